// rpf_grow.cu -- rpTree growth for all T trees at once (Sec. 2, Algorithm 1
// per tree, Algorithm 2 for the split direction).
//
// A tree is a permutation `perm` of 0..n-1 in which every node is a
// contiguous segment.  Growth runs in two phases:
//
//  Phase A (this file), level-synchronous over every tree, for nodes of more
//  than 4096 points: each level cuts the frontier into chunks of <= 4096
//  positions of one node and runs
//    k_dirs_a      nTry directions per node (FP64 r, FP32 copy) and the FP64
//                  projection b_j of the node's first member o
//    k_proj_a      centred FP32 projections q' = r . (x - o) (rows staged per
//                  warp through shared-memory tiles), per-point error radius,
//                  per-chunk FP32 statistics (sum, sum of squares, sum of
//                  |q'|, min, max, max radius, sum of squared radii)
//    k_certify_a   Algorithm 2's choice certified from the bounds, or the
//                  node is marked exact with its tries still in contention
//    k_cand        exact FP64 min / max among the candidates the bound leaves;
//                  lists the chunks of exact nodes
//    k_proj64, k_csum_*   canonical FP64 statistics of exact nodes (tries in
//                  contention only)
//    k_med_*       median rule: radix selection over q', the band, a direct
//                  selection for small bands (k_med_direct), exact passes
//    k_split_a     c = fma(u, b - a, a) with redraws ("c ~ runif[a, b]"), or
//                  the median
//    k_side_count  p < c per point (certified from q', else FP64), counts
//    k_node_scan / k_scatter   stable partition; children of <= 4096 points
//                  go straight to the final permutation
//    k_frontier    next frontier (> 4096 points), subtree items (L < len <=
//                  4096), new leaves (<= L)
//  Phase B (rpf_subtree.cu): one CTA grows each item's whole subtree.
//
//  Afterwards the node table is compacted (phase B reserves id ranges) and
//  the chosen direction of every split node is regenerated into it.
#include <cuda_runtime.h>

#include <type_traits>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "rpf_decide.cuh"
#include "rpf_proj.cuh"
#include "rpf_scan.cuh"

namespace {

constexpr int kBlock = 256;
static_assert(RPF_CHUNK % kBlock == 0, "a chunk is a whole number of block strides");
constexpr int kSub = RPF_CHUNK;  // nodes of at most this many points grow in one CTA
constexpr int kCandList = 256;   // min / max candidates listed per chunk for the warp pass
constexpr int kMedList = 256;    // median rule: bands up to this size are selected directly
constexpr int kPaStages = 2;     // row-tile units in flight per warp in k_proj_a

struct Level {
  int64_t cap_f = 0, cap_c = 0, cap_dir = 0;
  int32_t *fr_node[2]{}, *fr_tree[2]{}, *fr_begin[2]{}, *fr_len[2]{}, *fr_cb[2]{}, *fr_nc[2]{};
  uint64_t* fr_key[2]{};
  int32_t *fr_ogid{}, *fr_exact{}, *fr_jstar{}, *fr_flag{}, *fr_nl{};
  double *fr_a{}, *fr_b{}, *fr_c{}, *fr_base{};
  double *fr_mu{}, *fr_min{}, *fr_max{};
  float *fr_tl{}, *fr_tr{}, *fr_rad{}, *fr_wlo{}, *fr_whi{};
  unsigned long long *fr_akey{}, *fr_bkey{};
  unsigned long long* fr_cmask{};  // tries still in contention at an exact node
  // median rule: selected key, point index and remaining rank per node, and
  // a 256-bin histogram per node for the radix passes
  unsigned long long* md_key{};
  uint32_t *md_id{}, *md_fk{};
  int32_t *md_rank{}, *md_hist{}, *md_l0{};
  float *md_lo{}, *md_hi{};
  // median rule: each certified node's band as (key, point index) pairs, at
  // most kMedList of them, and whether the direct selection settled the node
  int32_t *md_bn{}, *md_done{};
  unsigned long long* md_bk{};
  uint32_t* md_bi{};
  int32_t *ch_node[2]{}, *ch_start[2]{}, *ch_len[2]{};
  int32_t *ch_nleft{}, *ch_loff{};
  double *cp_sum{}, *cp_min{}, *cp_max{};
  double *cp_s1{}, *cp_s2{}, *cp_a{};
  float *cp_min32{}, *cp_max32{}, *cp_rad{}, *cp_rad2{};
  double* dir64{};
  float* dir32{};
};

struct Counts {
  int32_t f_next, c_next, n_leaves_new, n_items_new;
  int32_t n_radix;  // median rule: nodes whose exact selection needs the radix passes
};

template <typename T>
int grow_buf(T** p, int64_t old_n, int64_t new_n, cudaStream_t s, bool keep) {
  void* q = nullptr;
  if (rpf_alloc(&q, sizeof(T) * (size_t)std::max<int64_t>(new_n, 1), s)) return RPF_ENOMEM;
  if (*p) {
    if (keep && old_n > 0) {
      cudaError_t e = cudaMemcpyAsync(q, *p, sizeof(T) * (size_t)old_n, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return rpf_cuda_err(e);
    }
    rpf_release(*p, s);
  }
  *p = (T*)q;
  return RPF_OK;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ---------------------------------------------------------------------------
__global__ void k_init_perm(int32_t* perm, int64_t n, int T) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * T) return;
  perm[i] = (int32_t)(i % n);
}

// |x|_2 rounded up (FP32 sum of squares, relative margin for its roundings)
__global__ void k_xnorm(const float* X, int64_t n, int d, float* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* x = X + i * d;
  float s = 0.0f;
  for (int k = 0; k < d; ++k) s = __fmaf_rn(x[k], x[k], s);
  out[i] = __fmul_ru(__fsqrt_ru(s), 1.0f + (float)(d + 4) * 0x1p-23f);
}

// Directions of the frontier nodes and the base projections b_j = r_j . o
// of each node's first member o; one warp per (node, try).  The lanes draw
// the Box-Muller pairs; the normalisation's sum keeps its sequential order
// (one lane), so r equals rpf_gen_direction bit for bit.  b_j is summed
// lane-strided and then by a butterfly (depth ceil(d / 32) + 5): the radius
// covers b_j summed in any order of depth <= d + 38.
__global__ void __launch_bounds__(128) k_dirs_a(int F, int ntry, int d, uint64_t seed, int t_base,
                                                int64_t n,
                                                const int32_t* fr_tree, const int32_t* fr_begin,
                                                const uint64_t* fr_key, const int32_t* perm_cur,
                                                const float* X, double* dir64, float* dir32,
                                                double* fr_base, int32_t* fr_ogid) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= (int64_t)F * ntry) return;  // whole warp
  const int f = (int)(g / ntry), j = (int)(g % ntry);
  const int tl = fr_tree[f];
  const uint64_t t = (uint64_t)(tl + t_base), key = fr_key[f];
  double* r = dir64 + g * d;
  float* r32 = dir32 + g * d;
  for (int i = lane; 2 * i < d; i += 32) {
    float g0, g1;
    rpf_gauss_pair(seed, t, key, (uint64_t)j, i, &g0, &g1);
    r32[2 * i] = g0;
    if (2 * i + 1 < d) r32[2 * i + 1] = g1;
  }
  __syncwarp();
  float inv = 0.0f;
  if (lane == 0) inv = rpf_inv_norm32(r32, d);
  inv = __shfl_sync(RPF_FULL, inv, 0);
  __syncwarp();
  for (int k = lane; k < d; k += 32) {
    const float v = inv == 0.0f ? (k == 0 ? 1.0f : 0.0f) : __fmul_rn(r32[k], inv);
    r32[k] = v;
    r[k] = (double)v;
  }
  const int32_t og = perm_cur[(int64_t)tl * n + fr_begin[f]];
  const float* xo = X + (int64_t)og * d;
  double b = 0.0;
  for (int k = lane; k < d; k += 32) b = __fma_rn((double)xo[k], r[k], b);  // r[k]: this lane's
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) b = __dadd_rn(b, __shfl_xor_sync(RPF_FULL, b, off));
  if (lane == 0) {
    fr_base[g] = b;
    if (j == 0) fr_ogid[f] = og;
  }
}

// Directions for explicit keys (inspection entry point).
__global__ void k_dirs_keys(uint64_t seed, int32_t t, const uint64_t* keys, int nk, int j, int d,
                            double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk) return;
  // the FP32 draw is staged in the upper half of the output row's bytes
  double* r = out + (int64_t)i * d;
  float* g = reinterpret_cast<float*>(r) + d;
  rpf_gen_direction(seed, (uint64_t)t, keys[i], (uint64_t)j, d, g, r);
}

template <int TG>
__global__ void __launch_bounds__(kBlock) k_proj_a(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, const int32_t* fr_ogid, const float* __restrict__ X,
    const int32_t* __restrict__ perm_cur, const float* __restrict__ xnorm, int64_t n, int64_t Tn,
    int d, int ntry, const float* dir32, float* p32, double* cp_s1, double* cp_s2, double* cp_a,
    float* cp_min, float* cp_max, float* cp_rad, float* cp_rad2) {
  extern __shared__ __align__(16) float smf[];
  float* sr = smf;                   // ntry x d
  float* so = smf + ntry * d;        // d
  float* red = so + ((d + 3) & ~3);  // 8 x TG x 5 statistics, then 33 for the radius
  float* tiles = red + 8 * 5 * 8 + 40;  // d % 4 == 0: kPaStages 32-row tiles per warp
  const int c = blockIdx.x;
  const int f = ch_node[c];
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const int len = ch_len[c];
  const int og = fr_ogid[f];
  const float on = xnorm[og];
  for (int i = threadIdx.x; i < ntry * d; i += blockDim.x) sr[i] = dir32[(int64_t)f * ntry * d + i];
  for (int k = threadIdx.x; k < d; k += blockDim.x) so[k] = X[(int64_t)og * d + k];
  __syncthreads();
  float radmax = 0.0f, rad2 = 0.0f;  // rad2: rounded-up sum of the points' rad^2
  for (int j0 = 0; j0 < ntry; j0 += TG) {
    const int nj = min(TG, ntry - j0);
    float s1[TG], s2[TG], a1[TG], mn[TG], mx[TG];
#pragma unroll
    for (int q = 0; q < TG; ++q) {
      s1[q] = s2[q] = a1[q] = 0.0f;
      mn[q] = INFINITY;
      mx[q] = -INFINITY;
    }
    if ((d & 3) == 0) {
      // batches of 32 positions, one per lane, rows staged through row
      // tiles, kPaStages units in flight per warp
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      // TG is nTry itself when nTry <= 5 (the launch picks it so): one pass
      // then covers every try, with the sum of squares
      auto project = [&](auto dfull) {
        rpf_warp_project<TG, RPF_TILE_DC, kPaStages, (TG <= 5), decltype(dfull)::value>(
            X, d, perm_cur + base, len, warp, kBlock / 32, tiles + warp * kPaStages * RPF_TILE_FLOATS,
            so, sr + j0 * d, nj, j0 == 0, lane, j0 == 0 ? xnorm : nullptr,
            [&](int pos, int gid, const float(&acc)[TG], float nn, float xn) {
              if (TG <= 5 || j0 == 0) {
                const float r = rpf_point_rad(d, nn, xn, on);
                radmax = fmaxf(radmax, r);
                rad2 = __fmaf_ru(r, r, rad2);
              }
#pragma unroll
              for (int q = 0; q < TG; ++q) {
                if (TG <= 5 || q < nj) {
                  p32[(int64_t)((TG <= 5 ? 0 : j0) + q) * Tn + base + pos] = acc[q];
                  rpf_stat_add(acc[q], s1[q], s2[q], a1[q], mn[q], mx[q]);
                }
              }
            });
      };
      // whole chunks when d is a multiple of the chunk width
      if (d % RPF_TILE_DC == 0) project(std::true_type{});
      else project(std::false_type{});
    } else {
      for (int u0 = 0; u0 * kBlock < len; u0 += 4) {
        int gid[4], pos[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          pos[p] = threadIdx.x + kBlock * (u0 + p);
          gid[p] = pos[p] < len ? perm_cur[base + pos[p]] : -1;
        }
        float acc[4][TG], nn[4];
        rpf_proj4<TG>(X, d, gid, so, sr + j0 * d, nj, acc, nn, j0 == 0);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (gid[p] < 0) continue;
          if (j0 == 0) {
            const float r = rpf_point_rad(d, nn[p], xnorm[gid[p]], on);
            radmax = fmaxf(radmax, r);
            rad2 = __fmaf_ru(r, r, rad2);
          }
#pragma unroll
          for (int q = 0; q < TG; ++q) {
            if (q < nj) {
              const float v = acc[p][q];
              p32[(int64_t)(j0 + q) * Tn + base + pos[p]] = v;
              rpf_stat_add(v, s1[q], s2[q], a1[q], mn[q], mx[q]);
            }
          }
        }
      }
    }
    const int64_t o = (int64_t)c * ntry + j0;
    rpf_block_stats<TG>(nj, s1, s2, a1, mn, mx, red, cp_s1 + o, cp_s2 + o, cp_a + o, cp_min + o,
                        cp_max + o, j0 == 0 ? &radmax : nullptr, &rad2);
  }
  if (threadIdx.x == 0) {
    cp_rad[c] = radmax;
    cp_rad2[c] = rad2;
  }
}

// Per node: merge the chunk statistics, certify Algorithm 2's choice.  One
// warp per node: lane j merges try j's chunk partials (in chunk order) and
// bounds its dispersion; the radius and the winner's extremes are lane-
// strided min / max reductions; lane 0 selects.
__global__ void __launch_bounds__(128) k_certify_a(
    int F, int ntry, int exact_only, const int32_t* fr_cb, const int32_t* fr_nc,
    const int32_t* fr_len, const double* cp_s1, const double* cp_s2, const double* cp_a,
    const float* cp_min, const float* cp_max, const float* cp_rad, const float* cp_rad2,
    const double* fr_base,
    int32_t* fr_exact, int32_t* fr_jstar, float* fr_rad, float* fr_wlo, float* fr_whi,
    unsigned long long* fr_akey, unsigned long long* fr_bkey, unsigned long long* fr_cmask) {
  __shared__ double s_vh[4][RPF_MAX_TRY];
  __shared__ float s_lo[4][RPF_MAX_TRY], s_hi[4][RPF_MAX_TRY];
  const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (f >= F) return;  // whole warp
  const int cb = fr_cb[f], nc = fr_nc[f];
  float rad = 0.0f, r2 = 0.0f;  // max radius; rounded-up sum of rad^2
  for (int c = cb + lane; c < cb + nc; c += 32) {
    rad = fmaxf(rad, cp_rad[c]);
    r2 = __fadd_ru(r2, cp_rad2[c]);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    rad = fmaxf(rad, __shfl_xor_sync(RPF_FULL, rad, off));
    r2 = __fadd_ru(r2, __shfl_xor_sync(RPF_FULL, r2, off));
  }
  const float l2 = __fsqrt_ru(r2);
  if (lane == 0) fr_rad[f] = rad;
  const int m = fr_len[f];
  const double inv_m = 1.0 / (double)m;
  for (int j = lane; j < ntry; j += 32) {
    double a = 0.0, b = 0.0, e = 0.0;
    int c = cb;
    for (; c + 3 < cb + nc; c += 4) {  // partials fetched ahead, added in chunk order
      double va[4], vb[4], ve[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        va[u] = cp_s1[(int64_t)(c + u) * ntry + j];
        vb[u] = cp_s2[(int64_t)(c + u) * ntry + j];
        ve[u] = cp_a[(int64_t)(c + u) * ntry + j];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a = __dadd_rn(a, va[u]);
        b = __dadd_rn(b, vb[u]);
        e = __dadd_rn(e, ve[u]);
      }
    }
    for (; c < cb + nc; ++c) {
      a = __dadd_rn(a, cp_s1[(int64_t)c * ntry + j]);
      b = __dadd_rn(b, cp_s2[(int64_t)c * ntry + j]);
      e = __dadd_rn(e, cp_a[(int64_t)c * ntry + j]);
    }
    rpf_try_bounds(m, inv_m, a, b, e, fr_base[(int64_t)f * ntry + j], rad, l2, &s_vh[wib][j],
                   &s_lo[wib][j], &s_hi[wib][j]);
  }
  __syncwarp();
  int w = -1;
  if (lane == 0) w = exact_only ? -1 : rpf_certify_select(ntry, s_vh[wib], s_lo[wib], s_hi[wib]);
  w = __shfl_sync(RPF_FULL, w, 0);
  if (w < 0) {
    if (lane == 0) {
      fr_exact[f] = 1;
      fr_cmask[f] = exact_only ? (ntry >= 64 ? ~0ull : (1ull << ntry) - 1ull)
                               : rpf_contenders(ntry, s_lo[wib], s_hi[wib]);
    }
    return;
  }
  float lo = INFINITY, hi = -INFINITY;
  for (int c = cb + lane; c < cb + nc; c += 32) {
    lo = fminf(lo, cp_min[(int64_t)c * ntry + w]);
    hi = fmaxf(hi, cp_max[(int64_t)c * ntry + w]);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(RPF_FULL, lo, off));
    hi = fmaxf(hi, __shfl_xor_sync(RPF_FULL, hi, off));
  }
  if (lane == 0) {
    const float r2 = __fmul_ru(2.0f, rad);
    fr_exact[f] = 0;
    fr_jstar[f] = w;
    fr_wlo[f] = __fadd_ru(lo, r2);  // min candidates: q' <= wlo
    fr_whi[f] = __fsub_rd(hi, r2);  // max candidates: q' >= whi
    fr_akey[f] = rpf_dkey(INFINITY);
    fr_bkey[f] = rpf_dkey(-INFINITY);
  }
}

// Exact FP64 projections of the min / max candidates of certified nodes;
// chunks of exact nodes are listed instead.
__global__ void __launch_bounds__(kBlock) k_cand(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, const int32_t* fr_exact, const int32_t* fr_jstar, const float* fr_wlo,
    const float* fr_whi, const float* X, const int32_t* perm_cur, int64_t n, int64_t Tn, int d,
    int ntry, const float* p32, const double* dir64, unsigned long long* fr_akey,
    unsigned long long* fr_bkey, int32_t* ex_list, int32_t* ex_count) {
  const int c = blockIdx.x;
  const int f = ch_node[c];
  if (fr_exact[f]) {  // listed for the exact path instead
    if (threadIdx.x == 0) ex_list[atomicAdd(ex_count, 1)] = c;
    return;
  }
  const int js = fr_jstar[f];
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const int len = ch_len[c];
  const float lo = fr_wlo[f], hi = fr_whi[f];
  const float* p = p32 + (int64_t)js * Tn + base;
  const double* r = dir64 + ((int64_t)f * ntry + js) * d;
  // candidates are few: list them, then one warp evaluates them two at a
  // time (rpf_p64_pair); beyond the list's room a thread evaluates its own
  __shared__ int s_n;
  __shared__ int s_e[kCandList];
  if (threadIdx.x == 0) s_n = 0;
  constexpr int kPer = RPF_CHUNK / kBlock;
  float qv[kPer];  // the chunk's q', fetched at once
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = threadIdx.x + u * kBlock;
    qv[u] = i < len ? p[i] : 0.0f;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = threadIdx.x + u * kBlock;
    if (i >= len) break;
    const float v = qv[u];
    const bool a = v <= lo, b = v >= hi;
    if (!a && !b) continue;
    const int slot = atomicAdd(&s_n, 1);
    if (slot < kCandList) {
      s_e[slot] = (i << 2) | (a ? 1 : 0) | (b ? 2 : 0);
      continue;
    }
    const double q = rpf_p64(X + (int64_t)perm_cur[base + i] * d, r, d);
    if (a) atomicMin(&fr_akey[f], rpf_dkey(q));
    if (b) atomicMax(&fr_bkey[f], rpf_dkey(q));
  }
  __syncthreads();
  const int nc = min(s_n, kCandList);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int q0 = 0; q0 < nc; q0 += 2) {
      const int e0 = s_e[q0], e1 = q0 + 1 < nc ? s_e[q0 + 1] : e0;
      const double q = rpf_p64_pair(X + (int64_t)perm_cur[base + (e0 >> 2)] * d,
                                    X + (int64_t)perm_cur[base + (e1 >> 2)] * d, r, d, lane);
      if (lane < 2) {
        const int e = lane == 0 ? e0 : e1;
        if (e & 1) atomicMin(&fr_akey[f], rpf_dkey(q));
        if (e & 2) atomicMax(&fr_bkey[f], rpf_dkey(q));
      }
    }
  }
}

// --- exact path: canonical FP64 projections and statistics (Algorithm 2) ---
// Grid-stride over (listed chunk, slice of 256 positions): canonical FP64
// projections of every try still in contention.
__global__ void __launch_bounds__(kBlock) k_proj64(
    const int32_t* list, const int32_t* count, const int32_t* ch_node, const int32_t* ch_start,
    const int32_t* ch_len, const int32_t* fr_tree, const int32_t* fr_begin, const float* X,
    const int32_t* perm_cur, int64_t n, int64_t Tn, int d, int ntry, const double* dir64,
    const unsigned long long* fr_cmask, double* p64) {
  constexpr int kSlices = RPF_CHUNK / kBlock;
  const int total = *count * kSlices;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int c = list[item / kSlices], sl = item % kSlices;
    const int i = sl * kBlock + threadIdx.x;
    if (i >= ch_len[c]) continue;
    const int f = ch_node[c];
    const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
    const float* x = X + (int64_t)perm_cur[base + i] * d;
    const unsigned long long mask = fr_cmask[f];
    for (int j = 0; j < ntry; ++j)
      if ((mask >> j) & 1ull)
        p64[(int64_t)j * Tn + base + i] = rpf_p64(x, dir64 + ((int64_t)f * ntry + j) * d, d);
  }
}

// One warp per (listed exact chunk, try in contention), grid-stride.
// pass 0: canonical chunk sum of p and exact min / max; pass 1: canonical
// chunk sum of (p - mu)^2.
__global__ void k_csum_chunks(int pass, const int32_t* list, const int32_t* count, int ntry,
                              const int32_t* ch_node, const int32_t* ch_start,
                              const int32_t* ch_len, const int32_t* fr_tree,
                              const int32_t* fr_begin, const unsigned long long* fr_cmask,
                              int64_t n, int64_t Tn, const double* p64, const double* fr_mu,
                              double* cp_sum, double* cp_min, double* cp_max) {
  const int lane = threadIdx.x & 31;
  const int64_t total = (int64_t)*count * ntry;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wid < total; wid += nw) {
    const int c = list[wid / ntry], j = (int)(wid % ntry);
    const int f = ch_node[c];
    if (!((fr_cmask[f] >> j) & 1ull)) continue;
    const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
    const int len = ch_len[c];
    const double* p = p64 + (int64_t)j * Tn + base;
    if (pass == 0) {
      double S = rpf_warp_chunk_sum(len, lane, [&](int64_t k) { return p[k]; });
      double a = INFINITY, b = -INFINITY;
      for (int k = lane; k < len; k += 32) {
        a = fmin(a, p[k]);
        b = fmax(b, p[k]);
      }
      for (int off = 16; off >= 1; off >>= 1) {
        a = fmin(a, __shfl_xor_sync(RPF_FULL, a, off));
        b = fmax(b, __shfl_xor_sync(RPF_FULL, b, off));
      }
      if (lane == 0) {
        cp_sum[(int64_t)c * ntry + j] = S;
        cp_min[(int64_t)c * ntry + j] = a;
        cp_max[(int64_t)c * ntry + j] = b;
      }
    } else {
      const double mu = fr_mu[(int64_t)f * ntry + j];
      double V = rpf_warp_chunk_sum(len, lane, [&](int64_t k) {
        double e = __dsub_rn(p[k], mu);
        return __dmul_rn(e, e);
      });
      if (lane == 0) cp_sum[(int64_t)c * ntry + j] = V;
    }
  }
}

// Canonical reduction of a node's chunk partials for one try (stride ntry),
// recursing in place beyond 4096 chunks.
__device__ double node_reduce(double* part, int64_t nc, int ntry, int lane) {
  while (nc > RPF_CHUNK) {
    const int64_t nc2 = (nc + RPF_CHUNK - 1) / RPF_CHUNK;
    for (int64_t c2 = 0; c2 < nc2; ++c2) {
      const int64_t len = min((int64_t)RPF_CHUNK, nc - c2 * RPF_CHUNK);
      const double* src = part + c2 * RPF_CHUNK * ntry;
      double s = rpf_warp_chunk_sum(len, lane, [&](int64_t k) { return src[k * ntry]; });
      __syncwarp();
      if (lane == 0) part[c2 * ntry] = s;
      __syncwarp();
    }
    nc = nc2;
  }
  return rpf_warp_chunk_sum(nc, lane, [&](int64_t k) { return part[k * ntry]; });
}

// One warp per exact node.  pass 0: S_j -> mu_j, exact min / max; pass 1:
// V_j and Algorithm 2's choice (first try with V > best, best from 0).
__global__ void k_csum_nodes(int pass, int F, int ntry, const int32_t* fr_cb, const int32_t* fr_nc,
                             const int32_t* fr_len, const int32_t* fr_exact,
                             const unsigned long long* fr_cmask, double* cp_sum,
                             const double* cp_min, const double* cp_max, double* fr_mu,
                             double* fr_min, double* fr_max, int32_t* fr_jstar, double* fr_a,
                             double* fr_b) {
  const int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= F || !fr_exact[f]) return;
  const int cb = fr_cb[f], nc = fr_nc[f];
  const double m = (double)fr_len[f];
  double best = 0.0;
  int js = -1;
  const unsigned long long mask = fr_cmask[f];
  for (int j = 0; j < ntry; ++j) {
    if (!((mask >> j) & 1ull)) continue;  // certainly below a contender
    double v = node_reduce(cp_sum + (int64_t)cb * ntry + j, nc, ntry, lane);
    if (pass == 0) {
      double a = INFINITY, b = -INFINITY;
      for (int c = cb + lane; c < cb + nc; c += 32) {
        a = fmin(a, cp_min[(int64_t)c * ntry + j]);
        b = fmax(b, cp_max[(int64_t)c * ntry + j]);
      }
      for (int off = 16; off >= 1; off >>= 1) {
        a = fmin(a, __shfl_xor_sync(RPF_FULL, a, off));
        b = fmax(b, __shfl_xor_sync(RPF_FULL, b, off));
      }
      if (lane == 0) {
        fr_mu[f * ntry + j] = __ddiv_rn(v, m);
        fr_min[f * ntry + j] = a;
        fr_max[f * ntry + j] = b;
      }
    } else if (v > best) {
      best = v;
      js = j;
    }
  }
  if (pass == 1 && lane == 0) {
    fr_jstar[f] = js;
    if (js >= 0) {
      fr_a[f] = fr_min[f * ntry + js];
      fr_b[f] = fr_max[f * ntry + js];
    }
  }
}

// Split point (Algorithm 1) and node record; certified side thresholds.
// ---------------------------------------------------------------------------
// Median rule (split_rule 1, Sec. 2's other usual split point): the floor(m/2)
// points smallest in (p64 of the winning try, point index) order go left and
// c is the p64 of the first point that goes right.
//
// Radix selection in 16 passes of 8 bits; per pass every chunk adds its
// shared-memory histogram of the keys that match the node's prefix so far
// into the node's 256 bins, and one warp per node picks the digit that holds
// the remaining rank.
//   passes 0-3  (certified nodes): v32 = the rank-floor(m/2) FP32 projection
//               q' of the winner.  With R the node's certified radius
//               (|q' - (p64 - b)| <= R), the median's p64 - b lies within
//               v32 +- R, so points with q' < v32 - 2R are certainly left,
//               points with q' > v32 + 2R certainly right, and only the band
//               between gets its p64 computed (k_med_band);
//   passes 4-11: the order-preserving 64-bit key of p64 (band points, or
//               every point of an exact node), rank floor(m/2) minus the
//               certainly-left count;
//   passes 12-15: the point index among equal keys.
// ---------------------------------------------------------------------------
__global__ void k_med_init(int F, const int32_t* fr_len, uint32_t* md_fk,
                           unsigned long long* md_key, uint32_t* md_id, int32_t* md_rank,
                           int32_t* md_l0, int32_t* md_bn, int32_t* md_done) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  md_fk[f] = 0u;
  md_key[f] = 0ull;
  md_id[f] = 0u;
  md_rank[f] = fr_len[f] >> 1;
  md_l0[f] = 0;
  md_bn[f] = 0;
  md_done[f] = 0;
}

// Median rule, a node's band of at most kMedList points (one warp per node):
// the band point with exactly md_rank smaller (key, index) pairs in the band
// is the selection (the pairs are distinct).  Exact nodes and larger bands
// are counted for the radix passes.
__global__ void __launch_bounds__(128) k_med_direct(
    int F, const int32_t* fr_exact, const int32_t* fr_jstar, const int32_t* md_bn,
    const unsigned long long* md_bk, const uint32_t* md_bi, const int32_t* md_rank,
    unsigned long long* md_key, uint32_t* md_id, int32_t* md_done, int32_t* n_radix) {
  const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= F || fr_jstar[f] < 0) return;  // whole warp
  const int nb = md_bn[f];
  if (fr_exact[f] || nb > kMedList) {
    if (lane == 0) atomicAdd(n_radix, 1);
    return;
  }
  const unsigned long long* K = md_bk + (int64_t)f * kMedList;
  const uint32_t* I = md_bi + (int64_t)f * kMedList;
  const int r = md_rank[f];
  for (int e = lane; e < nb; e += 32) {
    const unsigned long long k = K[e];
    const uint32_t id = I[e];
    int below = 0;
    for (int g = 0; g < nb; ++g) below += K[g] < k || (K[g] == k && I[g] < id);
    if (below == r) {
      md_key[f] = k;
      md_id[f] = id;
    }
  }
  if (lane == 0) md_done[f] = 1;
}

__global__ void __launch_bounds__(kBlock) k_med_hist(
    int pass, const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len,
    const int32_t* fr_tree, const int32_t* fr_begin, const int32_t* fr_exact,
    const int32_t* fr_jstar, const int32_t* perm_cur, int64_t n, int64_t Tn, const float* p32,
    const double* p64, const uint32_t* md_fk, const unsigned long long* md_key,
    const uint32_t* md_id, const float* md_lo, const float* md_hi, const int32_t* md_done,
    int32_t* md_hist) {
  __shared__ int h[256];
  const int c = blockIdx.x;
  const int f = ch_node[c];
  const int js = fr_jstar[f];
  const int exact = fr_exact[f];
  if (js < 0 || (pass < 4 && exact) || (pass >= 4 && md_done[f])) return;  // nothing to count
  for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const float* q = p32 + (int64_t)js * Tn + base;
  const double* p = p64 + (int64_t)js * Tn + base;
  const uint32_t pf = md_fk[f];
  const unsigned long long pk = md_key[f];
  const uint32_t pid = md_id[f];
  const float lo = md_lo[f], hi = md_hi[f];
  const int len = ch_len[c];
  constexpr int kPer = RPF_CHUNK / kBlock;
  float qv[kPer];  // the chunk's q', fetched at once
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = threadIdx.x + u * kBlock;
    qv[u] = (!exact && i < len) ? q[i] : 0.0f;
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = threadIdx.x + u * kBlock;
    if (i >= len) break;
    int dig;
    bool match;
    if (pass < 4) {
      const int sh = 24 - 8 * pass;
      const uint32_t k = rpf_fkey(qv[u]);
      dig = (int)((k >> sh) & 255u);
      match = pass == 0 || ((k ^ pf) >> (sh + 8)) == 0u;
    } else {
      if (!exact && !(qv[u] >= lo && qv[u] <= hi)) continue;  // decided without p64
      match = rpf_med_digit(pass - 4, rpf_mkey(p[i]), (uint32_t)perm_cur[base + i], pk, pid, &dig);
    }
    if (match) atomicAdd(&h[dig], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x)
    if (h[b]) atomicAdd(&md_hist[(int64_t)f * 256 + b], h[b]);
}

// one warp per node: the digit whose bin holds the remaining rank; the bins
// are cleared for the next pass
__global__ void __launch_bounds__(128) k_med_select(int pass, int F, const int32_t* fr_exact,
                                                    const int32_t* fr_jstar, const int32_t* md_done,
                                                    uint32_t* md_fk, unsigned long long* md_key,
                                                    uint32_t* md_id, int32_t* md_rank,
                                                    int32_t* md_hist) {
  const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= F || fr_jstar[f] < 0 || (pass < 4 && fr_exact[f]) || (pass >= 4 && md_done[f]))
    return;  // whole warp
  int32_t* hb = md_hist + (int64_t)f * 256 + 8 * lane;
  int v[8], sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    v[q] = hb[q];
    sum += v[q];
  }
  int x = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(RPF_FULL, x, off);
    if (lane >= off) x += y;
  }
  const int pre = x - sum;
  const int rank = md_rank[f];
  if (rank >= pre && rank < pre + sum) {  // exactly one lane holds the rank
    int cum = pre, dig = -1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (dig < 0) {
        if (rank < cum + v[q]) dig = 8 * lane + q;
        else cum += v[q];
      }
    }
    md_rank[f] = rank - cum;
    if (pass < 4) md_fk[f] |= (uint32_t)dig << (24 - 8 * pass);
    else if (pass < 12) md_key[f] |= (unsigned long long)dig << (56 - 8 * (pass - 4));
    else md_id[f] |= (uint32_t)dig << (24 - 8 * (pass - 12));
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) hb[q] = 0;
}

// Certified nodes: the band around v32; p64 of the winner for the points in
// it; the count of points certainly left of the band.
__global__ void __launch_bounds__(kBlock) k_med_band(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, const int32_t* fr_exact, const int32_t* fr_jstar,
    const float* fr_rad, const float* X, const int32_t* perm_cur, int64_t n, int64_t Tn, int d,
    int ntry, const double* dir64, const float* p32, const uint32_t* md_fk, double* p64,
    int32_t* md_l0, int32_t* md_bn, unsigned long long* md_bk, uint32_t* md_bi) {
  __shared__ int wc[kBlock / 32];
  const int c = blockIdx.x;
  const int f = ch_node[c];
  const int js = fr_jstar[f];
  if (js < 0 || fr_exact[f]) return;  // exact nodes hold every p64 already
  float lo, hi;
  rpf_med_band(md_fk[f], fr_rad[f], &lo, &hi);
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const double* r = dir64 + ((int64_t)f * ntry + js) * d;
  const float* q = p32 + (int64_t)js * Tn + base;
  const int len = ch_len[c];
  constexpr int kPer = RPF_CHUNK / kBlock;
  float qv[kPer];  // the chunk's q', fetched at once
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = threadIdx.x + u * kBlock;
    qv[u] = i < len ? q[i] : 0.0f;
  }
  int cnt = 0;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = threadIdx.x + u * kBlock;
    if (i >= len) break;
    const float v = qv[u];
    if (v < lo) {
      ++cnt;
    } else if (v <= hi) {
      const int32_t id = perm_cur[base + i];
      const double pv = rpf_p64(X + (int64_t)id * d, r, d);
      p64[(int64_t)js * Tn + base + i] = pv;
      const int e = atomicAdd(&md_bn[f], 1);
      if (e < kMedList) {
        md_bk[(int64_t)f * kMedList + e] = rpf_mkey(pv);
        md_bi[(int64_t)f * kMedList + e] = (uint32_t)id;
      }
    }
  }
  for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(RPF_FULL, cnt, off);
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int u = 0; u < kBlock / 32; ++u) t += wc[u];
    if (t) atomicAdd(&md_l0[f], t);
  }
}

// Certified nodes: the exact stage selects rank floor(m/2) - (certainly left)
// among the band; the band is kept for the sides.
__global__ void k_med_rank(int F, const int32_t* fr_len, const int32_t* fr_exact,
                           const int32_t* fr_jstar, const float* fr_rad, const uint32_t* md_fk,
                           const int32_t* md_l0, int32_t* md_rank, float* md_lo, float* md_hi) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F || fr_jstar[f] < 0) return;
  if (fr_exact[f]) {
    md_lo[f] = -INFINITY;
    md_hi[f] = INFINITY;
    return;
  }
  float lo, hi;
  rpf_med_band(md_fk[f], fr_rad[f], &lo, &hi);
  md_lo[f] = lo;
  md_hi[f] = hi;
  md_rank[f] = (fr_len[f] >> 1) - md_l0[f];
}

// (a, b: the exact path's for exact nodes, else the candidates' extremes;
// the fallback counter gains the level's exact nodes)
__global__ void k_split_a(int F, int ntry, uint64_t seed, int t_base, int median,
                          const int32_t* fr_node,
                          const int32_t* fr_tree, const uint64_t* fr_key, const int32_t* fr_exact,
                          const int32_t* fr_jstar, const double* fr_a, const double* fr_b,
                          const unsigned long long* fr_akey, const unsigned long long* fr_bkey,
                          const double* fr_base, const float* fr_rad,
                          const unsigned long long* md_key, double* fr_c, int32_t* fr_flag,
                          float* fr_tl, float* fr_tr, int32_t* node_jstar, int32_t* node_flag,
                          double* node_c, unsigned long long* n_exact) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int js = fr_jstar[f];
  const int exact = fr_exact[f];
  if (exact) atomicAdd(n_exact, 1ULL);
  double c = NAN;
  int acc = 0;
  if (js >= 0 && median) {  // c = the p64 of the first point that goes right
    c = rpf_dkey_inv(md_key[f]);
    acc = 1;
  } else if (js >= 0) {
    const double a = exact ? fr_a[f] : rpf_dkey_inv(fr_akey[f]);
    const double b = exact ? fr_b[f] : rpf_dkey_inv(fr_bkey[f]);
    acc = rpf_split_point(seed, (uint64_t)(fr_tree[f] + t_base), fr_key[f], a, b, &c);
  }
  fr_c[f] = c;
  fr_flag[f] = acc ? 0 : 1;
  if (acc && !median && !exact) {
    float tl, tr;
    rpf_side_thresholds(c, fr_base[(int64_t)f * ntry + js], (double)fr_rad[f], &tl, &tr);
    fr_tl[f] = tl;
    fr_tr[f] = tr;
  }
  const int id = fr_node[f];
  node_jstar[id] = js;
  node_flag[id] = (acc ? 0 : 1) | (exact ? 2 : 0);
  node_c[id] = c;
}

__global__ void __launch_bounds__(kBlock) k_side_count(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, const int32_t* fr_len, const int32_t* fr_exact,
    const int32_t* fr_jstar, const int32_t* fr_flag, const double* fr_c, const float* fr_tl,
    const float* fr_tr, const float* X, const int32_t* perm_cur, int64_t n, int64_t Tn, int d,
    int ntry, const float* p32, const double* p64, const double* dir64, int median,
    const unsigned long long* md_key, const uint32_t* md_id, const float* md_lo,
    const float* md_hi, uint8_t* side, int32_t* ch_nleft) {
  const int c = blockIdx.x;
  const int f = ch_node[c];
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const int len = ch_len[c];
  const int m = fr_len[f];
  const int flag = fr_flag[f];
  const int exact = fr_exact[f];
  const int js = fr_jstar[f];
  const double cc = fr_c[f];
  const float tl = fr_tl[f], tr = fr_tr[f];
  // the chunk's q' of the winner, fetched at once (<= 16 per thread)
  constexpr int kPer = RPF_CHUNK / kBlock;
  float qv[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = threadIdx.x + u * kBlock;
    qv[u] = (!flag && !exact && i < len) ? p32[(int64_t)js * Tn + base + i] : 0.0f;
  }
  int cnt = 0;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = threadIdx.x + u * kBlock;
    if (i >= len) break;
    bool left;
    if (flag) {
      left = (ch_start[c] + i) < (m >> 1);
    } else if (median) {  // certainly below / above the band, else (key, index) order
      const float q = qv[u];
      if (!exact && q < md_lo[f]) {
        left = true;
      } else if (!exact && q > md_hi[f]) {
        left = false;
      } else {
        const unsigned long long key = rpf_mkey(p64[(int64_t)js * Tn + base + i]);
        left = key < md_key[f] ||
               (key == md_key[f] && (uint32_t)perm_cur[base + i] < md_id[f]);
      }
    } else if (exact) {
      left = p64[(int64_t)js * Tn + base + i] < cc;
    } else {
      const float v = qv[u];
      if (v < tl) {
        left = true;
      } else if (v >= tr) {
        left = false;
      } else {
        left = rpf_p64(X + (int64_t)perm_cur[base + i] * d,
                       dir64 + ((int64_t)f * ntry + js) * d, d) < cc;
      }
    }
    side[base + i] = left ? 1 : 0;
    cnt += left ? 1 : 0;
  }
  for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(RPF_FULL, cnt, off);
  __shared__ int wc[kBlock / 32];
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int u = 0; u < kBlock / 32; ++u) s += wc[u];
    ch_nleft[c] = s;
  }
}

__global__ void k_node_scan(int F, int64_t id_base, const int32_t* fr_node, const int32_t* fr_tree,
                            const int32_t* fr_begin, const int32_t* fr_len, const uint64_t* fr_key,
                            const int32_t* fr_cb, const int32_t* fr_nc, const int32_t* ch_nleft,
                            int32_t* ch_loff, int32_t* fr_nl, uint64_t* node_key,
                            int32_t* node_tree, int32_t* node_begin, int32_t* node_len,
                            int32_t* node_left, int32_t* node_right, int32_t* node_jstar,
                            int32_t* node_flag, double* node_c) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  int run = 0;
  for (int c = fr_cb[f]; c < fr_cb[f] + fr_nc[f]; ++c) {
    ch_loff[c] = run;
    run += ch_nleft[c];
  }
  fr_nl[f] = run;
  const int m = fr_len[f];
  const int64_t idL = id_base + 2 * (int64_t)f, idR = idL + 1;
  const int parent = fr_node[f];
  node_left[parent] = (int32_t)idL;
  node_right[parent] = (int32_t)idR;
  const uint64_t key = fr_key[f];
  node_key[idL] = rpf_child_key(key, 0);
  node_key[idR] = rpf_child_key(key, 1);
  node_tree[idL] = node_tree[idR] = fr_tree[f];
  node_begin[idL] = fr_begin[f];
  node_begin[idR] = fr_begin[f] + run;
  node_len[idL] = run;
  node_len[idR] = m - run;
  node_left[idL] = node_right[idL] = node_left[idR] = node_right[idR] = -1;
  node_jstar[idL] = node_jstar[idR] = -1;
  node_flag[idL] = node_flag[idR] = 0;
  node_c[idL] = node_c[idR] = NAN;
}

// Stable scatter of one chunk: lefts at begin + (lefts before the chunk) +
// rank, rights at begin + nl + (rights before the chunk) + rank.  A child of
// at most 4096 points is written to the final permutation (a leaf, or a
// subtree that phase B reads from there).
__global__ void __launch_bounds__(kBlock) k_scatter(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* ch_loff,
    const int32_t* fr_tree, const int32_t* fr_begin, const int32_t* fr_len, const int32_t* fr_nl,
    int64_t n, int sub, const uint8_t* side, const int32_t* perm_cur, int32_t* perm_nxt,
    int32_t* perm_final) {
  const int c = blockIdx.x;
  const int f = ch_node[c];
  const int64_t tbase = (int64_t)fr_tree[f] * n;
  const int begin = fr_begin[f];
  const int64_t base = tbase + begin + ch_start[c];
  const int len = ch_len[c];
  const int m = fr_len[f], nl = fr_nl[f];
  const int loff = ch_loff[c];
  const int roff = ch_start[c] - loff;
  int32_t* dstL = (nl <= sub) ? perm_final : perm_nxt;
  int32_t* dstR = ((m - nl) <= sub) ? perm_final : perm_nxt;
  __shared__ int wsum[kBlock / 32];
  __shared__ int tile_l;
  int carryL = 0, carryR = 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // the chunk's sides and point ids, fetched at once (<= 16 per thread)
  constexpr int kPer = RPF_CHUNK / kBlock;
  int sv[kPer];
  int32_t pv[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = u * kBlock + threadIdx.x;
    sv[u] = i < len ? side[base + i] : 0;
    pv[u] = i < len ? perm_cur[base + i] : 0;
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int t0 = u * kBlock;
    if (t0 >= len) break;
    const int i = t0 + threadIdx.x;
    const bool valid = i < len;
    const int s = sv[u];
    int x = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int y = __shfl_up_sync(RPF_FULL, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int r = 0;
      for (int u = 0; u < kBlock / 32; ++u) {
        int v = wsum[u];
        wsum[u] = r;
        r += v;
      }
      tile_l = r;
    }
    __syncthreads();
    const int rankL = x - s + wsum[w];
    if (valid) {
      const int32_t v = pv[u];
      if (s) dstL[tbase + begin + loff + carryL + rankL] = v;
      else dstR[tbase + begin + nl + roff + carryR + (int)threadIdx.x - rankL] = v;
    }
    const int tl = tile_l;
    carryL += tl;
    carryR += min(kBlock, len - t0) - tl;
    __syncthreads();
  }
}

// Single block: classify the 2F children: > 4096 points -> next frontier,
// L < len <= 4096 -> subtree item, <= L -> leaf; build the next chunk list.
__global__ void __launch_bounds__(1024) k_frontier(
    int F, int L, int sub, int64_t id_base, const int32_t* fr_tree, const int32_t* fr_begin,
    const int32_t* fr_len, const uint64_t* fr_key, const int32_t* fr_nl, int32_t* nf_node,
    int32_t* nf_tree, int32_t* nf_begin, int32_t* nf_len, uint64_t* nf_key, int32_t* nf_cb,
    int32_t* nf_nc, int32_t* nch_node, int32_t* nch_start, int32_t* nch_len, int64_t leaf_base,
    int32_t* leaf_tree, int32_t* leaf_begin, int32_t* leaf_len, int64_t item_base,
    int32_t* it_node, int32_t* it_tree, int32_t* it_begin, int32_t* it_len, uint64_t* it_key,
    Counts* out) {
  __shared__ int ws_a[32], ws_l[32], ws_i[32], ws_c[32];
  __shared__ int tot_a, tot_l, tot_i, tot_c;
  __shared__ int run_a, run_l, run_i, run_c;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) run_a = run_l = run_i = 0;
  __syncthreads();
  const int NC = 2 * F;
  for (int t0 = 0; t0 < NC; t0 += 1024) {
    const int ci = t0 + threadIdx.x;
    int len = 0, active = 0, leaf = 0, item = 0;
    if (ci < NC) {
      const int f = ci >> 1, sd = ci & 1;
      len = sd ? fr_len[f] - fr_nl[f] : fr_nl[f];
      active = len > sub;
      leaf = len <= L;
      item = !active && !leaf;
    }
    int xa = active, xl = leaf, xi = item;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int ya = __shfl_up_sync(RPF_FULL, xa, off), yl = __shfl_up_sync(RPF_FULL, xl, off);
      int yi = __shfl_up_sync(RPF_FULL, xi, off);
      if (lane >= off) {
        xa += ya;
        xl += yl;
        xi += yi;
      }
    }
    if (lane == 31) {
      ws_a[w] = xa;
      ws_l[w] = xl;
      ws_i[w] = xi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int ra = 0, rl = 0, ri = 0;
      for (int u = 0; u < 32; ++u) {
        int va = ws_a[u], vl = ws_l[u], vi = ws_i[u];
        ws_a[u] = ra;
        ws_l[u] = rl;
        ws_i[u] = ri;
        ra += va;
        rl += vl;
        ri += vi;
      }
      tot_a = ra;
      tot_l = rl;
      tot_i = ri;
    }
    __syncthreads();
    if (ci < NC) {
      const int f = ci >> 1, sd = ci & 1;
      const int begin = sd ? fr_begin[f] + fr_nl[f] : fr_begin[f];
      if (active) {
        const int o = run_a + xa - active + ws_a[w];
        nf_node[o] = (int32_t)(id_base + ci);
        nf_tree[o] = fr_tree[f];
        nf_begin[o] = begin;
        nf_len[o] = len;
        nf_key[o] = rpf_child_key(fr_key[f], sd);
        nf_nc[o] = (len + RPF_CHUNK - 1) / RPF_CHUNK;
      } else if (leaf) {
        const int64_t o = leaf_base + run_l + xl - leaf + ws_l[w];
        leaf_tree[o] = fr_tree[f];
        leaf_begin[o] = begin;
        leaf_len[o] = len;
      } else {
        const int64_t o = item_base + run_i + xi - item + ws_i[w];
        it_node[o] = (int32_t)(id_base + ci);
        it_tree[o] = fr_tree[f];
        it_begin[o] = begin;
        it_len[o] = len;
        it_key[o] = rpf_child_key(fr_key[f], sd);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      run_a += tot_a;
      run_l += tot_l;
      run_i += tot_i;
    }
    __syncthreads();
  }
  const int FN = run_a;
  if (threadIdx.x == 0) run_c = 0;
  __syncthreads();
  for (int t0 = 0; t0 < FN; t0 += 1024) {
    const int fi = t0 + threadIdx.x;
    const int nc = fi < FN ? nf_nc[fi] : 0;
    int x = nc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int y = __shfl_up_sync(RPF_FULL, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) ws_c[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int r = 0;
      for (int u = 0; u < 32; ++u) {
        int v = ws_c[u];
        ws_c[u] = r;
        r += v;
      }
      tot_c = r;
    }
    __syncthreads();
    if (fi < FN) {
      const int cb = run_c + x - nc + ws_c[w];
      nf_cb[fi] = cb;
      const int len = nf_len[fi];
      for (int q = 0; q < nc; ++q) {
        nch_node[cb + q] = fi;
        nch_start[cb + q] = q * RPF_CHUNK;
        nch_len[cb + q] = min(RPF_CHUNK, len - q * RPF_CHUNK);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) run_c += tot_c;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out->f_next = FN;
    out->c_next = run_c;
    out->n_leaves_new = run_l;
    out->n_items_new = run_i;
  }
}

// --- node table compaction: valid slots (tree >= 0) keep their order -------
__global__ void k_compact_nodes(int64_t N, const int32_t* new_id, const uint64_t* key,
                                const int32_t* tree, const int32_t* begin, const int32_t* len,
                                const int32_t* left, const int32_t* right, const int32_t* jstar,
                                const int32_t* flag, const double* c, uint64_t* okey,
                                int32_t* otree, int32_t* obegin, int32_t* olen, int32_t* oleft,
                                int32_t* oright, int32_t* ojstar, int32_t* oflag, double* oc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int32_t o = new_id[i];
  if (o < 0) return;
  okey[o] = key[i];
  otree[o] = tree[i];
  obegin[o] = begin[i];
  olen[o] = len[i];
  oleft[o] = left[i] >= 0 ? new_id[left[i]] : -1;
  oright[o] = right[i] >= 0 ? new_id[right[i]] : -1;
  ojstar[o] = jstar[i];
  oflag[o] = flag[i];
  oc[o] = c[i];
}

__global__ void k_compact_leaves(int64_t S, const int32_t* pos, const int32_t* tree,
                                 const int32_t* begin, const int32_t* len, int32_t* otree,
                                 int32_t* obegin, int32_t* olen) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S || pos[i] < 0) return;
  otree[pos[i]] = tree[i];
  obegin[pos[i]] = begin[i];
  olen[pos[i]] = len[i];
}

// r* of every split node (regenerated from its key and chosen try), one warp
// per node: lanes draw the Box-Muller pairs, lane 0 forms the sequential
// FP32 norm, so r equals rpf_gen_direction's bit for bit.
__global__ void __launch_bounds__(128) k_node_dirs(int64_t N, int d, uint64_t seed, int t_base,
                                                   const uint64_t* key, const int32_t* tree,
                                                   const int32_t* left, const int32_t* jstar,
                                                   const int32_t* flag, float* dir32) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;  // whole warp
  float* r32 = dir32 + i * d;
  if (left[i] < 0 || (flag[i] & 1) || jstar[i] < 0) {
    for (int k = lane; k < d; k += 32) r32[k] = 0.0f;
    return;
  }
  const uint64_t t = (uint64_t)(tree[i] + t_base), kk = key[i], j = (uint64_t)jstar[i];
  for (int p = lane; 2 * p < d; p += 32) {
    float g0, g1;
    rpf_gauss_pair(seed, t, kk, j, p, &g0, &g1);
    r32[2 * p] = g0;
    if (2 * p + 1 < d) r32[2 * p + 1] = g1;
  }
  __syncwarp();
  float inv = 0.0f;
  if (lane == 0) inv = rpf_inv_norm32(r32, d);
  inv = __shfl_sync(RPF_FULL, inv, 0);
  __syncwarp();
  for (int k = lane; k < d; k += 32)
    r32[k] = inv == 0.0f ? (k == 0 ? 1.0f : 0.0f) : __fmul_rn(r32[k], inv);
}

// Routing record of every node: c (two words), left child, and the right
// child -- or the left one for a rank split, which sends every query left.
__global__ void k_route_table(int64_t N, const int32_t* left, const int32_t* right,
                              const int32_t* flag, const double* c, const int32_t* begin,
                              const int32_t* len, int4* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int l = left[i];
  if (l < 0) {  // a leaf: its segment of the tree's permutation
    out[i] = make_int4(begin[i], len[i], -1, -1);
    return;
  }
  const double cc = c[i];
  const int r = (flag[i] & 1) ? l : right[i];
  out[i] = make_int4(__double2loint(cc), __double2hiint(cc), l, r);
}

}  // namespace

int rpf_build_route(rpf_forest* f, cudaStream_t s) {
  rpf_release(f->node_route, s);
  f->node_route = nullptr;
  const int64_t N = f->n_nodes;
  if (rpf_alloc((void**)&f->node_route, sizeof(int4) * (size_t)std::max<int64_t>(N, 1), s))
    return RPF_ENOMEM;
  if (N > 0)
    RPF_LAUNCH("k_route_table", s, k_route_table<<<nblk(N, 256), 256, 0, s>>>(
        N, f->node_left, f->node_right, f->node_flag, f->node_c, f->node_begin, f->node_len,
        f->node_route));
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

// Phase B (rpf_subtree.cu)
bool rpf_subtree_fits(int d, int ntry);
int rpf_grow_subtrees(rpf_forest* fo, int64_t n_items, const int32_t* ilen, const int32_t* it_node,
                      const int32_t* it_tree, const int32_t* it_begin, const int32_t* it_len,
                      const uint64_t* it_key, const int32_t* it_nbase, const int32_t* it_lbase,
                      float* p32, double* p64, unsigned long long* d_exact, int* d_err,
                      int32_t* dfr, int* dfr_cnt, int dfr_cap, cudaStream_t s);
int rpf_split_deferred(rpf_forest* fo, const int32_t* dfr, const int* dfr_cnt, int dfr_cap,
                       const int32_t* new_id, int* d_err, cudaStream_t s);

// ---------------------------------------------------------------------------
int rpf_grow(rpf_forest* fo, cudaStream_t s) {
  const int64_t n = fo->n;
  const int d = fo->d;
  const int T = fo->prm.n_trees, L = fo->prm.leaf_max, ntry = fo->prm.n_try;
  const int exact_only = fo->prm.growth == 1 ? 1 : 0;
  const int median = fo->prm.split_rule == 1 ? 1 : 0;  // split at the median (Sec. 2)
  const uint64_t seed = fo->prm.seed;
  const int64_t Tn = (int64_t)T * n;
  // nodes of at most `sub` points grow inside one CTA (phase B); when its
  // shared-memory layout does not fit, every node is grown level by level
  const int sub = rpf_subtree_fits(d, ntry) ? kSub : L;

  int32_t *perm_a = nullptr, *perm_b = nullptr;
  float* p32 = nullptr;
  double* p64 = nullptr;
  uint8_t* side = nullptr;
  Level lv;
  Counts* h_cnt = nullptr;
  Counts* d_cnt = nullptr;
  unsigned long long* d_exact = nullptr;
  int* d_err = nullptr;
  int32_t *it_node = nullptr, *it_tree = nullptr, *it_begin = nullptr, *it_len = nullptr;
  int32_t *it_nbase = nullptr, *it_lbase = nullptr;
  uint64_t* it_key = nullptr;
  std::vector<void*> tmp;
  auto talloc = [&](void** p, size_t bytes) -> int {
    if (rpf_alloc(p, bytes, s)) return RPF_ENOMEM;
    tmp.push_back(*p);
    return RPF_OK;
  };
  auto free_level = [&]() {
    void* ps[] = {lv.fr_ogid, lv.fr_exact, lv.fr_jstar, lv.fr_flag, lv.fr_nl, lv.fr_a, lv.fr_b,
                  lv.fr_c, lv.fr_base, lv.fr_mu, lv.fr_min, lv.fr_max, lv.fr_tl, lv.fr_tr,
                  lv.fr_rad, lv.fr_wlo, lv.fr_whi, lv.fr_akey, lv.fr_bkey, lv.ch_nleft, lv.ch_loff,
                  lv.cp_sum, lv.cp_min, lv.cp_max, lv.cp_s1, lv.cp_s2, lv.cp_a, lv.cp_min32,
                  lv.cp_max32, lv.cp_rad, lv.cp_rad2, lv.dir64, lv.dir32, lv.md_key, lv.md_id, lv.md_rank,
                  lv.md_hist, lv.md_fk, lv.md_l0, lv.md_lo, lv.md_hi, lv.fr_cmask, lv.md_bn,
                  lv.md_done, lv.md_bk, lv.md_bi};
    for (void* p : ps) rpf_release(p, s);
    for (int q = 0; q < 2; ++q) {
      void* qs[] = {lv.fr_node[q], lv.fr_tree[q], lv.fr_begin[q], lv.fr_len[q], lv.fr_cb[q],
                    lv.fr_nc[q], lv.fr_key[q], lv.ch_node[q], lv.ch_start[q], lv.ch_len[q]};
      for (void* p : qs) rpf_release(p, s);
    }
    lv = Level();
  };
  auto cleanup = [&]() {
    for (void* p : tmp) rpf_release(p, s);
    tmp.clear();
    free_level();
  };
#define RPF_TRY(x) \
  do {             \
    int r_ = (x);  \
    if (r_) {      \
      cleanup();   \
      return r_;   \
    }              \
  } while (0)
#define RPF_TRYCU(x) RPF_TRY(((x) == cudaSuccess) ? RPF_OK : rpf_cuda_err(cudaGetLastError()))

  RPF_TRY(talloc((void**)&perm_a, sizeof(int32_t) * Tn));
  RPF_TRY(talloc((void**)&perm_b, sizeof(int32_t) * Tn));
  RPF_TRY(talloc((void**)&side, Tn));
  RPF_TRY(talloc((void**)&d_cnt, sizeof(Counts)));
  RPF_TRY(talloc((void**)&d_exact, sizeof(unsigned long long)));
  RPF_TRY(talloc((void**)&d_err, sizeof(int)));
  int32_t* ex_count = nullptr;
  RPF_TRY(talloc((void**)&ex_count, sizeof(int32_t)));
  RPF_TRYCU(cudaMemsetAsync(d_exact, 0, sizeof(unsigned long long), s));
  RPF_TRYCU(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  {  // one pinned counter block per host thread, kept for the process
    static thread_local Counts* pinned = nullptr;
    if (!pinned && cudaMallocHost((void**)&pinned, sizeof(Counts)) != cudaSuccess) {
      cudaGetLastError();
      pinned = nullptr;
      cleanup();
      return RPF_ENOMEM;
    }
    h_cnt = pinned;
  }
  RPF_TRY(talloc((void**)&p32, sizeof(float) * Tn * ntry));
  RPF_TRY(talloc((void**)&p64, sizeof(double) * Tn * ntry));
  // subtree items are disjoint sets of > L points of one tree
  const int64_t item_cap = Tn / (L + 1) + T + 1;
  RPF_TRY(talloc((void**)&it_node, 4 * item_cap));
  RPF_TRY(talloc((void**)&it_tree, 4 * item_cap));
  RPF_TRY(talloc((void**)&it_begin, 4 * item_cap));
  RPF_TRY(talloc((void**)&it_len, 4 * item_cap));
  RPF_TRY(talloc((void**)&it_key, 8 * item_cap));
  RPF_TRY(talloc((void**)&it_nbase, 4 * item_cap));
  RPF_TRY(talloc((void**)&it_lbase, 4 * item_cap));

  RPF_LAUNCH("k_init_perm", s, k_init_perm<<<nblk(Tn, 256), 256, 0, s>>>(perm_a, n, T));
  RPF_LAUNCH("k_init_perm", s, k_init_perm<<<nblk(Tn, 256), 256, 0, s>>>(fo->perm, n, T));
  RPF_LAUNCH("k_xnorm", s, k_xnorm<<<nblk(n, 256), 256, 0, s>>>(fo->X, n, d, fo->xnorm));

  // node and leaf tables, grown as needed (slots keep their contents)
  int64_t node_cap = 0, leaf_cap = 0;
  auto ensure_nodes = [&](int64_t need) -> int {
    if (need <= node_cap) return RPF_OK;
    const int64_t nc = std::max<int64_t>(need, node_cap * 2);
    const int64_t old = node_cap;
    int r;
    if ((r = grow_buf(&fo->node_key, old, nc, s, true))) return r;
    if ((r = grow_buf(&fo->node_tree, old, nc, s, true))) return r;
    if ((r = grow_buf(&fo->node_begin, old, nc, s, true))) return r;
    if ((r = grow_buf(&fo->node_len, old, nc, s, true))) return r;
    if ((r = grow_buf(&fo->node_left, old, nc, s, true))) return r;
    if ((r = grow_buf(&fo->node_right, old, nc, s, true))) return r;
    if ((r = grow_buf(&fo->node_jstar, old, nc, s, true))) return r;
    if ((r = grow_buf(&fo->node_flag, old, nc, s, true))) return r;
    if ((r = grow_buf(&fo->node_c, old, nc, s, true))) return r;
    // unused slots are marked by tree = -1
    if (cudaMemsetAsync(fo->node_tree + old, 0xFF, 4 * (nc - old), s) != cudaSuccess)
      return RPF_ECUDA;
    node_cap = nc;
    return RPF_OK;
  };
  auto ensure_leaves = [&](int64_t need) -> int {
    if (need <= leaf_cap) return RPF_OK;
    const int64_t nc = std::max<int64_t>(need, leaf_cap * 2);
    int r;
    if ((r = grow_buf(&fo->leaf_tree, leaf_cap, nc, s, true))) return r;
    if ((r = grow_buf(&fo->leaf_begin, leaf_cap, nc, s, true))) return r;
    if ((r = grow_buf(&fo->leaf_len, leaf_cap, nc, s, true))) return r;
    // unused slots are marked by len = 0
    if (cudaMemsetAsync(fo->leaf_len + leaf_cap, 0, 4 * (nc - leaf_cap), s) != cudaSuccess)
      return RPF_ECUDA;
    leaf_cap = nc;
    return RPF_OK;
  };
  RPF_TRY(ensure_nodes(std::max<int64_t>(4 * T + 4, (Tn / kSub) * 4 + 4 * T)));
  RPF_TRY(ensure_leaves(std::max<int64_t>(2 * T + 2, (Tn / kSub) * 2 + 2 * T)));

  int64_t n_nodes = T, n_leaves = 0, n_items = 0;
  {
    std::vector<uint64_t> key(T, 1ULL);
    std::vector<int32_t> tree(T), zero(T, 0), len(T, (int32_t)n), neg(T, -1);
    std::vector<double> cn(T, NAN);
    for (int t = 0; t < T; ++t) tree[t] = t;
    RPF_TRYCU(cudaMemcpyAsync(fo->node_key, key.data(), 8 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(fo->node_tree, tree.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(fo->node_begin, zero.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(fo->node_len, len.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(fo->node_left, neg.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(fo->node_right, neg.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(fo->node_jstar, neg.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(fo->node_flag, zero.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(fo->node_c, cn.data(), 8 * T, cudaMemcpyHostToDevice, s));
    if (n <= L) {  // every root is a leaf
      RPF_TRYCU(cudaMemcpyAsync(fo->leaf_tree, tree.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaMemcpyAsync(fo->leaf_begin, zero.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaMemcpyAsync(fo->leaf_len, len.data(), 4 * T, cudaMemcpyHostToDevice, s));
      n_leaves = T;
    } else if (n <= sub) {  // every root is a subtree item
      RPF_TRYCU(cudaMemcpyAsync(it_node, tree.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaMemcpyAsync(it_tree, tree.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaMemcpyAsync(it_begin, zero.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaMemcpyAsync(it_len, len.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaMemcpyAsync(it_key, key.data(), 8 * T, cudaMemcpyHostToDevice, s));
      n_items = T;
    }
    RPF_TRYCU(cudaStreamSynchronize(s));
  }

  // level arrays
  auto ensure_level = [&](int64_t F, int64_t C) -> int {
    int r;
    if (F > lv.cap_f) {
      const int64_t nf = std::max<int64_t>(F, lv.cap_f * 2);
      for (int q = 0; q < 2; ++q) {
        if ((r = grow_buf(&lv.fr_node[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_tree[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_begin[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_len[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_cb[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_nc[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_key[q], lv.cap_f, nf, s, true))) return r;
      }
      int32_t** i32s[] = {&lv.fr_ogid, &lv.fr_exact, &lv.fr_jstar, &lv.fr_flag, &lv.fr_nl};
      for (auto pp : i32s)
        if ((r = grow_buf(pp, 0, nf, s, false))) return r;
      double** f64s[] = {&lv.fr_a, &lv.fr_b, &lv.fr_c};
      for (auto pp : f64s)
        if ((r = grow_buf(pp, 0, nf, s, false))) return r;
      double** f64t[] = {&lv.fr_base, &lv.fr_mu, &lv.fr_min, &lv.fr_max};
      for (auto pp : f64t)
        if ((r = grow_buf(pp, 0, nf * ntry, s, false))) return r;
      float** f32s[] = {&lv.fr_tl, &lv.fr_tr, &lv.fr_rad, &lv.fr_wlo, &lv.fr_whi};
      for (auto pp : f32s)
        if ((r = grow_buf(pp, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_akey, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_bkey, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_cmask, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.md_key, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.md_id, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.md_rank, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.md_hist, 0, nf * 256, s, false))) return r;
      if ((r = grow_buf(&lv.md_fk, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.md_l0, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.md_lo, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.md_hi, 0, nf, s, false))) return r;
      if (median) {
        if ((r = grow_buf(&lv.md_bn, 0, nf, s, false))) return r;
        if ((r = grow_buf(&lv.md_done, 0, nf, s, false))) return r;
        if ((r = grow_buf(&lv.md_bk, 0, nf * kMedList, s, false))) return r;
        if ((r = grow_buf(&lv.md_bi, 0, nf * kMedList, s, false))) return r;
      }
      lv.cap_f = nf;
    }
    if (F * ntry > lv.cap_dir) {
      const int64_t nd = std::max<int64_t>(F * ntry, lv.cap_dir * 2);
      if ((r = grow_buf(&lv.dir64, 0, nd * d, s, false))) return r;
      if ((r = grow_buf(&lv.dir32, 0, nd * d, s, false))) return r;
      lv.cap_dir = nd;
    }
    if (C > lv.cap_c) {
      const int64_t ncap = std::max<int64_t>(C, lv.cap_c * 2);
      for (int q = 0; q < 2; ++q) {
        if ((r = grow_buf(&lv.ch_node[q], lv.cap_c, ncap, s, true))) return r;
        if ((r = grow_buf(&lv.ch_start[q], lv.cap_c, ncap, s, true))) return r;
        if ((r = grow_buf(&lv.ch_len[q], lv.cap_c, ncap, s, true))) return r;
      }
      if ((r = grow_buf(&lv.ch_nleft, 0, ncap, s, false))) return r;
      if ((r = grow_buf(&lv.ch_loff, 0, ncap, s, false))) return r;
      double** f64c[] = {&lv.cp_sum, &lv.cp_min, &lv.cp_max, &lv.cp_s1, &lv.cp_s2, &lv.cp_a};
      for (auto pp : f64c)
        if ((r = grow_buf(pp, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_min32, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_max32, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_rad, 0, ncap, s, false))) return r;
      if ((r = grow_buf(&lv.cp_rad2, 0, ncap, s, false))) return r;
      lv.cap_c = ncap;
    }
    return RPF_OK;
  };

  // ---- phase A: nodes of more than 4096 points, level by level ----------
  int64_t F = 0, C = 0;
  int cur = 0, level = 0;
  if (n > sub) {
    F = T;
    const int nc1 = (int)((n + RPF_CHUNK - 1) / RPF_CHUNK);
    C = (int64_t)T * nc1;
    RPF_TRY(ensure_level(F, C));
    std::vector<int32_t> node(T), tree(T), begin(T, 0), len(T, (int32_t)n), cb(T), ncv(T, nc1);
    std::vector<uint64_t> key(T, 1ULL);
    std::vector<int32_t> chn(C), chs(C), chl(C);
    for (int t = 0; t < T; ++t) {
      node[t] = t;
      tree[t] = t;
      cb[t] = t * nc1;
      for (int q = 0; q < nc1; ++q) {
        chn[t * nc1 + q] = t;
        chs[t * nc1 + q] = q * RPF_CHUNK;
        chl[t * nc1 + q] = (int32_t)std::min<int64_t>(RPF_CHUNK, n - (int64_t)q * RPF_CHUNK);
      }
    }
    RPF_TRYCU(cudaMemcpyAsync(lv.fr_node[0], node.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.fr_tree[0], tree.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.fr_begin[0], begin.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.fr_len[0], len.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.fr_cb[0], cb.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.fr_nc[0], ncv.data(), 4 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.fr_key[0], key.data(), 8 * T, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.ch_node[0], chn.data(), 4 * C, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.ch_start[0], chs.data(), 4 * C, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(lv.ch_len[0], chl.data(), 4 * C, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaStreamSynchronize(s));
  }
  const int TG = ntry <= 5 ? ntry : 8;
  const size_t smem_a = sizeof(float) * ((size_t)ntry * d + ((d + 3) & ~3) + 8 * 5 * 8 + 40 +
                                         ((d & 3) == 0 ? (size_t)(kBlock / 32) * kPaStages * RPF_TILE_FLOATS : 0));
  int32_t* perm_cur = perm_a;
  int32_t* perm_nxt = perm_b;
  while (F > 0) {
    // room for this level and for what k_frontier writes (<= 2F children,
    // <= C + 2F chunks), grown before any pointer of this level is captured
    RPF_TRY(ensure_level(2 * F, C + 2 * F));
    RPF_TRY(ensure_nodes(n_nodes + 2 * F));
    RPF_TRY(ensure_leaves(n_leaves + 2 * F));
    const int Fi = (int)F, Ci = (int)C;
    int32_t *fr_node = lv.fr_node[cur], *fr_tree = lv.fr_tree[cur], *fr_begin = lv.fr_begin[cur],
            *fr_len = lv.fr_len[cur], *fr_cb = lv.fr_cb[cur], *fr_nc = lv.fr_nc[cur];
    uint64_t* fr_key = lv.fr_key[cur];
    int32_t *ch_node = lv.ch_node[cur], *ch_start = lv.ch_start[cur], *ch_len = lv.ch_len[cur];

    RPF_LAUNCH("k_dirs_a", s, k_dirs_a<<<nblk(F * ntry * 32, 128), 128, 0, s>>>(
        Fi, ntry, d, seed, fo->t_base, n, fr_tree, fr_begin, fr_key, perm_cur, fo->X, lv.dir64, lv.dir32,
        lv.fr_base, lv.fr_ogid));
#define RPF_PROJ_A(TGV)                                                                          \
  do {                                                                                           \
    if (smem_a > 48 * 1024)                                                                      \
      cudaFuncSetAttribute(k_proj_a<TGV>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                           (int)smem_a);                                                         \
    RPF_LAUNCH("k_proj_a", s, k_proj_a<TGV><<<Ci, kBlock, smem_a, s>>>(                          \
        ch_node, ch_start, ch_len, fr_tree, fr_begin, lv.fr_ogid, fo->X, perm_cur, fo->xnorm, n, \
        Tn, d, ntry, lv.dir32, p32, lv.cp_s1, lv.cp_s2, lv.cp_a, lv.cp_min32, lv.cp_max32,       \
        lv.cp_rad, lv.cp_rad2));                                                                 \
  } while (0)
    switch (TG) {
      case 1: RPF_PROJ_A(1); break;
      case 2: RPF_PROJ_A(2); break;
      case 3: RPF_PROJ_A(3); break;
      case 4: RPF_PROJ_A(4); break;
      case 5: RPF_PROJ_A(5); break;
      default: RPF_PROJ_A(8); break;
    }
#undef RPF_PROJ_A
    RPF_LAUNCH("k_certify_a", s, k_certify_a<<<nblk(F * 32, 128), 128, 0, s>>>(
        Fi, ntry, exact_only, fr_cb, fr_nc, fr_len, lv.cp_s1, lv.cp_s2, lv.cp_a, lv.cp_min32,
        lv.cp_max32, lv.cp_rad, lv.cp_rad2, lv.fr_base, lv.fr_exact, lv.fr_jstar, lv.fr_rad, lv.fr_wlo,
        lv.fr_whi, lv.fr_akey, lv.fr_bkey, lv.fr_cmask));
    // chunks of exact nodes are listed (in ch_loff, which k_node_scan fills
    // later) so that their FP64 work spreads over the GPU
    RPF_TRYCU(cudaMemsetAsync(ex_count, 0, sizeof(int32_t), s));
    RPF_LAUNCH("k_cand", s, k_cand<<<Ci, kBlock, 0, s>>>(
        ch_node, ch_start, ch_len, fr_tree, fr_begin, lv.fr_exact, lv.fr_jstar, lv.fr_wlo,
        lv.fr_whi, fo->X, perm_cur, n, Tn, d, ntry, p32, lv.dir64, lv.fr_akey, lv.fr_bkey,
        lv.ch_loff, ex_count));
    RPF_LAUNCH("k_proj64", s, k_proj64<<<4 * 152, kBlock, 0, s>>>(
        lv.ch_loff, ex_count, ch_node, ch_start, ch_len, fr_tree, fr_begin, fo->X, perm_cur, n,
        Tn, d, ntry, lv.dir64, lv.fr_cmask, p64));
    for (int pass = 0; pass < 2; ++pass) {
      RPF_LAUNCH("k_csum_chunks", s, k_csum_chunks<<<2 * 152, 256, 0, s>>>(
          pass, lv.ch_loff, ex_count, ntry, ch_node, ch_start, ch_len, fr_tree, fr_begin,
          lv.fr_cmask, n, Tn, p64, lv.fr_mu, lv.cp_sum, lv.cp_min, lv.cp_max));
      RPF_LAUNCH("k_csum_nodes", s, k_csum_nodes<<<nblk(F * 32, 256), 256, 0, s>>>(
          pass, Fi, ntry, fr_cb, fr_nc, fr_len, lv.fr_exact, lv.fr_cmask, lv.cp_sum, lv.cp_min, lv.cp_max,
          lv.fr_mu, lv.fr_min, lv.fr_max, lv.fr_jstar, lv.fr_a, lv.fr_b));
    }
    if (median) {
      RPF_LAUNCH("k_med_init", s, k_med_init<<<nblk(F, 128), 128, 0, s>>>(
          Fi, fr_len, lv.md_fk, lv.md_key, lv.md_id, lv.md_rank, lv.md_l0, lv.md_bn, lv.md_done));
      RPF_TRYCU(cudaMemsetAsync(lv.md_hist, 0, sizeof(int32_t) * 256 * (size_t)F, s));
      for (int pass = 0; pass < 16; ++pass) {
        if (pass == 4) {
          // the band around the FP32 median; exact keys only inside it; a
          // band of at most kMedList points is settled directly, and the
          // radix passes run only if some node still needs them
          RPF_LAUNCH("k_med_band", s, k_med_band<<<Ci, kBlock, 0, s>>>(
              ch_node, ch_start, ch_len, fr_tree, fr_begin, lv.fr_exact, lv.fr_jstar, lv.fr_rad,
              fo->X, perm_cur, n, Tn, d, ntry, lv.dir64, p32, lv.md_fk, p64, lv.md_l0, lv.md_bn,
              lv.md_bk, lv.md_bi));
          RPF_LAUNCH("k_med_rank", s, k_med_rank<<<nblk(F, 128), 128, 0, s>>>(
              Fi, fr_len, lv.fr_exact, lv.fr_jstar, lv.fr_rad, lv.md_fk, lv.md_l0, lv.md_rank,
              lv.md_lo, lv.md_hi));
          RPF_TRYCU(cudaMemsetAsync(&d_cnt->n_radix, 0, sizeof(int32_t), s));
          RPF_LAUNCH("k_med_direct", s, k_med_direct<<<nblk(F * 32, 128), 128, 0, s>>>(
              Fi, lv.fr_exact, lv.fr_jstar, lv.md_bn, lv.md_bk, lv.md_bi, lv.md_rank, lv.md_key,
              lv.md_id, lv.md_done, &d_cnt->n_radix));
          RPF_TRYCU(cudaMemcpyAsync(&h_cnt->n_radix, &d_cnt->n_radix, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, s));
          RPF_TRYCU(cudaStreamSynchronize(s));
          if (h_cnt->n_radix == 0) break;
        }
        RPF_LAUNCH("k_med_hist", s, k_med_hist<<<Ci, kBlock, 0, s>>>(
            pass, ch_node, ch_start, ch_len, fr_tree, fr_begin, lv.fr_exact, lv.fr_jstar, perm_cur,
            n, Tn, p32, p64, lv.md_fk, lv.md_key, lv.md_id, lv.md_lo, lv.md_hi, lv.md_done,
            lv.md_hist));
        RPF_LAUNCH("k_med_select", s, k_med_select<<<nblk(F * 32, 128), 128, 0, s>>>(
            pass, Fi, lv.fr_exact, lv.fr_jstar, lv.md_done, lv.md_fk, lv.md_key, lv.md_id,
            lv.md_rank, lv.md_hist));
      }
    }
    RPF_LAUNCH("k_split_a", s, k_split_a<<<nblk(F, 128), 128, 0, s>>>(
        Fi, ntry, seed, fo->t_base, median, fr_node, fr_tree, fr_key, lv.fr_exact, lv.fr_jstar, lv.fr_a,
        lv.fr_b, lv.fr_akey, lv.fr_bkey, lv.fr_base, lv.fr_rad, lv.md_key, lv.fr_c, lv.fr_flag,
        lv.fr_tl, lv.fr_tr, fo->node_jstar, fo->node_flag, fo->node_c, d_exact));
    RPF_LAUNCH("k_side_count", s, k_side_count<<<Ci, kBlock, 0, s>>>(
        ch_node, ch_start, ch_len, fr_tree, fr_begin, fr_len, lv.fr_exact, lv.fr_jstar,
        lv.fr_flag, lv.fr_c, lv.fr_tl, lv.fr_tr, fo->X, perm_cur, n, Tn, d, ntry, p32, p64,
        lv.dir64, median, lv.md_key, lv.md_id, lv.md_lo, lv.md_hi, side, lv.ch_nleft));
    RPF_LAUNCH("k_node_scan", s, k_node_scan<<<nblk(F, 128), 128, 0, s>>>(
        Fi, n_nodes, fr_node, fr_tree, fr_begin, fr_len, fr_key, fr_cb, fr_nc, lv.ch_nleft,
        lv.ch_loff, lv.fr_nl, fo->node_key, fo->node_tree, fo->node_begin, fo->node_len,
        fo->node_left, fo->node_right, fo->node_jstar, fo->node_flag, fo->node_c));
    RPF_LAUNCH("k_scatter", s, k_scatter<<<Ci, kBlock, 0, s>>>(
        ch_node, ch_start, ch_len, lv.ch_loff, fr_tree, fr_begin, fr_len, lv.fr_nl, n, sub,
        side, perm_cur, perm_nxt, fo->perm));
    const int nxt = cur ^ 1;
    RPF_LAUNCH("k_frontier", s, k_frontier<<<1, 1024, 0, s>>>(
        Fi, L, sub, n_nodes, fr_tree, fr_begin, fr_len, fr_key, lv.fr_nl, lv.fr_node[nxt],
        lv.fr_tree[nxt], lv.fr_begin[nxt], lv.fr_len[nxt], lv.fr_key[nxt], lv.fr_cb[nxt],
        lv.fr_nc[nxt], lv.ch_node[nxt], lv.ch_start[nxt], lv.ch_len[nxt], n_leaves, fo->leaf_tree,
        fo->leaf_begin, fo->leaf_len, n_items, it_node, it_tree, it_begin, it_len, it_key, d_cnt));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt, d_cnt, sizeof(Counts), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cleanup();
      return rpf_cuda_err(e);
    }
    n_nodes += 2 * F;
    n_leaves += h_cnt->n_leaves_new;
    n_items += h_cnt->n_items_new;
    F = h_cnt->f_next;
    C = h_cnt->c_next;
    std::swap(perm_cur, perm_nxt);
    cur = nxt;
    ++level;
  }
  free_level();

  // ---- phase B: every item's subtree inside one CTA -----------------------
  int64_t nodes_used = n_nodes, leaves_used = n_leaves;
  int32_t* dfr = nullptr;
  int* dfr_cnt = nullptr;
  int dfr_cap = 0;
  if (n_items > 0) {
    std::vector<int32_t> ilen(n_items), nb(n_items), lb(n_items);
    RPF_TRYCU(cudaMemcpyAsync(ilen.data(), it_len, 4 * n_items, cudaMemcpyDeviceToHost, s));
    RPF_TRYCU(cudaStreamSynchronize(s));
    int64_t nrun = n_nodes, lrun = n_leaves;
    for (int64_t i = 0; i < n_items; ++i) {
      nb[i] = (int32_t)nrun;  // a subtree of m points has at most 2m - 1 nodes
      lb[i] = (int32_t)lrun;  // and at most m leaves
      nrun += 2 * (int64_t)ilen[i] - 2;
      lrun += ilen[i];
    }
    if (nrun >= ((int64_t)1 << 31) || lrun >= ((int64_t)1 << 31)) {
      cleanup();
      return RPF_EINVAL;
    }
    RPF_TRY(ensure_nodes(nrun));
    RPF_TRY(ensure_leaves(lrun));
    RPF_TRYCU(cudaMemcpyAsync(it_nbase, nb.data(), 4 * n_items, cudaMemcpyHostToDevice, s));
    RPF_TRYCU(cudaMemcpyAsync(it_lbase, lb.data(), 4 * n_items, cudaMemcpyHostToDevice, s));
    // records of the deferred split points: room for four split nodes per
    // leaf-bound's worth of phase-B points (at most 64 MB); a subtree that
    // finds the list full decides its split point in place
    if (fo->prm.growth != 1 && fo->prm.split_rule == 0) {
      int64_t pts = 0;
      for (int64_t i = 0; i < n_items; ++i) pts += ilen[i];
      dfr_cap = (int)std::min<int64_t>(4 * pts / std::max(L, 1) + 1024,
                                       (64ll << 20) / (4 * RPF_DEFER_REC));
      RPF_TRY(talloc((void**)&dfr, 4 * (size_t)RPF_DEFER_REC * dfr_cap));
      RPF_TRY(talloc((void**)&dfr_cnt, sizeof(int)));
      RPF_TRYCU(cudaMemsetAsync(dfr_cnt, 0, sizeof(int), s));
    }
    RPF_TRY(rpf_grow_subtrees(fo, n_items, ilen.data(), it_node, it_tree, it_begin, it_len, it_key, it_nbase,
                              it_lbase, p32, p64, d_exact, d_err, dfr, dfr_cnt, dfr_cap, s));
    nodes_used = nrun;
    leaves_used = lrun;
  }

  // ---- compact the node and leaf tables, regenerate chosen directions ----
  {
    const int64_t N = nodes_used;
    int32_t *blk = nullptr, *new_id = nullptr, *d_tot = nullptr;
    const int64_t nbmax = (std::max(nodes_used, leaves_used) + 1023) / 1024 + 1;
    RPF_TRY(talloc((void**)&blk, 4 * (size_t)nbmax));
    RPF_TRY(talloc((void**)&new_id, 4 * (size_t)std::max<int64_t>(N, 1)));
    RPF_TRY(talloc((void**)&d_tot, 8));
    const int32_t* ntree = fo->node_tree;
    rpf_scan(
        N, [=] __device__(int64_t i) -> int { return ntree[i] >= 0 ? 1 : 0; },
        [=] __device__(int64_t i, int p) { new_id[i] = ntree[i] >= 0 ? p : -1; }, blk, d_tot, s);
    int32_t tot[2] = {0, 0};
    int err_h = 0;
    RPF_TRYCU(cudaMemcpyAsync(&tot[0], d_tot, 4, cudaMemcpyDeviceToHost, s));
    RPF_TRYCU(cudaMemcpyAsync(&err_h, d_err, 4, cudaMemcpyDeviceToHost, s));
    RPF_TRYCU(cudaStreamSynchronize(s));
    if (err_h) {
      cleanup();
      return RPF_EINTERNAL;
    }
    const int32_t total = tot[0];
    const int64_t M = std::max<int64_t>(total, 1);
    uint64_t* okey = nullptr;
    int32_t *otree = nullptr, *obegin = nullptr, *olen = nullptr, *oleft = nullptr,
            *oright = nullptr, *ojstar = nullptr, *oflag = nullptr;
    double* oc = nullptr;
    int rc = rpf_alloc((void**)&okey, 8 * M, s);
    if (!rc) rc = rpf_alloc((void**)&otree, 4 * M, s);
    if (!rc) rc = rpf_alloc((void**)&obegin, 4 * M, s);
    if (!rc) rc = rpf_alloc((void**)&olen, 4 * M, s);
    if (!rc) rc = rpf_alloc((void**)&oleft, 4 * M, s);
    if (!rc) rc = rpf_alloc((void**)&oright, 4 * M, s);
    if (!rc) rc = rpf_alloc((void**)&ojstar, 4 * M, s);
    if (!rc) rc = rpf_alloc((void**)&oflag, 4 * M, s);
    if (!rc) rc = rpf_alloc((void**)&oc, 8 * M, s);
    if (rc) {
      void* ps[] = {okey, otree, obegin, olen, oleft, oright, ojstar, oflag, oc};
      for (void* p : ps) rpf_release(p, s);
      cleanup();
      return RPF_ENOMEM;
    }
    RPF_LAUNCH("k_compact_nodes", s, k_compact_nodes<<<nblk(N, 256), 256, 0, s>>>(
        N, new_id, fo->node_key, fo->node_tree, fo->node_begin, fo->node_len, fo->node_left,
        fo->node_right, fo->node_jstar, fo->node_flag, fo->node_c, okey, otree, obegin, olen,
        oleft, oright, ojstar, oflag, oc));
    void* olds[] = {fo->node_key, fo->node_tree, fo->node_begin, fo->node_len, fo->node_left,
                    fo->node_right, fo->node_jstar, fo->node_flag, fo->node_c};
    for (void* p : olds) rpf_release(p, s);
    fo->node_key = okey;
    fo->node_tree = otree;
    fo->node_begin = obegin;
    fo->node_len = olen;
    fo->node_left = oleft;
    fo->node_right = oright;
    fo->node_jstar = ojstar;
    fo->node_flag = oflag;
    fo->node_c = oc;
    fo->n_nodes = total;
    fo->nodes_cap = total;
    if (rpf_alloc((void**)&fo->node_dir32, sizeof(float) * M * d, s)) {
      cleanup();
      return RPF_ENOMEM;
    }
    RPF_LAUNCH("k_node_dirs", s, k_node_dirs<<<nblk((int64_t)total * 32, 128), 128, 0, s>>>(
        total, d, seed, fo->t_base, fo->node_key, fo->node_tree, fo->node_left, fo->node_jstar, fo->node_flag,
        fo->node_dir32));
    RPF_TRY(rpf_split_deferred(fo, dfr, dfr_cnt, dfr_cap, new_id, d_err, s));
    RPF_TRY(rpf_build_route(fo, s));

    // leaves: keep the used slots (len > 0) in slot order
    const int64_t S = leaves_used;
    const int32_t* llen = fo->leaf_len;
    int32_t* lpos = new_id;  // reuse: S <= N + items is not guaranteed, so size check
    if (S > N) RPF_TRY(talloc((void**)&lpos, 4 * (size_t)S));
    rpf_scan(
        S, [=] __device__(int64_t i) -> int { return llen[i] > 0 ? 1 : 0; },
        [=] __device__(int64_t i, int p) { lpos[i] = llen[i] > 0 ? p : -1; }, blk, d_tot + 1, s);
    RPF_TRYCU(cudaMemcpyAsync(&tot[1], d_tot + 1, 4, cudaMemcpyDeviceToHost, s));
    RPF_TRYCU(cudaStreamSynchronize(s));
    const int64_t NL = std::max<int32_t>(tot[1], 1);
    int32_t *lt = nullptr, *lb = nullptr, *ll = nullptr;
    if (rpf_alloc((void**)&lt, 4 * NL, s) || rpf_alloc((void**)&lb, 4 * NL, s) ||
        rpf_alloc((void**)&ll, 4 * NL, s)) {
      rpf_release(lt, s);
      rpf_release(lb, s);
      cleanup();
      return RPF_ENOMEM;
    }
    const int32_t *st = fo->leaf_tree, *sb = fo->leaf_begin;
    RPF_LAUNCH("k_compact_leaves", s, k_compact_leaves<<<nblk(S, 256), 256, 0, s>>>(
        S, lpos, st, sb, llen, lt, lb, ll));
    rpf_release(fo->leaf_tree, s);
    rpf_release(fo->leaf_begin, s);
    rpf_release(fo->leaf_len, s);
    fo->leaf_tree = lt;
    fo->leaf_begin = lb;
    fo->leaf_len = ll;
    fo->n_leaves = tot[1];
  }
  {
    unsigned long long ex = 0;
    int err_h = 0;  // also covers the deferred split points
    RPF_TRYCU(cudaMemcpyAsync(&ex, d_exact, sizeof(ex), cudaMemcpyDeviceToHost, s));
    RPF_TRYCU(cudaMemcpyAsync(&err_h, d_err, 4, cudaMemcpyDeviceToHost, s));
    RPF_TRYCU(cudaStreamSynchronize(s));
    if (err_h) {
      cleanup();
      return RPF_EINTERNAL;
    }
    fo->n_exact = (int64_t)ex;
    fo->max_depth = level;  // phase-A levels
  }
  cleanup();
  return RPF_OK;
#undef RPF_TRY
#undef RPF_TRYCU
}

void rpf_launch_directions(uint64_t seed, int32_t t, const uint64_t* keys_dev, int32_t n_keys,
                           int32_t j, int32_t d, double* out_dev, cudaStream_t s) {
  RPF_LAUNCH("k_dirs_keys", s,
             k_dirs_keys<<<nblk(n_keys, 64), 64, 0, s>>>(seed, t, keys_dev, n_keys, j, d, out_dev));
}
