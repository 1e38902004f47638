// rpf_subtree.cu -- phase B of rpTree growth: one CTA grows the whole subtree
// of a node of at most 4096 points (Sec. 2, Algorithm 1 with Algorithm 2 for
// every split), with no launch or host round trip per level.
//
// The subtree's permutation segment lives in shared memory.  Nodes are taken
// depth first from a small stack; after a split the larger child is pushed
// first so the smaller one is processed next, which keeps the stack depth
// below log2(4096) + 2.  Per node the CTA
//   1. draws the nTry candidate directions (FP32 Box-Muller, FP32 normalise)
//   2. takes o = the node's first member and b_j = p64(o, r_j)
//   3. projects every point: q' = fl32-dot(r32, fl32(x - o)) with the rows
//      staged per warp through shared-memory tiles, error radius, block
//      statistics (FP32 per thread, FP64 across warps)
//   4. certifies Algorithm 2's choice, or recomputes the node in FP64 with the
//      canonical reduction (one chunk: the node has <= 4096 points) for the
//      tries the bounds leave in contention
//   5. finds the exact min / max (FP64 on the few candidates) and draws c,
//      or selects the median
//   6. decides every point's side (certified from q', else FP64) and
//      partitions the segment stably
//   7. records the node and its children; leaves are written to the final
//      permutation, inner children pushed.
// Node ids and leaf slots come from ranges reserved per subtree (2m - 2 ids,
// m leaf slots for m points), so the layout is deterministic.  CTAs have 128
// threads (at most 32 points per thread in the statistics).
#include <cuda_runtime.h>

#include <type_traits>
#include <math.h>

#include <algorithm>

#include "rpf_decide.cuh"
#include "rpf_proj.cuh"

namespace {

constexpr int kB = 128;  // 4 warps; 4 CTAs per SM hide each other's serial sections
constexpr int kSmallB = 32;  // small subtrees: one warp per CTA, many CTAs per SM
constexpr int kSubN = RPF_CHUNK;
constexpr int kStack = 24;
constexpr int kBandSel = 256;  // median rule: bands up to this size are selected by counting
constexpr int kDefCand = RPF_DEFER_CAND;  // candidates per extreme of a deferred split point
// the projection's row tiles (kTStages per warp, 32 rows of kTDC + 4 floats)
// live in sT and sSide, which are contiguous and idle during the projection,
// and in sTx, which follows them
constexpr int kTDC = 16, kTStages = 2;
__host__ __device__ constexpr size_t tile_bytes(int nt) {
  return (size_t)(nt / 32) * kTStages * 32 * (kTDC + 4) * 4;
}
// the median rule's band list and histogram also live in sT (idle while the
// median is selected): sT must hold them
constexpr int kBandBytes = 12 * kBandSel + 4 * 256;
static_assert(kBandBytes <= 4 * kSubN, "band list and histogram fit sT");

struct SubState {
  uint64_t key;
  int nb, m, id;
  int exact, js, flag, nl;
  double a, b, c;
  float tl, tr, rad, wlo, whi;
  unsigned long long akey, bkey;
  unsigned long long cmask;  // tries still in contention at an exact node
  int top, next_id, id_end, next_leaf, leaf_end;
  int leafL, leafR, err, ncand;
  unsigned long long mkey;  // median rule: key, point index and rank being selected
  uint32_t mid, mfk;        // ... and the FP32 key of the band's centre
  int mrank;
  float mlo, mhi;           // band of q' outside which the side is certain
  // deferred split point: certified interval thresholds of the sides and the
  // candidates of the exact minimum / maximum
  int defer, nmin, nmax;
  float dtl, dtr;
  double u0;  // uniform of split attempt 0
  int cmin[kDefCand], cmax[kDefCand];
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

struct SubLayout {
  size_t sP, sT, sSide, sTx, r64, r32, so, sbase, sS1, sS2, sA, sinv, smn, smx, svh, slo, shi, sdtl,
      sdtr, red, total;
};

// subn: the most points of a subtree (sP and sT hold one int per point, a
// multiple of 16); nt: threads of the CTA
__host__ __device__ inline SubLayout sub_layout(int d, int ntry, int TG, int nt, int subn) {
  SubLayout l{};
  size_t o = 0;
  const size_t tb = tile_bytes(nt);
  l.sP = o;
  o = align16(o + 4 * (size_t)subn);
  l.sT = o;
  o = align16(o + 4 * (size_t)subn);
  l.sSide = o;
  o = align16(o + (size_t)subn);
  l.sTx = o;
  o = align16(o + (tb > 5 * (size_t)subn ? tb - 5 * (size_t)subn : 0));
  l.r64 = o;
  o = align16(o + 8 * (size_t)ntry * d);
  l.r32 = o;
  o = align16(o + 4 * (size_t)ntry * d);
  l.so = o;
  o = align16(o + 4 * (size_t)d);
  l.sbase = o;
  o = align16(o + 8 * (size_t)ntry);
  l.sS1 = o;
  o = align16(o + 8 * (size_t)ntry);
  l.sS2 = o;
  o = align16(o + 8 * (size_t)ntry);
  l.sA = o;
  o = align16(o + 8 * (size_t)ntry);
  l.sinv = o;
  o = align16(o + 8 * (size_t)ntry);
  l.smn = o;
  o = align16(o + 4 * (size_t)ntry);
  l.smx = o;
  o = align16(o + 4 * (size_t)ntry);
  l.svh = o;
  o = align16(o + 8 * (size_t)ntry);
  l.slo = o;
  o = align16(o + 4 * (size_t)ntry);
  l.shi = o;
  o = align16(o + 4 * (size_t)ntry);
  l.sdtl = o;
  o = align16(o + 4 * (size_t)ntry);
  l.sdtr = o;
  o = align16(o + 4 * (size_t)ntry);
  l.red = o;
  o = align16(o + 4 * (size_t)(8 * TG * 5 + 40));
  l.total = o;
  return l;
}

// Subtree items: (root node id, tree, begin in the tree's permutation, point
// count, root key, first node id and first leaf slot reserved for it).
struct SubItems {
  int32_t *node, *tree, *begin, *len;
  uint64_t* key;
  int32_t *nbase, *lbase;
};

// NT threads per CTA.  Items: it_idx[blockIdx.x] of `in` (one per CTA) when
// it_count is null; else items 0 .. *it_count - 1 of `in`, CTAs taking them
// in turn.  subn: capacity of the shared permutation segment.  defer_max > 0:
// an inner node of at most defer_max points is not grown here; its segment is
// written back, 2m - 2 node ids and m leaf slots are reserved for it, and it
// becomes an item of `out` (slot from *out_cnt, at most out_cap).
template <int TG, int NT>
__global__ void __launch_bounds__(NT, NT == 32 ? 16 : 4) k_subtree(
    SubItems in, const int32_t* it_idx, int n_items, const int* it_count, int subn,
    int defer_max, SubItems out, int* out_cnt, int out_cap,
    const float* __restrict__ X, const float* __restrict__ xnorm, int64_t n, int64_t Tn, int d,
    int ntry, int L, uint64_t seed, int t_base, int exact_only, int median, int32_t* perm_final,
    float* p32,
    double* p64,
    uint64_t* node_key, int32_t* node_tree, int32_t* node_begin, int32_t* node_len,
    int32_t* node_left, int32_t* node_right, int32_t* node_jstar, int32_t* node_flag,
    double* node_c, int32_t* leaf_tree, int32_t* leaf_begin, int32_t* leaf_len,
    unsigned long long* d_exact, int* d_err, int32_t* dfr, int* dfr_cnt, int dfr_cap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const SubLayout lay = sub_layout(d, ntry, TG, NT, subn);
  int32_t* sP = reinterpret_cast<int32_t*>(smraw + lay.sP);
  int32_t* sT = reinterpret_cast<int32_t*>(smraw + lay.sT);
  uint8_t* sSide = smraw + lay.sSide;
  double* r64 = reinterpret_cast<double*>(smraw + lay.r64);
  float* r32 = reinterpret_cast<float*>(smraw + lay.r32);
  float* so = reinterpret_cast<float*>(smraw + lay.so);
  double* sbase = reinterpret_cast<double*>(smraw + lay.sbase);
  double* sS1 = reinterpret_cast<double*>(smraw + lay.sS1);
  double* sS2 = reinterpret_cast<double*>(smraw + lay.sS2);
  double* sA = reinterpret_cast<double*>(smraw + lay.sA);
  float* sinv = reinterpret_cast<float*>(smraw + lay.sinv);
  float* smn = reinterpret_cast<float*>(smraw + lay.smn);
  float* smx = reinterpret_cast<float*>(smraw + lay.smx);
  double* svh = reinterpret_cast<double*>(smraw + lay.svh);
  float* slo = reinterpret_cast<float*>(smraw + lay.slo);
  float* shi = reinterpret_cast<float*>(smraw + lay.shi);
  float* sdtl = reinterpret_cast<float*>(smraw + lay.sdtl);
  float* sdtr = reinterpret_cast<float*>(smraw + lay.sdtr);
  float* red = reinterpret_cast<float*>(smraw + lay.red);
  __shared__ SubState S;
  __shared__ int st_nb[kStack], st_m[kStack], st_id[kStack];
  __shared__ uint64_t st_key[kStack];
  __shared__ int wsc[NT / 32];
  // median rule: a small band's keys and point indices, and the radix histogram
  unsigned long long* bnd_key = reinterpret_cast<unsigned long long*>(smraw + lay.sT);
  uint32_t* bnd_id = reinterpret_cast<uint32_t*>(smraw + lay.sT + 8 * kBandSel);
  int* mhist = reinterpret_cast<int*>(smraw + lay.sT + 12 * kBandSel);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nit = it_count ? *it_count : n_items;
  for (int ii = blockIdx.x; ii < nit; ii += gridDim.x) {
  const int it = it_idx ? it_idx[ii] : ii;
  const int t = in.tree[it];
  const int m0 = in.len[it];
  const int64_t pbase = (int64_t)t * n + in.begin[it];
  for (int i = tid; i < m0; i += NT) sP[i] = perm_final[pbase + i];
  if (tid == 0) {
    S.top = 1;
    st_nb[0] = 0;
    st_m[0] = m0;
    st_id[0] = in.node[it];
    st_key[0] = in.key[it];
    S.next_id = in.nbase[it];
    S.id_end = in.nbase[it] + 2 * m0 - 2;
    S.next_leaf = in.lbase[it];
    S.leaf_end = in.lbase[it] + m0;
    S.err = 0;
  }
  __syncthreads();
  const int npairs = (d + 1) / 2;

  while (true) {
    if (tid == 0) {
      if (S.top == 0 || S.err) {
        S.m = -1;
      } else {
        const int k = --S.top;
        S.nb = st_nb[k];
        S.m = st_m[k];
        S.id = st_id[k];
        S.key = st_key[k];
      }
    }
    __syncthreads();
    if (S.m < 0) break;
    const int nb = S.nb, m = S.m, id = S.id;
    const uint64_t key = S.key;

    if (m <= defer_max) {  // a small subtree: handed to the one-warp kernel
      for (int i = tid; i < m; i += NT) perm_final[pbase + nb + i] = sP[nb + i];
      if (tid == 0) {
        const int nbase = S.next_id, lbase = S.next_leaf;
        S.next_id += 2 * m - 2;
        S.next_leaf += m;
        const int slot = S.next_id > S.id_end || S.next_leaf > S.leaf_end ? out_cap
                                                                           : atomicAdd(out_cnt, 1);
        if (slot >= out_cap) {
          S.err = 1;
        } else {
          out.node[slot] = id;
          out.tree[slot] = t;
          out.begin[slot] = in.begin[it] + nb;
          out.len[slot] = m;
          out.key[slot] = key;
          out.nbase[slot] = nbase;
          out.lbase[slot] = lbase;
        }
      }
      __syncthreads();
      continue;
    }

    // 1. candidate directions, all in FP32 (r32), widened copy in r64: the
    // Box-Muller pairs of all tries are spread over the threads, thread j
    // forms try j's sequential FP32 norm, then every value is scaled; 2. with
    // it, the centre o = the node's first member (its row and norm are
    // requested first, so their loads overlap the draws) and attempt 0's
    // uniform of the split point
    const int og = sP[nb];
    const float* xo = X + (int64_t)og * d;
    float oreg = tid < d ? xo[tid] : 0.0f;
    const float on = xnorm[og];
    if (tid == NT - 1) S.u0 = rpf_u53(rpf_word(seed, RPF_TAG_SPLIT, (uint64_t)(t + t_base), key, 0, 0));
    for (int w = tid; w < ntry * npairs; w += NT) {
      const int j = w / npairs, i = w - j * npairs;
      const uint64_t hj = rpf_word_prefix(seed, RPF_TAG_DIR, (uint64_t)(t + t_base), key, (uint64_t)j);
      float g0, g1;
      rpf_gauss_pair_h(hj, i, &g0, &g1);
      r32[j * d + 2 * i] = g0;
      if (2 * i + 1 < d) r32[j * d + 2 * i + 1] = g1;
    }
    if (tid < d) so[tid] = oreg;
    for (int k = tid + NT; k < d; k += NT) so[k] = xo[k];
    __syncthreads();
    if (tid < ntry) sinv[tid] = rpf_inv_norm32(r32 + tid * d, d);
    __syncthreads();
    for (int w = tid; w < ntry * d; w += NT) {
      const int j = w / d, k = w - j * d;
      const float inv = sinv[j];
      const float v = inv == 0.0f ? (k == 0 ? 1.0f : 0.0f) : __fmul_rn(r32[w], inv);
      r32[w] = v;
      r64[w] = (double)v;
    }
    __syncthreads();

    // 3. centred FP32 projections and statistics
    float radmax = 0.0f, rad2 = 0.0f;  // rad2: rounded-up sum of the points' rad^2
    if (!exact_only) {
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
          // batches of 32 positions, one per lane; each warp stages its
          // units (batch, kTDC-coordinate chunk) ahead into row tiles held in
          // the partition scratch
          float* tb = reinterpret_cast<float*>(smraw + lay.sT) + warp * kTStages * 32 * (kTDC + 4);
          // TG is nTry itself when nTry <= 5 (the launch picks it so): one pass
          // then covers every try, with the sum of squares
          auto project = [&](auto dfull) {
            rpf_warp_project<TG, kTDC, kTStages, (TG <= 5), decltype(dfull)::value>(
                X, d, sP + nb, m, warp, NT / 32, tb, so, r32 + j0 * d, nj, j0 == 0, lane,
                j0 == 0 ? xnorm : nullptr,
                [&](int pos, int gid, const float(&acc)[TG], float nn, float xn) {
                  if (TG <= 5 || j0 == 0) {
                    const float r = rpf_point_rad(d, nn, xn, on);
                    radmax = fmaxf(radmax, r);
                    rad2 = __fmaf_ru(r, r, rad2);
                  }
#pragma unroll
                  for (int q = 0; q < TG; ++q) {
                    if (TG <= 5 || q < nj) {
                      p32[(int64_t)((TG <= 5 ? 0 : j0) + q) * Tn + pbase + nb + pos] = acc[q];
                      rpf_stat_add(acc[q], s1[q], s2[q], a1[q], mn[q], mx[q]);
                    }
                  }
                });
          };
          // whole chunks when d is a multiple of the chunk width
          if (d % kTDC == 0) project(std::true_type{});
          else project(std::false_type{});
        } else {
          for (int u0 = 0; u0 * NT < m; u0 += 4) {
            int gid[4], pos[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              pos[p] = tid + NT * (u0 + p);
              gid[p] = pos[p] < m ? sP[nb + pos[p]] : -1;
            }
            float acc[4][TG], nn[4];
            rpf_proj4<TG>(X, d, gid, so, r32 + j0 * d, nj, acc, nn, j0 == 0);
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
                  p32[(int64_t)(j0 + q) * Tn + pbase + nb + pos[p]] = v;
                  rpf_stat_add(v, s1[q], s2[q], a1[q], mn[q], mx[q]);
                }
              }
            }
          }
        }
        rpf_block_stats<TG>(nj, s1, s2, a1, mn, mx, red, sS1 + j0, sS2 + j0, sA + j0, smn + j0,
                            smx + j0, j0 == 0 ? &radmax : nullptr, &rad2);
      }
    }

    // 4. certify the choice of Algorithm 2
    if (!exact_only) {
      // bounds of every try; with at most 32 tries warp 0 holds them all
      // and certifies right after (a warp sync instead of a block barrier)
      const double inv_m = 1.0 / (double)m;
      for (int j = tid; j < ntry; j += NT) {
        rpf_try_bounds(m, inv_m, sS1[j], sS2[j], sA[j], (double)on, radmax, __fsqrt_ru(rad2),
                       &svh[j], &slo[j], &shi[j]);
        // the deferred split point's interval for every try, in parallel
        // (independent of the bounds above, so the two chains overlap)
        if (!median && dfr_cap > 0) {
          // With beta = p64(o, r_j) and R the largest radius, every p64 lies
          // within R of beta + q', so the exact extremes a, b lie within R of
          // beta + min / max q', and c = fma(u, b - a, a) (attempt 0) within
          // R + 2^-52 (|beta| + |min| + |max| + 2R) of beta + mid, mid =
          // min + u (max - min) (computed here within 2^-52 (|min| + |max|)).
          // So with e = 2R + 2^-48 mag, q' < mid - e puts p64 < c, q' >=
          // mid + e puts p64 >= c, and mid - e > min, mid + e < max make
          // attempt 0 accepted (a < c <= b).  |beta| <= |o| |r| <= 1.01 on.
          const double mn = (double)smn[j], mx = (double)smx[j], R = (double)radmax;
          const double mid = __fma_rn(S.u0, __dsub_rn(mx, mn), mn);
          const double mag = __dadd_ru(__dadd_ru(__dmul_ru(1.01, (double)on), fabs(mn)),
                                       __dadd_ru(fabs(mx), R));
          const double e = __fma_ru(0x1p-48, mag, 2.0 * R);
          const double lo = __dsub_rd(mid, e), hi = __dadd_ru(mid, e);
          const bool ok = lo > mn && hi < mx;
          sdtl[j] = ok ? __double2float_rd(lo) : NAN;
          sdtr[j] = __double2float_ru(hi);
        }
      }
      if (ntry <= 32) __syncwarp();
      else __syncthreads();
    }
    if (tid == 0) {
      const int w = exact_only ? -1 : rpf_certify_select(ntry, svh, slo, shi);
      S.exact = w < 0;
      S.cmask = exact_only ? (ntry >= 64 ? ~0ull : (1ull << ntry) - 1ull)
                           : (w < 0 ? rpf_contenders(ntry, slo, shi) : 0ull);
      S.js = w;
      S.rad = radmax;
      S.defer = 0;
      S.nmin = 0;
      S.nmax = 0;
      if (w >= 0) {
        const float r2 = __fmul_ru(2.0f, radmax);
        S.wlo = __fadd_ru(smn[w], r2);
        S.whi = __fsub_rd(smx[w], r2);
        S.akey = rpf_dkey(INFINITY);
        S.bkey = rpf_dkey(-INFINITY);
        if (!median && dfr_cap > 0 && !(sdtl[w] != sdtl[w])) {  // interval of the winner
          S.defer = 1;
          S.dtl = sdtl[w];
          S.dtr = sdtr[w];
        }
      }
    }
    __syncthreads();

    // 4d. deferred split point (uniform rule, certified choice): the sides
    // follow from the interval of c alone when no point lies inside it; the
    // exact extremes -- and c -- are then computed after growth from the
    // few candidates recorded here (k_split_deferred), off this CTA's
    // critical path.  Otherwise the node takes the exact path below.
    if (S.defer) {
      const int w = S.js;
      const float tl = S.dtl, tr = S.dtr, lo = S.wlo, hi = S.whi;
      const float* p = p32 + (int64_t)w * Tn + pbase + nb;
      int und = 0;
      for (int i = tid; i < m; i += NT) {
        const float v = p[i];
        sSide[i] = (uint8_t)(v < tl ? 1 : 0);
        und |= (v >= tl && v < tr) ? 1 : 0;
        if (v <= lo) {
          const int k = atomicAdd(&S.nmin, 1);
          if (k < kDefCand) S.cmin[k] = sP[nb + i];
        }
        if (v >= hi) {
          const int k = atomicAdd(&S.nmax, 1);
          if (k < kDefCand) S.cmax[k] = sP[nb + i];
        }
      }
      if (__syncthreads_or(und)) {
        if (tid == 0) S.defer = 0;
      } else if (tid == 0) {
        int ok = S.nmin <= kDefCand && S.nmax <= kDefCand;
        int slot = -1;
        if (ok) {
          slot = atomicAdd(dfr_cnt, 1);
          ok = slot < dfr_cap;
        }
        if (ok) {
          int32_t* r = dfr + (int64_t)slot * RPF_DEFER_REC;
          r[0] = id;
          r[1] = S.nmin | (S.nmax << 8);
          for (int k = 0; k < kDefCand; ++k) {
            r[2 + k] = k < S.nmin ? S.cmin[k] : -1;
            r[2 + kDefCand + k] = k < S.nmax ? S.cmax[k] : -1;
          }
          node_jstar[id] = w;
          node_flag[id] = 0;
          node_c[id] = NAN;  // k_split_deferred writes c
        }
        S.defer = ok;
        S.flag = 0;
      }
      __syncthreads();
    }

    if (!S.defer) {
    if (S.exact) {
      // canonical FP64 projections and statistics
      const unsigned long long mask = S.cmask;
      for (int i = tid; i < m; i += NT) {
        const float* x = X + (int64_t)sP[nb + i] * d;
        for (int j = 0; j < ntry; ++j)
          if ((mask >> j) & 1ull) p64[(int64_t)j * Tn + pbase + nb + i] = rpf_p64(x, r64 + j * d, d);
      }
      __syncthreads();
      if (warp == 0) {
        double best = 0.0;
        int js = -1;
        for (int j = 0; j < ntry; ++j) {
          if (!((mask >> j) & 1ull)) continue;  // certainly below a contender
          const double* p = p64 + (int64_t)j * Tn + pbase + nb;
          const double Ssum = rpf_warp_chunk_sum(m, lane, [&](int64_t k) { return p[k]; });
          const double mu = __ddiv_rn(Ssum, (double)m);
          const double V = rpf_warp_chunk_sum(m, lane, [&](int64_t k) {
            const double e = __dsub_rn(p[k], mu);
            return __dmul_rn(e, e);
          });
          if (V > best) {
            best = V;
            js = j;
          }
        }
        double a = INFINITY, b = -INFINITY;
        if (js >= 0) {
          const double* p = p64 + (int64_t)js * Tn + pbase + nb;
          for (int k = lane; k < m; k += 32) {
            a = fmin(a, p[k]);
            b = fmax(b, p[k]);
          }
          for (int off = 16; off >= 1; off >>= 1) {
            a = fmin(a, __shfl_xor_sync(RPF_FULL, a, off));
            b = fmax(b, __shfl_xor_sync(RPF_FULL, b, off));
          }
        }
        if (lane == 0) {
          S.js = js;
          S.a = a;
          S.b = b;
          atomicAdd(d_exact, 1ULL);
        }
      }
      __syncthreads();
    } else if (!median) {
      // exact min / max among the candidates the bound leaves: compact the
      // candidates, then one warp evaluates their canonical FP64 projections
      // (FP64 warp instructions are expensive whatever the active lanes)
      const int w = S.js;
      const float lo = S.wlo, hi = S.whi;
      const float* p = p32 + (int64_t)w * Tn + pbase + nb;
      if (tid == 0) S.ncand = 0;
      __syncthreads();
      for (int i = tid; i < m; i += NT) {
        const float v = p[i];
        const int code = (v <= lo ? 1 : 0) | (v >= hi ? 2 : 0);
        if (code) {
          const int slot = atomicAdd(&S.ncand, 1);
          sT[slot] = (i << 2) | code;
        }
      }
      __syncthreads();
      const int nc = S.ncand;
      if (warp == 0) {
        unsigned long long ak = rpf_dkey(INFINITY), bk = rpf_dkey(-INFINITY);
        for (int q0 = 0; q0 < nc; q0 += 2) {  // two candidates per pass (lanes 0, 1)
          const int e0 = sT[q0], e1 = q0 + 1 < nc ? sT[q0 + 1] : e0;
          const double v = rpf_p64_pair(X + (int64_t)sP[nb + (e0 >> 2)] * d,
                                        X + (int64_t)sP[nb + (e1 >> 2)] * d, r64 + w * d, d, lane);
          if (lane < 2) {
            const int e = lane == 0 ? e0 : e1;
            if (e & 1) ak = min(ak, rpf_dkey(v));
            if (e & 2) bk = max(bk, rpf_dkey(v));
          }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
          ak = min(ak, __shfl_xor_sync(RPF_FULL, ak, off));
          bk = max(bk, __shfl_xor_sync(RPF_FULL, bk, off));
        }
        if (lane == 0) {
          S.a = rpf_dkey_inv(ak);
          S.b = rpf_dkey_inv(bk);
        }
      }
      if (warp == (NT > 32 ? 1 : 0)) {
        // b_w = r_w . o in FP64 (any order: the radius covers it)
        double acc = 0.0;
        for (int k = lane; k < d; k += 32) acc = __fma_rn((double)so[k], r64[w * d + k], acc);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(RPF_FULL, acc, off));
        if (lane == 0) sbase[w] = acc;
      }
      __syncthreads();
    }

    // 5m. median rule (Sec. 2's other usual split point): the floor(m/2)
    // points smallest in (p64 of the winner, point index) order go left.
    // Radix selection in shared memory, warp 0 picking each digit:
    //   certified nodes: 4 passes find v32, the rank-floor(m/2) FP32
    //   projection; with R the certified radius, points with q' < v32 - 2R
    //   are certainly left and q' > v32 + 2R certainly right, so only the
    //   band between gets its p64 computed;
    //   then, at rank floor(m/2) minus the certainly-left count, a band of
    //   at most 256 points is searched directly (the point with exactly
    //   that many smaller (key, index) pairs in the band); a larger band,
    //   and every point of an exact node, takes 8 radix passes over the
    //   order-preserving key of p64 and 4 over the point index.
    if (median && S.js >= 0) {
      const int js = S.js;
      double* pj = p64 + (int64_t)js * Tn + pbase + nb;
      const float* qj = p32 + (int64_t)js * Tn + pbase + nb;
      const bool exact = S.exact;
      if (tid == 0) {
        S.mkey = 0ull;
        S.mid = 0u;
        S.mfk = 0u;
        S.mrank = m >> 1;
        S.mlo = -INFINITY;
        S.mhi = INFINITY;
        S.ncand = 0;
      }
      __syncthreads();
      for (int pass = exact ? 4 : 0; pass < 16; ++pass) {
        if (pass == 4 && !exact) {  // the band; p64 inside it; certainly-left count
          float lo, hi;
          rpf_med_band(S.mfk, S.rad, &lo, &hi);
          int cnt = 0;
          for (int i = tid; i < m; i += NT) {
            const float v = qj[i];
            if (v < lo) {
              ++cnt;
            } else if (v <= hi) {
              const double p = rpf_p64(X + (int64_t)sP[nb + i] * d, r64 + js * d, d);
              pj[i] = p;
              const int e = atomicAdd(&S.ncand, 1);
              if (e < kBandSel) {
                bnd_key[e] = rpf_mkey(p);
                bnd_id[e] = (uint32_t)sP[nb + i];
              }
            }
          }
          for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(RPF_FULL, cnt, off);
          if (lane == 0) wsc[warp] = cnt;
          __syncthreads();
          if (tid == 0) {
            int t = 0;
            for (int u = 0; u < NT / 32; ++u) t += wsc[u];
            S.mrank = (m >> 1) - t;
            S.mlo = lo;
            S.mhi = hi;
          }
          __syncthreads();
          const int nc = S.ncand;
          if (nc <= kBandSel) {
            // a small band: the element with exactly mrank smaller (key,
            // index) pairs in it, by counting (the pairs are distinct)
            const int r = S.mrank;
            for (int e = tid; e < nc; e += NT) {
              const unsigned long long k = bnd_key[e];
              const uint32_t id = bnd_id[e];
              int below = 0;
              for (int f = 0; f < nc; ++f)
                below += bnd_key[f] < k || (bnd_key[f] == k && bnd_id[f] < id);
              if (below == r) {
                S.mkey = k;
                S.mid = id;
              }
            }
            __syncthreads();
            break;
          }
        }
        for (int b = tid; b < 256; b += NT) mhist[b] = 0;
        __syncthreads();
        const uint32_t pf = S.mfk;
        const unsigned long long pk = S.mkey;
        const uint32_t pid = S.mid;
        const float lo = S.mlo, hi = S.mhi;
        for (int i = tid; i < m; i += NT) {
          int dig;
          bool match;
          if (pass < 4) {
            const int sh = 24 - 8 * pass;
            const uint32_t k = rpf_fkey(qj[i]);
            dig = (int)((k >> sh) & 255u);
            match = pass == 0 || ((k ^ pf) >> (sh + 8)) == 0u;
          } else {
            if (!exact && !(qj[i] >= lo && qj[i] <= hi)) continue;
            match = rpf_med_digit(pass - 4, rpf_mkey(pj[i]), (uint32_t)sP[nb + i], pk, pid, &dig);
          }
          if (match) atomicAdd(&mhist[dig], 1);
        }
        __syncthreads();
        if (warp == 0) {
          int dig, rest;
          if (rpf_pick_digit(mhist, lane, S.mrank, &dig, &rest)) {
            S.mrank = rest;
            if (pass < 4) S.mfk = pf | ((uint32_t)dig << (24 - 8 * pass));
            else if (pass < 12) S.mkey = pk | ((unsigned long long)dig << (56 - 8 * (pass - 4)));
            else S.mid = pid | ((uint32_t)dig << (24 - 8 * (pass - 12)));
          }
        }
        __syncthreads();
      }
    }

    // 5. split point and node record
    if (tid == 0) {
      const int js = S.js;
      double c = NAN;
      int acc = 0;
      if (js >= 0 && median) {  // c = the p64 of the first point that goes right
        c = rpf_dkey_inv(S.mkey);
        acc = 1;
      } else if (js >= 0) {
        acc = rpf_split_point(seed, (uint64_t)(t + t_base), key, S.a, S.b, &c);
      }
      S.c = c;
      S.flag = acc ? 0 : 1;
      if (acc && !median && !S.exact) {
        float tl, tr;
        rpf_side_thresholds(c, sbase[js], (double)S.rad, &tl, &tr);
        S.tl = tl;
        S.tr = tr;
      }
      node_jstar[id] = js;
      node_flag[id] = (acc ? 0 : 1) | (S.exact ? 2 : 0);
      node_c[id] = c;
    }
    __syncthreads();

    // 6. sides and the stable partition
    {
      const int js = S.js, flag = S.flag, exact = S.exact;
      const double c = S.c;
      const float tl = S.tl, tr = S.tr;
      if (tid == 0) S.ncand = 0;
      __syncthreads();
      for (int i = tid; i < m; i += NT) {
        int left;
        if (flag) {
          left = i < (m >> 1);
        } else if (median) {  // certainly below / above the band, else (key, index)
          const float q = p32[(int64_t)js * Tn + pbase + nb + i];
          if (q < S.mlo) {
            left = 1;
          } else if (q > S.mhi) {
            left = 0;
          } else {
            const unsigned long long k = rpf_mkey(p64[(int64_t)js * Tn + pbase + nb + i]);
            left = k < S.mkey || (k == S.mkey && (uint32_t)sP[nb + i] < S.mid);
          }
        } else if (exact) {
          left = p64[(int64_t)js * Tn + pbase + nb + i] < c;
        } else {
          const float v = p32[(int64_t)js * Tn + pbase + nb + i];
          if (v < tl) {
            left = 1;
          } else if (v >= tr) {
            left = 0;
          } else {  // undecided by the bound: FP64 below
            left = 2;
            sT[atomicAdd(&S.ncand, 1)] = i;
          }
        }
        sSide[i] = (uint8_t)left;
      }
      __syncthreads();
      if (warp == 0) {
        const int na = S.ncand;
        for (int q0 = 0; q0 < na; q0 += 2) {  // two undecided points per pass (lanes 0, 1)
          const int i0 = sT[q0], i1 = q0 + 1 < na ? sT[q0 + 1] : i0;
          const double v = rpf_p64_pair(X + (int64_t)sP[nb + i0] * d, X + (int64_t)sP[nb + i1] * d,
                                        r64 + js * d, d, lane);
          if (lane < 2 && q0 + lane < na) sSide[lane == 0 ? i0 : i1] = v < c ? 1 : 0;
        }
      }
      __syncthreads();
    }
    }  // !S.defer
    {
      // stable partition from one block-wide scan: thread t takes the run
      // [t per, (t + 1) per) of positions (per odd, so the runs' shared-
      // memory reads fall in distinct banks); E = lefts before a position
      const int per = ((m + NT - 1) / NT) | 1;
      const int v0 = min(m, tid * per), v1 = min(m, v0 + per);
      int cnt = 0;
      for (int i = v0; i < v1; ++i) cnt += sSide[i];
      int x = cnt;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(RPF_FULL, x, off);
        if (lane >= off) x += y;
      }
      if (lane == 31) wsc[warp] = x;
      __syncthreads();
      int E = x - cnt, nl = 0;
#pragma unroll
      for (int u = 0; u < NT / 32; ++u) {
        const int w = wsc[u];
        if (u < warp) E += w;
        nl += w;
      }
      for (int i = v0; i < v1; ++i) {
        const int sd = sSide[i];
        sT[nb + (sd ? E : nl + (i - E))] = sP[nb + i];
        E += sd;
      }
      if (tid == 0) S.nl = nl;
      __syncthreads();
      for (int i = tid; i < m; i += NT) sP[nb + i] = sT[nb + i];
      __syncthreads();
    }

    // 7. children
    if (tid == 0) {
      const int nl = S.nl;
      const int mL = nl, mR = m - nl;
      const int idL = S.next_id, idR = S.next_id + 1;
      if (idR >= S.id_end) S.err = 1;  // reserved range [nbase, nbase + 2 m0 - 2)
      if (!S.err) {
        S.next_id += 2;
        node_left[id] = idL;
        node_right[id] = idR;
        const int bL = in.begin[it] + nb, bR = bL + nl;
        node_key[idL] = rpf_child_key(key, 0);
        node_key[idR] = rpf_child_key(key, 1);
        node_tree[idL] = node_tree[idR] = t;
        node_begin[idL] = bL;
        node_begin[idR] = bR;
        node_len[idL] = mL;
        node_len[idR] = mR;
        node_left[idL] = node_right[idL] = node_left[idR] = node_right[idR] = -1;
        node_jstar[idL] = node_jstar[idR] = -1;
        node_flag[idL] = node_flag[idR] = 0;
        node_c[idL] = node_c[idR] = NAN;
        S.leafL = mL <= L;
        S.leafR = mR <= L;
        if (S.leafL) {
          const int ls = S.next_leaf++;
          leaf_tree[ls] = t;
          leaf_begin[ls] = bL;
          leaf_len[ls] = mL;
        }
        if (S.leafR) {
          const int ls = S.next_leaf++;
          leaf_tree[ls] = t;
          leaf_begin[ls] = bR;
          leaf_len[ls] = mR;
        }
        if (S.next_leaf > S.leaf_end || S.top + 2 > kStack) {
          S.err = 1;
        } else {
          // push the larger inner child first: the smaller one is popped next
          const bool Lfirst = mL >= mR;
          for (int pass = 0; pass < 2; ++pass) {
            const bool isL = (pass == 0) == Lfirst;
            if (isL && !S.leafL) {
              st_nb[S.top] = nb;
              st_m[S.top] = mL;
              st_id[S.top] = idL;
              st_key[S.top] = rpf_child_key(key, 0);
              ++S.top;
            } else if (!isL && !S.leafR) {
              st_nb[S.top] = nb + nl;
              st_m[S.top] = mR;
              st_id[S.top] = idR;
              st_key[S.top] = rpf_child_key(key, 1);
              ++S.top;
            }
          }
        }
      }
    }
    __syncthreads();
    if (S.err) break;
    if (S.leafL)
      for (int i = tid; i < S.nl; i += NT) perm_final[pbase + nb + i] = sP[nb + i];
    if (S.leafR)
      for (int i = tid; i < m - S.nl; i += NT) perm_final[pbase + nb + S.nl + i] = sP[nb + S.nl + i];
    __syncthreads();
  }
  if (tid == 0 && S.err) atomicExch(d_err, 1);
  __syncthreads();  // before the next item takes the shared state
  }
}

// The deferred split points, after growth (node tables compacted, chosen
// directions regenerated): one thread per record evaluates the canonical
// FP64 projections of its candidates in turn (an FP64 warp instruction costs
// the same whatever its active lanes, so all 32 lanes carry a record), takes
// the exact minimum a and maximum b, and forms c = fma(u, b - a, a) of
// attempt 0, which the certified interval already showed to be accepted
// (checked again here: a failure is an internal error).
__global__ void __launch_bounds__(128) k_split_deferred(
    const int32_t* dfr, const int* dfr_cnt, int dfr_cap, const int32_t* new_id,
    const uint64_t* node_key, const int32_t* node_tree, const float* node_dir32,
    const float* __restrict__ X, int d, uint64_t seed, int t_base, double* node_c, int* d_err) {
  const int64_t rec = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (rec >= min(*dfr_cnt, dfr_cap)) return;
  const int32_t* r = dfr + rec * RPF_DEFER_REC;
  const int nid = new_id[r[0]];
  const int nmin = r[1] & 255, nmax = (r[1] >> 8) & 255;
  const float* dir = node_dir32 + (int64_t)nid * d;
  unsigned long long ak = rpf_dkey(INFINITY), bk = rpf_dkey(-INFINITY);
  for (int c = 0; c < nmin + nmax; ++c) {
    const int pt = c < nmin ? r[2 + c] : r[2 + kDefCand + (c - nmin)];
    const unsigned long long k = rpf_dkey(rpf_p64f(X + (int64_t)pt * d, dir, d));
    if (c < nmin) ak = min(ak, k);
    else bk = max(bk, k);
  }
  const double a = rpf_dkey_inv(ak), b = rpf_dkey_inv(bk);
  const uint64_t t = (uint64_t)(node_tree[nid] + t_base);
  const double u = rpf_u53(rpf_word(seed, RPF_TAG_SPLIT, t, node_key[nid], 0, 0));
  const double c = __fma_rn(u, __dsub_rn(b, a), a);
  if (!(c > a && c <= b) || nmin < 1 || nmax < 1) atomicExch(d_err, 1);
  node_c[nid] = c;
}

}  // namespace

int rpf_split_deferred(rpf_forest* fo, const int32_t* dfr, const int* dfr_cnt, int dfr_cap,
                       const int32_t* new_id, int* d_err, cudaStream_t s) {
  if (dfr_cap <= 0) return RPF_OK;
  RPF_LAUNCH("k_split_deferred", s,
             k_split_deferred<<<(unsigned)(((int64_t)dfr_cap + 127) / 128), 128, 0, s>>>(
                 dfr, dfr_cnt, dfr_cap, new_id, fo->node_key, fo->node_tree, fo->node_dir32, fo->X,
                 fo->d, fo->prm.seed, fo->t_base, fo->node_c, d_err));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RPF_OK : rpf_cuda_err(e);
}

bool rpf_subtree_fits(int d, int ntry) {
  return sub_layout(d, ntry, 8, kB, kSubN).total <= 200 * 1024;
}

namespace {

// Largest subtree (points) given to the one-warp kernel: above the leaf
// bound (so that it is an inner node), at most 1024 points (32 positions per
// lane in the statistics), and at least 1024 under the median rule (its
// band list lives in sT); 0: none.
int small_subtree_max(int L, int median) {
  const int m = median ? 1024 : ((std::max(512, 2 * L) + 15) & ~15);
  return m > 1024 || m <= L ? 0 : m;
}

__global__ void k_seed_small(int n_small, const int32_t* idx, SubItems in, SubItems out, int* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *cnt = n_small;
  if (i >= n_small) return;
  const int j = idx[i];
  out.node[i] = in.node[j];
  out.tree[i] = in.tree[j];
  out.begin[i] = in.begin[j];
  out.len[i] = in.len[j];
  out.key[i] = in.key[j];
  out.nbase[i] = in.nbase[j];
  out.lbase[i] = in.lbase[j];
}

}  // namespace

// Phase B: items of more than S points (S = small_subtree_max) are grown by
// the four-warp kernel, which hands every node of at most S points to the
// one-warp kernel (items of at most S points go there directly).  Both
// reserve node ids and leaf slots by subtree size, so the forest does not
// depend on the order in which the small subtrees are taken.
int rpf_grow_subtrees(rpf_forest* fo, int64_t n_items, const int32_t* ilen, const int32_t* it_node,
                      const int32_t* it_tree, const int32_t* it_begin, const int32_t* it_len,
                      const uint64_t* it_key, const int32_t* it_nbase, const int32_t* it_lbase,
                      float* p32, double* p64, unsigned long long* d_exact, int* d_err,
                      int32_t* dfr, int* dfr_cnt, int dfr_cap, cudaStream_t s) {
  const int d = fo->d, ntry = fo->prm.n_try, L = fo->prm.leaf_max;
  const int64_t n = fo->n, Tn = n * fo->prm.n_trees;
  const int exact_only = fo->prm.growth == 1 ? 1 : 0;
  const int median = fo->prm.split_rule == 1 ? 1 : 0;
  const int TG = ntry <= 5 ? ntry : 8;
  const size_t smem = sub_layout(d, ntry, TG, kB, kSubN).total;
  if (smem > 200 * 1024) return RPF_EINVAL;
  int S = small_subtree_max(L, median);
  const size_t smem_s = S ? sub_layout(d, ntry, TG, kSmallB, S).total : 0;
  if (smem_s > 48 * 1024) S = 0;

  std::vector<int32_t> big, small;
  int64_t big_pts = 0;
  for (int64_t i = 0; i < n_items; ++i) {
    if (ilen[i] > S) {
      big.push_back((int32_t)i);
      big_pts += ilen[i];
    } else {
      small.push_back((int32_t)i);
    }
  }
  // deferred nodes are disjoint segments of more than L points
  const int64_t cap = S ? (int64_t)small.size() + big_pts / (L + 1) + 1 : 0;
  if (cap >= ((int64_t)1 << 31)) return RPF_EINVAL;
  SubItems in{const_cast<int32_t*>(it_node), const_cast<int32_t*>(it_tree),
              const_cast<int32_t*>(it_begin), const_cast<int32_t*>(it_len),
              const_cast<uint64_t*>(it_key),  const_cast<int32_t*>(it_nbase),
              const_cast<int32_t*>(it_lbase)};
  SubItems sm{};
  int32_t *d_big = nullptr, *d_small = nullptr;
  int* sm_cnt = nullptr;
  void* bufs[10] = {};
  auto release_all = [&]() {
    for (void* p : bufs) rpf_release(p, s);
  };
#define SUB_CU(call)                  \
  do {                                \
    cudaError_t e_ = (call);          \
    if (e_ != cudaSuccess) {          \
      release_all();                  \
      return rpf_cuda_err(e_);        \
    }                                 \
  } while (0)
  int rc = RPF_OK;
  if (!big.empty()) rc = rpf_alloc((void**)&d_big, 4 * big.size(), s);
  bufs[0] = d_big;
  if (!rc && S) {
    rc = rpf_alloc((void**)&d_small, 4 * std::max<size_t>(small.size(), 1), s);
    bufs[1] = d_small;
    int32_t** f32[6] = {&sm.node, &sm.tree, &sm.begin, &sm.len, &sm.nbase, &sm.lbase};
    for (int k = 0; k < 6 && !rc; ++k) {
      rc = rpf_alloc((void**)f32[k], 4 * (size_t)cap, s);
      bufs[2 + k] = *f32[k];
    }
    if (!rc) rc = rpf_alloc((void**)&sm.key, 8 * (size_t)cap, s);
    bufs[8] = sm.key;
    if (!rc) rc = rpf_alloc((void**)&sm_cnt, sizeof(int), s);
    bufs[9] = sm_cnt;
  }
  if (rc) {
    release_all();
    return rc;
  }
  if (!big.empty())
    SUB_CU(cudaMemcpyAsync(d_big, big.data(), 4 * big.size(), cudaMemcpyHostToDevice, s));
  if (S) {
    if (!small.empty())
      SUB_CU(cudaMemcpyAsync(d_small, small.data(), 4 * small.size(), cudaMemcpyHostToDevice, s));
    const int ns = (int)small.size();
    RPF_LAUNCH("k_seed_small", s, k_seed_small<<<(unsigned)(ns / 256 + 1), 256, 0, s>>>(
        ns, d_small, in, sm, sm_cnt));
  }
  // (copies from pageable memory have read their source when they return)
  int dev = 0, n_sm = 1, occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
#define RPF_SUB(TGV)                                                                               \
  do {                                                                                             \
    SUB_CU(cudaFuncSetAttribute(k_subtree<TGV, kB>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                (int)smem));                                                       \
    if (!big.empty())                                                                              \
      RPF_LAUNCH("k_subtree", s, k_subtree<TGV, kB><<<(unsigned)big.size(), kB, smem, s>>>(        \
          in, d_big, (int)big.size(), nullptr, kSubN, S, sm, sm_cnt, (int)cap, fo->X, fo->xnorm, n, \
          Tn, d, ntry, L, fo->prm.seed, fo->t_base, exact_only, median, fo->perm, p32, p64,       \
          fo->node_key, fo->node_tree, fo->node_begin, fo->node_len, fo->node_left,                \
          fo->node_right, fo->node_jstar, fo->node_flag, fo->node_c, fo->leaf_tree,               \
          fo->leaf_begin, fo->leaf_len, d_exact, d_err, dfr, dfr_cnt, dfr_cap));                  \
    if (S) {                                                                                       \
      SUB_CU(cudaFuncSetAttribute(k_subtree<TGV, kSmallB>,                                         \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s));      \
      SUB_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_subtree<TGV, kSmallB>,          \
                                                           kSmallB, smem_s));                      \
      const int64_t grid = std::min<int64_t>((int64_t)std::max(occ, 1) * n_sm, cap);             \
      RPF_LAUNCH("k_subtree_w", s, k_subtree<TGV, kSmallB><<<(unsigned)grid, kSmallB, smem_s, s>>>( \
          sm, nullptr, 0, sm_cnt, S, 0, sm, sm_cnt, 0, fo->X, fo->xnorm, n, Tn, d, ntry, L,       \
          fo->prm.seed, fo->t_base, exact_only, median, fo->perm, p32, p64, fo->node_key,         \
          fo->node_tree, fo->node_begin, fo->node_len, fo->node_left, fo->node_right,             \
          fo->node_jstar, fo->node_flag, fo->node_c, fo->leaf_tree, fo->leaf_begin, fo->leaf_len, \
          d_exact, d_err, dfr, dfr_cnt, dfr_cap));                                                 \
    }                                                                                              \
  } while (0)
  switch (TG) {
    case 1: RPF_SUB(1); break;
    case 2: RPF_SUB(2); break;
    case 3: RPF_SUB(3); break;
    case 4: RPF_SUB(4); break;
    case 5: RPF_SUB(5); break;
    default: RPF_SUB(8); break;
  }
#undef RPF_SUB
#undef SUB_CU
  release_all();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RPF_OK : rpf_cuda_err(e);
}
