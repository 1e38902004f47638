// rpf_knn.cu -- distances inside every (tree, leaf) block and the cross-tree
// merge of Algorithm 3 (Sec. 2): N_q is the union of q's leaves over the T
// trees and its K closest points are the answer.  A point y in the K closest
// of N_q has at most K-1 points of N_q before it, hence at most K-1 points of
// any leaf containing it, so y is in that leaf's own top-K: merging per-leaf
// top-K lists (deduplicated by index) gives exactly the top-K of the union.
//
//   k_leaf_plain   one CTA per tile of packed small leaves; every row scans its
//                  leaf with the canonical FP32 d32 and keeps a sorted top-K
//   k_merge        per point, merge the per-tree lists of a group of trees
//                  into the running top-K (duplicates have identical keys
//                  because d32 is symmetric and deterministic)
//   k_route_w      drop each query through each tree (FP64 r* . q < c,
//                  certified from FP32 and recomputed in FP64 when undecided)
//   k_qscan_cta    per (query, tree): top-K of the leaf the query fell into
//                  (leaf rows TMA-staged, bitonic sort of 64-bit keys);
//                  k_qscan is the one-thread-per-pair form for leaves > 128
// The chosen form of the all-kNN leaf tiles is in rpf_leaf_tc.cu.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "rpf_allknn.cuh"
#include "rpf_internal.cuh"
#include "rpf_tma.cuh"
#include "rpf_scan.cuh"
#include "rpf_select.cuh"

namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// acc + the squares of a - v over four coordinates, added one at a time in
// coordinate order (the canonical d32 chain); the differences are taken in
// packed pairs, each lane rounding like __fsub_rn
__device__ __forceinline__ float sq_chain4(const float4 a, const float4 v, float acc) {
  const float2 e01 = rpf_sub2(make_float2(a.x, a.y), make_float2(v.x, v.y));
  const float2 e23 = rpf_sub2(make_float2(a.z, a.w), make_float2(v.z, v.w));
  acc = __fmaf_rn(e01.x, e01.x, acc);
  acc = __fmaf_rn(e01.y, e01.y, acc);
  acc = __fmaf_rn(e23.x, e23.x, acc);
  return __fmaf_rn(e23.y, e23.y, acc);
}

// Register-resident sorted list of the KMAX smallest (d, idx) offered so far
// (ascending; empty slots are (+inf, -1)).  Every caller needs the K <= KMAX
// smallest, which the first K entries are.  The length is a compile-time
// constant so the list stays in registers (a run-time length makes the
// compiler place it in local memory); insertion is a branch-free network.
template <int KMAX>
struct TopK {
  float kd[KMAX];
  int ki[KMAX];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
      kd[q] = INFINITY;
      ki[q] = -1;
    }
  }
  __device__ __forceinline__ bool better_than_last(float v, int j) const {
    return rpf_less(v, j, kd[KMAX - 1], ki[KMAX - 1]);
  }
  // insert (v, j); the caller checked better_than_last
  __device__ __forceinline__ void insert(float v, int j) {
#pragma unroll
    for (int q = KMAX - 1; q >= 1; --q) {
      const bool sh = rpf_less(v, j, kd[q - 1], ki[q - 1]);
      const bool pl = !sh && rpf_less(v, j, kd[q], ki[q]);
      kd[q] = sh ? kd[q - 1] : (pl ? v : kd[q]);
      ki[q] = sh ? ki[q - 1] : (pl ? j : ki[q]);
    }
    const bool p0 = rpf_less(v, j, kd[0], ki[0]);
    kd[0] = p0 ? v : kd[0];
    ki[0] = p0 ? j : ki[0];
  }
  __device__ __forceinline__ void offer(float v, int j) {
    if (better_than_last(v, j)) insert(v, j);
  }
  __device__ __forceinline__ bool contains(int j) const {
    bool f = false;
#pragma unroll
    for (int q = 0; q < KMAX; ++q) f |= ki[q] == j;
    return f;
  }
  // first K entries to out[0..K)
  __device__ __forceinline__ void store(int K, uint2* out) const {
#pragma unroll
    for (int q = 0; q < KMAX; ++q)
      if (q < K) out[q] = make_uint2(__float_as_uint(kd[q]), (unsigned)ki[q]);
  }
};

// ---------------------------------------------------------------------------
// Plain leaf tiles.  A tile is a run of consecutive leaves of one tree (the
// leaf list is sorted by begin), so its rows are the permutation positions
// b0 .. b0 + rows - 1.  Rows are staged in shared memory by bulk copies
// (TMA engine), padded to dp floats with zeros beyond d.  Work item = one
// leaf and a block of 32 of its rows, taken by one warp: lane l owns row
// lb + 32 w + l (its coordinates in registers when d <= 64) and scans every
// column of the leaf, whose coordinates are broadcast from shared memory.
// Each distance is the canonical fmaf chain over k in order, so d32 is
// bit-identical to the oracle's.
// cand layout: [(g * n + point) * K + k] as (d32 bits, idx).
// ---------------------------------------------------------------------------
template <int KMAX, bool REG, bool STAGE>
__global__ void __launch_bounds__(128, 4) k_leaf_plain(const int32_t* tile_cnt,
                                                    const int32_t* tile_off,
                                                    const int32_t* tile_leaf, int64_t tile_base,
                                                    const int32_t* leaf_tree,
                                                    const int32_t* leaf_begin,
                                                    const int32_t* leaf_len, const int32_t* perm,
                                                    const float* __restrict__ X, int64_t n, int d,
                                                    int dp, int K, int t0, uint2* cand, int* err,
                                                    uint64_t wlim) {
  extern __shared__ __align__(16) float xs[];
  __shared__ int leaf_off[257];  // a tile starts at most 256 leaves
  __shared__ int item_off[257];
  __shared__ int lbeg[256];
  __shared__ int b0s;
  __shared__ __align__(8) uint64_t bar;
  const int64_t tile = tile_base + blockIdx.x;
  const int nl = tile_cnt[tile];
  if (nl == 0) return;
  const int32_t* tl = tile_leaf + tile_off[tile];
  const int t = leaf_tree[tl[0]];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // the tile's leaves (at most 1024), ordered by begin: rank sort
  for (int q = threadIdx.x; q < nl; q += blockDim.x) lbeg[q] = leaf_begin[tl[q]];
  __syncthreads();
  for (int q = threadIdx.x; q < nl; q += blockDim.x) {
    const int b = lbeg[q];
    int rank = 0;
    for (int p = 0; p < nl; ++p) rank += lbeg[p] < b;
    leaf_off[rank] = b;
    if (rank == nl - 1) leaf_off[nl] = b + leaf_len[tl[q]];
    if (rank == 0) b0s = b;
  }
  __syncthreads();
  const int b0 = b0s;
  for (int q = threadIdx.x; q <= nl; q += blockDim.x) leaf_off[q] -= b0;
  __syncthreads();
  const int rows = leaf_off[nl];
  const int32_t* prow = perm + (int64_t)t * n + b0;
  if (warp == 0) {  // item_off[q] = sum over earlier leaves of ceil(len / 32)
    int run = 0;
    for (int q0 = 0; q0 < nl; q0 += 32) {
      const int q = q0 + lane;
      const int v = q < nl ? (leaf_off[q + 1] - leaf_off[q] + 31) >> 5 : 0;
      int x = v;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(RPF_FULL, x, off);
        if (lane >= off) x += y;
      }
      if (q < nl) item_off[q] = run + x - v;
      run += __shfl_sync(RPF_FULL, x, 31);
    }
    if (lane == 0) item_off[nl] = run;
  }
  if (STAGE && (d & 3) == 0) {
    if (threadIdx.x == 0) {
      rpf_mbar_init(&bar, 1);
      rpf_mbar_arrive_expect_tx(&bar, (uint32_t)rows * (uint32_t)d * 4u);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += blockDim.x)
      rpf_bulk_g2s(xs + r * dp, X + (int64_t)prow[r] * d, (uint32_t)d * 4u, &bar);
    for (int r = threadIdx.x; r < rows; r += blockDim.x)
      for (int k = d; k < dp; ++k) xs[r * dp + k] = 0.0f;
    // the whole CTA gives up together: one more bounded wait for copies in
    // flight, then return (the error word reports the call as failed)
    if (!__syncthreads_and(rpf_mbar_wait(&bar, 0, err, wlim))) {
      rpf_mbar_wait(&bar, 0, nullptr, wlim);
      return;
    }
  } else if (STAGE) {
    for (int r = warp; r < rows; r += nwarp) {
      const float* src = X + (int64_t)prow[r] * d;
      for (int k = lane; k < dp; k += 32) xs[r * dp + k] = k < d ? src[k] : 0.0f;
    }
  }
  __syncthreads();
  const int nitems = item_off[nl];
  const int d4 = (d + 3) & ~3;
  for (int it = warp; it < nitems; it += nwarp) {
    int lo = 0, hi = nl - 1;  // leaf of item it: last q with item_off[q] <= it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (item_off[mid] <= it) lo = mid;
      else hi = mid - 1;
    }
    const int lb = leaf_off[lo], le = leaf_off[lo + 1];
    const int r = lb + 32 * (it - item_off[lo]) + lane;
    const bool live = r < le;
    const int rr = live ? r : lb;
    // up to 16 entries (32 when the row is not held in registers): 64-bit
    // keys (d32 bits, index), which order like (d32, index), merged in four
    // at a time; longer lists keep one insertion per column (the batched
    // merge would not fit in registers)
    constexpr bool kBatch = KMAX <= 16 || (!REG && KMAX <= 32);
    std::conditional_t<kBatch, Top64<KMAX>, TopK<KMAX>> tk;
    tk.init();
    float xr[REG ? 64 : 1];
    if (REG) {
#pragma unroll
      for (int k = 0; k < 64; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(xs + rr * dp + k);
        xr[k] = v.x;
        xr[k + 1] = v.y;
        xr[k + 2] = v.z;
        xr[k + 3] = v.w;
      }
    }
    // four columns at a time: four independent canonical chains per lane
    for (int c0 = lb; c0 < le; c0 += 4) {
      int cc[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) cc[j] = min(c0 + j, le - 1);
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (REG) {
#pragma unroll
        for (int k = 0; k < 64; k += 4) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 v = *reinterpret_cast<const float4*>(xs + cc[j] * dp + k);
            acc[j] = sq_chain4(make_float4(xr[k], xr[k + 1], xr[k + 2], xr[k + 3]), v, acc[j]);
          }
        }
      } else if (STAGE) {
        const float* x = xs + rr * dp;
        for (int k = 0; k < d4; k += 4) {
          const float4 a = *reinterpret_cast<const float4*>(x + k);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 v = *reinterpret_cast<const float4*>(xs + cc[j] * dp + k);
            acc[j] = sq_chain4(a, v, acc[j]);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          acc[j] = rpf_d32(X + (int64_t)prow[rr] * d, X + (int64_t)prow[cc[j]] * d, d);
      }
      if constexpr (kBatch) {
        unsigned long long kb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + j;
          kb[j] = c < le && c != r ? key64(acc[j], prow[cc[j]]) : ~0ull;
        }
        tk.insert4(kb);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + j;
          if (c < le && c != r) tk.offer(acc[j], prow[c]);
        }
      }
    }
    if (live) tk.store(K, cand + ((int64_t)(t - t0) * n + prow[r]) * K);
  }
}

// Exact top-K of tile row r over the columns [lb, le) of its leaf: canonical
// d32 chains, four at a time (rows in shared memory, padded to dp floats).
template <int KMAX>
__device__ __forceinline__ void rpf_row_exact(const float* xs, int dp, int d4, int r, int lb,
                                              int le, const int32_t* prow, TopK<KMAX>& tk) {
  const float* x = xs + r * dp;
  for (int c0 = lb; c0 < le; c0 += 4) {
    int cc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cc[j] = min(c0 + j, le - 1);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int k = 0; k < d4; k += 4) {
      const float4 a = *reinterpret_cast<const float4*>(x + k);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 v = *reinterpret_cast<const float4*>(xs + cc[j] * dp + k);
        acc[j] = sq_chain4(a, v, acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + j;
      if (c < le && c != r) tk.offer(acc[j], prow[c]);
    }
  }
}

// Merge G per-tree lists (sorted, padded with (inf, -1)) into the running list
// of each point, read from run_in and written to run_out (each thread reads
// its point's list before writing, so the two may coincide).  first: no
// running list yet; last: write the final outputs instead of run_out.
template <int KMAX>
__global__ void k_merge(int64_t n, int K, int G, const uint2* cand, const uint2* run_in,
                        uint2* run_out, bool first, bool last, int32_t* idx, float* dist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  TopK<KMAX> tk;
  tk.init();
  if (!first) {
#pragma unroll
    for (int q = 0; q < KMAX; ++q)
      if (q < K) {
        const uint2 e = run_in[i * K + q];
        tk.kd[q] = __uint_as_float(e.x);
        tk.ki[q] = (int)e.y;
      }
  }
  for (int g = 0; g < G; ++g) {
    const uint2* c = cand + ((int64_t)g * n + i) * K;
    for (int q = 0; q < K; ++q) {
      const uint2 e = c[q];
      const int j = (int)e.y;
      if (j < 0) break;
      const float v = __uint_as_float(e.x);
      if (!tk.better_than_last(v, j)) break;  // sorted list: nothing later fits
      if (!tk.contains(j)) tk.insert(v, j);    // a duplicate has the same key
    }
  }
  if (last) {
#pragma unroll
    for (int q = 0; q < KMAX; ++q)
      if (q < K) {
        idx[i * K + q] = tk.ki[q];
        dist[i * K + q] = tk.ki[q] < 0 ? INFINITY : __fsqrt_rn(tk.kd[q]);
      }
  } else {
    tk.store(K, run_out + i * K);
  }
}

template <int KMAX>
__global__ void k_qscan(const float* Q, int64_t m, int d, int T, int K, const int2* qleaf,
                        const int32_t* perm, const float* X, int64_t n, uint2* cand) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m * T) return;
  const int64_t q = g / T;
  const int t = (int)(g % T);
  const int2 lf = qleaf[g];  // the leaf's (begin, length) in tree t's permutation
  const int b = lf.x, ln = lf.y;
  const int32_t* mem = perm + (int64_t)t * n + b;
  const float* x = Q + q * d;
  TopK<KMAX> tk;
  tk.init();
  for (int a = 0; a < ln; ++a) {
    const int j = mem[a];
    tk.offer(rpf_d32(x, X + (int64_t)j * d, d), j);
  }
  tk.store(K, cand + ((int64_t)t * m + q) * K);
}

// Routing, one group of RW = 8 lanes per (query q, tree t) (Sec. 2,
// Algorithm 3); a warp walks four (query, tree) paths at once, so four
// chains of dependent node loads are in flight.  A step reads the node's
// 16-byte routing record (c, left, right) and its FP32 direction, both
// addressed by the node id alone, so one round trip per level.  At a split
// node the decision is r* . q < c with the canonical FP64 chain p64 (fold of
// fma((double)q_k, r_k, p) over k in order).  The directions are FP32
// values, so the group first forms s = r* . q in FP32 (lane-strided fmaf
// over at most ceil(d / 8) terms, then a 3-level butterfly) with
// A = sum |q_k r_k|; p64 lies within
//   e = (ceil(d / 8) + 7) 2^-24 A_up
// of s (FP32 error of s: (ceil(d/8) + 3) u A; FP64 error of p64: d 2^-53 A;
// A_up bounds A despite its own rounding).  Only when c falls inside
// [s - e, s + e] does the group's first lane evaluate p64 itself.  A rank
// split stores its left child on both sides (every query goes left).
#define RW 8
__global__ void __launch_bounds__(256) k_route_w(const float* __restrict__ Q, int64_t m, int d,
                                                 int T, const int4* __restrict__ node_route,
                                                 const float* __restrict__ node_dir32,
                                                 int2* qleaf) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / RW;
  const int lane = threadIdx.x & 31, sub = lane & (RW - 1);
  const unsigned gmask = ((1u << RW) - 1u) << (lane & ~(RW - 1));
  if (g >= m * T) return;  // whole group
  const int64_t q = g / T;
  const int t = (int)(g % T);
  const float* x = Q + q * d;
  const int per = (d + RW - 1) / RW;
  const float kerr = (float)(per + 7) * 0x1p-24f;
  const float kA = 1.0f + (float)(per + 6) * 0x1p-23f;
  int node = t;
  int4 rec = __ldg(node_route + node);
  while (rec.z >= 0) {
    const double c = __hiloint2double(rec.y, rec.x);
    const float* r32 = node_dir32 + (int64_t)node * d;
    float sacc = 0.0f, aacc = 0.0f;
    for (int k = sub; k < d; k += RW) {
      const float xv = __ldg(x + k), rv = __ldg(r32 + k);
      sacc = __fmaf_rn(xv, rv, sacc);
      aacc = __fmaf_rn(fabsf(xv), fabsf(rv), aacc);
    }
#pragma unroll
    for (int off = RW / 2; off >= 1; off >>= 1) {
      sacc = __fadd_rn(sacc, __shfl_xor_sync(gmask, sacc, off, RW));
      aacc = __fadd_rn(aacc, __shfl_xor_sync(gmask, aacc, off, RW));
    }
    int go_left;
    if (rec.z == rec.w) {  // rank split: every query goes left
      go_left = 1;
    } else {
      // q . r lies in [sacc - e, sacc + e]; the test runs in FP32 against
      // c rounded down / up (a subset of what the FP64 test decides)
      const float e = __fmul_ru(kerr, __fmul_ru(aacc, kA));
      if (__fadd_ru(sacc, e) < __double2float_rd(c)) {
        go_left = 1;
      } else if (__fsub_rd(sacc, e) >= __double2float_ru(c)) {
        go_left = 0;
      } else {  // undecided by the bound: the canonical FP64 chain
        int v = 0;
        if (sub == 0) {
          double p = 0.0;
          for (int k = 0; k < d; ++k) p = __fma_rn((double)__ldg(x + k), (double)__ldg(r32 + k), p);
          v = p < c;
        }
        go_left = __shfl_sync(gmask, v, 0, RW);
      }
    }
    node = go_left ? rec.z : rec.w;
    rec = __ldg(node_route + node);
  }
  if (sub == 0) qleaf[g] = make_int2(rec.x, rec.y);  // the leaf's (begin, length)
}

// The same walk with the query's coordinates held in registers and the next
// node's direction requested together with its routing record (PM >=
// ceil(d / 8) coordinates per lane), so a level costs one round trip even
// though the loop first tests the record.  The sums run in the same order as
// k_route_w's, so the decisions are the same.
template <int PM>
__global__ void __launch_bounds__(256) k_route_p(const float* __restrict__ Q, int64_t m, int d,
                                                 int T, const int4* __restrict__ node_route,
                                                 const float* __restrict__ node_dir32,
                                                 int2* qleaf) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / RW;
  const int lane = threadIdx.x & 31, sub = lane & (RW - 1);
  const unsigned gmask = ((1u << RW) - 1u) << (lane & ~(RW - 1));
  if (g >= m * T) return;  // whole group
  const int64_t q = g / T;
  const int t = (int)(g % T);
  const float* x = Q + q * d;
  const int per = (d + RW - 1) / RW;
  const float kerr = (float)(per + 7) * 0x1p-24f;
  const float kA = 1.0f + (float)(per + 6) * 0x1p-23f;
  float xv[PM], rv[PM];
#pragma unroll
  for (int i = 0; i < PM; ++i) {
    const int k = sub + RW * i;
    xv[i] = k < d ? __ldg(x + k) : 0.0f;
  }
  int node = t;
  int4 rec = __ldg(node_route + node);
#pragma unroll
  for (int i = 0; i < PM; ++i) {
    const int k = sub + RW * i;
    rv[i] = k < d ? __ldg(node_dir32 + (int64_t)node * d + k) : 0.0f;
  }
  while (rec.z >= 0) {
    const double c = __hiloint2double(rec.y, rec.x);
    float sacc = 0.0f, aacc = 0.0f;
#pragma unroll
    for (int i = 0; i < PM; ++i) {
      if (sub + RW * i < d) {
        sacc = __fmaf_rn(xv[i], rv[i], sacc);
        aacc = __fmaf_rn(fabsf(xv[i]), fabsf(rv[i]), aacc);
      }
    }
#pragma unroll
    for (int off = RW / 2; off >= 1; off >>= 1) {
      sacc = __fadd_rn(sacc, __shfl_xor_sync(gmask, sacc, off, RW));
      aacc = __fadd_rn(aacc, __shfl_xor_sync(gmask, aacc, off, RW));
    }
    int go_left;
    if (rec.z == rec.w) {  // rank split: every query goes left
      go_left = 1;
    } else {
      const float e = __fmul_ru(kerr, __fmul_ru(aacc, kA));
      if (__fadd_ru(sacc, e) < __double2float_rd(c)) {
        go_left = 1;
      } else if (__fsub_rd(sacc, e) >= __double2float_ru(c)) {
        go_left = 0;
      } else {  // undecided by the bound: the canonical FP64 chain
        int v = 0;
        if (sub == 0) {
          const float* r32 = node_dir32 + (int64_t)node * d;
          double p = 0.0;
          for (int k = 0; k < d; ++k) p = __fma_rn((double)__ldg(x + k), (double)__ldg(r32 + k), p);
          v = p < c;
        }
        go_left = __shfl_sync(gmask, v, 0, RW);
      }
    }
    node = go_left ? rec.z : rec.w;
    rec = __ldg(node_route + node);
#pragma unroll
    for (int i = 0; i < PM; ++i) {
      const int k = sub + RW * i;
      rv[i] = k < d ? __ldg(node_dir32 + (int64_t)node * d + k) : 0.0f;
    }
  }
  if (sub == 0) qleaf[g] = make_int2(rec.x, rec.y);  // the leaf's (begin, length)
}

// Ascending bitonic sort of one 64-bit key per lane (all 32 lanes).
__device__ __forceinline__ unsigned long long rpf_warp_sort(unsigned long long v, int lane) {
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const unsigned long long o = __shfl_xor_sync(RPF_FULL, v, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & kk) == 0);
      v = keep_min ? min(v, o) : max(v, o);
    }
  }
  return v;
}

// The 32 smallest keys of two ascending lists a, b (lane l holds element l
// of each), ascending: min(a_l, b_{31-l}) holds them as a bitonic sequence,
// which a bitonic merge sorts.
__device__ __forceinline__ unsigned long long rpf_warp_merge_min(unsigned long long a,
                                                                 unsigned long long b, int lane) {
  unsigned long long v = min(a, __shfl_sync(RPF_FULL, b, 31 - lane));
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const unsigned long long o = __shfl_xor_sync(RPF_FULL, v, j);
    v = (lane & j) == 0 ? min(v, o) : max(v, o);
  }
  return v;
}

// Leaf scan for queries, one CTA of QS_T threads per (query q, tree t): the
// leaf's rows are staged in shared memory by bulk copies, thread j computes
// the canonical d32 of q and leaf point j, and a bitonic sort of the 64-bit
// keys (d32 bits << 32 | index, ordered exactly like (d32, index)) gives the
// leaf's top-K (for K <= 32: register sorts per warp and a merge of the four
// warps' lists).  Leaves of at most QS_T points.
#define QS_T 128
__global__ void __launch_bounds__(QS_T) k_qscan_cta(const float* __restrict__ Q, int64_t m, int d,
                                                    int dp, int T, int K, const int2* qleaf,
                                                    const int32_t* __restrict__ perm,
                                                    const float* __restrict__ X, int64_t n,
                                                    uint2* cand, int* err, uint64_t wlim) {
  extern __shared__ __align__(16) float qs_rows[];  // QS_T x dp, then the query (dp)
  __shared__ unsigned long long keys[QS_T];
  __shared__ int pid[QS_T];
  __shared__ __align__(8) uint64_t bar;
  const int64_t g = blockIdx.x;
  const int64_t q = g / T;
  const int t = (int)(g % T);
  const int tid = threadIdx.x;
  const int2 lf = qleaf[g];  // the leaf's (begin, length) in tree t's permutation
  const int len = lf.y;
  const int32_t* mem = perm + (int64_t)t * n + lf.x;
  float* qv = qs_rows + QS_T * dp;
  if (tid < len) pid[tid] = mem[tid];
  for (int k = tid; k < dp; k += QS_T) qv[k] = k < d ? Q[q * d + k] : 0.0f;
  if (tid == 0) {
    rpf_mbar_init(&bar, 1);
    rpf_mbar_arrive_expect_tx(&bar, (uint32_t)len * (uint32_t)d * 4u);
  }
  __syncthreads();
  if (tid < len) {
    rpf_bulk_g2s(qs_rows + tid * dp, X + (int64_t)pid[tid] * d, (uint32_t)d * 4u, &bar);
    for (int k = d; k < dp; ++k) qs_rows[tid * dp + k] = 0.0f;
  }
  const bool ok = __syncthreads_and(rpf_mbar_wait(&bar, 0, err, wlim)) != 0;
  if (!ok) {  // one more bounded wait for copies in flight, then give up
    rpf_mbar_wait(&bar, 0, nullptr, wlim);
    // empty list for this (query, tree): the merge still reads defined slots
    if (tid < K) cand[((int64_t)t * m + q) * K + tid] = make_uint2(0x7f800000u, 0xffffffffu);
    return;
  }
  unsigned long long key = ~0ull;
  if (tid < len) {
    const float* y = qs_rows + tid * dp;
    float acc = 0.0f;
    for (int k = 0; k < d; k += 4) {
      const float4 a = *reinterpret_cast<const float4*>(qv + k);
      const float4 b = *reinterpret_cast<const float4*>(y + k);
      acc = sq_chain4(a, b, acc);
    }
    key = ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)pid[tid];
  }
  if (K <= 32) {
    // every warp sorts its 32 keys in registers; warp 0 merges the four
    // sorted lists, keeping the 32 smallest at each merge (one barrier)
    keys[tid] = rpf_warp_sort(key, tid & 31);
    __syncthreads();
    if (tid < 32) {
      unsigned long long v = keys[tid];
#pragma unroll
      for (int w = 1; w < QS_T / 32; ++w) v = rpf_warp_merge_min(v, keys[32 * w + tid], tid);
      if (tid < K)
        cand[((int64_t)t * m + q) * K + tid] =
            v == ~0ull ? make_uint2(0x7f800000u, 0xffffffffu)
                       : make_uint2((unsigned)(v >> 32), (unsigned)v);
    }
    return;
  }
  keys[tid] = key;
  __syncthreads();
  for (int kk = 2; kk <= QS_T; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const int p = tid ^ j;
      if (p > tid) {
        const unsigned long long a = keys[tid], b = keys[p];
        const bool up = (tid & kk) == 0;
        if ((a > b) == up) {
          keys[tid] = b;
          keys[p] = a;
        }
      }
      __syncthreads();
    }
  }
  if (tid < K) {
    const unsigned long long v = keys[tid];
    cand[((int64_t)t * m + q) * K + tid] =
        v == ~0ull ? make_uint2(0x7f800000u, 0xffffffffu)
                   : make_uint2((unsigned)(v >> 32), (unsigned)v);
  }
}

// Final merge for a batch of queries, one CTA per query: its T per-tree
// lists (T K entries) are sorted together as 64-bit keys (bitonic sort in
// shared memory), duplicates -- the same point found in several trees, with
// identical keys -- are dropped, and the first K distinct keys are the answer
// (the same list the running merge k_merge produces).  T K <= QM_MAX.
#define QM_T 256
#define QM_MAX 4096
__global__ void __launch_bounds__(QM_T) k_qmerge_cta(int64_t m, int K, int T, int N,
                                                     const uint2* __restrict__ cand,
                                                     int32_t* idx, float* dist) {
  extern __shared__ unsigned long long mk[];  // N keys, N a power of two
  __shared__ int wsum[QM_T / 32];
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int TK = T * K;
  for (int i = tid; i < N; i += QM_T) {
    unsigned long long key = ~0ull;
    if (i < TK) {
      const int t = i / K, j = i - t * K;
      const uint2 e = cand[((int64_t)t * m + q) * K + j];
      if (e.y != 0xffffffffu) key = ((unsigned long long)e.x << 32) | e.y;
    }
    mk[i] = key;
  }
  __syncthreads();
  for (int kk = 2; kk <= N; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < N; i += QM_T) {
        const int p = i ^ j;
        if (p > i) {
          const unsigned long long a = mk[i], b = mk[p];
          if ((a > b) == ((i & kk) == 0)) {
            mk[i] = b;
            mk[p] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  // rank of every distinct key: each thread takes a contiguous segment
  const int S = (N + QM_T - 1) / QM_T;
  const int s0 = min(tid * S, N), s1 = min(s0 + S, N);
  int cnt = 0;
  for (int i = s0; i < s1; ++i)
    cnt += mk[i] != ~0ull && (i == 0 || mk[i] != mk[i - 1]);
  int x = cnt;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(RPF_FULL, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int base = 0, total = 0;
  for (int w = 0; w < QM_T / 32; ++w) {
    if (w < warp) base += wsum[w];
    total += wsum[w];
  }
  int r = base + x - cnt;
  for (int i = s0; i < s1 && r < K; ++i) {
    const unsigned long long v = mk[i];
    if (v != ~0ull && (i == 0 || v != mk[i - 1])) {
      idx[q * K + r] = (int)(unsigned)v;
      dist[q * K + r] = __fsqrt_rn(__uint_as_float((unsigned)(v >> 32)));
      ++r;
    }
  }
  for (int rr = total + tid; rr < K; rr += QM_T) {
    idx[q * K + rr] = -1;
    dist[q * K + rr] = INFINITY;
  }
}

// Exact kNN by brute force (ground truth for the Sec. 5.1 metrics): one
// thread per query row, every data row in order; all threads of a block read
// the same data row at a time (broadcast).
template <int KMAX>
__global__ void k_brute(const float* X, int64_t n, int d, const float* Q, int64_t m,
                        const int32_t* self, int K, int32_t* idx, float* dist) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = q < m;
  const float* x = X;
  const float* y = Q + (live ? q : 0) * d;
  const int me = (live && self) ? self[q] : -1;
  TopK<KMAX> tk;
  tk.init();
  for (int64_t j = 0; j < n; ++j) {
    if ((int)j == me) continue;
    tk.offer(rpf_d32(y, x + j * d, d), (int)j);
  }
  if (!live) return;
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
    if (k < K) {
      idx[q * K + k] = tk.ki[k];
      dist[q * K + k] = tk.ki[k] < 0 ? INFINITY : __fsqrt_rn(tk.kd[k]);
    }
}

template <int KMAX>
void launch_brute(const float* X, int64_t n, int d, const float* Q, int64_t m,
                  const int32_t* self, int K, int32_t* idx, float* dist, cudaStream_t s) {
  RPF_LAUNCH("k_brute", s, k_brute<KMAX><<<nblk(m, 64), 64, 0, s>>>(X, n, d, Q, m, self, K, idx, dist));
}

template <int KMAX>
void launch_leaf(const rpf_forest* f, int64_t tb, int64_t nt, int K, int t0, uint2* cand, int* err,
                 cudaStream_t s) {
  const int rows = f->tile_rows;
  const int dp = ((f->d + 3) & ~3) + 4;
  const size_t smem = sizeof(float) * (size_t)rows * dp;
#define RPF_LEAF(REGV, STAGEV, SM)                                                             \
  do {                                                                                         \
    cudaFuncSetAttribute(k_leaf_plain<KMAX, REGV, STAGEV>,                                     \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SM));              \
    RPF_LAUNCH("k_leaf_plain", s, k_leaf_plain<KMAX, REGV, STAGEV><<<(unsigned)nt, 128, SM, s>>>( \
        f->tile_cnt, f->tile_off, f->tile_leaf, tb, f->leaf_tree, f->leaf_begin, f->leaf_len,  \
        f->perm, f->X, f->n, f->d, dp, K, t0, cand, err, rpf_wait_limit_ns()));                \
  } while (0)
  if (smem > 200 * 1024) RPF_LEAF(false, false, 0);   // rows read from global memory
  else if (dp == 68) RPF_LEAF(true, true, smem);      // 64-float rows held in registers
  else RPF_LEAF(false, true, smem);
#undef RPF_LEAF
}

template <int KMAX>
void launch_merge(int64_t n, int K, int G, const uint2* cand, const uint2* run_in,
                  uint2* run_out, bool first, bool last, int32_t* idx, float* dist,
                  cudaStream_t s) {
  RPF_LAUNCH("k_merge", s, k_merge<KMAX><<<nblk(n, 128), 128, 0, s>>>(
      n, K, G, cand, run_in, run_out, first, last, idx, dist));
}

template <int KMAX>
void launch_qscan(const rpf_forest* f, const float* Q, int64_t m, int K, const int2* qleaf,
                  uint2* cand, cudaStream_t s) {
  const int T = f->prm.n_trees;
  RPF_LAUNCH("k_qscan", s, k_qscan<KMAX><<<nblk(m * T, 128), 128, 0, s>>>(
      Q, m, f->d, T, K, qleaf, f->perm, f->X, f->n, cand));
}

#define RPF_KDISPATCH(K, FN, ...)                 \
  do {                                            \
    if ((K) <= 8) FN<8>(__VA_ARGS__);             \
    else if ((K) <= 16) FN<16>(__VA_ARGS__);      \
    else if ((K) <= 32) FN<32>(__VA_ARGS__);      \
    else if ((K) <= 64) FN<64>(__VA_ARGS__);      \
    else FN<128>(__VA_ARGS__);                    \
  } while (0)
// the plain leaf tiles also get lists of exactly 10 and 20 (the common K)
#define RPF_LEAF_KDISPATCH(K, FN, ...)            \
  do {                                            \
    if ((K) <= 8) FN<8>(__VA_ARGS__);             \
    else if ((K) <= 10) FN<10>(__VA_ARGS__);      \
    else if ((K) <= 16) FN<16>(__VA_ARGS__);      \
    else if ((K) <= 20) FN<20>(__VA_ARGS__);      \
    else if ((K) <= 32) FN<32>(__VA_ARGS__);      \
    else if ((K) <= 64) FN<64>(__VA_ARGS__);      \
    else FN<128>(__VA_ARGS__);                    \
  } while (0)

}  // namespace

namespace {
__global__ void k_tile_count(int64_t nl, const int32_t* leaf_tree, const int32_t* leaf_begin,
                             int64_t ntile, int R, int32_t* cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl) return;
  atomicAdd(&cnt[leaf_tree[i] * ntile + leaf_begin[i] / R], 1);
}
__global__ void k_tile_fill(int64_t nl, const int32_t* leaf_tree, const int32_t* leaf_begin,
                            int64_t ntile, int R, const int32_t* off, int32_t* cur,
                            int32_t* tile_leaf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl) return;
  const int64_t tile = leaf_tree[i] * ntile + leaf_begin[i] / R;
  tile_leaf[off[tile] + atomicAdd(&cur[tile], 1)] = (int32_t)i;
}
}  // namespace

// ---------------------------------------------------------------------------
// All-kNN work list, on the device: tile (t, k) takes the leaves of tree t
// whose begin lies in [k R, (k + 1) R).  Leaves of a tree tile its
// permutation, so a tile's rows are contiguous and number at most R + L - 1;
// every tree has exactly ceil(n / R) tiles (possibly empty).  R is the
// largest multiple of 32 up to the leaf bound for which the tile's rows fit in
// shared memory.
// ---------------------------------------------------------------------------
// The largest valid tile region for leaf bound L: a multiple of 32, at most
// 256 (leaves starting in one tile) and with R + L - 1 <= 1024 rows.
int rpf_region_cap(int L) {
  const int R = std::min(256, 1024 - L + 1 > 0 ? std::max(32, ((1024 - L + 1) / 32) * 32) : 32);
  return std::max(32, R);
}

int rpf_build_tiles(rpf_forest* f, cudaStream_t s, int R_force) {
  const int T = f->prm.n_trees, L = f->prm.leaf_max;
  const int dp = ((f->d + 3) & ~3) + 4;
  // prefer tiles small enough for four CTAs per SM (<= 56 KB of rows),
  // unless the autotuner chose a region for this (d, L) or the caller forces one
  int R = std::max(32, ((L + 31) / 32) * 32);
  while (R > 32 && (size_t)(R + L - 1) * dp * 4 > 56 * 1024) R -= 32;
  const int tuned = R_force > 0 ? R_force : rpf_tuned_region(f->d, L);
  if (tuned > 0) R = tuned;
  R = std::min(std::max(32, R & ~31), rpf_region_cap(L));
  // a rebuild replaces the previous tables (stream-ordered)
  rpf_release(f->tile_cnt, s);
  rpf_release(f->tile_off, s);
  rpf_release(f->tile_leaf, s);
  f->tile_cnt = f->tile_off = f->tile_leaf = nullptr;
  const int64_t ntile = (f->n + R - 1) / R;
  const int64_t N = (int64_t)T * ntile;
  const int64_t nl = f->n_leaves;
  int32_t *blk = nullptr, *tot = nullptr, *cur = nullptr;
  if (rpf_alloc((void**)&f->tile_cnt, 4 * (size_t)N, s) ||
      rpf_alloc((void**)&f->tile_off, 4 * (size_t)(N + 1), s) ||
      rpf_alloc((void**)&f->tile_leaf, 4 * (size_t)std::max<int64_t>(nl, 1), s) ||
      rpf_alloc((void**)&cur, 4 * (size_t)N, s) ||
      rpf_alloc((void**)&blk, 4 * (size_t)((N + 1023) / 1024 + 1), s) ||
      rpf_alloc((void**)&tot, 4, s)) {
    rpf_release(cur, s);
    rpf_release(blk, s);
    return RPF_ENOMEM;
  }
  RPF_CU(cudaMemsetAsync(f->tile_cnt, 0, 4 * (size_t)N, s));
  RPF_CU(cudaMemsetAsync(cur, 0, 4 * (size_t)N, s));
  RPF_LAUNCH("k_tile_count", s, k_tile_count<<<nblk(nl, 256), 256, 0, s>>>(
      nl, f->leaf_tree, f->leaf_begin, ntile, R, f->tile_cnt));
  const int32_t* cnt = f->tile_cnt;
  int32_t* off = f->tile_off;
  rpf_scan(N, [=] __device__(int64_t i) -> int { return cnt[i]; },
           [=] __device__(int64_t i, int p) { off[i] = p; }, blk, tot, s);
  RPF_LAUNCH("k_tile_fill", s, k_tile_fill<<<nblk(nl, 256), 256, 0, s>>>(
      nl, f->leaf_tree, f->leaf_begin, ntile, R, f->tile_off, cur, f->tile_leaf));
  rpf_release(cur, s);
  rpf_release(blk, s);
  rpf_release(tot, s);
  f->tile_region = R;
  f->tile_rows = R + L - 1;
  f->tiles_per_tree = ntile;
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

// [error word of an enqueue-only call (RPF_QERR_BYTES)][running lists]
// [per-tree lists of every tree]
size_t rpf_all_knn_ws(const rpf_forest* f, int K) {
  const int64_t n = f->n;
  const int T = f->prm.n_trees;
  return RPF_QERR_BYTES + align256((size_t)T * n * K * 8) + align256((size_t)n * K * 8);
}

int rpf_leaf_plain(const rpf_forest* f, int t0, int g, int K, uint2* cand, cudaStream_t s) {
  const int64_t tb = (int64_t)t0 * f->tiles_per_tree, nt = (int64_t)g * f->tiles_per_tree;
  if (nt > 0) RPF_LEAF_KDISPATCH(K, launch_leaf, f, tb, nt, K, t0, cand, f->d_err, s);
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

int rpf_merge_dev(int64_t n, int K, int G, const uint2* lists, int32_t* idx, float* dist,
                  cudaStream_t s) {
  RPF_KDISPATCH(K, launch_merge, n, K, G, lists, nullptr, nullptr, true, true, idx, dist, s);
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

int rpf_all_knn_enqueue(rpf_forest* f, int T, int K, int32_t* idx, float* dist, void* ws,
                        size_t ws_bytes, cudaStream_t s, uint2* keys) {
  const int64_t n = f->n;
  const size_t run_b = align256((size_t)n * K * 8);
  const size_t per_tree = (size_t)n * K * 8;
  if (ws_bytes < run_b + align256(per_tree)) return RPF_EINVAL;
  int G = (int)std::min<int64_t>(T, (int64_t)((ws_bytes - run_b) / per_tree));
  while (G > 1 && align256((size_t)G * per_tree) + run_b > ws_bytes) --G;
  uint2* run = (uint2*)ws;
  uint2* cand = (uint2*)((char*)ws + run_b);
  for (int t0 = 0; t0 < T; t0 += G) {
    const int g = std::min(G, T - t0);
    const int64_t tb = (int64_t)t0 * f->tiles_per_tree;
    const int64_t nt = (int64_t)g * f->tiles_per_tree;
    if (nt > 0) {
      if (f->prm.form == 1 && rpf_tc_supported(f, K)) {
        const int rc = rpf_leaf_tc(f, t0, g, K, cand, s);
        if (rc) return rc;
      } else {
        if (f->prm.form == 1) ++f->plain_groups;  // chosen form not available here
        RPF_LEAF_KDISPATCH(K, launch_leaf, f, tb, nt, K, t0, cand, f->d_err, s);
      }
    }
    const bool first = t0 == 0, last = t0 + g >= T;
    // with keys, the last merge writes the running list into the caller's keys
    uint2* out_run = (last && keys) ? keys : run;
    RPF_KDISPATCH(K, launch_merge, n, K, g, cand, run, out_run, first, last && !keys, idx, dist,
                  s);
  }
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

int rpf_all_knn_dev(rpf_forest* f, int T, int K, int32_t* idx, float* dist, void* ws,
                    size_t ws_bytes, cudaStream_t s, uint2* keys) {
  const int rc = rpf_all_knn_enqueue(f, T, K, idx, dist, ws, ws_bytes, s, keys);
  if (rc) return rc;
  // a bounded device wait that gave up is reported here
  int herr = 0;
  RPF_CU(cudaMemcpyAsync(&herr, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  RPF_CU(cudaStreamSynchronize(s));
  if (herr) {
    cudaMemsetAsync(f->d_err, 0, sizeof(int), s);
    return herr;
  }
  return RPF_OK;
}

size_t rpf_query_core_ws(int64_t m, int T, int K) {
  return RPF_QERR_BYTES + align256((size_t)m * T * 8) + align256((size_t)T * m * K * 8);
}

size_t rpf_query_ws(const rpf_forest* f, int64_t m, int K) {
  return rpf_query_core_ws(m, f->prm.n_trees, K) + align256((size_t)m * f->d * 4) +
         align256((size_t)m * K * 4) + align256((size_t)m * K * 4);
}

// The leaf of each of m queries in every tree, as its (begin, length) in the
// tree's permutation, into qleaf (m x T).
int rpf_route_dev(const rpf_forest* f, const float* Q, int64_t m, int2* qleaf, cudaStream_t s) {
  const int T = f->prm.n_trees;
  const int per = (f->d + RW - 1) / RW;
  const unsigned grid = nblk(m * T * RW, 256);
#define RPF_ROUTE_P(PMV)                                                             \
  RPF_LAUNCH("k_route_w", s, k_route_p<PMV><<<grid, 256, 0, s>>>(Q, m, f->d, T,       \
                                                                  f->node_route,      \
                                                                  f->node_dir32, qleaf))
  if (per <= 4) RPF_ROUTE_P(4);
  else if (per <= 8) RPF_ROUTE_P(8);
  else if (per <= 12) RPF_ROUTE_P(12);
  else if (per <= 16) RPF_ROUTE_P(16);
  else
    RPF_LAUNCH("k_route_w", s, k_route_w<<<grid, 256, 0, s>>>(
        Q, m, f->d, T, f->node_route, f->node_dir32, qleaf));
#undef RPF_ROUTE_P
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

// Per-tree lists of the leaves in qleaf: the chosen form's BF16 scan when
// `bf` (and the scan covers (f, K)), else the FP32 scan.
int rpf_qscan_dev(const rpf_forest* f, const float* Q, int64_t m, int K, const int2* qleaf,
                  uint2* cand, int* qerr, bool bf, cudaStream_t s) {
  const int T = f->prm.n_trees;
  const int dp = ((f->d + 3) & ~3) + 4;
  const size_t qsm = (size_t)(QS_T + 1) * dp * 4;
  if (bf && rpf_qscan_bf_ok(f, K)) {  // BF16 rows, certified exact re-rank
    const int rc = rpf_qscan_bf(f, Q, m, K, qleaf, cand, qerr, s);
    if (rc) return rc;
  } else if (f->prm.leaf_max <= QS_T && (f->d % 4) == 0 && qsm <= 200 * 1024) {
    RPF_CU(cudaFuncSetAttribute(k_qscan_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm));
    RPF_LAUNCH("k_qscan_cta", s, k_qscan_cta<<<(unsigned)(m * T), QS_T, qsm, s>>>(
        Q, m, f->d, dp, T, K, qleaf, f->perm, f->X,
        f->n, cand, qerr, rpf_wait_limit_ns()));
  } else {
    RPF_KDISPATCH(K, launch_qscan, f, Q, m, K, qleaf, cand, s);
  }
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

// Query scratch: [error word (RPF_QERR_BYTES)][leaf id per (query, tree)]
// [per-tree candidate lists].  The error word is cleared here and set by a
// bounded device wait that gave up, so it describes this call only.  The
// chosen form scans the BF16 rows unless the forest asks for the FP32 scan,
// or leaves the pick to the autotuner and it found the FP32 scan faster for
// this shape (both give the same lists).
int rpf_query_dev(const rpf_forest* f, const float* Q, int64_t m, int K, int32_t* idx,
                  float* dist, void* ws, size_t ws_bytes, cudaStream_t s) {
  const int T = f->prm.n_trees;
  if (ws_bytes < rpf_query_core_ws(m, T, K)) return RPF_EINVAL;
  int* qerr = (int*)ws;
  RPF_CU(cudaMemsetAsync(qerr, 0, sizeof(int), s));
  int2* qleaf = (int2*)((char*)ws + RPF_QERR_BYTES);
  uint2* cand = (uint2*)((char*)qleaf + align256((size_t)m * T * 8));
  int rc = rpf_route_dev(f, Q, m, qleaf, s);
  if (rc) return rc;
  const bool bf = f->prm.form == 1 && (f->qscan_mode >= 0 ? f->qscan_mode == 1
                                                           : rpf_tuned_qscan(f->d, f->prm.leaf_max, K) != 0);
  if ((rc = rpf_qscan_dev(f, Q, m, K, qleaf, cand, qerr, bf, s))) return rc;
  if ((int64_t)T * K <= QM_MAX) {
    int N = 1;
    while (N < T * K) N <<= 1;
    RPF_LAUNCH("k_qmerge_cta", s, k_qmerge_cta<<<(unsigned)m, QM_T, (size_t)N * 8, s>>>(
        m, K, T, N, cand, idx, dist));
  } else {
    RPF_KDISPATCH(K, launch_merge, m, K, T, cand, nullptr, nullptr, true, true, idx, dist, s);
  }
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

int rpf_brute_dev(const float* X, int64_t n, int d, const float* Q, int64_t m,
                  const int32_t* self, int K, int32_t* idx, float* dist, cudaStream_t s) {
  RPF_KDISPATCH(K, launch_brute, X, n, d, Q, m, self, K, idx, dist, s);
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}
