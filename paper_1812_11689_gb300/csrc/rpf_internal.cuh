// rpf_internal.cuh -- device helpers and the forest object of the GB300
// rpForests library (arXiv 1812.11689).  Compiled with -fmad=false: every
// fused multiply-add below is written out with __fma_rn / __fmaf_rn, so the
// FP64 arithmetic that decides tree structure is the same sequence of IEEE
// operations on every run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rpforest.h"

#define RPF_GAMMA 0x9E3779B97F4A7C15ULL
#define RPF_TAG_DIR 1ULL
#define RPF_TAG_SPLIT 2ULL
#define RPF_SPLIT_ATTEMPTS 8
#define RPF_CHUNK 4096  // canonical reduction chunk; also the growth work chunk
#define RPF_MAX_TRY 64
#define RPF_MAX_D 4096
#define RPF_MAX_K 128
#define RPF_MAX_LEAF 1024  // a leaf is one CTA tile of at most 1024 rows
#define RPF_FULL 0xffffffffu
// deferred split points of the subtree kernel: candidates recorded per
// extreme, and int32 words per record (node id, counts, candidates)
#define RPF_DEFER_CAND 6
#define RPF_DEFER_REC 16

// ---------------------------------------------------------------------------
// Counter-based random numbers for the direction draws and the uniform split
// point of Algorithms 1-2 (Sec. 2).  mix64 is the SplitMix64 output function (Steele, Lea &
// Flood 2014); word() absorbs (tag, tree, node key, try/attempt, counter) into
// the seed one field at a time.  Root key 1; child key = mix64(key ^ (1 +
// side) * GAMMA), side 0 = left, 1 = right.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t rpf_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// word() in two parts: the chain over (tag, t, key, j), shared by every
// counter c of one (node, try), then the last field
__host__ __device__ __forceinline__ uint64_t rpf_word_prefix(uint64_t seed, uint64_t tag,
                                                             uint64_t t, uint64_t key, uint64_t j) {
  uint64_t h = seed;
  h = rpf_mix64((h ^ tag) + RPF_GAMMA);
  h = rpf_mix64((h ^ t) + RPF_GAMMA);
  h = rpf_mix64((h ^ key) + RPF_GAMMA);
  h = rpf_mix64((h ^ j) + RPF_GAMMA);
  return h;
}
__host__ __device__ __forceinline__ uint64_t rpf_word_last(uint64_t h, uint64_t c) {
  return rpf_mix64((h ^ c) + RPF_GAMMA);
}
__host__ __device__ __forceinline__ uint64_t rpf_word(uint64_t seed, uint64_t tag, uint64_t t,
                                                      uint64_t key, uint64_t j, uint64_t c) {
  return rpf_word_last(rpf_word_prefix(seed, tag, t, key, j), c);
}

__host__ __device__ __forceinline__ uint64_t rpf_child_key(uint64_t key, int side) {
  return rpf_mix64(key ^ ((uint64_t)(1 + side) * RPF_GAMMA));
}

// u53 = (w >> 11) 2^-53 in [0, 1)
__device__ __forceinline__ double rpf_u53(uint64_t w) {
  return __dmul_rn((double)(w >> 11), 0x1p-53);
}

// Coefficients of the FP32 series below, fixed at compile time from their
// definitions: 1/(2k+1) (atanh series) and (-1)^k / n! (cos / sin series,
// n! a running double product), each rounded once to FP32.
constexpr float rpf_lnc(int k) { return (float)(1.0 / (double)(2 * k + 1)); }
constexpr double rpf_inv_fact(int n) {
  double f = 1.0;
  for (int i = 1; i <= n; ++i) f = f * (double)i;
  return 1.0 / f;
}
constexpr float rpf_cosc(int k) { return (float)((k & 1) ? -rpf_inv_fact(2 * k) : rpf_inv_fact(2 * k)); }
constexpr float rpf_sinc(int k) {
  return (float)((k & 1) ? -rpf_inv_fact(2 * k + 1) : rpf_inv_fact(2 * k + 1));
}

// ---------------------------------------------------------------------------
// ln(u) in FP32 for normal u > 0: u = m 2^e, m folded into [sqrt(2)/2,
// sqrt(2)], ln m = 2 atanh(s), s = (m - 1)/(m + 1), atanh Taylor series
// s (1 + z/3 + ... + z^5/11), z = s^2 <= 0.0295.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rpf_lnf(float u) {
  const float LN2F = 0.693147180559945309f;
  const float SQRT2F = 1.41421356237309504f;
  uint32_t b = __float_as_uint(u);
  int e = (int)((b >> 23) & 0xff) - 127;
  float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
  if (m > SQRT2F) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  float z = __fmul_rn(s, s);
  constexpr float L0 = rpf_lnc(0), L1 = rpf_lnc(1), L2 = rpf_lnc(2), L3 = rpf_lnc(3);
  constexpr float L4 = rpf_lnc(4), L5 = rpf_lnc(5);
  float p = L5;
  p = __fmaf_rn(p, z, L4);
  p = __fmaf_rn(p, z, L3);
  p = __fmaf_rn(p, z, L2);
  p = __fmaf_rn(p, z, L1);
  p = __fmaf_rn(p, z, L0);
  float h = __fmul_rn(s, p);
  return __fmaf_rn((float)e, LN2F, __fadd_rn(h, h));
}

// ---------------------------------------------------------------------------
// cos(2 pi u), sin(2 pi u) in FP32, u in [0, 1): quadrant q = floor(4u),
// theta = (4u - q) pi/2, Taylor series of cos / sin to theta^12 / theta^13.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rpf_sincos2pif(float u, float* c_out, float* s_out) {
  const float PI_2F = 1.57079632679489662f;
  float x = __fmul_rn(u, 4.0f);
  int q = (int)x;
  float f = __fsub_rn(x, (float)q);
  float th = __fmul_rn(f, PI_2F);
  float z = __fmul_rn(th, th);
  constexpr float C0 = rpf_cosc(0), C1 = rpf_cosc(1), C2 = rpf_cosc(2), C3 = rpf_cosc(3);
  constexpr float C4 = rpf_cosc(4), C5 = rpf_cosc(5), C6 = rpf_cosc(6);
  constexpr float S0 = rpf_sinc(0), S1 = rpf_sinc(1), S2 = rpf_sinc(2), S3 = rpf_sinc(3);
  constexpr float S4 = rpf_sinc(4), S5 = rpf_sinc(5), S6 = rpf_sinc(6);
  float cs = C6, sn = S6;
  cs = __fmaf_rn(cs, z, C5);
  sn = __fmaf_rn(sn, z, S5);
  cs = __fmaf_rn(cs, z, C4);
  sn = __fmaf_rn(sn, z, S4);
  cs = __fmaf_rn(cs, z, C3);
  sn = __fmaf_rn(sn, z, S3);
  cs = __fmaf_rn(cs, z, C2);
  sn = __fmaf_rn(sn, z, S2);
  cs = __fmaf_rn(cs, z, C1);
  sn = __fmaf_rn(sn, z, S1);
  cs = __fmaf_rn(cs, z, C0);
  sn = __fmaf_rn(sn, z, S0);
  sn = __fmul_rn(sn, th);
  switch (q & 3) {
    case 0: *c_out = cs; *s_out = sn; break;
    case 1: *c_out = -sn; *s_out = cs; break;
    case 2: *c_out = -cs; *s_out = -sn; break;
    default: *c_out = sn; *s_out = -cs; break;
  }
}

// ---------------------------------------------------------------------------
// Canonical FP64 warp sum of one chunk (<= 4096 values): lane l adds
// v[l], v[l+32], ... in order from +0.0, then the lane sums are folded by
// xor-butterfly 16, 8, 4, 2, 1 (lane 0 follows s_l += s_{l+off}).  Every lane
// returns the result.  All 32 lanes must call it.  The values are fetched 8
// at a time ahead of the additions (same order of additions), so the FP64
// chain does not wait for a load at every step.
// ---------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ double rpf_warp_chunk_sum(int64_t len, int lane, F val) {
  double a = 0.0;
  int64_t k = lane;
  for (; k + 32 * 7 < len; k += 32 * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = val(k + 32 * u);
#pragma unroll
    for (int u = 0; u < 8; ++u) a = __dadd_rn(a, v[u]);
  }
  for (; k < len; k += 32) a = __dadd_rn(a, val(k));
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) a = __dadd_rn(a, __shfl_xor_sync(RPF_FULL, a, off));
  return a;
}

// Order-preserving map of doubles to uint64 (for atomicMin / atomicMax).
__device__ __forceinline__ unsigned long long rpf_dkey(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double rpf_dkey_inv(unsigned long long k) {
  unsigned long long b = (k & 0x8000000000000000ULL) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
  return __longlong_as_double((long long)b);
}

// Canonical FP32 squared distance (ranking key of every neighbour list).
__device__ __forceinline__ float rpf_d32(const float* x, const float* y, int d) {
  float s = 0.0f;
  for (int k = 0; k < d; ++k) {
    float e = __fsub_rn(x[k], y[k]);
    s = __fmaf_rn(e, e, s);
  }
  return s;
}

// (d, i) < (e, j) in the neighbour order; index -1 means "empty" (+inf).
__device__ __forceinline__ bool rpf_less(float d, int i, float e, int j) {
  return d < e || (d == e && (unsigned)i < (unsigned)j);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct rpf_dbuf {  // owned device allocation
  void* p = nullptr;
  size_t bytes = 0;
};

struct rpf_forest {
  int64_t n = 0;
  int32_t d = 0;
  rpf_params prm{};
  // global index of the forest's first tree: the random draws of tree t use
  // t_base + t (0 for a build; the current tree count while rpf_add_trees
  // grows new trees into a temporary forest)
  int32_t t_base = 0;
  int device = 0;

  float* X = nullptr;         // n x d
  float* xnorm = nullptr;     // n: upper bound of |x|_2
  // chosen form: BF16 copy of X (bits), rows padded to d8 = 8 ceil(d / 8)
  uint16_t* X16 = nullptr;
  int32_t d8 = 0;
  int32_t* perm = nullptr;    // T x n final permutation

  // node table (capacity nodes_cap)
  int64_t n_nodes = 0, nodes_cap = 0;
  uint64_t* node_key = nullptr;
  int32_t* node_tree = nullptr;
  int32_t* node_begin = nullptr;
  int32_t* node_len = nullptr;
  int32_t* node_left = nullptr;
  int32_t* node_right = nullptr;
  int32_t* node_jstar = nullptr;
  int32_t* node_flag = nullptr;
  double* node_c = nullptr;
  // n_nodes x d: r* of every split node (zeros for leaves and rank splits);
  // the directions are FP32 values, so widening them gives the FP64 r*
  // exactly
  float* node_dir32 = nullptr;
  // per node, what routing reads at one step: (c as two words, left child,
  // right child); a rank split stores its left child on both sides, a leaf
  // has left = -1 (rpf_build_route)
  int4* node_route = nullptr;

  // leaves
  int64_t n_leaves = 0;
  int32_t* leaf_tree = nullptr;
  int32_t* leaf_begin = nullptr;
  int32_t* leaf_len = nullptr;
  int32_t max_depth = 0;
  int64_t n_exact = 0;  // nodes decided by the FP64 fallback

  // all-kNN tiles: tile (t, k) holds the leaves of tree t whose begin lies in
  // [k R, (k + 1) R); a tile has at most R + L - 1 rows
  int32_t tile_region = 0;        // R
  int32_t tile_rows = 0;          // R + L - 1
  int64_t tiles_per_tree = 0;     // ceil(n / R)
  int32_t* tile_cnt = nullptr;    // leaves per tile
  int32_t* tile_off = nullptr;    // first entry of the tile in tile_leaf
  int32_t* tile_leaf = nullptr;   // leaf indices grouped by tile

  // chosen-form tiles: runs of consecutive leaves of one tree, <= 128 rows
  int4* pk_tiles = nullptr;          // (tree, first position, rows, 0), tree-major
  uint32_t* pk_bits = nullptr;       // T x pk_nwords: bit p set iff a leaf begins at p
  int64_t pk_nwords = 0;
  int32_t pk_rows = 128;             // tile row capacity: 128, or 256 when L > 128
  std::vector<int64_t> pk_tree_off;  // first tile of every tree (T + 1 entries)

  int* d_err = nullptr;  // device error word (RPF_ETIMEOUT from bounded waits)
  unsigned long long* d_fallback = nullptr;  // rows the BF16 form rescanned exactly
  // tree groups of rpf_all_knn calls that asked for the chosen form and ran
  // the plain one (leaf bound > 256, K > 32, or a row too wide for the tile)
  int64_t plain_groups = 0;
  // query leaf scan of the chosen form: -1 = the autotuner's pick (BF16 rows
  // when untuned), 0 = FP32 rows, 1 = BF16 rows (rpf_set_query_scan)
  int32_t qscan_mode = -1;

  // staging for host outputs of rpf_all_knn
  void* stage = nullptr;
  size_t stage_bytes = 0;

  std::vector<void*> owned;
};

// Packed FP32 pair arithmetic (one instruction, two lanes of work each, each
// half rounded exactly as the scalar operation would round it).
__device__ __forceinline__ float2 rpf_sub2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "sub.rn.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 rpf_add2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "add.rn.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 rpf_fma2(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, c, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "mov.b64 c, {%6, %7};\n\tfma.rn.f32x2 r, a, b, c;\n\tmov.b64 {%0, %1}, r;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

// Two FP32 values rounded to nearest-even BF16 in one instruction, packed
// (lo in bits 0-15, hi in bits 16-31).
__device__ __forceinline__ uint32_t rpf_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Launch accounting (rpf_trace.cu): RPF_LAUNCH(name, stream, kernel<<<...>>>(...));
struct rpf_trace_scope {
  rpf_trace_scope(const char* name, cudaStream_t s);
  ~rpf_trace_scope();
  cudaStream_t s_;
  int id_ = 0;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};
#define RPF_LAUNCH(name, stream, ...)          \
  do {                                         \
    rpf_trace_scope rpf_ts_((name), (stream)); \
    __VA_ARGS__;                               \
  } while (0)

#define RPF_CU(call)                                  \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return rpf_cuda_err(e_);   \
  } while (0)

int rpf_cuda_err(cudaError_t e);
// time limit of every bounded device wait (rpf_set_wait_limit), nanoseconds
uint64_t rpf_wait_limit_ns();
bool rpf_is_device_ptr(const void* p);
// Stream-ordered device allocation from the device's default pool, which is
// set to keep freed memory cached (repeated builds reuse it without syncs).
int rpf_alloc(void** p, size_t bytes, cudaStream_t s);
void rpf_release(void* p, cudaStream_t s);

// growth (rpf_grow.cu)
int rpf_grow(rpf_forest* f, cudaStream_t s);
// leaf tiles + merge + query (rpf_knn.cu); R_force > 0 sets the tile region
int rpf_build_tiles(rpf_forest* f, cudaStream_t s, int R_force = 0);
int rpf_region_cap(int L);
// plain-form leaf tiles of trees [t0, t0 + g) into cand
int rpf_leaf_plain(const rpf_forest* f, int t0, int g, int K, uint2* cand, cudaStream_t s);
// chosen-form leaf tiles (rpf_leaf_tc.cu); rows_force > 0 sets the tile rows
int rpf_build_packs(rpf_forest* f, cudaStream_t s, int rows_force = 0);
// build-time tile choices the autotuner kept for (d, leaf bound), 0 if none
int rpf_tuned_region(int d, int L);
int rpf_tuned_rows(int d, int L);
bool rpf_tc_supported(const rpf_forest* f, int K);
int rpf_leaf_tc(const rpf_forest* f, int t0, int g, int K, uint2* cand, cudaStream_t s);
// times the leaf-tile configurations on f's tiles (plain: region; chosen:
// rows, Gram chunk, CTAs per SM), keeps the fastest for the rest of the
// process and applies the tile shape to f; chosen = {chunk, CTAs, rows, R}
int rpf_tc_autotune(rpf_forest* f, int K, cudaStream_t s, int32_t* chosen);
// all-kNN over the first T trees (T <= n_trees: nested ensembles)
// keys != nullptr: the final lists go there as (d32 bits, index) pairs
// instead of (idx, dist)
int rpf_all_knn_dev(rpf_forest* f, int T, int K, int32_t* idx, float* dist, void* ws,
                    size_t ws_bytes, cudaStream_t s, uint2* keys = nullptr);
// merge of G sorted (d32 bits, index) lists per point into the final lists
int rpf_merge_dev(int64_t n, int K, int G, const uint2* lists, int32_t* idx, float* dist,
                  cudaStream_t s);
int rpf_query_dev(const rpf_forest* f, const float* Q, int64_t m, int K, int32_t* idx, float* dist,
                  void* ws, size_t ws_bytes, cudaStream_t s);
int rpf_brute_dev(const float* X, int64_t n, int d, const float* Q, int64_t m,
                  const int32_t* self, int K, int32_t* idx, float* dist, cudaStream_t s);
size_t rpf_all_knn_ws(const rpf_forest* f, int K);
size_t rpf_query_ws(const rpf_forest* f, int64_t m, int K);
// scratch of rpf_query_dev alone (error word, leaf ids, per-tree lists)
size_t rpf_query_core_ws(int64_t m, int T, int K);
// the query error word heads every query scratch
#define RPF_QERR_BYTES 256
// device address of the allocation-free query's scratch on the current
// device (rpf_static.cu), or nullptr with *rc set
void* rpf_static_scratch(int* rc);
// the routing records of every node (after growth or a merge of tables)
int rpf_build_route(rpf_forest* f, cudaStream_t s);
// chosen-form query scan (rpf_qscan_bf.cu): the BF16 copy of X, whether the
// scan covers (f, K), and the launch over m x T (query, tree) leaves
int rpf_build_x16(rpf_forest* f, cudaStream_t s);
bool rpf_qscan_bf_ok(const rpf_forest* f, int K);
int rpf_qscan_bf(const rpf_forest* f, const float* Q, int64_t m, int K, const int2* qleaf,
                 uint2* cand, int* err, cudaStream_t s);
// the query path in parts (rpf_knn.cu): routing, and the leaf scan in the
// BF16 (bf) or FP32 form
int rpf_route_dev(const rpf_forest* f, const float* Q, int64_t m, int2* qleaf, cudaStream_t s);
int rpf_qscan_dev(const rpf_forest* f, const float* Q, int64_t m, int K, const int2* qleaf,
                  uint2* cand, int* qerr, bool bf, cudaStream_t s);
// the query scan the autotuner kept for (d, leaf bound, K): 1 = BF16 rows,
// 0 = FP32 rows, -1 = not tuned
int rpf_tuned_qscan(int d, int L, int K);
void rpf_launch_directions(uint64_t seed, int32_t t, const uint64_t* keys_dev, int32_t n_keys,
                           int32_t j, int32_t d, double* out_dev, cudaStream_t s);
