// rpf_grow.cu -- rpTree growth for all T trees at once, level by level
// (Sec. 2, Algorithm 1 per tree, Algorithm 2 for the split direction).
//
// A tree is a permutation `perm` of 0..n-1 in which every node is a
// contiguous segment.  Each level takes the frontier (all nodes of all trees
// holding more than L points), cuts it into chunks of <= 4096 positions of one
// node, and runs:
//   k_dirs        nTry candidate directions per node (FP64 r, FP32 copy)
//   [G-B]         k_proj32 -> k_stats32 -> k_var32 -> k_certify -> k_cand:
//                 FP32 projections with a certified error radius decide the
//                 direction choice and the min/max whenever the bound allows;
//                 the rest of the node is marked "exact"
//   [exact]       k_proj64 -> k_csum_chunks/k_csum_nodes (S, then V): the
//                 canonical FP64 statistics of Algorithm 2
//   k_split       c = fma(u, b - a, a), redrawn until a < c <= b (Algorithm 1
//                 "c ~ runif[a, b]"), else a rank split
//   k_side_count  p < c per point (FP32 certified or FP64), chunk counts
//   k_node_scan   child sizes, node table, chunk offsets
//   k_scatter     stable partition into the next permutation (leaf children
//                 go straight to the final permutation)
//   k_frontier    next frontier, new leaves, next chunk list
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "rpf_internal.cuh"

namespace {

constexpr int kBlock = 256;

struct Level {  // per-level device arrays, grown on demand
  int64_t cap_f = 0, cap_c = 0, cap_dir = 0;
  // frontier (two sets: current and next)
  int32_t *fr_node[2]{}, *fr_tree[2]{}, *fr_begin[2]{}, *fr_len[2]{}, *fr_cb[2]{}, *fr_nc[2]{};
  uint64_t* fr_key[2]{};
  // per frontier node results
  int32_t *fr_exact{}, *fr_jstar{}, *fr_flag{}, *fr_nl{};
  double *fr_a{}, *fr_b{}, *fr_c{};
  double *fr_mu{}, *fr_min{}, *fr_max{};  // F x ntry
  float *fr_tl{}, *fr_tr{}, *fr_rad{};     // certified thresholds, error radius
  float *fr_min32{}, *fr_max32{};          // F x ntry
  double *fr_vhat{}, *fr_ebound{};         // F x ntry (G-B estimate, bound)
  unsigned long long *fr_akey{}, *fr_bkey{};
  // chunks (two sets)
  int32_t *ch_node[2]{}, *ch_start[2]{}, *ch_len[2]{};
  int32_t *ch_nleft{}, *ch_loff{};
  double *cp_sum{}, *cp_min{}, *cp_max{};  // C x ntry
  float *cp_min32{}, *cp_max32{}, *cp_xmax{};
  double *cp_s1{}, *cp_s2{};
  // directions of the level
  double* dir64{};
  float* dir32{};
};

struct Counts {
  int32_t f_next, c_next, n_leaves_new, pad;
};

template <typename T>
int grow_buf(T** p, int64_t old_n, int64_t new_n, cudaStream_t s, bool keep) {
  T* q = nullptr;
  cudaError_t e = cudaMalloc((void**)&q, sizeof(T) * (size_t)std::max<int64_t>(new_n, 1));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RPF_ENOMEM : rpf_cuda_err(e);
  if (*p) {
    if (keep && old_n > 0) {
      e = cudaMemcpyAsync(q, *p, sizeof(T) * (size_t)old_n, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return rpf_cuda_err(e);
    }
    cudaStreamSynchronize(s);
    cudaFree(*p);
  }
  *p = q;
  return RPF_OK;
}

// ---------------------------------------------------------------------------
__global__ void k_init_perm(int32_t* perm, int64_t n, int T) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * T) return;
  perm[i] = (int32_t)(i % n);
}

// |x|_2 rounded up: FP32 sum of squares then a relative margin covering the
// d + 2 roundings of the computation.
__global__ void k_xnorm(const float* X, int64_t n, int d, float* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* x = X + i * d;
  float s = 0.0f;
  for (int k = 0; k < d; ++k) s = __fmaf_rn(x[k], x[k], s);
  float r = __fsqrt_ru(s);
  out[i] = __fmul_ru(r, 1.0f + (float)(d + 4) * 0x1p-23f);
}

// Candidate direction r = g/|g| for (tree t, node key, try j) (Algorithms 1-2,
// "generate a random direction"): Box-Muller pairs from words 2i and 2i+1.
__device__ void gen_direction(uint64_t seed, uint64_t t, uint64_t key, uint64_t j, int d,
                              double* r) {
  for (int i = 0; 2 * i < d; ++i) {
    uint64_t w1 = rpf_word(seed, RPF_TAG_DIR, t, key, j, (uint64_t)(2 * i));
    uint64_t w2 = rpf_word(seed, RPF_TAG_DIR, t, key, j, (uint64_t)(2 * i + 1));
    double u1 = __dmul_rn((double)((w1 >> 11) + 1), 0x1p-53);
    double u2 = __dmul_rn((double)(w2 >> 11), 0x1p-53);
    double rho = __dsqrt_rn(__dmul_rn(-2.0, rpf_ln(u1)));
    double c, s;
    rpf_sincos2pi(u2, &c, &s);
    r[2 * i] = __dmul_rn(rho, c);
    if (2 * i + 1 < d) r[2 * i + 1] = __dmul_rn(rho, s);
  }
  double ss = 0.0;
  for (int k = 0; k < d; ++k) ss = __fma_rn(r[k], r[k], ss);
  double nrm = __dsqrt_rn(ss);
  if (nrm == 0.0) {
    for (int k = 0; k < d; ++k) r[k] = 0.0;
    r[0] = 1.0;
    return;
  }
  for (int k = 0; k < d; ++k) r[k] = __ddiv_rn(r[k], nrm);
}

__global__ void k_dirs(int F, int ntry, int d, uint64_t seed, const int32_t* fr_tree,
                       const uint64_t* fr_key, double* dir64, float* dir32) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)F * ntry) return;
  int f = (int)(g / ntry), j = (int)(g % ntry);
  double* r = dir64 + g * d;
  gen_direction(seed, (uint64_t)fr_tree[f], fr_key[f], (uint64_t)j, d, r);
  float* r32 = dir32 + g * d;
  for (int k = 0; k < d; ++k) r32[k] = __double2float_rn(r[k]);
}

// Standalone direction generation (inspection entry point).
__global__ void k_dirs_keys(uint64_t seed, int32_t t, const uint64_t* keys, int nk, int j, int d,
                            double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk) return;
  gen_direction(seed, (uint64_t)t, keys[i], (uint64_t)j, d, out + (int64_t)i * d);
}

// ---------------------------------------------------------------------------
// G-B: FP32 projections with a certified error radius.
//
// For a point x and a candidate r (|r| = 1 up to FP64 rounding), the FP32
// projection p32 (fmaf chain against r32 = fl32(r)) and the canonical FP64
// projection p64 differ by at most
//     |p32 - p64| <= ((d+2) u32 + d u64) sum_k |x_k r_k| <= kappa_d |x|_2,
// u32 = 2^-24, u64 = 2^-53 (fma-chain dot-product bound plus the rounding of
// r to FP32; Cauchy-Schwarz with |r| <= 1 + d u64).  kappa_d = (d + 4) 2^-24
// covers these terms for d <= 4096.  rad(node) = kappa_d max_x |x|_2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kappa_of(int d) { return (float)(d + 4) * 0x1p-24f * 1.0625f; }

// One block per chunk: p32 for every try, stored; per-chunk FP64 sum of p32
// and FP32 min/max per try, max |x|.
__global__ void __launch_bounds__(kBlock) k_proj32(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, const float* X, const int32_t* perm_cur, const float* xnorm, int64_t n,
    int64_t Tn, int d, int ntry, const float* dir32, float* p32, double* cp_s1, float* cp_min32,
    float* cp_max32, float* cp_xmax) {
  extern __shared__ float sm[];
  float* r = sm;                   // ntry x d
  float* red = sm + ntry * d;      // reduction scratch: kBlock floats
  const int c = blockIdx.x;
  const int f = ch_node[c];
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const int len = ch_len[c];
  for (int i = threadIdx.x; i < ntry * d; i += blockDim.x) r[i] = dir32[(int64_t)f * ntry * d + i];
  __syncthreads();
  float xmax = 0.0f;
  for (int j0 = 0; j0 < ntry; j0 += 8) {
    const int nj = min(8, ntry - j0);
    float s1[8], mn[8], mx[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      s1[q] = 0.0f;
      mn[q] = INFINITY;
      mx[q] = -INFINITY;
    }
    double s1d[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) s1d[q] = 0.0;
    int cnt = 0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const int32_t pid = perm_cur[base + i];
      const float* x = X + (int64_t)pid * d;
      if (j0 == 0) xmax = fmaxf(xmax, xnorm[pid]);
      float acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
      for (int k = 0; k < d; ++k) {
        const float xv = __ldg(x + k);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nj) acc[q] = __fmaf_rn(xv, r[(j0 + q) * d + k], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q < nj) {
          p32[(int64_t)(j0 + q) * Tn + base + i] = acc[q];
          s1[q] = __fadd_rn(s1[q], acc[q]);
          mn[q] = fminf(mn[q], acc[q]);
          mx[q] = fmaxf(mx[q], acc[q]);
        }
      }
      if (++cnt == 16) {  // flush the FP32 partial sums into FP64 every 16 points
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          s1d[q] = __dadd_rn(s1d[q], (double)s1[q]);
          s1[q] = 0.0f;
        }
        cnt = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s1d[q] = __dadd_rn(s1d[q], (double)s1[q]);
    // block reductions (sum in FP64 via warp shuffles, min/max in FP32)
    for (int q = 0; q < nj; ++q) {
      double sv = s1d[q];
      float a = mn[q], b = mx[q];
      for (int off = 16; off >= 1; off >>= 1) {
        sv = __dadd_rn(sv, __shfl_xor_sync(RPF_FULL, sv, off));
        a = fminf(a, __shfl_xor_sync(RPF_FULL, a, off));
        b = fmaxf(b, __shfl_xor_sync(RPF_FULL, b, off));
      }
      __shared__ double wsum[kBlock / 32];
      __shared__ float wmn[kBlock / 32], wmx[kBlock / 32];
      const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
      if (l == 0) {
        wsum[w] = sv;
        wmn[w] = a;
        wmx[w] = b;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double S = 0.0;
        float A = INFINITY, B = -INFINITY;
        for (int u = 0; u < kBlock / 32; ++u) {
          S = __dadd_rn(S, wsum[u]);
          A = fminf(A, wmn[u]);
          B = fmaxf(B, wmx[u]);
        }
        cp_s1[(int64_t)c * ntry + j0 + q] = S;
        cp_min32[(int64_t)c * ntry + j0 + q] = A;
        cp_max32[(int64_t)c * ntry + j0 + q] = B;
      }
      __syncthreads();
    }
  }
  // chunk max |x|
  for (int off = 16; off >= 1; off >>= 1) xmax = fmaxf(xmax, __shfl_xor_sync(RPF_FULL, xmax, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = xmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.0f;
    for (int u = 0; u < kBlock / 32; ++u) m = fmaxf(m, red[u]);
    cp_xmax[c] = m;
  }
}

// Per node: mean estimate of p32 per try, FP32 min/max, error radius.
__global__ void k_stats32(int F, int ntry, int d, const int32_t* fr_cb, const int32_t* fr_nc,
                          const int32_t* fr_len, const double* cp_s1, const float* cp_min32,
                          const float* cp_max32, const float* cp_xmax, double* fr_mu,
                          float* fr_min32, float* fr_max32, float* fr_rad) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int cb = fr_cb[f], nc = fr_nc[f];
  float xm = 0.0f;
  for (int c = cb; c < cb + nc; ++c) xm = fmaxf(xm, cp_xmax[c]);
  fr_rad[f] = __fmul_ru(xm, kappa_of(d));
  for (int j = 0; j < ntry; ++j) {
    double S = 0.0;
    float A = INFINITY, B = -INFINITY;
    for (int c = cb; c < cb + nc; ++c) {
      S = __dadd_rn(S, cp_s1[(int64_t)c * ntry + j]);
      A = fminf(A, cp_min32[(int64_t)c * ntry + j]);
      B = fmaxf(B, cp_max32[(int64_t)c * ntry + j]);
    }
    fr_mu[(int64_t)f * ntry + j] = __ddiv_rn(S, (double)fr_len[f]);
    fr_min32[(int64_t)f * ntry + j] = A;
    fr_max32[(int64_t)f * ntry + j] = B;
  }
}

// Per chunk: sum of (p32 - mu32)^2 (FP32 within a thread over <= 16 points,
// FP64 across) and sum of |p32 - mu32| (for the error bound).
__global__ void __launch_bounds__(kBlock) k_var32(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, int64_t n, int64_t Tn, int ntry, const float* p32,
    const double* fr_mu, double* cp_s2, double* cp_s1) {
  const int c = blockIdx.x;
  const int f = ch_node[c];
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const int len = ch_len[c];
  __shared__ double w2[kBlock / 32], w1[kBlock / 32];
  for (int j = 0; j < ntry; ++j) {
    const float mu = __double2float_rn(fr_mu[(int64_t)f * ntry + j]);
    const float* p = p32 + (int64_t)j * Tn + base;
    double a2 = 0.0, a1 = 0.0;
    float s2 = 0.0f, s1 = 0.0f;
    int cnt = 0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      float e = __fsub_rn(p[i], mu);
      s2 = __fmaf_rn(e, e, s2);
      s1 = __fadd_rn(s1, fabsf(e));
      if (++cnt == 16) {
        a2 = __dadd_rn(a2, (double)s2);
        a1 = __dadd_rn(a1, (double)s1);
        s2 = s1 = 0.0f;
        cnt = 0;
      }
    }
    a2 = __dadd_rn(a2, (double)s2);
    a1 = __dadd_rn(a1, (double)s1);
    for (int off = 16; off >= 1; off >>= 1) {
      a2 = __dadd_rn(a2, __shfl_xor_sync(RPF_FULL, a2, off));
      a1 = __dadd_rn(a1, __shfl_xor_sync(RPF_FULL, a1, off));
    }
    if ((threadIdx.x & 31) == 0) {
      w2[threadIdx.x >> 5] = a2;
      w1[threadIdx.x >> 5] = a1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double S2 = 0.0, S1 = 0.0;
      for (int u = 0; u < kBlock / 32; ++u) {
        S2 = __dadd_rn(S2, w2[u]);
        S1 = __dadd_rn(S1, w1[u]);
      }
      cp_s2[(int64_t)c * ntry + j] = S2;
      cp_s1[(int64_t)c * ntry + j] = S1;  // reused: sum |p32 - mu32|
    }
    __syncthreads();
  }
}

// Per node: certify the direction choice of Algorithm 2 from the FP32
// estimates.  With v_j = sqrt(Vhat_j), Vhat_j = sum (p32 - mu32)^2, the
// canonical FP64 dispersion V_j satisfies |sqrt(V_j) - v_j| <= E_j, where E_j
// collects
//   sqrt(m) rad                  p64 vs p32: sqrt of a centred sum of squares
//                                is 1-Lipschitz in the vector of projections
//   sqrt(m) (|mu - mu32| + 17 u32 mean|p32|)
//                                centring at mu32 instead of the exact mean
//                                (FP32 partial sums of <= 16 terms)
//   20 u32 v_j                   rounding of (p32 - mu32)^2 and its FP32
//                                accumulation (<= 16 terms per partial)
//   1e-12 v_j + sqrt(m) 1e-13 mean|p|   the canonical FP64 reduction itself
// and the whole sum is doubled for safety.  Certified iff the first argmax w has
// v_w - E_w > v_k + E_k for every k != w and v_w - E_w > 0.  Certified nodes
// also get the min/max candidate windows [min32, min32 + 2 rad] and
// [max32 - 2 rad, max32] for the exact a and b.
__global__ void k_certify(int F, int ntry, const int32_t* fr_cb, const int32_t* fr_nc,
                          const int32_t* fr_len, const double* cp_s2, const double* cp_s1,
                          const double* fr_mu, const float* fr_rad, const float* fr_min32,
                          const float* fr_max32, int32_t* fr_exact, int32_t* fr_jstar,
                          float* fr_tl, float* fr_tr, unsigned long long* fr_akey,
                          unsigned long long* fr_bkey, double* fr_vhat) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int cb = fr_cb[f], nc = fr_nc[f];
  const double m = (double)fr_len[f];
  const double rad = (double)fr_rad[f];
  const double sm = sqrt(m);
  int w = -1;
  double vw = -1.0, ew = 0.0;
  const double u32 = 0x1p-24;
  // first pass: estimates and the first argmax
  for (int j = 0; j < ntry; ++j) {
    double S2 = 0.0, S1 = 0.0;
    for (int c = cb; c < cb + nc; ++c) {
      S2 = __dadd_rn(S2, cp_s2[(int64_t)c * ntry + j]);
      S1 = __dadd_rn(S1, cp_s1[(int64_t)c * ntry + j]);
    }
    const double mu = fr_mu[(int64_t)f * ntry + j];
    const double mu32 = (double)__double2float_rn(mu);
    // exact variance sum about the exact mean <= about mu32 (drop the
    // non-negative shift term) -- so sqrt(S2) over-estimates by at most
    // sqrt(m)|mu_true - mu32|, folded into E below.
    const double v = sqrt(S2);
    const double mabs = S1 / m + fabs(mu);  // bounds the mean of |p32|
    const double shift = sm * (fabs(mu - mu32) + 17.0 * u32 * mabs);
    const double accum = 20.0 * u32 * v;
    const double e64 = 1e-12 * v + sm * 1e-13 * (mabs + rad);
    const double E = 2.0 * (sm * rad + shift + accum + e64);
    fr_vhat[(int64_t)f * ntry + j] = v;
    fr_vhat[(int64_t)F * ntry + (int64_t)f * ntry + j] = E;
    if (v > vw) {
      vw = v;
      ew = E;
      w = j;
    }
  }
  bool ok = (w >= 0) && (vw - ew > 0.0);
  for (int j = 0; j < ntry && ok; ++j) {
    if (j == w) continue;
    const double v = fr_vhat[(int64_t)f * ntry + j];
    const double E = fr_vhat[(int64_t)F * ntry + (int64_t)f * ntry + j];
    if (!(vw - ew > v + E)) ok = false;
  }
  if (!ok) {
    fr_exact[f] = 1;
    return;
  }
  fr_exact[f] = 0;
  fr_jstar[f] = w;
  const float r2 = __fmul_ru(2.0f, fr_rad[f]);
  fr_tl[f] = __fadd_ru(fr_min32[(int64_t)f * ntry + w], r2);  // min candidates: p32 <= tl
  fr_tr[f] = __fsub_rd(fr_max32[(int64_t)f * ntry + w], r2);  // max candidates: p32 >= tr
  fr_akey[f] = rpf_dkey(INFINITY);
  fr_bkey[f] = rpf_dkey(-INFINITY);
}

// Per chunk of a certified node: exact FP64 projections of the min / max
// candidates, folded into the node's a and b with ordered atomics.
__global__ void __launch_bounds__(kBlock) k_cand(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, const int32_t* fr_exact, const int32_t* fr_jstar, const float* fr_tl,
    const float* fr_tr, const float* X, const int32_t* perm_cur, int64_t n, int64_t Tn, int d,
    int ntry, const float* p32, const double* dir64, unsigned long long* fr_akey,
    unsigned long long* fr_bkey) {
  const int c = blockIdx.x;
  const int f = ch_node[c];
  if (fr_exact[f]) return;
  const int js = fr_jstar[f];
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const int len = ch_len[c];
  const float tl = fr_tl[f], tr = fr_tr[f];
  const float* p = p32 + (int64_t)js * Tn + base;
  const double* r = dir64 + ((int64_t)f * ntry + js) * d;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const float pv = p[i];
    const bool lo = pv <= tl, hi = pv >= tr;
    if (!lo && !hi) continue;
    const float* x = X + (int64_t)perm_cur[base + i] * d;
    double q = 0.0;
    for (int k = 0; k < d; ++k) q = __fma_rn((double)x[k], r[k], q);
    if (lo) atomicMin(&fr_akey[f], rpf_dkey(q));
    if (hi) atomicMax(&fr_bkey[f], rpf_dkey(q));
  }
}

__global__ void k_cand_finish(int F, const int32_t* fr_exact, const unsigned long long* fr_akey,
                              const unsigned long long* fr_bkey, double* fr_a, double* fr_b) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F || fr_exact[f]) return;
  fr_a[f] = rpf_dkey_inv(fr_akey[f]);
  fr_b[f] = rpf_dkey_inv(fr_bkey[f]);
}

// ---------------------------------------------------------------------------
// Exact path: canonical FP64 projections and statistics (Algorithm 2).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_proj64(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, const int32_t* fr_exact, const float* X, const int32_t* perm_cur,
    int64_t n, int64_t Tn, int d, int ntry, const double* dir64, double* p64) {
  const int c = blockIdx.x;
  const int f = ch_node[c];
  if (!fr_exact[f]) return;
  const int64_t base = (int64_t)fr_tree[f] * n + fr_begin[f] + ch_start[c];
  const int len = ch_len[c];
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const float* x = X + (int64_t)perm_cur[base + i] * d;
    for (int j = 0; j < ntry; ++j) {
      const double* r = dir64 + ((int64_t)f * ntry + j) * d;
      double p = 0.0;
      for (int k = 0; k < d; ++k) p = __fma_rn((double)__ldg(x + k), r[k], p);
      p64[(int64_t)j * Tn + base + i] = p;
    }
  }
}

// One warp per (chunk, try).  pass 0: canonical chunk sum of p, exact
// min/max; pass 1: canonical chunk sum of (p - mu)^2.
__global__ void k_csum_chunks(int pass, int C, int ntry, const int32_t* ch_node,
                              const int32_t* ch_start, const int32_t* ch_len,
                              const int32_t* fr_tree, const int32_t* fr_begin,
                              const int32_t* fr_exact, int64_t n, int64_t Tn, const double* p64,
                              const double* fr_mu, double* cp_sum, double* cp_min,
                              double* cp_max) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (int64_t)C * ntry) return;
  const int c = (int)(wid / ntry), j = (int)(wid % ntry);
  const int f = ch_node[c];
  if (!fr_exact[f]) return;
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

// Canonical reduction of a node's chunk partials for try j (stride ntry),
// recursing in place when there are more than 4096 chunks.
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

// One warp per exact node.  pass 0: S_j -> mu_j, min/max; pass 1: V_j, then
// Algorithm 2's choice: the first try with V > best, best starting at 0.
__global__ void k_csum_nodes(int pass, int F, int ntry, const int32_t* fr_cb, const int32_t* fr_nc,
                             const int32_t* fr_len, const int32_t* fr_exact, double* cp_sum,
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
  for (int j = 0; j < ntry; ++j) {
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

// ---------------------------------------------------------------------------
// Split point and node records.
// ---------------------------------------------------------------------------
__global__ void k_split(int F, int ntry, int d, uint64_t seed, const int32_t* fr_node,
                        const int32_t* fr_tree, const uint64_t* fr_key, const int32_t* fr_jstar,
                        const double* fr_a, const double* fr_b, const float* fr_rad,
                        double* fr_c, int32_t* fr_flag, float* fr_tl, float* fr_tr,
                        int32_t* node_jstar, int32_t* node_flag, double* node_c) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int js = fr_jstar[f];
  bool acc = false;
  double c = NAN;
  if (js >= 0) {
    const double a = fr_a[f], b = fr_b[f];
    for (int att = 0; att < RPF_SPLIT_ATTEMPTS; ++att) {
      double u = rpf_u53(rpf_word(seed, RPF_TAG_SPLIT, (uint64_t)fr_tree[f], fr_key[f],
                                  (uint64_t)att, 0));
      double cc = __fma_rn(u, __dsub_rn(b, a), a);
      if (cc > a && cc <= b) {
        c = cc;
        acc = true;
        break;
      }
    }
  }
  fr_c[f] = c;
  fr_flag[f] = acc ? 0 : 1;
  if (acc) {  // certified side thresholds: p32 < tl => p64 < c; p32 >= tr => p64 >= c
    const double rad = (double)fr_rad[f];
    float tl = __double2float_rd(__dsub_rd(c, rad));
    float tr = __double2float_ru(__dadd_ru(c, rad));
    fr_tl[f] = nextafterf(tl, -INFINITY);
    fr_tr[f] = nextafterf(tr, INFINITY);
  }
  const int id = fr_node[f];
  node_jstar[id] = js;
  node_flag[id] = acc ? 0 : 1;
  node_c[id] = c;
}

// Copy r* of every split node into the node table (one block per node).
__global__ void k_store_dirs(int F, int ntry, int d, const int32_t* fr_node, const int32_t* fr_jstar,
                             const int32_t* fr_flag, const double* dir64, double* node_dir,
                             float* node_dir32) {
  const int f = blockIdx.x;
  if (f >= F) return;
  const int id = fr_node[f];
  const int js = fr_jstar[f];
  const bool ok = js >= 0 && !fr_flag[f];
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double v = ok ? dir64[((int64_t)f * ntry + js) * d + k] : 0.0;
    node_dir[(int64_t)id * d + k] = v;
    node_dir32[(int64_t)id * d + k] = __double2float_rn(v);
  }
}

// ---------------------------------------------------------------------------
// Partition.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_side_count(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* fr_tree,
    const int32_t* fr_begin, const int32_t* fr_len, const int32_t* fr_exact,
    const int32_t* fr_jstar, const int32_t* fr_flag, const double* fr_c, const float* fr_tl,
    const float* fr_tr, const float* X, const int32_t* perm_cur, int64_t n, int64_t Tn, int d,
    int ntry, const float* p32, const double* p64, const double* dir64, uint8_t* side,
    int32_t* ch_nleft) {
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
  int cnt = 0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    bool left;
    if (flag) {
      left = (ch_start[c] + i) < (m >> 1);
    } else if (exact) {
      left = p64[(int64_t)js * Tn + base + i] < cc;
    } else {
      const float pv = p32[(int64_t)js * Tn + base + i];
      if (pv < tl) {
        left = true;
      } else if (pv >= tr) {
        left = false;
      } else {
        const float* x = X + (int64_t)perm_cur[base + i] * d;
        const double* r = dir64 + ((int64_t)f * ntry + js) * d;
        double q = 0.0;
        for (int k = 0; k < d; ++k) q = __fma_rn((double)x[k], r[k], q);
        left = q < cc;
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

__global__ void k_node_scan(int F, int L, int64_t id_base, const int32_t* fr_node,
                            const int32_t* fr_tree, const int32_t* fr_begin, const int32_t* fr_len,
                            const uint64_t* fr_key, const int32_t* fr_cb, const int32_t* fr_nc,
                            const int32_t* ch_nleft, int32_t* ch_loff, int32_t* fr_nl,
                            uint64_t* node_key, int32_t* node_tree, int32_t* node_begin,
                            int32_t* node_len, int32_t* node_left, int32_t* node_right,
                            int32_t* node_jstar, int32_t* node_flag, double* node_c) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
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
  (void)L;
}

// Stable scatter of one chunk: lefts keep their order at
// begin + (lefts before the chunk) + rank; rights at begin + nl + (rights
// before the chunk) + rank.  A child with <= L points is final.
__global__ void __launch_bounds__(kBlock) k_scatter(
    const int32_t* ch_node, const int32_t* ch_start, const int32_t* ch_len, const int32_t* ch_loff,
    const int32_t* fr_tree, const int32_t* fr_begin, const int32_t* fr_len, const int32_t* fr_nl,
    int L, int64_t n, const uint8_t* side, const int32_t* perm_cur, int32_t* perm_nxt,
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
  int32_t* dstL = (nl <= L) ? perm_final : perm_nxt;
  int32_t* dstR = ((m - nl) <= L) ? perm_final : perm_nxt;
  __shared__ int wsum[kBlock / 32];
  __shared__ int carry_s;
  int carryL = 0, carryR = 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t0 = 0; t0 < len; t0 += kBlock) {
    const int i = t0 + threadIdx.x;
    const bool valid = i < len;
    const int s = valid ? side[base + i] : 0;
    // block exclusive scan of s
    int x = s;
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
      carry_s = r;
    }
    __syncthreads();
    const int rankL = x - s + wsum[w];
    const int tileL = carry_s;
    if (valid) {
      const int32_t v = perm_cur[base + i];
      if (s) {
        dstL[tbase + begin + loff + carryL + rankL] = v;
      } else {
        const int rankR = threadIdx.x - rankL;
        dstR[tbase + begin + nl + roff + carryR + rankR] = v;
      }
    }
    const int nvalid = min(kBlock, len - t0);
    carryL += tileL;
    carryR += nvalid - tileL;
    __syncthreads();
  }
}

// Single block: next frontier (children with > L points, in child order),
// new leaves, and the next chunk list.
__global__ void __launch_bounds__(1024) k_frontier(
    int F, int L, int64_t id_base, const int32_t* fr_tree, const int32_t* fr_begin,
    const int32_t* fr_len, const uint64_t* fr_key, const int32_t* fr_nl, int32_t* nf_node,
    int32_t* nf_tree, int32_t* nf_begin, int32_t* nf_len, uint64_t* nf_key, int32_t* nf_cb,
    int32_t* nf_nc, int32_t* nch_node, int32_t* nch_start, int32_t* nch_len, int64_t leaf_base,
    int32_t* leaf_tree, int32_t* leaf_begin, int32_t* leaf_len, Counts* out) {
  __shared__ int ws_a[32], ws_l[32], ws_c[32];
  __shared__ int tot_a, tot_l, tot_c;
  __shared__ int run_a, run_l, run_c;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) run_a = run_l = 0;
  __syncthreads();
  const int NC = 2 * F;
  for (int t0 = 0; t0 < NC; t0 += 1024) {
    const int ci = t0 + threadIdx.x;
    int len = 0, active = 0, leaf = 0;
    if (ci < NC) {
      const int f = ci >> 1, side = ci & 1;
      len = side ? fr_len[f] - fr_nl[f] : fr_nl[f];
      active = len > L;
      leaf = !active;
    }
    int xa = active, xl = leaf;
    for (int off = 1; off < 32; off <<= 1) {
      int ya = __shfl_up_sync(RPF_FULL, xa, off), yl = __shfl_up_sync(RPF_FULL, xl, off);
      if (lane >= off) {
        xa += ya;
        xl += yl;
      }
    }
    if (lane == 31) {
      ws_a[w] = xa;
      ws_l[w] = xl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int ra = 0, rl = 0;
      for (int u = 0; u < 32; ++u) {
        int va = ws_a[u], vl = ws_l[u];
        ws_a[u] = ra;
        ws_l[u] = rl;
        ra += va;
        rl += vl;
      }
      tot_a = ra;
      tot_l = rl;
    }
    __syncthreads();
    if (ci < NC) {
      const int f = ci >> 1, side = ci & 1;
      const int begin = side ? fr_begin[f] + fr_nl[f] : fr_begin[f];
      if (active) {
        const int o = run_a + xa - active + ws_a[w];
        nf_node[o] = (int32_t)(id_base + ci);
        nf_tree[o] = fr_tree[f];
        nf_begin[o] = begin;
        nf_len[o] = len;
        nf_key[o] = rpf_child_key(fr_key[f], side);
        nf_nc[o] = (len + RPF_CHUNK - 1) / RPF_CHUNK;
      } else {
        const int64_t o = leaf_base + run_l + xl - leaf + ws_l[w];
        leaf_tree[o] = fr_tree[f];
        leaf_begin[o] = begin;
        leaf_len[o] = len;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      run_a += tot_a;
      run_l += tot_l;
    }
    __syncthreads();
  }
  const int FN = run_a;
  // chunk offsets of the next frontier
  if (threadIdx.x == 0) run_c = 0;
  __syncthreads();
  for (int t0 = 0; t0 < FN; t0 += 1024) {
    const int fi = t0 + threadIdx.x;
    const int nc = fi < FN ? nf_nc[fi] : 0;
    int x = nc;
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
  }
}

__global__ void k_count_exact(int F, const int32_t* fr_exact, unsigned long long* counter) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < F && fr_exact[f]) atomicAdd(counter, 1ULL);
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
int rpf_grow(rpf_forest* fo, cudaStream_t s) {
  const int64_t n = fo->n;
  const int d = fo->d;
  const int T = fo->prm.n_trees, L = fo->prm.leaf_max, ntry = fo->prm.n_try;
  const int growth = fo->prm.growth == 0 ? 2 : fo->prm.growth;
  const uint64_t seed = fo->prm.seed;
  const int64_t Tn = (int64_t)T * n;

  // permutations
  int32_t *perm_a = nullptr, *perm_b = nullptr;
  float* p32 = nullptr;
  double* p64 = nullptr;
  uint8_t* side = nullptr;
  Level lv;
  Counts* h_cnt = nullptr;
  Counts* d_cnt = nullptr;
  unsigned long long* d_exact = nullptr;
  std::vector<void*> tmp;
  auto talloc = [&](void** p, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RPF_ENOMEM : rpf_cuda_err(e);
    tmp.push_back(*p);
    return RPF_OK;
  };
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    for (void* p : tmp) cudaFree(p);
    tmp.clear();
    if (h_cnt) cudaFreeHost(h_cnt);
    h_cnt = nullptr;
  };
#define RPF_TRY(x)       \
  do {                   \
    int r_ = (x);        \
    if (r_) {            \
      cleanup();         \
      return r_;         \
    }                    \
  } while (0)
#define RPF_TRYCU(x) RPF_TRY(((x) == cudaSuccess) ? RPF_OK : rpf_cuda_err(cudaGetLastError()))

  RPF_TRY(talloc((void**)&perm_a, sizeof(int32_t) * Tn));
  RPF_TRY(talloc((void**)&perm_b, sizeof(int32_t) * Tn));
  RPF_TRY(talloc((void**)&side, Tn));
  RPF_TRY(talloc((void**)&d_cnt, sizeof(Counts)));
  RPF_TRY(talloc((void**)&d_exact, sizeof(unsigned long long)));
  RPF_TRYCU(cudaMemsetAsync(d_exact, 0, sizeof(unsigned long long), s));
  if (cudaMallocHost((void**)&h_cnt, sizeof(Counts)) != cudaSuccess) {
    cleanup();
    return RPF_ENOMEM;
  }
  if (growth == 2) RPF_TRY(talloc((void**)&p32, sizeof(float) * Tn * ntry));
  // the FP64 buffer is needed for every node under G-A, for the rare
  // undecided nodes under G-B
  RPF_TRY(talloc((void**)&p64, sizeof(double) * Tn * ntry));

  RPF_LAUNCH("k_init_perm", s, k_init_perm<<<nblk(Tn, 256), 256, 0, s>>>(perm_a, n, T));
  RPF_LAUNCH("k_init_perm", s, k_init_perm<<<nblk(Tn, 256), 256, 0, s>>>(fo->perm, n, T));
  RPF_LAUNCH("k_xnorm", s, k_xnorm<<<nblk(n, 256), 256, 0, s>>>(fo->X, n, d, fo->xnorm));

  // node table: roots 0..T-1
  auto ensure_nodes = [&](int64_t need) -> int {
    if (need <= fo->nodes_cap) return RPF_OK;
    int64_t nc = std::max<int64_t>(need, fo->nodes_cap * 2);
    int64_t old = fo->n_nodes;
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
    if ((r = grow_buf(&fo->node_dir, old * d, nc * d, s, true))) return r;
    if ((r = grow_buf(&fo->node_dir32, old * d, nc * d, s, true))) return r;
    // leaves never outnumber nodes
    if ((r = grow_buf(&fo->leaf_tree, fo->n_leaves, nc, s, true))) return r;
    if ((r = grow_buf(&fo->leaf_begin, fo->n_leaves, nc, s, true))) return r;
    if ((r = grow_buf(&fo->leaf_len, fo->n_leaves, nc, s, true))) return r;
    fo->nodes_cap = nc;
    return RPF_OK;
  };
  const int64_t est = (int64_t)T * (2 * ((n + L) / std::max(1, L / 2 + 1)) + 3);
  RPF_TRY(ensure_nodes(std::max<int64_t>(est, 2 * T + 2)));
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
    RPF_TRYCU(cudaMemsetAsync(fo->node_dir, 0, sizeof(double) * d * T, s));
    RPF_TRYCU(cudaMemsetAsync(fo->node_dir32, 0, sizeof(float) * d * T, s));
    fo->n_nodes = T;
    fo->n_leaves = 0;
    if (n <= L) {  // every root is a leaf
      RPF_TRYCU(cudaMemcpyAsync(fo->leaf_tree, tree.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaMemcpyAsync(fo->leaf_begin, zero.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaMemcpyAsync(fo->leaf_len, len.data(), 4 * T, cudaMemcpyHostToDevice, s));
      RPF_TRYCU(cudaStreamSynchronize(s));
      fo->n_leaves = T;
      fo->max_depth = 0;
      fo->n_exact = 0;
      cleanup();
      return RPF_OK;
    }
  }

  // level arrays
  auto ensure_level = [&](int64_t F, int64_t C) -> int {
    int r;
    if (F > lv.cap_f) {
      int64_t nf = std::max<int64_t>(F, lv.cap_f * 2);
      for (int q = 0; q < 2; ++q) {
        if ((r = grow_buf(&lv.fr_node[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_tree[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_begin[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_len[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_cb[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_nc[q], lv.cap_f, nf, s, true))) return r;
        if ((r = grow_buf(&lv.fr_key[q], lv.cap_f, nf, s, true))) return r;
      }
      if ((r = grow_buf(&lv.fr_exact, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_jstar, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_flag, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_nl, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_a, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_b, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_c, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_mu, 0, nf * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.fr_min, 0, nf * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.fr_max, 0, nf * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.fr_tl, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_tr, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_rad, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_min32, 0, nf * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.fr_max32, 0, nf * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.fr_vhat, 0, 2 * nf * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.fr_akey, 0, nf, s, false))) return r;
      if ((r = grow_buf(&lv.fr_bkey, 0, nf, s, false))) return r;
      lv.cap_f = nf;
    }
    if (F * ntry > lv.cap_dir) {
      int64_t nd = std::max<int64_t>(F * ntry, lv.cap_dir * 2);
      if ((r = grow_buf(&lv.dir64, 0, nd * d, s, false))) return r;
      if ((r = grow_buf(&lv.dir32, 0, nd * d, s, false))) return r;
      lv.cap_dir = nd;
    }
    if (C > lv.cap_c) {
      int64_t ncap = std::max<int64_t>(C, lv.cap_c * 2);
      for (int q = 0; q < 2; ++q) {
        if ((r = grow_buf(&lv.ch_node[q], lv.cap_c, ncap, s, true))) return r;
        if ((r = grow_buf(&lv.ch_start[q], lv.cap_c, ncap, s, true))) return r;
        if ((r = grow_buf(&lv.ch_len[q], lv.cap_c, ncap, s, true))) return r;
      }
      if ((r = grow_buf(&lv.ch_nleft, 0, ncap, s, false))) return r;
      if ((r = grow_buf(&lv.ch_loff, 0, ncap, s, false))) return r;
      if ((r = grow_buf(&lv.cp_sum, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_min, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_max, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_min32, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_max32, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_xmax, 0, ncap, s, false))) return r;
      if ((r = grow_buf(&lv.cp_s1, 0, ncap * ntry, s, false))) return r;
      if ((r = grow_buf(&lv.cp_s2, 0, ncap * ntry, s, false))) return r;
      lv.cap_c = ncap;
    }
    return RPF_OK;
  };
  auto free_level = [&]() {
    void* ps[] = {lv.fr_exact, lv.fr_jstar, lv.fr_flag, lv.fr_nl, lv.fr_a, lv.fr_b, lv.fr_c,
                  lv.fr_mu, lv.fr_min, lv.fr_max, lv.fr_tl, lv.fr_tr, lv.fr_rad, lv.fr_min32,
                  lv.fr_max32, lv.fr_vhat, lv.fr_akey, lv.fr_bkey, lv.ch_nleft, lv.ch_loff,
                  lv.cp_sum, lv.cp_min, lv.cp_max, lv.cp_min32, lv.cp_max32, lv.cp_xmax, lv.cp_s1,
                  lv.cp_s2, lv.dir64, lv.dir32};
    cudaStreamSynchronize(s);
    for (void* p : ps) cudaFree(p);
    for (int q = 0; q < 2; ++q) {
      void* qs[] = {lv.fr_node[q], lv.fr_tree[q], lv.fr_begin[q], lv.fr_len[q], lv.fr_cb[q],
                    lv.fr_nc[q], lv.fr_key[q], lv.ch_node[q], lv.ch_start[q], lv.ch_len[q]};
      for (void* p : qs) cudaFree(p);
    }
  };

  // root frontier
  int64_t F, C;
  int cur = 0;
  {
    F = T;
    const int nc1 = (int)((n + RPF_CHUNK - 1) / RPF_CHUNK);
    C = (int64_t)T * nc1;
    int rr = ensure_level(F, C);
    if (rr) {
      free_level();
      cleanup();
      return rr;
    }
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
    cudaMemcpyAsync(lv.fr_node[0], node.data(), 4 * T, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.fr_tree[0], tree.data(), 4 * T, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.fr_begin[0], begin.data(), 4 * T, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.fr_len[0], len.data(), 4 * T, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.fr_cb[0], cb.data(), 4 * T, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.fr_nc[0], ncv.data(), 4 * T, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.fr_key[0], key.data(), 8 * T, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.ch_node[0], chn.data(), 4 * C, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.ch_start[0], chs.data(), 4 * C, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lv.ch_len[0], chl.data(), 4 * C, cudaMemcpyHostToDevice, s);
    // the host vectors die at the end of this scope
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      free_level();
      cleanup();
      return rpf_cuda_err(e);
    }
  }

  int32_t* perm_cur = perm_a;
  int32_t* perm_nxt = perm_b;
  int level = 0;
  int err = RPF_OK;
  while (F > 0) {
    // room for this level and for the next frontier / chunk list written by
    // k_frontier (at most 2F children and C + 2F chunks); grown before any
    // pointer of this level is captured
    if ((err = ensure_level(2 * F, C + 2 * F))) break;
    if ((err = ensure_nodes(fo->n_nodes + 2 * F))) break;
    const int Fi = (int)F, Ci = (int)C;
    int32_t *fr_node = lv.fr_node[cur], *fr_tree = lv.fr_tree[cur], *fr_begin = lv.fr_begin[cur],
            *fr_len = lv.fr_len[cur], *fr_cb = lv.fr_cb[cur], *fr_nc = lv.fr_nc[cur];
    uint64_t* fr_key = lv.fr_key[cur];
    int32_t *ch_node = lv.ch_node[cur], *ch_start = lv.ch_start[cur], *ch_len = lv.ch_len[cur];

    RPF_LAUNCH("k_dirs", s, k_dirs<<<nblk((int64_t)F * ntry, 128), 128, 0, s>>>(Fi, ntry, d, seed, fr_tree, fr_key,
                                                          lv.dir64, lv.dir32));
    if (growth == 2) {
      const size_t smem = sizeof(float) * ((size_t)ntry * d + kBlock);
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_proj32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      RPF_LAUNCH("k_proj32", s, k_proj32<<<Ci, kBlock, smem, s>>>(ch_node, ch_start, ch_len, fr_tree, fr_begin, fo->X,
                                        perm_cur, fo->xnorm, n, Tn, d, ntry, lv.dir32, p32,
                                        lv.cp_s1, lv.cp_min32, lv.cp_max32, lv.cp_xmax));
      RPF_LAUNCH("k_stats32", s, k_stats32<<<nblk(F, 128), 128, 0, s>>>(Fi, ntry, d, fr_cb, fr_nc, fr_len, lv.cp_s1,
                                             lv.cp_min32, lv.cp_max32, lv.cp_xmax, lv.fr_mu,
                                             lv.fr_min32, lv.fr_max32, lv.fr_rad));
      RPF_LAUNCH("k_var32", s, k_var32<<<Ci, kBlock, 0, s>>>(ch_node, ch_start, ch_len, fr_tree, fr_begin, n, Tn, ntry, p32,
                                    lv.fr_mu, lv.cp_s2, lv.cp_s1));
      RPF_LAUNCH("k_certify", s, k_certify<<<nblk(F, 128), 128, 0, s>>>(Fi, ntry, fr_cb, fr_nc, fr_len, lv.cp_s2, lv.cp_s1,
                                             lv.fr_mu, lv.fr_rad, lv.fr_min32, lv.fr_max32,
                                             lv.fr_exact, lv.fr_jstar, lv.fr_tl, lv.fr_tr,
                                             lv.fr_akey, lv.fr_bkey, lv.fr_vhat));
      RPF_LAUNCH("k_cand", s, k_cand<<<Ci, kBlock, 0, s>>>(ch_node, ch_start, ch_len, fr_tree, fr_begin, lv.fr_exact,
                                   lv.fr_jstar, lv.fr_tl, lv.fr_tr, fo->X, perm_cur, n, Tn, d,
                                   ntry, p32, lv.dir64, lv.fr_akey, lv.fr_bkey));
      RPF_LAUNCH("k_cand_finish", s, k_cand_finish<<<nblk(F, 128), 128, 0, s>>>(Fi, lv.fr_exact, lv.fr_akey, lv.fr_bkey, lv.fr_a,
                                                 lv.fr_b));
    } else {
      RPF_LAUNCH("k_fill_i32", s, k_fill_i32<<<nblk(F, 256), 256, 0, s>>>(lv.fr_exact, F, 1));
      RPF_LAUNCH("k_fill_i32", s, k_fill_i32<<<nblk(F, 256), 256, 0, s>>>((int32_t*)lv.fr_rad, F, 0));
    }
    // exact path (all nodes under G-A; undecided nodes under G-B)
    RPF_LAUNCH("k_proj64", s, k_proj64<<<Ci, kBlock, 0, s>>>(ch_node, ch_start, ch_len, fr_tree, fr_begin, lv.fr_exact,
                                   fo->X, perm_cur, n, Tn, d, ntry, lv.dir64, p64));
    RPF_LAUNCH("k_csum_chunks", s, k_csum_chunks<<<nblk((int64_t)C * ntry * 32, 256), 256, 0, s>>>(
        0, Ci, ntry, ch_node, ch_start, ch_len, fr_tree, fr_begin, lv.fr_exact, n, Tn, p64,
        lv.fr_mu, lv.cp_sum, lv.cp_min, lv.cp_max));
    RPF_LAUNCH("k_csum_nodes", s, k_csum_nodes<<<nblk((int64_t)F * 32, 256), 256, 0, s>>>(
        0, Fi, ntry, fr_cb, fr_nc, fr_len, lv.fr_exact, lv.cp_sum, lv.cp_min, lv.cp_max, lv.fr_mu,
        lv.fr_min, lv.fr_max, lv.fr_jstar, lv.fr_a, lv.fr_b));
    RPF_LAUNCH("k_csum_chunks", s, k_csum_chunks<<<nblk((int64_t)C * ntry * 32, 256), 256, 0, s>>>(
        1, Ci, ntry, ch_node, ch_start, ch_len, fr_tree, fr_begin, lv.fr_exact, n, Tn, p64,
        lv.fr_mu, lv.cp_sum, lv.cp_min, lv.cp_max));
    RPF_LAUNCH("k_csum_nodes", s, k_csum_nodes<<<nblk((int64_t)F * 32, 256), 256, 0, s>>>(
        1, Fi, ntry, fr_cb, fr_nc, fr_len, lv.fr_exact, lv.cp_sum, lv.cp_min, lv.cp_max, lv.fr_mu,
        lv.fr_min, lv.fr_max, lv.fr_jstar, lv.fr_a, lv.fr_b));
    RPF_LAUNCH("k_count_exact", s, k_count_exact<<<nblk(F, 256), 256, 0, s>>>(Fi, lv.fr_exact, d_exact));
    RPF_LAUNCH("k_split", s, k_split<<<nblk(F, 128), 128, 0, s>>>(Fi, ntry, d, seed, fr_node, fr_tree, fr_key, lv.fr_jstar,
                                         lv.fr_a, lv.fr_b, lv.fr_rad, lv.fr_c, lv.fr_flag,
                                         lv.fr_tl, lv.fr_tr, fo->node_jstar, fo->node_flag,
                                         fo->node_c));
    RPF_LAUNCH("k_store_dirs", s, k_store_dirs<<<Fi, 128, 0, s>>>(Fi, ntry, d, fr_node, lv.fr_jstar, lv.fr_flag, lv.dir64,
                                    fo->node_dir, fo->node_dir32));
    RPF_LAUNCH("k_side_count", s, k_side_count<<<Ci, kBlock, 0, s>>>(ch_node, ch_start, ch_len, fr_tree, fr_begin, fr_len,
                                       lv.fr_exact, lv.fr_jstar, lv.fr_flag, lv.fr_c, lv.fr_tl,
                                       lv.fr_tr, fo->X, perm_cur, n, Tn, d, ntry, p32, p64,
                                       lv.dir64, side, lv.ch_nleft));
    RPF_LAUNCH("k_node_scan", s, k_node_scan<<<nblk(F, 128), 128, 0, s>>>(
        Fi, L, fo->n_nodes, fr_node, fr_tree, fr_begin, fr_len, fr_key, fr_cb, fr_nc, lv.ch_nleft,
        lv.ch_loff, lv.fr_nl, fo->node_key, fo->node_tree, fo->node_begin, fo->node_len,
        fo->node_left, fo->node_right, fo->node_jstar, fo->node_flag, fo->node_c));
    RPF_LAUNCH("k_scatter", s, k_scatter<<<Ci, kBlock, 0, s>>>(ch_node, ch_start, ch_len, lv.ch_loff, fr_tree, fr_begin,
                                    fr_len, lv.fr_nl, L, n, side, perm_cur, perm_nxt, fo->perm));
    const int nxt = cur ^ 1;
    RPF_LAUNCH("k_frontier", s, k_frontier<<<1, 1024, 0, s>>>(
        Fi, L, fo->n_nodes, fr_tree, fr_begin, fr_len, fr_key, lv.fr_nl, lv.fr_node[nxt],
        lv.fr_tree[nxt], lv.fr_begin[nxt], lv.fr_len[nxt], lv.fr_key[nxt], lv.fr_cb[nxt],
        lv.fr_nc[nxt], lv.ch_node[nxt], lv.ch_start[nxt], lv.ch_len[nxt], fo->n_leaves,
        fo->leaf_tree, fo->leaf_begin, fo->leaf_len, d_cnt));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt, d_cnt, sizeof(Counts), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      err = rpf_cuda_err(e);
      break;
    }
    fo->n_nodes += 2 * F;
    fo->n_leaves += h_cnt->n_leaves_new;
    F = h_cnt->f_next;
    C = h_cnt->c_next;
    std::swap(perm_cur, perm_nxt);
    cur = nxt;
    ++level;
  }
  if (!err) {
    unsigned long long ex = 0;
    cudaMemcpyAsync(&ex, d_exact, sizeof(ex), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) err = rpf_cuda_err(e);
    fo->n_exact = (int64_t)ex;
    fo->max_depth = level;
  }
  free_level();
  cleanup();
  return err;
#undef RPF_TRY
#undef RPF_TRYCU
}

void rpf_launch_directions(uint64_t seed, int32_t t, const uint64_t* keys_dev, int32_t n_keys,
                           int32_t j, int32_t d, double* out_dev, cudaStream_t s) {
  RPF_LAUNCH("k_dirs_keys", s, k_dirs_keys<<<nblk(n_keys, 64), 64, 0, s>>>(seed, t, keys_dev, n_keys, j, d, out_dev));
}
