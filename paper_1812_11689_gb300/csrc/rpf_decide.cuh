// rpf_decide.cuh -- the per-node decisions of rpTree growth, shared by the
// level-synchronous kernels (big nodes) and the CTA-local subtree kernel.
//
// Exact definitions (what the CPU oracle computes):
//   direction r_j   : Box-Muller N(0, I) from the node's counter words,
//                     normalised, all in FP32 (Algorithms 1-2, "random
//                     direction"); r is an FP32 vector
//   projection      : p64(x, r) = fold_k fma((double)x_k, r_k, p) from +0.0
//   dispersion V_j  : canonical-order FP64 sum of (p - mu)^2, mu = S / m
//   choice          : first j with V_j > best, best starting at 0 (Alg. 2)
//   split point     : c = fma(u, b - a, a), a / b = min / max of p64_{j*},
//                     accepted iff a < c <= b, 8 attempts, else rank split
//   sides           : left iff p64_{j*}(x) < c (Alg. 1)
//
// Fast path (FP32, certified): for o = the node's first member,
//   q'_j(x) = fl32-dot(r32_j, fl32(x - o)),   b_j = p64(o, r_j),
//   |q'_j(x) - (p64_j(x) - b_j)| <= rad(x)
//     rad(x) = kappa_d |x - o|_2 + (d + 40) 2^-53 1.02 (|x| + |o|),
//     kappa_d = (d + 4) 2^-24 1.0625
// (fma-chain dot-product bound, rounding of x - o to FP32, and the
// FP64 projections' own bound -- b_j may be summed in any order of depth
// <= d + 38; Cauchy-Schwarz with |r| <= 1 + d 2^-53).
// Decisions are taken from q' when the bound separates them, else in FP64.
#pragma once

#include "rpf_internal.cuh"

// Box-Muller pair i of the direction for (tree t, node key, try j): FP32
// from the top 24 bits of the words 2i and 2i+1 (u1 in (0, 1], u2 in [0, 1)).
// h = rpf_word_prefix(seed, RPF_TAG_DIR, t, key, j), shared by all pairs of
// one (node, try).
__device__ __forceinline__ void rpf_gauss_pair_h(uint64_t h, int i, float* g0, float* g1) {
  const uint64_t w1 = rpf_word_last(h, (uint64_t)(2 * i));
  const uint64_t w2 = rpf_word_last(h, (uint64_t)(2 * i + 1));
  const float u1 = __fmul_rn((float)((w1 >> 40) + 1), 0x1p-24f);
  const float u2 = __fmul_rn((float)(w2 >> 40), 0x1p-24f);
  const float rho = __fsqrt_rn(__fmul_rn(-2.0f, rpf_lnf(u1)));
  float c, s;
  rpf_sincos2pif(u2, &c, &s);
  *g0 = __fmul_rn(rho, c);
  *g1 = __fmul_rn(rho, s);
}
__device__ __forceinline__ void rpf_gauss_pair(uint64_t seed, uint64_t t, uint64_t key, uint64_t j,
                                               int i, float* g0, float* g1) {
  rpf_gauss_pair_h(rpf_word_prefix(seed, RPF_TAG_DIR, t, key, j), i, g0, g1);
}

// 1 / |g| in FP32: |g| = sqrtf(sequential fmaf sum of g_k^2); 0 if g = 0
__device__ __forceinline__ float rpf_inv_norm32(const float* g, int d) {
  float ss = 0.0f;
#pragma unroll 8
  for (int k = 0; k < d; ++k) ss = __fmaf_rn(g[k], g[k], ss);
  return ss == 0.0f ? 0.0f : __fdiv_rn(1.0f, __fsqrt_rn(ss));
}

// Direction r for (tree t, node key, try j), all in FP32: r_k = g_k * (1/|g|);
// the unreachable all-zero draw gives e_0.  One thread; g is scratch for d
// floats; r receives the FP32 values widened to FP64.
__device__ __forceinline__ void rpf_gen_direction(uint64_t seed, uint64_t t, uint64_t key, uint64_t j,
                                                  int d, float* g, double* r) {
  for (int i = 0; 2 * i < d; ++i) {
    float g0, g1;
    rpf_gauss_pair(seed, t, key, j, i, &g0, &g1);
    g[2 * i] = g0;
    if (2 * i + 1 < d) g[2 * i + 1] = g1;
  }
  const float inv = rpf_inv_norm32(g, d);
  for (int k = 0; k < d; ++k) r[k] = inv == 0.0f ? (k == 0 ? 1.0 : 0.0) : (double)__fmul_rn(g[k], inv);
}

// canonical FP64 projection
__device__ __forceinline__ double rpf_p64(const float* x, const double* r, int d) {
  double p = 0.0;
  for (int k = 0; k < d; ++k) p = __fma_rn((double)__ldg(x + k), r[k], p);
  return p;
}
// the same from the FP32 direction values (widened exactly)
__device__ __forceinline__ double rpf_p64f(const float* x, const float* r, int d) {
  double p = 0.0;
  for (int k = 0; k < d; ++k) p = __fma_rn((double)__ldg(x + k), (double)__ldg(r + k), p);
  return p;
}

// Warp-collective canonical FP64 projections of two rows x0, x1 on r; lane 0
// returns p64(x0, r), lane 1 p64(x1, r).  With x_k and r_k FP32 values the
// product x_k r_k has at most 48 significant bits and is exact in FP64, so
// each step fma(x_k, r_k, p) equals p + (x_k r_k) rounded once: the warp forms
// the products 32 coordinates at a time (coalesced loads) and lanes 0 / 1 add
// them in order, taking each from the lane that holds it.  The chain then waits
// only for its additions, not for loads.
__device__ __forceinline__ double rpf_p64_pair(const float* x0, const float* x1, const double* r,
                                               int d, int lane) {
  double p = 0.0;
  for (int k0 = 0; k0 < d; k0 += 32) {
    const int k = k0 + lane;
    double t0 = 0.0, t1 = 0.0;
    if (k < d) {
      const double rk = r[k];
      t0 = __dmul_rn((double)__ldg(x0 + k), rk);
      t1 = __dmul_rn((double)__ldg(x1 + k), rk);
    }
    const int kn = min(32, d - k0);
    for (int u = 0; u < kn; ++u) {
      const double v0 = __shfl_sync(RPF_FULL, t0, u);
      const double v1 = __shfl_sync(RPF_FULL, t1, u);
      p = __dadd_rn(p, lane == 0 ? v0 : v1);
    }
  }
  return p;
}

__device__ __forceinline__ float rpf_kappa(int d) { return (float)(d + 4) * 0x1p-24f * 1.0625f; }

// error radius of one point (FP32, rounded up); nn = computed sum of squares
// of fl(x - o), xn / on = upper bounds of |x| and |o|
__device__ __forceinline__ float rpf_point_rad(int d, float nn, float xn, float on) {
  const float nrm = __fmul_ru(__fsqrt_ru(nn), 1.0f + (float)(d + 4) * 0x1p-24f);
  const float e64 = __fmul_ru((float)(d + 40) * 0x1p-53f * 1.02f, __fadd_ru(xn, on));
  return __fmaf_ru(rpf_kappa(d), nrm, e64);
}

// gamma_h for the FP32 statistics: at most 32 sequential terms per thread,
// a warp butterfly (5) and an FP32 merge of at most 8 warp partials.
#define RPF_STAT_DEPTH 45

// Bounds of sqrt(V_j) (the canonical FP64 dispersion of Algorithm 2) from the
// FP32 statistics of try j: S1 = sum q', S2 = sum q'^2, A = sum |q'|
// (<= RPF_STAT_DEPTH roundings on any path), node size m, radius rad, and
// babs >= |b_j| (|o| bounds it).  With Vhat = S2 - S1^2 / m:
//   |Vhat - V_q| <= EV   (FP32 sums: gamma (S2 + 2|S1| A / m + gamma A^2 / m),
//                         plus 1e-14 S2 for the FP64 arithmetic here)
//   |sqrt(V_q) - sqrt(V_p)| <= |q - p|_2 <= min(sqrt(m) rad, l2)
//                         (sqrt of a centred sum of squares is 1-Lipschitz in
//                         the vector of projections; l2 >= sqrt(sum rad_i^2))
//   |sqrt(V) - sqrt(V_p)| <= 1e-12 sqrt(V) + sqrt(m) 1e-13 (|b| + A/m + rad)
//                         (the canonical FP64 reduction itself)
// all error terms doubled.  lo / hi are rounded outwards in FP32.
__device__ __forceinline__ void rpf_try_bounds(int m, double inv_m, double S1, double S2,
                                               double A, double babs, float rad, float l2,
                                               double* vhat, float* lo, float* hi) {
  const double u = 0x1p-24;
  const double gam = RPF_STAT_DEPTH * u / (1.0 - RPF_STAT_DEPTH * u);
  const double V = S2 - S1 * (S1 * inv_m);
  const double Am = A * (1.0 + 2.0 * gam);
  const double EV =
      2.0 * (gam * (S2 + 2.0 * fabs(S1) * Am * inv_m + gam * Am * Am * inv_m) + 1e-14 * fabs(S2)) +
      0x1p-50 * S1 * S1 * inv_m;
  const float sqm = __fsqrt_ru(__int2float_ru(m));
  const float vup = __fsqrt_ru(__double2float_ru(fmax(V + EV, 0.0)));
  const float lip = __fmul_ru(2.0f, fminf(__fmul_ru(sqm, rad), l2));
  const float mid = __fadd_ru(__double2float_ru(fabs(babs) + Am * inv_m), rad);
  const float e64 = __fmul_ru(2.0f, __fadd_ru(__fmul_ru(1e-12f, vup), __fmul_ru(__fmul_ru(sqm, 1e-13f), mid)));
  const float err = __fadd_ru(lip, e64);
  *vhat = V;
  *hi = __fadd_ru(vup, err);
  *lo = __fsub_rd(__fsqrt_rd(__double2float_rd(fmax(V - EV, 0.0))), err);
}

// Certified winner of Algorithm 2 from per-try bounds: the first argmax w of
// Vhat, accepted iff lo_w > 0 and lo_w > hi_k for every k != w (then V_w is
// the unique maximum and positive, so Algorithm 2 picks w); else -1.
__device__ __forceinline__ int rpf_certify_select(int ntry, const double* vhat, const float* lo,
                                                  const float* hi) {
  int w = -1;
  double vb = -1.0;
  for (int j = 0; j < ntry; ++j)
    if (vhat[j] > vb) {
      vb = vhat[j];
      w = j;
    }
  if (w < 0 || !(lo[w] > 0.0f)) return -1;
  for (int j = 0; j < ntry; ++j)
    if (j != w && !(lo[w] > hi[j])) return -1;
  return w;
}

// The tries that can still be Algorithm 2's choice when the certificate
// fails: those whose upper bound reaches the largest lower bound L (any
// other try has sqrt(V) <= hi < L <= sqrt(V) of the try holding L, so it is
// neither the maximum nor tied with it).  Every try if a bound is NaN.
__device__ __forceinline__ unsigned long long rpf_contenders(int ntry, const float* lo,
                                                             const float* hi) {
  const unsigned long long all = ntry >= 64 ? ~0ull : (1ull << ntry) - 1ull;
  float L = -INFINITY;
  for (int j = 0; j < ntry; ++j) {
    if (lo[j] != lo[j] || hi[j] != hi[j]) return all;
    L = fmaxf(L, lo[j]);
  }
  unsigned long long mask = 0ull;
  for (int j = 0; j < ntry; ++j)
    if (hi[j] >= L) mask |= 1ull << j;
  return mask;
}

// Split point of Algorithm 1 from the exact a = min, b = max.  Returns 1 if
// an attempt was accepted (c in (a, b]), 0 for a rank split.
__device__ __forceinline__ int rpf_split_point(uint64_t seed, uint64_t t, uint64_t key, double a,
                                               double b, double* c_out) {
  for (int att = 0; att < RPF_SPLIT_ATTEMPTS; ++att) {
    const double u = rpf_u53(rpf_word(seed, RPF_TAG_SPLIT, t, key, (uint64_t)att, 0));
    const double c = __fma_rn(u, __dsub_rn(b, a), a);
    if (c > a && c <= b) {
      *c_out = c;
      return 1;
    }
  }
  *c_out = NAN;
  return 0;
}

// Certified side thresholds on q' for split point c, base b, radius rad:
// q' < tl  =>  p64 < c;   q' >= tr  =>  p64 >= c   (directed roundings)
__device__ __forceinline__ void rpf_side_thresholds(double c, double base, double rad, float* tl,
                                                    float* tr) {
  *tl = __double2float_rd(__dsub_rd(__dsub_rd(c, base), rad));
  *tr = __double2float_ru(__dadd_ru(__dsub_ru(c, base), rad));
}

// Median rule: order-preserving key of p64 (+0.0 for -0.0, so that equal
// projections get equal keys)
__device__ __forceinline__ unsigned long long rpf_mkey(double p) {
  return rpf_dkey(__dadd_rn(p, 0.0));
}

// Median rule: digit of radix pass `pass` (8 passes over the 64-bit order-
// preserving key of p64, then 4 over the point index among equal keys) and
// whether the point matches the prefix selected so far.
__device__ __forceinline__ bool rpf_med_digit(int pass, unsigned long long key, uint32_t id,
                                              unsigned long long pk, uint32_t pid, int* dig) {
  if (pass < 8) {
    const int sh = 56 - 8 * pass;
    *dig = (int)((key >> sh) & 255ull);
    return pass == 0 || ((key ^ pk) >> (sh + 8)) == 0ull;
  }
  const int sh = 24 - 8 * (pass - 8);
  *dig = (int)((id >> sh) & 255u);
  return key == pk && (pass == 8 || ((id ^ pid) >> (sh + 8)) == 0u);
}

// Median rule, FP32 stage: order-preserving key of a float, its inverse,
// and the band around the FP32 median (directed roundings).
__device__ __forceinline__ uint32_t rpf_fkey(float v) {  // order-preserving float key
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float rpf_fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
// the band of a certified node around v32 (directed roundings)
__device__ __forceinline__ void rpf_med_band(uint32_t fk, float rad, float* lo, float* hi) {
  const float v = rpf_fkey_inv(fk), r2 = __fmul_ru(2.0f, rad);
  *lo = __fsub_rd(v, r2);
  *hi = __fadd_ru(v, r2);
}

// Warp-collective: the digit of a 256-bin histogram that holds `rank` (lane l
// looks at bins 8 l .. 8 l + 7); the lane that finds it returns true with the
// digit and the rank left inside its bin.
__device__ __forceinline__ bool rpf_pick_digit(const int* hist, int lane, int rank, int* dig_out,
                                               int* rest_out) {
  int v[8], sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    v[q] = hist[8 * lane + q];
    sum += v[q];
  }
  int x = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(RPF_FULL, x, off);
    if (lane >= off) x += y;
  }
  const int pre = x - sum;
  if (!(rank >= pre && rank < pre + sum)) return false;
  int cum = pre, dig = -1;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (dig < 0) {
      if (rank < cum + v[q]) dig = 8 * lane + q;
      else cum += v[q];
    }
  }
  *dig_out = dig;
  *rest_out = rank - cum;
  return true;
}
