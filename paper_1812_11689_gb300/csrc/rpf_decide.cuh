// rpf_decide.cuh -- the per-node decisions of rpTree growth, shared by the
// level-synchronous kernels (big nodes) and the CTA-local subtree kernel.
//
// Exact definitions (what the CPU oracle computes):
//   direction r_j   : Box-Muller N(0, I) from the node's counter words,
//                     normalised in FP64 (Algorithms 1-2, "random direction")
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
//     rad(x) = kappa_d |x - o|_2 + (d + 2) 2^-53 1.02 (|x| + |o|),
//     kappa_d = (d + 4) 2^-24 1.0625
// (fma-chain dot-product bound, rounding of r and of x - o to FP32, and the
// FP64 projections' own bound; Cauchy-Schwarz with |r| <= 1 + d 2^-53).
// Decisions are taken from q' when the bound separates them, else in FP64.
#pragma once

#include "rpf_internal.cuh"

// Box-Muller pair i of the direction for (tree t, node key, try j): FP32
// from the top 24 bits of the words 2i and 2i+1 (u1 in (0, 1], u2 in [0, 1)).
__device__ __forceinline__ void rpf_gauss_pair(uint64_t seed, uint64_t t, uint64_t key, uint64_t j,
                                               int i, float* g0, float* g1) {
  const uint64_t w1 = rpf_word(seed, RPF_TAG_DIR, t, key, j, (uint64_t)(2 * i));
  const uint64_t w2 = rpf_word(seed, RPF_TAG_DIR, t, key, j, (uint64_t)(2 * i + 1));
  const float u1 = __fmul_rn((float)((w1 >> 40) + 1), 0x1p-24f);
  const float u2 = __fmul_rn((float)(w2 >> 40), 0x1p-24f);
  const float rho = __fsqrt_rn(__fmul_rn(-2.0f, rpf_lnf(u1)));
  float c, s;
  rpf_sincos2pif(u2, &c, &s);
  *g0 = __fmul_rn(rho, c);
  *g1 = __fmul_rn(rho, s);
}

// 1 / |g| with |g| = sqrt(sequential fma sum of g_k^2) in FP64; 0 if g = 0
__device__ __forceinline__ double rpf_inv_norm(const double* g, int d) {
  double ss = 0.0;
  for (int k = 0; k < d; ++k) ss = __fma_rn(g[k], g[k], ss);
  const double nrm = __dsqrt_rn(ss);
  return nrm == 0.0 ? 0.0 : __ddiv_rn(1.0, nrm);
}

// Direction r (FP64) for (tree t, node key, try j): r_k = g_k * (1 / |g|);
// the unreachable all-zero draw gives e_0.  One thread.
__device__ __forceinline__ void rpf_gen_direction(uint64_t seed, uint64_t t, uint64_t key, uint64_t j,
                                                  int d, double* r) {
  for (int i = 0; 2 * i < d; ++i) {
    float g0, g1;
    rpf_gauss_pair(seed, t, key, j, i, &g0, &g1);
    r[2 * i] = (double)g0;
    if (2 * i + 1 < d) r[2 * i + 1] = (double)g1;
  }
  const double inv = rpf_inv_norm(r, d);
  if (inv == 0.0) {
    for (int k = 0; k < d; ++k) r[k] = 0.0;
    r[0] = 1.0;
    return;
  }
  for (int k = 0; k < d; ++k) r[k] = __dmul_rn(r[k], inv);
}

// canonical FP64 projection
__device__ __forceinline__ double rpf_p64(const float* x, const double* r, int d) {
  double p = 0.0;
  for (int k = 0; k < d; ++k) p = __fma_rn((double)__ldg(x + k), r[k], p);
  return p;
}

__device__ __forceinline__ float rpf_kappa(int d) { return (float)(d + 4) * 0x1p-24f * 1.0625f; }

// error radius of one point (FP32, rounded up); nn = computed sum of squares
// of fl(x - o), xn / on = upper bounds of |x| and |o|
__device__ __forceinline__ float rpf_point_rad(int d, float nn, float xn, float on) {
  const float nrm = __fmul_ru(__fsqrt_ru(nn), 1.0f + (float)(d + 4) * 0x1p-24f);
  const float e64 = __fmul_ru((float)(d + 2) * 0x1p-53f * 1.02f, __fadd_ru(xn, on));
  return __fmaf_ru(rpf_kappa(d), nrm, e64);
}

// gamma_h for the FP32 statistics: <= 16 sequential terms per thread, a warp
// butterfly (5) and a sequential merge of the 8 warp partials (8)
#define RPF_STAT_DEPTH 30

// Certify Algorithm 2's choice from the FP32 statistics.  Inputs per try j:
// S1 = sum q', S2 = sum q'^2, A = sum |q'| (FP32 accumulated, FP64 across
// chunks), base b_j; node size m and radius rad.  Returns the certified
// winner, or -1 when the bounds do not separate it (exact path).
__device__ __forceinline__ int rpf_certify(int ntry, double m, const double* S1, const double* S2,
                                           const double* A, const double* base, double rad) {
  const double u = 0x1p-24;
  const double gam = RPF_STAT_DEPTH * u / (1.0 - RPF_STAT_DEPTH * u);
  const double sm = sqrt(m);
  int w = -1;
  double vb = -1.0;
  for (int j = 0; j < ntry; ++j) {
    const double V = S2[j] - S1[j] * S1[j] / m;
    if (V > vb) {
      vb = V;
      w = j;
    }
  }
  if (w < 0) return -1;
  double lo_w = 0.0, hi_other = -1.0;
  for (int j = 0; j < ntry; ++j) {
    const double V = S2[j] - S1[j] * S1[j] / m;
    const double Am = A[j] * (1.0 + 2.0 * gam);
    const double EV = 2.0 * (gam * (S2[j] + 2.0 * fabs(S1[j]) * Am / m + gam * Am * Am / m) +
                             1e-14 * fabs(S2[j]));
    const double lip = 2.0 * sm * rad;
    const double e64 = 2.0 * (1e-12 * sqrt(fmax(V, 0.0)) + sm * 1e-13 * (fabs(base[j]) + Am / m + rad));
    if (j == w) {
      lo_w = sqrt(fmax(V - EV, 0.0)) - lip - e64;
    } else {
      const double hi = sqrt(fmax(V + EV, 0.0)) + lip + e64;
      hi_other = fmax(hi_other, hi);
    }
  }
  if (!(lo_w > 0.0) || !(lo_w > hi_other)) return -1;
  return w;
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
