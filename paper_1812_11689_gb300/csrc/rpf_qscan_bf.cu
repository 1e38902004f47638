// rpf_qscan_bf.cu -- chosen form of the query leaf scan (Sec. 2, Algorithm 3
// with Q outside U): for each (query, tree) the K nearest points of the leaf
// the query fell into, read from a BF16 copy of the data with a certified
// exact FP32 re-rank, so that every list equals the plain scan's bit for bit.
//
// The scan is bound by the leaf rows it gathers from HBM.  The BF16 copy
// halves those bytes; only a shortlist of FP32 rows is read again.  One CTA
// of 128 threads per (query, tree), thread j = leaf point j:
//   1. the leaf's BF16 rows are staged in shared memory by bulk copies (rows
//      padded to 16-byte multiples);
//   2. D~_j = fl32 sum_k (q_k - y_jk)^2 with y = bf16(x) (any order: only a
//      bound on its error is used);
//   3. tau = the K-th smallest D~ (register sorts per warp, a merge of the
//      four warps' lists);
//   4. certificate.  With delta_j = 2^-9 |x_j| >= |y_j - x_j| (BF16 rounds
//      to nearest with 8 stored mantissa bits) and gam = (d + 4) 2^-24
//      covering the FP32 sums of D~ and of the canonical key d32,
//        |D~_j - d32_j| <= eps_j = 2 (2 gam A_j + B_j (1 + gam)),
//        A_j = D~_j / (1 - gam) >= |q - y_j|^2,
//        B_j = delta_j (2 sqrt(A_j) + 3 delta_j) >= | |q - y_j|^2 - |q - x_j|^2 |
//      (error terms doubled).  The K points of smallest D~ all have d32 <=
//      U = tau + eps(tau, max_j |x_j|) (eps grows with both arguments), so
//      the K-th smallest d32 is <= U, and a point with D~_j - eps_j > U has
//      d32_j > U: it cannot be among the K nearest.  The others (the
//      shortlist) are re-ranked with the canonical FP32 d32 from their FP32
//      rows (staged with coalesced reads) and sorted as 64-bit keys (d32 bits
//      << 32 | index).
//   5. a shortlist longer than 32 (or any non-finite value) sends the leaf to
//      the exact scan of all its FP32 rows (counted with the all-kNN
//      rescans).
// Every device wait is bounded; on a timeout the CTA writes an empty list,
// records RPF_ETIMEOUT and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rpf_internal.cuh"
#include "rpf_tma.cuh"

namespace {

#define QB_T 128

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__global__ void k_x16(const float* __restrict__ X, int64_t n, int d, int d8, uint16_t* X16) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d8) return;
  const int64_t r = i / d8;
  const int k = (int)(i - r * d8);
  const float v = k < d ? X[r * d + k] : 0.0f;
  X16[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__device__ __forceinline__ unsigned long long warp_sort64(unsigned long long v, int lane) {
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

// the 32 smallest keys of two ascending warp lists, ascending
__device__ __forceinline__ unsigned long long warp_merge64(unsigned long long a,
                                                           unsigned long long b, int lane) {
  unsigned long long v = min(a, __shfl_sync(RPF_FULL, b, 31 - lane));
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const unsigned long long o = __shfl_xor_sync(RPF_FULL, v, j);
    v = (lane & j) == 0 ? min(v, o) : max(v, o);
  }
  return v;
}

// bound of |D~ - d32| for D~ (>= 0) and xn >= |x| (rounded up)
__device__ __forceinline__ float qb_eps(float D, float xn, float gam) {
  const float del = __fmaf_ru(0x1p-9f, xn, 0x1p-100f);
  const float A = __fdiv_ru(D, 1.0f - gam);
  const float B = __fmul_ru(del, __fmaf_ru(2.0f, __fsqrt_ru(A), __fmul_ru(3.0f, del)));
  return __fmul_ru(2.0f, __fmaf_ru(__fmul_ru(2.0f, gam), A, __fmul_ru(B, 1.0f + gam)));
}

// canonical d32 of the FP32 query (shared memory) and an FP32 data row
__device__ __forceinline__ float qb_d32(const float* qv, const float* __restrict__ x, int d) {
  float acc = 0.0f;
  if ((d & 3) == 0) {  // rows are 16-byte aligned: vector loads, same order
    for (int k = 0; k < d; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(x + k));
      float e;
      e = __fsub_rn(qv[k], v.x); acc = __fmaf_rn(e, e, acc);
      e = __fsub_rn(qv[k + 1], v.y); acc = __fmaf_rn(e, e, acc);
      e = __fsub_rn(qv[k + 2], v.z); acc = __fmaf_rn(e, e, acc);
      e = __fsub_rn(qv[k + 3], v.w); acc = __fmaf_rn(e, e, acc);
    }
    return acc;
  }
  for (int k = 0; k < d; ++k) {
    const float e = __fsub_rn(qv[k], __ldg(x + k));
    acc = __fmaf_rn(e, e, acc);
  }
  return acc;
}

__global__ void __launch_bounds__(QB_T) k_qscan_bf(
    const float* __restrict__ Q, int64_t m, int d, int d8, int dp16, int T, int K,
    const int2* qleaf, const int32_t* __restrict__ perm, const float* __restrict__ X,
    const uint16_t* __restrict__ X16, const float* __restrict__ xnorm, int64_t n, uint2* cand,
    int* err, unsigned long long* fallbacks, uint64_t wlim) {
  extern __shared__ __align__(16) unsigned char qb_raw[];
  uint16_t* rows = reinterpret_cast<uint16_t*>(qb_raw);  // QB_T x dp16 BF16
  float* qv = reinterpret_cast<float*>(qb_raw + (size_t)QB_T * dp16 * 2);  // d8 floats
  __shared__ unsigned long long keys[QB_T];
  __shared__ int pid[QB_T];
  __shared__ int slist[QB_T];
  __shared__ float wmax[QB_T / 32];
  __shared__ int wcnt[QB_T / 32];
  __shared__ float s_tau;
  __shared__ __align__(8) uint64_t bar;
  const int64_t g = blockIdx.x;
  const int64_t q = g / T;
  const int t = (int)(g % T);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int2 lf = qleaf[g];  // the leaf's (begin, length) in tree t's permutation
  const int len = lf.y;
  const int32_t* mem = perm + (int64_t)t * n + lf.x;
  uint2* out = cand + ((int64_t)t * m + q) * K;
  float xn = 0.0f;
  if (tid < len) {
    pid[tid] = mem[tid];
    xn = xnorm[pid[tid]];
  }
  for (int k = tid; k < d8; k += QB_T) qv[k] = k < d ? Q[q * d + k] : 0.0f;
  if (tid == 0) {
    rpf_mbar_init(&bar, 1);
    rpf_mbar_arrive_expect_tx(&bar, (uint32_t)len * (uint32_t)d8 * 2u);
  }
  __syncthreads();
  if (tid < len) rpf_bulk_g2s(rows + tid * dp16, X16 + (int64_t)pid[tid] * d8, (uint32_t)d8 * 2u, &bar);
  float xm = xn;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) xm = fmaxf(xm, __shfl_xor_sync(RPF_FULL, xm, off));
  if (lane == 0) wmax[warp] = xm;
  const bool ok = __syncthreads_and(rpf_mbar_wait(&bar, 0, err, wlim)) != 0;
  if (!ok) {  // one more bounded wait for copies in flight, then an empty list
    rpf_mbar_wait(&bar, 0, nullptr, wlim);
    if (tid < K) out[tid] = make_uint2(0x7f800000u, 0xffffffffu);
    return;
  }
  // 2. approximate squared distances from the BF16 rows
  float Dt = INFINITY;
  if (tid < len) {
    const uint16_t* y = rows + tid * dp16;
    float acc = 0.0f;
    for (int k = 0; k < d8; k += 8) {
      const uint4 v = *reinterpret_cast<const uint4*>(y + k);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float y0 = __uint_as_float(w[h] << 16), y1 = __uint_as_float(w[h] & 0xffff0000u);
        const float e0 = __fsub_rn(qv[k + 2 * h], y0), e1 = __fsub_rn(qv[k + 2 * h + 1], y1);
        acc = __fmaf_rn(e0, e0, acc);
        acc = __fmaf_rn(e1, e1, acc);
      }
    }
    Dt = acc;
  }
  // 3. tau: the K-th smallest D~ (keys of D~ bits and the tile position)
  const unsigned long long k64 =
      tid < len && Dt == Dt ? ((unsigned long long)__float_as_uint(Dt) << 32) | (unsigned)tid
                            : ~0ull;
  keys[tid] = warp_sort64(k64, lane);
  const float gam = (float)(d + 4) * 0x1p-24f * 1.01f;
  __syncthreads();
  if (tid < 32) {
    unsigned long long v = keys[tid];
#pragma unroll
    for (int w = 1; w < QB_T / 32; ++w) v = warp_merge64(v, keys[32 * w + tid], tid);
    const unsigned long long kth = __shfl_sync(RPF_FULL, v, K - 1);
    if (tid == 0) {
      float X = 0.0f;
      for (int w = 0; w < QB_T / 32; ++w) X = fmaxf(X, wmax[w]);
      const float tau = __uint_as_float((unsigned)(kth >> 32));
      // fewer than K finite values: every point is on the shortlist
      s_tau = kth == ~0ull ? INFINITY : __fadd_ru(tau, qb_eps(tau, X, gam));
    }
  }
  __syncthreads();
  // 4. the shortlist: D~_j - eps_j <= U
  const float U = s_tau;
  const bool take = tid < len && !(__fsub_rd(Dt, qb_eps(Dt, xn, gam)) > U);
  const unsigned bal = __ballot_sync(RPF_FULL, take);
  if (lane == 0) wcnt[warp] = __popc(bal);
  __syncthreads();
  int base = 0, C = 0;
#pragma unroll
  for (int w = 0; w < QB_T / 32; ++w) {
    if (w < warp) base += wcnt[w];
    C += wcnt[w];
  }
  if (take) slist[base + __popc(bal & ((1u << lane) - 1u))] = tid;
  __syncthreads();
  if (C <= 32 && U < INFINITY) {
    // 5. exact re-rank of the shortlist: its FP32 rows are staged in the
    // (now idle) BF16 row area, one warp per row (coalesced reads), then one
    // lane per point runs the canonical chain from shared memory
    float* fr = reinterpret_cast<float*>(qb_raw);
    const int dpf = ((d + 3) & ~3) + 4;
    for (int c = warp; c < C; c += QB_T / 32) {
      const float* src = X + (int64_t)pid[slist[c]] * d;
      for (int k = lane; k < d; k += 32) fr[c * dpf + k] = __ldg(src + k);
    }
    __syncthreads();
    if (tid < 32) {
      unsigned long long v = ~0ull;
      if (tid < C) {
        const int j = pid[slist[tid]];
        const float* y = fr + tid * dpf;  // row stride an odd number of 16-byte units
        float acc = 0.0f;
        int k = 0;
        if ((d & 3) == 0) {
          for (; k < d; k += 4) {
            const float4 v4 = *reinterpret_cast<const float4*>(y + k);
            const float4 q4 = *reinterpret_cast<const float4*>(qv + k);
            float e;
            e = __fsub_rn(q4.x, v4.x); acc = __fmaf_rn(e, e, acc);
            e = __fsub_rn(q4.y, v4.y); acc = __fmaf_rn(e, e, acc);
            e = __fsub_rn(q4.z, v4.z); acc = __fmaf_rn(e, e, acc);
            e = __fsub_rn(q4.w, v4.w); acc = __fmaf_rn(e, e, acc);
          }
        }
        for (; k < d; ++k) {
          const float e = __fsub_rn(qv[k], y[k]);
          acc = __fmaf_rn(e, e, acc);
        }
        v = ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)j;
      }
      v = warp_sort64(v, tid);
      if (tid < K)
        out[tid] = v == ~0ull ? make_uint2(0x7f800000u, 0xffffffffu)
                              : make_uint2((unsigned)(v >> 32), (unsigned)v);
    }
    return;
  }
  // long shortlist: every point of the leaf, exactly
  unsigned long long v = ~0ull;
  if (tid < len) {
    const int j = pid[tid];
    v = ((unsigned long long)__float_as_uint(qb_d32(qv, X + (int64_t)j * d, d)) << 32) |
        (unsigned)j;
  }
  keys[tid] = warp_sort64(v, lane);
  __syncthreads();
  if (tid < 32) {
    unsigned long long u = keys[tid];
#pragma unroll
    for (int w = 1; w < QB_T / 32; ++w) u = warp_merge64(u, keys[32 * w + tid], tid);
    if (tid < K)
      out[tid] = u == ~0ull ? make_uint2(0x7f800000u, 0xffffffffu)
                            : make_uint2((unsigned)(u >> 32), (unsigned)u);
    if (tid == 0) atomicAdd(fallbacks, 1ULL);
  }
}

}  // namespace

int rpf_build_x16(rpf_forest* f, cudaStream_t s) {
  rpf_release(f->X16, s);
  f->X16 = nullptr;
  f->d8 = (f->d + 7) & ~7;
  const int64_t N = f->n * f->d8;
  if (rpf_alloc((void**)&f->X16, 2 * (size_t)N, s)) return RPF_ENOMEM;
  RPF_LAUNCH("k_x16", s, k_x16<<<nblk(N, 256), 256, 0, s>>>(f->X, f->n, f->d, f->d8, f->X16));
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

bool rpf_qscan_bf_ok(const rpf_forest* f, int K) {
  if (!f->X16 || K > 32 || f->prm.leaf_max > QB_T) return false;
  const int dp16 = ((f->d8 * 2 / 16) & 1) ? f->d8 : f->d8 + 8;
  return (size_t)QB_T * dp16 * 2 + (size_t)f->d8 * 4 <= 200 * 1024;
}

int rpf_qscan_bf(const rpf_forest* f, const float* Q, int64_t m, int K, const int2* qleaf,
                 uint2* cand, int* err, cudaStream_t s) {
  const int T = f->prm.n_trees, d8 = f->d8;
  // row stride: an odd number of 16-byte units, so 16-byte row reads of
  // consecutive threads fall in distinct banks
  const int dp16 = ((d8 * 2 / 16) & 1) ? d8 : d8 + 8;
  const size_t smem = (size_t)QB_T * dp16 * 2 + (size_t)d8 * 4;
  RPF_CU(cudaFuncSetAttribute(k_qscan_bf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  RPF_LAUNCH("k_qscan_bf", s, k_qscan_bf<<<(unsigned)(m * T), QB_T, smem, s>>>(
      Q, m, f->d, d8, dp16, T, K, qleaf, f->perm, f->X,
      f->X16, f->xnorm, f->n, cand, err, f->d_fallback, rpf_wait_limit_ns()));
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}
