// rpf_select.cuh -- register-resident sorted lists of the smallest keys
// offered, for the leaf tiles' selections.
//
// Top64 keeps the KK smallest 64-bit keys (the exact distance key
// d32 bits << 32 | index, which orders like (d32, index) because d32 >= +0);
// TopU the KK smallest 32-bit keys.  Both insert one key with a branch-free
// min/max network, or a batch with a sorting network and a bitonic merge
// that keeps exactly the same keys in fewer operations.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

__host__ __device__ __forceinline__ uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint32_t umax32(uint32_t a, uint32_t b) { return a < b ? b : a; }
__host__ __device__ __forceinline__ void ucmpx(uint32_t& a, uint32_t& b) {  // a <= b after
  const uint32_t lo = umin32(a, b);
  b = umax32(a, b);
  a = lo;
}
__host__ __device__ __forceinline__ void ucmpx64(unsigned long long& a, unsigned long long& b) {
  const bool sw = b < a;
  const unsigned long long lo = sw ? b : a;
  b = sw ? a : b;
  a = lo;
}
__host__ __device__ constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }

// the exact distance key of (d32, idx)
__device__ __forceinline__ unsigned long long key64(float d32, int idx) {
  return ((unsigned long long)__float_as_uint(d32) << 32) | (unsigned)idx;
}

// Sorted list of the KK smallest 64-bit keys offered (ascending; empty slots
// are all-ones).  Insertion is a branch-free min/max network.
template <int KK>
struct Top64 {
  unsigned long long k[KK];
  __host__ __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < KK; ++q) k[q] = ~0ull;
  }
  __host__ __device__ __forceinline__ void insert(unsigned long long x) {
#pragma unroll
    for (int q = KK - 1; q >= 1; --q) {
      const unsigned long long lo = k[q] < x ? k[q] : x;
      k[q] = k[q - 1] < lo ? lo : k[q - 1];
    }
    k[0] = k[0] < x ? k[0] : x;
  }
  // The same list as four insert() calls: the batch is sorted (five
  // comparators), the elementwise minimum of the list and the reversed batch
  // (the KK smallest of both, rising then falling) is sorted by a bitonic
  // merge over a power of two P >= KK, with P - KK leading zero keys whose
  // comparisons fold away.
  __host__ __device__ __forceinline__ void insert4(unsigned long long (&b)[4]) {
    ucmpx64(b[0], b[1]); ucmpx64(b[2], b[3]);
    ucmpx64(b[0], b[2]); ucmpx64(b[1], b[3]);
    ucmpx64(b[1], b[2]);
    constexpr int P = pow2_at_least(KK);
    unsigned long long s[P];
#pragma unroll
    for (int i = 0; i < P - KK; ++i) s[i] = 0ull;
#pragma unroll
    for (int i = 0; i < KK; ++i) {
      const unsigned long long c = b[KK - 1 - i < 4 ? KK - 1 - i : 0];
      s[P - KK + i] = KK - 1 - i < 4 && c < k[i] ? c : k[i];
    }
#pragma unroll
    for (int st = P / 2; st >= 1; st >>= 1) {
#pragma unroll
      for (int i = 0; i < P; ++i)
        if ((i & st) == 0) ucmpx64(s[i], s[i + st]);
    }
#pragma unroll
    for (int i = 0; i < KK; ++i) k[i] = s[P - KK + i];
  }
  // d32 of the K-th entry: the list is sorted, so it is the smallest key at
  // or after position K - 1 (a reduction keeps the list in registers)
  __device__ __forceinline__ float kth_d32(int K) const {
    unsigned long long m = ~0ull;
#pragma unroll
    for (int q = 0; q < KK; ++q) m = min(m, q >= K - 1 ? k[q] : ~0ull);
    return __uint_as_float((unsigned)(m >> 32));
  }
  // first K entries as (d32 bits, index); empty slots as (+inf, -1)
  __device__ __forceinline__ void store(int K, uint2* out) const {
#pragma unroll
    for (int q = 0; q < KK; ++q)
      if (q < K) {
        const bool e = k[q] == ~0ull;
        out[q] = e ? make_uint2(0x7f800000u, 0xffffffffu)
                   : make_uint2((unsigned)(k[q] >> 32), (unsigned)k[q]);
      }
  }
};

// Sorted list of the KK smallest 32-bit keys offered (branch-free networks).
template <int KK>
struct TopU {
  uint32_t v[KK];
  __host__ __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < KK; ++q) v[q] = 0xffffffffu;
  }
  __host__ __device__ __forceinline__ void insert(uint32_t x) {
#pragma unroll
    for (int q = KK - 1; q >= 1; --q) v[q] = umax32(v[q - 1], umin32(v[q], x));
    v[0] = umin32(v[0], x);
  }
  // The same list as eight insert() calls, in fewer operations: the batch is
  // sorted (a 19-comparator network); the elementwise minimum of the list and
  // the reversed batch holds the KK smallest of both and rises then falls;
  // a bitonic merge sorts it.  The merge runs over a power of two P >= KK
  // with P - KK leading zeros (no key is smaller), whose comparisons fold
  // away.
  __host__ __device__ __forceinline__ void insert8(uint32_t (&b)[8]) {
    ucmpx(b[0], b[2]); ucmpx(b[1], b[3]); ucmpx(b[4], b[6]); ucmpx(b[5], b[7]);
    ucmpx(b[0], b[4]); ucmpx(b[1], b[5]); ucmpx(b[2], b[6]); ucmpx(b[3], b[7]);
    ucmpx(b[0], b[1]); ucmpx(b[2], b[3]); ucmpx(b[4], b[5]); ucmpx(b[6], b[7]);
    ucmpx(b[2], b[4]); ucmpx(b[3], b[5]);
    ucmpx(b[1], b[4]); ucmpx(b[3], b[6]);
    ucmpx(b[1], b[2]); ucmpx(b[3], b[4]); ucmpx(b[5], b[6]);
    constexpr int P = pow2_at_least(KK);
    uint32_t s[P];
#pragma unroll
    for (int i = 0; i < P - KK; ++i) s[i] = 0u;
#pragma unroll
    for (int i = 0; i < KK; ++i)
      s[P - KK + i] = KK - 1 - i < 8 ? umin32(v[i], b[KK - 1 - i < 8 ? KK - 1 - i : 0]) : v[i];
#pragma unroll
    for (int st = P / 2; st >= 1; st >>= 1) {
#pragma unroll
      for (int i = 0; i < P; ++i)
        if ((i & st) == 0) ucmpx(s[i], s[i + st]);
    }
#pragma unroll
    for (int i = 0; i < KK; ++i) v[i] = s[P - KK + i];
  }
  __host__ __device__ __forceinline__ uint32_t kth(int K) const {  // sorted: min over q >= K - 1
    uint32_t r = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < KK; ++q) r = umin32(r, q >= K - 1 ? v[q] : 0xffffffffu);
    return r;
  }
};
