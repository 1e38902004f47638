// rpf_leaf_tc.cu -- chosen form of the leaf distances of Algorithm 3 (Sec. 2):
// the K nearest points of every point inside each of its leaves, with the
// inner products on the 5th-generation tensor cores and a certified exact
// FP32 re-rank, so that every list is bit-identical to the plain form's.
//
// Work layout.  The leaves of one tree are contiguous segments of the tree's
// permutation.  k_pack_tiles packs runs of consecutive leaves greedily into
// tiles of at most 128 rows (a leaf never straddles two tiles); k_leaf_tc is a
// persistent kernel whose CTAs take tiles in turn.  Per tile (128 threads,
// thread r = row r):
//   1. rows are staged in shared memory by bulk copies (TMA engine, mbarrier)
//      when a row is a 16-byte multiple (d % 4 == 0), else by warp loads;
//      leaf boundaries come from a per-tree bitmask of leaf starts.
//   2. Leaves of fewer than TC_BIG_MIN points, or of at most K + 1 ("small"),
//      need no arithmetic shortcut: every row offers all of its leaf to the
//      exact re-rank.
//   3. Rows of larger leaves are centred on their leaf's FP32 mean (y = x - c)
//      and split into BF16 pairs y ~ hi + lo; G = hi hi^T + hi lo^T + lo hi^T
//      is accumulated by tcgen05.mma (kind::f16, M = 128, N = rows padded to
//      16, FP32 in TMEM) over chunks of at most 128 coordinates.
//   4. Row r reads its Gram row from TMEM (tcgen05.ld) and keeps the K + 2
//      smallest keys of the approximate squared distances
//      D~_rj = n_r + n_j - 2 G_rj (n = FP32 squared norm of y) with their
//      columns (a branch-free min/max network); tau, an upper bound of the
//      K-th smallest D~, comes from the K-th key, and every j with
//      D~_rj <= tau' (a certified margin above tau) from the kept keys, or
//      from a second pass over the row when the kept keys may not hold
//      them all.
//   5. The collected candidates are re-ranked with the canonical FP32 d32
//      (the plain form's exact key) into a sorted list of 64-bit keys
//      (d32 bits << 32 | index), which orders exactly like (d32, index).
//   6. Certificate.  Every j that was not collected has D~_rj > tau', and
//        | D~_rj - |y_r - y_j|^2 | <= eps_r = ce (n_r + N_leaf)
//        | |y_r - y_j| - |x_r - x_j| | <= eta_r = 2^-23 (|y_r| + Y_leaf)
//        sqrt(d32_rj) >= (1 - (d + 3) 2^-23) |x_r - x_j|
//      (ce: 2^-13 for the split-BF16 residual, 2^-16 |y_k| per element, and
//      the dropped lo lo^T term, doubled in D~, with room for underflow;
//      (d + 8) 2^-23 for the FP32 norms and combination; 3 (d16 + 4) 2^-21
//      for the tensor core's FP32 accumulation of 3 d16 products, taken at
//      2^-22 per addition so that truncating internal adds are covered,
//      doubled in D~).  So no excluded j can enter the top-K if
//        sqrt_ru(d32 of the K-th collected) < (1 - (d + 3) 2^-23)
//                                             (sqrt_rd(tau' - eps_r) - eta_r).
//      tau' = eps_r + (sqrt(tau + eps_r)(1 + 4 (d + 3) 2^-23) + 2 eta_r)^2
//      makes this hold whenever the bounds are not loose.  A row that fails
//      the certificate, or collects more than TC_SLOTS candidates, is
//      rescanned exactly (counted in *fallbacks).  The tensor path is used
//      only when 2^-90 <= max |y|^2 <= 2^120 in the leaf (every D~ finite,
//      BF16 subnormals negligible); other leaves are scanned exactly.
// Every device wait is bounded; on a timeout the kernel records RPF_ETIMEOUT,
// waits once more (bounded) for copies and MMAs in flight, frees its TMEM and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rpf_internal.cuh"
#include "rpf_scan.cuh"
#include "rpf_select.cuh"
#include "rpf_tma.cuh"
#include "rpf_umma.cuh"

#define TC_SLOTS 32       // exact re-rank candidates per row
#define TC_SLOT_STRIDE 36 // bytes per row's slots: rows 9 words apart, so a warp's
                          // slot accesses fall in distinct banks
#define TC_SEG 4096       // packing segment (positions) per thread
#define TC_SEG_TILES 72   // >= 2 (TC_SEG + 128) / 128 + 1 tiles per segment
#define TC_BIG_MIN 12     // leaves of at least this many points take the tensor path
static_assert(TC_BIG_MIN >= 2 && TC_BIG_MIN <= TC_SLOTS + 2, "a small leaf fits the slots");

namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// D~ = (n_r + n_c) - 2 G_rc for the eight columns c0 .. c0 + 7 (c0 a multiple
// of 8; nrm has room for them), in packed pair instructions
__device__ __forceinline__ void tc_dist8(const float (&g)[8], float nr, const float* nrm, int c0,
                                         float (&D)[8]) {
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const float2 nc = *reinterpret_cast<const float2*>(nrm + c0 + j);
    const float2 s = rpf_add2(make_float2(nr, nr), nc);
    const float2 v = rpf_fma2(make_float2(-2.0f, -2.0f), make_float2(g[j], g[j + 1]), s);
    D[j] = v.x;
    D[j + 1] = v.y;
  }
}

// Sorted list of the KK smallest floats offered (branch-free network).
template <int KK>
struct TopF {
  float v[KK];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < KK; ++q) v[q] = INFINITY;
  }
  __device__ __forceinline__ void insert(float x) {
#pragma unroll
    for (int q = KK - 1; q >= 1; --q) v[q] = fmaxf(v[q - 1], fminf(v[q], x));
    v[0] = fminf(v[0], x);
  }
  __device__ __forceinline__ float kth(int K) const {  // sorted: min over q >= K - 1
    float r = INFINITY;
#pragma unroll
    for (int q = 0; q < KK; ++q) r = fminf(r, q >= K - 1 ? v[q] : INFINITY);
    return r;
  }
};


// Exact d32 of tile row r against up to four tile rows c[0..3] (canonical
// chains over k in order; rows padded with zeros to d4).
__device__ __forceinline__ void d32x4(const float* xs, int dp, int d4, int r, const int (&c)[4],
                                      float (&acc)[4]) {
  const float* x = xs + r * dp;
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j] = 0.0f;
  for (int k = 0; k < d4; k += 4) {
    const float4 a = *reinterpret_cast<const float4*>(x + k);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // the differences in packed pairs (each lane rounds like __fsub_rn);
      // the squares still go into one chain in coordinate order
      const float4 v = *reinterpret_cast<const float4*>(xs + c[j] * dp + k);
      const float2 e01 = rpf_sub2(make_float2(a.x, a.y), make_float2(v.x, v.y));
      const float2 e23 = rpf_sub2(make_float2(a.z, a.w), make_float2(v.z, v.w));
      acc[j] = __fmaf_rn(e01.x, e01.x, acc[j]);
      acc[j] = __fmaf_rn(e01.y, e01.y, acc[j]);
      acc[j] = __fmaf_rn(e23.x, e23.x, acc[j]);
      acc[j] = __fmaf_rn(e23.y, e23.y, acc[j]);
    }
  }
}

// ---------------------------------------------------------------------------
// Packing
// ---------------------------------------------------------------------------
__global__ void k_leaf_bits(int64_t nl, const int32_t* leaf_tree, const int32_t* leaf_begin,
                            int64_t nwords, uint32_t* bits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl) return;
  const int b = leaf_begin[i];
  atomicOr(bits + (int64_t)leaf_tree[i] * nwords + (b >> 5), 1u << (b & 31));
}

// smallest leaf start >= p in one tree's bitmask, or n
__device__ int64_t next_start(const uint32_t* b, int64_t n, int64_t p) {
  if (p >= n) return n;
  int64_t w = p >> 5;
  uint32_t x = b[w] & (0xffffffffu << (p & 31));
  const int64_t nw = (n + 31) >> 5;
  while (x == 0) {
    if (++w >= nw) return n;
    x = b[w];
  }
  const int64_t s = (w << 5) + __ffs(x) - 1;
  return s < n ? s : n;
}

// largest leaf start in (p, lim], or -1 (lim < n)
__device__ int64_t last_start_le(const uint32_t* b, int64_t p, int64_t lim) {
  int64_t w = lim >> 5;
  uint32_t x = b[w] & (0xffffffffu >> (31 - (lim & 31)));
  const int64_t w0 = (p + 1) >> 5;
  while (true) {
    if (w == w0) x &= 0xffffffffu << ((p + 1) & 31);
    if (x) break;
    if (--w < w0) return -1;
    x = b[w];
  }
  return (w << 5) + 31 - __clz(x);
}

// One thread per (tree, segment of TC_SEG positions): the leaves that begin
// in the segment, packed greedily in order into tiles of <= cap rows.
__global__ void k_pack_tiles(int T, int64_t n, int64_t nseg, int64_t nwords, const uint32_t* bits,
                             int cap, int2* slot, int32_t* cnt) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)T * nseg) return;
  const int t = (int)(g / nseg);
  const int64_t sg = g % nseg;
  const uint32_t* b = bits + (int64_t)t * nwords;
  const int64_t s0 = sg * TC_SEG, s1 = std::min<int64_t>(n, s0 + TC_SEG);
  int64_t p = next_start(b, n, s0);
  int c = 0;
  if (p < s1) {
    const int64_t E = next_start(b, n, s1);  // end of the segment's last leaf
    while (p < E) {
      const int64_t lim = std::min<int64_t>(p + cap, E);
      int64_t e = lim == n ? n : -1;
      if (e < 0) {
        e = last_start_le(b, p, lim);
        if (e < 0) e = lim;  // cannot happen: the leaf at p ends by p + L
      }
      if (c < TC_SEG_TILES) slot[g * TC_SEG_TILES + c] = make_int2((int)p, (int)(e - p));
      ++c;
      p = e;
    }
  }
  cnt[g] = c;
}

__global__ void k_pack_fill(int64_t G, int64_t nseg, const int2* slot, const int32_t* cnt,
                            const int32_t* off, int4* tiles) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int t = (int)(g / nseg);
  const int c = min(cnt[g], TC_SEG_TILES);
  for (int j = 0; j < c; ++j) {
    const int2 s = slot[g * TC_SEG_TILES + j];
    tiles[off[g] + j] = make_int4(t, s.x, s.y, 0);
  }
}

// ---------------------------------------------------------------------------
// The persistent chosen-form kernel
// ---------------------------------------------------------------------------
// ROWS = 128: one M = 128 accumulator of N <= 128 columns (128 TMEM columns,
// up to four CTAs per SM).  ROWS = 256 (leaves of up to 256 points): two
// M = 128 blocks (rows 0-127 and 128-255) against all N <= 256 rows, the
// block-b accumulator at TMEM column 256 b (512 columns, one CTA per SM);
// warp w reads lane quarter w % 4 of block w / 4.
template <int KK, int ROWS>
__global__ void __launch_bounds__(ROWS, ROWS == 128 ? 4 : 1) k_leaf_tc(
    const int4* __restrict__ tiles, int64_t tlo, int64_t thi, const uint32_t* __restrict__ bits,
    int64_t nwords, const int32_t* __restrict__ perm, const float* __restrict__ X, int64_t n,
    int d, int dp, int d16, int KC, int K, int t0, uint2* cand, int* err,
    unsigned long long* fallbacks, uint64_t wlim) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  constexpr int RG = ROWS / 8;                  // 8-row groups of the BF16 tiles
  constexpr uint32_t TCOLS = ROWS == 128 ? 128u : 512u;
  const int d4 = (d + 3) & ~3;
  float* xs = reinterpret_cast<float*>(smraw);
  const size_t a_off = (((size_t)ROWS * dp * 4) + 1023) & ~(size_t)1023;
  __nv_bfloat16* Ahi = reinterpret_cast<__nv_bfloat16*>(smraw + a_off);
  __nv_bfloat16* Alo = Ahi + ROWS * KC;
  constexpr int MAXBIG = ROWS / TC_BIG_MIN + 1;  // large leaves in one tile
  float* cen = reinterpret_cast<float*>(Alo + ROWS * KC);  // MAXBIG x d4
  unsigned char* slots = reinterpret_cast<unsigned char*>(cen + MAXBIG * d4);
  __shared__ __align__(16) float nrm[ROWS];
  __shared__ float ynm[ROWS];
  __shared__ int prow_s[ROWS], big_of_start[ROWS];
  __shared__ uint32_t wmask[ROWS / 32];
  __shared__ unsigned nmax_bits[MAXBIG];
  __shared__ int big_lb[MAXBIG], big_le[MAXBIG], nbig;
  __shared__ __align__(8) uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    rpf_mbar_init(&bar_tma, 1);
    rpf_mbar_init(&bar_mma, 1);
  }
  if (warp == 0) rpf_tmem_alloc(&tmem_base, TCOLS);
  rpf_tc_fence_before();
  __syncthreads();
  rpf_tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t tlane =
      tbase + (uint32_t)(256 * (warp >> 2)) + ((uint32_t)(32 * (warp & 3)) << 16);
  const float ce = 0x1p-13f + (float)(d + 8) * 0x1p-23f + 3.0f * (float)(d16 + 4) * 0x1p-21f;
  const float gam = (float)(d + 3) * 0x1p-23f;
  uint32_t tma_phase = 0, mma_phase = 0;
  bool ok = true, tma_pending = false, mma_pending = false;
  const int r = tid;

  // a tile's row ids and leaf-start bits, read one tile ahead
  auto fetch_rows = [&](const int4& tv, int& prow, bool& st) {
    prow = 0;
    st = false;
    if (r < tv.z) {
      const int64_t p = (int64_t)tv.y + r;
      prow = perm[(int64_t)tv.x * n + p];
      st = (bits[(int64_t)tv.x * nwords + (p >> 5)] >> (p & 31)) & 1u;
    }
  };
  int64_t tile = tlo + blockIdx.x;
  int4 tl_c = make_int4(0, 0, 0, 0);
  int prow_c = 0;
  bool start_c = false;
  if (tile < thi) {
    tl_c = tiles[tile];
    fetch_rows(tl_c, prow_c, start_c);
  }
  for (; tile < thi && ok; tile += gridDim.x) {
    const int4 tl = tl_c;
    const int t = tl.x, rows = tl.z;
    // (1) rows, leaf starts, staging
    const bool start = start_c;
    if (r < rows) prow_s[r] = prow_c;
    if (tile + gridDim.x < thi) tl_c = tiles[tile + gridDim.x];  // its rows: before (5)
    const uint32_t bal = __ballot_sync(RPF_FULL, start);
    if (lane == 0) wmask[warp] = bal;
    // rows of 16-byte multiples go by bulk copy (TMA engine); other rows are
    // not 16-byte aligned in X, so the warps load them (the barrier's phase
    // then completes on thread 0's arrival alone)
    const bool bulk = (d & 3) == 0;
    if (tid == 0) {
      nbig = 0;
      rpf_mbar_arrive_expect_tx(&bar_tma, bulk ? (uint32_t)rows * (uint32_t)d * 4u : 0u);
    }
    if (tid < MAXBIG) nmax_bits[tid] = 0u;
    __syncthreads();
    if (bulk) {
      for (int q = tid; q < rows; q += ROWS)
        rpf_bulk_g2s(xs + q * dp, X + (int64_t)prow_s[q] * d, (uint32_t)d * 4u, &bar_tma);
      for (int k = d; k < dp; ++k) xs[r * dp + k] = 0.0f;
    } else {
      for (int q = warp; q < rows; q += ROWS / 32) {
        const float* src = X + (int64_t)prow_s[q] * d;
        for (int k = lane; k < dp; k += 32) xs[q * dp + k] = k < d ? src[k] : 0.0f;
      }
    }
    tma_pending = bulk;
    // leaf [lb, le) of row r (tile-relative)
    int lb = 0, le = rows;
    if (r < rows) {
      const int w = r >> 5, b = r & 31;
      uint32_t x = wmask[w] & (0xffffffffu >> (31 - b));
      int ww = w;
      while (x == 0 && ww > 0) x = wmask[--ww];
      lb = x ? (ww << 5) + 31 - __clz(x) : 0;
      x = b == 31 ? 0u : (wmask[w] & (0xffffffffu << (b + 1)));
      ww = w;
      while (x == 0 && ww < ROWS / 32 - 1) x = wmask[++ww];
      le = x ? min((ww << 5) + __ffs(x) - 1, rows) : rows;
    }
    const int m = le - lb;
    const bool live = r < rows;
    const bool big = live && m >= TC_BIG_MIN && m - 1 > K;
    if (big && r == lb) {
      const int sidx = atomicAdd(&nbig, 1);  // at most ROWS / TC_BIG_MIN large leaves
      big_of_start[r] = sidx;
      big_lb[sidx] = lb;
      big_le[sidx] = le;
    }
    {
      const bool w = rpf_mbar_wait(&bar_tma, tma_phase, err, wlim);
      tma_phase ^= 1u;
      tma_pending = false;
      ok = __syncthreads_and(w) != 0;
      if (!ok) break;
    }
    const int nb = nbig;
    const int bslot = big ? big_of_start[lb] : -1;
    bool cert_ok = true;  // the leaf is in the tensor path's certified range
    if (nb > 0) {
      // (2) FP32 mean of every large leaf: one thread per (leaf, coordinate),
      // two chains (even and odd rows; any fixed order serves as a centre)
      for (int w = tid; w < nb * d; w += ROWS) {
        const int j = w / d, k = w - j * d;
        const int b0 = big_lb[j], b1 = big_le[j];
        float s0 = 0.0f, s1 = 0.0f;
        int q = b0;
        for (; q + 1 < b1; q += 2) {
          s0 = __fadd_rn(s0, xs[q * dp + k]);
          s1 = __fadd_rn(s1, xs[(q + 1) * dp + k]);
        }
        if (q < b1) s0 = __fadd_rn(s0, xs[q * dp + k]);
        cen[j * d4 + k] = __fdiv_rn(__fadd_rn(s0, s1), (float)(b1 - b0));
      }
      for (int w = tid; w < nb * (d4 - d); w += ROWS)  // pairs read past d see zeros
        cen[(w / (d4 - d)) * d4 + d + w % (d4 - d)] = 0.0f;
      __syncthreads();
      // (3) centred split-BF16 tiles, FP32 squared norms, Gram on the tensor core
      const int npad = (rows + 15) & ~15;
      const uint32_t idesc = rpf_umma_idesc_bf16(128, npad);
      float2 yy2 = make_float2(0.0f, 0.0f);  // squared norm: even and odd coordinates
      for (int k0 = 0; k0 < d16 && ok; k0 += KC) {
        if (k0 > 0) {  // the previous chunk's MMAs must be done reading the tiles
          const bool w = rpf_mbar_wait(&bar_mma, mma_phase, err, wlim);
          mma_phase ^= 1u;
          mma_pending = false;
          ok = __syncthreads_and(w) != 0;
          if (!ok) break;
        }
        for (int kk = 0; kk < KC; kk += 8) {
          uint32_t hp[4], lp[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            // coordinates k, k + 1 as one pair (rows and centres are zero
            // beyond d): y = x - c, hi = bf16(y), lo = bf16(y - hi)
            const int k = k0 + kk + 2 * u;
            float2 y2 = make_float2(0.0f, 0.0f);
            if (bslot >= 0 && k < d)
              y2 = rpf_sub2(*reinterpret_cast<const float2*>(xs + r * dp + k),
                            *reinterpret_cast<const float2*>(cen + bslot * d4 + k));
            yy2 = rpf_fma2(y2, y2, yy2);
            hp[u] = rpf_bf16x2(y2.x, y2.y);
            const float2 h2 = make_float2(__uint_as_float(hp[u] << 16),
                                          __uint_as_float(hp[u] & 0xffff0000u));
            const float2 l2 = rpf_sub2(y2, h2);
            lp[u] = rpf_bf16x2(l2.x, l2.y);
          }
          const int idx = rpf_umma_index(r, kk, RG);  // 8 consecutive k: 16 bytes
          *reinterpret_cast<uint4*>(Ahi + idx) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
          *reinterpret_cast<uint4*>(Alo + idx) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
        }
        rpf_fence_proxy_async();  // BF16 tiles -> visible to the tensor core
        rpf_tc_fence_before();
        __syncthreads();
        if (tid == 0) {
          rpf_tc_fence_after();
          const uint32_t hb = rpf_saddr(Ahi), lbs = rpf_saddr(Alo);
          const uint32_t lbo = (uint32_t)RG * 128u;  // next 8-column group along K
          for (int blk = 0; blk < ROWS / 128; ++blk) {
            if (blk * 128 >= rows) break;
            const uint32_t dcol = tbase + (uint32_t)(256 * blk);
            const uint32_t aoff = (uint32_t)blk * 16u * 128u;  // rows 128 blk ...
            for (int s2 = 0; s2 < KC / 16; ++s2) {
              const uint32_t off = (uint32_t)s2 * 2u * lbo;
              const uint64_t ah = rpf_umma_desc(hb + off + aoff, lbo, 128u);
              const uint64_t al = rpf_umma_desc(lbs + off + aoff, lbo, 128u);
              const uint64_t bh = rpf_umma_desc(hb + off, lbo, 128u);
              const uint64_t bl = rpf_umma_desc(lbs + off, lbo, 128u);
              rpf_umma_bf16(dcol, ah, bh, idesc, (k0 > 0 || s2 > 0) ? 1u : 0u);
              rpf_umma_bf16(dcol, ah, bl, idesc, 1u);
              rpf_umma_bf16(dcol, al, bh, idesc, 1u);
            }
          }
          rpf_umma_commit(&bar_mma);
        }
        mma_pending = true;
      }
      if (!ok) break;
      const float yy = __fadd_rn(yy2.x, yy2.y);
      nrm[r] = yy;
      const float yup = __fmul_ru(yy, 1.0f + (float)(d + 4) * 0x1p-23f);
      ynm[r] = __fsqrt_ru(yup);
      if (bslot >= 0) atomicMax(&nmax_bits[bslot], __float_as_uint(yup));
      {
        const bool w = rpf_mbar_wait(&bar_mma, mma_phase, err, wlim);
        mma_phase ^= 1u;
        mma_pending = false;
        ok = __syncthreads_and(w) != 0;
        if (!ok) break;
      }
      rpf_tc_fence_after();
      if (bslot >= 0) {
        const float Nm = __uint_as_float(nmax_bits[bslot]);
        cert_ok = Nm >= 0x1p-90f && Nm <= 0x1p120f;
      }
    }
    // (4) per-row candidates: small leaves offer everything; large leaves
    // offer the certified margin around tau
    unsigned char* my = slots + r * TC_SLOT_STRIDE;
    int ns = 0;
    float tau2 = 0.0f, eps = 0.0f, eta = 0.0f;
    const bool tc_row = big && cert_ok;
    if (__any_sync(RPF_FULL, tc_row)) {
      int lo = tc_row ? lb : ROWS, hi = tc_row ? le : 0;
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(RPF_FULL, lo, off));
        hi = max(hi, __shfl_xor_sync(RPF_FULL, hi, off));
      }
      lo &= ~7;
      const float nr = nrm[r];
      // One pass keeps the KK + 2 smallest keys (D~ bits with the low 8 bits
      // replaced by the column; D~ >= 0 after clamping, which moves no
      // value away from its bound): a key's bucket [lower, upper] holds its
      // D~, keys order like buckets, so the K-th key's upper edge is an
      // upper bound tau of the K-th smallest D~.  The margin's columns are
      // the kept keys whose lower edge is <= tau'; when the last kept key's
      // lower edge is also <= tau', further columns may lie within the
      // margin and the row collects them in a second pass.
      TopU<KK + 2> th;
      th.init();
#pragma unroll 1
      for (int c0 = lo; c0 < hi; c0 += 8) {
        float g[8], D[8];
        rpf_tmem_ld8(tlane + (uint32_t)c0, g);
        tc_dist8(g, nr, nrm, c0, D);
        uint32_t kb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = c0 + j;
          const bool use = tc_row && c >= lb && c < le && c != r;
          const uint32_t key = (__float_as_uint(fmaxf(D[j], 0.0f)) & 0xffffff00u) | (uint32_t)c;
          kb[j] = use ? key : 0xffffffffu;
        }
        th.insert8(kb);
      }
      bool more = false;  // the kept keys may not hold every margin column
      if (tc_row) {
        const uint32_t kk = th.kth(K);
        const float tlow = __uint_as_float(kk & 0xffffff00u);
        const float tau = kk == 0xffffffffu || isinf(tlow) ? INFINITY : __uint_as_float(kk | 0xffu);
        const float Nm = __uint_as_float(nmax_bits[bslot]);
        eps = __fmul_ru(ce, __fadd_ru(nr, Nm));
        eta = __fmul_ru(0x1p-23f, __fadd_ru(ynm[r], __fsqrt_ru(Nm)));
        const float s = __fadd_ru(__fmul_ru(__fsqrt_ru(__fadd_ru(tau, eps)), 1.0f + 4.0f * gam),
                                  2.0f * eta);
        tau2 = __fadd_ru(eps, __fmul_ru(s, s));
        const uint32_t last = th.v[KK + 1];
        more = last != 0xffffffffu && !(__uint_as_float(last & 0xffffff00u) > tau2);
        if (!more) {
#pragma unroll
          for (int q = 0; q < KK + 2; ++q) {
            const uint32_t v = th.v[q];
            if (v != 0xffffffffu && __uint_as_float(v & 0xffffff00u) <= tau2) {
              if (ns < TC_SLOTS) my[ns] = (unsigned char)(v & 0xffu);
              ++ns;
            }
          }
        }
      }
      if (__any_sync(RPF_FULL, more)) {
        // the columns within the margin, eight at a time as a bit mask; the
        // few set bits are then written out (no divergent store per column)
        const int cl = more ? lb : 0, ch = more ? le : 0;
#pragma unroll 1
        for (int c0 = lo; c0 < hi; c0 += 8) {
          float g[8], D[8];
          rpf_tmem_ld8(tlane + (uint32_t)c0, g);
          tc_dist8(g, nr, nrm, c0, D);
          uint32_t msk = 0u;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = c0 + j;
            const bool take = c >= cl && c < ch && c != r && D[j] <= tau2;
            msk |= (uint32_t)take << j;
          }
          while (msk) {
            const int j = __ffs(msk) - 1;
            msk &= msk - 1u;
            if (ns < TC_SLOTS) my[ns] = (unsigned char)(c0 + j);
            ++ns;
          }
        }
      }
    }
    const bool exact_row = live && (!big || !cert_ok);
    if (live && !big) {  // small leaf: everything is a candidate
      for (int c = lb; c < le; ++c)
        if (c != r) my[ns++] = (unsigned char)c;
    }
    if (tile + gridDim.x < thi) fetch_rows(tl_c, prow_c, start_c);
    // (5) exact re-rank of the candidates
    Top64<KK> ex;
    ex.init();
    bool redo = false;
    if (live && (!big || tc_row)) {
      const int nc = min(ns, TC_SLOTS);
#pragma unroll 1
      for (int e0 = 0; e0 < nc; e0 += 4) {
        int cc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cc[j] = my[e0 + j < nc ? e0 + j : e0];
        float acc[4];
        d32x4(xs, dp, d4, r, cc, acc);
        unsigned long long kb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) kb[j] = e0 + j < nc ? key64(acc[j], prow_s[cc[j]]) : ~0ull;
        ex.insert4(kb);
      }
      if (tc_row) {
        // (6) certificate
        if (ns > TC_SLOTS) {
          redo = true;
        } else {
          const float rk = ex.kth_d32(K);
          const float base = __fsub_rd(__fsqrt_rd(fmaxf(__fsub_rd(tau2, eps), 0.0f)), eta);
          const float lower = __fmul_rd(1.0f - gam, base);
          redo = !(__fsqrt_ru(rk) < lower);
        }
      }
    }
    if (redo || exact_row) {  // exact scan of the whole leaf
      ex.init();
#pragma unroll 1
      for (int c0 = lb; c0 < le; c0 += 4) {
        int cc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cc[j] = min(c0 + j, le - 1);
        float acc[4];
        d32x4(xs, dp, d4, r, cc, acc);
        unsigned long long kb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          kb[j] = c0 + j < le && c0 + j != r ? key64(acc[j], prow_s[c0 + j]) : ~0ull;
        ex.insert4(kb);
      }
      if (redo) atomicAdd(fallbacks, 1ULL);
    }
    if (live) ex.store(K, cand + ((int64_t)(t - t0) * n + prow_s[r]) * K);
    // (7) the tile's shared memory and TMEM are reused by the next tile
    rpf_fence_proxy_async();
    rpf_tc_fence_before();
    __syncthreads();
  }
  // after a timed-out wait: one more bounded wait for work in flight
  if (tma_pending) rpf_mbar_wait(&bar_tma, tma_phase, nullptr, wlim);
  if (mma_pending) rpf_mbar_wait(&bar_mma, mma_phase, nullptr, wlim);
  rpf_tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    rpf_tc_fence_after();
    rpf_tmem_dealloc(tbase, TCOLS);  // exactly the columns allocated
  }
}

size_t tc_need(int d, int dp, int rows, int KC) {
  const int d4 = (d + 3) & ~3;
  const size_t a_off = (((size_t)rows * dp * 4) + 1023) & ~(size_t)1023;
  return a_off + (size_t)2 * rows * KC * 2 + (size_t)(rows / TC_BIG_MIN + 1) * d4 * 4 +
         (size_t)rows * TC_SLOT_STRIDE;
}

// Dynamic shared memory of a CTA.  128-row tiles: if the tile fits 52 KB,
// at least 46 KB (four CTAs per SM, 4 x 128 TMEM columns), else at least
// 60 KB (three CTAs); 256-row tiles hold all 512 TMEM columns (one CTA).
size_t tc_smem(int d, int dp, int rows, int KC) {
  const size_t need = tc_need(d, dp, rows, KC);
  if (rows == 256) return std::max<size_t>(need, 120 * 1024);
  return need <= 52 * 1024 ? std::max<size_t>(need, 46 * 1024) : std::max<size_t>(need, 60 * 1024);
}

// Gram coordinates per chunk (a multiple of 16, <= 128): with 128-row tiles
// the largest that lets four CTAs share an SM, if any; otherwise the largest
// for which the CTA fits 220 KB (the opt-in limit is 227 KB); 0 if none.
int tc_chunk(int d, int rows) {
  const int d16 = (d + 15) & ~15, dp = ((d + 3) & ~3) + 4;
  if (rows == 128)
    for (int kc = std::min(d16, 128); kc >= 16; kc -= 16)
      if (tc_need(d, dp, rows, kc) <= 52 * 1024) return kc;
  for (int kc = std::min(d16, 128); kc >= 16; kc -= 16)
    if (tc_smem(d, dp, rows, kc) <= 220 * 1024) return kc;
  return 0;
}

// Launch configuration of the chosen-form kernel: Gram coordinates per
// chunk and CTAs per SM of the persistent grid.  rpf_tc_autotune times the
// candidates on a forest's own tiles and keeps the fastest per (d, tile rows,
// K bucket) for the rest of the process; without a tuned entry the
// heuristic (largest chunk that fits four CTAs, else three) is used.
struct TcConf {
  int kc = 0, occ = 0;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TcConf> g_tune;
// build-time tile shapes per (d, leaf bound): chosen-form tile rows and the
// plain form's tile region (0: the heuristic)
struct ShapeConf {
  int rows = 0, region = 0;
};
std::map<std::pair<int, int>, ShapeConf> g_shape;
// query leaf scan per (d, leaf bound, K bucket): 1 = BF16 rows, 0 = FP32 rows
std::map<std::tuple<int, int, int>, int> g_qscan;

template <int KK, int ROWS>
int launch_tc(const rpf_forest* f, int64_t tlo, int64_t thi, int K, int t0, uint2* cand,
              cudaStream_t s, const TcConf* force = nullptr) {
  if (thi <= tlo) return RPF_OK;
  const int d = f->d, dp = ((d + 3) & ~3) + 4, d16 = (d + 15) & ~15;
  TcConf conf;
  if (force) {
    conf = *force;
  } else {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(d, ROWS, KK));
    if (it != g_tune.end()) conf = it->second;
  }
  const int KC = conf.kc > 0 ? conf.kc : tc_chunk(d, ROWS);
  const size_t smem = tc_smem(d, dp, ROWS, KC);
  if (smem > 220 * 1024) return RPF_EINVAL;
  RPF_CU(cudaFuncSetAttribute(k_leaf_tc<KK, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
  int dev = 0, sms = 0, smem_sm = 0;
  RPF_CU(cudaGetDevice(&dev));
  RPF_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  RPF_CU(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  RPF_CU(cudaFuncSetAttribute(k_leaf_tc<KK, ROWS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              100));
  cudaFuncAttributes fa;
  RPF_CU(cudaFuncGetAttributes(&fa, k_leaf_tc<KK, ROWS>));
  // CTAs per SM that shared memory allows (1 KB per CTA is reserved by the
  // system), and that TMEM allows: four of 128 columns or one of 512
  const size_t per_cta = smem + fa.sharedSizeBytes + 1024;
  const int tmem_cap = ROWS == 128 ? 4 : 1;
  int occ = std::max(1, std::min(tmem_cap, (int)((size_t)smem_sm / per_cta)));
  if (conf.occ > 0) occ = std::min(occ, conf.occ);
  const int64_t grid = std::min<int64_t>(thi - tlo, (int64_t)sms * occ);
  RPF_LAUNCH("k_leaf_tc", s, k_leaf_tc<KK, ROWS><<<(unsigned)grid, ROWS, smem, s>>>(
      f->pk_tiles, tlo, thi, f->pk_bits, f->pk_nwords, f->perm, f->X, f->n, d, dp, d16, KC, K,
      t0, cand, f->d_err, f->d_fallback, rpf_wait_limit_ns()));
  return RPF_OK;
}

template <int KK>
int launch_tc_rows(const rpf_forest* f, int64_t tlo, int64_t thi, int K, int t0, uint2* cand,
                   cudaStream_t s, const TcConf* force = nullptr) {
  return f->pk_rows == 128 ? launch_tc<KK, 128>(f, tlo, thi, K, t0, cand, s, force)
                           : launch_tc<KK, 256>(f, tlo, thi, K, t0, cand, s, force);
}

// sorted-list length for K: only the first K slots are read, so common K
// (10, 20) get lists of exactly K
int kk_of(int K) {
  return K <= 4 ? 4 : K <= 8 ? 8 : K <= 10 ? 10 : K <= 12 ? 12 : K <= 16 ? 16 : K <= 20 ? 20
         : K <= 24 ? 24 : 32;
}

int launch_tc_k(const rpf_forest* f, int64_t tlo, int64_t thi, int K, int t0, uint2* cand,
                cudaStream_t s, const TcConf* force = nullptr) {
  switch (kk_of(K)) {
    case 4: return launch_tc_rows<4>(f, tlo, thi, K, t0, cand, s, force);
    case 8: return launch_tc_rows<8>(f, tlo, thi, K, t0, cand, s, force);
    case 10: return launch_tc_rows<10>(f, tlo, thi, K, t0, cand, s, force);
    case 12: return launch_tc_rows<12>(f, tlo, thi, K, t0, cand, s, force);
    case 16: return launch_tc_rows<16>(f, tlo, thi, K, t0, cand, s, force);
    case 20: return launch_tc_rows<20>(f, tlo, thi, K, t0, cand, s, force);
    case 24: return launch_tc_rows<24>(f, tlo, thi, K, t0, cand, s, force);
    default: return launch_tc_rows<32>(f, tlo, thi, K, t0, cand, s, force);
  }
}

}  // namespace

int rpf_tuned_region(int d, int L) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_shape.find(std::make_pair(d, L));
  return it == g_shape.end() ? 0 : it->second.region;
}

int rpf_tuned_rows(int d, int L) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_shape.find(std::make_pair(d, L));
  return it == g_shape.end() ? 0 : it->second.rows;
}

int rpf_tuned_qscan(int d, int L, int K) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_qscan.find(std::make_tuple(d, L, kk_of(K)));
  return it == g_qscan.end() ? -1 : it->second;
}

bool rpf_tc_supported(const rpf_forest* f, int K) {
  return f->pk_tiles != nullptr && f->prm.leaf_max <= 256 && K <= 32 &&
         tc_chunk(f->d, f->pk_rows) > 0;
}

int rpf_build_packs(rpf_forest* f, cudaStream_t s, int rows_force) {
  const int T = f->prm.n_trees;
  const int64_t n = f->n, nl = f->n_leaves;
  const int64_t nwords = (n + 31) >> 5, nseg = (n + TC_SEG - 1) / TC_SEG;
  const int64_t G = (int64_t)T * nseg;
  int2* slot = nullptr;
  int32_t *cnt = nullptr, *off = nullptr, *blk = nullptr, *tot = nullptr;
  // a rebuild replaces the previous tables (stream-ordered)
  rpf_release(f->pk_bits, s);
  rpf_release(f->pk_tiles, s);
  f->pk_bits = nullptr;
  f->pk_tiles = nullptr;
  if (rpf_alloc((void**)&f->pk_bits, 4 * (size_t)(T * nwords), s) ||
      rpf_alloc((void**)&slot, 8 * (size_t)G * TC_SEG_TILES, s) ||
      rpf_alloc((void**)&cnt, 4 * (size_t)G, s) || rpf_alloc((void**)&off, 4 * (size_t)G, s) ||
      rpf_alloc((void**)&blk, 4 * (size_t)((G + 1023) / 1024 + 1), s) ||
      rpf_alloc((void**)&tot, 4, s)) {
    rpf_release(slot, s);
    rpf_release(cnt, s);
    rpf_release(off, s);
    rpf_release(blk, s);
    return RPF_ENOMEM;
  }
  f->pk_nwords = nwords;
  RPF_CU(cudaMemsetAsync(f->pk_bits, 0, 4 * (size_t)(T * nwords), s));
  RPF_LAUNCH("k_leaf_bits", s, k_leaf_bits<<<nblk(nl, 256), 256, 0, s>>>(
      nl, f->leaf_tree, f->leaf_begin, nwords, f->pk_bits));
  // tile rows: 128 for leaf bounds up to 128, else 256; leaves of up to 128
  // points may also go in 256-row tiles when the autotuner found them faster
  int rows = f->prm.leaf_max <= 128 ? 128 : 256;
  const int want = rows_force > 0 ? rows_force : rpf_tuned_rows(f->d, f->prm.leaf_max);
  if (want == 256) rows = 256;
  f->pk_rows = rows;
  RPF_LAUNCH("k_pack_tiles", s, k_pack_tiles<<<nblk(G, 128), 128, 0, s>>>(
      T, n, nseg, nwords, f->pk_bits, f->pk_rows, slot, cnt));
  const int32_t* cn = cnt;
  int32_t* of = off;
  rpf_scan(G, [=] __device__(int64_t i) -> int { return min(cn[i], TC_SEG_TILES); },
           [=] __device__(int64_t i, int p) { of[i] = p; }, blk, tot, s);
  // per-tree tile offsets (segments are tree-major) and the tile count
  std::vector<int32_t> h_off(G), h_cnt(G);
  int32_t h_tot = 0;
  RPF_CU(cudaMemcpyAsync(h_off.data(), off, 4 * (size_t)G, cudaMemcpyDeviceToHost, s));
  RPF_CU(cudaMemcpyAsync(h_cnt.data(), cnt, 4 * (size_t)G, cudaMemcpyDeviceToHost, s));
  RPF_CU(cudaMemcpyAsync(&h_tot, tot, 4, cudaMemcpyDeviceToHost, s));
  RPF_CU(cudaStreamSynchronize(s));
  bool over = false;
  for (int64_t g = 0; g < G; ++g) over |= h_cnt[g] > TC_SEG_TILES;
  if (over) {  // cannot happen: a segment packs into at most TC_SEG_TILES tiles
    rpf_release(slot, s);
    rpf_release(cnt, s);
    rpf_release(off, s);
    rpf_release(blk, s);
    rpf_release(tot, s);
    return RPF_EINTERNAL;
  }
  f->pk_tree_off.assign(T + 1, 0);
  for (int t = 0; t < T; ++t) f->pk_tree_off[t] = h_off[(int64_t)t * nseg];
  f->pk_tree_off[T] = h_tot;
  if (rpf_alloc((void**)&f->pk_tiles, 16 * (size_t)std::max(h_tot, 1), s)) {
    rpf_release(slot, s);
    rpf_release(cnt, s);
    rpf_release(off, s);
    rpf_release(blk, s);
    rpf_release(tot, s);
    return RPF_ENOMEM;
  }
  RPF_LAUNCH("k_pack_fill", s, k_pack_fill<<<nblk(G, 128), 128, 0, s>>>(G, nseg, slot, cnt, off,
                                                                       f->pk_tiles));
  rpf_release(slot, s);
  rpf_release(cnt, s);
  rpf_release(off, s);
  rpf_release(blk, s);
  rpf_release(tot, s);
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

int rpf_leaf_tc(const rpf_forest* f, int t0, int g, int K, uint2* cand, cudaStream_t s) {
  return launch_tc_k(f, f->pk_tree_off[t0], f->pk_tree_off[t0 + g], K, t0, cand, s);
}

namespace {
// best of three timed runs (the first warms caches) of fn on stream s, ms
template <typename Fn>
int time_best(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, Fn fn, float* best) {
  *best = INFINITY;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s);
    const int rc = fn();
    cudaEventRecord(e1, s);
    if (rc) return rc;
    if (cudaEventSynchronize(e1) != cudaSuccess) return RPF_ECUDA;
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) *best = std::min(*best, t);
  }
  return RPF_OK;
}
}  // namespace

// Autotuner of the leaf tiles, timed on the forest's own tiles (its first
// trees).  Plain form: the tile region R (multiples of 32 up to the cap).
// Chosen form: tile rows (128 or 256 where the leaf bound allows both), Gram
// coordinates per chunk, CTAs per SM, and the query leaf scan (BF16 or FP32
// rows).  Every candidate gives the same lists.
// The tile shape is kept per (d, leaf bound) for later builds and applied to
// this forest; the launch choice per (d, tile rows, K bucket).
int rpf_tc_autotune(rpf_forest* f, int K, cudaStream_t s, int32_t* chosen) {
  if (chosen) {
    chosen[0] = chosen[1] = chosen[2] = chosen[3] = 0;
    chosen[4] = -1;
  }
  const int d = f->d, L = f->prm.leaf_max;
  const int g = std::min(f->prm.n_trees, 4);  // the tiles of the first trees
  uint2* cand = nullptr;
  if (rpf_alloc((void**)&cand, (size_t)g * f->n * K * 8, s)) return RPF_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = RPF_OK;
  if (f->prm.form == 0) {
    int best_r = 0;
    float best_ms = INFINITY;
    for (int R = 32; R <= rpf_region_cap(L) && !rc; R += 32) {
      rc = rpf_build_tiles(f, s, R);
      float ms = INFINITY;
      if (!rc) rc = time_best(s, e0, e1, [&] { return rpf_leaf_plain(f, 0, g, K, cand, s); }, &ms);
      if (!rc && ms < best_ms) {
        best_ms = ms;
        best_r = R;
      }
    }
    if (!rc) {
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_shape[std::make_pair(d, L)].region = best_r;
      }
      rc = rpf_build_tiles(f, s, best_r);
    }
    if (chosen && !rc) chosen[3] = best_r;
  } else if (rpf_tc_supported(f, K)) {
    const int dp = ((d + 3) & ~3) + 4, d16 = (d + 15) & ~15;
    TcConf best;
    int best_rows = f->pk_rows;
    float best_ms = INFINITY;
    const int rows_opts[2] = {128, 256};
    for (int ri = 0; ri < 2 && !rc; ++ri) {
      const int rows = rows_opts[ri];
      if ((rows == 128 && L > 128) || tc_chunk(d, rows) == 0) continue;
      rc = rpf_build_packs(f, s, rows);
      const int max_occ = rows == 128 ? 4 : 1;
      for (int kc = 16; kc <= std::min(d16, 128) && !rc; kc += 16) {
        if (tc_smem(d, dp, rows, kc) > 220 * 1024) continue;
        for (int occ = 1; occ <= max_occ && !rc; ++occ) {
          const TcConf c{kc, occ};
          float ms = INFINITY;
          rc = time_best(s, e0, e1, [&] {
            return launch_tc_k(f, f->pk_tree_off[0], f->pk_tree_off[g], K, 0, cand, s, &c);
          }, &ms);
          if (!rc && ms < best_ms) {
            best_ms = ms;
            best = c;
            best_rows = rows;
          }
        }
      }
    }
    if (!rc) {
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[std::make_tuple(d, best_rows, kk_of(K))] = best;
        g_shape[std::make_pair(d, L)].rows = best_rows;
      }
      rc = rpf_build_packs(f, s, best_rows);
    }
    if (chosen && !rc) {
      chosen[0] = best.kc;
      chosen[1] = best.occ;
      chosen[2] = best_rows;
      chosen[3] = f->tile_region;
    }
    // the query leaf scan: BF16 rows with the certified re-rank against the
    // FP32 rows, timed on the first (up to 4096) data points as queries
    if (!rc && rpf_qscan_bf_ok(f, K)) {
      const int T = f->prm.n_trees;
      const int64_t mq = std::min<int64_t>(f->n, 4096);
      int2* qleaf = nullptr;
      uint2* qc = nullptr;
      int* qe = nullptr;
      if (rpf_alloc((void**)&qleaf, 8 * (size_t)mq * T, s) ||
          rpf_alloc((void**)&qc, 8 * (size_t)mq * T * K, s) || rpf_alloc((void**)&qe, 4, s)) {
        rc = RPF_ENOMEM;
      } else {
        rc = rpf_route_dev(f, f->X, mq, qleaf, s);
        float ms_bf = INFINITY, ms_32 = INFINITY;
        if (!rc)
          rc = time_best(s, e0, e1, [&] {
            return rpf_qscan_dev(f, f->X, mq, K, qleaf, qc, qe, true, s);
          }, &ms_bf);
        if (!rc)
          rc = time_best(s, e0, e1, [&] {
            return rpf_qscan_dev(f, f->X, mq, K, qleaf, qc, qe, false, s);
          }, &ms_32);
        if (!rc) {
          const int pick = ms_bf < ms_32 ? 1 : 0;
          {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_qscan[std::make_tuple(d, L, kk_of(K))] = pick;
          }
          if (chosen) chosen[4] = pick;
        }
      }
      rpf_release(qleaf, s);
      rpf_release(qc, s);
      rpf_release(qe, s);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  rpf_release(cand, s);
  if (!rc) {
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = rpf_cuda_err(e);
  }
  return rc;
}
