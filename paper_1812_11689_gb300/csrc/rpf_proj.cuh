// rpf_proj.cuh -- centred FP32 projections and their block statistics,
// shared by the level-synchronous and the CTA-local growth kernels.
//
// Statistics of the FP32 projections q' of a node for one try: S1 = sum q',
// S2 = sum q'^2, A = sum |q'|, min, max.  Every thread accumulates at most 32
// points in FP32, the warp folds with a butterfly in FP32, and one thread per
// try adds the (at most 8) warp partials in FP32; the error analysis of
// rpf_try_bounds assumes this depth (RPF_STAT_DEPTH).
#pragma once

#include "rpf_internal.cuh"

// q'_j(x) = fl32-dot(r32_j, fl32(x - o)) for up to 4 points (gid < 0: none)
// and tries [j0, j0 + nj) (r32 of try j0 at sr, stride d); nn = FP32 sum of
// squares of fl32(x - o) when want_nn.
template <int TG>
__device__ __forceinline__ void rpf_proj4(const float* __restrict__ X, int d, const int (&gid)[4],
                                          const float* so, const float* sr, int nj,
                                          float (&acc)[4][TG], float (&nn)[4], bool want_nn) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    nn[p] = 0.0f;
#pragma unroll
    for (int q = 0; q < TG; ++q) acc[p][q] = 0.0f;
  }
  if ((d & 3) == 0) {
    // unrolled so that the next coordinates' row loads are issued while the
    // current ones are multiplied (each chain still runs over k in order)
#pragma unroll 2
    for (int k = 0; k < d; k += 4) {
      const float4 o4 = *reinterpret_cast<const float4*>(so + k);
      float4 r4[TG];
#pragma unroll
      for (int q = 0; q < TG; ++q)
        if (q < nj) r4[q] = *reinterpret_cast<const float4*>(sr + q * d + k);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        if (gid[p] < 0) continue;
        const float4 x4 = __ldg(reinterpret_cast<const float4*>(X + (int64_t)gid[p] * d + k));
        const float e0 = __fsub_rn(x4.x, o4.x), e1 = __fsub_rn(x4.y, o4.y);
        const float e2 = __fsub_rn(x4.z, o4.z), e3 = __fsub_rn(x4.w, o4.w);
        if (want_nn) {
          nn[p] = __fmaf_rn(e0, e0, nn[p]);
          nn[p] = __fmaf_rn(e1, e1, nn[p]);
          nn[p] = __fmaf_rn(e2, e2, nn[p]);
          nn[p] = __fmaf_rn(e3, e3, nn[p]);
        }
#pragma unroll
        for (int q = 0; q < TG; ++q) {
          if (q < nj) {
            float a = acc[p][q];
            a = __fmaf_rn(e0, r4[q].x, a);
            a = __fmaf_rn(e1, r4[q].y, a);
            a = __fmaf_rn(e2, r4[q].z, a);
            a = __fmaf_rn(e3, r4[q].w, a);
            acc[p][q] = a;
          }
        }
      }
    }
  } else {
    for (int k = 0; k < d; ++k) {
      const float ok = so[k];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        if (gid[p] < 0) continue;
        const float e = __fsub_rn(__ldg(X + (int64_t)gid[p] * d + k), ok);
        if (want_nn) nn[p] = __fmaf_rn(e, e, nn[p]);
#pragma unroll
        for (int q = 0; q < TG; ++q)
          if (q < nj) acc[p][q] = __fmaf_rn(e, sr[q * d + k], acc[p][q]);
      }
    }
  }
}

// The same projections for a warp's 32 points, one per lane, with the rows
// staged through shared memory (needs d % 4 == 0).  Rows are read 8 lanes
// per 32-coordinate chunk (one coalesced 128-byte line per row) by cp.async
// straight into a padded tile (row stride 36 floats, an odd number of 16-byte
// units, so that the lanes' row reads fall in distinct banks); each lane then
// runs its own point's chains from the tile (even and odd coordinates in
// order, see rpf_tile_chunk).  Gathering
// whole lines this way reaches about 4x the L2 bandwidth of one 16-byte load
// per lane per row, and two tiles per warp let the next chunk's copy overlap
// the current chunk's arithmetic.
// DC coordinates per chunk; row stride DC + 4 floats (DC = 16 or 32 keeps it
// an odd number of 16-byte units)
#define RPF_TILE_DC 32
#define RPF_TILE_STRIDE 36
#define RPF_TILE_FLOATS (32 * RPF_TILE_STRIDE)

__device__ __forceinline__ void rpf_cp16(float* sdst, const float* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void rpf_cp_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void rpf_cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Warp-collective: copy coordinates [k0, k0 + DC) of the 32 rows gid (lane
// l's row to tile row l; gid < 0: none) into the tile (DC / 4 lanes per row).
// DFULL: d is a multiple of DC (every chunk is whole).
template <int DC = RPF_TILE_DC, bool DFULL = false>
__device__ __forceinline__ void rpf_stage_rows(const float* __restrict__ X, int d, int gid, int k0,
                                               float* tile, int lane) {
  constexpr int LPR = DC / 4, RPI = 32 / LPR;  // lanes per row, rows per instruction
  const int c4 = 4 * (lane % LPR);
  const int kc = min(DC, d - k0);
#pragma unroll
  for (int i = 0; i < 32 / RPI; ++i) {
    const int row = RPI * i + lane / LPR;
    const int g = __shfl_sync(RPF_FULL, gid, row);
    if (g >= 0 && (DFULL || c4 < kc))
      rpf_cp16(tile + row * (DC + 4) + c4, X + (int64_t)g * d + k0 + c4);
  }
}

// Chains of the lane's row over coordinates [k0, k0 + kc) from the tile.
// Every dot product (and the sum of squares) runs as two FP32 chains, one
// over the even and one over the odd coordinates, in packed pair
// instructions; the caller adds the halves.  Each half has at most d / 2
// terms, so the computed value obeys the error bound of a d-term sequential
// chain that the radius and the statistics bounds assume.
// FULL: all TG tries and the sum of squares (the caller guarantees nj == TG
// and want_nn), so that no per-try predicate is kept across the loop.
template <int TG, int DC, bool FULL, bool DFULL>
__device__ __forceinline__ void rpf_tile_chunk(const float* tile, int lane, int k0, int kc,
                                                 const float* so, const float* sr, int d, int nj,
                                                 float2 (&acc)[TG], float2& nn, bool want_nn) {
  const float* xr = tile + lane * (DC + 4);
  const int kcc = DFULL ? DC : kc;
#pragma unroll(DFULL ? DC / 4 : 4)
  for (int k = 0; k < kcc; k += 4) {
    const float4 x4 = *reinterpret_cast<const float4*>(xr + k);
    const float4 o4 = *reinterpret_cast<const float4*>(so + k0 + k);
    const float2 e01 = rpf_sub2(make_float2(x4.x, x4.y), make_float2(o4.x, o4.y));
    const float2 e23 = rpf_sub2(make_float2(x4.z, x4.w), make_float2(o4.z, o4.w));
    if (FULL || want_nn) {
      nn = rpf_fma2(e01, e01, nn);
      nn = rpf_fma2(e23, e23, nn);
    }
#pragma unroll
    for (int q = 0; q < TG; ++q) {
      if (FULL || q < nj) {
        const float4 r4 = *reinterpret_cast<const float4*>(sr + q * d + k0 + k);
        acc[q] = rpf_fma2(e23, make_float2(r4.z, r4.w),
                          rpf_fma2(e01, make_float2(r4.x, r4.y), acc[q]));
      }
    }
  }
}

// Warp-collective driver of the staged projections: the warp's batches of 32
// positions (batch bfirst + i bstride, position 32 b + lane, point id
// ids[position]; npos positions) are cut into units (batch, DC-coordinate
// chunk), and unit u + NS - 1 is copied into tile (u + NS - 1) % NS while
// unit u is computed (NS tiles of 32 rows x (DC + 4) floats at `tiles`).
// After a batch's last chunk fin(position, id, acc, nn, xn) runs on every
// lane whose position holds a point, xn = xnorm[id] (0 when xnorm is null).
// Point ids and their norms are read NS batches ahead.  FULL: nj == TG and
// want_nn on every call (one pass over all tries).  DFULL: d % DC == 0.
template <int TG, int DC, int NS, bool FULL, bool DFULL, typename IdT, typename Fin>
__device__ __forceinline__ void rpf_warp_project(const float* __restrict__ X, int d, const IdT* ids,
                                                 int npos, int bfirst, int bstride, float* tiles,
                                                 const float* so, const float* sr, int nj,
                                                 bool want_nn, int lane,
                                                 const float* __restrict__ xnorm, Fin fin) {
  constexpr int TF = 32 * (DC + 4);
  const int nch = (d + DC - 1) / DC;
  const int nbt = (npos + 31) >> 5;
  const int nbw = bfirst < nbt ? (nbt - bfirst + bstride - 1) / bstride : 0;
  if (nbw == 0) return;
  int g[NS];     // ids of batches i .. i + NS - 1 (-1: none)
  float xv[NS];  // their norms
  int pb = bfirst;
#pragma unroll
  for (int k = 0; k < NS; ++k, pb += bstride) {
    const int p = pb * 32 + lane;
    g[k] = (pb < nbt && p < npos) ? (int)ids[p] : -1;
    xv[k] = (xnorm && g[k] >= 0) ? xnorm[g[k]] : 0.0f;
  }
  // the next unit to copy: batch i + sk, chunk sc, into tile ss
  int sk = 0, sc = 0, ss = 0;
  auto stage_next = [&](int i) {
    int gs = g[0];
#pragma unroll
    for (int kk = 1; kk < NS; ++kk)
      if (sk == kk) gs = g[kk];
    if (i + sk < nbw) rpf_stage_rows<DC, DFULL>(X, d, gs, sc * DC, tiles + ss * TF, lane);
    ss = ss + 1 == NS ? 0 : ss + 1;
    if (++sc == nch) {
      sc = 0;
      ++sk;
    }
  };
#pragma unroll
  for (int v = 0; v < NS - 1; ++v) {
    stage_next(0);
    rpf_cp_commit();
  }
  int cs = 0;  // tile of the unit being computed
  for (int i = 0; i < nbw; ++i) {
    float2 acc2[TG], nn2 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < TG; ++q) acc2[q] = make_float2(0.0f, 0.0f);
    for (int c = 0; c < nch; ++c) {
      stage_next(i);
      rpf_cp_commit();
      rpf_cp_wait<NS - 1>();  // this unit's copies are done
      __syncwarp();
      if (g[0] >= 0)
        rpf_tile_chunk<TG, DC, FULL, DFULL>(tiles + cs * TF, lane, c * DC, min(DC, d - c * DC), so, sr,
                                     d, nj, acc2, nn2, want_nn);
      __syncwarp();  // before this tile takes a later unit
      cs = cs + 1 == NS ? 0 : cs + 1;
    }
    if (g[0] >= 0) {
      float acc[TG];
#pragma unroll
      for (int q = 0; q < TG; ++q) acc[q] = __fadd_rn(acc2[q].x, acc2[q].y);
      fin((bfirst + i * bstride) * 32 + lane, g[0], acc, __fadd_rn(nn2.x, nn2.y), xv[0]);
    }
#pragma unroll
    for (int k = 0; k + 1 < NS; ++k) {
      g[k] = g[k + 1];
      xv[k] = xv[k + 1];
    }
    const int p = pb * 32 + lane;
    g[NS - 1] = (pb < nbt && p < npos) ? (int)ids[p] : -1;
    xv[NS - 1] = (xnorm && g[NS - 1] >= 0) ? xnorm[g[NS - 1]] : 0.0f;
    pb += bstride;
    --sk;
  }
  rpf_cp_wait<0>();
}

__device__ __forceinline__ void rpf_stat_add(float v, float& s1, float& s2, float& a1, float& mn,
                                             float& mx) {
  s1 = __fadd_rn(s1, v);
  s2 = __fmaf_rn(v, v, s2);
  a1 = __fadd_rn(a1, fabsf(v));
  mn = fminf(mn, v);
  mx = fmaxf(mx, v);
}

// Block reduction of per-thread statistics for nj tries into o*[q] (written
// by thread q; visible to all threads after the trailing barrier).
// red: 8 warps x TG x 5 floats of shared memory (+ 34 when rad is given).
// With rad non-null, the block-wide max of the non-negative *rad and the sum
// of *rad2, added with upward rounding (an upper bound of the exact sum), are
// folded in (slots 8 TG 5 .. + 33 of red) and returned to every thread.
template <int TG>
__device__ __forceinline__ void rpf_block_stats(int nj, float (&s1)[TG], float (&s2)[TG],
                                                float (&a1)[TG], float (&mn)[TG], float (&mx)[TG],
                                                float* red, double* o1, double* o2, double* oa,
                                                float* omn, float* omx, float* rad = nullptr,
                                                float* rad2 = nullptr) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* rred = red + 8 * TG * 5;
  if (rad) {
    float v = *rad, q = *rad2;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      v = fmaxf(v, __shfl_xor_sync(RPF_FULL, v, off));
      q = __fadd_ru(q, __shfl_xor_sync(RPF_FULL, q, off));
    }
    if (lane == 0) {
      rred[w] = v;
      rred[8 + w] = q;
    }
  }
#pragma unroll
  for (int q = 0; q < TG; ++q) {
    if (!(TG <= 5 || q < nj)) continue;  // TG <= 5: nj == TG (the callers' launch)
    float a = s1[q], b = s2[q], c = a1[q], lo = mn[q], hi = mx[q];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      a = __fadd_rn(a, __shfl_xor_sync(RPF_FULL, a, off));
      b = __fadd_rn(b, __shfl_xor_sync(RPF_FULL, b, off));
      c = __fadd_rn(c, __shfl_xor_sync(RPF_FULL, c, off));
      lo = fminf(lo, __shfl_xor_sync(RPF_FULL, lo, off));
      hi = fmaxf(hi, __shfl_xor_sync(RPF_FULL, hi, off));
    }
    if (lane == 0) {
      float* r = red + (w * TG + q) * 5;
      r[0] = a;
      r[1] = b;
      r[2] = c;
      r[3] = lo;
      r[4] = hi;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < nj) {  // one thread per try
    const int nw = blockDim.x >> 5;
    const int q = threadIdx.x;
    {
      float A = 0.0f, B = 0.0f, C = 0.0f;
      float lo = INFINITY, hi = -INFINITY;
      for (int u = 0; u < nw; ++u) {
        const float* r = red + (u * TG + q) * 5;
        A = __fadd_rn(A, r[0]);
        B = __fadd_rn(B, r[1]);
        C = __fadd_rn(C, r[2]);
        lo = fminf(lo, r[3]);
        hi = fmaxf(hi, r[4]);
      }
      o1[q] = (double)A;
      o2[q] = (double)B;
      oa[q] = (double)C;
      omn[q] = lo;
      omx[q] = hi;
    }
  }
  if (rad && threadIdx.x == 0) {
    float m = 0.0f, q = 0.0f;
    for (int u = 0; u < (int)(blockDim.x >> 5); ++u) {
      m = fmaxf(m, rred[u]);
      q = __fadd_ru(q, rred[8 + u]);
    }
    rred[32] = m;
    rred[33] = q;
  }
  __syncthreads();
  if (rad) {
    *rad = rred[32];
    *rad2 = rred[33];
  }
}

