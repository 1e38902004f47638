// rpf_scan.cuh -- device-wide exclusive prefix sums of int32 arrays (three
// passes: per-1024-block sums, one-block scan of the block sums, per-block
// scan), used to compact tables and to lay out leaf tiles.
#pragma once

#include "rpf_internal.cuh"

namespace {  // each translation unit gets its own copies

// sum of v(i) over each 1024-element block
template <typename F>
__global__ void __launch_bounds__(1024) k_block_sums(int64_t N, F v, int32_t* blk) {
  __shared__ int ws[32];
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  int x = i < N ? v(i) : 0;
  for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(RPF_FULL, x, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int u = 0; u < 32; ++u) s += ws[u];
    blk[blockIdx.x] = s;
  }
}

// in-place exclusive scan of nb block sums by one block; total to *total
__global__ void __launch_bounds__(1024) k_scan_blocks(int32_t* blk, int nb, int32_t* total) {
  __shared__ int ws[32];
  __shared__ int run, tile_tot;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) run = 0;
  __syncthreads();
  for (int t0 = 0; t0 < nb; t0 += 1024) {
    const int i = t0 + threadIdx.x;
    const int v = i < nb ? blk[i] : 0;
    int x = v;
    for (int off = 1; off < 32; off <<= 1) {
      int y = __shfl_up_sync(RPF_FULL, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int r = 0;
      for (int u = 0; u < 32; ++u) {
        int a = ws[u];
        ws[u] = r;
        r += a;
      }
      tile_tot = r;
    }
    __syncthreads();
    if (i < nb) blk[i] = run + x - v + ws[w];
    __syncthreads();
    if (threadIdx.x == 0) run += tile_tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = run;
}

// out(i, exclusive prefix of v up to i) for every element
template <typename F, typename G>
__global__ void __launch_bounds__(1024) k_scan_apply(int64_t N, F v, const int32_t* blk_off, G out) {
  __shared__ int ws[32];
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int x0 = i < N ? v(i) : 0;
  int x = x0;
  for (int off = 1; off < 32; off <<= 1) {
    int y = __shfl_up_sync(RPF_FULL, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int u = 0; u < 32; ++u) {
      int a = ws[u];
      ws[u] = r;
      r += a;
    }
  }
  __syncthreads();
  if (i < N) out(i, blk_off[blockIdx.x] + x - x0 + ws[w]);
}

}  // namespace

// Exclusive scan driver: v(i) -> out(i, prefix); *total receives the sum.
// blk needs (N + 1023) / 1024 + 1 ints of device scratch.
template <typename F, typename G>
inline void rpf_scan(int64_t N, F v, G out, int32_t* blk, int32_t* total, cudaStream_t s) {
  const int nb = (int)((N + 1023) / 1024);
  if (nb == 0) {
    cudaMemsetAsync(total, 0, sizeof(int32_t), s);
    return;
  }
  RPF_LAUNCH("k_block_sums", s, k_block_sums<<<nb, 1024, 0, s>>>(N, v, blk));
  RPF_LAUNCH("k_scan_blocks", s, k_scan_blocks<<<1, 1024, 0, s>>>(blk, nb, total));
  RPF_LAUNCH("k_scan_apply", s, k_scan_apply<<<nb, 1024, 0, s>>>(N, v, blk, out));
}
