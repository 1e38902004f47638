// rpf_probe.cu -- the row-gather ceiling of the growth kernels.
//
// The growth kernels read whole rows of X in the order of a tree's
// permutation: random rows, each read once per level, served from L2 when X
// fits there.  k_gather_probe reads rows the same way with nothing else to
// do: d / 4 lanes (at most 32) take one row as one coalesced read of 16
// bytes per lane (four rows per lane in flight), the row index is a
// multiplicative hash of the row's position (a fixed pseudo-random order),
// and every lane sums what it reads so that nothing is dropped.  Its rate
// (bytes of rows per second) is the ceiling against which the growth
// kernels' algorithmic bytes are compared.
#include <cuda_runtime.h>

#include "rpf_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) k_gather_probe(const float* __restrict__ X, int64_t n,
                                                      int d, int64_t rows, int64_t seed,
                                                      float* out) {
  const int lpr = min(32, d / 4);     // lanes per row
  const int rpw = 32 / lpr;           // rows per warp instruction
  const int lane = threadIdx.x & 31;
  const int sub = lane / lpr, c4 = 4 * (lane % lpr);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const uint32_t nn = n < 0xffffffffll ? (uint32_t)n : 0xffffffffu;
  // four rows per lane in flight; row = the high word of hash(pos) * n
  for (int64_t r0 = warp * 4 * rpw; r0 < rows; r0 += nwarp * 4 * rpw) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t pos = r0 + u * rpw + sub;
      v[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (sub < rpw && pos < rows) {
        const uint32_t h = (uint32_t)(pos + seed) * 2654435761u;
        const int64_t row = (int64_t)(((uint64_t)h * nn) >> 32);
        const float* src = X + row * d;
        for (int k = c4; k < d; k += 4 * lpr) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(src + k));
          v[u].x += t.x;
          v[u].y += t.y;
          v[u].z += t.z;
          v[u].w += t.w;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc.x += v[u].x;
      acc.y += v[u].y;
      acc.z += v[u].z;
      acc.w += v[u].w;
    }
  }
  const float s = acc.x + acc.y + acc.z + acc.w;
  if (s == 1.2345678e30f) out[0] = s;  // keeps the loads; never taken in practice
}

}  // namespace

extern "C" int rpf_gather_probe(const float* X, int64_t n, int32_t d, int64_t rows,
                                int64_t seed, float* out, void* stream) {
  if (!X || !out || n < 1 || d < 4 || (d & 3) != 0 || rows < 0) return RPF_EINVAL;
  if (((uintptr_t)X & 15) != 0) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, n_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  RPF_LAUNCH("k_gather_probe", s,
             k_gather_probe<<<(unsigned)(8 * n_sm), 256, 0, s>>>(X, n, d, rows, seed, out));
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}
