// rpf_static.cu -- rpf_query_static: the query path of rpf_query with its
// scratch in a fixed device array instead of a caller workspace or a
// stream-ordered allocation.
//
// It exists for callers that must not allocate device memory once they are
// running: a serving process that has handed the rest of HBM to its own pool,
// or a latency-critical thread for which a device allocation (and the
// synchronisation it may imply) is not acceptable.  Such a caller can answer
// queries with memory it already owns (Q, idx, dist) and nothing else.
//
// The scratch is one file-scope __device__ array per device (its backing is
// set up by the CUDA runtime when this module is loaded, not by this call).
// The first call on a device, with that device current, looks the array up
// with cudaGetSymbolAddress and caches the address; later calls on the
// device only reuse it.  The cache does not survive a device reset
// (cudaDeviceReset, or the primary context released and created again): the
// array may then live at another address, so a process that resets a device
// must not call rpf_query_static on it afterwards.
#include <cuda_runtime.h>

#include <mutex>

#include "rpf_internal.cuh"

// The scratch itself: file scope, one copy per device that loads the library,
// held until the process exits.  In host code this name is only a stand-in;
// kernels get the device address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_query_scratch[RPF_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

void* rpf_static_scratch(int* rc) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *rc = rpf_cuda_err(e);
    return nullptr;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *rc = RPF_EINVAL;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_query_scratch);
    if (e != cudaSuccess) {
      *rc = rpf_cuda_err(e);
      return nullptr;
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

extern "C" int rpf_query_static(const rpf_forest* f, const float* Q, int64_t m, int32_t K,
                                int32_t* idx, float* dist, void* stream) {
  if (!f || K < 1 || K > RPF_MAX_K || m < 0) return RPF_EINVAL;
  if (m == 0) return RPF_OK;
  if (!Q || !idx || !dist) return RPF_EINVAL;
  // error word, leaf id per (query, tree), T per-tree candidate lists of K
  if (rpf_query_core_ws(m, f->prm.n_trees, K) > (size_t)RPF_STATIC_SCRATCH_BYTES)
    return RPF_EINVAL;
  if (!rpf_is_device_ptr(Q) || !rpf_is_device_ptr(idx) || !rpf_is_device_ptr(dist))
    return RPF_EINVAL;
  int dev = -1;
  RPF_CU(cudaGetDevice(&dev));
  if (dev != f->device) return RPF_EINVAL;
  int rc = RPF_OK;
  void* ws = rpf_static_scratch(&rc);
  if (!ws) return rc;
  return rpf_query_dev(f, Q, m, K, idx, dist, ws, (size_t)RPF_STATIC_SCRATCH_BYTES,
                       (cudaStream_t)stream);
}
