// rpf_api.cu -- the C ABI declared in include/rpforest.h: argument checks,
// staging of host buffers through device memory, forest lifetime.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <atomic>

#include "rpf_allknn.cuh"
#include "rpf_internal.cuh"
#include "rpf_tma.cuh"

namespace {
// limit of every bounded device wait, nanoseconds (0 = the default)
constexpr uint64_t kDefaultWaitNs = 2000000000ull;
std::atomic<uint64_t> g_wait_ns{kDefaultWaitNs};
// allocation-failure injection: allocations left before one fails (-1 = off)
std::atomic<int64_t> g_fail_after{-1};
}  // namespace

uint64_t rpf_wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

int rpf_cuda_err(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return RPF_ENOMEM;
  return RPF_ECUDA;
}

bool rpf_is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int rpf_alloc(void** p, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static bool tuned[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> g(mu);
    if (!tuned[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      cudaGetLastError();
      tuned[dev] = true;
    }
  }
  *p = nullptr;
  if (g_fail_after.load() >= 0 && g_fail_after.fetch_sub(1) == 0) {
    g_fail_after.store(-1);  // one injected failure, then normal service
    return RPF_ENOMEM;
  }
  if (cudaMallocAsync(p, std::max<size_t>(bytes, 256), s) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return RPF_ENOMEM;
  }
  return RPF_OK;
}

void rpf_release(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

namespace {

template <typename T>
int dalloc(rpf_forest* f, T** p, size_t count, cudaStream_t s) {
  void* q = nullptr;
  int rc = rpf_alloc(&q, count * sizeof(T), s);
  if (rc) return rc;
  f->owned.push_back(q);
  *p = (T*)q;
  return RPF_OK;
}

// The forest's memory is released in stream order on the legacy stream:
// callers make sure no work that uses the forest is still in flight.
void free_forest(rpf_forest* f) {
  if (!f) return;
  for (void* p : f->owned) rpf_release(p, 0);
  void* ps[] = {f->node_key,  f->node_tree,  f->node_begin, f->node_len,  f->node_left,
                f->node_right, f->node_jstar, f->node_flag, f->node_c,    f->node_route,
                f->node_dir32, f->leaf_tree,  f->leaf_begin, f->leaf_len, f->tile_cnt,
                f->tile_off,  f->tile_leaf,  f->stage,      f->pk_tiles, f->pk_bits,
                f->X16};
  for (void* p : ps) rpf_release(p, 0);
  delete f;
}

// Node table of a forest grown in two parts (rpf_add_trees): part A (T trees,
// Na nodes, roots at ids 0..T-1) and part B (dT trees, roots at ids
// 0..dT-1).  Routing starts tree t at node t, so the merged table puts the
// roots first: A's roots, B's roots, then A's other nodes, then B's.
__device__ __forceinline__ int64_t merged_id(int64_t i, bool is_b, int T, int dT, int64_t Na) {
  if (!is_b) return i < T ? i : i + dT;
  return i < dT ? T + i : Na + i;
}

__global__ void k_merge_nodes(int64_t N, int is_b, int T, int dT, int64_t Na, int d,
                              const uint64_t* key, const int32_t* tree, const int32_t* begin,
                              const int32_t* len, const int32_t* left, const int32_t* right,
                              const int32_t* jstar, const int32_t* flag, const double* c,
                              const float* dir32, uint64_t* okey,
                              int32_t* otree, int32_t* obegin, int32_t* olen, int32_t* oleft,
                              int32_t* oright, int32_t* ojstar, int32_t* oflag, double* oc,
                              float* odir32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t o = merged_id(i, is_b != 0, T, dT, Na);
  okey[o] = key[i];
  otree[o] = tree[i] + (is_b ? T : 0);
  obegin[o] = begin[i];
  olen[o] = len[i];
  oleft[o] = left[i] >= 0 ? (int32_t)merged_id(left[i], is_b != 0, T, dT, Na) : -1;
  oright[o] = right[i] >= 0 ? (int32_t)merged_id(right[i], is_b != 0, T, dT, Na) : -1;
  ojstar[o] = jstar[i];
  oflag[o] = flag[i];
  oc[o] = c[i];
  for (int k = 0; k < d; ++k) odir32[o * d + k] = dir32[i * d + k];
}

__global__ void k_shift_tree(int64_t N, int add, const int32_t* in, int32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = in[i] + add;
}

// One bounded wait on a barrier that nothing completes: no thread arrives on
// it and no copy is posted to it, so nothing is in flight when the wait gives
// up and the kernel returns.
__global__ void k_wait_selftest(uint64_t wlim, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) rpf_mbar_init(&bar, 1);
  __syncthreads();
  rpf_mbar_wait(&bar, 0, err, wlim);
}

}  // namespace

extern "C" {

void rpf_default_params(rpf_params* p) {
  if (!p) return;
  p->n_trees = 10;
  p->leaf_max = 50;
  p->n_try = 5;
  p->split_rule = 0;
  p->form = 0;
  p->growth = 0;
  p->seed = 0;
}

void rpf_set_wait_limit(uint64_t limit_ns) {
  g_wait_ns.store(limit_ns ? limit_ns : kDefaultWaitNs);
}

int rpf_wait_selftest(uint64_t limit_ns, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int* d_err = nullptr;
  int rc = rpf_alloc((void**)&d_err, sizeof(int), s);
  if (rc) return rc;
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    RPF_LAUNCH("k_wait_selftest", s, k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, d_err));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  rpf_release(d_err, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return rpf_cuda_err(e);
  return h ? h : RPF_OK;
}

void rpf_debug_fail_alloc(int64_t after) { g_fail_after.store(after < 0 ? -1 : after); }

int rpf_query_status(const void* scratch, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const void* w = scratch;
  if (!w) {
    int rc = RPF_OK;
    w = rpf_static_scratch(&rc);
    if (!w) return rc;
  } else if (!rpf_is_device_ptr(w)) {
    return RPF_EINVAL;
  }
  int h = 0;
  RPF_CU(cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, s));
  RPF_CU(cudaStreamSynchronize(s));
  return h ? h : RPF_OK;
}

const char* rpf_error_string(int code) {
  switch (code) {
    case RPF_OK: return "success";
    case RPF_EINVAL: return "invalid argument";
    case RPF_ENOMEM: return "out of memory";
    case RPF_ECUDA: return "CUDA error";
    case RPF_ETIMEOUT: return "device wait timed out";
    case RPF_EINTERNAL: return "internal error";
    default: return "unknown error";
  }
}

}  // extern "C"

namespace {
// Grow trees t_base .. t_base + p->n_trees - 1 of the ensemble (every draw of
// tree t is keyed by its global index).
int build_impl(const float* X, int64_t n, int32_t d, const rpf_params* p, int32_t t_base,
               void* stream, rpf_forest** out) {
  if (!out) return RPF_EINVAL;
  *out = nullptr;
  if (!X || !p || n < 1 || d < 1 || d > RPF_MAX_D) return RPF_EINVAL;
  if (t_base < 0 || (int64_t)t_base + p->n_trees > (1 << 20)) return RPF_EINVAL;
  if (p->n_trees < 1 || p->leaf_max < 1 || p->leaf_max > RPF_MAX_LEAF || p->n_try < 1 || p->n_try > RPF_MAX_TRY) return RPF_EINVAL;
  if (p->split_rule < 0 || p->split_rule > 1 || p->form < 0 || p->form > 1 || p->growth < 0 || p->growth > 2)
    return RPF_EINVAL;
  if (n * (int64_t)p->n_trees >= ((int64_t)1 << 31)) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  rpf_forest* f = new (std::nothrow) rpf_forest();
  if (!f) return RPF_ENOMEM;
  f->n = n;
  f->d = d;
  f->prm = *p;
  f->t_base = t_base;
  if (f->prm.growth == 0) f->prm.growth = 2;
  // the G-B projection kernel stages nTry x d FP32 directions in shared memory
  if (f->prm.growth == 2 && (size_t)p->n_try * d * 4 + 2048 > 200 * 1024) f->prm.growth = 1;
  cudaGetDevice(&f->device);
  int rc;
  if ((rc = dalloc(f, &f->X, (size_t)n * d, s)) || (rc = dalloc(f, &f->xnorm, (size_t)n, s)) ||
      (rc = dalloc(f, &f->perm, (size_t)n * p->n_trees, s)) || (rc = dalloc(f, &f->d_err, 1, s)) ||
      (rc = dalloc(f, &f->d_fallback, 1, s))) {
    free_forest(f);
    return rc;
  }
  cudaError_t e = cudaMemsetAsync(f->d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->d_fallback, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->X, X, sizeof(float) * n * d, cudaMemcpyDefault, s);
  if (e != cudaSuccess) {
    free_forest(f);
    return rpf_cuda_err(e);
  }
  if ((rc = rpf_grow(f, s)) || (rc = rpf_build_tiles(f, s)) ||
      (f->prm.form == 1 && (rc = rpf_build_packs(f, s))) ||
      (f->prm.form == 1 && (rc = rpf_build_x16(f, s)))) {
    free_forest(f);
    return rc;
  }
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    free_forest(f);
    return rpf_cuda_err(e);
  }
  *out = f;
  return RPF_OK;
}
}  // namespace

extern "C" {

int rpf_build(const float* X, int64_t n, int32_t d, const rpf_params* p, void* stream,
              rpf_forest** out) {
  return build_impl(X, n, d, p, 0, stream, out);
}

int rpf_build_shard(const float* X, int64_t n, int32_t d, const rpf_params* p,
                    int32_t tree_first, void* stream, rpf_forest** out) {
  return build_impl(X, n, d, p, tree_first, stream, out);
}

void rpf_free(rpf_forest* f) { free_forest(f); }

int rpf_set_form(rpf_forest* f, int32_t form, void* stream) {
  if (!f || form < 0 || form > 1) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = RPF_OK;
  if (form == 1 && !f->pk_tiles) rc = rpf_build_packs(f, s);
  if (!rc && form == 1 && !f->X16) rc = rpf_build_x16(f, s);
  if (rc) return rc;
  f->prm.form = form;
  RPF_CU(cudaStreamSynchronize(s));
  return RPF_OK;
}

int rpf_set_query_scan(rpf_forest* f, int32_t mode) {
  if (!f || mode < -1 || mode > 1) return RPF_EINVAL;
  f->qscan_mode = mode;
  return RPF_OK;
}

int rpf_autotune(rpf_forest* f, int32_t K, void* stream, int32_t* chosen) {
  if (!f || K < 1 || K > RPF_MAX_K) return RPF_EINVAL;
  return rpf_tc_autotune(f, K, (cudaStream_t)stream, chosen);
}

int rpf_add_trees(rpf_forest* f, int32_t n_new, void* stream) {
  if (!f || n_new < 1) return RPF_EINVAL;
  const int T = f->prm.n_trees;
  const int64_t n = f->n;
  const int d = f->d;
  if ((int64_t)(T + n_new) * n >= ((int64_t)1 << 31) || T + n_new > (1 << 20)) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // the new trees grow in a temporary forest over the same points (X and
  // the norms borrowed, not owned), their draws keyed by T + t
  rpf_forest* g = new rpf_forest();
  g->n = n;
  g->d = d;
  g->prm = f->prm;
  g->prm.n_trees = n_new;
  g->device = f->device;
  g->t_base = f->t_base + T;
  g->X = f->X;
  g->xnorm = f->xnorm;
  g->d_err = f->d_err;
  g->d_fallback = f->d_fallback;
  int rc = dalloc(g, &g->perm, (size_t)n * n_new, s);
  if (!rc) rc = rpf_grow(g, s);
  if (rc) {
    g->X = nullptr;
    free_forest(g);
    return rc;
  }
  // merged permutation and node / leaf tables
  const int64_t Na = f->n_nodes, Nb = g->n_nodes, N = Na + Nb;
  const int64_t La = f->n_leaves, Lb = g->n_leaves;
  int32_t* perm = nullptr;
  uint64_t* key = nullptr;
  int32_t *tree = nullptr, *begin = nullptr, *len = nullptr, *left = nullptr, *right = nullptr,
          *jstar = nullptr, *flag = nullptr, *ltree = nullptr, *lbegin = nullptr, *llen = nullptr;
  double* c = nullptr;
  float* dir32 = nullptr;
  void** bufs[] = {(void**)&perm, (void**)&key, (void**)&tree, (void**)&begin, (void**)&len,
                   (void**)&left, (void**)&right, (void**)&jstar, (void**)&flag, (void**)&c,
                   (void**)&dir32, (void**)&ltree, (void**)&lbegin, (void**)&llen};
  const size_t sizes[] = {4 * (size_t)(T + n_new) * n, 8 * (size_t)N, 4 * (size_t)N,
                          4 * (size_t)N, 4 * (size_t)N, 4 * (size_t)N, 4 * (size_t)N,
                          4 * (size_t)N, 4 * (size_t)N, 8 * (size_t)N,
                          4 * (size_t)N * d, 4 * (size_t)(La + Lb), 4 * (size_t)(La + Lb),
                          4 * (size_t)(La + Lb)};
  for (int i = 0; i < 14 && !rc; ++i) rc = rpf_alloc(bufs[i], sizes[i], s);
  if (rc) {
    for (auto b : bufs) rpf_release(*b, s);
    g->X = nullptr;
    free_forest(g);
    return RPF_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(perm, f->perm, 4 * (size_t)T * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(perm + (size_t)T * n, g->perm, 4 * (size_t)n_new * n,
                        cudaMemcpyDeviceToDevice, s);
  const rpf_forest* parts[2] = {f, g};
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    const rpf_forest* q = parts[b];
    const int64_t Nq = q->n_nodes;
    if (Nq > 0) {
      k_merge_nodes<<<(unsigned)((Nq + 127) / 128), 128, 0, s>>>(
          Nq, b, T, n_new, Na, d, q->node_key, q->node_tree, q->node_begin, q->node_len,
          q->node_left, q->node_right, q->node_jstar, q->node_flag, q->node_c,
          q->node_dir32, key, tree, begin, len, left, right, jstar, flag, c, dir32);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && La > 0)
    e = cudaMemcpyAsync(ltree, f->leaf_tree, 4 * (size_t)La, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && Lb > 0) {
    k_shift_tree<<<(unsigned)((Lb + 255) / 256), 256, 0, s>>>(Lb, T, g->leaf_tree, ltree + La);
    e = cudaGetLastError();
  }
  const int32_t* lsrc[2][2] = {{f->leaf_begin, f->leaf_len}, {g->leaf_begin, g->leaf_len}};
  if (e == cudaSuccess && La > 0) e = cudaMemcpyAsync(lbegin, lsrc[0][0], 4 * (size_t)La, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && La > 0) e = cudaMemcpyAsync(llen, lsrc[0][1], 4 * (size_t)La, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && Lb > 0) e = cudaMemcpyAsync(lbegin + La, lsrc[1][0], 4 * (size_t)Lb, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && Lb > 0) e = cudaMemcpyAsync(llen + La, lsrc[1][1], 4 * (size_t)Lb, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    for (auto b : bufs) rpf_release(*b, s);
    g->X = nullptr;
    free_forest(g);
    return rpf_cuda_err(e);
  }
  // install: the old tables go back to the pool, the tile layouts are rebuilt
  for (auto& o : f->owned)
    if (o == f->perm) o = perm;
  void* olds[] = {f->perm, f->node_key, f->node_tree, f->node_begin, f->node_len, f->node_left,
                  f->node_right, f->node_jstar, f->node_flag, f->node_c, f->node_route,
                  f->node_dir32, f->leaf_tree, f->leaf_begin, f->leaf_len, f->tile_cnt,
                  f->tile_off, f->tile_leaf, f->pk_tiles, f->pk_bits};
  for (void* o : olds) rpf_release(o, s);
  f->perm = perm;
  f->node_key = key;
  f->node_tree = tree;
  f->node_begin = begin;
  f->node_len = len;
  f->node_left = left;
  f->node_right = right;
  f->node_jstar = jstar;
  f->node_flag = flag;
  f->node_c = c;
  f->node_route = nullptr;
  f->node_dir32 = dir32;
  f->leaf_tree = ltree;
  f->leaf_begin = lbegin;
  f->leaf_len = llen;
  f->tile_cnt = f->tile_off = f->tile_leaf = nullptr;
  f->pk_tiles = nullptr;
  f->pk_bits = nullptr;
  f->n_nodes = f->nodes_cap = N;
  f->n_leaves = La + Lb;
  f->n_exact += g->n_exact;
  f->max_depth = std::max(f->max_depth, g->max_depth);
  f->prm.n_trees = T + n_new;
  g->X = nullptr;
  g->xnorm = nullptr;
  free_forest(g);  // its own tables only (X, norms and error words are f's)
  if ((rc = rpf_build_route(f, s)) || (rc = rpf_build_tiles(f, s)) ||
      (f->prm.form == 1 && (rc = rpf_build_packs(f, s))))
    return rc;
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? RPF_OK : rpf_cuda_err(e);
}

size_t rpf_workspace_bytes(const rpf_forest* f, int64_t m, int32_t K, int32_t for_all_knn) {
  if (!f || K < 1 || K > RPF_MAX_K || m < 0) return 0;
  return for_all_knn ? rpf_all_knn_ws(f, K) : rpf_query_ws(f, m, K);
}

int rpf_all_knn(rpf_forest* f, int32_t K, int32_t* idx, float* dist, void* workspace,
                size_t ws_bytes, void* stream) {
  if (!f) return RPF_EINVAL;
  return rpf_all_knn_trees(f, f->prm.n_trees, K, idx, dist, workspace, ws_bytes, stream);
}

int rpf_all_knn_trees(rpf_forest* f, int32_t n_trees, int32_t K, int32_t* idx, float* dist,
                      void* workspace, size_t ws_bytes, void* stream) {
  if (!f || !idx || !dist || K < 1 || K > RPF_MAX_K) return RPF_EINVAL;
  if (n_trees < 1 || n_trees > f->prm.n_trees) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = f->n;
  const bool dev_out = rpf_is_device_ptr(idx) && rpf_is_device_ptr(dist);
  int32_t* di = idx;
  float* dd = dist;
  if (!dev_out) {
    const size_t need = (size_t)n * K * 8;
    if (f->stage_bytes < need) {
      rpf_release(f->stage, s);
      f->stage = nullptr;
      f->stage_bytes = 0;
      if (rpf_alloc(&f->stage, need, s)) return RPF_ENOMEM;
      f->stage_bytes = need;
    }
    di = (int32_t*)f->stage;
    dd = (float*)((char*)f->stage + (size_t)n * K * 4);
  }
  void* ws = workspace;
  size_t wsb = ws_bytes;
  bool own_ws = false;
  if (!ws) {
    wsb = rpf_all_knn_ws(f, K);
    if (rpf_alloc(&ws, wsb, s)) return RPF_ENOMEM;
    own_ws = true;
  }
  int rc = rpf_all_knn_dev(f, n_trees, K, di, dd, ws, wsb, s);
  if (own_ws) rpf_release(ws, s);
  if (rc) return rc;
  if (!dev_out) {
    RPF_CU(cudaMemcpyAsync(idx, di, (size_t)n * K * 4, cudaMemcpyDefault, s));
    RPF_CU(cudaMemcpyAsync(dist, dd, (size_t)n * K * 4, cudaMemcpyDefault, s));
    RPF_CU(cudaStreamSynchronize(s));
  }
  RPF_CU(cudaGetLastError());
  return RPF_OK;
}

int rpf_all_knn_async(rpf_forest* f, int32_t K, int32_t* idx, float* dist, void* workspace,
                      size_t ws_bytes, void* stream) {
  if (!f || !idx || !dist || !workspace || K < 1 || K > RPF_MAX_K) return RPF_EINVAL;
  if (!rpf_is_device_ptr(idx) || !rpf_is_device_ptr(dist) || !rpf_is_device_ptr(workspace))
    return RPF_EINVAL;
  if (ws_bytes < rpf_all_knn_ws(f, K)) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  RPF_CU(cudaMemsetAsync(f->d_err, 0, sizeof(int), s));
  const int rc = rpf_all_knn_enqueue(f, f->prm.n_trees, K, idx, dist,
                                     (char*)workspace + RPF_QERR_BYTES,
                                     ws_bytes - RPF_QERR_BYTES, s, nullptr);
  if (rc) return rc;
  // this call's outcome, for rpf_query_status(workspace, stream)
  RPF_CU(cudaMemcpyAsync(workspace, f->d_err, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return RPF_OK;
}

int rpf_all_knn_keys(rpf_forest* f, int32_t K, int32_t* keys, void* workspace, size_t ws_bytes,
                     void* stream) {
  if (!f || !keys || K < 1 || K > RPF_MAX_K) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = f->n;
  const bool dev_out = rpf_is_device_ptr(keys);
  const size_t need = (size_t)n * K * 8;
  void* ws = workspace;
  size_t wsb = ws_bytes;
  bool own_ws = false;
  if (!ws) {
    wsb = rpf_all_knn_ws(f, K);
    if (rpf_alloc(&ws, wsb, s)) return RPF_ENOMEM;
    own_ws = true;
  }
  void* kd = keys;
  if (!dev_out && rpf_alloc(&kd, need, s)) {
    if (own_ws) rpf_release(ws, s);
    return RPF_ENOMEM;
  }
  int rc = rpf_all_knn_dev(f, f->prm.n_trees, K, nullptr, nullptr, ws, wsb, s, (uint2*)kd);
  cudaError_t e = cudaSuccess;
  if (!rc && !dev_out) e = cudaMemcpyAsync(keys, kd, need, cudaMemcpyDefault, s);
  if (own_ws) rpf_release(ws, s);
  if (!dev_out) rpf_release(kd, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return rpf_cuda_err(e);
  return rc;
}

int rpf_merge_keys(int64_t n, int32_t K, int32_t n_lists, const int32_t* lists, int32_t* idx,
                   float* dist, void* stream) {
  if (n < 0 || K < 1 || K > RPF_MAX_K || n_lists < 1) return RPF_EINVAL;
  if (n == 0) return RPF_OK;
  if (!lists || !idx || !dist) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t lb = (size_t)n_lists * n * K * 8, ob = (size_t)n * K * 4;
  const bool ld = rpf_is_device_ptr(lists);
  const bool od = rpf_is_device_ptr(idx) && rpf_is_device_ptr(dist);
  auto a256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bl = ld ? 0 : a256(lb), bo = od ? 0 : 2 * a256(ob);
  char* w = nullptr;
  if (bl + bo && rpf_alloc((void**)&w, bl + bo, s)) return RPF_ENOMEM;
  const int32_t* L = ld ? lists : (const int32_t*)w;
  int32_t* I = od ? idx : (int32_t*)(w + bl);
  float* D = od ? dist : (float*)(w + bl + bo / 2);
  cudaError_t e = cudaSuccess;
  if (!ld) e = cudaMemcpyAsync((void*)L, lists, lb, cudaMemcpyDefault, s);
  int rc = RPF_OK;
  if (e == cudaSuccess) rc = rpf_merge_dev(n, K, n_lists, (const uint2*)L, I, D, s);
  if (e == cudaSuccess && !rc && !od) {
    e = cudaMemcpyAsync(idx, I, ob, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dist, D, ob, cudaMemcpyDefault, s);
  }
  rpf_release(w, s);
  if (e == cudaSuccess && !od) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return rpf_cuda_err(e);
  return rc;
}

int rpf_query(const rpf_forest* f, const float* Q, int64_t m, int32_t K, int32_t* idx,
              float* dist, void* workspace, size_t ws_bytes, void* stream) {
  if (!f || K < 1 || K > RPF_MAX_K || m < 0) return RPF_EINVAL;
  if (m == 0) return RPF_OK;
  if (!Q || !idx || !dist) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int T = f->prm.n_trees;
  const size_t need = rpf_query_ws(f, m, K);
  void* ws = workspace;
  bool own_ws = false;
  if (!ws) {
    if (rpf_alloc(&ws, need, s)) return RPF_ENOMEM;
    own_ws = true;
  } else if (ws_bytes < need) {
    return RPF_EINVAL;
  }
  auto a256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* w = (char*)ws;
  const size_t core = rpf_query_core_ws(m, T, K);
  float* dQ = (float*)(w + core);
  int32_t* di = (int32_t*)(w + core + a256((size_t)m * f->d * 4));
  float* dd = (float*)(w + core + a256((size_t)m * f->d * 4) + a256((size_t)m * K * 4));
  const bool q_dev = rpf_is_device_ptr(Q);
  const bool o_dev = rpf_is_device_ptr(idx) && rpf_is_device_ptr(dist);
  int rc = RPF_OK;
  cudaError_t e = cudaSuccess;
  if (!q_dev) e = cudaMemcpyAsync(dQ, Q, (size_t)m * f->d * 4, cudaMemcpyDefault, s);
  if (e == cudaSuccess) {
    rc = rpf_query_dev(f, q_dev ? Q : dQ, m, K, o_dev ? idx : di, o_dev ? dist : dd, ws, core, s);
    if (!rc && !o_dev) {
      e = cudaMemcpyAsync(idx, di, (size_t)m * K * 4, cudaMemcpyDefault, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dist, dd, (size_t)m * K * 4, cudaMemcpyDefault, s);
    }
  }
  // the call's error word (first bytes of the scratch) is read whenever the
  // call synchronises: host outputs, or a scratch the library allocated
  const bool sync = !o_dev || own_ws;
  int herr = 0;
  if (sync && e == cudaSuccess && !rc)
    e = cudaMemcpyAsync(&herr, ws, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (own_ws) rpf_release(ws, s);
  if (sync && e == cudaSuccess && !rc) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return rpf_cuda_err(e);
  if (rc) return rc;
  return herr ? herr : RPF_OK;
}

int rpf_forest_info(const rpf_forest* f, int64_t* n, int32_t* d, int32_t* n_trees,
                    int64_t* n_nodes, int64_t* n_leaves, int32_t* max_depth,
                    int64_t* n_exact_nodes) {
  if (!f) return RPF_EINVAL;
  if (n) *n = f->n;
  if (d) *d = f->d;
  if (n_trees) *n_trees = f->prm.n_trees;
  if (n_nodes) *n_nodes = f->n_nodes;
  if (n_leaves) *n_leaves = f->n_leaves;
  if (max_depth) *max_depth = f->max_depth;
  if (n_exact_nodes) *n_exact_nodes = f->n_exact;
  return RPF_OK;
}

int rpf_forest_counters(const rpf_forest* f, int64_t* out, int32_t n_out) {
  if (!f || !out || n_out < 0) return RPF_EINVAL;
  unsigned long long fb = 0;
  RPF_CU(cudaMemcpy(&fb, f->d_fallback, sizeof(fb), cudaMemcpyDeviceToHost));
  const int64_t v[5] = {f->n_exact, (int64_t)fb, f->max_depth, f->tile_region, f->plain_groups};
  for (int i = 0; i < n_out && i < 5; ++i) out[i] = v[i];
  return RPF_OK;
}

int rpf_forest_perm(const rpf_forest* f, int32_t t, int32_t* perm_host) {
  if (!f || !perm_host || t < 0 || t >= f->prm.n_trees) return RPF_EINVAL;
  RPF_CU(cudaMemcpy(perm_host, f->perm + (int64_t)t * f->n, sizeof(int32_t) * f->n,
                    cudaMemcpyDefault));
  return RPF_OK;
}

int rpf_forest_leaves(const rpf_forest* f, int32_t* tree, int32_t* begin, int32_t* len) {
  if (!f) return RPF_EINVAL;
  const size_t b = sizeof(int32_t) * f->n_leaves;
  if (tree) RPF_CU(cudaMemcpy(tree, f->leaf_tree, b, cudaMemcpyDefault));
  if (begin) RPF_CU(cudaMemcpy(begin, f->leaf_begin, b, cudaMemcpyDefault));
  if (len) RPF_CU(cudaMemcpy(len, f->leaf_len, b, cudaMemcpyDefault));
  return RPF_OK;
}

int rpf_forest_nodes(const rpf_forest* f, uint64_t* key, int32_t* tree, int32_t* begin,
                     int32_t* len, int32_t* left, int32_t* right, int32_t* jstar, int32_t* flag,
                     double* c) {
  if (!f) return RPF_EINVAL;
  const size_t nn = (size_t)f->n_nodes;
  if (key) RPF_CU(cudaMemcpy(key, f->node_key, 8 * nn, cudaMemcpyDefault));
  if (tree) RPF_CU(cudaMemcpy(tree, f->node_tree, 4 * nn, cudaMemcpyDefault));
  if (begin) RPF_CU(cudaMemcpy(begin, f->node_begin, 4 * nn, cudaMemcpyDefault));
  if (len) RPF_CU(cudaMemcpy(len, f->node_len, 4 * nn, cudaMemcpyDefault));
  if (left) RPF_CU(cudaMemcpy(left, f->node_left, 4 * nn, cudaMemcpyDefault));
  if (right) RPF_CU(cudaMemcpy(right, f->node_right, 4 * nn, cudaMemcpyDefault));
  if (jstar) RPF_CU(cudaMemcpy(jstar, f->node_jstar, 4 * nn, cudaMemcpyDefault));
  if (flag) RPF_CU(cudaMemcpy(flag, f->node_flag, 4 * nn, cudaMemcpyDefault));
  if (c) RPF_CU(cudaMemcpy(c, f->node_c, 8 * nn, cudaMemcpyDefault));
  return RPF_OK;
}

int rpf_directions(uint64_t seed, int32_t t, const uint64_t* keys_host, int32_t n_keys, int32_t j,
                   int32_t d, double* out, void* stream) {
  if (!keys_host || !out || n_keys < 0 || d < 1 || d > RPF_MAX_D || j < 0) return RPF_EINVAL;
  if (n_keys == 0) return RPF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t* dk = nullptr;
  double* dout = nullptr;
  if (rpf_alloc((void**)&dk, 8 * (size_t)n_keys, s)) return RPF_ENOMEM;
  const bool o_dev = rpf_is_device_ptr(out);
  if (!o_dev && rpf_alloc((void**)&dout, 8 * (size_t)n_keys * d, s)) {
    rpf_release(dk, s);
    return RPF_ENOMEM;
  }
  RPF_CU(cudaMemcpyAsync(dk, keys_host, 8 * (size_t)n_keys, cudaMemcpyDefault, s));
  rpf_launch_directions(seed, t, dk, n_keys, j, d, o_dev ? out : dout, s);
  RPF_CU(cudaGetLastError());
  if (!o_dev) RPF_CU(cudaMemcpyAsync(out, dout, 8 * (size_t)n_keys * d, cudaMemcpyDefault, s));
  rpf_release(dk, s);
  rpf_release(dout, s);
  RPF_CU(cudaStreamSynchronize(s));
  return RPF_OK;
}

int rpf_brute_knn(const float* X, int64_t n, int32_t d, const float* Q, int64_t m,
                  const int32_t* self, int32_t K, int32_t* idx, float* dist, void* stream) {
  if (!X || n < 1 || d < 1 || d > RPF_MAX_D || m < 0 || K < 1 || K > RPF_MAX_K) return RPF_EINVAL;
  if (m == 0) return RPF_OK;
  if (!Q || !idx || !dist || n >= ((int64_t)1 << 31)) return RPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // stage host buffers through one stream-ordered device block
  const bool xd = rpf_is_device_ptr(X), qd = rpf_is_device_ptr(Q);
  const bool sd = !self || rpf_is_device_ptr(self);
  const bool od = rpf_is_device_ptr(idx) && rpf_is_device_ptr(dist);
  auto a256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bx = xd ? 0 : a256((size_t)n * d * 4), bq = qd ? 0 : a256((size_t)m * d * 4);
  const size_t bs = sd ? 0 : a256((size_t)m * 4), bo = od ? 0 : 2 * a256((size_t)m * K * 4);
  char* w = nullptr;
  if (bx + bq + bs + bo) {
    if (rpf_alloc((void**)&w, bx + bq + bs + bo, s)) return RPF_ENOMEM;
  }
  const float* Xd = xd ? X : (const float*)w;
  const float* Qd = qd ? Q : (const float*)(w + bx);
  const int32_t* Sd = sd ? self : (const int32_t*)(w + bx + bq);
  int32_t* Id = od ? idx : (int32_t*)(w + bx + bq + bs);
  float* Dd = od ? dist : (float*)(w + bx + bq + bs + bo / 2);
  cudaError_t e = cudaSuccess;
  if (!xd) e = cudaMemcpyAsync((void*)Xd, X, (size_t)n * d * 4, cudaMemcpyDefault, s);
  if (e == cudaSuccess && !qd) e = cudaMemcpyAsync((void*)Qd, Q, (size_t)m * d * 4, cudaMemcpyDefault, s);
  if (e == cudaSuccess && !sd) e = cudaMemcpyAsync((void*)Sd, self, (size_t)m * 4, cudaMemcpyDefault, s);
  int rc = RPF_OK;
  if (e == cudaSuccess) rc = rpf_brute_dev(Xd, n, d, Qd, m, Sd, K, Id, Dd, s);
  if (e == cudaSuccess && !rc && !od) {
    e = cudaMemcpyAsync(idx, Id, (size_t)m * K * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dist, Dd, (size_t)m * K * 4, cudaMemcpyDefault, s);
  }
  rpf_release(w, s);
  if (e == cudaSuccess && !od) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return rpf_cuda_err(e);
  return rc;
}

}  // extern "C"
