// rpf_trace.cu -- launch accounting and optional per-kernel CUDA-event timing.
//
// Every kernel launch of the library goes through RPF_LAUNCH(name, stream, ...),
// which counts it; when tracing is on, an event pair is recorded around it on
// the launching stream and rpf_trace_read sums the elapsed times per kernel.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rpf_internal.cuh"

namespace {

struct Rec {
  int name;
  cudaEvent_t a, b;
};

struct Registry {
  std::mutex mu;
  std::map<std::string, int> index;
  std::vector<std::string> names;
  std::vector<long long> launches;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  bool on = false;
  long long total = 0;
};

Registry& reg() {
  static Registry* r = new Registry();  // never destroyed: safe at process exit
  return *r;
}

int name_id(Registry& r, const char* name) {
  auto it = r.index.find(name);
  if (it != r.index.end()) return it->second;
  const int id = (int)r.names.size();
  r.index.emplace(name, id);
  r.names.emplace_back(name);
  r.launches.push_back(0);
  return id;
}

cudaEvent_t take_event(Registry& r) {
  if (!r.pool.empty()) {
    cudaEvent_t e = r.pool.back();
    r.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

rpf_trace_scope::rpf_trace_scope(const char* name, cudaStream_t s) : s_(s) {
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  id_ = name_id(r, name);
  r.launches[id_] += 1;
  r.total += 1;
  if (r.on) {
    a_ = take_event(r);
    b_ = take_event(r);
    cudaEventRecord(a_, s);
  }
}

rpf_trace_scope::~rpf_trace_scope() {
  if (!a_) return;
  Registry& r = reg();
  cudaEventRecord(b_, s_);
  std::lock_guard<std::mutex> g(r.mu);
  r.recs.push_back({id_, a_, b_});
}

extern "C" {

int rpf_trace_enable(int on) {
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  r.on = on != 0;
  return RPF_OK;
}

int64_t rpf_launch_count(void) {
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  return r.total;
}

int rpf_trace_read(int32_t max_names, char* names, int64_t* launches, double* ms,
                   int32_t* n_names) {
  Registry& r = reg();
  std::lock_guard<std::mutex> g(r.mu);
  std::vector<double> acc(r.names.size(), 0.0);
  std::vector<long long> cnt(r.names.size(), 0);
  int rc = RPF_OK;
  for (Rec& e : r.recs) {
    float t = 0.0f;
    if (cudaEventSynchronize(e.b) != cudaSuccess || cudaEventElapsedTime(&t, e.a, e.b) != cudaSuccess) {
      cudaGetLastError();
      rc = RPF_ECUDA;
    }
    acc[e.name] += t;
    cnt[e.name] += 1;
    r.pool.push_back(e.a);
    r.pool.push_back(e.b);
  }
  r.recs.clear();
  const int k = (int)r.names.size();
  if (n_names) *n_names = k;
  for (int i = 0; i < k && i < max_names; ++i) {
    if (names) {
      std::strncpy(names + 48 * i, r.names[i].c_str(), 47);
      names[48 * i + 47] = 0;
    }
    if (launches) launches[i] = cnt[i];
    if (ms) ms[i] = acc[i];
  }
  return rc;
}

}  // extern "C"
