// Grouped solve of many independent problems (a batch of scatterers, each
// with its own H-matrix, scaling and right-hand sides) in one CUDA-graph
// launch.  The first call for a given set of (handle, X, B, nrhs) records
// every problem's power-series solve on its own stream, forked from and
// joined to a private capture stream (the caller's stream may be the legacy
// default stream, which cannot be captured), into one graph with one branch
// per problem; every call launches the instantiated graph on the caller's
// stream (one launch for the whole batch; the GPU overlaps the branches'
// kernels).
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "hm_internal.h"

namespace {

struct GroupGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned long long> gens;   // each handle's gen at capture
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaStream_t cap = nullptr;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    cap = nullptr;
    for (auto s : streams) cudaStreamDestroy(s);
    for (auto e : events) cudaEventDestroy(e);
    exec = nullptr;
    streams.clear();
    events.clear();
    gens.clear();
  }
};

std::mutex g_mu;
std::map<std::vector<const void*>, GroupGraph> g_cache;

hm_status capture(hm_handle* hs, void** X, const void** B, const int* nrhs, int count,
                  GroupGraph& gg) {
  HM_CUDA(cudaStreamCreateWithFlags(&gg.cap, cudaStreamNonBlocking));
  cudaStream_t main = gg.cap;
  for (int i = 0; i < count + 1; ++i) {
    cudaEvent_t e;
    HM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    gg.events.push_back(e);
  }
  for (int i = 0; i < count; ++i) {
    cudaStream_t s;
    HM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    gg.streams.push_back(s);
  }
  std::vector<cudaStream_t> saved(count);
  for (int i = 0; i < count; ++i) saved[i] = hs[i]->stream;
  HM_CUDA(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
  hm_status st = HM_OK;
  cudaError_t e = cudaEventRecord(gg.events[count], main);
  for (int i = 0; i < count && st == HM_OK && e == cudaSuccess; ++i) {
    e = cudaStreamWaitEvent(gg.streams[i], gg.events[count], 0);
    if (e != cudaSuccess) break;
    hs[i]->stream = gg.streams[i];
    st = hm_power_series_solve(hs[i], X[i], B[i], nrhs[i]);
    if (st != HM_OK) break;
    e = cudaEventRecord(gg.events[i], gg.streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(main, gg.events[i], 0);
  }
  for (int i = 0; i < count; ++i) hs[i]->stream = saved[i];
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(main, &graph);
  if (st != HM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return hm::cuda_status(e != cudaSuccess ? e : e2);
  }
  cudaError_t e3 = cudaGraphInstantiate(&gg.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return hm::cuda_status(e3);
  for (int i = 0; i < count; ++i) gg.gens.push_back(hs[i]->gen);
  return HM_OK;
}

// Cross-stream ordering of a grouped call that runs on `main`: with
// before = true, main waits for the work already queued on every other handle
// stream (a branch reuses its handle's work panels); with before = false,
// every other handle stream waits for what main has queued so far (later work
// on a handle starts after the graph).  One event per crossing, destroyed
// right away (the runtime keeps it until the wait is satisfied).
hm_status order_streams(hm_handle* hs, int count, cudaStream_t main, bool before) {
  std::vector<cudaStream_t> seen;
  for (int i = 0; i < count; ++i) {
    cudaStream_t si = hs[i]->stream;
    if (si == main || std::find(seen.begin(), seen.end(), si) != seen.end()) continue;
    seen.push_back(si);
  }
  if (seen.empty()) return HM_OK;
  if (before) {
    for (cudaStream_t si : seen) {
      cudaEvent_t e;
      HM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      cudaError_t r = cudaEventRecord(e, si);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(main, e, 0);
      cudaEventDestroy(e);
      HM_CUDA(r);
    }
  } else {
    cudaEvent_t e;
    HM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t r = cudaEventRecord(e, main);
    for (cudaStream_t si : seen)
      if (r == cudaSuccess) r = cudaStreamWaitEvent(si, e, 0);
    cudaEventDestroy(e);
    HM_CUDA(r);
  }
  return HM_OK;
}

}  // namespace

extern "C" hm_status hm_solve_grouped(hm_handle* hs, void** X, const void** B, const int* nrhs,
                                      int count) {
  if (!hs || !X || !B || !nrhs || count <= 0) return HM_ERR_INVALID;
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !X[i] || !B[i] || nrhs[i] <= 0) return HM_ERR_INVALID;
    if (!hs[i]->has_scaling || !hs[i]->sched_ready) return HM_ERR_STATE;
    if (hs[i]->prof) return HM_ERR_STATE;        // per-launch timing events cannot be captured
    if (hs[i]->p.term_tol > 0.0) return HM_ERR_STATE;   // host decisions per term
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return HM_ERR_INVALID;  // a handle's work panels serve one solve
  }
  cudaStream_t main = hs[0]->stream;
  std::vector<const void*> key;
  for (int i = 0; i < count; ++i) {
    key.push_back(hs[i]);
    key.push_back(X[i]);
    key.push_back(B[i]);
    key.push_back((const void*)(long long)nrhs[i]);
  }
  std::lock_guard<std::mutex> lk(g_mu);
  hm_status so = order_streams(hs, count, main, true);
  if (so != HM_OK) return so;
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    bool stale = false;
    for (int i = 0; i < count; ++i) stale |= it->second.gens[i] != hs[i]->gen;
    if (stale) {
      it->second.release();
      g_cache.erase(it);
      it = g_cache.end();
    }
  }
  if (it == g_cache.end()) {
    // one ordinary solve per problem first: sizes every work panel and runs
    // the lazy set-up that must not happen inside a capture
    for (int i = 0; i < count; ++i) {
      cudaStream_t sv = hs[i]->stream;
      hs[i]->stream = main;
      hm_status st = hm_power_series_solve(hs[i], X[i], B[i], nrhs[i]);
      hs[i]->stream = sv;
      if (st != HM_OK) return st;
    }
    HM_CUDA(cudaStreamSynchronize(main));
    GroupGraph gg;
    hm_status st = capture(hs, X, B, nrhs, count, gg);
    if (st != HM_OK) {
      gg.release();
      return st;
    }
    it = g_cache.emplace(key, gg).first;
  }
  HM_CUDA(cudaGraphLaunch(it->second.exec, main));
  return order_streams(hs, count, main, false);
}

namespace hm {
// Graphs that refer to a handle are dropped when it is destroyed.
void hm_group_forget(hm_ctx* h) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_cache.begin(); it != g_cache.end();) {
    bool uses = false;
    // key layout: 4 entries (handle, X, B, nrhs) per problem
    for (size_t i = 0; i < it->first.size(); i += 4)
      if (it->first[i] == (const void*)h) uses = true;
    if (uses) {
      it->second.release();
      it = g_cache.erase(it);
    } else {
      ++it;
    }
  }
}
}  // namespace hm
