// Batched PSD: many independent instances of uneven size solved
// concurrently on one GPU from ONE CUDA graph launch.  Each instance keeps
// its own handle (workspace, control blocks) and stream; its whole solve --
// the iteration loops are WHILE conditional nodes driven by the instance's
// device-resident stop flags -- is captured as an independent branch of a
// single graph (fork / join events on the instances' streams), which the
// GPU then runs without any host round trip: the kernels of different
// instances overlap, and an instance that stops early (converged, or failed
// on a non-finite value) ends its own branch only.  Nothing waits on a flag
// written by another kernel, so there is no spin-wait to bound.
//
// The graph is cached on the batch for the last set of f, g, u pointers.
// When a capture is not possible (kernel tracing on an instance, or a
// capture failure) every instance's own solve graph is launched on its own
// stream from this thread (or, for a handle whose graphs are off, its
// direct loop runs); psd_batch_set_mode selects either of these schedules
// or a pool of host threads explicitly.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "../../include/psd.h"

namespace psd_internal {
psd_status prepare(psd_handle c, const double* f, const double* g, double* u);
psd_status capture(psd_handle c, const double* f, const double* g, double* u, cudaStream_t st);
psd_status finish(psd_handle c, psd_info* info);
psd_status launch(psd_handle c, const double* f, const double* g, double* u, bool* ran);
cudaStream_t stream(psd_handle c);
psd_status tune(psd_handle c);
}  // namespace psd_internal

struct psd_batch_ctx {
  std::vector<psd_handle> inst;
  std::vector<cudaStream_t> streams;
  int workers = 1;
  std::string err;
  // the single-graph driver
  cudaStream_t main = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t graph = nullptr;
  std::vector<const void*> key;  // f, g, u of every instance
  bool graph_off = false;
  int mode = 0;       // requested schedule (psd_batch_set_mode); 0 = the default
  int last_mode = 0;  // schedule of the last solve: 1, 2 or 3 (see psd_batch_set_mode)
};

namespace {
thread_local std::string g_batch_error;

// The schedule used when none is set: 1 = one graph with a branch per
// instance.  On a GB300, the 96-instance 2D workload (64^2 .. 1024^2,
// mixed precision) took 144 ms this way, 195 ms with each instance's own
// graph on its stream (2) and 160 ms from host threads (3).
constexpr int kDefaultMode = 1;

// Capture the solves of all instances as parallel branches of one graph.
psd_status build_graph(psd_batch_ctx* b, const double* const* f, const double* const* g, double* const* u) {
  const int n = (int)b->inst.size();
  if (cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PSD_ERR_CUDA;
  psd_status s = PSD_OK;
  if (cudaEventRecord(b->fork, b->main) != cudaSuccess) s = PSD_ERR_CUDA;
  for (int i = 0; i < n && s == PSD_OK; ++i) {
    if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) {
      s = PSD_ERR_CUDA;
      break;
    }
    s = psd_internal::capture(b->inst[i], f[i], g ? g[i] : nullptr, u[i], b->streams[i]);
    if (s != PSD_OK) break;
    if (cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess ||
        cudaStreamWaitEvent(b->main, b->join[i], 0) != cudaSuccess)
      s = PSD_ERR_CUDA;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamEndCapture(b->main, &graph) != cudaSuccess) graph = nullptr;
  if (s != PSD_OK || graph == nullptr || cudaGraphInstantiate(&b->graph, graph, 0) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    b->graph = nullptr;
    return s != PSD_OK ? s : PSD_ERR_CUDA;
  }
  cudaGraphDestroy(graph);
  return PSD_OK;
}

}  // namespace

extern "C" {

psd_status psd_batch_create(const psd_params* per_instance, int count, int workers, psd_batch* out) {
  if (!out) return PSD_ERR_INVALID;
  *out = nullptr;
  if (!per_instance || count < 1) {
    g_batch_error = "per_instance must hold count >= 1 parameter sets";
    return PSD_ERR_INVALID;
  }
  psd_batch_ctx* b = new psd_batch_ctx();
  b->workers = workers > 0 ? std::min(workers, count) : std::min(count, 16);
  if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    g_batch_error = "stream or event creation failed";
    psd_batch_destroy(b);
    return PSD_ERR_CUDA;
  }
  for (int i = 0; i < count; ++i) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (st) cudaStreamDestroy(st);
      g_batch_error = "stream or event creation failed";
      psd_batch_destroy(b);
      return PSD_ERR_CUDA;
    }
    b->streams.push_back(st);
    b->join.push_back(ev);
    psd_params p = per_instance[i];
    p.stream = st;
    psd_handle h = nullptr;
    psd_status s = psd_create(&p, &h);
    if (s != PSD_OK) {
      char buf[256];
      psd_last_error(nullptr, buf, sizeof buf);
      g_batch_error = "instance " + std::to_string(i) + ": " + buf;
      psd_batch_destroy(b);
      return s;
    }
    b->inst.push_back(h);
    // tile widths of the FP32 passes, timed once per distinct grid (cached)
    if (p.precision == PSD_MIXED && (s = psd_internal::tune(h)) != PSD_OK) {
      g_batch_error = "instance " + std::to_string(i) + ": autotuning failed";
      psd_batch_destroy(b);
      return s;
    }
  }
  *out = b;
  return PSD_OK;
}

psd_status psd_batch_destroy(psd_batch b) {
  if (!b) return PSD_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (psd_handle h : b->inst) psd_destroy(h);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->main) cudaStreamDestroy(b->main);
  delete b;
  return PSD_OK;
}

psd_status psd_batch_solve(psd_batch b, const double* const* f, const double* const* g, double* const* u,
                           psd_info* infos) {
  if (!b || !f || !u) return PSD_ERR_INVALID;
  const int n = (int)b->inst.size();
  for (int i = 0; i < n; ++i)
    if (!f[i] || !u[i]) {
      b->err = "f[i] and u[i] are required for every instance";
      return PSD_ERR_INVALID;
    }
  // callers' data may still be in flight on the legacy stream
  if (cudaDeviceSynchronize() != cudaSuccess) {
    b->err = "cudaDeviceSynchronize failed";
    return PSD_ERR_CUDA;
  }
  std::vector<psd_status> st(n, PSD_OK);
  std::vector<psd_info> inf(n);
  bool done = false;
  const int mode = b->mode != 0 ? b->mode : kDefaultMode;
  if (mode == 1 && !b->graph_off) {
    // host part of every solve (asynchronous uploads), then one graph launch
    // for all of them
    psd_status ps = PSD_OK;
    for (int i = 0; i < n && ps == PSD_OK; ++i) ps = psd_internal::prepare(b->inst[i], f[i], g ? g[i] : nullptr, u[i]);
    if (ps == PSD_OK && cudaDeviceSynchronize() != cudaSuccess) ps = PSD_ERR_CUDA;
    if (ps == PSD_OK) {
      std::vector<const void*> key;
      for (int i = 0; i < n; ++i) {
        key.push_back(f[i]);
        key.push_back(g ? g[i] : nullptr);
        key.push_back(u[i]);
      }
      if (b->graph && key != b->key) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      if (!b->graph && build_graph(b, f, g, u) == PSD_OK) b->key = key;
      if (b->graph && cudaGraphLaunch(b->graph, b->main) == cudaSuccess &&
          cudaStreamSynchronize(b->main) == cudaSuccess) {
        for (int i = 0; i < n; ++i) st[i] = psd_internal::finish(b->inst[i], &inf[i]);
        done = true;
        b->last_mode = 1;
      } else {
        cudaGetLastError();
        b->graph_off = true;
      }
    } else {
      b->graph_off = true;
    }
  }
  if (!done && mode != 3) {
    // every instance's own solve graph on its own stream, launched from this
    // thread; the host waits once per instance at the end
    std::vector<char> ran(n, 0);
    for (int i = 0; i < n; ++i) {
      bool r = false;
      st[i] = psd_internal::prepare(b->inst[i], f[i], g ? g[i] : nullptr, u[i]);
      if (st[i] == PSD_OK) st[i] = psd_internal::launch(b->inst[i], f[i], g ? g[i] : nullptr, u[i], &r);
      ran[i] = r ? 1 : 0;
    }
    for (int i = 0; i < n; ++i) {
      if (ran[i])
        st[i] = psd_internal::finish(b->inst[i], &inf[i]);
      else if (st[i] == PSD_OK)  // graphs off for this handle: its direct loop
        st[i] = psd_solve(b->inst[i], f[i], g ? g[i] : nullptr, u[i], nullptr, &inf[i]);
    }
    done = true;
    b->last_mode = 2;
  }
  if (!done) {
    std::atomic<int> next(0);
    auto work = [&]() {
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= n) return;
        st[i] = psd_solve(b->inst[i], f[i], g ? g[i] : nullptr, u[i], nullptr, &inf[i]);
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < b->workers; ++t) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
    b->last_mode = 3;
  }
  psd_status worst = PSD_OK;
  for (int i = 0; i < n; ++i) {
    if (infos) infos[i] = inf[i];
    if (st[i] != PSD_OK && (worst == PSD_OK || st[i] == PSD_ERR_CUDA)) {
      worst = st[i];
      char buf[256];
      psd_last_error(b->inst[i], buf, sizeof buf);
      b->err = "instance " + std::to_string(i) + ": " + (buf[0] ? std::string(buf) : psd_status_string(st[i]));
    }
  }
  return worst;
}

psd_status psd_batch_last_error(psd_batch b, char* buf, size_t len) {
  if (!buf || len == 0) return PSD_ERR_INVALID;
  const std::string& e = b ? b->err : g_batch_error;
  snprintf(buf, len, "%s", e.c_str());
  return PSD_OK;
}

int psd_batch_mode(psd_batch b) { return b ? b->last_mode : 0; }

psd_status psd_batch_set_mode(psd_batch b, int mode) {
  if (!b || mode < 0 || mode > 3) return PSD_ERR_INVALID;
  b->mode = mode;
  return PSD_OK;
}

}  // extern "C"
