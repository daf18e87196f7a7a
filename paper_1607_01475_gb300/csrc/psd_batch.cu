// Batched PSD: many independent instances of uneven size solved
// concurrently on one GPU.  Each instance gets its own handle and its own
// non-blocking stream; a pool of host threads drives the instances' solve
// loops, so the kernels of different instances overlap on the device and
// the per-chunk host checks of one instance never stall another.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "../../include/psd.h"

struct psd_batch_ctx {
  std::vector<psd_handle> inst;
  std::vector<cudaStream_t> streams;
  int workers = 1;
  std::string err;
};

namespace {
thread_local std::string g_batch_error;
}

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
  for (int i = 0; i < count; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      g_batch_error = "cudaStreamCreateWithFlags failed";
      psd_batch_destroy(b);
      return PSD_ERR_CUDA;
    }
    b->streams.push_back(st);
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
  }
  *out = b;
  return PSD_OK;
}

psd_status psd_batch_destroy(psd_batch b) {
  if (!b) return PSD_OK;
  for (psd_handle h : b->inst) psd_destroy(h);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
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
  psd_status worst = PSD_OK;
  for (int i = 0; i < n; ++i) {
    if (infos) infos[i] = inf[i];
    if (st[i] != PSD_OK && (worst == PSD_OK || st[i] == PSD_ERR_CUDA)) {
      worst = st[i];
      char buf[256];
      psd_last_error(b->inst[i], buf, sizeof buf);
      b->err = "instance " + std::to_string(i) + ": " + buf;
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

}  // extern "C"
