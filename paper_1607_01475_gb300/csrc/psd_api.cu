// C ABI of the PSD library (include/psd.h): context management, the PSD
// driver loops (plain FP64 and mixed FP32/FP64 with outer FP64 residual
// correction), and the stand-alone residual / preconditioner calls.
//
// One PSD iteration (Algorithm 1 structure, Sec. 2.2, Sec. 6.1) is a fixed
// sequence of launches on the handle's stream:
//   DHT x -> [DHT y] -> middle pass (last axis: DHT, divide by the symbol of
//   L_h, Parseval sums, inverse DHT) -> [DHT y] -> DHT x (= d)
//   -> line search (alpha) -> residual at u + alpha d (fused update).
// The step size, the iteration count and the stop flag live in device memory
// (Ctrl); every kernel returns at once when the stop flag is set, so the host
// enqueues chunks of iterations and reads the flag once per chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/psd.h"
#include "kernels.h"

using psd::AxisTables;
using psd::Ctrl;
using psd::KParams;
using psd::ResArgs;

namespace {

thread_local std::string g_create_error;

constexpr int kChunk = 8;          // iterations enqueued between host checks (direct mode)
constexpr int kBody = 2;           // iterations per WHILE-loop body of a captured solve
static_assert(kBody % 2 == 0, "a loop body must start and end on the same ping-pong parity");
constexpr int kCapDepth = 3;       // nesting of WHILE loops: outer, inner, general-p line search
constexpr int kSolveGraphs = 4;    // solve graphs cached per handle (by pointer set)
static_assert(kChunk % 2 == 0, "a chunk must start and end on the same ping-pong parity");
constexpr int kLsPassesGen = 16;   // Newton passes of the general-p line search
constexpr double kInnerEta = 1e-4;  // inner FP32 solve: relative drop of the preconditioned norm
constexpr int kInnerStall = 5;      // ... or this many iterations without halving it
constexpr int kInnerMaxIter = 400;  // inner FP32 iterations per outer correction

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

struct psd_context {
  psd_params prm{};
  KParams kp{};
  int pk = psd::PK_GEN;
  cudaStream_t st = nullptr;
  size_t N = 0;
  std::string err;

  void* tables = nullptr;
  AxisTables<double> tb64{};
  AxisTables<float> tb32{};
  AxisTables<psd::ff> tbff{};

  // FP64 work arrays
  double* ub = nullptr;     // second iterate buffer (ping-pong with the caller's u)
  double* W = nullptr;      // residual / transform work array
  double* D = nullptr;      // search direction
  double* Z = nullptr;      // order 6: plain solve: xi = -DHT(u - g)/mu; mixed: DHT(u - g)
  double* Dsp = nullptr;    // order 6: DHT spectrum of T_h d for the last direction d
  double* Ftf = nullptr;    // time loops: right-hand side f of the current step
  double* Gtf = nullptr;    // SPFC time loop: g = u^n of the current step
  double* adj_q = nullptr;  // adjoint CG: H p (FP64), second direction buffer, copy of u
  double* adj_pb = nullptr;
  double* adj_u = nullptr;
  float* adj32[2] = {nullptr, nullptr};  // mixed adjoint: FP32 correction, H p
  // FP32 work arrays (mixed)
  float* u32 = nullptr;
  float* da = nullptr;
  float* db = nullptr;
  float* W32 = nullptr;
  float* D32 = nullptr;
  float* R32 = nullptr;
  float* Dsp32 = nullptr;

  double* partials = nullptr;
  Ctrl* ctrl = nullptr;   // PSD run state
  Ctrl* ctrl2 = nullptr;  // auxiliary reductions (outer residual, norms)
  Ctrl* ctrl3 = nullptr;  // mixed solve: outer-loop state of the captured solve
  Ctrl* ctrl_tmpl = nullptr;  // mixed solve: control block of a fresh inner solve
  Ctrl* h_ctrl = nullptr; // pinned host mirror: [0] synchronous transfers, [1..3] staging of
                          // asynchronous uploads (a batch's host part)

  double* d_hist = nullptr;
  double* user_alpha = nullptr;
  double* user_res = nullptr;
  int hist_cap = 0;

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // tracing: event pairs around every launch while enabled
  bool prof = false;
  unsigned prof_mask = ~0u;  // classes bracketed while prof is on
  std::vector<cudaEvent_t> ev_pool;
  struct Rec {
    int cls;
    int a, b;
  };
  std::vector<Rec> recs;
  double prof_ms[PSD_PROF_CLASSES] = {};
  long long prof_n[PSD_PROF_CLASSES] = {};
  std::vector<float> prof_durs[PSD_PROF_CLASSES];  // per-launch durations (ms)

  // The whole solve as one CUDA graph (its loops are WHILE conditional
  // nodes), captured on private streams and replayed on st.
  cudaStream_t gst = nullptr;
  cudaStream_t capst[kCapDepth] = {};
  int cap_depth = 0;
  bool capturing = false;
  // the last kSolveGraphs solve graphs by (u, f, g), least recently used
  // replaced: a caller that alternates buffer sets (copies of the next
  // step's inputs overlapping this step's solve) replays instead of
  // capturing again
  struct SolveGraph {
    cudaGraphExec_t exec = nullptr;
    const void* key[3] = {nullptr, nullptr, nullptr};
    unsigned long long used = 0;
  };
  SolveGraph g_solve[kSolveGraphs];
  unsigned long long g_tick = 0;
  cudaGraphExec_t g_cg32 = nullptr;  // adjoint CG chunks: FP32 (mixed inner, own buffers)
  cudaGraphExec_t g_cg64 = nullptr;  // and FP64 (own buffers: u is copied in)
  bool graphs_off = false;  // a capture failed once: launch directly from then on
};

namespace {

psd_status fail(psd_context* c, psd_status s, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_error = msg;
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(c, PSD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

template <typename T>
psd_status alloc(psd_context* c, T** p, size_t n) {
  if (*p) return PSD_OK;
  if (c->prm.alloc) {
    void* q = c->prm.alloc(n * sizeof(T), c->prm.alloc_ctx);
    if (!q) return fail(c, PSD_ERR_NOMEM, "the allocator callback returned NULL");
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
      c->prm.free_fn(q, c->prm.alloc_ctx);
      return fail(c, PSD_ERR_NOMEM, "the allocator callback returned memory not aligned to 256 bytes");
    }
    *p = static_cast<T*>(q);
    return PSD_OK;
  }
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, PSD_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return PSD_OK;
}

void dev_free(psd_context* c, void* p) {
  if (!p) return;
  if (c->prm.free_fn)
    c->prm.free_fn(p, c->prm.alloc_ctx);
  else
    cudaFree(p);
}

#define TRY(x)                   \
  do {                           \
    psd_status s_ = (x);         \
    if (s_ != PSD_OK) return s_; \
  } while (0)

psd_status validate(const psd_params* p, std::string& why) {
  if (!p) return why = "params is NULL", PSD_ERR_INVALID;
  if (p->order != 4 && p->order != 6) return why = "order must be 4 or 6", PSD_ERR_INVALID;
  if (p->dim != 2 && p->dim != 3) return why = "dim must be 2 or 3", PSD_ERR_INVALID;
  for (int a = 0; a < p->dim; ++a)
    if (!is_pow2(p->n[a]) || p->n[a] < 8 || p->n[a] > 1024)
      return why = "n[a] must be a power of two in [8, 1024]", PSD_ERR_INVALID;
  if (p->dim == 2 && p->n[2] != 1) return why = "n[2] must be 1 in 2D", PSD_ERR_INVALID;
  if (!(p->h > 0) || !std::isfinite(p->h)) return why = "h must be positive", PSD_ERR_INVALID;
  if (!(p->p >= 2) || !std::isfinite(p->p)) return why = "p must be >= 2", PSD_ERR_INVALID;
  if (p->dim == 3 && p->p > 6) return why = "3D requires p <= 6", PSD_ERR_INVALID;
  if (!(p->s > 0) || !std::isfinite(p->s)) return why = "s must be positive", PSD_ERR_INVALID;
  if (!(p->eps > 0) || !std::isfinite(p->eps)) return why = "eps must be positive", PSD_ERR_INVALID;
  if (!(p->lambda >= 0) || !std::isfinite(p->lambda)) return why = "lambda must be >= 0", PSD_ERR_INVALID;
  if (p->precision != PSD_FP64 && p->precision != PSD_MIXED)
    return why = "precision must be PSD_FP64 or PSD_MIXED", PSD_ERR_INVALID;
  if (!(p->tol >= 0) || !std::isfinite(p->tol)) return why = "tol must be >= 0", PSD_ERR_INVALID;
  if (p->max_iter < 0) return why = "max_iter must be >= 0", PSD_ERR_INVALID;
  if (p->precision == PSD_MIXED && p->max_outer < 1) return why = "max_outer must be >= 1", PSD_ERR_INVALID;
  if (!(p->inner_eta >= 0 && p->inner_eta < 1)) return why = "inner_eta must be in [0, 1)", PSD_ERR_INVALID;
  if (p->inner_stall < 0) return why = "inner_stall must be >= 0", PSD_ERR_INVALID;
  if ((p->alloc == nullptr) != (p->free_fn == nullptr))
    return why = "alloc and free_fn must both be set or both be NULL", PSD_ERR_INVALID;
  return PSD_OK;
}

psd_status build_tables(psd_context* c) {
  const int dim = c->prm.dim;
  int n[3] = {c->prm.n[0], c->prm.n[1], dim == 3 ? c->prm.n[2] : 1};
  size_t tot = 0;
  for (int a = 0; a < 3; ++a) tot += 3 * (size_t)n[a];
  std::vector<double> h64(tot);
  std::vector<float> h32(tot);
  size_t off = 0;
  size_t offs[3][3];
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double h = c->prm.h;
  for (int a = 0; a < 3; ++a) {
    offs[a][0] = off;
    for (int t = 0; t < n[a]; ++t) h64[off + t] = (double)cosl(2.0L * pi * t / n[a]);
    off += n[a];
    offs[a][1] = off;
    for (int t = 0; t < n[a]; ++t) h64[off + t] = (double)sinl(2.0L * pi * t / n[a]);
    off += n[a];
    offs[a][2] = off;
    for (int k = 0; k < n[a]; ++k) {
      const long double sn = (n[a] > 1) ? sinl(pi * k / n[a]) : 0.0L;
      h64[off + k] = (double)(4.0L / (h * h) * sn * sn);
    }
    off += n[a];
  }
  for (size_t i = 0; i < tot; ++i) h32[i] = (float)h64[i];
  // float-float twiddles: hi = the nearest float, lo = the nearest float to
  // the remainder, both from the long-double value
  std::vector<psd::ff> hff(tot);
  for (int a = 0; a < 3; ++a)
    for (int t = 0; t < n[a]; ++t)
      for (int w = 0; w < 3; ++w) {
        long double v;
        if (w == 0)
          v = cosl(2.0L * pi * t / n[a]);
        else if (w == 1)
          v = sinl(2.0L * pi * t / n[a]);
        else {
          const long double sn = (n[a] > 1) ? sinl(pi * t / n[a]) : 0.0L;
          v = 4.0L / (h * h) * sn * sn;
        }
        const float hi = (float)v;
        hff[offs[a][w] + t] = psd::ff(hi, (float)(v - (long double)hi));
      }
  {
    unsigned char* t = nullptr;
    TRY(alloc(c, &t, tot * (sizeof(double) + sizeof(float) + sizeof(psd::ff))));
    c->tables = t;
  }
  double* d64 = (double*)c->tables;
  psd::ff* dff = (psd::ff*)(d64 + tot);
  float* d32 = (float*)(dff + tot);
  CK(cudaMemcpy(d64, h64.data(), tot * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dff, hff.data(), tot * sizeof(psd::ff), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d32, h32.data(), tot * sizeof(float), cudaMemcpyHostToDevice));
  for (int a = 0; a < 3; ++a) {
    c->tb64.twc[a] = d64 + offs[a][0];
    c->tb64.tws[a] = d64 + offs[a][1];
    c->tb64.sym[a] = d64 + offs[a][2];
    c->tb32.twc[a] = d32 + offs[a][0];
    c->tb32.tws[a] = d32 + offs[a][1];
    c->tb32.sym[a] = d32 + offs[a][2];
    c->tbff.twc[a] = dff + offs[a][0];
    c->tbff.tws[a] = dff + offs[a][1];
    c->tbff.sym[a] = dff + offs[a][2];
  }
  return PSD_OK;
}

// ---------------------------------------------------------------- tracing
// Fold finished event pairs into the per-class totals and recycle the pool.
psd_status prof_flush(psd_context* c) {
  if (c->recs.empty()) return PSD_OK;
  CK(cudaStreamSynchronize(c->st));
  for (const auto& r : c->recs) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev_pool[r.a], c->ev_pool[r.b]));
    c->prof_ms[r.cls] += ms;
    c->prof_n[r.cls] += 1;
    c->prof_durs[r.cls].push_back(ms);
  }
  c->recs.clear();
  return PSD_OK;
}

// RAII bracket of one launch: records a start event now and a stop event at
// scope exit (both on the handle's stream).
struct ProfScope {
  psd_context* c;
  int cls;
  int a = -1;
  ProfScope(psd_context* c_, int cls_) : c(c_), cls(cls_) {
    if (!c->prof || !((c->prof_mask >> cls_) & 1u)) return;
    const size_t need = 2 * (c->recs.size() + 1);
    if (need > c->ev_pool.size()) {
      if (c->ev_pool.size() >= 4096) {
        if (prof_flush(c) != PSD_OK) return;
      } else {
        const size_t grow = std::max<size_t>(256, c->ev_pool.size());
        for (size_t i = 0; i < grow; ++i) {
          cudaEvent_t e;
          if (cudaEventCreate(&e) != cudaSuccess) return;
          c->ev_pool.push_back(e);
        }
      }
    }
    a = (int)(2 * c->recs.size());
    if (cudaEventRecord(c->ev_pool[a], c->st) != cudaSuccess) a = -1;
  }
  ~ProfScope() {
    if (a < 0) return;
    if (cudaEventRecord(c->ev_pool[a + 1], c->st) == cudaSuccess) c->recs.push_back({cls, a, a + 1});
  }
};

// Enqueue one chunk of iterations through a cached CUDA graph (captured the
// first time on the private stream and launched on st, whose stream order
// then places it after the work queued before), or directly while tracing
// is on or after a failed capture.
template <typename Enq>
psd_status run_chunk(psd_context* c, cudaGraphExec_t* cache, Enq&& enqueue) {
  if (c->prof || c->graphs_off) return enqueue();
  if (!*cache) {
    if (!c->gst && cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      c->graphs_off = true;
      return enqueue();
    }
    cudaStream_t saved = c->st;
    c->st = c->gst;
    cudaGraph_t g = nullptr;
    psd_status s = PSD_OK;
    if (cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      s = enqueue();
      if (cudaStreamEndCapture(c->gst, &g) != cudaSuccess) g = nullptr;
    }
    c->st = saved;
    if (s != PSD_OK || g == nullptr || cudaGraphInstantiate(cache, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      *cache = nullptr;
      c->graphs_off = true;
      return enqueue();
    }
    cudaGraphDestroy(g);
  }
  CK(cudaGraphLaunch(*cache, c->st));
  return PSD_OK;
}

template <typename T>
constexpr int cls_of(int fp64cls) {
  return sizeof(T) == 8 ? fp64cls : fp64cls + 1;
}

void init_ctrl(Ctrl& h, double tol, int max_iter) {
  std::memset(&h, 0, sizeof(h));
  h.tol = tol;
  h.max_iter = max_iter;
  h.res_linf = -1.0;
  h.c2 = -1.0;
}

psd_status upload_ctrl(psd_context* c, Ctrl* dst, const Ctrl& h) {
  *c->h_ctrl = h;
  CK(cudaMemcpyAsync(dst, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return PSD_OK;
}

// Upload without waiting, from staging slot `slot` (1..3) of the pinned
// mirror; the slot must not be reused before the copy has run.
psd_status upload_ctrl_async(psd_context* c, Ctrl* dst, const Ctrl& h, int slot) {
  c->h_ctrl[slot] = h;
  CK(cudaMemcpyAsync(dst, c->h_ctrl + slot, sizeof(Ctrl), cudaMemcpyHostToDevice, c->st));
  return PSD_OK;
}

psd_status read_ctrl(psd_context* c, const Ctrl* src, Ctrl& out) {
  CK(cudaMemcpyAsync(c->h_ctrl, src, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  out = *c->h_ctrl;
  return PSD_OK;
}

// Full separable DHT of x in place, multiplied by `scale` (its own inverse
// when scale = 1/N).
template <typename T>
psd_status full_dht(psd_context* c, T* x, T scale, const AxisTables<T>& tb) {
  const KParams& kp = c->kp;
  const int nrows = kp.ny * kp.nz;
  if (kp.dim == 2) {
    { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_ROWS_FP64)); CK(psd::launch_dht_rows<T>(x, x, kp.nx, nrows, T(1), nullptr, tb, c->st)); }
    { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_COLS_FP64)); CK(psd::launch_dht_cols<T>(x, kp, 1, scale, nullptr, tb, c->st)); }
  } else {
    { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_ROWS_FP64)); CK(psd::launch_dht_rows<T>(x, x, kp.nx, nrows, T(1), nullptr, tb, c->st)); }
    { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_COLS_FP64)); CK(psd::launch_dht_cols<T>(x, kp, 1, T(1), nullptr, tb, c->st)); }
    { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_COLS_FP64)); CK(psd::launch_dht_cols<T>(x, kp, 2, scale, nullptr, tb, c->st)); }
  }
  return PSD_OK;
}

// theta += DHT(v) / mu (order 6, mixed): v is src64 (FP64, transformed in
// place) or src32 (FP32, transformed into D); theta lives in Z.  skip
// (device, may be null): the passes return at once when *skip != 0.
psd_status dht_theta_ff(psd_context* c, const double* src64, const float* src32, double* dc = nullptr,
                        const int* skip = nullptr) {
  const KParams& kp = c->kp;
  const int nrows = kp.ny * kp.nz;
  psd::ff* x = reinterpret_cast<psd::ff*>(c->D);  // float-float pairs between the passes
  if (src32) {
    ProfScope p_(c, PSD_PROF_DHT_ROWS_FF);
    CK(psd::launch_dht_rows_ff_from_f32(src32, x, kp.nx, nrows, c->tbff, c->st, skip));
  } else {
    ProfScope p_(c, PSD_PROF_DHT_ROWS_FF);
    CK(psd::launch_dht_rows_ff(src64, x, kp.nx, nrows, c->tbff, c->st, skip));
  }
  if (kp.dim == 3) { ProfScope p_(c, PSD_PROF_DHT_COLS_FF); CK(psd::launch_dht_cols_ff(x, kp, 1, c->tbff, c->st, skip)); }
  { ProfScope p_(c, PSD_PROF_DHT_COLS_FF); CK(psd::launch_dht_last_ff(x, c->Z, nullptr, kp, nullptr, c->partials, c->tbff, c->st, dc, skip)); }
  return PSD_OK;
}

// The search-direction solve L_h d = W of one PSD iteration (W is consumed).
template <typename T>
psd_status precond_passes(psd_context* c, T* W, T* D, Ctrl* ctrl, T* xi, T* dspec, const AxisTables<T>& tb) {
  const KParams& kp = c->kp;
  const int* done = &ctrl->done;
  const int nrows = kp.ny * kp.nz;
  { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_ROWS_FP64)); CK(psd::launch_dht_rows<T>(W, W, kp.nx, nrows, T(1), done, tb, c->st)); }
  if (kp.dim == 3) { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_COLS_FP64)); CK(psd::launch_dht_cols<T>(W, kp, 1, T(1), done, tb, c->st)); }
  { ProfScope p_(c, cls_of<T>(PSD_PROF_MID_FP64)); CK(psd::launch_mid<T>(W, kp, ctrl, c->partials, xi, dspec, tb, c->st)); }
  if (kp.dim == 3) { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_COLS_FP64)); CK(psd::launch_dht_cols<T>(W, kp, 1, T(1), done, tb, c->st)); }
  { ProfScope p_(c, cls_of<T>(PSD_PROF_DHT_ROWS_FP64)); CK(psd::launch_dht_rows<T>(W, D, kp.nx, nrows, T(1), done, tb, c->st)); }
  return PSD_OK;
}

// ------------------------------------------------------ graph capture
// Stream of nesting depth d for capturing the bodies of WHILE nodes (depth 0
// is the graph itself, captured on gst).
psd_status cap_stream(psd_context* c, int d, cudaStream_t* out) {
  if (d <= 0) {
    if (!c->gst) CK(cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking));
    *out = c->gst;
    return PSD_OK;
  }
  if (d > kCapDepth) return fail(c, PSD_ERR_CUDA, "graph loops nested too deep");
  if (!c->capst[d - 1]) CK(cudaStreamCreateWithFlags(&c->capst[d - 1], cudaStreamNonBlocking));
  *out = c->capst[d - 1];
  return PSD_OK;
}

// Insert a WHILE conditional node at the current position of the capture on
// c->st and capture its body: body(handle) enqueues on c->st (a stream of the
// next depth) and must end with a kernel that sets the condition.  A kernel
// just before the node sets the condition to 1, so the body runs at least
// once every time the node is reached.
template <typename Body>
psd_status capture_while(psd_context* c, Body&& body) {
  cudaStream_t s = c->st, s2 = nullptr;
  TRY(cap_stream(c, c->cap_depth + 1, &s2));
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) return fail(c, PSD_ERR_CUDA, "capture_while outside a capture");
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  // a node nested in another loop's body is reached again with the value of
  // its last exit: arm it first
  CK(psd::launch_cond_arm(h, s));
  CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
  CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(s2, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  c->st = s2;
  ++c->cap_depth;
  psd_status r = body(h);
  --c->cap_depth;
  c->st = s;
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s2, &out);
  if (r != PSD_OK) return r;
  if (e != cudaSuccess) return fail(c, PSD_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  return PSD_OK;
}

// Capture enqueue() (which enqueues on c->st) into a graph and instantiate
// it into *exec.  Any failure leaves *exec null and returns the status.
template <typename Enq>
psd_status capture_graph(psd_context* c, cudaGraphExec_t* exec, Enq&& enqueue) {
  cudaStream_t s = nullptr;
  TRY(cap_stream(c, 0, &s));
  cudaStream_t saved = c->st;
  c->st = s;
  c->cap_depth = 0;
  cudaGraph_t g = nullptr;
  psd_status r = PSD_ERR_CUDA;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    r = enqueue();
    if (cudaStreamEndCapture(s, &g) != cudaSuccess) g = nullptr;
  }
  c->st = saved;
  if (r != PSD_OK || g == nullptr || cudaGraphInstantiate(exec, g, 0) != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    *exec = nullptr;
    return r != PSD_OK ? r : fail(c, PSD_ERR_CUDA, "graph capture or instantiation failed");
  }
  cudaGraphDestroy(g);
  return PSD_OK;
}

// The line search of one iteration: one pass (p = 4, 6), or for a general p
// one safeguarded Newton pass per launch -- a fixed run of kLsPassesGen
// launches (each returns at once after convergence) when enqueued directly,
// a WHILE loop that stops at convergence inside a captured graph.
template <typename T>
psd_status linesearch(psd_context* c, const T* u, const T* ubase, const T* D, Ctrl* ctrl) {
  if (c->pk != psd::PK_GEN) {
    ProfScope p_(c, cls_of<T>(PSD_PROF_LINESEARCH_FP64));
    CK(psd::launch_linesearch<T>(u, ubase, D, c->pk, c->kp, ctrl, c->partials, c->st));
    return PSD_OK;
  }
  if (c->capturing) {
    return capture_while(c, [&](cudaGraphConditionalHandle h) -> psd_status {
      CK(psd::launch_linesearch<T>(u, ubase, D, c->pk, c->kp, ctrl, c->partials, c->st));
      CK(psd::launch_ls_cond(h, ctrl, kLsPassesGen, c->st));
      return PSD_OK;
    });
  }
  for (int i = 0; i < kLsPassesGen; ++i) {
    ProfScope p_(c, cls_of<T>(PSD_PROF_LINESEARCH_FP64));
    CK(psd::launch_linesearch<T>(u, ubase, D, c->pk, c->kp, ctrl, c->partials, c->st));
  }
  return PSD_OK;
}

psd_status ensure_fp64(psd_context* c) {
  TRY(alloc(c, &c->ub, c->N));
  TRY(alloc(c, &c->W, c->N));
  TRY(alloc(c, &c->D, c->N));
  if (c->prm.order == 6) {
    TRY(alloc(c, &c->Z, c->N));
    TRY(alloc(c, &c->Dsp, c->N));
  }
  return PSD_OK;
}

psd_status ensure_fp32(psd_context* c) {
  TRY(alloc(c, &c->u32, c->N));
  TRY(alloc(c, &c->da, c->N));
  TRY(alloc(c, &c->db, c->N));
  TRY(alloc(c, &c->W32, c->N));
  TRY(alloc(c, &c->D32, c->N));
  TRY(alloc(c, &c->R32, c->N));
  if (c->prm.order == 6) TRY(alloc(c, &c->Dsp32, c->N));
  return PSD_OK;
}

// Whether the FP64 residual of the current iterate (its FP32 copy in u32)
// may take the fixed-point linear part and the float-float flux part: p = 4,
// 3D column kernel, and a worst-case error bound of the flux part,
//   |Omega|^{1/2} * 24 * 2^-47 * s q^4 * (2 max|G|)^3
// (24 flux values per cell in the divergence, 2^-47 the double-word
// precision, a factor 2 of margin on the FP32 estimate of max|G|), below
// tol / 20.  *fxs receives the fixed-point scale S (0: plain FP64): with
// max|u| < 2^e (max|u32| (1 + 2^-20) bounds it, as u32 = fl32(u)),
// S = 55 - e keeps |q| = |u| 2^S below 2^55; S must lie in [15, 120].
psd_status use_fluxff(psd_context* c, int* fxs) {
  *fxs = 0;
  const KParams& kp = c->kp;
  if (c->pk != psd::PK_4 || kp.dim != 3 || kp.nx < 32 || kp.ny < 8 || !(c->prm.tol > 0)) return PSD_OK;
  Ctrl h;
  init_ctrl(h, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h));
  { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_gradmax(c->u32, kp, c->ctrl2, c->partials, c->st)); }
  Ctrl h2;
  TRY(read_ctrl(c, c->ctrl2, h2));
  const double gmax = 2.0 * std::sqrt(std::max(h2.res_linf, 0.0));
  const double bound = std::sqrt((double)c->N * kp.hd) * 24.0 * std::ldexp(1.0, -47) * kp.cdiv * gmax * gmax * gmax;
  const double umax = h2.res_l2;
  if (!(std::isfinite(bound) && bound < 0.05 * c->prm.tol) || !std::isfinite(umax)) return PSD_OK;
  int e = 0;
  if (umax > 0.0) std::frexp(umax * (1.0 + std::ldexp(1.0, -20)), &e);  // umax (1 + 2^-20) < 2^e
  const int S = 55 - e;
  if (S >= 15 && S <= 120) *fxs = S;
  return PSD_OK;
}

// Whether the FP64 outer residuals of this handle may take the fixed-point /
// float-float variant at all (the per-iterate bound is checked on device in
// graph mode, by use_fluxff in direct mode).
bool fluxff_eligible(const psd_context* c) {
  const KParams& kp = c->kp;
  return c->pk == psd::PK_4 && kp.dim == 3 && kp.nx >= 32 && kp.ny >= 8 && c->prm.tol > 0;
}

// FP64 residual r = f - N_h[u] into r (order 6: P0[...] including T_h[u - g]),
// norms into ctrl2 (res_l2, res_linf), all enqueued (ctrl2 reset on device).
// fxs: fixed-point scale from the host (direct mode); fxs_dev: from device
// memory (graph mode).  Uses W, Z as scratch (order 6).
psd_status residual64(psd_context* c, const double* u, const double* f, const double* g, double* r, int fxs = 0,
                      const int* fxs_dev = nullptr) {
  const KParams& kp = c->kp;
  CK(psd::launch_ctrl_reset(c->ctrl2, c->st));
  ResArgs<double> a{u, nullptr, nullptr, f, nullptr, r, kp.order == 4 ? 1 : 0, 0, fxs ? 1 : 0, fxs, fxs_dev};
  { ProfScope p_(c, PSD_PROF_RESIDUAL_FP64); CK(psd::launch_residual<double>(a, psd::RM_PLAIN, c->pk, kp, c->ctrl2, c->partials, c->st)); }
  if (kp.order == 6) {
    // r <- P0[r_loc - T_h[u - g]] through the spectrum
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_axpby<double>(c->Z, u, g, 1.0, -1.0, 0.0, c->N, c->st)); }
    TRY(full_dht<double>(c, c->Z, 1.0, c->tb64));
    TRY(full_dht<double>(c, r, 1.0, c->tb64));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_spec6_combine<double>(r, c->Z, kp, c->tb64, c->st)); }
    TRY(full_dht<double>(c, r, kp.inv_ntot, c->tb64));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_norms(r, c->N, kp.hd, c->ctrl2, c->partials, c->st)); }
  }
  return PSD_OK;
}

// Sixth-order outer residual in the transform domain (mixed precision):
// R32 <- (float) DHT(P0[f - N_h^{loc}[u]] - T_h[u - g]) = DHT(r_loc) - theta
// with theta = DHT(T_h[u - g]) in Z (the subtraction, the rounding and the
// Parseval norm fused into the last transform pass); ||R||_2 into
// ctrl2->res_l2 (enqueued).
psd_status outer_residual6_spec(psd_context* c, const double* u, const double* f, int fxs,
                                const int* fxs_dev = nullptr) {
  const KParams& kp = c->kp;
  CK(psd::launch_ctrl_reset(c->ctrl2, c->st));
  ResArgs<double> a{u, nullptr, nullptr, f, nullptr, c->W, 0, 0, fxs ? 1 : 0, fxs, fxs_dev};
  { ProfScope p_(c, PSD_PROF_RESIDUAL_FP64); CK(psd::launch_residual<double>(a, psd::RM_PLAIN, c->pk, kp, c->ctrl2, c->partials, c->st)); }
  const int nrows = kp.ny * kp.nz;
  psd::ff* x = reinterpret_cast<psd::ff*>(c->W);  // transformed in place, float-float pairs after the x pass
  { ProfScope p_(c, PSD_PROF_DHT_ROWS_FF); CK(psd::launch_dht_rows_ff(c->W, x, kp.nx, nrows, c->tbff, c->st)); }
  if (kp.dim == 3) { ProfScope p_(c, PSD_PROF_DHT_COLS_FF); CK(psd::launch_dht_cols_ff(x, kp, 1, c->tbff, c->st)); }
  { ProfScope p_(c, PSD_PROF_DHT_COLS_FF); CK(psd::launch_dht_last_ff(x, c->Z, c->R32, kp, c->ctrl2, c->partials, c->tbff, c->st)); }
  return PSD_OK;
}

// ------------------------------------------------------------- plain FP64
// The part of the FP64 solve before the loop: order 6 xi_0 = DHT(-T_h[u0 -
// g]) = -DHT(u0 - g) / mu (direction spectrum 0), then the initial residual.
psd_status fp64_start(psd_context* c, const double* f, const double* g, double* u) {
  const KParams& kp = c->kp;
  if (kp.order == 6) {
    CK(cudaMemsetAsync(c->Dsp, 0, c->N * sizeof(double), c->st));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_axpby<double>(c->Z, u, g, 1.0, -1.0, 0.0, c->N, c->st)); }
    TRY(full_dht<double>(c, c->Z, 1.0, c->tb64));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_spec_apply_T<double>(c->Z, -1.0, kp, c->tb64, c->st)); }
  }
  ResArgs<double> a{u, nullptr, nullptr, f, nullptr, c->W, kp.order == 4 ? 1 : 0, 0};
  { ProfScope p_(c, PSD_PROF_RESIDUAL_FP64); CK(psd::launch_residual<double>(a, psd::RM_PLAIN, c->pk, kp, c->ctrl, c->partials, c->st)); }
  return PSD_OK;
}

// count (even) FP64 PSD iterations from u (iterates ping-pong between u and
// ub: an even count starts and ends on u).
psd_status fp64_iterations(psd_context* c, const double* f, double* u, int count) {
  const KParams& kp = c->kp;
  for (int i = 0; i < count; ++i) {
    double* cur = (i % 2 == 0) ? u : c->ub;
    double* nxt = (i % 2 == 0) ? c->ub : u;
    TRY(precond_passes<double>(c, c->W, c->D, c->ctrl, c->Z, c->Dsp, c->tb64));
    TRY(linesearch<double>(c, cur, nullptr, c->D, c->ctrl));
    ResArgs<double> a{cur, c->D, nxt, f, nullptr, c->W, kp.order == 4 ? 1 : 0, 1};
    { ProfScope p_(c, PSD_PROF_RESIDUAL_FP64); CK(psd::launch_residual<double>(a, psd::RM_PLAIN, c->pk, kp, c->ctrl, c->partials, c->st)); }
  }
  return PSD_OK;
}

// The whole FP64 solve after the control block upload, as graph work: the
// start, a WHILE loop of kBody iterations per body, and the copy of an odd
// final iterate back into u.
psd_status fp64_graph_body(psd_context* c, const double* f, const double* g, double* u) {
  TRY(fp64_start(c, f, g, u));
  const int guard = c->prm.max_iter / kBody + 3;
  TRY(capture_while(c, [&](cudaGraphConditionalHandle h) -> psd_status {
    TRY(fp64_iterations(c, f, u, kBody));
    CK(psd::launch_loop_cond(h, c->ctrl, guard, c->st));
    return PSD_OK;
  }));
  CK(psd::launch_copy_if_odd<double>(u, c->ub, c->ctrl, c->N, c->st));
  return PSD_OK;
}

void fill_info(psd_info* info, int iters, int outer, double res, double resinf, double alpha, float ms, int status) {
  if (!info) return;
  info->iters = iters;
  info->outer_iters = outer;
  info->res_l2 = res;
  info->res_linf = resinf;
  info->energy = NAN;
  info->last_alpha = alpha;
  info->wall_ms = ms;
  info->status = status;
}

// Launch the cached graph of this handle's solve for the key (u, f, g),
// capturing it first if needed; false in *ran when graphs are off (direct
// mode) or the capture failed (then direct mode from now on).
template <typename Enq>
psd_status launch_solve_graph(psd_context* c, const double* f, const double* g, double* u, bool* ran, Enq&& enq) {
  *ran = false;
  if (c->prof || c->graphs_off) return PSD_OK;
  psd_context::SolveGraph* e = nullptr;
  for (auto& x : c->g_solve)
    if (x.exec && x.key[0] == u && x.key[1] == f && x.key[2] == g) e = &x;
  if (!e) {
    e = &c->g_solve[0];  // an empty slot, else the least recently used
    for (auto& x : c->g_solve)
      if (!x.exec || (e->exec && x.used < e->used)) e = &x;
    if (e->exec) {
      cudaGraphExecDestroy(e->exec);
      e->exec = nullptr;
    }
    c->capturing = true;
    const psd_status s = capture_graph(c, &e->exec, enq);
    c->capturing = false;
    if (s != PSD_OK || !e->exec) {
      c->graphs_off = true;
      c->err.clear();
      return PSD_OK;
    }
    e->key[0] = u;
    e->key[1] = f;
    e->key[2] = g;
  }
  e->used = ++c->g_tick;
  CK(cudaGraphLaunch(e->exec, c->st));
  *ran = true;
  return PSD_OK;
}

// Plain FP64 PSD.
psd_status solve_fp64(psd_context* c, const double* f, const double* g, double* u, psd_info* info) {
  TRY(ensure_fp64(c));
  Ctrl h;
  init_ctrl(h, c->prm.tol, c->prm.max_iter);
  if (c->hist_cap > 0) {
    h.hist_cap = c->hist_cap;
    h.hist_alpha = c->d_hist;
    h.hist_res = c->d_hist + c->hist_cap;
  }
  TRY(upload_ctrl(c, c->ctrl, h));
  CK(cudaEventRecord(c->ev0, c->st));
  bool ran = false;
  TRY(launch_solve_graph(c, f, g, u, &ran, [&]() { return fp64_graph_body(c, f, g, u); }));
  Ctrl hc;
  if (!ran) {
    // direct: chunks of kChunk iterations, the stop flag read after each
    TRY(fp64_start(c, f, g, u));
    int k = 0;
    for (;;) {
      TRY(fp64_iterations(c, f, u, kChunk));
      k += kChunk;
      TRY(read_ctrl(c, c->ctrl, hc));
      if (hc.done) break;
      if (k > c->prm.max_iter + 2 * kChunk) {  // host-side guard: never loop unbounded
        hc.status = PSD_ERR_NOCONV;
        break;
      }
    }
    if (hc.iter % 2 == 1) CK(cudaMemcpyAsync(u, c->ub, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  }
  CK(cudaEventRecord(c->ev1, c->st));
  TRY(read_ctrl(c, c->ctrl, hc));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  fill_info(info, hc.iter, 0, hc.res_l2, hc.res_linf, hc.alpha, ms, hc.status);
  return (psd_status)hc.status;
}

// ------------------------------------------------------------------ mixed
// Mixed precision: outer FP64 residual R = f - N_h[u] (order 6: P0[...]
// with the exact T_h[u - g]); inner FP32 PSD on the correction delta with
// residual R - (N_h[u + delta] - N_h[u]) (order 6: mean-projected, the T_h
// term kept as the DHT spectrum of delta); u += delta in FP64.
//
// The FP32 inner iterations (count even) of one inner solve.
psd_status inner_iterations(psd_context* c, int count) {
  const KParams& kp = c->kp;
  const bool six = kp.order == 6;
  const float* rphys = six ? nullptr : c->R32;
  for (int i = 0; i < count; ++i) {
    float* cur = (i % 2 == 0) ? c->da : c->db;
    float* nxt = (i % 2 == 0) ? c->db : c->da;
    TRY(precond_passes<float>(c, c->W32, c->D32, c->ctrl, six ? c->R32 : nullptr, c->Dsp32, c->tb32));
    TRY(linesearch<float>(c, cur, c->u32, c->D32, c->ctrl));
    ResArgs<float> a{cur, c->D32, nxt, rphys, c->u32, c->W32, six ? 0 : 1, 1};
    { ProfScope p_(c, PSD_PROF_RESIDUAL_FP32); CK(psd::launch_residual<float>(a, psd::RM_INNER, c->pk, kp, c->ctrl, c->partials, c->st)); }
  }
  return PSD_OK;
}

// The start of an inner solve: delta = 0, the direction spectrum 0 (order
// 6), and the inner residual at delta = 0.
psd_status inner_start(psd_context* c) {
  const KParams& kp = c->kp;
  const bool six = kp.order == 6;
  CK(cudaMemsetAsync(c->da, 0, c->N * sizeof(float), c->st));
  if (six) CK(cudaMemsetAsync(c->Dsp32, 0, c->N * sizeof(float), c->st));
  // order 6: the outer residual enters in the middle pass as the initial xi
  // (R32 holds its spectrum and is advanced in place by the inner solve)
  ResArgs<float> a{c->da, nullptr, nullptr, six ? nullptr : c->R32, c->u32, c->W32, six ? 0 : 1, 0};
  { ProfScope p_(c, PSD_PROF_RESIDUAL_FP32); CK(psd::launch_residual<float>(a, psd::RM_INNER, c->pk, kp, c->ctrl, c->partials, c->st)); }
  return PSD_OK;
}

// The control block of an inner FP32 solve.  The FP32 residual of
// s eps^2 Delta_h^2 delta carries rounding noise of order eps32 * 64 s eps^2
// / h^4 * |delta|, which on fine grids is as large as the residual itself,
// so ||r||_2 cannot serve as the inner stopping test.  The preconditioned
// norm (r, L_h^{-1} r)^{1/2} damps that noise by the symbol of L_h; the inner
// solve stops when it has dropped by inner_eta, or when it has stopped
// halving (its FP32 floor).
void inner_ctrl(psd_context* c, Ctrl& h, int max_iter) {
  init_ctrl(h, 0.0, max_iter);
  h.pre_eta = c->prm.inner_eta > 0.0 ? c->prm.inner_eta : kInnerEta;
  h.pre_stall_max = c->prm.inner_stall > 0 ? c->prm.inner_stall : kInnerStall;
}

// Order 6: the problem lives on mean(u) = mean(g); project u0 once
// (enqueued: the mean difference is formed and added on the device).
psd_status mixed_project_mean(psd_context* c, const double* g, double* u) {
  ProfScope p_(c, PSD_PROF_OTHER);
  CK(psd::launch_mean_project(u, g, c->N, c->ctrl2, c->partials, c->st));
  return PSD_OK;
}

// The device part of the mixed solve's start: u32 = fl32(u); order 6:
// theta = DHT(T_h[u0 - g]) (advanced with DHT(T_h delta) after every
// correction).
psd_status mixed_start(psd_context* c, const double* g, double* u) {
  { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_round_f32(c->u32, u, c->N, c->st)); }
  if (c->kp.order == 6) {
    CK(cudaMemsetAsync(c->Z, 0, c->N * sizeof(double), c->st));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_axpby<double>(c->D, u, g, 1.0, -1.0, 0.0, c->N, c->st)); }
    TRY(dht_theta_ff(c, c->D, nullptr));
  }
  return PSD_OK;
}

// The whole mixed solve after the host uploads, as graph work: an outer
// WHILE loop (device decisions in ctrl3) around the FP64 outer residual, the
// inner FP32 solve (an inner WHILE loop) and the FP64 accumulation.
psd_status mixed_graph_body(psd_context* c, const double* f, const double* g, double* u) {
  const KParams& kp = c->kp;
  const bool six = kp.order == 6;
  const bool elig = fluxff_eligible(c);
  TRY(mixed_start(c, g, u));
  const int guard_outer = std::max(c->prm.max_outer, 1) + 3;
  const int inner_cap = std::min(std::max(c->prm.max_iter, 1), kInnerMaxIter);
  const int guard_inner = inner_cap / kBody + 3;
  return capture_while(c, [&](cudaGraphConditionalHandle ho) -> psd_status {
    const int* fxs_dev = nullptr;
    if (elig) {
      CK(psd::launch_ctrl_reset(c->ctrl2, c->st));
      { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_gradmax(c->u32, kp, c->ctrl2, c->partials, c->st)); }
      CK(psd::launch_fluxff_decide(c->ctrl3, c->ctrl2, std::sqrt((double)c->N * kp.hd), kp.cdiv, c->prm.tol, c->st));
      fxs_dev = &c->ctrl3->fxs;
    }
    if (six) {
      TRY(outer_residual6_spec(c, u, f, 0, fxs_dev));
    } else {
      TRY(residual64(c, u, f, g, c->W, 0, fxs_dev));
      { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_round_f32(c->R32, c->W, c->N, c->st)); }
    }
    CK(psd::launch_mixed_check(c->ctrl3, c->ctrl2, c->ctrl, c->ctrl_tmpl, c->prm.tol, c->prm.max_iter,
                               c->prm.max_outer, kInnerMaxIter, six ? 1 : 0, c->st));
    TRY(inner_start(c));
    TRY(capture_while(c, [&](cudaGraphConditionalHandle hi) -> psd_status {
      TRY(inner_iterations(c, kBody));
      CK(psd::launch_loop_cond(hi, c->ctrl, guard_inner, c->st));
      return PSD_OK;
    }));
    CK(psd::launch_copy_if_odd<float>(c->da, c->db, c->ctrl, c->N, c->st));
    CK(psd::launch_mixed_after(c->ctrl3, c->ctrl, c->st));
    // order 6: theta += DHT(T_h delta) with sum(delta) recorded; u += delta
    // (mean removed for order 6), u32 = fl32(u) -- skipped once the outer
    // loop is done
    double* dsum = six ? &c->ctrl2->c3 : nullptr;
    if (six) TRY(dht_theta_ff(c, nullptr, c->da, dsum, &c->ctrl3->done));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_accumulate_f64(u, c->da, c->u32, c->N, dsum, c->st, &c->ctrl3->done)); }
    CK(psd::launch_loop_cond(ho, c->ctrl3, guard_outer, c->st));
    (void)inner_cap;
    return PSD_OK;
  });
}

psd_status solve_mixed(psd_context* c, const double* f, const double* g, double* u, psd_info* info) {
  TRY(ensure_fp64(c));
  TRY(ensure_fp32(c));
  const KParams& kp = c->kp;
  const bool six = kp.order == 6;
  CK(cudaEventRecord(c->ev0, c->st));
  if (six) TRY(mixed_project_mean(c, g, u));
  // device state of the graph-driven loops: the outer decisions (ctrl3) and
  // the template of an inner solve's control block
  {
    Ctrl h3;
    init_ctrl(h3, -1.0, 1 << 30);
    h3.status = PSD_ERR_NOCONV;
    TRY(upload_ctrl(c, c->ctrl3, h3));
    Ctrl ht;
    inner_ctrl(c, ht, 0);
    TRY(upload_ctrl(c, c->ctrl_tmpl, ht));
  }
  bool ran = false;
  TRY(launch_solve_graph(c, f, g, u, &ran, [&]() { return mixed_graph_body(c, f, g, u); }));
  if (ran) {
    CK(cudaEventRecord(c->ev1, c->st));
    Ctrl h3;
    TRY(read_ctrl(c, c->ctrl3, h3));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    fill_info(info, h3.inner_total, h3.outer, h3.res_l2, h3.res_linf, h3.last_alpha, ms, h3.status);
    return (psd_status)h3.status;
  }
  // direct: the same steps with the decisions on the host
  TRY(mixed_start(c, g, u));
  int inner_total = 0, outer = 0;
  int status = PSD_ERR_NOCONV;
  double res = NAN, resinf = -1, last_alpha = 0;
  bool have_delta = false;
  for (;;) {
    if (have_delta) {
      // order 6: theta += DHT(T_h delta); the zero-frequency coefficient of the
      // transform, sum(delta), is recorded on the device and the accumulation
      // removes the mean of delta, which is zero only up to FP32 rounding,
      // so that mean(u) = mean(g) holds throughout
      double* dsum = six ? &c->ctrl2->c3 : nullptr;
      if (six) TRY(dht_theta_ff(c, nullptr, c->da, dsum));
      { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_accumulate_f64(u, c->da, c->u32, c->N, dsum, c->st)); }
    }
    int fxs = 0;
    TRY(use_fluxff(c, &fxs));
    if (six) {
      // the outer residual stays in the transform domain; the inner solve adds
      // it to its own transformed residual in the middle pass
      TRY(outer_residual6_spec(c, u, f, fxs));
    } else {
      TRY(residual64(c, u, f, g, c->W, fxs));
    }
    Ctrl h2;
    TRY(read_ctrl(c, c->ctrl2, h2));
    res = h2.res_l2;
    resinf = six ? -1.0 : h2.res_linf;
    ++outer;
    if (!six) { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_round_f32(c->R32, c->W, c->N, c->st)); }
    if (!std::isfinite(res)) {
      status = PSD_ERR_NONFINITE;
      break;
    }
    if (res < c->prm.tol) {
      status = PSD_OK;
      break;
    }
    if (outer > c->prm.max_outer || inner_total >= c->prm.max_iter) {
      status = PSD_ERR_NOCONV;
      break;
    }
    Ctrl h;
    inner_ctrl(c, h, std::min(c->prm.max_iter - inner_total, kInnerMaxIter));
    TRY(upload_ctrl(c, c->ctrl, h));
    TRY(inner_start(c));
    int k = 0;
    Ctrl hc;
    for (;;) {
      TRY(inner_iterations(c, kChunk));
      k += kChunk;
      TRY(read_ctrl(c, c->ctrl, hc));
      if (hc.done) break;
      if (k > h.max_iter + 2 * kChunk) break;  // host-side guard
    }
    inner_total += hc.iter;
    last_alpha = hc.alpha;
    if (hc.status == PSD_ERR_NONFINITE) {
      status = PSD_ERR_NONFINITE;
      break;
    }
    if (hc.iter % 2 == 1) CK(cudaMemcpyAsync(c->da, c->db, c->N * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    have_delta = hc.iter > 0;
  }
  CK(cudaEventRecord(c->ev1, c->st));
  CK(cudaStreamSynchronize(c->st));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  fill_info(info, inner_total, outer, res, resinf, last_alpha, ms, status);
  return (psd_status)status;
}

// ------------------------------------------------------------- autotuner
// Tile widths (line pairs per block) of the FP32 row, strided and middle
// passes of a mixed-precision handle: each pass in turn, every candidate
// cap is timed on the handle's own buffers (kernel times do not depend on
// the values) over a few preconditioner solves, and the fastest is kept.
// Results are cached for the process by (dim, n, order).
std::mutex g_tune_mu;
std::map<std::array<int, 5>, std::array<int, 3>> g_tune_cache;

psd_status autotune(psd_context* c) {
  if (c->prm.precision != PSD_MIXED) return PSD_OK;
  const KParams& kp = c->kp;
  const std::array<int, 5> key = {kp.dim, kp.nx, kp.ny, kp.nz, kp.order};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int k = 0; k < 3; ++k) c->tb32.tile_cap[k] = it->second[k];
      return PSD_OK;
    }
  }
  TRY(ensure_fp32(c));
  const bool six = kp.order == 6;
  const size_t bytes = c->N * sizeof(float);
  CK(cudaMemsetAsync(c->W32, 0, bytes, c->st));
  CK(cudaMemsetAsync(c->R32, 0, bytes, c->st));
  if (six) CK(cudaMemsetAsync(c->Dsp32, 0, bytes, c->st));
  Ctrl h;
  init_ctrl(h, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h));
  const bool prof = c->prof;
  c->prof = false;
  auto run = [&](int reps, float* ms) -> psd_status {
    for (int r = 0; r < reps; ++r)
      TRY(precond_passes<float>(c, c->W32, c->D32, c->ctrl2, six ? c->R32 : nullptr, c->Dsp32, c->tb32));
    if (ms) {
      CK(cudaEventRecord(c->ev0, c->st));
      for (int r = 0; r < reps; ++r)
        TRY(precond_passes<float>(c, c->W32, c->D32, c->ctrl2, six ? c->R32 : nullptr, c->Dsp32, c->tb32));
      CK(cudaEventRecord(c->ev1, c->st));
      CK(cudaEventSynchronize(c->ev1));
      CK(cudaEventElapsedTime(ms, c->ev0, c->ev1));
    }
    return PSD_OK;
  };
  static const int kCaps[] = {0, 16, 8, 4, 2, 1};
  psd_status st = PSD_OK;
  for (int pass = 0; pass < 3 && st == PSD_OK; ++pass) {
    int best = 0;
    float best_ms = 1e30f;
    for (int cap : kCaps) {
      c->tb32.tile_cap[pass] = cap;
      float ms = 0.f;
      st = run(5, &ms);
      if (st != PSD_OK) break;
      if (ms < 0.97f * best_ms) {  // a clear gain over the previous best
        best_ms = ms;
        best = cap;
      }
    }
    c->tb32.tile_cap[pass] = best;
  }
  c->prof = prof;
  TRY(st);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {c->tb32.tile_cap[0], c->tb32.tile_cap[1], c->tb32.tile_cap[2]};
  return PSD_OK;
}

// ------------------------------------------------ batch (internal hooks)
// The host part of a solve before its graph work: control blocks uploaded
// (and, order 6 mixed, the mean projection of u0).
// The uploads are asynchronous on the handle's stream (work enqueued on that
// stream after them sees them).
psd_status solve_prepare(psd_context* c, const double* f, const double* g, double* u) {
  TRY(ensure_fp64(c));
  if (c->prm.precision == PSD_MIXED) {
    TRY(ensure_fp32(c));
    if (c->kp.order == 6) TRY(mixed_project_mean(c, g, u));
    Ctrl h3;
    init_ctrl(h3, -1.0, 1 << 30);
    h3.status = PSD_ERR_NOCONV;
    TRY(upload_ctrl_async(c, c->ctrl3, h3, 1));
    Ctrl ht;
    inner_ctrl(c, ht, 0);
    TRY(upload_ctrl_async(c, c->ctrl_tmpl, ht, 2));
  } else {
    Ctrl h;
    init_ctrl(h, c->prm.tol, c->prm.max_iter);
    TRY(upload_ctrl_async(c, c->ctrl, h, 1));
  }
  (void)f;
  return PSD_OK;
}

// Launch the handle's own solve graph (captured first if needed) on its
// stream after solve_prepare; *ran false when graphs are off.
psd_status solve_launch(psd_context* c, const double* f, const double* g, double* u, bool* ran) {
  CK(cudaEventRecord(c->ev0, c->st));
  if (c->prm.precision == PSD_MIXED)
    TRY(launch_solve_graph(c, f, g, u, ran, [&]() { return mixed_graph_body(c, f, g, u); }));
  else
    TRY(launch_solve_graph(c, f, g, u, ran, [&]() { return fp64_graph_body(c, f, g, u); }));
  CK(cudaEventRecord(c->ev1, c->st));
  return PSD_OK;
}

// The solve's graph work enqueued on st (inside a capture), bracketed by the
// handle's timing events (recorded as event nodes of the graph).
psd_status solve_capture(psd_context* c, const double* f, const double* g, double* u, cudaStream_t st) {
  cudaStream_t saved = c->st;
  c->st = st;
  c->cap_depth = 0;
  c->capturing = true;
  psd_status s = PSD_OK;
  if (cudaEventRecordWithFlags(c->ev0, st, cudaEventRecordExternal) != cudaSuccess) s = PSD_ERR_CUDA;
  if (s == PSD_OK)
    s = (c->prm.precision == PSD_MIXED) ? mixed_graph_body(c, f, g, u) : fp64_graph_body(c, f, g, u);
  if (s == PSD_OK && cudaEventRecordWithFlags(c->ev1, st, cudaEventRecordExternal) != cudaSuccess) s = PSD_ERR_CUDA;
  c->capturing = false;
  c->st = saved;
  return s;
}

// The statistics of a solve whose graph work has completed.
psd_status solve_finish(psd_context* c, psd_info* info) {
  float ms = 0.f;
  CK(cudaEventSynchronize(c->ev1));  // the solve may still run on its stream
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  if (c->prm.precision == PSD_MIXED) {
    Ctrl h3;
    TRY(read_ctrl(c, c->ctrl3, h3));
    fill_info(info, h3.inner_total, h3.outer, h3.res_l2, h3.res_linf, h3.last_alpha, ms, h3.status);
    return (psd_status)h3.status;
  }
  Ctrl hc;
  TRY(read_ctrl(c, c->ctrl, hc));
  fill_info(info, hc.iter, 0, hc.res_l2, hc.res_linf, hc.alpha, ms, hc.status);
  return (psd_status)hc.status;
}

// Preconditioned conjugate gradients for H x = b in precision T, H = dN_h/du
// at `base` (order 4; the second variation of Sec. 5.3, symmetric positive
// definite), preconditioned by the FFT solve of L_h (the PSD search-direction
// operator).  Device resident: alpha, beta, (r, z) and the stop flag live in
// ctrl, the direction update p = z + beta p is fused into the Hessian-vector
// kernel, and chunks of kChunk iterations are replayed from a CUDA graph,
// the host reading the stop flag once per chunk.  x is zeroed first; r, q,
// w, z, pa, pb are work arrays (b may alias r).  Stops when ||r||_2 <=
// tol_abs or after max_iter iterations.
template <typename T>
psd_status cg_solve(psd_context* c, const T* base, const T* b, T* x, T* r, T* q, T* w, T* z, T* pa, T* pb,
                    const AxisTables<T>& tb, double tol_abs, int max_iter, cudaGraphExec_t* cache, Ctrl* out) {
  const KParams& kp = c->kp;
  const size_t bytes = c->N * sizeof(T);
  Ctrl h;
  init_ctrl(h, tol_abs, max_iter);
  h.cg = 1;
  h.rz = 0.0;
  TRY(upload_ctrl(c, c->ctrl, h));
  CK(cudaMemsetAsync(x, 0, bytes, c->st));
  CK(cudaMemsetAsync(pa, 0, bytes, c->st));  // p_0 = 0, so p_1 = z_0
  if (r != b) CK(cudaMemcpyAsync(r, b, bytes, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(w, b, bytes, cudaMemcpyDeviceToDevice, c->st));
  TRY(precond_passes<T>(c, w, z, c->ctrl, nullptr, nullptr, tb));  // z_0, (r_0, z_0), beta = 0
  auto chunk = [&]() -> psd_status {
    for (int i = 0; i < kChunk; ++i) {
      T* pold = (i % 2 == 0) ? pa : pb;
      T* pnew = (i % 2 == 0) ? pb : pa;
      // p_new = z + beta p_old (fused) and q = H p_new, alpha = (r, z) / (p, q)
      ResArgs<T> a{z, pold, pnew, nullptr, base, q, 0, 0};
      { ProfScope p_(c, cls_of<T>(PSD_PROF_RESIDUAL_FP64)); CK(psd::launch_residual<T>(a, psd::RM_HVP, c->pk, kp, c->ctrl, c->partials, c->st)); }
      { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_cg_update<T>(x, pnew, r, q, w, c->N, kp.hd, c->ctrl, c->partials, c->st)); }
      TRY(precond_passes<T>(c, w, z, c->ctrl, nullptr, nullptr, tb));  // z = L_h^{-1} r, beta
    }
    return PSD_OK;
  };
  int k = 0;
  Ctrl hc;
  for (;;) {
    TRY(run_chunk(c, cache, chunk));
    k += kChunk;
    TRY(read_ctrl(c, c->ctrl, hc));
    if (hc.done) break;
    if (k > max_iter + 2 * kChunk) {  // host-side guard: never loop unbounded
      hc.status = PSD_ERR_NOCONV;
      break;
    }
  }
  *out = hc;
  return PSD_OK;
}

// E_h[u] (Sec. 5.3 / 5.4 discrete energies; order 6 in the u = nu + gbar
// variables, with 1/2 ||u - g||_{-1}^2 = 1/2 (u - g, T_h[u - g])_2 by
// Parseval), FP64.  Uses W and ctrl2.
psd_status compute_energy(psd_context* c, const double* u, const double* f, const double* g, double* out) {
  const KParams& kp = c->kp;
  TRY(ensure_fp64(c));
  double gbar = 0.0;
  if (kp.order == 6) {
    Ctrl hg;
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_norms(g, c->N, kp.hd, c->ctrl2, c->partials, c->st)); }
    TRY(read_ctrl(c, c->ctrl2, hg));
    gbar = hg.rd / (double)c->N;
  }
  Ctrl h;
  init_ctrl(h, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h));
  { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_energy_terms(u, f, gbar, kp, c->ctrl2, c->partials, c->st)); }
  Ctrl t;
  TRY(read_ctrl(c, c->ctrl2, t));
  const double h2 = kp.h * kp.h;
  double E = kp.s / kp.p * kp.hd * std::pow(kp.q, kp.p) * t.tdd + 0.5 * kp.s * kp.eps2 * kp.hd * t.lapdd / (h2 * h2);
  if (kp.order == 4) {
    E += 0.5 * kp.hd * t.rd;
  } else {
    E += 0.5 * kp.lam * kp.s * kp.hd * t.rd - kp.hd * t.dd;
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_axpby<double>(c->W, u, g, 1.0, -1.0, 0.0, c->N, c->st)); }
    TRY(full_dht<double>(c, c->W, 1.0, c->tb64));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_spec_quad<double>(c->W, kp, c->ctrl2, c->partials, c->tb64, c->st)); }
    Ctrl q;
    TRY(read_ctrl(c, c->ctrl2, q));
    E += 0.5 * kp.hd * q.rd * kp.inv_ntot;
  }
  *out = E;
  return PSD_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

const char* psd_status_string(psd_status s) {
  switch (s) {
    case PSD_OK: return "PSD_OK";
    case PSD_ERR_INVALID: return "PSD_ERR_INVALID";
    case PSD_ERR_NOMEM: return "PSD_ERR_NOMEM";
    case PSD_ERR_CUDA: return "PSD_ERR_CUDA";
    case PSD_ERR_NOCONV: return "PSD_ERR_NOCONV";
    case PSD_ERR_TIMEOUT: return "PSD_ERR_TIMEOUT";
    case PSD_ERR_UNSUPPORTED: return "PSD_ERR_UNSUPPORTED";
    case PSD_ERR_NONFINITE: return "PSD_ERR_NONFINITE";
  }
  return "PSD_UNKNOWN_STATUS";
}

psd_status psd_create(const psd_params* params, psd_handle* out) {
  psd_context* c = nullptr;
  if (!out) return fail(nullptr, PSD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  std::string why;
  psd_status s = validate(params, why);
  if (s != PSD_OK) return fail(nullptr, s, why);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, PSD_ERR_CUDA, "no CUDA device");
  }
  c = new psd_context();
  c->prm = *params;
  c->st = (cudaStream_t)params->stream;
  KParams& kp = c->kp;
  kp.nx = params->n[0];
  kp.ny = params->n[1];
  kp.nz = params->dim == 3 ? params->n[2] : 1;
  kp.dim = params->dim;
  kp.h = params->h;
  kp.inv_h = 1.0 / params->h;
  kp.s = params->s;
  kp.eps2 = params->eps * params->eps;
  kp.lam = params->lambda;
  kp.p = params->p;
  kp.order = params->order;
  kp.cu = params->order == 4 ? 1.0 : params->s * params->lambda;
  kp.hd = params->dim == 3 ? params->h * params->h * params->h : params->h * params->h;
  c->N = (size_t)kp.nx * kp.ny * kp.nz;
  kp.inv_ntot = 1.0 / (double)c->N;
  psd::finish_kparams(kp);
  c->pk = (params->p == 4.0) ? psd::PK_4 : (params->p == 6.0) ? psd::PK_6 : psd::PK_GEN;
  static const bool attrs = (psd::init_dht_attributes(), true);  // once, thread-safe
  (void)attrs;

  auto bail = [&](psd_status st) {
    g_create_error = c->err;
    psd_destroy(c);
    return st;
  };
  if ((s = build_tables(c)) != PSD_OK) return bail(s);
  const size_t npart = std::max<size_t>(c->N / 16, 4096) * 8;
  if ((s = alloc(c, &c->partials, npart)) != PSD_OK) return bail(s);
  if ((s = alloc(c, &c->ctrl, 1)) != PSD_OK) return bail(s);
  if ((s = alloc(c, &c->ctrl2, 1)) != PSD_OK) return bail(s);
  if ((s = alloc(c, &c->ctrl3, 1)) != PSD_OK) return bail(s);
  if ((s = alloc(c, &c->ctrl_tmpl, 1)) != PSD_OK) return bail(s);
  if (cudaMemset(c->ctrl, 0, sizeof(Ctrl)) != cudaSuccess || cudaMemset(c->ctrl2, 0, sizeof(Ctrl)) != cudaSuccess ||
      cudaMemset(c->ctrl3, 0, sizeof(Ctrl)) != cudaSuccess || cudaMemset(c->ctrl_tmpl, 0, sizeof(Ctrl)) != cudaSuccess) {
    c->err = "cudaMemset failed";
    return bail(PSD_ERR_CUDA);
  }
  if (cudaMallocHost((void**)&c->h_ctrl, 4 * sizeof(Ctrl)) != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaMallocHost failed";
    return bail(PSD_ERR_NOMEM);
  }
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
    c->err = "cudaEventCreate failed";
    return bail(PSD_ERR_CUDA);
  }
  if ((s = ensure_fp64(c)) != PSD_OK) return bail(s);
  if (params->precision == PSD_MIXED && (s = ensure_fp32(c)) != PSD_OK) return bail(s);
  *out = c;
  return PSD_OK;
}

psd_status psd_destroy(psd_handle c) {
  if (!c) return PSD_OK;
  void* ptrs[] = {c->tables, c->ub, c->W, c->D, c->Z, c->Dsp, c->Ftf, c->Gtf, c->u32, c->da, c->db, c->W32, c->D32,
                  c->R32, c->Dsp32, c->partials, c->ctrl, c->ctrl2, c->ctrl3, c->ctrl_tmpl, c->d_hist, c->adj_q, c->adj_pb,
                  c->adj_u, c->adj32[0], c->adj32[1]};
  for (void* p : ptrs) dev_free(c, p);
  if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
  for (auto& x : c->g_solve)
    if (x.exec) cudaGraphExecDestroy(x.exec);
  if (c->g_cg32) cudaGraphExecDestroy(c->g_cg32);
  if (c->g_cg64) cudaGraphExecDestroy(c->g_cg64);
  if (c->gst) cudaStreamDestroy(c->gst);
  for (cudaStream_t q : c->capst)
    if (q) cudaStreamDestroy(q);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
  return PSD_OK;
}

psd_status psd_profile(psd_handle c, int enable) {
  if (!c) return PSD_ERR_INVALID;
  if (enable) {
    if (c->prof) TRY(prof_flush(c));
    c->recs.clear();
    for (int k = 0; k < PSD_PROF_CLASSES; ++k) {
      c->prof_ms[k] = 0.0;
      c->prof_n[k] = 0;
      c->prof_durs[k].clear();
    }
    // create the whole event pool now rather than while kernels are queued
    while (c->ev_pool.size() < 4096) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      c->ev_pool.push_back(e);
    }
  } else {
    TRY(prof_flush(c));
  }
  c->prof = enable != 0;
  c->prof_mask = ~0u;
  return PSD_OK;
}

psd_status psd_profile_classes(psd_handle c, unsigned mask) {
  if (!c) return PSD_ERR_INVALID;
  TRY(psd_profile(c, mask != 0 ? 1 : 0));
  c->prof_mask = mask;
  return PSD_OK;
}

psd_status psd_profile_read(psd_handle c, double* ms, long long* launches, double* eff_ms, long long* eff_launches,
                            double eff_us, int n) {
  if (!c || n < 0 || n > PSD_PROF_CLASSES) return PSD_ERR_INVALID;
  TRY(prof_flush(c));
  for (int k = 0; k < n; ++k) {
    if (ms) ms[k] = c->prof_ms[k];
    if (launches) launches[k] = c->prof_n[k];
    double em = 0.0;
    long long en = 0;
    for (float d : c->prof_durs[k])
      if (d * 1000.0 > eff_us) {
        em += d;
        ++en;
      }
    if (eff_ms) eff_ms[k] = em;
    if (eff_launches) eff_launches[k] = en;
  }
  return PSD_OK;
}

const char* psd_profile_class_name(int k) {
  static const char* names[PSD_PROF_CLASSES] = {
      "residual_fp64", "residual_fp32", "dht_rows_fp64", "dht_rows_fp32", "dht_cols_fp64", "dht_cols_fp32",
      "mid_fp64",      "mid_fp32",      "linesearch_fp64", "linesearch_fp32", "other",
      "dht_rows_ff",   "dht_cols_ff"};
  return (k >= 0 && k < PSD_PROF_CLASSES) ? names[k] : nullptr;
}

psd_status psd_last_error(psd_handle c, char* buf, size_t len) {
  if (!buf || len == 0) return PSD_ERR_INVALID;
  const std::string& e = c ? c->err : g_create_error;
  std::snprintf(buf, len, "%s", e.c_str());
  return PSD_OK;
}

psd_status psd_set_history(psd_handle c, double* alpha_hist, double* res_hist, int cap) {
  if (!c) return PSD_ERR_INVALID;
  if (cap < 0) return fail(c, PSD_ERR_INVALID, "cap must be >= 0");
  if (c->d_hist) {
    dev_free(c, c->d_hist);
    c->d_hist = nullptr;
  }
  c->hist_cap = 0;
  c->user_alpha = alpha_hist;
  c->user_res = res_hist;
  if ((alpha_hist || res_hist) && cap > 0) {
    TRY(alloc(c, &c->d_hist, 2 * (size_t)cap));
    c->hist_cap = cap;
  }
  return PSD_OK;
}

psd_status psd_residual(psd_handle c, const double* u, const double* f, const double* g, double* r,
                        double* res_l2, double* res_linf) {
  if (!c) return PSD_ERR_INVALID;
  if (!u || !f) return fail(c, PSD_ERR_INVALID, "u and f are required");
  if (c->prm.order == 6 && !g) return fail(c, PSD_ERR_INVALID, "order 6 requires g");
  TRY(ensure_fp64(c));
  double* out = r ? r : c->D;
  TRY(residual64(c, u, f, g, out));
  Ctrl h;
  TRY(read_ctrl(c, c->ctrl2, h));
  if (res_l2) *res_l2 = h.res_l2;
  if (res_linf) *res_linf = h.res_linf;
  return PSD_OK;
}

psd_status psd_residual_f32(psd_handle c, const float* u, const float* f, float* r) {
  if (!c) return PSD_ERR_INVALID;
  if (!u || !f || !r) return fail(c, PSD_ERR_INVALID, "u, f and r are required");
  Ctrl h;
  init_ctrl(h, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h));
  ResArgs<float> a{u, nullptr, nullptr, f, nullptr, r, 0, 0};
  { ProfScope p_(c, PSD_PROF_RESIDUAL_FP32); CK(psd::launch_residual<float>(a, psd::RM_PLAIN, c->pk, c->kp, c->ctrl2, c->partials, c->st)); }
  CK(cudaStreamSynchronize(c->st));
  return PSD_OK;
}

psd_status psd_residual_fixed(psd_handle c, const double* u, const double* f, double* r, int* scale) {
  if (!c) return PSD_ERR_INVALID;
  if (!u || !f || !r || !scale) return fail(c, PSD_ERR_INVALID, "u, f, r and scale are required");
  *scale = 0;
  const KParams& kp = c->kp;
  if (c->pk != psd::PK_4 || kp.dim != 3 || kp.nx < 32 || kp.ny < 8) return PSD_OK;
  Ctrl h;
  init_ctrl(h, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h));
  { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_norms(u, c->N, kp.hd, c->ctrl2, c->partials, c->st)); }
  Ctrl h2;
  TRY(read_ctrl(c, c->ctrl2, h2));
  const double umax = h2.res_linf;
  if (!std::isfinite(umax)) return PSD_OK;
  int e = 0;
  if (umax > 0.0) std::frexp(umax * (1.0 + std::ldexp(1.0, -20)), &e);
  const int S = 55 - e;
  if (S < 15 || S > 120) return PSD_OK;
  TRY(upload_ctrl(c, c->ctrl2, h));
  ResArgs<double> a{u, nullptr, nullptr, f, nullptr, r, 0, 0, 1, S};
  { ProfScope p_(c, PSD_PROF_RESIDUAL_FP64); CK(psd::launch_residual<double>(a, psd::RM_PLAIN, c->pk, kp, c->ctrl2, c->partials, c->st)); }
  CK(cudaStreamSynchronize(c->st));
  *scale = S;
  return PSD_OK;
}

psd_status psd_theta_ff(psd_handle c, const double* x, double* theta) {
  if (!c) return PSD_ERR_INVALID;
  if (!x || !theta) return fail(c, PSD_ERR_INVALID, "x and theta are required");
  TRY(ensure_fp64(c));
  const KParams& kp = c->kp;
  const int nrows = kp.ny * kp.nz;
  psd::ff* w = reinterpret_cast<psd::ff*>(c->D);
  { ProfScope p_(c, PSD_PROF_DHT_ROWS_FF); CK(psd::launch_dht_rows_ff(x, w, kp.nx, nrows, c->tbff, c->st)); }
  if (kp.dim == 3) { ProfScope p_(c, PSD_PROF_DHT_COLS_FF); CK(psd::launch_dht_cols_ff(w, kp, 1, c->tbff, c->st)); }
  { ProfScope p_(c, PSD_PROF_DHT_COLS_FF); CK(psd::launch_dht_last_ff(w, theta, nullptr, kp, nullptr, c->partials, c->tbff, c->st)); }
  CK(cudaStreamSynchronize(c->st));
  return PSD_OK;
}

psd_status psd_autotune(psd_handle c, int* caps) {
  if (!c) return PSD_ERR_INVALID;
  TRY(autotune(c));
  if (caps)
    for (int k = 0; k < 3; ++k) caps[k] = c->tb32.tile_cap[k];
  // captured solve graphs hold the old launch shapes
  for (auto& x : c->g_solve)
    if (x.exec) {
      cudaGraphExecDestroy(x.exec);
      x.exec = nullptr;
    }
  return PSD_OK;
}

psd_status psd_precond_solve(psd_handle c, const double* r, double* d) {
  if (!c) return PSD_ERR_INVALID;
  if (!r || !d) return fail(c, PSD_ERR_INVALID, "r and d are required");
  TRY(ensure_fp64(c));
  Ctrl h;
  init_ctrl(h, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h));
  if (d != r) CK(cudaMemcpyAsync(d, r, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  if (c->prm.order == 6) {
    CK(cudaMemsetAsync(c->Z, 0, c->N * sizeof(double), c->st));
    CK(cudaMemsetAsync(c->Dsp, 0, c->N * sizeof(double), c->st));
  }
  TRY(precond_passes<double>(c, d, d, c->ctrl2, c->Z, c->Dsp, c->tb64));
  return PSD_OK;
}

psd_status psd_precond_solve_f32(psd_handle c, const float* r, float* d) {
  if (!c) return PSD_ERR_INVALID;
  if (!r || !d) return fail(c, PSD_ERR_INVALID, "r and d are required");
  TRY(ensure_fp32(c));
  Ctrl h;
  init_ctrl(h, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h));
  if (d != r) CK(cudaMemcpyAsync(d, r, c->N * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
  if (c->prm.order == 6) {
    CK(cudaMemsetAsync(c->R32, 0, c->N * sizeof(float), c->st));
    CK(cudaMemsetAsync(c->Dsp32, 0, c->N * sizeof(float), c->st));
  }
  TRY(precond_passes<float>(c, d, d, c->ctrl2, c->prm.order == 6 ? c->R32 : nullptr, c->Dsp32, c->tb32));
  return PSD_OK;
}

psd_status psd_hvp(psd_handle c, const double* u, const double* v, double* y, double* dot) {
  if (!c) return PSD_ERR_INVALID;
  if (!u || !v || !y) return fail(c, PSD_ERR_INVALID, "u, v and y are required");
  if (c->prm.order != 4) return fail(c, PSD_ERR_UNSUPPORTED, "psd_hvp handles order 4");
  Ctrl h;
  init_ctrl(h, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h));
  ResArgs<double> a{v, nullptr, nullptr, nullptr, u, y, 0, 0};
  { ProfScope p_(c, PSD_PROF_RESIDUAL_FP64); CK(psd::launch_residual<double>(a, psd::RM_HVP, c->pk, c->kp, c->ctrl2, c->partials, c->st)); }
  Ctrl o;
  TRY(read_ctrl(c, c->ctrl2, o));
  if (dot) *dot = o.c1;
  return PSD_OK;
}

psd_status psd_adjoint(psd_handle c, const double* u, const double* grad_u, double* grad_f, double* grad_s,
                       double tol_rel, int max_iter, psd_info* info) {
  if (!c) return PSD_ERR_INVALID;
  if (!u || !grad_u || !grad_f) return fail(c, PSD_ERR_INVALID, "u, grad_u and grad_f are required");
  if (c->prm.order != 4) return fail(c, PSD_ERR_UNSUPPORTED, "psd_adjoint handles order 4");
  if (max_iter < 1) return fail(c, PSD_ERR_INVALID, "max_iter must be >= 1");
  if (!(tol_rel > 0)) tol_rel = 1e-12;
  TRY(ensure_fp64(c));
  TRY(alloc(c, &c->Z, c->N));
  TRY(alloc(c, &c->Dsp, c->N));
  TRY(alloc(c, &c->adj_q, c->N));
  const bool mixed = c->prm.precision == PSD_MIXED;
  if (mixed) {
    TRY(ensure_fp32(c));
    TRY(alloc(c, &c->adj32[0], c->N));
    TRY(alloc(c, &c->adj32[1], c->N));
  } else {
    TRY(alloc(c, &c->adj_pb, c->N));
    TRY(alloc(c, &c->adj_u, c->N));
  }
  const KParams& kp = c->kp;
  const size_t bytes = c->N * sizeof(double);
  // lambda lives in Dsp and is copied to grad_f at the end (grad_f may alias
  // grad_u); the FP64 solve works on a copy of u, so that every buffer of
  // its CG chunk belongs to the handle and one captured graph serves all calls
  double* lam = c->Dsp;
  CK(cudaEventRecord(c->ev0, c->st));
  Ctrl h0;
  init_ctrl(h0, -1.0, 1 << 30);
  TRY(upload_ctrl(c, c->ctrl2, h0));
  { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_norms(grad_u, c->N, kp.hd, c->ctrl2, c->partials, c->st)); }
  Ctrl hb;
  TRY(read_ctrl(c, c->ctrl2, hb));
  const double bnorm = hb.res_l2;
  int status = PSD_OK, iters = 0, outer = 0;
  double rel = 0.0;
  if (!std::isfinite(bnorm)) {
    status = PSD_ERR_NONFINITE;
  } else if (bnorm == 0.0) {
    CK(cudaMemsetAsync(lam, 0, bytes, c->st));
  } else if (!mixed) {
    // FP64: one device-resident CG solve to tol_rel ||b||
    CK(cudaMemcpyAsync(c->adj_u, u, bytes, cudaMemcpyDeviceToDevice, c->st));
    Ctrl hc;
    TRY(cg_solve<double>(c, c->adj_u, grad_u, lam, c->Z, c->adj_q, c->W, c->D, c->ub, c->adj_pb, c->tb64,
                         tol_rel * bnorm, max_iter, &c->g_cg64, &hc));
    iters = hc.iter;
    rel = hc.res_l2 / bnorm;
    status = hc.status;
  } else {
    // Mixed: FP64 outer residual R = b - H lambda (H at u), inner FP32 CG on
    // H delta = R (H at the FP32 copy of u) to kAdjInnerEta ||R||, lambda += delta
    CK(cudaMemsetAsync(lam, 0, bytes, c->st));
    CK(cudaMemsetAsync(c->adj_q, 0, bytes, c->st));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_round_f32(c->u32, u, c->N, c->st)); }
    const double eta = c->prm.inner_eta > 0.0 ? c->prm.inner_eta : kInnerEta;
    status = PSD_ERR_NOCONV;
    for (;;) {
      // R32 = (float)(b - H lambda), ||R||
      TRY(upload_ctrl(c, c->ctrl2, h0));
      { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_sub_round(grad_u, c->adj_q, c->R32, c->N, kp.hd, c->ctrl2, c->partials, c->st)); }
      Ctrl hr;
      TRY(read_ctrl(c, c->ctrl2, hr));
      ++outer;
      rel = hr.res_l2 / bnorm;
      if (!std::isfinite(rel)) {
        status = PSD_ERR_NONFINITE;
        break;
      }
      if (rel <= tol_rel) {
        status = PSD_OK;
        break;
      }
      if (iters >= max_iter || outer > std::max(c->prm.max_outer, 1) + 1) break;
      Ctrl hc;
      TRY(cg_solve<float>(c, c->u32, c->R32, c->adj32[0], c->R32, c->adj32[1], c->W32, c->D32, c->da, c->db, c->tb32,
                          eta * hr.res_l2, std::min(max_iter - iters, kInnerMaxIter), &c->g_cg32, &hc));
      iters += hc.iter;
      if (hc.status == PSD_ERR_NONFINITE) {
        status = PSD_ERR_NONFINITE;
        break;
      }
      if (hc.iter == 0) break;
      { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_add_f32(lam, c->adj32[0], c->N, c->st)); }
      // q = H lambda in FP64 (fresh control block: no CG bookkeeping)
      TRY(upload_ctrl(c, c->ctrl2, h0));
      ResArgs<double> a{lam, nullptr, nullptr, nullptr, u, c->adj_q, 0, 0};
      { ProfScope p_(c, PSD_PROF_RESIDUAL_FP64); CK(psd::launch_residual<double>(a, psd::RM_HVP, c->pk, kp, c->ctrl2, c->partials, c->st)); }
    }
  }
  // grad_s = -sum lam dN/ds, dN/ds = (N_h[u] - u)/s = (-r0 - u)/s with r0 = 0 - N_h[u]
  double gs = 0.0;
  {
    Ctrl hz;
    init_ctrl(hz, -1.0, 1 << 30);
    TRY(upload_ctrl(c, c->ctrl2, hz));
    ResArgs<double> a{u, nullptr, nullptr, nullptr, nullptr, c->W, 0, 0};
    { ProfScope p_(c, PSD_PROF_RESIDUAL_FP64); CK(psd::launch_residual<double>(a, psd::RM_PLAIN, c->pk, kp, c->ctrl2, c->partials, c->st)); }
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_dot(lam, c->W, u, c->N, c->ctrl2, c->partials, c->st)); }
    Ctrl o;
    TRY(read_ctrl(c, c->ctrl2, o));
    gs = o.rd / kp.s;  // -sum lam (-W - u)/s
  }
  CK(cudaMemcpyAsync(grad_f, lam, bytes, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaEventRecord(c->ev1, c->st));
  CK(cudaStreamSynchronize(c->st));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  if (grad_s) *grad_s = gs;
  if (info) {
    info->iters = iters;
    info->outer_iters = outer;
    info->res_l2 = rel;
    info->res_linf = -1.0;
    info->energy = NAN;
    info->last_alpha = 0.0;
    info->wall_ms = ms;
    info->status = status;
  }
  if (status != PSD_OK) fail(c, (psd_status)status, std::string("adjoint ended with ") + psd_status_string((psd_status)status));
  return (psd_status)status;
}

psd_status psd_solve(psd_handle c, const double* f, const double* g, double* u, double* w, psd_info* info) {
  if (!c) return PSD_ERR_INVALID;
  if (!f || !u) return fail(c, PSD_ERR_INVALID, "f and u are required");
  if (c->prm.order == 6 && !g) return fail(c, PSD_ERR_INVALID, "order 6 requires g");
  psd_status s = (c->prm.precision == PSD_MIXED) ? solve_mixed(c, f, g, u, info) : solve_fp64(c, f, g, u, info);
  if (s == PSD_ERR_CUDA || s == PSD_ERR_NOMEM || s == PSD_ERR_UNSUPPORTED) return s;
  if (c->hist_cap > 0 && c->prm.precision == PSD_FP64) {
    if (c->user_alpha)
      CK(cudaMemcpy(c->user_alpha, c->d_hist, c->hist_cap * sizeof(double), cudaMemcpyDeviceToHost));
    if (c->user_res)
      CK(cudaMemcpy(c->user_res, c->d_hist + c->hist_cap, c->hist_cap * sizeof(double), cudaMemcpyDeviceToHost));
  }
  if (c->prm.order == 6 && w) {
    // w = -T_h[u - g] + s lambda mean(g) - mean(f)
    const KParams& kp = c->kp;
    Ctrl hg, hf;
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_norms(g, c->N, kp.hd, c->ctrl2, c->partials, c->st)); }
    TRY(read_ctrl(c, c->ctrl2, hg));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_norms(f, c->N, kp.hd, c->ctrl2, c->partials, c->st)); }
    TRY(read_ctrl(c, c->ctrl2, hf));
    const double gbar = hg.rd / (double)c->N, fbar = hf.rd / (double)c->N;
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_axpby<double>(w, u, g, 1.0, -1.0, 0.0, c->N, c->st)); }
    TRY(full_dht<double>(c, w, 1.0, c->tb64));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_spec_apply_T<double>(w, 1.0, kp, c->tb64, c->st)); }
    TRY(full_dht<double>(c, w, kp.inv_ntot, c->tb64));
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_axpby<double>(w, w, nullptr, -1.0, 0.0, kp.s * kp.lam * gbar - fbar, c->N, c->st)); }
    CK(cudaStreamSynchronize(c->st));
  }
  if (c->prm.report_energy && info) TRY(compute_energy(c, u, f, g, &info->energy));
  if (s != PSD_OK)
    fail(c, s, std::string("solve ended with ") + psd_status_string(s));
  return s;
}

}  // extern "C"

namespace {
// Time loop shared by the thin-film and SPFC schemes: per step, rhs() forms
// the right-hand side(s) from u^n, then psd_solve runs from u^n.
template <typename Rhs>
psd_status run_steps(psd_context* c, double* u, int nsteps, psd_info* info, const double* g, Rhs&& rhs) {
  psd_info acc{};
  acc.status = PSD_OK;
  // own events: every psd_solve records the handle's ev0 / ev1
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  CK(cudaEventCreate(&t0));
  if (cudaEventCreate(&t1) != cudaSuccess) {
    cudaEventDestroy(t0);
    return fail(c, PSD_ERR_CUDA, "cudaEventCreate failed");
  }
  struct Events {
    cudaEvent_t a, b;
    ~Events() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev_guard{t0, t1};
  CK(cudaEventRecord(t0, c->st));
  psd_status s = PSD_OK;
  for (int n = 0; n < nsteps; ++n) {
    { ProfScope p_(c, PSD_PROF_OTHER); CK(rhs()); }
    psd_info one{};
    s = psd_solve(c, c->Ftf, g, u, nullptr, &one);
    acc.iters += one.iters;
    acc.outer_iters += one.outer_iters;
    acc.res_l2 = one.res_l2;
    acc.res_linf = one.res_linf;
    acc.energy = one.energy;
    acc.last_alpha = one.last_alpha;
    acc.status = one.status;
    if (s != PSD_OK) break;
  }
  CK(cudaEventRecord(t1, c->st));
  CK(cudaEventSynchronize(t1));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, t0, t1));
  acc.wall_ms = ms;
  if (info) *info = acc;
  return s;
}
}  // namespace

extern "C" {

psd_status psd_thinfilm_steps(psd_handle c, double* u, int nsteps, psd_info* info) {
  if (!c) return PSD_ERR_INVALID;
  if (!u || nsteps < 0) return fail(c, PSD_ERR_INVALID, "u is required and nsteps must be >= 0");
  if (c->prm.order != 4) return fail(c, PSD_ERR_INVALID, "the thin-film time loop needs a fourth-order handle");
  TRY(alloc(c, &c->Ftf, c->N));
  return run_steps(c, u, nsteps, info, nullptr, [&]() { return psd::launch_thinfilm_rhs(u, c->Ftf, c->kp, c->st); });
}

psd_status psd_spfc_steps(psd_handle c, double* u, double gamma1, int nsteps, psd_info* info) {
  if (!c) return PSD_ERR_INVALID;
  if (!u || nsteps < 0) return fail(c, PSD_ERR_INVALID, "u is required and nsteps must be >= 0");
  if (c->prm.order != 6) return fail(c, PSD_ERR_INVALID, "the SPFC time loop needs a sixth-order handle");
  if (!(gamma1 >= 0.0) || !std::isfinite(gamma1)) return fail(c, PSD_ERR_INVALID, "gamma1 must be finite and >= 0");
  TRY(alloc(c, &c->Ftf, c->N));
  TRY(alloc(c, &c->Gtf, c->N));
  const double cf = c->kp.s * gamma1;
  return run_steps(c, u, nsteps, info, c->Gtf,
                   [&]() { return psd::launch_spfc_rhs(u, c->Ftf, c->Gtf, cf, c->kp, c->st); });
}

psd_status psd_thinfilm_adjoint(psd_handle c, const double* u0, int nsteps, const double* grad_uN, double* grad_u0,
                                double* grad_s, int checkpoints, double tol_rel, int max_iter, psd_info* info) {
  if (!c) return PSD_ERR_INVALID;
  if (!u0 || !grad_uN || !grad_u0 || nsteps < 0)
    return fail(c, PSD_ERR_INVALID, "u0, grad_uN and grad_u0 are required and nsteps must be >= 0");
  if (c->prm.order != 4) return fail(c, PSD_ERR_INVALID, "the thin-film adjoint needs a fourth-order handle");
  if (max_iter < 1) return fail(c, PSD_ERR_INVALID, "max_iter must be >= 1");
  const size_t N = c->N, bytes = N * sizeof(double);
  const int ncp = checkpoints > 0 ? std::min(checkpoints, std::max(nsteps, 1))
                                  : std::max(1, (int)std::ceil(std::sqrt((double)nsteps)));
  const int K = nsteps > 0 ? (nsteps + ncp - 1) / ncp : 1;  // steps per segment
  const int nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;
  // workspace, released on return: the checkpoints u^{jK}, the states of one
  // segment, lambda, mu and a temporary
  struct Work {
    psd_context* c;
    double* p[5];
    ~Work() {
      for (double* q : p) dev_free(c, q);
    }
  } w{c, {nullptr, nullptr, nullptr, nullptr, nullptr}};
  TRY(alloc(c, &w.p[0], (size_t)std::max(nseg, 1) * N));
  TRY(alloc(c, &w.p[1], (size_t)(K + 1) * N));
  TRY(alloc(c, &w.p[2], N));
  TRY(alloc(c, &w.p[3], N));
  TRY(alloc(c, &w.p[4], N));
  TRY(alloc(c, &c->Ftf, N));
  double *ck = w.p[0], *seg = w.p[1], *lam = w.p[2], *mu = w.p[3], *tmp = w.p[4];
  const KParams& kp = c->kp;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  CK(cudaEventCreate(&t0));
  if (cudaEventCreate(&t1) != cudaSuccess) {
    cudaEventDestroy(t0);
    return fail(c, PSD_ERR_CUDA, "cudaEventCreate failed");
  }
  struct Events {
    cudaEvent_t a, b;
    ~Events() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev_guard{t0, t1};
  CK(cudaEventRecord(t0, c->st));
  int fwd_iters = 0, adj_iters = 0;
  auto step = [&](double* u) -> psd_status {  // one thin-film step in place
    { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_thinfilm_rhs(u, c->Ftf, kp, c->st)); }
    psd_info one{};
    const psd_status s = psd_solve(c, c->Ftf, nullptr, u, nullptr, &one);
    fwd_iters += one.iters;
    return s;
  };
  // forward: record u^{jK}; the last segment is recomputed by the backward pass
  CK(cudaMemcpyAsync(seg, u0, bytes, cudaMemcpyDeviceToDevice, c->st));
  for (int j = 0; j < nseg; ++j) {
    CK(cudaMemcpyAsync(ck + (size_t)j * N, seg, bytes, cudaMemcpyDeviceToDevice, c->st));
    if (j == nseg - 1) break;
    for (int t = 0; t < K; ++t) TRY(step(seg));
  }
  // backward: lambda_N = grad_uN; per step mu = H(u^{n+1})^{-1} lambda,
  // dJ/ds += -(mu . dN/ds) - (mu . Delta_h^v u^n), lambda = mu - s Delta_h^v mu
  CK(cudaMemcpyAsync(lam, grad_uN, bytes, cudaMemcpyDeviceToDevice, c->st));
  double gs = 0.0;
  for (int j = nseg - 1; j >= 0; --j) {
    const int len = std::min(K, nsteps - j * K);
    CK(cudaMemcpyAsync(seg, ck + (size_t)j * N, bytes, cudaMemcpyDeviceToDevice, c->st));
    for (int t = 1; t <= len; ++t) {
      double* ut = seg + (size_t)t * N;
      CK(cudaMemcpyAsync(ut, ut - N, bytes, cudaMemcpyDeviceToDevice, c->st));
      TRY(step(ut));
    }
    for (int t = len - 1; t >= 0; --t) {
      double* un = seg + (size_t)t * N;
      double gs_n = 0.0;
      psd_info ai{};
      TRY(psd_adjoint(c, un + N, lam, mu, &gs_n, tol_rel, max_iter, &ai));
      adj_iters += ai.iters;
      gs += gs_n;
      // -(mu . Delta_h^v u^n) = (mu . (u^n - s Delta_h^v u^n - u^n)) / s
      Ctrl h0;
      init_ctrl(h0, -1.0, 1 << 30);
      TRY(upload_ctrl(c, c->ctrl2, h0));
      {
        ProfScope p_(c, PSD_PROF_OTHER);
        CK(psd::launch_thinfilm_rhs(un, tmp, kp, c->st));
        CK(psd::launch_axpby<double>(tmp, tmp, un, 1.0, -1.0, 0.0, N, c->st));
        CK(psd::launch_dot(mu, tmp, nullptr, N, c->ctrl2, c->partials, c->st));
      }
      Ctrl hd;
      TRY(read_ctrl(c, c->ctrl2, hd));
      gs += hd.rd / kp.s;
      { ProfScope p_(c, PSD_PROF_OTHER); CK(psd::launch_thinfilm_rhs(mu, lam, kp, c->st)); }
    }
  }
  CK(cudaMemcpyAsync(grad_u0, lam, bytes, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaEventRecord(t1, c->st));
  CK(cudaEventSynchronize(t1));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, t0, t1));
  if (grad_s) *grad_s = gs;
  if (info) {
    *info = psd_info{};
    info->iters = adj_iters;
    info->outer_iters = fwd_iters;
    info->wall_ms = ms;
    info->status = PSD_OK;
  }
  return PSD_OK;
}

psd_status psd_energy(psd_handle c, const double* u, const double* f, const double* g, double* energy) {
  if (!c) return PSD_ERR_INVALID;
  if (!u || !f || !energy) return fail(c, PSD_ERR_INVALID, "u, f and energy are required");
  if (c->prm.order == 6 && !g) return fail(c, PSD_ERR_INVALID, "order 6 requires g");
  return compute_energy(c, u, f, g, energy);
}

}  // extern "C"

// Internal entry points of the batch driver (psd_batch.cu); not part of the C ABI.
namespace psd_internal {
psd_status prepare(psd_handle c, const double* f, const double* g, double* u) { return solve_prepare(c, f, g, u); }
psd_status capture(psd_handle c, const double* f, const double* g, double* u, cudaStream_t st) {
  return solve_capture(c, f, g, u, st);
}
psd_status finish(psd_handle c, psd_info* info) { return solve_finish(c, info); }
psd_status launch(psd_handle c, const double* f, const double* g, double* u, bool* ran) {
  return solve_launch(c, f, g, u, ran);
}
cudaStream_t stream(psd_handle c) { return c->st; }
psd_status tune(psd_handle c) { return autotune(c); }
void set_error(psd_handle c, const char* msg) { c->err = msg; }
}  // namespace psd_internal
