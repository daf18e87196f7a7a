// psd_residual_noalloc: the fourth-order FP64 residual with its norms, for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is
// being captured into a CUDA graph under an allocator that forbids new
// allocations, plug-ins living inside a host application that owns every
// device allocation (and offers no hook to borrow from it), and real-time
// or fixed-budget deployments that must not grow their device footprint
// after start-up.  This entry point needs no handle and allocates nothing:
// the per-block partial sums and the reduction control block of the residual
// kernel live in one file-scope __device__ array of fixed size.
//
// Costs and limits of that choice:
//  * every GPU that loads this library holds the array (kScratchBytes) until
//    the process exits;
//  * problem sizes whose residual launch needs more than kMaxBlocks blocks
//    are rejected with PSD_ERR_INVALID;
//  * all calls share the array: calls that overlap on the GPU (different
//    streams, or different host threads) race and give wrong norms;
//  * the first call on each device looks the array's device address up with
//    cudaGetSymbolAddress; make that first call before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/psd.h"
#include "kernels.h"

namespace {

constexpr int kMaxBlocks = 2048;  // residual blocks: every valid grid needs at most 2048 on up to 1024 SMs
constexpr size_t kCtrlBytes = (sizeof(psd::Ctrl) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCtrlBytes + (size_t)kMaxBlocks * 2 * sizeof(double);
constexpr int kMaxDevices = 64;

// The scratch: [Ctrl, padded to 256 B][kMaxBlocks x 2 partial sums].
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};
thread_local std::string g_noalloc_error;

psd_status err(psd_status s, const std::string& m) {
  g_noalloc_error = m;
  return s;
}

bool pow2_in_range(int n) { return n >= 8 && n <= 1024 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" psd_status psd_residual_noalloc(const psd_params* prm, const double* u, const double* f, double* r,
                                           double* res_l2, double* res_linf) {
  if (!prm || !u || !f || !r) return err(PSD_ERR_INVALID, "params, u, f and r are required");
  if (prm->order != 4) return err(PSD_ERR_INVALID, "psd_residual_noalloc handles order 4 only");
  if (prm->dim != 2 && prm->dim != 3) return err(PSD_ERR_INVALID, "dim must be 2 or 3");
  for (int a = 0; a < prm->dim; ++a)
    if (!pow2_in_range(prm->n[a])) return err(PSD_ERR_INVALID, "n[a] must be a power of two in [8, 1024]");
  if (prm->dim == 2 && prm->n[2] != 1) return err(PSD_ERR_INVALID, "n[2] must be 1 in 2D");
  if (!(prm->h > 0) || !std::isfinite(prm->h) || !(prm->p >= 2) || !std::isfinite(prm->p) ||
      !(prm->s > 0) || !std::isfinite(prm->s) || !(prm->eps > 0) || !std::isfinite(prm->eps))
    return err(PSD_ERR_INVALID, "h, s, eps must be positive and p >= 2");
  if (prm->dim == 3 && prm->p > 6) return err(PSD_ERR_INVALID, "3D requires p <= 6");
  psd::KParams kp{};
  kp.nx = prm->n[0];
  kp.ny = prm->n[1];
  kp.nz = prm->dim == 3 ? prm->n[2] : 1;
  kp.dim = prm->dim;
  kp.h = prm->h;
  kp.inv_h = 1.0 / prm->h;
  kp.s = prm->s;
  kp.eps2 = prm->eps * prm->eps;
  kp.lam = 0.0;
  kp.p = prm->p;
  kp.order = 4;
  kp.cu = 1.0;
  kp.hd = prm->dim == 3 ? prm->h * prm->h * prm->h : prm->h * prm->h;
  kp.inv_ntot = 1.0 / ((double)kp.nx * kp.ny * kp.nz);
  psd::finish_kparams(kp);
  const long long blocks = psd::residual_grid_blocks(kp, false);
  if (blocks > kMaxBlocks) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "grid needs %lld residual blocks; the static scratch holds %d", blocks,
                  kMaxBlocks);
    return err(PSD_ERR_INVALID, buf);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return err(PSD_ERR_CUDA, "cudaGetDevice failed");
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_dev_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_dev_ptr[dev] = nullptr;
        return err(PSD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    base = g_dev_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)prm->stream;
  psd::Ctrl* ctrl = reinterpret_cast<psd::Ctrl*>(base);
  double* partials = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kCtrlBytes);
  // the last-block counter (and everything else in the control block) must
  // start at zero; the previous call left its values there
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(psd::Ctrl), st);
  if (e != cudaSuccess) return err(PSD_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  psd::ResArgs<double> a{u, nullptr, nullptr, f, nullptr, r, 1, 0};
  const int pk = (prm->p == 4.0) ? psd::PK_4 : (prm->p == 6.0) ? psd::PK_6 : psd::PK_GEN;
  e = psd::launch_residual<double>(a, psd::RM_PLAIN, pk, kp, ctrl, partials, st);
  if (e != cudaSuccess) return err(PSD_ERR_CUDA, std::string("residual launch: ") + cudaGetErrorString(e));
  double norms[2];
  e = cudaMemcpyAsync(norms, &ctrl->res_l2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return err(PSD_ERR_CUDA, std::string("norm read-back: ") + cudaGetErrorString(e));
  if (res_l2) *res_l2 = norms[0];
  if (res_linf) *res_linf = norms[1];
  return PSD_OK;
}

extern "C" psd_status psd_noalloc_last_error(char* buf, size_t len) {
  if (!buf || len == 0) return PSD_ERR_INVALID;
  std::snprintf(buf, len, "%s", g_noalloc_error.c_str());
  return PSD_OK;
}
