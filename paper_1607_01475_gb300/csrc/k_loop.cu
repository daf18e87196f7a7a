// Device-side control of the graph-driven solves.  A PSD solve (Algorithm 1
// structure, Sec. 2.2) is captured once into a CUDA graph whose loops are
// WHILE conditional nodes; the single-thread kernels here, at the end of a
// loop body, set the node's condition from the device-resident run state
// (Ctrl), so a whole solve -- and a whole batch of solves -- runs from one
// graph launch with no host round trip.  Every loop also counts its bodies
// against a hard cap, so a loop ends even if a stop flag were never set.
#include <cmath>

#include "kernels.h"

namespace psd {
namespace {

__global__ void k_loop_cond(cudaGraphConditionalHandle h, Ctrl* c, int guard_max) {
  unsigned v = 0u;
  if (!c->done) {
    const int g = ++c->guard;
    if (g < guard_max) {
      v = 1u;
    } else {  // the iteration limits should have stopped the loop before
      c->status = 4;
      c->done = 1;
    }
  }
  cudaGraphSetConditional(h, v);
}

// Arm a WHILE node: its condition keeps the value of the loop's last exit
// (0) when the enclosing body runs again, so a kernel placed just before the
// node sets it to 1 (the body then runs at least once).
__global__ void k_cond_arm(cudaGraphConditionalHandle h) { cudaGraphSetConditional(h, 1u); }

__global__ void k_ls_cond(cudaGraphConditionalHandle h, Ctrl* c, int max_passes) {
  unsigned v = 0u;
  if (!c->done && c->c3 == 0.0) v = (++c->ls_pass < max_passes) ? 1u : 0u;
  cudaGraphSetConditional(h, v);
}

template <typename T>
__global__ void k_copy_if_odd(T* dst, const T* src, const Ctrl* c, size_t n) {
  if ((c->iter & 1) == 0) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_mixed_check(Ctrl* c3, const Ctrl* c2, Ctrl* c, const Ctrl* tmpl, double tol, int max_iter,
                              int max_outer, int inner_cap, int order6) {
  if (c3->done) {
    c->done = 1;
    return;
  }
  const int outer = ++c3->outer;
  const double res = c2->res_l2;
  c3->res_l2 = res;
  c3->res_linf = order6 ? -1.0 : c2->res_linf;
  if (!isfinite(res)) {
    c3->status = 7;
    c3->done = 1;
  } else if (res < tol) {
    c3->status = 0;
    c3->done = 1;
  } else if (outer > max_outer || c3->inner_total >= max_iter) {
    c3->status = 4;
    c3->done = 1;
  }
  if (c3->done) {  // no further inner solve: its kernels return at once
    c->done = 1;
    c->iter = 0;
    return;
  }
  *c = *tmpl;
  const int left = max_iter - c3->inner_total;
  c->max_iter = left < inner_cap ? left : inner_cap;
}

__global__ void k_mixed_after(Ctrl* c3, const Ctrl* c) {
  if (c3->done) return;
  c3->inner_total += c->iter;
  c3->last_alpha = c->alpha;
  if (c->status == 7) {
    c3->status = 7;
    c3->done = 1;
  }
}

// The host rule of the direct mixed solve: the fixed-point / float-float
// residual applies when |Omega|^{1/2} 24 2^-47 cdiv (2 max|G|)^3 < tol / 20
// and S = 55 - e (max|u| (1 + 2^-20) < 2^e) lies in [15, 120].
__global__ void k_fluxff_decide(Ctrl* c3, const Ctrl* c2, double sqrt_vol, double cdiv, double tol) {
  int fxs = 0;
  const double gmax = 2.0 * sqrt(fmax(c2->res_linf, 0.0));
  const double bound = sqrt_vol * 24.0 * ldexp(1.0, -47) * cdiv * gmax * gmax * gmax;
  const double umax = c2->res_l2;
  if (tol > 0.0 && isfinite(bound) && bound < 0.05 * tol && isfinite(umax)) {
    int e = 0;
    if (umax > 0.0) frexp(umax * (1.0 + ldexp(1.0, -20)), &e);
    const int S = 55 - e;
    if (S >= 15 && S <= 120) fxs = S;
  }
  c3->fxs = fxs;
}

__global__ void k_ctrl_reset(Ctrl* c) {
  Ctrl z;
  memset(&z, 0, sizeof(z));
  z.tol = -1.0;
  z.max_iter = 1 << 30;
  z.res_linf = -1.0;
  z.c2 = -1.0;
  *c = z;
}

inline int grid1d(size_t n) { return (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16); }

}  // namespace

cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, Ctrl* c, int guard_max, cudaStream_t st) {
  k_loop_cond<<<1, 1, 0, st>>>(h, c, guard_max);
  return cudaGetLastError();
}
cudaError_t launch_cond_arm(cudaGraphConditionalHandle h, cudaStream_t st) {
  k_cond_arm<<<1, 1, 0, st>>>(h);
  return cudaGetLastError();
}
cudaError_t launch_ls_cond(cudaGraphConditionalHandle h, Ctrl* c, int max_passes, cudaStream_t st) {
  k_ls_cond<<<1, 1, 0, st>>>(h, c, max_passes);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_copy_if_odd(T* dst, const T* src, const Ctrl* c, size_t n, cudaStream_t st) {
  k_copy_if_odd<T><<<grid1d(n), 256, 0, st>>>(dst, src, c, n);
  return cudaGetLastError();
}
template cudaError_t launch_copy_if_odd<float>(float*, const float*, const Ctrl*, size_t, cudaStream_t);
template cudaError_t launch_copy_if_odd<double>(double*, const double*, const Ctrl*, size_t, cudaStream_t);
cudaError_t launch_mixed_check(Ctrl* c3, const Ctrl* c2, Ctrl* c, const Ctrl* tmpl, double tol, int max_iter,
                               int max_outer, int inner_cap, int order6, cudaStream_t st) {
  k_mixed_check<<<1, 1, 0, st>>>(c3, c2, c, tmpl, tol, max_iter, max_outer, inner_cap, order6);
  return cudaGetLastError();
}
cudaError_t launch_mixed_after(Ctrl* c3, const Ctrl* c, cudaStream_t st) {
  k_mixed_after<<<1, 1, 0, st>>>(c3, c);
  return cudaGetLastError();
}
cudaError_t launch_fluxff_decide(Ctrl* c3, const Ctrl* c2, double sqrt_vol, double cdiv, double tol,
                                 cudaStream_t st) {
  k_fluxff_decide<<<1, 1, 0, st>>>(c3, c2, sqrt_vol, cdiv, tol);
  return cudaGetLastError();
}
cudaError_t launch_ctrl_reset(Ctrl* c, cudaStream_t st) {
  k_ctrl_reset<<<1, 1, 0, st>>>(c);
  return cudaGetLastError();
}

}  // namespace psd
