// Internal launchers of the PSD CUDA kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "ffloat.cuh"
#include "psd_common.cuh"

namespace psd {

// Per-axis tables owned by a context, in FP64, FP32 and float-float.
template <typename T>
struct AxisTables {
  const T* twc[3];  // cos(2 pi t / n_a), t < n_a
  const T* tws[3];  // sin(2 pi t / n_a)
  const T* sym[3];  // (4/h^2) sin^2(pi k / n_a), k < n_a
  // tile widths chosen by the autotuner: at most this many line pairs per
  // block in the row, strided and middle passes (0: as many as fill 256
  // threads)
  int tile_cap[3];
};

// ----------------------------------------------------------------- DHT passes
// 1D DHT of every line along x (contiguous rows), src -> dst (may alias),
// multiplied by `scale`.  Skipped when *done != 0 (done may be null).
template <typename T>
cudaError_t launch_dht_rows(const T* src, T* dst, int nx, int nrows, T scale, const int* done,
                            const AxisTables<T>& tb, cudaStream_t st);

// 1D DHT of every line along axis `ax` (1 = y, 2 = z), in place.
template <typename T>
cudaError_t launch_dht_cols(T* data, const KParams& kp, int ax, T scale, const int* done,
                            const AxisTables<T>& tb, cudaStream_t st);

// Passes in float-float arithmetic (about 48 significant bits; tables of
// double-word twiddles).  Between passes the data stays in float-float form
// (hi, lo pairs in the 8 bytes of an FP64 element): the x pass reads FP64
// (or FP32) and writes pairs; the strided pass transforms pairs in place.
// skip (device, may be null): the pass returns at once when *skip != 0.
cudaError_t launch_dht_rows_ff(const double* src, ff* dst, int nx, int nrows, const AxisTables<ff>& tb,
                               cudaStream_t st, const int* skip = nullptr);
cudaError_t launch_dht_rows_ff_from_f32(const float* src, ff* dst, int nx, int nrows, const AxisTables<ff>& tb,
                                        cudaStream_t st, const int* skip = nullptr);
cudaError_t launch_dht_cols_ff(ff* data, const KParams& kp, int ax, const AxisTables<ff>& tb, cudaStream_t st,
                               const int* skip = nullptr);
// The last pass (z in 3D, y in 2D) with a fused epilogue: out32 == nullptr:
// theta += DHT(data) / mu, and (dc != null) *dc = the zero-frequency
// coefficient (the sum of the transformed field); else out32 = (float)(DHT(data)
// - theta) and ctrl->res_l2 = its Parseval norm (h^d / N sum)^{1/2}.  mu = 0
// gives 0.
cudaError_t launch_dht_last_ff(const ff* data, double* theta, float* out32, const KParams& kp, Ctrl* ctrl,
                               double* partials, const AxisTables<ff>& tb, cudaStream_t st, double* dc = nullptr,
                               const int* skip = nullptr);

// The middle pass along the slowest axis (y in 2D, z in 3D) of the
// preconditioner: forward DHT, division by the symbol of L_h, Parseval sums
// into ctrl, inverse DHT (with the 1/N of the whole transform).  Order 6
// also advances xi -= alpha_prev dspec (xi: the transformed linear part
// of the residual not formed by the stencil kernel, -T_h[u - g] or
// R_outer - T_h[delta]), adds it to the transformed local residual, stores
// the spectrum of T_h d for the new direction d in dspec and decides
// convergence on the spectral residual norm.
template <typename T>
cudaError_t launch_mid(T* data, const KParams& kp, Ctrl* ctrl, double* partials, T* xi, T* dspec,
                       const AxisTables<T>& tb, cudaStream_t st);

// Spectral helpers (order 6, off the hot loop).
// spec6_combine: a <- (mu == 0) ? 0 : a - b / mu   (a, b full DHT spectra)
// spec_apply_T:  a <- (mu == 0) ? 0 : scale * a / mu
template <typename T>
cudaError_t launch_spec6_combine(T* a, const T* b, const KParams& kp, const AxisTables<T>& tb,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_spec_apply_T(T* a, T scale, const KParams& kp, const AxisTables<T>& tb, cudaStream_t st);

// ------------------------------------------------------------------ stencils
// RM_PLAIN: r = f - N_h^{loc}[u];  RM_INNER: r = R - (N_h^{loc}[ubase + delta]
// - N_h^{loc}[ubase]);  RM_HVP: r = H v (H = dN_h/du at ubase, v = u_in),
// with h^d sum v.(H v) into ctrl->c1 and max|H v| into ctrl->c2.
enum ResMode { RM_PLAIN = 0, RM_INNER = 1, RM_HVP = 2 };

template <typename T>
struct ResArgs {
  const T* u_in;   // plain: iterate u; inner: correction delta
  const T* d;      // direction applied before evaluation (null: none)
  T* u_out;        // receives u_in + alpha d (only when d != null)
  const T* f;      // plain: right-hand side f; inner: outer residual R (null: 0)
  const T* ubase;  // inner: the outer iterate (rounded); else null
  T* r;            // residual (order 6: local part, without T_h)
  int norm;        // 1: reduce ||r|| into ctrl and decide convergence
  int update_iter; // 1: this call advances the iteration count
  int fluxff;      // FP64 plain without d, p = 4, 3D: fixed-point linear part and
                   // float-float flux (see k_res3d_col)
  int fxs;         // with fluxff: the fixed-point scale S (u = q 2^-S), in [15, 120]
  const int* fxs_dev;  // or (non-null) S read from device memory at launch: the fixed-point
                       // variant and the plain FP64 kernel are both launched and the one that
                       // does not apply (S outside [15, 120] / inside) returns at once
};

// r = f - N_h^{loc}[u_in + alpha d] (plain) or
// r = R - (N_h^{loc}[ubase + delta] - N_h^{loc}[ubase]) (inner, in a
// cancellation-free form), N_h^{loc} = cu I - s plap + s eps^2 Delta_h^2.
template <typename T>
cudaError_t launch_residual(const ResArgs<T>& a, int mode, int pk, const KParams& kp, Ctrl* ctrl,
                            double* partials, cudaStream_t st);

// Line search reduction over the vertices: a = grad(u [+ ubase]), b = grad(d).
// p = 4: the cubic coefficients, then the step size alpha by safeguarded
// Newton in the last block.  General p: one Newton step per launch.
template <typename T>
cudaError_t launch_linesearch(const T* u, const T* ubase, const T* d, int pk, const KParams& kp,
                              Ctrl* ctrl, double* partials, cudaStream_t st);

// max over vertices of |G|^2, G the unscaled vertex gradient sums of the
// FP32 field u (g = q G), into ctrl->res_linf (an estimate for choosing the
// float-float flux of the FP64 residual).  3D grids with nx >= 32, ny >= 8.
cudaError_t launch_gradmax(const float* u, const KParams& kp, Ctrl* ctrl, double* partials, cudaStream_t st);
// Right-hand side of the thin-film convex-splitting step (Sec. 6.1):
// f = u - s Delta_h^v u (FP64, 2D and 3D).
cudaError_t launch_thinfilm_rhs(const double* u, double* f, const KParams& kp, cudaStream_t st);
// Right-hand side of the SPFC convex-splitting step (Sec. 6.2):
// f = -c Delta_h u (c = s gamma_1), g = u (FP64, 2D and 3D).
cudaError_t launch_spfc_rhs(const double* u, double* f, double* g, double c, const KParams& kp, cudaStream_t st);

// Local sums of the discrete energy of u (FP64) into ctrl->rd, dd, lapdd,
// tdd: sum (u - f)^2 (order 4) or sum u^2 (order 6); sum (u - gbar) f
// (order 6); sum (h^2 Delta_h u)^2; sum over vertices |G|^p.
cudaError_t launch_energy_terms(const double* u, const double* f, double gbar, const KParams& kp, Ctrl* ctrl,
                                double* partials, cudaStream_t st);
// sum over the spectrum of a^2 / mu (mu > 0) into ctrl->rd (a: a DHT).
template <typename T>
cudaError_t launch_spec_quad(const T* a, const KParams& kp, Ctrl* ctrl, double* partials, const AxisTables<T>& tb,
                             cudaStream_t st);

// Number of blocks launch_residual<T> uses for this problem size (one
// partial sum record per block); fp32 = (T is float).
long long residual_grid_blocks(const KParams& kp, bool fp32);

// ------------------------------------------------- device-side loop control
// The conditional handles of CUDA graph WHILE nodes are set by these
// single-thread kernels at the end of each loop body.
// Loop while !c->done and the body count stays below guard_max (the guard
// trips PSD_ERR_NOCONV).
cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, Ctrl* c, int guard_max, cudaStream_t st);
// Set the condition to 1 just before a WHILE node (it keeps the value of the
// previous exit when an enclosing loop body runs the node again).
cudaError_t launch_cond_arm(cudaGraphConditionalHandle h, cudaStream_t st);
// General-p line search: another Newton pass while the bracket has not
// converged (c->c3 == 0), the run is not done, and fewer than max_passes ran.
cudaError_t launch_ls_cond(cudaGraphConditionalHandle h, Ctrl* c, int max_passes, cudaStream_t st);
// dst = src where c->iter is odd (the iterate ends in the second ping-pong buffer).
template <typename T>
cudaError_t launch_copy_if_odd(T* dst, const T* src, const Ctrl* c, size_t n, cudaStream_t st);
// Mixed solve, after each FP64 outer residual (norm in c2->res_l2): count it,
// decide convergence / failure into c3, and either stop the inner solve
// (c->done = 1) or initialise it from the template tmpl with max_iter =
// min(max_iter - inner_total, inner_cap).  cond: the outer WHILE handle.
cudaError_t launch_mixed_check(Ctrl* c3, const Ctrl* c2, Ctrl* c, const Ctrl* tmpl, double tol, int max_iter,
                               int max_outer, int inner_cap, int order6, cudaStream_t st);
// Mixed solve, after the inner solve: inner_total += c->iter, last alpha,
// non-finite inner residual -> c3 failed (done).
cudaError_t launch_mixed_after(Ctrl* c3, const Ctrl* c, cudaStream_t st);
// Mixed solve: the choice of the fixed-point / float-float FP64 residual
// (the host rule of the direct solve, on device) from the max |G|^2 and
// max|u| estimates in c2 (res_linf, res_l2) into c3->fxs.
cudaError_t launch_fluxff_decide(Ctrl* c3, const Ctrl* c2, double sqrt_vol, double cdiv, double tol, cudaStream_t st);
// c = a fresh control block (tol -1, no iteration limit), on device.
cudaError_t launch_ctrl_reset(Ctrl* c, cudaStream_t st);

// ------------------------------------------------------------ adjoint CG
// lam += alpha p, r -= alpha q, w = r; ||r||_2, iteration count and stopping
// test into ctrl (alpha = ctrl->alpha); no-op once ctrl->done is set.
template <typename T>
cudaError_t launch_cg_update(T* lam, const T* p, T* r, const T* q, T* w, size_t n, double hd, Ctrl* ctrl,
                             double* partials, cudaStream_t st);
// out32 = (float)(b - q), ||b - q||_2 into ctrl->res_l2.
cudaError_t launch_sub_round(const double* b, const double* q, float* out32, size_t n, double hd, Ctrl* ctrl,
                             double* partials, cudaStream_t st);
// y += (double) x.
cudaError_t launch_add_f32(double* y, const float* x, size_t n, cudaStream_t st);

// ------------------------------------------------------------------ misc
// y = a * x + b * z + c elementwise (x or z may be null = 0; may alias y).
template <typename T>
cudaError_t launch_axpby(T* y, const T* x, const T* z, double a, double b, double c, size_t n, cudaStream_t st);
// sum x (y + z) -> c->rd (z may be null).
cudaError_t launch_dot(const double* x, const double* y, const double* z, size_t n, Ctrl* c, double* partials,
                       cudaStream_t st);
// sum x -> c->rd, sqrt(hd sum x^2) -> c->res_l2, max|x| -> c->res_linf.
cudaError_t launch_norms(const double* x, size_t n, double hd, Ctrl* c, double* partials, cudaStream_t st);
// out = (float) in;  u += delta, u32 = (float) u  (mixed precision bookkeeping)
// u += mean(g - u) (order 6 mean projection), the mean kept in c->c2.
cudaError_t launch_mean_project(double* u, const double* g, size_t n, Ctrl* c, double* partials, cudaStream_t st);
cudaError_t launch_round_f32(float* out, const double* in, size_t n, cudaStream_t st);
// u += delta - mean(delta) (dsum: device pointer to sum(delta), or null for
// no mean removal), u32 = (float) u.
cudaError_t launch_accumulate_f64(double* u, const float* delta, float* u32, size_t n, const double* dsum,
                                  cudaStream_t st, const int* skip = nullptr);

void init_dht_attributes();

}  // namespace psd
