/*
 * psd.h -- C ABI of the GB300 (sm_103a) preconditioned steepest descent (PSD)
 * solver for the periodic finite-difference regularized p-Laplacian problems
 * of Feng, Salgado, Wang & Wise, arXiv:1607.01475.
 *
 * Problems (cell-centred periodic grid, spacing h, Sec. 5):
 *   order 4 (Eq. "discrete-4th-order", Sec. 5.3):
 *       N_h[u] := u - s grad_h^v.(|grad_h^v u|^{p-2} grad_h^v u) + s eps^2 Delta_h^2 u = f
 *   order 6 (Sec. 5.4, operator form of Sec. 6.2 with gamma_0 = lambda):
 *       u - Delta_h w = g,
 *       s lambda u - s grad_h^v.(...) + s eps^2 Delta_h^2 u - w = f,
 *     solved for u with mean(u) = mean(g) as N_h[u] := s lambda u - s grad.(..)
 *       + s eps^2 Delta_h^2 u + T_h[u - g] = f on the mean-zero space,
 *     T_h = -Delta_h^{-1}; then w = -T_h[u - g] + s lambda mean(g) - mean(f).
 *
 * The PSD step (Sec. 2.2, Sec. 6.1): d^k solves L_h d^k = r^k := f - N_h[u^k]
 * with the constant-coefficient preconditioner L_h = I - s Delta_h +
 * s eps^2 Delta_h^2 (order 4, Sec. 5.3) or s lambda I - s Delta_h +
 * s eps^2 Delta_h^2 + T_h (order 6, Sec. 5.4); u^{k+1} = u^k + alpha_k d^k with
 * alpha_k the unique root of q(alpha) = (N_h[u^k + alpha d^k] - f, d^k)_2
 * (Eq. "eqn-search").  3D operators are the tensor extension of the 2D ones.
 *
 * Conventions for every entry point:
 *  - Arrays are DEVICE pointers to contiguous float64 grids laid out
 *    [nz][ny][nx] (x fastest; 2D: [ny][nx], n[2] = 1).  The caller owns them.
 *  - Work is enqueued on the stream given in psd_params.stream (NULL = the
 *    legacy default stream).  Calls that return scalars to the host
 *    (psd_residual, psd_solve, psd_adjoint) synchronise that stream before
 *    returning; psd_precond_solve is asynchronous.
 *  - Every call returns a psd_status; nothing aborts.  After an error,
 *    psd_last_error() returns a one-line description.
 *  - A handle is not thread safe: one host thread at a time.
 */
#ifndef PSD_H
#define PSD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PSD_OK = 0,
  PSD_ERR_INVALID = 1,     /* bad parameter, size or pointer                 */
  PSD_ERR_NOMEM = 2,       /* device allocation failed                       */
  PSD_ERR_CUDA = 3,        /* a CUDA runtime call failed                     */
  PSD_ERR_NOCONV = 4,      /* max_iter / max_outer reached above tol         */
  PSD_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                  */
  PSD_ERR_UNSUPPORTED = 6, /* valid but not implemented combination          */
  PSD_ERR_NONFINITE = 7    /* NaN/Inf met in a residual or step size         */
} psd_status;

enum { PSD_FP64 = 0, PSD_MIXED = 1 };

typedef struct psd_params {
  int order;        /* 4 or 6                                                  */
  int dim;          /* 2 or 3                                                  */
  int n[3];         /* cells per axis (x, y, z): powers of two in [8, 1024];
                       n[2] = 1 in 2D                                          */
  double h;         /* isotropic grid spacing (Sec. 5.1), h > 0                */
  double p;         /* p >= 2 (Sec. 3.1; 3D requires p <= 6)                   */
  double s;         /* s > 0                                                   */
  double eps;       /* 0 < eps (the paper takes eps <= 1)                      */
  double lambda;    /* lambda >= 0, order 6 only                               */
  int precision;    /* PSD_FP64 or PSD_MIXED (FP32 inner PSD + FP64 outer
                       residual correction)                                    */
  double tol;       /* stop when ||r||_2 = (h^d sum r^2)^{1/2} < tol           */
  int max_iter;     /* PSD iterations (mixed: total inner iterations)         */
  int max_outer;    /* mixed mode: outer FP64 residual corrections             */
  void* stream;     /* cudaStream_t                                            */
  double inner_eta; /* mixed mode: an inner FP32 solve stops when its
                       preconditioned norm (r, L_h^{-1} r)^{1/2} has dropped by
                       this factor; 0 = default (1e-4); in [0, 1)               */
  int inner_stall;  /* ... or when that norm has not halved in this many
                       iterations (its FP32 floor); 0 = default (5)            */
  /* Optional device allocator for the handle's workspace (both NULL:
   * cudaMalloc / cudaFree).  alloc(bytes, alloc_ctx) returns device memory
   * aligned to 256 bytes or NULL; free_fn(ptr, alloc_ctx) releases it.  Every
   * workspace allocation of the handle goes through them, in psd_create or
   * on first use of a precision, and psd_destroy returns all of it.        */
  void* (*alloc)(size_t bytes, void* alloc_ctx);
  void (*free_fn)(void* ptr, void* alloc_ctx);
  void* alloc_ctx;
  int report_energy; /* 1: psd_solve also evaluates E_h of the result into
                        psd_info.energy (one extra FP64 pass)               */
} psd_params;

typedef struct psd_info {
  int iters;          /* PSD iterations (mixed: inner FP32 iterations)        */
  int outer_iters;    /* mixed: FP64 outer residual evaluations               */
  double res_l2;      /* final ||f - N_h[u]||_2 (order 6: mean-projected)     */
  double res_linf;    /* final max |r| (order 4 FP64; -1 when not formed)     */
  double energy;      /* E_h of the result when report_energy was set (Sec.
                         5.3 / 5.4 discrete energies), else NaN              */
  double last_alpha;  /* last step size                                       */
  double wall_ms;     /* device time of the solve (CUDA events)               */
  int status;         /* psd_status of the solve                              */
} psd_info;

typedef struct psd_context* psd_handle;

/* Create a solver for one problem size and parameter set.  Validates every
 * field (PSD_ERR_INVALID on a bad one), builds the transform tables and
 * allocates the device workspace with cudaMalloc (PSD_ERR_NOMEM).  The
 * workspace is owned by the handle and freed by psd_destroy.             */
psd_status psd_create(const psd_params* params, psd_handle* out);

/* Free the workspace and the handle (NULL is accepted).                  */
psd_status psd_destroy(psd_handle h);

/* Residual r = f - N_h[u] (order 6: P0[f - N_h[u]] with g required) as in
 * Sec. 6.1 and 6.2.  r may be NULL; res_l2 / res_linf are host pointers
 * (either may be NULL) receiving ||r||_2 and max|r|.  Always FP64.        */
psd_status psd_residual(psd_handle h, const double* u, const double* f,
                        const double* g, double* r, double* res_l2,
                        double* res_linf);

/* Discrete energy E_h[u] (Sec. 5.3, Eq. "diseng4"; order 6: Sec. 5.4 in the
 * u = nu + mean(g) variables) into *energy (host).  FP64; synchronises the
 * handle's stream.  g is required for order 6.                             */
psd_status psd_energy(psd_handle h, const double* u, const double* f,
                      const double* g, double* energy);

/* Search direction: solve L_h d = r by the FFT (Sec. 6; symbol of L_h from
 * Sec. 5.3 / 5.4).  Order 6 returns the mean-zero solution for P0 r.
 * r and d may alias.  Asynchronous on the handle's stream.  Always FP64.  */
psd_status psd_precond_solve(psd_handle h, const double* r, double* d);

/* The same solve in FP32 with the kernels of the mixed solver's inner
 * iteration.  r, d: float32 device grids; may alias.  Asynchronous.        */
psd_status psd_precond_solve_f32(psd_handle h, const float* r, float* d);

/* PSD solve of N_h[u] = f (order 6: with g) from the initial guess in u; u
 * is overwritten with the result.  w (order 6, may be NULL) receives
 * w = -T_h[u - g] + s lambda mean(g) - mean(f).  info (host, may be NULL)
 * receives the statistics.  Returns PSD_ERR_NOCONV if the tolerance was
 * not met within the iteration limits (u then holds the last iterate).
 * The whole solve runs from one CUDA graph (loops as conditional WHILE
 * nodes), captured on the first call with a given (u, f, g) and replayed
 * afterwards; a handle keeps the graphs of its last four pointer sets, so a
 * caller that alternates buffer sets (the next step's inputs copied in on
 * another stream while this step is solved) replays without capturing.
 * Returns when the solve is done (the handle's stream is synchronised).    */
psd_status psd_solve(psd_handle h, const double* f, const double* g,
                     double* u, double* w, psd_info* info);

/* Hessian-vector product y = H v, H = dN_h/du at u (the second variation of
 * E_h, Sec. 5.3, in the Euclidean product): H v = v - s grad_h^v.(W(Du) Dv)
 * + s eps^2 Delta_h^2 v with W(g) = |g|^{p-2} I + (p-2)|g|^{p-4} g g^T.
 * Order 4, FP64, device arrays; synchronises the stream.  dot (host, may be
 * NULL) receives h^d sum v.y.                                             */
psd_status psd_hvp(psd_handle h, const double* u, const double* v, double* y,
                   double* dot);

/* Gradient of a loss J(u) of the converged solution u of N_h[u] = f with
 * respect to f and s (order 4).  Not in the paper: by the implicit function
 * theorem, H lambda = grad_u (H = dN_h/du, the second variation of Sec. 5.3,
 * symmetric positive definite, solved by conjugate gradients preconditioned
 * with the FFT solve of L_h), grad_f = lambda and grad_s = -sum_i lambda_i
 * (dN_h/ds)_i, dN_h/ds = -grad_h^v.(|Du|^{p-2}Du) + eps^2 Delta_h^2 u.
 * The CG loop is device resident (step lengths and the stop flag in device
 * memory, chunks of iterations replayed from a CUDA graph).  On a PSD_FP64
 * handle it runs in FP64; on a PSD_MIXED handle the FP64 residual
 * R = grad_u - H lambda is corrected by FP32 CG solves of H delta = R (H at
 * the FP32 copy of u) to inner_eta ||R|| (default 1e-4).
 * u, grad_u: device arrays (grad_u = dJ/du entrywise); grad_f: device output
 * (may alias grad_u); grad_s: host double (may be NULL).  The solve stops
 * when ||grad_u - H lambda||_2 <= tol_rel ||grad_u||_2 (tol_rel <= 0 selects
 * 1e-12) or after max_iter CG iterations (PSD_ERR_NOCONV).  info (may be
 * NULL): iters = CG iterations (mixed: FP32 inner iterations), outer_iters =
 * FP64 residual evaluations (mixed), res_l2 = final relative residual.
 * Uses the handle's workspace; synchronises the stream.                   */
psd_status psd_adjoint(psd_handle h, const double* u, const double* grad_u,
                       double* grad_f, double* grad_s, double tol_rel,
                       int max_iter, psd_info* info);

/* Record per-iteration step sizes alpha_k and residual norms ||r_k||_2 of
 * subsequent psd_solve calls into host arrays of capacity cap (both may be
 * NULL to stop recording).  res_hist[0] is ||r_0||.                        */
psd_status psd_set_history(psd_handle h, double* alpha_hist, double* res_hist,
                           int cap);

/* FP32 residual of the stencil kernel (used by the mixed path), for tests:
 * r = f - N_h[u] in float (order 6: the local part, without T_h).          */
psd_status psd_residual_f32(psd_handle h, const float* u, const float* f,
                            float* r);

/* Thin-film epitaxy time loop (Sec. 6.1, Eq. "thin-film-fully-discrete"):
 * nsteps steps of the convex-splitting scheme N_h[u^{n+1}] = u^n -
 * s Delta_h^v u^n with the handle's fourth-order operator (s is the time
 * step), each solve started from u^n and run like psd_solve (the handle's
 * precision and tolerance).  u: device, N doubles, u^0 in, u^{nsteps} out.
 * info (host, may be NULL): iters and outer_iters summed over the steps,
 * res_l2, res_linf, last_alpha and status of the last solve, wall_ms of the
 * whole loop (CUDA events).  Stops at the first step whose solve fails and
 * returns its status.  Errors: PSD_ERR_INVALID for a null u, nsteps < 0 or
 * a sixth-order handle.                                                     */
psd_status psd_thinfilm_steps(psd_handle h, double* u, int nsteps,
                              psd_info* info);

/* Gradient of a loss J(u^N) of the thin-film time loop with respect to the
 * initial state u^0 and to s (order 4; entrywise, like psd_adjoint).  Not in
 * the paper: the chain rule backwards through the steps of
 * psd_thinfilm_steps.  With mu_n = H(u^{n+1})^{-1} lambda_{n+1} (one
 * psd_adjoint solve per step, tol_rel and max_iter as there):
 * lambda_n = mu_n - s Delta_h^v mu_n, and grad_s collects
 * -(mu_n . dN_h/ds(u^{n+1})) - (mu_n . Delta_h^v u^n).  The forward states
 * are recomputed from checkpoints: every K-th state is kept (K =
 * ceil(nsteps / checkpoints); checkpoints <= 0 selects ceil(sqrt(nsteps))),
 * and each segment is recomputed once on the way back, so the workspace is
 * about (checkpoints + K + 5) N doubles, allocated for the call (through
 * the allocator callback if set) and released before it returns.
 * u0, grad_uN (= dJ/du^N): device inputs; grad_u0: device output;
 * grad_s: host double or NULL.  info (host, may be NULL): iters = adjoint
 * CG iterations, outer_iters = forward PSD iterations (the recomputation
 * included), wall_ms.  Errors: PSD_ERR_INVALID (null pointers, nsteps < 0,
 * max_iter < 1, a sixth-order handle); the status of a failing solve.     */
psd_status psd_thinfilm_adjoint(psd_handle h, const double* u0, int nsteps,
                                const double* grad_uN, double* grad_u0,
                                double* grad_s, int checkpoints,
                                double tol_rel, int max_iter, psd_info* info);

/* Square phase field crystal time loop (Sec. 6.2, Eq. "scheme-spfc", with
 * the s-scaled explicit term of the scheme in Sec. 1): nsteps steps of the
 * sixth-order problem of Sec. 5.4 (lambda of the handle = gamma_0, p = 4
 * expected) with g = u^n and f = -s gamma1 Delta_h u^n, each solve started
 * from u^n.  mean(u) is kept.  u, info and errors as psd_thinfilm_steps,
 * for a sixth-order handle; gamma1 >= 0, finite.                           */
psd_status psd_spfc_steps(psd_handle h, double* u, double gamma1, int nsteps,
                          psd_info* info);

/* FP64 residual by the kernel variant of the mixed solve's outer residual,
 * for tests: r = f - N_h[u] (order 6: the local part, without T_h) with the
 * linear part (z-pair sums, vertex gradients, both Laplacian passes of
 * Sec. 5.1) in exact 64-bit fixed point, q = round(u 2^S), and the p = 4
 * flux part in float-float; only the final combination is FP64.  S = 55 - e
 * for max|u| (1 + 2^-20) < 2^e, returned in *scale.  Applies to p = 4 on 3D
 * grids with nx >= 32 and ny >= 8, and max|u| in [2^-65, 2^40); otherwise
 * *scale = 0 and r is not written.  u, f, r: device, N doubles; scale: host.
 * The solver's bound on the float-float error of the flux part is not
 * checked here.  Errors: PSD_ERR_INVALID for null pointers.                */
psd_status psd_residual_fixed(psd_handle h, const double* u, const double* f,
                              double* r, int* scale);

/* The float-float transform passes of the mixed sixth-order solver's outer
 * loop, for tests: theta += H[T_h x], with H the unnormalised separable
 * discrete Hartley transform (kernel prod_a cas(2 pi j_a k_a / n_a), which
 * diagonalises the symbols of Sec. 5.1 like the DFT of Sec. 6 does) and
 * T_h = -Delta_h^{-1} on the mean-zero space (Sec. 5.1; the zero mode
 * gives 0), computed in double-word arithmetic (about 48 significant bits)
 * on FP64 storage.  x, theta: device, N doubles each, must not alias; the
 * handle's direction buffer is used as scratch.  Synchronises the stream.
 * Errors: PSD_ERR_INVALID for null pointers.                               */
psd_status psd_theta_ff(psd_handle h, const double* x, double* theta);

/* Autotuner (not in the paper): choose the tile widths -- line pairs per
 * thread block -- of the FP32 row, strided-axis and middle transform passes
 * of a PSD_MIXED handle by timing each candidate on the handle's own buffers
 * over a few preconditioner solves, and use the fastest from then on.  The
 * choice is cached for the process by grid shape and order, so tuning a
 * second handle of the same shape costs nothing; psd_batch_create tunes
 * every mixed instance.  caps (host, 3 ints, may be NULL) receives the
 * chosen caps (0 = the widest tile, 256 threads).  A no-op for PSD_FP64
 * handles.  Synchronises the handle's stream.                              */
psd_status psd_autotune(psd_handle h, int* caps);

/* Kernel classes reported by psd_profile_read (index = class).            */
enum {
  PSD_PROF_RESIDUAL_FP64 = 0, PSD_PROF_RESIDUAL_FP32 = 1,
  PSD_PROF_DHT_ROWS_FP64 = 2, PSD_PROF_DHT_ROWS_FP32 = 3,
  PSD_PROF_DHT_COLS_FP64 = 4, PSD_PROF_DHT_COLS_FP32 = 5,
  PSD_PROF_MID_FP64 = 6,      PSD_PROF_MID_FP32 = 7,
  PSD_PROF_LINESEARCH_FP64 = 8, PSD_PROF_LINESEARCH_FP32 = 9,
  PSD_PROF_OTHER = 10,
  PSD_PROF_DHT_ROWS_FF = 11,  PSD_PROF_DHT_COLS_FF = 12,  /* float-float passes */
  PSD_PROF_CLASSES = 13
};

/* Per-kernel timing (tracing).  While enabled, every kernel launch of this
 * handle is bracketed by CUDA events on the handle's stream; the events
 * cost a few microseconds of host time per launch and do not change the
 * order of work.  psd_profile(h, 1) enables and clears the counters,
 * psd_profile(h, 0) disables.                                              */
psd_status psd_profile(psd_handle h, int enable);

/* As psd_profile(h, 1), but brackets only the launches of the classes whose
 * bit (1 << class) is set in mask (mask 0 disables).  Timing one class costs
 * the others nothing.                                                       */
psd_status psd_profile_classes(psd_handle h, unsigned mask);

/* Accumulated device milliseconds and launch counts per kernel class since
 * the last psd_profile(h, 1) (synchronises the stream).  Kernels launched
 * after the stop flag is set return at once; the "effective" figures count
 * only launches that ran longer than eff_us microseconds.  All arrays are
 * host arrays of length n (n <= PSD_PROF_CLASSES); any may be NULL.        */
psd_status psd_profile_read(psd_handle h, double* ms, long long* launches,
                            double* eff_ms, long long* eff_launches,
                            double eff_us, int n);

/* Static name of a kernel class ("residual_fp64", ...), or NULL.           */
const char* psd_profile_class_name(int k);

/* Fourth-order FP64 residual r = f - N_h[u] with ||r||_2 and max|r| (as
 * psd_residual), without a handle and without allocating any device memory.
 * The paper has no counterpart; this exists for callers that must not call
 * cudaMalloc -- code running during stream capture under an allocator that
 * refuses new allocations, plug-ins whose host application owns every device
 * allocation, and fixed-budget deployments.  The kernel's scratch (block
 * partial sums and the reduction control block) is a file-scope __device__
 * array of about 33 KB that every GPU loading the library keeps until exit.
 * params: order must be 4 and, as for psd_create, p <= 6 in 3D; its stream
 * is used; tol, max_iter, max_outer and precision are ignored.  u, f, r: device arrays as for psd_residual (r is
 * required); res_l2 / res_linf: host pointers or NULL.  Synchronises the
 * stream.  Returns PSD_ERR_INVALID for a bad size or parameter, including
 * grids whose residual launch needs more than 2048 blocks (none of the
 * valid sizes on a device with up to 1024 SMs: 3D grids run one wave of at
 * most 2 blocks per SM, 2D grids at most 1024 tiles, 3D grids with
 * nx < 32 at most 2048 blocks).  All calls share the scratch: calls
 * that overlap on the GPU race.  The first call on a device looks up the
 * scratch address; make it before any stream capture.                    */
psd_status psd_residual_noalloc(const psd_params* params, const double* u,
                                const double* f, double* r, double* res_l2,
                                double* res_linf);

/* Text of the last error of psd_residual_noalloc in this host thread.     */
psd_status psd_noalloc_last_error(char* buf, size_t len);

/* ---- Batches of independent instances (many uneven problem sizes). ----
 * Not in the paper.  psd_batch_create makes one solver per parameter set
 * (each with its own non-blocking stream; the stream fields of per_instance
 * are ignored).  psd_batch_solve solves every instance i from the initial
 * guess in u[i] (device arrays of instance i's size; g[i] for order-6
 * instances, g may be NULL when none is order 6) concurrently, from ONE CUDA
 * graph launch: each instance's solve -- its loops are conditional WHILE
 * nodes driven by its device-resident stop flags -- is a branch of a single
 * graph captured on the first call (and again when a pointer changes), so
 * the instances' kernels overlap on the GPU with no host round trip.  How
 * many branches run at once is bounded by the process's hardware work
 * queues: set CUDA_DEVICE_MAX_CONNECTIONS=32 in the environment before the
 * CUDA context is created (the default, 8, leaves ~7 instances running at a
 * time; on a GB300 the 96-instance 2D workload took 118 ms with 32 against
 * 143 ms with 8).  When a capture is not possible (kernel tracing on, or a
 * capture failure) each instance's own solve graph is launched on its
 * stream instead; psd_batch_set_mode can also select a pool of `workers`
 * host threads (<= 0: min(count, 16)).  It synchronises the device before starting and returns when all
 * instances are done; infos (host, count entries, may be NULL) receives
 * per-instance statistics (wall_ms: the instance's own span inside the
 * graph); the status is PSD_OK or the first failing instance's status
 * (psd_batch_last_error names it).  A failing instance does not stop the
 * others.                                                                 */
typedef struct psd_batch_ctx* psd_batch;
psd_status psd_batch_create(const psd_params* per_instance, int count,
                            int workers, psd_batch* out);
psd_status psd_batch_solve(psd_batch b, const double* const* f,
                           const double* const* g, double* const* u,
                           psd_info* infos);
psd_status psd_batch_destroy(psd_batch b);
psd_status psd_batch_last_error(psd_batch b, char* buf, size_t len);
/* Schedule of psd_batch_solve: 1 = one graph launch with a branch per
 * instance; 2 = every instance's own solve graph launched on its own stream
 * from the calling thread (no host round trip inside a solve); 3 = a pool
 * of host threads, one solve per thread at a time; 0 = the default (1).
 * PSD_ERR_INVALID for another value.  psd_batch_mode returns the schedule
 * the last solve used (a graph capture that fails falls back to 2;
 * 0 = no solve yet or b NULL).                                             */
psd_status psd_batch_set_mode(psd_batch b, int mode);
int psd_batch_mode(psd_batch b);

/* Text of the last error on this handle (or of the last psd_create failure
 * when h is NULL), copied into buf (always NUL-terminated).                */
psd_status psd_last_error(psd_handle h, char* buf, size_t len);

/* Static name of a status code.                                           */
const char* psd_status_string(psd_status s);

#ifdef __cplusplus
}
#endif

#endif /* PSD_H */
