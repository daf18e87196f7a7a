// Shared device-side definitions of the PSD library: parameter blocks, the
// device-resident control block, and deterministic grid reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace psd {

// Kinds of the vertex factor |g|^{p-2}: specialised p = 4 (|g|^2) and
// p = 6 (|g|^4 = (|g|^2)^2), and a general p (pow).
enum PKind { PK_GEN = 0, PK_4 = 4, PK_6 = 6 };

// Slots of the "last block" counters in the control block.
enum CounterSlot { CS_RES = 0, CS_MID = 1, CS_LS = 2, CS_MISC = 3, CS_COUNT = 8 };

// Device-resident state of one PSD run.  Written only by the last block of
// a reducing kernel (or by the host between runs).
struct Ctrl {
  int done;        // 1: converged, failed or stopped -> later kernels return
  int iter;        // completed PSD iterations
  int status;      // psd_status of the run
  int max_iter;    // iteration limit for this run
  double alpha;    // step size of the current iteration
  double tol;      // stop when res_l2 < tol
  double res_l2;   // ||r||_2 of the current iterate
  double res_linf; // max |r| of the current iterate (-1 if not formed)
  // Parseval sums of the current direction (already weighted by h^d / N):
  double rd;       // (r, d)_2
  double dd;       // (d, d)_2
  double lapdd;    // (Delta_h d, Delta_h d)_2
  double tdd;      // (T_h d, d)_2 (order 6)
  // line search: the first three polynomial coefficients of q (p = 4, 6;
  // weighted by h^d and s), or the general-p Newton state (c1, c2 = bracket,
  // c3 = converged flag)
  double c1, c2, c3;
  // inner (mixed-precision) stop on the preconditioned residual norm
  // (r, L_h^{-1} r)^{1/2} = ||d||_L (Eq. "RRT-1"): done when it drops below
  // pre_eta times its first value pre_ref (pre_eta <= 0 disables).
  double pre_eta;
  double pre_ref;
  double pre_win;  // value at the start of the current stall window
  int pre_stall;   // iterations without halving pre_win
  int pre_stall_max;
  // conjugate gradients (the adjoint solve): cg = 1 switches the middle pass
  // and the Hessian-vector kernel to their CG bookkeeping -- the middle pass
  // forms beta = (r, z) / rz into alpha and stores rz = (r, z); the
  // Hessian-vector kernel forms alpha = rz / (p, H p)
  int cg;
  int cg_pad_;
  double rz;
  // device-side loop control of graph-driven solves (WHILE nodes)
  int guard;        // body executions of the current loop (a hard cap)
  int ls_pass;      // general-p line search: Newton passes of this iteration
  int outer;        // mixed solve: FP64 outer residual evaluations
  int inner_total;  // mixed solve: inner iterations so far
  int fxs;          // mixed solve: fixed-point scale of the next outer residual (0: plain FP64)
  int max_outer;
  double last_alpha;
  unsigned int counter[CS_COUNT];
  int hist_cap;
  int pad_;
  double* hist_alpha;  // device arrays of length hist_cap (or null)
  double* hist_res;
};

// Problem scalars passed by value to the kernels.
// Constants of the operator in a kernel's arithmetic type, formed once on
// the host.  (Formed in a kernel from the FP64 parameters, a value such as
// (float)(s * eps2) may be recomputed inside unrolled loops when registers
// are short, and GB300 issues FP64 at 1/64 of the FP32 rate.)
template <typename T>
struct KConst {
  T s, se2, sl, cu;  // s, s eps^2, s lambda, coefficient of u
  T cdiv, cbih;      // see KParams
  T inv_h, inv_ntot;
  T beta, pm2;       // (p - 2) / 2, p - 2
};

struct KParams {
  int nx, ny, nz;       // cells per axis (nz = 1 in 2D)
  int dim;
  double h, inv_h;      // spacing
  double s, eps2, lam;  // s, eps^2, lambda
  double p;             // exponent
  double cu;            // coefficient of u in N_h: 1 (order 4) or s*lambda (6)
  double hd;            // h^d (cell volume)
  double inv_ntot;      // 1 / (nx ny nz)
  int order;
  int nsm;              // SMs of the current device (finish_kparams; sizes one-wave grids)
  // derived constants (set by finish_kparams): the column kernels work with
  // unscaled vertex-gradient sums G = g / q and Laplacian sums h^2 Delta_h.
  double q;             // 1 / (2^(d-1) h): g = q G
  double cdiv;          // s q^p: s d.(|g|^{p-2} g) = cdiv * (sum of differences of |G|^{p-2} G)
  double cbih;          // s eps^2 / h^4: s eps^2 Delta_h^2 u = cbih * (h^4 Delta_h^2 u)
  KConst<double> c64;   // the constants in FP64 and FP32 (finish_kparams)
  KConst<float> c32;
};

template <typename T>
__device__ __forceinline__ const KConst<T>& kconst(const KParams& kp);
template <>
__device__ __forceinline__ const KConst<double>& kconst<double>(const KParams& kp) {
  return kp.c64;
}
template <>
__device__ __forceinline__ const KConst<float>& kconst<float>(const KParams& kp) {
  return kp.c32;
}

// Fill the derived constants of KParams (host side).
inline void finish_kparams(KParams& kp) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    sms = 152;
  kp.nsm = sms;
  kp.q = kp.inv_h / (kp.dim == 3 ? 4.0 : 2.0);
  const double qp = (kp.p == 4.0) ? kp.q * kp.q * kp.q * kp.q : std::pow(kp.q, kp.p);
  kp.cdiv = kp.s * qp;
  kp.cbih = kp.s * kp.eps2 * kp.inv_h * kp.inv_h * kp.inv_h * kp.inv_h;
  KConst<double>& d = kp.c64;
  d.s = kp.s;
  d.se2 = kp.s * kp.eps2;
  d.sl = kp.s * kp.lam;
  d.cu = kp.cu;
  d.cdiv = kp.cdiv;
  d.cbih = kp.cbih;
  d.inv_h = kp.inv_h;
  d.inv_ntot = kp.inv_ntot;
  d.beta = 0.5 * (kp.p - 2.0);
  d.pm2 = kp.p - 2.0;
  KConst<float>& f = kp.c32;
  f.s = (float)d.s;
  f.se2 = (float)d.se2;
  f.sl = (float)d.sl;
  f.cu = (float)d.cu;
  f.cdiv = (float)d.cdiv;
  f.cbih = (float)d.cbih;
  f.inv_h = (float)d.inv_h;
  f.inv_ntot = (float)d.inv_ntot;
  f.beta = (float)d.beta;
  f.pm2 = (float)d.pm2;
}

// ------------------------------------------------------------------ reductions

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Reduce M values of type A over the block (fixed order: warp butterflies,
// then warp 0 over the warp results); the result is valid in thread 0.  The
// last value is reduced with max when LASTMAX is set, every value when
// ALLMAX is.  FP32 kernels reduce
// in float (GB300 issues FP64 at 1/64 of the FP32 rate), FP64 kernels in
// double.  Requires blockDim to be a multiple of 32 (<= 1024) or smaller
// than 32 (then thread 0 sums serially); uses a shared scratch of 32*M A's.
template <typename A, int M, bool LASTMAX, bool ALLMAX = false>
__device__ __forceinline__ void block_reduce(A (&v)[M], A* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  if (nthr < 32) {
    __syncthreads();
#pragma unroll
    for (int m = 0; m < M; ++m) sh[tid * M + m] = v[m];
    __syncthreads();
    if (tid == 0) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        A acc = sh[m];
        for (int t = 1; t < nthr; ++t) acc = (ALLMAX || (LASTMAX && m == M - 1)) ? fmax(acc, sh[t * M + m]) : acc + sh[t * M + m];
        v[m] = acc;
      }
    }
    __syncthreads();
    return;
  }
  const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
  for (int m = 0; m < M; ++m) v[m] = (ALLMAX || (LASTMAX && m == M - 1)) ? warp_max(v[m]) : warp_sum(v[m]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) sh[wid * M + m] = v[m];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      A x = (lane < nw) ? sh[lane * M + m] : ((ALLMAX || (LASTMAX && m == M - 1)) ? A(-1) : A(0));
      v[m] = (ALLMAX || (LASTMAX && m == M - 1)) ? warp_max(x) : warp_sum(x);
    }
  }
  __syncthreads();
}

// Write this block's partials, then return true in every thread of the
// block that finished last (threadFenceReduction pattern).  The last block
// can then read all partials with __ldcg.
template <typename A>
__device__ __forceinline__ bool publish_and_check_last(const A* v, int M, A* partials, unsigned int* counter,
                                                       int* sh_flag) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
  if (tid == 0) {
    for (int m = 0; m < M; ++m) partials[(size_t)bid * M + m] = v[m];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    *sh_flag = (prev == nb - 1) ? 1 : 0;
  }
  __syncthreads();
  return *sh_flag != 0;
}

// In the last block: sum the partials of all blocks in a fixed order (each
// thread a strided subset, then the block tree), result in thread 0.
template <typename A, int M, bool LASTMAX, bool ALLMAX = false>
__device__ __forceinline__ void gather_partials(A (&out)[M], const A* partials, A* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
#pragma unroll
  for (int m = 0; m < M; ++m) out[m] = (ALLMAX || (LASTMAX && m == M - 1)) ? A(-1) : A(0);
  for (unsigned int b = tid; b < nb; b += nthr) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      A x = __ldcg(partials + (size_t)b * M + m);
      out[m] = (ALLMAX || (LASTMAX && m == M - 1)) ? fmax(out[m], x) : out[m] + x;
    }
  }
  block_reduce<A, M, LASTMAX, ALLMAX>(out, sh);
}

// Tile order of the one-wave column march (residual and line-search
// kernels).  The column-planes w = column * nz + z are split into G =
// gridDim.x equal contiguous shares; the shares of CTAs b and b + G / g
// (g = gcd(G, ncol)) start exactly ncol / g whole columns apart, so those
// CTAs march the same plane at the same time.  The columns that agree
// modulo m = ncol / g are therefore in lockstep, and they are given
// consecutive tiles (whole rows of tiles when ncol / m is a multiple of the
// row length): a tile's x-neighbours are then read in the same plane step,
// and the halo reads they share hit L2 instead of DRAM.
__device__ __forceinline__ int lockstep_classes(int G, int ncol) {
  int a = G, b = ncol;
  while (b != 0) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return ncol / a;
}
__device__ __forceinline__ int lockstep_tile(int col, int m, int ncol) { return (col % m) * (ncol / m) + col / m; }

__device__ __forceinline__ int wrapi(int i, int n) {  // n a power of two
  return i & (n - 1);
}

// Asynchronous global -> shared copies (cp.async, 8 or 16 bytes, both
// addresses aligned to the size); a thread that reads back only its own
// copies needs cp_async_wait_all() and no barrier.
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Close the current group of this thread's cp.async copies; wait until at
// most N of its groups are still in flight.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// 1/x for finite x >= 1 (the preconditioner symbols).  FP32: the hardware
// reciprocal estimate (rcp.approx) refined by one Newton-Raphson step
// r <- r + r (1 - x r), which squares the estimate's relative error, so the
// result is within an ulp or so of 1/x; x >= 1 keeps it clear of
// denormals.  FP64: the IEEE quotient.
__device__ __forceinline__ float recip_ge1(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double recip_ge1(double x) { return 1.0 / x; }

}  // namespace psd
