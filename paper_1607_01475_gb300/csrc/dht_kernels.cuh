// Discrete Hartley transform passes of the FFT preconditioner (Sec. 6: the
// search-direction equation L_h d = r is solved with the FFT), and the middle
// pass that divides by the symbol of L_h (Sec. 5.3, 5.4) and forms the
// Parseval sums the line search needs.
//
// Shared by the translation units k_dht_f32.cu, k_dht_f64.cu and
// k_dht_ff.cu, each of which instantiates one arithmetic type.
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "fft_line.cuh"
#include "kernels.h"

namespace psd {
namespace {

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};
struct __align__(16) ff2 {
  ff x, y;
};
template <>
struct Vec2<ff> {
  using type = ff2;
};

// x * scale, skipping the (double-word) product when scale is 1
template <typename T>
__device__ __forceinline__ T scaled(T x, T scale) {
  return x * scale;
}
template <>
__device__ __forceinline__ ff scaled<ff>(ff x, ff scale) {
  return (scale.hi == 1.0f && scale.lo == 0.0f) ? x : x * scale;
}

// Storage <-> compute element conversions (FP32, FP64, or float-float on
// FP64 storage).
template <typename C, typename S>
__device__ __forceinline__ C to_compute(S v) {
  return C(v);
}
template <typename S, typename C>
__device__ __forceinline__ S to_storage(C v) {
  return S(v);
}
template <>
__device__ __forceinline__ ff to_compute<ff, double>(double v) {
  return ff_from_double_bits(v);
}
template <>
__device__ __forceinline__ ff to_compute<ff, float>(float v) {
  return ff(v, 0.0f);
}
template <>
__device__ __forceinline__ double to_storage<double, ff>(ff v) {
  return ff_to_double_bits(v);
}

constexpr int kThreads = 256;

// Elements between the real arrays of consecutive line pairs in shared
// memory (each pair holds its real and imaginary line of F::L elements): the
// smallest LS >= F::L with LS = r (mod M), chosen so that the accesses of a
// warp in every pass of the line FFT spread over the 32 banks.  With EW the
// element size in 4-byte words: row passes (a warp spans 32/TS pairs) want
// r = m/2, M = m for m = TS/EW (odd LS when m < 2, free when m >= 32);
// column passes (a warp spans `pairs` pairs, 32/pairs threads each) want
// r = 16/k, M = 32/k for k = min(pairs EW, 16).  The rule was fitted to a
// wavefront count of the access pattern of every pass over N = 16..1024.
template <typename T, int N, int RM, bool ROWS>
__host__ __device__ constexpr int line_stride_words() {
  constexpr int L = LineFFT<T, N, RM>::L, TS = LineFFT<T, N, RM>::TS, EW = (int)(sizeof(T) / 4);
  int r = 0, M = 1;
  if (ROWS) {
    const int m = TS / EW;
    if (m >= 32) return L;
    r = m < 2 ? 1 : m / 2;
    M = m < 2 ? 2 : m;
  } else {
    const int k = (kThreads / TS) * EW < 16 ? (kThreads / TS) * EW : 16;
    r = 16 / k;
    M = 32 / k;
  }
  return L + (((r - L) % M) + M) % M;
}
constexpr size_t kMaxSmem = 96 * 1024;       // line-pair buffers of a block
constexpr size_t kMaxSmemPre = 200 * 1024;   // with the prefetch buffers of the last-axis passes

// Bytes of the line-pair region rounded up to 16 (the prefetch region follows).
__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// -------------------------------------------------------------- x (rows)
// S: element type in memory (SI of the source); T: arithmetic type.
template <typename S, typename T, int N, int RM, typename SI = S>
__global__ void __launch_bounds__(kThreads)
    k_dht_rows(const SI* src, S* dst, int nrows, T scale, const int* done, const T* __restrict__ twc,
               const T* __restrict__ tws) {
  using F = LineFFT<T, N, RM>;
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x;
  const int pairs = blockDim.x / F::TS;
  const int p = tid / F::TS, j = tid - p * F::TS;
  const int row0 = 2 * (blockIdx.x * pairs + p);
  const bool valid = row0 < nrows;
  constexpr int LS = line_stride_words<T, N, RM, true>();
  T* sr = sm + (size_t)p * 2 * LS;
  T* si = sr + LS;
  T vr[F::R], vi[F::R];
  const SI* s0 = src + (size_t)row0 * N;
#pragma unroll
  for (int q = 0; q < F::R; ++q) {
    vr[q] = valid ? to_compute<T>(s0[j + q * F::TS]) : T(0);
    vi[q] = valid ? to_compute<T>(s0[N + j + q * F::TS]) : T(0);
  }
  if constexpr (F::TS <= 32) {
    // a line's team is TS consecutive lanes: the last pass ends in registers
    // and the Hartley split takes X[N - k] from the partner lane by shuffle
    F::run_tw_regs(vr, vi, j, sr, si, TwPair<T>{twc, tws});
    T h1[F::R], h2[F::R];
    dht_split_regs<T, N, F::R, F::TS>(vr, vi, j, h1, h2);
    if (valid) {
      S* d0 = dst + (size_t)row0 * N;
#pragma unroll
      for (int q = 0; q < F::R; ++q) {
        const int k = j + q * F::TS;
        d0[k] = to_storage<S>(scaled(h1[q], scale));
        d0[N + k] = to_storage<S>(scaled(h2[q], scale));
      }
    }
  } else {
    F::run(vr, vi, j, sr, si, twc, tws);
    if (valid) {
      S* d0 = dst + (size_t)row0 * N;
#pragma unroll
      for (int q = 0; q < F::R; ++q) {
        const int k = j + q * F::TS;
        T h1, h2;
        dht_split(sr, si, k, N, h1, h2);
        d0[k] = to_storage<S>(scaled(h1, scale));
        d0[N + k] = to_storage<S>(scaled(h2, scale));
      }
    }
  }
}

// ------------------------------------------------------ strided lines (y, z)
// Block: `pairs` pairs of adjacent x-columns (x, x+1) packed as re/im, lines
// along the strided axis; thread (p, j) = (tid % pairs, tid / pairs) so that a
// warp reads whole row segments.
template <typename S, typename T, int N, int RM>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 || std::is_same<T, ff>::value ? 3 : 1)  // FP32 / float-float: 80 registers
    k_dht_cols(S* data, size_t line_stride, size_t outer_stride, T scale, const int* done,
               const T* __restrict__ twc, const T* __restrict__ tws) {
  using F = LineFFT<T, N, RM>;
  using V = typename Vec2<S>::type;
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x;
  const int pairs = blockDim.x / F::TS;
  const int p = tid % pairs, j = tid / pairs;
  const size_t base = (size_t)blockIdx.y * outer_stride + (size_t)blockIdx.x * 2 * pairs + 2 * p;
  constexpr int LS = line_stride_words<T, N, RM, false>();
  T* sr = sm + (size_t)p * 2 * LS;
  T* si = sr + LS;
  T vr[F::R], vi[F::R];
#pragma unroll
  for (int q = 0; q < F::R; ++q) {
    const V v = *reinterpret_cast<const V*>(data + base + (size_t)(j + q * F::TS) * line_stride);
    vr[q] = to_compute<T>(v.x);
    vi[q] = to_compute<T>(v.y);
  }
  F::run(vr, vi, j, sr, si, twc, tws);
#pragma unroll
  for (int q = 0; q < F::R; ++q) {
    const int k = j + q * F::TS;
    T h1, h2;
    dht_split(sr, si, k, N, h1, h2);
    V o;
    o.x = to_storage<S>(scaled(h1, scale));
    o.y = to_storage<S>(scaled(h2, scale));
    *reinterpret_cast<V*>(data + base + (size_t)k * line_stride) = o;
  }
}

// ------------------------------------ last axis, float-float, fused epilogue
// The last 1D DHT (z in 3D, y in 2D) of FP64 lines in float-float
// arithmetic; the transformed values h are not stored but consumed:
//   EPI_THETA:  theta += h / mu            (theta = DHT(T_h v) accumulates)
//   EPI_RESID:  out32 = h - theta (FP32), and sum of (h - theta)^2 into
//               ctrl->res_l2 = (h^d / N sum)^{1/2} (Parseval)
// with mu the symbol of -Delta_h at the element; the zero mode gives 0
// (mean-zero projection).  Same thread mapping as k_dht_cols.
enum { EPI_THETA = 0, EPI_RESID = 1 };
template <int N, int RM, int EPI>
__global__ void __launch_bounds__(kThreads, 3)  // 80 registers, 3 CTAs per SM
    k_dht_last_ff(const ff* data, double* theta, float* out32, size_t line_stride, size_t outer_stride,
                  KParams kp, Ctrl* ctrl, double* partials, const ff* __restrict__ twc,
                  const ff* __restrict__ tws, const ff* __restrict__ symx, const ff* __restrict__ symo,
                  const ff* __restrict__ syml, double* dc, const int* skip) {
  using T = ff;
  using F = LineFFT<T, N, RM>;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ float sred[32];
  __shared__ int sflag;
  const int tid = threadIdx.x;
  const int pairs = blockDim.x / F::TS;
  const int p = tid % pairs, j = tid / pairs;
  const int x = blockIdx.x * 2 * pairs + 2 * p;
  const size_t base = (size_t)blockIdx.y * outer_stride + x;
  constexpr int LS = line_stride_words<T, N, RM, false>();
  T* sr = sm + (size_t)p * 2 * LS;
  T* si = sr + LS;
  // theta of this thread's elements, copied asynchronously while the
  // forward transform runs: [q][j][p] double2
  double2* pre = reinterpret_cast<double2*>(smem_raw + align16((size_t)pairs * 2 * LS * sizeof(T)));
  T vr[F::R], vi[F::R];
#pragma unroll
  for (int q = 0; q < F::R; ++q) {
    const size_t idx = base + (size_t)(j + q * F::TS) * line_stride;
    const ff2 v = *reinterpret_cast<const ff2*>(data + idx);
    cp_async_16(pre + ((size_t)(q * F::TS + j) * pairs + p), theta + idx);
    vr[q] = v.x;
    vi[q] = v.y;
  }
  F::run(vr, vi, j, sr, si, twc, tws);
  cp_async_wait_all();
  const ff mo = symo != nullptr ? ld_tw(symo + blockIdx.y) : ff(0.0f, 0.0f);
  const ff mx[2] = {ff_add(ld_tw(symx + x), mo), ff_add(ld_tw(symx + x + 1), mo)};
  float acc = 0.0f;
#pragma unroll
  for (int q = 0; q < F::R; ++q) {
    const int k = j + q * F::TS;
    T h[2];
    dht_split(sr, si, k, N, h[0], h[1]);
    const ff ml = ld_tw(syml + k);
    const size_t idx = base + (size_t)k * line_stride;
    const double2 th = pre[(size_t)(q * F::TS + j) * pairs + p];
    const double thv[2] = {th.x, th.y};
    double outv[2];
    float o32[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const ff mu = ff_add(mx[c], ml);
      const bool live = mu.hi > 0.0f;
      if (EPI == EPI_THETA) {
        if (dc != nullptr && c == 0 && x == 0 && blockIdx.y == 0 && k == 0) *dc = ff_to_double_bits(h[0]);
        const ff t = live ? ff_mul(h[c], ff_recip(mu)) : ff(0.0f, 0.0f);
        outv[c] = ff_to_double_bits(ff_add(ff_from_double_bits(thv[c]), t));
      } else {
        const ff w = live ? ff_sub(h[c], ff_from_double_bits(thv[c])) : ff(0.0f, 0.0f);
        o32[c] = w.hi;
        acc = fmaf(w.hi, w.hi, acc);
      }
    }
    if (EPI == EPI_THETA) {
      *reinterpret_cast<double2*>(theta + idx) = make_double2(outv[0], outv[1]);
    } else {
      *reinterpret_cast<float2*>(out32 + idx) = make_float2(o32[0], o32[1]);
    }
  }
  if (EPI == EPI_RESID) {
    float v[1] = {acc};
    block_reduce<float, 1, false>(v, sred);
    if (publish_and_check_last<float>(v, 1, reinterpret_cast<float*>(partials), &ctrl->counter[CS_MID], &sflag)) {
      float tt[1];
      gather_partials<float, 1, false>(tt, reinterpret_cast<const float*>(partials), sred);
      if (tid == 0) {
        ctrl->res_l2 = sqrt((double)tt[0] * kp.hd * kp.inv_ntot);
        ctrl->res_linf = -1.0;
        ctrl->counter[CS_MID] = 0;
      }
    }
  }
}

// Block and grid reduction of the middle pass's five Parseval sums (fixed
// order) and the last block's bookkeeping: the sums into ctrl, the inner
// stopping rule on the preconditioned norm, the order-6 residual norm and
// convergence test, and the reset of the line-search state.
template <typename T, int ORDER>
__device__ __forceinline__ void mid_finish(T (&acc)[5], T* sred, double* partials, Ctrl* ctrl, const KParams& kp,
                                           int* sflag_) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  int& sflag = *sflag_;
  T v[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) v[m] = acc[m];
  block_reduce<T, 5, false>(v, sred);
  if (publish_and_check_last<T>(v, 5, reinterpret_cast<T*>(partials), &ctrl->counter[CS_MID], &sflag)) {
    T tt[5];
    gather_partials<T, 5, false>(tt, reinterpret_cast<const T*>(partials), sred);
    double tot[5];
    for (int m_ = 0; m_ < 5; ++m_) tot[m_] = (double)tt[m_];
    if (tid == 0 && ctrl->cg) {
      // conjugate gradients: z = L_h^{-1} r was just formed; beta = (r, z) /
      // (r, z)_previous goes to alpha for the direction update p = z + beta p
      // fused into the next Hessian-vector kernel (beta = 0 on the first pass)
      const double rz_new = tot[0] * kp.hd * kp.inv_ntot;
      ctrl->rd = rz_new;
      ctrl->alpha = (ctrl->rz > 0.0) ? rz_new / ctrl->rz : 0.0;
      ctrl->rz = rz_new;
      if (!isfinite(rz_new)) {
        ctrl->status = 7;
        ctrl->done = 1;
      }
      ctrl->counter[CS_MID] = 0;
    } else if (tid == 0) {
      const double w = kp.hd * kp.inv_ntot;
      ctrl->rd = tot[0] * w;
      ctrl->dd = tot[1] * w;
      ctrl->lapdd = tot[2] * w;
      ctrl->tdd = tot[3] * w;
      if (ctrl->pre_eta > 0.0) {
        // inner solve: stop when the preconditioned norm has dropped by
        // pre_eta, or when it has stopped halving (its rounding floor)
        const double pn = sqrt(fmax(ctrl->rd, 0.0));
        if (ctrl->pre_ref <= 0.0) {
          ctrl->pre_ref = pn;
          ctrl->pre_win = pn;
          ctrl->pre_stall = 0;
        } else if (pn < ctrl->pre_eta * ctrl->pre_ref) {
          ctrl->status = 0;
          ctrl->done = 1;
        } else if (pn < 0.5 * ctrl->pre_win) {
          ctrl->pre_win = pn;
          ctrl->pre_stall = 0;
        } else if (++ctrl->pre_stall >= ctrl->pre_stall_max) {
          ctrl->status = 0;
          ctrl->done = 1;
        }
      }
      if (ORDER == 6) {
        const double res = sqrt(tot[4] * w);
        ctrl->res_l2 = res;
        ctrl->res_linf = -1.0;
        const int it = ctrl->iter;
        if (ctrl->hist_res != nullptr && it < ctrl->hist_cap) ctrl->hist_res[it] = res;
        if (!isfinite(res)) {
          ctrl->status = 7;
          ctrl->done = 1;
        } else if (res < ctrl->tol) {
          ctrl->status = 0;
          ctrl->done = 1;
        } else if (it >= ctrl->max_iter) {
          ctrl->status = 4;
          ctrl->done = 1;
        }
      }
      // reset the line-search state for this iteration (general-p Newton:
      // bracket [c1, c2] with c2 < 0 meaning "no upper end yet", c3 = done)
      ctrl->c1 = 0.0;
      ctrl->c2 = -1.0;
      ctrl->c3 = 0.0;
      ctrl->alpha = 0.0;
      ctrl->ls_pass = 0;
      ctrl->counter[CS_MID] = 0;
    }
  }
}

// ------------------------------------------------------------- middle pass
// Tiles of 2 * pairs x-columns at one outer index (y in 3D), lines along the
// last axis.  PERSIST (the FP32 passes of the inner iteration): a grid of a
// few CTAs per SM loops over the tiles, and every thread prefetches, with
// cp.async into shared memory, its own elements of the next tile's data and
// of the current tile's xi / dspec, so that loads stay in flight while the
// transforms of the current tile run (no barrier is needed for the staged
// data: each thread reads only what it copied).  Otherwise one tile per CTA
// with direct loads.
template <typename T, int N, int ORDER, int RM, bool PERSIST>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 && ORDER == 4 && !PERSIST ? 3 : 2)
    k_mid(T* data, unsigned line_stride, unsigned outer_stride, int ntx, int ntiles, KParams kp, Ctrl* ctrl,
          double* partials, T* xi, T* dspec, const T* __restrict__ symx, const T* __restrict__ symo,
          const T* __restrict__ syml, const T* __restrict__ twc, const T* __restrict__ tws) {
  using F = LineFFT<T, N, RM>;
  using V = typename Vec2<T>::type;
  if (ctrl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ T sred[32 * 5];
  __shared__ int sflag;
  const int tid = threadIdx.x;
  const int pairs = blockDim.x / F::TS;
  const int p = tid % pairs, j = tid / pairs;
  constexpr int LS = line_stride_words<T, N, RM, false>();
  T* sr = sm + (size_t)p * 2 * LS;
  T* si = sr + LS;
  // staging ([q][j][p] pairs of columns): order 6 xi and dspec of the
  // current tile, then (PERSIST) two buffers of the data
  V* pre_x = reinterpret_cast<V*>(smem_raw + align16((size_t)pairs * 2 * LS * sizeof(T)));
  V* pre_d = pre_x + (size_t)N * pairs;
  V* pre_w = pre_x + (ORDER == 6 ? 2 : 0) * (size_t)N * pairs;
  // element offsets in 32 bits: every grid has fewer than 2^32 cells
  // staging index and line offset of the thread's q-th element; order 6
  // forms them from per-thread offsets taken once (with the inline form the
  // compiler spills there), order 4 keeps the inline form (no spill)
  constexpr bool HOIST = ORDER == 6;
  const unsigned e0 = (unsigned)j * pairs + p, estep = (unsigned)F::TS * pairs;
  const unsigned jl = (unsigned)j * line_stride, ql = (unsigned)F::TS * line_stride;
  auto elem = [&](int q) { return HOIST ? e0 + (unsigned)q * estep : (unsigned)(q * F::TS + j) * pairs + p; };
  auto goff = [&](int q) { return HOIST ? jl + (unsigned)q * ql : (unsigned)(j + q * F::TS) * line_stride; };
  auto tile_base = [&](int t) {
    const int xb = t % ntx, yo = t / ntx;
    return (unsigned)yo * outer_stride + (unsigned)(xb * 2 * pairs + 2 * p);
  };
  auto copy_vec = [&](V* dst, const T* src) {
    if (sizeof(V) == 8)
      cp_async_8(dst, src);
    else
      cp_async_16(dst, src);
  };
  const KConst<T>& C = kconst<T>(kp);
  const T s = C.s, se2 = C.se2, sl = C.sl;
  const T alpha_prev = (ORDER == 6) ? (T)ctrl->alpha : T(0);
  T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
  if (PERSIST && (int)blockIdx.x < ntiles) {
    const unsigned b0 = tile_base(blockIdx.x);
#pragma unroll
    for (int q = 0; q < F::R; ++q) copy_vec(pre_w + elem(q), data + (b0 + goff(q)));
    cp_async_commit();
  }
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int xb = t % ntx, yo = t / ntx;
    const int x = xb * 2 * pairs + 2 * p;
    const unsigned base = tile_base(t);
    V* wst = pre_w + (unsigned)(it & 1) * N * pairs;
    if (ORDER == 6) {
#pragma unroll
      for (int q = 0; q < F::R; ++q) {
        const unsigned idx = base + goff(q);
        copy_vec(pre_x + elem(q), xi + idx);
        copy_vec(pre_d + elem(q), dspec + idx);
      }
      cp_async_commit();
    }
    T vr[F::R], vi[F::R];
    if (PERSIST) {
      const int tn = t + gridDim.x;
      if (tn < ntiles) {
        const unsigned bn = tile_base(tn);
        V* wnx = pre_w + (unsigned)((it + 1) & 1) * N * pairs;
#pragma unroll
        for (int q = 0; q < F::R; ++q) copy_vec(wnx + elem(q), data + (bn + goff(q)));
      }
      cp_async_commit();
      // this tile's data is the oldest group in flight
      if (ORDER == 6)
        cp_async_wait_group<2>();
      else
        cp_async_wait_group<1>();
#pragma unroll
      for (int q = 0; q < F::R; ++q) {
        const V v = wst[elem(q)];
        vr[q] = v.x;
        vi[q] = v.y;
      }
    } else {
#pragma unroll
      for (int q = 0; q < F::R; ++q) {
        const V v = *reinterpret_cast<const V*>(data + (base + (unsigned)(j + q * F::TS) * line_stride));
        vr[q] = v.x;
        vi[q] = v.y;
      }
    }
    F::run(vr, vi, j, sr, si, twc, tws);
    if (ORDER == 6) {
      if (PERSIST)
        cp_async_wait_group<1>();
      else
        cp_async_wait_all();
    }

    const T mo = (symo != nullptr) ? symo[yo] : T(0);
    const T mxa = symx[x] + mo, mxb = symx[x + 1] + mo;
#pragma unroll
    for (int q = 0; q < F::R; ++q) {
      const int k = j + q * F::TS;
      T h[2];
      dht_split(sr, si, k, N, h[0], h[1]);
      const T ml = syml[k];
      T dv[2];
      if (ORDER == 4) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const T mu = (c ? mxb : mxa) + ml;
          const T dd = h[c] * recip_ge1(T(1) + mu * (s + se2 * mu));
          dv[c] = dd;
          acc[0] += h[c] * dd;
          acc[1] += dd * dd;
          acc[2] += (mu * dd) * (mu * dd);
        }
      } else {
        // xi holds the transformed part of the residual that is linear in the
        // iterate and not formed by the stencil kernel: -T_h[u - g] (plain
        // FP64) or R_outer - T_h[delta] (inner solve); it advances with the
        // previous step, xi -= alpha_prev T_h d_prev, where dspec keeps the
        // transform of T_h d_prev.  With L = lam s + s mu + s eps^2 mu^2 + 1/mu,
        // d = rt / L = mu rt / P and T_h d = d / mu = rt / P, where
        // P = 1 + mu (lam s + mu (s + s eps^2 mu)) >= 1: one reciprocal.
        const unsigned idx = base + (unsigned)k * line_stride;
        const V xv = pre_x[elem(q)];
        const V dp = pre_d[elem(q)];
        const T xs[2] = {xv.x, xv.y}, ds[2] = {dp.x, dp.y};
        T xn[2], tn[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const T mu = (c ? mxb : mxa) + ml;
          T rt = T(0), dd = T(0), xc = T(0), td = T(0);
          if (mu > T(0)) {
            xc = xs[c] - alpha_prev * ds[c];
            rt = h[c] + xc;
            td = rt * recip_ge1(T(1) + mu * (sl + mu * (s + se2 * mu)));
            dd = mu * td;
            acc[3] += dd * td;
          }
          xn[c] = xc;
          tn[c] = td;
          dv[c] = dd;
          acc[0] += rt * dd;
          acc[1] += dd * dd;
          acc[2] += (mu * dd) * (mu * dd);
          acc[4] += rt * rt;
        }
        V xo, o;
        xo.x = xn[0];
        xo.y = xn[1];
        o.x = tn[0];
        o.y = tn[1];
        *reinterpret_cast<V*>(xi + idx) = xo;
        *reinterpret_cast<V*>(dspec + idx) = o;
      }
      vr[q] = dv[0];
      vi[q] = dv[1];
    }
    __syncthreads();  // every thread has read the forward spectrum
    F::run(vr, vi, j, sr, si, twc, tws);
    const T scale = C.inv_ntot;
#pragma unroll
    for (int q = 0; q < F::R; ++q) {
      const int k = j + q * F::TS;
      T h1, h2;
      dht_split(sr, si, k, N, h1, h2);
      V o;
      o.x = h1 * scale;
      o.y = h2 * scale;
      *reinterpret_cast<V*>(data + (base + (unsigned)k * line_stride)) = o;
    }
    __syncthreads();  // the line buffers are rewritten by the next tile
  }
  if (PERSIST) cp_async_wait_all();
  mid_finish<T, ORDER>(acc, sred, partials, ctrl, kp, &sflag);
}

// ------------------------------------------------------ spectral helpers
template <typename T>
__device__ __forceinline__ T mu_at(size_t i, const KParams& kp, const T* sx, const T* sy, const T* sz) {
  const int x = (int)(i % kp.nx);
  const size_t rest = i / kp.nx;
  const int y = (int)(rest % kp.ny);
  const int z = (int)(rest / kp.ny);
  return sx[x] + sy[y] + (kp.dim == 3 ? sz[z] : T(0));
}

template <typename T>
__global__ void k_spec6_combine(T* a, const T* b, KParams kp, const T* sx, const T* sy, const T* sz, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T mu = mu_at(i, kp, sx, sy, sz);
    a[i] = (mu > T(0)) ? a[i] - b[i] / mu : T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_spec_quad(const T* a, KParams kp, const T* sx, const T* sy, const T* sz,
                                                   size_t n, Ctrl* ctrl, double* partials) {
  __shared__ double sred[32];
  __shared__ int sflag;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double mu = (double)mu_at(i, kp, sx, sy, sz);
    if (mu > 0.0) acc += (double)a[i] * (double)a[i] / mu;
  }
  double v[1] = {acc};
  block_reduce<double, 1, false>(v, sred);
  if (publish_and_check_last<double>(v, 1, partials, &ctrl->counter[CS_MID], &sflag)) {
    double tt[1];
    gather_partials<double, 1, false>(tt, partials, sred);
    if (threadIdx.x == 0) {
      ctrl->rd = tt[0];
      ctrl->counter[CS_MID] = 0;
    }
  }
}

template <typename T>
__global__ void k_spec_apply_T(T* a, T scale, KParams kp, const T* sx, const T* sy, const T* sz, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T mu = mu_at(i, kp, sx, sy, sz);
    a[i] = (mu > T(0)) ? scale * a[i] / mu : T(0);
  }
}

// ------------------------------------------------------------ launch helpers
// Radix of the register passes: 16 for the FP32 row/column passes; 8 where
// radix 16's register footprint would halve the occupancy (FP64, and the
// middle pass, which also holds the symbol-division state).
template <typename T>
constexpr int radix_pass() {
  return sizeof(T) == 8 ? 8 : 16;
}
template <typename T>
constexpr int radix_mid() {
  return 8;
}
template <typename T, int N, int RM, bool ROWS>
size_t pair_smem() {
  return 2 * (size_t)line_stride_words<T, N, RM, ROWS>() * sizeof(T);
}

// Number of column pairs per block: fill 256 threads, bounded by the shared
// memory budget, by the available pairs and by the autotuner's cap (0: no
// cap); a power of two.
template <typename T, int N, int RM, bool ROWS>
int pick_pairs(int avail_pairs, int cap = 0) {
  using F = LineFFT<T, N, RM>;
  int pairs = kThreads / F::TS;
  while (pairs > 1 && (size_t)pairs * pair_smem<T, N, RM, ROWS>() > kMaxSmem) pairs >>= 1;
  while (pairs > 1 && pairs > avail_pairs) pairs >>= 1;
  while (cap > 0 && pairs > 1 && pairs > cap) pairs >>= 1;
  return pairs < 1 ? 1 : pairs;
}

template <typename S, typename T, int N, typename SI = S>
cudaError_t rows_impl(const SI* src, S* dst, int nrows, T scale, const int* done, const T* twc,
                      const T* tws, cudaStream_t st, int cap = 0) {
  constexpr int RM = radix_pass<T>();
  using F = LineFFT<T, N, RM>;
  const int pairs = pick_pairs<T, N, RM, true>(1 << 30, cap);
  const int rows_per_block = 2 * pairs;
  const int grid = (nrows + rows_per_block - 1) / rows_per_block;
  k_dht_rows<S, T, N, RM, SI><<<grid, pairs * F::TS, pairs * pair_smem<T, N, RM, true>(), st>>>(
      src, dst, nrows, scale, done, twc, tws);
  return cudaGetLastError();
}

template <typename S, typename T, int N>
cudaError_t cols_impl(S* data, int nx, int nouter, size_t line_stride, size_t outer_stride, T scale,
                      const int* done, const T* twc, const T* tws, cudaStream_t st, int cap = 0) {
  constexpr int RM = radix_pass<T>();
  using F = LineFFT<T, N, RM>;
  const int pairs = pick_pairs<T, N, RM, false>(nx / 2, cap);
  dim3 grid(nx / (2 * pairs), nouter);
  k_dht_cols<S, T, N, RM><<<grid, pairs * F::TS, pairs * pair_smem<T, N, RM, false>(), st>>>(
      data, line_stride, outer_stride, scale, done, twc, tws);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t mid_impl(T* data, const KParams& kp, Ctrl* ctrl, double* partials, T* xi, T* dspec,
                     const AxisTables<T>& tb, cudaStream_t st) {
  constexpr int RM = radix_mid<T>();
  constexpr bool PERSIST = sizeof(T) == 4;
  using F = LineFFT<T, N, RM>;
  using V = typename Vec2<T>::type;
  const int nx = kp.nx;
  const int pairs = pick_pairs<T, N, RM, false>(nx / 2, tb.tile_cap[2]);
  size_t line_stride, outer_stride;
  int nouter;
  const T* symo;
  const T* syml;
  const T* twc;
  const T* tws;
  if (kp.dim == 2) {
    line_stride = nx;
    outer_stride = 0;
    nouter = 1;
    symo = nullptr;
    syml = tb.sym[1];
    twc = tb.twc[1];
    tws = tb.tws[1];
  } else {
    line_stride = (size_t)nx * kp.ny;
    outer_stride = nx;
    nouter = kp.ny;
    symo = tb.sym[1];
    syml = tb.sym[2];
    twc = tb.twc[2];
    tws = tb.tws[2];
  }
  const int ntx = nx / (2 * pairs);
  const int ntiles = ntx * nouter;
  // persistent: the CTAs that __launch_bounds__ keeps resident on every SM
  const int per_sm = 2;
  const int grid = PERSIST ? std::min(ntiles, per_sm * kp.nsm) : ntiles;
  const size_t sm = align16(pairs * pair_smem<T, N, RM, false>()) +
                    ((kp.order == 6 ? 2 : 0) + (PERSIST ? 2 : 0)) * (size_t)N * pairs * sizeof(V);
  if (sm > kMaxSmemPre) return cudaErrorInvalidConfiguration;
  if (kp.order == 4)
    k_mid<T, N, 4, RM, PERSIST><<<grid, pairs * F::TS, sm, st>>>(data, (unsigned)line_stride, (unsigned)outer_stride, ntx, ntiles, kp,
                                                                 ctrl, partials, xi, dspec, tb.sym[0], symo, syml,
                                                                 twc, tws);
  else
    k_mid<T, N, 6, RM, PERSIST><<<grid, pairs * F::TS, sm, st>>>(data, (unsigned)line_stride, (unsigned)outer_stride, ntx, ntiles, kp,
                                                                 ctrl, partials, xi, dspec, tb.sym[0], symo, syml,
                                                                 twc, tws);
  return cudaGetLastError();
}

template <typename T, int N>
void set_attrs_T() {
  constexpr int RP = radix_pass<T>(), RD = radix_mid<T>();
  cudaFuncSetAttribute(k_dht_rows<T, T, N, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
  cudaFuncSetAttribute(k_dht_cols<T, T, N, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
  constexpr bool PST = sizeof(T) == 4;
  cudaFuncSetAttribute(k_mid<T, N, 4, RD, PST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmemPre);
  cudaFuncSetAttribute(k_mid<T, N, 6, RD, PST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmemPre);
}

#define PSD_DISPATCH_N(n, CALL)      \
  switch (n) {                       \
    case 8: { constexpr int NN = 8; return CALL; }       \
    case 16: { constexpr int NN = 16; return CALL; }     \
    case 32: { constexpr int NN = 32; return CALL; }     \
    case 64: { constexpr int NN = 64; return CALL; }     \
    case 128: { constexpr int NN = 128; return CALL; }   \
    case 256: { constexpr int NN = 256; return CALL; }   \
    case 512: { constexpr int NN = 512; return CALL; }   \
    case 1024: { constexpr int NN = 1024; return CALL; } \
    default: return cudaErrorInvalidValue;               \
  }


}  // namespace

template <typename T>
cudaError_t launch_dht_rows(const T* src, T* dst, int nx, int nrows, T scale, const int* done,
                            const AxisTables<T>& tb, cudaStream_t st) {
  PSD_DISPATCH_N(nx, (rows_impl<T, T, NN>(src, dst, nrows, scale, done, tb.twc[0], tb.tws[0], st, tb.tile_cap[0])));
}

template <typename T>
cudaError_t launch_dht_cols(T* data, const KParams& kp, int ax, T scale, const int* done,
                            const AxisTables<T>& tb, cudaStream_t st) {
  const int n = ax == 1 ? kp.ny : kp.nz;
  size_t line_stride, outer_stride;
  int nouter;
  if (ax == 1) {
    line_stride = kp.nx;
    outer_stride = (size_t)kp.nx * kp.ny;
    nouter = kp.nz;
  } else {
    line_stride = (size_t)kp.nx * kp.ny;
    outer_stride = kp.nx;
    nouter = kp.ny;
  }
  PSD_DISPATCH_N(n, (cols_impl<T, T, NN>(data, kp.nx, nouter, line_stride, outer_stride, scale, done,
                                         tb.twc[ax], tb.tws[ax], st, tb.tile_cap[1])));
}

template <typename T>
cudaError_t launch_mid(T* data, const KParams& kp, Ctrl* ctrl, double* partials, T* xi, T* dspec,
                       const AxisTables<T>& tb, cudaStream_t st) {
  const int n = kp.dim == 2 ? kp.ny : kp.nz;
  PSD_DISPATCH_N(n, (mid_impl<T, NN>(data, kp, ctrl, partials, xi, dspec, tb, st)));
}

template <typename T>
cudaError_t launch_spec6_combine(T* a, const T* b, const KParams& kp, const AxisTables<T>& tb,
                                 cudaStream_t st) {
  const size_t n = (size_t)kp.nx * kp.ny * kp.nz;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
  k_spec6_combine<T><<<grid, 256, 0, st>>>(a, b, kp, tb.sym[0], tb.sym[1], tb.sym[2], n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_apply_T(T* a, T scale, const KParams& kp, const AxisTables<T>& tb, cudaStream_t st) {
  const size_t n = (size_t)kp.nx * kp.ny * kp.nz;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
  k_spec_apply_T<T><<<grid, 256, 0, st>>>(a, scale, kp, tb.sym[0], tb.sym[1], tb.sym[2], n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_quad(const T* a, const KParams& kp, Ctrl* ctrl, double* partials, const AxisTables<T>& tb,
                             cudaStream_t st) {
  const size_t n = (size_t)kp.nx * kp.ny * kp.nz;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 1024);
  k_spec_quad<T><<<grid, 256, 0, st>>>(a, kp, tb.sym[0], tb.sym[1], tb.sym[2], n, ctrl, partials);
  return cudaGetLastError();
}

}  // namespace psd
