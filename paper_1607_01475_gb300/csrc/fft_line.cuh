// Line FFTs in shared memory and the discrete Hartley transform (DHT) built
// on them.
//
// Why the DHT: the preconditioner L_h, the Poisson inverse T_h and Delta_h
// all have Fourier symbols that depend on sin^2(pi k_a / n_a) only, i.e. are
// real and even in each wavenumber separately.  The separable Hartley
// transform H = H_x H_y H_z (kernel cas(2 pi j k / n) = cos + sin per axis)
// therefore diagonalises them with the same symbols, maps real grids to real
// grids of the same shape, and is its own inverse up to 1/N.  A 1D DHT of
// two real lines x, y is read off one complex FFT of z = x + i y:
//   with Z_k = A + iB and Z_{n-k} = C + iD,
//   H[x]_k = (A - B + C + D)/2,  H[y]_k = (A + B - C + D)/2.
//
// The complex FFT is a Stockham autosort FFT: a line of N points is handled
// by a team of TS = N/R threads holding R points each in registers; each pass
// of radix RP (RP | R) does R/RP butterflies per thread and exchanges data
// through shared memory.  Pass with Ns = product of earlier radices:
// butterfly j' reads x[j' + r N/RP], twiddles by W_N^{(j' mod Ns) r N/(Ns RP)},
// does an RP-point DFT and writes y[(j'/Ns) Ns RP + (j' mod Ns) + r Ns].
#pragma once

#include <cuda_runtime.h>

#include "ffloat.cuh"

namespace psd {

// Twiddle load through the read-only path, and x/2, for each element type.
template <typename T>
__device__ __forceinline__ T ld_tw(const T* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ ff ld_tw<ff>(const ff* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return ff(v.x, v.y);
}
template <typename T>
__device__ __forceinline__ T half_of(T x) {
  return T(0.5) * x;
}
template <>
__device__ __forceinline__ ff half_of<ff>(ff x) {
  return ff_scale2(x, 0.5f);
}

// a * b + c and c - a * b with one rounding where the type allows it.
template <typename T>
__device__ __forceinline__ T mul_add(T a, T b, T c) {
  return a * b + c;
}
template <>
__device__ __forceinline__ float mul_add<float>(float a, float b, float c) {
  return fmaf(a, b, c);
}
template <>
__device__ __forceinline__ double mul_add<double>(double a, double b, double c) {
  return fma(a, b, c);
}
template <typename T>
__device__ __forceinline__ T neg_mul_add(T a, T b, T c) {
  return c - a * b;
}
template <>
__device__ __forceinline__ float neg_mul_add<float>(float a, float b, float c) {
  return fmaf(-a, b, c);
}
template <>
__device__ __forceinline__ double neg_mul_add<double>(double a, double b, double c) {
  return fma(-a, b, c);
}

// Twiddle source: (cos, sin)(2 pi t / N) from two tables of the element type.
template <typename T>
struct TwPair {
  const T* __restrict__ c;
  const T* __restrict__ s;
  __device__ __forceinline__ void get(int t, T& cv, T& sv) const {
    cv = ld_tw(c + t);
    sv = ld_tw(s + t);
  }
};

// cos(2 pi m / 16), the 16th roots of unity (exact values of cos(pi/8),
// sin(pi/8) and sqrt(2)/2).
__host__ __device__ constexpr double cos16(int m) {
  return (m & 15) == 0 ? 1.0
       : (m & 15) == 1 ? 0.92387953251128675613
       : (m & 15) == 2 ? 0.70710678118654752440
       : (m & 15) == 3 ? 0.38268343236508977173
       : (m & 15) == 4 ? 0.0
       : (m & 15) == 5 ? -0.38268343236508977173
       : (m & 15) == 6 ? -0.70710678118654752440
       : (m & 15) == 7 ? -0.92387953251128675613
       : (m & 15) == 8 ? -1.0
       : (m & 15) == 9 ? -0.92387953251128675613
       : (m & 15) == 10 ? -0.70710678118654752440
       : (m & 15) == 11 ? -0.38268343236508977173
       : (m & 15) == 12 ? 0.0
       : (m & 15) == 13 ? 0.38268343236508977173
       : (m & 15) == 14 ? 0.70710678118654752440
                        : 0.92387953251128675613;
}
__host__ __device__ constexpr double sin16(int m) { return cos16(m - 4); }

// In-register DFT of size R (R | 16): radix-2 decimation in time, in-order
// input and output.  X_k = sum_j x_j exp(-2 pi i j k / R).
template <int R>
struct DFT {
  template <typename T>
  __device__ __forceinline__ static void run(T (&re)[R], T (&im)[R]) {
    T er[R / 2], ei[R / 2], orr[R / 2], oi[R / 2];
#pragma unroll
    for (int j = 0; j < R / 2; ++j) {
      er[j] = re[2 * j];
      ei[j] = im[2 * j];
      orr[j] = re[2 * j + 1];
      oi[j] = im[2 * j + 1];
    }
    DFT<R / 2>::run(er, ei);
    DFT<R / 2>::run(orr, oi);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      if (4 * k == R) {  // W = -i: (tr, ti) = (oi, -orr)
        re[k] = er[k] + oi[k];
        im[k] = ei[k] - orr[k];
        re[k + R / 2] = er[k] - oi[k];
        im[k + R / 2] = ei[k] + orr[k];
        continue;
      }
      T tr, ti;
      if (k == 0) {
        tr = orr[k];
        ti = oi[k];
      } else {  // W = c - i sn
        const T c = (T)cos16(k * 16 / R), sn = (T)sin16(k * 16 / R);
        tr = mul_add(oi[k], sn, orr[k] * c);
        ti = neg_mul_add(orr[k], sn, oi[k] * c);
      }
      re[k] = er[k] + tr;
      im[k] = ei[k] + ti;
      re[k + R / 2] = er[k] - tr;
      im[k + R / 2] = ei[k] - ti;
    }
  }
};
template <>
struct DFT<1> {
  template <typename T>
  __device__ __forceinline__ static void run(T (&)[1], T (&)[1]) {}
};

// Complex FFT of one line of N points by a team of TS threads (team index
// j).  Input: registers vr/vi holding x[j + q TS], q < R.  Output: the
// transform in natural order in sr/si (shared memory, length N), visible to
// the whole block on return.  Every thread of the block must call this
// (it contains __syncthreads).  twc/tws: cos/sin(2 pi t / N), t < N.
template <typename T, int N, int RMAX = 16>
struct LineFFT {
  static_assert(RMAX == 2 || RMAX == 4 || RMAX == 8 || RMAX == 16, "radix must divide 16");
  static constexpr int R = N < RMAX ? N : RMAX;
  static constexpr int TS = N / R;
  // Shared-memory index of point i: one padding word every 16 points, so
  // that the radix-R scatter of the first pass (stride R) and the strided
  // gathers hit distinct banks.  A line occupies L = N + N/16 words.
  static constexpr int L = N + N / 16;
  __device__ __forceinline__ static int pix(int i) { return i + (i >> 4); }

  template <int NS, typename Tw>
  __device__ __forceinline__ static void pass(T (&vr)[R], T (&vi)[R], int j, T* sr, T* si, const Tw& tw) {
    constexpr int RP = (N / NS >= R) ? R : N / NS;
    constexpr int M = R / RP;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const int jp = j + b * TS;
      const int jm = jp & (NS - 1);
      T xr[RP], xi[RP];
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        xr[r] = vr[b + r * M];
        xi[r] = vi[b + r * M];
      }
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < RP; ++r) {
          const int t = jm * r * (N / (NS * RP));
          T c, sn;
          tw.get(t, c, sn);
          const T a = xr[r], bb = xi[r];
          xr[r] = mul_add(bb, sn, a * c);
          xi[r] = neg_mul_add(a, sn, bb * c);
        }
      }
      DFT<RP>::run(xr, xi);
      const int base = (jp / NS) * NS * RP + jm;
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        sr[pix(base + r * NS)] = xr[r];
        si[pix(base + r * NS)] = xi[r];
      }
    }
  }

  template <int NS, typename Tw>
  __device__ __forceinline__ static void rest(T (&vr)[R], T (&vi)[R], int j, T* sr, T* si, const Tw& tw) {
    if constexpr (NS < N) {
      constexpr int RP = (N / NS >= R) ? R : N / NS;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < R; ++q) {
        vr[q] = sr[pix(j + q * TS)];
        vi[q] = si[pix(j + q * TS)];
      }
      __syncthreads();
      pass<NS>(vr, vi, j, sr, si, tw);
      rest<NS * RP>(vr, vi, j, sr, si, tw);
    }
  }

  // The last pass (NS * RP == N) with its results kept in registers: the
  // butterfly b of this thread writes outputs jp + r NS = j + TS (b + M r),
  // so after it the thread holds X[j + q TS] in vr[q] / vi[q] (q < R), the
  // same points it loaded.
  template <int NS, typename Tw>
  __device__ __forceinline__ static void last_pass_regs(T (&vr)[R], T (&vi)[R], int j, const Tw& tw) {
    constexpr int RP = N / NS;
    constexpr int M = R / RP;
    static_assert(RP * M == R, "last pass must cover the thread's points");
    T outr[R], outi[R];
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const int jp = j + b * TS;  // < NS, so jp mod NS = jp
      T xr[RP], xi[RP];
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        xr[r] = vr[b + r * M];
        xi[r] = vi[b + r * M];
      }
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < RP; ++r) {
          T c, sn;
          tw.get(jp * r, c, sn);
          const T a = xr[r], bb = xi[r];
          xr[r] = mul_add(bb, sn, a * c);
          xi[r] = neg_mul_add(a, sn, bb * c);
        }
      }
      DFT<RP>::run(xr, xi);
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        outr[b + M * r] = xr[r];
        outi[b + M * r] = xi[r];
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      vr[q] = outr[q];
      vi[q] = outi[q];
    }
  }

  template <int NS, typename Tw>
  __device__ __forceinline__ static void rest_regs(T (&vr)[R], T (&vi)[R], int j, T* sr, T* si, const Tw& tw) {
    constexpr int RP = (N / NS >= R) ? R : N / NS;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < R; ++q) {
      vr[q] = sr[pix(j + q * TS)];
      vi[q] = si[pix(j + q * TS)];
    }
    if constexpr (NS * RP < N) {
      __syncthreads();
      pass<NS>(vr, vi, j, sr, si, tw);
      rest_regs<NS * RP>(vr, vi, j, sr, si, tw);
    } else {
      last_pass_regs<NS>(vr, vi, j, tw);
    }
  }

  // As run_tw, but the transform ends in registers (vr[q] / vi[q] = X[j + q
  // TS]) instead of shared memory.  The line buffer is free on return only
  // after a barrier.
  template <typename Tw>
  __device__ __forceinline__ static void run_tw_regs(T (&vr)[R], T (&vi)[R], int j, T* sr, T* si, const Tw& tw) {
    if constexpr (R == N) {
      DFT<R>::run(vr, vi);  // one team thread holds the whole line
    } else {
      pass<1>(vr, vi, j, sr, si, tw);
      rest_regs<R>(vr, vi, j, sr, si, tw);
    }
  }

  template <typename Tw>
  __device__ __forceinline__ static void run_tw(T (&vr)[R], T (&vi)[R], int j, T* sr, T* si, const Tw& tw) {
    pass<1>(vr, vi, j, sr, si, tw);
    rest<R>(vr, vi, j, sr, si, tw);
    __syncthreads();
  }
  __device__ __forceinline__ static void run(T (&vr)[R], T (&vi)[R], int j, T* sr, T* si,
                                             const T* __restrict__ twc, const T* __restrict__ tws) {
    run_tw(vr, vi, j, sr, si, TwPair<T>{twc, tws});
  }
};

// Value of lane src of the same warp (float, double, or float-float as two
// shuffles of its words).
template <typename T>
__device__ __forceinline__ T shfl_from(unsigned mask, T v, int src) {
  return __shfl_sync(mask, v, src);
}
template <>
__device__ __forceinline__ ff shfl_from<ff>(unsigned mask, ff v, int src) {
  return ff(__shfl_sync(mask, v.hi, src), __shfl_sync(mask, v.lo, src));
}

// Hartley outputs of the two real lines of a spectrum held in registers by
// a team of TS <= 32 consecutive lanes (team thread j holds X[j + q TS] in
// vr[q] / vi[q], as run_tw_regs leaves it): X[N - k] for k = j + q TS is
// point R - 1 - q of team thread TS - j (j > 0), or this thread's own point
// (R - q) mod R (j = 0), so one shuffle per value replaces the round trip
// through shared memory.  Every thread of the block must call this (the
// block is a power of two threads).
template <typename T, int N, int R, int TS>
__device__ __forceinline__ void dht_split_regs(const T (&vr)[R], const T (&vi)[R], int j, T (&h1)[R], T (&h2)[R]) {
  static_assert(TS <= 32 && (TS & (TS - 1)) == 0 && TS * R == N, "team must fit in a warp");
  const int lane = threadIdx.x & 31;
  const int src = (lane & ~(TS - 1)) | ((TS - j) & (TS - 1));
  // blocks are a power of two threads: whole warps, or one partial warp
  const unsigned mask = blockDim.x >= 32 ? 0xffffffffu : (1u << blockDim.x) - 1u;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    T C = shfl_from(mask, vr[R - 1 - q], src);
    T D = shfl_from(mask, vi[R - 1 - q], src);
    if (j == 0) {
      C = vr[(R - q) % R];
      D = vi[(R - q) % R];
    }
    const T A = vr[q], B = vi[q];
    h1[q] = half_of((A - B) + (C + D));
    h2[q] = half_of((A + B) - (C - D));
  }
}

// Hartley outputs of the two real lines packed in a complex spectrum (the
// line stored with the padded index i + i/16).
template <typename T>
__device__ __forceinline__ void dht_split(const T* sr, const T* si, int k, int N, T& h1, T& h2) {
  const int k2 = (N - k) & (N - 1);
  const int a = k + (k >> 4), b = k2 + (k2 >> 4);
  const T A = sr[a], B = si[a], C = sr[b], D = si[b];
  h1 = half_of((A - B) + (C + D));
  h2 = half_of((A + B) - (C - D));
}

}  // namespace psd
