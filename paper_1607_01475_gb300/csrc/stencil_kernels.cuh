// Residual and line-search kernels of the PSD iteration (included by the
// per-vertex-factor translation units k_res_p4.cu, k_res_p6.cu and
// k_res_pgen.cu, each of which instantiates one kind):
//   r = f - N_h[u],  N_h[u] = cu u - s d.(|D u|^{p-2} D u) + s eps^2 Delta_h^2 u
// (Eq. "discrete-4th-order", Sec. 5.3; the local part of the sixth-order
// operator of Sec. 5.4 / 6.2 with cu = s lambda), fused with the deferred
// update u <- u + alpha d (Eq. "eq:psd4"); and the line-search reduction that
// gives the step size alpha as the root of q(alpha) = (N_h[u + alpha d] - f, d)_2
// (Eq. "eqn-search", Sec. 6.1).
//
// D is the centre-to-vertex gradient and d. the vertex-to-centre divergence
// of Sec. 5.1; in 3D the tensor extension (D_x A_y A_z, d_x a_y a_z).  A CTA
// owns a TX x TY column of cells and marches along z keeping rolling planes
// of u (5, halo 2 in x/y), of Delta_h u (3, halo 1) and of the vertex fluxes
// (2 vertex planes) in shared memory.  Every vertex flux and every Laplacian
// value is computed once per CTA.
#pragma once

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "stencil_geom.h"

namespace psd {
namespace {

// |g|^{p-2} from g2 = |g|^2: g2 (p = 4), g2^2 (p = 6), else pow.
template <int PK, typename T>
__device__ __forceinline__ T vfactor(T g2, T beta) {
  if (PK == PK_4) return g2;
  if (PK == PK_6) return g2 * g2;
  return pow(g2, beta);  // beta = (p-2)/2; pow(0, 0) = 1, pow(0, b>0) = 0
}

// Flux difference F(a + e) - F(a), F(g) = |g|^{p-2} g, in a form whose
// rounding error scales with |e| (no cancellation of F(a) against itself).
template <int PK, typename T>
__device__ __forceinline__ void flux_diff(const T (&a)[3], const T (&e)[3], T beta, T (&out)[3]) {
  const T a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  // |a+e|^2 - |a|^2 = (2a + e).e, formed from e
  const T dl = (T(2) * a[0] + e[0]) * e[0] + (T(2) * a[1] + e[1]) * e[1] + (T(2) * a[2] + e[2]) * e[2];
  const T c2 = a2 + dl;  // |a+e|^2
  if (PK == PK_4) {
    // |a+e|^2 (a+e) - |a|^2 a = |a+e|^2 e + (|a+e|^2 - |a|^2) a
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = c2 * e[c] + dl * a[c];
  } else if (PK == PK_6) {
    // |a+e|^4 (a+e) - |a|^4 a = |a+e|^4 e + (|a+e|^2 - |a|^2)(|a+e|^2 + |a|^2) a
    const T c4 = c2 * c2, w = dl * (c2 + a2);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = c4 * e[c] + w * a[c];
  } else {
    const T fc = pow(c2 > T(0) ? c2 : T(0), beta);
    T dfac;  // |a+e|^{p-2} - |a|^{p-2}
    if (a2 > T(0))
      dfac = pow(a2, beta) * expm1(beta * log1p(dl / a2));
    else
      dfac = fc;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = fc * e[c] + dfac * a[c];
  }
}

template <int PK, typename T>
__device__ __forceinline__ void flux(const T (&g)[3], T beta, T (&out)[3]) {
  const T g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  const T f = vfactor<PK>(g2, beta);
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = f * g[c];
}

// Linearised flux W(a) e = |a|^{p-2} e + (p-2)|a|^{p-4} (a.e) a (the second
// variation of Sec. 5.3; the (p-2)-term is 0 where a = 0 for p < 4).
template <int PK, typename T>
__device__ __forceinline__ void flux_lin(const T (&a)[3], const T (&e)[3], T beta, T (&out)[3]) {
  const T a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  const T ae = a[0] * e[0] + a[1] * e[1] + a[2] * e[2];
  if (PK == PK_4) {
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = a2 * e[c] + T(2) * ae * a[c];
  } else if (PK == PK_6) {
    // |a|^4 e + 4 |a|^2 (a.e) a
    const T a4 = a2 * a2, w = T(4) * a2 * ae;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = a4 * e[c] + w * a[c];
  } else {
    const T f = pow(a2, beta);
    const T w = (a2 > T(0)) ? T(2) * beta * pow(a2, beta - T(1)) * ae : T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = f * e[c] + w * a[c];
  }
}

// Last-block bookkeeping of the residual kernel.
__device__ void residual_epilogue(Ctrl* ctrl, const KParams& kp, double sum2, double maxabs, int norm,
                                  int update_iter, bool hvp = false) {
  if (hvp) {
    const double pq = sum2 * kp.hd;  // (v, H v)_2
    ctrl->c1 = pq;
    ctrl->c2 = maxabs;
    if (ctrl->cg) {
      // CG step length alpha = (r, z) / (p, H p); H is positive definite
      // (the second variation, Sec. 5.3), so pq <= 0 means a breakdown
      if (pq > 0.0 && isfinite(pq)) {
        ctrl->alpha = ctrl->rz / pq;
      } else {
        ctrl->status = 7;
        ctrl->done = 1;
      }
    }
    ctrl->counter[CS_RES] = 0;
    return;
  }
  if (update_iter) {
    const int it = ctrl->iter;
    if (ctrl->hist_alpha != nullptr && it < ctrl->hist_cap) ctrl->hist_alpha[it] = ctrl->alpha;
    ctrl->iter = it + 1;
  }
  if (norm) {
    const double res = sqrt(sum2 * kp.hd);
    ctrl->res_l2 = res;
    ctrl->res_linf = maxabs;
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
  ctrl->counter[CS_RES] = 0;
}

// ------------------------------------------------------------- 3D residual
template <typename T, int PK, int MODE>
__global__ void __launch_bounds__(NT)
    k_res3d(ResArgs<T> a, KParams kp, Ctrl* ctrl, double* partials, int zc) {
  if (ctrl->done) return;
  constexpr int SXM = BX + 4, SYM = BY3 + 4;
  constexpr int NB = (MODE != RM_PLAIN) ? 2 : 1;
  __shared__ T su[5][SYM][SXM];
  __shared__ T sb[NB][SYM][SXM];
  __shared__ T sl[3][BY3 + 2][BX + 2];
  __shared__ T sf[2][3][BY3 + 1][BX + 1];
  __shared__ T sred[32 * 2];
  __shared__ int sflag;

  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const int TX = nx < BX ? nx : BX, TY = ny < BY3 ? ny : BY3;
  const int SX = TX + 4, SY = TY + 4;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
  const size_t plane = (size_t)nx * ny;
  const bool upd = a.d != nullptr;
  const T alpha = upd ? (T)ctrl->alpha : T(0);
  const KConst<T>& C = kconst<T>(kp);
  const T ih = C.inv_h, ih2 = ih * ih, q4 = T(0.25) * ih;
  const T s = C.s, se2 = C.se2, cu = C.cu;
  const T beta = C.beta;

  auto uslot = [&](int zz) { return (zz - z0 + 2) % 5; };
  auto lslot = [&](int zz) { return (zz - z0 + 1) % 3; };
  auto fslot = [&](int zz) { return (zz - z0 + 1) & 1; };  // vertex plane zz + 1/2
  auto bslot = [&](int zz) { return (zz - z0 + 2) & 1; };

  auto load_plane = [&](int zz) {
    const int sl_ = uslot(zz);
    const size_t gz = (size_t)wrapi(zz, nz) * plane;
    const bool own = (zz >= z0) && (zz < z0 + zc);
    for (int idx = tid; idx < SX * SY; idx += NT) {
      const int ly = idx / SX, lx = idx - ly * SX;
      const int gx = wrapi(x0 + lx - 2, nx), gy = wrapi(y0 + ly - 2, ny);
      const size_t g = gz + (size_t)gy * nx + gx;
      T v = a.u_in[g];
      if (upd) {
        v = v + alpha * a.d[g];
        if (own && lx >= 2 && lx < TX + 2 && ly >= 2 && ly < TY + 2) a.u_out[g] = v;
      }
      su[sl_][ly][lx] = v;
    }
  };
  auto load_base = [&](int zz) {
    if (MODE == RM_PLAIN) return;
    const int sl_ = bslot(zz);
    const size_t gz = (size_t)wrapi(zz, nz) * plane;
    for (int idx = tid; idx < SX * SY; idx += NT) {
      const int ly = idx / SX, lx = idx - ly * SX;
      const int gx = wrapi(x0 + lx - 2, nx), gy = wrapi(y0 + ly - 2, ny);
      sb[sl_ % NB][ly][lx] = a.ubase[gz + (size_t)gy * nx + gx];
    }
  };
  auto comp_lap = [&](int zz) {
    const int cm = uslot(zz - 1), c0 = uslot(zz), cp = uslot(zz + 1), ls = lslot(zz);
    const int LX = TX + 2, LY = TY + 2;
    for (int idx = tid; idx < LX * LY; idx += NT) {
      const int ly = idx / LX, lx = idx - ly * LX;
      const T c = su[c0][ly + 1][lx + 1];
      const T sum = (su[c0][ly + 1][lx] + su[c0][ly + 1][lx + 2]) + (su[c0][ly][lx + 1] + su[c0][ly + 2][lx + 1]) +
                    (su[cm][ly + 1][lx + 1] + su[cp][ly + 1][lx + 1]);
      sl[ls][ly][lx] = (sum - T(6) * c) * ih2;
    }
  };
  auto grad8 = [&](T (&fld)[SYM][SXM], T (&fld1)[SYM][SXM], int vy, int vx, T (&g)[3]) {
    const T u000 = fld[vy + 1][vx + 1], u001 = fld[vy + 1][vx + 2];
    const T u010 = fld[vy + 2][vx + 1], u011 = fld[vy + 2][vx + 2];
    const T u100 = fld1[vy + 1][vx + 1], u101 = fld1[vy + 1][vx + 2];
    const T u110 = fld1[vy + 2][vx + 1], u111 = fld1[vy + 2][vx + 2];
    g[0] = q4 * (((u001 - u000) + (u011 - u010)) + ((u101 - u100) + (u111 - u110)));
    g[1] = q4 * (((u010 - u000) + (u011 - u001)) + ((u110 - u100) + (u111 - u101)));
    g[2] = q4 * (((u100 - u000) + (u101 - u001)) + ((u110 - u010) + (u111 - u011)));
  };
  auto comp_flux = [&](int zz) {  // vertex plane zz + 1/2
    const int c0 = uslot(zz), c1 = uslot(zz + 1), fs = fslot(zz);
    const int VX = TX + 1, VY = TY + 1;
    for (int idx = tid; idx < VX * VY; idx += NT) {
      const int vy = idx / VX, vx = idx - vy * VX;
      T g[3], F[3];
      grad8(su[c0], su[c1], vy, vx, g);
      if (MODE != RM_PLAIN) {
        T ab[3];
        grad8(sb[bslot(zz) % NB], sb[bslot(zz + 1) % NB], vy, vx, ab);
        if (MODE == RM_INNER)
          flux_diff<PK>(ab, g, beta, F);
        else
          flux_lin<PK>(ab, g, beta, F);
      } else {
        flux<PK>(g, beta, F);
      }
      sf[fs][0][vy][vx] = F[0];
      sf[fs][1][vy][vx] = F[1];
      sf[fs][2][vy][vx] = F[2];
    }
  };

  T acc2 = T(0), accm = T(0);
  auto comp_out = [&](int zz) {
    const int lm = lslot(zz - 1), l0 = lslot(zz), lp = lslot(zz + 1);
    const int fm = fslot(zz - 1), fp = fslot(zz), c0 = uslot(zz);
    const size_t gz = (size_t)wrapi(zz, nz) * plane;
    for (int idx = tid; idx < TX * TY; idx += NT) {
      const int ty = idx / TX, tx = idx - ty * TX;
      const T bih = (((sl[l0][ty + 1][tx] + sl[l0][ty + 1][tx + 2]) + (sl[l0][ty][tx + 1] + sl[l0][ty + 2][tx + 1])) +
                     (sl[lm][ty + 1][tx + 1] + sl[lp][ty + 1][tx + 1]) - T(6) * sl[l0][ty + 1][tx + 1]) *
                    ih2;
      const T dx = q4 * (((sf[fm][0][ty][tx + 1] - sf[fm][0][ty][tx]) + (sf[fm][0][ty + 1][tx + 1] - sf[fm][0][ty + 1][tx])) +
                         ((sf[fp][0][ty][tx + 1] - sf[fp][0][ty][tx]) + (sf[fp][0][ty + 1][tx + 1] - sf[fp][0][ty + 1][tx])));
      const T dy = q4 * (((sf[fm][1][ty + 1][tx] - sf[fm][1][ty][tx]) + (sf[fm][1][ty + 1][tx + 1] - sf[fm][1][ty][tx + 1])) +
                         ((sf[fp][1][ty + 1][tx] - sf[fp][1][ty][tx]) + (sf[fp][1][ty + 1][tx + 1] - sf[fp][1][ty][tx + 1])));
      const T dz = q4 * (((sf[fp][2][ty][tx] - sf[fm][2][ty][tx]) + (sf[fp][2][ty][tx + 1] - sf[fm][2][ty][tx + 1])) +
                         ((sf[fp][2][ty + 1][tx] - sf[fm][2][ty + 1][tx]) + (sf[fp][2][ty + 1][tx + 1] - sf[fm][2][ty + 1][tx + 1])));
      const T div = dx + dy + dz;
      const T uc = su[c0][ty + 2][tx + 2];
      const size_t g = gz + (size_t)(y0 + ty) * nx + (x0 + tx);
      T r;
      if (MODE == RM_INNER)
        r = (a.f ? a.f[g] : T(0)) - ((cu * uc + se2 * bih) - s * div);
      else if (MODE == RM_HVP)
        r = (cu * uc + se2 * bih) - s * div;
      else
        r = (a.f ? a.f[g] : T(0)) - cu * uc + s * div - se2 * bih;
      a.r[g] = r;
      acc2 += (MODE == RM_HVP) ? uc * r : r * r;
      accm = fmax(accm, fabs(r));
    }
  };

  // prologue: planes z0-2 .. z0+1, Laplacians at z0-1, z0, fluxes at z0-1/2
  for (int zz = z0 - 2; zz <= z0 + 1; ++zz) load_plane(zz);
  load_base(z0 - 1);
  load_base(z0);
  __syncthreads();
  comp_lap(z0 - 1);
  comp_lap(z0);
  comp_flux(z0 - 1);
  // base slot of z0 - 1, read just above, is the one the first step refills
  if (MODE != RM_PLAIN) __syncthreads();
  for (int z = z0; z < z0 + zc; ++z) {
    load_plane(z + 2);
    load_base(z + 1);
    __syncthreads();
    comp_lap(z + 1);
    comp_flux(z);
    __syncthreads();
    comp_out(z);
  }

  T v[2] = {acc2, accm};
  block_reduce<T, 2, true>(v, sred);
  if (publish_and_check_last<T>(v, 2, reinterpret_cast<T*>(partials), &ctrl->counter[CS_RES], &sflag)) {
    T tt[2];
    gather_partials<T, 2, true>(tt, reinterpret_cast<const T*>(partials), sred);
    double tot[2];
    for (int m_ = 0; m_ < 2; ++m_) tot[m_] = (double)tt[m_];
    if (tid == 0) residual_epilogue(ctrl, kp, tot[0], tot[1], a.norm, a.update_iter, MODE == RM_HVP);
  }
}

// ------------------------------------------------------------- 2D residual
template <typename T, int PK, int MODE>
__global__ void __launch_bounds__(NT) k_res2d(ResArgs<T> a, KParams kp, Ctrl* ctrl, double* partials) {
  if (ctrl->done) return;
  constexpr int SXM = BX + 4, SYM = BY2 + 4;
  constexpr int NB = (MODE == RM_INNER) ? 1 : 1;
  __shared__ T su[SYM][SXM];
  __shared__ T sb[(MODE != RM_PLAIN) ? SYM : 1][SXM];
  __shared__ T sl[BY2 + 2][BX + 2];
  __shared__ T sf[2][BY2 + 1][BX + 1];
  __shared__ T sred[32 * 2];
  __shared__ int sflag;
  (void)NB;

  const int nx = kp.nx, ny = kp.ny;
  const int TX = nx < BX ? nx : BX, TY = ny < BY2 ? ny : BY2;
  const int SX = TX + 4, SY = TY + 4;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const bool upd = a.d != nullptr;
  const T alpha = upd ? (T)ctrl->alpha : T(0);
  const KConst<T>& C = kconst<T>(kp);
  const T ih = C.inv_h, ih2 = ih * ih, q2 = T(0.5) * ih;
  const T s = C.s, se2 = C.se2, cu = C.cu;
  const T beta = C.beta;

  for (int idx = tid; idx < SX * SY; idx += NT) {
    const int ly = idx / SX, lx = idx - ly * SX;
    const int gx = wrapi(x0 + lx - 2, nx), gy = wrapi(y0 + ly - 2, ny);
    const size_t g = (size_t)gy * nx + gx;
    T v = a.u_in[g];
    if (upd) {
      v = v + alpha * a.d[g];
      if (lx >= 2 && lx < TX + 2 && ly >= 2 && ly < TY + 2) a.u_out[g] = v;
    }
    su[ly][lx] = v;
    if (MODE != RM_PLAIN) sb[ly][lx] = a.ubase[g];
  }
  __syncthreads();
  {
    const int LX = TX + 2, LY = TY + 2;
    for (int idx = tid; idx < LX * LY; idx += NT) {
      const int ly = idx / LX, lx = idx - ly * LX;
      const T sum = (su[ly + 1][lx] + su[ly + 1][lx + 2]) + (su[ly][lx + 1] + su[ly + 2][lx + 1]);
      sl[ly][lx] = (sum - T(4) * su[ly + 1][lx + 1]) * ih2;
    }
    const int VX = TX + 1, VY = TY + 1;
    for (int idx = tid; idx < VX * VY; idx += NT) {
      const int vy = idx / VX, vx = idx - vy * VX;
      T g[3], F[3];
      {
        const T u00 = su[vy + 1][vx + 1], u01 = su[vy + 1][vx + 2], u10 = su[vy + 2][vx + 1], u11 = su[vy + 2][vx + 2];
        g[0] = q2 * ((u01 - u00) + (u11 - u10));
        g[1] = q2 * ((u10 - u00) + (u11 - u01));
        g[2] = T(0);
      }
      if (MODE != RM_PLAIN) {
        const T u00 = sb[vy + 1][vx + 1], u01 = sb[vy + 1][vx + 2], u10 = sb[vy + 2][vx + 1], u11 = sb[vy + 2][vx + 2];
        T ab[3] = {q2 * ((u01 - u00) + (u11 - u10)), q2 * ((u10 - u00) + (u11 - u01)), T(0)};
        if (MODE == RM_INNER)
          flux_diff<PK>(ab, g, beta, F);
        else
          flux_lin<PK>(ab, g, beta, F);
      } else {
        flux<PK>(g, beta, F);
      }
      sf[0][vy][vx] = F[0];
      sf[1][vy][vx] = F[1];
    }
  }
  __syncthreads();
  T acc2 = T(0), accm = T(0);
  for (int idx = tid; idx < TX * TY; idx += NT) {
    const int ty = idx / TX, tx = idx - ty * TX;
    const T bih = (((sl[ty + 1][tx] + sl[ty + 1][tx + 2]) + (sl[ty][tx + 1] + sl[ty + 2][tx + 1])) - T(4) * sl[ty + 1][tx + 1]) * ih2;
    const T dx = q2 * ((sf[0][ty][tx + 1] - sf[0][ty][tx]) + (sf[0][ty + 1][tx + 1] - sf[0][ty + 1][tx]));
    const T dy = q2 * ((sf[1][ty + 1][tx] - sf[1][ty][tx]) + (sf[1][ty + 1][tx + 1] - sf[1][ty][tx + 1]));
    const T div = dx + dy;
    const T uc = su[ty + 2][tx + 2];
    const size_t g = (size_t)(y0 + ty) * nx + (x0 + tx);
    T r;
    if (MODE == RM_INNER)
      r = (a.f ? a.f[g] : T(0)) - ((cu * uc + se2 * bih) - s * div);
    else if (MODE == RM_HVP)
      r = (cu * uc + se2 * bih) - s * div;
    else
      r = (a.f ? a.f[g] : T(0)) - cu * uc + s * div - se2 * bih;
    a.r[g] = r;
    acc2 += (MODE == RM_HVP) ? uc * r : r * r;
    accm = fmax(accm, fabs(r));
  }
  T v[2] = {acc2, accm};
  block_reduce<T, 2, true>(v, sred);
  if (publish_and_check_last<T>(v, 2, reinterpret_cast<T*>(partials), &ctrl->counter[CS_RES], &sflag)) {
    T tt[2];
    gather_partials<T, 2, true>(tt, reinterpret_cast<const T*>(partials), sred);
    double tot[2];
    for (int m_ = 0; m_ < 2; ++m_) tot[m_] = (double)tt[m_];
    if (tid == 0) residual_epilogue(ctrl, kp, tot[0], tot[1], a.norm, a.update_iter, MODE == RM_HVP);
  }
}

// ------------------------------------------------------------ line search
// alpha = root of q(alpha) = -rd + lin alpha + sum_{j=1..5} c_j alpha^j, the
// polynomial form of q(alpha) = (N_h[u + alpha d] - f, d)_2 for p = 4 (a
// cubic) and p = 6 (a quintic) of Sec. 6.1, with the s factor folded into
// c_j.  q(0) = -rd < 0 and q is strictly increasing (Sec. 2.3), so the root
// is unique; Newton's method with a bisection safeguard on a bracket.
__device__ double solve_poly_alpha(double rd, double lin, const double (&c)[5], int* status) {
  auto q = [&](double al) { return -rd + al * (lin + c[0] + al * (c[1] + al * (c[2] + al * (c[3] + al * c[4])))); };
  auto dq = [&](double al) {
    return lin + c[0] + al * (2.0 * c[1] + al * (3.0 * c[2] + al * (4.0 * c[3] + al * 5.0 * c[4])));
  };
  const double d0 = dq(0.0);
  if (!(rd > 0.0) || !(d0 > 0.0) || !isfinite(rd) || !isfinite(d0)) {
    *status = (isfinite(rd) && isfinite(d0)) ? 0 : 7;
    return 0.0;
  }
  double lo = 0.0, hi = -1.0;
  double alpha = rd / d0;
  double b = alpha;
  for (int i = 0; i < 200; ++i) {
    if (q(b) > 0.0) {
      hi = b;
      break;
    }
    lo = b;
    b *= 2.0;
  }
  if (hi < 0.0) {
    *status = 7;
    return alpha;
  }
  alpha = fmin(fmax(alpha, lo), hi);
  for (int it = 0; it < 200; ++it) {
    const double qa = q(alpha);
    if (qa == 0.0) return alpha;
    if (qa < 0.0)
      lo = alpha;
    else
      hi = alpha;
    const double step = qa / dq(alpha);
    if (fabs(step) <= 4e-16 * fabs(alpha)) return alpha - step;  // Newton step below rounding
    double nw = alpha - step;
    if (!(lo < nw && nw < hi)) nw = 0.5 * (lo + hi);
    if (hi - lo <= 4e-16 * hi) return nw;
    alpha = nw;
  }
  return alpha;
}

// Whether the line search of this vertex-factor kind is one pass (p = 4, 6:
// the coefficients of a polynomial q) or one pass per Newton step (general
// p: P(alpha) - P(0) and P'(alpha) at a trial alpha), and how many vertex
// sums a pass reduces.
template <int PK>
__host__ __device__ constexpr bool ls_closed_form() {
  return PK == PK_4 || PK == PK_6;
}
template <int PK>
__host__ __device__ constexpr int ls_nsums() {
  return PK == PK_6 ? 5 : 3;
}

// Vertex sums for one vertex with a = grad u (+ grad ubase), b = grad d.
// With A = |a|^2, B = a.b, C = |b|^2, the vertex term of P(alpha) =
// sum_v |a + alpha b|^{p-2} (a + alpha b).b is (A + 2 alpha B + alpha^2 C)^k
// (B + alpha C) for p = 2k + 2; its alpha^j coefficients (j >= 1) are summed:
//   p = 4: AC + 2B^2, 3BC, C^2;
//   p = 6: A^2 C + 4AB^2, 6ABC + 4B^3, 8B^2 C + 2AC^2, 5BC^2, C^3.
template <int PK, typename T>
__device__ __forceinline__ void ls_accumulate(const T (&av)[3], const T (&bv)[3], T trial, T beta, T pm2,
                                              T (&acc)[ls_nsums<PK>()]) {
  if (PK == PK_4 || PK == PK_6) {
    const T A = av[0] * av[0] + av[1] * av[1] + av[2] * av[2];
    const T B = av[0] * bv[0] + av[1] * bv[1] + av[2] * bv[2];
    const T C = bv[0] * bv[0] + bv[1] * bv[1] + bv[2] * bv[2];
    if (PK == PK_4) {
      acc[0] += A * C + T(2) * B * B;
      acc[1] += T(3) * B * C;
      acc[2] += C * C;
    } else {
      const T B2 = B * B, C2 = C * C;
      acc[0] += A * (A * C + T(4) * B2);
      acc[1] += B * (T(6) * A * C + T(4) * B2);
      acc[ls_nsums<PK>() - 3] += C * (T(8) * B2 + T(2) * A * C);
      acc[ls_nsums<PK>() - 2] += T(5) * B * C2;
      acc[ls_nsums<PK>() - 1] += C * C2;
    }
  } else {
    T e[3] = {trial * bv[0], trial * bv[1], trial * bv[2]};
    T df[3];
    flux_diff<PK>(av, e, beta, df);
    acc[0] += df[0] * bv[0] + df[1] * bv[1] + df[2] * bv[2];
    const T c[3] = {av[0] + e[0], av[1] + e[1], av[2] + e[2]};
    const T c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    const T cb = c[0] * bv[0] + c[1] * bv[1] + c[2] * bv[2];
    const T b2 = bv[0] * bv[0] + bv[1] * bv[1] + bv[2] * bv[2];
    T t = pow(c2, beta) * b2;
    if (c2 > T(0)) t += pm2 * pow(c2, beta - T(1)) * cb * cb;
    acc[1] += t;
  }
}

// Last-block logic of the line search.
template <int PK>
__device__ void linesearch_epilogue(Ctrl* ctrl, const KParams& kp, const double (&tot)[ls_nsums<PK>()]) {
  const double lin = kp.cu * ctrl->dd + ctrl->tdd + kp.s * kp.eps2 * ctrl->lapdd;
  if (ls_closed_form<PK>()) {
    int st = 0;
    // the kernels sum unscaled vertex gradients G = g / q: s g^p-terms = cdiv G^p-terms
    double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < ls_nsums<PK>(); ++j) c[j] = kp.cdiv * kp.hd * tot[j];
    const double al = solve_poly_alpha(ctrl->rd, lin, c, &st);
    ctrl->c1 = c[0];
    ctrl->c2 = c[1];
    ctrl->c3 = c[2];
    ctrl->alpha = al;
    if (st != 0) {
      ctrl->status = st;
      ctrl->done = 1;
    }
  } else {
    // one safeguarded Newton step per launch; state in c1 (lo), c2 (hi), c3 (done flag)
    const double trial = ctrl->alpha;
    const double qv = -ctrl->rd + trial * lin + kp.cdiv * kp.hd * tot[0];
    const double dqv = lin + kp.cdiv * kp.hd * tot[1];
    double lo = ctrl->c1, hi = ctrl->c2;
    if (qv < 0.0)
      lo = trial;
    else if (qv > 0.0)
      hi = trial;
    const double step = (dqv > 0.0) ? qv / dqv : 0.0;
    double nw = (dqv > 0.0) ? trial - step : 0.5 * (lo + hi);
    const bool tiny = (dqv > 0.0) && fabs(step) <= 4e-16 * fabs(trial);  // Newton step below rounding
    if (!tiny) {
      if (hi > 0.0) {
        if (!(lo < nw && nw < hi)) nw = 0.5 * (lo + hi);
      } else if (!(nw > lo)) {
        nw = 2.0 * (lo > 0.0 ? lo : 1.0);
      }
    }
    if (qv == 0.0 || tiny || (hi > 0.0 && hi - lo <= 4e-16 * hi)) {
      ctrl->c3 = 1.0;  // converged
      nw = (qv == 0.0) ? trial : nw;
    }
    ctrl->c1 = lo;
    ctrl->c2 = hi;
    ctrl->alpha = nw;
    if (!isfinite(nw) || !isfinite(qv)) {
      ctrl->status = 7;
      ctrl->done = 1;
    }
  }
  ctrl->counter[CS_LS] = 0;
}

// Block and grid reduction of a line-search pass (fixed order; the last
// block runs the epilogue).  sred: 32 * ls_nsums<PK>() shared elements.
template <typename T, int PK>
__device__ __forceinline__ void ls_finish(T (&acc)[ls_nsums<PK>()], T* sred, double* partials, Ctrl* ctrl,
                                          const KParams& kp, int* sflag) {
  constexpr int M = ls_nsums<PK>();
  block_reduce<T, M, false>(acc, sred);
  if (publish_and_check_last<T>(acc, M, reinterpret_cast<T*>(partials), &ctrl->counter[CS_LS], sflag)) {
    T tt[M];
    gather_partials<T, M, false>(tt, reinterpret_cast<const T*>(partials), sred);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (tid == 0) {
      double tot[M];
#pragma unroll
      for (int m = 0; m < M; ++m) tot[m] = (double)tt[m];
      linesearch_epilogue<PK>(ctrl, kp, tot);
    }
  }
}

}  // namespace
}  // namespace psd
#include "stencil3d_col.cuh"
#include "stencil3d_rb.cuh"
namespace psd {
namespace {

template <typename T, int PK, bool INNER>
__global__ void __launch_bounds__(NT)
    k_ls3d(const T* __restrict__ u, const T* __restrict__ ubase, const T* __restrict__ d, KParams kp, Ctrl* ctrl,
           double* partials, int zc) {
  if (ctrl->done) return;
  if (!ls_closed_form<PK>() && ctrl->c3 != 0.0) return;  // Newton already converged
  constexpr int SXM = BX + 1, SYM = BY3 + 1;
  __shared__ T su[2][SYM][SXM];
  __shared__ T sd[2][SYM][SXM];
  __shared__ T sred[32 * ls_nsums<PK>()];
  __shared__ int sflag;
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const int TX = nx < BX ? nx : BX, TY = ny < BY3 ? ny : BY3;
  const int SX = TX + 1, SY = TY + 1;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
  const size_t plane = (size_t)nx * ny;
  const T beta = kconst<T>(kp).beta, pm2 = kconst<T>(kp).pm2;
  const T trial = ls_closed_form<PK>() ? T(0) : (T)ctrl->alpha;
  auto load = [&](int zz) {
    const int sl_ = (zz - z0) & 1;
    const size_t gz = (size_t)wrapi(zz, nz) * plane;
    for (int idx = tid; idx < SX * SY; idx += NT) {
      const int ly = idx / SX, lx = idx - ly * SX;
      const size_t g = gz + (size_t)wrapi(y0 + ly, ny) * nx + wrapi(x0 + lx, nx);
      T v = u[g];
      if (INNER) v += ubase[g];
      su[sl_][ly][lx] = v;
      sd[sl_][ly][lx] = d[g];
    }
  };
  auto grad = [&](T (&f0)[SYM][SXM], T (&f1)[SYM][SXM], int vy, int vx, T (&g)[3]) {
    const T u000 = f0[vy][vx], u001 = f0[vy][vx + 1], u010 = f0[vy + 1][vx], u011 = f0[vy + 1][vx + 1];
    const T u100 = f1[vy][vx], u101 = f1[vy][vx + 1], u110 = f1[vy + 1][vx], u111 = f1[vy + 1][vx + 1];
    g[0] = ((u001 - u000) + (u011 - u010)) + ((u101 - u100) + (u111 - u110));
    g[1] = ((u010 - u000) + (u011 - u001)) + ((u110 - u100) + (u111 - u101));
    g[2] = ((u100 - u000) + (u101 - u001)) + ((u110 - u010) + (u111 - u011));
  };
  T acc[ls_nsums<PK>()] = {};
  load(z0);
  for (int z = z0; z < z0 + zc; ++z) {
    load(z + 1);
    __syncthreads();
    const int s0 = (z - z0) & 1, s1 = (z + 1 - z0) & 1;
    for (int idx = tid; idx < TX * TY; idx += NT) {
      const int vy = idx / TX, vx = idx - vy * TX;
      T av[3], bv[3];
      grad(su[s0], su[s1], vy, vx, av);
      grad(sd[s0], sd[s1], vy, vx, bv);
      ls_accumulate<PK>(av, bv, trial, beta, pm2, acc);
    }
    __syncthreads();
  }
  ls_finish<T, PK>(acc, sred, partials, ctrl, kp, &sflag);
}

template <typename T, int PK, bool INNER>
__global__ void __launch_bounds__(NT)
    k_ls2d(const T* __restrict__ u, const T* __restrict__ ubase, const T* __restrict__ d, KParams kp, Ctrl* ctrl,
           double* partials) {
  if (ctrl->done) return;
  if (!ls_closed_form<PK>() && ctrl->c3 != 0.0) return;
  constexpr int SXM = BX + 1, SYM = BY2 + 1;
  __shared__ T su[SYM][SXM];
  __shared__ T sd[SYM][SXM];
  __shared__ T sred[32 * ls_nsums<PK>()];
  __shared__ int sflag;
  const int nx = kp.nx, ny = kp.ny;
  const int TX = nx < BX ? nx : BX, TY = ny < BY2 ? ny : BY2;
  const int SX = TX + 1, SY = TY + 1;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const T beta = kconst<T>(kp).beta, pm2 = kconst<T>(kp).pm2;
  const T trial = ls_closed_form<PK>() ? T(0) : (T)ctrl->alpha;
  for (int idx = tid; idx < SX * SY; idx += NT) {
    const int ly = idx / SX, lx = idx - ly * SX;
    const size_t g = (size_t)wrapi(y0 + ly, ny) * nx + wrapi(x0 + lx, nx);
    T v = u[g];
    if (INNER) v += ubase[g];
    su[ly][lx] = v;
    sd[ly][lx] = d[g];
  }
  __syncthreads();
  T acc[ls_nsums<PK>()] = {};
  for (int idx = tid; idx < TX * TY; idx += NT) {
    const int vy = idx / TX, vx = idx - vy * TX;
    T av[3] = {(su[vy][vx + 1] - su[vy][vx]) + (su[vy + 1][vx + 1] - su[vy + 1][vx]),
               (su[vy + 1][vx] - su[vy][vx]) + (su[vy + 1][vx + 1] - su[vy][vx + 1]), T(0)};
    T bv[3] = {(sd[vy][vx + 1] - sd[vy][vx]) + (sd[vy + 1][vx + 1] - sd[vy + 1][vx]),
               (sd[vy + 1][vx] - sd[vy][vx]) + (sd[vy + 1][vx + 1] - sd[vy][vx + 1]), T(0)};
    ls_accumulate<PK>(av, bv, trial, beta, pm2, acc);
  }
  ls_finish<T, PK>(acc, sred, partials, ctrl, kp, &sflag);
}

}  // namespace

namespace detail {

template <typename T, int PK, int MODE>
cudaError_t res_impl(const ResArgs<T>& a, const KParams& kp, Ctrl* ctrl, double* partials, cudaStream_t st) {
  const ResGeom g = residual_geometry(kp, sizeof(T) == 4);
  switch (g.kind) {
    case RK_RB4:
      if constexpr (sizeof(T) == 4) k_res3d_rb<T, PK, MODE, 4><<<g.grid, NT, 0, st>>>(a, kp, ctrl, partials);
      break;
    case RK_COL:
      if constexpr (sizeof(T) == 8 && MODE == RM_PLAIN && PK == PK_4) {
        if (a.fxs_dev != nullptr && a.d == nullptr) {
          // both variants; the one that does not apply returns at once
          k_res3d_col<T, PK, MODE, true><<<g.grid, NT, 0, st>>>(a, kp, ctrl, partials);
          k_res3d_col<T, PK, MODE><<<g.grid, NT, 0, st>>>(a, kp, ctrl, partials);
          break;
        }
        if (a.fluxff && a.d == nullptr && a.fxs >= 15 && a.fxs <= 120) {
          k_res3d_col<T, PK, MODE, true><<<g.grid, NT, 0, st>>>(a, kp, ctrl, partials);
          break;
        }
      }
      k_res3d_col<T, PK, MODE><<<g.grid, NT, 0, st>>>(a, kp, ctrl, partials);
      break;
    case RK_SMALL3D:
      k_res3d<T, PK, MODE><<<g.grid, NT, 0, st>>>(a, kp, ctrl, partials, g.zc);
      break;
    default:
      k_res2d<T, PK, MODE><<<g.grid, NT, 0, st>>>(a, kp, ctrl, partials);
  }
  return cudaGetLastError();
}

template <typename T, int PK, bool INNER>
cudaError_t ls_impl(const T* u, const T* ubase, const T* d, const KParams& kp, Ctrl* ctrl, double* partials,
                    cudaStream_t st) {
  // the same tiles as the residual; __launch_bounds__(256, 3)
  const ResGeom g = res_geometry(kp, sizeof(T) == 4, 3);
  switch (g.kind) {
    case RK_RB4:
      if constexpr (sizeof(T) == 4) k_ls3d_rb<T, PK, INNER, 4><<<g.grid, NT, 0, st>>>(u, ubase, d, kp, ctrl, partials);
      break;
    case RK_COL:
      k_ls3d_col<T, PK, INNER><<<g.grid, NT, 0, st>>>(u, ubase, d, kp, ctrl, partials);
      break;
    case RK_SMALL3D:
      k_ls3d<T, PK, INNER><<<g.grid, NT, 0, st>>>(u, ubase, d, kp, ctrl, partials, g.zc);
      break;
    default:
      k_ls2d<T, PK, INNER><<<g.grid, NT, 0, st>>>(u, ubase, d, kp, ctrl, partials);
  }
  return cudaGetLastError();
}


}  // namespace detail
}  // namespace psd
