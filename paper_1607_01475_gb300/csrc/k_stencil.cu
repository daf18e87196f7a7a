// Stencil kernels off the inner PSD loop (vertex-gradient maxima, energy
// sums, time-loop right-hand sides, vector helpers), the launch geometry of
// the residual and line-search kernels, and the launchers that dispatch them
// by vertex-factor kind to the translation units that instantiate them.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "stencil_geom.h"

namespace psd {
namespace {

// max |G|^2 over the vertices of an FP32 field (G from the 8 surrounding
// cells) into ctrl->res_linf, and max |u| into ctrl->res_l2 (+inf if a
// value is not finite).  Each thread takes four consecutive vertices of a
// row (x fastest, nx a multiple of 4, the field 16-byte aligned): the four
// cell rows around them are read as float4 plus one scalar each.
__global__ void __launch_bounds__(NT) k_gradmax(const float* __restrict__ u, KParams kp, Ctrl* ctrl,
                                                double* partials) {
  __shared__ float sred[32 * 2];
  __shared__ int sflag;
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const int lq = __ffs(nx / 4) - 1, lqy = lq + __ffs(ny) - 1;  // sizes are powers of two
  const size_t plane = (size_t)nx * ny, nq = plane * nz / 4;
  float m = 0.0f, um = 0.0f;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < nq; i += (size_t)gridDim.x * NT) {
    const int x = 4 * (int)(i & (nx / 4 - 1)), y = (int)((i >> lq) & (ny - 1)), z = (int)(i >> lqy);
    const int x4 = (x + 4) & (nx - 1), y1 = (y + 1) & (ny - 1), z1 = (z + 1) & (nz - 1);
    const float* r00 = u + (size_t)z * plane + (size_t)y * nx;  // rows (z, y), (z, y1), (z1, y), (z1, y1)
    const float* r01 = u + (size_t)z * plane + (size_t)y1 * nx;
    const float* r10 = u + (size_t)z1 * plane + (size_t)y * nx;
    const float* r11 = u + (size_t)z1 * plane + (size_t)y1 * nx;
    const float4 a = *reinterpret_cast<const float4*>(r00 + x), b = *reinterpret_cast<const float4*>(r01 + x);
    const float4 c = *reinterpret_cast<const float4*>(r10 + x), d = *reinterpret_cast<const float4*>(r11 + x);
    const float av[5] = {a.x, a.y, a.z, a.w, r00[x4]}, bv[5] = {b.x, b.y, b.z, b.w, r01[x4]};
    const float cv[5] = {c.x, c.y, c.z, c.w, r10[x4]}, dv[5] = {d.x, d.y, d.z, d.w, r11[x4]};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // u000 = av[k], u001 = av[k+1] (x), u010 = bv[k] (y), u100 = cv[k] (z)
      const float g0 = ((av[k + 1] - av[k]) + (bv[k + 1] - bv[k])) + ((cv[k + 1] - cv[k]) + (dv[k + 1] - dv[k]));
      const float g1 = ((bv[k] - av[k]) + (bv[k + 1] - av[k + 1])) + ((dv[k] - cv[k]) + (dv[k + 1] - cv[k + 1]));
      const float g2 = ((cv[k] - av[k]) + (cv[k + 1] - av[k + 1])) + ((dv[k] - bv[k]) + (dv[k + 1] - bv[k + 1]));
      m = fmaxf(m, g0 * g0 + g1 * g1 + g2 * g2);
      const float au = fabsf(av[k]);
      um = (au <= FLT_MAX) ? fmaxf(um, au) : INFINITY;  // NaN or infinity: +inf
    }
  }
  float v[2] = {m, um};
  block_reduce<float, 2, true, true>(v, sred);
  if (publish_and_check_last<float>(v, 2, reinterpret_cast<float*>(partials), &ctrl->counter[CS_MID], &sflag)) {
    float tt[2];
    gather_partials<float, 2, true, true>(tt, reinterpret_cast<const float*>(partials), sred);
    if (threadIdx.x == 0) {
      ctrl->res_linf = (double)tt[0];
      ctrl->res_l2 = (double)tt[1];
      ctrl->counter[CS_MID] = 0;
    }
  }
}

// Local sums of the discrete energies (Sec. 5.3 / 5.4), FP64, one cell (and
// its vertex at +1/2 in every axis) per thread, grid-stride:
//   t0 = sum (u - f)^2 (order 4) or sum u^2 (order 6),
//   t1 = sum (u - gbar) f (order 6),  t2 = sum (h^2 Delta_h u)^2,
//   t3 = sum over vertices |G|^p (G = g / q, unscaled vertex gradient),
// into ctrl->rd, dd, lapdd, tdd.
__global__ void __launch_bounds__(NT) k_energy_terms(const double* __restrict__ u, const double* __restrict__ f,
                                                     double gbar, KParams kp, Ctrl* ctrl, double* partials) {
  __shared__ double sred[32 * 4];
  __shared__ int sflag;
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const int lx = __ffs(nx) - 1, lxy = lx + __ffs(ny) - 1;  // sizes are powers of two
  const size_t plane = (size_t)nx * ny, n = plane * nz;
  const bool d3 = kp.dim == 3;
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    const int x = (int)(i & (nx - 1)), y = (int)((i >> lx) & (ny - 1)), z = (int)(i >> lxy);
    const int xp = (x + 1) & (nx - 1), xm = (x - 1) & (nx - 1), yp = (y + 1) & (ny - 1), ym = (y - 1) & (ny - 1);
    auto at = [&](int zz, int yy, int xx) { return u[(size_t)zz * plane + (size_t)yy * nx + xx]; };
    const double c = u[i];
    const double sum = (at(z, y, xm) + at(z, y, xp)) + (at(z, ym, x) + at(z, yp, x));
    double lapc = sum - 4.0 * c;
    if (d3) {
      const int zp = (z + 1) & (nz - 1), zm = (z - 1) & (nz - 1);
      lapc = (sum + (at(zm, y, x) + at(zp, y, x))) - 6.0 * c;
    }
    t[2] += lapc * lapc;
    double G2;
    if (d3) {
      const int z1 = (z + 1) & (nz - 1);
      const double u000 = c, u001 = at(z, y, xp), u010 = at(z, yp, x), u011 = at(z, yp, xp);
      const double u100 = at(z1, y, x), u101 = at(z1, y, xp), u110 = at(z1, yp, x), u111 = at(z1, yp, xp);
      const double g0 = ((u001 - u000) + (u011 - u010)) + ((u101 - u100) + (u111 - u110));
      const double g1 = ((u010 - u000) + (u011 - u001)) + ((u110 - u100) + (u111 - u101));
      const double g2 = ((u100 - u000) + (u101 - u001)) + ((u110 - u010) + (u111 - u011));
      G2 = g0 * g0 + g1 * g1 + g2 * g2;
    } else {
      const double u00 = c, u01 = at(0, y, xp), u10 = at(0, yp, x), u11 = at(0, yp, xp);
      const double g0 = (u01 - u00) + (u11 - u10), g1 = (u10 - u00) + (u11 - u01);
      G2 = g0 * g0 + g1 * g1;
    }
    t[3] += (kp.p == 4.0) ? G2 * G2 : pow(G2, 0.5 * kp.p);
    if (kp.order == 4) {
      const double e = c - f[i];
      t[0] += e * e;
    } else {
      t[0] += c * c;
      t[1] += (c - gbar) * f[i];
    }
  }
  block_reduce<double, 4, false>(t, sred);
  if (publish_and_check_last<double>(t, 4, partials, &ctrl->counter[CS_RES], &sflag)) {
    double tt[4];
    gather_partials<double, 4, false>(tt, partials, sred);
    if (threadIdx.x == 0) {
      ctrl->rd = tt[0];
      ctrl->dd = tt[1];
      ctrl->lapdd = tt[2];
      ctrl->tdd = tt[3];
      ctrl->counter[CS_RES] = 0;
    }
  }
}

// ------------------------------------------------------------------ misc
template <typename T>
__global__ void k_axpby(T* y, const T* x, const T* z, double a, double b, double c, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T xv = x ? x[i] : T(0);
    const T zv = z ? z[i] : T(0);
    y[i] = (T)a * xv + (T)b * zv + (T)c;
  }
}

// Element-wise helpers over whole fields.  Grids have an even number of
// cells, so when the pointers are 16-byte aligned (always for the
// handle's own buffers, not necessarily for a caller's) two elements move
// per access; each thread keeps two such accesses in flight.
__device__ __forceinline__ bool aligned16(const void* p) { return ((unsigned long long)p & 15ull) == 0; }

// sum x, sum x^2, max |x| over n values -> ctrl (rd, res_l2 = sqrt(hd sum x^2), res_linf)
__global__ void __launch_bounds__(NT) k_norms(const double* x, size_t n, double hd, Ctrl* c, double* partials) {
  __shared__ double sred[32 * 3];
  __shared__ int sflag;
  double v[3] = {0.0, 0.0, -1.0}, w[3] = {0.0, 0.0, -1.0};
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  auto add = [](double (&a)[3], double t) {
    a[0] += t;
    a[1] += t * t;
    a[2] = fmax(a[2], fabs(t));
  };
  if (aligned16(x) && (n & 1) == 0) {
    const double2* x2 = reinterpret_cast<const double2*>(x);
    const size_t n2 = n / 2;
    size_t i = t0;
    for (; i + stride < n2; i += 2 * stride) {
      const double2 a = x2[i], b = x2[i + stride];
      add(v, a.x);
      add(w, a.y);
      add(v, b.x);
      add(w, b.y);
    }
    if (i < n2) {
      const double2 a = x2[i];
      add(v, a.x);
      add(w, a.y);
    }
  } else {
    for (size_t i = t0; i < n; i += stride) add(v, x[i]);
  }
  v[0] += w[0];
  v[1] += w[1];
  v[2] = fmax(v[2], w[2]);
  block_reduce<double, 3, true>(v, sred);
  if (publish_and_check_last<double>(v, 3, partials, &c->counter[CS_MISC], &sflag)) {
    double tt[3];
    gather_partials<double, 3, true>(tt, partials, sred);
    if (threadIdx.x == 0) {
      c->rd = tt[0];
      c->res_l2 = sqrt(hd * tt[1]);
      c->res_linf = tt[2];
      c->counter[CS_MISC] = 0;
    }
  }
}
// The mean projection of order 6 on the device: c->c2 = mean(g - u), then
// u += c->c2 (k_add_mean), with no host round trip.
__global__ void __launch_bounds__(NT) k_mean_diff(const double* g, const double* u, size_t n, Ctrl* c,
                                                  double* partials) {
  __shared__ double sred[32];
  __shared__ int sflag;
  double v[1] = {0.0}, w = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    v[0] += g[i];
    w += u[i];
  }
  v[0] -= w;
  block_reduce<double, 1, false>(v, sred);
  if (publish_and_check_last<double>(v, 1, partials, &c->counter[CS_MISC], &sflag)) {
    double tt[1];
    gather_partials<double, 1, false>(tt, partials, sred);
    if (threadIdx.x == 0) {
      c->c2 = tt[0] / (double)n;
      c->counter[CS_MISC] = 0;
    }
  }
}
__global__ void k_add_mean(double* u, const Ctrl* c, size_t n) {
  const double m = c->c2;
  if (m == 0.0) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    u[i] += m;
}
__global__ void k_round_f32(float* out, const double* in, size_t n) {
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  if (aligned16(in) && aligned16(out) && (n & 1) == 0) {
    const double2* in2 = reinterpret_cast<const double2*>(in);
    float2* out2 = reinterpret_cast<float2*>(out);
    for (size_t i = t0; i < n / 2; i += stride) {
      const double2 a = in2[i];
      out2[i] = make_float2((float)a.x, (float)a.y);
    }
  } else {
    for (size_t i = t0; i < n; i += stride) out[i] = (float)in[i];
  }
}
__global__ void k_accumulate_f64(double* u, const float* delta, float* u32, size_t n, const double* dsum,
                                 const int* skip) {
  if (skip != nullptr && *skip) return;
  const double m = dsum ? *dsum / (double)n : 0.0;  // mean of delta, removed
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  if (aligned16(u) && aligned16(delta) && aligned16(u32) && (n & 1) == 0) {
    double2* u2 = reinterpret_cast<double2*>(u);
    const float2* d2 = reinterpret_cast<const float2*>(delta);
    float2* o2 = reinterpret_cast<float2*>(u32);
    for (size_t i = t0; i < n / 2; i += stride) {
      const double2 a = u2[i];
      const float2 d = d2[i];
      const double2 v = make_double2(a.x + ((double)d.x - m), a.y + ((double)d.y - m));
      u2[i] = v;
      o2[i] = make_float2((float)v.x, (float)v.y);
    }
  } else {
    for (size_t i = t0; i < n; i += stride) {
      const double v = u[i] + ((double)delta[i] - m);
      u[i] = v;
      u32[i] = (float)v;
    }
  }
}

// One conjugate-gradient update of the adjoint solve H lambda = b:
// lam += alpha p, r -= alpha q (q = H p), w = r (the preconditioner's input,
// transformed in place), with ||r||_2 = (h^d sum r^2)^{1/2}, the iteration
// count and the stopping test (ctrl->tol absolute, ctrl->max_iter) in the
// last block.  Returns at once when ctrl->done is set.
template <typename T>
__global__ void __launch_bounds__(NT) k_cg_update(T* lam, const T* p, T* r, const T* q, T* w, size_t n, double hd,
                                                  Ctrl* ctrl, double* partials) {
  __shared__ T sred[32];
  __shared__ int sflag;
  if (ctrl->done) return;
  const T al = (T)ctrl->alpha;
  T acc = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T ri = r[i] - al * q[i];
    lam[i] += al * p[i];
    r[i] = ri;
    w[i] = ri;
    acc += ri * ri;
  }
  T v[1] = {acc};
  block_reduce<T, 1, false>(v, sred);
  if (publish_and_check_last<T>(v, 1, reinterpret_cast<T*>(partials), &ctrl->counter[CS_MISC], &sflag)) {
    T tt[1];
    gather_partials<T, 1, false>(tt, reinterpret_cast<const T*>(partials), sred);
    if (threadIdx.x == 0) {
      const double res = sqrt((double)tt[0] * hd);
      const int it = ctrl->iter + 1;
      ctrl->iter = it;
      ctrl->res_l2 = res;
      if (!isfinite(res)) {
        ctrl->status = 7;
        ctrl->done = 1;
      } else if (res <= ctrl->tol) {
        ctrl->status = 0;
        ctrl->done = 1;
      } else if (it >= ctrl->max_iter) {
        ctrl->status = 4;
        ctrl->done = 1;
      }
      ctrl->counter[CS_MISC] = 0;
    }
  }
}

// Outer residual of the mixed adjoint solve: out32 = (float)(b - q) with
// (h^d sum (b - q)^2)^{1/2} into ctrl->res_l2 (FP64).
__global__ void __launch_bounds__(NT) k_sub_round(const double* b, const double* q, float* out32, size_t n, double hd,
                                                  Ctrl* ctrl, double* partials) {
  __shared__ double sred[32];
  __shared__ int sflag;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double e = b[i] - q[i];
    out32[i] = (float)e;
    acc += e * e;
  }
  double v[1] = {acc};
  block_reduce<double, 1, false>(v, sred);
  if (publish_and_check_last<double>(v, 1, partials, &ctrl->counter[CS_MISC], &sflag)) {
    double tt[1];
    gather_partials<double, 1, false>(tt, partials, sred);
    if (threadIdx.x == 0) {
      ctrl->res_l2 = sqrt(tt[0] * hd);
      ctrl->counter[CS_MISC] = 0;
    }
  }
}

// y += (double) x (FP64 accumulation of an FP32 correction).
__global__ void k_add_f32(double* y, const float* x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] += (double)x[i];
}

// Thin-film right-hand side f = u - s Delta_h^v u (Sec. 6.1, Eq.
// "thin-film-fully-discrete"), one cell per thread, FP64.  The skew
// Laplacian is sum_a d_a D_a with D_a and d_a the vertex difference
// operators of Sec. 5.1 (3D: the tensor extension), i.e. along each axis
// the second difference (1, -2, 1) times the average (1, 2, 1)/4 along the
// other axes: integer weights 2 (corners) and -8 (centre) over 4 h^2 in 2D;
// 3 (corners), 2 (edges), -4 (faces), -24 (centre) over 16 h^2 in 3D.
__global__ void __launch_bounds__(NT) k_thinfilm_rhs(const double* __restrict__ u, double* __restrict__ f,
                                                     KParams kp) {
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const size_t plane = (size_t)nx * ny, n = plane * nz;
  const double sc = kp.s * kp.inv_h * kp.inv_h * (kp.dim == 3 ? 1.0 / 16.0 : 0.25);
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / plane);
    double acc = 0.0;
    if (kp.dim == 2) {
      const int xm = (x - 1) & (nx - 1), xp = (x + 1) & (nx - 1);
      const int ym = (y - 1) & (ny - 1), yp = (y + 1) & (ny - 1);
      acc = 2.0 * ((u[(size_t)ym * nx + xm] + u[(size_t)ym * nx + xp]) + (u[(size_t)yp * nx + xm] + u[(size_t)yp * nx + xp])) -
            8.0 * u[i];
    } else {
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int k = (dx != 0) + (dy != 0) + (dz != 0);  // 0 centre, 1 face, 2 edge, 3 corner
            const double w = k == 0 ? -24.0 : (k == 1 ? -4.0 : (k == 2 ? 2.0 : 3.0));
            const size_t j = (size_t)((z + dz) & (nz - 1)) * plane + (size_t)((y + dy) & (ny - 1)) * nx +
                             (size_t)((x + dx) & (nx - 1));
            acc += w * u[j];
          }
    }
    f[i] = u[i] - sc * acc;
  }
}

// SPFC right-hand side (Sec. 6.2, Eq. "scheme-spfc", with the s-scaled
// explicit term of the scheme in Sec. 1): f = -c Delta_h u, c = s gamma_1,
// Delta_h the 5- or 7-point Laplacian; g = u.  One cell per thread, FP64.
__global__ void __launch_bounds__(NT) k_spfc_rhs(const double* __restrict__ u, double* __restrict__ f,
                                                 double* __restrict__ g, double c, KParams kp) {
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const size_t plane = (size_t)nx * ny, n = plane * nz;
  const double sc = c * kp.inv_h * kp.inv_h;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / plane);
    const size_t row = i - x, pl = (size_t)z * plane;
    const double uc = u[i];
    double sum = (u[row + ((x + 1) & (nx - 1))] + u[row + ((x - 1) & (nx - 1))]) +
                 (u[pl + (size_t)((y + 1) & (ny - 1)) * nx + x] + u[pl + (size_t)((y - 1) & (ny - 1)) * nx + x]);
    double cw = 4.0;
    if (kp.dim == 3) {
      const size_t xy = i - pl;
      sum += u[(size_t)((z + 1) & (nz - 1)) * plane + xy] + u[(size_t)((z - 1) & (nz - 1)) * plane + xy];
      cw = 6.0;
    }
    f[i] = -sc * (sum - cw * uc);
    g[i] = uc;
  }
}

// sum x (y + z) (z may be null) -> c->rd
__global__ void __launch_bounds__(NT) k_dot(const double* x, const double* y, const double* z, size_t n, Ctrl* c,
                                            double* partials) {
  __shared__ double sred[32];
  __shared__ int sflag;
  double v[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[0] += x[i] * (z ? y[i] + z[i] : y[i]);
  block_reduce<double, 1, false>(v, sred);
  if (publish_and_check_last<double>(v, 1, partials, &c->counter[CS_MISC], &sflag)) {
    double tt[1];
    gather_partials<double, 1, false>(tt, partials, sred);
    if (threadIdx.x == 0) {
      c->rd = tt[0];
      c->counter[CS_MISC] = 0;
    }
  }
}

inline int grid1d(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

int pick_zc(int nz, int nblk_xy) {
  // z planes per CTA: enough CTAs to fill the GPU, long enough marches
  int zc = nz;
  while (zc > 8 && (size_t)nblk_xy * (nz / zc) < 152 * 8) zc >>= 1;
  return zc;
}

}  // namespace

// Launch geometry of the residual and line-search kernels (ctas_per_sm =
// the residency their __launch_bounds__ guarantee).  3D FP32 grids large
// enough to fill the GPU with 32 x 32 tiles take the register-blocked
// kernels (the FP32 residual is bound by instruction issue and shared-memory
// traffic); FP64 and smaller grids the column kernels; tiles below 32 x 8
// the general kernel.  The register-blocked and column kernels run one wave
// of CTAs: the CTAs per SM times the SMs (cached in KParams at setup, so
// captured and direct launches agree and the partial sums come in the same
// order), at most one CTA per 16 (8) column-planes.
ResGeom res_geometry(const KParams& kp, bool fp32, int ctas_per_sm) {
  ResGeom g{RK_2D, dim3(1, 1, 1), 1};
  if (kp.dim != 3) {
    const int TX = kp.nx < BX ? kp.nx : BX, TY = kp.ny < BY2 ? kp.ny : BY2;
    g.grid = dim3(kp.nx / TX, kp.ny / TY);
    return g;
  }
  const long long wave = (long long)ctas_per_sm * kp.nsm;
  if (fp32 && kp.nx % 32 == 0 && kp.ny % 32 == 0 && kp.nz >= 16 &&
      (long long)(kp.nx / 32) * (kp.ny / 32) * (kp.nz / 16) >= 2 * 152 &&
      (long long)(kp.nx / 32) * (kp.ny / 32) * kp.nz < (1LL << 31)) {
    const long long w = (long long)(kp.nx / 32) * (kp.ny / 32) * kp.nz;
    g.kind = RK_RB4;
    g.grid = dim3((unsigned)std::min(wave, w / 16));
    g.zc = 0;
    return g;
  }
  const int TX = kp.nx < BX ? kp.nx : BX, TY = kp.ny < BY3 ? kp.ny : BY3;
  const int gx = kp.nx / TX, gy = kp.ny / TY;
  const long long w = (long long)gx * gy * kp.nz;
  if (kp.nx >= 32 && kp.ny >= 8 && w < (1LL << 31)) {
    g.kind = RK_COL;
    g.grid = dim3((unsigned)std::max(1LL, std::min(wave, w / 8)));
    g.zc = 0;
    return g;
  }
  g.zc = pick_zc(kp.nz, gx * gy);
  g.grid = dim3(gx, gy, kp.nz / g.zc);
  g.kind = RK_SMALL3D;
  return g;
}


template <typename T>
cudaError_t launch_residual(const ResArgs<T>& a, int mode, int pk, const KParams& kp, Ctrl* ctrl,
                            double* partials, cudaStream_t st) {
  using detail::res_impl;
#define PSD_RES_BY_PK(MODE_)                                                              \
  switch (pk) {                                                                           \
    case PK_4: return res_impl<T, PK_4, MODE_>(a, kp, ctrl, partials, st);                \
    case PK_6: return res_impl<T, PK_6, MODE_>(a, kp, ctrl, partials, st);                \
    default: return res_impl<T, PK_GEN, MODE_>(a, kp, ctrl, partials, st);               \
  }
  if (mode == RM_INNER) PSD_RES_BY_PK(RM_INNER)
  if (mode == RM_HVP) PSD_RES_BY_PK(RM_HVP)
  PSD_RES_BY_PK(RM_PLAIN)
#undef PSD_RES_BY_PK
}

ResGeom residual_geometry(const KParams& kp, bool fp32) {
  const ResGeom g = res_geometry(kp, fp32, 2);
  return g.kind == RK_COL ? res_geometry(kp, fp32, 3) : g;
}

long long residual_grid_blocks(const KParams& kp, bool fp32) {
  const ResGeom g = residual_geometry(kp, fp32);
  return (long long)g.grid.x * g.grid.y * g.grid.z;
}

template <typename T>
cudaError_t launch_linesearch(const T* u, const T* ubase, const T* d, int pk, const KParams& kp, Ctrl* ctrl,
                              double* partials, cudaStream_t st) {
  using detail::ls_impl;
#define PSD_LS_BY_PK(INNER_)                                                              \
  switch (pk) {                                                                           \
    case PK_4: return ls_impl<T, PK_4, INNER_>(u, ubase, d, kp, ctrl, partials, st);      \
    case PK_6: return ls_impl<T, PK_6, INNER_>(u, ubase, d, kp, ctrl, partials, st);      \
    default: return ls_impl<T, PK_GEN, INNER_>(u, ubase, d, kp, ctrl, partials, st);     \
  }
  if (ubase != nullptr) PSD_LS_BY_PK(true)
  PSD_LS_BY_PK(false)
#undef PSD_LS_BY_PK
}

template <typename T>
cudaError_t launch_cg_update(T* lam, const T* p, T* r, const T* q, T* w, size_t n, double hd, Ctrl* ctrl,
                             double* partials, cudaStream_t st) {
  k_cg_update<T><<<std::min(grid1d(n), 1024), NT, 0, st>>>(lam, p, r, q, w, n, hd, ctrl, partials);
  return cudaGetLastError();
}
template cudaError_t launch_cg_update<float>(float*, const float*, float*, const float*, float*, size_t, double,
                                             Ctrl*, double*, cudaStream_t);
template cudaError_t launch_cg_update<double>(double*, const double*, double*, const double*, double*, size_t,
                                              double, Ctrl*, double*, cudaStream_t);
cudaError_t launch_sub_round(const double* b, const double* q, float* out32, size_t n, double hd, Ctrl* ctrl,
                             double* partials, cudaStream_t st) {
  k_sub_round<<<std::min(grid1d(n), 1024), NT, 0, st>>>(b, q, out32, n, hd, ctrl, partials);
  return cudaGetLastError();
}
cudaError_t launch_add_f32(double* y, const float* x, size_t n, cudaStream_t st) {
  k_add_f32<<<grid1d(n), 256, 0, st>>>(y, x, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpby(T* y, const T* x, const T* z, double a, double b, double c, size_t n, cudaStream_t st) {
  k_axpby<T><<<grid1d(n), 256, 0, st>>>(y, x, z, a, b, c, n);
  return cudaGetLastError();
}
cudaError_t launch_dot(const double* x, const double* y, const double* z, size_t n, Ctrl* c, double* partials,
                       cudaStream_t st) {
  k_dot<<<std::min(grid1d(n), 1024), NT, 0, st>>>(x, y, z, n, c, partials);
  return cudaGetLastError();
}
cudaError_t launch_gradmax(const float* u, const KParams& kp, Ctrl* ctrl, double* partials, cudaStream_t st) {
  const size_t n = (size_t)kp.nx * kp.ny * kp.nz;
  k_gradmax<<<std::min(grid1d(n / 4), 1024), NT, 0, st>>>(u, kp, ctrl, partials);  // 3D, nx % 4 == 0
  return cudaGetLastError();
}
cudaError_t launch_thinfilm_rhs(const double* u, double* f, const KParams& kp, cudaStream_t st) {
  const size_t n = (size_t)kp.nx * kp.ny * kp.nz;
  k_thinfilm_rhs<<<grid1d(n), NT, 0, st>>>(u, f, kp);
  return cudaGetLastError();
}
cudaError_t launch_spfc_rhs(const double* u, double* f, double* g, double c, const KParams& kp, cudaStream_t st) {
  const size_t n = (size_t)kp.nx * kp.ny * kp.nz;
  k_spfc_rhs<<<grid1d(n), NT, 0, st>>>(u, f, g, c, kp);
  return cudaGetLastError();
}
cudaError_t launch_energy_terms(const double* u, const double* f, double gbar, const KParams& kp, Ctrl* ctrl,
                                double* partials, cudaStream_t st) {
  const size_t n = (size_t)kp.nx * kp.ny * kp.nz;
  k_energy_terms<<<std::min(grid1d(n), 1024), NT, 0, st>>>(u, f, gbar, kp, ctrl, partials);
  return cudaGetLastError();
}
cudaError_t launch_norms(const double* x, size_t n, double hd, Ctrl* c, double* partials, cudaStream_t st) {
  k_norms<<<std::min(grid1d(n), 1024), NT, 0, st>>>(x, n, hd, c, partials);
  return cudaGetLastError();
}
cudaError_t launch_mean_project(double* u, const double* g, size_t n, Ctrl* c, double* partials, cudaStream_t st) {
  k_mean_diff<<<std::min(grid1d(n), 1024), NT, 0, st>>>(g, u, n, c, partials);
  k_add_mean<<<grid1d(n), 256, 0, st>>>(u, c, n);
  return cudaGetLastError();
}
cudaError_t launch_round_f32(float* out, const double* in, size_t n, cudaStream_t st) {
  k_round_f32<<<grid1d(n), 256, 0, st>>>(out, in, n);
  return cudaGetLastError();
}
cudaError_t launch_accumulate_f64(double* u, const float* delta, float* u32, size_t n, const double* dsum,
                                  cudaStream_t st, const int* skip) {
  k_accumulate_f64<<<grid1d(n), 256, 0, st>>>(u, delta, u32, n, dsum, skip);
  return cudaGetLastError();
}

template cudaError_t launch_residual<float>(const ResArgs<float>&, int, int, const KParams&, Ctrl*, double*,
                                            cudaStream_t);
template cudaError_t launch_residual<double>(const ResArgs<double>&, int, int, const KParams&, Ctrl*, double*,
                                             cudaStream_t);
template cudaError_t launch_linesearch<float>(const float*, const float*, const float*, int, const KParams&, Ctrl*,
                                              double*, cudaStream_t);
template cudaError_t launch_linesearch<double>(const double*, const double*, const double*, int, const KParams&,
                                               Ctrl*, double*, cudaStream_t);
template cudaError_t launch_axpby<float>(float*, const float*, const float*, double, double, double, size_t,
                                         cudaStream_t);
template cudaError_t launch_axpby<double>(double*, const double*, const double*, double, double, double, size_t,
                                          cudaStream_t);

}  // namespace psd
