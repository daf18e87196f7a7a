// Column-owning 3D kernels (tiles of 32 x 8; nx >= 32, ny >= 8): the
// residual and the line-search reduction, organised for a low operation
// count (GB300 issues FP64 at 1/64 of the FP32 rate, so the FP64 variants
// are bound by their operation count).
//
// Arithmetic (same operators as Sec. 5.1 with the tensor reading in 3D):
//  * vertex gradient g = q G, q = 1/(4h), from per-cell z-pair sums
//    P = u(z) + u(z+1) and differences M = u(z+1) - u(z) of the two cell
//    planes around the vertex plane:
//      G_x = (P[x+1,y] - P[x,y]) + (P[x+1,y+1] - P[x,y+1])
//      G_y = (P[x,y+1] - P[x,y]) + (P[x+1,y+1] - P[x+1,y])
//      G_z = (M[x,y] + M[x+1,y]) + (M[x,y+1] + M[x+1,y+1]);
//  * flux Phi = |G|^{p-2} G (|g|^{p-2} g = q^{p-1} Phi);
//  * divergence from per-vertex z-sums S_c = Phi_c(z-1/2) + Phi_c(z+1/2)
//    (c = x, y) and D_z = Phi_z(z+1/2) - Phi_z(z-1/2), so that
//    s d.(|g|^{p-2} g) = cdiv * div', cdiv = s q^p;
//  * Laplacian sums lap' = h^2 Delta_h u, bih' = h^4 Delta_h^2 u.
//
// Each thread owns one (x, y) column and marches in z; z-neighbours are
// kept in registers, xy-neighbours go through shared memory, and the next
// plane's global loads are issued a step ahead.
//
// Residual, per step z (output plane z):
//   P/M of the vertex plane z+1/2 from the register history of U(z),
//   U(z+1) (and of the base field B); store U(z+2)          -> sync
//   prefetch U(z+3), B(z+2), f(z+1)
//   lap'(z+1) over tile + halo 1 -> sL ring
//   Phi(z+1/2) at own (+ halo) vertex; S/D with Phi(z-1/2) -> sS
//   -> sync -> residual at plane z.
// U = u_in + alpha d (the fused update; the owner writes it to u_out);
// B = the base field of the correction form (RM_INNER only).
#pragma once

namespace psd {
namespace {

// FFX (FP64, plain mode without an update, p = 4): no FP64 arithmetic
// before the final combination.  The linear part runs in 64-bit fixed
// point: each u enters as q = round(u 2^S) (a.fxs = S, picked by the caller
// from a bound on |u| so that |q| <= 2^55), and the z-pair sums, vertex
// gradients and both Laplacian passes are exact integer sums (|h^4 Delta_h^2
// q| <= 144 2^55 < 2^63).  The flux part -- |G|^2 G, its z-sums S and the
// divergence -- is evaluated in float-float from the exact gradients
// (converted by integer operations).  Only r = (f - cu u) + (cdiv div -
// cbih bih) and the norms are FP64, with cu u from the FP64 u itself; the
// flux and biharmonic terms are those of u rounded to the grid 2^-S (at
// most 2^-56 max|u| away, below the rounding of the FP64 Laplacian sums they
// replace).  The caller
// selects it only when the worst-case float-float error of the flux part is
// far below the solve tolerance (it scales with s q^4 max|G|^3).
template <typename T, int PK, int MODE, bool FFX = false>
__global__ void __launch_bounds__(256, 3)  // 80 registers (FP64 fixed-point variant), 3 CTAs per SM
    k_res3d_col(ResArgs<T> a, KParams kp, Ctrl* ctrl, double* partials) {
  static_assert(!FFX || (sizeof(T) == 8 && MODE == RM_PLAIN && PK == PK_4), "FFX: FP64 plain p = 4 only");
  using FT = typename std::conditional<FFX, ff, T>::type;         // arithmetic type of the flux part
  using LT = typename std::conditional<FFX, long long, T>::type;  // and of the linear part
  if (ctrl->done) return;
  constexpr int TX = 32, TY = 8;
  constexpr int UX = TX + 4, UY = TY + 4, UN = UX * UY;  // U tile, halo 2
  constexpr int LX = TX + 2, LY = TY + 2, LN = LX * LY;  // halo-1 tile (Laplacian, P/M)
  constexpr int VX = TX + 1, VY = TY + 1;                // vertex tile
  constexpr bool INNER = MODE == RM_INNER;
  constexpr bool HVP = MODE == RM_HVP;
  constexpr bool BASE = MODE != RM_PLAIN;  // a base field B enters the flux
  constexpr int NLH = 2 * LX + 2 * TY;                   // Laplacian halo cells (84)
  constexpr int NVH = VY + TX;                           // vertex halo (41)
  __shared__ LT sU[3][UY][UX];
  __shared__ LT sL[2][LY][LX];
  __shared__ LT sP[LY][LX];
  __shared__ LT sM[LY][LX];
  __shared__ T sPb[BASE ? LY : 1][BASE ? LX : 1];
  __shared__ T sMb[BASE ? LY : 1][BASE ? LX : 1];
  __shared__ T sS[3][VY][VX];
  __shared__ T sred[32 * 2];
  __shared__ int sflag;

  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const size_t plane = (size_t)nx * ny;
  const bool upd = a.d != nullptr;
  const T alpha = upd ? (T)ctrl->alpha : T(0);
  const KConst<T>& C = kconst<T>(kp);
  const T cdiv = C.cdiv, cbih = C.cbih, cu = C.cu;
  const T beta = C.beta;
  // fixed point (FFX): u = q 2^-S (S in [15, 120]); the gradients enter the
  // flux as float-float values of G 2^-S, cbih absorbs 2^-S
  int fxs = FFX ? a.fxs : 0;
  if constexpr (FFX || (sizeof(T) == 8 && MODE == RM_PLAIN && PK == PK_4)) {
    if (a.fxs_dev != nullptr) {  // the scale decided on device: exactly one variant computes
      const int S = *a.fxs_dev;
      const bool fixed = S >= 15 && S <= 120;
      if (fixed != FFX) return;
      if (FFX) fxs = S;
    }
  }
  const T cbihq = FFX ? cbih * (T)fx_unit(fxs) : cbih;

  // One wave of CTAs: the column-planes (w = column * nz + z) are split
  // into equal contiguous shares, each marched as one or more z-segments
  // with their own prologue; columns map to tiles in lockstep order
  // (lockstep_tile).
  const int gx = nx / TX;
  const int ncol = gx * (ny / TY);
  const int wtot = ncol * nz;
  const int wend = (int)((long long)wtot * (blockIdx.x + 1) / gridDim.x);
  const int mls = lockstep_classes(gridDim.x, ncol);
  T acc2 = T(0), accm = T(0);
  for (int w = (int)((long long)wtot * blockIdx.x / gridDim.x); w < wend;) {
    const int col = w / nz, z0 = w - col * nz;
    const int zc = min(nz - z0, wend - w);
    w += zc;
    const int tile = lockstep_tile(col, mls, ncol);
    const int x0 = (tile % gx) * TX, y0 = (tile / gx) * TY;

    // this thread's U-tile elements (flattened e = tid, tid + 256) and where
    // they land in the halo-1 P/M tile
    int uoff[2], upm[2];
    bool uval[2], uown[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = tid + 256 * k;
      uval[k] = e < UN;
      const int ly = e / UX, lx = e - ly * UX;
      uoff[k] = ((y0 + ly - 2) & (ny - 1)) * nx + ((x0 + lx - 2) & (nx - 1));
      uown[k] = uval[k] && lx >= 2 && lx < TX + 2 && ly >= 2 && ly < TY + 2;
      upm[k] = (uval[k] && ly >= 1 && ly <= LY && lx >= 1 && lx <= LX) ? (ly - 1) * LX + (lx - 1) : -1;
    }
    int boff[2];
    bool bval[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = tid + 256 * k;
      bval[k] = BASE && e < LN;
      const int ly = e / LX, lx = e - ly * LX;
      boff[k] = ((y0 + ly - 1) & (ny - 1)) * nx + ((x0 + lx - 1) & (nx - 1));
    }
    const int gown = (y0 + ty) * nx + x0 + tx;

    T pu[2] = {T(0), T(0)}, pd[2] = {T(0), T(0)}, pb[2] = {T(0), T(0)};
    LT h1[2] = {LT(0), LT(0)}, h0[2] = {LT(0), LT(0)};  // U history: h1 newest stored plane, h0 the one before
    T bprev[2] = {T(0), T(0)};
    auto fetchU = [&](int zz) {
      const size_t gz = (size_t)(zz & (nz - 1)) * plane;
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (uval[k]) {
          pu[k] = a.u_in[gz + uoff[k]];
          if (upd) pd[k] = a.d[gz + uoff[k]];
        }
    };
    // store the prefetched plane zz into ring slot `slot` and shift the
    // register history (h0 <- h1 <- new)
    auto storeU = [&](int zz, int slot) {
      const size_t gz = (size_t)(zz & (nz - 1)) * plane;
      const bool ownplane = zz >= z0 && zz < z0 + zc;
      LT* dst = &sU[slot][0][0];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (uval[k]) {
          LT v;
          if constexpr (FFX) {
            v = fx_from_double(pu[k], fxs);
          } else {
            v = pu[k];
            if (upd) {
              v = v + alpha * pd[k];
              if (ownplane && uown[k]) a.u_out[gz + uoff[k]] = v;
            }
          }
          dst[tid + 256 * k] = v;
          h0[k] = h1[k];
          h1[k] = v;
        }
    };
    // P/M of the vertex plane between the two newest history planes
    auto storePM = [&]() {
      LT* P = &sP[0][0];
      LT* M = &sM[0][0];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (upm[k] >= 0) {
          P[upm[k]] = h0[k] + h1[k];
          M[upm[k]] = h1[k] - h0[k];
        }
    };
    auto fetchB = [&](int zz) {
      if (!BASE) return;
      const size_t gz = (size_t)(zz & (nz - 1)) * plane;
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (bval[k]) pb[k] = a.ubase[gz + boff[k]];
    };
    // base P/M between bprev and the prefetched plane (first: only record)
    auto storeB = [&](bool first) {
      if (!BASE) return;
      T* P = &sPb[0][0];
      T* M = &sMb[0][0];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (bval[k]) {
          if (!first) {
            P[tid + 256 * k] = bprev[k] + pb[k];
            M[tid + 256 * k] = pb[k] - bprev[k];
          }
          bprev[k] = pb[k];
        }
    };
    // h^2 Delta_h U at halo-1 cell (ly, lx) of the plane in slot s0
    auto lap_at = [&](int ly, int lx, int sm, int s0, int sp) -> LT {
      const LT c = sU[s0][ly + 1][lx + 1];
      const LT sum = (sU[s0][ly + 1][lx] + sU[s0][ly + 1][lx + 2]) + (sU[s0][ly][lx + 1] + sU[s0][ly + 2][lx + 1]) +
                     (sU[sm][ly + 1][lx + 1] + sU[sp][ly + 1][lx + 1]);
      return sum - LT(6) * c;
    };
    auto halo_lap_cell = [&](int h, int& ly, int& lx) {
      if (h < LX) {
        ly = 0;
        lx = h;
      } else if (h < 2 * LX) {
        ly = LY - 1;
        lx = h - LX;
      } else if (h < 2 * LX + TY) {
        ly = 1 + h - 2 * LX;
        lx = 0;
      } else {
        ly = 1 + h - 2 * LX - TY;
        lx = LX - 1;
      }
    };
    auto lap_plane = [&](int sm, int s0, int sp, int ls) -> LT {
      const LT own = lap_at(ty + 1, tx + 1, sm, s0, sp);
      sL[ls][ty + 1][tx + 1] = own;
      const int h = tid - (256 - NLH);
      if (h >= 0) {
        int ly, lx;
        halo_lap_cell(h, ly, lx);
        sL[ls][ly][lx] = lap_at(ly, lx, sm, s0, sp);
      }
      return own;
    };
    // Phi at vertex (vy, vx) of the current vertex plane (from sP/sM)
    auto vphi = [&](int vy, int vx, FT (&F)[3]) {
      LT G[3];
      G[0] = (sP[vy][vx + 1] - sP[vy][vx]) + (sP[vy + 1][vx + 1] - sP[vy + 1][vx]);
      G[1] = (sP[vy + 1][vx] - sP[vy][vx]) + (sP[vy + 1][vx + 1] - sP[vy][vx + 1]);
      G[2] = (sM[vy][vx] + sM[vy][vx + 1]) + (sM[vy + 1][vx] + sM[vy + 1][vx + 1]);
      if constexpr (FFX) {
        // exact integer gradients -> float-float values of G 2^-S (within 2^-47)
        const ff g0 = fx_to_ff(G[0], fxs), g1 = fx_to_ff(G[1], fxs), g2 = fx_to_ff(G[2], fxs);
        const ff q2 = ff_add_fast(ff_add_fast(g0 * g0, g1 * g1), g2 * g2);
        F[0] = q2 * g0;
        F[1] = q2 * g1;
        F[2] = q2 * g2;
      } else if (BASE) {
        T A[3];
        A[0] = (sPb[vy][vx + 1] - sPb[vy][vx]) + (sPb[vy + 1][vx + 1] - sPb[vy + 1][vx]);
        A[1] = (sPb[vy + 1][vx] - sPb[vy][vx]) + (sPb[vy + 1][vx + 1] - sPb[vy][vx + 1]);
        A[2] = (sMb[vy][vx] + sMb[vy][vx + 1]) + (sMb[vy + 1][vx] + sMb[vy + 1][vx + 1]);
        if (INNER)
          flux_diff<PK>(A, G, beta, F);
        else
          flux_lin<PK>(A, G, beta, F);
      } else {
        flux<PK>(G, beta, F);
      }
    };
    // the S sums in the arithmetic type of the flux (float-float pairs occupy
    // the 8 bytes of an FP64 slot)
    FT(*SS)[VY][VX] = reinterpret_cast<FT(*)[VY][VX]>(&sS[0][0][0]);
    // own vertex (ty+1, tx+1) and, for tid < NVH, one halo vertex
    const bool hv = tid < NVH;
    const int hvy = tid < VY ? tid : 0;
    const int hvx = tid < VY ? 0 : tid - VY + 1;
    FT Fo[3] = {FT(0), FT(0), FT(0)}, Fh[3] = {FT(0), FT(0), FT(0)};  // Phi of the previous vertex plane
    auto phi_plane = [&](bool first) {
      FT F[3];
      vphi(ty + 1, tx + 1, F);
      if (!first) {
        SS[0][ty + 1][tx + 1] = Fo[0] + F[0];
        SS[1][ty + 1][tx + 1] = Fo[1] + F[1];
        SS[2][ty + 1][tx + 1] = F[2] - Fo[2];
      }
      Fo[0] = F[0];
      Fo[1] = F[1];
      Fo[2] = F[2];
      if (hv) {
        vphi(hvy, hvx, F);
        if (!first) {
          SS[0][hvy][hvx] = Fh[0] + F[0];
          SS[1][hvy][hvx] = Fh[1] + F[1];
          SS[2][hvy][hvx] = F[2] - Fh[2];
        }
        Fh[0] = F[0];
        Fh[1] = F[1];
        Fh[2] = F[2];
      }
    };

    // ---- prologue
    // ring slots 0, 1, 2 hold U(z0-2), U(z0-1), U(z0); P/M of vertex plane z0-1/2
    fetchU(z0 - 2);
    storeU(z0 - 2, 0);
    fetchU(z0 - 1);
    storeU(z0 - 1, 1);
    fetchU(z0);
    storeU(z0, 2);
    storePM();  // from (U(z0-1), U(z0))
    fetchB(z0 - 1);
    storeB(true);
    fetchB(z0);
    storeB(false);  // base P/M of plane z0 - 1/2
    __syncthreads();
    LT Lm = lap_at(ty + 1, tx + 1, 0, 1, 2);  // lap'(z0 - 1), own column only
    phi_plane(true);                         // Phi(z0 - 1/2) into registers
    __syncthreads();
    fetchU(z0 + 1);
    storeU(z0 + 1, 0);  // history now (U(z0), U(z0+1))
    __syncthreads();
    int lz = 0;
    LT L0 = lap_plane(1, 2, 0, lz);  // lap'(z0)
    __syncthreads();  // lap'(z0) read slot 1, which the first loop step overwrites
    // loop convention: um = slot of U(z-1), u0 = U(z), u1 = U(z+1)
    int um = 1, u0 = 2, u1 = 0;
    fetchU(z0 + 2);
    fetchB(z0 + 1);
    T fr = a.f ? a.f[(size_t)(z0 & (nz - 1)) * plane + gown] : T(0);
    // FFX: the own cell's u in FP64 for the cu u term (the shared tile holds q)
    T ur = FFX ? a.u_in[(size_t)(z0 & (nz - 1)) * plane + gown] : T(0);

    for (int z = z0; z < z0 + zc; ++z) {
      const int u2 = um;
      storePM();        // vertex plane z + 1/2 from (U(z), U(z+1))
      storeU(z + 2, u2);
      storeB(false);    // base P/M of plane z + 1/2
      __syncthreads();  // (A)
      const T fcur = fr, ucur = ur;
      fetchU(z + 3);
      fetchB(z + 2);
      fr = a.f ? a.f[(size_t)((z + 1) & (nz - 1)) * plane + gown] : T(0);
      if constexpr (FFX) ur = a.u_in[(size_t)((z + 1) & (nz - 1)) * plane + gown];
      const LT Lp = lap_plane(u0, u1, u2, lz ^ 1);  // lap'(z+1)
      phi_plane(false);                             // S/D for the cells of plane z
      const LT ucl = sU[u0][ty + 2][tx + 2];
      __syncthreads();  // (B)
      const LT bihl = (((sL[lz][ty + 1][tx] + sL[lz][ty + 1][tx + 2]) + (sL[lz][ty][tx + 1] + sL[lz][ty + 2][tx + 1])) +
                       (Lm + Lp)) -
                      LT(6) * L0;
      // FFX: bih in units of 2^-S (cbihq carries the factor), u from FP64
      T uc, bih;
      if constexpr (FFX) {
        (void)ucl;
        uc = ucur;
        bih = fx_to_double(bihl);
      } else {
        (void)ucur;
        uc = ucl;
        bih = bihl;
      }
      const FT dx = (SS[0][ty][tx + 1] - SS[0][ty][tx]) + (SS[0][ty + 1][tx + 1] - SS[0][ty + 1][tx]);
      const FT dy = (SS[1][ty + 1][tx] - SS[1][ty][tx]) + (SS[1][ty + 1][tx + 1] - SS[1][ty][tx + 1]);
      const FT dz = (SS[2][ty][tx] + SS[2][ty][tx + 1]) + (SS[2][ty + 1][tx] + SS[2][ty + 1][tx + 1]);
      T div;
      if constexpr (FFX)
        div = ff_to_double_bits((dx + dy) + dz);
      else
        div = (dx + dy) + dz;
      T r;
      if (INNER)
        r = fcur - ((cu * uc + cbih * bih) - cdiv * div);
      else if (HVP)
        r = (cu * uc + cbih * bih) - cdiv * div;
      else
        r = (fcur - cu * uc) + (cdiv * div - cbihq * bih);
      a.r[(size_t)(z & (nz - 1)) * plane + gown] = r;
      acc2 += HVP ? uc * r : r * r;
      accm = fmax(accm, fabs(r));
      Lm = L0;
      L0 = Lp;
      lz ^= 1;
      um = u0;
      u0 = u1;
      u1 = u2;
    }
    __syncthreads();  // the next segment's prologue refills the shared tiles
  }

  T v[2] = {acc2, accm};
  block_reduce<T, 2, true>(v, sred);
  if (publish_and_check_last<T>(v, 2, reinterpret_cast<T*>(partials), &ctrl->counter[CS_RES], &sflag)) {
    T tt[2];
    gather_partials<T, 2, true>(tt, reinterpret_cast<const T*>(partials), sred);
    if (tid == 0) residual_epilogue(ctrl, kp, (double)tt[0], (double)tt[1], a.norm, a.update_iter, HVP);
  }
}

// Column-owning 3D line-search reduction (tiles of 32 x 8 vertices).  Each
// thread owns a vertex column; the z-pair sums / differences of u (+ base)
// and d are formed from a per-element register history as each plane
// arrives, double-buffered in shared memory (one barrier per plane).  The
// sums use the unscaled gradients A = a/q, B = b/q; the epilogue applies q^p.
template <typename T, int PK, bool INNER>
__global__ void __launch_bounds__(256, 3)
    k_ls3d_col(const T* __restrict__ u, const T* __restrict__ ubase, const T* __restrict__ d, KParams kp,
               Ctrl* ctrl, double* partials) {
  if (ctrl->done) return;
  if (!ls_closed_form<PK>() && ctrl->c3 != 0.0) return;  // Newton already converged
  constexpr int TX = 32, TY = 8;
  constexpr int SX = TX + 1, SY = TY + 1, SN = SX * SY;  // cells x0..x0+TX, y0..y0+TY
  __shared__ T sPu[2][SY][SX], sMu[2][SY][SX], sPd[2][SY][SX], sMd[2][SY][SX];
  __shared__ T sred[32 * ls_nsums<PK>()];
  __shared__ int sflag;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const size_t plane = (size_t)nx * ny;
  const T beta = kconst<T>(kp).beta, pm2 = kconst<T>(kp).pm2;
  const T trial = ls_closed_form<PK>() ? T(0) : (T)ctrl->alpha;
  // one wave of CTAs, each marching an equal share of the column-planes (as
  // the residual column kernel)
  const int gx = nx / TX;
  const int ncol = gx * (ny / TY);
  const int wtot = ncol * nz;
  const int wend = (int)((long long)wtot * (blockIdx.x + 1) / gridDim.x);
  const int mls = lockstep_classes(gridDim.x, ncol);
  int off[2], ely[2], elx[2];
  bool val[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int e = tid + 256 * k;
    val[k] = e < SN;
    ely[k] = e / SX;
    elx[k] = e - ely[k] * SX;
    off[k] = 0;
  }
  // prefetched plane: u, base and d kept apart until used a step later
  T pu[2] = {T(0), T(0)}, pbv[2] = {T(0), T(0)}, pdv[2] = {T(0), T(0)}, hu[2] = {T(0), T(0)},
    hdd[2] = {T(0), T(0)};
  auto fetch = [&](int zz) {
    const size_t gz = (size_t)(zz & (nz - 1)) * plane;
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (val[k]) {
        pu[k] = u[gz + off[k]];
        if (INNER) pbv[k] = ubase[gz + off[k]];
        pdv[k] = d[gz + off[k]];
      }
  };
  auto store = [&](int buf, bool first) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (val[k] && INNER) pu[k] += pbv[k];
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (val[k]) {
        if (!first) {
          (&sPu[buf][0][0])[tid + 256 * k] = hu[k] + pu[k];
          (&sMu[buf][0][0])[tid + 256 * k] = pu[k] - hu[k];
          (&sPd[buf][0][0])[tid + 256 * k] = hdd[k] + pdv[k];
          (&sMd[buf][0][0])[tid + 256 * k] = pdv[k] - hdd[k];
        }
        hu[k] = pu[k];
        hdd[k] = pdv[k];
      }
  };
  auto grad = [&](T (&P)[SY][SX], T (&M)[SY][SX], T (&g)[3]) {
    g[0] = (P[ty][tx + 1] - P[ty][tx]) + (P[ty + 1][tx + 1] - P[ty + 1][tx]);
    g[1] = (P[ty + 1][tx] - P[ty][tx]) + (P[ty + 1][tx + 1] - P[ty][tx + 1]);
    g[2] = (M[ty][tx] + M[ty][tx + 1]) + (M[ty + 1][tx] + M[ty + 1][tx + 1]);
  };
  T acc[ls_nsums<PK>()] = {};
  for (int w = (int)((long long)wtot * blockIdx.x / gridDim.x); w < wend;) {
    const int col = w / nz, z0 = w - col * nz;
    const int zc = min(nz - z0, wend - w);
    w += zc;
    const int tile = lockstep_tile(col, mls, ncol);
    const int x0 = (tile % gx) * TX, y0 = (tile / gx) * TY;
#pragma unroll
    for (int k = 0; k < 2; ++k) off[k] = ((y0 + ely[k]) & (ny - 1)) * nx + ((x0 + elx[k]) & (nx - 1));
    fetch(z0);
    store(0, true);
    fetch(z0 + 1);
    for (int z = z0; z < z0 + zc; ++z) {
      const int buf = (z - z0) & 1;
      store(buf, false);  // vertex plane z + 1/2
      __syncthreads();
      fetch(z + 2);
      T av[3], bv[3];
      grad(sPu[buf], sMu[buf], av);
      grad(sPd[buf], sMd[buf], bv);
      ls_accumulate<PK>(av, bv, trial, beta, pm2, acc);
    }
    __syncthreads();  // the next segment writes the shared buffers again
  }
  ls_finish<T, PK>(acc, sred, partials, ctrl, kp, &sflag);
}

}  // namespace
}  // namespace psd
