// Register-blocked 3D residual (tiles of 32 x 8*NY cells; nx % 32 == 0,
// ny % (8*NY) == 0): the residual kernel of the PSD iteration with the
// arithmetic of the column kernel (unscaled vertex gradients from z-pair
// sums P = U(z) + U(z+1), differences M = U(z+1) - U(z); Laplacian sums
// lap' = h^2 Delta_h U; vertex z-sums S of the flux), organised so that
// each value crosses shared memory as few times as possible.
//
// Each thread owns NY consecutive rows (y) of one column (x) of the tile
// and marches in z.  Values of its own cells (U history, P/M, lap', the
// flux of its own vertex, the S sums) stay in registers; shared memory
// carries only what another thread needs: the x-neighbours (lane +-1) and
// the rows above and below a thread's strip.  The ring of halo cells and
// vertices around the tile is computed by designated threads.  Per cell
// this reads about 17 words from shared memory (the column kernel: 47).
//
// Vertex (vy, vx) of the tile sits at (y0 + vy - 1/2, x0 + vx - 1/2); the
// own vertex of cell (cy, cx) is (cy + 1, cx + 1).  The halo-1 cell tile
// (P/M, lap') is indexed [cy + 1][cx + 1], the U tile (halo 2) [cy + 2][cx + 2].
//
// Step z (output plane z), ring slot of plane zz: (zz - z0 + 3) % 3:
//   store U(z+2); P/M of vertex plane z+1/2 from U(z), U(z+1)   -> sync A
//   prefetch U(z+3), B(z+2), f(z+1)
//   lap'(z+1) (own + halo ring) -> sL; flux at z+1/2 (own + halo vertices),
//   S = flux(z-1/2) +- flux(z+1/2) -> sS                        -> sync B
//   residual of plane z.
#pragma once

namespace psd {
namespace {

template <typename T, int PK, int MODE, int NY>
__global__ void __launch_bounds__(256, 2)
    k_res3d_rb(ResArgs<T> a, KParams kp, Ctrl* ctrl, double* partials) {
  if (ctrl->done) return;
  constexpr int TX = 32, TYT = 8 * NY;
  constexpr int UX = TX + 4, UY = TYT + 4;  // U tile, halo 2
  constexpr int LX = TX + 2, LY = TYT + 2;  // halo-1 cell tile
  constexpr int VX = TX + 1, VY = TYT + 1;  // vertex tile
  constexpr bool INNER = MODE == RM_INNER;
  constexpr bool HVP = MODE == RM_HVP;
  constexpr bool BASE = MODE != RM_PLAIN;
  constexpr int NUH = UX * UY - TX * TYT;  // U halo elements (2 rows top/bottom, 2 columns left/right)
  constexpr int NRING = 2 * LX + 2 * TYT;  // halo-1 ring cells
  constexpr int NLAP = 2 * TX + 2 * TYT;   // halo lap' cells (ring without corners)
  constexpr int NHV = VY + TX;             // halo vertices: column vx = 0 and row vy = 0
  static_assert(NRING <= 256 && NLAP <= 256 && NHV <= 256 && NUH <= 512, "halo work exceeds the block");
  __shared__ T sU[3][UY][UX];
  __shared__ T sL[2][LY][LX];
  __shared__ T sP[LY][LX];
  __shared__ T sM[LY][LX];
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
  const T cdiv = kconst<T>(kp).cdiv, cbih = kconst<T>(kp).cbih, cu = kconst<T>(kp).cu;
  const T beta = kconst<T>(kp).beta;
  const int cy0 = ty * NY;  // first own row (tile-local)

  // The grid is one wave of CTAs.  The column-planes (w = column * nz + z)
  // are split into equal contiguous shares; a CTA marches its share as one
  // or two z-segments, each with its own prologue, so no CTA waits for a
  // second wave.  Columns map to tiles in lockstep order (lockstep_tile).
  const int gx = nx / TX;
  const int ncol = gx * (ny / TYT);
  const int wtot = ncol * nz;
  const int wend = (int)((long long)wtot * (blockIdx.x + 1) / gridDim.x);
  const int mls = lockstep_classes(gridDim.x, ncol);
  T acc2 = T(0), accm = T(0);
  for (int w = (int)((long long)wtot * blockIdx.x / gridDim.x); w < wend;) {
    const int col = w / nz, z0 = w - col * nz;
    const int zc = min(nz - z0, wend - w);
    w += zc;
    const int tile = lockstep_tile(col, mls, ncol);
    const int x0 = (tile % gx) * TX, y0 = (tile / gx) * TYT;

    // global offsets (within a plane) of the own cells
    int ooff[NY];
#pragma unroll
    for (int i = 0; i < NY; ++i) ooff[i] = (y0 + cy0 + i) * nx + x0 + tx;

    // U halo elements of this thread: h = tid, tid + 256 (< NUH)
    int hoff[2], huy[2], hux[2];
    bool hval[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int h = tid + 256 * k;
      hval[k] = h < NUH;
      int uy = 0, ux = 0;
      if (h < 2 * UX) {
        uy = h / UX;
        ux = h - uy * UX;
      } else if (h < 4 * UX) {
        uy = UY - 2 + (h - 2 * UX) / UX;
        ux = (h - 2 * UX) % UX;
      } else {
        const int m = h - 4 * UX;  // middle rows: 4 per row
        uy = 2 + (m >> 2);
        const int c = m & 3;
        ux = c < 2 ? c : UX - 4 + c;
      }
      huy[k] = uy;
      hux[k] = ux;
      hoff[k] = ((y0 + uy - 2) & (ny - 1)) * nx + ((x0 + ux - 2) & (nx - 1));
    }
    // halo-1 ring cell of this thread (tid < NRING): P/M and base history
    const bool rv = tid < NRING;
    int rly = 0, rlx = 0;
    if (tid < LX) {
      rly = 0;
      rlx = tid;
    } else if (tid < 2 * LX) {
      rly = LY - 1;
      rlx = tid - LX;
    } else if (tid < 2 * LX + TYT) {
      rly = 1 + tid - 2 * LX;
      rlx = 0;
    } else {
      rly = 1 + tid - 2 * LX - TYT;
      rlx = LX - 1;
    }
    const int roff = ((y0 + rly - 1) & (ny - 1)) * nx + ((x0 + rlx - 1) & (nx - 1));
    // halo lap' cell of this thread (tid < NLAP), halo-1 tile coordinates
    const bool lv = tid < NLAP;
    int lly = 0, llx = 0;
    if (tid < TX) {
      lly = 0;
      llx = 1 + tid;
    } else if (tid < 2 * TX) {
      lly = LY - 1;
      llx = 1 + tid - TX;
    } else if (tid < 2 * TX + TYT) {
      lly = 1 + tid - 2 * TX;
      llx = 0;
    } else {
      lly = 1 + tid - 2 * TX - TYT;
      llx = LX - 1;
    }
    // halo vertex of this thread (tid < NHV)
    const bool hv = tid < NHV;
    const int hvy = tid < VY ? tid : 0;
    const int hvx = tid < VY ? 0 : tid - VY + 1;

    // ---- registers
    T pu[NY], pd[NY], ph[2], phd[2];  // prefetched U plane (own, halo) and d
    T pb[NY], pbr = T(0);             // prefetched base plane (own, ring)
    T u0[NY], u1[NY], u2[NY];         // own U(z), U(z+1), U(z+2)
    T Po[NY], Mo[NY], Pbo[NY], Mbo[NY];
    T bprev[NY], bring = T(0);
    T Lm[NY], L0[NY];
    T Fo[NY][3], Fh[3] = {T(0), T(0), T(0)};
    T pf[NY];
#pragma unroll
    for (int i = 0; i < NY; ++i) {
      pu[i] = pd[i] = pb[i] = u0[i] = u1[i] = u2[i] = T(0);
      Po[i] = Mo[i] = Pbo[i] = Mbo[i] = bprev[i] = Lm[i] = L0[i] = pf[i] = T(0);
      Fo[i][0] = Fo[i][1] = Fo[i][2] = T(0);
    }
    ph[0] = ph[1] = phd[0] = phd[1] = T(0);

    auto slot = [&](int zz) { return (zz - z0 + 3) % 3; };
    auto fetchU = [&](int zz) {
      const size_t gz = (size_t)(zz & (nz - 1)) * plane;
#pragma unroll
      for (int i = 0; i < NY; ++i) {
        pu[i] = a.u_in[gz + ooff[i]];
        if (upd) pd[i] = a.d[gz + ooff[i]];
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (hval[k]) {
          ph[k] = a.u_in[gz + hoff[k]];
          if (upd) phd[k] = a.d[gz + hoff[k]];
        }
    };
    // store the prefetched plane zz (own + halo) into its ring slot; the
    // updated own values go to u2 (and to u_out inside the block's z range)
    auto storeU = [&](int zz, int sl) {  // sl = slot(zz)
      const size_t gz = (size_t)(zz & (nz - 1)) * plane;
      const bool ownplane = zz >= z0 && zz < z0 + zc;
      T(*S)[UX] = sU[sl];
#pragma unroll
      for (int i = 0; i < NY; ++i) {
        T v = pu[i];
        if (upd) {
          v = v + alpha * pd[i];
          if (ownplane) a.u_out[gz + ooff[i]] = v;
        }
        S[cy0 + i + 2][tx + 2] = v;
        u2[i] = v;
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (hval[k]) {
          T v = ph[k];
          if (upd) v = v + alpha * phd[k];
          S[huy[k]][hux[k]] = v;
        }
    };
    auto fetchB = [&](int zz) {
      if constexpr (BASE) {
        const size_t gz = (size_t)(zz & (nz - 1)) * plane;
#pragma unroll
        for (int i = 0; i < NY; ++i) pb[i] = a.ubase[gz + ooff[i]];
        if (rv) pbr = a.ubase[gz + roff];
      }
    };
    // P/M of the vertex plane between U planes zl and zl+1 (own from the
    // registers ua, ub; ring from the U ring), and of the base field between
    // bprev and the prefetched base plane (first: only record)
    auto storePM = [&](const T (&ua)[NY], const T (&ub)[NY], int sa, int sb) {  // slots of zl, zl + 1
#pragma unroll
      for (int i = 0; i < NY; ++i) {
        Po[i] = ua[i] + ub[i];
        Mo[i] = ub[i] - ua[i];
        sP[cy0 + i + 1][tx + 1] = Po[i];
        sM[cy0 + i + 1][tx + 1] = Mo[i];
      }
      if (rv) {
        const T va = sU[sa][rly + 1][rlx + 1], vb = sU[sb][rly + 1][rlx + 1];
        sP[rly][rlx] = va + vb;
        sM[rly][rlx] = vb - va;
      }
    };
    auto storeB = [&](bool first) {
      if constexpr (BASE) {
#pragma unroll
        for (int i = 0; i < NY; ++i) {
          if (!first) {
            Pbo[i] = bprev[i] + pb[i];
            Mbo[i] = pb[i] - bprev[i];
            sPb[cy0 + i + 1][tx + 1] = Pbo[i];
            sMb[cy0 + i + 1][tx + 1] = Mbo[i];
          }
          bprev[i] = pb[i];
        }
        if (rv) {
          if (!first) {
            sPb[rly][rlx] = bring + pbr;
            sMb[rly][rlx] = pbr - bring;
          }
          bring = pbr;
        }
      }
    };
    // lap' of the own cells of plane zc_ (U ring slot s0) with z-neighbours
    // in registers um, up
    auto lap_own = [&](const T (&um)[NY], const T (&uc)[NY], const T (&up)[NY], int s0, T (&out)[NY]) {
      T(*S)[UX] = sU[s0];
      const T above = S[cy0 + 1][tx + 2];   // row cy0 - 1
      const T below = S[cy0 + NY + 2][tx + 2];  // row cy0 + NY
#pragma unroll
      for (int i = 0; i < NY; ++i) {
        const T yn = (i == 0 ? above : uc[i - 1]) + (i == NY - 1 ? below : uc[i + 1]);
        const T xn = S[cy0 + i + 2][tx + 1] + S[cy0 + i + 2][tx + 3];
        out[i] = ((xn + yn) + (um[i] + up[i])) - T(6) * uc[i];
      }
    };
    // lap' at halo cell (ly, lx) of the halo-1 tile from three ring slots
    auto lap_halo = [&](int ly, int lx, int sm, int s0, int sp) -> T {
      const T c = sU[s0][ly + 1][lx + 1];
      const T sum = (sU[s0][ly + 1][lx] + sU[s0][ly + 1][lx + 2]) + (sU[s0][ly][lx + 1] + sU[s0][ly + 2][lx + 1]) +
                    (sU[sm][ly + 1][lx + 1] + sU[sp][ly + 1][lx + 1]);
      return sum - T(6) * c;
    };
    auto flux_of = [&](const T (&G)[3], const T (&A)[3], T (&F)[3]) {
      if (BASE) {
        if (INNER)
          flux_diff<PK>(A, G, beta, F);
        else
          flux_lin<PK>(A, G, beta, F);
      } else {
        flux<PK>(G, beta, F);
      }
    };
    // flux at a halo vertex (all from shared memory)
    auto vphi_halo = [&](int vy, int vx, T (&F)[3]) {
      T G[3], A[3] = {T(0), T(0), T(0)};
      G[0] = (sP[vy][vx + 1] - sP[vy][vx]) + (sP[vy + 1][vx + 1] - sP[vy + 1][vx]);
      G[1] = (sP[vy + 1][vx] - sP[vy][vx]) + (sP[vy + 1][vx + 1] - sP[vy][vx + 1]);
      G[2] = (sM[vy][vx] + sM[vy][vx + 1]) + (sM[vy + 1][vx] + sM[vy + 1][vx + 1]);
      if (BASE) {
        A[0] = (sPb[vy][vx + 1] - sPb[vy][vx]) + (sPb[vy + 1][vx + 1] - sPb[vy + 1][vx]);
        A[1] = (sPb[vy + 1][vx] - sPb[vy][vx]) + (sPb[vy + 1][vx + 1] - sPb[vy][vx + 1]);
        A[2] = (sMb[vy][vx] + sMb[vy][vx + 1]) + (sMb[vy + 1][vx] + sMb[vy + 1][vx + 1]);
      }
      flux_of(G, A, F);
    };
    // fluxes of the own vertices (cy0 + i + 1, tx + 1), i < NY: P/M of the
    // own cells from registers, of column tx + 1 and of row cy0 + NY from
    // shared memory.  Writes the S sums and shifts Fo (first: only record).
    T So[NY][3];
    auto phi_own = [&](bool first) {
      T Px[NY + 1], Mx[NY + 1], Pbx[NY + 1], Mbx[NY + 1];
#pragma unroll
      for (int i = 0; i <= NY; ++i) {
        Px[i] = sP[cy0 + i + 1][tx + 2];
        Mx[i] = sM[cy0 + i + 1][tx + 2];
        if (BASE) {
          Pbx[i] = sPb[cy0 + i + 1][tx + 2];
          Mbx[i] = sMb[cy0 + i + 1][tx + 2];
        }
      }
      const T Pn = sP[cy0 + NY + 1][tx + 1], Mn = sM[cy0 + NY + 1][tx + 1];
      T Pbn = T(0), Mbn = T(0);
      if (BASE) {
        Pbn = sPb[cy0 + NY + 1][tx + 1];
        Mbn = sMb[cy0 + NY + 1][tx + 1];
      }
#pragma unroll
      for (int i = 0; i < NY; ++i) {
        // cells (i, x), (i, x+1), (i+1, x), (i+1, x+1) of the strip
        const T p00 = Po[i], p01 = Px[i], p10 = (i == NY - 1) ? Pn : Po[i + 1], p11 = Px[i + 1];
        const T m00 = Mo[i], m01 = Mx[i], m10 = (i == NY - 1) ? Mn : Mo[i + 1], m11 = Mx[i + 1];
        T G[3], A[3] = {T(0), T(0), T(0)}, F[3];
        G[0] = (p01 - p00) + (p11 - p10);
        G[1] = (p10 - p00) + (p11 - p01);
        G[2] = (m00 + m01) + (m10 + m11);
        if (BASE) {
          const T q00 = Pbo[i], q01 = Pbx[i], q10 = (i == NY - 1) ? Pbn : Pbo[i + 1], q11 = Pbx[i + 1];
          const T n00 = Mbo[i], n01 = Mbx[i], n10 = (i == NY - 1) ? Mbn : Mbo[i + 1], n11 = Mbx[i + 1];
          A[0] = (q01 - q00) + (q11 - q10);
          A[1] = (q10 - q00) + (q11 - q01);
          A[2] = (n00 + n01) + (n10 + n11);
        }
        flux_of(G, A, F);
        if (!first) {
          So[i][0] = Fo[i][0] + F[0];
          So[i][1] = Fo[i][1] + F[1];
          So[i][2] = F[2] - Fo[i][2];
          sS[0][cy0 + i + 1][tx + 1] = So[i][0];
          sS[1][cy0 + i + 1][tx + 1] = So[i][1];
          sS[2][cy0 + i + 1][tx + 1] = So[i][2];
        }
        Fo[i][0] = F[0];
        Fo[i][1] = F[1];
        Fo[i][2] = F[2];
      }
    };
    auto phi_halo = [&](bool first) {
      if (!hv) return;
      T F[3];
      vphi_halo(hvy, hvx, F);
      if (!first) {
        sS[0][hvy][hvx] = Fh[0] + F[0];
        sS[1][hvy][hvx] = Fh[1] + F[1];
        sS[2][hvy][hvx] = F[2] - Fh[2];
      }
      Fh[0] = F[0];
      Fh[1] = F[1];
      Fh[2] = F[2];
    };

    // ---- prologue: U(z0-2) own only; U(z0-1), U(z0) in the ring; P/M of the
    // vertex plane z0-1/2 and the fluxes there; lap'(z0-1) own; U(z0+1);
    // lap'(z0) own + halo
    T um2[NY];
    fetchU(z0 - 2);
#pragma unroll
    for (int i = 0; i < NY; ++i) um2[i] = upd ? pu[i] + alpha * pd[i] : pu[i];
    fetchU(z0 - 1);
    storeU(z0 - 1, slot(z0 - 1));
#pragma unroll
    for (int i = 0; i < NY; ++i) u1[i] = u2[i];  // u1 = U(z0-1) for now
    fetchU(z0);
    storeU(z0, slot(z0));  // u2 = U(z0)
    fetchB(z0 - 1);
    storeB(true);
    fetchB(z0);
    storeB(false);  // base P/M of vertex plane z0 - 1/2
    __syncthreads();
    lap_own(um2, u1, u2, slot(z0 - 1), Lm);  // lap'(z0-1)
    storePM(u1, u2, slot(z0 - 1), slot(z0));  // P/M of vertex plane z0 - 1/2
#pragma unroll
    for (int i = 0; i < NY; ++i) u0[i] = u2[i];  // u0 = U(z0)
    __syncthreads();
    phi_own(true);
    phi_halo(true);
    fetchU(z0 + 1);
    storeU(z0 + 1, slot(z0 + 1));  // u2 = U(z0+1)
#pragma unroll
    for (int i = 0; i < NY; ++i) {
      um2[i] = u1[i];  // U(z0-1)
      u1[i] = u2[i];   // U(z0+1)
    }
    __syncthreads();
    int lb = 0;  // sL buffer of lap'(z)
    lap_own(um2, u0, u1, slot(z0), L0);
#pragma unroll
    for (int i = 0; i < NY; ++i) sL[lb][cy0 + i + 1][tx + 1] = L0[i];
    if (lv) sL[lb][lly][llx] = lap_halo(lly, llx, slot(z0 - 1), slot(z0), slot(z0 + 1));
    __syncthreads();  // the ring slot of U(z0-1) is refilled by the first step
    fetchU(z0 + 2);
    fetchB(z0 + 1);
    const size_t fz0 = (size_t)(z0 & (nz - 1)) * plane;
#pragma unroll
    for (int i = 0; i < NY; ++i) pf[i] = a.f ? a.f[fz0 + ooff[i]] : T(0);

    int s0 = 0, s1 = 1, s2 = 2;  // ring slots of U(z), U(z+1), U(z+2)
    for (int z = z0; z < z0 + zc; ++z) {
      // invariant: u0 = U(z), u1 = U(z+1); Lm = lap'(z-1), L0 = lap'(z) (own;
      // lap'(z) with halo in sL[lb]); Fo = flux at z - 1/2; U(z+2), B(z+1),
      // f(z) prefetched
      storeU(z + 2, s2);  // u2 = U(z+2)
      storePM(u0, u1, s0, s1);
      storeB(false);
      T fcur[NY];
#pragma unroll
      for (int i = 0; i < NY; ++i) fcur[i] = pf[i];
      __syncthreads();  // (A)
      fetchU(z + 3);
      fetchB(z + 2);
      {
        const size_t fz = (size_t)((z + 1) & (nz - 1)) * plane;
#pragma unroll
        for (int i = 0; i < NY; ++i) pf[i] = a.f ? a.f[fz + ooff[i]] : T(0);
      }
      T Lp[NY];
      lap_own(u0, u1, u2, s1, Lp);  // lap'(z+1)
#pragma unroll
      for (int i = 0; i < NY; ++i) sL[lb ^ 1][cy0 + i + 1][tx + 1] = Lp[i];
      if (lv) sL[lb ^ 1][lly][llx] = lap_halo(lly, llx, s0, s1, s2);
      phi_own(false);
      phi_halo(false);
      __syncthreads();  // (B)
      // residual of plane z
      {
        T(*L)[LX] = sL[lb];
        const T Labove = L[cy0][tx + 1], Lbelow = L[cy0 + NY + 1][tx + 1];
        T Sx[3][NY + 1];  // S at the vertices of column tx (x - 1/2), rows cy0 .. cy0 + NY
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int i = 0; i <= NY; ++i) Sx[c][i] = sS[c][cy0 + i][tx];
        T Stop[3];  // S at vertex (cy0, tx + 1), the row above the strip
#pragma unroll
        for (int c = 0; c < 3; ++c) Stop[c] = sS[c][cy0][tx + 1];
        const size_t gz = (size_t)(z & (nz - 1)) * plane;
#pragma unroll
        for (int i = 0; i < NY; ++i) {
          const T yn = (i == 0 ? Labove : L0[i - 1]) + (i == NY - 1 ? Lbelow : L0[i + 1]);
          const T xn = L[cy0 + i + 1][tx] + L[cy0 + i + 1][tx + 2];
          const T bih = ((xn + yn) + (Lm[i] + Lp[i])) - T(6) * L0[i];
          // vertices: (i, x-1/2) = Sx[.][i], (i+1, x-1/2) = Sx[.][i+1],
          // (i, x+1/2) = row above (Stop or So[i-1]), (i+1, x+1/2) = So[i]
          T up3[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) up3[c] = (i == 0) ? Stop[c] : So[i - 1][c];
          const T dx = (up3[0] - Sx[0][i]) + (So[i][0] - Sx[0][i + 1]);
          const T dy = (Sx[1][i + 1] - Sx[1][i]) + (So[i][1] - up3[1]);
          const T dz = (Sx[2][i] + up3[2]) + (Sx[2][i + 1] + So[i][2]);
          const T div = (dx + dy) + dz;
          const T uc = u0[i];
          T r;
          if (INNER)
            r = fcur[i] - ((cu * uc + cbih * bih) - cdiv * div);
          else if (HVP)
            r = (cu * uc + cbih * bih) - cdiv * div;
          else
            r = (fcur[i] - cu * uc) + (cdiv * div - cbih * bih);
          a.r[gz + ooff[i]] = r;
          acc2 += HVP ? uc * r : r * r;
          accm = fmax(accm, fabs(r));
        }
      }
#pragma unroll
      for (int i = 0; i < NY; ++i) {
        Lm[i] = L0[i];
        L0[i] = Lp[i];
        u0[i] = u1[i];
        u1[i] = u2[i];
      }
      lb ^= 1;
      const int st = s0;
      s0 = s1;
      s1 = s2;
      s2 = st;
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

// Register-blocked 3D line-search reduction (tiles of 32 x 8*NY vertices).
// Vertex (cy, cx) of the tile sits at (y0 + cy + 1/2, x0 + cx + 1/2); each
// thread owns the vertices of NY consecutive rows of one column.  The z-pair
// sums / differences of u (+ base) and d of its own cells are formed in
// registers; those of the cells at x + 1 and of the row below the strip come
// through shared memory (double-buffered, one barrier per plane).  The extra
// column (x0 + 32) and row (y0 + 8 NY) of cells are carried by threads
// tid < 8 NY + 33.  Same unscaled vertex sums as the column kernel.
template <typename T, int PK, bool INNER, int NY>
__global__ void __launch_bounds__(256, 3)
    k_ls3d_rb(const T* __restrict__ u, const T* __restrict__ ubase, const T* __restrict__ d, KParams kp,
              Ctrl* ctrl, double* partials) {
  if (ctrl->done) return;
  if (!ls_closed_form<PK>() && ctrl->c3 != 0.0) return;  // Newton already converged
  constexpr int TX = 32, TYT = 8 * NY;
  constexpr int SX = TX + 1, SY = TYT + 1;  // cells x0 .. x0+TX, y0 .. y0+TYT
  constexpr int NH = SY + TX;               // halo cells: column TX (SY) and row TYT (TX)
  __shared__ T sPu[2][SY][SX], sMu[2][SY][SX], sPd[2][SY][SX], sMd[2][SY][SX];
  __shared__ T sred[32 * ls_nsums<PK>()];
  __shared__ int sflag;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
  const size_t plane = (size_t)nx * ny;
  const T beta = kconst<T>(kp).beta, pm2 = kconst<T>(kp).pm2;
  const T trial = ls_closed_form<PK>() ? T(0) : (T)ctrl->alpha;
  const int cy0 = ty * NY;
  const bool hv = tid < NH;
  const int hly = tid < SY ? tid : TYT, hlx = tid < SY ? TX : tid - SY;
  // one wave of CTAs, each marching an equal share of the column-planes in
  // one or two z-segments (as the register-blocked residual)
  const int gx = nx / TX;
  const int ncol = gx * (ny / TYT);
  const int wtot = ncol * nz;
  const int wend = (int)((long long)wtot * (blockIdx.x + 1) / gridDim.x);
  const int mls = lockstep_classes(gridDim.x, ncol);
  int x0 = 0, y0 = 0, ooff0 = 0, hoff = 0;

  // prefetched plane: u, base and d kept apart until the plane is used a
  // step later (summing them at fetch time would wait on the loads there)
  T pu[NY], pb[NY], pd[NY], hu[NY], hd[NY], Pu[NY], Mu[NY], Pd[NY], Md[NY];
  T puh = T(0), pbh = T(0), pdh = T(0), huh = T(0), hdh = T(0);
#pragma unroll
  for (int i = 0; i < NY; ++i) pu[i] = pb[i] = pd[i] = hu[i] = hd[i] = Pu[i] = Mu[i] = Pd[i] = Md[i] = T(0);
  auto fetch = [&](int zz) {
    const size_t gz = (size_t)(zz & (nz - 1)) * plane;
#pragma unroll
    for (int i = 0; i < NY; ++i) {
      const size_t g = gz + ooff0 + (size_t)i * nx;
      pu[i] = u[g];
      if (INNER) pb[i] = ubase[g];
      pd[i] = d[g];
    }
    if (hv) {
      puh = u[gz + hoff];
      if (INNER) pbh = ubase[gz + hoff];
      pdh = d[gz + hoff];
    }
  };
  // P/M of the vertex plane between the history and the fetched plane
  auto store = [&](int buf, bool first) {
    if (INNER) {
#pragma unroll
      for (int i = 0; i < NY; ++i) pu[i] += pb[i];
      puh += pbh;
    }
#pragma unroll
    for (int i = 0; i < NY; ++i) {
      if (!first) {
        Pu[i] = hu[i] + pu[i];
        Mu[i] = pu[i] - hu[i];
        Pd[i] = hd[i] + pd[i];
        Md[i] = pd[i] - hd[i];
        sPu[buf][cy0 + i][tx] = Pu[i];
        sMu[buf][cy0 + i][tx] = Mu[i];
        sPd[buf][cy0 + i][tx] = Pd[i];
        sMd[buf][cy0 + i][tx] = Md[i];
      }
      hu[i] = pu[i];
      hd[i] = pd[i];
    }
    if (hv) {
      if (!first) {
        sPu[buf][hly][hlx] = huh + puh;
        sMu[buf][hly][hlx] = puh - huh;
        sPd[buf][hly][hlx] = hdh + pdh;
        sMd[buf][hly][hlx] = pdh - hdh;
      }
      huh = puh;
      hdh = pdh;
    }
  };
  T acc[ls_nsums<PK>()] = {};
  for (int w = (int)((long long)wtot * blockIdx.x / gridDim.x); w < wend;) {
    const int col = w / nz, z0 = w - col * nz;
    const int zc = min(nz - z0, wend - w);
    w += zc;
    const int tile = lockstep_tile(col, mls, ncol);
    x0 = (tile % gx) * TX;
    y0 = (tile / gx) * TYT;
    ooff0 = (y0 + cy0) * nx + x0 + tx;  // own cell of row i: ooff0 + i nx
    hoff = ((y0 + hly) & (ny - 1)) * nx + ((x0 + hlx) & (nx - 1));
    fetch(z0);
    store(0, true);
    fetch(z0 + 1);
    for (int z = z0; z < z0 + zc; ++z) {
      const int buf = (z - z0) & 1;
      store(buf, false);  // vertex plane z + 1/2
      __syncthreads();
      fetch(z + 2);
      T xPu[NY + 1], xMu[NY + 1], xPd[NY + 1], xMd[NY + 1];  // cells (cy0 + i, tx + 1)
#pragma unroll
      for (int i = 0; i <= NY; ++i) {
        xPu[i] = sPu[buf][cy0 + i][tx + 1];
        xMu[i] = sMu[buf][cy0 + i][tx + 1];
        xPd[i] = sPd[buf][cy0 + i][tx + 1];
        xMd[i] = sMd[buf][cy0 + i][tx + 1];
      }
      const T nPu = sPu[buf][cy0 + NY][tx], nMu = sMu[buf][cy0 + NY][tx];  // cell (cy0 + NY, tx)
      const T nPd = sPd[buf][cy0 + NY][tx], nMd = sMd[buf][cy0 + NY][tx];
#pragma unroll
      for (int i = 0; i < NY; ++i) {
        const T p10 = i == NY - 1 ? nPu : Pu[i + 1], m10 = i == NY - 1 ? nMu : Mu[i + 1];
        const T q10 = i == NY - 1 ? nPd : Pd[i + 1], n10 = i == NY - 1 ? nMd : Md[i + 1];
        T av[3], bv[3];
        av[0] = (xPu[i] - Pu[i]) + (xPu[i + 1] - p10);
        av[1] = (p10 - Pu[i]) + (xPu[i + 1] - xPu[i]);
        av[2] = (Mu[i] + xMu[i]) + (m10 + xMu[i + 1]);
        bv[0] = (xPd[i] - Pd[i]) + (xPd[i + 1] - q10);
        bv[1] = (q10 - Pd[i]) + (xPd[i + 1] - xPd[i]);
        bv[2] = (Md[i] + xMd[i]) + (n10 + xMd[i + 1]);
        ls_accumulate<PK>(av, bv, trial, beta, pm2, acc);
      }
    }
    __syncthreads();  // the next segment writes the shared buffers again
  }
  ls_finish<T, PK>(acc, sred, partials, ctrl, kp, &sflag);
}

}  // namespace
}  // namespace psd
