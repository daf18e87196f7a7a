"""Readings of the thin-film Cauchy convergence test (Sec. 6.1.1, Table 1)
run with the CPU oracle, to record which readings of the experiment match
the printed differences ||delta_u||_2 (p = 4: 6.2192e-3 for 16 -> 32,
1.2685e-3 for 32 -> 64).

Each reading runs the convex-splitting scheme N_h[u^{n+1}] = f(u^n) on the
coarse and the fine grid from the initial data of Eq. "init1" on (0, 3.2)^2
to the final time T with s = 0.1 h^2 (each grid its own h), every step
solved by the oracle's PSD to ||r||_2 < 1e-12, and prints ||u_f -
I(u_c)||_2 on the fine grid (I: cell-centred bilinear interpolation,
weights 3/4, 1/4) with its RMS and max.  Not a test (minutes per reading):

    python tests/table1_readings.py [--pairs 1|2] [--reading NAME ...]

Readings:
  baseline      f = u - s Delta_h^v u, eps = 0.1, T = 0.32, cell centres
  explicit_lap  the explicit term with the 5-point Delta_h
  vertex_grid   data sampled at x_i = i h, vertex-grid interpolation
  T_0032        T = 0.032
  stable_sign   f = u + s Delta_h^v u (a decaying, non-physical sign)
  eps_0.2, eps_0.5   other eps
  eps2_0.1      eps^2 = 0.1 (eps = 0.316); eps2_0.1_p6 the same at p = 6
  s_coarse      both grids step with s = 0.1 h_c^2 (the coarse grid's h), T / s steps
  s_fine        both grids step with s = 0.1 h_f^2 (the fine grid's h)
"""

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import psd_oracle as O  # noqa: E402

L = 3.2
READINGS = {
    "baseline": dict(),
    "explicit_lap": dict(explicit="lap"),
    "vertex_grid": dict(grid="vertex"),
    "T_0032": dict(T=0.032),
    "stable_sign": dict(explicit="plus"),
    "eps_0.2": dict(eps=0.2),
    "eps_0.5": dict(eps=0.5),
    "eps2_0.1": dict(eps=float(np.sqrt(0.1))),
    "eps2_0.1_p6": dict(eps=float(np.sqrt(0.1)), p=6.0),
    "s_coarse": dict(s_from="coarse"),
    "s_fine": dict(s_from="fine"),
}


def init1(n, grid):
    """Eq. "init1" at cell centres (i + 1/2) h or at vertices i h."""
    h = L / n
    x = (np.arange(n) + (0.5 if grid == "cell" else 0.0)) * h
    y = x[:, None]
    return (0.1 * np.sin(2 * np.pi * x / L) ** 2 * np.sin(4 * np.pi * (y - 1.4) / L)
            - 0.1 * np.cos(2 * np.pi * (x - 2.0) / L) * np.sin(2 * np.pi * y / L))


def run(n, p=4.0, T=0.32, eps=0.1, explicit="skew", grid="cell", s_h=None):
    """s_h: the grid spacing that sets s = 0.1 s_h^2 (default: this grid's h)."""
    h = L / n
    s = 0.1 * (s_h if s_h is not None else h) ** 2
    P = O.Problem(4, h, p, s, eps)
    u = init1(n, grid)
    for _ in range(int(round(T / s))):
        if explicit == "skew":
            f = u - s * O.skew_lap(u, h)
        elif explicit == "lap":
            f = u - s * O.lap(u, h)
        else:
            f = u + s * O.skew_lap(u, h)
        u, _ = O.psd_solve(P, f, u, tol=1e-12, kmax=500)
    return u


def up(v, grid):
    """Coarse -> fine bilinear interpolation on the periodic grid."""
    def one(w, ax):
        wp = np.roll(w, -1, axis=ax)
        if grid == "cell":  # fine centres 1/4 and 3/4 between coarse centres
            wm = np.roll(w, 1, axis=ax)
            out = np.stack([0.75 * w + 0.25 * wm, 0.75 * w + 0.25 * wp], axis=ax + 1)
        else:  # fine vertices on and halfway between coarse vertices
            out = np.stack([w, 0.5 * (w + wp)], axis=ax + 1)
        shape = list(w.shape)
        shape[ax] *= 2
        return out.reshape(shape)
    return one(one(v, 0), 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=1, help="grid pairs from 16 -> 32 on (2 adds 32 -> 64)")
    ap.add_argument("--reading", nargs="*", default=list(READINGS))
    args = ap.parse_args()
    print("printed (p = 4): 16->32 6.2192e-3, 32->64 1.2685e-3")
    for name in args.reading:
        cfg = dict(READINGS[name])
        grid = cfg.get("grid", "cell")
        s_from = cfg.pop("s_from", None)
        for k in range(args.pairs):
            nc = 16 * 2 ** k
            s_h = None if s_from is None else L / (nc if s_from == "coarse" else 2 * nc)
            uc, uf = run(nc, s_h=s_h, **cfg), run(2 * nc, s_h=s_h, **cfg)
            d = uf - up(uc, grid)
            hf = L / (2 * nc)
            print(f"{name:14s} {nc:3d}->{2 * nc:3d}  l2 {np.sqrt(hf * hf * np.sum(d * d)):.4e}  "
                  f"rms {np.sqrt(np.mean(d * d)):.4e}  max {np.abs(d).max():.4e}", flush=True)


if __name__ == "__main__":
    main()
