"""Parity at the benchmark's grid size n = 256, against the FP64 CPU oracle.

The 256^3 sixth-order benchmark runs length-256 instantiations of every
transform kernel (FP64 and FP32 row, column and middle passes; the
float-float passes of the mixed solver's outer loop).  Each of them is
checked here on grids that put n = 256 on one axis at a time (and on a
full 256^2 cross-section), element by element against the oracle; the
benchmark's own answers (mixed and plain FP64) are then checked by the
oracle's residual, evaluated with its own FFT for T_h.

Tolerances (relative L-infinity, max|a - b| / max|b|): 1e-12 for FP64 and
float-float outputs (each output is a sum of O(n) terms with rounding of a
few eps64 log2(n) of the largest term; double-word arithmetic carries about
48 bits); converged answers: ||r||_2 of the oracle below 1.05 tol.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01475_gb300 import PSD_FP64, PSD_MIXED, Solver  # noqa: E402
from paper_1607_01475_gb300 import synthetic  # noqa: E402

rng = np.random.default_rng(256)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# n = 256 along z (the middle pass), y (the strided pass), x (the row pass),
# a full 256 x 256 cross-section, and the 2D middle and row passes
SHAPES_256 = [(256, 8, 16), (8, 256, 16), (8, 16, 256), (16, 256, 256), (256, 64), (64, 256)]


def _problem(oracle, order, shape, p=4.0, s=0.05, eps=0.1, lam=1.0):
    h = 2 * np.pi / 256
    return oracle.Problem(order, h, p, s, eps, lam), h


@pytest.mark.parametrize("shape", SHAPES_256)
@pytest.mark.parametrize("order", [4, 6])
def test_precond_parity_n256(oracle, shape, order):
    """FP64 search-direction solve L_h d = r (Sec. 6, the symbols of Sec. 5.3
    and 5.4) by the length-256 DHT passes."""
    P, h = _problem(oracle, order, shape)
    r = rng.standard_normal(shape)
    S = Solver(order, shape, h, 4.0, P.s, P.eps, P.lam)
    d = torch.empty(shape, dtype=torch.float64, device="cuda")
    S.precond_solve(dev(r), d)
    ref = oracle.precond4(r, P) if order == 4 else oracle.precond6(r, P)
    assert rel(host(d), ref) <= 1e-12


def test_precond_parity_full_256_cube(oracle):
    """The sixth-order FP64 preconditioner on the benchmark grid itself."""
    shape = (256, 256, 256)
    P, h = _problem(oracle, 6, shape)
    r = synthetic.fourier_field(shape, 2 * np.pi, 16, 4242)
    S = Solver(6, shape, h, 4.0, P.s, P.eps, P.lam)
    d = torch.empty(shape, dtype=torch.float64, device="cuda")
    S.precond_solve(dev(r), d)
    ref = oracle.precond6(r, P)
    assert rel(host(d), ref) <= 1e-12


@pytest.mark.parametrize("shape", SHAPES_256)
@pytest.mark.parametrize("order,p", [(4, 4.0), (6, 4.0), (4, 3.0)])
def test_residual_parity_n256(oracle, shape, order, p):
    """FP64 residual f - N_h[u] (order 6 with T_h[u - g] through the
    length-256 transforms) at h = 2 pi / 256."""
    P, h = _problem(oracle, order, shape, p)
    u = rng.standard_normal(shape) * 0.3
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape) if order == 6 else None
    if order == 6:
        u = u - u.mean() + g.mean()
    S = Solver(order, shape, h, p, P.s, P.eps, P.lam)
    r = torch.empty(shape, dtype=torch.float64, device="cuda")
    S.residual(dev(u), dev(f), None if g is None else dev(g), r)
    ref = oracle.residual4(u, f, P) if order == 4 else oracle.residual6(u, f, g, P)
    assert rel(host(r), ref) <= 1e-12


def _hartley(oracle, v):
    """Separable discrete Hartley transform from the oracle's DFT:
    per axis, cas(t) = cos(t) + sin(t) gives Re F - Im F for
    F_k = sum_j v_j exp(-2 pi i j k / n)."""
    out = np.asarray(v, dtype=np.float64)
    for ax in range(out.ndim):
        F = oracle.fft_axis(out, ax)
        out = F.real - F.imag
    return out


@pytest.mark.parametrize("shape", SHAPES_256 + [(256, 256, 256), (16, 16, 16), (8, 8, 8), (32, 32)])
def test_theta_ff_parity(oracle, shape):
    """The float-float transform passes of the mixed sixth-order outer loop,
    theta += H[T_h x], element by element against the oracle's T_h (its own
    FFT) and a Hartley transform composed from its DFT."""
    h = 2 * np.pi / 256
    x = rng.standard_normal(shape)
    theta0 = rng.standard_normal(shape) * 1e-3
    S = Solver(6, shape, h, 4.0, 0.05, 0.1, 1.0, precision=PSD_MIXED)
    th = dev(theta0)
    S.theta_ff(dev(x), th)
    ref = theta0 + _hartley(oracle, oracle.T_h(x, h))
    assert rel(host(th), ref) <= 1e-12


@pytest.mark.parametrize("shape", [(16, 256, 256), (256, 16, 32)])
def test_mixed_sixth_order_n256_checked_by_oracle(oracle, shape):
    """Mixed-precision sixth-order solves whose outer loop runs the
    length-256 float-float transforms: the oracle's residual at the answer
    is below the tolerance and mean(u) = mean(g)."""
    h = 2 * np.pi / 256
    f = synthetic.fourier_field(shape, 2 * np.pi, 16, 5001)
    g = synthetic.fourier_field(shape, 2 * np.pi, 16, 5002)
    P = oracle.Problem(6, h, 4.0, 0.05, 0.1, 1.0)
    S = Solver(6, shape, h, 4.0, 0.05, 0.1, 1.0, precision=PSD_MIXED, tol=1e-10, max_iter=5000)
    u = dev(np.full(shape, g.mean()))
    info = S.solve(dev(f), u, dev(g))
    assert info["status"] == 0 and info["outer_iters"] >= 2
    uh = host(u)
    assert abs(uh.mean() - g.mean()) < 1e-13
    r = oracle.residual6(uh, f, g, P)
    assert oracle.norm2(r, h) < 1e-10 * 1.05


@pytest.mark.parametrize("precision", [PSD_MIXED, PSD_FP64])
def test_bench_workload_checked_by_oracle(oracle, precision):
    """The benchmark workload itself (3D 256^3, sixth order, p = 4,
    lambda = 1, s = 0.05, eps = 0.1): the oracle's residual (numpy, its own
    FFT for T_h) at the GPU's answer is below the 1e-10 tolerance, and the
    mean constraint holds."""
    shape = (256, 256, 256)
    wl = synthetic.workload_spfc(shape)
    h = wl["L"] / shape[-1]
    P = oracle.Problem(6, h, wl["p"], wl["s"], wl["eps"], wl["lam"])
    S = Solver(6, shape, h, wl["p"], wl["s"], wl["eps"], wl["lam"], precision=precision, tol=1e-10,
               max_iter=5000, max_outer=30)
    u = dev(wl["u0"])
    info = S.solve(dev(wl["f"]), u, dev(wl["g"]))
    assert info["status"] == 0 and info["res_l2"] < 1e-10
    uh = host(u)
    S.close()
    del u
    torch.cuda.empty_cache()
    assert abs(uh.mean() - wl["g"].mean()) < 1e-13
    r = oracle.residual6(uh, wl["f"], wl["g"], P)
    assert oracle.norm2(r, h) < 1e-10 * 1.05
