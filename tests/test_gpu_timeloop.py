"""The thin-film convex-splitting time loop (Sec. 6.1) through
psd_thinfilm_steps against the oracle's loop (thinfilm_steps), element by
element after the same number of steps: the initial data of Eq. "init1" on
(0, 3.2)^2 with s = 0.1 h^2 and eps = 0.1 (the parameters printed with
Table 1), p = 4 and 6, FP64 and mixed precision; and a smooth 3D field.
Every solve stops at ||r||_2 < 1e-12 on both sides, and the slow growth of
the unstable modes over a few dozen steps keeps the difference near 1e-10
of |u|."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01475_gb300 import PSD_FP64, PSD_MIXED, PSDError, Solver, synthetic  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _init1(n):
    return synthetic.thin_film_init1(n)


@pytest.mark.parametrize("n,p,nsteps", [(16, 4.0, 20), (32, 4.0, 40), (32, 6.0, 20)])
@pytest.mark.parametrize("precision", [PSD_FP64, PSD_MIXED])
def test_thinfilm_steps_match_oracle(oracle, n, p, nsteps, precision):
    u0, h = _init1(n)
    s, eps = 0.1 * h * h, 0.1
    P = oracle.Problem(4, h, p, s, eps)
    ref, _ = oracle.thinfilm_steps(P, u0, nsteps, tol=1e-12)
    S = Solver(4, (n, n), h, p, s, eps, precision=precision, tol=1e-12)
    u = dev(u0)
    info = S.thinfilm_steps(u, nsteps)
    got = u.cpu().numpy()
    assert info["status"] == 0 and info["res_l2"] < 1e-12
    assert info["iters"] >= nsteps and info["wall_ms"] > 0
    assert rel(got, ref) <= 1e-8
    assert abs(got.sum() - u0.sum()) <= 1e-10 * np.abs(u0).sum()


def test_thinfilm_steps_3d(oracle):
    shape = (16, 16, 32)
    h = 2 * np.pi / 32
    u0 = 0.05 * synthetic.fourier_field(shape, 2 * np.pi, 4, 77, nmodes=16)
    s, eps = 0.1 * h * h, 0.1
    P = oracle.Problem(4, h, 4.0, s, eps)
    ref, _ = oracle.thinfilm_steps(P, u0, 6, tol=1e-12)
    S = Solver(4, shape, h, 4.0, s, eps, precision=PSD_MIXED, tol=1e-12)
    u = dev(u0)
    info = S.thinfilm_steps(u, 6)
    assert info["status"] == 0
    assert rel(u.cpu().numpy(), ref) <= 1e-8


def test_thinfilm_steps_arguments():
    u0, h = _init1(16)
    S = Solver(4, (16, 16), h, 4.0, 0.1 * h * h, 0.1)
    u = dev(u0)
    info = S.thinfilm_steps(u, 0)
    assert info["iters"] == 0 and np.array_equal(u.cpu().numpy(), u0)
    with pytest.raises(PSDError):
        S.thinfilm_steps(u, -1)
    S6 = Solver(6, (16, 16), h, 4.0, 0.1, 0.1, 1.0)
    with pytest.raises(PSDError):
        S6.thinfilm_steps(u, 1)


# ------------------------------------------------------------------ SPFC

@pytest.mark.parametrize("shape,nsteps", [((32, 32), 10), ((16, 16, 16), 4)])
@pytest.mark.parametrize("precision", [PSD_FP64, PSD_MIXED])
def test_spfc_steps_match_oracle(oracle, shape, nsteps, precision):
    """SPFC steps (Sec. 6.2: eps = 1, gamma_0 = lambda = 0.5, gamma_1 = 2)
    from random data of the shape of Eq. "init2" around a mean, against the
    oracle's loop; the mean of u is kept."""
    rng = np.random.default_rng(9)
    L = 20.0
    h = L / shape[-1]
    s, eps, g0, g1 = 0.1, 1.0, 0.5, 2.0
    u0 = 0.2 + 0.05 * (2 * rng.random(shape) - 1)
    P = oracle.Problem(6, h, 4.0, s, eps, g0)
    ref, _ = oracle.spfc_steps(P, u0, g1, nsteps, tol=1e-12)
    S = Solver(6, shape, h, 4.0, s, eps, g0, precision=precision, tol=1e-12)
    u = dev(u0)
    info = S.spfc_steps(u, g1, nsteps)
    got = u.cpu().numpy()
    assert info["status"] == 0
    assert rel(got - u0.mean(), ref - u0.mean()) <= 1e-8
    assert abs(got.mean() - u0.mean()) <= 1e-13


def test_spfc_steps_arguments():
    S4 = Solver(4, (16, 16), 0.1, 4.0, 0.1, 0.1)
    u = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(PSDError):
        S4.spfc_steps(u, 2.0, 1)
    S6 = Solver(6, (16, 16), 0.5, 4.0, 0.1, 1.0, 0.5)
    with pytest.raises(PSDError):
        S6.spfc_steps(u, -1.0, 1)
    assert S6.spfc_steps(u, 2.0, 0)["iters"] == 0


# -------------------------------------------------- adjoint through the loop

@pytest.mark.parametrize("checkpoints", [0, 1, 2, 6])
def test_thinfilm_adjoint_matches_oracle(oracle, checkpoints):
    """dJ/du^0 and dJ/ds through 6 thin-film steps (J = 1/2 |u^N - target|^2)
    against the oracle's backward recursion (itself pinned by finite
    differences); the checkpoint count changes only the recomputation, so
    every setting gives the same bits."""
    rng = np.random.default_rng(4)
    n, h, s, eps, N = 16, 0.4, 0.05, 0.3, 6
    P = oracle.Problem(4, h, 4.0, s, eps)
    u0 = 0.3 * rng.standard_normal((n, n))
    tgt = 0.2 * rng.standard_normal((n, n))
    uN, _ = oracle.thinfilm_steps(P, u0, N, tol=1e-13)
    ref_u, ref_s = oracle.thinfilm_adjoint(P, u0, N, uN - tgt, tol=1e-13)
    S = Solver(4, (n, n), h, 4.0, s, eps, tol=1e-13)
    u = dev(u0)
    S.thinfilm_steps(u, N)
    gu0 = torch.empty_like(u)
    gs, info = S.thinfilm_adjoint(dev(u0), N, u - dev(tgt), gu0, checkpoints=checkpoints, tol_rel=1e-13)
    assert info["status"] == 0 and info["iters"] > 0
    assert rel(gu0.cpu().numpy(), ref_u) <= 1e-8
    assert abs(gs - ref_s) <= 1e-8 * abs(ref_s)
    if checkpoints == 6:
        g2 = torch.empty_like(u)
        gs2, _ = S.thinfilm_adjoint(dev(u0), N, u - dev(tgt), g2, checkpoints=1, tol_rel=1e-13)
        assert torch.equal(g2, gu0) and gs2 == gs


def test_thinfilm_adjoint_zero_steps_is_identity():
    S = Solver(4, (16, 16), 0.4, 4.0, 0.05, 0.3)
    g = torch.randn((16, 16), dtype=torch.float64, device="cuda")
    out = torch.empty_like(g)
    gs, _ = S.thinfilm_adjoint(torch.zeros_like(g), 0, g, out)
    assert torch.equal(out, g) and gs == 0.0
