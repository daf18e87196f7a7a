"""Pins of the oracle's adjoint: the Hessian-vector product against central
differences of N_h, the adjoint solve against a dense solve built from the
explicit stencil matrices, and the end-to-end gradients against central
finite differences of the loss through the oracle's own PSD solve."""

import numpy as np
import pytest

from test_oracle_solver import DenseModel

rng = np.random.default_rng(4242)


@pytest.mark.parametrize("shape,p", [((16, 16), 4.0), ((8, 8, 8), 4.0), ((16, 16), 3.0)])
def test_hvp_is_the_derivative_of_N(oracle, shape, p):
    P = oracle.Problem(4, 2 * np.pi / shape[-1], p, 0.07, 0.2)
    u = rng.standard_normal(shape) * 0.5
    v = rng.standard_normal(shape)
    t = 1e-6
    fd = (oracle.N4(u + t * v, P) - oracle.N4(u - t * v, P)) / (2 * t)
    hv = oracle.hvp4(u, v, P)
    assert np.max(np.abs(fd - hv)) <= 1e-6 * np.max(np.abs(hv))
    # symmetry (x, H y) = (H x, y)
    x = rng.standard_normal(shape)
    assert abs(np.sum(x * hv) - np.sum(oracle.hvp4(u, x, P) * v)) <= 1e-10 * np.sum(np.abs(x * hv))


def test_adjoint_matches_dense_solve(oracle):
    shape = (8, 8)
    h = 2 * np.pi / 8
    P = oracle.Problem(4, h, 4.0, 0.05, 0.2)
    u = rng.standard_normal(shape) * 0.5
    gu = rng.standard_normal(shape)
    lam, gs, it = oracle.adjoint4(u, gu, P)
    J = DenseModel(shape, h, 4.0, 0.05, 0.2).jac(u.ravel())
    lam_dense = np.linalg.solve(J, gu.ravel()).reshape(shape)
    assert np.max(np.abs(lam - lam_dense)) <= 1e-11 * np.max(np.abs(lam_dense))


@pytest.mark.parametrize("shape", [(16, 16), (8, 8, 8)])
def test_adjoint_gradients_match_finite_differences(oracle, shape):
    """J(u) = 1/2 h^d sum (u - u_t)^2 with u the PSD solution for (f, s):
    dJ/df . v and dJ/ds against central differences of J (forward solves to
    the FP64 floor)."""
    h = 2 * np.pi / shape[-1]
    s, eps = 0.05, 0.2
    f = rng.standard_normal(shape) * 0.5
    ut = rng.standard_normal(shape) * 0.2
    hd = h ** len(shape)

    def solve(ff, ss):
        P = oracle.Problem(4, h, 4.0, ss, eps)
        u, _ = oracle.psd_solve(P, ff, np.zeros(shape), tol=1e-14, kmax=3000)
        return u

    def J(u):
        return 0.5 * hd * float(np.sum((u - ut) ** 2))

    u = solve(f, s)
    P = oracle.Problem(4, h, 4.0, s, eps)
    gf, gs, _ = oracle.adjoint4(u, hd * (u - ut), P)
    t = 1e-6
    for _ in range(2):
        v = rng.standard_normal(shape)
        fd = (J(solve(f + t * v, s)) - J(solve(f - t * v, s))) / (2 * t)
        an = float(np.sum(gf * v))
        assert abs(fd - an) <= 1e-5 * (abs(an) + 1e-12)
    fds = (J(solve(f, s + t)) - J(solve(f, s - t))) / (2 * t)
    assert abs(fds - gs) <= 1e-5 * abs(gs)
