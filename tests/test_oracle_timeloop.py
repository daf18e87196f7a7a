"""Pins of the oracle's thin-film time loop (Sec. 6.1, convex splitting),
each independent of the loop's own code:

* linear regime: for a small single Fourier mode the p-term is cubic in the
  amplitude, so each step multiplies the mode by the closed-form factor
  (1 + s mu_v) / (1 + s eps^2 mu^2), mu the symbol of -Delta_h and mu_v that
  of the skew Laplacian -Delta_h^v (2D: (2/h^2)(1 - cos t_x cos t_y); 3D:
  (4/h^2) sum_j sin^2(t_j/2) prod_{i != j} cos^2(t_i/2)).  Swapping Delta_h^v
  for Delta_h, a sign, or the eps^2 factor changes the factor at the chosen
  wave numbers by far more than the tolerance;
* mass: every step preserves sum u (the right-hand side and N_h - I are
  sums of differences);
* energy: convex splitting never increases the discrete energy
  h^d sum_v (1/p |grad u|^p - 1/2 |grad u|^2) + eps^2/2 ||Delta_h u||^2,
  whatever the step s (checked at s = 0.1 h^2 and at s = 10 h^2);
* the initial data of Eq. "init1" on (0, 3.2)^2 is sampled at cell centres.
"""

import numpy as np
import pytest


def _mode(shape, h, k, amp):
    axes = [(np.arange(n) + 0.5) * h for n in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    # array axis a is spatial axis a (any assignment works for a cosine mode)
    phase = sum((2 * np.pi * kk / (n * h)) * g for kk, n, g in zip(k, shape, grids))
    return amp * np.cos(phase)


def _factor(shape, h, k, s, eps):
    t = [2 * np.pi * kk / n for kk, n in zip(k, shape)]
    mu = sum((4 / h ** 2) * np.sin(tt / 2) ** 2 for tt in t)
    if len(shape) == 2:
        mu_v = (2 / h ** 2) * (1 - np.cos(t[0]) * np.cos(t[1]))
    else:
        mu_v = 0.0
        for j in range(3):
            prod = 1.0
            for i in range(3):
                if i != j:
                    prod *= np.cos(t[i] / 2) ** 2
            mu_v += (4 / h ** 2) * np.sin(t[j] / 2) ** 2 * prod
    return (1 + s * mu_v) / (1 + s * eps ** 2 * mu ** 2)


@pytest.mark.parametrize("shape,k", [((16, 16), (3, 2)), ((16, 32), (1, 5)), ((8, 8, 16), (1, 2, 3))])
def test_linear_regime_matches_closed_form(oracle, shape, k):
    h = 0.2
    s, eps = 0.3 * h ** 2, 0.1
    P = oracle.Problem(4, h, 4.0, s, eps)
    u0 = _mode(shape, h, k, 1e-6)
    u, _ = oracle.thinfilm_steps(P, u0, 3, tol=1e-20, kmax=60)
    g = _factor(shape, h, k, s, eps)
    assert np.max(np.abs(u - g ** 3 * u0)) <= 1e-8 * np.max(np.abs(u0))
    # the factor differs from the one with Delta_h in place of Delta_h^v
    t = [2 * np.pi * kk / n for kk, n in zip(k, shape)]
    mu = sum((4 / h ** 2) * np.sin(tt / 2) ** 2 for tt in t)
    assert abs(g - (1 + s * mu) / (1 + s * eps ** 2 * mu ** 2)) > 1e-3


def _init1(n):
    L = 3.2
    h = L / n
    x = (np.arange(n) + 0.5) * h
    y = x[:, None]
    return (0.1 * np.sin(2 * np.pi * x / L) ** 2 * np.sin(4 * np.pi * (y - 1.4) / L)
            - 0.1 * np.cos(2 * np.pi * (x - 2.0) / L) * np.sin(2 * np.pi * y / L)), h


@pytest.mark.parametrize("p,s_over_h2", [(4.0, 0.1), (4.0, 10.0), (6.0, 0.1)])
def test_mass_and_energy(oracle, p, s_over_h2):
    u, h = _init1(16)
    P = oracle.Problem(4, h, p, s_over_h2 * h * h, 0.1)
    m0 = float(np.sum(u))
    e = [oracle.thinfilm_energy(u, P)]
    for _ in range(12):
        u, _ = oracle.thinfilm_steps(P, u, 1, tol=1e-12)
        e.append(oracle.thinfilm_energy(u, P))
        assert abs(float(np.sum(u)) - m0) <= 1e-11 * max(1.0, abs(m0)) + 1e-11 * np.sum(np.abs(u))
    de = np.diff(e)
    assert np.all(de <= 1e-12 * np.max(np.abs(e))), de
    assert e[-1] < e[0]


def test_init1_sampling():
    u, h = _init1(32)
    assert h == pytest.approx(0.1)
    # value at the first cell centre (0.05, 0.05), from the formula by hand
    x = y = 0.05
    ref = (0.1 * np.sin(2 * np.pi * x / 3.2) ** 2 * np.sin(4 * np.pi * (y - 1.4) / 3.2)
           - 0.1 * np.cos(2 * np.pi * (x - 2.0) / 3.2) * np.sin(2 * np.pi * y / 3.2))
    assert u[0, 0] == pytest.approx(ref, rel=1e-15)


# ------------------------------------------------------------------ SPFC
# Sec. 6.2: order 6 with lambda = gamma_0, g = u^n, f = -s gamma_1 Delta_h u^n.
# A small mode on a constant background is multiplied per step by
# (1 + s gamma_1 mu^2) / (1 + s gamma_0 mu + s eps^2 mu^3) (the T_h term
# contributes 1/mu times the difference to the previous step); the mean of u
# is that of g = u^n, so it never changes.

def _spfc_factor(shape, h, k, s, eps, g0, g1):
    t = [2 * np.pi * kk / n for kk, n in zip(k, shape)]
    mu = sum((4 / h ** 2) * np.sin(tt / 2) ** 2 for tt in t)
    return (1 + s * g1 * mu ** 2) / (1 + s * g0 * mu + s * eps ** 2 * mu ** 3)


@pytest.mark.parametrize("shape,k", [((16, 16), (3, 2)), ((8, 8, 16), (1, 2, 3))])
def test_spfc_linear_regime_matches_closed_form(oracle, shape, k):
    h, s, eps, g0, g1 = 1.25, 0.5, 1.0, 0.5, 2.0
    P = oracle.Problem(6, h, 4.0, s, eps, g0)
    u0 = 0.3 + _mode(shape, h, k, 1e-6)
    u, _ = oracle.spfc_steps(P, u0, g1, 3, tol=1e-14, kmax=80)
    G = _spfc_factor(shape, h, k, s, eps, g0, g1)
    assert abs(G - 1.0) > 0.05
    assert np.max(np.abs(u - (0.3 + G ** 3 * (u0 - 0.3)))) <= 1e-8 * 1e-6
    # a missing s on the right-hand side (the printed Sec. 6.2 form) gives another factor
    t = [2 * np.pi * kk / n for kk, n in zip(k, shape)]
    mu = sum((4 / h ** 2) * np.sin(tt / 2) ** 2 for tt in t)
    assert abs(G - (1 + g1 * mu ** 2) / (1 + s * g0 * mu + s * eps ** 2 * mu ** 3)) > 0.05


@pytest.mark.parametrize("s", [0.01, 1.0])
def test_spfc_mass_and_energy(oracle, s):
    rng = np.random.default_rng(5)
    n, L = 16, 20.0
    h = L / n
    u = 0.2 + 0.05 * (2 * rng.random((n, n)) - 1)  # the shape of Eq. "init2" around a mean
    P = oracle.Problem(6, h, 4.0, s, 1.0, 0.5)
    m0 = float(u.mean())
    e = [oracle.spfc_energy(u, P, 2.0)]
    for _ in range(8):
        u, _ = oracle.spfc_steps(P, u, 2.0, 1, tol=1e-12)
        e.append(oracle.spfc_energy(u, P, 2.0))
        assert abs(float(u.mean()) - m0) <= 1e-13
    de = np.diff(e)
    assert np.all(de <= 1e-12 * np.max(np.abs(e))), de
    assert e[-1] < e[0]


# ------------------------------------------------ adjoint through the loop

def test_thinfilm_adjoint_matches_finite_differences(oracle):
    """dJ/du^0 and dJ/ds of J = 1/2 |u^N - target|^2 through 3 thin-film
    steps against central differences of J (step 1e-5, solves to 1e-14):
    both agree to about 1e-9; leaving out the right-hand side's dependence
    on s (the -Delta_h^v u^n term) changes dJ/ds by far more."""
    rng = np.random.default_rng(1)
    n, h, s, eps, N = 8, 0.4, 0.05, 0.3, 3
    P = oracle.Problem(4, h, 4.0, s, eps)
    u0 = 0.3 * rng.standard_normal((n, n))
    tgt = 0.2 * rng.standard_normal((n, n))
    v = rng.standard_normal((n, n))

    def J(u_init, s_=s):
        u, _ = oracle.thinfilm_steps(oracle.Problem(4, h, 4.0, s_, eps), u_init, N, tol=1e-14, kmax=3000)
        return 0.5 * float(np.sum((u - tgt) ** 2)), u

    _, uN = J(u0)
    gu, gs = oracle.thinfilm_adjoint(P, u0, N, uN - tgt, tol=1e-14)
    e = 1e-5
    fd_u = (J(u0 + e * v)[0] - J(u0 - e * v)[0]) / (2 * e)
    fd_s = (J(u0, s * (1 + e))[0] - J(u0, s * (1 - e))[0]) / (2 * e * s)
    assert abs(float(np.sum(gu * v)) - fd_u) <= 1e-7 * abs(fd_u)
    assert abs(gs - fd_s) <= 1e-7 * abs(fd_s)
    # the s-dependence of the right-hand side matters
    us = [u0]
    for _ in range(N):
        us.append(oracle.thinfilm_steps(P, us[-1], 1, tol=1e-14, kmax=3000)[0])
    lam, rhs_part = uN - tgt, 0.0
    for k in reversed(range(N)):
        mu, _, _ = oracle.adjoint4(us[k + 1], lam, P, tol=1e-14)
        rhs_part -= float(np.sum(mu * oracle.skew_lap(us[k], h)))
        lam = mu - s * oracle.skew_lap(mu, h)
    assert abs(rhs_part) > 1e-3 * abs(fd_s)
