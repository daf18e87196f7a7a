"""Pins of the oracle's PSD iteration against results fixed independently of
its code: an exactly solvable linear case (p = 2) with the classical rate
bound of Sec. 2.1, the manufactured-solution protocol of Sec. 6.1.1, dense
Newton brute force built from explicit stencil matrices, the energy-decrease
and positivity results of Sec. 2.3, the exact line search as an energy
minimiser, and conservation of mass."""

import itertools

import numpy as np
import pytest

rng = np.random.default_rng(777)


# ---------------------------------------------------------------- helpers

def _dense_grad(shape, h):
    """Dense matrices of the vertex gradient, assembled entry by entry: the
    a-derivative at vertex v is the mean over the 2^(d-1) a-edges of the
    vertex cube of (u[v + e_a] - u[v]) / h (Sec. 5.1; 3D tensor reading)."""
    dim = len(shape)
    N = int(np.prod(shape))
    mats = []
    for ax in range(dim):
        M = np.zeros((N, N))
        others = [o for o in range(dim) if o != ax]
        c = 1.0 / (h * 2 ** (dim - 1))
        for cell in itertools.product(*[range(n) for n in shape]):
            i = np.ravel_multi_index(cell, shape)
            for bits in itertools.product((0, 1), repeat=dim - 1):
                base = list(cell)
                for o, b in zip(others, bits):
                    base[o] += b
                hi = list(base)
                hi[ax] += 1
                M[i, np.ravel_multi_index(tuple(x % n for x, n in zip(hi, shape)), shape)] += c
                M[i, np.ravel_multi_index(tuple(x % n for x, n in zip(base, shape)), shape)] -= c
        mats.append(M)
    return mats


def _dense_lap(shape, h):
    N = int(np.prod(shape))
    M = np.zeros((N, N))
    for cell in itertools.product(*[range(n) for n in shape]):
        i = np.ravel_multi_index(cell, shape)
        for ax in range(len(shape)):
            for sgn in (1, -1):
                nb = list(cell)
                nb[ax] = (nb[ax] + sgn) % shape[ax]
                M[i, np.ravel_multi_index(tuple(nb), shape)] += 1 / h ** 2
            M[i, i] -= 2 / h ** 2
    return M


class DenseModel:
    """N_h and its Jacobian from dense matrices; the divergence is -G^T
    (summation by parts, pinned in test_oracle_operators)."""

    def __init__(self, shape, h, p, s, eps, lam=0.0, order=4):
        self.G = _dense_grad(shape, h)
        self.L = _dense_lap(shape, h)
        self.p, self.s, self.eps, self.lam, self.order = p, s, eps, lam, order
        self.T = np.linalg.pinv(-self.L)  # -Delta_h^{-1} on mean-zero functions
        self.N = int(np.prod(shape))

    def op(self, u, g=None):
        gr = [G @ u for G in self.G]
        g2 = sum(x * x for x in gr)
        r = g2 ** ((self.p - 2) / 2)
        plap = -sum(G.T @ (r * x) for G, x in zip(self.G, gr))
        base = -self.s * plap + self.s * self.eps ** 2 * (self.L @ (self.L @ u))
        if self.order == 4:
            return u + base
        return self.s * self.lam * u + base + self.T @ (u - g)

    def jac(self, u):
        gr = [G @ u for G in self.G]
        g2 = sum(x * x for x in gr)
        r = g2 ** ((self.p - 2) / 2)
        with np.errstate(divide="ignore", invalid="ignore"):
            q = np.where(g2 > 0, (self.p - 2) * g2 ** ((self.p - 4) / 2), 0.0)
        J = self.s * self.eps ** 2 * self.L @ self.L
        for a_, Ga in enumerate(self.G):
            for b_, Gb in enumerate(self.G):
                w = q * gr[a_] * gr[b_] + (r if a_ == b_ else 0.0)
                J += self.s * Ga.T @ (w[:, None] * Gb)
        if self.order == 4:
            J += np.eye(self.N)
        else:
            J += self.s * self.lam * np.eye(self.N) + self.T
        return J

    def newton(self, f, u0, g=None, iters=40):
        u = u0.ravel().copy()
        fv = f.ravel()
        if self.order == 6:
            # Newton restricted to the mean-zero directions
            Q, _ = np.linalg.qr(np.eye(self.N) - 1.0 / self.N)
            Q = Q[:, : self.N - 1]
        for _ in range(iters):
            res = fv - self.op(u, None if g is None else g.ravel())
            J = self.jac(u)
            if self.order == 4:
                du = np.linalg.solve(J, res)
            else:
                res = res - res.mean()
                du = Q @ np.linalg.solve(Q.T @ J @ Q, Q.T @ res)
            u = u + du
            if np.max(np.abs(du)) < 1e-15 * (1 + np.max(np.abs(u))):
                break
        return u.reshape(u0.shape)


# ---------------------------------------------------------------- tests

def test_dense_model_agrees_with_oracle_operator(oracle):
    """Cross-check of the two independent constructions of N_h."""
    for shape in [(8, 8), (4, 4, 4)]:
        h, p = 0.5, 4.0
        P = oracle.Problem(4, h, p, 0.2, 0.3)
        m = DenseModel(shape, h, p, 0.2, 0.3)
        u = rng.standard_normal(shape)
        np.testing.assert_allclose(oracle.N4(u, P).ravel(), m.op(u.ravel()), atol=1e-10)


@pytest.mark.parametrize("shape,p", [((8, 8), 4.0), ((8, 8), 3.0), ((8, 8, 8), 4.0)])
def test_psd_matches_dense_newton_4th(oracle, shape, p):
    h = 2 * np.pi / shape[0]
    s, eps = 0.05, 0.2
    P = oracle.Problem(4, h, p, s, eps)
    f = rng.standard_normal(shape) * 0.5
    u_psd, info = oracle.psd_solve(P, f, np.zeros(shape), tol=1e-13, kmax=500)
    assert info["res"][-1] < 1e-13
    m = DenseModel(shape, h, p, s, eps)
    u_n = m.newton(f, f.copy())  # start where the vertex gradients are non-zero
    assert np.max(np.abs(u_psd - u_n)) <= 1e-12


@pytest.mark.parametrize("shape", [(8, 8), (8, 8, 8)])
def test_psd_matches_dense_newton_6th(oracle, shape):
    h = 2 * np.pi / shape[0]
    s, eps, lam = 0.05, 0.2, 1.0
    P = oracle.Problem(6, h, 4.0, s, eps, lam)
    f = rng.standard_normal(shape) * 0.5
    g = rng.standard_normal(shape) * 0.5
    u0 = np.full(shape, g.mean())
    u_psd, info = oracle.psd_solve(P, f, u0, g=g, tol=1e-13, kmax=500)
    assert info["res"][-1] < 1e-13
    m = DenseModel(shape, h, 4.0, s, eps, lam, order=6)
    u_n = m.newton(f, u0, g=g)
    assert abs(u_n.mean() - g.mean()) < 1e-14
    assert np.max(np.abs(u_psd - u_n)) <= 1e-12
    # the recovered w solves both equations of the mixed system (Sec. 5.4)
    w = oracle.recover_w(u_psd, f, g, P)
    np.testing.assert_allclose(u_psd - oracle.lap(w, h), g, atol=1e-11)
    lhs = (s * lam * u_psd - s * oracle.plap(u_psd, h, 4.0)
           + s * eps ** 2 * oracle.lap(oracle.lap(u_psd, h), h) - w)
    np.testing.assert_allclose(lhs, f, atol=1e-11)


@pytest.mark.parametrize("shape", [(32, 32), (16, 16, 16)])
def test_p2_exact_solution_and_classical_rate(oracle, shape):
    """p = 2: N_h = I - s Delta_h^v + s eps^2 Delta_h^2 is linear with symbol
    1 + s mu_v + s eps^2 mu^2 (mu_v from the skew-Laplacian symbol); PSD with
    exact line search is Algorithm 1 and contracts the A-norm error by at most
    (kappa - 1)/(kappa + 1) per step (Sec. 2.1)."""
    h = 2 * np.pi / shape[0]
    s, eps = 0.3, 0.2
    P = oracle.Problem(4, h, 2.0, s, eps)
    f = rng.standard_normal(shape)
    grids = np.meshgrid(*[2 * np.pi * np.arange(n) / n for n in shape], indexing="ij")
    if len(shape) == 2:
        mu_v = (2 / h ** 2) * (1 - np.cos(grids[0]) * np.cos(grids[1]))
    else:
        mu_v = 0.0
        for j in range(3):
            t = np.sin(grids[j] / 2) ** 2
            for i in range(3):
                if i != j:
                    t = t * np.cos(grids[i] / 2) ** 2
            mu_v = mu_v + t
        mu_v = mu_v * 4 / h ** 2
    mu = sum((4 / h ** 2) * np.sin(t / 2) ** 2 for t in grids)
    symA = 1 + s * mu_v + s * eps ** 2 * mu ** 2
    symL = 1 + s * mu + s * eps ** 2 * mu ** 2
    u_star = np.real(np.fft.ifftn(np.fft.fftn(f) / symA))
    kappa = np.max(symA / symL) / np.min(symA / symL)
    bound = (kappa - 1) / (kappa + 1)
    u, info = oracle.psd_solve(P, f, np.zeros(shape), tol=1e-12, kmax=500, record=True)
    assert np.max(np.abs(u - u_star)) < 1e-12
    errs = []
    for uk in info["u"]:
        e = uk - u_star
        errs.append(np.sqrt(np.sum(np.real(np.fft.ifftn(symA * np.fft.fftn(e))) * e)))
    for k in range(len(errs) - 1):
        if errs[k] > 1e-9:
            assert errs[k + 1] <= bound * errs[k] * (1 + 1e-9)


def test_manufactured_solution_protocol(oracle):
    """Sec. 6.1.1: f := N_h[I_h u~] with u~ = sin(2 pi x) cos(2 pi y) cos(s)/(2 pi)
    on (0,1)^2; PSD from u0 = u~(.,.,0) + s^2 sin(4 pi x) sin(6 pi y) recovers
    I_h u~ (the paper stops at 1e-8 in the max norm; we go to 1e-11)."""
    n, s, eps, p = 32, 0.01, 0.03, 4.0
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Y, X = np.meshgrid(x, x, indexing="ij")
    ut = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) * np.cos(s) / (2 * np.pi)
    P = oracle.Problem(4, h, p, s, eps)
    f = oracle.N4(ut, P)
    u0 = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) / (2 * np.pi) + s * s * np.sin(4 * np.pi * X) * np.sin(6 * np.pi * Y)
    u, info = oracle.psd_solve(P, f, u0, tol=1e-12, kmax=2000)
    assert np.max(np.abs(u - ut)) < 1e-11


@pytest.mark.parametrize("order", [4, 6])
def test_energy_decrease_positive_alpha_and_contraction(oracle, order):
    """Prop. "energy-decrease": E_h[u^{k+1}] <= E_h[u^k] and alpha_k > 0;
    Theorem "generic-convergence": E_h[u^k] - E_h[u] decays geometrically."""
    shape = (32, 32)
    h = 2 * np.pi / 32
    P = oracle.Problem(order, h, 4.0, 0.1, 0.1, lam=1.0)
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape) if order == 6 else None
    u0 = np.zeros(shape) if order == 4 else np.full(shape, g.mean())
    u, info = oracle.psd_solve(P, f, u0, g=g, tol=1e-11, kmax=500, record=True)
    E = np.array(info["energy"])
    assert np.all(np.diff(E) <= 4e-16 * np.abs(E[1:]) * 8)
    assert all(al > 0 for al in info["alpha"])
    Einf = E[-1]
    gaps = E[:-1] - Einf
    good = gaps[1:] > 1e-8 * gaps[0]
    ratios = gaps[1:][good] / gaps[:-1][good]
    assert len(ratios) >= 3 and np.all(ratios < 1.0)
    if order == 6:
        for uk in info["u"]:
            assert abs(uk.mean() - g.mean()) < 1e-13
    else:
        # mass: (u - f, 1)_2 = 0 at the solution (Sec. 3.2)
        assert abs(u.mean() - f.mean()) < 1e-11


@pytest.mark.parametrize("p", [3.0, 4.0, 6.0])
def test_line_search_minimises_energy(oracle, p):
    """alpha_k = argmin_alpha E_h[u + alpha d] (Eq. "eqn-search"), checked by
    golden-section search on the plain energy sum; alpha > 0."""
    shape = (16, 16)
    h = 2 * np.pi / 16
    P = oracle.Problem(4, h, p, 0.1, 0.1)
    f = rng.standard_normal(shape)
    u = rng.standard_normal(shape) * 0.3
    r = oracle.residual4(u, f, P)
    d = oracle.precond4(r, P)
    q = lambda al: oracle.ip2(oracle.N4(u + al * d, P) - f, d, h)
    dq = lambda al: oracle.second_variation4(u + al * d, d, P)
    alpha = oracle.line_search(q, dq, oracle.ip2(r, d, h) / dq(0.0))
    assert alpha > 0
    E = lambda al: oracle.energy4(u + al * d, f, P)
    lo, hi = 0.0, 4 * alpha
    gr = (np.sqrt(5) - 1) / 2
    for _ in range(200):
        m1, m2 = hi - gr * (hi - lo), lo + gr * (hi - lo)
        if E(m1) < E(m2):
            hi = m2
        else:
            lo = m1
    assert abs(0.5 * (lo + hi) - alpha) <= 1e-7 * alpha
    if p == 4.0:
        # q is a cubic for p = 4 (Sec. 6.1): 4th differences vanish
        vals = [q(k * 0.3 * alpha) for k in range(5)]
        d4 = vals[4] - 4 * vals[3] + 6 * vals[2] - 4 * vals[1] + vals[0]
        assert abs(d4) <= 1e-10 * max(abs(v) for v in vals)


@pytest.mark.parametrize("shape", [(16, 32), (8, 8, 16)])
def test_preconditioner_inverts_stencil_operator(oracle, shape):
    h, s, eps, lam = 0.2, 0.1, 0.3, 0.5
    P4 = oracle.Problem(4, h, 4.0, s, eps)
    r = rng.standard_normal(shape)
    dd = oracle.precond4(r, P4)
    Ld = dd - s * oracle.lap(dd, h) + s * eps ** 2 * oracle.lap(oracle.lap(dd, h), h)
    np.testing.assert_allclose(Ld, r, atol=1e-11)
    P6 = oracle.Problem(6, h, 4.0, s, eps, lam)
    d6 = oracle.precond6(r, P6)
    assert abs(d6.mean()) < 1e-14
    Ld6 = (s * lam * d6 - s * oracle.lap(d6, h) + s * eps ** 2 * oracle.lap(oracle.lap(d6, h), h)
           + oracle.T_h(d6, h))
    np.testing.assert_allclose(Ld6, r - r.mean(), atol=1e-11)


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("p", [2.0, 4.0, 6.0])
@pytest.mark.parametrize("shape", [(16, 16), (8, 8, 8)])
def test_line_search_polynomial(oracle, order, p, shape):
    """q(alpha) = (N_h[u + alpha d] - f, d)_2 is a polynomial of degree p - 1
    for even p (Sec. 6.1: a cubic for p = 4, a quintic for p = 6); the
    oracle's coefficients reproduce the literal q at seven step sizes, and a
    perturbed coefficient would not."""
    h = 0.3
    P = oracle.Problem(order, h, p, 0.1, 0.4, 0.7)
    u = 0.5 * rng.standard_normal(shape)
    d = 0.5 * rng.standard_normal(shape)
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape) if order == 6 else None

    def q(al):
        v = u + al * d
        nv = oracle.N4(v, P) if order == 4 else oracle.N6(v, g, P)
        return oracle.ip2(nv - f, d, h)

    c = oracle.line_search_poly(u, d, f, P, g)
    assert len(c) == int(p)
    alphas = (-1.3, -0.4, 0.0, 0.2, 0.7, 1.5, 2.2)
    qs = [q(al) for al in alphas]
    scale = max(abs(x) for x in qs)
    for al, qa in zip(alphas, qs):
        assert abs(sum(ck * al ** k for k, ck in enumerate(c)) - qa) <= 1e-12 * scale
    # the top coefficient is s <|b|^p> > 0 and matters at these step sizes
    assert c[-1] > 0 and abs(c[-1]) * 2.2 ** (len(c) - 1) > 1e-6 * scale
