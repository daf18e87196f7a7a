"""Pins of the oracle's grid operators and FFT against facts the paper and the
mathematics fix independently of the oracle's code:

* the FFT against the DFT definition (direct O(n^2) sum) and a library FFT;
* every difference operator against dense matrices assembled entry by entry
  from the explicit stencils printed in Sec. 5.1;
* discrete Fourier symbols (the appendix's w_l = -2 i sin(l pi h/L)/h and the
  skew-Laplacian symbol implied by its stencil);
* summation by parts (frak{d} = -frak{D}^T), the gradient identity
  delta E_h[u](xi) = (N_h[u] - f, xi)_2 by central differences of the plain
  energy sum, and the second variation by second differences;
* second-order consistency with the continuous operator (sympy);
* lattice symmetries.
"""

import itertools

import numpy as np
import pytest

rng = np.random.default_rng(12345)


# ---------------------------------------------------------------- FFT

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64])
def test_fft_matches_dft_definition(oracle, n):
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(j, j) / n)
    np.testing.assert_allclose(oracle.fft_axis(x, 0), F @ x, rtol=0, atol=1e-12 * max(1, n))
    Finv = np.exp(2j * np.pi * np.outer(j, j) / n) / n
    np.testing.assert_allclose(oracle.fft_axis(x, 0, inverse=True), Finv @ x, atol=1e-13 * max(1, n))


@pytest.mark.parametrize("shape", [(8, 16), (4, 8, 16), (32, 32)])
def test_fftn_matches_library_and_roundtrip(oracle, shape):
    x = rng.standard_normal(shape)
    np.testing.assert_allclose(oracle.fftn(x), np.fft.fftn(x), atol=1e-11)
    np.testing.assert_allclose(np.real(oracle.ifftn(oracle.fftn(x))), x, atol=1e-14)


def test_fft_rejects_non_power_of_two(oracle):
    with pytest.raises(ValueError):
        oracle.fft_axis(np.ones(6), 0)


# ------------------------------------------- dense operators from Sec. 5.1

def _idx(shape, cell):
    return np.ravel_multi_index(tuple(c % n for c, n in zip(cell, shape)), shape)


def _dense_from_stencil(shape, stencil):
    """Matrix M with (M u)[i] = sum_{(offset, c)} c u[i + offset] (periodic)."""
    N = int(np.prod(shape))
    M = np.zeros((N, N))
    for cell in itertools.product(*[range(n) for n in shape]):
        i = _idx(shape, cell)
        for off, c in stencil:
            M[i, _idx(shape, tuple(ci + oi for ci, oi in zip(cell, off)))] += c
    return M


def _vertex_grad_stencils_2d(h):
    """Explicit formulas of Sec. 5.1 in (y, x) array order; vertex (i+1/2,
    j+1/2) stored at array (j, i):
    frak{D}_x = (u_{i+1,j+1} - u_{i,j+1} + u_{i+1,j} - u_{i,j}) / 2h
    frak{D}_y = (u_{i+1,j+1} - u_{i+1,j} + u_{i,j+1} - u_{i,j}) / 2h"""
    c = 1.0 / (2 * h)
    Dx = [((1, 1), c), ((1, 0), -c), ((0, 1), c), ((0, 0), -c)]
    Dy = [((1, 1), c), ((0, 1), -c), ((1, 0), c), ((0, 0), -c)]
    return Dy, Dx


def _vertex_div_stencils_2d(h):
    """frak{d}_x v_{ij} = (v_{i+1/2,j+1/2} - v_{i-1/2,j+1/2} + v_{i+1/2,j-1/2}
    - v_{i-1/2,j-1/2}) / 2h; vertex (i+1/2, j+1/2) at array (j, i), so
    (i-1/2, j+1/2) is array offset (0, -1) etc.  frak{d}_y likewise."""
    c = 1.0 / (2 * h)
    dx = [((0, 0), c), ((0, -1), -c), ((-1, 0), c), ((-1, -1), -c)]
    dy = [((0, 0), c), ((-1, 0), -c), ((0, -1), c), ((-1, -1), -c)]
    return dy, dx


def _apply(M, u):
    return (M @ u.ravel()).reshape(u.shape)


def test_vertex_gradient_and_divergence_2d_match_printed_stencils(oracle):
    shape, h = (8, 8), 0.37
    u = rng.standard_normal(shape)
    for ax, st in enumerate(_vertex_grad_stencils_2d(h)):
        np.testing.assert_allclose(oracle.vgrad(u, h)[ax],
                                   _apply(_dense_from_stencil(shape, st), u), atol=1e-13)
    w = [rng.standard_normal(shape) for _ in range(2)]
    dy, dx = _vertex_div_stencils_2d(h)
    ref = _apply(_dense_from_stencil(shape, dy), w[0]) + _apply(_dense_from_stencil(shape, dx), w[1])
    np.testing.assert_allclose(oracle.vdiv(w, h), ref, atol=1e-13)


def test_laplacian_and_skew_laplacian_2d_match_printed_stencils(oracle):
    shape, h = (8, 8), 0.21
    u = rng.standard_normal(shape)
    c = 1.0 / h ** 2
    five = [((0, 1), c), ((0, -1), c), ((1, 0), c), ((-1, 0), c), ((0, 0), -4 * c)]
    np.testing.assert_allclose(oracle.lap(u, h), _apply(_dense_from_stencil(shape, five), u), atol=1e-11)
    # skew Laplacian (Sec. 5.1): (u_{i+1,j+1}+u_{i-1,j+1}+u_{i+1,j-1}+u_{i-1,j-1}-4u_ij)/(2h^2)
    c2 = 1.0 / (2 * h ** 2)
    skew = [((1, 1), c2), ((1, -1), c2), ((-1, 1), c2), ((-1, -1), c2), ((0, 0), -4 * c2)]
    np.testing.assert_allclose(oracle.skew_lap(u, h), _apply(_dense_from_stencil(shape, skew), u), atol=1e-11)
    # p = 2: the discrete p-Laplacian is the skew Laplacian (Sec. 5.1)
    np.testing.assert_allclose(oracle.plap(u, h, 2.0), oracle.skew_lap(u, h), atol=1e-11)


def test_vertex_gradient_3d_tensor_reading(oracle):
    """3D reading: frak{D}_x at vertex (i+1/2,j+1/2,k+1/2) is the mean over the
    four x-edges of the vertex cube of (u_{i+1,.,.} - u_{i,.,.})/h."""
    shape, h = (4, 8, 8), 0.5
    u = rng.standard_normal(shape)
    c = 1.0 / (4 * h)
    stx = []
    for b, e in itertools.product((0, 1), repeat=2):
        stx += [((e, b, 1), c), ((e, b, 0), -c)]
    sty = []
    for b, e in itertools.product((0, 1), repeat=2):
        sty += [((e, 1, b), c), ((e, 0, b), -c)]
    stz = []
    for b, e in itertools.product((0, 1), repeat=2):
        stz += [((1, e, b), c), ((0, e, b), -c)]
    g = oracle.vgrad(u, h)
    for ax, st in zip(range(3), [stz, sty, stx]):
        np.testing.assert_allclose(g[ax], _apply(_dense_from_stencil(shape, st), u), atol=1e-13)
    seven = [((0, 0, 1), 1), ((0, 0, -1), 1), ((0, 1, 0), 1), ((0, -1, 0), 1),
             ((1, 0, 0), 1), ((-1, 0, 0), 1), ((0, 0, 0), -6)]
    seven = [(o, cc / h ** 2) for o, cc in seven]
    np.testing.assert_allclose(oracle.lap(u, h), _apply(_dense_from_stencil(shape, seven), u), atol=1e-12)


@pytest.mark.parametrize("shape", [(8, 8), (4, 4, 8)])
def test_summation_by_parts(oracle, shape):
    """(frak{d}.w, xi)_2 = -<w, frak{D} xi> for all w, xi (Sec. 5.1-5.3)."""
    h = 0.3
    xi = rng.standard_normal(shape)
    w = [rng.standard_normal(shape) for _ in shape]
    lhs = oracle.ip2(oracle.vdiv(w, h), xi, h)
    g = oracle.vgrad(xi, h)
    rhs = -sum(oracle.ipv(wa, ga, h) for wa, ga in zip(w, g))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_biharmonic_coefficients(oracle):
    """Delta_h^2 stencil: 2D centre 20, axis +-1 -8, diagonals 2, axis +-2 1;
    3D centre 42, axis +-1 -12, edge diagonals 2, axis +-2 1 (all / h^4);
    coefficients sum to zero."""
    h = 1.0
    e = np.zeros((8, 8)); e[4, 4] = 1
    b = oracle.lap(oracle.lap(e, h), h)
    assert b[4, 4] == 20 and b[4, 5] == -8 and b[5, 5] == 2 and b[4, 6] == 1
    assert abs(b.sum()) < 1e-12 and np.count_nonzero(b) == 13
    e = np.zeros((8, 8, 8)); e[4, 4, 4] = 1
    b = oracle.lap(oracle.lap(e, h), h)
    assert b[4, 4, 4] == 42 and b[4, 4, 5] == -12 and b[4, 5, 5] == 2 and b[6, 4, 4] == 1
    assert abs(b.sum()) < 1e-12 and np.count_nonzero(b) == 25


# ---------------------------------------------------------------- symbols

@pytest.mark.parametrize("shape", [(16, 8), (8, 4, 16)])
def test_fourier_symbols(oracle, shape):
    """Mode e^{i theta.x}: Delta_h -> -sum (4/h^2) sin^2(theta/2) (|w_l|^2 of
    the appendix); 2D skew Laplacian -> -(2/h^2)(1 - cos th_x cos th_y);
    3D -> -(4/h^2) sum_j sin^2(th_j/2) prod_{i!=j} cos^2(th_i/2)."""
    h = 0.25
    for trial in range(5):
        k = [int(rng.integers(0, n)) for n in shape]
        grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
        th = [2 * np.pi * kk / n for kk, n in zip(k, shape)]
        phase = sum(t * gg for t, gg in zip(th, grids))
        e = np.exp(1j * phase)
        lap_e = oracle.lap(e.real, h) + 1j * oracle.lap(e.imag, h)
        mu = sum(4 / h ** 2 * np.sin(t / 2) ** 2 for t in th)
        np.testing.assert_allclose(lap_e, -mu * e, atol=1e-10)
        skew_e = oracle.skew_lap(e.real, h) + 1j * oracle.skew_lap(e.imag, h)
        if len(shape) == 2:
            sym = -(2 / h ** 2) * (1 - np.cos(th[0]) * np.cos(th[1]))
        else:
            sym = 0.0
            for j in range(3):
                t = np.sin(th[j] / 2) ** 2
                for i in range(3):
                    if i != j:
                        t *= np.cos(th[i] / 2) ** 2
                sym += t
            sym *= -4 / h ** 2
        np.testing.assert_allclose(skew_e, sym * e, atol=1e-10)
        # the oracle's mu_symbol at FFT index k equals the mode's eigenvalue
        assert abs(oracle.mu_symbol(shape, h)[tuple(k)] - mu) < 1e-10


# ------------------------------------------- energy, gradient, 2nd variation

@pytest.mark.parametrize("shape,p", [((8, 8), 4.0), ((8, 8), 3.0), ((8, 8), 6.0),
                                     ((4, 4, 8), 4.0), ((4, 4, 4), 3.0), ((8, 8), 2.0)])
def test_gradient_identity_4th(oracle, shape, p):
    """delta E_h[u](xi) = (N_h[u] - f, xi)_2 (Sec. 5.3): the residual equals
    -h^{-d} dE_h/du, checked by central differences of the plain energy."""
    P = oracle.Problem(4, 0.4, p, 0.3, 0.2)
    u = rng.standard_normal(shape)
    f = rng.standard_normal(shape)
    r = oracle.residual4(u, f, P)
    for _ in range(4):
        xi = rng.standard_normal(shape)
        t = 1e-5
        fd = (oracle.energy4(u + t * xi, f, P) - oracle.energy4(u - t * xi, f, P)) / (2 * t)
        an = -oracle.ip2(r, xi, P.h)
        assert abs(fd - an) <= 1e-7 * (abs(an) + 1)
        # second variation against a second difference of the energy
        t = 1e-4
        fd2 = (oracle.energy4(u + t * xi, f, P) - 2 * oracle.energy4(u, f, P)
               + oracle.energy4(u - t * xi, f, P)) / t ** 2
        sv = oracle.second_variation4(u, xi, P)
        assert abs(fd2 - sv) <= 1e-4 * abs(sv)


@pytest.mark.parametrize("shape", [(8, 8), (4, 8, 8)])
def test_gradient_identity_6th(oracle, shape):
    """Sixth order: for mean-zero xi, delta E_h[u](xi) = -(P0[f - N_h[u]], xi)."""
    P = oracle.Problem(6, 0.4, 4.0, 0.3, 0.2, lam=0.7)
    g = rng.standard_normal(shape)
    f = rng.standard_normal(shape)
    u = rng.standard_normal(shape)
    u = u - u.mean() + g.mean()
    r = oracle.residual6(u, f, g, P)
    assert abs(r.mean()) < 1e-14
    for _ in range(4):
        xi = rng.standard_normal(shape)
        xi -= xi.mean()
        t = 1e-5
        fd = (oracle.energy6(u + t * xi, f, g, P) - oracle.energy6(u - t * xi, f, g, P)) / (2 * t)
        an = -oracle.ip2(r, xi, P.h)
        assert abs(fd - an) <= 1e-7 * (abs(an) + 1)
        t = 1e-4
        fd2 = (oracle.energy6(u + t * xi, f, g, P) - 2 * oracle.energy6(u, f, g, P)
               + oracle.energy6(u - t * xi, f, g, P)) / t ** 2
        sv = oracle.second_variation6(u, xi, P)
        assert abs(fd2 - sv) <= 1e-4 * abs(sv)


def test_T_h_inverts_minus_laplacian(oracle):
    """-Delta_h T_h[zeta] = zeta for mean-zero zeta (Sec. 5.1)."""
    for shape in [(16, 8), (8, 8, 4)]:
        h = 0.3
        z = rng.standard_normal(shape)
        z -= z.mean()
        t = oracle.T_h(z, h)
        np.testing.assert_allclose(-oracle.lap(t, h), z, atol=1e-12)
        assert abs(t.mean()) < 1e-14


# ------------------------------------------- second-order consistency

def _continuous_N4(p, s, eps):
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    ut = sp.sin(x) * sp.cos(2 * y) + sp.Rational(3, 10) * sp.cos(x + y)
    ux, uy = sp.diff(ut, x), sp.diff(ut, y)
    g2 = ux ** 2 + uy ** 2
    r = g2 ** sp.Rational(int(p) - 2, 2)
    plap = sp.diff(r * ux, x) + sp.diff(r * uy, y)
    lap = sp.diff(ut, x, 2) + sp.diff(ut, y, 2)
    bih = sp.diff(lap, x, 2) + sp.diff(lap, y, 2)
    N = ut - s * plap + s * eps ** 2 * bih
    return sp.lambdify((x, y), ut, "numpy"), sp.lambdify((x, y), N, "numpy")


@pytest.mark.parametrize("p", [4.0, 6.0])
def test_second_order_consistency(oracle, p):
    """N_h[I_h u] - I_h(N u) = O(h^2) for smooth periodic u (Sec. 5.3)."""
    s, eps = 0.1, 0.3
    uf, Nf = _continuous_N4(p, s, eps)
    P = None
    errs, hs = [], []
    for n in (32, 64, 128, 256, 512):
        h = 2 * np.pi / n
        c = (np.arange(n) + 0.5) * h
        Y, X = np.meshgrid(c, c, indexing="ij")
        P = oracle.Problem(4, h, p, s, eps)
        e = oracle.N4(uf(X, Y), P) - Nf(X, Y)
        errs.append(np.max(np.abs(e)))
        hs.append(h)
    errs, hs = np.array(errs), np.array(hs)
    rates = np.log2(errs[:-1] / errs[1:])
    # Second order, reached from the pre-asymptotic side: at p = 6 the flux
    # |grad u|^4 grad u carries a large h^4 term, so the coarse rates are
    # 1.82, 1.93, 1.99 before 2.00.  The finest rate must be 2 within 0.01,
    # every rate above 1.7, and the error constant e / h^2 settled to 1%
    # between the two finest grids (a first-order or O(h^3) error fails both).
    const = errs / hs ** 2
    assert 1.99 < rates[-1] < 2.01 and np.all(rates > 1.7), rates
    assert abs(const[-1] - const[-2]) < 0.01 * const[-1], const


# ------------------------------------------- symmetries

@pytest.mark.parametrize("shape", [(8, 16), (4, 8, 8)])
def test_lattice_symmetries(oracle, shape):
    """A periodic shift, an axis reflection or (cubic grids) an axis swap of
    (u, f) commutes with N_h."""
    P = oracle.Problem(4, 0.3, 4.0, 0.2, 0.3)
    u = rng.standard_normal(shape)
    N = oracle.N4(u, P)
    for ax in range(len(shape)):
        np.testing.assert_allclose(oracle.N4(np.roll(u, 3, axis=ax), P), np.roll(N, 3, axis=ax), atol=1e-10)
        # reflection i -> n-1-i maps cells to cells and vertices to vertices
        np.testing.assert_allclose(oracle.N4(np.flip(u, axis=ax), P), np.flip(N, axis=ax), atol=1e-10)
    if len(set(shape[-2:])) == 1:
        np.testing.assert_allclose(oracle.N4(np.swapaxes(u, -1, -2), P), np.swapaxes(N, -1, -2), atol=1e-10)
