"""Plain FP64 CPU oracle for the preconditioned steepest descent (PSD) method of
Feng, Salgado, Wang & Wise, "Preconditioned steepest descent methods for some
nonlinear elliptic equations involving p-Laplacian terms" (arXiv:1607.01475).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: it exists so that tests, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` leg of ``bench.py`` can check the CUDA path against an
independent, slow, obviously correct restatement of the paper.  It shares no
code with the CUDA library.

Everything is plain numpy in float64.  Operators are written as compositions
of the paper's one-dimensional difference and average operators, exactly as
defined in Sec. 5.1; the FFT is this module's own radix-2 Cooley-Tukey
transform (``fft_axis``), not a library call.

Array conventions
-----------------
* A cell-centred grid function (the paper's C_per) is an array of shape
  ``(ny, nx)`` in 2D or ``(nz, ny, nx)`` in 3D; the LAST axis is x.  Array
  index ``i`` is the paper's cell ``i+1`` (centre at ``(i + 1/2) h``).
* A vertex-centred function (V_per) uses the same shape; array index ``v``
  holds the vertex at position ``(v + 1) h`` along each axis, i.e. the corner
  shared by cells ``v`` and ``v+1``.  With this storage the centre-to-vertex
  operators are forward differences/averages and the vertex-to-centre
  operators are backward ones, all with periodic wrap.
* Edge functions (E^ew, E^ns) are handled implicitly with the same rule per
  axis.

Readings of the paper (where it is silent or garbled)
------------------------------------------------------
* 3D operators are not written out (remark after Lemma "dis-lemma3" in
  Sec. 5.2).  We use the tensor extension: the x-derivative at a vertex is
  D_x A_y A_z, the vertex-to-centre x-derivative is d_x a_y a_z, Delta_h is
  the 7-point Laplacian, and vertex sums are h^3 sum over vertices.
* The vertex-to-centre average calA (Sec. 5.1) is printed with cell indices;
  it is read as the average of the 2^d vertices surrounding the cell.
* The cell inner product (.,.)_2 is printed with a stray psi; read as xi.
* For p < 4 the factor |grad u|^{p-4} (nabla u . nabla xi)^2 in the second
  variation is taken as 0 where the vertex gradient vanishes (its continuous
  extension); |0|^{p-2} = 0 for p > 2.
* Stopping: the residual norm is the paper's ||r||_2 = (h^d sum r^2)^{1/2};
  the iteration stops when it drops below ``tol`` (Algorithm 1).
* Sixth order: T_h (Sec. 5.1) is applied to the mean-zero projection of its
  argument; the residual is the mean-zero projection P0 of f - N_h[u]
  (the discrete problem lives on the mean-zero space, Sec. 5.4), and the
  line-search argument of T_h is u - g (Sec. 6.2 prints u - f; for the SPFC
  operator of Sec. 6.2 the argument is u - g).
"""

import numpy as np

__all__ = [
    "fft_axis", "fftn", "ifftn",
    "D", "A", "d", "a", "vgrad", "vdiv", "vavg", "lap", "skew_lap", "plap",
    "ip2", "ipv", "norm2", "mu_symbol",
    "N4", "residual4", "energy4", "second_variation4", "precond4",
    "T_h", "N6", "residual6", "energy6", "second_variation6", "precond6",
    "recover_w", "line_search", "line_search_poly", "psd_solve", "Problem", "hvp4", "dN4_ds", "adjoint4",
    "thinfilm_rhs", "thinfilm_energy", "thinfilm_steps", "thinfilm_adjoint",
    "spfc_rhs", "spfc_energy", "spfc_steps",
]


# --------------------------------------------------------------------------
# Radix-2 Cooley-Tukey FFT (Sec. 6: the search-direction and Poisson
# equations are solved with the FFT).  Own implementation, iterative,
# decimation in time with a bit-reversal permutation.
# --------------------------------------------------------------------------

def _bit_reverse_indices(n):
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft_axis(x, axis, inverse=False):
    """DFT along ``axis``: X_k = sum_j x_j exp(-2 pi i j k / n) (forward) or
    x_j = (1/n) sum_k X_k exp(+2 pi i j k / n) (inverse).  n a power of two."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    if n & (n - 1):
        raise ValueError("fft_axis: length must be a power of two")
    lead = x.shape[:-1]
    y = x[..., _bit_reverse_indices(n)].copy()
    sign = 1.0 if inverse else -1.0
    m = 1
    while m < n:
        # combine pairs of length-m transforms into length-2m transforms
        w = np.exp(sign * 1j * np.pi * np.arange(m) / m)
        y = y.reshape(lead + (n // (2 * m), 2, m))
        even = y[..., 0, :]
        odd = y[..., 1, :] * w
        y = np.stack([even + odd, even - odd], axis=-2).reshape(lead + (n,))
        m *= 2
    if inverse:
        y = y / n
    return np.moveaxis(y, -1, axis)


def fftn(x):
    y = np.asarray(x, dtype=np.complex128)
    for ax in range(y.ndim):
        y = fft_axis(y, ax)
    return y


def ifftn(x):
    y = np.asarray(x, dtype=np.complex128)
    for ax in range(y.ndim):
        y = fft_axis(y, ax, inverse=True)
    return y


# --------------------------------------------------------------------------
# Difference and average operators (Sec. 5.1).  ``ax`` is a numpy axis.
# --------------------------------------------------------------------------

def D(u, ax, h):
    """D_x: (u_{i+1} - u_i)/h, centre -> edge (or edge -> vertex)."""
    return (np.roll(u, -1, axis=ax) - u) / h


def A(u, ax):
    """A_x: (u_{i+1} + u_i)/2, centre -> edge (or edge -> vertex)."""
    return 0.5 * (np.roll(u, -1, axis=ax) + u)


def d(w, ax, h):
    """d_x: (w_{i+1/2} - w_{i-1/2})/h, edge -> centre (or vertex -> edge)."""
    return (w - np.roll(w, 1, axis=ax)) / h


def a(w, ax):
    """a_x: (w_{i+1/2} + w_{i-1/2})/2, edge -> centre (or vertex -> edge)."""
    return 0.5 * (w + np.roll(w, 1, axis=ax))


def vgrad(u, h):
    """Centre-to-vertex gradient nabla_h^v u: for each axis, D along it and
    A along every other axis (Sec. 5.1; 3D by the tensor extension)."""
    out = []
    for ax in range(u.ndim):
        t = u
        for other in range(u.ndim):
            if other != ax:
                t = A(t, other)
        out.append(D(t, ax, h))
    return out


def vdiv(w, h):
    """Vertex-to-centre divergence sum_a frak{d}_a w_a, frak{d}_a = d_a times
    a along every other axis (Sec. 5.1)."""
    total = 0.0
    nd = len(w)
    for ax in range(nd):
        t = w[ax]
        for other in range(nd):
            if other != ax:
                t = a(t, other)
        total = total + d(t, ax, h)
    return total


def vavg(nu):
    """calA: average of the 2^d vertices surrounding each cell (Sec. 5.1)."""
    t = nu
    for ax in range(nu.ndim):
        t = a(t, ax)
    return t


def lap(u, h):
    """Standard Laplacian Delta_h = sum_a d_a D_a (5-point / 7-point)."""
    total = 0.0
    for ax in range(u.ndim):
        total = total + d(D(u, ax, h), ax, h)
    return total


def skew_lap(u, h):
    """Skew Laplacian Delta_h^v = sum_a frak{d}_a frak{D}_a (Sec. 5.1)."""
    return vdiv(vgrad(u, h), h)


def _vertex_factor(g2, p):
    """|g|^{p-2} from |g|^2 at the vertices."""
    if p == 2:
        return np.ones_like(g2)
    return g2 ** ((p - 2.0) / 2.0)


def plap(u, h, p):
    """Discrete p-Laplacian nabla_h^v . (|nabla_h^v u|^{p-2} nabla_h^v u)
    with r = [sum_a (frak{D}_a u)^2]^{(p-2)/2} at the vertices (Sec. 5.1)."""
    g = vgrad(u, h)
    g2 = sum(c * c for c in g)
    r = _vertex_factor(g2, p)
    return vdiv([r * c for c in g], h)


# --------------------------------------------------------------------------
# Inner products and norms (Sec. 5.1)
# --------------------------------------------------------------------------

def ip2(u, v, h):
    """(u, v)_2 = h^d sum u v over the periodic cells."""
    return float(h ** u.ndim * np.sum(u * v))


def ipv(nu, xi, h):
    """<nu, xi> = (calA(nu xi), 1)_2, the vertex inner product."""
    return ip2(vavg(nu * xi), np.ones_like(nu), h)


def norm2(u, h):
    return np.sqrt(ip2(u, u, h))


def mu_symbol(shape, h):
    """Eigenvalue of -Delta_h on the Fourier mode with FFT indices k:
    mu(k) = sum_a (4/h^2) sin^2(pi k_a / n_a)  (the squared modulus of the
    per-axis difference symbol w_l = -2 i sin(l pi h / L)/h of the appendix)."""
    mu = np.zeros(shape)
    for ax, n in enumerate(shape):
        k = np.arange(n)
        s = (4.0 / h ** 2) * np.sin(np.pi * k / n) ** 2
        bshape = [1] * len(shape)
        bshape[ax] = n
        mu = mu + s.reshape(bshape)
    return mu


# --------------------------------------------------------------------------
# Problem description
# --------------------------------------------------------------------------

class Problem:
    """Parameters of one discrete problem.

    order 4: u - s plap(u) + s eps^2 Delta_h^2 u = f          (Sec. 5.3)
    order 6: u - Delta_h w = g,
             s lam u - s plap(u) + s eps^2 Delta_h^2 u - w = f  (Sec. 5.4)
    """

    def __init__(self, order, h, p, s, eps, lam=0.0):
        if order not in (4, 6):
            raise ValueError("order must be 4 or 6")
        self.order, self.h, self.p = order, float(h), float(p)
        self.s, self.eps, self.lam = float(s), float(eps), float(lam)


# --------------------------------------------------------------------------
# Fourth order (Sec. 5.3; thin-film form Sec. 6.1)
# --------------------------------------------------------------------------

def N4(u, P):
    """N_h[u] = u - s plap(u) + s eps^2 Delta_h^2 u."""
    h = P.h
    return u - P.s * plap(u, h, P.p) + P.s * P.eps ** 2 * lap(lap(u, h), h)


def residual4(u, f, P):
    """r = f - N_h[u] = -(grad of E_h) in the (.,.)_2 metric."""
    return f - N4(u, P)


def energy4(u, f, P):
    """E_h[u] = 1/2 ||u - f||_2^2 + s/p ||nabla_h^v u||_p^p
    + s eps^2/2 ||Delta_h u||_2^2   (Eq. "diseng4")."""
    h = P.h
    g = vgrad(u, h)
    g2 = sum(c * c for c in g)
    ones = np.ones_like(u)
    lu = lap(u, h)
    return (0.5 * ip2(u - f, u - f, h)
            + P.s / P.p * ipv(g2 ** (P.p / 2.0), ones, h)
            + 0.5 * P.s * P.eps ** 2 * ip2(lu, lu, h))


def _pterm_second_variation(u, xi, P):
    """s <|g|^{p-2} D xi, D xi> + (p-2) s <|g|^{p-4} (g . D xi)^2, 1>."""
    h = P.h
    g = vgrad(u, h)
    b = vgrad(xi, h)
    g2 = sum(c * c for c in g)
    gb = sum(c * e for c, e in zip(g, b))
    b2 = sum(e * e for e in b)
    ones = np.ones_like(u)
    t1 = ipv(_vertex_factor(g2, P.p) * b2, ones, h)
    if P.p == 2:
        t2 = 0.0
    else:
        with np.errstate(divide="ignore", invalid="ignore"):
            w = np.where(g2 > 0, g2 ** ((P.p - 4.0) / 2.0) * gb * gb, 0.0)
        t2 = (P.p - 2.0) * ipv(w, ones, h)
    return P.s * (t1 + t2)


def second_variation4(u, xi, P):
    """delta^2 E_h[u](xi, xi) (Sec. 5.3)."""
    h = P.h
    lx = lap(xi, h)
    return (ip2(xi, xi, h) + _pterm_second_variation(u, xi, P)
            + P.s * P.eps ** 2 * ip2(lx, lx, h))


def precond4(r, P):
    """Solve L_h d = r, L_h = I - s Delta_h + s eps^2 Delta_h^2, with the FFT
    (Sec. 5.3 and Sec. 6.1): divide by 1 + s mu + s eps^2 mu^2."""
    mu = mu_symbol(r.shape, P.h)
    lam = 1.0 + P.s * mu + P.s * P.eps ** 2 * mu * mu
    return np.real(ifftn(fftn(r) / lam))


# --------------------------------------------------------------------------
# Sixth order (Sec. 5.4; SPFC form Sec. 6.2)
# --------------------------------------------------------------------------

def T_h(zeta, h):
    """T_h = -Delta_h^{-1} on mean-zero functions (Sec. 5.1), applied to the
    mean-zero projection of ``zeta``: divide the spectrum by mu, zero mode 0."""
    mu = mu_symbol(zeta.shape, h)
    zh = fftn(zeta)
    out = np.zeros_like(zh)
    nz = mu > 0
    out[nz] = zh[nz] / mu[nz]
    return np.real(ifftn(out))


def _p0(v):
    return v - v.mean()


def N6(u, g, P):
    """N_h[u] = s lam u - s plap(u) + s eps^2 Delta_h^2 u + T_h[u - g]
    (Sec. 6.2 with gamma_0 = lam; -T_h[-u + g] = T_h[u - g])."""
    h = P.h
    return (P.s * P.lam * u - P.s * plap(u, h, P.p)
            + P.s * P.eps ** 2 * lap(lap(u, h), h) + T_h(u - g, h))


def residual6(u, f, g, P):
    """r = P0[f - N_h[u]]: the residual lives on the mean-zero space."""
    return _p0(f - N6(u, g, P))


def energy6(u, f, g, P):
    """E_h of Sec. 5.4 written in u = nu + gbar (nu mean-zero):
    1/2 ||u - g||_{-1}^2 + lam s/2 ||u||_2^2 - (u - gbar, f)_2
    + s/p ||nabla_h^v u||_p^p + s eps^2/2 ||Delta_h u||_2^2."""
    h = P.h
    gbar = g.mean()
    z = u - g
    g_ = vgrad(u, h)
    g2 = sum(c * c for c in g_)
    ones = np.ones_like(u)
    lu = lap(u, h)
    return (0.5 * ip2(z, T_h(z, h), h)
            + 0.5 * P.lam * P.s * ip2(u, u, h)
            - ip2(u - gbar, f, h)
            + P.s / P.p * ipv(g2 ** (P.p / 2.0), ones, h)
            + 0.5 * P.s * P.eps ** 2 * ip2(lu, lu, h))


def second_variation6(u, xi, P):
    """delta^2 E_h[u](xi, xi) for the sixth-order energy (Sec. 4, discrete)."""
    h = P.h
    lx = lap(xi, h)
    return (ip2(xi, T_h(xi, h), h) + P.lam * P.s * ip2(xi, xi, h)
            + _pterm_second_variation(u, xi, P)
            + P.s * P.eps ** 2 * ip2(lx, lx, h))


def precond6(r, P):
    """Solve L_h d = r on the mean-zero space,
    L_h = s lam I - s Delta_h + s eps^2 Delta_h^2 + T_h  (Sec. 5.4, 6.2):
    divide by s lam + s mu + s eps^2 mu^2 + 1/mu, zero mode 0."""
    mu = mu_symbol(r.shape, P.h)
    rh = fftn(r)
    out = np.zeros_like(rh)
    nz = mu > 0
    m = mu[nz]
    out[nz] = rh[nz] / (P.s * P.lam + P.s * m + P.s * P.eps ** 2 * m * m + 1.0 / m)
    return np.real(ifftn(out))


def recover_w(u, f, g, P):
    """w = -T_h[u - g] + s lam gbar - fbar  (Sec. 4, change of variables)."""
    return -T_h(u - g, P.h) + P.s * P.lam * g.mean() - f.mean()


# --------------------------------------------------------------------------
# Line search (Eq. "eqn-search"): alpha = argzero q, q(alpha) =
# (N_h[u + alpha d] - f, d)_2 = delta E_h[u + alpha d](d).
# --------------------------------------------------------------------------

def line_search(q, dq, alpha0, max_iter=200):
    """Root of the strictly increasing q with q(0) < 0 (Prop. "energy-decrease":
    alpha > 0).  Newton's method with a bisection safeguard on a bracket
    [lo, hi]; q' is the second variation delta^2 E_h[u + alpha d](d, d)."""
    lo, hi = 0.0, None
    alpha = alpha0 if alpha0 > 0 else 1.0
    # find an upper end of the bracket
    b = alpha
    for _ in range(200):
        if q(b) > 0:
            hi = b
            break
        lo = b
        b *= 2.0
    if hi is None:
        raise RuntimeError("line search: no sign change found")
    alpha = min(max(alpha, lo), hi)
    for _ in range(max_iter):
        qa = q(alpha)
        if qa == 0.0:
            return alpha
        if qa < 0:
            lo = alpha
        else:
            hi = alpha
        step = qa / dq(alpha)
        new = alpha - step
        if not (lo < new < hi):
            new = 0.5 * (lo + hi)
        if abs(new - alpha) <= 4e-16 * abs(new) or hi - lo <= 4e-16 * hi:
            return new
        alpha = new
    return alpha


def line_search_poly(u, d, f, P, g=None):
    """Coefficients (lowest power first) of q(alpha) = (N_h[u + alpha d] - f, d)_2
    for even p = 2, 4, 6, where q is a polynomial of degree p - 1 (Sec. 6.1:
    a cubic for p = 4, a quintic for p = 6).  The linear part of N_h gives
    (Lin u - f, d)_2 + alpha (Lin d, d)_2 (order 6: T_h[u - g] in Lin u, T_h d
    in Lin d); by summation by parts the p-term is
    s <|a + alpha b|^{p-2} (a + alpha b), b> with a = grad_h^v u and
    b = grad_h^v d at the vertices, expanded in A = |a|^2, B = a.b, C = |b|^2."""
    if P.p not in (2.0, 4.0, 6.0):
        raise ValueError("q is a polynomial for even p only")
    h = P.h
    s, se2 = P.s, P.s * P.eps ** 2
    if P.order == 4:
        lin_u = u + se2 * lap(lap(u, h), h)
        lin_d = d + se2 * lap(lap(d, h), h)
    else:
        lin_u = s * P.lam * u + se2 * lap(lap(u, h), h) + T_h(u - g, h)
        lin_d = s * P.lam * d + se2 * lap(lap(d, h), h) + T_h(d, h)
    ga, gb = vgrad(u, h), vgrad(d, h)
    A = sum(c * c for c in ga)
    B = sum(x * y for x, y in zip(ga, gb))
    C = sum(c * c for c in gb)
    if P.p == 2.0:
        terms = [B, C]
    elif P.p == 4.0:
        terms = [A * B, A * C + 2 * B * B, 3 * B * C, C * C]
    else:
        terms = [A * A * B, A * A * C + 4 * A * B * B, 6 * A * B * C + 4 * B ** 3,
                 8 * B * B * C + 2 * A * C * C, 5 * B * C * C, C ** 3]
    w = s * h ** u.ndim
    coef = [w * float(np.sum(t)) for t in terms]
    coef[0] += ip2(lin_u - f, d, h)
    coef[1] += ip2(lin_d, d, h)
    return coef


# --------------------------------------------------------------------------
# PSD iteration (Algorithm 1 structure; search direction Eq.
# "search-direction-pb", update Eq. "eq:psd4", step Eq. "eqn-search")
# --------------------------------------------------------------------------

def _ops(P, f, g):
    if P.order == 4:
        res = lambda u: residual4(u, f, P)
        pre = lambda r: precond4(r, P)
        nop = lambda u: N4(u, P)
        sv = lambda u, x: second_variation4(u, x, P)
        en = lambda u: energy4(u, f, P)
    else:
        res = lambda u: residual6(u, f, g, P)
        pre = lambda r: precond6(r, P)
        nop = lambda u: N6(u, g, P)
        sv = lambda u, x: second_variation6(u, x, P)
        en = lambda u: energy6(u, f, g, P)
    return res, pre, nop, sv, en


def psd_solve(P, f, u0, g=None, tol=1e-10, kmax=1000, record=False):
    """Run PSD from u0 until ||r||_2 < tol or kmax iterations.

    Returns (u, info) where info holds the iteration count, the residual
    history ||r_k||_2 (k = 0..iters), the step sizes alpha_k and, if
    ``record``, the energies and iterates."""
    res, pre, nop, sv, en = _ops(P, f, g)
    h = P.h
    u = np.array(u0, dtype=np.float64, copy=True)
    r = res(u)
    info = {"iters": 0, "res": [norm2(r, h)], "alpha": [], "energy": [],
            "u": [], "d": []}
    if record:
        info["energy"].append(en(u))
        info["u"].append(u.copy())
    if info["res"][0] < tol:
        return u, info
    for k in range(kmax):
        dk = pre(r)
        rd = ip2(r, dk, h)

        def q(al, u=u, dk=dk):
            return ip2(nop(u + al * dk) - f, dk, h)

        def dq(al, u=u, dk=dk):
            return sv(u + al * dk, dk)

        alpha0 = rd / dq(0.0)
        alpha = line_search(q, dq, alpha0)
        u = u + alpha * dk
        r = res(u)
        info["iters"] = k + 1
        info["alpha"].append(alpha)
        info["res"].append(norm2(r, h))
        if record:
            info["energy"].append(en(u))
            info["u"].append(u.copy())
            info["d"].append(dk.copy())
        if info["res"][-1] < tol:
            break
    return u, info


# --------------------------------------------------------------------------
# Adjoint (gradient of a loss of the converged solution).  Not in the paper:
# by the implicit function theorem at the solution of N_h[u] = f,
#   dJ/df = lambda,  dJ/ds = -(lambda . dN_h/ds),  H lambda = dJ/du,
# with H = dN_h/du (the array Jacobian, symmetric: h^{-d} times the Hessian
# of E_h, i.e. the second variation of Sec. 5.3 in the Euclidean product).
# Gradients are with respect to the array entries (Euclidean).
# --------------------------------------------------------------------------

def hvp4(u, v, P):
    """H v = v - s d.(W(g) D v) + s eps^2 Delta_h^2 v with g = D u and
    W(g) = |g|^{p-2} I + (p-2)|g|^{p-4} g g^T (second variation, Sec. 5.3;
    the (p-2)-term is 0 where g = 0 for p < 4)."""
    h = P.h
    g = vgrad(u, h)
    b = vgrad(v, h)
    g2 = sum(c * c for c in g)
    gb = sum(c * e for c, e in zip(g, b))
    r = _vertex_factor(g2, P.p)
    if P.p == 2:
        w = 0.0 * g2
    else:
        with np.errstate(divide="ignore", invalid="ignore"):
            w = np.where(g2 > 0, (P.p - 2.0) * g2 ** ((P.p - 4.0) / 2.0) * gb, 0.0)
    flux = [r * e + w * c for c, e in zip(g, b)]
    return v - P.s * vdiv(flux, h) + P.s * P.eps ** 2 * lap(lap(v, h), h)


def dN4_ds(u, P):
    """Partial derivative of N_h[u] with respect to s."""
    h = P.h
    return -plap(u, h, P.p) + P.eps ** 2 * lap(lap(u, h), h)


def adjoint4(u, grad_u, P, tol=1e-13, kmax=2000):
    """Solve H lam = grad_u by conjugate gradients preconditioned with L_h
    (the PSD preconditioner); return (grad_f, grad_s, iterations)."""
    lam = np.zeros_like(grad_u)
    r = grad_u.copy()
    z = precond4(r, P)
    p = z.copy()
    rz = float(np.sum(r * z))
    bnorm = np.sqrt(float(np.sum(grad_u * grad_u)))
    it = 0
    for it in range(1, kmax + 1):
        Hp = hvp4(u, p, P)
        a = rz / float(np.sum(p * Hp))
        lam = lam + a * p
        r = r - a * Hp
        if np.sqrt(float(np.sum(r * r))) <= tol * bnorm:
            break
        z = precond4(r, P)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    grad_s = -float(np.sum(lam * dN4_ds(u, P)))
    return lam, grad_s, it


# --------------------------------------------------------------------------
# Thin-film epitaxy with slope selection, convex-splitting time loop (Sec.
# 6.1, Eq. "thin-film-fully-discrete"): each step solves N_h[u^{n+1}] = f
# with the fourth-order operator of Sec. 5.3 (s = the time step) and
# f = u^n - s Delta_h^v u^n, the concave part -1/2 |grad u|^2 of the energy
# taken explicitly with the skew Laplacian.
# --------------------------------------------------------------------------

def thinfilm_rhs(u, P):
    """f = u^n - s Delta_h^v u^n (Sec. 6.1)."""
    return u - P.s * skew_lap(u, P.h)


def thinfilm_energy(u, P):
    """Discrete thin-film energy (Sec. 6.1 with the operators of Sec. 5.1):
    h^d sum_v (1/p |grad_h^v u|^p - 1/2 |grad_h^v u|^2) + eps^2/2 ||Delta_h u||_2^2.
    The convex-splitting scheme does not increase it, for any step s."""
    h = P.h
    g = vgrad(u, h)
    g2 = sum(c * c for c in g)
    vertex = h ** u.ndim * float(np.sum(g2 ** (P.p / 2.0) / P.p - 0.5 * g2))
    lu = lap(u, h)
    return vertex + 0.5 * P.eps ** 2 * ip2(lu, lu, h)


def thinfilm_steps(P, u0, nsteps, tol=1e-12, kmax=1000):
    """nsteps steps of the scheme from u0, each PSD solve started from the
    previous step's solution; returns (u, per-step iteration counts)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    iters = []
    for _ in range(nsteps):
        u, info = psd_solve(P, thinfilm_rhs(u, P), u, tol=tol, kmax=kmax)
        iters.append(info["iters"])
    return u, iters


# --------------------------------------------------------------------------
# Square phase field crystal (SPFC), convex-splitting time loop (Sec. 6.2,
# Eq. "scheme-spfc"; the s-scaled right-hand side of the scheme in Sec. 1):
# each step solves the sixth-order problem of Sec. 5.4 with lambda = gamma_0,
# g = u^n and f = -s gamma_1 Delta_h u^n.
# --------------------------------------------------------------------------

def spfc_rhs(u, P, gamma1):
    """(f, g) = (-s gamma_1 Delta_h u^n, u^n)."""
    return -P.s * gamma1 * lap(u, P.h), u.copy()


def spfc_energy(u, P, gamma1):
    """Discrete SPFC energy (Sec. 6.2 with the operators of Sec. 5.1):
    gamma_0/2 ||u||^2 + gamma_1/2 (u, Delta_h u)_2 + eps^2/2 ||Delta_h u||^2
    + 1/4 h^d sum_v |grad_h^v u|^4, gamma_0 = lambda.  The convex-splitting
    scheme does not increase it, for any step s."""
    h = P.h
    lu = lap(u, h)
    g = vgrad(u, h)
    g2 = sum(c * c for c in g)
    return (0.5 * P.lam * ip2(u, u, h) + 0.5 * gamma1 * ip2(u, lu, h) + 0.5 * P.eps ** 2 * ip2(lu, lu, h)
            + 0.25 * h ** u.ndim * float(np.sum(g2 * g2)))


def spfc_steps(P, u0, gamma1, nsteps, tol=1e-12, kmax=1000):
    """nsteps SPFC steps from u0 (order 6, p = 4), each PSD solve started
    from the previous step's solution; returns (u, per-step iterations)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    iters = []
    for _ in range(nsteps):
        f, g = spfc_rhs(u, P, gamma1)
        u, info = psd_solve(P, f, u, g=g, tol=tol, kmax=kmax)
        iters.append(info["iters"])
    return u, iters


def thinfilm_adjoint(P, u0, nsteps, grad_uN, tol=1e-13):
    """Gradient of a loss J(u^N) of the thin-film time loop with respect to
    u^0 and s (Euclidean, like adjoint4), given dJ/du^N.  Not in the paper:
    the chain rule through the steps of Sec. 6.1.  Step n maps u^n to the
    solution u^{n+1} of N_h[u] = f_n, f_n = u^n - s Delta_h^v u^n; with
    mu_n = H(u^{n+1})^{-1} lambda_{n+1} (adjoint4, dJ/df_n = mu_n):
      lambda_n = mu_n - s Delta_h^v mu_n          (Delta_h^v is symmetric)
      dJ/ds   += -(mu_n . dN_h/ds(u^{n+1})) - (mu_n . Delta_h^v u^n).
    Returns (dJ/du^0, dJ/ds); every forward state is kept."""
    us = [np.array(u0, dtype=np.float64, copy=True)]
    for _ in range(nsteps):
        u, _ = psd_solve(P, thinfilm_rhs(us[-1], P), us[-1], tol=tol, kmax=2000)
        us.append(u)
    lam = np.array(grad_uN, dtype=np.float64, copy=True)
    gs = 0.0
    for n in reversed(range(nsteps)):
        mu, gs_n, _ = adjoint4(us[n + 1], lam, P, tol=tol)
        gs += gs_n - float(np.sum(mu * skew_lap(us[n], P.h)))
        lam = mu - P.s * skew_lap(mu, P.h)
    return lam, gs
