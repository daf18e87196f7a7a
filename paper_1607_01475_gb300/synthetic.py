"""Seeded synthetic inputs for the PSD workloads.

This module holds only input synthesis (random numbers and smooth random
fields); it contains none of the solver's arithmetic, so that the CPU oracle
used by the tests and the CUDA library can both be fed the same arrays.

Random numbers come from SplitMix64 used as a counter-based generator: the
i-th output of stream ``seed`` is mix(seed + (i+1) * 0x9E3779B97F4A7C15),
with the published SplitMix64 finaliser (Steele, Lea & Flood, 2014).
Uniforms take the top 53 bits; normals use the Box-Muller transform.

Seeds follow ``1607014750 + 1000*workload + 10*instance + field`` with
field 0 = f, 1 = g, 2 = u_target, 3 = the random phase field.

All fields live on the periodic box (0, L)^d with cell centres at
(i + 1/2) h, h = L / n, arrays shaped (ny, nx) or (nz, ny, nx), x last.
"""

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 1607014750


def seed_for(workload, instance=0, field=0):
    return SEED_BASE + 1000 * workload + 10 * instance + field


def splitmix64(seed, n, offset=0):
    """n consecutive SplitMix64 outputs of stream ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n, offset=0):
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed, n, offset=0):
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    u = uniform(seed, 2 * n, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def cell_centres(n, L):
    h = L / n
    return (np.arange(n) + 0.5) * h


def fourier_field(shape, L, K, seed, nmodes=32):
    """sum_{j<nmodes} (a_j cos(k_j.x) + b_j sin(k_j.x)) / (1 + |k_j|^2) with
    a_j, b_j ~ N(0,1) and k_j uniform over non-zero integer wave vectors with
    |k| <= K (angular wavenumbers 2 pi k / L), evaluated at cell centres."""
    dim = len(shape)
    # wave vectors by rejection from the cube [-K, K]^dim
    ks = []
    off = 0
    while len(ks) < nmodes:
        cand = np.floor(uniform(seed + 7, dim, off) * (2 * K + 1)).astype(np.int64) - K
        off += dim
        if 0 < int(np.sum(cand * cand)) <= K * K:
            ks.append(cand)
    amp = normal(seed, 2 * nmodes).reshape(nmodes, 2)
    # per-axis complex exponentials, axis order (.., y, x) = reversed dims
    axes = [cell_centres(n, L) for n in shape]
    out = np.zeros(shape)
    for j in range(nmodes):
        k = ks[j]  # k[0] pairs with the last array axis (x)
        e = None
        for ax in range(dim):
            kk = k[dim - 1 - ax]
            v = np.exp(1j * 2.0 * np.pi * kk * axes[ax] / L)
            e = v if e is None else np.multiply.outer(e, v)
        w = (amp[j, 0] - 1j * amp[j, 1]) / (1.0 + float(np.sum(k * k)))
        out += np.real(w * e)
    return out


def smoothed_uniform_field(shape, L, seed, amp=0.1, width=64.0):
    """Real part of F^{-1}[exp(-|k|^2/width) F[U]], U ~ uniform(-amp, amp) per
    cell (the random initial data shape of the coarsening runs, smoothed)."""
    n_tot = int(np.prod(shape))
    U = amp * (2.0 * uniform(seed, n_tot) - 1.0)
    U = U.reshape(shape)
    k2 = _wavenumber_sq(shape, L)
    return np.real(np.fft.ifftn(np.exp(-k2 / width) * np.fft.fftn(U)))


def thin_film_rhs(phi, L, s):
    """phi - s Delta phi with the exact (spectral) continuous Laplacian: a
    right-hand side shaped like the thin-film convex-splitting step."""
    k2 = _wavenumber_sq(phi.shape, L)
    return np.real(np.fft.ifftn((1.0 + s * k2) * np.fft.fftn(phi)))


def _wavenumber_sq(shape, L):
    k2 = np.zeros(shape)
    for ax, n in enumerate(shape):
        k = np.fft.fftfreq(n, d=1.0 / n) * (2.0 * np.pi / L)
        b = [1] * len(shape)
        b[ax] = n
        k2 = k2 + (k * k).reshape(b)
    return k2


# --------------------------------------------------------------------------
# The benchmark workloads (problem sizes and parameters)
# --------------------------------------------------------------------------

TWO_PI = 2.0 * np.pi


def workload_small_2d(n=64):
    """2D fourth order, p=4, s=0.01, eps=0.1 on (0, 2pi)^2; f = Fourier field
    with K=8; u0 = 0."""
    shape = (n, n)
    f = fourier_field(shape, TWO_PI, 8, seed_for(0, 0, 0))
    return dict(order=4, shape=shape, L=TWO_PI, p=4.0, s=0.01, eps=0.1,
                lam=0.0, f=f, g=None, u0=np.zeros(shape))


def workload_thin_film(shape):
    """Fourth order, p=4, s=0.1, eps=0.05 on (0, 2pi)^d; phi a smoothed random
    phase field, f = phi - s Delta phi; u0 = 0 (2D 1024^2 and 3D 128^3)."""
    s = 0.1
    phi = smoothed_uniform_field(shape, TWO_PI, seed_for(1, 0, 3))
    f = thin_film_rhs(phi, TWO_PI, s)
    return dict(order=4, shape=tuple(shape), L=TWO_PI, p=4.0, s=s, eps=0.05,
                lam=0.0, f=f, g=None, u0=np.zeros(shape))


def workload_spfc(shape=(256, 256, 256)):
    """Sixth order, p=4, lam=1, s=0.05, eps=0.1 on (0, 2pi)^d; f and g Fourier
    fields with K=16; u0 = mean(g) (3D 256^3 in the benchmark)."""
    f = fourier_field(shape, TWO_PI, 16, seed_for(2, 0, 0))
    g = fourier_field(shape, TWO_PI, 16, seed_for(2, 0, 1))
    u0 = np.full(shape, g.mean())
    return dict(order=6, shape=tuple(shape), L=TWO_PI, p=4.0, s=0.05, eps=0.1,
                lam=1.0, f=f, g=g, u0=u0)


def thin_film_init1(n, L=3.2):
    """The analytic initial data of the thin-film convergence test (Sec. 6.1.1,
    Eq. "init1") on (0, L)^2 at cell centres:
    0.1 sin^2(2 pi x / L) sin(4 pi (y - 1.4) / L) - 0.1 cos(2 pi (x - 2) / L) sin(2 pi y / L).
    Returns (u0, h)."""
    h = L / n
    x = (np.arange(n) + 0.5) * h
    y = x[:, None]
    return (0.1 * np.sin(2 * np.pi * x / L) ** 2 * np.sin(4 * np.pi * (y - 1.4) / L)
            - 0.1 * np.cos(2 * np.pi * (x - 2.0) / L) * np.sin(2 * np.pi * y / L)), h


def workload_batch(count=96, max_exp=5):
    """Uneven 2D fourth-order instances on (0, 2pi)^2: n = 2^(6 + floor(max_exp U))
    (64..1024 for max_exp = 5), s = 10^(-3 + 2U), eps uniform in [0.02, 0.2],
    p = 3 or 4 with probability 1/2, f a Fourier field with K = 8; u0 = 0.

    ``tol`` is the instance's residual target: 1e-10, raised to the FP64
    rounding floor of the residual where that is larger.  Delta_h^2 applied
    as two Laplacian passes carries a rounding error of about
    64 eps64 |u| per cell, scaled by s eps^2 / h^4, so
    floor = 64 eps64 (s eps^2 / h^4) max|f| |Omega|^(1/2) (|u| <= max|f|
    for these problems)."""
    out = []
    for i in range(count):
        u = uniform(seed_for(3, i, 5), 4)
        n = 2 ** (6 + int(np.floor(max_exp * u[0])))
        s = 10.0 ** (-3.0 + 2.0 * u[1])
        eps = 0.02 + 0.18 * u[2]
        p = 3.0 if u[3] < 0.5 else 4.0
        shape = (n, n)
        f = fourier_field(shape, TWO_PI, 8, seed_for(3, i, 0))
        h = TWO_PI / n
        floor = 64.0 * np.finfo(np.float64).eps * (s * eps * eps / h ** 4) * float(np.max(np.abs(f))) * TWO_PI
        out.append(dict(order=4, shape=shape, L=TWO_PI, p=p, s=s, eps=eps, lam=0.0, f=f, g=None,
                        u0=np.zeros(shape), tol=max(1e-10, floor)))
    return out
