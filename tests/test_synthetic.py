"""The seeded input generators (paper_1607_01475_gb300/synthetic.py), which
feed both the oracle and the CUDA path: SplitMix64 against the published
generator's first outputs for seed 0 and a scalar restatement, offsets,
uniform and normal ranges and moments, and the shapes and parameter ranges
of the workloads."""

import numpy as np

from paper_1607_01475_gb300 import synthetic as S

M64 = (1 << 64) - 1


def _splitmix_scalar(seed, n):
    state, out = seed & M64, []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_known_outputs_and_offsets():
    # the first outputs of SplitMix64 seeded with 0
    assert [int(x) for x in S.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    seed = S.seed_for(2, 3, 1)
    assert [int(x) for x in S.splitmix64(seed, 64, offset=5)] == _splitmix_scalar(seed, 69)[5:]


def test_uniform_and_normal():
    u = S.uniform(S.seed_for(0), 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    z = S.normal(S.seed_for(1), 200000)
    assert np.all(np.isfinite(z))
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.02
    assert np.array_equal(S.normal(7, 10, offset=3), S.normal(7, 13)[3:])


def test_fourier_field_is_seeded_periodic_and_band_limited():
    shape = (16, 32)
    a = S.fourier_field(shape, 2 * np.pi, 4, 11, nmodes=8)
    assert a.shape == shape and np.array_equal(a, S.fourier_field(shape, 2 * np.pi, 4, 11, nmodes=8))
    assert not np.array_equal(a, S.fourier_field(shape, 2 * np.pi, 4, 12, nmodes=8))
    spec = np.abs(np.fft.fft2(a))
    kx = np.fft.fftfreq(shape[1], 1 / shape[1])[None, :]
    ky = np.fft.fftfreq(shape[0], 1 / shape[0])[:, None]
    outside = spec[(kx ** 2 + ky ** 2) > 16 + 1e-9]
    assert outside.max() <= 1e-9 * spec.max()  # only |k| <= K carries energy
    assert abs(a.mean()) <= 1e-12  # no k = 0 mode


def test_workload_batch_ranges():
    wl = S.workload_batch(96)
    assert len(wl) == 96
    ns = {w["shape"][0] for w in wl}
    assert ns <= {64, 128, 256, 512, 1024} and len(ns) >= 4
    assert all(1e-3 <= w["s"] <= 1e-1 and 0.02 <= w["eps"] <= 0.2 and w["p"] in (3.0, 4.0) for w in wl)
    assert all(w["tol"] >= 1e-10 for w in wl)
    assert {w["p"] for w in wl} == {3.0, 4.0}
