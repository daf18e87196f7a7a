"""Entry points beyond the solve: the discrete energy (psd_energy and
psd_info.energy) against the oracle's E_h, and the optional allocator
callback of psd_params (every workspace allocation goes through it and
psd_destroy returns all of it; results do not depend on it)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01475_gb300 import PSD_FP64, PSD_MIXED, Solver, synthetic  # noqa: E402

rng = np.random.default_rng(77)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("shape", [(64, 64), (16, 16, 16), (8, 16, 32)])
@pytest.mark.parametrize("order,p", [(4, 4.0), (4, 3.0), (6, 4.0)])
def test_energy_matches_oracle(oracle, shape, order, p):
    h = 2 * np.pi / shape[-1]
    P = oracle.Problem(order, h, p, 0.1, 0.2, 0.7)
    u = rng.standard_normal(shape) * 0.3
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape) if order == 6 else None
    S = Solver(order, shape, h, p, P.s, P.eps, P.lam)
    e = S.energy(dev(u), dev(f), None if g is None else dev(g))
    ref = oracle.energy4(u, f, P) if order == 4 else oracle.energy6(u, f, g, P)
    assert abs(e - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("precision", [PSD_FP64, PSD_MIXED])
def test_solve_reports_energy(precision):
    """psd_info.energy of a solve equals psd_energy of its result, and the
    minimiser's energy is below the start's (PSD decreases E_h)."""
    wl = synthetic.workload_small_2d(64)
    shape = wl["shape"]
    h = wl["L"] / shape[-1]
    S = Solver(4, shape, h, wl["p"], wl["s"], wl["eps"], precision=precision, tol=1e-11, report_energy=True)
    f = dev(wl["f"])
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    e0 = S.energy(u, f)
    info = S.solve(f, u)
    assert info["status"] == 0
    assert info["energy"] == pytest.approx(S.energy(u, f), rel=1e-14)
    assert info["energy"] < e0


def test_allocator_callback():
    """A caller-supplied allocator (here torch's caching allocator) receives
    every workspace allocation; psd_destroy frees each of them once, and the
    solution is bit-identical to the one with the default allocator."""
    live, calls = {}, {"alloc": 0, "free": 0}

    def alloc(nbytes):
        ptr = torch.cuda.caching_allocator_alloc(nbytes)
        live[ptr] = nbytes
        calls["alloc"] += 1
        return ptr

    def free(ptr):
        assert ptr in live
        del live[ptr]
        torch.cuda.caching_allocator_delete(ptr)
        calls["free"] += 1

    wl = synthetic.workload_spfc((32, 32, 32))
    shape = wl["shape"]
    h = wl["L"] / shape[-1]
    outs = []
    for allocator in (None, (alloc, free)):
        S = Solver(6, shape, h, wl["p"], wl["s"], wl["eps"], wl["lam"], precision=PSD_MIXED, tol=1e-10,
                   allocator=allocator)
        u = dev(wl["u0"])
        info = S.solve(dev(wl["f"]), u, dev(wl["g"]))
        assert info["status"] == 0
        outs.append(u.cpu().numpy())
        S.close()
    assert calls["alloc"] > 5 and calls["free"] == calls["alloc"] and not live
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("order,precision,shape", [(6, PSD_MIXED, (64, 64, 64)), (4, PSD_FP64, (128, 128)),
                                                   (4, PSD_MIXED, (32, 32, 64))])
def test_graph_replay_matches_direct_launches(order, precision, shape):
    """Chunks replayed from captured CUDA graphs give bit-identical results
    to the same kernels launched one by one (tracing on forces direct
    launches); a second solve into a different u buffer re-keys the FP64
    graph and agrees too."""
    h = 2 * np.pi / shape[-1]
    f = synthetic.fourier_field(shape, 2 * np.pi, 6, 4242, nmodes=16)
    g = synthetic.fourier_field(shape, 2 * np.pi, 6, 4243, nmodes=16) if order == 6 else None
    u0 = np.full(shape, g.mean()) if order == 6 else np.zeros(shape)
    S = Solver(order, shape, h, 4.0, 0.05, 0.1, 1.0, precision=precision, tol=1e-10, max_iter=4000)
    fd, gd = dev(f), (None if g is None else dev(g))
    S.profile(True)
    ud = dev(u0)
    S.solve(fd, ud, gd)
    S.profile(False)
    outs = [ud.cpu().numpy()]
    for _ in range(2):
        ug = dev(u0)
        info = S.solve(fd, ug, gd)
        assert info["status"] == 0
        outs.append(ug.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
