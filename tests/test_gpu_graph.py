"""The graph-driven solve (the whole PSD run captured once into a CUDA graph
whose loops are WHILE conditional nodes set by device kernels) against the
same solve driven from the host (kernel tracing on, which launches every
kernel directly and reads the stop flags on the host): the same kernels in
the same order, so the iterates must agree bit for bit -- for the plain FP64
loop, the nested mixed outer / inner loops, and the general-p Newton line
search nested inside the iteration loop."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01475_gb300 import PSD_FP64, PSD_MIXED, Solver, synthetic  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


CASES = [((64, 64), 4, 4.0), ((32, 32, 32), 4, 4.0), ((64, 64), 6, 4.0), ((32, 32, 32), 6, 4.0),
         ((64, 64), 4, 3.0), ((16, 16, 16), 4, 6.0), ((32, 64, 64), 6, 4.0)]


@pytest.mark.parametrize("shape,order,p", CASES)
@pytest.mark.parametrize("precision", [PSD_FP64, PSD_MIXED])
def test_graph_solve_matches_host_driven_solve(shape, order, p, precision):
    h = 2 * np.pi / shape[-1]
    f = synthetic.fourier_field(shape, 2 * np.pi, 6, 11, nmodes=16)
    g = synthetic.fourier_field(shape, 2 * np.pi, 6, 12, nmodes=16) if order == 6 else None
    u0 = np.zeros(shape) if order == 4 else np.full(shape, g.mean())
    out = {}
    for mode in ("graph", "host"):
        S = Solver(order, shape, h, p, 0.05, 0.15, 1.0, precision=precision, tol=1e-10, max_iter=3000,
                   max_outer=30)
        if mode == "host":
            S.profile(True)
        u = dev(u0)
        info = S.solve(dev(f), u, None if g is None else dev(g))
        assert info["status"] == 0 and info["res_l2"] < 1e-10
        out[mode] = (info, u)
        # a second solve replays the captured graph
        u2 = dev(u0)
        info2 = S.solve(dev(f), u2, None if g is None else dev(g))
        assert torch.equal(u, u2) and info2["iters"] == info["iters"]
        S.close()
    ig, ih = out["graph"][0], out["host"][0]
    assert (ig["iters"], ig["outer_iters"], ig["status"]) == (ih["iters"], ih["outer_iters"], ih["status"])
    assert ig["res_l2"] == ih["res_l2"]
    assert torch.equal(out["graph"][1], out["host"][1])


@pytest.mark.parametrize("precision", [PSD_FP64, PSD_MIXED])
def test_graph_cache_over_pointer_sets(precision):
    """A handle keeps the solve graphs of its last four (u, f, g) pointer
    sets: alternating two buffer sets, and cycling through six (more than
    the cache holds, so graphs are replaced), every solve gives the answer
    of a fresh handle bit for bit."""
    shape, order = (32, 32, 32), 6
    h = 2 * np.pi / shape[-1]
    f = synthetic.fourier_field(shape, 2 * np.pi, 6, 21, nmodes=16)
    g = synthetic.fourier_field(shape, 2 * np.pi, 6, 22, nmodes=16)
    u0 = np.full(shape, g.mean())
    kw = dict(precision=precision, tol=1e-10, max_iter=3000, max_outer=30)
    ref = Solver(order, shape, h, 4.0, 0.05, 0.15, 1.0, **kw)
    u_ref = dev(u0)
    info_ref = ref.solve(dev(f), u_ref, dev(g))
    ref.close()
    S = Solver(order, shape, h, 4.0, 0.05, 0.15, 1.0, **kw)
    sets = [(dev(f), dev(g), dev(u0)) for _ in range(6)]
    for k in [0, 1, 0, 1, 2, 3, 4, 5, 0, 1, 5]:
        fb, gb, ub = sets[k]
        ub.copy_(dev(u0))
        info = S.solve(fb, ub, gb)
        assert info["iters"] == info_ref["iters"] and info["res_l2"] == info_ref["res_l2"]
        assert torch.equal(ub, u_ref)
    S.close()
