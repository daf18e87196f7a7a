"""Batched solves of many independent, uneven instances (psd_batch_*):
each instance against the CPU oracle and bitwise against the same solve on
a single handle, and the 96-instance workload end to end."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01475_gb300 import PSD_FP64, PSD_MIXED, Batch, Solver, synthetic  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _small_instances():
    shapes = [(16, 16), (32, 32), (64, 64), (32, 64), (16, 16, 16), (64, 32)]
    out = []
    for i, sh in enumerate(shapes):
        out.append(dict(order=4, shape=sh, h=2 * np.pi / sh[-1], p=3.0 if i % 2 else 4.0,
                        s=0.01 * (1 + i), eps=0.1 + 0.02 * i))
    return out


@pytest.mark.parametrize("precision", [PSD_FP64, PSD_MIXED])
def test_batch_matches_oracle_and_single_handle(oracle, precision):
    insts = _small_instances()
    fs = [synthetic.fourier_field(it["shape"], 2 * np.pi, 6, 500 + i, nmodes=16) for i, it in enumerate(insts)]
    tol = 1e-11
    B = Batch([dict(it, precision=precision, tol=tol, max_iter=3000) for it in insts], workers=3)
    us = [torch.zeros(it["shape"], dtype=torch.float64, device="cuda") for it in insts]
    infos = B.solve([dev(f) for f in fs], us)
    assert B.mode() == 1  # one graph launch for the whole batch
    for mode in (2, 3):  # the other schedules give the same bits
        B.set_mode(mode)
        us_m = [torch.zeros_like(u) for u in us]
        B.solve([dev(f) for f in fs], us_m)
        assert B.mode() == mode and all(torch.equal(a, b) for a, b in zip(us, us_m))
    B.set_mode(0)
    for i, (it, f, u, info) in enumerate(zip(insts, fs, us, infos)):
        assert info["status"] == 0 and info["res_l2"] < tol
        P = oracle.Problem(4, it["h"], it["p"], it["s"], it["eps"])
        ref, _ = oracle.psd_solve(P, f, np.zeros(it["shape"]), tol=0.0, kmax=200)
        assert rel(u.cpu().numpy(), ref) <= (1e-11 if precision == PSD_FP64 else 1e-9), i
        S = Solver(4, it["shape"], it["h"], it["p"], it["s"], it["eps"], precision=precision, tol=tol,
                   max_iter=3000)
        S.autotune()  # the batch tunes its mixed instances: same tiles, same reduction order
        u1 = torch.zeros_like(u)
        S.solve(dev(f), u1)
        assert torch.equal(u1, u), i


def test_batch_workload_96_instances(oracle):
    """The 96-instance uneven 2D workload (64^2 .. 1024^2, p in {3, 4}) in
    mixed precision: every instance converges to its own tolerance (1e-10,
    or its FP64 rounding floor where larger); for a sample of instances the
    oracle's FP64 residual of the returned iterate agrees."""
    wl = synthetic.workload_batch(96)
    insts = [dict(order=4, shape=w["shape"], h=w["L"] / w["shape"][-1], p=w["p"], s=w["s"], eps=w["eps"],
                  precision=PSD_MIXED, tol=w["tol"], max_iter=20000, max_outer=40) for w in wl]
    B = Batch(insts)
    fs = [dev(w["f"]) for w in wl]
    us = [torch.zeros(w["shape"], dtype=torch.float64, device="cuda") for w in wl]
    infos = B.solve(fs, us)
    bad = [(k, i["status"], i["res_l2"], w["tol"]) for k, (i, w) in enumerate(zip(infos, wl))
           if i["status"] != 0 or not i["res_l2"] < w["tol"]]
    assert not bad, bad
    assert sum(w["tol"] == 1e-10 for w in wl) >= 40  # most instances at the plain 1e-10 target
    for k in (0, 17, 50, 95):
        w = wl[k]
        P = oracle.Problem(4, w["L"] / w["shape"][-1], w["p"], w["s"], w["eps"])
        r = oracle.residual4(us[k].cpu().numpy(), w["f"], P)
        assert oracle.norm2(r, P.h) < 1.05 * w["tol"] + 1e-12, k


def test_batch_poisoned_instance_fails_alone():
    """Fault injection on the host: one instance's f carries a NaN.  That
    instance reports PSD_ERR_NONFINITE (7), the batch returns that status and
    names the instance, and every other instance still converges."""
    insts = _small_instances()
    fs = [synthetic.fourier_field(it["shape"], 2 * np.pi, 6, 500 + i, nmodes=16) for i, it in enumerate(insts)]
    fs[2][1, 1] = np.nan
    B = Batch([dict(it, precision=PSD_FP64, tol=1e-10, max_iter=3000) for it in insts], workers=3)
    us = [torch.zeros(it["shape"], dtype=torch.float64, device="cuda") for it in insts]
    status, msg, infos = B.solve([dev(f) for f in fs], us, check=False)
    assert status == 7 and "instance 2" in msg
    for i, info in enumerate(infos):
        if i == 2:
            assert info["status"] == 7
        else:
            assert info["status"] == 0 and info["res_l2"] < 1e-10, i


def test_batch_graph_replays_and_recaptures():
    """The batch graph is replayed for the same arrays (bitwise the same
    answers) and captured again for new arrays."""
    insts = _small_instances()
    fs = [dev(synthetic.fourier_field(it["shape"], 2 * np.pi, 6, 600 + i, nmodes=16)) for i, it in enumerate(insts)]
    B = Batch([dict(it, precision=PSD_MIXED, tol=1e-10, max_iter=3000) for it in insts])
    us = [torch.zeros(it["shape"], dtype=torch.float64, device="cuda") for it in insts]
    B.solve(fs, us)
    first = [u.clone() for u in us]
    for u in us:
        u.zero_()
    B.solve(fs, us)
    assert B.mode() == 1 and all(torch.equal(a, b) for a, b in zip(first, us))
    us2 = [torch.zeros_like(u) for u in us]
    infos = B.solve(fs, us2)
    assert B.mode() == 1 and all(torch.equal(a, b) for a, b in zip(first, us2))
    assert all(i["status"] == 0 and i["res_l2"] < 1e-10 and i["wall_ms"] > 0 for i in infos)
