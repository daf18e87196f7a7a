"""The adjoint (gradients of a loss of the converged solution) through the
C ABI and the torch.autograd.Function, against the CPU oracle's adjoint,
against central finite differences, and the Hessian-vector product kernel
against the oracle's second variation."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01475_gb300 import PSD_FP64, PSD_MIXED, Solver, synthetic  # noqa: E402
from paper_1607_01475_gb300.autograd import psd_solve_autograd  # noqa: E402

rng = np.random.default_rng(99)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("shape,p", [((64, 64), 4.0), ((16, 16, 16), 4.0), ((32, 32, 64), 4.0),
                                     ((8, 16, 32), 3.0), ((1024, 1024), 4.0)])
def test_hvp_parity(oracle, shape, p):
    h = 2 * np.pi / shape[-1]
    P = oracle.Problem(4, h, p, 0.07, 0.15)
    u = rng.standard_normal(shape) * 0.3
    v = rng.standard_normal(shape)
    S = Solver(4, shape, h, p, P.s, P.eps)
    y = torch.empty(shape, dtype=torch.float64, device="cuda")
    dot = S.hvp(dev(u), dev(v), y)
    ref = oracle.hvp4(u, v, P)
    assert rel(y.cpu().numpy(), ref) <= 1e-12
    assert abs(dot - h ** len(shape) * np.sum(v * ref)) <= 1e-10 * abs(dot)


@pytest.mark.parametrize("precision", [PSD_FP64, PSD_MIXED])
@pytest.mark.parametrize("shape", [(32, 32), (16, 16, 16), (32, 32, 64)])
def test_adjoint_matches_oracle(oracle, shape, precision):
    """dJ/df and dJ/ds of the device-resident CG (FP64, or FP32 inner CG with
    FP64 outer residual correction) against the oracle's adjoint at 1e-9."""
    h = 2 * np.pi / shape[-1]
    s, eps = 0.05, 0.15
    P = oracle.Problem(4, h, 4.0, s, eps)
    f = synthetic.fourier_field(shape, 2 * np.pi, 6, 77, nmodes=16)
    ut = synthetic.fourier_field(shape, 2 * np.pi, 6, 78, nmodes=16)
    u, _ = oracle.psd_solve(P, f, np.zeros(shape), tol=0.0, kmax=150)
    hd = h ** len(shape)
    gu = hd * (u - ut)
    gf_ref, gs_ref, _ = oracle.adjoint4(u, gu, P)
    S = Solver(4, shape, h, 4.0, s, eps, precision=precision)
    gf = torch.empty(shape, dtype=torch.float64, device="cuda")
    gs, info = S.adjoint(dev(u), dev(gu), gf, tol_rel=1e-13, max_iter=2000)
    assert info["status"] == 0 and info["res_l2"] <= 1e-13
    assert rel(gf.cpu().numpy(), gf_ref) <= 1e-9
    assert abs(gs - gs_ref) <= 1e-9 * abs(gs_ref)
    # a second call on the same handle (replayed CG graphs) gives the same bits
    gf2 = torch.empty_like(gf)
    gs2, _ = S.adjoint(dev(u), dev(gu), gf2, tol_rel=1e-13, max_iter=2000)
    assert torch.equal(gf, gf2) and gs == gs2


def test_adjoint_aliasing_and_zero_rhs(oracle):
    """grad_f may alias grad_u; a zero dJ/du gives zero gradients."""
    shape = (16, 16, 16)
    h = 2 * np.pi / 16
    P = oracle.Problem(4, h, 4.0, 0.05, 0.15)
    f = synthetic.fourier_field(shape, 2 * np.pi, 6, 91, nmodes=16)
    u, _ = oracle.psd_solve(P, f, np.zeros(shape), tol=0.0, kmax=150)
    gu = rng.standard_normal(shape)
    gf_ref, _, _ = oracle.adjoint4(u, gu, P)
    for prec in (PSD_FP64, PSD_MIXED):
        S = Solver(4, shape, h, 4.0, P.s, P.eps, precision=prec)
        g = dev(gu)
        S.adjoint(dev(u), g, g, tol_rel=1e-13)
        assert rel(g.cpu().numpy(), gf_ref) <= 1e-9
        z = torch.zeros(shape, dtype=torch.float64, device="cuda")
        out = torch.full_like(z, 5.0)
        gs, info = S.adjoint(dev(u), z, out)
        assert info["status"] == 0 and gs == 0.0 and bool((out == 0).all())


def test_adjoint_gradient_by_central_differences_and_autograd():
    """J = 1/2 h^d sum (u - u_t)^2: torch.autograd through PSDSolve against
    central differences (step 1e-6) of J through forward solves run to the
    FP64 floor."""
    shape = (32, 32, 32)
    h = 2 * np.pi / 32
    eps = 0.1
    f0 = dev(synthetic.fourier_field(shape, 2 * np.pi, 6, 81, nmodes=16))
    ut = dev(synthetic.fourier_field(shape, 2 * np.pi, 6, 82, nmodes=16))
    hd = h ** 3

    def J(f, s):
        u = psd_solve_autograd(f, s, h, 4.0, eps, tol=1e-13, max_iter=5000)
        return 0.5 * hd * torch.sum((u - ut) ** 2)

    f = f0.clone().requires_grad_(True)
    s = torch.tensor(0.05, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = J(f, s)
    gf, gs = torch.autograd.grad(loss, (f, s))
    t = 1e-6
    with torch.no_grad():
        for k in range(3):
            v = dev(rng.standard_normal(shape))
            fd = (J(f0 + t * v, 0.05) - J(f0 - t * v, 0.05)).item() / (2 * t)
            an = torch.sum(gf * v).item()
            assert abs(fd - an) <= 2e-5 * abs(an), (k, fd, an)
        fds = (J(f0, 0.05 + t) - J(f0, 0.05 - t)).item() / (2 * t)
        assert abs(fds - gs.item()) <= 2e-5 * abs(gs.item())


@pytest.mark.parametrize("precision", [PSD_FP64, PSD_MIXED])
def test_adjoint_full_size_128cubed(precision):
    """The adjoint workload: 3D 128^3, p=4, s=0.1, eps=0.05 (thin-film shaped
    f), J = 1/2 h^3 sum (u - u_t)^2; the adjoint solve converges and the
    directional derivative along a random direction matches central
    differences of J."""
    shape = (128, 128, 128)
    wl = synthetic.workload_thin_film(shape)
    h = wl["L"] / 128
    ut = dev(synthetic.fourier_field(shape, wl["L"], 8, synthetic.seed_for(4, 0, 2)))
    f0 = dev(wl["f"])
    hd = h ** 3
    S = Solver(4, shape, h, 4.0, wl["s"], wl["eps"], precision=precision, tol=1e-11, max_iter=5000, max_outer=30)

    def solve(f):
        u = torch.zeros_like(f)
        S.solve(f, u)
        return u

    u = solve(f0)
    gf = torch.empty_like(u)
    gs, info = S.adjoint(u, hd * (u - ut), gf, tol_rel=1e-12, max_iter=3000)
    assert info["status"] == 0
    v = dev(rng.standard_normal(shape))
    t = 1e-5
    Jp = 0.5 * hd * torch.sum((solve(f0 + t * v) - ut) ** 2).item()
    Jm = 0.5 * hd * torch.sum((solve(f0 - t * v) - ut) ** 2).item()
    fd = (Jp - Jm) / (2 * t)
    an = torch.sum(gf * v).item()
    assert abs(fd - an) <= 1e-4 * abs(an)


def test_mixed_adjoint_matches_fp64_at_128cubed():
    """The mixed adjoint (FP32 inner CG, FP64 outer correction) agrees with
    the FP64 adjoint to 1e-9 on the 128^3 adjoint workload."""
    shape = (128, 128, 128)
    wl = synthetic.workload_thin_film(shape)
    h = wl["L"] / 128
    ut = dev(synthetic.fourier_field(shape, wl["L"], 8, synthetic.seed_for(4, 0, 2)))
    S64 = Solver(4, shape, h, 4.0, wl["s"], wl["eps"], tol=1e-11, max_iter=5000)
    u = torch.zeros_like(ut)
    S64.solve(dev(wl["f"]), u)
    gu = h ** 3 * (u - ut)
    out = {}
    for prec in (PSD_FP64, PSD_MIXED):
        S = Solver(4, shape, h, 4.0, wl["s"], wl["eps"], precision=prec)
        gf = torch.empty_like(u)
        gs, info = S.adjoint(u, gu, gf, tol_rel=1e-12, max_iter=3000)
        assert info["status"] == 0
        out[prec] = (gf.cpu().numpy(), gs)
    assert rel(out[PSD_MIXED][0], out[PSD_FP64][0]) <= 1e-9
    assert abs(out[PSD_MIXED][1] - out[PSD_FP64][1]) <= 1e-9 * abs(out[PSD_FP64][1])
