"""The adjoint (K11) on the GPU: link force and mass derivative of the exponents against the
oracle's analytic force, against central finite differences of the GPU estimate, in FP64 and
mixed precision, and through the torch.autograd.Function."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as oc
from paper_1211_1214_gb300 import autograd, binding, synth

pytestmark = pytest.mark.gpu


def perturb(U, omega, t):
    X = np.einsum("lna,aij->lnij", omega, synth.gell_mann() / 2.0).reshape(-1, 3, 3)
    E = synth._expm_i_traceless_hermitian(t * X).reshape(U.shape)
    return np.einsum("lnij,lnjk->lnik", E, U)


@pytest.mark.parametrize("dims,l,eps,csw,m1,m2", [((4, 4, 4, 4), 2, 0.3, 1.0, 0.20, 0.17),
                                                  ((8, 8, 8, 8), 4, 0.25, 1.5, 0.10, 0.09)])
def test_force_matches_oracle(dims, l, eps, csw, m1, m2):
    U = synth.gauge_field(dims, eps, seed=1)
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(U)
    ctx.set_params(csw, m1, m2)
    ctx.set_solver(binding.FP64, tol_outer=1e-13, tol_block=1e-14)
    lat = oc.Lattice(dims, (l,) * 4, U, csw)
    eta = oc.noise_packed(2, 0, 1, 12 * ctx.nP)
    dU = np.zeros((ctx.V, 4, 8))
    e, dm2, _ = ctx.force(1, eta=eta.reshape(1, ctx.nP, 4, 3).copy(), dU=dU)
    e_o, dU_o, dm2_o = lat.force(m1, m2, lat.unpack(eta[0]), tol_block=1e-14, tol_outer=1e-13)
    assert abs(e[0] - e_o) <= 1e-9 * max(abs(e_o), 1)
    assert np.linalg.norm(dU - dU_o) <= 1e-8 * np.linalg.norm(dU_o)
    assert abs(dm2[0] - dm2_o) <= 1e-8 * max(abs(dm2_o), 1e-3)
    ctx.close()


@pytest.fixture(scope="module")
def c5():
    """16^4, 4^4 blocks, eps 0.25, csw 1.5, m1 0.05, m2 0.045, N_hit 4."""
    dims, l = (16, 16, 16, 16), 4
    U = synth.gauge_field(dims, 0.25, seed=1)
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(U)
    ctx.set_params(1.5, 0.05, 0.045)
    yield ctx, U, dims
    ctx.close()


def fd_exponent_sum(ctx, U, omega, h, w, nhit):
    """central difference of sum_j w_j e_j along omega, with FP64 solves to 1e-13 / 1e-14"""
    vals = []
    ctx.set_solver(binding.FP64, tol_outer=1e-13, tol_block=1e-14)
    for t in (+h, -h):
        ctx.load_gauge(perturb(U, omega, t))
        ctx.set_params(1.5, 0.05, 0.045)
        e, _, _, _ = ctx.estimate(nhit, seed=2)
        vals.append(float(np.dot(w, e)))
    ctx.load_gauge(U)
    ctx.set_params(1.5, 0.05, 0.045)
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("prec", [binding.FP64, binding.MIXED_FP32])
def test_c5_force_against_finite_differences(c5, prec):
    ctx, U, dims = c5
    nhit = 4
    w = np.array([1.0, 0.5, -0.25, 2.0])
    tol = dict(tol_outer=1e-13, tol_block=1e-14) if prec == binding.FP64 else dict(tol_outer=1e-11, tol_block=1e-12)
    ctx.set_solver(prec, **tol)
    dU = torch.zeros((ctx.V, 4, 8), dtype=torch.float64, device="cuda")
    e, dm2, _ = ctx.force(nhit, seed=2, weights=w, dU=dU)
    F = dU.cpu().numpy()
    rng = np.random.default_rng(1000)
    ndir = 64 if prec == binding.FP64 else 8
    h = 1e-5
    bad = []
    for k in range(ndir):
        omega = rng.standard_normal((ctx.V, 4, 8))
        fd = fd_exponent_sum(ctx, U, omega, h, w, nhit)
        an = float(np.sum(omega * F))
        if abs(fd - an) > 1e-6 * max(abs(an), 1.0):
            bad.append((k, fd, an))
    assert not bad, bad[:4]
    # mass derivative (FP64 solves for the difference quotient)
    ctx.set_solver(binding.FP64, tol_outer=1e-13, tol_block=1e-14)
    vals = []
    for m2 in (0.045 + h, 0.045 - h):
        ctx.set_params(1.5, 0.05, m2)
        ee, _, _, _ = ctx.estimate(nhit, seed=2)
        vals.append(ee)
    ctx.set_params(1.5, 0.05, 0.045)
    fd_m = (vals[0] - vals[1]) / (2 * h)
    assert np.allclose(dm2, fd_m, rtol=1e-6, atol=1e-6 * np.abs(fd_m).max())
    # the analytic force of the mixed path matches its FP64 force, so the difference quotients in
    # FP64 pin both


def test_mixed_force_matches_fp64(c5):
    ctx, U, dims = c5
    outs = []
    for prec, tol in ((binding.FP64, (1e-13, 1e-14)), (binding.MIXED_FP32, (1e-10, 1e-12)),
                      (binding.MIXED_FP16, (1e-10, 1e-12))):
        ctx.set_solver(prec, tol_outer=tol[0], tol_block=tol[1])
        dU = torch.zeros((ctx.V, 4, 8), dtype=torch.float64, device="cuda")
        e, dm2, _ = ctx.force(2, seed=5, dU=dU)
        outs.append((e, dm2, dU.cpu().numpy()))
    e0, m0, F0 = outs[0]
    for e1, m1, F1 in outs[1:]:
        assert np.allclose(e1, e0, rtol=1e-8)
        assert np.allclose(m1, m0, rtol=1e-7)
        assert np.linalg.norm(F1 - F0) <= 1e-7 * np.linalg.norm(F0)


def test_autograd_function(c5):
    ctx, U, dims = c5
    ctx.set_solver(binding.FP64, tol_outer=1e-12, tol_block=1e-13)
    omega = torch.zeros((ctx.V, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    m2 = torch.tensor(0.045, dtype=torch.float64, requires_grad=True)
    e = autograd.exponents(ctx, omega, m2, nhit=2, seed=9)
    w = torch.tensor([0.3, -1.2], dtype=torch.float64, device="cuda")
    (e * w).sum().backward()
    dU = torch.zeros((ctx.V, 4, 8), dtype=torch.float64, device="cuda")
    e2, dm2, _ = ctx.force(2, seed=9, weights=w.cpu().numpy(), dU=dU)
    assert torch.allclose(e.detach().cpu(), torch.from_numpy(e2), rtol=1e-12)
    assert torch.allclose(omega.grad, dU, rtol=1e-10, atol=1e-14)
    assert abs(m2.grad.item() - float(np.dot(w.cpu().numpy(), dm2))) <= 1e-10 * max(1.0, abs(m2.grad.item()))
