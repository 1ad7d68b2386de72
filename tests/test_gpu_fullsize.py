"""Parity at the benchmark's full size (64x32^3, 8^4 blocks, eps 0.2, csw 1.9): the FP64 operator
against the oracle over the whole lattice, the true residuals of a block solve and of the outer
solve measured with the oracle's operator, and the mixed-precision estimate against the FP64 path
on the same noise vector (the oracle's own solves at this size are out of reach in a test)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as oc
from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu

DIMS, L, EPS, CSW, M1, M2 = (64, 32, 32, 32), 8, 0.2, 1.9, 0.02, 0.015


@pytest.fixture(scope="module")
def full():
    U = synth.gauge_field(DIMS, EPS, seed=1)
    ctx = binding.Context(DIMS, (L,) * 4)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_params(CSW, M1, M2)
    lat = oc.Lattice(DIMS, (L,) * 4, U, CSW)
    yield ctx, lat
    ctx.close()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_operator_full_lattice(full):
    ctx, lat = full
    x = synth.spinor_field(DIMS, seed=71)
    y = torch.empty(x.shape, dtype=torch.complex128, device="cuda")
    ctx.apply_D(M2, torch.from_numpy(x).cuda(), y)
    assert rel(y.cpu().numpy(), lat.apply(M2, x)) < 1e-12


@pytest.mark.parametrize("prec", [binding.MIXED_FP32, binding.MIXED_FP16], ids=["fp32", "fp16"])
def test_solves_reach_their_true_residual(full, prec):
    ctx, lat = full
    ctx.set_solver(prec, tol_outer=1e-10, tol_block=1e-10)
    b = synth.spinor_field(DIMS, seed=72)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    ctx.solve_D(M2, bt, x)
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - lat.apply(M2, xh)) / np.linalg.norm(b) <= 1e-10
    xb = torch.zeros_like(bt)
    ctx.solve_block(0, M1, bt, xb)
    col = lat.colour()
    bc = b.copy()
    bc[col != 0] = 0
    res = bc - lat.apply(M1, xb.cpu().numpy(), rows=0, cols=0)
    assert np.linalg.norm(res) / np.linalg.norm(bc) <= 1e-10


@pytest.mark.parametrize("prec", [binding.MIXED_FP32, binding.MIXED_FP16], ids=["fp32", "fp16"])
def test_mixed_estimate_matches_fp64_at_full_size(full, prec):
    ctx, lat = full
    ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    e64, lw64, _, _ = ctx.estimate(1, seed=2, hit_offset=0)
    ctx.set_solver(prec, tol_outer=1e-10, tol_block=1e-10)
    e32, lw32, _, info = ctx.estimate(1, seed=2, hit_offset=0)
    assert abs(e32[0] - e64[0]) <= 1e-8 * max(abs(e64[0]), 1.0)
    assert abs(lw32 - lw64) <= 1e-8 * max(abs(lw64), 1.0)
    assert info["true_rel_residual"] <= 1e-10
