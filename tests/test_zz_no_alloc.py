"""ddrw_solve_block_noalloc: the block solve for callers that cannot allocate device memory.

It must agree with ddrw_solve_block on two calls in a row (its scratch array keeps the previous
call's contents, so the second call checks that everything that must start at zero is cleared),
and refuse what its fixed scratch cannot serve.  Collected last so that a stop at the first
failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def ctx():
    dims, l = (8, 8, 8, 16), 4
    c = binding.Context(dims, (l,) * 4)
    c.load_gauge(torch.from_numpy(synth.gauge_field(dims, 0.25, seed=1)).cuda())
    c.set_params(1.5, 0.05, 0.045)
    c.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    yield c, dims
    c.close()


def test_two_calls_match_the_allocating_entry_point(ctx):
    c, dims = ctx
    for call, (colour, m, seed) in enumerate([(0, 0.045, 41), (1, 0.05, 42)]):
        b = torch.from_numpy(synth.spinor_field(dims, seed=seed)).cuda()
        x_ref = torch.zeros_like(b)
        c.solve_block(colour, m, b, x_ref)
        x = torch.full_like(b, float("nan"))
        info = c.solve_block_noalloc(colour, m, b, x)
        assert info["true_rel_residual"] <= 1e-13, (call, info)
        assert rel(x.cpu().numpy(), x_ref.cpu().numpy()) < 1e-11, call


def test_rejects_what_the_scratch_cannot_serve(ctx):
    c, dims = ctx
    b = torch.from_numpy(synth.spinor_field(dims, seed=43)).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(binding.DDRWError, match="m1 or m2"):
        c.solve_block_noalloc(0, 0.123, b, x)
    with pytest.raises(binding.DDRWError, match="device pointers"):
        c.solve_block_noalloc(0, 0.045, b.cpu().numpy(), x)
    big_dims = (16, 16, 16, 16)
    big = binding.Context(big_dims, (4,) * 4)
    try:
        big.load_gauge(torch.from_numpy(synth.gauge_field(big_dims, 0.25, seed=1)).cuda())
        big.set_params(1.5, 0.05, 0.045)
        bb = torch.zeros((int(np.prod(big_dims)), 4, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(binding.DDRWError, match="at most 20736 sites"):
            big.solve_block_noalloc(0, 0.045, bb, torch.zeros_like(bb))
    finally:
        big.close()


def test_non_finite_right_hand_side_is_an_error(ctx):
    c, dims = ctx
    b = torch.from_numpy(synth.spinor_field(dims, seed=44)).cuda()
    b[3, 1, 2] = complex(float("nan"), 0.0)
    x = torch.zeros_like(b)
    with pytest.raises(binding.DDRWError, match="non-finite"):
        c.solve_block_noalloc(0, 0.045, b, x)


def test_calls_allocate_no_device_memory():
    """On a fresh context (no allocating solve before it), after one warm-up call, further calls
    leave the device's free memory unchanged: no cudaMalloc and no allocating library routine."""
    dims, l = (8, 8, 8, 8), 4
    c = binding.Context(dims, (l,) * 4)
    try:
        c.load_gauge(torch.from_numpy(synth.gauge_field(dims, 0.25, seed=2)).cuda())
        c.set_params(1.5, 0.05, 0.045)
        c.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
        bs = [torch.from_numpy(synth.spinor_field(dims, seed=50 + k)).cuda() for k in range(3)]
        xs = [torch.zeros_like(b) for b in bs]
        for colour in (0, 1):  # warm-up: first launches of each shape (stencil autotuning)
            c.solve_block_noalloc(colour, 0.045, bs[0], xs[0])
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        c.solve_block_noalloc(1, 0.05, bs[1], xs[1])
        c.solve_block_noalloc(0, 0.05, bs[2], xs[2])
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
    finally:
        c.close()
