"""Parity of the CUDA operator kernels (K1, K2, K4, K5) against the CPU oracle, through the C ABI.

Bar: 1e-12 relative (2-norm over the whole lattice) for a single FP64 application.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as oc
from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu

GEOMS = [
    # dims, block, eps, csw
    ((4, 4, 4, 4), 2, 0.3, 1.0),
    ((8, 4, 4, 12), 2, 0.25, 1.5),
    ((8, 8, 8, 16), 4, 0.25, 1.5),
    ((12, 12, 12, 24), 6, 0.2, 1.9),
    ((16, 16, 16, 16), 8, 0.2, 1.9),
]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module", params=GEOMS, ids=lambda g: "x".join(map(str, g[0])) + f"_l{g[1]}")
def setup(request):
    dims, l, eps, csw = request.param
    U = synth.gauge_field(dims, eps, seed=1)
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_params(csw, 0.05, 0.045)
    lat = oc.Lattice(dims, (l,) * 4, U, csw)
    yield ctx, lat, dims
    ctx.close()


@pytest.mark.parametrize("m", [0.045, -0.3])
def test_apply_D_fp64(setup, m):
    ctx, lat, dims = setup
    x = synth.spinor_field(dims, seed=5)
    y = torch.empty(x.shape, dtype=torch.complex128, device="cuda")
    ctx.apply_D(m, torch.from_numpy(x).cuda(), y)
    assert rel(y.cpu().numpy(), lat.apply(m, x)) < 1e-12


def test_apply_D_host_pointers_and_multi_rhs(setup):
    ctx, lat, dims = setup
    x = synth.spinor_field(dims, seed=6, nrhs=3)
    y = np.zeros_like(x)
    ctx.apply_D(0.1, x, y, nrhs=3)
    for r in range(3):
        assert rel(y[r], lat.apply(0.1, x[r])) < 1e-12


@pytest.mark.parametrize("form", [None, (1, 64, 1, 0), (1, 128, 1, 1), (1, 64, 1, 11)],
                         ids=["tuned", "unrolled", "rolled", "fully_rolled"])
@pytest.mark.parametrize("m", [0.045, -0.3])
def test_apply_D_double_single(setup, m, form):
    """The double-single stencil of the mixed defect correction: FP32 pairs carry ~48 significant
    bits and each two-sum / two-product loses a few units of 2^-48, so the result must sit within
    1e-12 of the oracle's FP64 operator -- five orders below what FP32 arithmetic could give; in
    the tuned launch form and pinned to the unrolled, the rolled and the fully rolled hop code."""
    ctx, lat, dims = setup
    x = synth.spinor_field(dims, seed=7, nrhs=2)
    y = np.zeros_like(x)
    if form:
        ctx.stencil_config(*form)
    try:
        ctx.apply_D_ds(m, x, y, nrhs=2)
    finally:
        ctx.stencil_config(0)
    for r in range(2):
        assert rel(y[r], lat.apply(m, x[r])) < 1e-12


@pytest.mark.parametrize("nr,nt,nw,roll", [(1, 64, 1, 0), (1, 64, 1, 1), (2, 128, 1, 0), (2, 128, 2, 1),
                                           (4, 32, 2, 0), (4, 256, 1, 1), (1, 32, 8, 1), (1, 128, 1, 2),
                                           (1, 64, 2, 3), (1, 256, 1, 4), (1, 128, 2, 5),
                                           (2, 128, 1, 5), (1, 64, 1, 6), (2, 128, 1, 6), (1, 128, 2, 7),
                                           (1, 64, 1, 9), (1, 128, 1, 10)])
def test_every_stencil_configuration(setup, nr, nt, nw, roll):
    """Each pinned launch configuration of the all-hop stencil (right-hand sides per thread, CTA
    shape, hop code form, computed or tabulated neighbours) gives the oracle's operator on 4
    right-hand sides."""
    ctx, lat, dims = setup
    x = synth.spinor_field(dims, seed=9, nrhs=4)
    y = np.zeros_like(x)
    ctx.stencil_config(nr, nt, nw, roll)
    try:
        ctx.apply_D(0.07, x, y, nrhs=4)
    finally:
        ctx.stencil_config(0)
    for r in range(4):
        assert rel(y[r], lat.apply(0.07, x[r])) < 1e-12


# relative error bound of one storage-precision stencil launch against the FP64 oracle: the input,
# links and clover terms are rounded to the storage (FP32 2^-24, FP16 with a per-site scale 2^-11,
# BF16 2^-8 relative per component), the arithmetic is FP32; a wrong hop, link or clover term
# gives errors of order 1e-1
LOW_TOL = {binding.MIXED_FP32: 2e-6, binding.MIXED_FP16: 3e-3, binding.MIXED_BF16: 2e-2}


def ainv_apply(lat, m, v):
    """A(m)^-1 v site by site, A(m) = (4 + m) + C(x) from the oracle's clover matrices."""
    out = np.empty_like(v)
    for x in range(v.shape[0]):
        out[x] = np.linalg.solve(lat.clover(x) + (4 + m) * np.eye(12), v[x].reshape(12)).reshape(4, 3)
    return out


@pytest.mark.parametrize("post", [False, True], ids=["D", "AinvD"])
@pytest.mark.parametrize("prec,cfg", [(binding.MIXED_FP32, None), (binding.MIXED_FP32, (1, 64, 1, 5)),
                                      (binding.MIXED_FP32, (2, 128, 1, 0)), (binding.MIXED_FP32, (1, 64, 1, 6)),
                                      (binding.MIXED_FP32, (1, 64, 4, 8)), (binding.MIXED_FP32, (1, 128, 2, 8)),
                                      (binding.MIXED_FP32, (1, 32, 8, 8)), (binding.MIXED_FP16, None),
                                      (binding.MIXED_FP16, (1, 64, 1, 6)), (binding.MIXED_FP16, (1, 64, 4, 8)),
                                      (binding.MIXED_BF16, None), (binding.MIXED_FP32, (1, 64, 1, 9)),
                                      (binding.MIXED_FP32, (1, 128, 2, 10)), (binding.MIXED_FP32, (1, 32, 8, 9)),
                                      (binding.MIXED_FP16, (1, 64, 1, 9))],
                         ids=["s-tuned", "s-f5", "s-u2", "s-table", "s-staged64x4", "s-staged128x2",
                              "s-staged32x8", "h-tuned", "h-table", "h-staged-falls-back", "b-tuned",
                              "s-pipe64", "s-pipe128x2", "s-pipe32x8", "h-pipe-falls-back"])
def test_apply_D_in_storage_precision(setup, prec, cfg, post):
    """One stencil launch in FP32 / FP16 / BF16 storage, in each launch form (computed or tabulated
    neighbours, links and clover terms staged in shared memory by bulk copies), against the oracle's
    D(m) and A(m)^-1 D(m) on 3 right-hand sides (fewer than some forms' right-hand-side rows)."""
    ctx, lat, dims = setup
    x = synth.spinor_field(dims, seed=11, nrhs=3)
    y = np.zeros_like(x)
    if cfg:
        ctx.stencil_config(*cfg)
    try:
        ctx.apply_D_low(prec, 0.07, x, y, nrhs=3, post=post)
    finally:
        ctx.stencil_config(0)
    for r in range(3):
        ref = lat.apply(0.07, x[r])
        if post:
            ref = ainv_apply(lat, 0.07, ref)
        assert rel(y[r], ref) < LOW_TOL[prec], (r, rel(y[r], ref))


@pytest.mark.parametrize("rows,cols", [(0, 0), (1, 1), (0, 1), (1, 0), (2, 0), (1, 2)])
def test_apply_block(setup, rows, cols):
    ctx, lat, dims = setup
    x = synth.spinor_field(dims, seed=7)
    y = torch.empty(x.shape, dtype=torch.complex128, device="cuda")
    ctx.apply_block(rows, cols, 0.045, torch.from_numpy(x).cuda(), y)
    ref = lat.apply(0.045, x, rows=rows, cols=cols)
    assert rel(y.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("cfg", [(1, 64, 1, 9), (1, 128, 2, 10), (1, 64, 1, 6)], ids=["pipe", "pipe3", "table"])
def test_antiperiodic_time_fp32_forms(cfg):
    """The time-boundary sign in the FP32 forms that read it from the neighbour table (one launch in
    FP32 storage against the oracle's operator)."""
    dims, l = (8, 4, 4, 4), 2
    U = synth.gauge_field(dims, 0.3, seed=3)
    ctx = binding.Context(dims, (l,) * 4)
    try:
        ctx.load_gauge(torch.from_numpy(U).cuda())
        ctx.set_params(1.2, 0.1, 0.09, antiperiodic_t=True)
        lat = oc.Lattice(dims, (l,) * 4, U, 1.2, antiperiodic_t=True)
        x = synth.spinor_field(dims, seed=8, nrhs=2)
        y = np.zeros_like(x)
        ctx.stencil_config(*cfg)
        ctx.apply_D_low(binding.MIXED_FP32, 0.1, x, y, nrhs=2)
        for r in range(2):
            assert rel(y[r], lat.apply(0.1, x[r])) < LOW_TOL[binding.MIXED_FP32]
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg", [None, (1, 64, 1, 6), (1, 64, 1, 7)], ids=["tuned", "table128", "table85"])
def test_antiperiodic_time(cfg):
    """Antiperiodic time boundary: the sign of the hops across t = T-1 -> 0, also in the forms that
    read the time-boundary bit from the neighbour table."""
    dims, l = (8, 4, 4, 4), 2
    U = synth.gauge_field(dims, 0.3, seed=3)
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_params(1.2, 0.1, 0.09, antiperiodic_t=True)
    lat = oc.Lattice(dims, (l,) * 4, U, 1.2, antiperiodic_t=True)
    x = synth.spinor_field(dims, seed=8)
    y = np.zeros_like(x)
    if cfg:
        ctx.stencil_config(*cfg)
    ctx.apply_D(0.1, x, y)
    assert rel(y, lat.apply(0.1, x)) < 1e-12
    # the same context back to periodic: the table does not depend on the boundary condition
    ctx.set_params(1.2, 0.1, 0.09, antiperiodic_t=False)
    ctx.apply_D(0.1, x, y)
    assert rel(y, oc.Lattice(dims, (l,) * 4, U, 1.2).apply(0.1, x)) < 1e-12
    ctx.close()


def test_free_field_plane_wave_on_gpu():
    """U = 1: the GPU operator reproduces the closed form of the free Wilson operator."""
    dims, l = (8, 8, 4, 12), 2
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(U)
    ctx.set_params(1.0, 0.1, 0.1)
    X = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), axis=-1).reshape(-1, 4)
    p = 2 * np.pi * np.array([1, 3, 1, 5]) / np.array(dims)
    chi = synth.complex_gaussian((4, 3), seed=4)
    psi = np.exp(1j * X @ p)[:, None, None] * chi[None]
    y = np.zeros_like(psi)
    m = 0.1
    ctx.apply_D(m, psi, y)
    g = [oc.gamma(mu) for mu in range(4)]
    Dp = (m + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
    want = np.exp(1j * X @ p)[:, None, None] * (Dp @ chi)[None]
    assert np.max(np.abs(y - want)) < 1e-13
    ctx.close()
