"""Parity of the solver and estimate path (K3, K6, K7, K8, K9, K10) with the CPU oracle.

Bars: block solves to the block tolerance, the full solve to the outer tolerance (true FP64
residual), r and delta to 1e-10 relative, exponents e_j and log W to 1e-8 relative
(|d| <= 1e-8 max(|x|, 1)), noise to 1e-15 (same Philox integers, libm vs CUDA transcendental
rounding).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as oc
from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu

CASES = [
    # name, dims, l, eps, csw, m1, m2, nhit
    ("c1_4x4x4x4_l2", (4, 4, 4, 4), 2, 0.3, 1.0, 0.20, 0.19, 8),
    ("8x8x8x8_l4", (8, 8, 8, 8), 4, 0.25, 1.5, 0.10, 0.09, 2),
    ("12x12x12x12_l6", (12, 12, 12, 12), 6, 0.2, 1.9, 0.10, 0.08, 1),
]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def close(a, b, tol=1e-8):
    return abs(a - b) <= tol * max(abs(b), 1.0)


@pytest.fixture(scope="module", params=CASES, ids=lambda c: c[0])
def case(request):
    name, dims, l, eps, csw, m1, m2, nhit = request.param
    U = synth.gauge_field(dims, eps, seed=1)
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_params(csw, m1, m2)
    ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    lat = oc.Lattice(dims, (l,) * 4, U, csw)
    yield dict(ctx=ctx, lat=lat, dims=dims, m1=m1, m2=m2, nhit=nhit, l=l)
    ctx.close()


def test_noise_matches_oracle_philox(case):
    ctx = case["ctx"]
    eta = torch.zeros((3, ctx.nP, 4, 3), dtype=torch.complex128, device="cuda")
    ctx.noise(2, 5, 3, eta)
    want = oc.noise_packed(2, 5, 3, ctx.nP * 12).reshape(3, ctx.nP, 4, 3)
    assert np.max(np.abs(eta.cpu().numpy() - want)) < 1e-14
    # P has the size the oracle's projector has
    assert ctx.nP == len(case["lat"].suppP_sites())


@pytest.mark.parametrize("colour", [0, 1])
def test_block_solve(case, colour):
    ctx, lat, dims = case["ctx"], case["lat"], case["dims"]
    b = synth.spinor_field(dims, seed=31, nrhs=2)
    x = np.zeros_like(b)
    info = ctx.solve_block(colour, case["m2"], b, x, nrhs=2)
    col = lat.colour()
    for r in range(2):
        bc = b[r].copy()
        bc[col != colour] = 0
        res = bc - lat.apply(case["m2"], x[r], rows=colour, cols=colour)
        assert np.linalg.norm(res) / np.linalg.norm(bc) < 2e-13
        assert np.max(np.abs(x[r][col != colour])) == 0.0
    assert info["block_iters_max"] > 0


@pytest.mark.parametrize("max_rhs", [1, 3])
def test_chunked_estimates_agree_with_one_chunk(case, max_rhs):
    """The batched estimates split into chunks of at most max_rhs right-hand sides (one mass and
    some of its hits per chunk) give the one-chunk exponents and log W to the solver tolerance: the
    mass sweep of Eq. 3 over two target masses and the N = 2 interpolation of Eq. 8, FP16 storage."""
    ctx, m1, m2 = case["ctx"], case["m1"], case["m2"]
    m2s, nhit = [m2, 0.5 * (m1 + m2)], 4
    ctx.set_solver(binding.MIXED_FP16, tol_outer=1e-10, tol_block=1e-10)
    try:
        E0, L0, _, _ = ctx.estimate_masses(m2s, nhit, seed=13, hit_offset=2)
        I0 = ctx.estimate_interp(2, 2, seed=14, hit_offset=1)
        ctx.set_max_rhs(max_rhs)
        E1, L1, _, _ = ctx.estimate_masses(m2s, nhit, seed=13, hit_offset=2)
        I1 = ctx.estimate_interp(2, 2, seed=14, hit_offset=1)
    finally:
        ctx.set_max_rhs(0)
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    E0, E1 = np.asarray(E0).reshape(-1), np.asarray(E1).reshape(-1)
    assert np.all(np.abs(E1 - E0) <= 1e-8 * np.maximum(np.abs(E0), 1.0)), (E0, E1)
    for a, b in zip(np.asarray(L1).reshape(-1), np.asarray(L0).reshape(-1)):
        assert close(a, b)
    a, b = np.asarray(I1["exponents"]).reshape(-1), np.asarray(I0["exponents"]).reshape(-1)
    assert np.all(np.abs(a - b) <= 1e-8 * np.maximum(np.abs(b), 1.0))
    assert close(I1["logW"], I0["logW"])


@pytest.mark.parametrize("form", [0, 1, 2], ids=["nt", "2nt", "pairs"])
def test_block_solver_launch_shapes(case, form):
    """The persistent block solver in each launch shape (one right-hand side per CTA of NT or 2 NT
    threads, or pairs of right-hand sides per CTA sharing every link and clover load; blocks of at
    least 512 sites per parity, else the single shape), FP32 inner solves with FP64 defect
    correction, on 4 right-hand sides: the true residual of every block system by the oracle's block
    operator, nothing written outside the colour."""
    ctx, lat, dims = case["ctx"], case["lat"], case["dims"]
    ctx.set_solver(binding.MIXED_FP32, tol_outer=1e-10, tol_block=1e-12)
    ctx.block_config(form)
    try:
        b = synth.spinor_field(dims, seed=38, nrhs=4)
        x = np.zeros_like(b)
        info = ctx.solve_block(1, case["m1"], b, x, nrhs=4)
        col = lat.colour()
        for r in range(4):
            bc = b[r].copy()
            bc[col != 1] = 0
            res = bc - lat.apply(case["m1"], x[r], rows=1, cols=1)
            assert np.linalg.norm(res) / np.linalg.norm(bc) <= 1e-12, r
            assert np.max(np.abs(x[r][col != 1])) == 0.0
        assert info["block_iters_max"] > 0
    finally:
        ctx.block_config(-1)
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)


@pytest.mark.parametrize("form", [(1, 64, 1, 0), (1, 128, 1, 1), (1, 64, 1, 11)],
                         ids=["unrolled", "rolled", "fully_rolled"])
def test_mixed_block_solve_double_single_forms(case, form):
    """Mixed block solves (FP32 persistent kernel, FP64 defect correction) whose block-restricted
    double-single residuals run in the unrolled, the rolled and the fully rolled hop code: the true
    residual of every block system by the oracle's block operator."""
    ctx, lat, dims = case["ctx"], case["lat"], case["dims"]
    ctx.set_solver(binding.MIXED_FP32, tol_outer=1e-10, tol_block=1e-12)
    ctx.stencil_config(*form)
    try:
        b = synth.spinor_field(dims, seed=35, nrhs=2)
        x = np.zeros_like(b)
        ctx.solve_block(0, case["m2"], b, x, nrhs=2)
        col = lat.colour()
        for r in range(2):
            bc = b[r].copy()
            bc[col != 0] = 0
            res = bc - lat.apply(case["m2"], x[r], rows=0, cols=0)
            assert np.linalg.norm(res) / np.linalg.norm(bc) <= 1e-12
    finally:
        ctx.stencil_config(0)
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)


@pytest.mark.parametrize("prec", [binding.MIXED_FP16, binding.MIXED_BF16], ids=["fp16", "bf16"])
def test_16bit_krylov_block_solves_with_reliable_updates(case, prec):
    """16-bit block solves through the Krylov-loop BiCGStab on a colour's blocks with reliable
    updates into FP32: the true residual of every block system by the oracle's block operator,
    and the estimate through them against the oracle's chain."""
    ctx, lat, dims = case["ctx"], case["lat"], case["dims"]
    ctx.set_solver(prec, tol_outer=1e-10, tol_block=1e-12)
    ctx.set_low_precision(True, True)
    ctx.set_block_solver(1)
    try:
        b = synth.spinor_field(dims, seed=36, nrhs=2)
        col = lat.colour()
        for colour in (0, 1):
            x = np.zeros_like(b)
            info = ctx.solve_block(colour, case["m2"], b, x, nrhs=2)
            for r in range(2):
                bc = b[r].copy()
                bc[col != colour] = 0
                res = bc - lat.apply(case["m2"], x[r], rows=colour, cols=colour)
                assert np.linalg.norm(res) / np.linalg.norm(bc) <= 1e-12, (colour, r)
                assert np.max(np.abs(x[r][col != colour])) == 0.0
            assert info["block_iters_max"] > 0
        nhit = 1
        eta = oc.noise_packed(2, 8, nhit, ctx.nP * 12)
        e, _, _, _ = ctx.estimate(nhit, eta=torch.from_numpy(eta.reshape(nhit, ctx.nP, 4, 3)).cuda())
        want = lat.exponent(case["m1"], case["m2"], lat.unpack(eta[0]))["e"]
        assert close(e[0], want), (e[0], want)
    finally:
        ctx.set_block_solver(0)
        ctx.set_low_precision(True, False)
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)


@pytest.mark.parametrize("colour", [0, 1])
def test_block_solve_krylov_loop(case, colour):
    """Block solves through the graph-captured BiCGStab on all blocks of the colour at once (FP32
    inner solves, FP64 defect correction): the true residual of every block system by the oracle's
    block operator, and nothing written outside the colour."""
    ctx, lat, dims = case["ctx"], case["lat"], case["dims"]
    ctx.set_solver(binding.MIXED_FP32, tol_outer=1e-10, tol_block=1e-12)
    ctx.set_block_solver(1)
    try:
        b = synth.spinor_field(dims, seed=34, nrhs=2)
        x = np.zeros_like(b)
        info = ctx.solve_block(colour, case["m1"], b, x, nrhs=2)
        col = lat.colour()
        for r in range(2):
            bc = b[r].copy()
            bc[col != colour] = 0
            res = bc - lat.apply(case["m1"], x[r], rows=colour, cols=colour)
            assert np.linalg.norm(res) / np.linalg.norm(bc) <= 1e-12
            assert np.max(np.abs(x[r][col != colour])) == 0.0
        assert info["block_iters_max"] > 0
        # the estimate through these block solves against the oracle's chain
        nhit = 1
        eta = oc.noise_packed(2, 7, nhit, ctx.nP * 12)
        e, _, _, _ = ctx.estimate(nhit, eta=torch.from_numpy(eta.reshape(nhit, ctx.nP, 4, 3)).cuda())
        want = lat.exponent(case["m1"], case["m2"], lat.unpack(eta[0]))["e"]
        assert close(e[0], want), (e[0], want)
    finally:
        ctx.set_block_solver(0)
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)


def test_fused_inner_products(case):
    """The BiCGStab inner products fused into the stencil epilogue and in separate kernels give the
    same solves up to the rounding of the sums: both reach the outer tolerance by the oracle's
    operator and the exponents agree."""
    ctx, lat, dims = case["ctx"], case["lat"], case["dims"]
    ctx.set_solver(binding.MIXED_FP32, tol_outer=1e-10, tol_block=1e-12)
    try:
        b = synth.spinor_field(dims, seed=36, nrhs=2)
        e = {}
        for fuse in (True, False):
            ctx.fuse_reductions(fuse)
            x = np.zeros_like(b)
            ctx.solve_D(case["m2"], b, x, nrhs=2)
            for r in range(2):
                assert rel(lat.apply(case["m2"], x[r]), b[r]) <= 1e-10, (fuse, r)
            e[fuse], _, _, _ = ctx.estimate(1, seed=2, hit_offset=3)
        assert close(e[True][0], e[False][0], tol=1e-9)
    finally:
        ctx.fuse_reductions(False)
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)


@pytest.mark.parametrize("prec", [binding.MIXED_FP16, binding.MIXED_BF16], ids=["fp16", "bf16"])
def test_16bit_reliable_updates(case, prec):
    """16-bit Krylov vectors with reliable updates into FP32: the full solve reaches the outer
    tolerance by the oracle's operator in no more defect-correction cycles than FP32 storage needs
    (the plain 16-bit form restarts more often), with 16-bit and with FP32 block solves, and the
    estimate agrees with the oracle's exponents."""
    ctx, lat, dims = case["ctx"], case["lat"], case["dims"]
    b = synth.spinor_field(dims, seed=37, nrhs=2)
    try:
        cycles = {}
        for reliable, block16 in ((True, True), (True, False), (False, True)):
            ctx.set_solver(prec, tol_outer=1e-10, tol_block=1e-12)
            ctx.set_low_precision(reliable, block16)
            x = np.zeros_like(b)
            info = ctx.solve_D(case["m2"], b, x, nrhs=2)
            for r in range(2):
                assert rel(lat.apply(case["m2"], x[r]), b[r]) <= 1e-10, (reliable, block16, r)
            cycles[(reliable, block16)] = info["cycles"]
        assert cycles[(True, True)] <= 3 and cycles[(True, True)] <= cycles[(False, True)], cycles
        ctx.set_low_precision(True, True)
        nhit = 1
        eta = oc.noise_packed(2, 9, nhit, ctx.nP * 12)
        e, _, _, _ = ctx.estimate(nhit, eta=torch.from_numpy(eta.reshape(nhit, ctx.nP, 4, 3)).cuda())
        want = lat.exponent(case["m1"], case["m2"], lat.unpack(eta[0]))["e"]
        assert close(e[0], want), (e[0], want)
    finally:
        ctx.set_low_precision(True, False)
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)


def test_full_solve(case):
    ctx, lat, dims = case["ctx"], case["lat"], case["dims"]
    b = synth.spinor_field(dims, seed=32)
    x = np.zeros_like(b)
    info = ctx.solve_D(case["m2"], b, x)
    res = np.linalg.norm(b - lat.apply(case["m2"], x)) / np.linalg.norm(b)
    assert res <= 1e-10
    assert info["true_rel_residual"] <= 1e-10


def oracle_schur(lat, m, v_full):
    """A(m) v = v - P D_bb^-1 D_bw D_ww^-1 D_wb v from the oracle's operator and CGNR."""
    u = lat.apply(m, v_full, rows=oc.WHITE, cols=oc.BLACK)
    a, _, _ = lat.solve(m, u, sel=oc.WHITE, tol=1e-13)
    c = lat.apply(m, a, rows=oc.BLACK, cols=oc.WHITE)
    y, _, _ = lat.solve(m, c, sel=oc.BLACK, tol=1e-13)
    P = lat.suppP().astype(bool)
    out = v_full - y
    out[~P] = 0
    return out


def test_apply_schur(case):
    ctx, lat = case["ctx"], case["lat"]
    v = synth.complex_gaussian((1, ctx.nP, 4, 3), seed=33)
    out = np.zeros_like(v)
    ctx.apply_schur(case["m2"], v, out)
    want = lat.pack(oracle_schur(lat, case["m2"], lat.unpack(v[0].reshape(-1))))
    assert rel(out[0].reshape(-1), want) < 1e-11


def test_apply_schur_dagger(case):
    """A(m)^dag on supp P (Sec. 1, with D^dag = g5 D g5): <x, A y> = <A^dag x, y>, and on the 4^4
    lattice A^dag x equals the conjugate transpose of the oracle's dense A(m) applied to x."""
    ctx, lat = case["ctx"], case["lat"]
    m = case["m2"]
    x = synth.complex_gaussian((1, ctx.nP, 4, 3), seed=34)
    y = synth.complex_gaussian((1, ctx.nP, 4, 3), seed=35)
    ay = np.zeros_like(y)
    adx = np.zeros_like(x)
    ctx.apply_schur(m, y, ay)
    ctx.apply_schur(m, x, adx, dagger=True)
    lhs, rhs = np.vdot(x, ay), np.vdot(adx, y)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    if lat.V <= 256:
        from oracle import dense as od
        want = od.schur_on_P(lat, m).conj().T @ x.reshape(-1)
        assert rel(adx.reshape(-1), want) < 1e-11
        # and it is not A itself (the test is not vacuous)
        ax = np.zeros_like(x)
        ctx.apply_schur(m, x, ax)
        assert rel(ax.reshape(-1), want) > 1e-3


def test_dA_and_delta_and_exponent(case):
    """r = (A(m1) - A(m2)) eta, delta = A(m2)^-1 r and e_j against the oracle's own chain."""
    ctx, lat = case["ctx"], case["lat"]
    nhit = case["nhit"]
    eta = oc.noise_packed(2, 0, nhit, ctx.nP * 12)
    eta_t = torch.from_numpy(eta.reshape(nhit, ctx.nP, 4, 3)).cuda()
    r = torch.zeros_like(eta_t)
    ctx.apply_dA(eta_t, r, nrhs=nhit)
    delta = torch.zeros_like(eta_t)
    e, logw, relvar, info = ctx.estimate(nhit, eta=eta_t, delta=delta)
    r_h, d_h = r.cpu().numpy().reshape(nhit, -1), delta.cpu().numpy().reshape(nhit, -1)
    e_orc = []
    for j in range(nhit):
        res = lat.exponent(case["m1"], case["m2"], lat.unpack(eta[j]))
        assert rel(r_h[j], lat.pack(res["r"])) < 1e-10
        assert rel(d_h[j], lat.pack(res["delta"])) < 1e-8
        assert close(e[j], res["e"]), (j, e[j], res["e"])
        e_orc.append(res["e"])
    assert close(logw, oc.log_w(e_orc))
    assert info["true_rel_residual"] <= 1e-10
    assert info["iters_inner_total"] >= info["block_iters_max"] > 0


def test_estimate_with_own_noise_equals_estimate_with_passed_noise(case):
    ctx = case["ctx"]
    nhit = 2
    eta = torch.zeros((nhit, ctx.nP, 4, 3), dtype=torch.complex128, device="cuda")
    ctx.noise(7, 3, nhit, eta)
    e1, lw1, _, _ = ctx.estimate(nhit, seed=7, hit_offset=3)
    e2, lw2, _, _ = ctx.estimate(nhit, eta=eta)
    assert np.allclose(e1, e2, rtol=1e-12, atol=1e-14)


def test_zero_mass_shift():
    dims, l = (4, 4, 4, 8), 2
    U = synth.gauge_field(dims, 0.3, seed=2)
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(U)
    ctx.set_params(1.0, 0.15, 0.15)
    e, lw, _, _ = ctx.estimate(2)
    assert np.all(e == 0.0) and lw == 0.0
    ctx.close()


@pytest.mark.parametrize("prec", [binding.MIXED_FP32, binding.MIXED_FP16, binding.MIXED_BF16],
                         ids=["fp32", "fp16", "bf16"])
def test_mixed_precision_estimate_matches_fp64(case, prec):
    ctx = case["ctx"]
    nhit = min(case["nhit"], 4)
    e64, lw64, _, _ = ctx.estimate(nhit, seed=2)
    ctx.set_solver(prec, tol_outer=1e-10, tol_block=1e-12)
    try:
        e, lw, _, info = ctx.estimate(nhit, seed=2)
    finally:
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    for j in range(nhit):
        assert close(e[j], e64[j]), (j, e[j], e64[j])
    assert close(lw, lw64)
    assert info["true_rel_residual"] <= 1e-10


@pytest.mark.parametrize("prec", [binding.MIXED_FP32, binding.MIXED_FP16], ids=["fp32", "fp16"])
@pytest.mark.parametrize("cfg", [(1, 128, 1, 1), (4, 64, 1, 0), (2, 64, 2, 1), (1, 128, 1, 2), (1, 64, 1, 3),
                                 (1, 64, 1, 6), (2, 128, 1, 6), (1, 64, 2, 7)],
                         ids=["r1", "u4", "r2w2", "b4", "b8", "t1", "t2", "t1w2"])
def test_mixed_estimate_under_pinned_stencil_configs(case, prec, cfg):
    """The low-precision stencils in each pinned launch configuration lead to the FP64 result."""
    ctx = case["ctx"]
    nhit = min(case["nhit"], 4)
    e64, lw64, _, _ = ctx.estimate(nhit, seed=3)
    ctx.set_solver(prec, tol_outer=1e-10, tol_block=1e-12)
    ctx.stencil_config(*cfg)
    try:
        e, lw, _, info = ctx.estimate(nhit, seed=3)
    finally:
        ctx.stencil_config(0)
        ctx.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    for j in range(nhit):
        assert close(e[j], e64[j]), (j, e[j], e64[j])
    assert close(lw, lw64)
    assert info["true_rel_residual"] <= 1e-10


def test_batched_masses_match_single_mass_calls(case):
    ctx = case["ctx"]
    m1 = case["m1"]
    m2s = [m1 - 0.002, m1 - 0.005, m1 - 0.01]
    nhit = 2
    E, LW, RV, _ = ctx.estimate_masses(m2s, nhit, seed=4)
    for k, m2 in enumerate(m2s):
        ctx.set_params(ctx_csw(case), m1, m2)
        e, lw, _, _ = ctx.estimate(nhit, seed=4)
        assert np.allclose(E[k], e, rtol=1e-9, atol=1e-12)
        assert close(LW[k], lw, 1e-9)
    ctx.set_params(ctx_csw(case), m1, case["m2"])


def ctx_csw(case):
    return case["lat"].csw
