"""CUDA graphs (the outer Krylov loop; whole estimate chunks with device-controlled cycles) and the
stencil autotuner: same results with and without them, and the graph path is actually taken."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    dims, l = (16, 16, 16, 16), 4
    c = binding.Context(dims, (l,) * 4)
    c.load_gauge(torch.from_numpy(synth.gauge_field(dims, 0.25, seed=1)).cuda())
    c.set_params(1.5, 0.05, 0.045)
    yield c, dims
    c.close()


@pytest.mark.parametrize("prec", [binding.MIXED_FP32, binding.FP64])
def test_graph_and_eager_krylov_loops_agree(ctx, prec):
    c, dims = ctx
    c.set_solver(prec, tol_outer=1e-10, tol_block=1e-12)
    b = torch.from_numpy(synth.spinor_field(dims, seed=61, nrhs=3)).cuda()
    xs = []
    for graphs in (False, True):
        c.use_graphs(graphs)
        n0 = c.use_graphs()
        x = torch.zeros_like(b)
        info = c.solve_D(0.045, b, x, nrhs=3)
        assert info["true_rel_residual"] <= 1e-10
        xs.append(x.cpu().numpy())
        if graphs:
            assert c.use_graphs() > n0  # the loop ran as a graph
    assert np.array_equal(xs[0], xs[1])
    c.use_graphs(2)  # the default mode


def test_estimate_same_with_graphs_and_without(ctx):
    c, dims = ctx
    c.set_solver(binding.MIXED_FP32, tol_outer=1e-10, tol_block=1e-12)
    c.use_graphs(False)
    e0, lw0, _, _ = c.estimate(4, seed=3)
    c.use_graphs(2)
    e1, lw1, _, _ = c.estimate(4, seed=3)
    assert np.array_equal(e0, e1)


def test_autotuner_off_gives_the_same_numbers(ctx):
    c, dims = ctx
    c.set_solver(binding.MIXED_FP32, tol_outer=1e-10, tol_block=1e-12)
    c.autotune(True)
    e0, _, _, _ = c.estimate(2, seed=4)
    report = c.autotune_report()
    assert "nr=" in report
    c.autotune(False)
    e1, _, _, _ = c.estimate(2, seed=4)
    c.autotune(True)
    # a different launch shape changes only the order of nothing: each site's arithmetic is the same
    assert np.allclose(e0, e1, rtol=1e-9)


@pytest.mark.parametrize("prec", [binding.MIXED_FP32, binding.FP64, binding.MIXED_FP16], ids=["fp32", "fp64", "fp16"])
def test_whole_estimate_graph_replays_the_eager_estimate(ctx, prec):
    """The second call of a chunk shape captures the whole estimate (noise, the four block solves,
    the outer solve, the reductions) as one graph with device-controlled loops; later calls replay
    it.  Same seeds give bit-identical exponents to the host-controlled path, for fresh noise on
    every replay, and the replay counts the kernels its loops ran.  16-bit storage: this mode runs
    the plain inner solves (no reliable updates) on all its calls, so the host-controlled reference
    runs them too; the reliable-update estimate agrees with it to the solver tolerance."""
    c, dims = ctx
    c.set_solver(prec, tol_outer=1e-10, tol_block=1e-12)
    m2s = [0.045, 0.04]
    c.use_graphs(False)
    if prec == binding.MIXED_FP16:
        rel_ref = c.estimate_masses(m2s, 3, seed=11)[0]
        c.set_low_precision(False)
    ref = [c.estimate_masses(m2s, 3, seed=s)[0] for s in (11, 12, 13)]
    c.set_low_precision(True)
    if prec == binding.MIXED_FP16:
        a, b = np.asarray(rel_ref), np.asarray(ref[0])
        assert np.all(np.abs(a - b) <= 1e-8 * np.maximum(np.abs(b), 1.0))
    c.use_graphs(1)
    n0 = c.use_graphs()
    c.profile(True)
    try:
        got = [c.estimate_masses(m2s, 3, seed=s) for s in (11, 12, 13)]  # eager, capture + replay, replay
        launches = c.profile_read(binding.PROF_LAUNCHES)[0]
    finally:
        c.profile(False)
        n1 = c.use_graphs(2)
    assert n1 >= n0 + 2  # two replays of the whole estimate (plus Krylov-loop graphs)
    for (e, lw, rv, info), e_ref in zip(got, ref):
        assert np.array_equal(np.asarray(e), np.asarray(e_ref))
        assert info["true_rel_residual"] <= 1e-10
    assert not np.array_equal(np.asarray(got[1][0]), np.asarray(got[2][0]))  # new noise per replay
    assert launches > 1000


def test_krylov_only_graph_mode_gives_the_same_estimate_without_whole_chunk_graphs(ctx):
    """Mode 2 (Krylov-loop graphs, host-driven cycles) gives the eager numbers bitwise on repeated
    calls; an unknown mode is refused."""
    c, dims = ctx
    m2s = [0.045, 0.04]
    c.set_solver(binding.MIXED_FP32, tol_outer=1e-10, tol_block=1e-10)
    try:
        c.use_graphs(False)
        ref = c.estimate_masses(m2s, 3, seed=21)[0]
        c.use_graphs(2)
        got = [c.estimate_masses(m2s, 3, seed=21)[0] for _ in range(3)]
    finally:
        c.use_graphs(2)
        c.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    for e in got:
        assert np.array_equal(np.asarray(e), np.asarray(ref))
    with pytest.raises(binding.DDRWError) as ei:
        c.use_graphs(3)
    assert ei.value.status == 1


@pytest.mark.parametrize("mode", [2, 1], ids=["krylov_graphs", "whole_estimate_graphs"])
def test_new_configuration_reuses_graphs_and_inverses(mode):
    """A context that loads a second gauge field (host buffer, as an ensemble loop does) and then
    sets the same parameters again keeps its captured graphs and the addresses of its in-block
    inverses, whose contents are recomputed: its estimate on the second field is bit-identical to
    that of a fresh context on that field, and a changed target mass is picked up."""
    dims, l, m2s = (8, 8, 8, 16), 4, [0.045, 0.04]
    U1 = synth.gauge_field(dims, 0.25, seed=1)
    U2 = synth.gauge_field(dims, 0.25, seed=2)
    a = binding.Context(dims, (l,) * 4)
    b = binding.Context(dims, (l,) * 4)
    try:
        for c in (a, b):
            c.set_solver(binding.MIXED_FP16, tol_outer=1e-10, tol_block=1e-12)
            c.use_graphs(mode)
        a.load_gauge(U1)
        a.set_params(1.5, 0.05, m2s[0])
        for _ in range(3):  # eager, captured, replayed
            a.estimate_masses(m2s, 2, seed=5)
        n0 = a.use_graphs()
        a.load_gauge(U2)
        a.set_params(1.5, 0.05, m2s[0])  # unchanged: no rebuild
        e_a = [a.estimate_masses(m2s, 2, seed=s)[0] for s in (6, 7, 8)]
        b.load_gauge(U2)
        b.set_params(1.5, 0.05, m2s[0])
        e_b = [b.estimate_masses(m2s, 2, seed=s)[0] for s in (6, 7, 8)]
        for x, y in zip(e_a, e_b):
            assert np.array_equal(np.asarray(x), np.asarray(y))
        assert a.use_graphs() > n0  # the graphs captured on the first field were replayed
        # a new m1 rebuilds the inverses: the same as a fresh context with that m1
        a.set_params(1.5, 0.06, m2s[0])
        b.set_params(1.5, 0.06, m2s[0])
        ea = np.asarray(a.estimate_masses(m2s, 2, seed=9)[0])
        c = binding.Context(dims, (l,) * 4)
        try:
            c.set_solver(binding.MIXED_FP16, tol_outer=1e-10, tol_block=1e-12)
            c.use_graphs(mode)
            c.load_gauge(U2)
            c.set_params(1.5, 0.06, m2s[0])
            ec = np.asarray(c.estimate_masses(m2s, 2, seed=9)[0])
        finally:
            c.close()
        assert np.allclose(ea, ec, rtol=1e-9, atol=1e-12)
    finally:
        a.close()
        b.close()
