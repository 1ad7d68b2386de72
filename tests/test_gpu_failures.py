"""Failure detection without a GPU fault: every failure is made on the host (bad arguments,
an iteration cap of 1, NaN in a host input buffer) or is a bounded device-side wait that a test
switch lets run out, and must come back as a status code with a message, leaving the context
usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    dims, l = (8, 8, 8, 8), 4
    c = binding.Context(dims, (l,) * 4)
    c.load_gauge(synth.gauge_field(dims, 0.25, seed=1))
    c.set_params(1.5, 0.05, 0.045)
    yield c, dims
    c.close()


def test_iteration_cap_reports_no_convergence_and_fills_outputs(ctx):
    c, dims = ctx
    c.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13, maxiter=1)
    b = synth.spinor_field(dims, seed=81)
    x = np.zeros_like(b)
    with pytest.raises(binding.DDRWError) as ei:
        c.solve_D(0.045, b, x)
    assert ei.value.status == 4  # DDRW_ENOCONV
    assert np.linalg.norm(x) > 0  # the last iterate is returned
    c.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13, maxiter=20000)
    info = c.solve_D(0.045, b, x)  # the context still works
    assert info["true_rel_residual"] <= 1e-10


def test_nan_in_a_host_input_is_reported(ctx):
    c, dims = ctx
    c.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    b = synth.spinor_field(dims, seed=82)
    b[17, 2, 1] = np.nan
    x = np.zeros_like(b)
    with pytest.raises(binding.DDRWError) as ei:
        c.solve_D(0.045, b, x)
    assert ei.value.status in (4, 5)  # no convergence or a non-finite reduction
    b2 = synth.spinor_field(dims, seed=83)
    assert c.solve_D(0.045, b2, x)["true_rel_residual"] <= 1e-10


def test_bad_arguments(ctx):
    c, dims = ctx
    b = synth.spinor_field(dims, seed=84)
    with pytest.raises(binding.DDRWError) as ei:
        c.solve_block(2, 0.045, b, np.zeros_like(b))  # colour must be black or white
    assert ei.value.status == 1
    with pytest.raises(binding.DDRWError) as ei:
        c.set_solver(9)  # no such precision
    assert ei.value.status == 1
    with pytest.raises(binding.DDRWError) as ei:
        c.estimate_interp(9, 2)  # at most 8 interpolation steps
    assert ei.value.status == 1
    for cfg in [(2, 64, 1, 7), (4, 64, 1, 6), (2, 64, 1, 4), (1, 64, 1, 12), (2, 64, 1, 11), (2, 64, 1, 8), (1, 256, 1, 8),
                (2, 64, 1, 9), (2, 128, 1, 10), (1, 48, 1, 0), (1, 256, 2, 0)]:
        with pytest.raises(binding.DDRWError) as ei:
            c.stencil_config(*cfg)  # form, right-hand sides per thread or CTA shape out of range
        assert ei.value.status == 1
    for form in (-2, 3):
        with pytest.raises(binding.DDRWError) as ei:
            c.block_config(form)  # no such block-solver launch shape
        assert ei.value.status == 1
    with pytest.raises(binding.DDRWError) as ei:
        c.set_max_rhs(-1)  # chunks hold at least one right-hand side (0: from free memory)
    assert ei.value.status == 1
    st = c.L.ddrw_apply_D(c._h, 0.1, None, None, 1)
    assert st == 1
    assert b"bad argument" in c.L.ddrw_last_error(c._h)


def test_calls_before_a_gauge_field_are_refused():
    c = binding.Context((4, 4, 4, 4), (2, 2, 2, 2))
    b = synth.spinor_field((4, 4, 4, 4), seed=85)
    with pytest.raises(binding.DDRWError) as ei:
        c.apply_D(0.1, b, np.zeros_like(b))
    assert ei.value.status == 7  # DDRW_ESTATE
    c.close()


def test_empty_and_oversized_requests_are_refused(ctx):
    c, dims = ctx
    b = synth.spinor_field(dims, seed=86)
    assert c.L.ddrw_apply_D(c._h, 0.1, b.ctypes.data, b.ctypes.data, 0) == 1      # nrhs = 0
    with pytest.raises(binding.DDRWError) as ei:
        c.estimate(0)                                                            # no noise vectors
    assert ei.value.status == 1
    with pytest.raises(binding.DDRWError) as ei:
        c.estimate_masses([0.04] * 9, 2)                                         # at most 8 mass slots
    assert ei.value.status == 1
    with pytest.raises(binding.DDRWError) as ei:
        c.estimate_variant(3, 1, 2)                                              # no such operator variant
    assert ei.value.status == 1


def test_eight_mass_slots_in_one_pass(ctx):
    """The largest batch of target masses (8 slots) agrees with single-mass estimates."""
    c, dims = ctx
    c.set_solver(binding.FP64, tol_outer=1e-10, tol_block=1e-13)
    m2s = [0.045 - 0.002 * k for k in range(8)]
    e, lw, _, _ = c.estimate_masses(m2s, 2, seed=4)
    e = np.asarray(e).reshape(8, 2)
    for k in (0, 7):
        c.set_params(1.5, 0.05, m2s[k])
        e1, _, _, _ = c.estimate(2, seed=4)
        assert np.all(np.abs(e[k] - e1) <= 1e-8 * np.maximum(np.abs(e1), 1.0))
    c.set_params(1.5, 0.05, 0.045)


def test_staged_stencil_wait_runs_out_and_the_context_recovers(ctx):
    """The staged stencil's shared-memory barrier is told to expect 16 bytes that never arrive: every
    CTA stops polling after its bounded number of tries, sets the device error flag and returns; the
    call reports DDRW_ETIMEOUT, and with the switch off the same context computes the right result."""
    c, dims = ctx
    x = synth.spinor_field(dims, seed=85, nrhs=2)
    y = np.zeros_like(x)
    c.stencil_config(1, 64, 2, 8)
    try:
        c.test_stall_staging(True)
        with pytest.raises(binding.DDRWError) as ei:
            c.apply_D_low(binding.MIXED_FP32, 0.07, x, y, nrhs=2)
        assert ei.value.status == 8
        c.test_stall_staging(False)
        c.apply_D_low(binding.MIXED_FP32, 0.07, x, y, nrhs=2)
    finally:
        c.test_stall_staging(False)
        c.stencil_config(0)
    ref = np.zeros_like(x)
    c.apply_D(0.07, x, ref, nrhs=2)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 2e-6
