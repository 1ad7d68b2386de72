"""Mass interpolation (Eq. 8) and the one-flavour estimator (Eq. 11) on the GPU against the oracle:
each factor's exponents e_ij with its own noise, the complex one-flavour exponents <eta, delta>,
and the assembled log W, log |W_1f| and root-trick values."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as oc
from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def close(a, b, tol=1e-8):
    return abs(a - b) <= tol * max(abs(b), 1.0)


@pytest.mark.parametrize("dims,l", [((4, 4, 4, 4), 2), ((8, 8, 8, 8), 4)])
def test_interpolation_and_one_flavour_match_oracle(dims, l):
    U = synth.gauge_field(dims, 0.3, seed=1)
    m1, m2, N, nhit, hit0 = 0.20, 0.14, 3, 2, 5
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(U)
    ctx.set_params(1.0, m1, m2)
    ctx.set_solver(binding.FP64, tol_outer=1e-11, tol_block=1e-13)
    out = ctx.estimate_interp(N, nhit, seed=2, hit_offset=hit0)
    lat = oc.Lattice(dims, (l,) * 4, U, 1.0)
    ms = [(i / N) * m2 + ((N - i) / N) * m1 for i in range(N + 1)]
    logw, logw1, sign = 0.0, 0.0, 1.0
    for i in range(1, N + 1):
        eta = oc.noise_packed(2, hit0 + (i - 1) * nhit, nhit, 12 * ctx.nP)
        e, e1 = [], []
        for j in range(nhit):
            res = lat.exponent(ms[i - 1], ms[i], lat.unpack(eta[j]), tol_block=1e-13, tol_outer=1e-11)
            e.append(res["e"])
            e1.append(np.vdot(eta[j], lat.pack(res["delta"])))
            assert close(out["exponents"][i - 1, j], res["e"]), (i, j)
            assert abs(out["exponents_1f"][i - 1, j] - e1[-1]) <= 1e-8 * max(abs(e1[-1]), 1.0), (i, j)
        logw += oc.log_w(e)
        X = np.exp(-np.array(e1))  # Eq. 12's sample form: E|X|^2 - |E X|^2 over |E X|^2
        want_rv1 = np.sum(np.abs(X - X.mean()) ** 2) / (nhit - 1) / abs(X.mean()) ** 2
        assert abs(out["rel_var_1f"][i - 1] - want_rv1) <= 1e-6 * max(want_rv1, 1e-12), (i, want_rv1)
        f1 = np.mean(np.exp(-np.array(e1))).real
        logw1 += np.log(abs(f1))
        sign *= np.sign(f1)
    assert close(out["logW"], logw)
    assert close(out["logW_1f"], logw1)
    assert out["sign_1f"] == sign
    assert close(out["logW_root"], 0.5 * logw)
    ctx.close()


def test_one_step_interpolation_is_the_plain_estimate():
    dims, l = (8, 8, 8, 8), 4
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(synth.gauge_field(dims, 0.25, seed=3))
    ctx.set_params(1.5, 0.10, 0.09)
    out = ctx.estimate_interp(1, 4, seed=7, hit_offset=11)
    e, lw, _, _ = ctx.estimate(4, seed=7, hit_offset=11)
    assert np.allclose(out["exponents"][0], e, rtol=1e-12, atol=1e-14)
    assert close(out["logW"], lw, 1e-12)
    ctx.close()
