"""Parity of the operator variants of Fig. 1's comparison (ddrw_estimate_variant) with the dense
oracle: the total operator Mh = D(m_i)^-1 D(m_{i-1}), the even-odd Schur complement and the block
Schur complement, each with mass interpolation (Eq. 8).  Bar: exponents 1e-8 max(|e|, 1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as oc
from oracle import dense as od
from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu

DIMS, L, EPS, CSW, M1, M2 = (4, 4, 4, 4), 2, 0.3, 1.0, 0.20, 0.15


@pytest.fixture(scope="module")
def setup():
    U = synth.gauge_field(DIMS, EPS, seed=1)
    ctx = binding.Context(DIMS, (L,) * 4)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_params(CSW, M1, M2)
    ctx.set_solver(binding.FP64, tol_outer=1e-12, tol_block=1e-13)
    lat = oc.Lattice(DIMS, (L,) * 4, U, CSW)
    yield ctx, lat
    ctx.close()


def masses(N):
    return [((N - i) * M1 + i * M2) / N for i in range(N + 1)]


def support(lat, variant):
    if variant == 0:
        return np.arange(12 * lat.V)
    return od.even_components(lat)


@pytest.mark.parametrize("variant", [0, 1], ids=["total", "even_odd"])
@pytest.mark.parametrize("N", [1, 2])
def test_variant_exponents_match_the_dense_oracle(setup, variant, N):
    ctx, lat = setup
    nhit = 3
    dim = len(support(lat, variant))
    eta = synth.complex_gaussian((N, nhit, dim), seed=40 + N + 10 * variant)
    e, lw, rv, d, info = ctx.estimate_variant(variant, N, nhit, eta=eta)
    assert d == dim
    m = masses(N)
    ratio = od.ratio_matrix_total if variant == 0 else od.ratio_matrix_eo
    lw_o = 0.0
    for i in range(N):
        e_o = od.exponent(ratio(lat, m[i], m[i + 1]), eta[i])
        assert np.all(np.abs(e[i] - e_o) <= 1e-8 * np.maximum(np.abs(e_o), 1.0)), (i, e[i], e_o)
        lw_o += np.log(np.mean(np.exp(-e_o)))
    assert abs(lw - lw_o) <= 1e-8 * max(abs(lw_o), 1.0)


def test_block_variant_is_the_interpolated_estimate(setup):
    ctx, lat = setup
    e, lw, rv, d, _ = ctx.estimate_variant(2, 2, 4, seed=7)
    assert d == 12 * len(lat.suppP_sites())
    r = ctx.estimate_interp(2, 4, seed=7)
    assert np.array_equal(e, r["exponents"])
    assert lw == r["logW"]


def test_philox_noise_of_the_total_variant(setup):
    """Without caller noise the support components come from Philox (component index in the
    lexicographic packed order): the same exponents as with that noise passed explicitly."""
    ctx, lat = setup
    e, _, _, dim, _ = ctx.estimate_variant(0, 1, 2, seed=9, hit_offset=5)
    eta = oc.noise_packed(9, 5, 2, dim)
    e2, _, _, _, _ = ctx.estimate_variant(0, 1, 2, eta=eta.reshape(1, 2, dim))
    assert np.all(np.abs(e - e2) <= 1e-10 * np.maximum(np.abs(e2), 1.0))
