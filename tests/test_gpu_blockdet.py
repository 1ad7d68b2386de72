"""Parity of the block determinants of Eq. 7 (csrc/blockdet.cu) with the oracle (oracle/blockdet.py).

Bars: log |det D_k(m)| per block to 1e-10 absolute (the values are O(100): about 1e-12 relative),
equal signs; the block factor log prod_k det D_k^2(m2) / det D_k^2(m1) to 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blockdet as ob
from oracle import core as oc
from paper_1211_1214_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def make(dims, l, eps, csw, m1, m2, seed=1, U=None):
    U = synth.gauge_field(dims, eps, seed=seed) if U is None else U
    ctx = binding.Context(dims, (l,) * 4)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_params(csw, m1, m2)
    return ctx, oc.Lattice(dims, (l,) * 4, U, csw)


def test_block_logdets_4x4x4x4_l2():
    ctx, lat = make((4, 4, 4, 4), 2, 0.3, 1.0, 0.20, 0.19)
    for m in (0.20, 0.19, -0.3):
        ld, sg = ctx.block_logdet(m)
        ld_o, sg_o = ob.block_logdets(lat, m)
        assert np.max(np.abs(ld - ld_o)) < 1e-10
        assert np.array_equal(sg, np.real(sg_o).round())
    assert abs(ctx.block_factor() - ob.log_block_factor(lat, 0.20, 0.19)) < 1e-9
    ctx.close()


def test_block_logdets_8x8x8x8_l4():
    """4^4 blocks (the 16^4 configuration's block size): Schur complements of dimension 1536."""
    ctx, lat = make((8, 8, 8, 8), 4, 0.25, 1.5, 0.05, 0.045)
    ld, sg = ctx.block_logdet(0.045)
    ld_o, sg_o = ob.block_logdets(lat, 0.045)
    assert np.max(np.abs(ld - ld_o)) < 1e-10 * max(1.0, np.max(np.abs(ld_o)))
    assert np.array_equal(sg, np.real(sg_o).round())
    ctx.close()


def test_block_factor_is_gauge_invariant_and_vanishes_at_equal_masses():
    dims, l = (8, 8, 8, 8), 4
    U = synth.gauge_field(dims, 0.25, seed=5)
    g = synth.gauge_transform(dims, seed=6)
    X = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1).reshape(-1, 4)
    Ug = np.empty_like(U)
    for mu in range(4):
        Y = X.copy()
        Y[:, mu] = (Y[:, mu] + 1) % dims[mu]
        ym = ((Y[:, 0] * dims[1] + Y[:, 1]) * dims[2] + Y[:, 2]) * dims[3] + Y[:, 3]
        Ug[:, mu] = g @ U[:, mu] @ g[ym].conj().transpose(0, 2, 1)
    ctx, _ = make(dims, l, 0.25, 1.5, 0.05, 0.045, U=U)
    ctxg, _ = make(dims, l, 0.25, 1.5, 0.05, 0.045, U=Ug)
    f, fg = ctx.block_factor(), ctxg.block_factor()
    assert abs(f - fg) < 1e-9 * max(1.0, abs(f))
    # a lighter target mass moves every eigenvalue (real part above dm / 2) towards zero, so the
    # block determinants shrink and the factor is below one
    assert f < 0
    ctx.set_params(1.5, 0.05, 0.05)
    assert ctx.block_factor() == 0.0
    ctx.close()
    ctxg.close()


def test_block_determinants_refuse_large_blocks():
    ctx = binding.Context((16, 16, 16, 16), (8, 8, 8, 8))
    ctx.load_gauge(synth.gauge_field((16, 16, 16, 16), 0.2, seed=1))
    ctx.set_params(1.0, 0.1, 0.09)
    with pytest.raises(binding.DDRWError) as ei:
        ctx.block_factor()
    assert ei.value.status == 1
    ctx.close()
