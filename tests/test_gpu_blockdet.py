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


# ---- the nested decomposition of large blocks (Sec. 2.2, caption of Fig. 2)

def test_nested_block_factor_parts_match_the_oracle():
    """8^4 lattice, blocks of length 4 decomposed into 2^4 sub-blocks: the exact sub-block part
    against the oracle's dense sub-block determinants, the exponents of the stochastic Schur part
    against the oracle's five-solve chain on the Dirichlet-cut operator (same Philox noise), and the
    stochastic part is the log-sum-exp of those exponents."""
    dims, l, eps, csw, m1, m2, nhit, seed = (8, 8, 8, 8), 4, 0.25, 1.5, 0.10, 0.08, 3, 5
    U = synth.gauge_field(dims, eps, seed=1)
    ctx, _ = make(dims, l, eps, csw, m1, m2, U=U)
    try:
        ctx.set_solver(binding.FP64, tol_outer=1e-12, tol_block=1e-13)
        tot, ex, sto, e, rv = ctx.block_factor_nested(2, nhit, seed=seed)
        cut2 = ob.dirichlet_lattice(dims, (2,) * 4, U, csw, cut=l)
        assert abs(ex - ob.log_block_factor(cut2, m1, m2)) <= 1e-9 * max(1.0, abs(ex))
        nP = len(cut2.suppP_sites())
        eta = oc.noise_packed(seed, 0, nhit, 12 * nP)
        for j in range(nhit):
            want = cut2.exponent(m1, m2, cut2.unpack(eta[j]))["e"]
            assert abs(e[j] - want) <= 1e-8 * max(abs(want), 1.0), (j, e[j], want)
        assert abs(sto - oc.log_w(e)) <= 1e-12 * max(1.0, abs(sto))
        assert abs(tot - (ex + sto)) <= 1e-12 * max(1.0, abs(tot))
    finally:
        ctx.close()


def test_nested_block_factor_estimates_the_exact_block_factor():
    """Where the exact factor of Eq. 7 is computable (4^4 blocks) the nested estimate (2^4
    sub-blocks exact, the blocks' Schur complements by Eq. 3) agrees with it within its
    statistical error."""
    dims, l, eps, csw, m1, m2, nhit = (8, 8, 8, 8), 4, 0.25, 1.5, 0.10, 0.095, 64
    ctx, _ = make(dims, l, eps, csw, m1, m2)
    try:
        ctx.set_solver(binding.MIXED_FP32, tol_outer=1e-10, tol_block=1e-12)
        exact = ctx.block_factor()
        tot, ex, sto, e, rv = ctx.block_factor_nested(2, nhit, seed=9)
        sigma = np.sqrt(rv / nhit)
        assert abs(tot - exact) <= 5 * sigma + 1e-6, (tot, exact, sigma)
        assert abs(ex - exact) > 5 * sigma + 1e-6  # without the Schur part the check would fail
    finally:
        ctx.close()


def test_nested_block_factor_8x8x8x8_blocks_of_a_16x16x16x16_lattice():
    """8^4 blocks (the 64x32^3 block size) decomposed into 4^4 sub-blocks: the exponents of the
    Schur part against the oracle on the Dirichlet-cut operator; the sub-block part equals the
    exact factor of a context with 4^4 blocks (whose parity with the oracle is tested above)."""
    dims, l, eps, csw, m1, m2, nhit, seed = (16, 16, 16, 16), 8, 0.2, 1.9, 0.05, 0.045, 1, 3
    U = synth.gauge_field(dims, eps, seed=1)
    ctx, _ = make(dims, l, eps, csw, m1, m2, U=U)
    ctx4, _ = make(dims, 4, eps, csw, m1, m2, U=U)
    try:
        ctx.set_solver(binding.FP64, tol_outer=1e-12, tol_block=1e-13)
        tot, ex, sto, e, rv = ctx.block_factor_nested(4, nhit, seed=seed)
        assert abs(ex - ctx4.block_factor()) <= 1e-10 * max(1.0, abs(ex))
        cut4 = ob.dirichlet_lattice(dims, (4,) * 4, U, csw, cut=l)
        nP = len(cut4.suppP_sites())
        eta = oc.noise_packed(seed, 0, nhit, 12 * nP)
        want = cut4.exponent(m1, m2, cut4.unpack(eta[0]))["e"]
        assert abs(e[0] - want) <= 1e-8 * max(abs(want), 1.0), (e[0], want)
    finally:
        ctx.close()
        ctx4.close()


def test_dirichlet_cut_is_validated():
    ctx = binding.Context((8, 8, 8, 8), (4,) * 4)
    try:
        with pytest.raises(binding.DDRWError):
            ctx.set_dirichlet(6)  # not a multiple of the block length
        ctx.set_dirichlet(8)
        ctx.load_gauge(torch.from_numpy(synth.gauge_field((8, 8, 8, 8), 0.2, seed=1)).cuda())
        with pytest.raises(binding.DDRWError):
            ctx.set_dirichlet(0)  # after the field is loaded
    finally:
        ctx.close()
