"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms (free field,
Abelian clover field), algebraic invariants (Clifford algebra, gamma5-hermiticity, gauge
covariance), the paper's exact identities on dense matrices (det factorisation and the inverse
on supp P of Sec. 1, Eq. 5, Eq. 6), its Gaussian integral and variance (Eq. 3, Eq. 4) by
sampling, and the published known-answer vectors of Philox4x32-10.
"""
import os

import numpy as np
import pytest

from oracle import core as oc
from oracle import dense as od
from paper_1211_1214_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def g5():
    return np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128)


def apply_spin(M, v):
    """Apply a 4x4 spin matrix to a field of shape (V, 4, 3)."""
    return np.einsum("ab,xbc->xac", M, v)


def coords(dims):
    return np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), axis=-1).reshape(-1, 4)


# ----------------------------------------------------------------------------- gamma matrices

def test_gamma_clifford_and_chiral_basis():
    g = [oc.gamma(mu) for mu in range(4)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * (a == b) * np.eye(4))
    assert np.allclose(g[0] @ g[1] @ g[2] @ g[3], g5())


# ----------------------------------------------------------------------------- Philox

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oc.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_noise_moments():
    """E eta = 0, E eta^2 = 0, E|eta|^2 = 1: the measure of Eq. 3 normalised to one."""
    eta = oc.noise_packed(seed=2, hit0=0, nhit=4, n=50000).reshape(-1)
    n = eta.size
    assert abs(np.mean(eta)) < 5 / np.sqrt(n)
    assert abs(np.mean(eta * eta)) < 5 / np.sqrt(n)
    assert abs(np.mean(np.abs(eta) ** 2) - 1.0) < 5 / np.sqrt(n)
    # the real part is N(0, 1/2): fourth moment 3/4
    assert abs(np.mean(eta.real ** 4) - 0.75) < 10 * np.sqrt(105 / 16 - 9 / 16) / np.sqrt(n)


# ----------------------------------------------------------------------------- free field

@pytest.mark.parametrize("antiperiodic", [False, True])
def test_free_field_plane_wave(antiperiodic):
    """U = 1: D e^{ipx} chi = [m + sum_mu (1 - cos p_mu) + i sum_mu g_mu sin p_mu] e^{ipx} chi."""
    dims = (6, 4, 2, 8)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.7, antiperiodic_t=antiperiodic)
    X = coords(dims)
    rng = np.random.default_rng(5)
    g = [oc.gamma(mu) for mu in range(4)]
    m = 0.13
    for n in [(0, 0, 0, 0), (1, 0, 1, 3), (2, 3, 1, 5), (5, 1, 0, 7)]:
        p = np.array([2 * np.pi * n[mu] / dims[mu] for mu in range(4)])
        if antiperiodic:
            p[0] += np.pi / dims[0]
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * X @ p)
        psi = phase[:, None, None] * chi[None]
        Dp = (m + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        want = phase[:, None, None] * (Dp @ chi)[None]
        got = lat.apply(m, psi)
        assert np.max(np.abs(got - want)) < 1e-13


def test_free_field_spectrum_multiplicity():
    """Dense spectrum at U = 1: m + sum(1 - cos p) +- i sqrt(sum sin^2 p), each 6-fold per momentum."""
    dims = (4, 2, 2, 4)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.0)
    m = 0.07
    ev = np.linalg.eigvals(od.dense_D(lat, m))
    want = []
    for n in np.ndindex(*dims):
        p = 2 * np.pi * np.array(n) / np.array(dims)
        re = m + np.sum(1 - np.cos(p))
        im = np.sqrt(np.sum(np.sin(p) ** 2))
        want += [re + 1j * im] * 6 + [re - 1j * im] * 6
    want = np.array(want)
    key = lambda z: np.lexsort((np.round(z.imag, 9), np.round(z.real, 9)))
    assert np.allclose(np.sort_complex(np.round(ev, 9)), np.sort_complex(np.round(want, 9)), atol=1e-8)


# ----------------------------------------------------------------------------- clover term

@pytest.mark.parametrize("plane", [(0, 1), (1, 3), (2, 0)])
def test_clover_abelian_constant_field(plane):
    """Constant Abelian field: every leaf is e^{i phi q}, so Fhat_{mu nu} = i sin(phi q) and
    C = -(csw/2) sigma_{mu nu} (x) diag(sin(phi q_a)) at every site."""
    mu, nu = plane
    dims = (4, 6, 4, 8)
    V = int(np.prod(dims))
    X = coords(dims)
    q = np.array([1.0, -2.0, 1.0])
    phi = 2 * np.pi * 1 / (dims[mu] * dims[nu])
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    for a in range(3):
        U[:, nu, a, a] = np.exp(1j * phi * q[a] * X[:, mu])
        last = X[:, mu] == dims[mu] - 1
        U[last, mu, a, a] = np.exp(-1j * phi * q[a] * dims[mu] * X[last, nu])
    csw = 1.3
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=csw)
    g = [oc.gamma(k) for k in range(4)]
    sigma = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
    want = -(csw / 2) * np.kron(sigma, np.diag(np.sin(phi * q)))
    for x in [0, 17, V // 2 + 3, V - 1]:
        assert np.max(np.abs(lat.clover(x) - want)) < 1e-13


def test_clover_hermitian_commutes_gamma5_and_vanishes_at_unit_links():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=1)
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.0)
    G5 = np.kron(g5(), np.eye(3))
    for x in [0, 5, 100, 255]:
        C = lat.clover(x)
        assert np.max(np.abs(C - C.conj().T)) < 1e-14
        assert np.max(np.abs(G5 @ C - C @ G5)) < 1e-14
        assert np.max(np.abs(C)) > 1e-3
    V = 256
    lat1 = oc.Lattice(dims, (2, 2, 2, 2), np.broadcast_to(np.eye(3), (V, 4, 3, 3)).astype(np.complex128), csw=1.0)
    assert np.max(np.abs(lat1.clover(7))) == 0.0


# ----------------------------------------------------------------------------- invariants at random U

@pytest.fixture(scope="module")
def c1():
    """4^4 lattice, blocks 2^4, eps = 0.3, seed 1, csw = 1.0, m1 = 0.20, m2 = 0.19."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=1)
    return oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.0)


def test_gamma5_hermiticity(c1):
    """<x, g5 D g5 y> = <D x, y>, with D^dag written out independently in the oracle."""
    x = synth.spinor_field(c1.dims, seed=11)
    y = synth.spinor_field(c1.dims, seed=12)
    m = 0.2
    lhs = np.vdot(x, apply_spin(g5(), c1.apply(m, apply_spin(g5(), y))))
    rhs = np.vdot(c1.apply(m, x), y)
    assert abs(lhs - rhs) < 1e-13 * abs(rhs)
    # the adjoint the oracle applies equals g5 D g5
    assert np.max(np.abs(c1.apply(m, y, dagger=True) - apply_spin(g5(), c1.apply(m, apply_spin(g5(), y))))) < 1e-13


def test_gauge_covariance():
    """D[U^g] (g psi) = g D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    dims = (4, 4, 2, 6)
    V = int(np.prod(dims))
    U = synth.gauge_field(dims, 0.4, seed=3)
    g = synth.gauge_transform(dims, seed=4)
    X = coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        Y = X.copy()
        Y[:, mu] = (Y[:, mu] + 1) % dims[mu]
        ym = ((Y[:, 0] * dims[1] + Y[:, 1]) * dims[2] + Y[:, 2]) * dims[3] + Y[:, 3]
        Ug[:, mu] = g @ U[:, mu] @ g[ym].conj().transpose(0, 2, 1)
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.4)
    latg = oc.Lattice(dims, (2, 2, 2, 2), Ug, csw=1.4)
    psi = synth.spinor_field(dims, seed=9)
    gpsi = np.einsum("xab,xsb->xsa", g, psi)
    lhs = latg.apply(0.1, gpsi)
    rhs = np.einsum("xab,xsb->xsa", g, lat.apply(0.1, psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-13


# ----------------------------------------------------------------------------- block structure (Eq. 1, Sec. 1)

def test_blocks_are_block_diagonal(c1):
    """D_bb couples only sites of the same black block; D_bw only sites of neighbouring blocks."""
    D = od.dense_D(c1, 0.2)
    X = coords(c1.dims)
    blk = ((X[:, 0] // 2 * 2 + X[:, 1] // 2) * 2 + X[:, 2] // 2) * 2 + X[:, 3] // 2
    col = c1.colour()
    assert np.all(col == (X // 2).sum(axis=1) % 2)
    nz = np.abs(D.reshape(c1.V, 12, c1.V, 12)).max(axis=(1, 3)) > 0
    i, j = np.nonzero(nz)
    same_colour = col[i] == col[j]
    assert np.all(blk[i][same_colour] == blk[j][same_colour])
    # 4^4 with 2^4 blocks: supp P is every black site (P = all black sites)
    assert np.all(c1.suppP() == (col == 0))


def test_det_factorisation(c1):
    """det D = det Dhat det D_ww det D_bb (Sec. 1), and det D is real (gamma5-hermiticity)."""
    for m in (0.2, 0.19, -0.3):
        D = od.dense_D(c1, m)
        Dbb, Dbw, Dwb, Dww = od.blocks(c1, m)
        s, ld = od.logdet(D)
        s1, l1 = od.logdet(od.schur(c1, m))
        s2, l2 = od.logdet(Dbb)
        s3, l3 = od.logdet(Dww)
        assert abs(ld - (l1 + l2 + l3)) < 1e-9 * abs(ld)
        assert abs(s - s1 * s2 * s3) < 1e-8
        assert abs(s.imag) < 1e-8


def test_schur_inverse_on_supp_P():
    """On supp P: (P Dhat P)^-1 = P (1 - Dcal_bw D_wb) P and det(P Dhat P) = det Dhat (Sec. 1)."""
    # blocks 4x4x2x2 (one block in y and z, which wrap onto themselves): sites with t and x
    # inside the block have no white neighbour, so supp P is a proper subset of the black sites
    dims = (8, 8, 2, 2)
    U = synth.gauge_field(dims, 0.3, seed=7)
    lat = oc.Lattice(dims, (4, 4, 2, 2), U, csw=1.2)
    b, w, p = od.component_sets(lat)
    assert 0 < len(p) < len(b)
    m = 0.15
    D = od.dense_D(lat, m)
    Dinv = np.linalg.inv(D)
    Dcal_bw = Dinv[np.ix_(b, w)]
    Dwb = D[np.ix_(w, b)]
    # D_wb P = D_wb: columns of D_wb outside supp P vanish
    pos = np.searchsorted(b, p)
    outside = np.setdiff1d(np.arange(len(b)), pos)
    assert np.max(np.abs(Dwb[:, outside])) == 0.0
    S = od.schur(lat, m)
    A = S[np.ix_(pos, pos)]
    want = (np.eye(len(b)) - Dcal_bw @ Dwb)[np.ix_(pos, pos)]
    assert np.max(np.abs(np.linalg.inv(A) - want)) < 1e-10
    assert abs(od.logdet(A)[1] - od.logdet(S)[1]) < 1e-9


def test_even_odd_is_the_l1_case():
    """Blocks of length 1 give the even-odd Schur complement: D_bb is site-diagonal on even sites."""
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, 0.3, seed=2)
    lat = oc.Lattice(dims, (1, 1, 1, 1), U, csw=1.0)
    X = coords(dims)
    assert np.all(lat.colour() == X.sum(axis=1) % 2)
    Dbb, _, _, _ = od.blocks(lat, 0.1)
    nb = Dbb.shape[0] // 12
    R = Dbb.reshape(nb, 12, nb, 12)
    off = R.copy()
    for k in range(nb):
        off[k, :, k, :] = 0
    assert np.max(np.abs(off)) == 0.0
    assert np.all(lat.suppP() == (lat.colour() == 0))


# ----------------------------------------------------------------------------- mass structure (Eq. 5, Eq. 6)

def test_mass_shift_spectrum(c1):
    """D(m1) - D(m2) = dm; lambda(M) = 1 + dm/lambda(D(m2)); det M^-1 = prod lambda/(lambda + dm)."""
    m1, m2 = 0.20, 0.19
    dm = m1 - m2
    D1, D2 = od.dense_D(c1, m1), od.dense_D(c1, m2)
    assert np.max(np.abs(D1 - D2 - dm * np.eye(D1.shape[0]))) < 1e-15
    lam = np.linalg.eigvals(D2)
    M = np.linalg.solve(D2, D1)
    lamM = np.linalg.eigvals(M)
    want = 1 + dm / lam
    # match each eigenvalue of M to the prediction
    d = np.abs(lamM[:, None] - want[None, :]).min(axis=1)
    assert d.max() < 1e-9
    s, ldM = np.linalg.slogdet(M)
    assert abs(-ldM - np.sum(np.log(np.abs(lam / (lam + dm))))) < 1e-9


# ----------------------------------------------------------------------------- solver and estimator

def test_cgnr_block_solve_matches_dense(c1):
    D = od.dense_D(c1, 0.19)
    b_idx, w_idx, _ = od.component_sets(c1)
    rhs = synth.spinor_field(c1.dims, seed=21)
    col = c1.colour()
    rhs[col == 1] = 0
    x, it, rel = c1.solve(0.19, rhs, sel=oc.BLACK, tol=1e-13)
    assert rel <= 1e-13
    want = np.linalg.solve(D[np.ix_(b_idx, b_idx)], rhs.reshape(-1)[b_idx])
    assert np.max(np.abs(x.reshape(-1)[b_idx] - want)) < 1e-11 * np.max(np.abs(want))
    assert np.max(np.abs(x[col == 1])) == 0.0


def test_exponent_matches_dense(c1):
    """Oracle e_j (five CGNR solves, resolvent form of r) against eta^dag (Mh^dag Mh - 1) eta."""
    m1, m2 = 0.20, 0.19
    Mh = od.ratio_matrix(c1, m1, m2)
    A1, A2 = od.schur_on_P(c1, m1), od.schur_on_P(c1, m2)
    n = Mh.shape[0]
    eta_p = oc.noise_packed(seed=2, hit0=0, nhit=3, n=n)
    for j in range(3):
        res = c1.exponent(m1, m2, c1.unpack(eta_p[j]))
        e_dense = od.exponent(Mh, eta_p[j])[0]
        assert abs(res["e"] - e_dense) < 1e-10 * max(abs(e_dense), 1.0)
        r_dense = (A1 - A2) @ eta_p[j]
        assert np.max(np.abs(c1.pack(res["r"]) - r_dense)) < 1e-11 * np.max(np.abs(r_dense))
        d_dense = Mh @ eta_p[j] - eta_p[j]
        assert np.max(np.abs(c1.pack(res["delta"]) - d_dense)) < 1e-10 * np.max(np.abs(d_dense))


def test_zero_mass_shift_gives_zero_exponent(c1):
    eta_p = oc.noise_packed(seed=3, hit0=0, nhit=1, n=len(c1.suppP_sites()) * 12)[0]
    res = c1.exponent(0.2, 0.2, c1.unpack(eta_p))
    assert res["e"] == 0.0
    assert np.max(np.abs(res["r"])) == 0.0


def test_estimator_mean_and_variance():
    """Eq. 3: mean of exp(-e_j) -> 1/det(Mh^dag Mh); Eq. 4: its variance, by sampling the
    oracle's own Philox noise (a wrong noise normalisation or exponent fails both)."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=1)
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.0)
    m1, m2 = 0.20, 0.15
    Mh = od.ratio_matrix(lat, m1, m2)
    W = od.inv_det_MdagM(Mh)
    var = od.stochastic_variance(Mh)
    ns = 12000
    eta = oc.noise_packed(seed=77, hit0=0, nhit=ns, n=Mh.shape[0])
    e = od.exponent(Mh, eta)
    w = np.exp(-e)
    # the test is sensitive: a noise of the wrong variance moves the mean by many standard errors
    assert abs(np.log(W)) > 20 * np.sqrt(var / ns) / W
    assert abs(w.mean() - W) < 4 * np.sqrt(var / ns)
    # sample variance against Eq. 4 (fourth moment finite for this spectrum; 25% slack)
    assert abs(w.var() / var - 1) < 0.25
    # the oracle's C estimator agrees with the dense exponent on a few of these samples
    for j in range(2):
        res = lat.exponent(m1, m2, lat.unpack(eta[j]))
        assert abs(res["e"] - e[j]) < 1e-10 * max(abs(e[j]), 1.0)


def test_variance_expansion_and_hutchinson_moments():
    """Eq. 4 at small dm, the form the large-volume check uses.  With A = Mh^dag Mh and X = A - 1:
    det(A)^2 / det(2A - 1) = det(1 + X^2 (1 + 2X)^-1) exactly, so sigma_s^2/W^2 = exp(tr X^2 + O(X^3)) - 1;
    for complex Gaussian noise (E|eta|^2 = 1) the exponent e = eta^dag X eta has mean tr X and
    variance tr X^2 (Hutchinson).  Both sides are checked on the dense 4^4 ratio matrix."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=1)
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.0)
    m1 = 0.20
    prev = None
    for m2 in (0.199, 0.198):
        Mh = od.ratio_matrix(lat, m1, m2)
        A = Mh.conj().T @ Mh
        n = A.shape[0]
        X = A - np.eye(n)
        W = od.inv_det_MdagM(Mh)
        rel = od.stochastic_variance(Mh) / W ** 2           # Eq. 4 divided by W^2
        trX, trX2 = np.real(np.trace(X)), np.real(np.trace(X @ X))
        # the exact rewrite and its leading order
        _, ld = np.linalg.slogdet(np.eye(n) + X @ X @ np.linalg.inv(np.eye(n) + 2 * X))
        assert abs(np.expm1(ld) - rel) < 1e-10 * rel
        assert abs(np.expm1(trX2) - rel) < 0.05 * rel
        # Hutchinson: sample mean and variance of the exponents
        ns = 20000
        eta = oc.noise_packed(seed=91, hit0=0, nhit=ns, n=n)
        e = od.exponent(Mh, eta)
        assert abs(e.mean() - trX) < 5 * np.sqrt(trX2 / ns)
        assert abs(e.var() / trX2 - 1) < 0.1
        # the fluctuations grow like dm^2
        if prev is not None:
            assert abs(trX2 / prev - 4.0) < 0.1
        prev = trX2


# ----------------------------------------------------------------------------- one flavour (Eq. 11, Eq. 12), interpolation (Eq. 8)

def test_one_flavour_integral_and_variance():
    """Eq. 11: the mean of exp(-eta^dag (Mh - 1) eta) -> 1/det Mh (real by g5-hermiticity);
    Eq. 12: its variance 1/det(Mh^dag + Mh - 1) - 1/det(Mh^dag Mh), by sampling."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=1)
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.0)
    Mh = od.ratio_matrix(lat, 0.20, 0.15)
    n = Mh.shape[0]
    ev = np.linalg.eigvals(Mh)
    assert np.all(ev.real > 0)                                      # integral defined
    assert np.all(np.linalg.eigvalsh(Mh + Mh.conj().T) > 1)         # variance defined
    s, ld = np.linalg.slogdet(Mh)
    W1 = np.exp(-ld) / s                                            # 1/det Mh
    assert abs(W1.imag) < 1e-10 * abs(W1)
    W1 = W1.real
    s2, ld2 = np.linalg.slogdet(Mh + Mh.conj().T - np.eye(n))
    _, ldMM = np.linalg.slogdet(Mh.conj().T @ Mh)
    var = float(np.exp(-ld2).real - np.exp(-ldMM))
    ns = 12000
    eta = oc.noise_packed(seed=91, hit0=0, nhit=ns, n=n)
    e1 = np.sum(eta.conj() * (eta @ (Mh - np.eye(n)).T), axis=1)   # eta^dag (Mh - 1) eta
    x = np.exp(-e1)
    assert abs(x.mean().real - W1) < 4 * np.sqrt(var / ns)
    assert abs(x.mean().imag) < 4 * np.sqrt(var / ns)
    assert abs(np.mean(np.abs(x - x.mean()) ** 2) / var - 1) < 0.25
    # sensitivity: the two-flavour value is many standard errors away
    assert abs(W1 - np.exp(-ldMM)) > 20 * np.sqrt(var / ns)
    # the oracle's delta gives the same complex exponent
    for j in range(2):
        res = lat.exponent(0.20, 0.15, lat.unpack(eta[j]))
        e1_orc = np.vdot(eta[j], lat.pack(res["delta"]))
        assert abs(e1_orc - e1[j]) < 1e-10 * max(abs(e1[j]), 1.0)


def test_mass_interpolation_telescopes():
    """Eq. 8: with m_i = (i/N) m2 + ((N-i)/N) m1 the factors Mh_i = A(m_i)^-1 A(m_{i-1}) multiply to
    det Mh: prod_i 1/det(Mh_i^dag Mh_i) = 1/det(Mh^dag Mh)."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, seed=1)
    lat = oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.0)
    m1, m2, N = 0.20, 0.14, 3
    ms = [(i / N) * m2 + ((N - i) / N) * m1 for i in range(N + 1)]
    tot = 0.0
    for i in range(1, N + 1):
        Mi = od.ratio_matrix(lat, ms[i - 1], ms[i])
        tot += np.linalg.slogdet(Mi.conj().T @ Mi)[1]
    one = od.ratio_matrix(lat, m1, m2)
    assert abs(tot - np.linalg.slogdet(one.conj().T @ one)[1]) < 1e-9


# ---- block determinants of Eq. 7 (oracle/blockdet.py)

def test_block_determinants_factorise_det_D(c1):
    """Sum over the blocks of one colour of log|det D_k| is log|det D_bb| (D_ww), and with the
    Schur complement they give log|det D| (Sec. 1) -- every determinant of D_k real (Eq. 7 uses
    det D_k^2)."""
    from oracle import blockdet as ob
    for m in (0.2, -0.3):
        ld, sg = ob.block_logdets(c1, m)
        blocks = ob.block_list(c1)
        nb = len(blocks) // 2
        assert all(c == 0 for c, _ in blocks[:nb]) and all(c == 1 for c, _ in blocks[nb:])
        Dbb, _, _, Dww = od.blocks(c1, m)
        sb, lb = od.logdet(Dbb)
        sw, lw = od.logdet(Dww)
        assert abs(ld[:nb].sum() - lb) < 1e-9 * max(1.0, abs(lb))
        assert abs(ld[nb:].sum() - lw) < 1e-9 * max(1.0, abs(lw))
        s, lD = od.logdet(od.dense_D(c1, m))
        _, lS = od.logdet(od.schur(c1, m))
        assert abs(ld.sum() + lS - lD) < 1e-8 * max(1.0, abs(lD))
        assert np.all(np.abs(np.imag(sg)) < 1e-9)


def test_single_site_blocks_reduce_to_the_site_term():
    """With l = 1 every block is one site and D_k = A(x) = (4 + m) + C(x): its determinant is the
    determinant of the 12x12 site matrix, read from the oracle's clover routine."""
    from oracle import blockdet as ob
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.4, seed=17)
    lat = oc.Lattice(dims, (1, 1, 1, 1), U, 1.3)
    m = 0.11
    ld, sg = ob.block_logdets(lat, m)
    for k, (_, o) in enumerate(ob.block_list(lat)):
        x = ((o[0] * dims[1] + o[1]) * dims[2] + o[2]) * dims[3] + o[3]
        s, l = np.linalg.slogdet(lat.clover(x) + (4 + m) * np.eye(12))
        assert abs(ld[k] - l) < 1e-12 and abs(sg[k] - s) < 1e-12


def test_block_determinants_are_gauge_invariant():
    """A gauge transformation acts on each block operator as a similarity transform, so every
    block determinant is unchanged; a wrong link index or a missing conjugate breaks this."""
    from oracle import blockdet as ob
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.4, seed=21)
    g = synth.gauge_transform(dims, seed=23)
    X = coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        Y = X.copy()
        Y[:, mu] = (Y[:, mu] + 1) % dims[mu]
        ym = ((Y[:, 0] * dims[1] + Y[:, 1]) * dims[2] + Y[:, 2]) * dims[3] + Y[:, 3]
        Ug[:, mu] = g @ U[:, mu] @ g[ym].conj().transpose(0, 2, 1)
    ld0, _ = ob.block_logdets(oc.Lattice(dims, (2, 2, 2, 2), U, csw=1.2), 0.07)
    ld1, _ = ob.block_logdets(oc.Lattice(dims, (2, 2, 2, 2), Ug, csw=1.2), 0.07)
    assert np.max(np.abs(ld1 - ld0)) < 1e-10
    # and they do change when the links change (the test is not vacuous)
    ld2, _ = ob.block_logdets(oc.Lattice(dims, (2, 2, 2, 2), synth.gauge_field(dims, 0.4, seed=22), csw=1.2), 0.07)
    assert np.max(np.abs(ld2 - ld0)) > 1e-3


# ---- the operators of Fig. 1's comparison (oracle/dense.py): total, even-odd, block Schur

def test_estimator_operators_factorise_the_determinant_ratio(c1):
    """det D = det A_oo det S (even-odd) and det D = det Dhat det D_bb det D_ww (Sec. 1), so the
    three ratio matrices carry the same determinant ratio up to exactly known site and block
    factors: log det M_total = log det M_eo + log det A_oo(m1) - log det A_oo(m2)
                             = log det Mh + sum_k [log det D_k(m1) - log det D_k(m2)]   (Eq. 7)."""
    from oracle import blockdet as ob
    m1, m2 = 0.20, 0.15
    st, lt = od.logdet(od.ratio_matrix_total(c1, m1, m2))
    se, le = od.logdet(od.ratio_matrix_eo(c1, m1, m2))
    sh, lh = od.logdet(od.ratio_matrix(c1, m1, m2))
    # det A_oo(m): product over odd sites of det((4 + m) + C(x)) from the oracle's clover matrix
    X = np.stack(np.unravel_index(np.arange(c1.V), c1.dims), -1)
    odd = np.nonzero(X.sum(1) % 2 == 1)[0]
    lA = lambda m: sum(np.linalg.slogdet(c1.clover(x) + (4 + m) * np.eye(12))[1] for x in odd)
    assert abs(lt - (le + lA(m1) - lA(m2))) < 1e-9
    b1, _ = ob.block_logdets(c1, m1)
    b2, _ = ob.block_logdets(c1, m2)
    assert abs(lt - (lh + b1.sum() - b2.sum())) < 1e-9
    # the ratio matrices differ (the estimator's variance depends on the choice, Fig. 1)
    assert abs(lt - lh) > 1e-3


# ---- the log-sum-exp of Eq. 3 / Eq. 8 (oracle.core.log_w) and the block factor of Eq. 7
# (oracle.blockdet.log_block_factor): both serve as checkers of the GPU's log W

def _log_w_decimal(exponents, digits=60):
    """log((1/N) sum_j exp(-e_j)) in 60-digit decimal arithmetic: no shift, no overflow."""
    from decimal import Decimal, localcontext
    with localcontext() as ctx:
        ctx.prec = digits
        s = sum((-Decimal(repr(float(e)))).exp() for e in exponents)
        return float((s / len(exponents)).ln())


def test_log_w_against_the_direct_sum():
    """Eq. 3: W = (1/N_hit) sum_j exp(-e_j).  On moderate exponents log_w equals the direct
    formula evaluated in FP64 and in high precision."""
    rng = np.random.default_rng(31)
    for n in (1, 2, 7, 16, 48):
        e = rng.normal(3.0, 2.0, size=n)
        direct = float(np.log(np.mean(np.exp(-e))))
        assert abs(oc.log_w(e) - direct) <= 1e-13 * max(1.0, abs(direct))
        assert abs(oc.log_w(e) - _log_w_decimal(e)) <= 1e-13 * max(1.0, abs(direct))


def test_log_w_at_exponents_where_the_direct_form_overflows():
    """Exponents of -710 .. +760 overflow (exp(710) = inf) or underflow (exp(-760) = 0) in the
    direct form; log_w must stay exact there (the paper's log W at 64x32^3 is O(10^3))."""
    for e in ([-710.0, -711.5, -709.25], [700.0, 745.0, 760.0, 701.0], [-700.0, 700.0], [2571.8, 2570.1]):
        with np.errstate(over="ignore", divide="ignore"):
            direct = np.log(np.mean(np.exp(-np.asarray(e))))
        want = _log_w_decimal(e)
        got = oc.log_w(e)
        assert np.isfinite(got)
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want))
        if not np.isfinite(direct):
            continue
        assert abs(got - direct) <= 1e-12 * max(1.0, abs(want))


def test_log_w_normalisation_and_sign():
    """Equal exponents give log W = -e exactly (the -log N_hit offset cancels N equal terms); one
    finite term among N whose others vanish gives -e - log N; W decreases as an exponent grows."""
    for n in (1, 3, 16):
        assert abs(oc.log_w([2.5] * n) - (-2.5)) < 1e-15
        assert abs(oc.log_w([0.25] + [5000.0] * (n - 1)) - (-0.25 - np.log(n))) < 1e-14
    assert oc.log_w([1.0]) == -1.0
    assert oc.log_w([1.0, 2.0]) > oc.log_w([1.0, 3.0])


def test_log_block_factor_completes_the_determinant_ratio(c1):
    """Eq. 7 with Eq. 3: W = W_gl prod_k det D_k^2(m2)/det D_k^2(m1) with W_gl = 1/det(Mh^dag Mh)
    (its exact value, dense), and by det D = det Dhat det D_bb det D_ww (Sec. 1) the product is
    det D(m2)^2 / det D(m1)^2 = the two-flavour ratio 1/det(M^dag M) of the total operator, Eq. 2.
    Swapped masses, a missing square or a lost block fail this."""
    from oracle import blockdet as ob
    for m1, m2 in ((0.20, 0.19), (0.20, 0.12)):
        Mh = od.ratio_matrix(c1, m1, m2)
        log_w_gl = float(np.log(od.inv_det_MdagM(Mh)))
        _, l1 = od.logdet(od.dense_D(c1, m1))
        _, l2 = od.logdet(od.dense_D(c1, m2))
        want = 2.0 * (l2 - l1)
        got = ob.log_block_factor(c1, m1, m2) + log_w_gl
        assert abs(got - want) <= 1e-9 * max(1.0, abs(want))
        # the block factor alone is not the whole ratio (the test is not vacuous)
        assert abs(ob.log_block_factor(c1, m1, m2) - want) > 1e-3


# ---- nested decomposition of large blocks (Sec. 2.2, Fig. 2 caption): a block determinant is the
# Schur complement of the block's Dirichlet operator with respect to its sub-blocks times the
# sub-block determinants (oracle.blockdet.dirichlet_links / dirichlet_lattice)

@pytest.fixture(scope="module")
def boxes():
    """8x4x4x4 lattice cut into two 4^4 Dirichlet boxes along t (hops across every box face,
    including the periodic wrap in x, y, z, removed), as blocks of length 4 and 2."""
    from oracle import blockdet as ob
    dims, csw = (8, 4, 4, 4), 1.2
    U = synth.gauge_field(dims, 0.3, seed=5)
    full = oc.Lattice(dims, (4, 4, 4, 4), U, csw)
    cut4 = ob.dirichlet_lattice(dims, (4, 4, 4, 4), U, csw, cut=4)
    cut2 = ob.dirichlet_lattice(dims, (2, 2, 2, 2), U, csw, cut=4)
    return dims, full, cut4, cut2


def test_dirichlet_operator_is_the_direct_sum_of_the_box_operators(boxes):
    """The cut operator keeps exactly the site terms (the clover term of the full field) and the
    hops that stay inside a box, with the full operator's entries, and couples no two boxes."""
    dims, full, cut4, cut2 = boxes
    m = 0.07
    Dc = od.dense_D(cut2, m).reshape(cut2.V, 12, cut2.V, 12).transpose(0, 2, 1, 3)  # [x][y][12][12]
    D = od.dense_D(full, m).reshape(full.V, 12, full.V, 12).transpose(0, 2, 1, 3)
    X = coords(dims)
    keep = np.eye(full.V, dtype=bool)
    for mu in range(4):
        for d in (1, -1):
            Y = X.copy()
            Y[:, mu] = (Y[:, mu] + d) % dims[mu]
            inside = (X[:, mu] // 4 == Y[:, mu] // 4) & (np.abs(X[:, mu] - Y[:, mu]) == 1)
            y = ((Y[:, 0] * dims[1] + Y[:, 1]) * dims[2] + Y[:, 2]) * dims[3] + Y[:, 3]
            keep[np.arange(full.V)[inside], y[inside]] = True
    assert np.max(np.abs(Dc[keep] - D[keep])) < 1e-15
    assert np.max(np.abs(Dc[~keep])) == 0.0
    assert np.max(np.abs(D[~keep])) > 0.1  # the removed hops were there
    for x in (0, 37, 200, 511):
        assert np.max(np.abs(cut2.clover(x) - full.clover(x))) == 0.0


def test_nested_block_determinant_equals_the_block_determinant(boxes):
    """For the Dirichlet boxes D_k: sum_k log|det D_k| = sum over the 2^4 sub-blocks of
    log|det D_sub| + log|det Dhat'| (Dhat' the Schur complement of the cut operator with respect
    to the sub-blocks, Sec. 1); and for a mass pair the block factor of Eq. 7 equals the sub-block
    factor times 1/det(Mh'^dag Mh'), Mh' the sub-block ratio matrix of the cut operator -- the
    quantity the nested estimate samples."""
    from oracle import blockdet as ob
    dims, full, cut4, cut2 = boxes
    for m in (0.07, -0.2):
        ld4, _ = ob.block_logdets(cut4, m)
        ld2, _ = ob.block_logdets(cut2, m)
        _, lS = od.logdet(od.schur(cut2, m))
        assert abs(ld4.sum() - (ld2.sum() + lS)) < 1e-9 * max(1.0, abs(ld4.sum()))
    m1, m2 = 0.10, 0.06
    exact = ob.log_block_factor(cut4, m1, m2)
    sub = ob.log_block_factor(cut2, m1, m2)
    schur_part = float(np.log(od.inv_det_MdagM(od.ratio_matrix(cut2, m1, m2))))
    assert abs(exact - (sub + schur_part)) < 1e-9 * max(1.0, abs(exact))
    assert abs(schur_part) > 1e-3 and abs(sub) > 1e-3  # both parts carry weight
