"""Pins of the oracle's adjoint (no GPU): its analytic link and mass derivatives of
e = eta^dag (Mh^dag Mh - 1) eta against central finite differences of the oracle's own estimate.

Direction convention: d/dt e(exp(i t X) U) with X = sum_a w_a lambda_a / 2 on every link, which
equals sum_{links, a} w_a dU[link, a]."""
import numpy as np
import pytest

from oracle import core as oc
from paper_1211_1214_gb300 import synth


def perturb(U, omega, t):
    """exp(i t X) U per link, X = sum_a omega_a lambda_a / 2 (omega shape (V, 4, 8))."""
    X = np.einsum("lna,aij->lnij", omega, synth.gell_mann() / 2.0).reshape(-1, 3, 3)
    E = synth._expm_i_traceless_hermitian(t * X).reshape(U.shape)
    return np.einsum("lnij,lnjk->lnik", E, U)


@pytest.mark.parametrize("csw", [0.0, 1.3])
def test_link_and_mass_derivatives_match_finite_differences(csw):
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.3, seed=1)
    m1, m2 = 0.20, 0.17
    lat = oc.Lattice(dims, block, U, csw)
    eta = lat.unpack(oc.noise_packed(2, 0, 1, 12 * len(lat.suppP_sites()))[0])
    e0, dU, dm2 = lat.force(m1, m2, eta, tol_block=1e-14, tol_outer=1e-14)
    assert abs(e0 - lat.exponent(m1, m2, eta)["e"]) < 1e-9 * max(1, abs(e0))
    h = 1e-5
    rng = np.random.default_rng(11)
    for k in range(1):
        omega = rng.standard_normal((lat.V, 4, 8))
        ep = oc.Lattice(dims, block, perturb(U, omega, +h), csw).exponent(m1, m2, eta, 1e-14, 1e-14)["e"]
        em = oc.Lattice(dims, block, perturb(U, omega, -h), csw).exponent(m1, m2, eta, 1e-14, 1e-14)["e"]
        fd = (ep - em) / (2 * h)
        an = float(np.sum(omega * dU))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (k, fd, an)
    ep = lat.exponent(m1, m2 + h, eta, 1e-14, 1e-14)["e"]
    em = lat.exponent(m1, m2 - h, eta, 1e-14, 1e-14)["e"]
    fd = (ep - em) / (2 * h)
    assert abs(fd - dm2) <= 1e-6 * max(abs(dm2), 1e-3), (fd, dm2)


def test_single_link_derivative():
    """One link, one generator: the force entry itself against a finite difference."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.3, seed=5)
    lat = oc.Lattice(dims, block, U, 1.0)
    eta = lat.unpack(oc.noise_packed(3, 0, 1, 12 * len(lat.suppP_sites()))[0])
    _, dU, _ = lat.force(0.20, 0.15, eta, tol_block=1e-14, tol_outer=1e-14)
    h = 1e-5
    for (x, mu, a) in [(37, 2, 7), (200, 3, 4)]:
        omega = np.zeros((lat.V, 4, 8))
        omega[x, mu, a] = 1.0
        ep = oc.Lattice(dims, block, perturb(U, omega, +h), 1.0).exponent(0.20, 0.15, eta, 1e-14, 1e-14)["e"]
        em = oc.Lattice(dims, block, perturb(U, omega, -h), 1.0).exponent(0.20, 0.15, eta, 1e-14, 1e-14)["e"]
        fd = (ep - em) / (2 * h)
        assert abs(fd - dU[x, mu, a]) <= 1e-6 * max(abs(dU[x, mu, a]), 1e-4), (x, mu, a, fd, dU[x, mu, a])
