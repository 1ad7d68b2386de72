"""Dense linear algebra on tiny lattices (V <= 4^4, dim D = 12V <= 3072).

TEST INFRASTRUCTURE ONLY.  The dense matrix of D(m) is assembled column by column from the C
oracle's operator; everything else here is textbook dense algebra on that matrix, written to
mirror the paper's statements:

* Eq. 1   block notation D = [[D_bb, D_bw], [D_wb, D_ww]] and D^-1 = [[Dcal_bb, Dcal_bw], ...];
* Sec. 1  Dhat = 1 - D_bb^-1 D_bw D_ww^-1 D_wb, det D = det Dhat det D_ww det D_bb, and on the
          support of the projector P (D_wb P = D_wb) the inverse Dhat^-1 = 1 - P Dcal_bw D_wb;
* Eq. 3   the Gaussian integral 1/det(M^dag M) and its estimator exp(-eta^dag (M^dag M - 1) eta);
* Eq. 4   sigma_s^2 = 1/det(2 M^dag M - 1) - 1/det(M^dag M)^2;
* Eq. 5/6 det M^-1 = prod lambda/(lambda + dm), lambda(M) = 1 + dm lambda(D^-1(m2)).
* Sec. 2   the other operators whose ratio the estimator can sample (Fig. 1's variants): the total
          operator, M = D(m2)^-1 D(m1), and the even-odd Schur complement
          S = A_ee - D_eo A_oo^-1 D_oe (the block Schur complement for blocks of one site),
          M = S(m2)^-1 S(m1); supports in lexicographic site order.
"""
from __future__ import annotations

import numpy as np

from . import core


def dense_D(lat: "core.Lattice", m: float) -> np.ndarray:
    """The 12V x 12V matrix of D(m); built once at m = 0 and shifted, since D(m) = D(0) + m."""
    key = "_dense_D0"
    D0 = getattr(lat, key, None)
    if D0 is None:
        n = 12 * lat.V
        D0 = np.zeros((n, n), dtype=np.complex128)
        e = np.zeros(n, dtype=np.complex128)
        for j in range(n):
            e[:] = 0
            e[j] = 1
            D0[:, j] = lat.apply(0.0, e).reshape(-1)
        setattr(lat, key, D0)
    return D0 + m * np.eye(D0.shape[0])


def component_sets(lat: "core.Lattice"):
    """Component indices (into 12V) of black sites, white sites and supp P, ascending."""
    col = lat.colour()
    P = lat.suppP()
    comp = lambda mask: (np.nonzero(mask)[0][:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
    return comp(col == 0), comp(col == 1), comp(P == 1)


def blocks(lat, m):
    D = dense_D(lat, m)
    b, w, _ = component_sets(lat)
    return D[np.ix_(b, b)], D[np.ix_(b, w)], D[np.ix_(w, b)], D[np.ix_(w, w)]


def schur(lat, m) -> np.ndarray:
    """Dhat(m) = 1 - D_bb^-1 D_bw D_ww^-1 D_wb on the black components."""
    Dbb, Dbw, Dwb, Dww = blocks(lat, m)
    return np.eye(Dbb.shape[0]) - np.linalg.solve(Dbb, Dbw @ np.linalg.solve(Dww, Dwb))


def schur_on_P(lat, m) -> np.ndarray:
    """A(m) = P Dhat(m) P, as a matrix on the supp P components (packed order)."""
    b, _, p = component_sets(lat)
    pos = np.searchsorted(b, p)
    S = schur(lat, m)
    return S[np.ix_(pos, pos)]


def ratio_matrix(lat, m1, m2) -> np.ndarray:
    """Mhat = A(m2)^-1 A(m1) on supp P (Eq. 8 with N = 1, restricted to the support of P)."""
    return np.linalg.solve(schur_on_P(lat, m2), schur_on_P(lat, m1))


def ratio_matrix_total(lat, m1, m2) -> np.ndarray:
    """M = D(m2)^-1 D(m1) on all 12 V components (lexicographic site order)."""
    return np.linalg.solve(dense_D(lat, m2), dense_D(lat, m1))


def even_components(lat) -> np.ndarray:
    """Component indices (into 12 V) of the even sites (t + x + y + z even), ascending."""
    X = np.stack(np.unravel_index(np.arange(lat.V), lat.dims), -1)
    even = np.nonzero(X.sum(1) % 2 == 0)[0]
    return (even[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)


def schur_eo(lat, m) -> np.ndarray:
    """S(m) = D_ee - D_eo D_oo^-1 D_oe on the even components (D_ee = A_ee, D_oo = A_oo)."""
    D = dense_D(lat, m)
    e = even_components(lat)
    o = np.setdiff1d(np.arange(12 * lat.V), e)
    return D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])


def ratio_matrix_eo(lat, m1, m2) -> np.ndarray:
    """M = S(m2)^-1 S(m1) on the even components."""
    return np.linalg.solve(schur_eo(lat, m2), schur_eo(lat, m1))


def exponent(Mh: np.ndarray, eta_packed: np.ndarray) -> np.ndarray:
    """e = eta^dag (Mh^dag Mh - 1) eta for one or more packed vectors (rows of eta_packed)."""
    eta = np.atleast_2d(eta_packed)
    y = eta @ Mh.T
    return np.real(np.sum(np.conj(y) * y, axis=1) - np.sum(np.conj(eta) * eta, axis=1))


def logdet(A: np.ndarray):
    """(sign, log|det A|) by LU."""
    return np.linalg.slogdet(A)


def inv_det_MdagM(Mh: np.ndarray) -> float:
    """1/det(Mh^dag Mh) (Eq. 3's left-hand side)."""
    s, ld = np.linalg.slogdet(Mh.conj().T @ Mh)
    return float(np.exp(-ld))


def stochastic_variance(Mh: np.ndarray) -> float:
    """sigma_s^2 = 1/det(2 Mh^dag Mh - 1) - 1/det(Mh^dag Mh)^2 (Eq. 4), N_hit = 1."""
    A = Mh.conj().T @ Mh
    s2, ld2 = np.linalg.slogdet(2 * A - np.eye(A.shape[0]))
    s1, ld1 = np.linalg.slogdet(A)
    if np.real(s2) <= 0:
        raise ValueError("variance undefined: an eigenvalue of M^dag M is below 1/2")
    return float(np.exp(-ld2) - np.exp(-2 * ld1))
