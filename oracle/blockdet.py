"""Block determinants of Eq. 7: log |det D_k(m)| and the sign of det D_k(m) for every block k.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Eq. 7 writes the reweighting factor as
W = W_gl prod_k det D_k^2(m2) / det D_k^2(m1), k over the black and the white blocks, D_k the
block Dirac operators on the diagonal of D_bb and D_ww (Eq. 1: hops inside the block only).

Each D_k is assembled densely from the C oracle's block-restricted operator (rows and columns of
one colour): a unit vector placed at the same in-block site and component of every block of that
colour gives one column of every block matrix at once, because the blocks of a colour do not
couple.  The determinant is a textbook LU (numpy.linalg.slogdet).  Blocks are numbered as the
library numbers them: black blocks first, then white, each in lexicographic order of the block
coordinates (t slowest).
"""
from __future__ import annotations

import numpy as np

from . import core


def block_list(lat: "core.Lattice"):
    """[(colour, origin (t, x, y, z))] in the library's block numbering."""
    NB = [L // b for L, b in zip(lat.dims, lat.block)]
    out = {0: [], 1: []}
    for B in range(int(np.prod(NB))):
        c, r = [0] * 4, B
        for mu in (3, 2, 1, 0):
            c[mu] = r % NB[mu]
            r //= NB[mu]
        out[sum(c) % 2].append(tuple(ci * b for ci, b in zip(c, lat.block)))
    return [(0, o) for o in out[0]] + [(1, o) for o in out[1]]


def _block_sites(lat, origin):
    """Lexicographic site indices of the block at `origin`, in in-block lexicographic order."""
    L, b = lat.dims, lat.block
    idx = []
    for t in range(b[0]):
        for x in range(b[1]):
            for y in range(b[2]):
                for z in range(b[3]):
                    tt, xx, yy, zz = origin[0] + t, origin[1] + x, origin[2] + y, origin[3] + z
                    idx.append(((tt * L[1] + xx) * L[2] + yy) * L[3] + zz)
    return np.array(idx)


def block_matrices(lat: "core.Lattice", m: float):
    """Dense D_k(m) (12 l^4 square) for every block, in the library's numbering."""
    blocks = block_list(lat)
    nsite = int(np.prod(lat.block))
    n = 12 * nsite
    mats = [np.zeros((n, n), dtype=np.complex128) for _ in blocks]
    sites = [_block_sites(lat, o) for _, o in blocks]
    for colour in (0, 1):
        members = [k for k, (c, _) in enumerate(blocks) if c == colour]
        for q in range(nsite):
            for a in range(12):
                v = np.zeros((lat.V, 12), dtype=np.complex128)
                for k in members:
                    v[sites[k][q], a] = 1.0
                w = lat.apply(m, v.reshape(lat.V, 4, 3), rows=colour, cols=colour).reshape(lat.V, 12)
                for k in members:
                    mats[k][:, 12 * q + a] = w[sites[k]].reshape(-1)
    return mats


def block_logdets(lat: "core.Lattice", m: float):
    """(log |det D_k(m)|, sign of det D_k(m)) for every block; det D_k is real (g5-hermiticity of
    the block operator), so the sign is the real part of the phase."""
    ld, sg = [], []
    for A in block_matrices(lat, m):
        s, l = np.linalg.slogdet(A)
        ld.append(l)
        sg.append(s)
    return np.array(ld), np.array(sg)


def log_block_factor(lat: "core.Lattice", m1: float, m2: float) -> float:
    """log prod_k det D_k^2(m2) / det D_k^2(m1) (Eq. 7, two flavours)."""
    l2, _ = block_logdets(lat, m2)
    l1, _ = block_logdets(lat, m1)
    return float(2.0 * (l2.sum() - l1.sum()))


# ---- the nested decomposition of large blocks (Sec. 2.2, caption of Fig. 2: the 8^4 blocks are
# decomposed further into an 8^4 Schur complement with Dirichlet boundaries and 4^4 blocks)

def dirichlet_links(U: np.ndarray, dims, cut: int) -> np.ndarray:
    """The links with every hop across a face of the cut^4 boxes removed (U_mu(x) = 0 where
    x_mu = cut - 1 mod cut): with them the hopping term of D is the direct sum of the boxes'
    Dirichlet operators D_k (hops inside the box).  The clover term is not computed from these."""
    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    X = np.stack(np.unravel_index(np.arange(V), dims), -1)
    out = np.array(U, dtype=np.complex128, copy=True).reshape(V, 4, 3, 3)
    for mu in range(4):
        out[X[:, mu] % cut == cut - 1, mu] = 0.0
    return out


def dirichlet_lattice(dims, block, U, csw, cut, antiperiodic_t=False) -> "core.Lattice":
    """A lattice whose operator is the direct sum of the cut^4 boxes' Dirichlet operators (clover
    term of the full field U, hops inside the boxes only), cut into blocks of length `block`."""
    lat = core.Lattice(dims, block, U, csw, antiperiodic_t)
    lat.set_hopping_links(dirichlet_links(U, dims, cut))
    return lat
