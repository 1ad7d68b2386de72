"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and nothing else of the method: it holds no Dirac operator,
no block decomposition, no solver and no estimator.  Both the CUDA path and the CPU oracle
receive what it returns as plain arrays.

Layouts (the library's boundary layout):

* site index ``((t*L1 + x)*L2 + y)*L3 + z`` with ``dims = (L0, L1, L2, L3) = (T, X, Y, Z)``;
* gauge field ``U[site][mu][a][b]`` complex128, ``mu = 0..3`` is ``t, x, y, z``;
* spinor ``psi[site][alpha][a]`` complex128, 4 spins x 3 colours.

The gauge links follow the recipe of the workloads: ``U = exp(i eps H)`` with
``H = sum_a w_a lambda_a / 2`` (Gell-Mann matrices ``lambda_a``) and ``w_a ~ N(0, 1)``, which
makes every link an SU(3) matrix whose distance from the identity is set by ``eps``.  The
paper's CLS configurations (Sec. 2, 48x24^3 and 64x32^3 at beta = 5.3) are not available; these
fields have the same lattice shapes and stand in for them.
"""
from __future__ import annotations

import numpy as np

__all__ = ["gell_mann", "gauge_field", "spinor_field", "complex_gaussian", "gauge_transform"]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3), complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _expm_batch(A: np.ndarray) -> np.ndarray:
    """exp(A) for a batch of small anti-Hermitian 3x3 matrices by scaling and squaring of a Taylor
    series; the result is projected back to SU(3) by the caller."""
    nrm = np.abs(A).sum(axis=(-2, -1)).max() if A.size else 0.0
    s = max(0, int(np.ceil(np.log2(max(nrm, 1e-300)))) + 1)
    As = A / (2.0 ** s)
    out = np.broadcast_to(np.eye(3, dtype=A.dtype), A.shape).copy()
    term = out.copy()
    for k in range(1, 18):
        term = term @ As / k
        out += term
    for _ in range(s):
        out = out @ out
    return out


def _expm_i_traceless_hermitian(Q: np.ndarray) -> np.ndarray:
    """exp(iQ) for a batch of traceless Hermitian 3x3 Q, from the spectral decomposition.

    The eigenvalues solve l^3 - c1 l - c0 = 0 with c1 = tr(Q^2)/2 and c0 = det Q (trigonometric
    solution of the cubic); exp(iQ) = sum_j e^{i l_j} (Q - l_k)(Q - l_m) / ((l_j - l_k)(l_j - l_m)).
    Matrices with nearly degenerate eigenvalues fall back to the Taylor series.
    """
    Q2 = Q @ Q
    c1 = 0.5 * np.real(np.einsum("nii->n", Q2))
    a, b, c = Q[:, 0], Q[:, 1], Q[:, 2]
    c0 = np.real(a[:, 0] * (b[:, 1] * c[:, 2] - b[:, 2] * c[:, 1]) - a[:, 1] * (b[:, 0] * c[:, 2] - b[:, 2] * c[:, 0])
                 + a[:, 2] * (b[:, 0] * c[:, 1] - b[:, 1] * c[:, 0]))
    c1s = np.maximum(c1, 1e-300)
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        arg = np.clip(0.5 * c0 * (3.0 / c1s) ** 1.5, -1.0, 1.0)
    phi = np.arccos(arg) / 3.0
    rad = 2.0 * np.sqrt(c1s / 3.0)
    lam = np.stack([rad * np.cos(phi - 2.0 * np.pi * k / 3.0) for k in range(3)], axis=-1)
    l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
    d = np.stack([(l0 - l1) * (l0 - l2), (l1 - l0) * (l1 - l2), (l2 - l0) * (l2 - l1)], axis=-1)
    e = np.exp(1j * lam)
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        w = e / np.where(np.abs(d) > 0, d, 1.0)
    A = w.sum(-1)
    B = (w * lam).sum(-1)
    C = w[:, 0] * l1 * l2 + w[:, 1] * l0 * l2 + w[:, 2] * l0 * l1
    out = A[:, None, None] * Q2 + B[:, None, None] * Q + C[:, None, None] * np.eye(3)
    # nearly degenerate spectra (and Q = 0, where the trigonometric solution is 0/0) take the series
    bad = ~(np.abs(d).min(axis=-1) >= 1e-6 * np.maximum(c1, 1e-30)) | ~np.isfinite(out).all(axis=(-2, -1))
    if np.any(bad):
        out[bad] = _expm_batch(1j * Q[bad])
    return out


def _project_su3(U: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1): unitary with det exactly 1."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - (np.sum(np.conj(r0) * r1, axis=-1, keepdims=True)) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 16) -> np.ndarray:
    """SU(3) links U = exp(i eps H), H = sum_a w_a lambda_a/2, w_a ~ N(0,1); shape (V, 4, 3, 3).

    All 8*4*V normals are drawn from one ``numpy.random.default_rng(seed)`` stream in the order
    (site, mu, a), so the field depends on neither ``chunk`` nor the number of threads that
    exponentiate the chunks.
    """
    import concurrent.futures as cf
    import os

    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    omega = rng.standard_normal((V * 4, 8))
    lam_half = (gell_mann() / 2.0).reshape(8, 9)
    U = np.empty((V * 4, 3, 3), dtype=np.complex128)

    def work(lo):
        hi = min(V * 4, lo + chunk)
        w = omega[lo:hi] * eps
        H = (w @ lam_half.real + 1j * (w @ lam_half.imag)).reshape(-1, 3, 3)
        U[lo:hi] = _project_su3(_expm_i_traceless_hermitian(H))

    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        list(ex.map(work, range(0, V * 4, chunk)))
    return U.reshape(V, 4, 3, 3)


def complex_gaussian(shape, seed: int) -> np.ndarray:
    """Complex Gaussian entries with E|z|^2 = 1 (real and imaginary parts ~ N(0, 1/2))."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(tuple(shape) + (2,)) * np.sqrt(0.5)
    return z[..., 0] + 1j * z[..., 1]


def spinor_field(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Random spinor field(s), shape (V, 4, 3) or (nrhs, V, 4, 3), complex128."""
    V = int(np.prod(dims))
    shape = (V, 4, 3) if nrhs is None else (nrhs, V, 4, 3)
    return complex_gaussian(shape, seed)


def gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix per site, shape (V, 3, 3), for gauge-covariance checks."""
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    omega = rng.standard_normal((V, 8))
    H = np.einsum("na,aij->nij", omega, gell_mann() / 2.0)
    return _project_su3(_expm_i_traceless_hermitian(H))
