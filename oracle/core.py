"""ctypes binding of the C oracle (``ddrw_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Vectors are numpy complex128 arrays in the
boundary layout: ``[site][spin 4][colour 3]`` with lexicographic sites ``((t*X + x)*Y + y)*Z + z``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddrw_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libddrw_oracle.so")

BLACK, WHITE, ALL = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no target-specific flags); returns the .so path."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ip, ip, dp, ctypes.c_double, ctypes.c_int]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_hopping_links.argtypes = [ctypes.c_void_p, dp]
        L.orc_volume.restype = ctypes.c_long
        L.orc_volume.argtypes = [ctypes.c_void_p]
        L.orc_clover_matrix.argtypes = [ctypes.c_void_p, ctypes.c_long, dp]
        L.orc_colour.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_suppP.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_apply.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_solve.restype = ctypes.c_long
        L.orc_solve.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, dp, dp, ctypes.c_double,
                                ctypes.c_long, dp]
        L.orc_exponent.restype = ctypes.c_int
        L.orc_exponent.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, dp, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_long, dp, dp, dp, ctypes.POINTER(ctypes.c_long)]
        L.orc_force.restype = ctypes.c_int
        L.orc_force.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double,
                                ctypes.c_long, dp, dp, dp]
        L.orc_gamma.argtypes = [ctypes.c_int, dp]
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_noise.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_long, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gamma(mu: int) -> np.ndarray:
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().orc_gamma(mu, _dp(out))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def noise_packed(seed: int, hit0: int, nhit: int, n: int) -> np.ndarray:
    """Packed complex Gaussian noise, shape (nhit, n): component k of hit h from Philox (k, hit0+h)."""
    out = np.zeros((nhit, n), dtype=np.complex128)
    lib().orc_noise(ctypes.c_uint64(seed), ctypes.c_uint64(hit0), nhit, n, _dp(out))
    return out


class Lattice:
    """A gauge configuration with its clover term and block geometry, held by the C oracle."""

    def __init__(self, dims, block, U: np.ndarray, csw: float, antiperiodic_t: bool = False):
        self.dims = tuple(int(d) for d in dims)
        self.block = tuple(int(b) for b in block)
        self.V = int(np.prod(self.dims))
        for L, b in zip(self.dims, self.block):
            if L % b:
                raise ValueError("block must divide the lattice")
        U = np.ascontiguousarray(U, dtype=np.complex128)
        if U.shape != (self.V, 4, 3, 3):
            raise ValueError("U must have shape (V, 4, 3, 3)")
        Ld = (ctypes.c_int * 4)(*self.dims)
        Bd = (ctypes.c_int * 4)(*self.block)
        self.csw = float(csw)
        self._h = lib().orc_create(Ld, Bd, _dp(U), self.csw, int(antiperiodic_t))
        if not self._h:
            raise MemoryError("oracle allocation failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    def set_hopping_links(self, U: np.ndarray) -> None:
        """Links of the hopping term from now on; the clover term stays the one of the creation links."""
        U = np.ascontiguousarray(U, dtype=np.complex128)
        if U.shape != (self.V, 4, 3, 3):
            raise ValueError("U must have shape (V, 4, 3, 3)")
        lib().orc_set_hopping_links(self._h, _dp(U))

    # -- geometry
    def colour(self) -> np.ndarray:
        out = np.zeros(self.V, dtype=np.uint8)
        lib().orc_colour(self._h, out.ctypes.data)
        return out

    def suppP(self) -> np.ndarray:
        out = np.zeros(self.V, dtype=np.uint8)
        lib().orc_suppP(self._h, out.ctypes.data)
        return out

    def suppP_sites(self) -> np.ndarray:
        return np.nonzero(self.suppP())[0]

    def pack(self, v: np.ndarray) -> np.ndarray:
        """Full-lattice vector (V,4,3) -> packed supp P list (n,) in ascending site order."""
        return np.ascontiguousarray(v.reshape(self.V, 12)[self.suppP_sites()].reshape(-1))

    def unpack(self, p: np.ndarray) -> np.ndarray:
        out = np.zeros((self.V, 12), dtype=np.complex128)
        out[self.suppP_sites()] = p.reshape(-1, 12)
        return out.reshape(self.V, 4, 3)

    # -- operator
    def clover(self, site: int) -> np.ndarray:
        out = np.zeros((12, 12), dtype=np.complex128)
        lib().orc_clover_matrix(self._h, site, _dp(out))
        return out

    def apply(self, m: float, v: np.ndarray, dagger: bool = False, rows: int = ALL, cols: int = ALL) -> np.ndarray:
        """out = D_{rows,cols}(m) v (or the adjoint), full-lattice vectors of shape (V, 4, 3)."""
        v = np.ascontiguousarray(v, dtype=np.complex128).reshape(self.V, 4, 3)
        out = np.zeros_like(v)
        lib().orc_apply(self._h, float(m), int(dagger), int(rows), int(cols), _dp(v), _dp(out))
        return out

    def solve(self, m: float, b: np.ndarray, sel: int = ALL, tol: float = 1e-12, maxiter: int = 100000):
        """CGNR solve of D_{sel,sel}(m) x = b.  Returns (x, iterations, true relative residual)."""
        b = np.ascontiguousarray(b, dtype=np.complex128).reshape(self.V, 4, 3)
        x = np.zeros_like(b)
        rel = ctypes.c_double(0)
        it = lib().orc_solve(self._h, float(m), int(sel), _dp(b), _dp(x), float(tol), int(maxiter),
                             ctypes.byref(rel))
        if it < 0:
            raise RuntimeError(f"oracle CGNR did not converge (relres {rel.value:.3e})")
        return x, int(it), rel.value

    def exponent(self, m1: float, m2: float, eta: np.ndarray, tol_block: float = 1e-13,
                 tol_outer: float = 1e-12, maxiter: int = 100000):
        """e = eta^dag (Mh^dag Mh - 1) eta for one full-lattice eta supported on supp P.

        Returns a dict with e, r, delta (full-lattice) and the CGNR counts of the five solves.
        """
        eta = np.ascontiguousarray(eta, dtype=np.complex128).reshape(self.V, 4, 3)
        r = np.zeros_like(eta)
        delta = np.zeros_like(eta)
        e = ctypes.c_double(0)
        iters = (ctypes.c_long * 5)()
        st = lib().orc_exponent(self._h, float(m1), float(m2), _dp(eta), float(tol_block), float(tol_outer),
                                int(maxiter), ctypes.byref(e), _dp(r), _dp(delta), iters)
        if st != 0:
            raise RuntimeError("oracle solve did not converge")
        return {"e": e.value, "r": r, "delta": delta, "iters": list(iters)}


def _force(self, m1, m2, eta, tol_block=1e-13, tol_outer=1e-13, maxiter=100000, links=True):
    """Link derivatives dU[x, mu, a] = de/dt for U_mu(x) -> exp(i t lambda_a/2) U_mu(x) and de/dm2."""
    eta = np.ascontiguousarray(eta, dtype=np.complex128).reshape(self.V, 4, 3)
    e = ctypes.c_double(0)
    dm2 = ctypes.c_double(0)
    dU = np.zeros((self.V, 4, 8), dtype=np.float64) if links else None
    st = lib().orc_force(self._h, float(m1), float(m2), _dp(eta), float(tol_block), float(tol_outer), int(maxiter),
                         ctypes.byref(e), _dp(dU) if links else None, ctypes.byref(dm2))
    if st != 0:
        raise RuntimeError("oracle solve did not converge")
    return e.value, dU, dm2.value


Lattice.force = _force


def log_w(exponents) -> float:
    """log W_gl = log((1/N_hit) sum_j exp(-e_j)) by log-sum-exp in FP64 (Eq. 3, Eq. 8 with N = 1)."""
    e = -np.asarray(exponents, dtype=np.float64)
    mx = e.max()
    return float(mx + np.log(np.mean(np.exp(e - mx))))
