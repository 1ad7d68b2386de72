"""Python binding of the C ABI in ``include/ddrw.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/libddrw.so``; this module only converts
arrays to pointers and status codes to exceptions.  Arrays may be torch tensors (CUDA or CPU) or
numpy arrays, of dtype complex128 or float64 (interleaved re, im), C-contiguous.  If the library
is missing, loading fails with an error: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FP64, MIXED_FP32, MIXED_FP16, MIXED_BF16 = 0, 1, 2, 3
BLACK, WHITE, ALL = 0, 1, 2

_STATUS = {0: "DDRW_OK", 1: "DDRW_EINVAL", 2: "DDRW_ENOMEM", 3: "DDRW_ECUDA", 4: "DDRW_ENOCONV",
           5: "DDRW_ENUMERIC", 6: "DDRW_EDOMAIN", 7: "DDRW_ESTATE", 8: "DDRW_ETIMEOUT"}

#: every entry point declared in include/ddrw.h
EXPORTS = ["ddrw_create", "ddrw_destroy", "ddrw_last_error", "ddrw_suppP_size", "ddrw_volume", "ddrw_load_gauge",
           "ddrw_set_params", "ddrw_set_solver", "ddrw_set_outer_solver", "ddrw_set_block_solver",
           "ddrw_fuse_reductions", "ddrw_set_low_precision", "ddrw_block_config", "ddrw_set_max_rhs", "ddrw_set_dirichlet",
           "ddrw_block_factor_nested", "ddrw_apply_sap", "ddrw_apply_D", "ddrw_apply_block", "ddrw_solve_block",
           "ddrw_solve_D", "ddrw_apply_schur", "ddrw_apply_dA", "ddrw_solve_schur", "ddrw_noise", "ddrw_estimate",
           "ddrw_estimate_masses", "ddrw_profile", "ddrw_profile_read", "ddrw_solve_block_noalloc",
           "ddrw_autotune", "ddrw_autotune_report", "ddrw_stencil_config", "ddrw_profile_units",
           "ddrw_block_logdet", "ddrw_block_factor", "ddrw_estimate_variant", "ddrw_force", "ddrw_use_graphs",
           "ddrw_estimate_interp", "ddrw_apply_D_ds", "ddrw_test_stall_staging", "ddrw_apply_D_low"]

#: kernel classes of ddrw_profile_read
PROF_DSLASH64, PROF_DSLASH32, PROF_DSLASH64_BLK, PROF_DSLASH32_BLK, PROF_BLOCK64, PROF_BLOCK32, PROF_BLAS, PROF_DSLASH_DS, \
    PROF_DSLASH16, PROF_DSLASH16_BLK, PROF_BLOCK16, PROF_SAP, PROF_LAUNCHES = range(13)


class DDRWError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters_outer", ctypes.c_int), ("iters_inner_total", ctypes.c_int), ("cycles", ctypes.c_int),
                ("fp64_dslash_calls", ctypes.c_int),
                ("block_iters_max", ctypes.c_int), ("true_rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the CUDA library (build it first with ``paper_1211_1214_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)
    st = ctypes.c_int
    sig = {
        "ddrw_create": (st, [ctypes.POINTER(vp), ip, ip, ctypes.c_int, vp]),
        "ddrw_destroy": (None, [vp]),
        "ddrw_last_error": (ctypes.c_char_p, [vp]),
        "ddrw_suppP_size": (st, [vp, ctypes.POINTER(ctypes.c_long)]),
        "ddrw_volume": (st, [vp, ctypes.POINTER(ctypes.c_long)]),
        "ddrw_load_gauge": (st, [vp, dp]),
        "ddrw_set_params": (st, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
        "ddrw_set_solver": (st, [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
        "ddrw_set_outer_solver": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "ddrw_apply_sap": (st, [vp, ctypes.c_double, dp, dp, ctypes.c_int]),
        "ddrw_set_dirichlet": (st, [vp, ctypes.c_int]),
        "ddrw_set_block_solver": (st, [vp, ctypes.c_int]),
        "ddrw_fuse_reductions": (st, [vp, ctypes.c_int]),
        "ddrw_set_low_precision": (st, [vp, ctypes.c_int, ctypes.c_int]),
        "ddrw_block_config": (st, [vp, ctypes.c_int]),
        "ddrw_set_max_rhs": (st, [vp, ctypes.c_int]),
        "ddrw_block_factor_nested": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, dp, dp, dp]),
        "ddrw_apply_D": (st, [vp, ctypes.c_double, dp, dp, ctypes.c_int]),
        "ddrw_apply_D_ds": (st, [vp, ctypes.c_double, dp, dp, ctypes.c_int]),
        "ddrw_apply_D_low": (st, [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp, ctypes.c_int]),
        "ddrw_apply_block": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_int]),
        "ddrw_solve_block": (st, [vp, ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_int, ctypes.POINTER(SolveInfo)]),
        "ddrw_solve_D": (st, [vp, ctypes.c_double, dp, dp, ctypes.c_int, ctypes.POINTER(SolveInfo)]),
        "ddrw_apply_schur": (st, [vp, ctypes.c_double, ctypes.c_int, dp, dp, ctypes.c_int]),
        "ddrw_apply_dA": (st, [vp, dp, dp, ctypes.c_int, ctypes.POINTER(SolveInfo)]),
        "ddrw_solve_schur": (st, [vp, ctypes.c_double, dp, dp, ctypes.c_int, ctypes.POINTER(SolveInfo)]),
        "ddrw_noise": (st, [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, dp]),
        "ddrw_estimate": (st, [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, dp, dp, dp, dp, dp,
                               ctypes.POINTER(SolveInfo)]),
        "ddrw_estimate_masses": (st, [vp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, dp, dp,
                                      dp, ctypes.POINTER(SolveInfo)]),
        "ddrw_profile": (st, [vp, ctypes.c_int]),
        "ddrw_autotune": (st, [vp, ctypes.c_int]),
        "ddrw_stencil_config": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "ddrw_test_stall_staging": (st, [vp, ctypes.c_int]),
        "ddrw_profile_units": (st, [vp, ctypes.c_int, dp]),
        "ddrw_block_logdet": (st, [vp, ctypes.c_double, dp, dp]),
        "ddrw_block_factor": (st, [vp, dp]),
        "ddrw_estimate_variant": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                       dp, dp, dp, dp, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(SolveInfo)]),
        "ddrw_use_graphs": (st, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_long)]),
        "ddrw_estimate_interp": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, dp, dp, dp, dp,
                                      dp, dp, ctypes.POINTER(SolveInfo)]),
        "ddrw_force": (st, [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, dp, dp, dp, dp, dp,
                            ctypes.POINTER(SolveInfo)]),
        "ddrw_autotune_report": (st, [vp, ctypes.c_char_p, ctypes.c_long]),
        "ddrw_solve_block_noalloc": (st, [vp, ctypes.c_int, ctypes.c_double, dp, dp, ctypes.POINTER(SolveInfo)]),
        "ddrw_profile_read": (st, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """Data pointer of a contiguous complex128/float64 torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(a.dtype) not in ("torch.complex128", "torch.float64"):
            raise ValueError("tensor must be complex128 or float64")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if a.dtype not in (np.complex128, np.float64):
            raise ValueError("array must be complex128 or float64")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


class Context:
    """One ``ddrw_ctx``: a lattice with its blocks on one GPU.  Methods mirror the C calls."""

    def __init__(self, dims, block, device: int = 0, stream: int | None = None):
        self.L = load()
        self.dims = tuple(int(d) for d in dims)
        self.block = tuple(int(b) for b in (block if hasattr(block, "__len__") else [block] * 4))
        h = ctypes.c_void_p()
        st = self.L.ddrw_create(ctypes.byref(h), (ctypes.c_int * 4)(*self.dims), (ctypes.c_int * 4)(*self.block),
                                int(device), ctypes.c_void_p(stream) if stream else None)
        if st != 0:
            raise DDRWError(st, f"ddrw_create(dims={self.dims}, block={self.block})")
        self._h = h
        n = ctypes.c_long()
        self.L.ddrw_suppP_size(self._h, ctypes.byref(n))
        self.nP = n.value
        self.L.ddrw_volume(self._h, ctypes.byref(n))
        self.V = n.value

    def close(self):
        if getattr(self, "_h", None):
            self.L.ddrw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.L.ddrw_last_error(self._h)
            raise DDRWError(st, f"{what}: {msg.decode() if msg else ''}")

    def load_gauge(self, U):
        self._check(self.L.ddrw_load_gauge(self._h, _ptr(U)), "ddrw_load_gauge")

    def set_params(self, csw, m1, m2, antiperiodic_t=False):
        self._csw, self._m1, self._m2 = float(csw), float(m1), float(m2)
        self._check(self.L.ddrw_set_params(self._h, float(csw), float(m1), float(m2), int(antiperiodic_t)),
                    "ddrw_set_params")

    def set_solver(self, prec=FP64, tol_outer=1e-10, tol_block=1e-13, maxiter=20000):
        self._check(self.L.ddrw_set_solver(self._h, int(prec), float(tol_outer), float(tol_block), int(maxiter)),
                    "ddrw_set_solver")

    def set_outer_solver(self, method=1, ncy=4, nmr=4, nkv=8):
        """Krylov method of the FP32 inner solves: 0 even-odd BiCGStab, 1 Schwarz-preconditioned GCR."""
        self._check(self.L.ddrw_set_outer_solver(self._h, int(method), int(ncy), int(nmr), int(nkv)),
                    "ddrw_set_outer_solver")

    def apply_sap(self, m, x, out, nrhs=1):
        self._check(self.L.ddrw_apply_sap(self._h, float(m), _ptr(x), _ptr(out), int(nrhs)), "ddrw_apply_sap")

    def apply_D(self, m, x, out, nrhs=1):
        self._check(self.L.ddrw_apply_D(self._h, float(m), _ptr(x), _ptr(out), int(nrhs)), "ddrw_apply_D")

    def apply_D_ds(self, m, x, out, nrhs=1):
        self._check(self.L.ddrw_apply_D_ds(self._h, float(m), _ptr(x), _ptr(out), int(nrhs)), "ddrw_apply_D_ds")

    def apply_D_low(self, prec, m, x, out, nrhs=1, post=False):
        """out = D(m) x (post: A(m)^-1 D(m) x) by one stencil launch in storage precision prec."""
        self._check(self.L.ddrw_apply_D_low(self._h, int(prec), float(m), int(bool(post)), _ptr(x), _ptr(out),
                                            int(nrhs)), "ddrw_apply_D_low")

    def apply_block(self, rows, cols, m, x, out, nrhs=1):
        self._check(self.L.ddrw_apply_block(self._h, int(rows), int(cols), float(m), _ptr(x), _ptr(out), int(nrhs)),
                    "ddrw_apply_block")

    def solve_block(self, colour, m, b, x, nrhs=1):
        info = SolveInfo()
        st = self.L.ddrw_solve_block(self._h, int(colour), float(m), _ptr(b), _ptr(x), int(nrhs), ctypes.byref(info))
        self._check(st, "ddrw_solve_block")
        return info.as_dict()

    def solve_block_noalloc(self, colour, m, b, x):
        """ddrw_solve_block without device allocation (one right-hand side, device pointers)."""
        info = SolveInfo()
        st = self.L.ddrw_solve_block_noalloc(self._h, int(colour), float(m), _ptr(b), _ptr(x), ctypes.byref(info))
        self._check(st, "ddrw_solve_block_noalloc")
        return info.as_dict()

    def solve_D(self, m, b, x, nrhs=1):
        info = SolveInfo()
        st = self.L.ddrw_solve_D(self._h, float(m), _ptr(b), _ptr(x), int(nrhs), ctypes.byref(info))
        self._check(st, "ddrw_solve_D")
        return info.as_dict()

    def apply_schur(self, m, x, out, nrhs=1, dagger=False):
        self._check(self.L.ddrw_apply_schur(self._h, float(m), int(bool(dagger)), _ptr(x), _ptr(out), int(nrhs)),
                    "ddrw_apply_schur")

    def apply_dA(self, eta, r, nrhs=1):
        info = SolveInfo()
        self._check(self.L.ddrw_apply_dA(self._h, _ptr(eta), _ptr(r), int(nrhs), ctypes.byref(info)), "ddrw_apply_dA")
        return info.as_dict()

    def solve_schur(self, m, b, x, nrhs=1):
        info = SolveInfo()
        st = self.L.ddrw_solve_schur(self._h, float(m), _ptr(b), _ptr(x), int(nrhs), ctypes.byref(info))
        self._check(st, "ddrw_solve_schur")
        return info.as_dict()

    def noise(self, seed, hit_offset, nhit, eta):
        self._check(self.L.ddrw_noise(self._h, ctypes.c_uint64(seed), ctypes.c_uint64(hit_offset), int(nhit),
                                      _ptr(eta)), "ddrw_noise")

    def estimate(self, nhit, seed=2, hit_offset=0, eta=None, delta=None):
        """Returns (exponents as numpy float64 array, logW, rel_var, solve info dict)."""
        e = np.zeros(nhit, dtype=np.float64)
        lw = np.zeros(1, dtype=np.float64)
        rv = np.zeros(1, dtype=np.float64)
        info = SolveInfo()
        st = self.L.ddrw_estimate(self._h, int(nhit), ctypes.c_uint64(seed), ctypes.c_uint64(hit_offset), _ptr(eta),
                                  _ptr(e), _ptr(lw), _ptr(rv), _ptr(delta), ctypes.byref(info))
        self._check(st, "ddrw_estimate")
        return e, float(lw[0]), float(rv[0]), info.as_dict()

    def force(self, nhit, seed=2, hit_offset=0, eta=None, weights=None, dU=None, want_dm2=True):
        """Exponents, link force sum_j w_j de_j/dU (written into dU, [V,4,8] float64, if given) and
        de_j/dm2.  Returns (exponents, dm2, solve info)."""
        e = np.zeros(nhit, dtype=np.float64)
        dm = np.zeros(nhit, dtype=np.float64) if want_dm2 else None
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
        info = SolveInfo()
        st = self.L.ddrw_force(self._h, int(nhit), ctypes.c_uint64(seed), ctypes.c_uint64(hit_offset), _ptr(eta),
                               _ptr(w), _ptr(e), _ptr(dU), _ptr(dm), ctypes.byref(info))
        self._check(st, "ddrw_force")
        return e, dm, info.as_dict()

    def use_graphs(self, enable=None):
        """Graph mode (2, the default: Krylov loops; True / 1: Krylov loops and whole estimate chunks
        with device-controlled cycles; False / 0: none; None: keep); returns graph launches so far."""
        n = ctypes.c_long()
        self._check(self.L.ddrw_use_graphs(self._h, -1 if enable is None else int(enable), ctypes.byref(n)),
                    "ddrw_use_graphs")
        return n.value

    def autotune(self, enable=True):
        self._check(self.L.ddrw_autotune(self._h, int(enable)), "ddrw_autotune")

    def block_logdet(self, m):
        """log |det D_k(m)| and sign for every block (Eq. 7), library block numbering."""
        nb = self.V // (self.block[0] * self.block[1] * self.block[2] * self.block[3])
        ld = np.zeros(nb)
        sg = np.zeros(nb)
        self._check(self.L.ddrw_block_logdet(self._h, float(m), _ptr(ld), _ptr(sg)), "ddrw_block_logdet")
        return ld, sg

    def estimate_variant(self, variant, N, nhit, seed=2, hit_offset=0, eta=None):
        """Fig. 1's operator variants (0 total, 1 even-odd, 2 blocks) of the interpolated estimate:
        returns (exponents [N, nhit], log W, rel_var [N], support dimension, solve info)."""
        e = np.zeros((N, nhit))
        rv = np.zeros(N)
        lw = ctypes.c_double(0)
        dim = ctypes.c_long(0)
        info = SolveInfo()
        ep = None if eta is None else np.ascontiguousarray(eta, dtype=np.complex128)
        st = self.L.ddrw_estimate_variant(self._h, int(variant), int(N), int(nhit), int(seed), int(hit_offset),
                                          None if ep is None else _ptr(ep), _ptr(e), ctypes.byref(lw), _ptr(rv),
                                          ctypes.byref(dim), ctypes.byref(info))
        self._check(st, "ddrw_estimate_variant")
        return e, lw.value, rv, dim.value, info.as_dict()

    def block_factor(self):
        """log prod_k det D_k^2(m2) / det D_k^2(m1) for the current m1, m2 (Eq. 7)."""
        v = ctypes.c_double(0)
        self._check(self.L.ddrw_block_factor(self._h, ctypes.byref(v)), "ddrw_block_factor")
        return v.value

    def block_factor_nested(self, lsub, nhit, seed=2):
        """Eq. 7's block factor by the nested decomposition (Sec. 2.2): returns (total, exact sub-block
        part, stochastic Schur part, exponents[nhit], relative sample variance)."""
        out, e, rv = np.zeros(3), np.zeros(int(nhit)), np.zeros(1)
        self._check(self.L.ddrw_block_factor_nested(self._h, int(lsub), int(nhit), ctypes.c_uint64(seed),
                                                     _ptr(out), _ptr(e), _ptr(rv)), "ddrw_block_factor_nested")
        return float(out[0]), float(out[1]), float(out[2]), e, float(rv[0])

    def set_low_precision(self, reliable_updates=True, block_solves_16bit=False):
        """16-bit precisions: reliable updates in the inner solves; 16-bit or FP32 block solves."""
        self._check(self.L.ddrw_set_low_precision(self._h, int(bool(reliable_updates)), int(bool(block_solves_16bit))),
                    "ddrw_set_low_precision")

    def set_max_rhs(self, max_rhs=0):
        """Right-hand sides per chunk of the batched estimates (0: sized from free device memory)."""
        self._check(self.L.ddrw_set_max_rhs(self._h, int(max_rhs)), "ddrw_set_max_rhs")

    def block_config(self, form=-1):
        """Persistent block-solver launch shape: -1 tuned, 0 / 1 one right-hand side per CTA of 256 /
        512 threads, 2 two right-hand sides per CTA."""
        self._check(self.L.ddrw_block_config(self._h, int(form)), "ddrw_block_config")

    def fuse_reductions(self, enable=True):
        """Inner products of the BiCGStab recurrence in the stencil epilogue (True) or separate kernels."""
        self._check(self.L.ddrw_fuse_reductions(self._h, int(bool(enable))), "ddrw_fuse_reductions")

    def set_block_solver(self, method):
        """Block solves of the mixed precisions: 0 persistent kernel, 1 Krylov-loop BiCGStab."""
        self._check(self.L.ddrw_set_block_solver(self._h, int(method)), "ddrw_set_block_solver")

    def set_dirichlet(self, cut):
        """Remove the hops across the faces of cut^4 boxes (before load_gauge)."""
        self._check(self.L.ddrw_set_dirichlet(self._h, int(cut)), "ddrw_set_dirichlet")

    def stencil_config(self, nr=0, nt=128, nw=1, roll=0):
        """Pin the stencil launch configuration (nr = 0: back to the autotuner)."""
        self._check(self.L.ddrw_stencil_config(self._h, int(nr), int(nt), int(nw), int(roll)), "ddrw_stencil_config")

    def test_stall_staging(self, enable):
        """Test switch: staged stencil launches wait for bytes that never come (bounded wait, then
        DDRW_ETIMEOUT); False restores normal operation."""
        self._check(self.L.ddrw_test_stall_staging(self._h, int(bool(enable))), "ddrw_test_stall_staging")

    def autotune_report(self):
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self.L.ddrw_autotune_report(self._h, buf, len(buf)), "ddrw_autotune_report")
        return buf.value.decode()

    def profile(self, enable=True):
        self._check(self.L.ddrw_profile(self._h, int(enable)), "ddrw_profile")

    def profile_units(self, kind):
        """Site updates (sites x right-hand sides) of the timed launches of a stencil class."""
        u = ctypes.c_double(0)
        self._check(self.L.ddrw_profile_units(self._h, int(kind), ctypes.byref(u)), "ddrw_profile_units")
        return u.value

    def profile_read(self, kind):
        """(launches, summed device ms, summed compulsory bytes) of one kernel class."""
        n, ms, b = ctypes.c_long(), ctypes.c_double(), ctypes.c_double()
        self._check(self.L.ddrw_profile_read(self._h, int(kind), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b)),
                    "ddrw_profile_read")
        return n.value, ms.value, b.value

    def estimate_interp(self, N, nhit, seed=2, hit_offset=0):
        """Mass interpolation in N steps (Eq. 8) with the one-flavour estimator (Eq. 11).  Returns a
        dict: exponents [N, nhit], exponents_1f [N, nhit] complex, logW (two flavours), logW_1f,
        sign_1f, logW_root, logW_factors [N], rel_var [N], info."""
        e = np.zeros((N, nhit), dtype=np.float64)
        e1 = np.zeros((N, nhit, 2), dtype=np.float64)
        lw = np.zeros(4, dtype=np.float64)
        lf = np.zeros(N, dtype=np.float64)
        rv = np.zeros(N, dtype=np.float64)
        rv1 = np.zeros(N, dtype=np.float64)
        info = SolveInfo()
        st = self.L.ddrw_estimate_interp(self._h, int(N), int(nhit), ctypes.c_uint64(seed), ctypes.c_uint64(hit_offset),
                                         _ptr(e), _ptr(e1), _ptr(lw), _ptr(lf), _ptr(rv), _ptr(rv1), ctypes.byref(info))
        self._check(st, "ddrw_estimate_interp")
        return {"exponents": e, "exponents_1f": e1[..., 0] + 1j * e1[..., 1], "logW": lw[0], "logW_1f": lw[1],
                "sign_1f": lw[2], "logW_root": lw[3], "logW_factors": lf, "rel_var": rv, "rel_var_1f": rv1,
                "info": info.as_dict()}

    def estimate_masses(self, m2s, nhit, seed=2, hit_offset=0):
        """Batched estimate for several target masses: (exponents [nmass, nhit], logW [nmass],
        rel_var [nmass], solve info)."""
        m = np.ascontiguousarray(m2s, dtype=np.float64)
        e = np.zeros((len(m), nhit), dtype=np.float64)
        lw = np.zeros(len(m), dtype=np.float64)
        rv = np.zeros(len(m), dtype=np.float64)
        info = SolveInfo()
        st = self.L.ddrw_estimate_masses(self._h, len(m), _ptr(m), int(nhit), ctypes.c_uint64(seed),
                                         ctypes.c_uint64(hit_offset), _ptr(e), _ptr(lw), _ptr(rv), ctypes.byref(info))
        self._check(st, "ddrw_estimate_masses")
        return e, lw, rv, info.as_dict()
