"""Thin ctypes binding of libomm_gb300.so (argument marshalling only).

Every step of the solve runs in the library's CUDA kernels; this module only
turns numpy arrays (host memory) and torch CUDA tensors (device memory) into
the plain pointers and sizes of the C ABI declared in include/omm.h.  There
is no fallback: if the library is missing, importing a function raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libomm_gb300.so")

OK = 0
ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_NOT_SPD, ERR_LINESEARCH = -1, -2, -3, -4, -5
ERR_MAXITER, ERR_PATTERN, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = -6, -7, -8, -9, -10, -11
PREC_FP64, PREC_MIXED = 0, 1
REFINE_EXACT, REFINE_FP64 = 0, 1

ARRAY_W, ARRAY_HW, ARRAY_SW, ARRAY_G, ARRAY_D, ARRAY_HW_N, ARRAY_SW_N = range(7)
PATTERN_H, PATTERN_W, PATTERN_HW, PATTERN_N = range(4)
DENSITY_RHO, DENSITY_RHO_E = 0, 1


class Options(C.Structure):
    _fields_ = [("eta", C.c_double), ("eta_auto", C.c_int32), ("precision", C.c_int32),
                ("cholesky", C.c_int32), ("max_iter", C.c_int32), ("orth_tol", C.c_double),
                ("filter_eps", C.c_double), ("stream", C.c_void_p), ("refine", C.c_int32),
                ("exact_digits", C.c_int32), ("split_digits", C.c_int32), ("graphs", C.c_int32),
                ("n_occupied", C.c_int32), ("precon", C.c_int32), ("tau_T", C.c_double),
                ("screen_eps", C.c_double), ("gemm_pair", C.c_int32),
                ("gemm_persistent", C.c_int32), ("dir_digits", C.c_int32)]


class Pattern(C.Structure):
    _fields_ = [("bm", C.c_int32), ("bn", C.c_int32), ("nbr", C.c_int64), ("nbc", C.c_int64),
                ("H_rowptr", C.c_void_p), ("H_col", C.c_void_p),
                ("W_rowptr", C.c_void_p), ("W_col", C.c_void_p)]


class Diag(C.Structure):
    _fields_ = [("E", C.c_double), ("E_rel_change", C.c_double), ("orth", C.c_double),
                ("charge", C.c_double), ("eta", C.c_double), ("iters", C.c_int32),
                ("status", C.c_int32), ("iters_mixed", C.c_int32), ("iters_refine", C.c_int32),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double), ("nnzb_H", C.c_int64),
                ("nnzb_W", C.c_int64), ("nnzb_HW", C.c_int64), ("nnzb_N", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_SIGS = {
    "omm_default_options": (None, [C.POINTER(Options)]),
    "omm_create": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, C.c_void_p, C.POINTER(Options),
                             C.POINTER(C.c_void_p)]),
    "omm_set_HS": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "omm_set_H": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "omm_set_T": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "omm_md_guess": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "omm_selftest_bounded_wait": (C.c_int, [C.c_int64, C.POINTER(C.c_int32), C.c_void_p]),
    "omm_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_int32,
                            C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "omm_get_diag": (C.c_int, [C.c_void_p, C.POINTER(Diag)]),
    "omm_get_array": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "omm_get_density": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "omm_destroy": (None, [C.c_void_p]),
    "omm_status_str": (C.c_char_p, [C.c_int]),
    "omm_op_dgemm": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_double,
                               C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                               C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]),
    "omm_op_quartic_coeffs_scratch_bytes": (C.c_int64, [C.c_int64]),
    "omm_op_quartic_coeffs": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.c_void_p, C.c_int64, C.c_void_p]),
    "omm_op_line_min": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "omm_op_convert": (C.c_int, [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "omm_op_quartic_coeffs_static_max_bytes": (C.c_int64, []),
    "omm_op_quartic_coeffs_static": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                               C.c_void_p]),
    "omm_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "omm_get_stage_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "omm_kernel_launches": (C.c_int64, []),
    "omm_last_error": (C.c_char_p, []),
    "omm_get_pattern": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "omm_solve_begin": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double]),
    "omm_solve_progress": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "omm_solve_end": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "omm_batch_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_double, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "omm_batch_solve_grouped": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_double, C.c_int32,
                                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "omm_batch_last_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "omm_op_exact_gemm_workspace_bytes": (C.c_int64, [C.c_int64, C.c_int64, C.c_int64, C.c_int32]),
    "omm_op_exact_gemm": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                    C.c_double, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.c_double, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.c_void_p, C.c_int64, C.c_void_p]),
    "omm_op_split_gemm_workspace_bytes": (C.c_int64, [C.c_int64, C.c_int64, C.c_int64, C.c_int32]),
    "omm_op_split_gemm": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                    C.c_double, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.c_double, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.c_void_p, C.c_int64, C.c_void_p]),
}

NSTAGES = 11


def lib():
    """Load libomm_gb300.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build(); "
                               "there is no non-CUDA implementation")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class OmmError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = lib().omm_status_str(status).decode()
        detail = lib().omm_last_error().decode()
        msg = f"{msg} ({status})" + (f" [{detail}]" if detail else "")
        super().__init__(f"{what}: {msg}" if what else msg)


def check(status, what=""):
    if status != OK:
        raise OmmError(status, what)
    return status


def status_str(status: int) -> str:
    return lib().omm_status_str(status).decode()


# ---------------------------------------------------------------- marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device) of a numpy array or a torch tensor; None -> (None, 0)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        return C.c_void_p(x.data_ptr()), int(x.is_cuda)
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 and x.dtype not in (np.int64, np.int32):
            raise TypeError("expected float64 arrays")
        return C.c_void_p(x.ctypes.data), 0
    raise TypeError(f"unsupported array type {type(x)}")


def colmajor(A: np.ndarray) -> np.ndarray:
    return np.asfortranarray(np.asarray(A, dtype=np.float64))


def _check_colmajor(x, rows, cols, name):
    if _is_torch(x):
        if tuple(x.shape) != (rows, cols):
            raise ValueError(f"{name}: shape {tuple(x.shape)} != {(rows, cols)}")
        if cols > 1 and rows > 1 and x.stride() != (1, rows):
            raise ValueError(f"{name}: must be column-major contiguous (stride (1, {rows}))")
        if str(x.dtype) != "torch.float64":
            raise TypeError(f"{name}: float64 required")
    else:
        if x.shape != (rows, cols):
            raise ValueError(f"{name}: shape {x.shape} != {(rows, cols)}")
        if not x.flags["F_CONTIGUOUS"] or x.dtype != np.float64:
            raise ValueError(f"{name}: must be a float64 Fortran-ordered array")


def selftest_bounded_wait(limit_ns: int, stream=None) -> int:
    """Run one bounded mbarrier wait that nothing completes; returns its status
    (ERR_TIMEOUT expected); see omm_selftest_bounded_wait."""
    st = C.c_int32(0)
    check(lib().omm_selftest_bounded_wait(int(limit_ns), C.byref(st), C.c_void_p(stream) if stream else None),
          "omm_selftest_bounded_wait")
    return st.value


def default_options(**kw) -> Options:
    o = Options()
    lib().omm_default_options(C.byref(o))
    known = {name for name, _ in Options._fields_}
    unknown = sorted(set(kw) - known)
    if unknown:
        raise TypeError(f"unknown omm option(s) {unknown}; known: {sorted(known)}")
    for k, v in kw.items():
        if k == "stream":
            v = C.c_void_p(v) if v is not None else None
        setattr(o, k, v)
    return o


class Solver:
    """One omm_handle (dense form)."""

    def __init__(self, m: int, n: int, block_size: int = 8, pattern=None, **options):
        self.m, self.n = m, n
        self._opts = default_options(**options)
        h = C.c_void_p()
        pat = None
        if pattern is not None:
            pat = C.byref(pattern)
        check(lib().omm_create(m, n, block_size, pat, C.byref(self._opts), C.byref(h)), "omm_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().omm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_HS(self, H, S):
        _check_colmajor(H, self.m, self.m, "H")
        _check_colmajor(S, self.m, self.m, "S")
        pH, dH = _ptr(H)
        pS, dS = _ptr(S)
        if dH != dS:
            raise ValueError("H and S must both be host or both device arrays")
        return check(lib().omm_set_HS(self._h, pH, pS, dH), "omm_set_HS")

    def set_H(self, H):
        """New H with the previous S (and Cholesky factor) kept; see omm_set_H."""
        _check_colmajor(H, self.m, self.m, "H")
        pH, dH = _ptr(H)
        return check(lib().omm_set_H(self._h, pH, dH), "omm_set_H")

    def set_T(self, T):
        """Kinetic-energy matrix of the preconditioner P = (S + T/tau_T)^-1; see omm_set_T."""
        _check_colmajor(T, self.m, self.m, "T")
        pT, dT = _ptr(T)
        return check(lib().omm_set_T(self._h, pT, dT), "omm_set_T")

    def md_guess(self, prev, prev2=None):
        """Resident W <- prev's solution carried onto this handle's pattern, or the
        linear extrapolation 2 W_prev - W_prev2; see omm_md_guess."""
        return check(lib().omm_md_guess(self._h, prev._h, prev2._h if prev2 is not None else None),
                     "omm_md_guess")

    def solve(self, W0=None, tol: float = 1e-10, W_out=None, raise_on_error=True):
        if W0 is not None:
            _check_colmajor(W0, self.m, self.n, "W0")
        if W_out is not None:
            _check_colmajor(W_out, self.m, self.n, "W_out")
        p0, d0 = _ptr(W0)
        po, do = _ptr(W_out)
        E = C.c_double(0.0)
        it = C.c_int32(0)
        st = lib().omm_solve(self._h, p0, d0, float(tol), po, do, C.byref(E), C.byref(it))
        if raise_on_error and st not in (OK,):
            raise OmmError(st, "omm_solve")
        return E.value, it.value, st

    def diag(self) -> Diag:
        d = Diag()
        check(lib().omm_get_diag(self._h, C.byref(d)), "omm_get_diag")
        return d

    # asynchronous driver
    def begin(self, W0=None, tol: float = 1e-10):
        p0, d0 = _ptr(W0)
        return check(lib().omm_solve_begin(self._h, p0, d0, float(tol)), "omm_solve_begin")

    def progress(self, blocking: bool = False) -> bool:
        done = C.c_int32(0)
        check(lib().omm_solve_progress(self._h, int(blocking), C.byref(done)), "omm_solve_progress")
        return bool(done.value)

    def end(self, W_out=None, raise_on_error=True):
        po, do = _ptr(W_out)
        E = C.c_double(0.0)
        it = C.c_int32(0)
        st = lib().omm_solve_end(self._h, po, do, C.byref(E), C.byref(it))
        if raise_on_error and st != OK:
            raise OmmError(st, "omm_solve_end")
        return E.value, it.value, st

    def set_profiling(self, on: bool):
        check(lib().omm_set_profiling(self._h, int(on)), "omm_set_profiling")

    def stage_times(self, reset: bool = False):
        ms = np.zeros(NSTAGES)
        cnt = np.zeros(NSTAGES, dtype=np.int64)
        check(lib().omm_get_stage_times(self._h, C.c_void_p(ms.ctypes.data), C.c_void_p(cnt.ctypes.data),
                                        NSTAGES, int(reset)), "omm_get_stage_times")
        return ms, cnt

    def get_array(self, which: int) -> np.ndarray:
        rows = self.n if which in (ARRAY_HW_N, ARRAY_SW_N) else self.m
        out = np.zeros((rows, self.n), order="F")
        check(lib().omm_get_array(self._h, which, C.c_void_p(out.ctypes.data), 0), "omm_get_array")
        return out

    def get_density(self, which: int = DENSITY_RHO, out=None):
        """rho (Eq. 5) or rho_E of the last solve, m x m; into `out` (column-major
        host or device array) or a new host array."""
        if out is None:
            out = np.zeros((self.m, self.m), order="F")
        _check_colmajor(out, self.m, self.m, "out")
        p, d = _ptr(out)
        check(lib().omm_get_density(self._h, which, p, d), "omm_get_density")
        return out


class SparseSolver:
    """omm_handle of the linear-scaling form: H, S on a block pattern P_H of
    bm x bm blocks, W on a localisation pattern P_W of bm x bn blocks (block CSR
    over basis-atom rows, int64 rowptr / int32 col).  Values are passed as
    (nnzb, bm, bm) / (nnzb, bm, bn) float64 arrays, blocks row-major."""

    def __init__(self, m, n, bm, bn, H_rowptr, H_col, W_rowptr, W_col, **options):
        self.m, self.n, self.bm, self.bn = m, n, bm, bn
        self._keep = [np.ascontiguousarray(H_rowptr, dtype=np.int64), np.ascontiguousarray(H_col, dtype=np.int32),
                      np.ascontiguousarray(W_rowptr, dtype=np.int64), np.ascontiguousarray(W_col, dtype=np.int32)]
        self.nbr = len(self._keep[0]) - 1
        self.nbc = n // bn
        pat = Pattern(bm, bn, self.nbr, self.nbc, *[C.c_void_p(a.ctypes.data) for a in self._keep])
        self._opts = default_options(**options)
        h = C.c_void_p()
        check(lib().omm_create(m, n, bm, C.byref(pat), C.byref(self._opts), C.byref(h)), "omm_create")
        self._h = h
        d = self.diag()
        self.nnzb = {"H": d.nnzb_H, "W": d.nnzb_W, "HW": d.nnzb_HW, "N": d.nnzb_N}

    close = Solver.close
    __del__ = Solver.__del__
    diag = Solver.diag
    begin = Solver.begin
    progress = Solver.progress
    end = Solver.end
    set_profiling = Solver.set_profiling
    stage_times = Solver.stage_times
    md_guess = Solver.md_guess

    def set_HS(self, Hv, Sv):
        for a, name in ((Hv, "H"), (Sv, "S")):
            if tuple(a.shape) != (self.nnzb["H"], self.bm, self.bm):
                raise ValueError(f"{name}: expected {(self.nnzb['H'], self.bm, self.bm)}, got {tuple(a.shape)}")
        pH, dH = _ptr(Hv)
        pS, dS = _ptr(Sv)
        if dH != dS:
            raise ValueError("H and S must both be host or both device arrays")
        st = check(lib().omm_set_HS(self._h, pH, pS, dH), "omm_set_HS")
        self.nnzb["H_kept"] = self.diag().nnzb_H
        return st

    def solve(self, W0=None, tol=1e-10, W_out=None, raise_on_error=True):
        shape = (self.nnzb["W"], self.bm, self.bn)
        for a, name in ((W0, "W0"), (W_out, "W_out")):
            if a is not None and tuple(a.shape) != shape:
                raise ValueError(f"{name}: expected {shape}")
        p0, d0 = _ptr(W0)
        po, do = _ptr(W_out)
        E = C.c_double(0.0)
        it = C.c_int32(0)
        st = lib().omm_solve(self._h, p0, d0, float(tol), po, do, C.byref(E), C.byref(it))
        if raise_on_error and st != OK:
            raise OmmError(st, "omm_solve")
        return E.value, it.value, st

    def get_density(self, which: int = DENSITY_RHO):
        """rho (Eq. 5) or rho_E of the last solve on the pattern of S: (nnzb_H, bm, bm)."""
        out = np.zeros((len(self._keep[1]), self.bm, self.bm))
        check(lib().omm_get_density(self._h, which, C.c_void_p(out.ctypes.data), 0), "omm_get_density")
        return out

    def get_array(self, which):
        sizes = {ARRAY_W: ("W", self.bm * self.bn), ARRAY_HW: ("HW", self.bm * self.bn),
                 ARRAY_SW: ("HW", self.bm * self.bn), ARRAY_G: ("W", self.bm * self.bn),
                 ARRAY_D: ("W", self.bm * self.bn), ARRAY_HW_N: ("N", self.bn * self.bn),
                 ARRAY_SW_N: ("N", self.bn * self.bn)}
        key, bs = sizes[which]
        out = np.zeros(self.nnzb[key] * bs)
        check(lib().omm_get_array(self._h, which, C.c_void_p(out.ctypes.data), 0), "omm_get_array")
        return out

    def get_pattern(self, which):
        nrows = self.nbc if which == PATTERN_N else self.nbr
        nnz = {PATTERN_H: self.nnzb.get("H_kept", self.nnzb["H"]), PATTERN_W: self.nnzb["W"],
               PATTERN_HW: self.nnzb["HW"], PATTERN_N: self.nnzb["N"]}[which]
        rp = np.zeros(nrows + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        check(lib().omm_get_pattern(self._h, which, C.c_void_p(rp.ctypes.data), C.c_void_p(col.ctypes.data)),
              "omm_get_pattern")
        return rp, col[:nnz]


def _batch_args(solvers, W0s):
    k = len(solvers)
    hs = (C.c_void_p * k)(*[s._h.value for s in solvers])
    if W0s is None:
        return hs, None, 0
    ptrs = [_ptr(a) for a in W0s]
    on = {d for p, d in ptrs if p is not None}
    if len(on) > 1:
        raise ValueError("W0s must be all host or all device arrays")
    on_dev = on.pop() if on else 0
    return hs, (C.c_void_p * k)(*[p.value if p is not None else None for p, _ in ptrs]), on_dev


def batch_solve_grouped(solvers, W0s=None, tol: float = 1e-10, tile_mode: int = -1):
    """Minimise several dense mixed handles as one group (omm_batch_solve_grouped):
    grouped persistent tensor-core launches per CG step, autotuned tile mode
    (tile_mode -1), or 0 single CTA / 1 CTA pairs.  Returns (E, iters, status, rc)."""
    k = len(solvers)
    hs, w, on_dev = _batch_args(solvers, W0s)
    E = np.zeros(k)
    it = np.zeros(k, dtype=np.int32)
    st = np.zeros(k, dtype=np.int32)
    rc = lib().omm_batch_solve_grouped(hs, k, w, on_dev, float(tol), int(tile_mode), C.c_void_p(E.ctypes.data),
                                       C.c_void_p(it.ctypes.data), C.c_void_p(st.ctypes.data))
    return E, it, st, rc


def batch_last_tuning():
    """(modes[3], ms[3][2]) of the last grouped batch: products, contractions, gradient."""
    modes = np.zeros(3, dtype=np.int32)
    ms = np.zeros(6, dtype=np.float32)
    check(lib().omm_batch_last_tuning(C.c_void_p(modes.ctypes.data), C.c_void_p(ms.ctypes.data)),
          "omm_batch_last_tuning")
    return modes, ms.reshape(3, 2)


def batch_solve(solvers, W0s=None, tol: float = 1e-10):
    """Minimise several handles together (omm_batch_solve); returns (E, iters, status) arrays."""
    k = len(solvers)
    hs = (C.c_void_p * k)(*[s._h.value for s in solvers])
    if W0s is None:
        w = None
        on_dev = 0
    else:
        ptrs = [_ptr(a) for a in W0s]
        on = {d for p, d in ptrs if p is not None}
        if len(on) > 1:
            raise ValueError("W0s must be all host or all device arrays")
        on_dev = on.pop() if on else 0
        w = (C.c_void_p * k)(*[p.value if p is not None else None for p, _ in ptrs])
    E = np.zeros(k)
    it = np.zeros(k, dtype=np.int32)
    st = np.zeros(k, dtype=np.int32)
    lib().omm_batch_solve(hs, k, w, on_dev, float(tol), C.c_void_p(E.ctypes.data), C.c_void_p(it.ctypes.data),
                          C.c_void_p(st.ctypes.data))
    return E, it, st


# ---------------------------------------------------------------- op-level calls
def op_dgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldcin, Cout, ldc, stream=0):
    return lib().omm_op_dgemm(int(transA), int(transB), M, N, K, float(alpha), _ptr(A)[0], lda,
                              _ptr(B)[0], ldb, float(beta), _ptr(Cin)[0], ldcin, _ptr(Cout)[0], ldc,
                              C.c_void_p(stream) if stream else None)


def kernel_launches() -> int:
    return int(lib().omm_kernel_launches())


def op_exact_gemm_workspace_bytes(M, N, K, ndigits) -> int:
    return int(lib().omm_op_exact_gemm_workspace_bytes(M, N, K, ndigits))


def op_exact_gemm(transA, transB, M, N, K, ndigits, alpha, A, lda, B, ldb, beta, Cin, ldcin, Cout, ldc,
                  workspace, workspace_bytes, stream=0):
    return lib().omm_op_exact_gemm(int(transA), int(transB), M, N, K, int(ndigits), float(alpha),
                                   _ptr(A)[0], lda, _ptr(B)[0], ldb, float(beta), _ptr(Cin)[0], ldcin,
                                   _ptr(Cout)[0], ldc, _ptr(workspace)[0], workspace_bytes,
                                   C.c_void_p(stream) if stream else None)


def op_split_gemm_workspace_bytes(M, N, K, ndigits) -> int:
    return int(lib().omm_op_split_gemm_workspace_bytes(M, N, K, ndigits))


def op_split_gemm(transA, transB, M, N, K, ndigits, alpha, A, lda, B, ldb, beta, Cin, ldcin, Cout, ldc,
                  workspace, workspace_bytes, stream=0):
    return lib().omm_op_split_gemm(int(transA), int(transB), M, N, K, int(ndigits), float(alpha),
                                   _ptr(A)[0], lda, _ptr(B)[0], ldb, float(beta), _ptr(Cin)[0], ldcin,
                                   _ptr(Cout)[0], ldc, _ptr(workspace)[0], workspace_bytes,
                                   C.c_void_p(stream) if stream else None)


def op_quartic_coeffs_scratch_bytes(n: int) -> int:
    return lib().omm_op_quartic_coeffs_scratch_bytes(n)


def op_quartic_coeffs(n, h0, s0, ld_h, X, Y, h2, s2, ld_z, coeffs, scratch, scratch_bytes, stream=0):
    return lib().omm_op_quartic_coeffs(n, _ptr(h0)[0], _ptr(s0)[0], ld_h, _ptr(X)[0], _ptr(Y)[0],
                                       _ptr(h2)[0], _ptr(s2)[0], ld_z, _ptr(coeffs)[0],
                                       _ptr(scratch)[0], scratch_bytes,
                                       C.c_void_p(stream) if stream else None)


def op_quartic_coeffs_static(n, h0, s0, ld_h, X, Y, h2, s2, ld_z, coeffs, stream=0):
    """Allocation-free variant: the library's static device scratch instead of a caller buffer."""
    return lib().omm_op_quartic_coeffs_static(n, _ptr(h0)[0], _ptr(s0)[0], ld_h, _ptr(X)[0], _ptr(Y)[0],
                                              _ptr(h2)[0], _ptr(s2)[0], ld_z, _ptr(coeffs)[0],
                                              C.c_void_p(stream) if stream else None)


def op_convert(op, inp, out, e=None, stream=0):
    """Integer-pipe conversion self-test (omm_op_convert): device tensors in, out (and e)."""
    return lib().omm_op_convert(op, inp.numel(), _ptr(inp)[0], _ptr(e)[0] if e is not None else None,
                                _ptr(out)[0], C.c_void_p(stream) if stream else None)


def op_line_min(coeffs, x_out, status_out, stream=0):
    return lib().omm_op_line_min(_ptr(coeffs)[0], _ptr(x_out)[0], _ptr(status_out)[0],
                                 C.c_void_p(stream) if stream else None)
