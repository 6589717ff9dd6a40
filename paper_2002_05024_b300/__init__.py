"""Robust eigenvectors of real Schur forms on one B300 GPU.

A thin ctypes binding over the C ABI in ``include/evec.h`` (library
``_lib/libevec.so``, built by ``paper_2002_05024_b300.build``).  Every step of
the computation runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies device memory and the current stream.

Matrices are float64 CUDA tensors in column-major layout: shape (n, n) with
strides (1, ld), ld >= n -- e.g. ``torch.from_numpy(np.asfortranarray(A)).cuda()``
or ``colmajor(t)``.  Results follow the library's conventions: the true
eigenvector j is ``X[:, j] * 2**(-scale_exp[j])`` with max |X[:, j]| in
[1, 2) (a complex pair occupies two columns (Re, Im) and shares one
exponent; its norm is max |re| + |im|).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libevec.so")
# the checked build (bounds checks of the kernels' main device accesses,
# reported as EVEC_EBOUNDS); use_checked_build() selects it
CHECK_LIB_PATH = os.path.join(_HERE, "_lib", "libevec_check.so")

STATUS = {0: "EVEC_OK", 1: "EVEC_EINVAL", 2: "EVEC_ENOTSCHUR", 3: "EVEC_ENONFINITE",
          4: "EVEC_ENOMEM", 5: "EVEC_ECUDA", 6: "EVEC_ETIMEOUT", 7: "EVEC_ERESIDUAL",
          8: "EVEC_ECAPACITY", 9: "EVEC_EBOUNDS"}
EVEC_OK, EVEC_EINVAL, EVEC_ENOTSCHUR, EVEC_ENONFINITE = 0, 1, 2, 3
EVEC_ENOMEM, EVEC_ECUDA, EVEC_ETIMEOUT, EVEC_ERESIDUAL = 4, 5, 6, 7
EVEC_ECAPACITY = 8
KERNELS = ("gather", "tile_norms", "diag_solve", "tile_update", "finalize",
           "backtransform", "canonicalize", "batched", "refine", "left", "hess_panel",
           "hess_update", "window")


class EvecError(RuntimeError):
    def __init__(self, status: int, where: str, bad: int = -1):
        msg = f"{where}: {STATUS.get(status, status)}"
        if bad >= 0:
            msg += f" (index {bad})"
        if status in (4, 5) and _lib is not None:
            msg += f" [{_lib.evec_last_cuda_error().decode()}]"
        super().__init__(msg)
        self.status = status
        self.bad = bad


class _Opts(ctypes.Structure):
    """evec_opts, in the header's field order."""
    _fields_ = [("mode", ctypes.c_int), ("tile", ctypes.c_int), ("slices", ctypes.c_int),
                ("refine", ctypes.c_int), ("check", ctypes.c_int)]


MODES = {"fp64": 0, "split": 1}


_lib = None
_lock = threading.Lock()


def use_checked_build() -> None:
    """Load the checked build instead of the normal one; call before the
    first use of the library in the process."""
    global LIB_PATH
    if _lib is not None:
        raise RuntimeError("the library is already loaded")
    LIB_PATH = CHECK_LIB_PATH


def lib() -> ctypes.CDLL:
    """The loaded C library; raises if it has not been built (there is no
    fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH}; run "
                               "`python -m paper_2002_05024_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        i64, p, i32 = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32
        L.evec_create.argtypes = [ctypes.POINTER(p), ctypes.c_int, p]
        L.evec_destroy.argtypes = [p]
        L.evec_set_stream.argtypes = [p, p]
        L.evec_count.argtypes = [p, i64, p, i64, p, ctypes.POINTER(i64)]
        L.evec_standard.argtypes = [p, i64, p, i64, p, i64, p, p, i64, p, p, p,
                                    ctypes.POINTER(_Opts)]
        L.evec_standard_left.argtypes = L.evec_standard.argtypes
        L.evec_standard_host.argtypes = [p, i64, p, p, p, p, p, p, p, ctypes.POINTER(_Opts)]
        L.evec_sync.argtypes = [p, ctypes.POINTER(i64)]
        L.evec_plan_query.argtypes = [i64, p, p, p, p, ctypes.c_int, ctypes.POINTER(i64),
                                      ctypes.POINTER(i32), p, ctypes.POINTER(i64)]
        L.evec_profile.argtypes = [p, ctypes.c_int]
        L.evec_set_lookahead.argtypes = [p, ctypes.c_int]
        L.evec_hessenberg.argtypes = [p, i64, p, i64, p, i64, ctypes.POINTER(_Opts)]
        L.evec_set_hessenberg_panel.argtypes = [p, ctypes.c_int]
        L.evec_window_update.argtypes = [p, i64, p, i64, p, i64, ctypes.c_int, p, p, p, p,
                                         ctypes.POINTER(_Opts)]
        L.evec_window_update_set.argtypes = [p, i64, p, i64, p, i64, ctypes.c_int, p, p, p, p,
                                             ctypes.POINTER(_Opts)]
        L.evec_gate_stats.argtypes = [p, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int)]
        L.evec_profile_read.argtypes = [p, p, p, ctypes.c_int]
        L.evec_last_cuda_error.argtypes = []
        L.evec_last_cuda_error.restype = ctypes.c_char_p
        L.evec_strerror.argtypes = [ctypes.c_int]
        L.evec_strerror.restype = ctypes.c_char_p
        L.evec_trsolve.argtypes = [p, i64, p, i64, i64, p, i64, p, i64, p,
                                   ctypes.POINTER(_Opts)]
        L.evec_generalized.argtypes = [p, i64, p, i64, p, i64, p, i64, p, p, i64, p, p, p, p,
                                       ctypes.POINTER(_Opts)]
        L.evec_generalized_left.argtypes = L.evec_generalized.argtypes
        L.evec_batched_count.argtypes = [p, i64, p, p, p, p, p]
        L.evec_count_generalized.argtypes = [p, i64, p, i64, p, i64, p, ctypes.POINTER(i64)]
        L.evec_batched_generalized_count.argtypes = [p, i64, p, p, p, p, p, p, p]
        L.evec_batched.argtypes = [p, i64, p, p, p, p, p, p, p, p, p, p, p, p,
                                   ctypes.POINTER(_Opts)]
        L.evec_batched_generalized.argtypes = [p, i64, p, p, p, p, p, p, p, p, p, p, p, p, p,
                                               ctypes.POINTER(_Opts)]
        L.evec_set_wait_limit.argtypes = [p, i64]
        L.evec_set_gate_factor.argtypes = [p, ctypes.c_double]
        L.evec_opts_default.argtypes = [ctypes.POINTER(_Opts)]
        L.evec_opts_default.restype = None
        L.evec_standard_noalloc.argtypes = [i64, p, i64, p, p, i64, p, ctypes.c_int, p,
                                            ctypes.POINTER(i64)]
        L.evec_tune_get.argtypes = [p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.evec_tune_set.argtypes = [p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        for f in ("evec_create", "evec_destroy", "evec_set_stream", "evec_count",
                  "evec_standard", "evec_standard_left", "evec_standard_host", "evec_sync",
                  "evec_plan_query", "evec_trsolve",
                  "evec_profile", "evec_profile_read", "evec_batched_count", "evec_batched",
                  "evec_batched_generalized", "evec_set_lookahead", "evec_hessenberg",
                  "evec_set_hessenberg_panel", "evec_gate_stats", "evec_window_update",
                  "evec_window_update_set",
                  "evec_generalized", "evec_count_generalized", "evec_set_wait_limit",
                  "evec_generalized_left",
                  "evec_set_gate_factor", "evec_standard_noalloc",
                  "evec_batched_generalized_count",
                  "evec_tune_get", "evec_tune_set"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
        return L


def strerror(status: int) -> str:
    return lib().evec_strerror(int(status)).decode()


def _check(status: int, where: str, bad: int = -1):
    if status != EVEC_OK:
        raise EvecError(status, where, bad)


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _mask(select, n):
    if select is None:
        return None
    if hasattr(select, "detach"):
        select = select.detach().cpu().numpy()
    s = np.ascontiguousarray(select, dtype=np.uint8)
    if s.shape != (n,):
        raise ValueError("selection mask must have n entries")
    return s


def _opts(tile, check, mode="fp64", slices=0, refine=1):
    return _Opts(mode=MODES[mode], tile=int(tile), slices=int(slices), refine=int(refine),
                 check=1 if check else 0)


# ---------------------------------------------------------------------------
# handles: one per device, bound to the caller's current stream at each call
# ---------------------------------------------------------------------------
class Handle:
    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        _check(lib().evec_create(ctypes.byref(self._h), int(device),
                                 ctypes.c_void_p(stream or 0)), "evec_create")
        self.device = int(device)

    @property
    def ptr(self):
        return self._h

    def set_stream(self, stream):
        _check(lib().evec_set_stream(self._h, ctypes.c_void_p(stream or 0)), "evec_set_stream")

    def sync(self):
        bad = ctypes.c_int64(-1)
        st = lib().evec_sync(self._h, ctypes.byref(bad))
        _check(st, "evec_sync", bad.value)

    def gate_stats(self):
        """(eigenvalues that failed the residual gate in the last refine = 2
        call's first solve, repeated solves)."""
        f = ctypes.c_int64(0)
        r = ctypes.c_int(0)
        _check(lib().evec_gate_stats(self._h, ctypes.byref(f), ctypes.byref(r)), "evec_gate_stats")
        return int(f.value), int(r.value)

    def wait_limit(self, polls: int):
        """Polls of a bounded device-side wait before it gives up (0 = the
        built-in limit)."""
        _check(lib().evec_set_wait_limit(self._h, int(polls)), "evec_set_wait_limit")

    def gate_factor(self, factor: float):
        """Bound of the residual gate (refine = 2): factor * n (default 10)."""
        _check(lib().evec_set_gate_factor(self._h, float(factor)), "evec_set_gate_factor")

    def hessenberg_panel(self, cooperative: bool):
        """Hessenberg panels as one cooperative launch (default) or six
        launches per column."""
        _check(lib().evec_set_hessenberg_panel(self._h, 1 if cooperative else 0),
               "evec_set_hessenberg_panel")

    def lookahead(self, enable: bool):
        """Look-ahead schedule of the split-mode solve (off by default)."""
        _check(lib().evec_set_lookahead(self._h, 1 if enable else 0), "evec_set_lookahead")

    def profile(self, enable: bool):
        _check(lib().evec_profile(self._h, 1 if enable else 0), "evec_profile")

    def profile_read(self):
        """{kernel class: (milliseconds, launches)} since the last read."""
        ms = np.zeros(len(KERNELS))
        cnt = np.zeros(len(KERNELS), dtype=np.int64)
        _check(lib().evec_profile_read(self._h, _np_ptr(ms), _np_ptr(cnt), len(KERNELS)),
               "evec_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNELS)}

    def close(self):
        if self._h:
            lib().evec_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles: dict = {}


def handle(device=None) -> Handle:
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)
    h = _handles.get(dev)
    if h is None:
        h = Handle(dev)
        _handles[dev] = h
    h.set_stream(torch.cuda.current_stream(dev).cuda_stream)
    return h


def colmajor(t):
    """Column-major copy (strides (1, n)) of a 2-D tensor."""
    return t.t().contiguous().t()


def _check_colmajor(t, name, n=None, ncols=None):
    import torch
    if t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2:
        raise ValueError(f"{name} must be a float64 CUDA matrix")
    rows, cols = t.shape
    if ncols is None:
        ncols = n
    if n is not None and (rows != n or cols != ncols):
        raise ValueError(f"{name} must be {n} x {ncols}")
    if rows > 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); use colmajor()")
    ld = t.stride(1) if cols > 1 else max(rows, 1)
    if ld < rows:
        raise ValueError(f"{name}: leading dimension below the row count")
    return ld


# ---------------------------------------------------------------------------
# public functions
# ---------------------------------------------------------------------------
def plan_query(diag, sub, sup, select=None, tile: int = 64):
    """Host-only: number of output columns and tile boundaries for T's
    diagonal / subdiagonal / superdiagonal (numpy arrays)."""
    d = np.ascontiguousarray(diag, dtype=np.float64)
    n = d.shape[0]
    s = np.ascontiguousarray(sub, dtype=np.float64)
    u = np.ascontiguousarray(sup, dtype=np.float64)
    sel = _mask(select, n)
    m = ctypes.c_int64(0)
    nt = ctypes.c_int32(0)
    starts = np.zeros(n // max(tile - 1, 1) + 3, dtype=np.int32)
    bad = ctypes.c_int64(-1)
    st = lib().evec_plan_query(n, _np_ptr(d), _np_ptr(s), _np_ptr(u), _np_ptr(sel), int(tile),
                               ctypes.byref(m), ctypes.byref(nt), _np_ptr(starts),
                               ctypes.byref(bad))
    _check(st, "evec_plan_query", bad.value)
    return int(m.value), starts[: nt.value + 1].copy()


def count(T, select=None) -> int:
    ldt = _check_colmajor(T, "T")
    n = T.shape[0]
    sel = _mask(select, n)
    m = ctypes.c_int64(0)
    h = handle(T.device.index)
    _check(lib().evec_count(h.ptr, n, T.data_ptr(), ldt, _np_ptr(sel), ctypes.byref(m)),
           "evec_count")
    return int(m.value)


def standard(T, Q=None, select=None, tile: int = 0, check: bool = False, out=None,
             mode: str = "fp64", slices: int = 0, refine: int = 1):
    """Eigenvectors of the quasi-triangular T (optionally X = Q Y).

    refine (split mode; evec_opts.refine): 1 (the library's default) one
    FP64 residual-correction sweep after the solve, 0 none, 2 the sweep and
    the residual gate.
    Returns (X, scale_exp, lam_re, lam_im) as CUDA tensors; X is (n, m)
    column-major.  The call is asynchronous on the current stream; device
    detected input errors surface at ``sync()`` (or immediately with
    check=True)."""
    return _standard_call("evec_standard", T, Q, select, tile, check, out, mode, slices, refine)


def left(T, Q=None, select=None, tile: int = 0, check: bool = False, out=None,
         mode: str = "fp64", slices: int = 0, refine: int = 1):
    """Left eigenvectors u^H T = lambda u^H (optionally X = Q U), same
    arguments, outputs and column order as ``standard``; a pair gives
    (Re u, Im u) for lambda = a + i w, w > 0."""
    return _standard_call("evec_standard_left", T, Q, select, tile, check, out, mode, slices,
                          refine)


def _standard_call(fn, T, Q, select, tile, check, out, mode, slices, refine):
    import torch
    n = T.shape[0]
    ldt = _check_colmajor(T, "T", n)
    ldq = _check_colmajor(Q, "Q", n) if Q is not None else max(n, 1)
    sel = _mask(select, n)
    dev = T.device
    h = handle(dev.index)
    m = count(T, sel) if n else 0
    if out is not None:
        X, e, lr, li = out
    else:
        X = torch.empty((m, n), dtype=torch.float64, device=dev).t()
        e = torch.empty(m, dtype=torch.int32, device=dev)
        lr = torch.empty(m, dtype=torch.float64, device=dev)
        li = torch.empty(m, dtype=torch.float64, device=dev)
    ldx = X.stride(1) if m > 1 else max(n, 1)
    if m == 0:
        return X, e, lr, li
    opts = _opts(tile, False, mode, slices, refine)
    st = getattr(lib(), fn)(h.ptr, n, T.data_ptr(), ldt,
                            Q.data_ptr() if Q is not None else None, ldq, _np_ptr(sel),
                            X.data_ptr(), ldx, e.data_ptr(), lr.data_ptr(), li.data_ptr(),
                            ctypes.byref(opts))
    _check(st, fn)
    if check:
        h.sync()
    return X, e, lr, li


def count_generalized(S, T, select=None) -> int:
    """Output columns of evec_generalized for the pencil (S, T)."""
    n = S.shape[0]
    lds = _check_colmajor(S, "S", n)
    ldt = _check_colmajor(T, "T", n)
    sel = _mask(select, n)
    m = ctypes.c_int64(0)
    h = handle(S.device.index)
    _check(lib().evec_count_generalized(h.ptr, n, S.data_ptr(), lds, T.data_ptr(), ldt,
                                        _np_ptr(sel), ctypes.byref(m)), "evec_count_generalized")
    return int(m.value)


def generalized(S, T, Z=None, select=None, tile: int = 0, check: bool = False,
                mode: str = "fp64", slices: int = 0, left: bool = False):
    """Generalized eigenvectors of the pencil (S, T) (optionally X = Z Y).

    Returns (X, scale_exp, alpha_re, alpha_im, beta) as CUDA tensors; X is
    (n, m) column-major; column j is the eigenvector of alpha_j / beta_j.
    left: the left eigenvectors u^H (beta S - alpha T) = 0 (evec_generalized_left)."""
    import torch
    n = S.shape[0]
    lds = _check_colmajor(S, "S", n)
    ldt = _check_colmajor(T, "T", n)
    ldz = _check_colmajor(Z, "Z", n) if Z is not None else max(n, 1)
    sel = _mask(select, n)
    dev = S.device
    h = handle(dev.index)
    m = count_generalized(S, T, sel) if n else 0
    X = torch.empty((m, n), dtype=torch.float64, device=dev).t()
    e = torch.empty(m, dtype=torch.int32, device=dev)
    ar = torch.empty(m, dtype=torch.float64, device=dev)
    ai = torch.empty(m, dtype=torch.float64, device=dev)
    be = torch.empty(m, dtype=torch.float64, device=dev)
    if m == 0:
        return X, e, ar, ai, be
    ldx = X.stride(1) if m > 1 else max(n, 1)
    opts = _opts(tile, False, mode, slices)
    name = "evec_generalized_left" if left else "evec_generalized"
    st = getattr(lib(), name)(h.ptr, n, S.data_ptr(), lds, T.data_ptr(), ldt,
                              Z.data_ptr() if Z is not None else None, ldz, _np_ptr(sel),
                              X.data_ptr(), ldx, e.data_ptr(), ar.data_ptr(), ai.data_ptr(),
                              be.data_ptr(), ctypes.byref(opts))
    _check(st, name)
    if check:
        h.sync()
    return X, e, ar, ai, be


def generalized_left(S, T, Z=None, select=None, tile: int = 0, check: bool = False,
                     mode: str = "fp64", slices: int = 0):
    """Left eigenvectors of the pencil (S, T): u^H (beta S - alpha T) = 0
    (optionally X = Z U); outputs as generalized()."""
    return generalized(S, T, Z, select, tile, check, mode, slices, left=True)


def trsolve(T, B, tile: int = 0, check: bool = False, mode: str = "fp64", slices: int = 0,
            out=None):
    """Robust solve of T x_j = b_j for every column of B (T upper
    quasi-triangular, CUDA tensors, column-major).  Returns (X, scale_exp)
    with x_j = X[:, j] * 2**(-scale_exp[j]), |X[:, j]|_inf in [1, 2); out =
    (X, e) to write into (X may be B for an in-place solve)."""
    import torch
    n = T.shape[0]
    ldt = _check_colmajor(T, "T", n)
    if B.dim() == 1:
        B = B.view(n, 1)
    nrhs = B.shape[1]
    ldb = _check_colmajor(B, "B", n, nrhs)
    h = handle(T.device.index)
    if out is not None:
        X, e = out
        if X.dim() == 1:
            X = X.view(n, 1)
        if e.dtype != torch.int32 or not e.is_cuda or e.numel() < nrhs:
            raise ValueError(f"scale_exp must be an int32 CUDA vector of {nrhs} entries")
    else:
        X = torch.empty((nrhs, n), dtype=torch.float64, device=T.device).t()
        e = torch.empty(nrhs, dtype=torch.int32, device=T.device)
    ldx = _check_colmajor(X, "X", n, nrhs)
    if n == 0 or nrhs == 0:
        return X, e
    opts = _opts(tile, False, mode, slices)
    st = lib().evec_trsolve(h.ptr, n, T.data_ptr(), ldt, nrhs, B.data_ptr(), ldb, X.data_ptr(),
                            ldx, e.data_ptr(), ctypes.byref(opts))
    _check(st, "evec_trsolve")
    if check:
        h.sync()
    return X, e


def pack_windows(windows, device):
    """[(begin, Z), ...] (Z k x k) -> (begin int64, size int32, zoff int64
    host arrays, the Z matrices packed column-major into one float64
    device vector)."""
    import torch
    begin = np.array([int(a) for a, _ in windows], dtype=np.int64)
    size = np.array([int(Z.shape[0]) for _, Z in windows], dtype=np.int32)
    zoff = np.zeros(len(windows), dtype=np.int64)
    if len(windows):
        zoff[1:] = np.cumsum(size.astype(np.int64) ** 2)[:-1]
    parts = [torch.as_tensor(np.asarray(Z) if not torch.is_tensor(Z) else Z,
                             dtype=torch.float64).t().reshape(-1) for _, Z in windows]
    Zp = (torch.cat(parts) if parts else torch.zeros(1, dtype=torch.float64)).to(device)
    return begin, size, zoff, Zp


def window_update(T, Q, windows, check: bool = False, packed=None, disjoint: bool = False,
                  mode: str = "fp64", slices: int = 0):
    """Eigenvalue reordering's off-diagonal updates, in place: for each
    (begin, Z) in windows, in order, T[a:b, a:] <- Z^T T[a:b, a:],
    T[:b, a:b] <- T[:b, a:b] Z and Q[:, a:b] <- Q[:, a:b] Z (T, Q float64
    CUDA, column-major; Q may be None).  disjoint: the windows are pairwise
    disjoint and are applied as one concurrent set (evec_window_update_set).
    packed: the result of pack_windows, to skip packing.  mode "split": the
    products in split precision (BF16 digit slices, FP64 results).  Returns
    (T, Q)."""
    n = T.shape[0]
    ldt = _check_colmajor(T, "T", n)
    ldq = _check_colmajor(Q, "Q", n) if Q is not None else 1
    begin, size, zoff, Zp = packed if packed is not None else pack_windows(windows, T.device)
    h = handle(T.device.index)
    opts = _opts(0, False, mode, slices)
    fn = lib().evec_window_update_set if disjoint else lib().evec_window_update
    st = fn(h.ptr, n, T.data_ptr(), ldt, Q.data_ptr() if Q is not None else None, ldq, len(begin),
            _np_ptr(begin), _np_ptr(size), Zp.data_ptr(), _np_ptr(zoff), ctypes.byref(opts))
    _check(st, "evec_window_update_set" if disjoint else "evec_window_update")
    if check:
        h.sync()
    return T, Q


def hessenberg(A, calc_q: bool = True, check: bool = False, overwrite: bool = False,
               mode: str = "fp64", slices: int = 0):
    """Hessenberg reduction A = Q H Q^T of a float64 CUDA matrix
    (column-major).  Returns (H, Q or None); with overwrite, H is A itself.
    mode "split": the panels' large products through the split GEMM."""
    import torch
    n = A.shape[0]
    lda = _check_colmajor(A, "A", n)
    H = A if overwrite else A.t().contiguous().t()
    Q = torch.empty((n, n), dtype=torch.float64, device=A.device).t() if calc_q else None
    if n == 0:
        return H, Q
    h = handle(A.device.index)
    opts = _opts(0, False, mode, slices)
    st = lib().evec_hessenberg(h.ptr, n, H.data_ptr(), H.stride(1) if n > 1 else lda,
                               Q.data_ptr() if Q is not None else None,
                               Q.stride(1) if (Q is not None and n > 1) else max(n, 1),
                               ctypes.byref(opts))
    _check(st, "evec_hessenberg")
    if check:
        h.sync()
    return H, Q


def standard_host(T, Q=None, select=None, tile: int = 0, device: int = 0,
                  mode: str = "fp64", slices: int = 0, refine: int = 1):
    """The same computation from host numpy arrays (column-major float64);
    copies in, computes, copies out.  Returns numpy arrays."""
    Tf = np.asfortranarray(T, dtype=np.float64)
    n = Tf.shape[0]
    Qf = None if Q is None else np.asfortranarray(Q, dtype=np.float64)
    sel = _mask(select, n)
    d = np.ascontiguousarray(np.diagonal(Tf))
    sub = np.ascontiguousarray(np.diagonal(Tf, -1))
    sup = np.ascontiguousarray(np.diagonal(Tf, 1))
    m, _ = plan_query(d, sub, sup, sel, tile or 64) if n else (0, None)
    X = np.zeros((n, m), dtype=np.float64, order="F")
    e = np.zeros(m, dtype=np.int32)
    lr = np.zeros(m)
    li = np.zeros(m)
    import torch
    h = handle(device)
    h.set_stream(torch.cuda.current_stream(device).cuda_stream)
    opts = _opts(tile, False, mode, slices, refine)
    st = lib().evec_standard_host(h.ptr, n, _np_ptr(Tf), _np_ptr(Qf), _np_ptr(sel), _np_ptr(X),
                                  _np_ptr(e), _np_ptr(lr), _np_ptr(li), ctypes.byref(opts))
    _check(st, "evec_standard_host")
    return X, e, lr, li


def sync(device=None):
    handle(device).sync()


# ---------------------------------------------------------------------------
# batched mode
# ---------------------------------------------------------------------------
SIZE_CLASSES = 5   # n <= 64, <= 128, <= 256, <= 512, larger


def pack_batch(Ts, device=None):
    """Pack square matrices (numpy or torch, any layout) column-major into one
    CUDA tensor; returns (packed, n array, element offsets)."""
    import torch
    ns = np.array([int(t.shape[0]) for t in Ts], dtype=np.int64)
    offs = np.zeros(len(Ts), dtype=np.int64)
    if len(Ts):
        offs[1:] = np.cumsum(ns * ns)[:-1]
    host = np.empty(int((ns * ns).sum()), dtype=np.float64)
    for t, n, o in zip(Ts, ns, offs):
        a = t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)
        host[o:o + n * n] = np.asarray(a, dtype=np.float64).ravel(order="F")
    dev = torch.device("cuda", device if device is not None else torch.cuda.current_device())
    return torch.from_numpy(host).to(dev), ns, offs


def batched_count(T_packed, ns, t_offs, select=None):
    """Output columns m_i of each matrix of a packed batch."""
    h = handle(T_packed.device.index)
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    t_offs = np.ascontiguousarray(t_offs, dtype=np.int64)
    sel = None if select is None else np.ascontiguousarray(select, dtype=np.uint8)
    if sel is not None and sel.shape != (int(ns.sum()),):
        raise ValueError("selection must hold n_i bytes per matrix")
    m = np.zeros(len(ns), dtype=np.int64)
    _check(lib().evec_batched_count(h.ptr, len(ns), _np_ptr(ns), T_packed.data_ptr(),
                                    _np_ptr(t_offs), _np_ptr(sel), _np_ptr(m)),
           "evec_batched_count")
    return m


def batched_packed(T_packed, ns, t_offs, select=None, tile: int = 0, mode: str = "fp64",
                   check: bool = False, out=None, slices: int = 0, Q_packed=None, q_offs=None,
                   x_offs=None, e_offs=None):
    """evec_batched on a packed device buffer.  select: concatenated n_i-byte
    masks or None.  Q_packed / q_offs: per-matrix back-transformations
    (q_offs[i] < 0: none for matrix i).  Returns (X_packed, scale_exp,
    lam_re, lam_im, m) with the output packing of the C entry point (X_i at
    x_offs[i], default sum_{k<i} n_k m_k, leading dimension n_i; the others
    at e_offs[i], default sum_{k<i} m_k).  out = (X, e, lr, li, m) from an
    earlier call on the same batch layout skips the column count."""
    import torch
    h = handle(T_packed.device.index)
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    t_offs = np.ascontiguousarray(t_offs, dtype=np.int64)
    sel = None if select is None else np.ascontiguousarray(select, dtype=np.uint8)
    q_offs = None if q_offs is None else np.ascontiguousarray(q_offs, dtype=np.int64)
    x_offs = None if x_offs is None else np.ascontiguousarray(x_offs, dtype=np.int64)
    e_offs = None if e_offs is None else np.ascontiguousarray(e_offs, dtype=np.int64)
    if out is not None:
        X, e, lr, li, m = out
    else:
        m = batched_count(T_packed, ns, t_offs, sel)
        dev = T_packed.device
        nx = int((ns * m).sum()) if x_offs is None else int((x_offs + ns * m).max(initial=0))
        ne = int(m.sum()) if e_offs is None else int((e_offs + m).max(initial=0))
        X = torch.empty(max(nx, 1), dtype=torch.float64, device=dev)
        e = torch.empty(max(ne, 1), dtype=torch.int32, device=dev)
        lr = torch.empty(max(ne, 1), dtype=torch.float64, device=dev)
        li = torch.empty(max(ne, 1), dtype=torch.float64, device=dev)
    opts = _opts(tile, False, mode, slices)
    st = lib().evec_batched(h.ptr, len(ns), _np_ptr(ns), T_packed.data_ptr(), _np_ptr(t_offs),
                            None if Q_packed is None else Q_packed.data_ptr(), _np_ptr(q_offs),
                            _np_ptr(sel), X.data_ptr(), _np_ptr(x_offs), e.data_ptr(),
                            _np_ptr(e_offs), lr.data_ptr(), li.data_ptr(), ctypes.byref(opts))
    _check(st, "evec_batched")
    if check:
        h.sync()
    return X, e, lr, li, m


def batched(Ts, selects=None, tile: int = 0, mode: str = "fp64", check: bool = True,
            slices: int = 0, Qs=None):
    """Eigenvectors of a list of quasi-triangular matrices in one persistent
    launch; Qs: a list of orthogonal factors (None entries: no
    back-transformation for that matrix).  Returns a list of (X_i (n_i,
    m_i), scale_exp_i, lam_re_i, lam_im_i) CUDA tensors, X_i column-major."""
    Tp, ns, offs = pack_batch(Ts)
    sel = None
    if selects is not None:
        sel = np.concatenate([np.ones(n, np.uint8) if s is None else
                              np.ascontiguousarray(s, dtype=np.uint8) for s, n in zip(selects, ns)])
    Qp = qoffs = None
    if Qs is not None and any(q is not None for q in Qs):
        have = [q for q in Qs if q is not None]
        Qp, _, ho = pack_batch(have)
        qoffs = np.full(len(Ts), -1, dtype=np.int64)
        k = 0
        for i, q in enumerate(Qs):
            if q is not None:
                qoffs[i] = ho[k]
                k += 1
    X, e, lr, li, m = batched_packed(Tp, ns, offs, sel, tile, mode, check, slices=slices,
                                     Q_packed=Qp, q_offs=qoffs)
    out = []
    xo = eo = 0
    for n, mi in zip(ns, m):
        n, mi = int(n), int(mi)
        out.append((X[xo:xo + n * mi].view(mi, n).t(), e[eo:eo + mi], lr[eo:eo + mi],
                    li[eo:eo + mi]))
        xo += n * mi
        eo += mi
    return out


def batched_generalized_packed(S_packed, T_packed, ns, s_offs, t_offs, select=None,
                               tile: int = 0, check: bool = False, out=None, Z_packed=None,
                               z_offs=None, mode: str = "fp64", slices: int = 0):
    """evec_batched_generalized on packed device buffers (FP64).  Returns
    (X_packed, scale_exp, alpha_re, alpha_im, beta, m) with the output
    packing of evec_batched; out = that tuple from an earlier call on the
    same layout skips the column count.  Z_packed / z_offs: pencil i with
    z_offs[i] >= 0 gets X_i = Z_i Y_i.  mode "split": the updates as split
    products on the tensor cores."""
    import torch
    h = handle(S_packed.device.index)
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    s_offs = np.ascontiguousarray(s_offs, dtype=np.int64)
    t_offs = np.ascontiguousarray(t_offs, dtype=np.int64)
    sel = None if select is None else np.ascontiguousarray(select, dtype=np.uint8)
    if out is not None:
        X, e, ar, ai, be, m = out
    else:
        m = np.zeros(len(ns), dtype=np.int64)
        _check(lib().evec_batched_generalized_count(h.ptr, len(ns), _np_ptr(ns),
                                                    S_packed.data_ptr(), _np_ptr(s_offs),
                                                    T_packed.data_ptr(), _np_ptr(t_offs),
                                                    _np_ptr(sel), _np_ptr(m)),
               "evec_batched_generalized_count")
        dev = S_packed.device
        X = torch.empty(int((ns * m).sum()), dtype=torch.float64, device=dev)
        e = torch.empty(int(m.sum()), dtype=torch.int32, device=dev)
        ar = torch.empty(int(m.sum()), dtype=torch.float64, device=dev)
        ai = torch.empty(int(m.sum()), dtype=torch.float64, device=dev)
        be = torch.empty(int(m.sum()), dtype=torch.float64, device=dev)
    opts = _opts(tile, False, mode, slices)
    zo = None if Z_packed is None else np.ascontiguousarray(z_offs, dtype=np.int64)
    st = lib().evec_batched_generalized(h.ptr, len(ns), _np_ptr(ns), S_packed.data_ptr(),
                                        _np_ptr(s_offs), T_packed.data_ptr(), _np_ptr(t_offs),
                                        None if Z_packed is None else Z_packed.data_ptr(),
                                        _np_ptr(zo), _np_ptr(sel), X.data_ptr(), e.data_ptr(),
                                        ar.data_ptr(), ai.data_ptr(), be.data_ptr(),
                                        ctypes.byref(opts))
    _check(st, "evec_batched_generalized")
    if check:
        h.sync()
    return X, e, ar, ai, be, m


def batched_generalized(pairs, selects=None, tile: int = 0, check: bool = True, Zs=None,
                        mode: str = "fp64", slices: int = 0):
    """Generalized eigenvectors of a list of pencils [(S_i, T_i), ...] (numpy
    or torch matrices, packed here) in one persistent launch (FP64); Zs (a
    list with a matrix or None per pencil): X_i = Z_i Y_i.  Returns a list
    of (X_i (n_i, m_i), scale_exp_i, alpha_re_i, alpha_im_i, beta_i)."""
    Sp, ns, soffs = pack_batch([S for S, _ in pairs])
    Tp, _, toffs = pack_batch([T for _, T in pairs])
    Zp = zoffs = None
    if Zs is not None and any(z is not None for z in Zs):
        have = [z for z in Zs if z is not None]
        Zp, _, zo = pack_batch(have)
        zoffs = np.full(len(pairs), -1, dtype=np.int64)
        j = 0
        for i, z in enumerate(Zs):
            if z is not None:
                zoffs[i] = zo[j]
                j += 1
    sel = None
    if selects is not None:
        sel = np.concatenate([np.ones(n, np.uint8) if s is None else
                              np.ascontiguousarray(s, dtype=np.uint8) for s, n in zip(selects, ns)])
    X, e, ar, ai, be, m = batched_generalized_packed(Sp, Tp, ns, soffs, toffs, sel, tile, check,
                                                     Z_packed=Zp, z_offs=zoffs, mode=mode,
                                                     slices=slices)
    out = []
    xo = eo = 0
    for n, mi in zip(ns, m):
        n, mi = int(n), int(mi)
        out.append((X[xo:xo + n * mi].view(mi, n).t(), e[eo:eo + mi], ar[eo:eo + mi],
                    ai[eo:eo + mi], be[eo:eo + mi]))
        xo += n * mi
        eo += mi
    return out


TUNE_TABLES = {"fp64": 0, "split": 1, "pencil": 2}   # "pencil": EVEC_TUNE_PENCIL


def tune_table(device: int = 0, mode: str = "fp64"):
    """The handle's tile per size class (0 = not tuned yet); mode "fp64" or
    "split" (evec_batched) or "pencil" (evec_batched_generalized)."""
    h = handle(device)
    out = []
    for c in range(SIZE_CLASSES):
        t = ctypes.c_int(0)
        _check(lib().evec_tune_get(h.ptr, TUNE_TABLES[mode], c, ctypes.byref(t)),
               "evec_tune_get")
        out.append(t.value)
    return out


def set_tune_table(table, device: int = 0, mode: str = "fp64"):
    """Load a tile table (e.g. one saved as JSON by an earlier run)."""
    h = handle(device)
    for c, t in enumerate(table):
        _check(lib().evec_tune_set(h.ptr, TUNE_TABLES[mode], c, int(t)), "evec_tune_set")
