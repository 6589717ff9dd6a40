"""CPU oracle for the robust eigenvector method -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  It wraps ``evec_oracle.c`` (plain C, FP64, one column at
a time, OpenMP over independent columns), built here with gcc -O2 and without
fast-math, so no flush-to-zero and IEEE rounding throughout.

Functions return numpy arrays; matrices are float64 column-major.  The
canonical output is X with |X[:, j]|_inf in [1, 2) (pairs share one exponent
and use max_i |re_i| + |im_i|), and the true eigenvector is
X[:, j] * 2**(-scale_exp[j])  (y_j = x_j / alpha_j with alpha_j =
2**scale_exp[j], the augmented representation of Sec. 3.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evec_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

OK, EINVAL, ENOTSCHUR, ENONFINITE, ENOMEM = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, status, bad):
        super().__init__(f"oracle status {status} (bad index {bad})")
        self.status = status
        self.bad = bad


def compile_library(src: str, out: str) -> str:
    """gcc -O2 (no fast-math, OpenMP) of one C source into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def source_path() -> str:
    return _SRC


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    return compile_library(_SRC, _LIB)


class Oracle:
    """Bindings to one build of the oracle library (the default build, or a
    test's own variant of it)."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.evo_count.argtypes = [i64, p, i64, p, p, p]
        lib.evo_count.restype = ctypes.c_int
        lib.evo_standard.argtypes = [i64, p, i64, p, i64, p, p, i64, p, p, p,
                                     ctypes.c_int, p]
        lib.evo_standard.restype = ctypes.c_int
        lib.evo_standard_left.argtypes = lib.evo_standard.argtypes
        lib.evo_standard_left.restype = ctypes.c_int
        lib.evo_generalized.argtypes = [i64, p, i64, p, i64, p, i64, p, p, i64,
                                        p, p, p, p, ctypes.c_int, p]
        lib.evo_generalized.restype = ctypes.c_int
        lib.evo_generalized_left.argtypes = lib.evo_generalized.argtypes
        lib.evo_generalized_left.restype = ctypes.c_int
        lib.evo_trsolve.argtypes = [i64, p, i64, i64, p, i64, p, i64, p, ctypes.c_int, p]
        lib.evo_trsolve.restype = ctypes.c_int
        lib.evo_hessenberg.argtypes = [i64, p, i64, p, i64, p, p]
        lib.evo_hessenberg.restype = ctypes.c_int
        lib.evo_window_update.argtypes = [i64, p, i64, p, i64, ctypes.c_int, p, p, p, p]
        lib.evo_window_update.restype = ctypes.c_int
        lib.evo_naive_standard.argtypes = [i64, p, i64, p, p, i64]
        lib.evo_naive_standard.restype = i64
        self.lib = lib
        self.path = path

    def count(self, S, select=None) -> int:
        S = _fortran(S)
        n = S.shape[0]
        sel = _mask(select, n)
        m = np.zeros(1, dtype=np.int64)
        bad = np.full(1, -1, dtype=np.int64)
        st = self.lib.evo_count(n, _ptr(S), max(n, 1), _ptr(sel), _ptr(m), _ptr(bad))
        if st:
            raise OracleError(st, int(bad[0]))
        return int(m[0])

    def standard(self, S, Q=None, select=None, threads: int = 0, left: bool = False):
        """Eigenvectors of the quasi-triangular S (optionally back-transformed
        by Q).  Returns (X, scale_exp, lam_re, lam_im).  left: the left
        eigenvectors, u^H S = lambda u^H (pairs: columns Re u, Im u for
        lambda = a + i w, w > 0), zero above their block."""
        S = _fortran(S)
        n = S.shape[0]
        sel = _mask(select, n)
        m = self.count(S, sel) if n else 0
        X = np.zeros((n, m), dtype=np.float64, order="F")
        e = np.zeros(m, dtype=np.int32)
        lr = np.zeros(m)
        li = np.zeros(m)
        Qf = None if Q is None else _fortran(Q)
        bad = np.full(1, -1, dtype=np.int64)
        fn = self.lib.evo_standard_left if left else self.lib.evo_standard
        st = fn(n, _ptr(S), max(n, 1), _ptr(Qf), max(n, 1), _ptr(sel), _ptr(X), max(n, 1),
                _ptr(e), _ptr(lr), _ptr(li), int(threads), _ptr(bad))
        if st:
            raise OracleError(st, int(bad[0]))
        return X, e, lr, li

    def generalized(self, S, T, Z=None, select=None, threads: int = 0, left: bool = False):
        """Generalized eigenvectors of (S, T) (optionally back-transformed by
        Z).  Returns (X, scale_exp, alpha_re, alpha_im, beta).  left: the
        left eigenvectors, u^H (beta S - alpha T) = 0 (pairs: columns Re u,
        Im u for Im alpha > 0), zero above their block."""
        S = _fortran(S)
        T = _fortran(T)
        n = S.shape[0]
        sel = _mask(select, n)
        m = self.count(S, sel) if n else 0
        X = np.zeros((n, m), dtype=np.float64, order="F")
        e = np.zeros(m, dtype=np.int32)
        ar = np.zeros(m)
        ai = np.zeros(m)
        be = np.zeros(m)
        Zf = None if Z is None else _fortran(Z)
        bad = np.full(1, -1, dtype=np.int64)
        fn = self.lib.evo_generalized_left if left else self.lib.evo_generalized
        st = fn(n, _ptr(S), max(n, 1), _ptr(T), max(n, 1), _ptr(Zf), max(n, 1), _ptr(sel),
                _ptr(X), max(n, 1), _ptr(e), _ptr(ar), _ptr(ai), _ptr(be), int(threads),
                _ptr(bad))
        if st:
            raise OracleError(st, int(bad[0]))
        return X, e, ar, ai, be

    def trsolve(self, S, B, threads: int = 0):
        """Robust solve of S x_j = b_j for every column of B (S upper
        quasi-triangular).  Returns (X, scale_exp): x_j = X[:, j] *
        2**(-scale_exp[j]), |X[:, j]|_inf in [1, 2)."""
        S = _fortran(S)
        B = _fortran(np.atleast_2d(B.T).T if np.ndim(B) == 1 else B)
        n = S.shape[0]
        nrhs = B.shape[1]
        X = np.zeros((n, nrhs), dtype=np.float64, order="F")
        e = np.zeros(nrhs, dtype=np.int32)
        bad = np.full(1, -1, dtype=np.int64)
        st = self.lib.evo_trsolve(n, _ptr(S), max(n, 1), nrhs, _ptr(B), max(n, 1), _ptr(X),
                                  max(n, 1), _ptr(e), int(threads), _ptr(bad))
        if st:
            raise OracleError(st, int(bad[0]))
        return X, e

    def hessenberg(self, A, calc_q: bool = True):
        """Hessenberg reduction A = Q H Q^T by one Householder reflector per
        column (unblocked).  Returns (H, Q or None, tau)."""
        H = np.array(_fortran(A), order="F", copy=True)
        n = H.shape[0]
        Q = np.zeros((n, n), order="F") if calc_q else None
        tau = np.zeros(max(n, 1))
        bad = np.full(1, -1, dtype=np.int64)
        st = self.lib.evo_hessenberg(n, _ptr(H), max(n, 1), _ptr(Q), max(n, 1), _ptr(tau),
                                     _ptr(bad))
        if st:
            raise OracleError(st, int(bad[0]))
        return H, Q, tau[:n]

    def window_update(self, T, Q, windows):
        """Eigenvalue reordering's off-diagonal updates: for each (a, Z) in
        windows, in order, T <- Zhat^T T Zhat and Q <- Q Zhat with Zhat the
        identity carrying the k x k orthogonal Z on rows and columns
        [a, a + k).  Returns updated copies (T, Q or None)."""
        T = np.array(_fortran(T), order="F", copy=True)
        n = T.shape[0]
        Q = None if Q is None else np.array(_fortran(Q), order="F", copy=True)
        begin = np.array([int(a) for a, _ in windows], dtype=np.int64)
        size = np.array([np.asarray(Z).shape[0] for _, Z in windows], dtype=np.int32)
        zoff = np.zeros(len(windows), dtype=np.int64)
        if len(windows):
            zoff[1:] = np.cumsum(size.astype(np.int64) ** 2)[:-1]
        Zp = np.concatenate([np.asarray(Z, dtype=np.float64).ravel(order="F") for _, Z in windows]
                            + [np.zeros(1)])
        st = self.lib.evo_window_update(n, _ptr(T), max(n, 1), _ptr(Q), max(n, 1), len(windows),
                                        _ptr(begin), _ptr(size), _ptr(Zp), _ptr(zoff))
        if st:
            raise OracleError(st, -1)
        return T, Q

    def naive_standard(self, S, select=None):
        """Unscaled textbook substitution (overflow witness).  Returns
        (X, number of columns containing Inf or NaN)."""
        S = _fortran(S)
        n = S.shape[0]
        sel = _mask(select, n)
        m = self.count(S, sel)
        X = np.zeros((n, m), dtype=np.float64, order="F")
        with np.errstate(all="ignore"):
            bad = self.lib.evo_naive_standard(n, _ptr(S), max(n, 1), _ptr(sel), _ptr(X),
                                              max(n, 1))
        return X, int(bad)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _fortran(a):
    return np.asfortranarray(a, dtype=np.float64)


def _mask(select, n):
    if select is None:
        return None
    s = np.ascontiguousarray(select, dtype=np.uint8)
    if s.shape != (n,):
        raise ValueError("selection mask must have length n")
    return s


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def count(S, select=None) -> int:
    return default().count(S, select)


def standard(S, Q=None, select=None, threads: int = 0):
    return default().standard(S, Q, select, threads)


def left(S, Q=None, select=None, threads: int = 0):
    """Left eigenvectors u^H S = lambda u^H (see Oracle.standard)."""
    return default().standard(S, Q, select, threads, left=True)


def generalized(S, T, Z=None, select=None, threads: int = 0):
    return default().generalized(S, T, Z, select, threads)


def generalized_left(S, T, Z=None, select=None, threads: int = 0):
    """Left eigenvectors u^H (beta S - alpha T) = 0 (see Oracle.generalized)."""
    return default().generalized(S, T, Z, select, threads, left=True)


def naive_standard(S, select=None):
    return default().naive_standard(S, select)


def trsolve(S, B, threads: int = 0):
    return default().trsolve(S, B, threads)


def hessenberg(A, calc_q: bool = True):
    return default().hessenberg(A, calc_q)


def window_update(T, Q, windows):
    return default().window_update(T, Q, windows)
