"""The pins must catch plausible mistakes in the oracle.

Each case copies the oracle's C source, plants one mistake (a flipped sign,
a dropped term, a wrong or transposed index, a disabled protection step),
compiles the copy into a temporary library and runs a fast detector suite
built only from independent checks (hand-derived golden vectors, the
residual definition, an overflow case, arbitrary-precision brute force).
The unmodified oracle must pass the suite; every mutant must fail it.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads
from evec_checks import (U, canonical_norms, column_groups, flip_pencil,
                         generalized_left_residuals, generalized_residuals, left_residuals,
                         mp_canonical, mp_eigvec, mp_left_eigvec, standard_residuals)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")

MUTANTS = [
    ("update_sign", "yr[r] -= Sc[r] * zr;", "yr[r] += Sc[r] * zr;"),
    ("imag_update_dropped",
     "for (int64_t r = 0; r < q; r++) yi[r] -= Sc[r] * zi;", ";"),
    ("own_block_wrong_entry", "o[3] = w / b;", "o[3] = w / c;"),
    ("protect_update_disabled",
     "if (tau > (OMEGA - nu) / mu) return -1 - ((int64_t)ilogb(mu) + 1);",
     "if (tau > (OMEGA - nu) / mu) return 0;"),
    ("small_system_transposed",
     "double sv = AT(P->S, P->lds, i0 + a, i0 + b);",
     "double sv = AT(P->S, P->lds, i0 + b, i0 + a);"),
    ("canonical_exponent_sign", "    e -= tcan;\n            if (Q) {",
     "    e += tcan;\n            if (Q) {"),
    ("backtransform_transposed", "x[r] += Qc[r] * v;", "x[r] += AT(Q, ldq, j, r) * v;"),
    ("division_scale_not_applied",
     "zr[i] = ldexp(hr[i], (int)(kr + s));", "zr[i] = ldexp(hr[i], (int)(kr));"),
    ("generalized_alpha_sign",
     "yr[r] -= sv * zr - tr * (ar * zr - ai * zi);",
     "yr[r] -= sv * zr + tr * (ar * zr - ai * zi);"),
    ("generalized_cross_term",
     "if (cplx) yi[r] -= sv * zi - tr * (ar * zi + ai * zr);",
     "if (cplx) yi[r] -= sv * zi - tr * (ar * zi - ai * zr);"),
    ("pivot_permutation_not_undone",
     "hr[colp[0]] = w1r; hi[colp[0]] = w1i;\n        hr[colp[1]] = w2r; hi[colp[1]] = w2i;",
     "hr[0] = w1r; hi[0] = w1i;\n        hr[1] = w2r; hi[1] = w2i;"),
    ("eigenvalue_imag_sign", "lre[k] = a; lim[k] = w;", "lre[k] = a; lim[k] = -w;"),
    ("left_update_sign", "wr[c] -= sv * zr;", "wr[c] += sv * zr;"),
    ("left_small_system_not_transposed",
     "const double sv = AT(P->S, P->lds, i0 + b, i0 + a);",
     "const double sv = AT(P->S, P->lds, i0 + a, i0 + b);"),
    ("left_own_block_sign", "o[2] = w / b;", "o[2] = -w / b;"),
    ("left_conjugation_dropped", "for (int64_t r = 0; r < n; r++) yi[r] = -yi[r];", "(void)0;"),
    ("left_update_unprotected",
     ": P->tauL[cur];\n            int64_t s = protect_update(nu, tau, mu);",
     ": P->tauL[cur];\n            int64_t s = 0;"),
    ("generalized_left_T_update_dropped",
     "tv = AT(P->T, P->ldt, q + j, c);", "tv = AT(P->T, P->ldt, c, q + j);"),
    ("generalized_left_T_bound_dropped",
     "cabs1(ar, ai) * P->tauLT[cur]", "0.0 * P->tauLT[cur]"),
    ("generalized_left_own_block_not_reversed",
     "double t = o[0]; o[0] = o[1]; o[1] = t;", "double t = o[0];"),
    ("generalized_left_alpha_sign",
     "wr[c] -= bsv * zr - tv * (ar * zr - ai * zi);",
     "wr[c] -= bsv * zr + tv * (ar * zr - ai * zi);"),
    ("hessenberg_beta_sign", "if (alpha >= 0.0) beta = -beta;", "if (alpha < 0.0) beta = -beta;"),
    ("hessenberg_tau", "const double t = (beta - alpha) / beta;",
     "const double t = (beta - alpha) / alpha;"),
    ("window_left_not_transposed",
     "for (int64_t l = 0; l < k; l++) s += AT(Zw, k, l, i) * AT(T, ldt, a + l, j);",
     "for (int64_t l = 0; l < k; l++) s += AT(Zw, k, i, l) * AT(T, ldt, a + l, j);"),
    ("window_left_skips_block", "for (int64_t j = a; j < n; j++) {", "for (int64_t j = b; j < n; j++) {"),
    ("window_right_rows_short", "for (int64_t r = 0; r < b; r++) {", "for (int64_t r = 0; r < a; r++) {"),
    ("window_q_dropped", "        if (Q)\n            for (int64_t r = 0; r < n; r++) {\n                for (int64_t i = 0; i < k; i++) {",
     "        if (0)\n            for (int64_t r = 0; r < n; r++) {\n                for (int64_t i = 0; i < k; i++) {"),
    ("hessenberg_left_columns", "for (int64_t c = j + 1; c < n; c++) {\n            double s = 0.0;\n            for (int64_t i = j + 1",
     "for (int64_t c = j + 2; c < n; c++) {\n            double s = 0.0;\n            for (int64_t i = j + 1"),
]


def detector_failures(orc):
    """Run the independent checks against one oracle build; return the names
    of the checks that fail."""
    fails = []

    def check(name, fn):
        try:
            with np.errstate(all="ignore"):
                ok = fn()
        except Exception:  # a crash or a rejected input counts as a failure
            ok = False
        if not ok:
            fails.append(name)

    def golden():
        for case in json.load(open(GOLDEN))["cases"]:
            S = np.array(case["S"], dtype=np.float64)
            X, e, lr, li = orc.standard(S)
            for (j, pair), ref in zip(column_groups(li), case["eigen"]):
                y_ref = np.array([complex(a, b) for a, b in ref["y"]])
                y = np.ldexp(X[:, j], -int(e[j])).astype(complex)
                if pair:
                    y = y + 1j * np.ldexp(X[:, j + 1], -int(e[j]))
                if not np.allclose(y, y_ref, rtol=0, atol=8 * U * np.abs(y_ref).max()):
                    return False
                lam = complex(*ref["lambda"])
                if abs(complex(lr[j], li[j]) - lam) > 8 * U * abs(lam):
                    return False
        return True

    T0, _ = workloads.config0_schur(96, seed=5)
    Q0 = workloads.householder_orthogonal(96, seed=6)

    def residual_std():
        X, e, lr, li = orc.standard(T0)
        if not np.isfinite(X).all():
            return False
        nr = canonical_norms(X, li)
        return standard_residuals(T0, X, lr, li).max() <= 10 * 96 and nr.min() >= 1 and nr.max() < 2

    def residual_backtransformed():
        X, e, lr, li = orc.standard(T0, Q=Q0)
        A = Q0 @ T0 @ Q0.T
        return np.isfinite(X).all() and standard_residuals(A, X, lr, li).max() <= 10 * 96

    def adversarial():
        T, _ = workloads.adversarial_schur(128, seed=8)
        X, e, lr, li = orc.standard(T)
        return np.isfinite(X).all() and standard_residuals(T, X, lr, li).max() <= 10 * 128

    def brute_force():
        T, blocks = workloads.config0_schur(20, seed=9)
        X, e, lr, li = orc.standard(T)
        col = 0
        for (p, sz) in blocks:
            y, _ = mp_eigvec(T, p, sz)
            xr, xi, emp = mp_canonical(y, sz == 2)
            de = int(e[col]) - emp
            if abs(de) > 1:
                return False
            err = np.abs(np.ldexp(X[:, col], -de) - xr)
            if sz == 2:
                err = err + np.abs(np.ldexp(X[:, col + 1], -de) - xi)
            if err.max() > 1e-12 * np.max(np.abs(xr) + np.abs(xi)):
                return False
            col += sz
        return True

    def generalized():
        S, T, _ = workloads.generalized_pair(80, seed=10)
        Z = workloads.householder_orthogonal(80, seed=11)
        X, e, ar, ai, be = orc.generalized(S, T, Z=Z)
        # residual of the original pencil (Z S Z^T, Z T Z^T) for X = Z Y
        A = Z @ S @ Z.T
        B = Z @ T @ Z.T
        return np.isfinite(X).all() and generalized_residuals(A, B, X, ar, ai, be).max() <= 10 * 80

    def left_residual():
        X, e, lr, li = orc.standard(T0, left=True)
        if not np.isfinite(X).all():
            return False
        nr = canonical_norms(X, li)
        return left_residuals(T0, X, lr, li).max() <= 10 * 96 and nr.min() >= 1 and nr.max() < 2

    def left_adversarial():
        T, _ = workloads.adversarial_schur(128, seed=8)
        X, e, lr, li = orc.standard(T, left=True)
        return np.isfinite(X).all() and left_residuals(T, X, lr, li).max() <= 10 * 128

    def left_brute_force():
        T, blocks = workloads.config0_schur(20, seed=9)
        X, e, lr, li = orc.standard(T, left=True)
        col = 0
        for (p, sz) in blocks:
            u, _ = mp_left_eigvec(T, p, sz)
            xr, xi, emp = mp_canonical(u, sz == 2)
            de = int(e[col]) - emp
            if abs(de) > 1:
                return False
            err = np.abs(np.ldexp(X[:, col], -de) - xr)
            if sz == 2:
                err = err + np.abs(np.ldexp(X[:, col + 1], -de) - xi)
            if err.max() > 1e-12 * np.max(np.abs(xr) + np.abs(xi)):
                return False
            col += sz
        return True

    def generalized_left():
        S, T, _ = workloads.generalized_pair(80, seed=12)
        Z = workloads.householder_orthogonal(80, seed=13)
        X, e, ar, ai, be = orc.generalized(S, T, Z=Z, left=True)
        A = Z @ S @ Z.T
        B = Z @ T @ Z.T
        if not (np.isfinite(X).all() and
                generalized_left_residuals(A, B, X, ar, ai, be).max() <= 10 * 80):
            return False
        # the flipped pencil's right eigenvalues, in reverse block order
        _, _, arf, aif, bef = orc.generalized(*flip_pencil(S, T))
        lam = np.sort_complex((ar + 1j * ai) / be)
        lamf = np.sort_complex((arf + 1j * aif) / bef)
        return np.allclose(lam, lamf, rtol=1e-12, atol=0)

    def generalized_left_adversarial():
        # T-dominated growth: large upper part in T, clusters 1e-9 apart
        rng = np.random.default_rng(14)
        n = 64
        S = np.triu(rng.standard_normal((n, n)), 1)
        T = np.triu(rng.standard_normal((n, n)) * 1e3, 1)
        d = rng.uniform(0.5, 2.0, n)
        lam = np.concatenate([-0.5 + (rng.permutation(32) - 16) * 1e-9,
                              0.5 + (rng.permutation(32) - 16) * 1e-9])
        S[np.arange(n), np.arange(n)] = lam * d
        T[np.arange(n), np.arange(n)] = d
        X, e, ar, ai, be = orc.generalized(S, T, left=True)
        return np.isfinite(X).all() and \
            generalized_left_residuals(S, T, X, ar, ai, be).max() <= 10 * n

    def hessenberg():
        A = np.random.default_rng(3).standard_normal((40, 40))
        H, Q, _ = orc.hessenberg(A)
        Hs, Qs = sl.hessenberg(A, calc_q=True)
        return (np.abs(H - Hs).max() <= 1e-11 and np.abs(Q @ H @ Q.T - A).max() <= 1e-11 and
                np.all(np.tril(H, -2) == 0.0))

    def window():
        # an orthogonal similarity keeps Q T Q^T; a cyclic permutation
        # window permutes by index arithmetic alone
        n = 48
        T, blocks = workloads.config0_schur(n, seed=21)
        Q = workloads.householder_orthogonal(n, seed=22)
        A = Q @ T @ Q.T
        T2, Q2 = orc.window_update(T, Q, workloads.window_chain(n, 16, 16, seed=23,
                                                                blocks=blocks))
        ok = np.abs(Q2 @ T2 @ Q2.T - A).max() <= 1e-12 * np.abs(A).max()
        a, k = 6, 5
        P = np.zeros((k, k))
        P[np.roll(np.arange(k), 1), np.arange(k)] = 1.0
        T3, _ = orc.window_update(T, None, [(a, P)])
        idx = np.arange(n)
        idx[a:a + k] = a + np.roll(np.arange(k), 1)
        Te = T.copy()
        Te[a:a + k, a:] = T[idx[a:a + k], a:]
        Te[:a + k, a:a + k] = Te[:a + k, idx[a:a + k]].copy()
        return ok and np.array_equal(T3, Te)

    check("golden", golden)
    check("residual_std", residual_std)
    check("residual_backtransformed", residual_backtransformed)
    check("adversarial", adversarial)
    check("brute_force", brute_force)
    check("generalized", generalized)
    check("left_residual", left_residual)
    check("left_adversarial", left_adversarial)
    check("left_brute_force", left_brute_force)
    check("generalized_left", generalized_left)
    check("generalized_left_adversarial", generalized_left_adversarial)
    check("hessenberg", hessenberg)
    check("window", window)
    return fails


def test_unmodified_oracle_passes_detectors():
    assert detector_failures(oracle.default()) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(oracle.source_path()).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / f"mut_{name}.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.compile_library(str(mutated), str(tmp_path / f"libmut_{name}.so"))
    fails = detector_failures(oracle.Oracle(lib))
    assert fails, f"mutant {name} passed every pin"
