"""Pins for the oracle's generalized path, (S - lambda T) y = 0 in
homogeneous form (beta S - alpha T) y = 0 (Sec. 2, Eq. evec_solve; Sec. 3.3
for the robust scaling; the generalized solver is the subject of the
paper's reference [ppam2019cckm])."""
import numpy as np

import oracle
import workloads
from evec_checks import (U, canonical_norms, column_groups, generalized_residuals,
                         mp_canonical, mp_gen_eigvec, standard_residuals)


def _true(X, e, j, pair):
    v = np.ldexp(X[:, j], -int(e[j])).astype(complex)
    if pair:
        v = v + 1j * np.ldexp(X[:, j + 1], -int(e[j]))
    return v


def test_upper_triangular_2x2_closed_form():
    rng = np.random.default_rng(21)
    for _ in range(50):
        s11, s22, s12 = rng.uniform(-2, 2, 3)
        t11, t22 = rng.uniform(0.5, 2, 2)
        t12 = rng.standard_normal()
        S = np.array([[s11, s12], [0, s22]])
        T = np.array([[t11, t12], [0, t22]])
        X, e, ar, ai, be = oracle.generalized(S, T)
        # lambda_2 = s22 / t22; x = (-(s12 - lambda t12) / (s11 - lambda t11), 1)
        lam = s22 / t22
        assert abs(ar[1] / be[1] - lam) <= 8 * U * abs(lam) + 1e-300
        x = _true(X, e, 1, False).real
        ref = np.array([-(s12 - lam * t12) / (s11 - lam * t11), 1.0])
        assert np.allclose(x, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
        # (alpha, beta) normalised: max(|alpha|, beta) in [1, 2)
        for j in range(2):
            mx = max(abs(ar[j]), abs(ai[j]), be[j])
            assert 1.0 <= mx < 2.0


def test_identity_T_reduces_to_standard():
    S, blocks = workloads.config0_schur(128, seed=31)
    T = np.eye(128)
    Xg, eg, ar, ai, be = oracle.generalized(S, T)
    Xs, es, lr, li = oracle.standard(S)
    for j, pair in column_groups(li):
        assert abs(int(eg[j]) - int(es[j])) <= 1
        cols = [j, j + 1] if pair else [j]
        a = np.ldexp(Xg[:, cols], int(es[j]) - int(eg[j]))
        assert np.abs(a - Xs[:, cols]).max() <= 1e-12
        assert np.allclose(ar[j] / be[j], lr[j], rtol=1e-15, atol=1e-15)
        assert np.allclose(ai[j] / be[j], li[j], rtol=1e-15, atol=1e-15)


def test_config4_residual_and_structure():
    S, T, blocks = workloads.generalized_pair(300, seed=41)
    X, e, ar, ai, be = oracle.generalized(S, T)
    res = generalized_residuals(S, T, X, ar, ai, be)
    assert res.max() <= 10 * 300
    nr = canonical_norms(X, ai)
    assert np.all(nr >= 1.0) and np.all(nr < 2.0)
    col = 0
    for (p, sz) in blocks:
        for k in range(sz):
            assert np.all(X[p + sz:, col + k] == 0.0)
        col += sz
    # near-infinite eigenvalues are present and handled: beta tiny
    assert (be < 1e-10).sum() >= 5


def test_mpmath_generalized_small():
    S, T, blocks = workloads.generalized_pair(40, seed=51)
    X, e, ar, ai, be = oracle.generalized(S, T)
    col = 0
    worst = 0.0
    for (p, sz) in blocks:
        y = mp_gen_eigvec(S, T, p, sz)
        xr, xi, emp = mp_canonical(y, sz == 2)
        de = int(e[col]) - emp
        assert abs(de) <= 1
        got = np.ldexp(X[:, col], -de)
        err = np.abs(got - xr)
        den = np.max(np.abs(xr) + np.abs(xi))
        if sz == 2:
            err = err + np.abs(np.ldexp(X[:, col + 1], -de) - xi)
        worst = max(worst, err.max() / den)
        col += sz
    assert worst <= 1e-11, worst


def test_unequal_diagonal_T_pair():
    """A 2x2 block of S over a diagonal (not scalar) block of T."""
    S = np.array([[0.3, 1.0, 0.5], [0.0, 0.2, 1.5], [0.0, -1.0, 0.4]])
    T = np.array([[1.0, 0.3, -0.2], [0.0, 0.5, 0.0], [0.0, 0.0, 2.0]])
    X, e, ar, ai, be = oracle.generalized(S, T)
    res = generalized_residuals(S, T, X, ar, ai, be)
    assert res.max() <= 30
    y = mp_gen_eigvec(S, T, 1, 2)
    xr, xi, emp = mp_canonical(y, True)
    got = np.ldexp(X[:, 1], emp - int(e[1])) + 1j * np.ldexp(X[:, 2], emp - int(e[1]))
    assert np.abs(got - (xr + 1j * xi)).max() <= 1e-13


def test_backtransform_Z():
    S, T, blocks = workloads.generalized_pair(96, seed=61)
    Z = workloads.householder_orthogonal(96, seed=62)
    X, e, ar, ai, be = oracle.generalized(S, T)
    Xz, ez, _, _, _ = oracle.generalized(S, T, Z=Z)
    for j, pair in column_groups(ai):
        cols = [j, j + 1] if pair else [j]
        ref = Z @ X[:, cols]
        got = np.ldexp(Xz[:, cols], int(e[j]) - int(ez[j]))
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_generalized_standard_residual_equivalence():
    """With T = diag(d) scalar d on every block, (S, dI) has the eigenvectors
    of S; the residual of the standard problem must be small too."""
    S, blocks = workloads.config0_schur(64, seed=71)
    T = 0.75 * np.eye(64)
    X, e, ar, ai, be = oracle.generalized(S, T)
    # S x = lambda (0.75 I) x: the standard eigenvalue is 0.75 alpha / beta
    lr = 0.75 * ar / be
    li = 0.75 * ai / be
    res = standard_residuals(S, X, lr, li)
    assert res.max() <= 10 * 64
