"""Pins for the oracle's robust triangular solve (T x_j = b_j for every
column of B, the xLATRS generalisation the eigenvector solve rests on,
Sec. 3.3): library solvers on well-conditioned inputs, closed forms,
arbitrary-precision brute force on a matrix whose unscaled solve overflows,
and exact power-of-two relations.  Output convention: x_j = X[:, j] *
2**(-scale_exp[j]) with |X[:, j]|_inf in [1, 2)."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads


def _true(X, e):
    return np.ldexp(X, -e.astype(np.int64)[None, :])


def _upper(n, seed, diag=(1.0, 2.0)):
    rng = np.random.default_rng(seed)
    T = np.triu(rng.standard_normal((n, n)) / np.sqrt(n), 1)
    d = rng.uniform(*diag, n) * rng.choice([-1.0, 1.0], n)
    T[np.arange(n), np.arange(n)] = d
    return T


def test_against_scipy_triangular_solve():
    n = 200
    T = _upper(n, 1)
    B = np.random.default_rng(2).standard_normal((n, 7))
    X, e = oracle.trsolve(T, B)
    ref = sl.solve_triangular(T, B)
    assert np.abs(X).max(axis=0).min() >= 1.0 and np.abs(X).max(axis=0).max() < 2.0
    rel = np.abs(_true(X, e) - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert rel.max() <= 1e-12, rel.max()


def test_quasi_triangular_against_lapack_dense_solve():
    # 2x2 blocks (config-0 form) and the same blocks made non-standard:
    # the solve does not need the eigenvalue form of a block
    n = 150
    T, blocks = workloads.config0_schur(n, seed=3)
    T2 = T.copy()
    for p, sz in blocks:
        if sz == 2:
            T2[p, p] += 0.3
            T2[p + 1, p] *= 1.7
    B = np.random.default_rng(4).standard_normal((n, 5))
    for M in (T, T2):
        X, e = oracle.trsolve(M, B)
        ref = np.linalg.solve(M, B)
        rel = np.abs(_true(X, e) - ref).max(axis=0) / np.abs(ref).max(axis=0)
        cond = np.linalg.cond(M, 1)
        assert rel.max() <= 1e-15 * cond * n, (rel.max(), cond)


def test_two_by_two_closed_form():
    # a lone 2x2 block [[a, b], [c, d]]: x = (d b1 - b b2, a b2 - c b1) / det
    a, b, c, d = 1.5, -0.75, 0.5, 2.25
    T = np.array([[a, b], [c, d]])
    rhs = np.array([1.0, -3.0])
    X, e = oracle.trsolve(T, rhs)
    det = a * d - b * c
    x = np.array([(d * rhs[0] - b * rhs[1]) / det, (a * rhs[1] - c * rhs[0]) / det])
    np.testing.assert_allclose(_true(X, e)[:, 0], x, rtol=4e-16, atol=0)


def test_growth_witness_against_mpmath():
    # diagonal 2^-600, upper part 1: the true solution grows by about 2^600
    # per row, the unscaled substitution overflows after two rows; the
    # robust one stays finite and matches 256-bit backsubstitution
    import mpmath as mp
    mp.mp.prec = 256
    n = 12
    T = np.triu(np.ones((n, n)), 1)
    T[np.arange(n), np.arange(n)] = np.ldexp(1.0, -600) * (1 + np.arange(n) / n)
    b = np.linspace(1.0, 2.0, n)
    with np.errstate(all="ignore"):
        naive = np.zeros(n)
        for i in range(n - 1, -1, -1):
            naive[i] = (b[i] - T[i, i + 1:] @ naive[i + 1:]) / T[i, i]
    assert not np.isfinite(naive).all()
    X, e = oracle.trsolve(T, b)
    assert np.isfinite(X).all() and e[0] < -5000
    t = [[mp.mpf(float(T[i, j])) for j in range(n)] for i in range(n)]
    y = [mp.mpf(0)] * n
    for i in range(n - 1, -1, -1):
        s = mp.mpf(float(b[i])) - sum(t[i][j] * y[j] for j in range(i + 1, n))
        y[i] = s / t[i][i]
    top = max(abs(v) for v in y)
    for i in range(n):
        got = mp.mpf(float(X[i, 0])) * mp.mpf(2) ** (-int(e[0]))
        assert abs(got - y[i]) <= mp.mpf(1e-14) * top, i


def test_power_of_two_right_hand_side_and_zero_columns():
    # 2^k b gives the same X and an exponent lower by k; a zero column gives
    # X = 0, exponent 0
    n = 90
    T, _ = workloads.config0_schur(n, seed=5)
    B = np.random.default_rng(6).standard_normal((n, 4))
    B[:, 2] = 0.0
    X0, e0 = oracle.trsolve(T, B)
    for k in (-40, 17):
        X1, e1 = oracle.trsolve(T, np.ldexp(B, k))
        np.testing.assert_array_equal(X0, X1)
        nz = np.abs(B).max(axis=0) > 0
        np.testing.assert_array_equal(e1[nz], e0[nz] - k)
    assert np.all(X0[:, 2] == 0.0) and e0[2] == 0


def test_residual_and_thread_invariance():
    n = 300
    T, _ = workloads.config0_schur(n, seed=7)
    B = np.random.default_rng(8).standard_normal((n, 6))
    X1, e1 = oracle.trsolve(T, B, threads=1)
    X4, e4 = oracle.trsolve(T, B, threads=4)
    np.testing.assert_array_equal(X1, X4)
    np.testing.assert_array_equal(e1, e4)
    x = _true(X1, e1)
    Tl = T.astype(np.longdouble)
    r = Tl @ x.astype(np.longdouble) - B.astype(np.longdouble)
    nrm = np.abs(Tl).sum(axis=0).max() * np.abs(x).sum(axis=0)
    assert float((np.abs(r).sum(axis=0) / (nrm * 2.0 ** -53)).max()) <= 10 * n


def test_errors():
    n = 20
    T, blocks = workloads.config0_schur(n, seed=9)
    B = np.ones((n, 3))
    bad = B.copy()
    bad[4, 1] = np.nan
    with pytest.raises(oracle.OracleError) as ei:
        oracle.trsolve(T, bad)
    assert ei.value.status == oracle.ENONFINITE and ei.value.bad == n * n + 4 + 1 * n
    bad = B.copy()
    bad[0, 2] = 2.0 ** 1001
    with pytest.raises(oracle.OracleError) as ei:
        oracle.trsolve(T, bad)
    assert ei.value.status == oracle.EINVAL
    T2 = T.copy()
    p = next(q for q, sz in blocks if sz == 2)
    T2[p + 2, p + 1] = 0.5                      # two nonzero subdiagonals in a row
    with pytest.raises(oracle.OracleError) as ei:
        oracle.trsolve(T2, B)
    assert ei.value.status == oracle.ENOTSCHUR
