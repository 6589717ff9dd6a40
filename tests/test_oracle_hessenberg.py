"""Pins for the oracle's Hessenberg reduction (A = Q H Q^T, Sec. 3.1's first
phase; one Householder reflector per column, unblocked): LAPACK's dgehrd
(scipy.linalg.hessenberg, the same reflector convention), orthogonality and
backward error, the exact zero pattern, the symmetric special case
(tridiagonal H), an input already in Hessenberg form, exact power-of-two
scaling and input errors."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle

U = 2.0 ** -53


def _rand(n, seed):
    return np.random.default_rng(seed).standard_normal((n, n))


@pytest.mark.parametrize("n", [3, 17, 200])
def test_against_lapack_dgehrd(n):
    A = _rand(n, n)
    H, Q, tau = oracle.hessenberg(A)
    Hs, Qs = sl.hessenberg(A, calc_q=True)
    nrm = np.abs(A).max()
    assert np.abs(H - Hs).max() <= 16 * n * U * nrm * np.sqrt(n)
    assert np.abs(Q - Qs).max() <= 16 * n * U * np.sqrt(n)


def test_orthogonality_backward_error_and_zeros():
    n = 300
    A = _rand(n, 7)
    H, Q, tau = oracle.hessenberg(A)
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 4 * n * U
    assert np.abs(Q @ H @ Q.T - A).max() <= 4 * n * U * np.abs(A).max() * np.sqrt(n)
    assert np.all(np.tril(H, -2) == 0.0)
    # the reflectors leave row and column 0 of Q alone
    assert Q[0, 0] == 1.0 and np.all(Q[0, 1:] == 0.0) and np.all(Q[1:, 0] == 0.0)
    assert np.all(tau[n - 2:] == 0.0) and np.all((tau[: n - 2] >= 1.0) & (tau[: n - 2] <= 2.0))


def test_symmetric_input_gives_tridiagonal():
    n = 120
    B = _rand(n, 9)
    A = B + B.T
    H, Q, _ = oracle.hessenberg(A)
    nrm = np.abs(A).max()
    assert np.abs(np.triu(H, 2)).max() <= 8 * n * U * nrm
    assert np.abs(H - H.T).max() <= 8 * n * U * nrm
    w = np.sort(np.linalg.eigvalsh((H + H.T) / 2))
    assert np.abs(w - np.sort(np.linalg.eigvalsh(A))).max() <= 8 * n * U * nrm


def test_already_hessenberg_is_left_alone():
    n = 40
    A = np.triu(_rand(n, 3), -1)
    H, Q, tau = oracle.hessenberg(A)
    assert np.array_equal(H, A) and np.array_equal(Q, np.eye(n)) and np.all(tau == 0.0)


@pytest.mark.parametrize("k", [-900, -300, 200, 900])
def test_power_of_two_scaling(k):
    # (the GPU test at 2^+-900 compares the scaled results with this oracle)
    A = _rand(60, 11)
    H, Q, tau = oracle.hessenberg(A)
    H2, Q2, tau2 = oracle.hessenberg(np.ldexp(A, k))
    assert np.array_equal(H2, np.ldexp(H, k))
    assert np.array_equal(Q2, Q) and np.array_equal(tau2, tau)


def test_large_entries_do_not_overflow():
    # entries near the input limit: the scaled norms keep every square finite
    A = np.ldexp(_rand(50, 13), 990)
    H, Q, _ = oracle.hessenberg(A)
    assert np.isfinite(H).all()
    Hs, _ = sl.hessenberg(np.ldexp(A, -990), calc_q=True)
    assert np.abs(np.ldexp(H, -990) - Hs).max() <= 1e-12 * np.abs(Hs).max()


def test_errors():
    A = _rand(20, 1)
    bad = A.copy()
    bad[4, 7] = np.nan
    with pytest.raises(oracle.OracleError) as ei:
        oracle.hessenberg(bad)
    assert ei.value.status == oracle.ENONFINITE and ei.value.bad == 4 + 7 * 20
    bad = A.copy()
    bad[2, 3] = 2.0 ** 1001
    with pytest.raises(oracle.OracleError) as ei:
        oracle.hessenberg(bad)
    assert ei.value.status == oracle.EINVAL

