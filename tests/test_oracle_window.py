"""Pins for the oracle's eigenvalue-reordering off-diagonal updates
(oracle.window_update: each window's accumulated orthogonal transform Z
applied as T <- Zhat^T T Zhat, Q <- Q Zhat; the left and right update
tasks of the paper's reordering phase, Sec. 3.2).  Each pin is fixed by the
mathematics, not by the oracle's own formula: the identity, exact
permutations by index arithmetic, the invariant Q T Q^T of an orthogonal
similarity, disjoint windows commuting, untouched regions, eigenvalues of a
small case, and bad windows."""
import numpy as np
import pytest

import oracle
import workloads

U = 2.0 ** -53


def _setup(n, seed=3):
    T, blocks = workloads.config0_schur(n, seed=seed)
    Q = workloads.householder_orthogonal(n, seed=seed + 1)
    return T, Q, blocks


def test_identity_windows_change_nothing():
    T, Q, blocks = _setup(30)
    T2, Q2 = oracle.window_update(T, Q, [(4, np.eye(9)), (0, np.eye(30))])
    np.testing.assert_array_equal(T2, T)
    np.testing.assert_array_equal(Q2, Q)


def test_permutation_window_is_exact():
    # Z = P, a cyclic shift (not symmetric): T <- P^T T P permutes rows and
    # columns of the window by index arithmetic alone
    n, a, k = 20, 5, 7
    T, Q, blocks = _setup(n)
    perm = np.roll(np.arange(k), 1)              # column i of P is e_perm[i]
    P = np.zeros((k, k))
    P[perm, np.arange(k)] = 1.0
    T2, Q2 = oracle.window_update(T, Q, [(a, P)])
    idx = np.arange(n)
    idx[a:a + k] = a + perm
    Te = T.copy()
    Te[a:a + k, a:] = T[idx[a:a + k], a:]        # rows a..b-1 from column a on
    Tc = Te.copy()
    Tc[:a + k, a:a + k] = Te[:a + k, idx[a:a + k]]
    np.testing.assert_array_equal(T2, Tc)
    np.testing.assert_array_equal(Q2, Q[:, idx])


def test_similarity_invariant_and_orthogonality():
    # disjoint windows: each one's rows below it and columns left of it are
    # still the zeros of the quasi-triangular form when it is applied, so
    # the structured update is the full similarity (overlapping windows need
    # accumulators that keep the window's diagonal block quasi-triangular,
    # as the window task's do)
    n = 90
    T, Q, blocks = _setup(n)
    A = Q @ T @ Q.T
    wins = workloads.window_chain(n, 24, 24, seed=5, blocks=blocks)
    T2, Q2 = oracle.window_update(T, Q, wins)
    assert np.abs(Q2 @ T2 @ Q2.T - A).max() <= 64 * n * U * np.abs(A).max()
    assert np.abs(Q2.T @ Q2 - np.eye(n)).max() <= 64 * n * U


def test_disjoint_windows_commute():
    # transforms on disjoint index sets commute: either order gives the same
    # matrices up to rounding
    n = 40
    T, Q, blocks = _setup(n, seed=7)
    w = workloads.window_chain(n, 13, 13, seed=11, blocks=blocks)
    T1, Q1 = oracle.window_update(T, Q, w)
    T2, Q2 = oracle.window_update(T, Q, w[::-1])
    assert np.abs(T1 - T2).max() <= 64 * n * U * np.abs(T).max()
    assert np.abs(Q1 - Q2).max() <= 64 * n * U


def test_untouched_regions_stay_exact():
    n, a, k = 50, 17, 11
    T, Q, blocks = _setup(n, seed=13)
    Z = workloads.window_chain(k, k, k, seed=17)[0][1]
    T2, Q2 = oracle.window_update(T, None, [(a, Z)])
    b = a + k
    # rows above the window outside its columns, and rows below it
    np.testing.assert_array_equal(T2[:a, :a], T[:a, :a])
    np.testing.assert_array_equal(T2[:a, b:], T[:a, b:])
    np.testing.assert_array_equal(T2[b:, :], T[b:, :])
    # the window's rows left of it (zeros below the diagonal)
    np.testing.assert_array_equal(T2[a:b, :a], T[a:b, :a])
    assert Q2 is None


def test_eigenvalues_preserved_small():
    n = 12
    T, _ = workloads.config0_schur(n, seed=19)
    Z = workloads.window_chain(6, 6, 6, seed=23)[0][1]
    T2, _ = oracle.window_update(T, None, [(3, Z)])
    e1 = np.sort_complex(np.linalg.eigvals(T))
    e2 = np.sort_complex(np.linalg.eigvals(T2))
    assert np.abs(e1 - e2).max() <= 1e-10 * max(1.0, np.abs(e1).max())


@pytest.mark.parametrize("a,k", [(-1, 3), (8, 3), (0, 11)])
def test_bad_windows_rejected(a, k):
    T, Q, blocks = _setup(10)
    with pytest.raises(oracle.OracleError):
        oracle.window_update(T, Q, [(a, np.eye(k))])
