"""Pins for the CPU oracle: closed forms, the paper's invariants, brute force
in arbitrary precision, a library special case, overflow witnesses and
metamorphic relations.  None of these re-types the oracle's formulas: each
compares it with something the mathematics fixes independently.

Paper: Sec. 2 (Eq. evec_solve, Eq. evec_backtransform); Sec. 3.3 (robust
computation of eigenvectors: augmented representation y = x / alpha,
power-of-two scale factors, no overflow).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads
from evec_checks import (U, canonical_norms, column_groups, compare_canonical,
                         complex_columns, extended_errors, ld_real_eigvec,
                         longdouble_is_extended, mp_canonical, mp_eigvec,
                         standard_residuals)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _true_vec(X, e, j, pair):
    if pair:
        return np.ldexp(X[:, j], -int(e[j])) + 1j * np.ldexp(X[:, j + 1], -int(e[j]))
    return np.ldexp(X[:, j], -int(e[j])).astype(complex)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def test_hand_derived_golden_examples():
    cases = json.load(open(GOLDEN))["cases"]
    for case in cases:
        S = np.array(case["S"], dtype=np.float64)
        X, e, lr, li = oracle.standard(S)
        groups = list(column_groups(li))
        assert len(groups) == len(case["eigen"])
        for (j, pair), ref in zip(groups, case["eigen"]):
            y_ref = np.array([complex(a, b) for a, b in ref["y"]])
            lam = complex(*ref["lambda"])
            # w = sqrt(|b|) sqrt(|c|) is rounded: allow a few ulps
            assert abs(lr[j] - lam.real) <= 4 * U * abs(lam) and abs(li[j] - lam.imag) <= 4 * U * abs(lam), case["name"]
            y = _true_vec(X, e, j, pair)
            assert np.allclose(y, y_ref, rtol=0, atol=4 * U * np.abs(y_ref).max()), (case["name"], y, y_ref)
            assert abs(int(e[j]) - ref["canonical_exponent"]) <= 1


def test_one_by_one():
    for v in (-3.5, 0.0, 1e-300, 7.0):
        X, e, lr, li = oracle.standard(np.array([[v]]))
        assert X[0, 0] == 1.0 and e[0] == 0 and lr[0] == v and li[0] == 0.0


def test_upper_triangular_2x2_distinct():
    rng = np.random.default_rng(1)
    for _ in range(50):
        t11, t22, t12 = rng.uniform(-2, 2, 3)
        S = np.array([[t11, t12], [0.0, t22]])
        X, e, lr, li = oracle.standard(S)
        y = _true_vec(X, e, 1, False)
        ref = np.array([-t12 / (t11 - t22), 1.0])
        assert np.allclose(y, ref, rtol=8 * U, atol=0)
        assert np.all(X[:, 0] == [1.0, 0.0])


def test_standardized_pair_is_null_vector():
    rng = np.random.default_rng(2)
    for _ in range(100):
        a = rng.uniform(-1, 1)
        b = rng.uniform(0.1, 3) * rng.choice([-1, 1])
        c = -np.sign(b) * rng.uniform(0.1, 3)
        B = np.array([[a, b], [c, a]])
        X, e, lr, li = oracle.standard(B)
        w = np.sqrt(abs(b) * abs(c))
        assert lr[0] == a and lr[1] == a and li[1] == -li[0]
        assert abs(li[0] - w) <= 4 * U * w
        w = li[0]
        v = _true_vec(X, e, 0, True)
        lam = a + 1j * w
        r = (B - lam * np.eye(2)) @ v
        assert np.abs(r).max() <= 8 * U * np.abs(B).max() * np.abs(v).max()
        # the block part follows the convention: (1, i w / b) or (-w / c, i)
        if abs(b) >= abs(c):
            assert np.allclose(v / v[0], [1.0, 1j * w / b], rtol=4 * U, atol=4 * U)
        else:
            assert np.allclose(v / v[1] * 1j, [-w / c, 1j], rtol=4 * U, atol=4 * U)


def test_three_by_three_pair_at_bottom():
    rng = np.random.default_rng(3)
    for _ in range(50):
        t11 = rng.uniform(-1, 1)
        t12, t13 = rng.standard_normal(2)
        a = rng.uniform(-1, 1)
        b = rng.uniform(0.5, 1.0)
        c = -rng.uniform(0.1, 0.4)     # |b| >= |c|: block part (1, i w / b)
        S = np.array([[t11, t12, t13], [0, a, b], [0, c, a]])
        X, e, lr, li = oracle.standard(S)
        w = np.sqrt(b * -c)
        lam = a + 1j * w
        v = _true_vec(X, e, 1, True)
        v1 = -(t12 + 1j * w * t13 / b) / (t11 - lam)
        ref = np.array([v1, 1.0, 1j * w / b])
        assert np.allclose(v, ref, rtol=16 * U, atol=16 * U)
        assert np.all(X[:, 0] == [1.0, 0.0, 0.0])


def test_three_by_three_real_at_bottom_cramer():
    rng = np.random.default_rng(4)
    for _ in range(50):
        a = rng.uniform(-1, 1)
        b = rng.uniform(0.1, 1.0)
        c = -rng.uniform(0.1, 1.0)
        mu = rng.uniform(-1, 1)
        t13, t23 = rng.standard_normal(2)
        S = np.array([[a, b, t13], [c, a, t23], [0, 0, mu]])
        X, e, lr, li = oracle.standard(S)
        assert li[2] == 0.0 and lr[2] == mu
        x = _true_vec(X, e, 2, False).real
        # [x1; x2] = -(B - mu I)^{-1} [t13; t23] by Cramer's rule
        m11, m12, m21, m22 = a - mu, b, c, a - mu
        det = m11 * m22 - m12 * m21
        x1 = -(t13 * m22 - m12 * t23) / det
        x2 = -(m11 * t23 - m21 * t13) / det
        assert np.allclose(x, [x1, x2, 1.0], rtol=32 * U, atol=32 * U * max(1, abs(x1), abs(x2)))


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg0_256():
    T, blocks = workloads.config0_schur(256)
    X, e, lr, li = oracle.standard(T)
    return T, blocks, X, e, lr, li


def test_zero_below_block_and_canonical_norm(cfg0_256):
    T, blocks, X, e, lr, li = cfg0_256
    col = 0
    for (p, sz) in blocks:
        for k in range(sz):
            assert np.all(X[p + sz:, col + k] == 0.0)
        col += sz
    nr = canonical_norms(X, li)
    assert np.all(nr >= 1.0) and np.all(nr < 2.0)
    for j, pair in column_groups(li):
        if pair:
            assert e[j] == e[j + 1]
            assert lr[j] == lr[j + 1] and li[j] == -li[j + 1] and li[j] > 0


def test_block_count_matches_layout(cfg0_256):
    T, blocks, X, e, lr, li = cfg0_256
    assert X.shape[1] == sum(sz for _, sz in blocks) == 256
    pairs = sum(1 for _, sz in blocks if sz == 2)
    assert sum(1 for _, p in column_groups(li) if p) == pairs


def test_residual_config0(cfg0_256):
    T, blocks, X, e, lr, li = cfg0_256
    res = standard_residuals(T, X, lr, li)
    assert res.max() <= 10 * T.shape[0]


def test_numpy_eig_directions(cfg0_256):
    """LAPACK dgeev (numpy.linalg.eig) is the library special case: on a
    well-conditioned input the directions must agree."""
    T, blocks, X, e, lr, li = cfg0_256
    w, V = np.linalg.eig(T)
    vecs = complex_columns(X, li)
    lams = [lr[j] + 1j * li[j] for j, _ in column_groups(li)]
    worst = 0.0
    for x, lam in zip(vecs, lams):
        k = np.argmin(np.abs(w - lam))
        v = V[:, k]
        c = abs(np.vdot(x, v)) / (np.linalg.norm(x) * np.linalg.norm(v))
        worst = max(worst, 1 - c)
    assert worst <= 1e-12


def test_selection_invariance(cfg0_256):
    T, blocks, X, e, lr, li = cfg0_256
    sel = workloads.random_eigen_selection(256, blocks, 0.35, seed=9)
    Xs, es, lrs, lis = oracle.standard(T, select=sel)
    # map selected columns back to the full result
    cols = []
    col = 0
    for (p, sz) in blocks:
        if sel[p] or (sz == 2 and sel[p + 1]):
            cols.extend(range(col, col + sz))
        col += sz
    assert Xs.shape[1] == len(cols)
    assert np.array_equal(Xs, X[:, cols])
    assert np.array_equal(es, e[cols])
    assert np.array_equal(lrs, lr[cols]) and np.array_equal(lis, li[cols])


def test_thread_count_invariance(cfg0_256):
    T, blocks, X, e, lr, li = cfg0_256
    X1, e1, _, _ = oracle.standard(T, threads=1)
    assert np.array_equal(X1, X) and np.array_equal(e1, e)


@pytest.mark.parametrize("k", [-100, 100, 6])
def test_power_of_two_metamorphic(cfg0_256, k):
    """T -> 2^k T leaves every eigenvector unchanged and every computed
    quantity scaled exactly, so the canonical output is bit-identical.
    k is even: a pair's w = sqrt(|b|) sqrt(|c|) scales exactly by 2^(k/2)
    only then (sqrt(2) is irrational)."""
    T, blocks, X, e, lr, li = cfg0_256
    X2, e2, lr2, li2 = oracle.standard(np.ldexp(T, k))
    assert np.array_equal(X2, X) and np.array_equal(e2, e)
    assert np.array_equal(lr2, np.ldexp(lr, k)) and np.array_equal(li2, np.ldexp(li, k))


def test_backtransform_matches_definition(cfg0_256):
    T, blocks, X, e, lr, li = cfg0_256
    Q = workloads.householder_orthogonal(256, seed=11)
    assert np.abs(Q.T @ Q - np.eye(256)).max() < 1e-13
    Xq, eq, _, _ = oracle.standard(T, Q=Q)
    for j, pair in column_groups(li):
        cols = [j, j + 1] if pair else [j]
        ref = Q @ X[:, cols]
        got = np.ldexp(Xq[:, cols], int(e[j]) - int(eq[j]))
        assert np.abs(got - ref).max() <= 64 * U * 16 * np.abs(ref).max()
    nr = canonical_norms(Xq, li)
    assert np.all(nr >= 1.0) and np.all(nr < 2.0)


# --------------------------------------------------------------------------
# brute force in arbitrary precision (mpmath, 256-bit, unbounded exponent)
# --------------------------------------------------------------------------

def _mp_compare(T, blocks, X, e, li, tol, max_cols=None):
    col = 0
    checked = 0
    worst = 0.0
    for (p, sz) in blocks:
        if max_cols is not None and checked >= max_cols:
            break
        y, lam = mp_eigvec(T, p, sz)
        xr, xi, emp = mp_canonical(y, sz == 2)
        de = int(e[col]) - emp
        assert abs(de) <= 1, (p, e[col], emp)
        got_r = np.ldexp(X[:, col], -de)
        err = np.abs(got_r - xr)
        if sz == 2:
            got_i = np.ldexp(X[:, col + 1], -de)
            err = err + np.abs(got_i - xi)
            den = np.max(np.abs(xr) + np.abs(xi))
        else:
            den = np.max(np.abs(xr))
        worst = max(worst, err.max() / den)
        col += sz
        checked += 1
    assert worst <= tol, worst
    return worst


def test_mpmath_config0_small():
    T, blocks = workloads.config0_schur(48, seed=123)
    X, e, lr, li = oracle.standard(T)
    _mp_compare(T, blocks, X, e, li, tol=1e-12)


def test_mpmath_adversarial_small():
    """Two clusters of 32 eigenvalues 1e-9 apart, upper part N(0,1)*1e3:
    exact solution entries grow past the double range.  The oracle must
    agree with the 256-bit reference in exponent (+-1) and, normwise, to
    the conditioning of the cluster (forward error ~ |T| / gap * u)."""
    rng = np.random.default_rng(5)
    n = 64
    T = np.triu(rng.standard_normal((n, n)) * 1e3, 1)
    diag = np.concatenate([-0.5 + (rng.permutation(32) - 16) * 1e-9,
                           0.5 + (rng.permutation(32) - 16) * 1e-9])
    T[np.arange(n), np.arange(n)] = diag
    blocks = [(i, 1) for i in range(n)]
    X, e, lr, li = oracle.standard(T)
    assert np.isfinite(X).all()
    assert e.min() < -1100       # the true vectors leave the double range
    _, bad = oracle.naive_standard(T)
    assert bad > 0
    _mp_compare(T, blocks, X, e, li, tol=1e-4)


def _ld_to_mpf(v):
    # exact: a longdouble is m 2^ex with a 64-bit integer significand
    import mpmath as mp
    m, ex = np.frexp(v)
    return mp.mpf(int(np.ldexp(m, 64))) * mp.mpf(2) ** (int(ex) - 64)


@pytest.mark.skipif(not longdouble_is_extended(), reason="no extended long double")
def test_extended_reference_against_mpmath():
    # the longdouble backsubstitution (the large-n reference) against the
    # 256-bit one on a config-0 matrix and on a growth witness past 2^1024
    import mpmath as mp
    T, blocks = workloads.config0_schur(40, seed=77)
    rng = np.random.default_rng(8)
    n = 40
    A = np.triu(rng.standard_normal((n, n)) * 1e3, 1)
    A[np.arange(n), np.arange(n)] = 0.5 + (rng.permutation(n) - 20) * 1e-9
    past_double = False
    for M, blk in ((T, blocks), (A, [(i, 1) for i in range(n)])):
        for p, sz in blk:
            if sz != 1 or p < 5:
                continue
            y_mp, _ = mp_eigvec(M, p, 1)
            y_ld = ld_real_eigvec(M, blk, p)
            top = max(abs(v) for v in y_mp[:p + 1])
            past_double |= top > mp.mpf(2) ** 1024
            for i in range(p + 1):
                assert abs(y_mp[i].real - _ld_to_mpf(y_ld[i])) <= mp.mpf(1e-15) * top, (p, i)
    assert past_double


@pytest.mark.skipif(not longdouble_is_extended(), reason="no extended long double")
def test_oracle_against_extended_reference():
    # n = 600 config-0: every real column of the oracle agrees with the
    # extended-precision backsubstitution in direction to 1e-13 and, with
    # its exponent, to 1e-10
    n = 600
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE + 9)
    X, e, lr, li = oracle.standard(T)
    col = 0
    worst = (0.0, 0.0)
    for p, sz in blocks:
        if sz == 1 and p % 7 == 0:
            d, s = extended_errors(ld_real_eigvec(T, blocks, p), X[:, col], e[col])
            worst = (max(worst[0], d), max(worst[1], s))
        col += sz
    assert worst[0] <= 1e-13 and worst[1] <= 1e-10, worst


def test_mpmath_pairs_dense():
    """Every other block a 2x2 pair, so complex shifts meet 2x2 blocks."""
    rng = np.random.default_rng(6)
    n = 40
    T = np.triu(rng.standard_normal((n, n)), 1)
    blocks = []
    i = 0
    while i < n:
        if i % 3 == 0 and i + 1 < n:
            a = rng.uniform(-1, 1)
            b = rng.uniform(0.1, 1)
            c = -b * rng.uniform(0.1, 1) if rng.random() < 0.5 else -rng.uniform(1, 3)
            T[i, i] = T[i + 1, i + 1] = a
            T[i, i + 1] = b
            T[i + 1, i] = c
            blocks.append((i, 2))
            i += 2
        else:
            T[i, i] = rng.uniform(-1, 1)
            blocks.append((i, 1))
            i += 1
    X, e, lr, li = oracle.standard(T)
    _mp_compare(T, blocks, X, e, li, tol=1e-11)


# --------------------------------------------------------------------------
# overflow witness and robustness
# --------------------------------------------------------------------------

def test_adversarial_overflow_witness():
    T, blocks = workloads.adversarial_schur(512, seed=77)
    _, bad = oracle.naive_standard(T)
    assert bad > 0, "the unscaled substitution was expected to overflow"
    X, e, lr, li = oracle.standard(T)
    assert np.isfinite(X).all()
    nr = canonical_norms(X, li)
    assert np.all(nr >= 1.0) and np.all(nr < 2.0)
    res = standard_residuals(T, X, lr, li)
    assert res.max() <= 10 * 512
    assert e.min() < -1074       # far outside the double range


def test_protect_division_near_singular_shift():
    """Equal eigenvalues: the pivot is perturbed to smin instead of
    dividing by zero; the result stays finite with a tiny residual."""
    S = np.array([[0.5, 1.0, 2.0], [0.0, 0.5, 1.0], [0.0, 0.0, 0.5]])
    X, e, lr, li = oracle.standard(S)
    assert np.isfinite(X).all()
    res = standard_residuals(S, X, lr, li)
    assert res.max() <= 10 * 3


# --------------------------------------------------------------------------
# input validation
# --------------------------------------------------------------------------

def test_rejects_non_standardized_pair():
    S = np.array([[1.0, 2.0], [-1.0, 1.5]])      # unequal diagonal
    with pytest.raises(oracle.OracleError) as ei:
        oracle.standard(S)
    assert ei.value.status == oracle.ENOTSCHUR
    S = np.array([[1.0, 2.0], [1.0, 1.0]])       # real eigenvalues
    with pytest.raises(oracle.OracleError) as ei:
        oracle.standard(S)
    assert ei.value.status == oracle.ENOTSCHUR


def test_rejects_consecutive_subdiagonals():
    S = np.triu(np.ones((4, 4)))
    S[1, 0] = -1.0
    S[2, 1] = -1.0
    with pytest.raises(oracle.OracleError) as ei:
        oracle.standard(S)
    assert ei.value.status == oracle.ENOTSCHUR and ei.value.bad == 1


def test_rejects_nonfinite_and_huge():
    S = np.triu(np.ones((3, 3)))
    S[0, 2] = np.inf
    with pytest.raises(oracle.OracleError) as ei:
        oracle.standard(S)
    assert ei.value.status == oracle.ENONFINITE
    S[0, 2] = 2.0 ** 1010
    with pytest.raises(oracle.OracleError) as ei:
        oracle.standard(S)
    assert ei.value.status == oracle.EINVAL


def test_empty():
    X, e, lr, li = oracle.standard(np.zeros((0, 0)))
    assert X.shape == (0, 0) and e.shape == (0,)
