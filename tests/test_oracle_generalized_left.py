"""Pins for the oracle's left eigenvectors of a pencil: u^H (beta S - alpha T)
= 0, the eigenvector problem of Sec. 2 for the transposed pencil, by robust
forward substitution (Sec. 3.3's protection, with the generalized bound of
the update C = beta S - alpha T, applied in the other direction).  Closed
forms, reduction to the standard left problem, LAPACK's left generalized
eigenvectors, biorthogonality with the right eigenvectors, arbitrary-
precision brute force on the flipped pencil, and metamorphic relations.

Output convention: X[:, j] * 2**(-e[j]) is u, zero above its block; a 2x2
block gives (Re u, Im u) for the member with Im alpha > 0, and (alpha, beta)
of a 2x2 block are those of the reversed transposed block (entries (s22,
s12; s21, s11) against diag(d2, d1)): the same eigenvalue, with the pair
normalised against d2."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads
from evec_checks import (U, canonical_norms, column_groups, compare_canonical, flip_pencil,
                         generalized_left_residuals, mp_canonical, mp_gen_left_eigvec)


def _u(X, e, j, pair):
    u = np.ldexp(X[:, j], -int(e[j])).astype(complex)
    if pair:
        u = u + 1j * np.ldexp(X[:, j + 1], -int(e[j]))
    return u


# --------------------------------------------------------------------------
# closed forms and special cases
# --------------------------------------------------------------------------

def test_upper_triangular_2x2_closed_form():
    rng = np.random.default_rng(121)
    for _ in range(50):
        s11, s22, s12 = rng.uniform(-2, 2, 3)
        t11, t22 = rng.uniform(0.5, 2, 2)
        t12 = rng.standard_normal()
        S = np.array([[s11, s12], [0, s22]])
        T = np.array([[t11, t12], [0, t22]])
        X, e, ar, ai, be = oracle.generalized_left(S, T)
        # lambda_1 = s11 / t11: u = (1, -(s12 - lambda t12) / (s22 - lambda t22))
        lam = s11 / t11
        assert abs(ar[0] / be[0] - lam) <= 8 * U * abs(lam) + 1e-300
        ref = np.array([1.0, -(s12 - lam * t12) / (s22 - lam * t22)])
        got = np.ldexp(X[:, 0], -int(e[0]))
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max()), (got, ref)
        # lambda_2 = s22 / t22: nothing above row 1 -> u = (0, 1)
        assert X[0, 1] == 0.0 and X[1, 1] == 1.0 and e[1] == 0
        assert abs(ar[1] / be[1] - s22 / t22) <= 8 * U * abs(s22 / t22) + 1e-300
        for j in range(2):
            mx = max(abs(ar[j]), abs(ai[j]), be[j])
            assert 1.0 <= mx < 2.0


def test_identity_T_reduces_to_standard_left():
    S, blocks = workloads.config0_schur(128, seed=131)
    Xg, eg, ar, ai, be = oracle.generalized_left(S, np.eye(128))
    Xs, es, lr, li = oracle.left(S)
    assert Xg.shape == Xs.shape
    for j, pair in column_groups(li):
        assert abs(int(eg[j]) - int(es[j])) <= 1
        cols = [j, j + 1] if pair else [j]
        a = np.ldexp(Xg[:, cols], int(es[j]) - int(eg[j]))
        assert np.abs(a - Xs[:, cols]).max() <= 1e-12
        assert np.allclose(ar[j] / be[j], lr[j], rtol=1e-15, atol=1e-15)
        assert np.allclose(ai[j] / be[j], li[j], rtol=1e-15, atol=1e-15)


def test_unequal_diagonal_T_pair_closed_form():
    """The 2x2 block of S on rows 0-1 over diag(d1, d2): u^H (S_b - lambda
    T_b) = 0 on the block; row 2 from the forward step
    w2 (s22' - lambda t22') = -(w0 (s02 - lambda t02) + w1 (s12 - lambda t12))
    with w = conj(u)."""
    S = np.array([[0.3, 1.0, 0.5], [-1.2, 0.2, 1.5], [0.0, 0.0, 0.4]])
    T = np.array([[0.5, 0.0, -0.2], [0.0, 2.0, 0.7], [0.0, 0.0, 1.5]])
    X, e, ar, ai, be = oracle.generalized_left(S, T)
    res = generalized_left_residuals(S, T, X, ar, ai, be)
    assert res.max() <= 30
    lam = (ar[0] + 1j * ai[0]) / be[0]
    assert ai[0] > 0 and ai[1] == -ai[0]
    # det(S_b - lambda T_b) = 0
    M = S[:2, :2] - lam * T[:2, :2]
    assert abs(np.linalg.det(M)) <= 1e-14 * np.abs(S[:2, :2]).max() ** 2
    w = np.conj(_u(X, e, 0, True))
    assert abs(w[:2] @ M[:, 0]) + abs(w[:2] @ M[:, 1]) <= 1e-14 * np.abs(w).max() * 4
    w2 = -(w[0] * (S[0, 2] - lam * T[0, 2]) + w[1] * (S[1, 2] - lam * T[1, 2])) / \
        (S[2, 2] - lam * T[2, 2])
    assert abs(w[2] - w2) <= 1e-14 * np.abs(w).max()


# --------------------------------------------------------------------------
# library special case, invariants, biorthogonality
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def pencil_left():
    S, T, blocks = workloads.generalized_pair(200, seed=141)
    X, e, ar, ai, be = oracle.generalized_left(S, T)
    return S, T, blocks, X, e, ar, ai, be


def test_structure_residual_and_normalisation(pencil_left):
    S, T, blocks, X, e, ar, ai, be = pencil_left
    col = 0
    for p, sz in blocks:
        for k in range(sz):
            assert np.all(X[:p, col + k] == 0.0)
        col += sz
    nr = canonical_norms(X, ai)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    assert generalized_left_residuals(S, T, X, ar, ai, be).max() <= 10 * S.shape[0]
    # near-infinite eigenvalues of the workload are handled: beta tiny
    assert (be < 1e-10).sum() >= 3
    mx = np.maximum(np.maximum(np.abs(ar), np.abs(ai)), be)
    assert mx.min() >= 1.0 and mx.max() < 2.0


def test_lapack_left_directions():
    """scipy.linalg.eig(S, T, left=True) returns LAPACK's left generalized
    eigenvectors (vl^H S = lambda vl^H T); on a well-conditioned pencil the
    directions agree."""
    n = 120
    S, blocks = workloads.config0_schur(n, seed=151)
    S[np.triu_indices(n, 1)] /= np.sqrt(n)
    rng = np.random.default_rng(152)
    T = np.triu(rng.standard_normal((n, n)) / np.sqrt(n), 1)
    d = rng.uniform(0.5, 2.0, n)
    for p, sz in blocks:
        if sz == 2:            # a standardized pair keeps complex eigenvalues
            T[p, p + 1] = 0.0  # over a scalar diagonal block of T
            d[p + 1] = d[p]
    T[np.arange(n), np.arange(n)] = d
    X, e, ar, ai, be = oracle.generalized_left(S, T)
    w, VL = sl.eig(S, T, left=True, right=False)
    worst = 0.0
    for j, pair in column_groups(ai):
        u = _u(X, e, j, pair)
        lam = (ar[j] + 1j * ai[j]) / be[j]
        k = np.argmin(np.abs(w - lam))
        assert abs(w[k] - lam) <= 1e-10 * max(1.0, abs(lam))
        v = VL[:, k]
        worst = max(worst, 1 - abs(np.vdot(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v)))
    assert worst <= 1e-12, worst


def test_biorthogonality_with_right_eigenvectors():
    """u_i^H T y_j = 0 and u_i^H S y_j = 0 whenever the eigenvalues differ
    (y_j from the right generalized oracle), on a well-separated pencil."""
    n = 120
    S, T, blocks = workloads.generalized_pair(n, seed=161)
    S = np.array(S)
    S[np.triu_indices(n, 1)] /= np.sqrt(n)
    T = np.array(T)
    T[np.triu_indices(n, 1)] /= np.sqrt(n)
    Xl, el, ar, ai, be = oracle.generalized_left(S, T)
    Xr, er, br, bi, bb = oracle.generalized(S, T)
    groups = list(column_groups(ai))
    U_ = [_u(Xl, el, j, p) for j, p in groups]
    Y_ = [_u(Xr, er, j, p) for j, p in groups]
    worst = 0.0
    for a, u in enumerate(U_):
        un = u / np.linalg.norm(u)
        for b, y in enumerate(Y_):
            if a == b:
                continue
            yn = y / np.linalg.norm(y)
            for v in (yn, yn.conj()):
                worst = max(worst, abs(np.vdot(un, T @ v)), abs(np.vdot(un, S @ v)))
    scale = max(np.abs(S).sum(axis=0).max(), np.abs(T).sum(axis=0).max())
    assert worst <= 1e-10 * scale, worst


# --------------------------------------------------------------------------
# arbitrary precision
# --------------------------------------------------------------------------

def _mp_compare(S, T, blocks, X, e, tol):
    col = 0
    worst = 0.0
    for p, sz in blocks:
        u = mp_gen_left_eigvec(S, T, p, sz)
        xr, xi, emp = mp_canonical(u, sz == 2)
        de = int(e[col]) - emp
        assert abs(de) <= 1, (p, e[col], emp)
        err = np.abs(np.ldexp(X[:, col], -de) - xr)
        den = np.max(np.abs(xr))
        if sz == 2:
            err = err + np.abs(np.ldexp(X[:, col + 1], -de) - xi)
            den = np.max(np.abs(xr) + np.abs(xi))
        worst = max(worst, float(err.max() / den))
        col += sz
    assert worst <= tol, worst


def test_mpmath_generalized_left_small():
    S, T, blocks = workloads.generalized_pair(40, seed=171)
    X, e, ar, ai, be = oracle.generalized_left(S, T)
    _mp_compare(S, T, blocks, X, e, 1e-11)


def test_mpmath_generalized_left_overflow_witness():
    """Two clusters of 24 eigenvalues 1e-9 apart, upper parts N(0,1)*1e3: the
    left vectors grow past the double range along the forward direction; the
    unscaled forward substitution overflows, the oracle stays finite and
    agrees with the 256-bit reference to the clusters' conditioning."""
    rng = np.random.default_rng(176)
    n = 48
    S = np.triu(rng.standard_normal((n, n)) * 1e3, 1)
    T = np.triu(rng.standard_normal((n, n)), 1)
    d = rng.uniform(0.5, 2.0, n)
    lam = np.concatenate([-0.5 + (rng.permutation(24) - 12) * 1e-9,
                          0.5 + (rng.permutation(24) - 12) * 1e-9])
    S[np.arange(n), np.arange(n)] = lam * d
    T[np.arange(n), np.arange(n)] = d
    X, e, ar, ai, be = oracle.generalized_left(S, T)
    assert np.isfinite(X).all()
    assert e.min() < -1024                 # |u| beyond the largest double
    with np.errstate(all="ignore"):
        l0 = S[0, 0] / T[0, 0]
        w = np.zeros(n)
        w[0] = 1.0
        for i in range(1, n):
            w[i] = -(w[:i] @ (S[:i, i] - l0 * T[:i, i])) / (S[i, i] - l0 * T[i, i])
    assert not np.isfinite(w).all()
    _mp_compare(S, T, [(i, 1) for i in range(n)], X, e, 1e-4)


# --------------------------------------------------------------------------
# metamorphic relations
# --------------------------------------------------------------------------

def test_flip_relation_with_right_oracle(pencil_left):
    """u = conj(J y') with y' the right eigenvectors of the flipped pencil:
    the left oracle against the right oracle (other direction and summation
    order: equal to rounding; (alpha, beta) bit-identical)."""
    S, T, blocks, X, e, ar, ai, be = pencil_left
    Sf, Tf = flip_pencil(S, T)
    Xf, ef, arf, aif, bef = oracle.generalized(Sf, Tf)
    m = X.shape[1]
    perm, sign = np.zeros(m, int), np.ones(m)
    col = 0
    for p, sz in blocks:
        cf = m - col - sz
        for k in range(sz):
            perm[col + k] = cf + k
        if sz == 2:
            sign[col + 1] = -1.0
        col += sz
    assert np.array_equal(arf[perm], ar) and np.array_equal(aif[perm], ai)
    assert np.array_equal(bef[perm], be)
    Xr = Xf[::-1, perm] * sign[None, :]
    de, rel = compare_canonical(X, e, Xr, ef[perm], ai)
    assert de <= 1 and rel <= 1e-10, (de, rel)


@pytest.mark.parametrize("k", [-200, 150])
def test_common_power_of_two(pencil_left, k):
    """(2^k S, 2^k T) has the same normalised (alpha, beta) and the same
    vectors, bit for bit."""
    S, T, blocks, X, e, ar, ai, be = pencil_left
    X2, e2, ar2, ai2, be2 = oracle.generalized_left(np.ldexp(S, k), np.ldexp(T, k))
    assert np.array_equal(X2, X) and np.array_equal(e2, e)
    assert np.array_equal(ar2, ar) and np.array_equal(ai2, ai) and np.array_equal(be2, be)


def test_selection_threads_and_backtransform(pencil_left):
    S, T, blocks, X, e, ar, ai, be = pencil_left
    n = S.shape[0]
    sel = workloads.random_eigen_selection(n, blocks, 0.35, seed=181)
    Xs, es, *_ = oracle.generalized_left(S, T, select=sel)
    cols, col = [], 0
    for p, sz in blocks:
        if sel[p] or (sz == 2 and sel[p + 1]):
            cols.extend(range(col, col + sz))
        col += sz
    assert np.array_equal(Xs, X[:, cols]) and np.array_equal(es, e[cols])
    X1, e1, *_ = oracle.generalized_left(S, T, threads=1)
    assert np.array_equal(X1, X) and np.array_equal(e1, e)
    Z = workloads.householder_orthogonal(n, seed=182)
    Xz, ez, *_ = oracle.generalized_left(S, T, Z=Z)
    for j, pair in column_groups(ai):
        c = [j, j + 1] if pair else [j]
        ref = Z @ X[:, c]
        got = np.ldexp(Xz[:, c], int(e[j]) - int(ez[j]))
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_generalized_left_errors():
    S, T, blocks = workloads.generalized_pair(30, seed=191)
    p = next(q for q, sz in blocks if sz == 2)
    bad = np.array(T, copy=True)
    bad[p, p + 1] = 0.5                    # T not diagonal on a 2x2 block
    with pytest.raises(oracle.OracleError) as ei:
        oracle.generalized_left(S, bad)
    assert ei.value.status == oracle.ENOTSCHUR
    bad = np.array(S, copy=True)
    bad[3, 20] = np.inf
    with pytest.raises(oracle.OracleError) as ei:
        oracle.generalized_left(bad, T)
    assert ei.value.status == oracle.ENONFINITE
