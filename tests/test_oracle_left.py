"""Pins for the oracle's left eigenvectors: u^H S = lambda u^H, the
eigenvector problem of Sec. 2 for S^T, by robust forward substitution
(Sec. 3.3's protection applied in the other direction).  Closed forms,
LAPACK's left eigenvectors, biorthogonality with the right eigenvectors,
arbitrary-precision brute force (the right-eigenvector reference on the
flipped matrix J S^T J), an overflow witness and metamorphic relations.

Output convention: X[:, j] * 2**(-e[j]) is u, zero above its block; a 2x2
block gives (Re u, Im u) for lambda = a + i w, w > 0, normalised on the
block to (-i w/b, 1) if |b| >= |c|, else (-i, -w/c) (the row-reversed,
conjugated form of the right-eigenvector convention)."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads
from evec_checks import (U, canonical_norms, column_groups, compare_canonical,
                         left_residuals, mp_canonical, mp_left_eigvec)


def _u(X, e, j, pair):
    u = np.ldexp(X[:, j], -int(e[j])).astype(complex)
    if pair:
        u = u + 1j * np.ldexp(X[:, j + 1], -int(e[j]))
    return u


def _flip(T):
    return np.asfortranarray(T.T[::-1, ::-1])


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def test_one_by_one_and_upper_triangular_2x2():
    X, e, lr, li = oracle.left(np.array([[-2.5]]))
    assert X[0, 0] == 1.0 and e[0] == 0 and lr[0] == -2.5
    rng = np.random.default_rng(3)
    for _ in range(20):
        t11, t22 = rng.uniform(-1, 1, 2)
        t12 = rng.standard_normal()
        T = np.array([[t11, t12], [0.0, t22]])
        X, e, lr, li = oracle.left(T)
        # lambda_1 = t11: u^T (T - t11 I) = 0 gives u = (1, t12 / (t11 - t22))
        u1 = np.array([1.0, t12 / (t11 - t22)])
        got = np.ldexp(X[:, 0], -int(e[0]))
        assert np.allclose(got, u1, rtol=8 * U, atol=0), (got, u1)
        # lambda_2 = t22: nothing above row 1 -> u = (0, 1)
        assert X[0, 1] == 0.0 and X[1, 1] == 1.0 and e[1] == 0


@pytest.mark.parametrize("b,c", [(2.0, -0.5), (-0.75, 3.0), (1.0, -1.0)])
def test_standardized_pair_closed_form(b, c):
    a = 0.3
    B = np.array([[a, b], [c, a]])
    X, e, lr, li = oracle.left(B)
    w = np.sqrt(abs(b)) * np.sqrt(abs(c))
    lam = a + 1j * w
    assert lr[0] == a and abs(li[0] - w) <= 2 * U * w and li[1] == -li[0]
    u = _u(X, e, 0, True)
    ref = np.array([-1j * w / b, 1.0]) if abs(b) >= abs(c) else np.array([-1j, -w / c])
    assert np.allclose(u, ref, rtol=0, atol=8 * U * np.abs(ref).max()), (u, ref)
    # and it is a left eigenvector: u^H B = lambda u^H
    r = u.conj() @ B - lam * u.conj()
    assert np.abs(r).max() <= 8 * U * np.abs(B).max()
    nr = canonical_norms(X, li)
    assert 1.0 <= nr[0] < 2.0


def test_three_by_three_pair_on_top():
    # pair [[a, b], [c, a]] on rows 0-1, 1x1 mu on row 2.  Left vector of
    # the pair: w = conj(u) = (i w/b, 1, w3) with w3 (mu - lambda) =
    # -(w0 t02 + w1 t12); of mu (last row): u = (0, 0, 1).
    a, b, c, mu = 0.2, 1.5, -0.4, -0.7
    t02, t12 = 0.9, -1.3
    T = np.array([[a, b, t02], [c, a, t12], [0.0, 0.0, mu]])
    X, e, lr, li = oracle.left(T)
    w = np.sqrt(abs(b)) * np.sqrt(abs(c))
    lam = a + 1j * w
    w0, w1 = 1j * w / b, 1.0
    w2 = -(w0 * t02 + w1 * t12) / (mu - lam)
    ref = np.conj(np.array([w0, w1, w2]))
    u = _u(X, e, 0, True)
    assert np.allclose(u, ref, rtol=0, atol=16 * U * np.abs(ref).max()), (u, ref)
    assert X[0, 2] == 0.0 and X[1, 2] == 0.0 and X[2, 2] == 1.0 and e[2] == 0


def test_three_by_three_real_on_top_cramer():
    # 1x1 mu on row 0, pair below: u = (1, v1, v2) with
    # (B - mu I)^T (v1, v2) = -(t01, t02), a real 2x2 solve (Cramer)
    mu, t01, t02 = 0.45, -0.8, 1.1
    a, b, c = -0.3, 0.7, -1.9
    T = np.array([[mu, t01, t02], [0.0, a, b], [0.0, c, a]])
    X, e, lr, li = oracle.left(T)
    M = np.array([[a - mu, c], [b, a - mu]])          # (B - mu I)^T
    rhs = -np.array([t01, t02])
    det = M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]
    v1 = (rhs[0] * M[1, 1] - M[0, 1] * rhs[1]) / det
    v2 = (M[0, 0] * rhs[1] - M[1, 0] * rhs[0]) / det
    ref = np.array([1.0, v1, v2])
    got = np.ldexp(X[:, 0], -int(e[0]))
    assert np.allclose(got, ref, rtol=0, atol=16 * U * np.abs(ref).max()), (got, ref)


# --------------------------------------------------------------------------
# library special case, invariants, biorthogonality
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg0_left():
    T, blocks = workloads.config0_schur(256, seed=workloads.SEED_BASE)
    X, e, lr, li = oracle.left(T)
    return T, blocks, X, e, lr, li


def test_lapack_left_directions(cfg0_left):
    """scipy.linalg.eig(left=True) returns LAPACK's left eigenvectors
    (vl^H T = lambda vl^H); on a well-conditioned input the directions agree."""
    T, blocks, X, e, lr, li = cfg0_left
    w, VL = sl.eig(T, left=True, right=False)
    worst = 0.0
    for j, pair in column_groups(li):
        u = _u(X, e, j, pair)
        k = np.argmin(np.abs(w - (lr[j] + 1j * li[j])))
        v = VL[:, k]
        worst = max(worst, 1 - abs(np.vdot(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v)))
    assert worst <= 1e-12, worst


def test_zero_above_block_canonical_and_residual(cfg0_left):
    T, blocks, X, e, lr, li = cfg0_left
    col = 0
    for p, sz in blocks:
        for k in range(sz):
            assert np.all(X[:p, col + k] == 0.0)
        col += sz
    nr = canonical_norms(X, li)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    assert left_residuals(T, X, lr, li).max() <= 10 * T.shape[0]


def test_biorthogonality_with_right_eigenvectors():
    """u_i^H y_j = 0 whenever lambda_i differs from lambda_j and from its
    conjugate (y_j from the right-eigenvector oracle); u_i^H y_i != 0."""
    n = 150
    T, blocks = workloads.config0_schur(n, seed=17)
    # well-separated spectrum: make the upper part smaller
    T[np.triu_indices(n, 1)] /= np.sqrt(n)
    Xl, el, lr, li = oracle.left(T)
    Xr, er, _, _ = oracle.standard(T)
    groups = list(column_groups(li))
    U_ = [_u(Xl, el, j, p) for j, p in groups]
    Y_ = [_u(Xr, er, j, p) for j, p in groups]
    lam = np.array([lr[j] + 1j * li[j] for j, _ in groups])
    worst = 0.0
    for a, u in enumerate(U_):
        un = u / np.linalg.norm(u)
        for b, y in enumerate(Y_):
            yn = y / np.linalg.norm(y)
            if a == b:
                assert abs(np.vdot(un, yn)) > 0.0
                continue
            for v in (yn, yn.conj()):
                worst = max(worst, abs(np.vdot(un, v)))
    gap = min(abs(lam[a] - lam[b]) for a in range(len(lam)) for b in range(a))
    assert worst <= 1e-11, (worst, gap)


# --------------------------------------------------------------------------
# arbitrary precision
# --------------------------------------------------------------------------

def _mp_compare_left(T, blocks, X, e, tol):
    col = 0
    worst = 0.0
    for p, sz in blocks:
        u, _ = mp_left_eigvec(T, p, sz)
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


def test_mpmath_left_config0_small():
    T, blocks = workloads.config0_schur(40, seed=321)
    X, e, lr, li = oracle.left(T)
    _mp_compare_left(T, blocks, X, e, 1e-12)


def test_mpmath_left_adversarial_overflow_witness():
    """Two clusters of 32 eigenvalues 1e-9 apart, upper part N(0,1)*1e3: the
    left vectors grow past the double range along the forward direction.
    The unscaled forward substitution overflows; the oracle stays finite
    and agrees with the 256-bit reference (to the cluster's conditioning)."""
    rng = np.random.default_rng(6)
    n = 64
    T = np.triu(rng.standard_normal((n, n)) * 1e3, 1)
    diag = np.concatenate([-0.5 + (rng.permutation(32) - 16) * 1e-9,
                           0.5 + (rng.permutation(32) - 16) * 1e-9])
    T[np.arange(n), np.arange(n)] = diag
    X, e, lr, li = oracle.left(T)
    assert np.isfinite(X).all()
    assert e.min() < -1100
    # unscaled forward substitution from the first row (lambda = T[0, 0])
    with np.errstate(all="ignore"):
        w = np.zeros(n)
        w[0] = 1.0
        for i in range(1, n):
            w[i] = -(w[:i] @ T[:i, i]) / (T[i, i] - T[0, 0])
    assert not np.isfinite(w).all()
    _mp_compare_left(T, [(i, 1) for i in range(n)], X, e, 1e-4)


# --------------------------------------------------------------------------
# metamorphic relations
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [-100, 100])
def test_left_power_of_two(cfg0_left, k):
    T, blocks, X, e, lr, li = cfg0_left
    X2, e2, lr2, li2 = oracle.left(np.ldexp(T, k))
    assert np.array_equal(X2, X) and np.array_equal(e2, e)
    assert np.array_equal(lr2, np.ldexp(lr, k)) and np.array_equal(li2, np.ldexp(li, k))


def test_left_selection_and_threads(cfg0_left):
    T, blocks, X, e, lr, li = cfg0_left
    sel = workloads.random_eigen_selection(256, blocks, 0.35, seed=19)
    Xs, es, _, _ = oracle.left(T, select=sel)
    cols, col = [], 0
    for p, sz in blocks:
        if sel[p] or (sz == 2 and sel[p + 1]):
            cols.extend(range(col, col + sz))
        col += sz
    assert np.array_equal(Xs, X[:, cols]) and np.array_equal(es, e[cols])
    X1, e1, _, _ = oracle.left(T, threads=1)
    assert np.array_equal(X1, X) and np.array_equal(e1, e)


def test_flip_relation_with_right_eigenvectors(cfg0_left):
    """u = conj(J y') with y' the right eigenvectors of J T^T J: the left
    oracle against the right oracle on the flipped matrix (different
    substitution direction and summation order: equal to rounding)."""
    T, blocks, X, e, lr, li = cfg0_left
    n = T.shape[0]
    Xf, ef, lrf, lif = oracle.standard(_flip(T))
    m = X.shape[1]
    # the flipped matrix lists the blocks in reverse order; a pair keeps its
    # (Re, Im) column order
    perm, sign = np.zeros(m, int), np.ones(m)
    col = 0
    for p, sz in blocks:
        cf = m - col - sz
        for k in range(sz):
            perm[col + k] = cf + k
        if sz == 2:
            sign[col + 1] = -1.0
        col += sz
    Xr = Xf[::-1, perm] * sign[None, :]
    assert np.array_equal(lrf[perm], lr) and np.array_equal(lif[perm], li)
    de, rel = compare_canonical(X, e, Xr, ef[perm], li)
    assert de <= 1 and rel <= 1e-12, (de, rel)


def test_left_backtransform():
    n = 120
    T, blocks = workloads.config0_schur(n, seed=23)
    Q = workloads.householder_orthogonal(n, seed=24)
    X, e, lr, li = oracle.left(T)
    Xq, eq, _, _ = oracle.left(T, Q=Q)
    for j, pair in column_groups(li):
        cols = [j, j + 1] if pair else [j]
        ref = Q @ X[:, cols]
        got = np.ldexp(Xq[:, cols], int(e[j]) - int(eq[j]))
        assert np.abs(got - ref).max() <= 64 * U * 16 * np.abs(ref).max()
    A = Q @ T @ Q.T
    assert left_residuals(A, Xq, lr, li).max() <= 10 * n


def test_left_errors():
    T, blocks = workloads.config0_schur(30, seed=29)
    p = next(q for q, sz in blocks if sz == 2)
    bad = T.copy()
    bad[p + 1, p + 1] += 0.1               # pair no longer standardized
    with pytest.raises(oracle.OracleError) as ei:
        oracle.left(bad)
    assert ei.value.status == oracle.ENOTSCHUR
    bad = T.copy()
    bad[3, 20] = np.inf
    with pytest.raises(oracle.OracleError) as ei:
        oracle.left(bad)
    assert ei.value.status == oracle.ENONFINITE and ei.value.bad == 3 + 20 * 30
