"""Left eigenvectors of a pencil (S, T) (evec_generalized_left) against the
CPU oracle: (alpha, beta) bit-identical, exponents +-1, columns within 1e-10
normwise relative (1e-9 at n = 8192), normalised residual
||u^H (beta S - alpha T)||_1 / ((|beta| ||S||_inf + |alpha| ||T||_inf)
||u||_1 u) <= 10 n (in Schur coordinates u = Z^T x when Z is given), zeros
above each block."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads
from evec_checks import canonical_norms, compare_canonical, generalized_left_residuals

pytestmark = pytest.mark.gpu


def _dev(A):
    return None if A is None else torch.from_numpy(np.asfortranarray(A)).cuda()


def _run(S, T, Z=None, select=None, tile=0, mode="fp64"):
    X, e, ar, ai, be = ev.generalized_left(_dev(S), _dev(T), _dev(Z), select=select, tile=tile,
                                           check=True, mode=mode)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in (X, e, ar, ai, be))


def _parity(S, T, Z, out, select=None, rel_tol=1e-10, blocks=None, cluster_beta=0.0):
    """cluster_beta > 0: columns of eigenvalues with beta below it (the
    nearly infinite ones, a cluster in the chordal metric: their (alpha,
    beta) differ by about beta) are compared by exponent (+-1) and residual
    only.  A left vector of such an eigenvalue passes through every other
    nearly singular pivot beta S_jj - alpha T_jj below its block, each of
    which multiplies the rounding error by about 1 / beta, so its direction
    is not determined to working precision (both sides' residuals stay
    small)."""
    X, e, ar, ai, be = out
    Xo, eo, aro, aio, beo = oracle.generalized_left(S, T, Z, select=select)
    assert X.shape == Xo.shape
    np.testing.assert_array_equal(ar, aro)
    np.testing.assert_array_equal(ai, aio)
    np.testing.assert_array_equal(be, beo)
    assert np.isfinite(X).all()
    nr = canonical_norms(X, ai)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    keep = np.asarray(beo) >= cluster_beta
    assert np.abs(np.asarray(eo)[~keep] - np.asarray(e)[~keep]).max(initial=0) <= 1
    de, rel = compare_canonical(Xo[:, keep], eo[keep], X[:, keep], e[keep], aio[keep])
    assert de <= 1, de
    assert rel <= rel_tol, rel
    U_ = X if Z is None else Z.T @ X
    r = generalized_left_residuals(S, T, U_, ar, ai, be)
    assert r.max() <= 10 * S.shape[0], r.max()
    if Z is None and blocks is not None and select is None:
        col = 0
        for p, sz in blocks:
            assert np.all(X[:p, col:col + sz] == 0.0)
            col += sz
    return rel


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("tile", [16, 32, 64, 256])
def test_generalized_left_tiles(tile, mode):
    n = 413
    S, T, blocks = workloads.generalized_pair(n, seed=tile + 207)
    _parity(S, T, None, _run(S, T, tile=tile, mode=mode), blocks=blocks)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_generalized_left_with_z_and_selection(mode):
    n = 600
    S, T, blocks = workloads.generalized_pair(n, seed=231)
    Z = workloads.householder_orthogonal(n, seed=232)
    sel = workloads.random_eigen_selection(n, blocks, 0.35, seed=233)
    _parity(S, T, Z, _run(S, T, Z, select=sel, tile=64, mode=mode), select=sel)
    _parity(S, T, Z, _run(S, T, Z, tile=128, mode=mode))


def test_generalized_left_unstandardized_pairs_and_unequal_diagonal():
    # 2x2 blocks of S with unequal diagonal entries over diag(d1, d2) with
    # d1 != d2: the left convention takes the pair against d2
    n = 200
    S, T, blocks = workloads.generalized_pair(n, seed=241)
    pairs = [p for p, sz in blocks if sz == 2]
    for p in pairs[:5]:
        S[p, p] += 0.05
        S[p + 1, p + 1] -= 0.05
        T[p + 1, p + 1] *= 1.5
    _parity(S, T, None, _run(S, T, tile=32), blocks=blocks)


def test_generalized_left_identity_T_matches_standard_left():
    n = 300
    S, blocks = workloads.config0_schur(n, seed=245)
    X, e, ar, ai, be = _run(S, np.eye(n), tile=64)
    Xs, es, lr, li = (t.cpu().numpy() for t in ev.left(_dev(S), tile=64, check=True))
    assert np.allclose(ar / be, lr, rtol=1e-15, atol=1e-15)
    assert np.allclose(ai / be, li, rtol=1e-15, atol=1e-15)
    de, rel = compare_canonical(Xs, es, X, e, li)
    assert de <= 1 and rel <= 1e-12, (de, rel)


def test_generalized_left_edge_sizes():
    for n in (1, 2, 3, 17, 65):
        S, T, blocks = workloads.generalized_pair(max(n, 2), seed=250 + n)
        S, T = S[:n, :n].copy(), T[:n, :n].copy()
        if n >= 2 and S[n - 1, n - 2] != 0.0:        # a pair cut in half: drop it
            S[n - 1, n - 2] = 0.0
        _parity(S, T, None, _run(S, T, tile=16))


def test_generalized_left_errors():
    n = 120
    S, T, blocks = workloads.generalized_pair(n, seed=251)
    p = next(q for q, sz in blocks if sz == 2)
    bad = T.copy()
    bad[p, p + 1] = 0.25                   # T's block under an S pair not diagonal
    with pytest.raises(ev.EvecError) as ei:
        _run(S, bad, tile=32)
    assert ei.value.status == ev.EVEC_ENOTSCHUR
    bad = T.copy()
    bad[7, 90] = np.inf                    # upper part of T, in T's coordinates
    with pytest.raises(ev.EvecError) as ei:
        _run(S, bad, tile=32)
    assert ei.value.status == ev.EVEC_ENONFINITE and ei.value.bad == 7 + 90 * n
    bad = S.copy()
    bad[5, 80] = np.nan                    # upper part of S
    with pytest.raises(ev.EvecError) as ei:
        _run(bad, T, tile=32)
    assert ei.value.status == ev.EVEC_ENONFINITE and ei.value.bad == 5 + 80 * n
    bad = T.copy()
    bad[90, 7] = np.nan                    # strictly lower part of T: never read
    bad[p + 1, p] = np.nan                 # T's subdiagonal under a pair: never read
    _parity(S, T, None, _run(S, bad, tile=32))
    with pytest.raises(ev.EvecError) as ei:   # tiles above 512 rows are refused
        _run(S, T, tile=513)
    assert ei.value.status == ev.EVEC_EINVAL


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_generalized_left_full_size_sampled(mode):
    # n = 8192 pencil with Z (nearly infinite eigenvalues every 50th row);
    # 192 sampled eigenvalues against the oracle (the nearly infinite ones
    # by exponent and residual)
    n = 8192
    S, T, blocks = workloads.generalized_pair(n, seed=workloads.SEED_BASE + 4)
    Z = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 104)
    X, e, ar, ai, be = _run(S, T, Z, tile=0, mode=mode)
    assert np.isfinite(X).all()
    rng = np.random.default_rng(16)
    chosen = rng.choice(len(blocks), size=192, replace=False)
    sel = np.zeros(n, np.uint8)
    for b in chosen:
        p, sz = blocks[b]
        sel[p:p + sz] = 1
    cols, col = [], 0
    for p, sz in blocks:
        if sel[p]:
            cols.extend(range(col, col + sz))
        col += sz
    _parity(S, T, Z, (X[:, cols], e[cols], ar[cols], ai[cols], be[cols]), select=sel,
            rel_tol=1e-9, cluster_beta=1e-10)
    assert (be[cols] < 1e-10).sum() >= 2      # the sample holds some of the cluster
