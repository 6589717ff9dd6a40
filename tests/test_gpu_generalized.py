"""Generalized eigenvectors of a pencil (S, T) (evec_generalized) against the
CPU oracle: (alpha, beta) bit-identical, exponents +-1, columns within 1e-10
normwise relative, normalised residual
||beta S y - alpha T y||_1 / ((|beta| ||S||_1 + |alpha| ||T||_1) ||y||_1 u)
<= 10 n (in Schur coordinates y = Z^T x when Z is given)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads
from evec_checks import canonical_norms, compare_canonical, generalized_residuals

pytestmark = pytest.mark.gpu


def _dev(A):
    return None if A is None else torch.from_numpy(np.asfortranarray(A)).cuda()


def _run(S, T, Z=None, select=None, tile=0, mode="fp64"):
    X, e, ar, ai, be = ev.generalized(_dev(S), _dev(T), _dev(Z), select=select, tile=tile,
                                      check=True, mode=mode)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in (X, e, ar, ai, be))


def _parity(S, T, Z, out, select=None, rel_tol=1e-10):
    X, e, ar, ai, be = out
    Xo, eo, aro, aio, beo = oracle.generalized(S, T, Z, select=select)
    assert X.shape == Xo.shape
    np.testing.assert_array_equal(ar, aro)
    np.testing.assert_array_equal(ai, aio)
    np.testing.assert_array_equal(be, beo)
    assert np.isfinite(X).all()
    nr = canonical_norms(X, ai)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    de, rel = compare_canonical(Xo, eo, X, e, aio)
    assert de <= 1, de
    assert rel <= rel_tol, rel
    Y = X if Z is None else Z.T @ X
    r = generalized_residuals(S, T, Y, ar, ai, be)
    assert r.max() <= 10 * S.shape[0], r.max()
    return rel


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("tile", [16, 32, 64])
def test_generalized_tiles(tile, mode):
    n = 413
    S, T, blocks = workloads.generalized_pair(n, seed=tile + 7)
    _parity(S, T, None, _run(S, T, tile=tile, mode=mode))


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_generalized_with_z_and_selection(mode):
    n = 600
    S, T, blocks = workloads.generalized_pair(n, seed=31)
    Z = workloads.householder_orthogonal(n, seed=32)
    sel = workloads.random_eigen_selection(n, blocks, 0.35, seed=33)
    _parity(S, T, Z, _run(S, T, Z, select=sel, tile=64, mode=mode), select=sel)


def test_generalized_unstandardized_pairs():
    # a 2x2 block of S with unequal diagonal entries (still complex
    # eigenvalues against T's diagonal block)
    n = 200
    S, T, blocks = workloads.generalized_pair(n, seed=41)
    pairs = [p for p, sz in blocks if sz == 2]
    for p in pairs[:5]:
        S[p, p] += 0.05
        S[p + 1, p + 1] -= 0.05
    _parity(S, T, None, _run(S, T, tile=32))


def test_generalized_errors():
    n = 120
    S, T, blocks = workloads.generalized_pair(n, seed=51)
    p = next(q for q, sz in blocks if sz == 2)
    bad = T.copy()
    bad[p, p + 1] = 0.25                   # T's block under an S pair not diagonal
    with pytest.raises(ev.EvecError) as ei:
        _run(S, bad, tile=32)
    assert ei.value.status == ev.EVEC_ENOTSCHUR
    bad = T.copy()
    bad[p + 1, p + 1] = -1.0               # not positive
    with pytest.raises(ev.EvecError) as ei:
        _run(S, bad, tile=32)
    assert ei.value.status == ev.EVEC_ENOTSCHUR
    bad = T.copy()
    bad[7, 90] = np.inf                    # upper part of T
    with pytest.raises(ev.EvecError) as ei:
        _run(S, bad, tile=32)
    assert ei.value.status == ev.EVEC_ENONFINITE and ei.value.bad == 7 + 90 * n
    bad = T.copy()
    bad[90, 7] = np.nan                    # strictly lower part of T: never read
    _parity(S, T, None, _run(S, bad, tile=32))
    with pytest.raises(ev.EvecError) as ei:   # tiles above 512 rows are refused
        _run(S, T, tile=513)
    assert ei.value.status == ev.EVEC_EINVAL


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_generalized_config4_full_size_sampled(mode):
    # n = 8192 pencil with Z (every 50th diagonal entry of T = 1e-12: nearly
    # infinite eigenvalues); 256 sampled eigenvalues against the oracle
    n = 8192
    S, T, blocks = workloads.generalized_pair(n, seed=workloads.SEED_BASE + 4)
    Z = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 104)
    X, e, ar, ai, be = _run(S, T, Z, tile=0, mode=mode)
    assert np.isfinite(X).all()
    rng = np.random.default_rng(6)
    chosen = rng.choice(len(blocks), size=256, replace=False)
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
            rel_tol=1e-9)


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("n,tile", [(700, 128), (900, 256), (1100, 512), (600, 200)])
def test_generalized_big_tiles(n, tile, mode):
    # pencil tiles above 64 rows: S's and T's sub-blocks of at most 64 rows
    # inside each tile, the rows above a sub-block updated in one protected
    # pass with both matrices; with Z and without
    S, T, blocks = workloads.generalized_pair(n, seed=n + tile)
    Z = workloads.householder_orthogonal(n, seed=n + tile + 1)
    _parity(S, T, Z, _run(S, T, Z, tile=tile, mode=mode))
    _parity(S, T, None, _run(S, T, tile=tile, mode=mode))
