"""Left eigenvectors on the GPU (evec_standard_left) against the CPU oracle's
robust forward substitution: eigenvalues bit-identical, exponents +-1,
columns within 1e-10 normwise relative, left residual
||u^H T - lambda u^H||_1 / (||T||_inf ||u||_1 u) <= 10 n, exact zeros above
each block; every tile path in FP64 and split mode, with Q and a
selection, the residual-correction sweep, edge sizes and errors."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads
from evec_checks import canonical_norms, compare_canonical, left_residuals

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


def _dev(A):
    return None if A is None else torch.from_numpy(np.asfortranarray(A)).cuda()


def _gpu(T, Q=None, select=None, tile=0, mode="fp64", slices=0, refine=False):
    X, e, lr, li = ev.left(_dev(T), _dev(Q), select=select, tile=tile, check=True, mode=mode,
                           slices=slices, refine=refine)
    torch.cuda.synchronize()
    return X.cpu().numpy(), e.cpu().numpy(), lr.cpu().numpy(), li.cpu().numpy()


def _parity(T, Q, out, select=None, rel_tol=REL_TOL):
    X, e, lr, li = out
    Xo, eo, lro, lio = oracle.left(T, Q=Q, select=select)
    assert X.shape == Xo.shape
    np.testing.assert_array_equal(lr, lro)
    np.testing.assert_array_equal(li, lio)
    assert np.isfinite(X).all()
    nr = canonical_norms(X, li)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    de, rel = compare_canonical(Xo, eo, X, e, lio)
    assert de <= 1, de
    assert rel <= rel_tol, rel
    A = T if Q is None else Q @ T @ Q.T
    res = left_residuals(A, X, lr, li)
    assert res.max() <= 10 * T.shape[0], res.max()
    return rel


def _zeros_above_blocks(blocks, X, select=None):
    col = 0
    for p, sz in blocks:
        if select is not None and not (select[p] or (sz == 2 and select[p + 1])):
            continue
        for k in range(sz):
            assert np.all(X[:p, col + k] == 0.0)
        col += sz


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("tile", [16, 32, 64, 128])
def test_left_tiles_and_modes(tile, mode):
    n = 613
    T, blocks = workloads.config0_schur(n, seed=900 + tile)
    out = _gpu(T, tile=tile, mode=mode)
    _zeros_above_blocks(blocks, out[0])
    _parity(T, None, out)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_left_with_q_and_selection(mode):
    n = 700
    T, blocks = workloads.config0_schur(n, seed=41)
    Q = workloads.householder_orthogonal(n, seed=42)
    sel = workloads.random_eigen_selection(n, blocks, 0.35, seed=43)
    _parity(T, Q, _gpu(T, Q, select=sel, tile=64, mode=mode), select=sel)
    # the selected columns equal the same columns of the full result
    X, e, lr, li = _gpu(T, Q, tile=64, mode=mode)
    Xs, es, _, _ = _gpu(T, Q, select=sel, tile=64, mode=mode)
    cols, col = [], 0
    for p, sz in blocks:
        if sel[p] or (sz == 2 and sel[p + 1]):
            cols.extend(range(col, col + sz))
        col += sz
    if mode == "fp64":
        np.testing.assert_array_equal(Xs, X[:, cols])
        np.testing.assert_array_equal(es, e[cols])


def test_left_refine_low_slices():
    # split at 5 slices misses the bar without the sweep, meets it with it
    n = 500
    T, blocks = workloads.config0_schur(n, seed=95)
    X, e, lr, li = _gpu(T, tile=64, mode="split", slices=5)
    Xo, eo, _, lio = oracle.left(T)
    _, rel_plain = compare_canonical(Xo, eo, X, e, lio)
    assert rel_plain > 10 * REL_TOL, rel_plain
    _parity(T, None, _gpu(T, tile=64, mode="split", slices=5, refine=True))


def test_left_adversarial_clusters():
    # clustered eigenvalues with growth past the double range: finite, exponents
    # +-1, within the clustered-input bound
    n = 512
    T, blocks = workloads.adversarial_schur(n, seed=61)
    out = _gpu(T, tile=64)
    assert out[1].min() < -1100
    _parity(T, None, out, rel_tol=1e-3)


def test_left_edge_sizes():
    for n in (1, 2, 3, 65):
        T, blocks = workloads.config0_schur(n, seed=n + 70)
        out = _gpu(T, tile=64)
        _zeros_above_blocks(blocks, out[0])
        _parity(T, None, out)


def test_left_errors():
    n = 120
    T, blocks = workloads.config0_schur(n, seed=51)
    bad = T.copy()
    bad[7, 90] = np.nan                     # strictly above the superdiagonal
    with pytest.raises(ev.EvecError) as ei:
        _gpu(bad, tile=32)
    assert ei.value.status == ev.EVEC_ENONFINITE and ei.value.bad == 7 + 90 * n
    bad = T.copy()
    bad[3, 50] = 2.0 ** 1001
    with pytest.raises(ev.EvecError) as ei:
        _gpu(bad, tile=32)
    assert ei.value.status == ev.EVEC_EINVAL and ei.value.bad == 3 + 50 * n
    p = next(q for q, sz in blocks if sz == 2)
    bad = T.copy()
    bad[p + 1, p + 1] += 0.25               # pair not standardized
    with pytest.raises(ev.EvecError) as ei:
        _gpu(bad, tile=32)
    assert ei.value.status == ev.EVEC_ENOTSCHUR
    bad = T.copy()
    bad[100, 5] = np.nan                    # strictly lower part: never read
    _parity(T, None, _gpu(bad, tile=32))


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_left_full_size_sampled(mode):
    # the benchmark's workload shape: n = 4096 with Q, tile 64; 16 sampled
    # eigenvalues against the oracle
    n = 4096
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE + 1)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 101)
    X, e, lr, li = _gpu(T, Q, tile=0, mode=mode)
    assert np.isfinite(X).all()
    rng = np.random.default_rng(8)
    chosen = rng.choice(len(blocks), size=16, replace=False)
    sel = np.zeros(n, np.uint8)
    for b in chosen:
        p, sz = blocks[b]
        sel[p:p + sz] = 1
    cols, col = [], 0
    for p, sz in blocks:
        if sel[p]:
            cols.extend(range(col, col + sz))
        col += sz
    _parity(T, Q, (X[:, cols], e[cols], lr[cols], li[cols]), select=sel, rel_tol=1e-9)
