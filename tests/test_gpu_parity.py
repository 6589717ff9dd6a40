"""GPU path vs the CPU oracle, through the C ABI (via the thin binding).

Tolerances (the library's stated parity bar):
  * scale exponents agree within +-1 (both sides take floor(log2 |y|) of the
    same true vector; a value next to a power of two may round either way);
  * well-conditioned inputs: every column agrees normwise within 1e-10
    relative after bringing both to one exponent;
  * every input: normalised residual ||T x - lambda x||_1 / (||T||_1 ||x||_1 u)
    <= 10 n, all entries finite, canonical norm in [1, 2), exact zeros below
    the diagonal block (before back-transformation).
Clustered adversarial inputs (eigenvalues 1e-9 apart, upper part 1e3) have
eigenvectors whose forward error is of order |T| / gap * u; there the columns
are compared to a looser bound stated in the test.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads
from evec_checks import (canonical_norms, column_groups, compare_canonical,
                         standard_residuals)

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


def _gpu(T, Q=None, select=None, tile=0, mode="fp64", slices=0, refine=0):
    # split mode here is the plain split solve (no residual-correction sweep;
    # the sweep has its own tests)
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    dQ = None if Q is None else torch.from_numpy(np.asfortranarray(Q)).cuda()
    X, e, lr, li = ev.standard(dT, dQ, select=select, tile=tile, check=True, mode=mode,
                               slices=slices, refine=refine)
    torch.cuda.synchronize()
    return X.cpu().numpy(), e.cpu().numpy(), lr.cpu().numpy(), li.cpu().numpy()


def _check_structure(T, blocks, X, li, select=None):
    assert np.isfinite(X).all()
    nr = canonical_norms(X, li)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    col = 0
    for p, sz in blocks:
        if select is not None and not (select[p] or (sz == 2 and select[p + 1])):
            continue
        for k in range(sz):
            assert np.all(X[p + sz:, col + k] == 0.0)
        col += sz


def _parity(T, Q, X, e, lr, li, select=None, rel_tol=REL_TOL):
    Xo, eo, lro, lio = oracle.standard(T, Q=Q, select=select)
    assert X.shape == Xo.shape
    np.testing.assert_array_equal(lr, lro)
    np.testing.assert_array_equal(li, lio)
    de, rel = compare_canonical(Xo, eo, X, e, lio)
    assert de <= 1, de
    assert rel <= rel_tol, rel
    A = T if Q is None else Q @ T @ Q.T
    res = standard_residuals(A, X, lr, li)
    assert res.max() <= 10 * T.shape[0], res.max()
    return rel, res.max()


@pytest.mark.parametrize("tile", [16, 32, 64, 128])
def test_config0_all_tiles(tile):
    T, blocks = workloads.config0_schur(256)
    X, e, lr, li = _gpu(T, tile=tile)
    _check_structure(T, blocks, X, li)
    _parity(T, None, X, e, lr, li)


@pytest.mark.parametrize("n,tile", [(517, 64), (1000, 128), (333, 16)])
def test_ragged_with_backtransform(n, tile):
    T, blocks = workloads.config0_schur(n, seed=n)
    Q = workloads.householder_orthogonal(n, seed=n + 1)
    X, e, lr, li = _gpu(T, Q, tile=tile)
    nr = canonical_norms(X, li)
    assert np.isfinite(X).all() and nr.min() >= 1.0 and nr.max() < 2.0
    _parity(T, Q, X, e, lr, li)


def test_selection_subset():
    T, blocks = workloads.config0_schur(700, seed=5)
    sel = workloads.random_eigen_selection(700, blocks, 0.35, seed=6)
    X, e, lr, li = _gpu(T, select=sel, tile=64)
    _check_structure(T, blocks, X, li, select=sel)
    _parity(T, None, X, e, lr, li, select=sel)


def test_adversarial_overflow_case():
    n = 512
    T, blocks = workloads.adversarial_schur(n, seed=77)
    _, bad = oracle.naive_standard(T)
    assert bad > 0                        # unscaled substitution overflows
    X, e, lr, li = _gpu(T, tile=64)
    _check_structure(T, blocks, X, li)
    assert e.min() < -1074                # true vectors far outside the double range
    # forward error of a 1e-9-cluster eigenvector ~ |T| / gap * u ~ 1e-3
    _parity(T, None, X, e, lr, li, rel_tol=1e-3)


def test_edge_sizes():
    for S in (np.array([[0.5]]), np.array([[0.2, 1.0], [-0.5, 0.2]]),
              np.array([[1.0, 2.0, 3.0], [0.0, 0.5, 1.0], [0.0, -2.0, 0.5]])):
        X, e, lr, li = _gpu(S, tile=16)
        _parity(S, None, X, e, lr, li)
    T, blocks = workloads.config0_schur(40, seed=2)
    X, e, lr, li = _gpu(T, select=np.zeros(40, np.uint8))
    assert X.shape == (40, 0)
    X, e, lr, li = _gpu(np.zeros((0, 0)))
    assert X.shape == (0, 0)


def test_errors_are_reported():
    S = np.triu(np.ones((6, 6)))
    S[1, 0] = -1.0
    S[2, 1] = -1.0
    with pytest.raises(ev.EvecError) as ei:
        _gpu(S)
    assert ei.value.status == ev.EVEC_ENOTSCHUR
    T, _ = workloads.config0_schur(200, seed=9)
    T[3, 150] = np.inf
    with pytest.raises(ev.EvecError) as ei:
        _gpu(T, tile=32)
    assert ei.value.status == ev.EVEC_ENONFINITE and ei.value.bad == 3 + 150 * 200
    T[3, 150] = 2.0 ** 1005
    with pytest.raises(ev.EvecError) as ei:
        _gpu(T, tile=32)
    assert ei.value.status == ev.EVEC_EINVAL
    # the handle stays usable after a reported error
    T[3, 150] = 0.5
    X, e, lr, li = _gpu(T, tile=32)
    _parity(T, None, X, e, lr, li)


@pytest.mark.parametrize("n,mode,frac", [(300, "fp64", None), (701, "split", None),
                                         (1300, "split", 0.6)])
def test_host_entry_point_matches_device(n, mode, frac):
    # the host-buffer entry point copies Q beside the solve and, in split
    # mode, brings X back in column chunks as the back-transformation
    # finishes them (pairs can straddle a chunk): the result equals the
    # device entry point's bit for bit
    T, blocks = workloads.config0_schur(n, seed=12 + n)
    Q = workloads.householder_orthogonal(n, seed=13 + n)
    sel = None if frac is None else workloads.random_eigen_selection(n, blocks, frac, seed=n)
    X, e, lr, li = _gpu(T, Q, select=sel, tile=64, mode=mode)
    Xh, eh, lrh, lih = ev.standard_host(T, Q, select=sel, tile=64, mode=mode, refine=0)
    np.testing.assert_array_equal(X, Xh)
    np.testing.assert_array_equal(e, eh)
    np.testing.assert_array_equal(lr, lrh)
    np.testing.assert_array_equal(li, lih)


def test_deterministic_and_power_of_two_invariant():
    n = 640
    T, _ = workloads.config0_schur(n, seed=21)
    X1, e1, _, _ = _gpu(T, tile=64)
    X2, e2, _, _ = _gpu(T, tile=64)
    np.testing.assert_array_equal(X1, X2)
    np.testing.assert_array_equal(e1, e2)
    # T -> 2^6 T: same eigenvectors, every operation scaled exactly
    X3, e3, _, _ = _gpu(np.ldexp(T, 6), tile=64)
    np.testing.assert_array_equal(X1, X3)
    np.testing.assert_array_equal(e1, e3)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_subset_columns_bit_identical_to_all_columns(mode):
    # columns are independent in the method: a subset's columns equal the
    # same columns of the all-columns run bit for bit.  The subset has far
    # fewer active units per step, so its diagonal solves run with more
    # lanes per unit (16 / 32 instead of 8): this pins those variants to
    # the default one.
    n = 1500
    T, blocks = workloads.config0_schur(n, seed=77)
    Q = workloads.householder_orthogonal(n, seed=78)
    Xa, ea, _, _ = _gpu(T, Q, tile=64, mode=mode)
    sel = workloads.random_eigen_selection(n, blocks, 0.1, seed=79)
    Xs, es, _, _ = _gpu(T, Q, select=sel, tile=64, mode=mode)
    cols, col = [], 0
    for p, sz in blocks:
        if sel[p] or (sz == 2 and sel[p + 1]):
            cols.extend(range(col, col + sz))
        col += sz
    assert Xs.shape[1] == len(cols) > 0
    np.testing.assert_array_equal(Xs, Xa[:, cols])
    np.testing.assert_array_equal(es, ea[cols])


def test_plan_reuse_follows_the_diagonals_and_selection():
    # the handle reuses its plan when T's three central diagonals, the
    # selection and the tile are those of the last call; anything else
    # replans.  Same diagonals with a different upper part, a changed
    # eigenvalue, a changed selection, then the first matrix again: each
    # result matches the oracle for its own input.
    n = 400
    T1, blocks = workloads.config0_schur(n, seed=301)
    T2 = T1.copy()
    rng = np.random.default_rng(302)
    iu = np.triu_indices(n, 2)
    T2[iu] = rng.standard_normal(len(iu[0]))        # same diagonals, new upper part
    T3 = T1.copy()
    p = next(q for q, sz in blocks if sz == 1 and q > 10)
    T3[p, p] += 0.125                               # one eigenvalue moved
    sel = workloads.random_eigen_selection(n, blocks, 0.3, seed=303)
    for T, s in ((T1, None), (T2, None), (T3, None), (T3, sel), (T1, None)):
        X, e, lr, li = _gpu(T, tile=32, select=s)
        _parity(T, None, X, e, lr, li, select=s)


# ---------------------------------------------------------------------------
# full size, in the benchmark's launch configuration (tile 64, with Q):
# the GPU computes every column, the oracle a seeded sample of columns
# ---------------------------------------------------------------------------
def _sampled_parity(T, blocks, Q, k, seed, rel_tol, mode="fp64", tile=0):
    n = T.shape[0]
    X, e, lr, li = _gpu(T, Q, tile=tile, mode=mode)
    assert np.isfinite(X).all()
    rng = np.random.default_rng(seed)
    chosen = rng.choice(len(blocks), size=k, replace=False)
    sel = np.zeros(n, np.uint8)
    for b in chosen:
        p, sz = blocks[b]
        sel[p:p + sz] = 1
    Xo, eo, lro, lio = oracle.standard(T, Q=Q, select=sel)
    cols = []
    col = 0
    for p, sz in blocks:
        if sel[p]:
            cols.extend(range(col, col + sz))
        col += sz
    de, rel = compare_canonical(Xo, eo, X[:, cols], e[cols], lio)
    assert de <= 1
    assert rel <= rel_tol, rel
    A = Q @ T @ Q.T
    res = standard_residuals(A, X[:, cols], lr[cols], li[cols])
    assert res.max() <= 10 * n
    nr = canonical_norms(X, li)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    return rel


@pytest.mark.parametrize("tile", [0, 256, 512])
def test_full_size_config1a_sampled(tile):
    # n = 4096 with Q across the tile sweep (0 = the default 64; 256 and 512
    # are solved in sub-blocks of at most 64 rows, one exponent per tile)
    n = 4096
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE + 1)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 101)
    _sampled_parity(T, blocks, Q, k=48, seed=1, rel_tol=REL_TOL, tile=tile)


@pytest.mark.parametrize("tile", [0, 256, 512])
def test_full_size_config1b_sampled(tile):
    n = 4096
    T, blocks = workloads.adversarial_schur(n, seed=workloads.SEED_BASE + 11)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 111)
    _sampled_parity(T, blocks, Q, k=32, seed=2, rel_tol=1e-3, tile=tile)


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("n,tile", [(1300, 200), (1300, 256), (1100, 512), (700, 512),
                                    (600, 130)])
def test_big_tiles(n, tile, mode):
    # tiles above 64 rows: sub-blocks of at most 64 rows inside each tile
    # (a boundary that would split a 2x2 block moves up a row), the rows
    # above a sub-block updated in one protected pass; ragged last tiles,
    # with Q, every column against the oracle
    T, blocks = workloads.config0_schur(n, seed=n + tile)
    Q = workloads.householder_orthogonal(n, seed=n + tile + 1)
    X, e, lr, li = _gpu(T, Q, tile=tile, mode=mode)
    _parity(T, Q, X, e, lr, li)
    X, e, lr, li = _gpu(T, None, tile=tile, mode=mode)
    _check_structure(T, blocks, X, li)
    _parity(T, None, X, e, lr, li)


@pytest.mark.parametrize("tile", [256, 512])
def test_big_tiles_adversarial_and_selection(tile):
    n = 1200
    T, blocks = workloads.adversarial_schur(n, seed=88 + tile)
    _, bad = oracle.naive_standard(T)
    assert bad > 0
    X, e, lr, li = _gpu(T, tile=tile)
    _check_structure(T, blocks, X, li)
    assert e.min() < -1074
    _parity(T, None, X, e, lr, li, rel_tol=1e-3)
    T, blocks = workloads.config0_schur(n, seed=89 + tile)
    sel = workloads.random_eigen_selection(n, blocks, 0.35, seed=90)
    X, e, lr, li = _gpu(T, select=sel, tile=tile, mode="split")
    _check_structure(T, blocks, X, li, select=sel)
    _parity(T, None, X, e, lr, li, select=sel)


# ---------------------------------------------------------------------------
# split precision (BF16 slices on the tensor cores) -- same parity bar at the
# default 8 slices: a product term's error is ~2^-55 of its row / column
# maxima, at the level of FP64 rounding
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,tile", [(300, 64), (517, 32), (1000, 128)])
def test_split_backtransform(n, tile):
    T, blocks = workloads.config0_schur(n, seed=n + 5)
    Q = workloads.householder_orthogonal(n, seed=n + 6)
    X, e, lr, li = _gpu(T, Q, tile=tile, mode="split")
    nr = canonical_norms(X, li)
    assert np.isfinite(X).all() and nr.min() >= 1.0 and nr.max() < 2.0
    _parity(T, Q, X, e, lr, li)


@pytest.mark.parametrize("tile", [16, 32, 64, 128])
def test_split_tile_update_paths(tile):
    # no Q: X is the solve's own output, so every tile update is on the
    # tensor cores (tiles <= 64: panel-resident kernel; 128: streamed panel)
    n = 613
    T, blocks = workloads.config0_schur(n, seed=640 + tile)
    X, e, lr, li = _gpu(T, tile=tile, mode="split")
    _check_structure(T, blocks, X, li)
    _parity(T, None, X, e, lr, li)


def test_split_seven_slices():
    # 7 slices: products carry ~2^-48 of their row / column maxima; the
    # residual gate holds and the column error stays within 1e-8 here
    n = 700
    T, blocks = workloads.config0_schur(n, seed=5)
    X, e, lr, li = _gpu(T, tile=16, mode="split", slices=7)
    _check_structure(T, blocks, X, li)
    rel, res = _parity(T, None, X, e, lr, li, rel_tol=1e-8)
    assert rel > 0.0


def test_split_slices_out_of_range():
    T, _ = workloads.config0_schur(64, seed=3)
    for bad in (1, 9):
        with pytest.raises(ev.EvecError) as ei:
            _gpu(T, mode="split", slices=bad)
        assert ei.value.status == ev.EVEC_EINVAL


def test_split_power_of_two_invariant():
    # rows and columns are normalised by powers of two before slicing, so
    # T -> 2^6 T leaves every digit, and so every result bit, unchanged
    n = 500
    T, _ = workloads.config0_schur(n, seed=31)
    Q = workloads.householder_orthogonal(n, seed=32)
    X1, e1, _, _ = _gpu(T, Q, tile=64, mode="split")
    X2, e2, _, _ = _gpu(np.ldexp(T, 6), Q, tile=64, mode="split")
    np.testing.assert_array_equal(X1, X2)
    np.testing.assert_array_equal(e1, e2)


def test_split_selection_and_determinism():
    n = 700
    T, blocks = workloads.config0_schur(n, seed=15)
    Q = workloads.householder_orthogonal(n, seed=16)
    sel = workloads.random_eigen_selection(n, blocks, 0.35, seed=17)
    X1, e1, lr, li = _gpu(T, Q, select=sel, tile=64, mode="split")
    X2, e2, _, _ = _gpu(T, Q, select=sel, tile=64, mode="split")
    np.testing.assert_array_equal(X1, X2)
    np.testing.assert_array_equal(e1, e2)
    _parity(T, Q, X1, e1, lr, li, select=sel)


def test_split_adversarial():
    n = 512
    T, blocks = workloads.adversarial_schur(n, seed=78)
    Q = workloads.householder_orthogonal(n, seed=79)
    X, e, lr, li = _gpu(T, Q, tile=64, mode="split")
    assert np.isfinite(X).all()
    _parity(T, Q, X, e, lr, li, rel_tol=1e-3)


def test_split_full_size_config1a_sampled():
    n = 4096
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE + 1)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 101)
    _sampled_parity(T, blocks, Q, k=48, seed=3, rel_tol=REL_TOL, mode="split")


SPLIT_16K_TOL = 5e-10


def _sample_blocks(blocks, n, k, seed):
    rng = np.random.default_rng(seed)
    chosen = rng.choice(len(blocks), size=k, replace=False)
    sel = np.zeros(n, np.uint8)
    for b in chosen:
        p, sz = blocks[b]
        sel[p:p + sz] = 1
    cols = []
    col = 0
    for p, sz in blocks:
        if sel[p]:
            cols.extend(range(col, col + sz))
        col += sz
    return sel, cols


def _column_errors(Xo, eo, X, e, li):
    """Per eigenvalue: normwise relative difference of two canonical
    results after bringing both to one exponent."""
    out = []
    for j, pair in column_groups(li):
        w = 2 if pair else 1
        de, rel = compare_canonical(Xo[:, j:j + w], eo[j:j + w], X[:, j:j + w], e[j:j + w],
                                    li[j:j + w])
        assert de <= 1, (j, de)
        out.append(rel)
    return np.asarray(out)


@pytest.mark.parametrize("refine", [0, 1])
def test_split_full_size_config2_sampled(refine):
    # n = 16384, split precision, with Q, the default launch configuration
    # (tile 64, 8 slices), without and with the residual-correction sweep:
    # 256 sampled eigenvalues against the oracle, and the residual of those
    # columns in Schur coordinates (y = Q^T x, FP64 BLAS; its rounding is
    # far below the 10 n gate).  16384 eigenvalues in [-1, 1] are about
    # 1e-4 apart, and these eigenvectors grow by up to 2^8000 between their
    # block and their top entry, so the scale of a column (top against
    # block) is ill-conditioned for any FP64 solve: the FP64 path differs
    # from the oracle by up to a few 1e-11 on such samples, the split path
    # (products carry ~2^-55 of their row / column maxima) somewhat more.
    # The column bound is SPLIT_16K_TOL; the residual gate is the method's.
    n = 16384
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE + 2)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 102)
    X, e, lr, li = _gpu(T, Q, tile=0, mode="split", refine=refine)
    assert np.isfinite(X).all()
    nr = canonical_norms(X, li)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    sel, cols = _sample_blocks(blocks, n, 256, seed=4)
    Xo, eo, lro, lio = oracle.standard(T, Q=Q, select=sel)
    np.testing.assert_array_equal(lr[cols], lro)
    np.testing.assert_array_equal(li[cols], lio)
    errs = _column_errors(Xo, eo, X[:, cols], e[cols], lio)
    print(f"config2 split refine={refine}: {len(errs)} eigenvalues, column error max "
          f"{errs.max():.3e} median {np.median(errs):.3e}")
    assert errs.max() <= SPLIT_16K_TOL, errs.max()
    Y = Q.T @ X[:, cols]
    res = standard_residuals(T, Y, lr[cols], li[cols])
    assert res.max() <= 10 * n, res.max()


@pytest.mark.parametrize("kind", ["standard", "refine", "trsolve"])
def test_lookahead_schedule_is_bit_identical(kind):
    # the look-ahead schedule (decisions as their own launch, each step's
    # update split at the next diagonal tile and run beside its solve)
    # changes the order of launches, not the arithmetic of any element
    n = 613
    T, _ = workloads.config0_schur(n, seed=404)
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    h = ev.handle(0)
    outs = []
    for la in (False, True):
        h.lookahead(la)
        try:
            if kind == "trsolve":
                B = np.random.default_rng(5).standard_normal((n, 300))
                dB = torch.from_numpy(np.asfortranarray(B)).cuda()
                X, e = ev.trsolve(dT, dB, tile=64, check=True, mode="split")
            else:
                X, e, _, _ = ev.standard(dT, tile=64, check=True, mode="split",
                                         slices=5 if kind == "refine" else 0,
                                         refine=kind == "refine")
        finally:
            h.lookahead(False)
        torch.cuda.synchronize()
        outs.append((X.cpu().numpy(), e.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("with_q,tile", [(False, 64), (True, 64), (True, 256)])
def test_outputs_stay_inside_their_buffers(mode, with_q, tile):
    # canary-padded outputs (the race-detection substitute for a sanitizer):
    # X with a leading dimension above n and spare columns, the exponent and
    # eigenvalue vectors with spare entries, all filled with a sentinel; the
    # call writes exactly the n x m block and the m entries
    n, pad_rows, pad_cols = 333, 19, 5
    T, _ = workloads.config0_schur(n, seed=42)
    Q = workloads.householder_orthogonal(n, seed=43) if with_q else None
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    dQ = None if Q is None else torch.from_numpy(np.asfortranarray(Q)).cuda()
    m = ev.count(dT)
    ld = n + pad_rows
    sentinel = -1.2345e300
    buf = torch.full((m + pad_cols, ld), sentinel, dtype=torch.float64, device="cuda")
    X = buf.t()[:n, :m]
    assert X.stride() == (1, ld)
    ebuf = torch.full((m + pad_cols,), 7777777, dtype=torch.int32, device="cuda")
    lbuf = torch.full((2, m + pad_cols), sentinel, dtype=torch.float64, device="cuda")
    out = (X, ebuf[:m], lbuf[0, :m], lbuf[1, :m])
    ev.standard(dT, dQ, tile=tile, check=True, out=out, mode=mode, refine=0)
    torch.cuda.synchronize()
    b = buf.t().cpu().numpy()
    assert np.all(b[n:, :] == sentinel)                  # rows between n and ld
    assert np.all(b[:, m:] == sentinel)                  # spare columns
    assert np.isfinite(b[:n, :m]).all()
    assert np.all(ebuf[m:].cpu().numpy() == 7777777)
    assert np.all(lbuf[:, m:].cpu().numpy() == sentinel)
    Xo, eo, _, lio = oracle.standard(T, Q=Q)
    de, rel = compare_canonical(Xo, eo, b[:n, :m], ebuf[:m].cpu().numpy(), lio)
    assert de <= 1 and rel <= REL_TOL, (de, rel)
