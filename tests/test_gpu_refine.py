"""The residual-correction sweep of split mode (opts.refine) against the CPU
oracle, with the single-matrix parity bar (exponents +-1, columns within 1e-10
normwise relative on well-conditioned inputs, residual <= 10 n).

One sweep is classical iterative refinement with an FP64 residual: if the
split solve carries a relative error eps (about 2^(-7 slices) of the row /
column maxima per product), the correction d solves for the residual to the
same relative eps, so the refined column carries about eps^2 plus the FP64
residual's own rounding.  The low-slice tests use that: 5 slices alone miss
the bar by orders of magnitude, one sweep brings them under it (4 slices,
eps ~ 1e-4 here: one sweep gains about four digits).  At 8 slices the split
solve is already as close to the exact eigenvectors as the FP64 solve
(checked against an extended-precision backsubstitution below), and the
sweep takes only corrections below 2^(20 - 7 slices) of a column."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads
from evec_checks import (canonical_norms, compare_canonical, extended_errors,
                         ld_real_eigvec, longdouble_is_extended, standard_residuals)

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


def _gpu(T, Q=None, select=None, tile=0, mode="split", slices=0, refine=True):
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    dQ = None if Q is None else torch.from_numpy(np.asfortranarray(Q)).cuda()
    X, e, lr, li = ev.standard(dT, dQ, select=select, tile=tile, check=True, mode=mode,
                               slices=slices, refine=refine)
    torch.cuda.synchronize()
    return X.cpu().numpy(), e.cpu().numpy(), lr.cpu().numpy(), li.cpu().numpy()


def _against_oracle(T, Q, out, select=None):
    X, e, lr, li = out
    Xo, eo, lro, lio = oracle.standard(T, Q=Q, select=select)
    assert X.shape == Xo.shape
    np.testing.assert_array_equal(lr, lro)
    np.testing.assert_array_equal(li, lio)
    assert np.isfinite(X).all()
    nr = canonical_norms(X, li)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    de, rel = compare_canonical(Xo, eo, X, e, lio)
    assert de <= 1, de
    A = T if Q is None else Q @ T @ Q.T
    res = standard_residuals(A, X, lr, li)
    assert res.max() <= 10 * T.shape[0], res.max()
    return rel


def _zeros_below_blocks(blocks, X, select=None):
    col = 0
    for p, sz in blocks:
        if select is not None and not (select[p] or (sz == 2 and select[p + 1])):
            continue
        for k in range(sz):
            assert np.all(X[p + sz:, col + k] == 0.0)
        col += sz


@pytest.mark.parametrize("tile", [16, 32, 64, 128, 256, 512])
def test_refine_all_tiles(tile):
    # no Q: the refined Y itself (tiles <= 64: panel-resident update kernel
    # in both sweeps; 128: streamed panel)
    n = 613
    T, blocks = workloads.config0_schur(n, seed=700 + tile)
    out = _gpu(T, tile=tile)
    _zeros_below_blocks(blocks, out[0])
    assert _against_oracle(T, None, out) <= REL_TOL


@pytest.mark.parametrize("slices", [4, 5])
def test_refine_recovers_low_slices(slices):
    # without the sweep the column error is ~2^(-7 slices) x growth, far
    # above the bar; with it the error is about its square
    n = 500
    T, blocks = workloads.config0_schur(n, seed=90 + slices)
    X, e, lr, li = _gpu(T, tile=64, slices=slices, refine=False)
    Xo, eo, _, lio = oracle.standard(T)
    _, rel_plain = compare_canonical(Xo, eo, X, e, lio)
    assert rel_plain > 10 * REL_TOL, rel_plain
    rel = _against_oracle(T, None, _gpu(T, tile=64, slices=slices))
    if slices >= 5:
        assert rel <= REL_TOL, (rel_plain, rel)
    else:
        assert rel <= 1e-3 * rel_plain, (rel_plain, rel)


def test_refine_with_backtransform_and_selection():
    n = 700
    T, blocks = workloads.config0_schur(n, seed=15)
    Q = workloads.householder_orthogonal(n, seed=16)
    sel = workloads.random_eigen_selection(n, blocks, 0.35, seed=17)
    out = _gpu(T, Q, select=sel, tile=64)
    assert _against_oracle(T, Q, out, select=sel) <= REL_TOL
    # deterministic: a second call gives the same bits
    out2 = _gpu(T, Q, select=sel, tile=64)
    np.testing.assert_array_equal(out[0], out2[0])
    np.testing.assert_array_equal(out[1], out2[1])


def test_refine_closer_to_fp64_than_plain_split():
    # the refined split result and the FP64 path agree better than the plain
    # split result and the FP64 path (4 slices, where the gap is large)
    n = 800
    T, blocks = workloads.config0_schur(n, seed=21)
    Xf, ef, _, lif = _gpu(T, tile=32, mode="fp64", refine=False)
    Xp, ep, _, _ = _gpu(T, tile=32, slices=4, refine=False)
    Xr, er, _, _ = _gpu(T, tile=32, slices=4)
    _, d_plain = compare_canonical(Xf, ef, Xp, ep, lif)
    _, d_ref = compare_canonical(Xf, ef, Xr, er, lif)
    assert d_ref < 1e-3 * d_plain, (d_plain, d_ref)


def test_refine_adversarial_overflow_case():
    # entries near the overflow threshold: the correction solve runs under
    # the same protection, the result stays finite and within the
    # clustered-input bound of the FP64 path
    n = 512
    T, blocks = workloads.adversarial_schur(n, seed=78)
    Q = workloads.householder_orthogonal(n, seed=79)
    out = _gpu(T, Q, tile=64)
    assert _against_oracle(T, Q, out) <= 1e-3


def test_refine_edge_sizes():
    # n = 1, 2 (no rows above any block: the correction is zero) and a
    # ragged n just above a tile
    for n in (1, 2, 3, 65):
        T, blocks = workloads.config0_schur(n, seed=n + 40)
        out = _gpu(T, tile=64)
        _zeros_below_blocks(blocks, out[0])
        assert _against_oracle(T, None, out) <= REL_TOL


def test_refine_ignored_in_fp64_mode():
    n = 300
    T, _ = workloads.config0_schur(n, seed=9)
    a = _gpu(T, tile=32, mode="fp64", refine=True)
    b = _gpu(T, tile=32, mode="fp64", refine=False)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def _real_columns(blocks):
    out, col = [], 0
    for p, sz in blocks:
        if sz == 1:
            out.append((p, col))
        col += sz
    return out


@pytest.mark.skipif(not longdouble_is_extended(), reason="no extended long double")
def test_split_fp64_refined_against_extended_precision():
    # n = 8192 config-0, no Q.  These eigenvectors grow by up to 2^8000
    # from their block to their top, so the ratio of the top entries to the
    # block (the scale) is ill-conditioned for any FP64 solve; the direction
    # is not.  On the columns where the split and FP64 results differ most,
    # and on random ones, all three (FP64, split, split + sweep) agree with
    # an extended-precision backsubstitution to 1e-13 in direction and to
    # 1e-9 with the scale (the FP64 path's own largest error here: 4.9e-10).
    n = 8192
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE + 2)
    runs = {
        "fp64": _gpu(T, tile=0, mode="fp64", refine=False),
        "split": _gpu(T, tile=0, refine=False),
        "refined": _gpu(T, tile=0),
    }
    Xf, ef = runs["fp64"][0], runs["fp64"][1]
    Xs, es = runs["split"][0], runs["split"][1]
    cols = _real_columns(blocks)
    gap = []
    for p, j in cols:
        a = Xf[:p + 1, j]
        b = np.ldexp(Xs[:p + 1, j], int(ef[j]) - int(es[j]))
        gap.append(np.max(np.abs(a - b)) / np.max(np.abs(a)))
    order = np.argsort(gap)[::-1]
    rng = np.random.default_rng(12)
    pick = list(order[:6]) + list(rng.choice(len(cols), 6, replace=False))
    for k in pick:
        p, j = cols[k]
        yref = ld_real_eigvec(T, blocks, p)
        for name, (X, e, _, _) in runs.items():
            d, s = extended_errors(yref, X[:, j], e[j])
            assert d <= 1e-13, (name, j, d)
            assert s <= 1e-9, (name, j, s)


def test_refine_full_size_config2_sampled():
    # n = 16384 with Q in the benchmark's launch configuration (tile 64,
    # 8 slices, one sweep): 16 sampled eigenvalues against the oracle with
    # the bound of the plain split test (the FP64 path itself is ~5e-10 from
    # the exact vectors at this growth), their residual in Schur coordinates,
    # and 4 sampled real columns against the extended-precision
    # backsubstitution (y = Q^T x in FP64: its rounding is ~1e-14 here)
    n = 16384
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE + 2)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 102)
    X, e, lr, li = _gpu(T, Q, tile=0)
    assert np.isfinite(X).all()
    nr = canonical_norms(X, li)
    assert nr.min() >= 1.0 and nr.max() < 2.0
    rng = np.random.default_rng(4)
    chosen = rng.choice(len(blocks), size=16, replace=False)
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
    assert rel <= 5e-10, rel
    Y = Q.T @ X[:, cols]
    res = standard_residuals(T, Y, lr[cols], li[cols])
    assert res.max() <= 10 * n, res.max()
    if longdouble_is_extended():
        real = _real_columns(blocks)
        for k in rng.choice(len(real), 4, replace=False):
            p, j = real[k]
            yref = ld_real_eigvec(T, blocks, p)
            d, s = extended_errors(yref, Q.T @ X[:, j], e[j])
            assert d <= 1e-12 and s <= 1e-9, (j, d, s)


def _spread(n, seed):
    # real eigenvalues spread over [-50, 50] (gaps up to 100): an error in
    # a vector shows in its residual (T - lambda I) dy, unlike the clustered
    # config-0 spectrum, where a residual gate passes errors that lie along
    # nearby eigenvectors
    rng = np.random.default_rng(seed)
    T = np.triu(rng.standard_normal((n, n)), 1)
    T[np.arange(n), np.arange(n)] = rng.permutation(np.linspace(-50.0, 50.0, n))
    return T, [(i, 1) for i in range(n)]


def test_residual_gate_repeats_a_failing_solve():
    # refine = 2: after the sweep, the gate ||(T - lambda I) y||_1 <= 10 n
    # ||T||_1 ||y||_1 u per eigenvalue.  At 2 slices (about 2^-14 per
    # product, 2^-28 after one sweep) the spread spectrum fails it; the
    # matrix is solved again with 8 slices and then meets the parity bar
    n = 400
    T, blocks = _spread(n, 61)
    out = _gpu(T, tile=64, slices=2, refine=2)
    failed, retries = ev.handle(0).gate_stats()
    assert failed > 0 and retries >= 1, (failed, retries)
    _zeros_below_blocks(blocks, out[0])
    assert _against_oracle(T, None, out) <= REL_TOL


def test_residual_gate_passes_at_8_slices():
    n = 613
    for T in (workloads.config0_schur(n, seed=62)[0], _spread(n, 65)[0]):
        out = _gpu(T, tile=64, refine=2)
        assert ev.handle(0).gate_stats() == (0, 0)
        assert _against_oracle(T, None, out) <= REL_TOL


def test_residual_gate_with_q_and_left():
    n = 300
    T, blocks = _spread(n, 63)
    Q = workloads.householder_orthogonal(n, seed=64)
    out = _gpu(T, Q, tile=32, slices=2, refine=2)
    failed, retries = ev.handle(0).gate_stats()
    assert failed > 0 and retries >= 1
    assert _against_oracle(T, Q, out) <= REL_TOL
    # the left eigenvectors run the same path on the flipped form
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    X, e, lr, li = ev.left(dT, tile=32, check=True, mode="split", slices=2, refine=2)
    assert ev.handle(0).gate_stats()[1] >= 1
    Xo, eo, _, lio = oracle.left(T)
    de, rel = compare_canonical(Xo, eo, X.cpu().numpy(), e.cpu().numpy(), lio)
    assert de <= 1 and rel <= REL_TOL, (de, rel)


def test_residual_gate_reports_eresidual_after_every_repeat():
    # a gate no result can pass (factor 1e-30 instead of 10): the split
    # solve fails it, the 8-slice repeat fails it, the FP64 repeat fails it
    # too, and evec_sync reports EVEC_ERESIDUAL with the output column of the
    # first failing eigenvalue; the result is the FP64 one
    n = 300
    T, blocks = workloads.config0_schur(n, seed=66)
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    h = ev.handle(0)
    L = ev.lib()
    L.evec_set_gate_factor.argtypes = [ctypes.c_void_p, ctypes.c_double]
    L.evec_set_gate_factor.restype = ctypes.c_int
    assert L.evec_set_gate_factor(h.ptr, 0.0) == ev.EVEC_EINVAL
    assert L.evec_set_gate_factor(h.ptr, 1e-30) == ev.EVEC_OK
    try:
        X, e, lr, li = ev.standard(dT, tile=32, mode="split", slices=4, refine=2)
        with pytest.raises(ev.EvecError) as ei:
            h.sync()
        assert ei.value.status == ev.EVEC_ERESIDUAL
        # the first block's vector has no rows above it: its residual is 0
        # and passes any gate; the first failure is the second block's
        assert ei.value.bad == blocks[0][1]
        assert ev.handle(0).gate_stats()[1] == 2       # 8 slices, then FP64
        Xf, ef, _, lif = ev.standard(dT, tile=32, mode="fp64", check=True)
        np.testing.assert_array_equal(X.cpu().numpy(), Xf.cpu().numpy())
        np.testing.assert_array_equal(e.cpu().numpy(), ef.cpu().numpy())
    finally:
        assert L.evec_set_gate_factor(h.ptr, 10.0) == ev.EVEC_OK
    # the default gate again: passes, and the status was cleared
    out = _gpu(T, tile=32, slices=4, refine=2)
    h.sync()
    assert _against_oracle(T, None, out) <= REL_TOL


def test_opts_struct_in_the_documented_field_order():
    # evec_opts filled by a C caller in the header's order {mode, tile,
    # slices, refine, check}: slices = 9 in the third field is refused, and
    # check = 1 in the fifth makes the call return the device status
    class Opts(ctypes.Structure):
        _fields_ = [("mode", ctypes.c_int), ("tile", ctypes.c_int), ("slices", ctypes.c_int),
                    ("refine", ctypes.c_int), ("check", ctypes.c_int)]

    n = 120
    T, _ = workloads.config0_schur(n, seed=67)
    # a private handle on the library: the prototype set here must not
    # replace the one the binding uses
    L = ctypes.CDLL(ev.LIB_PATH)
    f = L.evec_standard
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [p, i64, p, i64, p, i64, p, p, i64, p, p, p, ctypes.POINTER(Opts)]
    f.restype = ctypes.c_int
    h = ev.handle(0)
    X = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    e = torch.empty(n, dtype=torch.int32, device="cuda")
    bad_T = np.array(T, order="F", copy=True)
    bad_T[5, 100] = np.inf
    dT = torch.from_numpy(np.asfortranarray(bad_T)).cuda()

    def call(o):
        return f(h.ptr, n, dT.data_ptr(), n, None, n, None, X.data_ptr(), n, e.data_ptr(), None,
                 None, ctypes.byref(o))

    assert call(Opts(mode=1, tile=32, slices=9, refine=0, check=1)) == ev.EVEC_EINVAL
    assert call(Opts(mode=1, tile=32, slices=6, refine=0, check=1)) == ev.EVEC_ENONFINITE
    d = Opts()
    L.evec_opts_default.argtypes = [ctypes.POINTER(Opts)]
    L.evec_opts_default.restype = None
    L.evec_opts_default(ctypes.byref(d))
    assert (d.mode, d.tile, d.slices, d.refine, d.check) == (0, 0, 0, 1, 0)
