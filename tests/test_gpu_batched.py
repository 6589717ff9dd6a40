"""Batched mode (evec_batched): many independent Schur forms in one persistent
launch, against the CPU oracle matrix by matrix, with the parity bar of the
single-matrix tests (exponents +-1; columns within 1e-10 normwise relative on
well-conditioned inputs, 1e-3 on the clustered adversarial ones; residual
<= 10 n).  Both modes: FP64, and split precision (the updates as BF16 slice
products on the tensor cores inside the persistent kernel, 8 slices: the
same bar as the single-matrix split path)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads
from evec_checks import compare_canonical, standard_residuals

pytestmark = pytest.mark.gpu


def _members(sizes, seed, adversarial_every=0, fraction=0.3):
    Ts, sels, adv = [], [], []
    for i, n in enumerate(sizes):
        s = seed * 1000 + i
        a = bool(adversarial_every) and i % adversarial_every == adversarial_every - 1
        T, blocks = (workloads.adversarial_schur if a else workloads.config0_schur)(int(n), seed=s)
        Ts.append(T)
        sels.append(None if fraction is None else
                    workloads.block_selection(int(n), blocks, fraction, seed=s + 7))
        adv.append(a)
    return Ts, sels, adv


def _check_against_oracle(Ts, sels, adv, res, tol=1e-10):
    for T, sel, a, (X, e, lr, li) in zip(Ts, sels, adv, res):
        Xo, eo, lro, lio = oracle.standard(T, select=sel)
        X, e, lr, li = X.cpu().numpy(), e.cpu().numpy(), lr.cpu().numpy(), li.cpu().numpy()
        assert X.shape == Xo.shape
        if X.shape[1] == 0:
            continue
        np.testing.assert_array_equal(lr, lro)
        np.testing.assert_array_equal(li, lio)
        assert np.isfinite(X).all()
        de, rel = compare_canonical(Xo, eo, X, e, lio)
        assert de <= 1, de
        assert rel <= (1e-3 if a else tol), (T.shape[0], rel)
        r = standard_residuals(T, X, lr, li)
        assert r.max() <= 10 * T.shape[0], r.max()


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_batched_mixed_sizes(tile):
    sizes = [37, 300, 64, 65, 129, 1, 2, 513, 96, 250, 31, 200]
    Ts, sels, adv = _members(sizes, seed=11, adversarial_every=5)
    res = ev.batched(Ts, sels, tile=tile)
    _check_against_oracle(Ts, sels, adv, res)


def test_batched_all_columns_and_empty_selections():
    sizes = [120, 77, 300, 45]
    Ts, sels, adv = _members(sizes, seed=12, fraction=None)
    sels = [None, np.zeros(77, np.uint8), None, np.zeros(45, np.uint8)]
    res = ev.batched(Ts, sels, tile=32)
    assert res[1][0].shape == (77, 0) and res[3][0].shape == (45, 0)
    _check_against_oracle(Ts, sels, adv, res)


def test_batched_autotuned_tiles_and_table():
    sizes = [40, 90, 200, 400, 700, 60, 150]
    Ts, sels, adv = _members(sizes, seed=13)
    h = ev.handle(0)
    ev.set_tune_table([0] * ev.SIZE_CLASSES)
    res = ev.batched(Ts, sels, tile=0)
    _check_against_oracle(Ts, sels, adv, res)
    table = ev.tune_table()
    assert all(t in (16, 32, 64) for t in table)   # every class is present here
    # a loaded table is used as is, and gives the same answers
    ev.set_tune_table([16] * ev.SIZE_CLASSES)
    res2 = ev.batched(Ts, sels, tile=0)
    _check_against_oracle(Ts, sels, adv, res2)
    assert ev.tune_table() == [16] * ev.SIZE_CLASSES
    ev.set_tune_table(table)
    del h


def test_batched_repeat_is_deterministic():
    # the second call replays the cached graph of the first
    sizes = [100, 260, 33, 500]
    Ts, sels, adv = _members(sizes, seed=14)
    a = ev.batched(Ts, sels, tile=64)
    b = ev.batched(Ts, sels, tile=64)
    for (X1, e1, _, _), (X2, e2, _, _) in zip(a, b):
        np.testing.assert_array_equal(X1.cpu().numpy(), X2.cpu().numpy())
        np.testing.assert_array_equal(e1.cpu().numpy(), e2.cpu().numpy())


def test_batched_errors_name_the_packed_entry():
    sizes = [50, 60, 70]
    Ts, sels, adv = _members(sizes, seed=15, fraction=None)
    bad = [T.copy() for T in Ts]
    bad[1][5, 40] = np.nan                      # matrix 1, entry (5, 40)
    Tp, ns, offs = ev.pack_batch(bad)
    with pytest.raises(ev.EvecError) as ei:
        ev.batched_packed(Tp, ns, offs, tile=32, check=True)
    assert ei.value.status == ev.EVEC_ENONFINITE
    assert ei.value.bad == offs[1] + 5 + 40 * 60
    bad = [T.copy() for T in Ts]
    bad[2][11, 10] = 0.5                        # a second nonzero subdiagonal next to a pair
    bad[2][12, 11] = 0.5
    Tp, ns, offs = ev.pack_batch(bad)
    with pytest.raises(ev.EvecError) as ei:
        ev.batched_packed(Tp, ns, offs, tile=32)
    assert ei.value.status == ev.EVEC_ENOTSCHUR
    Tp, ns, offs = ev.pack_batch(Ts)
    for bad_slices in (1, 9):                     # split precision: 2..8 slices
        with pytest.raises(ev.EvecError) as ei:
            ev.batched_packed(Tp, ns, offs, mode="split", slices=bad_slices)
        assert ei.value.status == ev.EVEC_EINVAL
    # the handle stays usable
    res = ev.batched(Ts, None, tile=32)
    _check_against_oracle(Ts, [None] * 3, [False] * 3, res)


def test_batched_config3_full_size_sampled():
    # the benchmark's batch: 2000 matrices, sizes log-uniform in [32, 1024],
    # every 10th adversarial, 30% of the blocks selected; 24 members checked
    sizes, Ts, sels = workloads.batch_inputs(2000)
    res = ev.batched(Ts, sels, tile=0)
    rng = np.random.default_rng(5)
    pick = sorted(rng.choice(len(Ts), size=24, replace=False))
    pick += [int(np.argmax(sizes))]            # the largest member too
    adv = [i % 10 == 9 for i in range(len(Ts))]
    _check_against_oracle([Ts[i] for i in pick], [sels[i] for i in pick],
                          [adv[i] for i in pick], [res[i] for i in pick])
    for X, e, lr, li in res:
        assert bool(torch.isfinite(X).all())


# ---------------------------------------------------------------------------
# split precision inside the persistent kernel
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("tile", [16, 32, 64])
def test_batched_split_mixed_sizes(tile):
    # sizes around the 128-row blocks and 32-column chunks of the in-kernel
    # split update (127, 128, 129, 300, 513: several row blocks, ragged)
    sizes = [37, 300, 64, 65, 129, 1, 2, 513, 96, 250, 31, 200, 127, 128]
    Ts, sels, adv = _members(sizes, seed=21, adversarial_every=5)
    res = ev.batched(Ts, sels, tile=tile, mode="split")
    _check_against_oracle(Ts, sels, adv, res)


def test_batched_split_all_columns_and_determinism():
    sizes = [120, 77, 300, 45, 700]
    Ts, sels, adv = _members(sizes, seed=22, fraction=None)
    a = ev.batched(Ts, None, tile=64, mode="split")
    _check_against_oracle(Ts, [None] * len(Ts), adv, a)
    b = ev.batched(Ts, None, tile=64, mode="split")
    for (X1, e1, _, _), (X2, e2, _, _) in zip(a, b):
        np.testing.assert_array_equal(X1.cpu().numpy(), X2.cpu().numpy())
        np.testing.assert_array_equal(e1.cpu().numpy(), e2.cpu().numpy())


def test_batched_split_matches_single_matrix_split_bar_and_fp64():
    # the split batch and the FP64 batch agree to the parity bar, and the
    # split batch is not bit-identical to the FP64 one (the products really
    # are split)
    sizes = [400, 250, 600]
    Ts, sels, adv = _members(sizes, seed=23)
    rs = ev.batched(Ts, sels, tile=32, mode="split")
    rf = ev.batched(Ts, sels, tile=32, mode="fp64")
    differs = False
    for (Xs, es, _, li), (Xf, ef, _, _) in zip(rs, rf):
        Xs, es, Xf, ef = (t.cpu().numpy() for t in (Xs, es, Xf, ef))
        de, rel = compare_canonical(Xf, ef, Xs, es, li.cpu().numpy())
        assert de <= 1 and rel <= 1e-10, rel
        differs |= not np.array_equal(Xs, Xf)
    assert differs


def test_batched_split_seven_slices():
    # 7 slices: products carry ~2^-48 of their row / column maxima; the
    # residual gate holds and the columns stay within 1e-8 (as the
    # single-matrix split path at 7 slices)
    sizes = [200, 350]
    Ts, sels, adv = _members(sizes, seed=24)
    res = ev.batched(Ts, sels, tile=32, mode="split", slices=7)
    _check_against_oracle(Ts, sels, adv, res, tol=1e-8)


def test_batched_split_autotuned_table():
    sizes = [40, 90, 200, 400, 700, 60, 150]
    Ts, sels, adv = _members(sizes, seed=25)
    ev.set_tune_table([0] * ev.SIZE_CLASSES, mode="split")
    res = ev.batched(Ts, sels, tile=0, mode="split")
    _check_against_oracle(Ts, sels, adv, res)
    table = ev.tune_table(mode="split")
    assert all(t in (16, 32, 64) for t in table)


def test_batched_split_config3_full_size_sampled():
    # the benchmark's batch in split mode: 24 members and the largest
    # against the oracle, every output finite
    sizes, Ts, sels = workloads.batch_inputs(2000)
    res = ev.batched(Ts, sels, tile=0, mode="split")
    rng = np.random.default_rng(6)
    pick = sorted(rng.choice(len(Ts), size=24, replace=False))
    pick += [int(np.argmax(sizes))]
    adv = [i % 10 == 9 for i in range(len(Ts))]
    _check_against_oracle([Ts[i] for i in pick], [sels[i] for i in pick],
                          [adv[i] for i in pick], [res[i] for i in pick])
    for X, e, lr, li in res:
        assert bool(torch.isfinite(X).all())


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_batched_with_q_and_output_offsets(mode):
    # a nullable Q per matrix (every other one back-transformed, X_i = Q_i Y_i)
    # and outputs placed by x_off / e_off in reverse matrix order with gaps;
    # each matrix against oracle.standard(T_i, Q=Q_i), and a second identical
    # call (a replay of the captured graph) gives the same bits
    sizes = [150, 33, 300, 64, 97, 1, 260, 40]
    Ts, sels, adv = _members(sizes, seed=17, adversarial_every=4)
    Qs = [workloads.householder_orthogonal(int(n), seed=300 + i) if i % 2 == 0 else None
          for i, n in enumerate(sizes)]
    Tp, ns, toffs = ev.pack_batch(Ts)
    Qp, _, hoffs = ev.pack_batch([q for q in Qs if q is not None])
    qoffs = np.full(len(Ts), -1, dtype=np.int64)
    k = 0
    for i, q in enumerate(Qs):
        if q is not None:
            qoffs[i] = hoffs[k]
            k += 1
    sel = np.concatenate([np.ones(n, np.uint8) if s is None else s for s, n in zip(sels, ns)])
    m = ev.batched_count(Tp, ns, toffs, sel)
    xoffs = np.zeros(len(Ts), dtype=np.int64)
    eoffs = np.zeros(len(Ts), dtype=np.int64)
    xa = ea = 0
    for i in reversed(range(len(Ts))):          # reverse order, 7-element gaps
        xoffs[i], eoffs[i] = xa, ea
        xa += int(ns[i] * m[i]) + 7
        ea += int(m[i]) + 7
    X = torch.full((xa,), np.nan, dtype=torch.float64, device="cuda")
    e = torch.zeros(ea, dtype=torch.int32, device="cuda")
    lr = torch.zeros(ea, dtype=torch.float64, device="cuda")
    li = torch.zeros(ea, dtype=torch.float64, device="cuda")
    outs = []
    for _ in range(2):
        ev.batched_packed(Tp, ns, toffs, sel, tile=32, mode=mode, check=True,
                          out=(X, e, lr, li, m), Q_packed=Qp, q_offs=qoffs, x_offs=xoffs,
                          e_offs=eoffs)
        outs.append((X.cpu().numpy().copy(), e.cpu().numpy().copy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    Xh, eh, lrh, lih = X.cpu().numpy(), e.cpu().numpy(), lr.cpu().numpy(), li.cpu().numpy()
    for i, (T, s, a, Q) in enumerate(zip(Ts, sels, adv, Qs)):
        n, mi = int(ns[i]), int(m[i])
        Xo, eo, lro, lio = oracle.standard(T, Q=Q, select=s)
        assert Xo.shape == (n, mi)
        if mi == 0:
            continue
        Xi = Xh[xoffs[i]:xoffs[i] + n * mi].reshape(mi, n).T
        ei = eh[eoffs[i]:eoffs[i] + mi]
        np.testing.assert_array_equal(lrh[eoffs[i]:eoffs[i] + mi], lro)
        np.testing.assert_array_equal(lih[eoffs[i]:eoffs[i] + mi], lio)
        assert np.isfinite(Xi).all()
        de, rel = compare_canonical(Xo, eo, Xi, ei, lio)
        assert de <= 1, (i, de)
        assert rel <= (1e-3 if a else 1e-10), (i, n, rel)
        A = T if Q is None else Q @ T @ Q.T
        r = standard_residuals(A, Xi, lro, lio)
        assert r.max() <= 10 * n, (i, r.max())
    # the gaps between the outputs are untouched
    gaps = np.ones(xa, bool)
    for i in range(len(Ts)):
        gaps[xoffs[i]:xoffs[i] + int(ns[i] * m[i])] = False
    assert np.isnan(Xh[gaps]).all()
