"""Batched mode (evec_batched): many independent Schur forms in one persistent
launch, against the CPU oracle matrix by matrix, with the parity bar of the
single-matrix tests (exponents +-1; columns within 1e-10 normwise relative on
well-conditioned inputs, 1e-3 on the clustered adversarial ones; residual
<= 10 n)."""
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


def _check_against_oracle(Ts, sels, adv, res):
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
        assert rel <= (1e-3 if a else 1e-10), (T.shape[0], rel)
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
    with pytest.raises(ev.EvecError) as ei:      # split precision: not in batched mode
        ev.batched_packed(Tp, ns, offs, mode="split")
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
