"""Batched pencils (evec_batched_generalized: the persistent kernel's pencil
variant) against the CPU oracle, pencil by pencil: (alpha, beta)
bit-identical, exponents +-1, columns within 1e-10 normwise relative,
normalised residual ||beta S y - alpha T y||_1 / ((|beta| ||S||_1 +
|alpha| ||T||_1) ||y||_1 u) <= 10 n, zeros below each block; mixed sizes,
selections, every tile, edge sizes and errors."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads
from evec_checks import canonical_norms, compare_canonical, generalized_residuals

pytestmark = pytest.mark.gpu


def _batch(sizes, seed, fraction=None):
    pairs, sels = [], []
    for i, n in enumerate(sizes):
        S, T, blocks = workloads.generalized_pair(int(n), seed=seed + i)
        pairs.append((S, T))
        if fraction is None:
            sels.append(None)
        else:
            sels.append(workloads.random_eigen_selection(int(n), blocks, fraction, seed=seed + 500 + i))
    return pairs, sels


def _check(pairs, sels, outs, rel_tol=1e-10, Zs=None):
    worst = 0.0
    for i, ((S, T), sel, out) in enumerate(zip(pairs, sels, outs)):
        X, e, ar, ai, be = (t.cpu().numpy() for t in out)
        Z = None if Zs is None else Zs[i]
        Xo, eo, aro, aio, beo = oracle.generalized(S, T, Z, select=sel)
        assert X.shape == Xo.shape
        if Xo.shape[1] == 0:
            continue
        np.testing.assert_array_equal(ar, aro)
        np.testing.assert_array_equal(ai, aio)
        np.testing.assert_array_equal(be, beo)
        assert np.isfinite(X).all()
        nr = canonical_norms(X, ai)
        assert nr.min() >= 1.0 and nr.max() < 2.0
        de, rel = compare_canonical(Xo, eo, X, e, aio)
        assert de <= 1, de
        worst = max(worst, rel)
        r = generalized_residuals(S, T, X if Z is None else Z.T @ X, ar, ai, be)
        assert r.max() <= 10 * S.shape[0], r.max()
    assert worst <= rel_tol, worst
    return worst


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_batched_pencils_tiles(tile):
    sizes = workloads.batch_sizes(24, seed=31, lo=8, hi=200)
    pairs, sels = _batch(sizes, seed=1000 + tile)
    outs = ev.batched_generalized(pairs, tile=tile)
    _check(pairs, sels, outs)


def test_batched_pencils_selection_and_edges():
    sizes = [1, 2, 3, 40, 130, 7, 64, 65, 250]
    pairs, sels = _batch(sizes, seed=77, fraction=0.3)
    sels[1] = np.zeros(2, np.uint8)          # nothing selected in one pencil
    outs = ev.batched_generalized(pairs, selects=sels)
    _check(pairs, sels, outs)
    # the selected columns agree with the same columns of the full result
    full = ev.batched_generalized(pairs)
    for (S, T), sel, o, f in zip(pairs, sels, outs, full):
        if sel is None or not sel.any():
            continue
        n = S.shape[0]
        cols, col, i = [], 0, 0
        while i < n:
            sz = 2 if i + 1 < n and S[i + 1, i] != 0.0 else 1
            if sel[i] or (sz == 2 and sel[i + 1]):
                cols.extend(range(col, col + sz))
            col += sz
            i += sz
        Xf, ef, aif = (f[k].cpu().numpy() for k in (0, 1, 3))
        de, rel = compare_canonical(Xf[:, cols], ef[cols], o[0].cpu().numpy(),
                                    o[1].cpu().numpy(), aif[cols])
        assert de == 0 and rel <= 1e-13, (de, rel)


def test_batched_pencils_match_single_pencil_path():
    # the persistent kernel and the single-pencil launches run the same
    # per-tile steps: results agree to rounding
    sizes = [90, 150, 33]
    pairs, sels = _batch(sizes, seed=5)
    outs = ev.batched_generalized(pairs, tile=32)
    for (S, T), out in zip(pairs, outs):
        dS = torch.from_numpy(np.asfortranarray(S)).cuda()
        dT = torch.from_numpy(np.asfortranarray(T)).cuda()
        X1, e1, ar1, ai1, be1 = ev.generalized(dS, dT, None, tile=32, check=True)
        np.testing.assert_array_equal(out[2].cpu().numpy(), ar1.cpu().numpy())
        np.testing.assert_array_equal(out[4].cpu().numpy(), be1.cpu().numpy())
        de, rel = compare_canonical(X1.cpu().numpy(), e1.cpu().numpy(), out[0].cpu().numpy(),
                                    out[1].cpu().numpy(), ai1.cpu().numpy())
        assert de <= 1 and rel <= 1e-12, (de, rel)


def test_batched_pencils_errors():
    sizes = [40, 60, 30]
    pairs, _ = _batch(sizes, seed=9)
    S1, T1 = pairs[1]
    bad = T1.copy()
    bad[5, 50] = np.nan                      # T of the second pencil
    pairs_bad = [pairs[0], (S1, bad), pairs[2]]
    with pytest.raises(ev.EvecError) as ei:
        ev.batched_generalized(pairs_bad)
    assert ei.value.status == ev.EVEC_ENONFINITE
    assert ei.value.bad == 40 * 40 + 5 + 50 * 60      # offset in the packed T
    # a slice count outside 2..8 is refused
    Sp, ns, offs = ev.pack_batch([S for S, _ in pairs])
    Tp, _, _ = ev.pack_batch([T for _, T in pairs])
    h = ev.handle(0)
    opts = ev._opts(0, False, "split", 9)
    st = ev.lib().evec_batched_generalized(h.ptr, 3, ev._np_ptr(ns), Sp.data_ptr(),
                                           ev._np_ptr(offs), Tp.data_ptr(), ev._np_ptr(offs),
                                           None, None, None, None, None, None, None, None,
                                           ctypes.byref(opts))
    assert st == ev.EVEC_EINVAL
    # the handle stays usable
    _check(pairs, [None] * 3, ev.batched_generalized(pairs))


def _unpack(ns, out):
    X, e, ar, ai, be, m = out
    res, xo, eo = [], 0, 0
    for n, mi in zip(ns, m):
        n, mi = int(n), int(mi)
        res.append((X[xo:xo + n * mi].view(mi, n).t(), e[eo:eo + mi], ar[eo:eo + mi],
                    ai[eo:eo + mi], be[eo:eo + mi]))
        xo += n * mi
        eo += mi
    return res


def test_batched_pencils_graph_replay():
    """The same call again replays the captured launch (bit-identical);
    new values off the three central diagonals keep the plans and are read
    by the replay; new diagonal values rebuild the plans."""
    sizes = workloads.batch_sizes(40, seed=77, lo=8, hi=300)
    pairs, sels = _batch(sizes, seed=7700, fraction=0.4)
    Sp, ns, soffs = ev.pack_batch([S for S, _ in pairs])
    Tp, _, toffs = ev.pack_batch([T for _, T in pairs])
    sel = np.concatenate([np.ascontiguousarray(s, dtype=np.uint8) for s in sels])
    out = ev.batched_generalized_packed(Sp, Tp, ns, soffs, toffs, sel, check=True)
    first = [t.clone() for t in out[:5]]
    _check(pairs, sels, _unpack(ns, out))
    out2 = ev.batched_generalized_packed(Sp, Tp, ns, soffs, toffs, sel, check=True, out=out)
    for a, b in zip(first, out2[:5]):
        assert torch.equal(a, b)
    # halve every entry above the superdiagonal of S and T in place
    pairs2 = []
    for (S, T), so, to, n in zip(pairs, soffs, toffs, ns):
        n = int(n)
        S2, T2 = np.array(S, copy=True), np.array(T, copy=True)
        iu = np.triu_indices(n, 2)
        S2[iu] *= 0.5
        T2[iu] *= 0.5
        Sp[int(so):int(so) + n * n] = torch.from_numpy(np.asfortranarray(S2).ravel(order="F"))
        Tp[int(to):int(to) + n * n] = torch.from_numpy(np.asfortranarray(T2).ravel(order="F"))
        pairs2.append((S2, T2))
    out3 = ev.batched_generalized_packed(Sp, Tp, ns, soffs, toffs, sel, check=True, out=out)
    _check(pairs2, sels, _unpack(ns, out3))
    # a new diagonal of T in the first pencil: new plans (beta changes)
    S3, T3 = pairs2[0]
    T3 = np.array(T3, copy=True)
    n0 = int(ns[0])
    T3[np.arange(n0), np.arange(n0)] *= 2.0
    Tp[int(toffs[0]):int(toffs[0]) + n0 * n0] = torch.from_numpy(np.asfortranarray(T3).ravel(order="F"))
    pairs3 = [(S3, T3)] + pairs2[1:]
    out4 = ev.batched_generalized_packed(Sp, Tp, ns, soffs, toffs, sel, check=True, out=out)
    _check(pairs3, sels, _unpack(ns, out4))


def test_batched_pencils_with_z():
    """X_i = Z_i Y_i for the pencils given a Z (every other one), Y_i for the
    rest; against the oracle's back-transformed vectors."""
    sizes = workloads.batch_sizes(30, seed=88, lo=8, hi=260)
    pairs, sels = _batch(sizes, seed=8800, fraction=0.5)
    Zs = [workloads.householder_orthogonal(int(n), seed=8900 + i) if i % 2 == 0 else None
          for i, n in enumerate(sizes)]
    outs = ev.batched_generalized(pairs, sels, Zs=Zs)
    _check(pairs, sels, outs, Zs=Zs)
    # Z_packed without offsets is refused
    Sp, ns, offs = ev.pack_batch([S for S, _ in pairs])
    Tp, _, _ = ev.pack_batch([T for _, T in pairs])
    h = ev.handle(0)
    opts = ev._opts(0, False, "fp64", 0)
    st = ev.lib().evec_batched_generalized(h.ptr, len(ns), ev._np_ptr(ns), Sp.data_ptr(),
                                           ev._np_ptr(offs), Tp.data_ptr(), ev._np_ptr(offs),
                                           Sp.data_ptr(), None, None, None, None, None, None,
                                           None, ctypes.byref(opts))
    assert st == ev.EVEC_EINVAL


def test_batched_pencils_tile_tuning():
    """tile 0: each size class gets the fastest of 16 / 32 / 64 on its first
    use (timed on up to eight of its pencils); the tuned batch matches the
    oracle; a table set by hand is used as given."""
    h = ev.handle(0)
    for c in range(ev.SIZE_CLASSES):
        assert ev.lib().evec_tune_set(h.ptr, 2, c, 0) == ev.EVEC_OK
    sizes = workloads.batch_sizes(40, seed=99, lo=16, hi=600)
    pairs, sels = _batch(sizes, seed=9900, fraction=0.5)
    outs = ev.batched_generalized(pairs, sels)
    table = ev.tune_table(0, "pencil")
    classes = {0 if n <= 64 else 1 if n <= 128 else 2 if n <= 256 else 3 if n <= 512 else 4
               for n in sizes}
    for c in range(ev.SIZE_CLASSES):
        assert (table[c] in (16, 32, 64)) if c in classes else table[c] == 0, table
    _check(pairs, sels, outs)
    ev.set_tune_table([16] * ev.SIZE_CLASSES, 0, "pencil")
    assert ev.tune_table(0, "pencil") == [16] * ev.SIZE_CLASSES
    _check(pairs, sels, ev.batched_generalized(pairs, sels))
    with pytest.raises(ev.EvecError):
        ev.set_tune_table([100] * ev.SIZE_CLASSES, 0, "pencil")
    for c in range(ev.SIZE_CLASSES):
        assert ev.lib().evec_tune_set(h.ptr, 2, c, 0) == ev.EVEC_OK


@pytest.mark.parametrize("tile", [32, 64])
def test_batched_pencils_split(tile):
    """Split mode: the updates as one split product of [S_rs T_rs] against
    [beta X; -alpha X] per step, in the persistent kernel; with and without
    Z, against the oracle at the FP64 bar."""
    sizes = workloads.batch_sizes(30, seed=111 + tile, lo=8, hi=400)
    pairs, sels = _batch(sizes, seed=11100 + tile, fraction=0.5)
    outs = ev.batched_generalized(pairs, sels, tile=tile, mode="split")
    _check(pairs, sels, outs)
    Zs = [workloads.householder_orthogonal(int(n), seed=11200 + i) if i % 3 == 0 else None
          for i, n in enumerate(sizes)]
    outs = ev.batched_generalized(pairs, sels, tile=tile, mode="split", Zs=Zs)
    _check(pairs, sels, outs, Zs=Zs)
