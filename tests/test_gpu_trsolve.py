"""The robust triangular solve with many right-hand sides (evec_trsolve)
against the CPU oracle: exponents +-1, columns within 1e-10 normwise
relative after bringing both to one exponent, residual <= 10 n; the same
tiled steps as the eigenvectors with shift 0 (both update modes, every tile
path), right-hand sides that are zero or near the input limit, a matrix
whose unscaled solve overflows, edge sizes, in-place use, power-of-two
invariance and error reporting."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads

pytestmark = pytest.mark.gpu


def _well_conditioned(n, seed):
    T, blocks, _ = workloads.solve_system(n, 0, seed=seed)
    return T, blocks


def _gpu(T, B, tile=0, mode="fp64", slices=0):
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    dB = torch.from_numpy(np.asfortranarray(B)).cuda()
    X, e = ev.trsolve(dT, dB, tile=tile, check=True, mode=mode, slices=slices)
    torch.cuda.synchronize()
    return X.cpu().numpy(), e.cpu().numpy()


def _compare(T, B, X, e, rel_tol=1e-10):
    Xo, eo = oracle.trsolve(T, B)
    assert X.shape == Xo.shape and np.isfinite(X).all()
    nz = np.abs(B).max(axis=0) > 0
    assert np.all(X[:, ~nz] == 0.0) and np.all(e[~nz] == 0)
    worst = 0.0
    for j in np.nonzero(nz)[0]:
        de = int(eo[j]) - int(e[j])
        assert abs(de) <= 1, (j, eo[j], e[j])
        a = Xo[:, j]
        b = np.ldexp(X[:, j], de)
        worst = max(worst, np.abs(a - b).max() / np.abs(a).max())
        assert 1.0 <= np.abs(X[:, j]).max() < 2.0
    assert worst <= rel_tol, worst
    # residual of the GPU solution, in long double
    x = np.ldexp(X, -e.astype(np.int64)[None, :]).astype(np.longdouble)
    Tl = T.astype(np.longdouble)
    r = Tl @ x - B.astype(np.longdouble)
    T1 = np.abs(Tl).sum(axis=0).max()
    for j in np.nonzero(nz)[0]:
        res = np.abs(r[:, j]).sum() / (T1 * np.abs(x[:, j]).sum() * 2.0 ** -53)
        assert float(res) <= 10 * T.shape[0], (j, float(res))
    return worst


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("tile", [16, 32, 64, 128, 256, 512])
def test_trsolve_tiles_and_modes(tile, mode):
    n = 613
    T, _ = _well_conditioned(n, seed=500 + tile)
    rng = np.random.default_rng(tile)
    B = rng.standard_normal((n, 37))
    B[:, 5] = 0.0                               # a zero right-hand side
    B[:, 9] *= 2.0 ** 900                       # near the input limit
    B[:300, 11] = 0.0                           # rows above a point are zero
    X, e = _gpu(T, B, tile=tile, mode=mode)
    _compare(T, B, X, e)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_trsolve_growth_past_the_double_range(mode):
    # tiny pivots under a dense upper part: the unscaled solve overflows,
    # the robust one stays finite and matches the oracle
    n = 256
    rng = np.random.default_rng(7)
    T = np.triu(rng.uniform(0.5, 1.0, (n, n)), 1)
    T[np.arange(n), np.arange(n)] = np.ldexp(1.0, -40) * rng.uniform(1.0, 2.0, n)
    B = rng.standard_normal((n, 9))
    X, e = _gpu(T, B, tile=64, mode=mode)
    assert e.min() < -5000
    Xo, eo = oracle.trsolve(T, B)
    assert np.all(np.abs(eo - e) <= 1)
    for j in range(B.shape[1]):
        de = int(eo[j]) - int(e[j])
        a, b = Xo[:, j], np.ldexp(X[:, j], de)
        assert np.abs(a - b).max() / np.abs(a).max() <= 1e-6, j


def test_trsolve_edges_in_place_and_power_of_two():
    # n = 1 and 2, one right-hand side, none; an in-place solve; 2^k B gives
    # the same X and exponents lower by k
    for n in (1, 2, 3):
        T, _ = _well_conditioned(n, seed=40 + n)
        B = np.random.default_rng(n).standard_normal((n, 2))
        X, e = _gpu(T, B, tile=16)
        _compare(T, B, X, e)
    n = 300
    T, _ = _well_conditioned(n, seed=61)
    B = np.random.default_rng(62).standard_normal((n, 8))
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    dB = torch.from_numpy(np.asfortranarray(B)).cuda()
    e = torch.empty(8, dtype=torch.int32, device="cuda")
    ev.trsolve(dT, dB, tile=64, check=True, out=(dB, e))   # X is B
    X1, e1 = dB.cpu().numpy(), e.cpu().numpy()
    _compare(T, B, X1, e1)
    X2, e2 = _gpu(T, np.ldexp(B, 30), tile=64)
    np.testing.assert_array_equal(X1, X2)
    np.testing.assert_array_equal(e2, e1 - 30)
    empty = torch.empty((n, 0), dtype=torch.float64, device="cuda")
    Xe, ee = ev.trsolve(dT, empty)
    assert Xe.shape == (n, 0) and ee.shape == (0,)


def test_trsolve_errors():
    n = 120
    T, blocks = _well_conditioned(n, seed=81)
    B = np.ones((n, 4))
    bad = B.copy()
    bad[7, 2] = np.nan
    with pytest.raises(ev.EvecError) as ei:
        _gpu(T, bad, tile=32)
    assert ei.value.status == ev.EVEC_ENONFINITE and ei.value.bad == n * n + 7 + 2 * n
    bad = B.copy()
    bad[3, 1] = 2.0 ** 1001
    with pytest.raises(ev.EvecError) as ei:
        _gpu(T, bad, tile=32)
    assert ei.value.status == ev.EVEC_EINVAL
    T2 = T.copy()
    p = next(q for q, sz in blocks if sz == 2 and q + 2 < n)
    T2[p + 2, p + 1] = 0.25                     # two nonzero subdiagonal entries in a row
    with pytest.raises(ev.EvecError) as ei:
        _gpu(T2, B, tile=32)
    assert ei.value.status == ev.EVEC_ENOTSCHUR
    # the handle stays usable
    X, e = _gpu(T, B, tile=32)
    _compare(T, B, X, e)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_trsolve_full_size_sampled(mode):
    # the benchmark's solve: n = 4096, 4096 right-hand sides, tile 64; 24
    # sampled columns against the oracle
    n = 4096
    T, _, B = workloads.solve_system(n, n)
    X, e = _gpu(T, B, tile=0, mode=mode)
    assert np.isfinite(X).all()
    cols = np.sort(np.random.default_rng(9).choice(n, 24, replace=False))
    _compare(T, B[:, cols], X[:, cols], e[cols])
