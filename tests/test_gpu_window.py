"""Eigenvalue reordering's off-diagonal updates on the GPU
(evec_window_update: the left and right update tasks applying each
window's accumulator as FP64 products, or through the split-precision
GEMM) against the oracle's plain loops:
element by element within a dot-product rounding bound for chains of
overlapping windows of every kernel variant (k up to 256, ragged n), exact
results for permutation windows, the invariant Q T Q^T for disjoint
windows at the benchmark's size, edge windows and errors."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _dev(A):
    return torch.from_numpy(np.asfortranarray(A)).cuda()


def _gpu(T, Q, windows):
    dT = _dev(T)
    dQ = _dev(Q) if Q is not None else None
    ev.window_update(dT, dQ, windows, check=True)
    return dT.cpu().numpy(), (dQ.cpu().numpy() if dQ is not None else None)


def _bound(T, windows):
    kmax = max(Z.shape[0] for _, Z in windows)
    return 4 * kmax * len(windows) * U * max(1.0, np.abs(T).max())


@pytest.mark.parametrize("k,stride", [(17, 9), (32, 16), (64, 40), (100, 50), (128, 64),
                                      (200, 100), (256, 128)])
def test_window_chain_against_oracle(k, stride):
    n = 333 if k < 256 else 600
    T, blocks = workloads.config0_schur(n, seed=k)
    Q = workloads.householder_orthogonal(n, seed=k + 1)
    w = workloads.window_chain(n, k, stride, seed=k + 2, blocks=blocks)
    Tg, Qg = _gpu(T, Q, w)
    To, Qo = oracle.window_update(T, Q, w)
    assert np.abs(Tg - To).max() <= _bound(To, w), np.abs(Tg - To).max()
    assert np.abs(Qg - Qo).max() <= _bound(Qo, w)


def test_permutation_window_exact():
    n, a, k = 150, 37, 45
    T, _ = workloads.config0_schur(n, seed=3)
    Q = workloads.householder_orthogonal(n, seed=4)
    perm = np.roll(np.arange(k), 7)
    P = np.zeros((k, k))
    P[perm, np.arange(k)] = 1.0
    Tg, Qg = _gpu(T, Q, [(a, P)])
    To, Qo = oracle.window_update(T, Q, [(a, P)])
    np.testing.assert_array_equal(Tg, To)
    np.testing.assert_array_equal(Qg, Qo)


def test_edge_windows_and_no_q():
    n = 97
    T, _ = workloads.config0_schur(n, seed=5)
    rng = np.random.default_rng(6)
    w = []
    for a, k in ((0, 1), (96, 1), (0, 97), (60, 37), (0, 33)):
        Z, _ = np.linalg.qr(rng.standard_normal((k, k)))
        w.append((a, Z))
    Tg, Qg = _gpu(T, None, w)
    To, _ = oracle.window_update(T, None, w)
    assert Qg is None
    assert np.abs(Tg - To).max() <= _bound(To, w)
    # no windows: nothing changes
    Tn, _ = _gpu(T, None, [])
    np.testing.assert_array_equal(Tn, T)


def test_disjoint_windows_full_size_invariant():
    # the benchmark's workload: n = 4096 with Q, disjoint windows of 128
    # tiling the diagonal (boundaries off 2x2 blocks): Q T Q^T unchanged and
    # Q orthogonal, with the host BLAS; three windows against the oracle
    n = 4096
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 100)
    w = workloads.window_chain(n, 128, 128, seed=workloads.SEED_BASE + 9, blocks=blocks)
    Tg, Qg = _gpu(T, Q, w)
    A = Q @ T @ Q.T
    assert np.abs(Qg @ Tg @ Qg.T - A).max() <= 64 * n * U * np.abs(A).max()
    assert np.abs(Qg.T @ Qg - np.eye(n)).max() <= 64 * n * U
    sub = [w[0], w[len(w) // 2], w[-1]]
    Ts, Qs = _gpu(T, Q, sub)
    To, Qo = oracle.window_update(T, Q, sub)
    assert np.abs(Ts - To).max() <= _bound(To, sub)
    assert np.abs(Qs - Qo).max() <= _bound(Qo, sub)


def test_window_errors():
    n = 50
    T, _ = workloads.config0_schur(n, seed=8)
    dT = _dev(T)
    for a, k in ((-1, 4), (48, 4), (0, 257)):
        if k > n:
            dT2 = _dev(np.eye(300))
            with pytest.raises(ev.EvecError) as ei:
                ev.window_update(dT2, None, [(a, np.eye(k))])
        else:
            with pytest.raises(ev.EvecError) as ei:
                ev.window_update(dT, None, [(a, np.eye(k))])
        assert ei.value.status == ev.EVEC_EINVAL
    # nothing was applied, and the handle stays usable
    np.testing.assert_array_equal(dT.cpu().numpy(), T)
    Tg, _ = _gpu(T, None, [(3, np.eye(5))])
    np.testing.assert_array_equal(Tg, T)


def _mixed_disjoint(n, seed):
    # disjoint windows of mixed sizes (one per kernel variant), in shuffled order
    rng = np.random.default_rng(seed)
    out, a = [], 5
    for k in (37, 64, 128, 200, 20, 256):
        if a + k > n:
            break
        Z, _ = np.linalg.qr(rng.standard_normal((k, k)))
        out.append((a, Z))
        a += k + int(rng.integers(0, 9))
    rng.shuffle(out)
    return out


def test_disjoint_set_against_oracle():
    n = 777
    T, _ = workloads.config0_schur(n, seed=41)
    Q = workloads.householder_orthogonal(n, seed=42)
    w = _mixed_disjoint(n, 43)
    dT, dQ = _dev(T), _dev(Q)
    ev.window_update(dT, dQ, w, check=True, disjoint=True)
    To, Qo = oracle.window_update(T, Q, w)
    assert np.abs(dT.cpu().numpy() - To).max() <= _bound(To, w)
    assert np.abs(dQ.cpu().numpy() - Qo).max() <= _bound(Qo, w)
    # without Q, and a zero-size window in the list
    dT = _dev(T)
    ev.window_update(dT, None, w + [(3, np.zeros((0, 0)))], check=True, disjoint=True)
    assert np.abs(dT.cpu().numpy() - To).max() <= _bound(To, w)


def test_disjoint_set_full_size_matches_sequential():
    # the benchmark's windows: the set path against the one-window-at-a-time
    # path (the same products, another order of the commuting updates)
    n = 4096
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 100)
    w = workloads.window_chain(n, 128, 128, seed=workloads.SEED_BASE + 9, blocks=blocks)
    Ts, Qs = _dev(T), _dev(Q)
    ev.window_update(Ts, Qs, w, check=True, disjoint=True)
    Tq, Qq = _dev(T), _dev(Q)
    ev.window_update(Tq, Qq, w, check=True)
    assert torch.abs(Ts - Tq).max().item() <= _bound(T, w[:2])
    assert torch.equal(Qs, Qq)   # Q's updates touch disjoint columns: same products


def test_disjoint_set_rejects_overlap():
    n = 60
    T, _ = workloads.config0_schur(n, seed=44)
    dT = _dev(T)
    with pytest.raises(ev.EvecError) as ei:
        ev.window_update(dT, None, [(0, np.eye(10)), (9, np.eye(5))], disjoint=True)
    assert ei.value.status == ev.EVEC_EINVAL
    np.testing.assert_array_equal(dT.cpu().numpy(), T)


# --------------------------------------------------------------------------
# split precision (EVEC_SPLIT): the products through the split GEMM
# --------------------------------------------------------------------------

def _gpu_split(T, Q, windows, disjoint=False):
    dT = _dev(T)
    dQ = _dev(Q) if Q is not None else None
    ev.window_update(dT, dQ, windows, check=True, disjoint=disjoint, mode="split")
    return dT.cpu().numpy(), (dQ.cpu().numpy() if dQ is not None else None)


@pytest.mark.parametrize("k,stride", [(17, 9), (64, 40), (128, 64), (200, 100), (256, 128)])
def test_window_chain_split_against_oracle(k, stride):
    # 8 slices of 7 bits: each product within k 2^-55 max|row| max|column|
    # of the exact one, inside the FP64 path's bound
    n = 333 if k < 256 else 600
    T, blocks = workloads.config0_schur(n, seed=k + 50)
    Q = workloads.householder_orthogonal(n, seed=k + 51)
    w = workloads.window_chain(n, k, stride, seed=k + 52, blocks=blocks)
    Tg, Qg = _gpu_split(T, Q, w)
    To, Qo = oracle.window_update(T, Q, w)
    assert np.abs(Tg - To).max() <= _bound(To, w), np.abs(Tg - To).max()
    assert np.abs(Qg - Qo).max() <= _bound(Qo, w)


def test_window_split_edges_disjoint_set_and_errors():
    n = 97
    T, _ = workloads.config0_schur(n, seed=55)
    rng = np.random.default_rng(56)
    w = []
    for a, k in ((0, 1), (96, 1), (0, 97), (60, 37), (0, 33)):
        Z, _ = np.linalg.qr(rng.standard_normal((k, k)))
        w.append((a, Z))
    Tg, _ = _gpu_split(T, None, w)
    To, _ = oracle.window_update(T, None, w)
    assert np.abs(Tg - To).max() <= _bound(To, w)
    # the disjoint set in split mode (applied in the order of first rows)
    n = 777
    T, _ = workloads.config0_schur(n, seed=57)
    Q = workloads.householder_orthogonal(n, seed=58)
    w = _mixed_disjoint(n, 59)
    Tg, Qg = _gpu_split(T, Q, w, disjoint=True)
    To, Qo = oracle.window_update(T, Q, w)
    assert np.abs(Tg - To).max() <= _bound(To, w)
    assert np.abs(Qg - Qo).max() <= _bound(Qo, w)
    # a slice count outside 2..8 is refused and nothing is applied
    dT = _dev(T)
    with pytest.raises(ev.EvecError) as ei:
        ev.window_update(dT, None, w, mode="split", slices=9)
    assert ei.value.status == ev.EVEC_EINVAL
    np.testing.assert_array_equal(dT.cpu().numpy(), T)


def test_window_split_full_size_invariant_and_fp64_agreement():
    # the benchmark's workload in split mode: Q T Q^T unchanged, Q
    # orthogonal, and the result within the FP64 bound of the FP64 path's
    n = 4096
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 100)
    w = workloads.window_chain(n, 128, 128, seed=workloads.SEED_BASE + 9, blocks=blocks)
    Tg, Qg = _gpu_split(T, Q, w)
    A = Q @ T @ Q.T
    assert np.abs(Qg @ Tg @ Qg.T - A).max() <= 64 * n * U * np.abs(A).max()
    assert np.abs(Qg.T @ Qg - np.eye(n)).max() <= 64 * n * U
    Tf, Qf = _gpu(T, Q, w)
    assert np.abs(Tg - Tf).max() <= _bound(T, w[:2])
    assert np.abs(Qg - Qf).max() <= _bound(Q, w[:2])
