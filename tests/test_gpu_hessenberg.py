"""Hessenberg reduction on the GPU (evec_hessenberg: panels of 32 columns,
compact WY updates) against the oracle's unblocked reduction: H and Q
element by element within a rounding bound (16 n sqrt(n) u, relative to
max |A| for H), exact zeros below the subdiagonal, orthogonality and the
backward error of Q H Q^T; a leading dimension above n, the symmetric case,
errors, and the benchmark's size n = 4096 through its invariants."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _gpu(A, calc_q=True, mode="fp64"):
    dA = torch.from_numpy(np.asfortranarray(A)).cuda()
    H, Q = ev.hessenberg(dA, calc_q=calc_q, check=True, mode=mode)
    torch.cuda.synchronize()
    return H.cpu().numpy(), (Q.cpu().numpy() if Q is not None else None)


def _bound(n):
    return 16 * n * np.sqrt(n) * U


@pytest.mark.parametrize("n", [1, 2, 3, 33, 100, 257, 600])
def test_hessenberg_against_oracle(n):
    A = np.random.default_rng(n).standard_normal((n, n))
    H, Q = _gpu(A)
    Ho, Qo, _ = oracle.hessenberg(A)
    nrm = np.abs(A).max()
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.abs(H - Ho).max() <= _bound(n) * nrm, np.abs(H - Ho).max()
    assert np.abs(Q - Qo).max() <= _bound(n), np.abs(Q - Qo).max()
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 8 * n * U
    assert np.abs(Q @ H @ Q.T - A).max() <= _bound(n) * nrm


def test_hessenberg_leading_dimension_and_no_q():
    n, ld = 150, 173
    A = np.random.default_rng(5).standard_normal((n, n))
    buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    dA = buf.t()[:n, :]                      # column-major, leading dimension ld
    dA.copy_(torch.from_numpy(A))
    assert dA.stride() == (1, ld)
    H, Q = ev.hessenberg(dA, calc_q=False, check=True, overwrite=True)
    assert Q is None and H.data_ptr() == dA.data_ptr()
    Ho, _, _ = oracle.hessenberg(A)
    assert np.abs(H.cpu().numpy() - Ho).max() <= _bound(n) * np.abs(A).max()
    # the rows between n and ld are not touched
    assert torch.all(buf.t()[n:, :] == 0.0)


def test_hessenberg_symmetric_gives_tridiagonal():
    n = 300
    B = np.random.default_rng(9).standard_normal((n, n))
    A = B + B.T
    H, Q = _gpu(A)
    nrm = np.abs(A).max()
    assert np.abs(np.triu(H, 2)).max() <= _bound(n) * nrm
    assert np.abs(H - H.T).max() <= _bound(n) * nrm


def test_hessenberg_errors():
    n = 50
    A = np.random.default_rng(1).standard_normal((n, n))
    bad = A.copy()
    bad[4, 7] = np.nan
    with pytest.raises(ev.EvecError) as ei:
        _gpu(bad)
    assert ei.value.status == ev.EVEC_ENONFINITE and ei.value.bad == 4 + 7 * n
    bad = A.copy()
    bad[2, 3] = 2.0 ** 1001
    with pytest.raises(ev.EvecError) as ei:
        _gpu(bad)
    assert ei.value.status == ev.EVEC_EINVAL and ei.value.bad == 2 + 3 * n
    H, Q = _gpu(A)   # the handle stays usable
    assert np.abs(Q @ H @ Q.T - A).max() <= _bound(n) * np.abs(A).max()


def test_hessenberg_full_size_invariants():
    # n = 4096 (the benchmark's size): zero pattern, orthogonality and the
    # backward error, checked with the host BLAS
    n = 4096
    A = np.random.default_rng(2020).standard_normal((n, n))
    H, Q = _gpu(A)
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 8 * n * U
    R = Q @ H @ Q.T - A
    assert np.abs(R).max() <= _bound(n) * np.abs(A).max(), np.abs(R).max()


def test_hessenberg_panel_paths_agree():
    # the six-launch panel path (used when a device refuses the cooperative
    # launch) against the oracle and the cooperative path
    n = 333
    A = np.random.default_rng(31).standard_normal((n, n))
    h = ev.handle(0)
    out = {}
    for coop in (False, True):
        h.hessenberg_panel(coop)
        try:
            out[coop] = _gpu(A)
        finally:
            h.hessenberg_panel(True)
    Ho, Qo, _ = oracle.hessenberg(A)
    nrm = np.abs(A).max()
    for coop, (H, Q) in out.items():
        assert np.all(np.tril(H, -2) == 0.0)
        assert np.abs(H - Ho).max() <= _bound(n) * nrm, (coop, np.abs(H - Ho).max())
        assert np.abs(Q - Qo).max() <= _bound(n), coop
    assert np.abs(out[False][0] - out[True][0]).max() <= _bound(n) * nrm


@pytest.mark.parametrize("e2", [-900, 900])
def test_hessenberg_extreme_scales(e2):
    # entries near 2^900 and 2^-900: every column norm takes the scaled
    # branch (the plain sum of squares would overflow or lose digits);
    # scaling by a power of two commutes with the reduction
    n = 200
    A = np.random.default_rng(77).standard_normal((n, n))
    H, Q = _gpu(np.ldexp(A, e2))
    H = np.ldexp(H, -e2)
    Ho, Qo, _ = oracle.hessenberg(A)
    nrm = np.abs(A).max()
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.abs(H - Ho).max() <= _bound(n) * nrm, np.abs(H - Ho).max()
    assert np.abs(Q - Qo).max() <= _bound(n)
    assert np.abs(Q @ H @ Q.T - A).max() <= _bound(n) * nrm


def test_hessenberg_of_hessenberg_input_is_exact():
    # every column is already zero below the subdiagonal: every reflector
    # is the identity (tau = 0), so H = A and Q = I exactly
    n = 150
    A = np.triu(np.random.default_rng(12).standard_normal((n, n)), -1)
    H, Q = _gpu(A)
    np.testing.assert_array_equal(H, A)
    np.testing.assert_array_equal(Q, np.eye(n))


def test_hessenberg_several_chunks_per_cta():
    # n = 5000: more rows than 32 per CTA of the cooperative panel, so each
    # CTA's product runs over several 32-row chunks; invariants with the
    # host BLAS
    n = 5000
    A = np.random.default_rng(5000).standard_normal((n, n))
    H, Q = _gpu(A)
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 8 * n * U
    R = Q @ H @ Q.T - A
    assert np.abs(R).max() <= _bound(n) * np.abs(A).max(), np.abs(R).max()


def test_panel_barrier_wait_runs_out_then_recovers():
    # failure detection without a fault: a wait limit of one poll makes the
    # cooperative panel's grid-barrier waits give up (the other CTAs are not
    # there yet); every CTA returns, evec_sync reports EVEC_ETIMEOUT, and
    # the next call with the built-in limit matches the oracle
    import ctypes
    n = 300
    A = np.random.default_rng(31).standard_normal((n, n))
    h = ev.handle(0)
    L = ev.lib()
    L.evec_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    L.evec_set_wait_limit.restype = ctypes.c_int
    assert L.evec_set_wait_limit(h.ptr, -1) == ev.EVEC_EINVAL
    assert L.evec_set_wait_limit(h.ptr, 1) == ev.EVEC_OK
    try:
        dA = torch.from_numpy(np.asfortranarray(A)).cuda()
        ev.hessenberg(dA, calc_q=True, check=False, overwrite=True)
        with pytest.raises(ev.EvecError) as ei:
            h.sync()
        assert ei.value.status == ev.EVEC_ETIMEOUT
    finally:
        assert L.evec_set_wait_limit(h.ptr, 0) == ev.EVEC_OK
    h.sync()                                   # the status was cleared
    H, Q = _gpu(A)
    Ho, Qo, _ = oracle.hessenberg(A)
    assert np.abs(H - Ho).max() <= _bound(n) * np.abs(A).max()
    assert np.abs(Q - Qo).max() <= _bound(n)


# --------------------------------------------------------------------------
# split precision (EVEC_SPLIT): the five large products of every panel's
# update through the split GEMM, at the FP64 path's bounds
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [3, 33, 100, 257, 600])
def test_hessenberg_split_against_oracle(n):
    A = np.random.default_rng(n + 1000).standard_normal((n, n))
    H, Q = _gpu(A, mode="split")
    Ho, Qo, _ = oracle.hessenberg(A)
    nrm = np.abs(A).max()
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.abs(H - Ho).max() <= _bound(n) * nrm, np.abs(H - Ho).max()
    assert np.abs(Q - Qo).max() <= _bound(n), np.abs(Q - Qo).max()
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 8 * n * U
    assert np.abs(Q @ H @ Q.T - A).max() <= _bound(n) * nrm
    # without Q
    H2, Q2 = _gpu(A, calc_q=False, mode="split")
    assert Q2 is None and np.abs(H2 - Ho).max() <= _bound(n) * nrm


@pytest.mark.parametrize("e2", [-900, 900])
def test_hessenberg_split_extreme_scales(e2):
    n = 200
    A = np.random.default_rng(78).standard_normal((n, n))
    H, Q = _gpu(np.ldexp(A, e2), mode="split")
    H = np.ldexp(H, -e2)
    Ho, Qo, _ = oracle.hessenberg(A)
    nrm = np.abs(A).max()
    assert np.abs(H - Ho).max() <= _bound(n) * nrm, np.abs(H - Ho).max()
    assert np.abs(Q - Qo).max() <= _bound(n)


def test_hessenberg_split_full_size_invariants():
    n = 4096
    A = np.random.default_rng(2021).standard_normal((n, n))
    H, Q = _gpu(A, mode="split")
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 8 * n * U
    R = Q @ H @ Q.T - A
    assert np.abs(R).max() <= _bound(n) * np.abs(A).max(), np.abs(R).max()
    with pytest.raises(ev.EvecError) as ei:   # a slice count outside 2..8
        ev.hessenberg(torch.from_numpy(np.asfortranarray(A[:64, :64])).cuda(), mode="split",
                      slices=9)
    assert ei.value.status == ev.EVEC_EINVAL
