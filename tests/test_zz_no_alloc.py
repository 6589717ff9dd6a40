"""evec_standard_noalloc: the entry point for callers that cannot allocate GPU
memory while they run (a serving process whose memory pool owns the device,
code where a cudaMalloc would synchronise or fail, a fixed memory budget).
It keeps all scratch in one fixed array inside the library.

Called here through the C ABI, several times in a row on different inputs
(so each call starts from whatever the previous one left in the shared
array), and checked against the regular entry point evec_standard and
against the CPU oracle, within the parity tolerance of the GPU tests
(exponents +-1, columns within 1e-10 relative on well-conditioned inputs;
on the clustered adversarial input exponents +-1 and columns within 1e-3,
since their forward error grows like ||T|| / gap * u).  Also checked: the
device memory in use does not change across a call, a non-finite entry is
reported through the status word in the shared array with its index and
leaves the next call correct, and the largest plan the array takes
(n = 512 in 16-row tiles) fits.  This file is collected last, and it also
passes on its own in a fresh process, where its first call sets up the
array's device address.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2002_05024_b300 as ev
import workloads
from evec_checks import compare_canonical, standard_residuals

pytestmark = pytest.mark.gpu


def _noalloc(dT, n, ldt, sel, m, tile):
    L = ev.lib()
    f = L.evec_standard_noalloc
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [i64, p, i64, p, p, i64, p, ctypes.c_int, p, ctypes.POINTER(i64)]
    f.restype = ctypes.c_int
    X = torch.full((max(m, 1), n), np.nan, dtype=torch.float64, device="cuda").t()
    e = torch.zeros(max(m, 1), dtype=torch.int32, device="cuda")
    bad = i64(-1)
    st = f(n, dT.data_ptr(), ldt, None if sel is None else sel.ctypes.data_as(p), X.data_ptr(),
           n, e.data_ptr(), int(tile), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
           ctypes.byref(bad))
    return st, X[:, :m], e[:m], bad.value


def _run(T, select=None, tile=0):
    n = T.shape[0]
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    sel = None if select is None else np.ascontiguousarray(select, dtype=np.uint8)
    m = ev.count(dT, sel)
    return _noalloc(dT, n, n, sel, m, tile)


def _regular(T, select=None, tile=0):
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    X, e, lr, li = ev.standard(dT, select=select, tile=tile, check=True)
    return X.cpu().numpy(), e.cpu().numpy(), lr.cpu().numpy(), li.cpu().numpy()


def _check(T, sel, tile, col_tol):
    st, X, e, _ = _run(T, sel, tile)
    assert st == ev.EVEC_OK, ev.strerror(st)
    torch.cuda.synchronize()
    Xn, en = X.cpu().numpy(), e.cpu().numpy()
    Xr, er, lr, li = _regular(T, sel, tile)
    Xo, eo, _, _ = oracle.standard(T, select=sel)
    assert Xn.shape == Xr.shape == Xo.shape
    assert np.isfinite(Xn).all()
    de, rel = compare_canonical(Xr, er, Xn, en, li)
    assert de <= 1 and rel <= col_tol, ("vs evec_standard", de, rel)
    de, rel = compare_canonical(Xo, eo, Xn, en, li)
    assert de <= 1 and rel <= col_tol, ("vs oracle", de, rel)
    res = standard_residuals(T, Xn, lr, li)
    assert res.max() <= 10 * T.shape[0], res.max()


def test_noalloc_matches_regular_entry_point_and_oracle_in_a_row():
    T1, _ = workloads.config0_schur(300, seed=901)
    T2, blocks2 = workloads.config0_schur(200, seed=902)
    sel2 = workloads.random_eigen_selection(200, blocks2, 0.35, seed=903)
    for T, sel, tile in ((T1, None, 64), (T2, sel2, 32), (T1, None, 128)):
        _check(T, sel, tile, 1e-10)


def test_noalloc_adversarial_and_largest_plan():
    # clustered eigenvalues with large upper entries: the per-column
    # power-of-two scaling does the work (an unscaled solve overflows)
    Ta, _ = workloads.adversarial_schur(400, seed=905)
    _, overflowed = oracle.naive_standard(Ta)
    assert overflowed > 0
    _check(Ta, None, 32, 1e-3)
    # n = 512 in 16-row tiles: the most tiles, so the largest scratch layout
    Tb, _ = workloads.config0_schur(512, seed=906)
    _check(Tb, None, 16, 1e-10)


def test_noalloc_leaves_device_memory_unchanged():
    T, _ = workloads.config0_schur(256, seed=907)
    n = T.shape[0]
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    m = ev.count(dT, None)
    st, _, _, _ = _noalloc(dT, n, n, None, m, 64)      # loads every kernel it uses
    assert st == ev.EVEC_OK
    X = torch.empty((m, n), dtype=torch.float64, device="cuda").t()
    e = torch.empty(m, dtype=torch.int32, device="cuda")
    f = ev.lib().evec_standard_noalloc
    bad = ctypes.c_int64(-1)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        st = f(n, dT.data_ptr(), n, None, X.data_ptr(), n, e.data_ptr(), 64,
               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(bad))
        assert st == ev.EVEC_OK
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_reports_nonfinite_entry_then_recovers():
    T, _ = workloads.config0_schur(240, seed=908)
    bad_T = np.array(T, order="F", copy=True)
    i, j = 17, 201                      # strictly upper: found by the norm kernel
    bad_T[i, j] = np.nan
    st, _, _, bad = _run(bad_T, None, 32)
    assert st == ev.EVEC_ENONFINITE, ev.strerror(st)
    assert bad == i + j * 240
    # the next call starts from the array as the failed one left it
    _check(T, None, 32, 1e-10)


def test_noalloc_rejects_too_large():
    T, _ = workloads.config0_schur(513, seed=904)
    st, _, _, _ = _run(T)
    assert st == ev.EVEC_ECAPACITY
    assert "EVEC_ECAPACITY" in ev.strerror(st)
