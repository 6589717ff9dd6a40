"""evec_standard_noalloc: the entry point for callers that cannot allocate GPU
memory while they run (a serving process whose memory pool owns the device,
code where a cudaMalloc would synchronise or fail, a fixed memory budget).
It keeps all scratch in one fixed array inside the library.

Called here through the C ABI, twice in a row on different inputs (so a
second call starts from whatever the first left in the shared array), and
checked against the regular entry point evec_standard within the parity
tolerance of the GPU tests (exponents +-1, columns within 1e-10 relative).
This file is collected last, and it also passes on its own in a fresh
process, where its first call sets up the array's device address.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2002_05024_b300 as ev
import workloads
from evec_checks import compare_canonical

pytestmark = pytest.mark.gpu


def _noalloc(T, select=None, tile=0):
    L = ev.lib()
    f = L.evec_standard_noalloc
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [i64, p, i64, p, p, i64, p, ctypes.c_int, p, ctypes.POINTER(i64)]
    f.restype = ctypes.c_int
    n = T.shape[0]
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    sel = None if select is None else np.ascontiguousarray(select, dtype=np.uint8)
    m = ev.count(dT, sel)
    X = torch.full((m, n), np.nan, dtype=torch.float64, device="cuda").t()
    e = torch.zeros(m, dtype=torch.int32, device="cuda")
    bad = i64(-1)
    st = f(n, dT.data_ptr(), n, None if sel is None else sel.ctypes.data_as(p), X.data_ptr(),
           n, e.data_ptr(), int(tile), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
           ctypes.byref(bad))
    return st, X, e, bad.value


def _regular(T, select=None, tile=0):
    dT = torch.from_numpy(np.asfortranarray(T)).cuda()
    X, e, lr, li = ev.standard(dT, select=select, tile=tile, check=True)
    return X.cpu().numpy(), e.cpu().numpy(), li.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice():
    T1, _ = workloads.config0_schur(300, seed=901)
    T2, blocks2 = workloads.config0_schur(200, seed=902)
    sel2 = workloads.random_eigen_selection(200, blocks2, 0.35, seed=903)
    for T, sel, tile in ((T1, None, 64), (T2, sel2, 32)):
        st, X, e, _ = _noalloc(T, sel, tile)
        assert st == ev.EVEC_OK, ev.strerror(st)
        torch.cuda.synchronize()
        Xr, er, li = _regular(T, sel, tile)
        Xn, en = X.cpu().numpy(), e.cpu().numpy()
        assert Xn.shape == Xr.shape
        assert np.isfinite(Xn).all()
        de, rel = compare_canonical(Xr, er, Xn, en, li)
        assert de <= 1 and rel <= 1e-10, (de, rel)


def test_noalloc_rejects_too_large():
    T, _ = workloads.config0_schur(513, seed=904)
    st, _, _, _ = _noalloc(T)
    assert st == ev.EVEC_ECAPACITY
    assert "EVEC_ECAPACITY" in ev.strerror(st)
