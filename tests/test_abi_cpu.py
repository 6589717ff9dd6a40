"""CPU checks of the C ABI: the library loads, exports every entry point the
headers declare, plans correctly on the host, and refuses to run without a
GPU (there is no CPU fallback)."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_2002_05024_b300 as ev
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(evec_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    ev.lib()
    names = _declared_functions()
    assert "evec_standard" in names and "evec_sync" in names
    out = subprocess.run(["nm", "-D", "--defined-only", ev.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(ev.lib(), n)


def test_checked_build_exports_the_same_symbols():
    from paper_2002_05024_b300 import build as b
    b.build(checked=True)
    names = _declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", ev.CHECK_LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert not [n for n in names if n not in exported]
    # the flag itself, without a GPU
    Lc = ctypes.CDLL(ev.CHECK_LIB_PATH)
    assert Lc.evec_checked_build() == 1
    assert ev.lib().evec_checked_build() == 0


def test_strerror_names_every_status():
    for s in range(10):
        assert ev.strerror(s).startswith(ev.STATUS[s])


def _diags(T):
    return (np.ascontiguousarray(np.diagonal(T)), np.ascontiguousarray(np.diagonal(T, -1)),
            np.ascontiguousarray(np.diagonal(T, 1)))


@pytest.mark.parametrize("nb", [16, 17, 32, 64, 100, 128, 256, 512])
@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 300, 1029])
def test_plan_tiles_never_split_a_pair(n, nb):
    T, blocks = workloads.config0_schur(n, seed=n * 7 + nb)
    m, ts = ev.plan_query(*_diags(T), None, nb)
    assert m == n
    assert ts[0] == 0 and ts[-1] == n
    sizes = np.diff(ts)
    assert sizes.max() <= nb and (sizes[:-1] >= nb - 1).all() and sizes.min() >= 1
    pair_seconds = {p + 1 for p, sz in blocks if sz == 2}
    for b in ts[1:-1]:
        assert b not in pair_seconds


def test_plan_column_count_matches_oracle():
    T, blocks = workloads.config0_schur(500, seed=11)
    for frac in (0.0, 0.1, 0.35, 1.0):
        sel = workloads.random_eigen_selection(500, blocks, frac, seed=int(frac * 100))
        m, _ = ev.plan_query(*_diags(T), sel, 64)
        assert m == oracle.count(T, sel)


def test_plan_rejects_bad_forms():
    S = np.triu(np.ones((4, 4)))
    S[1, 0] = -1.0
    S[2, 1] = -1.0
    with pytest.raises(ev.EvecError) as e:
        ev.plan_query(*_diags(S), None, 16)
    assert e.value.status == ev.EVEC_ENOTSCHUR and e.value.bad == 1
    S = np.array([[1.0, 2.0], [-1.0, 1.5]])
    with pytest.raises(ev.EvecError) as e:
        ev.plan_query(*_diags(S), None, 16)
    assert e.value.status == ev.EVEC_ENOTSCHUR
    S = np.triu(np.ones((3, 3)))
    S[1, 1] = np.nan
    with pytest.raises(ev.EvecError) as e:
        ev.plan_query(*_diags(S), None, 16)
    assert e.value.status == ev.EVEC_ENONFINITE and e.value.bad == 1 + 1 * 3
    S[1, 1] = 2.0 ** 1001
    with pytest.raises(ev.EvecError) as e:
        ev.plan_query(*_diags(S), None, 16)
    assert e.value.status == ev.EVEC_EINVAL
    with pytest.raises(ev.EvecError) as e:
        ev.plan_query(*_diags(np.eye(3)), None, 8)      # tile below 16
    assert e.value.status == ev.EVEC_EINVAL


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert ev.lib().evec_create(ctypes.byref(h), 0, None) == ev.EVEC_ECUDA
    # the device entry points refuse a NULL handle before touching anything
    assert ev.lib().evec_standard(None, 4, None, 4, None, 4, None, None, 4, None, None,
                                  None, None) == ev.EVEC_EINVAL


def test_opts_defaults_in_the_documented_field_order():
    # evec_opts as the header lays it out: {mode, tile, slices, refine,
    # check}; the defaults (those of opt == NULL) set only refine
    class Opts(ctypes.Structure):
        _fields_ = [("mode", ctypes.c_int), ("tile", ctypes.c_int), ("slices", ctypes.c_int),
                    ("refine", ctypes.c_int), ("check", ctypes.c_int)]

    assert [f[0] for f in ev._Opts._fields_] == [f[0] for f in Opts._fields_]
    o = Opts(7, 7, 7, 7, 7)
    f = ctypes.CDLL(ev.LIB_PATH).evec_opts_default   # a private prototype
    f.argtypes = [ctypes.POINTER(Opts)]
    f.restype = None
    f(ctypes.byref(o))
    assert (o.mode, o.tile, o.slices, o.refine, o.check) == (0, 0, 0, 1, 0)
    f(None)                                   # a NULL pointer is ignored
