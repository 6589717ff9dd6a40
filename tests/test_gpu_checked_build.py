"""The checked build (libevec_check.so, compiled with -DEVEC_CHECK): the
kernels test the row, column, tile and segment indices of their main
device accesses against the plan and would report EVEC_EBOUNDS at
evec_sync.  Here it runs the hot paths (FP64 and split with Q, the sweep,
tiles 16 to 256, selections, left eigenvectors, a pencil with Z, the
triangular solve, the batch) in a process of its own: no check may fire,
and every result must match the oracle at the usual bars."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
import numpy as np, torch
import paper_2002_05024_b300 as ev
ev.use_checked_build()
import oracle, workloads
from evec_checks import compare_canonical, column_groups
assert ev.lib().evec_checked_build() == 1

def dev(A):
    return None if A is None else torch.from_numpy(np.asfortranarray(A)).cuda()

def check(Xo, eo, lio, out, tol):
    X, e = out[0].cpu().numpy(), out[1].cpu().numpy()
    de, rel = compare_canonical(Xo, eo, X, e, lio)
    assert de <= 1 and rel <= tol, (de, rel)

n = 333
T, blocks = workloads.config0_schur(n, seed=71)
Q = workloads.householder_orthogonal(n, seed=72)
sel = workloads.random_eigen_selection(n, blocks, 0.4, seed=73)
Xo, eo, lro, lio = oracle.standard(T, Q=Q)
for tile in (16, 64, 256):
    for mode, refine in (("fp64", 0), ("split", 0), ("split", 1)):
        out = ev.standard(dev(T), dev(Q), tile=tile, mode=mode, refine=refine, check=True)
        check(Xo, eo, lio, out, 1e-10)
Xs, es, _, lis = oracle.standard(T, Q=Q, select=sel)
check(Xs, es, lis, ev.standard(dev(T), dev(Q), select=sel, tile=32, check=True), 1e-10)
Xl, el, _, lil = oracle.left(T, Q=Q)
check(Xl, el, lil, ev.left(dev(T), dev(Q), tile=64, mode="split", check=True), 1e-10)
S, Tp, _ = workloads.generalized_pair(300, seed=74)
Z = workloads.householder_orthogonal(300, seed=75)
Xg, eg, _, aig, _ = oracle.generalized(S, Tp, Z)
check(Xg, eg, aig, ev.generalized(dev(S), dev(Tp), dev(Z), tile=32, check=True), 1e-10)
Ts, _, B = workloads.solve_system(257, 40, seed=76)
Xt, et = oracle.trsolve(Ts, B)
out = ev.trsolve(dev(Ts), dev(B), tile=32, check=True)
Xg2, eg2 = out[0].cpu().numpy(), out[1].cpu().numpy()
for j in range(B.shape[1]):
    d = int(et[j]) - int(eg2[j])
    assert abs(d) <= 1
    a, b = Xt[:, j], np.ldexp(Xg2[:, j], d)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
Ts3 = [workloads.config0_schur(k, seed=80 + k)[0] for k in (40, 130, 257)]
outs = ev.batched(Ts3, tile=32)
for Tb, o in zip(Ts3, outs):
    Xb, eb, _, lib_ = oracle.standard(Tb)
    check(Xb, eb, lib_, o, 1e-10)
ev.sync()
print("checked build ok")
"""


def test_checked_build_runs_clean():
    from paper_2002_05024_b300 import build as b
    b.build(checked=True)
    code = "import os\nROOT = %r\n" % ROOT + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
