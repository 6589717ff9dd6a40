#!/usr/bin/env python
"""Benchmark of the robust eigenvector path on one B300 (replicas across GPUs).

Workload (one step = the whole path once): all 16384 eigenvectors of an
n = 16384 real Schur form drawn from the config-0 distribution (75% real 1x1
blocks, 25% standardized 2x2 blocks, strictly upper part N(0, 1)),
back-transformed by an orthogonal Q (product of 64 Householder reflectors).
The timed steps run the FP64 path (DFMA throughout); the same line carries,
under "records", the split-precision path on the same input (8 BF16 digit
slices on the tensor cores, FP32 exact accumulation, FP64 recombination,
then one FP64 residual-correction sweep; also without the sweep) and the
batched workload (2000 Schur forms of n in [32, 1024] in one persistent
launch, FP64 and split), each with its rate, residuals and ratio to the
plain FP64 path.  Inputs are seeded and synthetic; T, Q and X are 2 GiB
each, larger than L2.

Metric: eigenvector columns per second (and achieved FP64 TFLOPS with the
algorithmic count F = sum_j [k_j^2 + 2 n (k_j + b_j)], k_j rows above the
column's block, b_j its size); split and batched against the plain FP64
path at normalised residual <= 10 n.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain column-by-column robust
substitution) on the machine's host cores, each step a bounded random sample of
the same workload's columns, extrapolated to all columns by the flop count.
Other workloads: --workload batched | generalized | trsolve |
batched_generalized | hessenberg | window, --side left.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 DFMA rate per SM and clock measured on this B300 (fp64 probe):
# 1.126 TFLOP/s at 1935 MHz over 148 SMs = 3.93 flop/clk/SM, i.e. 2 DFMA/clk/SM.
FP64_FLOP_PER_CLK_PER_SM = 4.0
N_SMS = 148

REASON_BITS = {
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
    0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
    0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
    0x100: "display_clock_setting",
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=0,
                    help="order (default: 16384 for the right eigenvectors, 8192 for the "
                         "generalized workload, 4096 otherwise)")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--mode", choices=["fp64", "split"], default="fp64")
    ap.add_argument("--slices", type=int, default=0)
    ap.add_argument("--refine", action="store_true",
                    help="split mode: one FP64 residual-correction sweep after the solve")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="columns of the CPU-oracle sample (default 512 at n >= 8192, "
                         "else 4096)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-records", dest="records", action="store_false",
                    help="single workload, FP64: leave out the split and batched records")
    ap.add_argument("--record-steps", type=int, default=3,
                    help="timed steps of the split records")
    ap.add_argument("--residual-cols", type=int, default=512,
                    help="columns whose residual the line reports")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="extra steps timed kernel by kernel (default 1 at n >= 8192, else 3)")
    ap.add_argument("--workload", choices=["single", "batched", "generalized", "trsolve",
                                           "batched_generalized", "hessenberg", "window"],
                    default="single",
                    help="single: one n x n Schur form with Q (default); batched: the "
                         "2000-matrix batch of evec_batched; generalized: an n x n pencil "
                         "(S, T) with Z; trsolve: robust solve of an n x n "
                         "quasi-triangular T with --nrhs right-hand sides; "
                         "batched_generalized: --batch pencils in one persistent launch")
    ap.add_argument("--nrhs", type=int, default=0, help="trsolve: right-hand sides (default n)")
    ap.add_argument("--window", type=int, default=128,
                    help="window: rows and columns of each reordering window")
    ap.add_argument("--lookahead", action="store_true",
                    help="split mode: the look-ahead schedule (evec_set_lookahead)")
    ap.add_argument("--side", choices=["right", "left"], default="right",
                    help="single: right eigenvectors (default) or left ones (u^H T = lambda u^H)")
    ap.add_argument("--batch", type=int, default=2000)
    ap.add_argument("--input", choices=["config0", "adversarial"], default="config0",
                    help="single workload: config-0 Schur form (default) or the clustered "
                         "adversarial one (4 clusters 1e-9 apart, upper part N(0, 1) x 1e3)")
    ap.add_argument("--no-other", dest="other", action="store_false",
                    help="default line: leave out the short runs of the other workloads")
    args = ap.parse_args()
    if not args.n:
        args.n = (16384 if args.workload == "single" and args.side == "right" else
                  8192 if args.workload == "generalized" else 4096)
    if not args.cpu_sample:
        args.cpu_sample = 512 if args.n >= 8192 else 4096
    if not args.profile_steps:
        args.profile_steps = 1 if args.n >= 8192 else 3
    return args


METRIC_SINGLE = ("eigvec columns/s (robust eigenvectors incl. back-transformation X = Q Y); "
                 "TFLOPS vs the FP64 roofline; split/batched vs plain at residual <= 10 n")


def workload(n, kind="config0"):
    if kind == "adversarial":
        T, blocks = workloads.adversarial_schur(n, seed=workloads.SEED_BASE + 11)
    else:
        T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE + 1)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 101)
    return T, blocks, Q


# Short runs of the other workloads that the default line carries under
# "other_workloads" (each a child process of this script, so its device
# memory and its own timing are separate): name, arguments, what it is.
OTHER_WORKLOADS = [
    ("n4096_fp64", ["--n", "4096", "--no-records"],
     "n = 4096 config-0 Schur form + Q, FP64, tile 64"),
    ("n4096_split_sweep", ["--n", "4096", "--no-records", "--mode", "split", "--refine"],
     "n = 4096 config-0 Schur form + Q, split (8 slices) + FP64 residual-correction sweep"),
    ("n4096_clustered_fp64", ["--n", "4096", "--no-records", "--input", "adversarial"],
     "n = 4096 clustered adversarial Schur form + Q, FP64, tile 64"),
    ("pencil_n8192_fp64", ["--workload", "generalized"],
     "n = 8192 pencil (S, T) + Z, FP64"),
    ("pencil_n8192_split", ["--workload", "generalized", "--mode", "split"],
     "n = 8192 pencil (S, T) + Z, split (8 slices)"),
    ("trsolve_n4096_split", ["--workload", "trsolve", "--mode", "split"],
     "robust triangular solve, n = 4096, 4096 right-hand sides, split"),
    ("left_n4096_split", ["--n", "4096", "--no-records", "--side", "left", "--mode", "split"],
     "left eigenvectors, n = 4096 + Q, split"),
    ("batched_pencils_fp64", ["--workload", "batched_generalized"],
     "2000 pencils, n in [32, 1024], 30% selected, FP64, one persistent launch"),
    ("window_n4096_split", ["--workload", "window", "--mode", "split"],
     "reordering off-diagonal updates, n = 4096 + Q, 32 windows of 128, split"),
    ("hessenberg_n4096_split", ["--workload", "hessenberg", "--mode", "split"],
     "Hessenberg reduction with Q, n = 4096, split updates"),
]
OTHER_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype",
              "tflops_fp64", "tflops_fp64_equivalent", "quality", "e2e")


def other_workloads_record(steps=3, warmup=2, timeout=600):
    """Each entry of OTHER_WORKLOADS as a child run of this script (no CPU
    baseline), reduced to its rate, quality and dominant kernel's roofline;
    a child that fails is recorded with its exit status, not raised."""
    out = {}
    for name, extra, what in OTHER_WORKLOADS:
        cmd = [sys.executable, os.path.abspath(__file__), "--steps", str(steps), "--warmup",
               str(warmup), "--no-cpu-baseline", *extra]
        t = time.time()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, cwd=ROOT)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode != 0 or not lines:
                out[name] = {"what": what, "error": f"exit {r.returncode}",
                             "tail": (r.stderr or r.stdout)[-300:]}
                continue
            line = json.loads(lines[-1])
        except Exception as exc:   # timeout, bad JSON: record it
            out[name] = {"what": what, "error": repr(exc)[:300]}
            continue
        rec = {"what": what, "args": " ".join(extra), "wall_s": round(time.time() - t, 1)}
        rec.update({k: line[k] for k in OTHER_KEYS if k in line})
        rec["workload"] = (line.get("config") or {}).get("workload")
        roof = line.get("roofline")
        if isinstance(roof, dict):
            rec["roofline"] = {k: roof.get(k) for k in ("kernel", "bound", "achieved", "peak",
                                                         "unit", "frac")}
        out[name] = rec
    return out


def default_tile(n, mode):
    """The library's tile when opt->tile is 0: 64 rows, 256 in split mode
    from n = 8192."""
    return 256 if mode == "split" and n >= 8192 else 64


def flop_counts(n, blocks, tile_start, with_q=True, res=None):
    """Algorithmic FP64 flops: total per the method's definition, and the
    parts done by the tile-update GEMMs and by the back-transformation (the
    diagonal-tile solves do the rest of the substitution: total - upd - bt).
    res (a list): receives the flops of the residual -(T - lambda I) y of the
    correction sweep, 2 (p (p + size) - p (p - 1) / 2) per column of a block
    at row p (rows above the block, T quasi-triangular)."""
    tile_start = np.asarray(tile_start)
    total = 0.0
    upd = 0.0
    bt = 0.0
    r = 0.0
    for p, sz in blocks:
        k = p
        r += sz * 2.0 * (k * (k + sz) - k * (k - 1) / 2.0)
        for _ in range(sz):
            total += k * k + (2.0 * n * (k + sz) if with_q else 0.0)
            bt += 2.0 * n * (k + sz) if with_q else 0.0
            # rows above the column's own tile are updated by the GEMMs
            c = int(np.searchsorted(tile_start, p, side="right") - 1)
            t0c = tile_start[c]
            upd += 2.0 * t0c * (p + sz - t0c)
            for s in range(1, c):
                upd += 2.0 * tile_start[s] * (tile_start[s + 1] - tile_start[s])
    if res is not None:
        res.append(r)
    return total, upd, bt


# kernel class -> source files whose content a stored DRAM-traffic figure
# belongs to (per mode)
KERNEL_SOURCES = {
    ("diag_solve", "fp64"): ["k_diag_solve.cu", "diag_tile.cuh"],
    ("diag_solve", "split"): ["k_diag_solve.cu", "diag_tile.cuh"],
    ("refine", "split"): ["k_gemm.cu", "k_finalize.cu"],
    ("tile_update", "fp64"): ["k_gemm.cu"],
    ("tile_update", "split"): ["k_split_update.cu", "k_split.cu", "split_common.cuh"],
    ("backtransform", "fp64"): ["k_gemm.cu"],
    ("backtransform", "split"): ["k_split.cu", "split_common.cuh"],
    ("left", "split"): ["k_left.cu"],
    ("left", "fp64"): ["k_left.cu"],
    ("hess_panel", "fp64"): ["k_hessenberg.cu"],
    ("hess_update", "fp64"): ["k_hessenberg.cu"],
    ("window", "fp64"): ["k_window.cu"],
    ("window", "split"): ["k_split.cu", "k_window.cu", "split_common.cuh"],
}
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def source_digest(files):
    import hashlib
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2002_05024_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(kernel, mode, n, tile, prefix=""):
    """DRAM bytes per launch from the committed ncu summary, or None when
    there is none for this kernel, workload and mode, or when the kernel's
    source changed since the capture (prefix: "" for the eigenvector
    workload, "trsolve:" for the triangular solve)."""
    try:
        rec = json.load(open(TRAFFIC))[f"{prefix}{kernel}/{mode}/n{n}/tile{tile}"]
    except Exception:
        return None
    files = KERNEL_SOURCES.get((kernel, mode))
    if not files or rec.get("source_sha1") != source_digest(files):
        return None
    return rec.get("dram_bytes_per_launch")


def rooflines(prof, steps, mode, slices, F_diag, F_upd, F_bt, peaks, n, tile, F_res=0.0,
              sweeps=1, prefix=""):
    """Per kernel class: algorithmic work per step / event-timed kernel time
    per step against the unit that bounds it.  Diagonal solves and FP64-mode
    GEMMs: FP64 flops on the FP64 pipe ("alu"; peak from the measured DFMA
    rate x SMs x max clock).  Split-mode GEMMs: the S (S + 1) / 2 BF16 slice
    products the method needs per FP64 multiply-add, on the tensor cores
    ("tensor"; peak = the measured sustained cuBLAS BF16 rate, as these
    kernels run inside a long step).  With the residual-correction sweep
    (sweeps = 2) the solve kernels run twice per step, and "refine" is the
    FP64 residual product (F_res) with its two small companions."""
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    fp64_peak = N_SMS * FP64_FLOP_PER_CLK_PER_SM * sm_max * 1e6 / 1e12
    bf16 = peaks.get("bf16_tflops_sustained")
    bf16_src = "of measured (sustained cuBLAS BF16)" if bf16 else "of fallback"
    bf16 = float(bf16 or 1400.0)
    pairs = slices * (slices + 1) // 2
    work = {"diag_solve": (sweeps * F_diag, False),
            "tile_update": (sweeps * F_upd, mode == "split"),
            "backtransform": (F_bt, mode == "split"), "refine": (F_res, False)}
    out = {}
    for k, (ms, nl) in prof.items():
        if k not in work or ms <= 0 or nl <= 0 or work[k][0] <= 0:
            continue
        f64, tensor = work[k]
        sec = ms / steps / 1e3
        if tensor:
            alg, peak, bound, src = pairs * f64, bf16, "tensor", bf16_src
        else:
            alg, peak, bound, src = f64, fp64_peak, "alu", \
                "of derived FP64 peak (measured 4 flop/clk/SM x 148 SMs x max SM clock)"
        achieved = alg / sec / 1e12
        tr = stored_traffic(k, mode, n, tile, prefix)
        out[k] = {"kernel": k, "bound": bound, "achieved": achieved, "peak": peak,
                  "unit": "TFLOP/s", "frac": achieved / peak, "traffic": tr,
                  "peak_source": src, "launches_per_step": nl / steps,
                  "ms_per_step": ms / steps,
                  "alg_flops_per_launch": alg / (nl / steps)}
    return out


def profiled_steps(h, step, steps, dev, k=3):
    """Per-kernel CUDA-event times of k extra steps, after the timed region
    (the events recorded around every launch are kept out of the timed
    steps), scaled to `steps` steps: {kind: (ms, launches)}."""
    import torch
    k = max(1, min(k, steps))
    h.profile(True)
    h.profile_read()
    for _ in range(k):
        step()
    torch.cuda.synchronize(dev)
    prof = h.profile_read()
    h.profile(False)
    return {kind: (ms * steps / k, int(round(c * steps / k))) for kind, (ms, c) in prof.items()}


def reduce_over_ranks(x, dist=None, device=None, op="max"):
    """The max (or sum) of a float over the ranks of the default process
    group (NCCL on the GPU, gloo on the host); x itself without a group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, seconds_max, world):
    """Whole-job throughput: every rank processed units_per_rank units per
    step (weak scaling); the slowest rank's time is the job's."""
    return world * units_per_rank * steps / seconds_max


def measured_peaks():
    try:
        return json.load(open(MEASURED))
    except Exception:
        return {}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                      text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                act = int(f[4], 16)
            except ValueError:
                continue
            for bit, name in REASON_BITS.items():
                if act & bit and name != "gpu_idle":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def block_columns(blocks):
    """First output column of every block (all eigenvalues selected)."""
    out, c = [], 0
    for _, sz in blocks:
        out.append(c)
        c += sz
    return out


def pick_eigenvalues(blocks, k, seed):
    """Seeded random blocks until they hold at least k columns."""
    rng = np.random.default_rng(seed)
    pick, cols = [], 0
    for b in rng.permutation(len(blocks)):
        if cols >= k:
            break
        pick.append(int(b))
        cols += blocks[b][1]
    return sorted(pick)


def sample_flops(n, blocks, sel, with_q):
    """The method's flops F = sum_j [k_j^2 + 2 n (k_j + b_j) [Q]] over the
    selected columns."""
    f = 0.0
    for p, sz in blocks:
        if sel is None or sel[p]:
            f += sz * (float(p) * p + (2.0 * n * (p + sz) if with_q else 0.0))
    return f


def compare_columns(Xa, ea, Xb, eb, lam_im):
    """Canonical columns a (reference) and b: per eigenvalue the exponent
    difference and the normwise relative difference after bringing b to a's
    exponent (a pair: row norms |re| + |im|).  Returns (max |exponent
    difference|, max and median relative difference)."""
    m = Xa.shape[1]
    rels, max_de = [], 0
    j = 0
    step = 512
    while j < m:
        j1 = min(m, j + step)
        if j1 < m and lam_im[j1 - 1] > 0:   # keep a pair together
            j1 += 1
        de = ea[j:j1].astype(np.int64) - eb[j:j1].astype(np.int64)
        A = Xa[:, j:j1]
        B = np.ldexp(Xb[:, j:j1], de.astype(np.int32))
        D = np.abs(A - B)
        N = np.abs(A)
        c = 0
        while c < j1 - j:
            if lam_im[j + c] != 0.0:
                rels.append((D[:, c] + D[:, c + 1]).max() / (N[:, c] + N[:, c + 1]).max())
                max_de = max(max_de, abs(int(de[c])))
                c += 2
            else:
                rels.append(D[:, c].max() / N[:, c].max())
                max_de = max(max_de, abs(int(de[c])))
                c += 1
        j = j1
    rels = np.asarray(rels) if rels else np.zeros(1)
    return max_de, float(rels.max()), float(np.median(rels))


def normalised_residuals(T, X, lr, li):
    """||T x - lambda x||_1 / (||T||_1 ||x||_1 u) per eigenvalue (FP64)."""
    T1 = np.abs(T).sum(axis=0).max()
    R = T @ X
    out = []
    j = 0
    while j < X.shape[1]:
        if li[j] != 0.0:
            x = X[:, j] + 1j * X[:, j + 1]
            r = (R[:, j] + 1j * R[:, j + 1]) - (lr[j] + 1j * li[j]) * x
            j += 2
        else:
            x = X[:, j]
            r = R[:, j] - lr[j] * x
            j += 1
        out.append(np.abs(r).sum() / (T1 * np.abs(x).sum() * 2.0 ** -53))
    return np.asarray(out)


def cpu_baseline(T, blocks, Q, sample_cols, seed=5, gpu=None, left=False, flops=None):
    """The oracle, as it stands, on a seeded random sample of the workload's
    columns, on all host cores.  flops = (n, with_q): the rate is
    extrapolated from the sample to the whole workload by the method's flop
    count (sum over all columns / sum over the sampled ones), and the
    oracle's result comes back with it: (record, (X, scale_exp, mask)).
    With gpu = (X, scale_exp) of the timed run, the sampled columns are also
    compared with the GPU's (largest exponent difference and normwise
    relative difference after bringing both to one exponent)."""
    import oracle
    n = T.shape[0]
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(blocks))
    sel = np.zeros(n, np.uint8)
    cols = 0
    for b in order:
        if cols >= sample_cols:
            break
        p, sz = blocks[b]
        sel[p:p + sz] = 1
        cols += sz
    oracle.build()
    t = time.perf_counter()
    X, e, lr, li = (oracle.left if left else oracle.standard)(T, Q=Q, select=sel)
    dt = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = int(os.environ.get("OMP_NUM_THREADS", cores))
    out = {"value": X.shape[1] / dt, "unit": "columns/s", "cores": threads, "kind": "oracle",
           "columns": X.shape[1], "seconds": dt,
           "sample": f"{X.shape[1]} randomly chosen columns (seed {seed}) of the n={n} "
                     f"workload incl. back-transformation"
                     + (" (left eigenvectors)" if left else "") + f", {dt:.2f} s"}
    if flops is not None:
        m = sum(sz for _, sz in blocks)
        f_all = sample_flops(n, blocks, None, flops[1])
        f_smp = sample_flops(n, blocks, sel, flops[1])
        out["value"] = m / (dt * f_all / f_smp)
        out["extrapolated"] = True
        out["sample_columns_per_s"] = X.shape[1] / dt
        out["sample"] += (f"; extrapolated to all {m} columns by the flop count "
                          f"({f_all:.3e} / {f_smp:.3e})")
    if gpu is not None:
        Xg, eg = gpu
        cidx = [c + k for c, (p, sz) in zip(block_columns(blocks), blocks) if sel[p]
                for k in range(sz)]
        de, rel, med = compare_columns(X, e, Xg[:, cidx], eg[cidx], li)
        out["gpu_vs_oracle"] = {"columns": len(cidx), "max_exponent_diff": de,
                                "max_rel_diff": rel, "median_rel_diff": med}
    if flops is not None:
        return out, (X, e, sel)
    return out


def residual_sample(T, Q, X, lr, li, blocks, pick, left=False):
    """Normalised residual ||T y - lambda y||_1 / (||T||_1 ||y||_1 u) of the
    picked eigenvalues of a GPU result, y = Q^T x (the Schur-coordinate
    residual of x), in FP64 on the host.  left: the residual of T^T conj(y)
    = lambda conj(y) (u^H T = lambda u^H) with ||T^T||_1."""
    starts = block_columns(blocks)
    cols = [starts[b] + k for b in pick for k in range(blocks[b][1])]
    Xs = np.array(X[:, cols], dtype=np.float64, order="F")
    lrs, lis = np.asarray(lr)[cols], np.asarray(li)[cols]
    if left:
        T = np.ascontiguousarray(T.T)
        Xs[:, lis < 0] = -Xs[:, lis < 0]
    Ys = Q.T @ Xs if Q is not None else Xs
    res = normalised_residuals(T, Ys, lrs, lis)
    n = T.shape[0]
    return {"eigenvalues": int(len(pick)), "columns": len(cols),
            "max_normalised_residual": float(res.max()),
            "median_normalised_residual": float(np.median(res)),
            "max_over_n": float(res.max()) / n, "gate": "<= 10 n",
            "how": "Schur coordinates y = Q^T x, FP64 on the host"}


def run_reference_trsolve(args):
    n = args.n
    nrhs = args.nrhs or n
    T, _, B = workloads.solve_system(n, nrhs)
    per_step = max(16, args.cpu_sample // 4)
    times, cols = [], []
    for i in range(args.warmup + args.steps):
        r = trsolve_cpu_baseline(T, B, per_step, seed=1000 + i)
        if i >= args.warmup:
            cols.append(r["columns"])
            times.append(r["seconds"])
    value = sum(cols) / sum(times)
    line = {
        "impl": "reference",
        "metric": "right-hand sides/s (robust FP64 triangular solve with per-column scaling)",
        "value": value, "unit": "right-hand sides/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"quasi-triangular T n={n}, B n x {nrhs} (oracle samples)"},
        "cpu_baseline": {"value": value, "unit": "right-hand sides/s", "cores": r["cores"],
                         "kind": "oracle",
                         "sample": f"{per_step} random right-hand sides per step of the "
                                   f"n={n} system, on the host cores"},
        "e2e": {"value": value, "unit": "right-hand sides/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reference_line(args, metric, unit, workload, value, sample, ms_per_step, cores):
    return {
        "impl": "reference", "metric": metric, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": workload},
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference_other(args):
    """The oracle on bounded samples of the batched, pencil, batched-pencil
    and Hessenberg workloads (same metric and unit as the GPU arm)."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cores = int(os.environ.get("OMP_NUM_THREADS", cores))
    units, secs = 0.0, 0.0
    if args.workload in ("batched", "batched_generalized"):
        if args.workload == "batched":
            _, mats, sels = workloads.batch_inputs(args.batch)
            run = lambda i: oracle.standard(mats[i], select=sels[i])[0].shape[1]  # noqa: E731
            metric = "eigvec columns/s, batched (robust FP64 eigenvectors, many Schur forms)"
            what = f"batch of {args.batch} Schur forms, n log-uniform in [32, 1024]"
        else:
            _, mats, sels = workloads.batch_pencils(args.batch)
            run = lambda i: oracle.generalized(mats[i][0], mats[i][1],  # noqa: E731
                                               select=sels[i])[0].shape[1]
            metric = ("eigvec columns/s, batched pencils (robust "
                      + ("generalized eigenvectors, split-precision updates)"
                         if args.mode == "split" else "FP64 generalized eigenvectors)"))
            what = f"batch of {args.batch} pencils, n log-uniform in [32, 1024]"
        per = max(8, min(len(mats), 50))
        for i in range(args.warmup + args.steps):
            pick = np.random.default_rng(2000 + i).choice(len(mats), size=per, replace=False)
            t = time.perf_counter()
            c = sum(run(int(k)) for k in pick)
            dt = time.perf_counter() - t
            if i >= args.warmup:
                units += c
                secs += dt
        unit = "columns/s"
        sample = f"{per} random matrices of the batch per step, on the host cores"
    elif args.workload == "generalized":
        n = args.n
        S, T, blocks = workloads.generalized_pair(n, seed=workloads.SEED_BASE + 4)
        Z = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 104)
        per = max(2, args.cpu_sample // 64)
        for i in range(args.warmup + args.steps):
            rng = np.random.default_rng(3000 + i)
            sel = np.zeros(n, np.uint8)
            for b in rng.choice(len(blocks), size=per, replace=False):
                p, sz = blocks[b]
                sel[p:p + sz] = 1
            t = time.perf_counter()
            c = oracle.generalized(S, T, Z, select=sel)[0].shape[1]
            dt = time.perf_counter() - t
            if i >= args.warmup:
                units += c
                secs += dt
        unit = "columns/s"
        metric = "eigvec columns/s, generalized (robust FP64 eigenvectors of a pencil incl. X = Z Y)"
        what = f"pencil (S, T) n={n} with Z, all columns"
        sample = f"{per} random eigenvalues per step of the n={n} pencil, on the host cores"
    elif args.workload == "window":
        n, k = args.n, args.window
        T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE)
        Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 100)
        wins = workloads.window_chain(n, k, k, seed=workloads.SEED_BASE + 9, blocks=blocks)
        per = 2
        for i in range(args.warmup + args.steps):
            pick = np.random.default_rng(5000 + i).choice(len(wins), size=per, replace=False)
            t = time.perf_counter()
            oracle.window_update(T, Q, [wins[int(j)] for j in sorted(pick)])
            dt = time.perf_counter() - t
            if i >= args.warmup:
                units += per
                secs += dt
        unit = "windows/s"
        metric = ("reordering windows/s (off-diagonal updates with Q, " +
                  (f"split precision, {args.slices or 8} slices)" if args.mode == "split"
                   else "FP64)"))
        what = window_what(n, k, len(wins))
        sample = f"{per} random windows of the chain per step, plain loops on one core"
        cores = 1
    else:   # hessenberg: one unblocked reduction at a reduced order per step
        n = args.n
        ns = min(n, 768)
        for i in range(args.warmup + args.steps):
            A = np.random.default_rng(4000 + i).standard_normal((ns, ns))
            t = time.perf_counter()
            oracle.hessenberg(A)
            dt = time.perf_counter() - t
            if i >= args.warmup:
                units += (ns / n) ** 3
                secs += dt
        unit = "reductions/s"
        metric = ("Hessenberg reductions/s (A = Q H Q^T with Q, "
                  + (f"split-precision updates, {args.slices or 8} slices)"
                     if args.mode == "split" else "FP64)"))
        what = f"Hessenberg reduction of an n={n} N(0, 1) matrix with Q"
        sample = (f"one unblocked reduction with Q at n = {ns} per step on one core, counted as "
                  f"(n / {ns})^3 reductions of order {n}")
        cores = 1
    value = units / secs if secs > 0 else 0.0
    print(json.dumps(reference_line(args, metric, unit, what + " (oracle samples)", value, sample,
                                    1e3 * secs / max(args.steps, 1), cores)), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload == "trsolve":
        return run_reference_trsolve(args)
    if args.workload in ("batched", "batched_generalized", "generalized", "hessenberg", "window"):
        return run_reference_other(args)
    n = args.n
    T, blocks, Q = workload(n, args.input)
    m = sum(sz for _, sz in blocks)
    # a bounded sample per step (about 1.5 s of oracle work at n = 16384),
    # extrapolated to the whole workload by the flop count
    per_step = 64 if n >= 8192 else max(16, args.cpu_sample // 4)
    times, cols = [], []
    for i in range(args.warmup + args.steps):
        r, _ = cpu_baseline(T, blocks, Q, per_step, seed=1000 + i, left=args.side == "left",
                            flops=(n, True))
        if i >= args.warmup:
            cols.append(m)
            times.append(m / r["value"])
    value = sum(cols) / sum(times)
    cores = r["cores"]
    line = {
        "impl": "reference",
        "metric": METRIC_SINGLE,
        "value": value, "unit": "columns/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"single large Schur form: n={n} real Schur form ("
                               + ("clustered adversarial" if args.input == "adversarial" else
                                  "config-0 distribution")
                               + ") + Q (product of 64 Householder reflectors), all "
                               f"{m} " + ("left eigenvectors" if args.side == "left" else
                                          "eigenvectors")
                               + "; the oracle on sampled columns, extrapolated",
                   "n": n, "columns": m},
        "cpu_baseline": {"value": value, "unit": "columns/s", "cores": cores, "kind": "oracle",
                         "extrapolated": True,
                         "sample": f"{per_step} random columns per step of the n={n} "
                                   "workload, on the host cores; each step's time scaled to "
                                   "all columns by the flop count (ms_per_step is that "
                                   "extrapolated time of a whole step)"},
        "e2e": {"value": value, "unit": "columns/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    """The eigenvector workload: all eigenvectors of one n x n Schur form with
    Q.  The timed steps run args.mode (FP64 by default); with --records (the
    default for FP64 right eigenvectors on one GPU) the line also carries the
    split-precision path on the same input, with and without the FP64
    residual-correction sweep, and the batched workload in both modes, each
    with its rate, its quality and its ratio to the plain FP64 path."""
    import ctypes

    import torch

    import paper_2002_05024_b300 as ev

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n = args.n
    T, blocks, Q = workload(n, args.input)
    m = sum(sz for _, sz in blocks)
    d = np.ascontiguousarray(np.diagonal(T))
    tile_used = args.tile or default_tile(n, args.mode)
    _, tile_start = ev.plan_query(d, np.ascontiguousarray(np.diagonal(T, -1)),
                                  np.ascontiguousarray(np.diagonal(T, 1)), None, tile_used)
    res = []
    F, F_upd, F_bt = flop_counts(n, blocks, tile_start, res=res)
    F_diag = max(F - F_upd - F_bt, 0.0)
    refine = bool(args.refine and args.mode == "split")
    F_res = res[0]

    dT = torch.from_numpy(T).to(dev)
    dQ = torch.from_numpy(Q).to(dev)
    X = torch.empty((m, n), dtype=torch.float64, device=dev).t()
    e = torch.empty(m, dtype=torch.int32, device=dev)
    lr = torch.empty(m, dtype=torch.float64, device=dev)
    li = torch.empty(m, dtype=torch.float64, device=dev)
    out = (X, e, lr, li)
    stream = torch.cuda.current_stream(dev)

    left = args.side == "left"
    solve = ev.left if left else ev.standard
    ev.handle(local_rank).lookahead(args.lookahead)

    def step():
        solve(dT, dQ, tile=args.tile, out=out, mode=args.mode, slices=args.slices,
              refine=1 if refine else 0)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    ev.sync(local_rank)
    h = ev.handle(local_rank)

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(gpu_id) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    elapsed_ms = t0.elapsed_time(t1)
    clocks = sampler.stop() if sampler else None
    ev.sync(local_rank)
    prof = profiled_steps(h, step, args.steps, dev, k=args.profile_steps)
    elapsed_ms = reduce_over_ranks(elapsed_ms, dist, dev)

    ms_per_step = elapsed_ms / args.steps
    value = whole_job_rate(m, args.steps, elapsed_ms / 1e3, world)
    tflops = world * F * args.steps / (elapsed_ms / 1e3) / 1e12

    # roofline of the dominant kernel (largest share of event-timed time)
    peaks = measured_peaks()
    slices = (args.slices or 8) if args.mode == "split" else 0
    roofs = rooflines(prof, args.steps, args.mode, slices, F_diag, F_upd, F_bt, peaks, n,
                      tile_used,
                      F_res=F_res if refine else 0.0, sweeps=2 if refine else 1,
                      prefix="left:" if left else "")
    dominant = max(prof.items(), key=lambda kv: kv[1][0])[0]
    roofline = roofs.get(dominant)
    gpu_launches = sum(c for _, c in prof.values())

    # end to end through the public API with host buffers (pinned host memory)
    e2e = None
    e2e_steps = args.steps if n <= 4096 else min(args.steps, 2)
    if left and not os.environ.get("EVEC_BENCH_NO_E2E"):
        # no host-buffer entry point for the left vectors: the public call on
        # device tensors with T and Q copied in from pinned memory and X,
        # the exponents and eigenvalues copied out, every step
        hT = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hT.copy_(torch.from_numpy(T))
        hQ = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hQ.copy_(torch.from_numpy(Q))
        hX = torch.empty((m, n), dtype=torch.float64, pin_memory=True).t()
        hE = torch.empty(m, dtype=torch.int32, pin_memory=True)
        hL = torch.empty((2, m), dtype=torch.float64, pin_memory=True)

        def host_step():
            dT.copy_(hT, non_blocking=True)
            dQ.copy_(hQ, non_blocking=True)
            step()
            hX.copy_(X, non_blocking=True)
            hE.copy_(e, non_blocking=True)
            hL[0].copy_(lr, non_blocking=True)
            hL[1].copy_(li, non_blocking=True)
            torch.cuda.synchronize(dev)
    elif not os.environ.get("EVEC_BENCH_NO_E2E"):
        pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()  # noqa: E731
        hT = pin((n, n), torch.float64)
        hT[...] = T.T          # row-major view of the column-major bytes
        hQ = pin((n, n), torch.float64)
        hQ[...] = Q.T
        hX = pin((m, n), torch.float64)
        hE = pin((m,), torch.int32)
        hLr = pin((m,), torch.float64)
        hLi = pin((m,), torch.float64)
        opts = ev._opts(args.tile, False, args.mode, args.slices, 1 if refine else 0)
        hh = ev.handle(local_rank)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731

        def host_step():
            st = ev.lib().evec_standard_host(hh.ptr, n, P(hT), P(hQ), None, P(hX), P(hE),
                                             P(hLr), P(hLi), ctypes.byref(opts))
            if st:
                raise ev.EvecError(st, "evec_standard_host")
    if not os.environ.get("EVEC_BENCH_NO_E2E"):
        host_step()
        if dist:
            dist.barrier()
        w0 = time.perf_counter()
        for _ in range(e2e_steps):
            host_step()
        w = time.perf_counter() - w0
        if dist:
            tt = torch.tensor([w], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            w = float(tt.item())
        e2e = {"value": world * m * e2e_steps / w, "unit": "columns/s",
               "h2d_bytes_per_step": 2 * n * n * 8,
               "d2h_bytes_per_step": n * m * 8 + m * 4 + 2 * m * 8,
               "steps": e2e_steps, "warmup": 1,
               "entry": "evec_standard_left on device tensors with pinned-memory copies"
                        if left else "evec_standard_host (C ABI, pinned host buffers)"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    Xh, eh = X.cpu().numpy(), e.cpu().numpy()
    lrh, lih = lr.cpu().numpy(), li.cpu().numpy()
    pick = pick_eigenvalues(blocks, args.residual_cols, seed=7)
    quality = residual_sample(T, Q, Xh, lrh, lih, blocks, pick, left=left)
    cpu = None
    oracle_ref = None
    if world == 1 and not args.no_cpu_baseline:
        cpu, oracle_ref = cpu_baseline(T, blocks, Q, args.cpu_sample, gpu=(Xh, eh), left=left,
                                       flops=(n, True))
        cpu.pop("columns")
        cpu.pop("seconds")
    records = None
    if world == 1 and args.records and not left and args.mode == "fp64":
        records = {}
        rec_steps = max(1, min(args.steps, args.record_steps))
        # the split path at its own tile (the library's default in split mode)
        s_tile = args.tile or default_tile(n, "split")
        _, s_start = ev.plan_query(d, np.ascontiguousarray(np.diagonal(T, -1)),
                                   np.ascontiguousarray(np.diagonal(T, 1)), None, s_tile)
        s_res = []
        sF, sF_upd, sF_bt = flop_counts(n, blocks, s_start, res=s_res)
        for name, ref in (("split", True), ("split_no_sweep", False)):
            r = split_record(ev, dev, stream, dT, dQ, T, Q, blocks, m, sF, sF_upd, sF_bt,
                             s_res[0], s_tile, ref, rec_steps, max(1, min(args.warmup, 2)),
                             peaks, pick, oracle_ref, (Xh, eh, lih), left=False)
            r["vs_plain"] = r["value"] / value
            records[name] = r
        records["split_vs_plain"] = records["split"]["vs_plain"]
        records["split_no_sweep_vs_plain"] = records["split_no_sweep"]["vs_plain"]
        records["batched"] = batched_record(ev, dev, stream, local_rank, args.batch,
                                            max(1, min(args.steps, 5)),
                                            max(1, min(args.warmup, 2)), peaks)
        records["batched_vs_plain"] = records["batched"]["batched_vs_plain"]
        if args.other:
            del dT, dQ, X, e, lr, li, out
            torch.cuda.empty_cache()
            records["other_workloads"] = other_workloads_record()
    if args.mode == "fp64":
        dtype, how = "f64", "FP64 (DFMA) throughout"
    else:
        dtype = "bf16 slice products + f64"
        how = (f"split precision ({slices} BF16 slices, FP32 exact accumulation, FP64 "
               "recombination)" + (", then one FP64 residual-correction sweep" if refine else ""))
    line = {
        "metric": METRIC_SINGLE,
        "value": value, "unit": "columns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": dtype,
        "data": "synthetic",
        "config": {"workload": f"single large Schur form: n={n} real Schur form "
                               + ("(clustered adversarial: 4 clusters of real eigenvalues "
                                  "1e-9 apart, strictly upper N(0, 1) x 1e3)"
                                  if args.input == "adversarial" else
                                  "(config-0 distribution: 75% 1x1 blocks, 25% standardized "
                                  "2x2 blocks, strictly upper N(0, 1))")
                               + " + Q (product of 64 Householder "
                               f"reflectors), all {m} "
                               + ("left eigenvectors; " if left else "eigenvectors; ")
                               + "timed path: " + how
                               + ("; the split-precision path with the FP64 residual-correction "
                                  "sweep, and the 2000-matrix batch, in 'records'"
                                  if records else ""),
                   "n": n, "columns": m, "tile": tile_used, "mode": args.mode,
                   "slices": slices or None,
                   "refine": refine, "side": args.side,
                   "lookahead": args.lookahead,
                   "parallelism": "replicas",
                   "l2": f"inputs larger than L2 (T, Q, X {n * n * 8 / 2**20:.0f} MiB each)"},
        "tflops_fp64": tflops,
        "quality": quality,
        "flops_per_step": F,
        "roofline": roofline,
        "rooflines": roofs,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "records": records,
        # the metric's comparisons, from the records (same input, same GPU)
        "split_vs_plain": records.get("split_vs_plain") if records else None,
        "split_no_sweep_vs_plain": records.get("split_no_sweep_vs_plain") if records else None,
        "batched_vs_plain": records.get("batched_vs_plain") if records else None,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def split_record(ev, dev, stream, dT, dQ, T, Q, blocks, m, F, F_upd, F_bt, F_res, tile, refine,
                 steps, warmup, peaks, pick, oracle_ref, fp64_out, left=False):
    """The split-precision path (8 BF16 slices) on the timed workload's
    input, with or without the FP64 residual-correction sweep: rate, the
    split kernels' rooflines, the residual on the same sampled eigenvalues as
    the main line, the difference to the oracle on its sampled columns and
    to the FP64 GPU result on every column."""
    import torch
    n = T.shape[0]
    X = torch.empty((m, n), dtype=torch.float64, device=dev).t()
    e = torch.empty(m, dtype=torch.int32, device=dev)
    lr = torch.empty(m, dtype=torch.float64, device=dev)
    li = torch.empty(m, dtype=torch.float64, device=dev)
    out = (X, e, lr, li)

    def step():
        ev.standard(dT, dQ, tile=tile, out=out, mode="split", slices=8,
                    refine=1 if refine else 0)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    ev.sync(dev.index)
    h = ev.handle(dev.index)
    prof = profiled_steps(h, step, steps, dev, k=1)
    F_diag = max(F - F_upd - F_bt, 0.0)
    roofs = rooflines(prof, steps, "split", 8, F_diag, F_upd, F_bt, peaks, n, tile,
                      F_res=F_res if refine else 0.0, sweeps=2 if refine else 1)
    Xh, eh = X.cpu().numpy(), e.cpu().numpy()
    lrh, lih = lr.cpu().numpy(), li.cpu().numpy()
    rec = {"value": m * steps / (ms / 1e3), "unit": "columns/s", "steps": steps,
           "warmup": warmup, "ms_per_step": ms / steps,
           "tflops_fp64_equivalent": F * steps / (ms / 1e3) / 1e12,
           "dtype": "bf16 slice products (FP32 exact accumulation) + f64",
           "path": "split precision, 8 BF16 digit slices per operand, FP64 recombination"
                   + (", then one FP64 residual-correction sweep" if refine else ""),
           "tile": tile,
           "quality": residual_sample(T, Q, Xh, lrh, lih, blocks, pick, left=left),
           "rooflines": roofs,
           "kernel_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[0] > 0}}
    if oracle_ref is not None:
        Xo, eo, sel = oracle_ref
        cols = [c for c, (p, sz) in zip(block_columns(blocks), blocks) if sel[p]
                for c in range(c, c + sz)]
        de, rel, med = compare_columns(Xo, eo, Xh[:, cols], eh[cols], lih[cols])
        rec["gpu_vs_oracle"] = {"columns": len(cols), "max_exponent_diff": de,
                                "max_rel_diff": rel, "median_rel_diff": med}
    X64, e64, li64 = fp64_out
    de, rel, med = compare_columns(X64, e64, Xh, eh, li64)
    rec["vs_fp64_gpu"] = {"columns": m, "max_exponent_diff": de, "max_rel_diff": rel,
                          "median_rel_diff": med}
    del X, e, lr, li, out
    torch.cuda.empty_cache()
    return rec


def batched_record(ev, dev, stream, local_rank, count, steps, warmup, peaks):
    """The batched workload (count Schur forms, n log-uniform in [32, 1024],
    every 10th clustered-adversarial, 30% of the blocks selected) in one
    persistent launch per step, FP64 and split, against the same batch one
    evec_standard call per matrix (FP64, "plain").  Quality: the normalised
    residual of every selected eigenvalue of 100 sampled matrices per mode."""
    import torch
    _, Ts, sels = workloads.batch_inputs(count)
    Tp, ns, offs = ev.pack_batch(Ts, device=local_rank)
    sel = np.concatenate(sels)
    F = 0.0
    for T, s_ in zip(Ts, sels):
        nn = T.shape[0]
        i = 0
        while i < nn:
            sz = 2 if i + 1 < nn and T[i + 1, i] != 0.0 else 1
            if s_[i] or (sz == 2 and s_[i + 1]):
                F += sz * float(i) * float(i)
            i += sz
    check = np.random.default_rng(11).choice(len(Ts), size=min(len(Ts), 100), replace=False)
    out = {}
    for mode in ("fp64", "split"):
        o = ev.batched_packed(Tp, ns, offs, sel, mode=mode)
        for _ in range(warmup):
            ev.batched_packed(Tp, ns, offs, sel, mode=mode, out=o)
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            ev.batched_packed(Tp, ns, offs, sel, mode=mode, out=o)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        ms = t0.elapsed_time(t1)
        ev.sync(local_rank)
        cols = int(o[4].sum())
        Xp, ep, lrp, lip = (t.cpu().numpy() for t in o[:4])
        mm = o[4]
        xo = np.concatenate([[0], np.cumsum(ns * mm)])
        eo = np.concatenate([[0], np.cumsum(mm)])
        worst = 0.0
        for i in check:
            nn, mi = int(ns[i]), int(mm[i])
            if mi == 0:
                continue
            Xi = Xp[xo[i]:xo[i] + nn * mi].reshape(mi, nn).T
            r = normalised_residuals(Ts[i], Xi, lrp[eo[i]:eo[i] + mi], lip[eo[i]:eo[i] + mi])
            worst = max(worst, float((r / nn).max()))
        out[mode] = {"value": cols * steps / (ms / 1e3), "unit": "columns/s", "steps": steps,
                     "warmup": warmup, "ms_per_step": ms / steps,
                     "tflops_fp64_equivalent": F * steps / (ms / 1e3) / 1e12,
                     "tile_table": ev.tune_table(local_rank, mode),
                     "quality": {"matrices": int(len(check)),
                                 "max_normalised_residual_over_n": worst, "gate": "<= 10 n"}}
        del o
    dTs = [torch.from_numpy(np.asfortranarray(T)).to(dev) for T in Ts]
    for T, s_ in zip(dTs, sels):
        ev.standard(T, select=s_, tile=64)
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    for T, s_ in zip(dTs, sels):
        ev.standard(T, select=s_, tile=64)
    torch.cuda.synchronize(dev)
    plain = cols / (time.perf_counter() - w0)
    del dTs, Tp
    torch.cuda.empty_cache()
    return {"workload": f"{count} Schur forms, n log-uniform in [32, 1024] (config-0 "
                        "distribution, every 10th clustered adversarial), 30% of the blocks "
                        "selected, no Q, one persistent launch per step (CUDA graph)",
            "columns": cols, "flops_per_step": F, "fp64": out["fp64"], "split": out["split"],
            "plain_fp64_one_call_per_matrix": {"value": plain, "unit": "columns/s"},
            "batched_vs_plain": out["fp64"]["value"] / plain,
            "batched_split_vs_plain": out["split"]["value"] / plain}


def run_batched(args, rank, world, local_rank):
    """The batched workload: --batch independent Schur forms, sizes
    log-uniform in [32, 1024], every 10th clustered-adversarial, 30% of the
    blocks selected, no Q; one evec_batched call per step (persistent
    launch; FP64, or --mode split: the updates as BF16 slice products inside
    the persistent kernel).  Also times the same batch matrix by matrix
    through evec_standard ("plain", FP64) on the same GPU."""
    import ctypes  # noqa: F401

    import torch

    import paper_2002_05024_b300 as ev

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sizes, Ts, sels = workloads.batch_inputs(args.batch)
    Tp, ns, offs = ev.pack_batch(Ts, device=local_rank)
    sel = np.concatenate(sels)
    mode = args.mode
    slices = (args.slices or 8) if mode == "split" else 0
    out = ev.batched_packed(Tp, ns, offs, sel, tile=args.tile, mode=mode, slices=args.slices)
    m = out[4]
    cols = int(m.sum())
    F = 0.0
    for T, s_ in zip(Ts, sels):
        n = T.shape[0]
        i = 0
        while i < n:
            sz = 2 if i + 1 < n and T[i + 1, i] != 0.0 else 1
            if s_[i] or (sz == 2 and s_[i + 1]):
                F += sz * float(i) * float(i)
            i += sz
    for _ in range(args.warmup):
        ev.batched_packed(Tp, ns, offs, sel, tile=args.tile, mode=mode, out=out,
                          slices=args.slices)
    torch.cuda.synchronize(dev)
    # the update share of F with each matrix's tile (the tuned table)
    table = ev.tune_table(local_rank, mode)
    F_upd = 0.0
    for T, s_ in zip(Ts, sels):
        n = T.shape[0]
        c = 0 if n <= 64 else 1 if n <= 128 else 2 if n <= 256 else 3 if n <= 512 else 4
        nb = args.tile or table[c] or 64
        blocks, i = [], 0
        while i < n:
            sz = 2 if i + 1 < n and T[i + 1, i] != 0.0 else 1
            if s_[i] or (sz == 2 and s_[i + 1]):
                blocks.append((i, sz))
            i += sz
        _, ts = ev.plan_query(np.ascontiguousarray(np.diagonal(T)),
                              np.ascontiguousarray(np.diagonal(T, -1)),
                              np.ascontiguousarray(np.diagonal(T, 1)), None, nb)
        F_upd += flop_counts(n, blocks, ts, with_q=False)[1]
    h = ev.handle(local_rank)
    sampler = ClockSampler() if rank == 0 else None
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        ev.batched_packed(Tp, ns, offs, sel, tile=args.tile, mode=mode, out=out,
                          slices=args.slices)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1)
    clocks = sampler.stop() if sampler else None
    prof = profiled_steps(
        h, lambda: ev.batched_packed(Tp, ns, offs, sel, tile=args.tile, mode=mode, out=out,
                                     slices=args.slices), args.steps, dev)
    ev.sync(local_rank)
    if dist:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    value = world * cols * args.steps / (elapsed / 1e3)
    # the same batch, matrix by matrix through evec_standard
    dTs = [torch.from_numpy(np.asfortranarray(T)).to(dev) for T in Ts]
    for _ in range(2):
        for T, s_ in zip(dTs, sels):
            ev.standard(T, select=s_, tile=64)
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    for T, s_ in zip(dTs, sels):
        ev.standard(T, select=s_, tile=64)
    torch.cuda.synchronize(dev)
    plain = cols / (time.perf_counter() - w0)
    # end to end: the packed inputs from pinned host memory, results back
    hT = torch.empty(Tp.numel(), dtype=torch.float64, pin_memory=True)
    hT.copy_(Tp.cpu())
    hX = torch.empty(out[0].numel(), dtype=torch.float64, pin_memory=True)
    hE = torch.empty(out[1].numel(), dtype=torch.int32, pin_memory=True)
    w0 = time.perf_counter()
    for _ in range(args.steps):
        Tp.copy_(hT, non_blocking=True)
        ev.batched_packed(Tp, ns, offs, sel, tile=args.tile, mode=mode, out=out,
                          slices=args.slices)
        hX.copy_(out[0], non_blocking=True)
        hE.copy_(out[1], non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e = {"value": world * cols * args.steps / (time.perf_counter() - w0),
           "unit": "columns/s", "h2d_bytes_per_step": Tp.numel() * 8,
           "d2h_bytes_per_step": out[0].numel() * 8 + out[1].numel() * 4}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    fp64_peak = N_SMS * FP64_FLOP_PER_CLK_PER_SM * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6
    kms = prof.get("batched", (0.0, 0))[0] / args.steps
    launches = prof.get("batched", (0.0, 0))[1] / args.steps
    achieved = F / (kms / 1e3) / 1e12 if kms > 0 else None
    fp64_view = {"kernel": "k_batched", "bound": "alu", "achieved": achieved, "peak": fp64_peak,
                 "unit": "TFLOP/s", "frac": achieved / fp64_peak if achieved else None,
                 "traffic": None,
                 "peak_source": "of derived FP64 peak (measured 4 flop/clk/SM x 148 SMs x max "
                                "SM clock)",
                 "launches_per_step": launches, "alg_flops_per_launch": F / max(launches, 1)}
    roofline = fp64_view
    rooflines = {"fp64": fp64_view}
    if mode == "split" and kms > 0:
        # the updates' slice products on the tensor cores (S (S + 1) / 2 per
        # FP64 multiply-add) against the sustained BF16 rate; the diagonal
        # solves (F - F_upd) stay on the FP64 pipe inside the same kernel
        bf16 = float(peaks.get("bf16_tflops_sustained") or 1400.0)
        pairs = slices * (slices + 1) // 2
        ach = pairs * F_upd / (kms / 1e3) / 1e12
        roofline = {"kernel": "k_batched (split)", "bound": "tensor", "achieved": ach,
                    "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16, "traffic": None,
                    "peak_source": "of measured (sustained cuBLAS BF16)"
                    if peaks.get("bf16_tflops_sustained") else "of fallback",
                    "launches_per_step": launches,
                    "alg_flops_per_launch": pairs * F_upd / max(launches, 1),
                    "fp64_flops_of_diagonal_solves_per_launch": (F - F_upd) / max(launches, 1)}
        rooflines["tensor"] = roofline
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rng = np.random.default_rng(9)
        pick = rng.choice(len(Ts), size=min(len(Ts), 200), replace=False)
        t = time.perf_counter()
        cc = 0
        for i in pick:
            X, _, _, _ = oracle.standard(Ts[i], select=sels[i])
            cc += X.shape[1]
        dt = time.perf_counter() - t
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        cpu = {"value": cc / dt, "unit": "columns/s",
               "cores": int(os.environ.get("OMP_NUM_THREADS", cores)), "kind": "oracle",
               "sample": f"{len(pick)} randomly chosen matrices of the batch ({cc} columns), "
                         f"{dt:.2f} s"}
    line = {
        "metric": "eigvec columns/s, batched (robust FP64 eigenvectors, many Schur forms)",
        "value": value, "unit": "columns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if mode == "fp64" else "bf16 slice products + f64", "data": "synthetic",
        "config": {"workload": f"batch of {args.batch} Schur forms, n log-uniform in [32, 1024] "
                               "(config-0, every 10th clustered adversarial), 30% of blocks "
                               "selected, no Q, one persistent launch per step",
                   "matrices": args.batch, "columns": cols, "tile": args.tile or "tuned",
                   "tile_table": ev.tune_table(local_rank, mode), "mode": mode,
                   "slices": slices or None,
                   "parallelism": "replicas",
                   "l2": f"inputs {Tp.numel() * 8 / 2**30:.1f} GiB, larger than L2"},
        "plain_value": plain,
        "plain": "the same batch through evec_standard, one call per matrix (columns/s)",
        "tflops_fp64": F * args.steps / (elapsed / 1e3) / 1e12,
        "flops_per_step": F,
        "update_flops_per_step": F_upd,
        "roofline": roofline,
        "rooflines": rooflines,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": sum(c for _, c in prof.values()),
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batched_generalized(args, rank, world, local_rank):
    """Batched pencils: --batch independent pencils (S_i, T_i) built like the
    single pencil workload (S config-0, T upper triangular, diagonal
    U[0.5, 2], every 50th 1e-12), sizes log-uniform in [32, 1024], 30% of the
    blocks selected, no Z; one evec_batched_generalized call per step (the
    persistent kernel's pencil variant, FP64).  Algorithmic flops 2 k_j^2
    per selected column (two products per substitution step)."""
    import torch

    import paper_2002_05024_b300 as ev

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sizes, pairs, sels = workloads.batch_pencils(args.batch)
    Sp, ns, soffs = ev.pack_batch([S for S, _ in pairs], device=local_rank)
    Tp, _, toffs = ev.pack_batch([T for _, T in pairs], device=local_rank)
    sel = np.concatenate(sels)
    out = ev.batched_generalized_packed(Sp, Tp, ns, soffs, toffs, sel, tile=args.tile,
                                        mode=args.mode, slices=args.slices)
    m = out[5]
    cols = int(m.sum())
    F = 0.0
    for (S, _), s_ in zip(pairs, sels):
        n = S.shape[0]
        i = 0
        while i < n:
            sz = 2 if i + 1 < n and S[i + 1, i] != 0.0 else 1
            if s_[i] or (sz == 2 and s_[i + 1]):
                F += sz * 2.0 * float(i) * float(i)
            i += sz

    def step():
        ev.batched_generalized_packed(Sp, Tp, ns, soffs, toffs, sel, tile=args.tile, out=out,
                                      mode=args.mode, slices=args.slices)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    h = ev.handle(local_rank)
    sampler = ClockSampler() if rank == 0 else None
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1)
    clocks = sampler.stop() if sampler else None
    prof = profiled_steps(h, step, args.steps, dev)
    ev.sync(local_rank)
    if dist:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    value = world * cols * args.steps / (elapsed / 1e3)
    # end to end: S and T from pinned host memory, X and exponents back
    hS = torch.empty(Sp.numel(), dtype=torch.float64, pin_memory=True)
    hS.copy_(Sp.cpu())
    hT = torch.empty(Tp.numel(), dtype=torch.float64, pin_memory=True)
    hT.copy_(Tp.cpu())
    hX = torch.empty(out[0].numel(), dtype=torch.float64, pin_memory=True)
    hE = torch.empty(out[1].numel(), dtype=torch.int32, pin_memory=True)
    w0 = time.perf_counter()
    for _ in range(args.steps):
        Sp.copy_(hS, non_blocking=True)
        Tp.copy_(hT, non_blocking=True)
        step()
        hX.copy_(out[0], non_blocking=True)
        hE.copy_(out[1], non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e = {"value": world * cols * args.steps / (time.perf_counter() - w0),
           "unit": "columns/s", "h2d_bytes_per_step": (Sp.numel() + Tp.numel()) * 8,
           "d2h_bytes_per_step": out[0].numel() * 8 + out[1].numel() * 4}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    fp64_peak = N_SMS * FP64_FLOP_PER_CLK_PER_SM * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6
    kms = prof.get("batched", (0.0, 0))[0] / args.steps
    launches = prof.get("batched", (0.0, 0))[1] / args.steps
    achieved = F / (kms / 1e3) / 1e12 if kms > 0 else None
    roofline = {"kernel": "k_batched (pencils)", "bound": "alu", "achieved": achieved,
                "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak if achieved else None, "traffic": None,
                "peak_source": "of derived FP64 peak (measured 4 flop/clk/SM x 148 SMs x max "
                               "SM clock)",
                "launches_per_step": launches, "alg_flops_per_launch": F / max(launches, 1)}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rng = np.random.default_rng(9)
        pick = rng.choice(len(pairs), size=min(len(pairs), 200), replace=False)
        t = time.perf_counter()
        cc = 0
        for i in pick:
            X = oracle.generalized(pairs[i][0], pairs[i][1], select=sels[i])[0]
            cc += X.shape[1]
        dt = time.perf_counter() - t
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        cpu = {"value": cc / dt, "unit": "columns/s",
               "cores": int(os.environ.get("OMP_NUM_THREADS", cores)), "kind": "oracle",
               "sample": f"{len(pick)} randomly chosen pencils of the batch ({cc} columns), "
                         f"{dt:.2f} s"}
    line = {
        "metric": "eigvec columns/s, batched pencils (robust "
                  + ("generalized eigenvectors, split-precision updates)" if args.mode == "split"
                     else "FP64 generalized eigenvectors)"),
        "value": value, "unit": "columns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 slice products + f64" if args.mode == "split" else "f64",
        "data": "synthetic",
        "config": {"workload": f"batch of {args.batch} pencils, n log-uniform in [32, 1024] "
                               "(S config-0, T diag U[0.5, 2] with every 50th 1e-12), 30% of "
                               "blocks selected, no Z, one persistent launch per step",
                   "matrices": args.batch, "columns": cols,
                   "tile": args.tile or ("tuned" if args.mode == "fp64" else 64),
                   "tile_table": ev.tune_table(local_rank, "pencil"),
                   "mode": args.mode, "parallelism": "replicas",
                   "l2": f"inputs {(Sp.numel() + Tp.numel()) * 8 / 2**30:.1f} GiB, larger "
                         "than L2"},
        "tflops_fp64": F * args.steps / (elapsed / 1e3) / 1e12,
        "flops_per_step": F,
        "roofline": roofline,
        "rooflines": {"fp64": roofline},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": sum(c for _, c in prof.values()),
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def hessenberg_counts(n):
    """Algorithmic work of the Hessenberg reduction of order n with Q: flops
    10/3 n^3 for H (the two-sided reflector products, LAPACK's count) plus
    4/3 n^3 for forming Q, and the bytes the panel reductions' trailing
    matrix-vector products read, sum_c 8 n (n - c - 1) over the reduced
    columns c = 0 .. n - 3."""
    F = 14.0 / 3.0 * n ** 3
    Bpan = sum(8.0 * n * (n - c - 1) for c in range(max(n - 2, 0)))
    return F, Bpan


def run_hessenberg(args, rank, world, local_rank):
    """Hessenberg reduction A = Q H Q^T of an n x n N(0, 1) matrix with Q
    (evec_hessenberg).  Metric: reductions per second; rooflines: the panel
    reductions against HBM (the bytes their trailing matrix-vector products
    read), the updates against the FP64 pipe."""
    import ctypes

    import torch

    import paper_2002_05024_b300 as ev

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n
    A = np.random.default_rng(workloads.SEED_BASE + 9).standard_normal((n, n))
    dA0 = torch.from_numpy(np.asfortranarray(A)).to(dev)
    dA = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    dQ = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    h = ev.handle(local_rank)
    split = args.mode == "split"
    slices = (args.slices or 8) if split else 0
    opts = ev._opts(0, False, args.mode, slices)

    def step():
        dA.copy_(dA0)
        st = ev.lib().evec_hessenberg(h.ptr, n, dA.data_ptr(), n, dQ.data_ptr(), n,
                                      ctypes.byref(opts))
        if st:
            raise ev.EvecError(st, "evec_hessenberg")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    ev.sync(local_rank)
    sampler = ClockSampler() if rank == 0 else None
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1)
    clocks = sampler.stop() if sampler else None
    prof = profiled_steps(h, step, args.steps, dev)
    ev.sync(local_rank)
    if dist:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    # end to end: A in from pinned memory, H and Q out
    e2e = None
    if not os.environ.get("EVEC_BENCH_NO_E2E"):
        hA = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hA.copy_(torch.from_numpy(A))
        hH = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hQ = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            dA0.copy_(hA, non_blocking=True)
            step()
            hH.copy_(dA, non_blocking=True)
            hQ.copy_(dQ, non_blocking=True)
            torch.cuda.synchronize(dev)
        e2e = {"value": world * args.steps / (time.perf_counter() - w0), "unit": "reductions/s",
               "h2d_bytes_per_step": 8 * n * n, "d2h_bytes_per_step": 16 * n * n}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    H, Q = dA.cpu().numpy(), dQ.cpu().numpy()
    nrm = np.abs(A).max()
    quality = {"max_backward_error_over_nu_maxA": float(np.abs(Q @ H @ Q.T - A).max() / (n * 2.0 ** -53 * nrm)),
               "max_orthogonality_error_over_nu": float(np.abs(Q.T @ Q - np.eye(n)).max() / (n * 2.0 ** -53)),
               "zeros_below_subdiagonal": bool(np.all(np.tril(H, -2) == 0.0))}
    F, Bpan = hessenberg_counts(n)
    peaks = measured_peaks()
    fp64_peak = N_SMS * FP64_FLOP_PER_CLK_PER_SM * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6
    hbm = float(peaks.get("hbm_gbs") or 6400.0)
    roofs = {}
    pm, pn = prof.get("hess_panel", (0.0, 0))
    if pm > 0:
        # the trailing products need 2 flops per 8 bytes read, above B300's
        # FP64 balance (1.2 TFLOP/s against 6.5 TB/s): the FP64 pipe bounds
        # them before HBM does; both views are reported
        sec = pm / args.steps / 1e3
        Fp = 2.0 * Bpan / 8.0
        ach = Fp / sec / 1e12
        achb = Bpan / sec / 1e9
        roofs["hess_panel"] = {"kernel": "panel reduction (k_hs_panel, one cooperative launch per "
                                         "panel)",
                               "bound": "alu", "achieved": ach, "peak": fp64_peak,
                               "unit": "TFLOP/s", "frac": ach / fp64_peak,
                               "traffic": stored_traffic("hess_panel", "fp64", n, 32,
                                                         "hessenberg:"),
                               "peak_source": "of derived FP64 peak (measured 4 flop/clk/SM x 148 "
                                              "SMs x max SM clock)",
                               "hbm_view": {"achieved": achb, "peak": hbm, "unit": "GB/s",
                                            "frac": achb / hbm,
                                            "peak_source": "of measured" if peaks.get("hbm_gbs")
                                            else "of fallback"},
                               "launches_per_step": pn / args.steps,
                               "alg_flops_per_step": Fp, "alg_bytes_per_step": Bpan,
                               "ms_per_step": pm / args.steps}
    um, un = prof.get("hess_update", (0.0, 0))
    if um > 0 and split:
        # BF16 slice products: S (S + 1) / 2 digit pairs per FP64 multiply-add
        Fu = (F - 2.0 * Bpan / 8.0) * slices * (slices + 1) / 2
        ach = Fu / (um / args.steps / 1e3) / 1e12
        bf16 = float(peaks.get("bf16_tflops_sustained") or 1400.0)
        roofs["hess_update"] = {"kernel": "trailing / top / Q updates through the split GEMM "
                                          "(k_split_gemm with its slicing kernels)",
                                "bound": "tensor", "achieved": ach, "peak": bf16,
                                "unit": "TFLOP/s", "frac": ach / bf16, "traffic": None,
                                "peak_source": "of measured sustained BF16 (MEASURED_PEAKS.json)",
                                "launches_per_step": un / args.steps, "alg_flops_per_step": Fu,
                                "fp64_equivalent_tflops":
                                    (F - 2.0 * Bpan / 8.0) / (um / args.steps / 1e3) / 1e12,
                                "ms_per_step": um / args.steps}
    elif um > 0:
        Fu = F - 2.0 * Bpan / 8.0   # the products not done by the matrix-vector steps
        ach = Fu / (um / args.steps / 1e3) / 1e12
        roofs["hess_update"] = {"kernel": "trailing / top / Q updates (k_hs_gemm)", "bound": "alu",
                                "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                "frac": ach / fp64_peak,
                                "traffic": stored_traffic("hess_update", "fp64", n, 32,
                                                          "hessenberg:"),
                                "peak_source": "of derived FP64 peak (measured 4 flop/clk/SM x 148 "
                                               "SMs x max SM clock)",
                                "launches_per_step": un / args.steps, "alg_flops_per_step": Fu,
                                "ms_per_step": um / args.steps}
    dominant = max(roofs.items(), key=lambda kv: kv[1]["ms_per_step"])[0] if roofs else None
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ns = min(n, 1024)
        As = np.random.default_rng(3).standard_normal((ns, ns))
        t = time.perf_counter()
        oracle.hessenberg(As)
        dt = time.perf_counter() - t
        cpu = {"value": (1.0 / dt) * (ns / n) ** 3, "unit": "reductions/s", "cores": 1,
               "kind": "oracle",
               "sample": f"one unblocked reduction with Q at n = {ns} in {dt:.2f} s on one core, "
                         f"extrapolated to n = {n} by (n / {ns})^3"}
    line = {
        "metric": "Hessenberg reductions/s (A = Q H Q^T with Q, "
                  + (f"split-precision updates, {slices} slices)" if split else "FP64)"),
        "value": world * args.steps / (elapsed / 1e3), "unit": "reductions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 slice products + f64" if split else "f64",
        "data": "synthetic",
        "config": {"workload": f"Hessenberg reduction of an n={n} N(0, 1) matrix with Q, panels of "
                               "32 columns", "n": n, "panel": 32, "mode": args.mode,
                   "parallelism": "replicas",
                   "l2": f"inputs larger than L2 (A, H, Q {8 * n * n >> 20} MiB each)"},
        "tflops_fp64": F * args.steps / (elapsed / 1e3) / 1e12,
        "flops_per_step": F,
        "quality": quality,
        "roofline": roofs.get(dominant),
        "rooflines": roofs,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": sum(c for _, c in prof.values()),
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def window_what(n, k, count):
    return (f"eigenvalue reordering's off-diagonal updates: {count} disjoint windows of {k} "
            f"tiling the diagonal of an n={n} config-0 Schur form (boundaries off 2x2 blocks), "
            f"random orthogonal accumulators, with Q")


def window_flops(n, wins):
    """FP64 flops of the left and right updates and Q: 2 k^2 ((n - a) + (a + k) + n)
    per window."""
    return sum(2.0 * Z.shape[0] ** 2 * ((n - a) + (a + Z.shape[0]) + n) for a, Z in wins)


def run_window(args, rank, world, local_rank):
    """Eigenvalue reordering's off-diagonal updates (evec_window_update_set):
    the disjoint windows of one pass over the diagonal applied as one
    concurrent set to T (left and right updates) and Q.  Metric: windows per second; roofline: the FP64
    products against the FP64 pipe."""
    import ctypes

    import torch

    import paper_2002_05024_b300 as ev

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n, k = args.n, args.window
    T, blocks = workloads.config0_schur(n, seed=workloads.SEED_BASE)
    Q = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 100)
    wins = workloads.window_chain(n, k, k, seed=workloads.SEED_BASE + 9, blocks=blocks)
    dT = torch.from_numpy(np.asfortranarray(T)).to(dev)
    dQ = torch.from_numpy(np.asfortranarray(Q)).to(dev)
    begin, size, zoff, Zp = ev.pack_windows(wins, dev)
    h = ev.handle(local_rank)
    split = args.mode == "split"
    slices = args.slices or 8
    opts = ev._opts(0, False, args.mode, slices)

    def step():
        # each pass is one more orthogonal similarity of the same matrices
        # the pass's windows are disjoint: one concurrent set
        st = ev.lib().evec_window_update_set(h.ptr, n, dT.data_ptr(), n, dQ.data_ptr(), n,
                                             len(wins), ev._np_ptr(begin), ev._np_ptr(size),
                                             Zp.data_ptr(), ev._np_ptr(zoff), ctypes.byref(opts))
        if st:
            raise ev.EvecError(st, "evec_window_update_set")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    ev.sync(local_rank)
    sampler = ClockSampler() if rank == 0 else None
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1)
    clocks = sampler.stop() if sampler else None
    prof = profiled_steps(h, step, args.steps, dev)
    ev.sync(local_rank)
    if dist:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    e2e = None
    if not os.environ.get("EVEC_BENCH_NO_E2E"):
        # T and Q in from pinned memory, T and Q out, every step
        hT = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hQ = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hT.copy_(torch.from_numpy(T))
        hQ.copy_(torch.from_numpy(Q))
        oT = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        oQ = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            dT.copy_(hT, non_blocking=True)
            dQ.copy_(hQ, non_blocking=True)
            step()
            oT.copy_(dT, non_blocking=True)
            oQ.copy_(dQ, non_blocking=True)
            torch.cuda.synchronize(dev)
        e2e = {"value": world * len(wins) * args.steps / (time.perf_counter() - w0),
               "unit": "windows/s", "h2d_bytes_per_step": 16 * n * n,
               "d2h_bytes_per_step": 16 * n * n}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # quality: one pass from the original matrices keeps Q T Q^T (disjoint
    # windows: a similarity) and matches the oracle on three windows
    dT.copy_(torch.from_numpy(np.asfortranarray(T)))
    dQ.copy_(torch.from_numpy(np.asfortranarray(Q)))
    step()
    Tg, Qg = dT.cpu().numpy(), dQ.cpu().numpy()
    A = Q @ T @ Q.T
    quality = {"max_similarity_error_over_nu_maxA":
               float(np.abs(Qg @ Tg @ Qg.T - A).max() / (n * 2.0 ** -53 * np.abs(A).max())),
               "max_orthogonality_error_over_nu":
               float(np.abs(Qg.T @ Qg - np.eye(n)).max() / (n * 2.0 ** -53))}
    F = window_flops(n, wins)
    peaks = measured_peaks()
    fp64_peak = N_SMS * FP64_FLOP_PER_CLK_PER_SM * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6
    roof = None
    wm, wn = prof.get("window", (0.0, 0))
    if wm > 0 and split:
        # BF16 slice products: S (S + 1) / 2 digit pairs per FP64 product
        Fs = F * slices * (slices + 1) / 2
        ach = Fs / (wm / args.steps / 1e3) / 1e12
        bf16 = float(peaks.get("bf16_tflops_sustained") or 1400.0)
        roof = {"kernel": "the split products of every window (k_split_gemm with its slicing "
                          "kernels)",
                "bound": "tensor",
                "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                "traffic": stored_traffic("window", "split", n, k, "window:"),
                "peak_source": "of measured sustained BF16 (MEASURED_PEAKS.json)",
                "launches_per_step": wn / args.steps, "alg_flops_per_step": Fs,
                "fp64_equivalent_tflops": F / (wm / args.steps / 1e3) / 1e12,
                "ms_per_step": wm / args.steps}
    elif wm > 0:
        ach = F / (wm / args.steps / 1e3) / 1e12
        roof = {"kernel": "left and right updates of the set (k_win_left_set, k_win_right_set)",
                "bound": "alu",
                "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                "traffic": stored_traffic("window", "fp64", n, k, "window:"),
                "peak_source": "of derived FP64 peak (measured 4 flop/clk/SM x 148 SMs x max "
                               "SM clock)",
                "launches_per_step": wn / args.steps, "alg_flops_per_step": F,
                "ms_per_step": wm / args.steps}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        pick = [wins[0], wins[len(wins) // 2]]
        t = time.perf_counter()
        To, Qo = oracle.window_update(T, Q, pick)
        dt = time.perf_counter() - t
        dT.copy_(torch.from_numpy(np.asfortranarray(T)))
        dQ.copy_(torch.from_numpy(np.asfortranarray(Q)))
        ev.window_update(dT, dQ, pick, check=True, disjoint=True, mode=args.mode, slices=slices)
        quality["gpu_vs_oracle_two_windows"] = float(
            max(np.abs(dT.cpu().numpy() - To).max(), np.abs(dQ.cpu().numpy() - Qo).max()))
        cpu = {"value": len(pick) / dt, "unit": "windows/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(pick)} windows of the pass (the first and the middle one), "
                         f"plain loops on one core, {dt:.2f} s"}
    line = {
        "metric": "reordering windows/s (off-diagonal updates with Q, "
                  + (f"split precision, {slices} slices)" if split else "FP64)"),
        "value": world * len(wins) * args.steps / (elapsed / 1e3), "unit": "windows/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 slice products + f64" if split else "f64",
        "data": "synthetic",
        "config": {"workload": window_what(n, k, len(wins)), "n": n, "window": k,
                   "windows_per_step": len(wins), "parallelism": "replicas",
                   "l2": f"inputs larger than L2 (T and Q {8 * n * n >> 20} MiB each)"},
        "tflops_fp64": F * args.steps / (elapsed / 1e3) / 1e12,
        "flops_per_step": F,
        "quality": quality,
        "roofline": roof,
        "kernel_ms_per_step": {kk: v[0] / args.steps for kk, v in prof.items()},
        "gpu_launches": sum(c for _, c in prof.values()),
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_generalized(args, rank, world, local_rank):
    """The pencil workload: S config-0 (n x n), T upper triangular with
    diagonal U[0.5, 2] (every 50th entry 1e-12) and N(0, 1) upper part, Z from
    64 Householder reflectors, all eigenvectors, X = Z Y."""
    import torch

    import paper_2002_05024_b300 as ev

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n
    S, T, blocks = workloads.generalized_pair(n, seed=workloads.SEED_BASE + 4)
    Z = workloads.householder_orthogonal(n, seed=workloads.SEED_BASE + 104)
    dS = torch.from_numpy(np.asfortranarray(S)).to(dev)
    dT = torch.from_numpy(np.asfortranarray(T)).to(dev)
    dZ = torch.from_numpy(np.asfortranarray(Z)).to(dev)
    tile = args.tile or 64
    m = n
    # algorithmic FP64 flops: 2 k^2 (two products per substitution step) +
    # 2 n (k + b) for X = Z Y, k rows above the column's block
    F = 0.0
    for p, sz in blocks:
        F += sz * (2.0 * p * p + 2.0 * n * (p + sz))

    def step():
        return ev.generalized(dS, dT, dZ, tile=tile, mode=args.mode, slices=args.slices)

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize(dev)
    h = ev.handle(local_rank)
    sampler = ClockSampler() if rank == 0 else None
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        out = step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1)
    clocks = sampler.stop() if sampler else None
    prof = profiled_steps(h, step, args.steps, dev)
    ev.sync(local_rank)
    if dist:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    X, e, ar, ai, be = out
    # residual of 16 sampled eigenvalues in Schur coordinates (y = Z^T x)
    rng = np.random.default_rng(7)
    starts, col = [], 0
    for p, sz in blocks:
        starts.append((col, sz))
        col += sz
    Xh, arh, aih, beh = X.cpu().numpy(), ar.cpu().numpy(), ai.cpu().numpy(), be.cpu().numpy()
    S1 = np.abs(S).sum(axis=0).max()
    T1 = np.abs(np.triu(T)).sum(axis=0).max()
    worst = 0.0
    for b in rng.choice(len(starts), size=16, replace=False):
        c, sz = starts[b]
        x = Xh[:, c] + (1j * Xh[:, c + 1] if sz == 2 else 0.0)
        y = Z.T @ x
        al = arh[c] + 1j * aih[c]
        r = beh[c] * (S @ y) - al * (np.triu(T) @ y)
        den = (abs(beh[c]) * S1 + abs(al) * T1) * np.abs(y).sum() * np.finfo(np.float64).eps / 2
        worst = max(worst, float(np.abs(r).sum() / den))
    peaks = measured_peaks()
    fp64_peak = N_SMS * FP64_FLOP_PER_CLK_PER_SM * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6
    line = {
        "metric": "eigvec columns/s, generalized (robust FP64 eigenvectors of a pencil incl. X = Z Y)",
        "value": world * m * args.steps / (elapsed / 1e3), "unit": "columns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.mode == "fp64" else "bf16 slice products + f64",
        "data": "synthetic",
        "config": {"workload": f"pencil (S, T) n={n}, S config-0, T diag U[0.5, 2] with every "
                               "50th 1e-12, Z from 64 Householder reflectors, all columns",
                   "n": n, "columns": m, "tile": tile, "mode": args.mode,
                   "slices": (args.slices or 8) if args.mode == "split" else None,
                   "parallelism": "replicas"},
        "tflops_fp64": F * args.steps / (elapsed / 1e3) / 1e12,
        "fp64_peak_tflops": fp64_peak,
        "flops_per_step": F,
        "quality": {"eigenvalues": 16, "max_normalised_residual": worst, "max_over_n": worst / n,
                    "gate": "<= 10 n"},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": sum(c for _, c in prof.values()),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def solve_tiles(n, sub, nb):
    """Tile boundaries of the solve (rows; a 2x2 block is never cut): the
    plan's own rule, restated for the flop accounting."""
    ts = [0]
    while ts[-1] < n:
        b = ts[-1] + nb
        if b >= n:
            b = n
        elif sub[b - 1] != 0.0:   # b is the second row of a 2x2 block
            b -= 1
        ts.append(b)
    return ts


def trsolve_cpu_baseline(T, B, cols, seed=5, gpu=None):
    """The oracle's robust triangular solve, as it stands, on `cols` seeded
    random right-hand sides of the workload, on all host cores; with gpu =
    (X, scale_exp) the sampled columns are compared with the GPU's."""
    import oracle
    rng = np.random.default_rng(seed)
    nrhs = B.shape[1]
    pick = np.sort(rng.choice(nrhs, size=min(cols, nrhs), replace=False))
    Bs = np.asfortranarray(B[:, pick])
    oracle.build()
    t = time.perf_counter()
    X, e = oracle.trsolve(T, Bs)
    dt = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = {"value": len(pick) / dt, "unit": "right-hand sides/s",
           "cores": int(os.environ.get("OMP_NUM_THREADS", cores)), "kind": "oracle",
           "columns": len(pick), "seconds": dt,
           "sample": f"{len(pick)} randomly chosen right-hand sides (seed {seed}) of the "
                     f"n={T.shape[0]} system, {dt:.2f} s"}
    if gpu is not None:
        Xg, eg = gpu
        de = e.astype(np.int64) - eg[pick].astype(np.int64)
        a = X
        b = np.ldexp(Xg[:, pick], de[None, :])
        rel = np.abs(a - b).max(axis=0) / np.maximum(np.abs(a).max(axis=0), 1e-300)
        out["gpu_vs_oracle"] = {"columns": len(pick), "max_exponent_diff": int(np.abs(de).max()),
                                "max_rel_diff": float(rel.max())}
    return out


def run_trsolve(args, rank, world, local_rank):
    """The robust triangular solve T X = B diag(2^scale_exp)^-1 with many
    right-hand sides: T the n x n quasi-triangular system of
    workloads.solve_system (config-0 block structure, well conditioned), B
    n x nrhs N(0, 1).  Algorithmic flops n^2 per right-hand side (one
    multiply-add per entry of the strictly upper part, one division per
    row), of which the tile updates do 2 r_s b_s for tile s (r_s rows above
    it, b_s its rows) and the diagonal-tile solves the rest."""
    import torch

    import paper_2002_05024_b300 as ev

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n
    nrhs = args.nrhs or n
    T, blocks, B = workloads.solve_system(n, nrhs)
    tile = args.tile or 64
    ts = solve_tiles(n, np.diagonal(T, -1), tile)
    F = float(n) * n * nrhs
    F_upd = sum(2.0 * ts[s] * (ts[s + 1] - ts[s]) for s in range(1, len(ts) - 1)) * nrhs
    F_diag = F - F_upd
    dT = torch.from_numpy(T).to(dev)
    dB = torch.from_numpy(B).to(dev)
    X = torch.empty((nrhs, n), dtype=torch.float64, device=dev).t()
    e = torch.empty(nrhs, dtype=torch.int32, device=dev)

    def step():
        ev.trsolve(dT, dB, tile=args.tile, mode=args.mode, slices=args.slices, out=(X, e))

    ev.handle(local_rank).lookahead(args.lookahead)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    ev.sync(local_rank)
    h = ev.handle(local_rank)
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(gpu_id) if rank == 0 else None
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1)
    clocks = sampler.stop() if sampler else None
    ev.sync(local_rank)
    prof = profiled_steps(h, step, args.steps, dev)
    if dist:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    peaks = measured_peaks()
    slices = (args.slices or 8) if args.mode == "split" else 0
    roofs = rooflines(prof, args.steps, args.mode, slices, F_diag, F_upd, 0.0, peaks, n, tile,
                      prefix="trsolve:")
    dominant = max(prof.items(), key=lambda kv: kv[1][0])[0]

    # end to end through the public call: T and B from pinned host memory,
    # X and the exponents back, every step
    e2e = None
    if not os.environ.get("EVEC_BENCH_NO_E2E"):
        hT = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hT.copy_(torch.from_numpy(T))
        hB = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True).t()
        hB.copy_(torch.from_numpy(B))
        hX = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True).t()
        hE = torch.empty(nrhs, dtype=torch.int32, pin_memory=True)

        def host_step():
            dT.copy_(hT, non_blocking=True)
            dB.copy_(hB, non_blocking=True)
            step()
            hX.copy_(X, non_blocking=True)
            hE.copy_(e, non_blocking=True)
            torch.cuda.synchronize(dev)

        for _ in range(args.warmup):
            host_step()
        if dist:
            dist.barrier()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        w = time.perf_counter() - w0
        if dist:
            tt = torch.tensor([w], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            w = float(tt.item())
        e2e = {"value": world * nrhs * args.steps / w, "unit": "right-hand sides/s",
               "h2d_bytes_per_step": 8 * n * (n + nrhs),
               "d2h_bytes_per_step": 8 * n * nrhs + 4 * nrhs}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    Xh, eh = X.cpu().numpy(), e.cpu().numpy()
    # normalised residual ||T x - b||_1 / (||T||_1 ||x||_1 u) of 16 sampled
    # right-hand sides, in long double
    rng = np.random.default_rng(7)
    Tl = T.astype(np.longdouble)
    T1 = np.abs(Tl).sum(axis=0).max()
    worst = 0.0
    for j in rng.choice(nrhs, size=min(16, nrhs), replace=False):
        x = np.ldexp(Xh[:, j], -int(eh[j])).astype(np.longdouble)
        r = Tl @ x - B[:, j].astype(np.longdouble)
        worst = max(worst, float(np.abs(r).sum() / (T1 * np.abs(x).sum() * 2.0 ** -53)))
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = trsolve_cpu_baseline(T, B, args.cpu_sample, gpu=(Xh, eh))
        cpu.pop("columns")
        cpu.pop("seconds")
    line = {
        "metric": "right-hand sides/s (robust FP64 triangular solve with per-column scaling)",
        "value": world * nrhs * args.steps / (elapsed / 1e3), "unit": "right-hand sides/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.mode == "fp64" else "bf16 slice products + f64",
        "data": "synthetic",
        "config": {"workload": f"quasi-triangular T n={n} (config-0 blocks, well conditioned), "
                               f"B n x {nrhs} N(0, 1), "
                               + ("FP64" if args.mode == "fp64" else
                                  f"split precision ({slices} BF16 slices)"),
                   "n": n, "nrhs": nrhs, "tile": tile, "mode": args.mode,
                   "slices": slices or None, "parallelism": "replicas",
                   "l2": f"inputs larger than L2 (T {8 * n * n >> 20} MiB, B and X "
                         f"{8 * n * nrhs >> 20} MiB each)"},
        "tflops_fp64": F * args.steps / (elapsed / 1e3) / 1e12,
        "flops_per_step": F,
        "quality": {"right_hand_sides": int(min(16, nrhs)), "max_normalised_residual": worst,
                    "max_over_n": worst / n, "gate": "<= 10 n"},
        "roofline": roofs.get(dominant),
        "rooflines": roofs,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": sum(c for _, c in prof.values()),
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.workload == "generalized":
        run_generalized(args, rank, world, local_rank)
    elif args.workload == "trsolve":
        run_trsolve(args, rank, world, local_rank)
    elif args.workload == "batched_generalized":
        run_batched_generalized(args, rank, world, local_rank)
    elif args.workload == "hessenberg":
        run_hessenberg(args, rank, world, local_rank)
    elif args.workload == "window":
        run_window(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
