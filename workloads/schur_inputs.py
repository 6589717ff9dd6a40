"""Seeded generators for synthetic (generalized) real Schur forms.

All matrices are float64 in column-major (Fortran) order, which is the
storage the C ABI and the oracle expect.  Every generator returns the matrix
together with the list of its diagonal blocks ``(start, size)`` that it
placed, so callers can build selection masks without re-deriving structure.

Distributions (the paper's eigenvector experiments use generated Schur forms
whose construction it does not describe; these are the recipes used here):

* ``config0_schur(n)``: walk the diagonal; with probability 0.25 (when two
  rows remain) place a standardized 2x2 block [[a, b], [c, a]] with
  a ~ U[-1, 1], b ~ U[0.1, 1], c = -b*s, s ~ U[0.1, 1]; otherwise a 1x1 block
  with lambda ~ U[-1, 1].  Strictly upper part i.i.d. N(0, 1).
* ``adversarial_schur(n)``: all 1x1 blocks; four contiguous clusters with
  centres -0.75, -0.25, 0.25, 0.75; inside a cluster of size c the
  eigenvalues are centre + (k - c/2) * 1e-9, k = 0..c-1 in a seeded random
  order; strictly upper part N(0, 1) * 1e3.  Unscaled backsubstitution
  overflows on it.
* ``householder_orthogonal(n)``: product of 64 Householder reflectors
  I - 2 v v^T / v^T v with v ~ N(0, I), formed in compact WY form.
* ``generalized_pair(n)``: S as config0; T upper triangular with diagonal
  U[0.5, 2], every 50th diagonal entry 1e-12 (on 1x1 blocks; moved to the
  next 1x1 block when it lands on a pair), T's 2x2 block under an S pair is
  d*I with d ~ U[0.5, 2], strictly upper part N(0, 1).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20020502


def _rng(seed):
    return np.random.default_rng(seed)


def _place_blocks(n, rng, pair_prob=0.25):
    """Draw the 1x1/2x2 block layout and the diagonal-block entries."""
    blocks = []
    vals = []
    i = 0
    while i < n:
        if n - i >= 2 and rng.random() < pair_prob:
            a = rng.uniform(-1.0, 1.0)
            b = rng.uniform(0.1, 1.0)
            s = rng.uniform(0.1, 1.0)
            blocks.append((i, 2))
            vals.append((a, b, -b * s))
            i += 2
        else:
            blocks.append((i, 1))
            vals.append((rng.uniform(-1.0, 1.0),))
            i += 1
    return blocks, vals


def _strict_upper_normal(n, rng, scale=1.0, dtype=np.float64):
    """n x n column-major matrix with i.i.d. N(0, scale^2) strictly above the
    diagonal and zeros elsewhere."""
    A = rng.standard_normal((n, n))
    if scale != 1.0:
        A *= scale
    A = np.triu(A, 1)
    return np.asfortranarray(A, dtype=dtype)


def config0_schur(n: int, seed: int = SEED_BASE):
    """Config-0 distribution real Schur form (see module docstring)."""
    rng = _rng(seed)
    blocks, vals = _place_blocks(n, rng)
    T = _strict_upper_normal(n, rng)
    for (p, sz), v in zip(blocks, vals):
        if sz == 1:
            T[p, p] = v[0]
        else:
            a, b, c = v
            T[p, p] = a
            T[p + 1, p + 1] = a
            T[p, p + 1] = b
            T[p + 1, p] = c
    return T, blocks


def _cluster_sizes(n, parts=4):
    base = n // parts
    rem = n % parts
    return [base + (1 if k < rem else 0) for k in range(parts)]


def adversarial_schur(n: int, seed: int = SEED_BASE + 1, spacing: float = 1e-9,
                      upper_scale: float = 1e3):
    """Clustered real eigenvalues, large upper part (see module docstring)."""
    rng = _rng(seed)
    centres = (-0.75, -0.25, 0.25, 0.75)
    diag = np.empty(n)
    pos = 0
    for centre, c in zip(centres, _cluster_sizes(n)):
        order = rng.permutation(c)
        diag[pos:pos + c] = centre + (order - c / 2.0) * spacing
        pos += c
    T = _strict_upper_normal(n, rng, scale=upper_scale)
    T[np.arange(n), np.arange(n)] = diag
    blocks = [(i, 1) for i in range(n)]
    return T, blocks


def householder_orthogonal(n: int, seed: int = SEED_BASE + 100, reflectors: int = 64):
    """Q = H_1 H_2 ... H_k, H_i = I - tau_i v_i v_i^T, in compact WY form
    Q = I - V W V^T (W upper triangular).  Column-major float64."""
    rng = _rng(seed)
    k = min(reflectors, n)
    V = rng.standard_normal((n, k))
    tau = 2.0 / np.einsum("ij,ij->j", V, V)
    W = np.zeros((k, k))
    G = V.T @ V
    for j in range(k):
        W[j, j] = tau[j]
        if j:
            W[:j, j] = -tau[j] * (W[:j, :j] @ G[:j, j])
    Q = np.asfortranarray(-(V @ W) @ V.T)
    Q[np.arange(n), np.arange(n)] += 1.0
    return Q


def generalized_pair(n: int, seed: int = SEED_BASE + 4):
    """Generalized real Schur pair (S, T) (see module docstring)."""
    rng = _rng(seed)
    S, blocks = config0_schur(n, seed=int(rng.integers(1 << 62)))
    T = _strict_upper_normal(n, rng)
    d = rng.uniform(0.5, 2.0, size=n)
    pair_start = {p for p, sz in blocks if sz == 2}
    in_pair = set()
    for p in pair_start:
        in_pair.update((p, p + 1))
    for p, sz in blocks:
        if sz == 1:
            T[p, p] = d[p]
        else:
            T[p, p] = d[p]
            T[p + 1, p + 1] = d[p]
            T[p, p + 1] = 0.0
    # near-infinite eigenvalues: every 50th diagonal position, moved forward
    # to the next 1x1 block when it falls on a pair
    for target in range(49, n, 50):
        i = target
        while i < n and i in in_pair:
            i += 1
        if i < n:
            T[i, i] = 1e-12
    return S, T, blocks


def solve_system(n: int, nrhs: int, seed: int = SEED_BASE + 7):
    """A quasi-triangular system T X = B for the robust triangular solve:
    the config-0 block structure, 1x1 pivots moved to magnitude [1, 2)
    (sign kept), 2x2 blocks shifted by 1.5 on the diagonal with the second
    entry a further U[0, 0.25] up (no longer in standard form), the strictly
    upper part scaled to N(0, 1/n) so that T is well conditioned; B is
    N(0, 1), n x nrhs, column-major."""
    rng = _rng(seed)
    T, blocks = config0_schur(n, seed=int(rng.integers(1 << 62)))
    iu = np.triu_indices(n, 1)
    T[iu] /= np.sqrt(n)
    shift = rng.uniform(0.0, 0.25, size=n)
    for p, sz in blocks:
        if sz == 1:
            T[p, p] = (1.0 if T[p, p] >= 0 else -1.0) * (1.0 + abs(T[p, p]))
        else:
            T[p, p] += 1.5
            T[p + 1, p + 1] += 1.5 + shift[p]
    B = np.asfortranarray(rng.standard_normal((n, nrhs)))
    return T, blocks, B


def random_eigen_selection(n: int, blocks, fraction: float, seed: int):
    """Eigenvalue selection mask (uint8, length n): ``fraction`` of the
    eigenvalues chosen uniformly at random (the paper's experiment picks 35%
    of the eigenvalues at random)."""
    rng = _rng(seed)
    count = int(round(fraction * n))
    sel = np.zeros(n, dtype=np.uint8)
    sel[rng.permutation(n)[:count]] = 1
    return sel


def block_selection(n: int, blocks, fraction: float, seed: int):
    """Selection mask choosing an exact ``round(fraction * len(blocks))`` of
    the diagonal blocks from a seeded permutation; both eigenvalues of a
    chosen 2x2 block are marked."""
    rng = _rng(seed)
    count = int(round(fraction * len(blocks)))
    chosen = rng.permutation(len(blocks))[:count]
    sel = np.zeros(n, dtype=np.uint8)
    for b in chosen:
        p, sz = blocks[b]
        sel[p:p + sz] = 1
    return sel


def batch_sizes(count: int, seed: int = SEED_BASE + 3, lo: int = 32, hi: int = 1024):
    """Orders log-uniform in [lo, hi]: round(exp(U[ln lo, ln hi]))."""
    rng = _rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    return np.rint(np.exp(u)).astype(np.int64)


def batch_inputs(count: int, seed: int = SEED_BASE + 3, fraction: float = 0.3,
                 adversarial_every: int = 10):
    """Batch of independent Schur forms: sizes from ``batch_sizes``; member i
    uses seed SEED_BASE*10 + i; every ``adversarial_every``-th member
    (i % adversarial_every == adversarial_every - 1) is built like the
    clustered adversarial case; ``fraction`` of each member's blocks is
    selected.  Returns (sizes, list of T, list of selection masks)."""
    sizes = batch_sizes(count, seed)
    Ts, sels = [], []
    for i, n in enumerate(sizes):
        s = SEED_BASE * 10 + i
        if adversarial_every and i % adversarial_every == adversarial_every - 1:
            T, blocks = adversarial_schur(int(n), seed=s)
        else:
            T, blocks = config0_schur(int(n), seed=s)
        Ts.append(T)
        sels.append(block_selection(int(n), blocks, fraction, seed=s + 7))
    return sizes, Ts, sels


def batch_pencils(count: int, seed: int = SEED_BASE + 5, fraction: float = 0.3):
    """Batch of independent pencils (S_i, T_i) built like ``generalized_pair``:
    sizes from ``batch_sizes``, member i with seed SEED_BASE*10 + 5000 + i,
    ``fraction`` of each member's blocks selected.  Returns (sizes, list of
    (S, T), list of selection masks)."""
    sizes = batch_sizes(count, seed)
    pairs, sels = [], []
    for i, n in enumerate(sizes):
        s = SEED_BASE * 10 + 5000 + i
        S, T, blocks = generalized_pair(int(n), seed=s)
        pairs.append((S, T))
        sels.append(block_selection(int(n), blocks, fraction, seed=s + 7))
    return sizes, pairs, sels


def window_chain(n: int, k: int, stride: int, seed: int = SEED_BASE + 9, blocks=None):
    """A chain of overlapping diagonal windows as eigenvalue reordering moves
    a group of eigenvalues towards the top: windows of k rows and columns
    starting at n - k, n - k - stride, ... and a top one from row 0 that
    keeps the same overlap (stride = k: disjoint windows tiling the diagonal),
    each with a random k x k orthogonal accumulator (QR of a Gaussian
    matrix, columns signed so that R has a positive diagonal).  With the
    Schur form's blocks [(p, size), ...] no window boundary falls inside a
    2x2 block (a boundary there moves up by one row).  Returns a list of
    (begin, Z) with Z column-major float64."""
    rng = _rng(seed)
    wins = []                      # (begin, size): the top one clipped at 0
    a = n - k
    while a > 0:
        wins.append((a, k))
        a -= stride
    end = wins[-1][0] + k - stride if wins else n
    if end > 0:
        wins.append((0, min(end, n)))
    if blocks is not None:
        inner = {p + 1 for p, sz in blocks if sz == 2}
        fixed = []
        for a, kk in wins:
            b = a + kk
            a = a - 1 if a in inner else a
            b = b - 1 if b in inner else b
            if b > a:
                fixed.append((a, b - a))
        wins = fixed
    out = []
    for a, kk in wins:
        Z, R = np.linalg.qr(rng.standard_normal((kk, kk)))
        Z = Z * np.sign(np.where(np.diag(R) == 0.0, 1.0, np.diag(R)))
        out.append((int(a), np.asfortranarray(Z)))
    return out
