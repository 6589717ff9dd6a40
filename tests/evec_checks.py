"""Checkers shared by the tests: residuals, canonical-form comparisons and an
arbitrary-precision reference.  Plain numpy/mpmath; nothing here is part of
the oracle or of the CUDA path.

Conventions (both the oracle and the CUDA path return them):
  X[:, j] canonical, |X[:, j]|_inf in [1, 2) (a (Re, Im) column pair uses
  max_i |re_i| + |im_i| and shares one exponent);
  true eigenvector = X[:, j] * 2**(-e[j]).
"""
from __future__ import annotations

import math

import numpy as np

U = 2.0 ** -53


def column_groups(lam_im):
    """Yield (j, is_pair) over output columns: a pair occupies j, j+1 and is
    marked by lam_im[j] > 0 followed by lam_im[j+1] < 0."""
    j = 0
    m = len(lam_im)
    while j < m:
        if lam_im[j] != 0.0:
            yield j, True
            j += 2
        else:
            yield j, False
            j += 1


def complex_columns(X, lam_im):
    """List of complex vectors, one per eigenvalue (pairs merged)."""
    out = []
    for j, pair in column_groups(lam_im):
        if pair:
            out.append(X[:, j] + 1j * X[:, j + 1])
        else:
            out.append(X[:, j].astype(complex))
    return out


def standard_residuals(T, X, lam_re, lam_im):
    """||T x - lambda x||_1 / (||T||_1 ||x||_1 u) per eigenvalue.  T X is
    one real product (a pair's (Re, Im) columns give T x_re and T x_im),
    so T is never copied to a complex array."""
    T1 = np.abs(T).sum(axis=0).max()
    TX = T @ X
    res = []
    for j, pair in column_groups(lam_im):
        if pair:
            x = X[:, j] + 1j * X[:, j + 1]
            lam = lam_re[j] + 1j * lam_im[j]
            tx = TX[:, j] + 1j * TX[:, j + 1]
        else:
            x = X[:, j]
            lam = lam_re[j]
            tx = TX[:, j]
        r = tx - lam * x
        res.append(np.abs(r).sum() / (T1 * np.abs(x).sum() * U))
    return np.array(res)


def left_residuals(T, X, lam_re, lam_im):
    """||u^H T - lambda u^H||_1 / (||T||_inf ||u||_1 u) per eigenvalue, for
    left eigenvectors stored as (Re u, Im u): the residual of
    T^T conj(u) = lambda conj(u)."""
    Xc = np.array(X, dtype=np.float64, copy=True)
    for j, pair in column_groups(lam_im):
        if pair:
            Xc[:, j + 1] = -Xc[:, j + 1]
    return standard_residuals(np.ascontiguousarray(T.T), Xc, lam_re, lam_im)


def generalized_residuals(S, T, X, a_re, a_im, beta):
    """||beta S x - alpha T x||_1 / ((|beta| ||S||_1 + |alpha| ||T||_1) ||x||_1 u)
    (S X and T X as real products, as in standard_residuals)."""
    S1 = np.abs(S).sum(axis=0).max()
    T1 = np.abs(T).sum(axis=0).max()
    SX = S @ X
    TX = T @ X
    res = []
    for j, pair in column_groups(a_im):
        if pair:
            x = X[:, j] + 1j * X[:, j + 1]
            al = a_re[j] + 1j * a_im[j]
            sx = SX[:, j] + 1j * SX[:, j + 1]
            tx = TX[:, j] + 1j * TX[:, j + 1]
        else:
            x = X[:, j]
            al = a_re[j]
            sx, tx = SX[:, j], TX[:, j]
        r = beta[j] * sx - al * tx
        den = (abs(beta[j]) * S1 + abs(al) * T1) * np.abs(x).sum() * U
        res.append(np.abs(r).sum() / den)
    return np.array(res)


def generalized_left_residuals(S, T, X, a_re, a_im, beta):
    """||u^H (beta S - alpha T)||_1 / ((|beta| ||S||_inf + |alpha| ||T||_inf)
    ||u||_1 u) per eigenvalue, for left eigenvectors stored as (Re u, Im u):
    the residual of (beta S^T - alpha T^T) conj(u) = 0."""
    Xc = np.array(X, dtype=np.float64, copy=True)
    for j, pair in column_groups(a_im):
        if pair:
            Xc[:, j + 1] = -Xc[:, j + 1]
    return generalized_residuals(np.ascontiguousarray(S.T), np.ascontiguousarray(T.T), Xc,
                                 a_re, a_im, beta)


def flip_pencil(S, T):
    """(J S^T J, J T^T J), J the reversal permutation: the pencil whose right
    eigenvectors are the reversed conjugated left eigenvectors of (S, T)."""
    return (np.asfortranarray(S.T[::-1, ::-1]), np.asfortranarray(T.T[::-1, ::-1]))


def canonical_norms(X, lam_im):
    out = []
    for j, pair in column_groups(lam_im):
        if pair:
            out.append(np.max(np.abs(X[:, j]) + np.abs(X[:, j + 1])))
        else:
            out.append(np.max(np.abs(X[:, j])))
    return np.array(out)


def compare_canonical(Xa, ea, Xb, eb, lam_im):
    """Compare two canonical results column by column.
    Returns (max |exponent difference|, max normwise relative difference),
    after bringing b to a's exponent (the difference is at most one binade
    because both normalise the same true vector)."""
    max_de = 0
    max_rel = 0.0
    for j, pair in column_groups(lam_im):
        de = int(ea[j]) - int(eb[j])
        max_de = max(max_de, abs(de))
        cols = [j, j + 1] if pair else [j]
        a = Xa[:, cols]
        b = np.ldexp(Xb[:, cols], de)
        den = np.max(np.abs(a).sum(axis=1))
        rel = np.max(np.abs(a - b).sum(axis=1)) / den
        max_rel = max(max_rel, float(rel))
    return max_de, max_rel


# ---------------------------------------------------------------------------
# Arbitrary-precision reference (mpmath: 256-bit significand, unbounded
# exponent), the textbook definition: y zero below the block, the block part
# fixed by the normalisation convention, rows above from
# (T - lambda I) y = 0 by backsubstitution.
# ---------------------------------------------------------------------------

def mp_eigvec(T, p, size, prec=256):
    import mpmath as mp
    mp.mp.prec = prec
    n = T.shape[0]
    t = [[mp.mpf(float(T[i, j])) for j in range(n)] for i in range(n)]
    if size == 1:
        lam = t[p][p]
        y = [mp.mpc(0)] * n
        y[p] = mp.mpc(1)
    else:
        a, b, c = t[p][p], t[p][p + 1], t[p + 1][p]
        w = mp.sqrt(abs(b)) * mp.sqrt(abs(c))
        lam = mp.mpc(a, w)
        y = [mp.mpc(0)] * n
        if abs(b) >= abs(c):
            y[p] = mp.mpc(1)
            y[p + 1] = mp.mpc(0, w / b)
        else:
            y[p] = mp.mpc(-w / c)
            y[p + 1] = mp.mpc(0, 1)
    # block structure above p from the subdiagonal
    blocks = []
    i = 0
    while i < p:
        if i + 1 < n and T[i + 1, i] != 0.0:
            blocks.append((i, 2))
            i += 2
        else:
            blocks.append((i, 1))
            i += 1
    for q, qs in reversed(blocks):
        rhs = []
        for a_ in range(qs):
            s = mp.mpc(0)
            for j in range(q + qs, p + size):
                s += t[q + a_][j] * y[j]
            rhs.append(-s)
        if qs == 1:
            y[q] = rhs[0] / (t[q][q] - lam)
        else:
            m11 = t[q][q] - lam
            m12 = t[q][q + 1]
            m21 = t[q + 1][q]
            m22 = t[q + 1][q + 1] - lam
            det = m11 * m22 - m12 * m21
            y[q] = (rhs[0] * m22 - m12 * rhs[1]) / det
            y[q + 1] = (m11 * rhs[1] - m21 * rhs[0]) / det
    return y, lam


def mp_left_eigvec(T, p, size, prec=256):
    """Left eigenvector u (u^H T = lambda u^H) of the block at p, from the
    right-eigenvector reference on the flipped matrix T' = J T^T J (J the
    reversal permutation): T' is upper quasi-triangular with the same
    blocks, T'(J conj(u)) = lambda (J conj(u)), so u = conj(J y') with y'
    the eigenvector of T' for the block at n - p - size.  Returns (u, lam)."""
    import mpmath as mp
    n = T.shape[0]
    Tf = np.ascontiguousarray(T.T[::-1, ::-1])
    y, lam = mp_eigvec(Tf, n - p - size, size, prec)
    return [mp.conj(v) for v in reversed(y)], lam


def mp_canonical(y, pair):
    """Canonical (x as float64 array(s), exponent) of an mpmath vector."""
    import mpmath as mp
    if pair:
        nrm = max(abs(mp.re(v)) + abs(mp.im(v)) for v in y)
    else:
        nrm = max(abs(mp.re(v)) for v in y)
    t = int(mp.floor(mp.log(nrm, 2)))
    # guard the floor against rounding of log2 at exact powers of two
    if mp.mpf(2) ** t > nrm:
        t -= 1
    elif mp.mpf(2) ** (t + 1) <= nrm:
        t += 1
    xr = np.array([float(mp.re(v) / mp.mpf(2) ** t) for v in y])
    xi = np.array([float(mp.im(v) / mp.mpf(2) ** t) for v in y])
    return xr, xi, -t


# ---------------------------------------------------------------------------
# Extended-precision reference for large n (numpy longdouble: a 64-bit
# significand, 11 bits beyond FP64, and a 15-bit exponent, so an eigenvector
# growing by up to 2^16000 stays in range with no scaling).  The same
# textbook backsubstitution as mp_eigvec, vectorised row by row, for a real
# eigenvalue (a 1x1 block at row p, y_p = 1).
# ---------------------------------------------------------------------------

def longdouble_is_extended():
    return np.finfo(np.longdouble).nmant >= 63 and np.finfo(np.longdouble).maxexp >= 16384


def ld_real_eigvec(T, blocks, p):
    """y[0 : p + 1] of the eigenvalue T[p, p]; blocks = [(row, size)] of T."""
    LD = np.longdouble
    lam = LD(T[p, p])
    TL = np.asarray(T[:p + 1, :p + 1], dtype=LD)
    y = np.zeros(p + 1, LD)
    y[p] = 1
    for q, sz in reversed([b for b in blocks if b[0] < p]):
        if sz == 1:
            y[q] = -(TL[q, q + 1:] @ y[q + 1:]) / (TL[q, q] - lam)
        else:
            r0 = -(TL[q, q + 2:] @ y[q + 2:])
            r1 = -(TL[q + 1, q + 2:] @ y[q + 2:])
            a, b = TL[q, q] - lam, TL[q, q + 1]
            c, d = TL[q + 1, q], TL[q + 1, q + 1] - lam
            det = a * d - b * c
            y[q] = (d * r0 - b * r1) / det
            y[q + 1] = (a * r1 - c * r0) / det
    return y


def extended_errors(yref, x, e):
    """(direction error, error with the scale) of the canonical column x with
    exponent e (true vector x 2^-e) against the extended reference yref:
    the first after scaling x onto yref at yref's largest entry, the second
    as returned; both max-norm, relative to max |yref|."""
    LD = np.longdouble
    x = np.asarray(x[:len(yref)], dtype=LD)
    den = np.max(np.abs(yref))
    k = int(np.argmax(np.abs(yref)))
    direction = float(np.max(np.abs(yref - x * (yref[k] / x[k]))) / den)
    scaled = float(np.max(np.abs(yref - np.ldexp(x, -int(e)))) / den)
    return direction, scaled


def ulp_scale_ok(e, lo=-(2 ** 31) + 1, hi=2 ** 31 - 1):
    return all(lo <= int(v) <= hi for v in e)


def log2_floor(x):
    return int(math.floor(math.log2(x)))


def mp_gen_eigvec(S, T, p, size, prec=256):
    """Generalized eigenvector of (S, T) for block (p, size) in mpmath,
    from (beta S - alpha T) y = 0 with lambda = alpha / beta; the block part
    follows the library convention (1x1: y_p = 1; 2x2 with M = S_b - lambda
    T_b: (1, -m11 / m12) when |m12| >= |m21|, else (-i m22 / m21, i))."""
    import mpmath as mp
    mp.mp.prec = prec
    n = S.shape[0]
    s = [[mp.mpf(float(S[i, j])) for j in range(n)] for i in range(n)]
    t = [[mp.mpf(float(T[i, j])) if j >= i else mp.mpf(0) for j in range(n)] for i in range(n)]
    y = [mp.mpc(0)] * n
    if size == 1:
        al, be = s[p][p], t[p][p]
        y[p] = mp.mpc(1)
    else:
        s11, s12, s21, s22 = s[p][p], s[p][p + 1], s[p + 1][p], s[p + 1][p + 1]
        d1, d2 = t[p][p], t[p + 1][p + 1]
        # det(S_b - lambda diag(d1, d2)) = 0, root with positive imaginary part
        qa = d1 * d2
        qb = -(s11 * d2 + s22 * d1)
        qc = s11 * s22 - s12 * s21
        disc = qb * qb - 4 * qa * qc
        lam = (-qb + mp.sqrt(mp.mpc(disc))) / (2 * qa)
        if mp.im(lam) < 0:
            lam = mp.conj(lam)
        al, be = lam, mp.mpf(1)
        m11 = s11 - lam * d1
        m22 = s22 - lam * d2
        if abs(s12) >= abs(s21):
            y[p] = mp.mpc(1)
            y[p + 1] = -m11 / s12
        else:
            y[p + 1] = mp.mpc(0, 1)
            y[p] = -m22 * mp.mpc(0, 1) / s21
    blocks = []
    i = 0
    while i < p:
        if S[i + 1, i] != 0.0:
            blocks.append((i, 2))
            i += 2
        else:
            blocks.append((i, 1))
            i += 1
    for q, qs in reversed(blocks):
        rhs = []
        for a_ in range(qs):
            acc = mp.mpc(0)
            for j in range(q + qs, p + size):
                acc += (be * s[q + a_][j] - al * t[q + a_][j]) * y[j]
            rhs.append(-acc)
        if qs == 1:
            y[q] = rhs[0] / (be * s[q][q] - al * t[q][q])
        else:
            m11 = be * s[q][q] - al * t[q][q]
            m12 = be * s[q][q + 1] - al * t[q][q + 1]
            m21 = be * s[q + 1][q]
            m22 = be * s[q + 1][q + 1] - al * t[q + 1][q + 1]
            det = m11 * m22 - m12 * m21
            y[q] = (rhs[0] * m22 - m12 * rhs[1]) / det
            y[q + 1] = (m11 * rhs[1] - m21 * rhs[0]) / det
    return y


def mp_gen_left_eigvec(S, T, p, size, prec=256):
    """Left eigenvector u of the pencil (S, T), u^H (beta S - alpha T) = 0,
    for the block at p: from the right-eigenvector reference on the flipped
    pencil (J S^T J, J T^T J) (upper quasi-triangular and upper triangular,
    the same blocks in reverse order), u = conj(J y')."""
    import mpmath as mp
    n = S.shape[0]
    Sf, Tf = flip_pencil(S, T)
    y = mp_gen_eigvec(Sf, Tf, n - p - size, size, prec)
    return [mp.conj(v) for v in reversed(y)]
