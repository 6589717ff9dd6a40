/*
 * evec_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, column-by-column CPU oracle for the robust eigenvector
 * computation of the paper "Task-based, GPU-accelerated and Robust Library
 * for Solving Dense Nonsymmetric Eigenvalue Problems" (StarNEig):
 *
 *   - eigenvectors of a real upper quasi-triangular Schur form S by
 *     backsubstitution, (S - lambda_i I) y_i = 0           (Sec. 2, Eq. evec_solve)
 *   - generalized eigenvectors of a pair (S, T),
 *     (S - lambda_i T) y_i = 0, in homogeneous form          (Sec. 2, Eq. evec_solve)
 *   - back-transformation x_i = Q y_i  /  x_i = Z y_i       (Sec. 2, Eq. evec_backtransform)
 *   - left eigenvectors of S, u_i^H S = lambda_i u_i^H, by robust forward
 *     substitution (the transposed problem of Sec. 2), back-transformed
 *     by the same Q
 *   - the Hessenberg reduction A = Q H Q^T that precedes the Schur form
 *     (Sec. 3.1), by one Householder reflector per column applied from
 *     both sides, unblocked
 *   - the off-diagonal updates of eigenvalue reordering (Sec. 3.2, the
 *     window, left-update and right-update tasks): each window's
 *     accumulated orthogonal transform Z applied as T <- Zhat^T T Zhat,
 *     Q <- Q Zhat (Zhat = I with Z on the window), window by window
 *   - the robust triangular solve with many right-hand sides that the
 *     eigenvector solve generalises (Sec. 3.3, the LAPACK xLATRS lineage):
 *     T x_j = b_j for every column of B, each x_j = X[:, j] / 2^scale_exp[j]
 *   - robustness: every intermediate and final value stays in range; the
 *     vector is returned as  y = x / alpha  with alpha an integer power of
 *     two (the augmented representation of Sec. 3.3, "Robust computation of
 *     eigenvectors"), the exponent held in a
 *     32-bit signed integer (Sec. 3.3, last paragraph).
 *
 * Only tests/, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library.  It shares no code with the CUDA path.
 *
 * One column at a time, one scale exponent per column (LAPACK xLATRS style,
 * Sec. 3.3): no tiling, no blocking.  OpenMP runs independent columns in
 * parallel; every column is computed by the same sequential code, so the
 * result does not depend on the thread count.
 *
 * Readings where the paper is silent (the paper states only the guarantee
 * "no overflow", Sec. 3.3):
 *   OMEGA = 2^1020 is the overflow threshold for every intermediate value;
 *   inputs must satisfy |entry| <= 2^1000, so that any row sum of n <= 2^20
 *   entries stays below OMEGA.
 *   Small 1x1/2x2 (real or complex) systems: normalise the right-hand side to
 *   norm < 1, solve by complete pivoting with pivots perturbed up to smin,
 *   then choose a power-of-two scale so the solution stays below OMEGA.
 *   Update protection: before r <- r - B z with nu = |r|, tau = |B|, mu = |z|
 *   choose a power of two xi <= 1 with xi*nu + tau*xi*mu <= OMEGA.
 *   Canonical output: |x|_inf in [1, 2) (pairs: max_i |re_i| + |im_i|);
 *   true eigenvector = x * 2^(-scale_exp).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EVO_OK 0
#define EVO_EINVAL 1
#define EVO_ENOTSCHUR 2
#define EVO_ENONFINITE 3
#define EVO_ENOMEM 4

#define OMEGA 0x1p1020
#define INPUT_MAX 0x1p1000
#define ULP 0x1p-52
#define SAFMIN 0x1p-1022

typedef struct {
    int64_t start;  /* first row/column of the diagonal block */
    int size;       /* 1 or 2 */
} block_t;

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */

/* |a|_1 of a complex number, a cheap upper bound of its modulus. */
static double cabs1(double re, double im) { return fabs(re) + fabs(im); }

/* Complex division (a / b) by Smith's method: no intermediate exceeds
 * max(|a|)*2 / max(|b_re|, |b_im|). */
static void cdiv(double ar, double ai, double br, double bi, double *cr, double *ci)
{
    if (fabs(br) >= fabs(bi)) {
        double t = bi / br, d = br + bi * t;
        *cr = (ar + ai * t) / d;
        *ci = (ai - ar * t) / d;
    } else {
        double t = br / bi, d = bi + br * t;
        *cr = (ar * t + ai) / d;
        *ci = (ai * t - ar) / d;
    }
}

/* Scale a vector by 2^q. */
static void scale_vec(int64_t len, double *v, int64_t q)
{
    if (q == 0) return;
    for (int64_t i = 0; i < len; i++) v[i] = ldexp(v[i], (int)q);
}

/* ------------------------------------------------------------------ */
/* The small shifted systems on the diagonal blocks                     */
/* ------------------------------------------------------------------ */

/*
 * Solve M z = r for a k x k complex M (k = 1 or 2, stored row-major in
 * mr/mi) robustly.  Returns the exponent s <= 0: the computed z satisfies
 * M z = 2^s r (up to rounding) and |z| <= OMEGA componentwise.
 *   1. rhs normalised by an exact power of two to norm < 1;
 *   2. complete pivoting; a pivot whose |.|_1 is below smin is replaced by
 *      smin (the near-singular perturbation);
 *   3. the exponent s is fitted to the computed solution.
 */
static int64_t small_solve(int k, const double *mr, const double *mi,
                           const double *rr, const double *ri, double smin,
                           double *zr, double *zi)
{
    double rn = 0.0;
    for (int i = 0; i < k; i++) {
        double a = fabs(rr[i]) > fabs(ri[i]) ? fabs(rr[i]) : fabs(ri[i]);
        if (a > rn) rn = a;
    }
    if (rn == 0.0) {
        for (int i = 0; i < k; i++) { zr[i] = 0.0; zi[i] = 0.0; }
        return 0;
    }
    int kr = ilogb(rn) + 1;              /* 2^-kr * rn < 1 */
    double br[2], bi[2];
    for (int i = 0; i < k; i++) { br[i] = ldexp(rr[i], -kr); bi[i] = ldexp(ri[i], -kr); }

    double hr[2], hi[2];                 /* normalised solution */
    if (k == 1) {
        double pr = mr[0], pi = mi[0];
        if (cabs1(pr, pi) < smin) { pr = smin; pi = 0.0; }
        cdiv(br[0], bi[0], pr, pi, &hr[0], &hi[0]);
    } else {
        /* complete pivoting on the 2x2 matrix */
        int pr_row = 0, pc_col = 0;
        double best = -1.0;
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                double a = cabs1(mr[2 * i + j], mi[2 * i + j]);
                if (a > best) { best = a; pr_row = i; pc_col = j; }
            }
        /* permuted matrix a[i][j] = M[rowp[i]][colp[j]] */
        int rowp[2] = {pr_row, 1 - pr_row}, colp[2] = {pc_col, 1 - pc_col};
        double a11r = mr[2 * rowp[0] + colp[0]], a11i = mi[2 * rowp[0] + colp[0]];
        double a12r = mr[2 * rowp[0] + colp[1]], a12i = mi[2 * rowp[0] + colp[1]];
        double a21r = mr[2 * rowp[1] + colp[0]], a21i = mi[2 * rowp[1] + colp[0]];
        double a22r = mr[2 * rowp[1] + colp[1]], a22i = mi[2 * rowp[1] + colp[1]];
        double c1r = br[rowp[0]], c1i = bi[rowp[0]];
        double c2r = br[rowp[1]], c2i = bi[rowp[1]];
        if (cabs1(a11r, a11i) < smin) { a11r = smin; a11i = 0.0; }
        double lr, li;                   /* multiplier l = a21 / a11 */
        cdiv(a21r, a21i, a11r, a11i, &lr, &li);
        double ur = a22r - (lr * a12r - li * a12i);
        double ui = a22i - (lr * a12i + li * a12r);
        if (cabs1(ur, ui) < smin) { ur = smin; ui = 0.0; }
        double d2r = c2r - (lr * c1r - li * c1i);
        double d2i = c2i - (lr * c1i + li * c1r);
        double w2r, w2i, w1r, w1i, gr, gi, qr, qi;
        cdiv(d2r, d2i, ur, ui, &w2r, &w2i);
        cdiv(c1r, c1i, a11r, a11i, &qr, &qi);      /* c1 / a11 */
        cdiv(a12r, a12i, a11r, a11i, &gr, &gi);    /* a12 / a11, |.| <= 2 */
        w1r = qr - (gr * w2r - gi * w2i);
        w1i = qi - (gr * w2i + gi * w2r);
        /* undo the column permutation: w_j is the unknown of column colp[j] */
        hr[colp[0]] = w1r; hi[colp[0]] = w1i;
        hr[colp[1]] = w2r; hi[colp[1]] = w2i;
    }
    double hn = 0.0;
    for (int i = 0; i < k; i++) {
        double a = fabs(hr[i]) > fabs(hi[i]) ? fabs(hr[i]) : fabs(hi[i]);
        if (a > hn) hn = a;
    }
    if (hn == 0.0) {
        for (int i = 0; i < k; i++) { zr[i] = 0.0; zi[i] = 0.0; }
        return 0;
    }
    /* s: largest exponent <= 0 with 2^(kr + s) * hn <= OMEGA */
    int64_t s = (int64_t)ilogb(OMEGA) - (int64_t)ilogb(hn) - 1 - kr;
    if (s > 0) s = 0;
    for (int i = 0; i < k; i++) {
        zr[i] = ldexp(hr[i], (int)(kr + s));
        zi[i] = ldexp(hi[i], (int)(kr + s));
    }
    return s;
}

/*
 * Update protection (Sec. 3.3: the preprocessing that makes z = y - T x
 * safe).  Given nu = |r|_inf <= OMEGA, tau = |B|_inf <= OMEGA and
 * mu = |z|_inf, return q <= 0 such that 2^q nu + tau 2^q mu <= OMEGA.
 */
static int64_t protect_update(double nu, double tau, double mu)
{
    if (mu <= 1.0) {
        if (tau * mu > OMEGA - nu) return -1;
    } else {
        if (tau > (OMEGA - nu) / mu) return -1 - ((int64_t)ilogb(mu) + 1);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Block scan and validation                                            */
/* ------------------------------------------------------------------ */

#define AT(M, ld, i, j) ((M)[(int64_t)(j) * (ld) + (i)])

/* Finiteness and magnitude of the referenced part (upper triangle plus the
 * first subdiagonal when sub != 0). */
static int check_entries(int64_t n, const double *A, int64_t lda, int sub, int64_t *bad)
{
    for (int64_t j = 0; j < n; j++) {
        int64_t iend = j + (sub ? 2 : 1);
        if (iend > n) iend = n;
        for (int64_t i = 0; i < iend; i++) {
            double v = AT(A, lda, i, j);
            if (!isfinite(v)) { if (bad) *bad = j * n + i; return EVO_ENONFINITE; }
            if (fabs(v) > INPUT_MAX) { if (bad) *bad = j * n + i; return EVO_EINVAL; }
        }
    }
    return EVO_OK;
}

/* 1x1 / 2x2 block structure from the first subdiagonal of S (Sec. 2: the
 * Schur form has 1x1 and 2x2 diagonal blocks).  standardized != 0 requires
 * the standard-problem form of a 2x2 block: equal diagonal entries and
 * off-diagonal entries of opposite sign. */
static int scan_blocks(int64_t n, const double *S, int64_t lds, int standardized,
                       block_t *blk, int64_t *nblk, int64_t *bad)
{
    int64_t i = 0, k = 0;
    while (i < n) {
        if (i + 1 < n && AT(S, lds, i + 1, i) != 0.0) {
            if (i + 2 < n && AT(S, lds, i + 2, i + 1) != 0.0) {
                if (bad) *bad = i + 1;
                return EVO_ENOTSCHUR;
            }
            if (standardized) {
                double a = AT(S, lds, i, i), d = AT(S, lds, i + 1, i + 1);
                double b = AT(S, lds, i, i + 1), c = AT(S, lds, i + 1, i);
                if (a != d || !((b > 0.0 && c < 0.0) || (b < 0.0 && c > 0.0))) {
                    if (bad) *bad = i;
                    return EVO_ENOTSCHUR;
                }
            }
            blk[k].start = i; blk[k].size = 2; k++; i += 2;
        } else {
            blk[k].start = i; blk[k].size = 1; k++; i += 1;
        }
    }
    *nblk = k;
    return EVO_OK;
}

/* |A[0:rows, c0:c0+cols]|_inf (largest row sum). */
static double block_col_norm(const double *A, int64_t lda, int64_t rows, int64_t c0, int cols)
{
    double m = 0.0;
    for (int64_t r = 0; r < rows; r++) {
        double s = 0.0;
        for (int j = 0; j < cols; j++) s += fabs(AT(A, lda, r, c0 + j));
        if (s > m) m = s;
    }
    return m;
}

/* |A[r0:r0+rows, c0:n]^T|_inf (largest column sum of the block rows right of
 * column c0): the bound of a forward-substitution update from those rows. */
static double block_row_norm(const double *A, int64_t lda, int64_t n, int64_t r0, int rows,
                             int64_t c0)
{
    double m = 0.0;
    for (int64_t c = c0; c < n; c++) {
        double s = 0.0;
        for (int a = 0; a < rows; a++) s += fabs(AT(A, lda, r0 + a, c));
        if (s > m) m = s;
    }
    return m;
}

/* Number of output columns: a 2x2 block is selected when either of its two
 * eigenvalues is, and then yields two real columns (Re, Im). */
static int64_t count_columns(const block_t *blk, int64_t nblk, const uint8_t *select)
{
    int64_t m = 0;
    for (int64_t k = 0; k < nblk; k++) {
        int64_t p = blk[k].start;
        int sel = select == NULL || select[p] || (blk[k].size == 2 && select[p + 1]);
        if (sel) m += blk[k].size;
    }
    return m;
}

/* ------------------------------------------------------------------ */
/* One eigenvector by robust backsubstitution                           */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    const double *S; int64_t lds;     /* quasi-triangular */
    const double *T; int64_t ldt;     /* upper triangular, generalized only */
    const block_t *blk; int64_t nblk;
    const double *tauS;               /* per block: |S[0:start, block]|_inf */
    const double *tauT;               /* per block: |T[0:start, block]|_inf */
    const double *tauL;               /* per block: |S[block, end:n]^T|_inf (left) */
    const double *tauLT;              /* per block: |T[block, end:n]^T|_inf (left, pencil) */
    double smax, tmax;                /* max |S_ii|, max |T_ii| (generalized smin) */
} problem_t;

/*
 * Backsubstitution for diagonal block k with eigenvalue  alpha / beta
 * (standard problem: beta = 1 and the matrix is S - lambda I).
 * On return y (yr, yi; yi unused when the eigenvalue is real) holds the
 * eigenvector scaled by 2^e: y_true = y * 2^-e.  Rows below the block are 0.
 */
static void solve_one(const problem_t *P, int generalized, int64_t k,
                      double ar, double ai, double beta,
                      const double *own_r, const double *own_i,
                      double *yr, double *yi, int64_t *e_out)
{
    const int64_t n = P->n;
    const int cplx = ai != 0.0;
    const block_t *B = P->blk;
    const int64_t p = B[k].start;
    const int bs = B[k].size;
    int64_t e = 0;
    double smin;
    if (generalized)
        smin = ULP * (fabs(beta) * P->smax + cabs1(ar, ai) * P->tmax);
    else
        smin = ULP * cabs1(ar, ai);
    double smlnum = SAFMIN * ((double)n / ULP);
    if (smin < smlnum) smin = smlnum;

    memset(yr, 0, sizeof(double) * n);
    if (cplx) memset(yi, 0, sizeof(double) * n);
    for (int j = 0; j < bs; j++) {
        yr[p + j] = own_r[j];
        if (cplx) yi[p + j] = own_i[j];
    }
    /* right-hand side rows 0..p-1 receive  -(beta S - alpha T)[0:p, block] y_block
       through the same protected update as every later block */
    int64_t cur = k;            /* the block whose solution was just fixed */
    for (;;) {
        const int64_t q = B[cur].start;
        const int cb = B[cur].size;
        if (q > 0) {
            /* --- protect, then apply r[0:q] -= C[0:q, block] z ---------- */
            double nu = 0.0, mu = 0.0;
            for (int64_t r = 0; r < q; r++) {
                double a = fabs(yr[r]);
                if (cplx && fabs(yi[r]) > a) a = fabs(yi[r]);
                if (a > nu) nu = a;
            }
            for (int j = 0; j < cb; j++) {
                double a = fabs(yr[q + j]);
                if (cplx && fabs(yi[q + j]) > a) a = fabs(yi[q + j]);
                if (a > mu) mu = a;
            }
            double tau;
            if (generalized)
                tau = fabs(beta) * P->tauS[cur] + cabs1(ar, ai) * P->tauT[cur];
            else
                tau = P->tauS[cur];
            int64_t s = protect_update(nu, tau, mu);
            if (s != 0) {
                scale_vec(n, yr, s);
                if (cplx) scale_vec(n, yi, s);
                e += s;
            }
            for (int j = 0; j < cb; j++) {
                const double zr = yr[q + j], zi = cplx ? yi[q + j] : 0.0;
                const double *Sc = &AT(P->S, P->lds, 0, q + j);
                if (!generalized) {
                    for (int64_t r = 0; r < q; r++) yr[r] -= Sc[r] * zr;
                    if (cplx)
                        for (int64_t r = 0; r < q; r++) yi[r] -= Sc[r] * zi;
                } else {
                    /* C = beta S - alpha T, alpha complex:
                       C z = beta S z - (ar + i ai) T (zr + i zi) */
                    const double *Tc = &AT(P->T, P->ldt, 0, q + j);
                    for (int64_t r = 0; r < q; r++) {
                        double sv = beta * Sc[r];
                        double tr = Tc[r];
                        yr[r] -= sv * zr - tr * (ar * zr - ai * zi);
                        if (cplx) yi[r] -= sv * zi - tr * (ar * zi + ai * zr);
                    }
                }
            }
        }
        if (cur == 0) break;
        /* --- solve the next block up: (C_ii) z = r_i ------------------ */
        cur -= 1;
        const int64_t i0 = B[cur].start;
        const int ib = B[cur].size;
        double mr[4], mi[4], rr[2], ri[2], zr[2], zi[2];
        for (int a = 0; a < ib; a++) {
            for (int b = 0; b < ib; b++) {
                double sv = AT(P->S, P->lds, i0 + a, i0 + b);
                if (!generalized) {
                    mr[a * ib + b] = sv - (a == b ? ar : 0.0);
                    mi[a * ib + b] = (a == b ? -ai : 0.0);
                } else {
                    double tv = (b >= a) ? AT(P->T, P->ldt, i0 + a, i0 + b) : 0.0;
                    mr[a * ib + b] = beta * sv - ar * tv;
                    mi[a * ib + b] = -ai * tv;
                }
            }
            rr[a] = yr[i0 + a];
            ri[a] = cplx ? yi[i0 + a] : 0.0;
        }
        int64_t s = small_solve(ib, mr, mi, rr, ri, smin, zr, zi);
        if (s != 0) {
            scale_vec(n, yr, s);
            if (cplx) scale_vec(n, yi, s);
            e += s;
        }
        for (int a = 0; a < ib; a++) {
            yr[i0 + a] = zr[a];
            if (cplx) yi[i0 + a] = zi[a];
        }
    }
    *e_out = e;
}

/*
 * Left eigenvector of block k of the standard problem, lambda = ar + i ai
 * (generalized: of the pencil, eigenvalue alpha / beta with alpha = ar + i ai;
 * the matrix S - lambda I below is then beta S - alpha T, and the bound of an
 * update |beta| |S[..]| + |alpha|_1 |T[..]|).
 * A left eigenvector satisfies u^H S = lambda u^H; with w = conj(u) this is
 * w^T (S - lambda I) = 0, the transposed system, solved by forward
 * substitution over the blocks after k: w is zero above block k, fixed on
 * it by own_r/own_i, and each later block i solves
 *   (S_ii - lambda I)^T w_i = r_i,   r = -(S[rows before i, block i])^T w,
 * with r accumulated block by block through protected updates (the bound of
 * an update from block q is |S[block q, after q]^T|_inf).  On return w (wr,
 * wi) holds w_true * 2^e; rows above the block are 0.
 */
static void solve_one_left(const problem_t *P, int generalized, int64_t k, double ar, double ai,
                           double beta, const double *own_r, const double *own_i,
                           double *wr, double *wi, int64_t *e_out)
{
    const int64_t n = P->n;
    const int cplx = ai != 0.0;
    const block_t *B = P->blk;
    const int64_t p = B[k].start;
    const int bs = B[k].size;
    int64_t e = 0;
    double smin;
    if (generalized)
        smin = ULP * (fabs(beta) * P->smax + cabs1(ar, ai) * P->tmax);
    else
        smin = ULP * cabs1(ar, ai);
    double smlnum = SAFMIN * ((double)n / ULP);
    if (smin < smlnum) smin = smlnum;

    memset(wr, 0, sizeof(double) * n);
    if (cplx) memset(wi, 0, sizeof(double) * n);
    for (int j = 0; j < bs; j++) {
        wr[p + j] = own_r[j];
        if (cplx) wi[p + j] = own_i[j];
    }
    int64_t cur = k;            /* the block whose part of w was just fixed */
    for (;;) {
        const int64_t q = B[cur].start;
        const int cb = B[cur].size;
        const int64_t q1 = q + cb;
        if (q1 < n) {
            /* --- protect, then apply r[q1:n] -= S[block, q1:n]^T z ------ */
            double nu = 0.0, mu = 0.0;
            for (int64_t r = q1; r < n; r++) {
                double a = fabs(wr[r]);
                if (cplx && fabs(wi[r]) > a) a = fabs(wi[r]);
                if (a > nu) nu = a;
            }
            for (int j = 0; j < cb; j++) {
                double a = fabs(wr[q + j]);
                if (cplx && fabs(wi[q + j]) > a) a = fabs(wi[q + j]);
                if (a > mu) mu = a;
            }
            const double tau = generalized
                                   ? fabs(beta) * P->tauL[cur] + cabs1(ar, ai) * P->tauLT[cur]
                                   : P->tauL[cur];
            int64_t s = protect_update(nu, tau, mu);
            if (s != 0) {
                scale_vec(n, wr, s);
                if (cplx) scale_vec(n, wi, s);
                e += s;
            }
            for (int j = 0; j < cb; j++) {
                const double zr = wr[q + j], zi = cplx ? wi[q + j] : 0.0;
                for (int64_t c = q1; c < n; c++) {
                    const double sv = AT(P->S, P->lds, q + j, c);
                    if (!generalized) {
                        wr[c] -= sv * zr;
                        if (cplx) wi[c] -= sv * zi;
                    } else {
                        /* C^T z with C = beta S - alpha T, alpha complex */
                        const double bsv = beta * sv, tv = AT(P->T, P->ldt, q + j, c);
                        wr[c] -= bsv * zr - tv * (ar * zr - ai * zi);
                        if (cplx) wi[c] -= bsv * zi - tv * (ar * zi + ai * zr);
                    }
                }
            }
        }
        if (cur == P->nblk - 1) break;
        /* --- solve the next block down: (S_ii - lambda I)^T z = r_i ------ */
        cur += 1;
        const int64_t i0 = B[cur].start;
        const int ib = B[cur].size;
        double mr[4], mi[4], rr[2], ri[2], zr[2], zi[2];
        for (int a = 0; a < ib; a++) {
            for (int b = 0; b < ib; b++) {
                /* the transposed block: entry (a, b) is C[i0 + b, i0 + a] */
                const double sv = AT(P->S, P->lds, i0 + b, i0 + a);
                if (!generalized) {
                    mr[a * ib + b] = sv - (a == b ? ar : 0.0);
                    mi[a * ib + b] = (a == b ? -ai : 0.0);
                } else {
                    const double tv = (a >= b) ? AT(P->T, P->ldt, i0 + b, i0 + a) : 0.0;
                    mr[a * ib + b] = beta * sv - ar * tv;
                    mi[a * ib + b] = -ai * tv;
                }
            }
            rr[a] = wr[i0 + a];
            ri[a] = cplx ? wi[i0 + a] : 0.0;
        }
        int64_t s = small_solve(ib, mr, mi, rr, ri, smin, zr, zi);
        if (s != 0) {
            scale_vec(n, wr, s);
            if (cplx) scale_vec(n, wi, s);
            e += s;
        }
        for (int a = 0; a < ib; a++) {
            wr[i0 + a] = zr[a];
            if (cplx) wi[i0 + a] = zi[a];
        }
    }
    *e_out = e;
}

/* Canonical form: scale by 2^-t with t = floor(log2 |y|), |y| = max_i |y_i|
 * (complex: max_i |re_i| + |im_i|), so |x| lies in [1, 2).  Returns t. */
static int64_t canonicalize(int64_t n, double *yr, double *yi, int cplx)
{
    double m = 0.0;
    for (int64_t r = 0; r < n; r++) {
        double a = cplx ? fabs(yr[r]) + fabs(yi[r]) : fabs(yr[r]);
        if (a > m) m = a;
    }
    if (m == 0.0) return 0;
    int64_t t = ilogb(m);
    scale_vec(n, yr, -t);
    if (cplx) scale_vec(n, yi, -t);
    return t;
}

/* x = Q y (Eq. evec_backtransform), plain loops. */
static void back_transform(int64_t n, const double *Q, int64_t ldq, const double *y, double *x)
{
    for (int64_t r = 0; r < n; r++) x[r] = 0.0;
    for (int64_t j = 0; j < n; j++) {
        double v = y[j];
        if (v == 0.0) continue;
        const double *Qc = &AT(Q, ldq, 0, j);
        for (int64_t r = 0; r < n; r++) x[r] += Qc[r] * v;
    }
}

/* ------------------------------------------------------------------ */
/* Drivers                                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t blk;       /* block index */
    int64_t col;       /* first output column */
} job_t;

static int run_jobs(const problem_t *P, int generalized, int left, const double *Q, int64_t ldq,
                    const job_t *jobs, int64_t njobs,
                    const double *lre, const double *lim, const double *lbeta,
                    const double *own, /* per block: 4 values (own_r[2], own_i[2]) */
                    double *X, int64_t ldx, int32_t *scale_exp, int nthreads)
{
    const int64_t n = P->n;
    int status = EVO_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *yr = (double *)malloc(sizeof(double) * n);
        double *yi = (double *)malloc(sizeof(double) * n);
        double *xr = Q ? (double *)malloc(sizeof(double) * n) : NULL;
        int ok = yr && yi && (!Q || xr);
        if (!ok) {
#pragma omp atomic write
            status = EVO_ENOMEM;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < njobs; t++) {
            if (!ok) continue;
            const int64_t k = jobs[t].blk, col = jobs[t].col;
            const double ar = lre[k], ai = lim[k], beta = lbeta ? lbeta[k] : 1.0;
            const int cplx = ai != 0.0;
            int64_t e = 0;
            if (left) {
                /* w = conj(u): the stored columns are (Re u, Im u) */
                solve_one_left(P, generalized, k, ar, ai, beta, &own[4 * k], &own[4 * k + 2], yr,
                               yi, &e);
                if (cplx)
                    for (int64_t r = 0; r < n; r++) yi[r] = -yi[r];
            } else {
                solve_one(P, generalized, k, ar, ai, beta, &own[4 * k], &own[4 * k + 2], yr, yi,
                          &e);
            }
            int64_t tcan = canonicalize(n, yr, yi, cplx);
            e -= tcan;
            if (Q) {
                back_transform(n, Q, ldq, yr, xr);
                memcpy(yr, xr, sizeof(double) * n);
                if (cplx) {
                    back_transform(n, Q, ldq, yi, xr);
                    memcpy(yi, xr, sizeof(double) * n);
                }
                tcan = canonicalize(n, yr, yi, cplx);
                e -= tcan;
            }
            if (e > INT32_MAX || e < INT32_MIN) {
#pragma omp atomic write
                status = EVO_EINVAL;
                continue;
            }
            memcpy(&AT(X, ldx, 0, col), yr, sizeof(double) * n);
            scale_exp[col] = (int32_t)e;
            if (cplx) {
                memcpy(&AT(X, ldx, 0, col + 1), yi, sizeof(double) * n);
                scale_exp[col + 1] = (int32_t)e;
            }
        }
        free(yr); free(yi); free(xr);
    }
    return status;
}

/* Number of output columns for a selection (NULL = all). */
int evo_count(int64_t n, const double *S, int64_t lds, const uint8_t *select,
              int64_t *m, int64_t *bad)
{
    if (n < 0 || lds < (n > 0 ? n : 1) || !m) return EVO_EINVAL;
    if (n == 0) { *m = 0; return EVO_OK; }
    block_t *blk = (block_t *)malloc(sizeof(block_t) * n);
    if (!blk) return EVO_ENOMEM;
    int64_t nblk = 0;
    int st = scan_blocks(n, S, lds, 0, blk, &nblk, bad);
    if (st == EVO_OK) *m = count_columns(blk, nblk, select);
    free(blk);
    return st;
}

/* Right (left = 0) or left (left = 1) eigenvectors of the standard problem. */
static int standard_impl(int left, int64_t n, const double *S, int64_t lds, const double *Q,
                         int64_t ldq, const uint8_t *select, double *X, int64_t ldx,
                         int32_t *scale_exp, double *lam_re, double *lam_im, int nthreads,
                         int64_t *bad)
{
    if (n < 0 || lds < (n > 0 ? n : 1) || ldx < (n > 0 ? n : 1)) return EVO_EINVAL;
    if (Q && ldq < (n > 0 ? n : 1)) return EVO_EINVAL;
    if (n == 0) return EVO_OK;
    int st = check_entries(n, S, lds, 1, bad);
    if (st) return st;
    block_t *blk = (block_t *)malloc(sizeof(block_t) * n);
    double *tau = (double *)malloc(sizeof(double) * n);
    double *lre = (double *)malloc(sizeof(double) * n);
    double *lim = (double *)malloc(sizeof(double) * n);
    double *own = (double *)malloc(sizeof(double) * 4 * n);
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * n);
    int64_t nblk = 0;
    if (!blk || !tau || !lre || !lim || !own || !jobs) { st = EVO_ENOMEM; goto done; }
    st = scan_blocks(n, S, lds, 1, blk, &nblk, bad);
    if (st) goto done;

    int64_t njobs = 0, col = 0;
    for (int64_t k = 0; k < nblk; k++) {
        const int64_t p = blk[k].start;
        tau[k] = left ? block_row_norm(S, lds, n, p, blk[k].size, p + blk[k].size)
                      : block_col_norm(S, lds, p, p, blk[k].size);
        double *o = &own[4 * k];
        if (blk[k].size == 1) {
            lre[k] = AT(S, lds, p, p); lim[k] = 0.0;
            o[0] = 1.0; o[1] = 0.0; o[2] = 0.0; o[3] = 0.0;
        } else {
            /* eigenvalues of [[a, b], [c, a]], bc < 0:  a +- i sqrt(|b|) sqrt(|c|) */
            double a = AT(S, lds, p, p), b = AT(S, lds, p, p + 1), c = AT(S, lds, p + 1, p);
            double w = sqrt(fabs(b)) * sqrt(fabs(c));
            lre[k] = a; lim[k] = w;
            if (!left) {
                /* null vector of [[-iw, b], [c, -iw]] */
                if (fabs(b) >= fabs(c)) { o[0] = 1.0; o[1] = 0.0; o[2] = 0.0; o[3] = w / b; }
                else { o[0] = -w / c; o[1] = 0.0; o[2] = 0.0; o[3] = 1.0; }
            } else {
                /* null vector of the transpose [[-iw, c], [b, -iw]] (w^T of
                   the block part), in the row-reversed form of the right
                   convention: (iw/b, 1) if |b| >= |c|, else (i, -w/c) */
                if (fabs(b) >= fabs(c)) { o[0] = 0.0; o[1] = 1.0; o[2] = w / b; o[3] = 0.0; }
                else { o[0] = 0.0; o[1] = -w / c; o[2] = 1.0; o[3] = 0.0; }
            }
        }
        int sel = select == NULL || select[p] || (blk[k].size == 2 && select[p + 1]);
        if (sel) {
            jobs[njobs].blk = k; jobs[njobs].col = col; njobs++;
            if (lam_re) { lam_re[col] = lre[k]; if (blk[k].size == 2) lam_re[col + 1] = lre[k]; }
            if (lam_im) { lam_im[col] = lim[k]; if (blk[k].size == 2) lam_im[col + 1] = -lim[k]; }
            col += blk[k].size;
        }
    }
    {
        problem_t P = {n, S, lds, NULL, 0, blk, nblk, left ? NULL : tau, NULL,
                       left ? tau : NULL, NULL, 0.0, 0.0};
        st = run_jobs(&P, 0, left, Q, ldq, jobs, njobs, lre, lim, NULL, own, X, ldx, scale_exp,
                      nthreads);
    }
done:
    free(blk); free(tau); free(lre); free(lim); free(own); free(jobs);
    return st;
}

/*
 * Standard problem: right eigenvectors of the quasi-triangular S
 * (column-major, ld lds), optional Q (NULL: X = Y).  Output columns follow
 * the block order; a 2x2 block yields (Re, Im) of the eigenvector of
 * lambda = a + i w with w > 0.  lam_re/lam_im (length m, may be NULL).
 */
int evo_standard(int64_t n, const double *S, int64_t lds, const double *Q, int64_t ldq,
                 const uint8_t *select, double *X, int64_t ldx, int32_t *scale_exp,
                 double *lam_re, double *lam_im, int nthreads, int64_t *bad)
{
    return standard_impl(0, n, S, lds, Q, ldq, select, X, ldx, scale_exp, lam_re, lam_im,
                         nthreads, bad);
}

/*
 * Left eigenvectors of the quasi-triangular S: u_i^H S = lambda_i u_i^H
 * (Sec. 2's eigenvector problem for S^T), optional Q (x_i = Q u_i, the
 * left eigenvectors of Q S Q^T).  Same arguments, column order, eigenvalue
 * outputs and canonical form as evo_standard; a 2x2 block yields (Re u,
 * Im u) for lambda = a + i w, w > 0, and u is zero above its block.
 */
int evo_standard_left(int64_t n, const double *S, int64_t lds, const double *Q, int64_t ldq,
                      const uint8_t *select, double *X, int64_t ldx, int32_t *scale_exp,
                      double *lam_re, double *lam_im, int nthreads, int64_t *bad)
{
    return standard_impl(1, n, S, lds, Q, ldq, select, X, ldx, scale_exp, lam_re, lam_im,
                         nthreads, bad);
}

/*
 * Generalized problem (S, T): S quasi-triangular, T upper triangular; the
 * 2x2 block of T under a 2x2 block of S must be diagonal with positive
 * entries.  Generalized eigenvalue lambda = alpha / beta with beta real >= 0,
 * (alpha, beta) scaled by a common power of two so max(|alpha|, beta) lies
 * in [1, 2) (|alpha| = max(|re|, |im|)).  For a 2x2 block the column pair is
 * (Re, Im) of the eigenvector of the member with Im alpha > 0.  Optional Z.
 */
static int generalized_impl(int left, int64_t n, const double *S, int64_t lds, const double *T,
                            int64_t ldt, const double *Z, int64_t ldz, const uint8_t *select,
                            double *X, int64_t ldx, int32_t *scale_exp,
                            double *alpha_re, double *alpha_im, double *beta_out,
                            int nthreads, int64_t *bad)
{
    if (n < 0 || lds < (n > 0 ? n : 1) || ldt < (n > 0 ? n : 1) || ldx < (n > 0 ? n : 1))
        return EVO_EINVAL;
    if (Z && ldz < (n > 0 ? n : 1)) return EVO_EINVAL;
    if (n == 0) return EVO_OK;
    int st = check_entries(n, S, lds, 1, bad);
    if (st) return st;
    st = check_entries(n, T, ldt, 0, bad);
    if (st) return st;
    block_t *blk = (block_t *)malloc(sizeof(block_t) * n);
    double *tauS = (double *)malloc(sizeof(double) * n);
    double *tauT = (double *)malloc(sizeof(double) * n);
    double *lre = (double *)malloc(sizeof(double) * n);
    double *lim = (double *)malloc(sizeof(double) * n);
    double *lbe = (double *)malloc(sizeof(double) * n);
    double *own = (double *)malloc(sizeof(double) * 4 * n);
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * n);
    int64_t nblk = 0;
    if (!blk || !tauS || !tauT || !lre || !lim || !lbe || !own || !jobs) { st = EVO_ENOMEM; goto done; }
    st = scan_blocks(n, S, lds, 0, blk, &nblk, bad);
    if (st) goto done;

    double smax = 0.0, tmax = 0.0;
    for (int64_t i = 0; i < n; i++) {
        if (fabs(AT(S, lds, i, i)) > smax) smax = fabs(AT(S, lds, i, i));
        if (fabs(AT(T, ldt, i, i)) > tmax) tmax = fabs(AT(T, ldt, i, i));
    }
    int64_t njobs = 0, col = 0;
    for (int64_t k = 0; k < nblk; k++) {
        const int64_t p = blk[k].start;
        const int64_t pe = p + blk[k].size;
        tauS[k] = left ? block_row_norm(S, lds, n, p, blk[k].size, pe)
                       : block_col_norm(S, lds, p, p, blk[k].size);
        tauT[k] = left ? block_row_norm(T, ldt, n, p, blk[k].size, pe)
                       : block_col_norm(T, ldt, p, p, blk[k].size);
        double ar, ai, be;
        double *o = &own[4 * k];
        if (blk[k].size == 1) {
            ar = AT(S, lds, p, p); ai = 0.0; be = AT(T, ldt, p, p);
            if (be < 0.0) { be = -be; ar = -ar; }
            if (ar == 0.0 && be == 0.0) {
                if (bad) *bad = p;
                st = EVO_ENOTSCHUR;
                goto done;
            }
            o[0] = 1.0; o[1] = 0.0; o[2] = 0.0; o[3] = 0.0;
        } else {
            double s11 = AT(S, lds, p, p), s12 = AT(S, lds, p, p + 1);
            double s21 = AT(S, lds, p + 1, p), s22 = AT(S, lds, p + 1, p + 1);
            double d1 = AT(T, ldt, p, p), d2 = AT(T, ldt, p + 1, p + 1);
            if (left) {
                /* the left eigenvalue pair is defined on the reversed
                   transposed block J B^T J (entries (s22, s12; s21, s11)
                   against diag(d2, d1)), the block a forward substitution
                   meets first from its last row */
                double t = s11; s11 = s22; s22 = t;
                t = d1; d1 = d2; d2 = t;
            }
            if (!(d1 > 0.0 && d2 > 0.0) || AT(T, ldt, p, p + 1) != 0.0) {
                if (bad) *bad = p;
                st = EVO_ENOTSCHUR;
                goto done;
            }
            /* det(S_b - lambda diag(d1, d2)) = 0:
               lambda = h +- i sqrt(-g),  h = (s11/d1 + s22/d2) / 2,
               g = ((s11/d1 - s22/d2) / 2)^2 + s12 s21 / (d1 d2) */
            double u = s11 / d1, v = s22 / d2;
            double hh = 0.5 * (u + v), dd = 0.5 * (u - v);
            double g = dd * dd + (s12 / d1) * (s21 / d2);
            if (!(g < 0.0)) {
                if (bad) *bad = p;
                st = EVO_ENOTSCHUR;
                goto done;
            }
            double w = sqrt(-g);
            /* alpha = lambda * d1, beta = d1 */
            ar = hh * d1; ai = w * d1; be = d1;
        }
        /* common power-of-two normalisation: max(|alpha|, beta) in [1, 2) */
        {
            double mx = fabs(ar);
            if (fabs(ai) > mx) mx = fabs(ai);
            if (be > mx) mx = be;
            if (!isfinite(mx) || mx == 0.0) {
                if (bad) *bad = p;
                st = EVO_EINVAL;
                goto done;
            }
            int t = ilogb(mx);
            ar = ldexp(ar, -t); ai = ldexp(ai, -t); be = ldexp(be, -t);
        }
        lre[k] = ar; lim[k] = ai; lbe[k] = be;
        if (blk[k].size == 2) {
            /* null vector of M = beta S_b - alpha T_b (complex alpha); left:
               of the reversed transposed block, stored in reverse below */
            double s11 = AT(S, lds, p, p), s12 = AT(S, lds, p, p + 1);
            double s21 = AT(S, lds, p + 1, p), s22 = AT(S, lds, p + 1, p + 1);
            double d1 = AT(T, ldt, p, p), d2 = AT(T, ldt, p + 1, p + 1);
            if (left) {
                double t = s11; s11 = s22; s22 = t;
                t = d1; d1 = d2; d2 = t;
            }
            double m12 = be * s12, m21 = be * s21;
            if (fabs(m12) >= fabs(m21)) {
                /* row 1: m11 v1 + m12 v2 = 0, v1 = 1, v2 = -m11 / m12 */
                double m11r = be * s11 - ar * d1, m11i = -ai * d1;
                o[0] = 1.0; o[2] = 0.0;
                o[1] = -m11r / m12; o[3] = -m11i / m12;
            } else {
                /* row 2: m21 v1 + m22 v2 = 0, v2 = i, v1 = -m22 i / m21 */
                double m22r = be * s22 - ar * d2, m22i = -ai * d2;
                /* -m22 * i = m22i - i m22r */
                o[0] = m22i / m21; o[2] = -m22r / m21;
                o[1] = 0.0; o[3] = 1.0;
            }
            if (left) {   /* w's block part is the reversed vector */
                double t = o[0]; o[0] = o[1]; o[1] = t;
                t = o[2]; o[2] = o[3]; o[3] = t;
            }
        }
        int sel = select == NULL || select[p] || (blk[k].size == 2 && select[p + 1]);
        if (sel) {
            jobs[njobs].blk = k; jobs[njobs].col = col; njobs++;
            for (int j = 0; j < blk[k].size; j++) {
                if (alpha_re) alpha_re[col + j] = ar;
                if (alpha_im) alpha_im[col + j] = j == 0 ? ai : -ai;
                if (beta_out) beta_out[col + j] = be;
            }
            col += blk[k].size;
        }
    }
    {
        problem_t P = {n, S, lds, T, ldt, blk, nblk, left ? NULL : tauS, left ? NULL : tauT,
                       left ? tauS : NULL, left ? tauT : NULL, smax, tmax};
        st = run_jobs(&P, 1, left, Z, ldz, jobs, njobs, lre, lim, lbe, own, X, ldx, scale_exp,
                      nthreads);
    }
done:
    free(blk); free(tauS); free(tauT); free(lre); free(lim); free(lbe); free(own); free(jobs);
    return st;
}

int evo_generalized(int64_t n, const double *S, int64_t lds, const double *T, int64_t ldt,
                    const double *Z, int64_t ldz, const uint8_t *select,
                    double *X, int64_t ldx, int32_t *scale_exp,
                    double *alpha_re, double *alpha_im, double *beta_out,
                    int nthreads, int64_t *bad)
{
    return generalized_impl(0, n, S, lds, T, ldt, Z, ldz, select, X, ldx, scale_exp, alpha_re,
                            alpha_im, beta_out, nthreads, bad);
}

/*
 * Left eigenvectors of the pencil (S, T): u_i^H (beta_i S - alpha_i T) = 0
 * (the eigenvector problem of Sec. 2 for the transposed pencil), by robust
 * forward substitution over the blocks after block i, optional Z (x_i =
 * Z u_i).  Requirements, column order, canonical form and outputs as
 * evo_generalized; u_i is zero above its block.  For a 2x2 block, (alpha,
 * beta) and the block part of u are those of the reversed transposed block
 * (entries (s22, s12; s21, s11) against diag(d2, d1)): the same eigenvalue
 * alpha / beta, the pair normalised against d2; the column pair is (Re u,
 * Im u) for the member with Im alpha > 0.
 */
int evo_generalized_left(int64_t n, const double *S, int64_t lds, const double *T, int64_t ldt,
                         const double *Z, int64_t ldz, const uint8_t *select,
                         double *X, int64_t ldx, int32_t *scale_exp,
                         double *alpha_re, double *alpha_im, double *beta_out,
                         int nthreads, int64_t *bad)
{
    return generalized_impl(1, n, S, lds, T, ldt, Z, ldz, select, X, ldx, scale_exp, alpha_re,
                            alpha_im, beta_out, nthreads, bad);
}

/* ------------------------------------------------------------------ */
/* Robust triangular solve, many right-hand sides                       */
/* ------------------------------------------------------------------ */

/*
 * T x = b for one column, robustly: the backsubstitution of solve_one with
 * the shift 0 and a general right-hand side instead of an eigenvector's
 * own block.  Every diagonal block is solved (pivots below
 * smlnum = 2^-1022 n / ulp perturbed up to it), and every update is
 * protected.  On return y = x * 2^e.
 */
static void solve_rhs(const problem_t *P, const double *b, double *y, int64_t *e_out)
{
    const int64_t n = P->n;
    const block_t *B = P->blk;
    const double smin = SAFMIN * ((double)n / ULP);
    const double zero2[2] = {0.0, 0.0};
    int64_t e = 0;
    memcpy(y, b, sizeof(double) * n);
    for (int64_t cur = P->nblk - 1; cur >= 0; cur--) {
        const int64_t i0 = B[cur].start;
        const int ib = B[cur].size;
        double mr[4], mi[4] = {0.0, 0.0, 0.0, 0.0}, rr[2], zr[2], zi[2];
        for (int a = 0; a < ib; a++) {
            for (int c = 0; c < ib; c++) mr[a * ib + c] = AT(P->S, P->lds, i0 + a, i0 + c);
            rr[a] = y[i0 + a];
        }
        int64_t s = small_solve(ib, mr, mi, rr, zero2, smin, zr, zi);
        if (s != 0) {
            scale_vec(n, y, s);
            e += s;
        }
        for (int a = 0; a < ib; a++) y[i0 + a] = zr[a];
        if (i0 == 0) break;
        /* protect, then r[0:i0] -= T[0:i0, block] z */
        double nu = 0.0, mu = 0.0;
        for (int64_t r = 0; r < i0; r++)
            if (fabs(y[r]) > nu) nu = fabs(y[r]);
        for (int a = 0; a < ib; a++)
            if (fabs(y[i0 + a]) > mu) mu = fabs(y[i0 + a]);
        s = protect_update(nu, P->tauS[cur], mu);
        if (s != 0) {
            scale_vec(n, y, s);
            e += s;
        }
        for (int a = 0; a < ib; a++) {
            const double z = y[i0 + a];
            const double *Tc = &AT(P->S, P->lds, 0, i0 + a);
            for (int64_t r = 0; r < i0; r++) y[r] -= Tc[r] * z;
        }
    }
    *e_out = e;
}

/*
 * Robust triangular solve: for each column b_j of B (n x nrhs, ld ldb),
 * the solution of T x_j = b_j as X[:, j] * 2^(-scale_exp[j]) with
 * |X[:, j]|_inf in [1, 2) (X[:, j] = 0 and scale_exp[j] = 0 for b_j = 0).
 * T (ld ldt) is upper quasi-triangular: 1x1 and 2x2 diagonal blocks from
 * its first subdiagonal, a 2x2 block in any form.  Entries of T (upper
 * part and first subdiagonal) and of B must be finite and at most 2^1000
 * in magnitude; *bad is i + j n for T and n n + i + j n for B.
 */
int evo_trsolve(int64_t n, const double *S, int64_t lds, int64_t nrhs, const double *Bm,
                int64_t ldb, double *X, int64_t ldx, int32_t *scale_exp, int nthreads,
                int64_t *bad)
{
    if (n < 0 || nrhs < 0 || lds < (n > 0 ? n : 1) || ldb < (n > 0 ? n : 1) ||
        ldx < (n > 0 ? n : 1))
        return EVO_EINVAL;
    if (n == 0 || nrhs == 0) return EVO_OK;
    int st = check_entries(n, S, lds, 1, bad);
    if (st) return st;
    for (int64_t j = 0; j < nrhs; j++)
        for (int64_t i = 0; i < n; i++) {
            double v = AT(Bm, ldb, i, j);
            if (!isfinite(v) || fabs(v) > INPUT_MAX) {
                if (bad) *bad = n * n + i + j * n;
                return isfinite(v) ? EVO_EINVAL : EVO_ENONFINITE;
            }
        }
    block_t *blk = (block_t *)malloc(sizeof(block_t) * n);
    double *tau = (double *)malloc(sizeof(double) * n);
    int64_t nblk = 0;
    if (!blk || !tau) { st = EVO_ENOMEM; goto done; }
    st = scan_blocks(n, S, lds, 0, blk, &nblk, bad);
    if (st) goto done;
    for (int64_t k = 0; k < nblk; k++)
        tau[k] = block_col_norm(S, lds, blk[k].start, blk[k].start, blk[k].size);
    {
        problem_t P = {n, S, lds, NULL, 0, blk, nblk, tau, NULL, NULL, NULL, 0.0, 0.0};
#ifdef _OPENMP
        if (nthreads > 0) omp_set_num_threads(nthreads);
#else
        (void)nthreads;
#endif
#pragma omp parallel
        {
            double *y = (double *)malloc(sizeof(double) * n);
            if (!y) {
#pragma omp atomic write
                st = EVO_ENOMEM;
            }
#pragma omp for schedule(dynamic, 1)
            for (int64_t j = 0; j < nrhs; j++) {
                if (!y) continue;
                int64_t e = 0;
                solve_rhs(&P, &AT(Bm, ldb, 0, j), y, &e);
                e -= canonicalize(n, y, NULL, 0);
                if (e > INT32_MAX || e < INT32_MIN) {
#pragma omp atomic write
                    st = EVO_EINVAL;
                    continue;
                }
                memcpy(&AT(X, ldx, 0, j), y, sizeof(double) * n);
                scale_exp[j] = (int32_t)e;
            }
            free(y);
        }
    }
done:
    free(blk); free(tau);
    return st;
}

/*
 * Overflow witness (test-only): the textbook unscaled substitution for the
 * standard problem, no scaling and no perturbation.  Writes the unnormalised
 * vectors to X and returns the number of columns that contain Inf or NaN.
 */
int64_t evo_naive_standard(int64_t n, const double *S, int64_t lds, const uint8_t *select,
                           double *X, int64_t ldx)
{
    block_t *blk = (block_t *)malloc(sizeof(block_t) * (n > 0 ? n : 1));
    double *yi = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    int64_t nblk = 0, col = 0, nonfinite = 0;
    if (!blk || !yi || scan_blocks(n, S, lds, 1, blk, &nblk, NULL) != EVO_OK) {
        free(blk); free(yi); return -1;
    }
    for (int64_t k = 0; k < nblk; k++) {
        const int64_t p = blk[k].start;
        int sel = select == NULL || select[p] || (blk[k].size == 2 && select[p + 1]);
        if (!sel) continue;
        double *yr = &AT(X, ldx, 0, col);
        double ar = AT(S, lds, p, p), ai = 0.0;
        memset(yr, 0, sizeof(double) * n);
        memset(yi, 0, sizeof(double) * n);
        if (blk[k].size == 1) {
            yr[p] = 1.0;
        } else {
            double b = AT(S, lds, p, p + 1), c = AT(S, lds, p + 1, p);
            ai = sqrt(fabs(b)) * sqrt(fabs(c));
            if (fabs(b) >= fabs(c)) { yr[p] = 1.0; yi[p + 1] = ai / b; }
            else { yr[p] = -ai / c; yi[p + 1] = 1.0; }
        }
        /* plain block backsubstitution: row block q solves
           (S_qq - lambda I) y_q = -sum_{j > q} S_qj y_j */
        for (int64_t kk = k - 1; kk >= 0; kk--) {
            const int64_t q = blk[kk].start;
            const int qb = blk[kk].size;
            double rr[2] = {0, 0}, ri[2] = {0, 0};
            for (int a = 0; a < qb; a++) {
                for (int64_t j = q + qb; j < p + blk[k].size; j++) {
                    rr[a] -= AT(S, lds, q + a, j) * yr[j];
                    ri[a] -= AT(S, lds, q + a, j) * yi[j];
                }
            }
            if (qb == 1) {
                double dr = AT(S, lds, q, q) - ar, di = -ai;
                cdiv(rr[0], ri[0], dr, di, &yr[q], &yi[q]);
            } else {
                /* Cramer's rule on the complex 2x2 system */
                double m11r = AT(S, lds, q, q) - ar, m11i = -ai;
                double m22r = AT(S, lds, q + 1, q + 1) - ar, m22i = -ai;
                double m12 = AT(S, lds, q, q + 1), m21 = AT(S, lds, q + 1, q);
                double detr = m11r * m22r - m11i * m22i - m12 * m21;
                double deti = m11r * m22i + m11i * m22r;
                double n1r = rr[0] * m22r - ri[0] * m22i - m12 * rr[1];
                double n1i = rr[0] * m22i + ri[0] * m22r - m12 * ri[1];
                double n2r = m11r * rr[1] - m11i * ri[1] - m21 * rr[0];
                double n2i = m11r * ri[1] + m11i * rr[1] - m21 * ri[0];
                cdiv(n1r, n1i, detr, deti, &yr[q], &yi[q]);
                cdiv(n2r, n2i, detr, deti, &yr[q + 1], &yi[q + 1]);
            }
        }
        int bad = 0;
        for (int64_t r = 0; r < n; r++)
            if (!isfinite(yr[r]) || !isfinite(yi[r])) { bad = 1; break; }
        nonfinite += bad;
        if (blk[k].size == 2) memcpy(&AT(X, ldx, 0, col + 1), yi, sizeof(double) * n);
        col += blk[k].size;
    }
    free(blk); free(yi);
    return nonfinite;
}

/* ------------------------------------------------------------------ */
/* Hessenberg reduction                                                 */
/* ------------------------------------------------------------------ */

/* |x|_2 of a vector, scaled by its largest magnitude so that no square
 * overflows or underflows to zero before the sum. */
static double scaled_norm2(int64_t len, const double *x, int64_t inc)
{
    double mx = 0.0;
    for (int64_t i = 0; i < len; i++)
        if (fabs(x[i * inc]) > mx) mx = fabs(x[i * inc]);
    if (mx == 0.0) return 0.0;
    double ss = 0.0;
    for (int64_t i = 0; i < len; i++) {
        double t = x[i * inc] / mx;
        ss += t * t;
    }
    return mx * sqrt(ss);
}

/*
 * Hessenberg reduction (Sec. 3.1: A = Q H Q^T with H upper Hessenberg and Q
 * orthogonal, the first phase of the eigenvalue pipeline), the unblocked
 * definition: for j = 0 .. n - 3 one Householder reflector
 * P_j = I - tau_j w_j w_j^T annihilates A[j+2:n, j]; A <- P_j A P_j, and
 * Q <- Q P_j (Q starts as the identity).  With alpha = A[j+1, j] and
 * x = A[j+2:n, j]: if x = 0 then tau_j = 0 (P_j = I); otherwise
 *   beta = -sign(alpha) |(alpha, x)|_2  (sign(0) = +1),
 *   tau_j = (beta - alpha) / beta,  w_j = (0 .. 0, 1, x / (alpha - beta)),
 * the 1 at row j + 1, so that P_j (alpha, x) = (beta, 0).  On return A
 * holds H (exact zeros below the first subdiagonal), Q (if not NULL, ld
 * ldq) the orthogonal factor and tau (if not NULL, length n) tau_j (0 for
 * j >= n - 2).  Entries must be finite and at most 2^1000 in magnitude
 * (*bad = i + j n).
 */
int evo_hessenberg(int64_t n, double *A, int64_t lda, double *Q, int64_t ldq, double *tau,
                   int64_t *bad)
{
    if (n < 0 || lda < (n > 0 ? n : 1) || (Q && ldq < (n > 0 ? n : 1))) return EVO_EINVAL;
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < n; i++) {
            double v = AT(A, lda, i, j);
            if (!isfinite(v)) { if (bad) *bad = i + j * n; return EVO_ENONFINITE; }
            if (fabs(v) > INPUT_MAX) { if (bad) *bad = i + j * n; return EVO_EINVAL; }
        }
    if (Q)
        for (int64_t j = 0; j < n; j++)
            for (int64_t i = 0; i < n; i++) AT(Q, ldq, i, j) = i == j ? 1.0 : 0.0;
    if (tau)
        for (int64_t j = 0; j < n; j++) tau[j] = 0.0;
    double *w = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    if (!w) return EVO_ENOMEM;
    for (int64_t j = 0; j + 2 < n; j++) {
        const double alpha = AT(A, lda, j + 1, j);
        const double xn = scaled_norm2(n - j - 2, &AT(A, lda, j + 2, j), 1);
        if (xn == 0.0) continue;                       /* P_j = I */
        double beta = scaled_norm2(2, (double[]){alpha, xn}, 1);
        if (alpha >= 0.0) beta = -beta;
        const double t = (beta - alpha) / beta;
        const double d = alpha - beta;
        for (int64_t i = 0; i < n; i++) w[i] = 0.0;
        w[j + 1] = 1.0;
        for (int64_t i = j + 2; i < n; i++) w[i] = AT(A, lda, i, j) / d;
        /* column j: (beta, 0, ..., 0) below the diagonal */
        AT(A, lda, j + 1, j) = beta;
        for (int64_t i = j + 2; i < n; i++) AT(A, lda, i, j) = 0.0;
        /* A <- P A on columns j+1 .. n-1 (rows j+1 .. n-1) */
        for (int64_t c = j + 1; c < n; c++) {
            double s = 0.0;
            for (int64_t i = j + 1; i < n; i++) s += w[i] * AT(A, lda, i, c);
            s *= t;
            for (int64_t i = j + 1; i < n; i++) AT(A, lda, i, c) -= s * w[i];
        }
        /* A <- A P on all rows (columns j+1 .. n-1) */
        for (int64_t r = 0; r < n; r++) {
            double s = 0.0;
            for (int64_t c = j + 1; c < n; c++) s += AT(A, lda, r, c) * w[c];
            s *= t;
            for (int64_t c = j + 1; c < n; c++) AT(A, lda, r, c) -= s * w[c];
        }
        /* Q <- Q P */
        if (Q)
            for (int64_t r = 0; r < n; r++) {
                double s = 0.0;
                for (int64_t c = j + 1; c < n; c++) s += AT(Q, ldq, r, c) * w[c];
                s *= t;
                for (int64_t c = j + 1; c < n; c++) AT(Q, ldq, r, c) -= s * w[c];
            }
        if (tau) tau[j] = t;
    }
    free(w);
    return EVO_OK;
}


/*
 * Eigenvalue reordering's off-diagonal updates (Sec. 3.2: a window task
 * gathers its local transformations in an accumulator matrix; the left and
 * right update tasks then apply it to the off-diagonal sections).  Windows
 * are applied in the order given; window w covers rows and columns
 * [a, a + k) with a = begin[w], k = size[w], and its accumulator Z is the
 * k x k column-major matrix at Z + zoff[w].  With Zhat = diag(I_a, Z, I):
 *   T <- Zhat^T T Zhat, touching only rows [a, a + k) from column a on (the
 *   rows' entries left of the window are the zeros below the diagonal) and
 *   columns [a, a + k) down to row a + k - 1 (the rows below are zero);
 *   Q <- Q Zhat (all n rows of the window's columns).
 * Plain definition: each updated entry is one dot product of length k.
 */
int evo_window_update(int64_t n, double *T, int64_t ldt, double *Q, int64_t ldq, int nwin,
                      const int64_t *begin, const int32_t *size, const double *Z,
                      const int64_t *zoff) {
    if (n < 0 || ldt < (n > 0 ? n : 1) || (Q && ldq < (n > 0 ? n : 1)) || nwin < 0)
        return EVO_EINVAL;
    for (int w = 0; w < nwin; w++)
        if (begin[w] < 0 || size[w] < 0 || begin[w] + size[w] > n || zoff[w] < 0)
            return EVO_EINVAL;
    double *t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!t) return EVO_ENOMEM;
    for (int w = 0; w < nwin; w++) {
        const int64_t a = begin[w], k = size[w], b = a + k;
        const double *Zw = Z + zoff[w];
        /* left: T[a:b, j] <- Z^T T[a:b, j] for j = a .. n-1 */
        for (int64_t j = a; j < n; j++) {
            for (int64_t i = 0; i < k; i++) {
                double s = 0.0;
                for (int64_t l = 0; l < k; l++) s += AT(Zw, k, l, i) * AT(T, ldt, a + l, j);
                t[i] = s;
            }
            for (int64_t i = 0; i < k; i++) AT(T, ldt, a + i, j) = t[i];
        }
        /* right: T[r, a:b] <- T[r, a:b] Z for r = 0 .. b-1 */
        for (int64_t r = 0; r < b; r++) {
            for (int64_t i = 0; i < k; i++) {
                double s = 0.0;
                for (int64_t l = 0; l < k; l++) s += AT(T, ldt, r, a + l) * AT(Zw, k, l, i);
                t[i] = s;
            }
            for (int64_t i = 0; i < k; i++) AT(T, ldt, r, a + i) = t[i];
        }
        /* Q[r, a:b] <- Q[r, a:b] Z for every row */
        if (Q)
            for (int64_t r = 0; r < n; r++) {
                for (int64_t i = 0; i < k; i++) {
                    double s = 0.0;
                    for (int64_t l = 0; l < k; l++) s += AT(Q, ldq, r, a + l) * AT(Zw, k, l, i);
                    t[i] = s;
                }
                for (int64_t i = 0; i < k; i++) AT(Q, ldq, r, a + i) = t[i];
            }
    }
    free(t);
    return EVO_OK;
}
