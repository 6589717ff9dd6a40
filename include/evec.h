/*
 * evec.h -- robust eigenvectors of real Schur forms on one GPU.
 *
 * The operation (Sec. 2, Eq. evec_solve and Eq. evec_backtransform of
 * "Task-based, GPU-accelerated and Robust Library for Solving Dense
 * Nonsymmetric Eigenvalue Problems"): given a real upper quasi-triangular
 * Schur form T (1x1 diagonal blocks for real eigenvalues, 2x2 blocks for
 * complex-conjugate pairs) and optionally its orthogonal factor Q, solve
 * (T - lambda_i I) y_i = 0 by backsubstitution for every selected eigenvalue
 * and return x_i = Q y_i.  The solve is robust (Sec. 3.3, "Robust computation of eigenvectors"): no intermediate
 * or final value overflows, because every tile segment of every column
 * carries an integer power-of-two scale factor (the augmented tile
 * <alpha, X> represents y_j = x_j / alpha_j) and every tile update
 * Y <- Y - T X is preceded by a scaling that bounds its result.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Matrices are FP64, column-major, with a leading dimension (ld >= n).
 *   Matrix arguments are DEVICE pointers unless the name ends in _host.
 *   Entries of T below the first subdiagonal are never read.
 * - A 2x2 diagonal block must be standardized: equal diagonal entries a and
 *   off-diagonal entries b, c of opposite sign; its eigenvalues are
 *   a +- i w, w = sqrt(|b|) sqrt(|c|).  Two consecutive nonzero
 *   subdiagonal entries, or a non-standardized 2x2 block, is EVEC_ENOTSCHUR.
 * - Every referenced entry must be finite (else EVEC_ENONFINITE) and of
 *   magnitude <= 2^1000 (else EVEC_EINVAL).  2^1020 is the overflow
 *   threshold of every intermediate bound.
 * - select_host: HOST array of n bytes; eigenvalue i is selected when
 *   select_host[i] != 0.  A 2x2 block is selected when either of its two
 *   eigenvalues is.  NULL selects all eigenvalues.
 * - Output columns follow the order of the diagonal blocks.  A real
 *   eigenvalue gives one column; a selected 2x2 block gives two columns
 *   (Re, Im) of the eigenvector for lambda = a + i w with w > 0 (the
 *   conjugate eigenvalue has the conjugate vector).  m, the number of
 *   output columns, is returned by evec_count.
 * - Scaling: on return the true eigenvector is  X[:, j] * 2^(-scale_exp[j])
 *   and X is canonical: max_i |X[i, j]| lies in [1, 2) (for a pair,
 *   max_i |X[i, p]| + |X[i, p+1]| lies in [1, 2) and both columns share one
 *   exponent).  scale_exp is int32 (the paper's 32-bit scale exponents).
 *   Entries far below the column maximum may underflow to subnormal or zero
 *   when the final consolidation (Sec. 3.3, post-processing) brings every
 *   segment of a column to one common exponent.
 * - The block part of each eigenvector is fixed: y_p = 1 for a 1x1 block at
 *   p; for a pair, (y_p, y_p+1) = (1, i w / b) when |b| >= |c|, otherwise
 *   (-w / c, i).  Rows below the block are zero before back-transformation.
 * - Calls are asynchronous on the handle's stream.  Argument errors
 *   (EVEC_EINVAL, EVEC_ENOTSCHUR found while planning) are returned
 *   synchronously and nothing is launched.  Errors found on the device
 *   (EVEC_ENONFINITE, EVEC_EINVAL for an entry above 2^1000) are reported
 *   by evec_sync, which also returns the offending index.  There is no CPU
 *   fallback: without a usable CUDA device every call returns EVEC_ECUDA.
 * - Ownership: the caller owns every matrix and output buffer.  The handle
 *   owns its workspace (working copy of Y when Q is given, per-segment
 *   exponents and norms, the plan), grows it on demand and frees it in
 *   evec_destroy.  One handle must not be used by two host threads at once.
 */
#ifndef EVEC_H
#define EVEC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct evec_ctx *evec_handle;

typedef enum {
    EVEC_OK = 0,
    EVEC_EINVAL = 1,     /* bad argument, or an entry above 2^1000 */
    EVEC_ENOTSCHUR = 2,  /* not a (standardized) quasi-triangular Schur form */
    EVEC_ENONFINITE = 3, /* NaN or Inf in a referenced entry */
    EVEC_ENOMEM = 4,     /* device or host allocation failed */
    EVEC_ECUDA = 5,      /* CUDA runtime error */
    EVEC_ETIMEOUT = 6,   /* a bounded device-side wait gave up (reported by evec_sync) */
    EVEC_ERESIDUAL = 7,  /* refine = 2: an eigenvalue failed the residual
                            gate in every repeat, FP64 included (evec_sync) */
    EVEC_ECAPACITY = 8,  /* problem larger than evec_standard_noalloc's fixed scratch */
    EVEC_EBOUNDS = 9     /* checked build only: a device access outside the range
                            the plan allows was skipped; index = the site */
} evec_status;

typedef enum {
    EVEC_FP64 = 0,  /* every operation in FP64 on the GPU (DFMA) */
    EVEC_SPLIT = 1  /* dense contractions as split-precision products on the
                       BF16 tensor cores (FP64 operands cut into `slices`
                       7-bit digit slices, exact FP32 accumulation per digit
                       diagonal, FP64 recombination); everything else FP64 */
} evec_mode;

typedef struct {
    int mode;    /* evec_mode */
    int tile;    /* tile size nb of the tiled solve, 16..512; 0 = 64, or
                    256 in EVEC_SPLIT mode for n >= 8192 (the faster
                    choice measured on B300).  Tiles above 64 rows are
                    solved in sub-blocks of at most 64 rows with one scale
                    exponent per tile segment */
    int slices;  /* EVEC_SPLIT: digit slices per operand, 2..8; 0 = 8
                    (relative error of a product ~2^(-7 slices)) */
    int refine;  /* EVEC_SPLIT, evec_standard and evec_standard_left:
                    1 (the default of evec_opts_default and of opt ==
                    NULL) = one residual-correction sweep after the solve:
                    the residual r = -(T - lambda I) y in FP64 on the rows
                    above each column's block, formed on the solver's scaled
                    segments (each tile row in its own power-of-two scale),
                    the correction (T - lambda I) d = r solved by the same
                    robust tiled solver, y <- y + d exactly (power-of-two
                    scaling, one FP64 addition per entry).  A column whose
                    correction exceeds 2^(20 - 7 slices) of it keeps its
                    unrefined value: there the residual's own FP64
                    rounding, amplified by an ill-conditioned column,
                    outweighs the split error.  Costs one FP64 product of
                    about n^3 / 3 flops for all columns, and an extra
                    n x m FP64 workspace.  0 = no sweep.  2 = the sweep,
                    then the residual gate of the refined vectors:
                    ||(T - lambda I) y||_1 <= 10 n ||T||_1 ||y||_1 u
                    (u = 2^-53) per eigenvalue, from a second FP64
                    residual; if any eigenvalue fails, the matrix is solved
                    again with 8 slices (and the gate), then in EVEC_FP64
                    mode, whose result is gated too: an eigenvalue that
                    still fails makes evec_sync return EVEC_ERESIDUAL with
                    the output column of the first one as its index
                    (evec_gate_stats reports what happened).  Ignored in
                    EVEC_FP64 mode and for pencils. */
    int check;   /* nonzero: synchronise at the end of the call and return
                    the device status directly */
} evec_opts;

/* The defaults that opt == NULL stands for: EVEC_FP64, tile 0 (64 rows in
 * FP64 mode), slices 0 (8), refine 1, check 0. */
void evec_opts_default(evec_opts *opt);

/* Create a handle on CUDA device `device` that launches on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).
 * Errors: EVEC_EINVAL (h NULL or bad device), EVEC_ECUDA, EVEC_ENOMEM. */
evec_status evec_create(evec_handle *h, int device, void *cuda_stream);

/* Release the handle and its workspace (after synchronising its stream). */
evec_status evec_destroy(evec_handle h);

/* Change the stream later calls launch on. */
evec_status evec_set_stream(evec_handle h, void *cuda_stream);

/* Number of output columns m of a selection (2 per selected pair).  Reads
 * the diagonal and the first sub- and super-diagonal of the device matrix T
 * (synchronises the handle's stream).
 * Errors: EVEC_EINVAL, EVEC_ENOTSCHUR, EVEC_ECUDA. */
evec_status evec_count(evec_handle h, int64_t n, const double *T, int64_t ldt,
                       const uint8_t *select_host, int64_t *m);

/*
 * Right eigenvectors of the quasi-triangular T (Eq. evec_solve), optionally
 * back-transformed by the orthogonal Q (Eq. evec_backtransform; Q == NULL
 * returns Y itself).  Device arrays:
 *   T [ldt x n], Q [ldq x n] or NULL, X [ldx x m] output,
 *   scale_exp [m] int32 output, lam_re / lam_im [m] FP64 outputs or NULL
 *   (lam_im[j] = w, lam_im[j+1] = -w for a pair).
 * X must not overlap T or Q.  opt may be NULL (defaults).
 * Errors (synchronous): EVEC_EINVAL, EVEC_ENOTSCHUR, EVEC_ENOMEM,
 * EVEC_ECUDA; (at evec_sync) EVEC_ENONFINITE, EVEC_EINVAL.
 */
evec_status evec_standard(evec_handle h, int64_t n, const double *T, int64_t ldt,
                          const double *Q, int64_t ldq, const uint8_t *select_host,
                          double *X, int64_t ldx, int32_t *scale_exp,
                          double *lam_re, double *lam_im, const evec_opts *opt);

/*
 * Left eigenvectors of the quasi-triangular T: u_j^H T = lambda_j u_j^H (the
 * eigenvector problem of Sec. 2 for T^T), optionally back-transformed by
 * Q (x_j = Q u_j, the left eigenvectors of Q T Q^T).  Same arguments,
 * selection, column order (T's block order), eigenvalue outputs, canonical
 * form and errors as evec_standard (mode, tile, slices, refine and check
 * as there).  u_j is zero above its block; for a 1x1 block u_p = 1, for a
 * pair [[a, b], [c, a]] the columns are (Re u, Im u) for lambda = a + i w,
 * w > 0, with the block part (-i w/b, 1) if |b| >= |c|, else (-i, -w/c).
 * Computed as the right eigenvectors of the flipped form T' = J T^T J (J
 * the reversal permutation; T' has T's blocks in reverse order) with
 * Q J for the back-transformation, so the handle holds two extra n x n
 * and one n x m FP64 workspaces.  A non-finite or over-range entry of T
 * strictly above the first superdiagonal is reported at evec_sync with
 * its index i + j ldt in T.
 */
evec_status evec_standard_left(evec_handle h, int64_t n, const double *T, int64_t ldt,
                               const double *Q, int64_t ldq, const uint8_t *select_host,
                               double *X, int64_t ldx, int32_t *scale_exp,
                               double *lam_re, double *lam_im, const evec_opts *opt);

/*
 * Hessenberg reduction A = Q H Q^T (Sec. 3.1, the first phase of the
 * eigenvalue pipeline), blocked by panels of 32 columns: each panel is
 * reduced column by column with Householder reflectors P_j = I - tau_j w_j
 * w_j^T (beta = -sign(alpha) |(alpha, x)|_2, alpha = A[j+1, j], x =
 * A[j+2:n, j], norms scaled by their largest entry; tau_j = 0 when x = 0),
 * accumulated in the compact WY form I - V T V^T with Y = A V T, whose
 * columns need the matrix-vector product of the trailing matrix with w_j;
 * then the trailing matrix gets (I - V T V^T)^T (A - Y V^T) and the rows
 * above the panel A - Y V^T.  All FP64 on the device, or with opt->mode
 * EVEC_SPLIT (opt->slices digit slices, 2..8; 0 = 8; n <= 65472) the five
 * large products of each panel's update (Q V, A^T V and the three rank-32
 * updates) through the split-precision GEMM: BF16 digit slices with row /
 * column power-of-two scales on the tensor cores, FP64 results; the panel
 * reductions stay FP64.  The split updates need slice buffers of about
 * 4 slices n^2 BF16 values (with Q; half without).
 *   A [lda x n] (device): overwritten with H, exact zeros below the first
 *     subdiagonal.  Entries must be finite and at most 2^1000 (else
 *     EVEC_ENONFINITE / EVEC_EINVAL at evec_sync, index i + j lda).
 *   Q [ldq x n] (device) or NULL: receives the orthogonal factor.
 *   opt: mode, slices and check are read.
 * The handle keeps a workspace of about 5 * 32 n + n doubles.
 */
evec_status evec_hessenberg(evec_handle h, int64_t n, double *A, int64_t lda, double *Q,
                            int64_t ldq, const evec_opts *opt);

/*
 * Off-diagonal updates of eigenvalue reordering (Sec. 3.2: a window task
 * accumulates the local transformations of a diagonal window into an
 * orthogonal k x k matrix Z; the left and right update tasks apply it to
 * the off-diagonal sections as level-3 products).  Windows are applied in
 * the order given.  Window w covers rows and columns [a, a + k), with
 * a = begin_host[w] and k = size_host[w].  Its accumulator is the k x k
 * column-major matrix at Z + zoff_host[w].  With Zhat = diag(I_a, Z, I):
 *   T[a:a+k, a:n] <- Z^T T[a:a+k, a:n]   (left update; the window's rows
 *                                         left of it are not read)
 *   T[0:a+k, a:a+k] <- T[0:a+k, a:a+k] Z (right update; the rows below it
 *                                         are not read)
 *   Q[:, a:a+k] <- Q[:, a:a+k] Z          (when Q is non-NULL)
 * This is T <- Zhat^T T Zhat, Q <- Q Zhat whenever the window's rows left
 * of it and its columns below it hold zeros.  That holds for a quasi-
 * triangular T whose windows do not split a 2x2 block, with
 * accumulators that keep each window's diagonal block quasi-triangular, as
 * a window task's do.  Otherwise the update is still the one stated above.
 *   T [ldt x n], Q [ldq x n], Z: device pointers on the handle's device;
 *     Z holds sum_w size_host[w]^2 doubles at the given offsets.
 *   begin_host, size_host, zoff_host [nwin]: host arrays.
 *   opt->mode: EVEC_FP64 (default): FP64 products, the Q updates on a
 *     second stream of the handle beside the T updates.  EVEC_SPLIT: the
 *     three products of each window through the split-precision GEMM of
 *     the back-transformation (opt->slices BF16 digit slices of 7 bits per
 *     operand, row and column power-of-two scales, FP64 results: each
 *     entry within about k 2^-(7 slices) max|row of the left operand|
 *     max|column of the right operand| of the exact product), one window
 *     after another on the handle's stream, for n <= 65472; the handle
 *     keeps the slice buffers (about 2 slices n pad(k) BF16 values).
 *   opt->check: synchronise and return the device status.
 * Errors: EVEC_EINVAL (n < 0, a bad leading dimension, a window outside
 * [0, n), a size above 256, a negative offset, a bad mode or slice count,
 * n > 65472 in EVEC_SPLIT mode).  Entries are not checked.
 */
evec_status evec_window_update(evec_handle h, int64_t n, double *T, int64_t ldt, double *Q,
                               int64_t ldq, int nwin, const int64_t *begin_host,
                               const int32_t *size_host, const double *Z,
                               const int64_t *zoff_host, const evec_opts *opt);

/*
 * The same updates for a set of pairwise disjoint windows, applied
 * concurrently (the paper's concurrent windows of different chains):
 * disjoint windows' updates commute, since (Z'^T X) Z = Z'^T (X Z) on the
 * block two windows share, so all left updates of T run in one launch,
 * then all right updates, with all Q updates beside them.  The result
 * equals evec_window_update on the same windows in any order, up to
 * rounding.  Arguments and errors as evec_window_update; also EVEC_EINVAL
 * when two windows of nonzero size overlap.  In EVEC_SPLIT mode the
 * windows are applied one after another in the order of their first rows.
 */
evec_status evec_window_update_set(evec_handle h, int64_t n, double *T, int64_t ldt, double *Q,
                                   int64_t ldq, int nwin, const int64_t *begin_host,
                                   const int32_t *size_host, const double *Z,
                                   const int64_t *zoff_host, const evec_opts *opt);

/* Polls (about 64 ns each) that a CTA of evec_hessenberg's cooperative
 * panel waits at a grid barrier before it gives up (0 = the built-in
 * limit, 2^22 polls).  A wait that gives up makes the kernel's CTAs return
 * and evec_sync report EVEC_ETIMEOUT; the matrix is then left partly
 * reduced.  The handle stays usable.  A small limit makes the waits run
 * out (a test of the failure path).  Errors: EVEC_EINVAL (polls < 0). */
evec_status evec_set_wait_limit(evec_handle h, int64_t polls);

/* How evec_hessenberg reduces a panel: 1 (default) one cooperative launch
 * per panel (every CTA co-resident, bounded grid barriers between the
 * column phases; falls back to 0 when the device refuses the launch), 0
 * six launches per column.  Same reflectors either way; the sums of the
 * partial reductions group differently (results agree to rounding). */
evec_status evec_set_hessenberg_panel(evec_handle h, int cooperative);

/*
 * The same computation with HOST buffers (column-major, ld = n): copies
 * T (and Q) to the device, computes, copies X [n x m], scale_exp [m],
 * lam_re [m] and lam_im [m] back (each output may be NULL) and
 * synchronises.  Page-locked host memory gives the fastest copies.  Device
 * errors are returned directly.
 */
evec_status evec_standard_host(evec_handle h, int64_t n, const double *T_host,
                               const double *Q_host, const uint8_t *select_host,
                               double *X_host, int32_t *scale_exp_host,
                               double *lam_re_host, double *lam_im_host,
                               const evec_opts *opt);

/* Host-only planning query (no GPU needed).  From the diagonal, the first
 * subdiagonal and the first superdiagonal of T (host arrays of n, n-1 and
 * n-1 values) compute the number of output columns m of a selection and
 * the tile boundaries used for tile size nb (16..512): tiles of nb rows,
 * one row shorter where a boundary would split a 2x2 block.  tile_start
 * (may be NULL) receives ntiles + 1 entries and must hold n / (nb - 1) + 2.
 * Errors: EVEC_EINVAL (bad argument or an entry above 2^1000),
 * EVEC_ENOTSCHUR, EVEC_ENONFINITE (*bad_index: linear index with ld = n). */
evec_status evec_plan_query(int64_t n, const double *diag, const double *sub,
                            const double *sup, const uint8_t *select_host, int nb,
                            int64_t *m, int32_t *ntiles, int32_t *tile_start,
                            int64_t *bad_index);

/* Wait for the handle's stream; return the first device-detected error of
 * the calls since the previous evec_sync (and its linear index i + j*ld into
 * the offending matrix when bad_index is non-NULL), then clear it. */
evec_status evec_sync(evec_handle h, int64_t *bad_index);

/* Kernel classes reported by evec_profile_read (array index). */
enum {
    EVEC_K_GATHER = 0,       /* diagonal gather for the plan */
    EVEC_K_NORMS = 1,        /* tile norms + input validation */
    EVEC_K_DIAG_SOLVE = 2,   /* robust diagonal-tile solves + decisions */
    EVEC_K_TILE_UPDATE = 3,  /* off-diagonal tile updates (FP64, or split:
                                slicing + tensor-core products) */
    EVEC_K_FINALIZE = 4,     /* consolidation + canonical form */
    EVEC_K_BACKTRANSFORM = 5,/* X = Q Y (FP64, or split: slicing + products) */
    EVEC_K_CANONICALIZE = 6, /* canonical form after Q */
    EVEC_K_BATCHED = 7,      /* the persistent kernel of evec_batched */
    EVEC_K_REFINE = 8,       /* residual, right-hand side, correction add
                                (the correction solve itself counts under
                                EVEC_K_DIAG_SOLVE / EVEC_K_TILE_UPDATE) */
    EVEC_K_LEFT = 9,         /* evec_standard_left: the flipped T' and Q J,
                                and the final scatter into T's column order */
    EVEC_K_HESS_PANEL = 10,  /* evec_hessenberg: panel reductions, with the
                                trailing matrix-vector products */
    EVEC_K_HESS_UPDATE = 11, /* evec_hessenberg: trailing / top updates, Q */
    EVEC_K_WINDOW = 12,      /* evec_window_update: left and right updates */
    EVEC_K_COUNT = 13
};

/* The residual gate of the last evec_standard call with refine = 2:
 * eigenvalues that failed it in the first solve, and the number of
 * repeated solves (more slices, then FP64). */
evec_status evec_gate_stats(evec_handle h, int64_t *failed_units, int *retries);

/* The bound of the residual gate (refine = 2) is factor * n (default 10,
 * the bound ||(T - lambda I) y||_1 <= 10 n ||T||_1 ||y||_1 u).  A smaller
 * factor asks for a tighter residual.  Errors: EVEC_EINVAL (factor not
 * positive and finite). */
evec_status evec_set_gate_factor(evec_handle h, double factor);

/* Look-ahead schedule of the split-mode solve (default off): the diagonal
 * solve of step s leaves its protection decisions to a separate launch, and
 * the update of step s is cut at the 128-row block holding tile s - 1: that
 * head runs before the next diagonal solve, the rest on a second stream of
 * the handle beside it, on the SMs the solve leaves free.  The results are
 * bit-identical either way (same arithmetic per element).  On B300 at
 * n = 4096 it is slower (the next diagonal solve needs most SMs, so the
 * rest of the update runs on few), hence off by default. */
evec_status evec_set_lookahead(evec_handle h, int enable);

/* Enable (1) or disable (0) per-kernel timing: while enabled, every kernel
 * launch of the handle is bracketed by CUDA events on the handle's stream. */
evec_status evec_profile(evec_handle h, int enable);

/* Synchronise the handle's stream and return, per kernel class, the summed
 * event-timed milliseconds and the number of kernel launches since the
 * previous read (arrays of nk entries, nk <= EVEC_K_COUNT; either may be
 * NULL); then reset the counters.  Kernels launched back to back for one
 * operation (a slicing kernel and its product) share one timed interval. */
evec_status evec_profile_read(evec_handle h, double *ms, int64_t *launches, int nk);

/*
 * Generalized right eigenvectors of the pencil (S, T) (Sec. 2: (S - lambda T)
 * y = 0, solved as (beta S - alpha T) y = 0): S upper quasi-triangular (1x1 /
 * 2x2 diagonal blocks, not necessarily standardized), T upper triangular
 * with a diagonal positive 2x2 block under each 2x2 block of S (else
 * EVEC_ENOTSCHUR); T's strictly lower part is not read.  Optional Z (NULL:
 * X = Y) for X = Z Y.  Per eigenvalue: 1x1 block (alpha, beta) = (S_pp,
 * T_pp) with beta >= 0; 2x2 block lambda = h +- i sqrt(-g) of det(S_b -
 * lambda T_b) = 0, alpha = lambda d1, beta = d1; both scaled by one power of
 * two so that max(|alpha|, beta) is in [1, 2).  Outputs and canonical form
 * as evec_standard; alpha_re, alpha_im, beta (length m, device, may be NULL)
 * per column (a pair: alpha_im = +w, -w).  Every bound is
 * |beta| |S_rs| + |alpha|_1 |T_rs|.  opt->tile: 16..512 (0 = 64; above 64 in
 * sub-blocks of at most 64 rows, as evec_standard); opt->mode
 * EVEC_SPLIT runs the back-transformation X = Z Y in split precision.
 */
evec_status evec_generalized(evec_handle h, int64_t n, const double *S, int64_t lds,
                             const double *T, int64_t ldt, const double *Z, int64_t ldz,
                             const uint8_t *select_host, double *X, int64_t ldx,
                             int32_t *scale_exp, double *alpha_re, double *alpha_im,
                             double *beta, const evec_opts *opt);

/*
 * Generalized left eigenvectors of the pencil (S, T): u_j^H (beta_j S -
 * alpha_j T) = 0 (the eigenvector problem of Sec. 2 for the transposed
 * pencil), optionally back-transformed by Z (NULL: X = U; else x_j = Z u_j).
 * Same requirements on (S, T), arguments, selection, column order (S's
 * block order), canonical form, options and errors as evec_generalized.
 * u_j is zero above its block; for a 1x1 block u_p = 1.  For a 2x2 block
 * the eigenvalue pair and the block part of u come from the reversed
 * transposed block (entries (s22, s12; s21, s11) against diag(d2, d1)):
 * alpha = lambda d2, beta = d2 before the power-of-two normalisation, and
 * the columns are (Re u, Im u) for Im alpha > 0 (alpha_im = +w, -w).
 * Computed as the right eigenvectors of the flipped pencil (J S^T J, J T^T
 * J) (J the reversal permutation; the blocks in reverse order) with Z J
 * for the back-transformation, so the handle holds three extra n x n and
 * one n x m FP64 workspaces.  A non-finite or over-range entry of S or T
 * strictly above the first superdiagonal is reported at evec_sync with its
 * index i + j lds (or ldt).
 */
evec_status evec_generalized_left(evec_handle h, int64_t n, const double *S, int64_t lds,
                                  const double *T, int64_t ldt, const double *Z, int64_t ldz,
                                  const uint8_t *select_host, double *X, int64_t ldx,
                                  int32_t *scale_exp, double *alpha_re, double *alpha_im,
                                  double *beta, const evec_opts *opt);

/* Number of output columns m of evec_generalized for a selection: S's 1x1
 * and 2x2 blocks (2 columns per selected 2x2 block), with the same checks
 * of the pencil's form as evec_generalized (synchronises the handle's
 * stream).  Errors: EVEC_EINVAL, EVEC_ENOTSCHUR, EVEC_ENONFINITE,
 * EVEC_ECUDA. */
evec_status evec_count_generalized(evec_handle h, int64_t n, const double *S, int64_t lds,
                                   const double *T, int64_t ldt, const uint8_t *select_host,
                                   int64_t *m);

/*
 * Robust triangular solve with many right-hand sides (the LAPACK xLATRS
 * generalisation the eigenvector solve of Sec. 3.3 rests on): for every
 * column b_j of B, the solution of T x_j = b_j, returned as
 *   x_j = X[:, j] * 2^(-scale_exp[j]),  max_i |X[i, j]| in [1, 2)
 * (X[:, j] = 0 and scale_exp[j] = 0 for b_j = 0), computed by the tiled
 * steps of evec_standard with shift 0 and b_j as the starting segments:
 * every intermediate stays below 2^1020, pivots below 2^-1022 n / ulp are
 * perturbed up to it (a singular T still gives a finite X).
 *   T [ldt x n]: upper quasi-triangular, 1x1 and 2x2 diagonal blocks from
 *     its first subdiagonal (a 2x2 block in any form; no two consecutive
 *     nonzero subdiagonal entries, else EVEC_ENOTSCHUR); the strictly lower
 *     part below the first subdiagonal is not read.
 *   B [ldb x nrhs], X [ldx x nrhs], scale_exp [nrhs]: device pointers on
 *     the handle's device; X may equal B (ldx == ldb) for an in-place solve.
 *   opt: mode (EVEC_FP64 or EVEC_SPLIT updates), tile, slices, check as for
 *     evec_standard; refine is ignored.
 * Errors: EVEC_EINVAL (bad argument or an entry above 2^1000),
 * EVEC_ENOTSCHUR, EVEC_ENONFINITE; device-detected ones through evec_sync
 * with index i + j ldt for T and ldt n + i + j ldb for B.
 */
evec_status evec_trsolve(evec_handle h, int64_t n, const double *T, int64_t ldt, int64_t nrhs,
                         const double *B, int64_t ldb, double *X, int64_t ldx,
                         int32_t *scale_exp, const evec_opts *opt);

/* ---- batched mode --------------------------------------------------------
 * count independent real Schur forms packed in one device buffer: T_i
 * (order n_host[i], column-major, leading dimension n_i) starts at
 * T_packed + t_off_host[i].  select_host: n_i bytes per matrix, back to back
 * in matrix order, with the meaning of evec_standard's mask (NULL: every
 * eigenvector of every matrix).  Host arrays are read during the call.
 */

/* Output columns m_i of each matrix (m_host: count entries, host). */
evec_status evec_batched_count(evec_handle h, int64_t count, const int64_t *n_host,
                               const double *T_packed, const int64_t *t_off_host,
                               const uint8_t *select_host, int64_t *m_host);

/*
 * Right eigenvectors of every matrix (evec_standard per matrix, with or
 * without its own Q) in one persistent launch: a device work queue hands
 * whole matrices to CTAs, largest estimated work first; the device part of
 * the call (plan upload, queue reset, launch) is a CUDA graph, replayed
 * while the batch layout, buffers and offsets stay the same.
 *   Q_packed (device, may be NULL) with q_off_host (host, count entries):
 *     matrix i with q_off_host[i] >= 0 is back-transformed, X_i = Q_i Y_i
 *     with Q_i (n_i x n_i, leading dimension n_i) at Q_packed +
 *     q_off_host[i], and brought to canonical form; q_off_host[i] < 0 (or
 *     Q_packed NULL) returns Y_i itself.  The CTA that solved the matrix
 *     forms the product (FP64; K runs to the block end of each 64-column
 *     block's last column), and the handle keeps Y_i in its workspace.
 *   X_i (n_i x m_i, leading dimension n_i) at X_packed + x_off_host[i],
 *     scale_exp_i and lam_re_i / lam_im_i (m_i each; lam may be NULL) at
 *     offset e_off_host[i] of their arrays; x_off_host / e_off_host NULL
 *     pack them in matrix order (X_i at sum_{k<i} n_k m_k, the others at
 *     sum_{k<i} m_k).  Outputs must not overlap.
 * opt->mode: EVEC_FP64, or EVEC_SPLIT (opt->slices digit slices, 2..8;
 * 0 = 8): the updates of every matrix as BF16 slice products on the tensor
 * cores inside the same persistent kernel (each CTA holds 256 TMEM columns;
 * two CTAs per SM); the diagonal solves, decisions, back-transformation
 * and canonical form stay FP64.  opt->refine is ignored here.
 * opt->tile: 16..64 for every matrix, or 0 = the tile of each matrix's size
 * class from the handle's table, tuned on first use of a class by timing
 * 16, 32 and 64 on up to eight of the batch's matrices of that class.
 * Errors: EVEC_EINVAL (a NULL q_off_host with Q_packed, a negative output
 * offset, ...); device-side errors (evec_sync / opt->check): index =
 * element offset in T_packed.
 */
evec_status evec_batched(evec_handle h, int64_t count, const int64_t *n_host,
                         const double *T_packed, const int64_t *t_off_host,
                         const double *Q_packed, const int64_t *q_off_host,
                         const uint8_t *select_host, double *X_packed,
                         const int64_t *x_off_host, int32_t *scale_exp_packed,
                         const int64_t *e_off_host, double *lam_re_packed,
                         double *lam_im_packed, const evec_opts *opt);

/*
 * Generalized right eigenvectors of a batch of pencils (S_i, T_i) (the
 * single-pencil computation of evec_generalized) in one persistent launch
 * of the pencil variant of the batched kernel: each CTA takes whole
 * pencils from the work queue, computes the norms of both matrices, runs
 * the diagonal-tile solves of (beta S - alpha T) and the updates
 * Y_r <- 2^dy Y_r - [S_rs (beta X~) - T_rs (alpha X~)] in FP64, and writes
 * the canonical form.  S_i, T_i (n_i x n_i, leading dimension n_i) at
 * S_packed + s_off_host[i] and T_packed + t_off_host[i], with the
 * requirements of evec_generalized.
 *   Z_packed (device, may be NULL) with z_off_host (host, count entries):
 *     pencil i with z_off_host[i] >= 0 is back-transformed, X_i = Z_i Y_i
 *     with Z_i (n_i x n_i, leading dimension n_i) at Z_packed +
 *     z_off_host[i], by the CTA that solved it (FP64), then brought to
 *     canonical form; z_off_host[i] < 0 (or Z_packed NULL) returns Y_i.
 *     The handle keeps Y_i in its workspace.
 * Output packing as evec_batched (X_i at sum_{k<i} n_k m_k; scale_exp_i,
 * alpha_re_i, alpha_im_i, beta_i at sum_{k<i} m_k; the last three may be
 * NULL); m_i from evec_batched_generalized_count.  opt->mode: EVEC_FP64,
 * or EVEC_SPLIT (opt->slices digit slices, 2..8; 0 = 8): each update as
 * one split product of the rows [S_rs T_rs] against the 2K-row right-hand
 * side [beta X~; -alpha X~] on the tensor cores inside the persistent
 * kernel; the diagonal solves, decisions, back-transformation and
 * canonical form stay FP64.  opt->tile 16..64 for every pencil (the solver
 * holds both matrices' diagonal tiles: one CTA per SM at 64), or 0 = in
 * EVEC_FP64 mode the tile of each pencil's size class from the handle's
 * pencil table (EVEC_TUNE_PENCIL), tuned on first use of a class by timing
 * 16, 32 and 64 on up to eight of the batch's pencils of that class; in
 * EVEC_SPLIT mode 64.  As in
 * evec_batched, the device
 * part of the call is a CUDA graph, replayed while the call is the same
 * (layout, buffers, offsets, selection, tile, and the three central
 * diagonals of every S_i and T_i; the entries above them may change); a
 * call of evec_batched_generalized_count in between ends the replay.
 * Errors: EVEC_EINVAL also for Z_packed without z_off_host.  Device-side
 * errors (evec_sync / opt->check): index = element offset in S_packed or
 * T_packed of the offending entry.
 */
evec_status evec_batched_generalized(evec_handle h, int64_t count, const int64_t *n_host,
                                     const double *S_packed, const int64_t *s_off_host,
                                     const double *T_packed, const int64_t *t_off_host,
                                     const double *Z_packed, const int64_t *z_off_host,
                                     const uint8_t *select_host, double *X_packed,
                                     int32_t *scale_exp_packed, double *alpha_re_packed,
                                     double *alpha_im_packed, double *beta_packed,
                                     const evec_opts *opt);

/* Output columns m_i of each pencil of a packed batch (m_host: count
 * entries, host), with the checks of evec_batched_generalized. */
evec_status evec_batched_generalized_count(evec_handle h, int64_t count, const int64_t *n_host,
                                           const double *S_packed, const int64_t *s_off_host,
                                           const double *T_packed, const int64_t *t_off_host,
                                           const uint8_t *select_host, int64_t *m_host);

/* Size classes of the tile table: n <= 64, <= 128, <= 256, <= 512, larger. */
#define EVEC_SIZE_CLASSES 5

/* The table of batched pencils (evec_batched_generalized, FP64) in
 * evec_tune_get / evec_tune_set. */
#define EVEC_TUNE_PENCIL 2

/* The handle's tile tables (mode = evec_mode for evec_batched, or
 * EVEC_TUNE_PENCIL; size_class < EVEC_SIZE_CLASSES); tile 0 = not tuned
 * yet.  evec_tune_set accepts 0 (forget) or 16..64. */
evec_status evec_tune_get(evec_handle h, int mode, int size_class, int *tile);
evec_status evec_tune_set(evec_handle h, int mode, int size_class, int tile);

/* Limits of evec_standard_noalloc. */
#define EVEC_NOALLOC_MAX_N 512
#define EVEC_NOALLOC_SCRATCH_BYTES (1 << 20)

/*
 * evec_standard_noalloc -- the paper has no counterpart to this entry point;
 * it exists for callers that cannot allocate GPU memory while they run: a
 * serving process whose own memory pool already owns the device, code where
 * a cudaMalloc would synchronise the device or fail, a program with a fixed,
 * pre-reserved memory budget.  It computes the same result as evec_standard
 * with Q == NULL (X = Y, canonical columns, scale_exp) for n <= 512, and
 * allocates nothing: no handle, no cudaMalloc / cudaFree, no pinned host
 * memory.  All scratch lives in one fixed device array of
 * EVEC_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits.
 *   T [ldt x n], X [ldx x m] output, scale_exp [m]: device pointers on the
 *   current device; select_host as for evec_standard (m from evec_count or
 *   evec_plan_query); tile: 16..128, 0 = 64; cuda_stream: stream of the
 *   current device (NULL = legacy default stream).
 * The first call on a device looks up the array's device address (with
 * that device current).
 * Every call shares the array and reuses whatever the previous call left in
 * it (the status word is cleared at the start of each call; everything else
 * is written before it is read).  Two calls that overlapped on the GPU
 * would race on the array, so the library prevents overlap: the call is
 * synchronous, calls are serialised inside the library, and each one
 * synchronises its stream before it returns, on success and on every error
 * after it queued work.  Each process that loads the library has its own
 * copy of the array.
 * Returns, synchronously: EVEC_ECAPACITY when n > EVEC_NOALLOC_MAX_N or the
 * chosen tile needs more than the fixed scratch; EVEC_EINVAL,
 * EVEC_ENOTSCHUR, EVEC_ENONFINITE (with *bad_index, linear index into T) as
 * evec_standard and evec_sync would; EVEC_ECUDA on a runtime error.
 */
evec_status evec_standard_noalloc(int64_t n, const double *T, int64_t ldt,
                                  const uint8_t *select_host, double *X, int64_t ldx,
                                  int32_t *scale_exp, int tile, void *cuda_stream,
                                  int64_t *bad_index);

/* Text of the most recent CUDA runtime error that made a call of this
 * library on the calling host thread return EVEC_ECUDA or EVEC_ENOMEM. */
const char *evec_last_cuda_error(void);

/* Static, human-readable name of a status code. */
const char *evec_strerror(evec_status s);

/* 1 when this library is the checked build (compiled with -DEVEC_CHECK:
 * the kernels test the row, column, tile and segment indices of their main
 * device accesses against the plan, skip an access that fails and report
 * EVEC_EBOUNDS at evec_sync with the site's number as the index), else 0.
 * Results are otherwise identical to the normal build's. */
int evec_checked_build(void);

#ifdef __cplusplus
}
#endif

#endif /* EVEC_H */
