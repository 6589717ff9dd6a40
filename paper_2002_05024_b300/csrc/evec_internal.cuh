// evec_internal.cuh -- shared declarations of the CUDA path (not installed).
//
// Data layout in device memory (all FP64 matrices column-major):
//   T [ldt x n]           caller's quasi-triangular Schur form
//   Y [ldy x m]           working eigenvector matrix; X itself when no Q
//   seg_* [N x m]         one entry per (tile row r, output column j), row
//                         major: index r * m + j.  Segment (r, j) is the part
//                         of column j in the rows of tile r; it holds
//                         y_true = Y * 2^(-seg_e) (the augmented tile
//                         <alpha, X> of Sec. 3.3 with alpha = 2^seg_e).
//   tau [N x N]           tau[r * N + s] = |T_rs|_inf for r < s
//   blk_tau [nblk]        |T[tile start : q, block q]|_inf inside the tile
// Units: one unit per selected real eigenvalue (one column) or selected
// complex pair (two columns, Re then Im), in block order.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace evec {

// Overflow threshold of every bound; 2^4 of headroom below DBL_MAX covers
// the rounding of the bound arithmetic itself.
constexpr double kOmega = 0x1p1020;
constexpr double kInputMax = 0x1p1000;
constexpr double kUlp = 0x1p-52;
constexpr double kSafeMin = 0x1p-1022;
constexpr int kOmegaExp = 1020;
// dy sentinel: the segment has never been written; treat it as zero.
constexpr int32_t kFresh = INT32_MIN;
constexpr int kMaxTile = 128;      // tiles solved whole in shared memory (pencils: 64)
constexpr int kMaxTileBig = 512;   // largest tile: solved in sub-blocks of 64 rows

struct DevStatus {
    int code;          // evec_status of the first device-detected error
    int timeout;       // nonzero: a bounded device-side wait gave up
    long long index;   // linear index of the offending entry
};

// The plan: everything the kernels need about blocks, tiles and units.
// All arrays live in one device buffer; pointers are set by the host.
struct Plan {
    int64_t n, m;
    int32_t ntiles, nblk, nunits;
    int32_t nb;                 // target tile size
    const int32_t *tile_start;  // [ntiles + 1]
    const int32_t *tile_blk;    // [ntiles + 1] first block of each tile
    const int32_t *tile_unit;   // [ntiles + 1] first unit whose block is in the tile
    const int32_t *tile_col;    // [ntiles + 1] first output column of the tile's units
    const int32_t *blk_start;   // [nblk]
    const int8_t *blk_size;     // [nblk]
    const int32_t *unit_col;    // [nunits] first output column
    const int32_t *unit_blk;    // [nunits] block index
    const int32_t *unit_tile;   // [nunits]
    const double *unit_lam;     // [2 * nunits] (re, im), im > 0 for a pair
    const double *unit_own;     // [4 * nunits] block part: re0, re1, im0, im1
    const int32_t *col_unit;    // [m] unit of each column
    // solve order: real units and complex units, each in unit order, so the
    // units active at step s (block in tile >= s) are a suffix of each list
    int32_t nreal, ncplx;
    const int32_t *ord_real;    // [nreal] unit indices
    const int32_t *ord_cplx;    // [ncplx]
    const int32_t *tile_real;   // [ntiles + 1] first position in ord_real with tile >= s
    const int32_t *tile_cplx;   // [ntiles + 1]
    // pencils (beta S - alpha T) only, else null: unit_lam holds alpha
    const double *unit_beta;    // [nunits]
    const double *unit_smin;    // [nunits] perturbation threshold of the small solves
    DevStatus *status;          // the handle's status word (bounds reports of a checked build)
};

// Bounds checks of the checked build (compiled with -DEVEC_CHECK): a
// guarded access runs only when evec_in(P, ok, site) holds; a failed check
// records EVEC_EBOUNDS (9) with the site's number as the index in the
// plan's status word, so evec_sync reports it, and the access is skipped.
// In the normal build evec_in is `true` and the compiler drops the test.
#ifdef EVEC_CHECK
__device__ __forceinline__ bool evec_in(const Plan &P, bool ok, int site) {
    if (!ok && P.status && atomicCAS(&P.status->code, 0, 9) == 0) P.status->index = site;
    return ok;
}
#else
__device__ __forceinline__ bool evec_in(const Plan &, bool, int) { return true; }
#endif

// The second matrix T of a pencil (upper triangular) with its tile norms
// (tau[r * N + s] = |T_rs|_inf) and in-tile block column norms.
struct Pencil {
    const double *T = nullptr;
    int64_t ldt = 0;
    const double *tau = nullptr;
    const double *blk_tau = nullptr;
};

// One matrix of the batched mode: its plan, input, output and workspaces.
struct BatchItem {
    Plan P;
    const double *T;
    int64_t ldt;
    int64_t t_base;   // element offset of T in the packed input (error indices)
    double *X;
    int64_t ldx;
    int32_t *scale_exp;
    double *tau, *blk_tau, *seg_nu;
    int32_t *seg_e, *seg_dx, *seg_dy;
    // pencils (beta S - alpha T): T here is S, T2 the upper triangular T
    // with its tile norms; null for a standard problem
    const double *T2;
    int64_t ldt2;
    int64_t t2_base;
    double *tau2, *blk_tau2;
    // back-transformation (standard problem): with Q non-null the solve
    // writes Y into X (a workspace, leading dimension n), then the CTA forms
    // Xout = Q Y and its canonical form; without Q, Xout == X
    const double *Q;
    int64_t ldq;
    double *Xout;
    int64_t ldxo;
    // eigenvalues per output column (may be null), written by the CTA
    double *lam_re, *lam_im;
};

// ---------------------------------------------------------------------------
// exact power-of-two scaling, from the IEEE-754 binary64 encoding
// ---------------------------------------------------------------------------

// 2^k for -1022 <= k <= 1023 (a normal number).
__device__ __forceinline__ double pow2_normal(int k) {
    return __longlong_as_double((long long)(k + 1023) << 52);
}

// x * 2^k for any integer k, by at most three exact multiplications; only a
// result in the subnormal range is rounded (once per step).
__device__ __forceinline__ double scale2(double x, int k) {
    if (k >= -1022 && k <= 1023) return x * pow2_normal(k);
    if (k < -1022) {
        if (k < -2200) return x * 0.0;
        x *= pow2_normal(-1022);
        k += 1022;
        if (k < -1022) { x *= pow2_normal(-1022); k += 1022; if (k < -1022) k = -1022; }
        return x * pow2_normal(k);
    }
    if (k > 2200) k = 2200;
    x *= pow2_normal(1023);
    k -= 1023;
    if (k > 1023) { x *= pow2_normal(1023); k -= 1023; }
    return x * pow2_normal(k);
}

// floor(log2 |x|) for finite nonzero x, from the exponent field (subnormals
// handled through one exact rescaling).
__device__ __forceinline__ int ilog2_abs(double x) {
    long long b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
    int ex = (int)(b >> 52);
    if (ex == 0) {  // subnormal
        double y = __longlong_as_double(b) * 0x1p64;
        long long c = __double_as_longlong(y);
        return (int)(c >> 52) - 1023 - 64;
    }
    return ex - 1023;
}

// Update protection (Sec. 3.3: before Z <- Y - T X, scale so the result
// cannot exceed the threshold).  nu = |y|, tau = |T|, mu = |x|, with
// nu <= Omega and tau <= Omega.  Returns q <= 0 such that
// 2^q nu + tau 2^q mu <= Omega.
// The test is tau * mu > Omega - nu: a product that overflows to +Inf
// (tau, mu <= Omega) still compares as "too large", so no division is needed.
__device__ __forceinline__ int protect_update(double nu, double tau, double mu) {
    if (!(tau * mu > kOmega - nu)) return 0;
    return mu <= 1.0 ? -1 : -2 - ilog2_abs(mu);
}

// protect_update for the decisions of a tile update, with nu and mu given
// as doubles times powers of two: q for (nu 2^kn, tau, mu 2^km).  The common
// case is decided on exponent fields alone (integer pipe): nu 2^kn <
// 2^(field(nu) - 1022 + kn) and likewise for tau and mu, so when the larger
// of the two bounds is at most 2^1019 the sum stays below 2^1020 = Omega and
// the FP64 test of protect_update would return 0 as well (its rounded
// product is at most 2^1019, its rounded Omega - nu at least 2^1019).
// Otherwise the scaled values are formed and the FP64 test decides.
__device__ __forceinline__ int protect_update_scaled(double nu, int kn, double tau, double mu,
                                                     int km) {
    const int fn = (__double2hiint(nu) >> 20) & 0x7ff, ft = (__double2hiint(tau) >> 20) & 0x7ff;
    const int fm = (__double2hiint(mu) >> 20) & 0x7ff;
    const int en = nu == 0.0 ? INT32_MIN / 2 : fn - 1022 + kn;
    const int ep = (tau == 0.0 || mu == 0.0) ? INT32_MIN / 2 : (ft - 1022) + (fm - 1022 + km);
    if (max(en, ep) <= kOmegaExp - 1) return 0;
    return protect_update(scale2(nu, kn), tau, scale2(mu, km));
}

// 1 / x for finite nonzero x without the IEEE division sequence: x = m 2^k
// with m in [1, 2) (exponent field), a hardware approximation of 1/m
// (rcp.approx.ftz.f64), two Newton-Raphson steps r <- r + r (1 - m r) in
// FP64, then the exact rescaling by 2^-k.  Relative error within a few ulp.
__device__ __forceinline__ double rcp_fast(double x) {
    long long b = __double_as_longlong(x);
    int ex = (int)((b >> 52) & 0x7ff);
    int adj = 0;
    if (ex == 0) {  // subnormal: rescale exactly first
        x *= 0x1p64;
        b = __double_as_longlong(x);
        ex = (int)((b >> 52) & 0x7ff);
        adj = 64;
    }
    const double m = __longlong_as_double((b & 0x800fffffffffffffLL) | (1023LL << 52));
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(m));
    double e = fma(-m, r, 1.0);
    r = fma(r, e, r);
    e = fma(-m, r, 1.0);
    r = fma(r, e, r);
    return scale2(r, 1023 - ex + adj);
}

// Biased exponent field of x (0 for zero and subnormals): |x| < 2^(field - 1022).
// Integer arithmetic on fields replaces FP64 compares on latency chains.
__device__ __forceinline__ int efield(double x) {
    return (__double2hiint(x) >> 20) & 0x7ff;
}

// max of |a| over doubles through their bit patterns (integer pipe): the
// order of non-negative IEEE doubles is the order of their encodings.
__device__ __forceinline__ long long abs_bits(double x) {
    return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

__device__ __forceinline__ void report(DevStatus *st, int code, long long index) {
    if (atomicCAS(&st->code, 0, code) == 0) st->index = index;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may be set up while the previous kernel of
// its stream still runs; grid_dependency_wait() blocks until that kernel has
// completed and its writes are visible (a no-op for a normal launch), so
// only reads of data no earlier kernel writes (the input matrix, the plan)
// may precede it.  The update kernels before a diagonal solve do not
// trigger their dependents early: measured on B300 at n = 4096, an early
// trigger at their start made the split solve 7% slower, while the launch
// alone (dependents released at the update's end) saved 1.4%.
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Slice buffers of the split-precision Hessenberg updates: the A chain (t*)
// and the Q chain (q*); *a: left-operand slices, S x split_pad_m(n) x
// split_pad_k(n) BF16; *b: right-operand slices, S x max(split_pad_m(n) x
// 64, 64 x split_pad_k(n)); *am / *ae and *bm / *be: maxima and exponents,
// split_pad_m(n) (at least 64) entries; tp / qp: partial products of a K
// split, kHSplitMax x split_pad_m(n) x 32 doubles.
constexpr int kHSplitMax = 16;
struct HessSplitWs {
    __nv_bfloat16 *ta, *tb, *qa, *qb;
    unsigned long long *tam, *tbm, *qam, *qbm;
    int *tae, *tbe, *qae, *qbe;
    double *tp, *qp;
};

// One window of a disjoint set for the reordering updates: rows and
// columns [a, a + k), accumulator at Z + zoff, first CTA of its tiles cta0.
struct WinDesc {
    int64_t a, zoff, cta0;
    int k, pad;
};

}  // namespace evec
