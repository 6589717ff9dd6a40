// k_finalize.cu -- the post-processing of Sec. 3.3: all segments of each
// column brought to one consistent scaling, in canonical form.
//
// Segment r of column j holds y_true = Y * 2^(-e_r).  With
//   t = floor(log2 |y_true|_inf) = max over nonzero segments of
//       (floor(log2 nu_r) - e_r)            (exact: e_r is an integer)
// every entry becomes x = Y * 2^(-e_r - t) in one exact power-of-two scaling,
// so |x|_inf lies in [1, 2) and scale_exp = -t (y_true = x * 2^-scale_exp).
// For a complex pair the norm is max_i |re_i| + |im_i| and both columns
// share t.  Rows below the column's own block are written as zeros.
// One CTA (8 warps) per unit; the column is read twice and written once:
// HBM-bound, about 3 * 8 * n bytes per column.
#include "evec_internal.cuh"

namespace evec {

namespace {
constexpr int kWarps = 8;

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_imax(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
}  // namespace

__global__ void __launch_bounds__(kWarps * 32)
    k_finalize(Plan P, double *__restrict__ Y, int64_t ldy, const int32_t *__restrict__ seg_e,
               int32_t *__restrict__ scale_exp) {
    const int u = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t m = P.m, n = P.n;
    const int col = P.unit_col[u];
    const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
    const int c = P.unit_tile[u];
    const int kb = P.unit_blk[u];
    const int row_end = P.blk_start[kb] + P.blk_size[kb];
    if (!evec_in(P, u < P.nunits && col + (cplx ? 1 : 0) < m && row_end <= n && c < P.ntiles,
                 131))
        return;
    double *yr = Y + (int64_t)col * ldy;
    double *yi = Y + (int64_t)(col + 1) * ldy;
    __shared__ int sbest[kWarps];

    // pass 1: per segment maximum, combined through the exponents
    int best = INT32_MIN;
    for (int r = warp; r <= c; r += kWarps) {
        const int a = P.tile_start[r];
        const int b = min(P.tile_start[r + 1], row_end);
        double mx = 0.0;
        for (int i = a + lane; i < b; i += 32) {
            double v = fabs(yr[i]);
            if (cplx) v += fabs(yi[i]);
            mx = fmax(mx, v);
        }
        mx = warp_max(mx);
        if (mx > 0.0) best = max(best, ilog2_abs(mx) - seg_e[(int64_t)r * m + col]);
    }
    best = warp_imax(best);
    if (lane == 0) sbest[warp] = best;
    __syncthreads();
    int t = INT32_MIN;
#pragma unroll
    for (int w = 0; w < kWarps; w++) t = max(t, sbest[w]);
    // an eigenvector's own block is never zero; a correction (residual
    // sweep) can be: then every entry is zero and any t will do
    if (t == INT32_MIN) t = 0;

    // pass 2: one exact scaling per entry
    for (int r = warp; r <= c; r += kWarps) {
        const int a = P.tile_start[r];
        const int b = min(P.tile_start[r + 1], row_end);
        const int k = -seg_e[(int64_t)r * m + col] - t;
        for (int i = a + lane; i < b; i += 32) {
            yr[i] = scale2(yr[i], k);
            if (cplx) yi[i] = scale2(yi[i], k);
        }
    }
    for (int64_t i = row_end + threadIdx.x; i < n; i += kWarps * 32) {
        yr[i] = 0.0;
        if (cplx) yi[i] = 0.0;
    }
    if (threadIdx.x == 0) {
        scale_exp[col] = -t;
        if (cplx) scale_exp[col + 1] = -t;
    }
}

// Re-canonicalise after the back-transformation: X[:, unit] <- X * 2^-t2,
// t2 = floor(log2 |X|), scale_exp -= t2.
__global__ void __launch_bounds__(kWarps * 32)
    k_canonicalize(Plan P, double *__restrict__ X, int64_t ldx, int32_t *__restrict__ scale_exp,
                   int u0) {
    const int u = u0 + blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = P.n;
    if (!evec_in(P, u < P.nunits, 132)) return;
    const int col = P.unit_col[u];
    const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
    if (!evec_in(P, col + (cplx ? 1 : 0) < P.m, 133)) return;
    double *xr = X + (int64_t)col * ldx;
    double *xi = X + (int64_t)(col + 1) * ldx;
    __shared__ double smax[kWarps];

    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kWarps * 32) {
        double v = fabs(xr[i]);
        if (cplx) v += fabs(xi[i]);
        mx = fmax(mx, v);
    }
    mx = warp_max(mx);
    if (lane == 0) smax[warp] = mx;
    __syncthreads();
    mx = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) mx = fmax(mx, smax[w]);
    if (mx == 0.0) return;
    const int t2 = ilog2_abs(mx);
    for (int64_t i = threadIdx.x; i < n; i += kWarps * 32) {
        xr[i] = scale2(xr[i], -t2);
        if (cplx) xi[i] = scale2(xi[i], -t2);
    }
    if (threadIdx.x == 0) {
        scale_exp[col] -= t2;
        if (cplx) scale_exp[col + 1] -= t2;
    }
}

// Right-hand side of the correction solve: the residual R holds, per
// segment, -(T - lambda I) y in that segment's own scale 2^e_r (the
// exponents of the solve stay in seg_e); its segment maxima start seg_nu.
// One CTA per unit.
__global__ void __launch_bounds__(kWarps * 32)
    k_rhs_init(Plan P, const double *__restrict__ R, int64_t ldr, double *__restrict__ seg_nu) {
    const int u = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t m = P.m;
    const int col = P.unit_col[u];
    const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
    const int c = P.unit_tile[u];
    for (int r = warp; r <= c; r += kWarps) {
        const int a = P.tile_start[r], b = P.tile_start[r + 1];
        double mr = 0.0, mi = 0.0;
        for (int i = a + lane; i < b; i += 32) {
            mr = fmax(mr, fabs(R[i + col * ldr]));
            if (cplx) mi = fmax(mi, fabs(R[i + (col + 1) * ldr]));
        }
        mr = warp_max(mr);
        mi = warp_max(mi);
        if (lane == 0) {
            seg_nu[(int64_t)r * m + col] = mr;
            if (cplx) seg_nu[(int64_t)r * m + col + 1] = mi;
        }
    }
}

// y <- y + d, segment by segment: y_r = Y_r 2^-ey_r, d_r = D_r 2^-ed_r, so
// Y_r <- Y_r + D_r 2^(ey_r - ed_r) (exact power-of-two scaling, one FP64
// addition per entry), the exponents of y unchanged.  With
//   t_y = max_r floor(log2 |Y_r|) - ey_r,  t_d = the same for D,
// the correction is taken only if |d| / |y| < 2^(t_d + 1 - t_y) stays at or
// below 2^max_rel and no scaled segment of D reaches 2^1000.  The caller
// sets max_rel from the split error (products carry ~2^(-7 slices) of their
// row / column maxima, grown through the solve): a larger correction is not
// that error but the FP64 rounding of the residual amplified by
// (T - lambda I)^-1 (an ill-conditioned column, clustered eigenvalues), and
// there the unrefined column is the better one.  One CTA per unit.
__global__ void __launch_bounds__(kWarps * 32)
    k_refine_combine(Plan P, double *__restrict__ Y, int64_t ldy,
                     const int32_t *__restrict__ ey, const double *__restrict__ D, int64_t ldd,
                     const int32_t *__restrict__ ed, int max_rel) {
    const int u = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t m = P.m;
    const int col = P.unit_col[u];
    const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
    const int c = P.unit_tile[u];
    const int kb = P.unit_blk[u];
    const int pend = P.blk_start[kb];   // rows above the block; the block is fixed
    __shared__ int sty[kWarps], std_[kWarps], sover[kWarps];
    int ty = INT32_MIN, td = INT32_MIN, over = 0;   // over: too large or not finite
    for (int r = warp; r <= c; r += kWarps) {
        const int a = P.tile_start[r];
        const int b = min(P.tile_start[r + 1], P.blk_start[kb] + P.blk_size[kb]);
        double my = 0.0, md = 0.0;
        for (int i = a + lane; i < b; i += 32) {
            double vy = fabs(Y[i + col * ldy]), vd = fabs(D[i + col * ldd]);
            if (cplx) {
                vy += fabs(Y[i + (col + 1) * ldy]);
                vd += fabs(D[i + (col + 1) * ldd]);
            }
            my = fmax(my, vy);
            md = fmax(md, vd);
            if (!isfinite(vd)) over = 1;
        }
        my = warp_max(my);
        md = warp_max(md);
        const int64_t at = (int64_t)r * m + col;
        if (my > 0.0) ty = max(ty, ilog2_abs(my) - ey[at]);
        if (md > 0.0) {
            td = max(td, ilog2_abs(md) - ed[at]);
            if (ilog2_abs(md) + ey[at] - ed[at] >= 1000) over = 1;
        }
    }
    ty = warp_imax(ty);
    td = warp_imax(td);
    over = warp_imax(over);
    if (lane == 0) {
        sty[warp] = ty;
        std_[warp] = td;
        sover[warp] = over;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kWarps; w++) {
        ty = max(ty, sty[w]);
        td = max(td, std_[w]);
        over |= sover[w];
    }
    // no correction (td unset), or one too large to be the split error
    if (td == INT32_MIN || over || ty == INT32_MIN || td + 1 - ty > max_rel) return;
    for (int r = warp; r <= c; r += kWarps) {
        const int a = P.tile_start[r];
        const int b = min(P.tile_start[r + 1], pend);
        const int64_t at = (int64_t)r * m + col;
        const int k = ey[at] - ed[at];
        for (int i = a + lane; i < b; i += 32) {
            Y[i + col * ldy] += scale2(D[i + col * ldd], k);
            if (cplx) Y[i + (col + 1) * ldy] += scale2(D[i + (col + 1) * ldd], k);
        }
    }
}

__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ||T||_1 over the referenced part (upper triangle and first subdiagonal):
// the largest column sum, merged by atomicMax on the bit patterns (the order
// of non-negative doubles); one warp per column.
__global__ void __launch_bounds__(kWarps * 32)
    k_norm1(const double *__restrict__ T, int64_t ldt, int64_t n,
            unsigned long long *__restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * kWarps + warp;
    if (j >= n) return;
    const int64_t iend = min(j + 2, n);
    double s = 0.0;
    for (int64_t i = lane; i < iend; i += 32) s += fabs(T[i + j * ldt]);
    s = warp_sumd(s);
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

// The residual gate of one unit (one CTA): the normalised residual
// ||(T - lambda I) y||_1 / (||T||_1 ||y||_1 u), u = 2^-53 (pairs: sums of
// |re| + |im|), from the segments Y_r (scale 2^-ey_r) and the residual R_r
// in the same scales (k_residual; zero at and below the block).  Both sums
// are taken in the common scale of the largest segment (exact powers of
// two), so nothing overflows.  Units above `limit` (or not finite) are
// counted in *fails; ratio[u] receives the value.
__global__ void __launch_bounds__(kWarps * 32)
    k_gate(Plan P, const double *__restrict__ Y, int64_t ldy, const int32_t *__restrict__ ey,
           const double *__restrict__ R, int64_t ldr, const unsigned long long *__restrict__ tn,
           double limit, int *__restrict__ fails, double *__restrict__ ratio,
           int *__restrict__ first_col) {
    const int u = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t m = P.m;
    const int col = P.unit_col[u];
    const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
    const int c = P.unit_tile[u];
    const int kb = P.unit_blk[u];
    const int bend = P.blk_start[kb] + P.blk_size[kb];
    __shared__ int sE[kWarps];
    __shared__ double sy[kWarps], sr[kWarps];
    int E = INT32_MIN;
    for (int r = warp; r <= c; r += kWarps) {
        const int a = P.tile_start[r], b = min(P.tile_start[r + 1], bend);
        double my = 0.0;
        for (int i = a + lane; i < b; i += 32) {
            double v = fabs(Y[i + (int64_t)col * ldy]);
            if (cplx) v += fabs(Y[i + (int64_t)(col + 1) * ldy]);
            my = fmax(my, v);
        }
        my = warp_max(my);
        if (my > 0.0) E = max(E, ilog2_abs(my) - ey[(int64_t)r * m + col]);
    }
    E = warp_imax(E);
    if (lane == 0) sE[warp] = E;
    __syncthreads();
    int Eall = INT32_MIN;
#pragma unroll
    for (int w = 0; w < kWarps; w++) Eall = max(Eall, sE[w]);
    double ty = 0.0, tr = 0.0;
    if (Eall != INT32_MIN) {
        for (int r = warp; r <= c; r += kWarps) {
            const int a = P.tile_start[r], b = min(P.tile_start[r + 1], bend);
            double yy = 0.0, rr = 0.0;
            for (int i = a + lane; i < b; i += 32) {
                yy += fabs(Y[i + (int64_t)col * ldy]);
                rr += fabs(R[i + (int64_t)col * ldr]);
                if (cplx) {
                    yy += fabs(Y[i + (int64_t)(col + 1) * ldy]);
                    rr += fabs(R[i + (int64_t)(col + 1) * ldr]);
                }
            }
            yy = warp_sumd(yy);
            rr = warp_sumd(rr);
            const int k = -ey[(int64_t)r * m + col] - Eall;
            ty += scale2(yy, k);
            tr += scale2(rr, k);
        }
    }
    if (lane == 0) { sy[warp] = ty; sr[warp] = tr; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double y1 = 0.0, r1 = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) { y1 += sy[w]; r1 += sr[w]; }
        const double tnorm = __longlong_as_double((long long)*tn);
        const double q = r1 / (tnorm * y1 * 0x1p-53);
        if (ratio) ratio[u] = q;
        if (!(q <= limit)) {
            atomicAdd(fails, 1);
            atomicMin(first_col, col);
        }
    }
}

void launch_gate(const Plan &p, const double *Y, int64_t ldy, const int32_t *ey, const double *R,
                 int64_t ldr, const double *T, int64_t ldt, double limit, void *buf,
                 double *ratio, cudaStream_t st) {
    // buf: [0] ||T||_1 bits, [1] the failure count (int) and the output
    // column of the first failing eigenvalue (int, 0x7f7f7f7f when none)
    unsigned long long *tn = (unsigned long long *)buf;
    int *fails = (int *)(tn + 1);
    cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned long long), st);
    cudaMemsetAsync(fails + 1, 0x7f, sizeof(int), st);
    k_norm1<<<(unsigned)((p.n + kWarps - 1) / kWarps), kWarps * 32, 0, st>>>(T, ldt, p.n, tn);
    k_gate<<<p.nunits, kWarps * 32, 0, st>>>(p, Y, ldy, ey, R, ldr, tn, limit, fails, ratio,
                                             fails + 1);
}

void launch_rhs_init(const Plan &p, const double *R, int64_t ldr, double *seg_nu,
                     cudaStream_t st) {
    if (p.nunits <= 0) return;
    k_rhs_init<<<p.nunits, kWarps * 32, 0, st>>>(p, R, ldr, seg_nu);
}

void launch_refine_combine(const Plan &p, double *Y, int64_t ldy, const int32_t *ey,
                           const double *D, int64_t ldd, const int32_t *ed, int max_rel,
                           cudaStream_t st) {
    if (p.nunits <= 0) return;
    k_refine_combine<<<p.nunits, kWarps * 32, 0, st>>>(p, Y, ldy, ey, D, ldd, ed, max_rel);
}

void launch_finalize(const Plan &p, double *Y, int64_t ldy, const int32_t *seg_e,
                     int32_t *scale_exp, cudaStream_t st) {
    if (p.nunits <= 0) return;
    k_finalize<<<p.nunits, kWarps * 32, 0, st>>>(p, Y, ldy, seg_e, scale_exp);
}

void launch_canonicalize(const Plan &p, double *X, int64_t ldx, int32_t *scale_exp,
                         cudaStream_t st) {
    if (p.nunits <= 0) return;
    k_canonicalize<<<p.nunits, kWarps * 32, 0, st>>>(p, X, ldx, scale_exp, 0);
}

// the same for units [u0, u1)
void launch_canonicalize_range(const Plan &p, double *X, int64_t ldx, int32_t *scale_exp, int u0,
                               int u1, cudaStream_t st) {
    if (u1 <= u0) return;
    k_canonicalize<<<u1 - u0, kWarps * 32, 0, st>>>(p, X, ldx, scale_exp, u0);
}

}  // namespace evec
