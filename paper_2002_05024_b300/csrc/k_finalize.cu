// k_finalize.cu -- the post-processing of Sec. 3.4: all segments of each
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
    // the own block is never zero, so t is set

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
    k_canonicalize(Plan P, double *__restrict__ X, int64_t ldx, int32_t *__restrict__ scale_exp) {
    const int u = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = P.n;
    const int col = P.unit_col[u];
    const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
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

void launch_finalize(const Plan &p, double *Y, int64_t ldy, const int32_t *seg_e,
                     int32_t *scale_exp, cudaStream_t st) {
    if (p.nunits <= 0) return;
    k_finalize<<<p.nunits, kWarps * 32, 0, st>>>(p, Y, ldy, seg_e, scale_exp);
}

void launch_canonicalize(const Plan &p, double *X, int64_t ldx, int32_t *scale_exp,
                         cudaStream_t st) {
    if (p.nunits <= 0) return;
    k_canonicalize<<<p.nunits, kWarps * 32, 0, st>>>(p, X, ldx, scale_exp);
}

}  // namespace evec
