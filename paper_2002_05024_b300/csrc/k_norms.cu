// k_norms.cu -- input gathering and tile norms (the bounds of Sec. 3.3).
//
// tau[r * N + s] = |T_rs|_inf (largest row sum of |T| over the rows of tile
// r and the columns of tile s, r < s) bounds every off-diagonal tile update
// Y_r <- Y_r - T_rs X_s; blk_tau[k] = |T[tile start : q, q : q + size_k]|_inf
// bounds the in-tile update from diagonal block k (start q).  The kernel
// also validates every referenced entry (finite, |t| <= 2^1000).
// Reads the upper triangle of T once: HBM-bound, n (n + 1) / 2 * 8 bytes.
#include <algorithm>

#include "evec_internal.cuh"

namespace evec {

__global__ void k_gather_diagonals(const double *__restrict__ T, int64_t ldt, int64_t n,
                                   double *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = T[i + i * ldt];
    if (i + 1 < n) {
        out[n + i] = T[(i + 1) + i * ldt];           // subdiagonal
        out[2 * n - 1 + i] = T[i + (i + 1) * ldt];   // superdiagonal
    }
}

void launch_gather_diagonals(const double *T, int64_t ldt, int64_t n, double *out,
                             cudaStream_t st) {
    int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    k_gather_diagonals<<<(unsigned)blocks, threads, 0, st>>>(T, ldt, n, out);
}

// The same three diagonals for a batch: matrix i (order n_i, column-major,
// ld = n_i, at T + t_off[i]) owns rows [row_off[i], row_off[i + 1]) of the
// batch and writes diag / sub / super at 3 row_off[i] + (0, n_i, 2 n_i - 1).
__global__ void k_gather_batched(const double *__restrict__ T, const int64_t *__restrict__ t_off,
                                 const int64_t *__restrict__ row_off, int count,
                                 int64_t total_rows, double *__restrict__ out) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total_rows) return;
    int lo = 0, hi = count - 1;   // last matrix with row_off[i] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const int64_t n = row_off[lo + 1] - row_off[lo], r = g - row_off[lo];
    const double *A = T + t_off[lo];
    double *o = out + 3 * row_off[lo];
    o[r] = A[r + r * n];
    if (r + 1 < n) {
        o[n + r] = A[(r + 1) + r * n];
        o[2 * n - 1 + r] = A[r + (r + 1) * n];
    }
}

void launch_gather_batched(const double *T, const int64_t *t_off, const int64_t *row_off,
                           int count, int64_t total_rows, double *out, cudaStream_t st) {
    if (total_rows <= 0) return;
    k_gather_batched<<<(unsigned)((total_rows + 255) / 256), 256, 0, st>>>(T, t_off, row_off, count,
                                                                           total_rows, out);
}

__device__ __forceinline__ void check_entry(double v, long long idx, DevStatus *st) {
    if (!isfinite(v)) report(st, 3 /* EVEC_ENONFINITE */, idx);
    else if (fabs(v) > kInputMax) report(st, 1 /* EVEC_EINVAL */, idx);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One CTA of 128 threads per tile pair (r, s), r <= s; blockIdx.x runs over
// the upper triangle of the tile grid, column by column.
// lower = 0: T is upper triangular (the second matrix of a pencil) and its
// first subdiagonal is neither read nor validated.
__global__ void __launch_bounds__(128) k_tile_norms(const double *__restrict__ T, int64_t ldt,
                                                    Plan P, double *__restrict__ tau,
                                                    double *__restrict__ blk_tau,
                                                    DevStatus *status, int lower) {
    const int idx = blockIdx.x;
    int s = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
    while (s * (s + 1) / 2 > idx) s--;
    while ((s + 1) * (s + 2) / 2 <= idx) s++;
    const int r = idx - s * (s + 1) / 2;
    const int r0 = P.tile_start[r], r1 = P.tile_start[r + 1];
    const int c0 = P.tile_start[s], c1 = P.tile_start[s + 1];
    const int tid = threadIdx.x;
    __shared__ double red[4];

    if (r < s) {
        double w = 0.0;
        for (int i = r0 + tid; i < r1; i += 128) {   // tiles of up to 512 rows
            double sum = 0.0;
            for (int j = c0; j < c1; j++) {
                double v = T[i + (int64_t)j * ldt];
                check_entry(v, (long long)i + (long long)j * ldt, status);
                sum += fabs(v);
            }
            w = fmax(w, sum);
        }
        w = warp_max(w);
        if ((tid & 31) == 0) red[tid >> 5] = w;
        __syncthreads();
        if (tid == 0) {
            double mx = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
            tau[(int64_t)r * P.ntiles + s] = mx;
        }
        return;
    }
    // diagonal tile: validate the upper part and the first subdiagonal
    for (int j = c0; j < c1; j++)
        for (int i = r0 + tid; i < r1 && i <= j + lower; i += 128)
            check_entry(T[i + (int64_t)j * ldt], (long long)i + (long long)j * ldt, status);
    // in-tile block column norms: one warp per block
    const int lane = tid & 31, warp = tid >> 5;
    const int kb0 = P.tile_blk[s], kb1 = P.tile_blk[s + 1];
    for (int k = kb0 + warp; k < kb1; k += 4) {
        const int q = P.blk_start[k];
        const int bs = P.blk_size[k];
        double mx = 0.0;
        for (int i = r0 + lane; i < q; i += 32) {
            double a = fabs(T[i + (int64_t)q * ldt]);
            if (bs == 2) a += fabs(T[i + (int64_t)(q + 1) * ldt]);
            mx = fmax(mx, a);
        }
        mx = warp_max(mx);
        if (lane == 0) blk_tau[k] = mx;
    }
}

// Validation of the right-hand sides of the triangular solve: every entry
// of B (n x nrhs, ld ldb) finite and at most 2^1000 in magnitude; an entry
// is reported as ldt n + i + j ldb (B placed after T).
__global__ void k_check_rhs(const double *__restrict__ B, int64_t ldb, int64_t n, int64_t nrhs,
                            int64_t base, DevStatus *status) {
    const int64_t j = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        check_entry(B[i + j * ldb], (long long)(base + i + j * ldb), status);
}

void launch_check_rhs(const double *B, int64_t ldb, int64_t n, int64_t nrhs, int64_t base,
                      DevStatus *status, cudaStream_t st) {
    if (n <= 0 || nrhs <= 0) return;
    const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 64);
    for (int64_t j0 = 0; j0 < nrhs; j0 += 65535) {
        const unsigned gy = (unsigned)std::min<int64_t>(nrhs - j0, 65535);
        k_check_rhs<<<dim3(gx, gy), 256, 0, st>>>(B + j0 * ldb, ldb, n, gy,
                                                  base + j0 * ldb, status);
    }
}

void launch_tile_norms(const double *T, int64_t ldt, const Plan &p, double *tau,
                       double *blk_tau, DevStatus *status, cudaStream_t st, int lower) {
    int64_t N = p.ntiles;
    int64_t pairs = N * (N + 1) / 2;
    k_tile_norms<<<(unsigned)pairs, 128, 0, st>>>(T, ldt, p, tau, blk_tau, status, lower);
}

}  // namespace evec
