// k_batched.cu -- many independent Schur forms in one persistent launch.
//
// Each CTA (4 warps) takes the next matrix from a device work queue (an
// atomic counter over the matrices, which the host orders by decreasing
// estimated work, so the longest solves start first) and runs the whole
// tiled robust solve of Sec. 3.4 for it on its own: tile norms and input
// validation, then for s = N-1 .. 0 the diagonal-tile solves of every
// active unit (the same device code as the per-step kernel, in chunks of
// 16 real or 8 complex units) followed by the updates Y_r <- 2^dy Y_r -
// 2^dx T_rs X_s for all r < s, and finally the consolidation into canonical
// form.  CTAs never wait on one another; the queue is the only shared state.
// Matrices of this workload are small (n <= 1024), so one SM per matrix
// keeps each solve's data in L1/L2 and the device busy across the batch.
#include "diag_tile.cuh"

namespace evec {

constexpr int kBThreads = 128;

namespace {

__device__ __forceinline__ double bwarp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int bwarp_imax(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void check_entry_b(double v, long long idx, DevStatus *st) {
    if (!isfinite(v)) report(st, 3 /* EVEC_ENONFINITE */, idx);
    else if (fabs(v) > kInputMax) report(st, 1 /* EVEC_EINVAL */, idx);
}

// tau[r N + s] = |T_rs|_inf for r < s, the in-tile block column norms, and
// validation of every referenced entry (upper part, first subdiagonal of
// the diagonal tiles).  smem: kBThreads doubles.
__device__ void cta_tile_norms(const BatchItem &B, double *red, DevStatus *status) {
    const Plan &P = B.P;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = P.ntiles;
    for (int s = 0; s < N; s++) {
        const int c0 = P.tile_start[s], c1 = P.tile_start[s + 1];
        for (int r = 0; r < s; r++) {
            const int r0 = P.tile_start[r], r1 = P.tile_start[r + 1];
            double sum = 0.0;
            for (int i = r0 + tid; i < r1; i += kBThreads) {
                double rs = 0.0;
                for (int j = c0; j < c1; j++) {
                    const double v = B.T[i + (int64_t)j * B.ldt];
                    check_entry_b(v, B.t_base + i + (int64_t)j * B.ldt, status);
                    rs += fabs(v);
                }
                sum = fmax(sum, rs);
            }
            sum = bwarp_max(sum);
            if (lane == 0) red[warp] = sum;
            __syncthreads();
            if (tid == 0)
                B.tau[(int64_t)r * N + s] = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
            __syncthreads();
        }
        for (int j = c0; j < c1; j++)
            for (int i = c0 + tid; i < c1 && i <= j + 1; i += kBThreads)
                check_entry_b(B.T[i + (int64_t)j * B.ldt], B.t_base + i + (int64_t)j * B.ldt,
                              status);
        for (int k = P.tile_blk[s] + warp; k < P.tile_blk[s + 1]; k += kBThreads / 32) {
            const int q = P.blk_start[k];
            const int bs = P.blk_size[k];
            double mx = 0.0;
            for (int i = c0 + lane; i < q; i += 32) {
                double a = fabs(B.T[i + (int64_t)q * B.ldt]);
                if (bs == 2) a += fabs(B.T[i + (int64_t)(q + 1) * B.ldt]);
                mx = fmax(mx, a);
            }
            mx = bwarp_max(mx);
            if (lane == 0) B.blk_tau[k] = mx;
        }
    }
}

// Updates of step s: for every 64-column block of the active columns and
// every tile r < s, Y_r <- 2^dy Y_r - T_rs (2^dx X_s) with the new column
// maxima.  Thread (tx, ty) = (tid % 16, tid / 16) owns rows ty + 8 i
// (i < 8) and columns tx + 16 j (j < 4) of the 64 x 64 block.  X_s is
// staged scaled by 2^dx[r, j] before the product (exact): the protection
// decisions bound the product of the scaled operands, not of the unscaled
// ones, which may overflow.
// smem: Bs [64][65], As [64][64], red [8][64] doubles, sdx / sdy [64] ints.
__device__ void cta_tile_update(const BatchItem &B, int s, double *smem) {
    const Plan &P = B.P;
    const int64_t m = P.m;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double *Bs = smem;                  // [k][65]
    double *As = Bs + 64 * 65;          // [k][64]
    double *red = As + 64 * 64;         // [8][64]
    int *sdx = (int *)(red + 8 * 64);   // [64]
    int *sdy = sdx + 64;                // [64]
    const int k0 = P.tile_start[s], K = P.tile_start[s + 1] - k0;
    double *Y = B.X;
    const int64_t ldy = B.ldx;
    for (int64_t j0 = P.tile_col[s]; j0 < m; j0 += 64) {
        const int nc = (int)min((int64_t)64, m - j0);
        for (int r = 0; r < s; r++) {
            const int r0 = P.tile_start[r], rows = P.tile_start[r + 1] - r0;
            __syncthreads();   // the previous block's readers of As / Bs / sdx are done
            if (tid < 64) {
                int dx = 0, dy = kFresh;
                if (tid < nc) {
                    dx = B.seg_dx[(int64_t)r * m + j0 + tid];
                    dy = B.seg_dy[(int64_t)r * m + j0 + tid];
                }
                sdx[tid] = dx;
                sdy[tid] = dy;
            }
            for (int e = tid; e < 64 * 64; e += kBThreads) {
                const int i = e % 64, k = e / 64;
                As[k * 64 + i] = (i < rows && k < K) ? B.T[(r0 + i) + (int64_t)(k0 + k) * B.ldt] : 0.0;
            }
            __syncthreads();   // sdx is read by the staging of X_s below
            for (int e = tid; e < 64 * 64; e += kBThreads) {
                const int k = e % 64, j = e / 64;
                Bs[k * 65 + j] =
                    (k < K && j < nc) ? scale2(Y[(k0 + k) + (j0 + j) * ldy], sdx[j]) : 0.0;
            }
            __syncthreads();
            double acc[8][4];
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
            for (int k = 0; k < K; k++) {
                double a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; i++) a[i] = As[k * 64 + ty + 8 * i];
#pragma unroll
                for (int j = 0; j < 4; j++) b[j] = Bs[k * 65 + tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 8; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            double cmax[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int jl = tx + 16 * j;
                if (jl >= nc) continue;
                const int dy = sdy[jl];
                double *c = Y + (j0 + jl) * ldy + r0;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int row = ty + 8 * i;
                    if (row < rows) {
                        const double old = (dy == kFresh) ? 0.0 : scale2(c[row], dy);
                        const double v = old - acc[i][j];
                        c[row] = v;
                        cmax[j] = fmax(cmax[j], fabs(v));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) red[ty * 64 + tx + 16 * j] = cmax[j];
            __syncthreads();
            if (tid < nc) {
                double mx = 0.0;
#pragma unroll
                for (int t = 0; t < 8; t++) mx = fmax(mx, red[t * 64 + tid]);
                B.seg_nu[(int64_t)r * m + j0 + tid] = mx;
            }
        }
    }
    __syncthreads();
}

// Consolidation of one unit's column(s) into canonical form (as k_finalize,
// with the CTA's 4 warps).  smem: 4 ints.
__device__ void cta_finalize_unit(const BatchItem &B, int u, int *sbest) {
    const Plan &P = B.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kW = kBThreads / 32;
    const int64_t m = P.m, n = P.n;
    const int col = P.unit_col[u];
    const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
    const int c = P.unit_tile[u];
    const int kb = P.unit_blk[u];
    const int row_end = P.blk_start[kb] + P.blk_size[kb];
    double *yr = B.X + (int64_t)col * B.ldx;
    double *yi = B.X + (int64_t)(col + 1) * B.ldx;
    int best = INT32_MIN;
    for (int r = warp; r <= c; r += kW) {
        const int a = P.tile_start[r];
        const int b = min(P.tile_start[r + 1], row_end);
        double mx = 0.0;
        for (int i = a + lane; i < b; i += 32) {
            double v = fabs(yr[i]);
            if (cplx) v += fabs(yi[i]);
            mx = fmax(mx, v);
        }
        mx = bwarp_max(mx);
        if (mx > 0.0) best = max(best, ilog2_abs(mx) - B.seg_e[(int64_t)r * m + col]);
    }
    best = bwarp_imax(best);
    if (lane == 0) sbest[warp] = best;
    __syncthreads();
    int t = INT32_MIN;
#pragma unroll
    for (int w = 0; w < kW; w++) t = max(t, sbest[w]);
    __syncthreads();
    for (int r = warp; r <= c; r += kW) {
        const int a = P.tile_start[r];
        const int b = min(P.tile_start[r + 1], row_end);
        const int k = -B.seg_e[(int64_t)r * m + col] - t;
        for (int i = a + lane; i < b; i += 32) {
            yr[i] = scale2(yr[i], k);
            if (cplx) yi[i] = scale2(yi[i], k);
        }
    }
    for (int64_t i = row_end + threadIdx.x; i < n; i += kBThreads) {
        yr[i] = 0.0;
        if (cplx) yi[i] = 0.0;
    }
    if (threadIdx.x == 0) {
        B.scale_exp[col] = -t;
        if (cplx) B.scale_exp[col + 1] = -t;
    }
}

}  // namespace

__global__ void __launch_bounds__(kBThreads)
    k_batched(const BatchItem *__restrict__ items, int count, int *queue, DevStatus *status) {
    extern __shared__ double smem[];
    __shared__ int next;
    __shared__ int sbest[kBThreads / 32];
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(queue, 1);
        __syncthreads();
        const int k = next;
        __syncthreads();
        if (k >= count) break;
        const BatchItem B = items[k];
        const Plan &P = B.P;
        cta_tile_norms(B, smem, status);
        __syncthreads();
        for (int s = P.ntiles - 1; s >= 0; s--) {
            for (int pos = P.tile_real[s]; pos < P.nreal; pos += Lanes<false>::U * 4) {
                diag_tile<4, false>(s, pos, B.T, B.ldt, P, B.tau, B.blk_tau, B.X, B.ldx,
                                    B.seg_e, B.seg_nu, B.seg_dx, B.seg_dy, smem);
                __syncthreads();
            }
            for (int pos = P.tile_cplx[s]; pos < P.ncplx; pos += Lanes<true>::U * 4) {
                diag_tile<4, true>(s, pos, B.T, B.ldt, P, B.tau, B.blk_tau, B.X, B.ldx,
                                   B.seg_e, B.seg_nu, B.seg_dx, B.seg_dy, smem);
                __syncthreads();
            }
            if (s > 0 && P.tile_col[s] < P.m) {
                cta_tile_update(B, s, smem);
                __syncthreads();
            }
        }
        for (int u = 0; u < P.nunits; u++) cta_finalize_unit(B, u, sbest);
        __syncthreads();
    }
}

size_t batched_smem_bytes() {
    const size_t upd = sizeof(double) * (64 * 65 + 64 * 64 + 8 * 64) + sizeof(int) * 128;
    return std::max(diag_smem<4>(64), upd);
}

// One persistent launch: grid = SMs x CTAs per SM (occupancy query).
cudaError_t launch_batched(const BatchItem *items, int count, int *queue, DevStatus *status,
                           int nsm, cudaStream_t st) {
    const size_t smem = batched_smem_bytes();
    cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_batched, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched, kBThreads, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int grid = std::min(count, nsm * per_sm);
    if (grid <= 0) return cudaSuccess;
    k_batched<<<grid, kBThreads, smem, st>>>(items, count, queue, status);
    return cudaGetLastError();
}

size_t batch_item_bytes() { return sizeof(BatchItem); }

}  // namespace evec
