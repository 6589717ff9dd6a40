// k_gemm.cu -- the dense contractions of the method, in FP64 on the DFMA pipe.
//
// tile update (Sec. 3.3, the single level-3 operation of Z <- Y - T X):
//   for every tile r < s and every active column j (its block in tile >= s)
//     Y_r[:, j] <- 2^dy[r, j] Y_r[:, j] - T_rs (2^dx[r, j] X_s[:, j])
//   with dy / dx from the diagonal-tile kernel (dy = fresh: Y_r[:, j] has not
//   been written yet and counts as zero), and the new column maxima
//   |Y_r[:, j]|_inf written to seg_nu for the next decisions.
// back-transformation (Eq. evec_backtransform): X = Q Y, where Y is block
//   upper triangular: column j is zero below its own diagonal block, so each
//   column block only runs K up to the end of its last column's block.
//
// On B300 the FP64 tensor path (mma.sync .f64) was measured below the plain
// DFMA rate, so both kernels are register-tiled DFMA GEMMs: a CTA of 256
// threads computes a BM x 64 tile, each thread (BM/16) x 4 outputs, with
// operands staged through double-buffered shared memory (K step 16, the next
// chunk prefetched into registers while the current one is consumed).
#include <math.h>

#include <algorithm>

#include "evec_internal.cuh"

namespace evec {

constexpr int kBN = 64;
constexpr int kBK = 16;
constexpr int kThreads = 256;
constexpr int kBPad = kBN + 1;   // B rows padded: conflict-free column-wise stores

template <int BM>
struct GemmSmem {
    double A[2][kBK][BM];
    double B[2][kBK][kBPad];
    int bexp[kBN];
};

// acc[i][jj] += sum_k A[row i][k] * B[k][col jj] over k in [0, K).
//   A(i, k) = A[i + k * lda], rows i < a_rows (rows beyond read as 0)
//   B(k, j) = B[k + j * ldb], columns j < ncols
//   scale_b: B column j is multiplied by 2^sm.bexp[j] while staged (exact)
//   zero: start from acc = 0 (else accumulate onto acc)
template <int BM>
__device__ __forceinline__ void dfma_mainloop(const double *__restrict__ A, int64_t lda, int a_rows,
                                              const double *__restrict__ B, int64_t ldb, int K,
                                              int ncols, GemmSmem<BM> &sm, bool scale_b,
                                              double (&acc)[BM / 16][4], bool zero = true) {
    constexpr int MI = BM / 16;
    constexpr int A_PER = BM * kBK / kThreads;   // A elements per thread per chunk
    constexpr int B_PER = kBK * kBN / kThreads;  // = 4
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    double ra[A_PER], rb[B_PER];

    auto load = [&](int kb) {
#pragma unroll
        for (int t = 0; t < A_PER; t++) {
            const int e = tid + kThreads * t;
            const int i = e % BM, k = e / BM;
            ra[t] = (i < a_rows && kb + k < K) ? A[i + (int64_t)(kb + k) * lda] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < B_PER; t++) {
            const int e = tid + kThreads * t;
            const int k = e % kBK, j = e / kBK;
            rb[t] = (j < ncols && kb + k < K) ? B[(kb + k) + (int64_t)j * ldb] : 0.0;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int t = 0; t < A_PER; t++) {
            const int e = tid + kThreads * t;
            sm.A[buf][e / BM][e % BM] = ra[t];
        }
#pragma unroll
        for (int t = 0; t < B_PER; t++) {
            const int e = tid + kThreads * t;
            const int k = e % kBK, j = e / kBK;
            sm.B[buf][k][j] = scale_b ? scale2(rb[t], sm.bexp[j]) : rb[t];
        }
    };

    if (zero)
#pragma unroll
        for (int i = 0; i < MI; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    if (K <= 0) return;
    load(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int kb = 0; kb < K; kb += kBK) {
        const bool more = kb + kBK < K;
        if (more) load(kb + kBK);
#pragma unroll
        for (int k = 0; k < kBK; k++) {
            double a[MI], b[4];
#pragma unroll
            for (int i = 0; i < MI; i++) a[i] = sm.A[buf][k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = sm.B[buf][k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < MI; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (more) {
            store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
}

// ---------------------------------------------------------------------------
// tile update at step s: grid (column blocks, r = 0..s-1)
// ---------------------------------------------------------------------------
// GEN (pencil beta S - alpha T): T holds S, B2 / ldb2 the second matrix, and
// the right-hand side comes from W = [beta X_s; -(alpha X_s)] (2 K x active
// columns, ld ldw) instead of Y: acc = S_rs W_top + T_rs W_bottom.
template <int BM, bool GEN>
__global__ void __launch_bounds__(kThreads)
    k_tile_update(int s, const double *__restrict__ T, int64_t ldt, Plan P,
                  double *__restrict__ Y, int64_t ldy, const int32_t *__restrict__ seg_dx,
                  const int32_t *__restrict__ seg_dy, double *__restrict__ seg_nu,
                  const double *__restrict__ B2, int64_t ldb2, const double *__restrict__ W,
                  int64_t ldw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    GemmSmem<BM> &sm = *reinterpret_cast<GemmSmem<BM> *>(smraw);
    __shared__ int sdy[kBN];
    __shared__ long long red[16][kBN + 1];
    constexpr int MI = BM / 16;

    // tiles of more than BM rows: blockIdx.z picks the BM-row chunk
    const int r = blockIdx.y;
    const int r0 = P.tile_start[r] + (int)blockIdx.z * BM;
    const int rows = min(BM, P.tile_start[r + 1] - r0);
    if (rows <= 0) return;
    const int k0 = P.tile_start[s];
    const int K = P.tile_start[s + 1] - k0;
    const int64_t m = P.m;
    const int64_t j0 = (int64_t)P.tile_col[s] + (int64_t)blockIdx.x * kBN;
    const int ncols = (int)min((int64_t)kBN, m - j0);
    if (!evec_in(P, r < s && r0 + rows <= P.n && k0 + K <= P.n && ncols > 0, 121)) return;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    if (tid < kBN) {
        int dx = 0, dy = kFresh;
        if (tid < ncols) {
            dx = seg_dx[(int64_t)r * m + j0 + tid];
            dy = seg_dy[(int64_t)r * m + j0 + tid];
        }
        sm.bexp[tid] = dx;
        sdy[tid] = dy;
    }
    __syncthreads();

    double acc[MI][4];
    if (!GEN) {
        dfma_mainloop<BM>(T + r0 + (int64_t)k0 * ldt, ldt, rows, Y + k0 + j0 * ldy, ldy, K, ncols,
                          sm, true, acc);
    } else {
        const double *w = W + (j0 - P.tile_col[s]) * ldw;
        dfma_mainloop<BM>(T + r0 + (int64_t)k0 * ldt, ldt, rows, w, ldw, K, ncols, sm, true, acc);
        __syncthreads();   // the staging buffers are reused
        dfma_mainloop<BM>(B2 + r0 + (int64_t)k0 * ldb2, ldb2, rows, w + K, ldw, K, ncols, sm, true,
                          acc, false);
    }

    // one FP64 operation per entry on the DFMA pipe: the power-of-two
    // scaling only when dy != 0 (2^0 Y is Y), the column maxima on the bit
    // patterns of |v| (the order of non-negative doubles) in integer code
    long long cmax[4] = {0, 0, 0, 0};
#pragma unroll
    for (int jj = 0; jj < 4; jj++) {
        const int jl = tx + 16 * jj;
        if (jl >= ncols) continue;
        const int dy = sdy[jl];
        double *c = Y + (j0 + jl) * ldy + r0;
#pragma unroll
        for (int i = 0; i < MI; i++) {
            const int row = ty + 16 * i;
            if (row < rows) {
                const double old = (dy == kFresh) ? 0.0 : (dy == 0 ? c[row] : scale2(c[row], dy));
                const double v = old - acc[i][jj];
                c[row] = v;
                cmax[jj] = max(cmax[jj], abs_bits(v));
            }
        }
    }
#pragma unroll
    for (int jj = 0; jj < 4; jj++) red[ty][tx + 16 * jj] = cmax[jj];
    __syncthreads();
    if (tid < ncols) {
        long long mx = 0;
#pragma unroll
        for (int t = 0; t < 16; t++) mx = max(mx, red[t][tid]);
        // the decisions zeroed seg_nu; the chunks of a tile merge their maxima
        if (gridDim.z == 1) seg_nu[(int64_t)r * m + j0 + tid] = __longlong_as_double(mx);
        else if (mx > 0)
            atomicMax((unsigned long long *)&seg_nu[(int64_t)r * m + j0 + tid],
                      (unsigned long long)mx);
    }
}

// ---------------------------------------------------------------------------
// back-transformation X = Q Y: grid (column blocks, heaviest first; row blocks)
// ---------------------------------------------------------------------------
// 1-D grid in groups of gw column blocks: within a group the row bands take
// turns with the group's column blocks fastest, so the CTAs resident at one
// time cover a few row bands x gw column blocks and share their Q rows and
// Y columns through L2; heaviest column blocks first.
template <int BM>
__global__ void __launch_bounds__(kThreads)
    k_backtransform(const double *__restrict__ Q, int64_t ldq, Plan P,
                    const double *__restrict__ Y, int64_t ldy, double *__restrict__ X,
                    int64_t ldx, int gw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    GemmSmem<BM> &sm = *reinterpret_cast<GemmSmem<BM> *>(smraw);
    constexpr int MI = BM / 16;
    const int64_t m = P.m, n = P.n;
    const int nblk_cols = (int)((m + kBN - 1) / kBN);
    const int nbands = (int)((n + BM - 1) / BM);
    const int per = gw * nbands;
    const int grp = (int)blockIdx.x / per;
    const int rem = (int)blockIdx.x - grp * per;
    const int w = min(gw, nblk_cols - grp * gw);
    const int band = rem / w;
    const int64_t cb = nblk_cols - 1 - (grp * gw + rem % w);   // heaviest blocks first
    const int64_t j0 = cb * kBN;
    const int ncols = (int)min((int64_t)kBN, m - j0);
    const int64_t i0 = (int64_t)band * BM;
    const int rows = (int)min((int64_t)BM, n - i0);
    // rows of Y beyond the last column's diagonal block are zero
    if (!evec_in(P, rows > 0 && ncols > 0, 141)) return;
    const int ul = P.col_unit[j0 + ncols - 1];
    const int kb = P.unit_blk[ul];
    const int K = P.blk_start[kb] + P.blk_size[kb];
    if (!evec_in(P, K <= n, 142)) return;

    double acc[MI][4];
    dfma_mainloop<BM>(Q + i0, ldq, rows, Y + j0 * ldy, ldy, K, ncols, sm, false, acc);

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int jj = 0; jj < 4; jj++) {
        const int jl = tx + 16 * jj;
        if (jl >= ncols) continue;
        double *c = X + (j0 + jl) * ldx + i0;
#pragma unroll
        for (int i = 0; i < MI; i++) {
            const int row = ty + 16 * i;
            if (row < rows) c[row] = acc[i][jj];
        }
    }
}

// Residual of the solved segments (the residual-correction sweep), before
// the consolidation: segment r of column j holds y_r = Y_r 2^-e_r, and the
// exponents never increase going up a column (e_r <= e_s for r < s: every
// decision takes a = min(e_r, e_s) and only scales down).  In segment r's
// own scale
//   R_r = -[(T_rr - lambda I) Y_r + sum_{s > r} T_rs (2^(e_r - e_s) Y_s)],
// every factor 2^(e_r - e_s) <= 1, so nothing overflows and no row loses
// the precision that a single exponent per column (the canonical form,
// which flushes a column with 2^1000+ of growth to zero near its block)
// would take away.  One CTA per (column block of 64, row tile r); row tile
// r is one tile, so one exponent per column; K runs from the tile's first
// row to the last column's block.  Rows at or below column j's block get
// 0.  The diagonal is left out of the product and applied as
// (t_ii - a) Y_i, the shifted entry the backsubstitution itself divides by:
// t_ii Y_i and a Y_i separately would cancel and leave u |Y_i| of rounding
// in place of u |t_ii - a| |Y_i|.  For a pair (Re, Im) of lambda = a + i w:
// ((T - lambda I) y)_re = (T - a) y_re + w y_im,
// ((T - lambda I) y)_im = (T - a) y_im - w y_re.
template <int BM>
__global__ void __launch_bounds__(kThreads)
    k_residual(const double *__restrict__ T, int64_t ldt, Plan P, const double *__restrict__ Y,
               int64_t ldy, const int32_t *__restrict__ seg_e,
               const int32_t *__restrict__ row_tile, double *__restrict__ R, int64_t ldr) {
    extern __shared__ __align__(16) unsigned char smraw[];
    GemmSmem<BM> &sm = *reinterpret_cast<GemmSmem<BM> *>(smraw);
    __shared__ int s_bend[kBN], s_er[kBN];
    constexpr int MI = BM / 16;
    constexpr int A_PER = BM * kBK / kThreads;
    constexpr int B_PER = kBK * kBN / kThreads;
    const int64_t m = P.m;
    const int64_t nblk_cols = (m + kBN - 1) / kBN;
    const int64_t j0 = (nblk_cols - 1 - blockIdx.x) * kBN;   // heaviest blocks first
    const int ncols = (int)min((int64_t)kBN, m - j0);
    const int r = blockIdx.y;
    const int i0 = P.tile_start[r];
    const int ic = (int)blockIdx.z * BM;   // this CTA's row chunk of tile r
    const int rows = min(BM, P.tile_start[r + 1] - i0 - ic);
    if (rows <= 0) return;
    const int tid = threadIdx.x;
    if (tid < kBN) {
        int be = 0, er = 0;
        if (tid < ncols) {
            const int u = P.col_unit[j0 + tid];
            const int kb = P.unit_blk[u];
            be = P.blk_start[kb] + P.blk_size[kb];
            if (r <= P.unit_tile[u]) er = seg_e[(int64_t)r * m + j0 + tid];
        }
        s_bend[tid] = be;
        s_er[tid] = er;
    }
    __syncthreads();
    const int K = s_bend[ncols - 1];   // block ends grow with the column
    double acc[MI][4];
#pragma unroll
    for (int i = 0; i < MI; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    if (i0 + ic < K) {
        const double *A = T + (i0 + ic) + (int64_t)i0 * ldt;
        const int KL = K - i0;
        double ra[A_PER], rb[B_PER];
        // A(i, k) = T(i0 + i, i0 + k) on and above the subdiagonal, diagonal
        // excluded; B(k, j) = Y(i0 + k, j0 + j) 2^(e_r - e_s(k)) above the
        // column's block end, else 0
        auto load = [&](int kb) {
#pragma unroll
            for (int t = 0; t < A_PER; t++) {
                const int e = tid + kThreads * t;
                const int i = e % BM, k = kb + e / BM;
                ra[t] = (i < rows && k < KL && k + 1 >= ic + i && k != ic + i)
                            ? A[i + (int64_t)k * ldt]
                            : 0.0;
            }
#pragma unroll
            for (int t = 0; t < B_PER; t++) {
                const int e = tid + kThreads * t;
                const int k = kb + e % kBK, j = e / kBK;
                const int gk = i0 + k;
                double v = 0.0;
                if (j < ncols && gk < s_bend[j]) {
                    v = Y[gk + (j0 + j) * ldy];
                    const int es = seg_e[(int64_t)row_tile[gk] * m + j0 + j];
                    v = scale2(v, s_er[j] - es);
                }
                rb[t] = v;
            }
        };
        auto store = [&](int buf) {
#pragma unroll
            for (int t = 0; t < A_PER; t++) {
                const int e = tid + kThreads * t;
                sm.A[buf][e / BM][e % BM] = ra[t];
            }
#pragma unroll
            for (int t = 0; t < B_PER; t++) {
                const int e = tid + kThreads * t;
                sm.B[buf][e % kBK][e / kBK] = rb[t];
            }
        };
        const int tx = tid & 15, ty = tid >> 4;
        load(0);
        store(0);
        __syncthreads();
        int buf = 0;
        for (int kb = 0; kb < KL; kb += kBK) {
            const bool more = kb + kBK < KL;
            if (more) load(kb + kBK);
#pragma unroll
            for (int k = 0; k < kBK; k++) {
                double a[MI], b[4];
#pragma unroll
                for (int i = 0; i < MI; i++) a[i] = sm.A[buf][k][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; j++) b[j] = sm.B[buf][k][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < MI; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            if (more) {
                store(buf ^ 1);
                __syncthreads();
                buf ^= 1;
            }
        }
    }
    const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int jj = 0; jj < 4; jj++) {
        const int jl = tx + 16 * jj;
        if (jl >= ncols) continue;
        const int64_t j = j0 + jl;
        const int u = P.col_unit[j];
        const int pj = P.blk_start[P.unit_blk[u]];
        const double lr = P.unit_lam[2 * u], li = P.unit_lam[2 * u + 1];
        const bool re = j == P.unit_col[u];
        const double *y = Y + j * ldy;
        const double *yp = Y + (re ? j + 1 : j - 1) * ldy;   // the pair's other column
        double *c = R + j * ldr;
#pragma unroll
        for (int i = 0; i < MI; i++) {
            const int row = ty + 16 * i;
            if (row >= rows) continue;
            const int64_t gi = i0 + ic + row;
            double v = 0.0;
            if (gi < pj) {   // same tile: Y_i is already in this scale
                v = -fma(T[gi + gi * ldt] - lr, y[gi], acc[i][jj]);
                if (li != 0.0) v = re ? fma(-li, yp[gi], v) : fma(li, yp[gi], v);
            }
            c[gi] = v;
        }
    }
}

template <int BM>
static void launch_residual_bm(const double *T, int64_t ldt, const Plan &p, int ntiles,
                               int max_tile, const double *Y, int64_t ldy, const int32_t *seg_e,
                               const int32_t *row_tile, double *R, int64_t ldr, cudaStream_t st) {
    cudaFuncSetAttribute(k_residual<BM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(GemmSmem<BM>));
    dim3 grid((unsigned)((p.m + kBN - 1) / kBN), (unsigned)ntiles,
              (unsigned)((max_tile + BM - 1) / BM));
    k_residual<BM><<<grid, kThreads, sizeof(GemmSmem<BM>), st>>>(T, ldt, p, Y, ldy, seg_e,
                                                                 row_tile, R, ldr);
}

void launch_residual(const double *T, int64_t ldt, const Plan &p, int ntiles, int max_tile,
                     const double *Y, int64_t ldy, const int32_t *seg_e,
                     const int32_t *row_tile, double *R, int64_t ldr, cudaStream_t st) {
    if (p.m <= 0 || ntiles <= 0) return;
    if (max_tile <= 64)
        launch_residual_bm<64>(T, ldt, p, ntiles, max_tile, Y, ldy, seg_e, row_tile, R, ldr, st);
    else
        launch_residual_bm<128>(T, ldt, p, ntiles, max_tile, Y, ldy, seg_e, row_tile, R, ldr,
                                st);
}

// W = [beta X_s; -(alpha X_s)] for the active columns of step s (pencils):
// column c of unit u (alpha = ar + i ai, beta) and its pair partner give
// (alpha x)_re = ar xr - ai xi, (alpha x)_im = ar xi + ai xr.
__global__ void k_pencil_rhs(int s, Plan P, const double *__restrict__ Y, int64_t ldy,
                             double *__restrict__ W, int64_t ldw) {
    const int t0 = P.tile_start[s], K = P.tile_start[s + 1] - t0;
    const int64_t c = P.tile_col[s] + blockIdx.x;
    if (c >= P.m) return;
    const int u = P.col_unit[c];
    const int cu = P.unit_col[u];
    const double ar = P.unit_lam[2 * u], ai = P.unit_lam[2 * u + 1], be = P.unit_beta[u];
    double *w = W + (c - P.tile_col[s]) * ldw;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {   // tiles of up to 512 rows
        const double x = Y[(t0 + k) + c * ldy];
        double ax;
        if (ai == 0.0) ax = ar * x;
        else if (c == cu) ax = fma(ar, x, -ai * Y[(t0 + k) + (c + 1) * ldy]);   // real part
        else ax = fma(ar, x, ai * Y[(t0 + k) + (c - 1) * ldy]);                 // imaginary part
        w[k] = be * x;
        w[K + k] = -ax;
    }
}

template <int BM>
static void set_smem_attr() {
    cudaFuncSetAttribute(k_tile_update<BM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(GemmSmem<BM>));
    cudaFuncSetAttribute(k_tile_update<BM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(GemmSmem<BM>));
    cudaFuncSetAttribute(k_backtransform<BM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(GemmSmem<BM>));
}

void launch_tile_update(int s, const double *T, int64_t ldt, const Plan &p, int max_tile,
                        const int32_t *tile_col_h, double *Y, int64_t ldy,
                        const int32_t *seg_dx, const int32_t *seg_dy, double *seg_nu,
                        cudaStream_t st) {
    if (s <= 0) return;
    const int64_t cols = p.m - tile_col_h[s];
    if (cols <= 0) return;
    dim3 grid((unsigned)((cols + kBN - 1) / kBN), (unsigned)s,
              (unsigned)(max_tile <= 64 ? 1 : (max_tile + 127) / 128));
    if (max_tile <= 64) {
        set_smem_attr<64>();
        k_tile_update<64, false><<<grid, kThreads, sizeof(GemmSmem<64>), st>>>(
            s, T, ldt, p, Y, ldy, seg_dx, seg_dy, seg_nu, nullptr, 0, nullptr, 0);
    } else {
        set_smem_attr<128>();
        k_tile_update<128, false><<<grid, kThreads, sizeof(GemmSmem<128>), st>>>(
            s, T, ldt, p, Y, ldy, seg_dx, seg_dy, seg_nu, nullptr, 0, nullptr, 0);
    }
}

// W = [beta X_s; -(alpha X_s)] of step s (ld ldw >= 2 |tile s|).
void launch_pencil_rhs(int s, const Plan &p, const int32_t *tile_col_h, const double *Y,
                       int64_t ldy, double *W, int64_t ldw, cudaStream_t st) {
    const int64_t cols = p.m - tile_col_h[s];
    if (cols <= 0) return;
    k_pencil_rhs<<<(unsigned)cols, 64, 0, st>>>(s, p, Y, ldy, W, ldw);
}

// Pencils: W = [beta X_s; -(alpha X_s)], then
// Y_r <- 2^dy Y_r - (S_rs W_top + T_rs W_bottom) 2^dx, one CTA per 64-row
// chunk of a tile (max_tile: the largest tile).  W: ldw x m doubles, ld
// ldw >= 2 |tile s|.  Returns the number of kernels launched.
int launch_tile_update_pencil(int s, const double *S, int64_t lds, const double *T2,
                              int64_t ldt2, const Plan &p, const int32_t *tile_start_h,
                              const int32_t *tile_col_h, double *Y, int64_t ldy,
                              const int32_t *seg_dx, const int32_t *seg_dy, double *seg_nu,
                              double *W, int64_t ldw, int max_tile, cudaStream_t st) {
    if (s <= 0) return 0;
    const int64_t cols = p.m - tile_col_h[s];
    if (cols <= 0) return 0;
    launch_pencil_rhs(s, p, tile_col_h, Y, ldy, W, ldw, st);
    dim3 grid((unsigned)((cols + kBN - 1) / kBN), (unsigned)s, (unsigned)((max_tile + 63) / 64));
    set_smem_attr<64>();
    k_tile_update<64, true><<<grid, kThreads, sizeof(GemmSmem<64>), st>>>(
        s, S, lds, p, Y, ldy, seg_dx, seg_dy, seg_nu, T2, ldt2, W, ldw);
    (void)tile_start_h;
    return 2;
}

void launch_backtransform(const double *Q, int64_t ldq, const Plan &p, const double *Y,
                          int64_t ldy, double *X, int64_t ldx, cudaStream_t st) {
    constexpr int BM = 128;
    set_smem_attr<BM>();
    const int ncb = (int)((p.m + kBN - 1) / kBN), nbands = (int)((p.n + BM - 1) / BM);
    // column blocks per group: about sqrt(resident CTAs x 2) (a row band of
    // Q is BM = 2 x kBN rows, a column block of Y kBN columns)
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, nsm = 148, per = 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_backtransform<BM>, kThreads,
                                                          sizeof(GemmSmem<BM>)) != cudaSuccess ||
            per < 1) {
            cudaGetLastError();
            nsm = 148;
            per = 1;
        }
        resident = nsm * per;
    }
    const int gw = std::max(1, std::min(ncb, (int)lround(sqrt(2.0 * resident))));
    k_backtransform<BM><<<(unsigned)(ncb * nbands), kThreads, sizeof(GemmSmem<BM>), st>>>(
        Q, ldq, p, Y, ldy, X, ldx, gw);
}

}  // namespace evec
