// k_window.cu -- the off-diagonal updates of eigenvalue reordering (Sec. 3:
// a window task gathers the local transformations of a diagonal window in
// an accumulator matrix Z; the left and right update tasks then apply it to
// the off-diagonal sections as level-3 products).  For a window of k rows
// and columns at a (b = a + k) and Zhat = diag(I_a, Z, I):
//   left:  T[a:b, a:n] <- Z^T T[a:b, a:n]   (the window's rows from its
//          first column on; left of it they are zeros of the Schur form)
//   right: T[0:b, a:b] <- T[0:b, a:b] Z     (its columns down to its last
//          row; below it they are zeros) and Q[:, a:b] <- Q[:, a:b] Z.
// Both are FP64 products with K = k.  Each CTA stages the strip it owns in
// shared memory before it writes, so the update runs in place; Z streams
// through shared memory in chunks of kWzc rows.  The left update must
// finish before the right one reads the window's diagonal block, so the
// two are separate launches on one stream.
#include <algorithm>

#include "evec_internal.cuh"

namespace evec {

constexpr int kWinMax = 256;   // largest window
constexpr int kWzc = 16;       // rows of Z per shared-memory chunk
constexpr int kWlc = 16;       // columns per CTA in the left update
constexpr int kWrr = 32;       // rows per CTA in the right update

// Z rows [l0, l0 + kWzc) into Zs[ll * (k + 1) + i] (the +1 keeps the
// column-wise stores out of one bank); rows past k are zeros.
__device__ __forceinline__ void stage_z(const double *__restrict__ Z, int k, int l0, double *Zs) {
    for (int e = threadIdx.x; e < kWzc * k; e += blockDim.x) {
        const int ll = e % kWzc, i = e / kWzc;
        Zs[ll * (k + 1) + i] = l0 + ll < k ? Z[(l0 + ll) + (int64_t)i * k] : 0.0;
    }
}

// Left update, kWlc columns per CTA (from column a + blockIdx.x kWlc); lane
// = output rows lane + 32 p (p < P, k <= 32 P), warp = columns warp + 8 q.
template <int P>
__global__ void __launch_bounds__(256)
    k_win_left(int64_t n, double *__restrict__ T, int64_t ldt, int64_t a, int k,
               const double *__restrict__ Z) {
    extern __shared__ __align__(16) double wsm[];
    double *Ws = wsm;                 // [kWlc][k]: column c of the strip at Ws + c k
    double *Zs = wsm + kWlc * k;      // [kWzc][k + 1]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col0 = a + (int64_t)blockIdx.x * kWlc;
    const int ncol = (int)min((int64_t)kWlc, n - col0);
    for (int e = threadIdx.x; e < kWlc * k; e += blockDim.x) {
        const int l = e % k, c = e / k;
        Ws[e] = c < ncol ? T[(a + l) + (col0 + c) * ldt] : 0.0;
    }
    constexpr int QN = kWlc / 8;
    double acc[P][QN];
#pragma unroll
    for (int p = 0; p < P; p++)
#pragma unroll
        for (int q = 0; q < QN; q++) acc[p][q] = 0.0;
    for (int l0 = 0; l0 < k; l0 += kWzc) {
        __syncthreads();   // the strip is staged / the previous chunk consumed
        stage_z(Z, k, l0, Zs);
        __syncthreads();
        const int lc = min(kWzc, k - l0);
        for (int ll = 0; ll < lc; ll++) {
            double w[QN], z[P];
#pragma unroll
            for (int q = 0; q < QN; q++) w[q] = Ws[(warp + 8 * q) * k + l0 + ll];
#pragma unroll
            for (int p = 0; p < P; p++) {
                const int i = lane + 32 * p;
                z[p] = i < k ? Zs[ll * (k + 1) + i] : 0.0;
            }
#pragma unroll
            for (int p = 0; p < P; p++)
#pragma unroll
                for (int q = 0; q < QN; q++) acc[p][q] = fma(z[p], w[q], acc[p][q]);
        }
    }
#pragma unroll
    for (int p = 0; p < P; p++) {
        const int i = lane + 32 * p;
#pragma unroll
        for (int q = 0; q < QN; q++) {
            const int c = warp + 8 * q;
            if (i < k && c < ncol) T[(a + i) + (col0 + c) * ldt] = acc[p][q];
        }
    }
}

// Right update, kWrr rows per CTA of T (blockIdx.y 0, rows [0, rows_t)) or
// Q (blockIdx.y 1, rows [0, rows_q)); lane = row, warp = output columns
// warp + 8 p (p < P, k <= 8 P).
template <int P>
__global__ void __launch_bounds__(256)
    k_win_right(int64_t rows_t, double *__restrict__ T, int64_t ldt, int64_t rows_q,
                double *__restrict__ Q, int64_t ldq, int64_t a, int k,
                const double *__restrict__ Z) {
    extern __shared__ __align__(16) double wsm[];
    double *Ws = wsm;                 // [k][kWrr]: row l of the strip's transpose
    double *Zs = wsm + kWrr * k;      // [kWzc][k + 1]
    double *C = blockIdx.y ? Q : T;
    const int64_t ld = blockIdx.y ? ldq : ldt, rows = blockIdx.y ? rows_q : rows_t;
    const int64_t r0 = (int64_t)blockIdx.x * kWrr;
    if (r0 >= rows) return;   // (uniform in the CTA)
    const int nr = (int)min((int64_t)kWrr, rows - r0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < kWrr * k; e += blockDim.x) {
        const int rr = e % kWrr, l = e / kWrr;
        Ws[e] = rr < nr ? C[(r0 + rr) + (a + l) * ld] : 0.0;
    }
    double acc[P];
#pragma unroll
    for (int p = 0; p < P; p++) acc[p] = 0.0;
    for (int l0 = 0; l0 < k; l0 += kWzc) {
        __syncthreads();
        stage_z(Z, k, l0, Zs);
        __syncthreads();
        const int lc = min(kWzc, k - l0);
        for (int ll = 0; ll < lc; ll++) {
            const double w = Ws[(l0 + ll) * kWrr + lane];
#pragma unroll
            for (int p = 0; p < P; p++) {
                const int i = warp + 8 * p;
                const double z = i < k ? Zs[ll * (k + 1) + i] : 0.0;
                acc[p] = fma(w, z, acc[p]);
            }
        }
    }
    if (lane < nr) {
#pragma unroll
        for (int p = 0; p < P; p++) {
            const int i = warp + 8 * p;
            if (i < k) C[(r0 + lane) + (a + i) * ld] = acc[p];
        }
    }
}

int window_max() { return kWinMax; }

template <int P>
static void left_t(int64_t n, double *T, int64_t ldt, int64_t a, int k, const double *Z,
                   cudaStream_t st) {
    const size_t smem = sizeof(double) * ((size_t)kWlc * k + (size_t)kWzc * (k + 1));
    cudaFuncSetAttribute(k_win_left<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned grid = (unsigned)((n - a + kWlc - 1) / kWlc);
    k_win_left<P><<<grid, 256, smem, st>>>(n, T, ldt, a, k, Z);
}

template <int P>
static void right_t(int64_t rows_t, double *T, int64_t ldt, int64_t rows_q, double *Q,
                    int64_t ldq, int64_t a, int k, const double *Z, cudaStream_t st) {
    const size_t smem = sizeof(double) * ((size_t)kWrr * k + (size_t)kWzc * (k + 1));
    cudaFuncSetAttribute(k_win_right<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t rows = std::max(rows_t, Q ? rows_q : 0);
    dim3 grid((unsigned)((rows + kWrr - 1) / kWrr), Q ? 2u : 1u);
    k_win_right<P><<<grid, 256, smem, st>>>(rows_t, T, ldt, rows_q, Q, ldq, a, k, Z);
}

// One window (1 <= k <= kWinMax, a + k <= n): the left update, then the
// right update of T and Q.  Returns the kernels launched.
int window_update(int64_t n, double *T, int64_t ldt, double *Q, int64_t ldq, int64_t a, int k,
                  const double *Z, cudaStream_t st) {
    if (k <= 0) return 0;
    if (k <= 32) left_t<1>(n, T, ldt, a, k, Z, st);
    else if (k <= 64) left_t<2>(n, T, ldt, a, k, Z, st);
    else if (k <= 128) left_t<4>(n, T, ldt, a, k, Z, st);
    else left_t<8>(n, T, ldt, a, k, Z, st);
    const int64_t b = a + k;
    if (k <= 32) right_t<4>(b, T, ldt, n, Q, ldq, a, k, Z, st);
    else if (k <= 64) right_t<8>(b, T, ldt, n, Q, ldq, a, k, Z, st);
    else if (k <= 128) right_t<16>(b, T, ldt, n, Q, ldq, a, k, Z, st);
    else right_t<32>(b, T, ldt, n, Q, ldq, a, k, Z, st);
    return 2;
}

}  // namespace evec
