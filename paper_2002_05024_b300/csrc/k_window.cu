// k_window.cu -- the off-diagonal updates of eigenvalue reordering (Sec. 3.2:
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
// two are separate launches on one stream; the Q updates read no part of T
// and run on a second stream beside them.
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
__device__ __forceinline__ void win_left_tile(int64_t n, double *__restrict__ T, int64_t ldt,
                                              int64_t a, int k, const double *__restrict__ Z,
                                              int64_t tile) {
    extern __shared__ __align__(16) double wsm[];
    double *Ws = wsm;                 // [kWlc][k]: column c of the strip at Ws + c k
    double *Zs = wsm + kWlc * k;      // [kWzc][k + 1]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col0 = a + tile * kWlc;
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

// Right update C[0:rows, a:a+k] <- C[0:rows, a:a+k] Z (C = T with rows =
// a + k, or Q with rows = n), kWrr rows per CTA; lane = row, warp = output
// columns warp + 8 p (p < P, k <= 8 P).
template <int P>
__device__ __forceinline__ void win_right_tile(int64_t rows, double *__restrict__ C, int64_t ld,
                                               int64_t a, int k, const double *__restrict__ Z,
                                               int64_t tile) {
    extern __shared__ __align__(16) double wsm[];
    double *Ws = wsm;                 // [k][kWrr]: row l of the strip's transpose
    double *Zs = wsm + kWrr * k;      // [kWzc][k + 1]
    const int64_t r0 = tile * kWrr;
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

template <int P>
__global__ void __launch_bounds__(256)
    k_win_left(int64_t n, double *__restrict__ T, int64_t ldt, int64_t a, int k,
               const double *__restrict__ Z) {
    win_left_tile<P>(n, T, ldt, a, k, Z, blockIdx.x);
}

template <int P>
__global__ void __launch_bounds__(256)
    k_win_right(int64_t rows, double *__restrict__ C, int64_t ld, int64_t a, int k,
                const double *__restrict__ Z) {
    win_right_tile<P>(rows, C, ld, a, k, Z, blockIdx.x);
}

// A set of pairwise disjoint windows in one launch: CTA blockIdx.x works
// on window w with cta0[w] <= blockIdx.x < cta0[w + 1] (its tile index is
// the difference).  Disjoint windows' updates commute, as (Z'^T X) Z =
// Z'^T (X Z) on the block two of them share, so the left updates of the
// whole set run in one launch, then the right updates.
__device__ __forceinline__ int find_window(const WinDesc *wd, int nwin) {
    int lo = 0, hi = nwin - 1;   // the last w with cta0 <= blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (wd[mid].cta0 <= (int64_t)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int P>
__global__ void __launch_bounds__(256)
    k_win_left_set(int64_t n, double *__restrict__ T, int64_t ldt, const WinDesc *__restrict__ wd,
                   int nwin, const double *__restrict__ Z) {
    const WinDesc d = wd[find_window(wd, nwin)];
    win_left_tile<P>(n, T, ldt, d.a, d.k, Z + d.zoff, (int64_t)blockIdx.x - d.cta0);
}

// rows of window w: a + k for T (q false), n for Q
template <int P>
__global__ void __launch_bounds__(256)
    k_win_right_set(int64_t n, double *__restrict__ C, int64_t ld, bool q,
                    const WinDesc *__restrict__ wd, int nwin, const double *__restrict__ Z) {
    const WinDesc d = wd[find_window(wd, nwin)];
    win_right_tile<P>(q ? n : d.a + d.k, C, ld, d.a, d.k, Z + d.zoff,
                      (int64_t)blockIdx.x - d.cta0);
}

int window_max() { return kWinMax; }
int window_left_tiles(int64_t n, int64_t a) { return (int)((n - a + kWlc - 1) / kWlc); }
int window_right_tiles(int64_t rows) { return (int)((rows + kWrr - 1) / kWrr); }

// Kernel variant of a window of k rows: the right update's columns per
// thread P (k <= 8 P); the left update's rows per lane are (P + 3) / 4.
// A window takes the smallest variant that holds it: a thread's columns
// past k are multiplied all the same (the FP64 pipe runs them like the
// others), so a variant twice too large costs twice the time.
int window_class(int k) {
    return k <= 32 ? 4 : k <= 64 ? 8 : k <= 128 ? 16 : k <= 160 ? 20 : 32;
}

template <int P>
static void set_left_t(int64_t n, double *T, int64_t ldt, int kmax, const WinDesc *wl, int ctas,
                       int nwin, const double *Z, cudaStream_t st) {
    constexpr int PL = (P + 3) / 4;
    const size_t sl = sizeof(double) * ((size_t)kWlc * kmax + (size_t)kWzc * (kmax + 1));
    cudaFuncSetAttribute(k_win_left_set<PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl);
    k_win_left_set<PL><<<ctas, 256, sl, st>>>(n, T, ldt, wl, nwin, Z);
}

template <int P>
static void set_right_t(int64_t n, double *C, int64_t ld, bool q, int kmax, const WinDesc *wr,
                        int ctas, int nwin, const double *Z, cudaStream_t st) {
    const size_t sr = sizeof(double) * ((size_t)kWrr * kmax + (size_t)kWzc * (kmax + 1));
    cudaFuncSetAttribute(k_win_right_set<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
    k_win_right_set<P><<<ctas, 256, sr, st>>>(n, C, ld, q, wr, nwin, Z);
}

// The left updates of a set of disjoint windows of one class (wl: their
// descriptor table, cta0 counting left tiles; kmax: their largest k).
void window_set_left(int pclass, int64_t n, double *T, int64_t ldt, int kmax, const WinDesc *wl,
                     int ctas, int nwin, const double *Z, cudaStream_t st) {
    if (ctas <= 0) return;
    switch (pclass) {
    case 4: set_left_t<4>(n, T, ldt, kmax, wl, ctas, nwin, Z, st); break;
    case 8: set_left_t<8>(n, T, ldt, kmax, wl, ctas, nwin, Z, st); break;
    case 16: set_left_t<16>(n, T, ldt, kmax, wl, ctas, nwin, Z, st); break;
    case 20: set_left_t<20>(n, T, ldt, kmax, wl, ctas, nwin, Z, st); break;
    default: set_left_t<32>(n, T, ldt, kmax, wl, ctas, nwin, Z, st); break;
    }
}

// Their right updates of C = T (q false: rows a + k) or Q (q true: n rows).
void window_set_right(int pclass, int64_t n, double *C, int64_t ld, bool q, int kmax,
                      const WinDesc *wr, int ctas, int nwin, const double *Z, cudaStream_t st) {
    if (ctas <= 0) return;
    switch (pclass) {
    case 4: set_right_t<4>(n, C, ld, q, kmax, wr, ctas, nwin, Z, st); break;
    case 8: set_right_t<8>(n, C, ld, q, kmax, wr, ctas, nwin, Z, st); break;
    case 16: set_right_t<16>(n, C, ld, q, kmax, wr, ctas, nwin, Z, st); break;
    case 20: set_right_t<20>(n, C, ld, q, kmax, wr, ctas, nwin, Z, st); break;
    default: set_right_t<32>(n, C, ld, q, kmax, wr, ctas, nwin, Z, st); break;
    }
}

template <int P>
static void left_t(int64_t n, double *T, int64_t ldt, int64_t a, int k, const double *Z,
                   cudaStream_t st) {
    const size_t smem = sizeof(double) * ((size_t)kWlc * k + (size_t)kWzc * (k + 1));
    cudaFuncSetAttribute(k_win_left<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned grid = (unsigned)((n - a + kWlc - 1) / kWlc);
    k_win_left<P><<<grid, 256, smem, st>>>(n, T, ldt, a, k, Z);
}

template <int P>
static void right_t(int64_t rows, double *C, int64_t ld, int64_t a, int k, const double *Z,
                    cudaStream_t st) {
    const size_t smem = sizeof(double) * ((size_t)kWrr * k + (size_t)kWzc * (k + 1));
    cudaFuncSetAttribute(k_win_right<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned grid = (unsigned)((rows + kWrr - 1) / kWrr);
    k_win_right<P><<<grid, 256, smem, st>>>(rows, C, ld, a, k, Z);
}

static void right(int64_t rows, double *C, int64_t ld, int64_t a, int k, const double *Z,
                  cudaStream_t st) {
    if (k <= 32) right_t<4>(rows, C, ld, a, k, Z, st);
    else if (k <= 64) right_t<8>(rows, C, ld, a, k, Z, st);
    else if (k <= 128) right_t<16>(rows, C, ld, a, k, Z, st);
    else if (k <= 160) right_t<20>(rows, C, ld, a, k, Z, st);
    else right_t<32>(rows, C, ld, a, k, Z, st);
}

// One window of T (1 <= k <= kWinMax, a + k <= n): the left update, then
// the right update.  Returns the kernels launched.
int window_update_t(int64_t n, double *T, int64_t ldt, int64_t a, int k, const double *Z,
                    cudaStream_t st) {
    if (k <= 0) return 0;
    if (k <= 32) left_t<1>(n, T, ldt, a, k, Z, st);
    else if (k <= 64) left_t<2>(n, T, ldt, a, k, Z, st);
    else if (k <= 128) left_t<4>(n, T, ldt, a, k, Z, st);
    else if (k <= 160) left_t<5>(n, T, ldt, a, k, Z, st);
    else left_t<8>(n, T, ldt, a, k, Z, st);
    right(a + k, T, ldt, a, k, Z, st);
    return 2;
}

// The same window's Q[:, a:a+k] <- Q[:, a:a+k] Z.  It reads no part of T,
// so the Q updates of a list of windows can run on their own stream.
int window_update_q(int64_t n, double *Q, int64_t ldq, int64_t a, int k, const double *Z,
                    cudaStream_t st) {
    if (k <= 0) return 0;
    right(n, Q, ldq, a, k, Z, st);
    return 1;
}

}  // namespace evec
