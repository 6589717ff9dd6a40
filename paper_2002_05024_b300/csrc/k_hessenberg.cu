// k_hessenberg.cu -- Hessenberg reduction A = Q H Q^T (Sec. 3.1), blocked by
// panels of kHb columns as the paper describes:
//   1. reduce the panel: column c = k + i of the panel gets the earlier
//      reflectors of the panel from the right (x = A[:, c] - Y V^T e_c) and
//      the left (x <- (I - V T V^T)^T x), then its reflector P_c = I - tau v
//      v^T (beta = -sign(alpha) |(alpha, x)|_2, v = (1, x / (alpha - beta))
//      below row c), and Y = A V T gains the column
//      y = tau (A[:, c+1:n] v - Y (V^T v))  -- the large matrix-vector
//      product over the part of the matrix that trails the column, the
//      HBM-bound step (8 n (n - c - 1) bytes per column);
//   2. update the trailing matrix: A <- (I - V T V^T)^T (A - Y V^T);
//   3. update the top part from the right: A <- A - Y V^T (rows above the
//      panel, which the left factor does not touch).
// Q (optional) accumulates Q <- Q (I - V T V^T).  All FP64.  Reductions
// across CTAs go through per-CTA partial sums and a second pass (no FP64
// atomics), so the result does not depend on scheduling.
#include <algorithm>

#include <cuda_bf16.h>

#include "evec_internal.cuh"

namespace evec {

constexpr int kHb = 32;          // panel width
constexpr int kHRowThreads = 256;
constexpr int kHPartStride = 2 * kHb + 4;

struct HessScal {
    double tau, d, beta;
};

__device__ __forceinline__ double hwarp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// merge two (scale, sum of squares) pairs: sum_i x_i^2 = s^2 q
__device__ __forceinline__ void ssq_merge(double &s, double &q, double s2, double q2) {
    if (s2 == 0.0) return;
    if (s < s2) {
        const double r = s / s2;
        q = q2 + q * r * r;
        s = s2;
    } else {
        const double r = s2 / s;
        q += q2 * r * r;
    }
}

// Block-wide sums of nv values per thread (nv <= kHb), written to
// part[blockIdx.x * kHPartStride + off + j].  smem: 8 x kHb doubles.
__device__ void block_sums(double *vals, int nv, double *red, double *part, int off) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < nv; j++) {
        const double v = hwarp_sum(vals[j]);
        if (lane == 0) red[warp * kHb + j] = v;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int w = 0; w < kHRowThreads / 32; w++) s += red[w * kHb + threadIdx.x];
        part[(int64_t)blockIdx.x * kHPartStride + off + threadIdx.x] = s;
    }
    __syncthreads();
}

// 1. x = A[:, c] - Y[:, 0:i] V[c, 0:i]^T for every row; partial sums of
//    V[:, 0:i]^T x.
__global__ void __launch_bounds__(kHRowThreads)
    k_hs_col(int64_t n, const double *__restrict__ A, int64_t lda, int64_t c, int i,
             const double *__restrict__ Y, const double *__restrict__ V, double *__restrict__ x,
             double *__restrict__ part) {
    __shared__ double vc[kHb];
    __shared__ double red[8 * kHb];
    if (threadIdx.x < i) vc[threadIdx.x] = V[c + (int64_t)threadIdx.x * n];
    __syncthreads();
    double acc[kHb];
#pragma unroll
    for (int j = 0; j < kHb; j++) acc[j] = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double xr = A[r + c * lda];
#pragma unroll
        for (int j = 0; j < kHb; j++)
            if (j < i) xr = fma(-Y[r + (int64_t)j * n], vc[j], xr);
        x[r] = xr;
#pragma unroll
        for (int j = 0; j < kHb; j++)
            if (j < i) acc[j] = fma(V[r + (int64_t)j * n], xr, acc[j]);
    }
    block_sums(acc, i, red, part, 0);
}

// 2. w = T[0:i, 0:i]^T (sum of the partials), one CTA.
__global__ void k_hs_w(int i, int nparts, const double *__restrict__ part,
                       const double *__restrict__ T, double *__restrict__ w) {
    __shared__ double u[kHb];
    const int j = threadIdx.x;
    if (j < i) {
        double s = 0.0;
        for (int p = 0; p < nparts; p++) s += part[(int64_t)p * kHPartStride + j];
        u[j] = s;
    }
    __syncthreads();
    if (j < i) {   // (T^T u)_j = sum_{l <= j} T[l, j] u_l
        double s = 0.0;
        for (int l = 0; l <= j; l++) s = fma(T[l + j * kHb], u[l], s);
        w[j] = s;
    }
}

// 3. x <- x - V[:, 0:i] w; column c of A for rows <= c; partials of the
//    norm of x[c+2:n] (scale, sum of squares) and of V[c+2:n, 0:i]^T x.
__global__ void __launch_bounds__(kHRowThreads)
    k_hs_apply(int64_t n, double *__restrict__ A, int64_t lda, int64_t c, int i,
               const double *__restrict__ V, const double *__restrict__ w,
               double *__restrict__ x, double *__restrict__ part) {
    __shared__ double ws[kHb];
    __shared__ double red[8 * kHb];
    __shared__ double rs[8], rq[8];
    if (threadIdx.x < i) ws[threadIdx.x] = w[threadIdx.x];
    __syncthreads();
    double acc[kHb];
#pragma unroll
    for (int j = 0; j < kHb; j++) acc[j] = 0.0;
    double sc = 0.0, sq = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double xr = x[r];
#pragma unroll
        for (int j = 0; j < kHb; j++)
            if (j < i) xr = fma(-V[r + (int64_t)j * n], ws[j], xr);
        x[r] = xr;
        if (r <= c) A[r + c * lda] = xr;
        if (r >= c + 2) {
            ssq_merge(sc, sq, fabs(xr), xr != 0.0 ? 1.0 : 0.0);
#pragma unroll
            for (int j = 0; j < kHb; j++)
                if (j < i) acc[j] = fma(V[r + (int64_t)j * n], xr, acc[j]);
        }
    }
    block_sums(acc, i, red, part, 0);
    // (scale, ssq) over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, sc, o);
        const double q2 = __shfl_xor_sync(0xffffffffu, sq, o);
        ssq_merge(sc, sq, s2, q2);
    }
    if (lane == 0) { rs[warp] = sc; rq[warp] = sq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, q = 0.0;
        for (int k = 0; k < kHRowThreads / 32; k++) ssq_merge(s, q, rs[k], rq[k]);
        part[(int64_t)blockIdx.x * kHPartStride + kHb] = s;
        part[(int64_t)blockIdx.x * kHPartStride + kHb + 1] = q;
    }
}

// 4. The reflector of column c (one CTA): beta, tau, d = alpha - beta,
//    s = V[:, 0:i]^T v, the new column of T, A[c+1, c] = beta.
__global__ void k_hs_reflector(int64_t n, double *__restrict__ A, int64_t lda, int64_t c, int i,
                               int nparts, const double *__restrict__ part,
                               const double *__restrict__ x, const double *__restrict__ V,
                               double *__restrict__ T, double *__restrict__ svec,
                               HessScal *scal) {
    __shared__ double sh[kHb];
    __shared__ double s_tau, s_d;
    const int j = threadIdx.x;
    if (j == 0) {
        double s = 0.0, q = 0.0;
        for (int p = 0; p < nparts; p++)
            ssq_merge(s, q, part[(int64_t)p * kHPartStride + kHb],
                      part[(int64_t)p * kHPartStride + kHb + 1]);
        const double xn = s * sqrt(q);
        const double alpha = x[c + 1];
        double tau = 0.0, d = 1.0, beta = alpha;
        if (xn != 0.0) {
            const double m = fmax(fabs(alpha), xn);
            const double a = alpha / m, b = xn / m;
            beta = m * sqrt(a * a + b * b);
            if (alpha >= 0.0) beta = -beta;
            tau = (beta - alpha) / beta;
            d = alpha - beta;
        }
        s_tau = tau;
        s_d = d;
        scal->tau = tau;
        scal->d = d;
        scal->beta = beta;
        A[(c + 1) + c * lda] = beta;
    }
    __syncthreads();
    const double tau = s_tau, d = s_d;
    if (j < i) {   // s_j = V[c+1, j] + (V[c+2:n, j]^T x[c+2:n]) / d
        double q = 0.0;
        for (int p = 0; p < nparts; p++) q += part[(int64_t)p * kHPartStride + j];
        sh[j] = tau == 0.0 ? 0.0 : V[(c + 1) + (int64_t)j * n] + q / d;
        svec[j] = sh[j];
    }
    __syncthreads();
    if (j < i) {   // T[j, i] = -tau sum_{l >= j, l < i} T[j, l] s_l
        double t = 0.0;
        for (int l = j; l < i; l++) t = fma(T[j + l * kHb], sh[l], t);
        T[j + i * kHb] = -tau * t;
    }
    if (j == 0) T[i + i * kHb] = tau;
}

// 5. v (column i of V): 0 above row c + 1, 1 at c + 1, x / d below; zeros
//    below the subdiagonal of column c of A.
__global__ void __launch_bounds__(kHRowThreads)
    k_hs_v(int64_t n, double *__restrict__ A, int64_t lda, int64_t c, int i,
           const double *__restrict__ x, double *__restrict__ V, const HessScal *scal) {
    const double tau = scal->tau, d = scal->d;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (r == c + 1) v = 1.0;
        else if (r > c + 1 && tau != 0.0) v = x[r] / d;
        V[r + (int64_t)i * n] = v;
        if (r > c + 1) A[r + c * lda] = 0.0;
    }
}

// 6. Y[:, i] = tau (A[:, c+1:n] v - Y[:, 0:i] s): 32 rows per CTA (lane =
//    row), its 16 warps split the columns; every warp load is 256
//    contiguous bytes of one column.
constexpr int kGvWarps = 16;
__global__ void __launch_bounds__(32 * kGvWarps)
    k_hs_gemv(int64_t n, const double *__restrict__ A, int64_t lda, int64_t c, int i,
              const double *__restrict__ V, const double *__restrict__ svec,
              double *__restrict__ Y, const HessScal *scal) {
    __shared__ double red[kGvWarps][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 32 + lane;
    const bool rv = r < n;
    const double *v = V + (int64_t)i * n;
    double acc = 0.0, acc2 = 0.0;
    int64_t j = c + 1 + warp;
    for (; j + kGvWarps < n; j += 2 * kGvWarps) {
        const double a0 = rv ? A[r + j * lda] : 0.0;
        const double a1 = rv ? A[r + (j + kGvWarps) * lda] : 0.0;
        acc = fma(a0, v[j], acc);
        acc2 = fma(a1, v[j + kGvWarps], acc2);
    }
    if (j < n && rv) acc = fma(A[r + j * lda], v[j], acc);
    red[warp][lane] = acc + acc2;
    __syncthreads();
    if (warp == 0 && rv) {
        double y = 0.0;
        for (int w = 0; w < kGvWarps; w++) y += red[w][lane];
        for (int l = 0; l < i; l++) y = fma(-Y[r + (int64_t)l * n], svec[l], y);
        Y[r + (int64_t)i * n] = scal->tau * y;
    }
}

// ---------------------------------------------------------------------------
// The panel as one cooperative launch (the paper's monolithic "reduce the
// panel" task): every CTA runs every column's phases, separated by a grid
// barrier; the small reductions are repeated in every CTA instead of taking
// another barrier.  The barrier waits are bounded: on expiry the kernel
// sets *err and every CTA returns.
// ---------------------------------------------------------------------------
constexpr long kGridWaitLimit = 1L << 22;

struct GridBar {
    unsigned count, gen;
};

// Sense-reversing grid barrier over gridDim.x co-resident CTAs; a CTA
// waits at most `limit` polls (about 64 ns each).  Returns false (and sets
// *err) when the wait gave up.  A CTA that gave up returns from the
// kernel, so the others give up at their next barrier: every CTA ends
// within a few limits.
__device__ bool grid_barrier(GridBar *bar, int *err, long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &bar->gen;
        const unsigned my_gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x) {
            bar->count = 0;
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            long it = 0;
            while (*vgen == my_gen) {
                if (++it > limit) {
                    ok = 0;
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// scalars of the column every CTA derives from the partials
struct ColScal {
    double tau, d;
    double w[kHb], s[kHb];
};

// Block sums of the kHb values every thread holds in registers (zero
// where unused), written to out[0 .. kHb): a reduce-scatter butterfly in
// each warp (31 shuffles and 31 FP64 additions per lane instead of 5 per
// value; lane j ends with the warp's sum of value j), then the warps' sums
// in shared memory.  A warp that held no rows (active false) skips the
// butterfly: it would share an FP64 pipe with a warp that did.  red: 8 x
// kHb doubles.
__device__ __forceinline__ void block_sums_rs(double (&v)[kHb], bool active, double *red,
                                              double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (active) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const bool hi = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < o; k++) {
                const double keep = hi ? v[o + k] : v[k];
                const double send = hi ? v[k] : v[o + k];
                v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
    red[warp * kHb + lane] = active ? v[0] : 0.0;
    __syncthreads();
    if (threadIdx.x < kHb) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kHRowThreads / 32; w++) t += red[w * kHb + threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// Sum over nparts rows of the partials (value j = 0 .. kHb-1 at column
// off + j) by all threads of the CTA: thread (group g, value j) sums rows
// g, g + 8, ..., then the groups in shared memory.  red: 8 x kHb doubles.
__device__ __forceinline__ void sum_partials(const double *part, int nparts, int off, double *red,
                                             double *out) {
    const int j = threadIdx.x & 31, g = threadIdx.x >> 5;
    double t = 0.0;
    for (int p = g; p < nparts; p += kHRowThreads / 32) t += part[(int64_t)p * kHPartStride + off + j];
    red[g * kHb + j] = t;
    __syncthreads();
    if (threadIdx.x < kHb) {
        double u = 0.0;
#pragma unroll
        for (int w = 0; w < kHRowThreads / 32; w++) u += red[w * kHb + threadIdx.x];
        out[threadIdx.x] = u;
    }
    __syncthreads();
}

// Column norm thresholds on the high word of |x| (sign cleared): while the
// largest entry lies in [2^-480, 2^480) the plain sum of squares neither
// overflows nor drops a term that matters (a term below 2^-537 is under
// 2^-114 of the largest square), so the reflector takes sqrt(alpha^2 +
// sum x^2) directly; outside that range every CTA recomputes the norm with
// a running scale.  The plain form keeps divisions off the column's
// critical path: on this part a dependent FP64 operation costs a whole
// pipe pass (64 cycles), a division about ten.
constexpr unsigned kNrmLo = (1023u - 480u) << 20, kNrmHi = (1023u + 480u) << 20;

__device__ __forceinline__ unsigned abs_hi(double v) {
    return (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
}

__global__ void __launch_bounds__(kHRowThreads)
    k_hs_panel(int64_t n, double *__restrict__ A, int64_t lda, int64_t k, int b,
               double *__restrict__ V, double *__restrict__ Y, double *__restrict__ T,
               double *__restrict__ x, double *__restrict__ part, double *__restrict__ part2,
               GridBar *bar, int *err, long wait_limit) {
    // part: the partials of phase 1 (read in phase 2), part2: those of
    // phase 3 (read in phase 4) -- a CTA done with phase 2 must not
    // overwrite the partials other CTAs are still reading
    __shared__ ColScal cs;
    __shared__ double red[8 * kHb];
    __shared__ double rs[8], rq[8];
    __shared__ unsigned rmh[8];
    __shared__ double gv[8][33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // rows of the row phases: a contiguous block of rpc rows per CTA
    // (ceil(n / grid) rounded up to 32), so that all SMs share the FP64
    // work; the reductions read the partials of the row-owning CTAs
    const int64_t rpc = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
    const int64_t rbeg = (int64_t)blockIdx.x * rpc, rend = min(rbeg + rpc, n);
    const int nparts = (int)min((int64_t)gridDim.x, (n + rpc - 1) / rpc);
    const bool warp_rows = rbeg + 32 * warp < rend;   // this warp holds rows
    // T and the subdiagonal entry are written by the last CTA, which owns
    // no rows whenever the grid outnumbers the row blocks: its serial
    // chain then runs while the row owners form v
    const bool scalar_cta = blockIdx.x == gridDim.x - 1;
    for (int i = 0; i < b; i++) {
        const int64_t c = k + i;
        // 1. x = A[:, c] - Y V[c, :]^T; partials of V^T x.  The sums run
        //    as four interleaved chains (a chain link is a pipe pass).
        {
            if (tid < i) cs.s[tid] = V[c + (int64_t)tid * n];   // V[c, j], reused below
            __syncthreads();
            double acc[kHb];
#pragma unroll
            for (int j = 0; j < kHb; j++) acc[j] = 0.0;
            for (int64_t r = rbeg + tid; r < rend; r += blockDim.x) {
                double x4[4] = {A[r + c * lda], 0.0, 0.0, 0.0};
#pragma unroll
                for (int j = 0; j < kHb; j++)
                    if (j < i) x4[j & 3] = fma(-Y[r + (int64_t)j * n], cs.s[j], x4[j & 3]);
                const double xr = (x4[0] + x4[1]) + (x4[2] + x4[3]);
                x[r] = xr;
#pragma unroll
                for (int j = 0; j < kHb; j++)
                    if (j < i) acc[j] = fma(V[r + (int64_t)j * n], xr, acc[j]);
            }
            if ((int64_t)blockIdx.x < nparts)
                block_sums_rs(acc, warp_rows, red, part + (int64_t)blockIdx.x * kHPartStride);
        }
        if (!grid_barrier(bar, err, wait_limit)) return;
        // 2. w = T^T (sum of partials), in every CTA
        sum_partials(part, nparts, 0, red, cs.s);
        if (tid < i) {
            double w4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int l = 0; l < kHb; l++)
                if (l <= tid) w4[l & 3] = fma(T[l + tid * kHb], cs.s[l], w4[l & 3]);
            cs.w[tid] = (w4[0] + w4[1]) + (w4[2] + w4[3]);
        }
        __syncthreads();
        // 3. x -= V w; column c rows <= c; below row c + 1: the V^T x
        //    partials, the sum of squares (value kHb - 1, which no V column
        //    uses as i < kHb) and the largest high word of |x|
        {
            double acc[kHb];
#pragma unroll
            for (int j = 0; j < kHb; j++) acc[j] = 0.0;
            unsigned mh = 0;
            for (int64_t r = rbeg + tid; r < rend; r += blockDim.x) {
                double x4[4] = {x[r], 0.0, 0.0, 0.0};
#pragma unroll
                for (int j = 0; j < kHb; j++)
                    if (j < i) x4[j & 3] = fma(-V[r + (int64_t)j * n], cs.w[j], x4[j & 3]);
                const double xr = (x4[0] + x4[1]) + (x4[2] + x4[3]);
                x[r] = xr;
                if (r <= c) A[r + c * lda] = xr;
                if (r >= c + 2) {
                    acc[kHb - 1] = fma(xr, xr, acc[kHb - 1]);
                    mh = max(mh, abs_hi(xr));
#pragma unroll
                    for (int j = 0; j < kHb; j++)
                        if (j < i) acc[j] = fma(V[r + (int64_t)j * n], xr, acc[j]);
                }
            }
            mh = __reduce_max_sync(0xffffffffu, mh);
            if (lane == 0) rmh[warp] = mh;
            if ((int64_t)blockIdx.x < nparts) {
                // (its barriers make rmh visible)
                block_sums_rs(acc, warp_rows, red, part2 + (int64_t)blockIdx.x * kHPartStride);
                if (tid == 0) {
                    unsigned m = 0;
                    for (int w8 = 0; w8 < kHRowThreads / 32; w8++) m = max(m, rmh[w8]);
                    reinterpret_cast<unsigned long long *>(
                        part2)[(int64_t)blockIdx.x * kHPartStride + kHb] = m;
                }
            }
        }
        if (!grid_barrier(bar, err, wait_limit)) return;
        // 4. the reflector, in every CTA; the partials of V^T x below row
        //    c + 1 (and the sum of squares) into cs.w (w is done with)
        sum_partials(part2, nparts, 0, red, cs.w);
        if (warp == 0) {
            unsigned m = 0;
            for (int p = lane; p < nparts; p += 32)
                m = max(m, (unsigned)reinterpret_cast<const unsigned long long *>(
                               part2)[(int64_t)p * kHPartStride + kHb]);
            m = __reduce_max_sync(0xffffffffu, m);
            if (lane == 0) rmh[0] = m;
        }
        __syncthreads();
        const double alpha = x[c + 1];
        const bool plain = rmh[0] >= kNrmLo && rmh[0] < kNrmHi && abs_hi(alpha) < kNrmHi;
        if (!plain) {   // (uniform) scaled sum of squares of x[c+2 : n], alike in every CTA
            double sc = 0.0, sq = 0.0;
            for (int64_t r = c + 2 + tid; r < n; r += blockDim.x) {
                const double xr = x[r];
                ssq_merge(sc, sq, fabs(xr), xr != 0.0 ? 1.0 : 0.0);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double s2 = __shfl_xor_sync(0xffffffffu, sc, o);
                const double q2 = __shfl_xor_sync(0xffffffffu, sq, o);
                ssq_merge(sc, sq, s2, q2);
            }
            if (lane == 0) { rs[warp] = sc; rq[warp] = sq; }
            __syncthreads();
        }
        if (tid == 0) {
            double tau = 0.0, d = 1.0, beta = alpha;
            if (plain) {   // the sum of squares is positive here
                beta = sqrt(fma(alpha, alpha, cs.w[kHb - 1]));
                if (alpha >= 0.0) beta = -beta;
                tau = (beta - alpha) / beta;
                d = alpha - beta;
            } else {
                double s0 = 0.0, q0 = 0.0;
                for (int w8 = 0; w8 < kHRowThreads / 32; w8++) ssq_merge(s0, q0, rs[w8], rq[w8]);
                const double xn = s0 * sqrt(q0);
                if (xn != 0.0) {
                    const double mx = fmax(fabs(alpha), xn);
                    const double a = alpha / mx, bb = xn / mx;
                    beta = mx * sqrt(a * a + bb * bb);
                    if (alpha >= 0.0) beta = -beta;
                    tau = (beta - alpha) / beta;
                    d = alpha - beta;
                }
            }
            cs.tau = tau;
            cs.d = d;
            if (scalar_cta) A[(c + 1) + c * lda] = beta;
        }
        __syncthreads();
        if (tid < i)
            cs.s[tid] = cs.tau == 0.0 ? 0.0 : V[(c + 1) + (int64_t)tid * n] + cs.w[tid] / cs.d;
        __syncthreads();
        if (scalar_cta) {
            if (tid < i) {
                double t4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
                for (int l = 0; l < kHb; l++)
                    if (l >= tid && l < i) t4[l & 3] = fma(T[tid + l * kHb], cs.s[l], t4[l & 3]);
                T[tid + i * kHb] = -cs.tau * ((t4[0] + t4[1]) + (t4[2] + t4[3]));
            }
            if (tid == 0) T[i + i * kHb] = cs.tau;
        }
        // 5. v and the zeros below the subdiagonal of column c
        for (int64_t r = rbeg + tid; r < rend; r += blockDim.x) {
            double v = 0.0;
            if (r == c + 1) v = 1.0;
            else if (r > c + 1 && cs.tau != 0.0) v = x[r] / cs.d;
            V[r + (int64_t)i * n] = v;
            if (r > c + 1) A[r + c * lda] = 0.0;
        }
        if (!grid_barrier(bar, err, wait_limit)) return;
        // 6. Y[:, i] = tau (A[:, c+1:n] v - Y s) for the CTA's own rows, in
        //    32-row chunks; the CTA's 8 warps split the columns.  No grid
        //    barrier follows: until the next column's first barrier a CTA
        //    touches only its own rows of A, x, Y and V (and reads V's row
        //    c + 1, final since the last barrier), while the product of a
        //    slower CTA reads only that CTA's rows and column i of V.
        {
            const double *v = V + (int64_t)i * n;
            for (int64_t r0 = rbeg; r0 < rend; r0 += 32) {
                const int64_t r = r0 + lane;
                const bool rv = r < rend;
                // warp w takes columns c+1+w, +8, ...: sixteen loads in
                // flight per lane (independent accumulators; 32 measured
                // the same, and a double-buffered batch was slower)
                constexpr int kU = 16;
                double as[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) as[u] = 0.0;
                int64_t j = c + 1 + warp;
                for (; j + 8 * (kU - 1) < n; j += 8 * kU) {
                    double a[kU];
#pragma unroll
                    for (int u = 0; u < kU; u++) a[u] = rv ? A[r + (j + 8 * u) * lda] : 0.0;
#pragma unroll
                    for (int u = 0; u < kU; u++) as[u] = fma(a[u], v[j + 8 * u], as[u]);
                }
                for (; j < n; j += 8)
                    if (rv) as[0] = fma(A[r + j * lda], v[j], as[0]);
#pragma unroll
                for (int h = kU / 2; h > 0; h >>= 1)
#pragma unroll
                    for (int u = 0; u < h; u++) as[u] += as[u + h];
                gv[warp][lane] = as[0];
                __syncthreads();
                if (warp == 0 && rv) {
                    double y4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
                    for (int w8 = 0; w8 < 8; w8++) y4[w8 & 3] += gv[w8][lane];
#pragma unroll
                    for (int l = 0; l < kHb; l++)
                        if (l < i) y4[l & 3] = fma(-Y[r + (int64_t)l * n], cs.s[l], y4[l & 3]);
                    Y[r + (int64_t)i * n] = cs.tau * ((y4[0] + y4[1]) + (y4[2] + y4[3]));
                }
                __syncthreads();
            }
        }
    }
}

// C = alpha op(A) op(B) + beta C (beta 0: C is not read); op(A) M x K,
// op(B) K x N.  Tiles of GM x GN outputs, RM x 4 per thread (256 threads):
// 128 x 64 (RM 8) for the rank-32 updates; 256 x 32 (RM 8) for the long
// products with the panel's 32 columns, which a 64-wide tile would run at
// half its multiply-adds; 32 x 32 (RM 1) for the small ones with K = 32,
// which need the CTAs more than the reuse.  16-deep K chunks
// double-buffered through registers; the shared rows are padded so that
// the transposed operand stores do not collide in a bank.
constexpr int kGK = 16;
template <int GN, int RM>
struct HsTile {
    static constexpr int TX = GN / 4, TY = 256 / TX, GM = RM * TY;
};
template <int GN, int RM>
struct HsGemmSmem {
    double A[2][kGK][HsTile<GN, RM>::GM + 1];
    double B[2][kGK][GN + 1];
};
template <int GN, int RM, bool TA, bool TB>
__device__ __forceinline__ void k_hs_gemm_body(int M, int N, int K, double alpha,
                                               const double *__restrict__ A, int64_t lda,
                                               const double *__restrict__ B, int64_t ldb,
                                               double beta, double *__restrict__ C, int64_t ldc) {
    using Tile = HsTile<GN, RM>;
    constexpr int TX = Tile::TX, TY = Tile::TY, GM = Tile::GM;
    extern __shared__ __align__(16) unsigned char hs_smraw[];
    HsGemmSmem<GN, RM> &sm = *reinterpret_cast<HsGemmSmem<GN, RM> *>(hs_smraw);
    auto &As = sm.A;
    auto &Bs = sm.B;
    constexpr int A_PER = GM * kGK / 256, B_PER = kGK * GN / 256;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
    double ra[A_PER], rb[B_PER];
    auto load = [&](int k0) {
#pragma unroll
        for (int t = 0; t < A_PER; t++) {
            const int e = tid + 256 * t;
            const int mm = TA ? e / kGK : e % GM, kk = TA ? e % kGK : e / GM;
            const int gm = m0 + mm, gk = k0 + kk;
            ra[t] = (gm < M && gk < K) ? (TA ? A[gk + (int64_t)gm * lda] : A[gm + (int64_t)gk * lda])
                                       : 0.0;
        }
#pragma unroll
        for (int t = 0; t < B_PER; t++) {
            const int e = tid + 256 * t;
            const int nn = TB ? e % GN : e / kGK, kk = TB ? e / GN : e % kGK;
            const int gn = n0 + nn, gk = k0 + kk;
            rb[t] = (gn < N && gk < K) ? (TB ? B[gn + (int64_t)gk * ldb] : B[gk + (int64_t)gn * ldb])
                                       : 0.0;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int t = 0; t < A_PER; t++) {
            const int e = tid + 256 * t;
            const int mm = TA ? e / kGK : e % GM, kk = TA ? e % kGK : e / GM;
            As[buf][kk][mm] = ra[t];
        }
#pragma unroll
        for (int t = 0; t < B_PER; t++) {
            const int e = tid + 256 * t;
            const int nn = TB ? e % GN : e / kGK, kk = TB ? e / GN : e % kGK;
            Bs[buf][kk][nn] = rb[t];
        }
    };
    double acc[RM][4];
#pragma unroll
    for (int a = 0; a < RM; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
    if (K > 0) {
        load(0);
        store(0);
        __syncthreads();
        int buf = 0;
        for (int k0 = 0; k0 < K; k0 += kGK) {
            const bool more = k0 + kGK < K;
            if (more) load(k0 + kGK);
#pragma unroll
            for (int kk = 0; kk < kGK; kk++) {
                double a[RM], b[4];
#pragma unroll
                for (int p = 0; p < RM; p++) a[p] = As[buf][kk][ty + TY * p];
#pragma unroll
                for (int q = 0; q < 4; q++) b[q] = Bs[buf][kk][tx + TX * q];
#pragma unroll
                for (int p = 0; p < RM; p++)
#pragma unroll
                    for (int q = 0; q < 4; q++) acc[p][q] = fma(a[p], b[q], acc[p][q]);
            }
            if (more) {
                store(buf ^ 1);
                __syncthreads();
                buf ^= 1;
            }
        }
    }
#pragma unroll
    for (int p = 0; p < RM; p++) {
        const int gm = m0 + ty + TY * p;
        if (gm >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int gn = n0 + tx + TX * q;
            if (gn >= N) continue;
            double *cp = C + gm + (int64_t)gn * ldc;
            *cp = beta == 0.0 ? alpha * acc[p][q] : fma(alpha, acc[p][q], beta * *cp);
        }
    }
}

template <int GN, int RM, bool TA, bool TB>
__global__ void __launch_bounds__(256)
    k_hs_gemm(int M, int N, int K, double alpha, const double *__restrict__ A, int64_t lda,
              const double *__restrict__ B, int64_t ldb, double beta, double *__restrict__ C,
              int64_t ldc) {
    k_hs_gemm_body<GN, RM, TA, TB>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// Split-K: the K range is cut into gridDim.z slices, each CTA writes its
// partial tile to P[z] (M x N, ld M); k_hs_sum adds them (fixed order).
template <int GN, bool TA, bool TB>
__global__ void __launch_bounds__(256)
    k_hs_gemm_part(int M, int N, int K, int kc, const double *__restrict__ A, int64_t lda,
                   const double *__restrict__ B, int64_t ldb, double *__restrict__ P) {
    const int k0 = blockIdx.z * kc;
    const int kl = min(kc, K - k0);
    k_hs_gemm_body<GN, 8, TA, TB>(M, N, kl, 1.0, TA ? A + k0 : A + (int64_t)k0 * lda, lda,
                               TB ? B + (int64_t)k0 * ldb : B + k0, ldb, 0.0,
                               P + (int64_t)blockIdx.z * M * N, M);
}

__global__ void k_hs_sum(int M, int N, int splits, const double *__restrict__ P, double alpha,
                         double beta, double *__restrict__ C, int64_t ldc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    const int64_t m = e % M, nn = e / M;
    double acc = 0.0;
    for (int z = 0; z < splits; z++) acc += P[(int64_t)z * M * N + e];
    double *cp = C + m + nn * ldc;
    *cp = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *cp);
}

template <int GN, int RM, bool TA, bool TB>
static void gemm_t(int M, int N, int K, double alpha, const double *A, int64_t lda,
                   const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                   cudaStream_t st) {
    constexpr int GM = HsTile<GN, RM>::GM;
    const int smem = (int)sizeof(HsGemmSmem<GN, RM>);
    cudaFuncSetAttribute(k_hs_gemm<GN, RM, TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    dim3 grid((unsigned)((M + GM - 1) / GM), (unsigned)((N + GN - 1) / GN));
    k_hs_gemm<GN, RM, TA, TB><<<grid, 256, smem, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C,
                                                      ldc);
}

// C = alpha op(A) op(B) + beta C with the K range split over gridDim.z
// when the M x N tiles alone would leave most SMs idle (the skinny products
// A^T V and Q V, N = 32): as many slices as fill both CTA slots of every
// SM (2 x 148), within the partial workspace P of p_cap doubles.
template <bool TA, bool TB>
static void gemm_splitk(int M, int N, int K, double alpha, const double *A, int64_t lda,
                        const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                        double *P, int64_t p_cap, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    constexpr int GN = 32, GM = HsTile<GN, 8>::GM;
    const int tiles = ((M + GM - 1) / GM) * ((N + GN - 1) / GN);
    const int max_splits = (int)std::min<int64_t>(1024, p_cap / ((int64_t)M * N));
    int splits = std::max(1, std::min(max_splits, 296 / std::max(tiles, 1)));
    const int kc = ((K + splits - 1) / splits + kGK - 1) / kGK * kGK;
    splits = std::max(1, (K + kc - 1) / std::max(kc, 1));
    const int smem = (int)sizeof(HsGemmSmem<GN, 8>);
    cudaFuncSetAttribute(k_hs_gemm_part<GN, TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    dim3 grid((unsigned)((M + GM - 1) / GM), (unsigned)((N + GN - 1) / GN), (unsigned)splits);
    k_hs_gemm_part<GN, TA, TB><<<grid, 256, smem, st>>>(M, N, K, kc, A, lda, B, ldb, P);
    const int64_t tot = (int64_t)M * N;
    k_hs_sum<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, splits, P, alpha, beta, C, ldc);
}

template <int GN, int RM>
static void gemm_n(bool ta, bool tb, int M, int N, int K, double alpha, const double *A,
                   int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                   cudaStream_t st) {
    if (ta && tb) gemm_t<GN, RM, true, true>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    else if (ta) gemm_t<GN, RM, true, false>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    else if (tb) gemm_t<GN, RM, false, true>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    else gemm_t<GN, RM, false, false>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
}

static void gemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A,
                 int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                 cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    if (N <= 32 && K <= 2 * kHb) gemm_n<32, 1>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    else if (N <= 32) gemm_n<32, 8>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    else gemm_n<64, 8>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
}

__global__ void k_hs_eye(int64_t n, double *Q, int64_t ldq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) Q[i + i * ldq] = 1.0;
}

int hess_panel_width() { return kHb; }

static int hess_parts(int64_t n) {
    return (int)std::max<int64_t>(
        std::min<int64_t>((n + kHRowThreads - 1) / kHRowThreads, 128), 1);
}

constexpr int kHMaxCoop = 1024;   // partials rows reserved for the cooperative panel
constexpr int kHSplits = 20;      // partial slices of n x kHb in each split-K workspace

// workspace doubles for order n: V, Y, VT, W, VTq (n x kHb each), Z (kHb x
// n), T (kHb x kHb), x (n), w and s (kHb each), the per-CTA partials,
// scalars, and the split-K partials of the A and the Q products
size_t hessenberg_workspace(int64_t n) {
    return (size_t)(6 * n * kHb + kHb * kHb + n + 2 * kHb +
                    2 * (int64_t)std::max(hess_parts(n), kHMaxCoop) * kHPartStride + 8 + 2 +
                    2 * (int64_t)kHSplits * n * kHb);
}

struct HessWs {
    double *V, *Y, *VT, *W, *VTq, *Z, *T, *x, *wv, *sv, *part, *part2, *P, *Pq;
    HessScal *scal;
    GridBar *bar;
};

static HessWs hess_ws(int64_t n, double *ws) {
    HessWs w;
    w.V = ws;
    w.Y = w.V + n * kHb;
    w.VT = w.Y + n * kHb;
    w.W = w.VT + n * kHb;
    w.VTq = w.W + n * kHb;
    w.Z = w.VTq + n * kHb;
    w.T = w.Z + kHb * n;
    w.x = w.T + kHb * kHb;
    w.wv = w.x + n;
    w.sv = w.wv + kHb;
    w.part = w.sv + kHb;
    w.part2 = w.part + (int64_t)std::max(hess_parts(n), kHMaxCoop) * kHPartStride;
    w.scal = (HessScal *)(w.part2 + (int64_t)std::max(hess_parts(n), kHMaxCoop) * kHPartStride);
    w.bar = (GridBar *)(w.scal + 2);
    w.P = (double *)(w.scal) + 10;
    w.Pq = w.P + (int64_t)kHSplits * n * kHb;
    return w;
}

// Q = I
void hess_init_q(int64_t n, double *Q, int64_t ldq, cudaStream_t st) {
    cudaMemset2DAsync(Q, ldq * sizeof(double), 0, n * sizeof(double), n, st);
    k_hs_eye<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, Q, ldq);
}

// Step 1 for the panel of b columns at k: one cooperative launch when the
// device grants it (co-resident CTAs, bounded grid barriers), else six
// launches per column.  Returns the kernels launched.
int hess_panel(int64_t n, double *A, int64_t lda, int64_t k, int b, double *ws, int *err,
               int nsm, bool cooperative, cudaStream_t st, long wait_limit) {
    if (wait_limit <= 0) wait_limit = kGridWaitLimit;
    const HessWs w = hess_ws(n, ws);
    const int parts = hess_parts(n);
    cudaMemsetAsync(w.T, 0, sizeof(double) * kHb * kHb, st);
    {
        static int per_sm = -1;
        if (per_sm < 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hs_panel, kHRowThreads,
                                                              0) != cudaSuccess)
                per_sm = 0;
            cudaGetLastError();
        }
        const int grid = cooperative ? std::min(std::min(per_sm, 2) * nsm, kHMaxCoop) : 0;
        if (grid > 0) {
            cudaMemsetAsync(w.bar, 0, sizeof(GridBar), st);
            int64_t nn = n, kk = k;
            int bb = b;
            double *V = w.V, *Y = w.Y, *T = w.T, *x = w.x, *pa = w.part, *pb = w.part2;
            GridBar *bar = w.bar;
            long wl = wait_limit;
            void *args[] = {&nn, &A, &lda, &kk, &bb, &V, &Y, &T, &x, &pa, &pb, &bar, &err, &wl};
            if (cudaLaunchCooperativeKernel((const void *)k_hs_panel, dim3(grid),
                                            dim3(kHRowThreads), args, 0, st) == cudaSuccess)
                return 1;
            cudaGetLastError();   // not granted: the launch-per-step path below
        }
    }
    for (int i = 0; i < b; i++) {
        const int64_t c = k + i;
        k_hs_col<<<parts, kHRowThreads, 0, st>>>(n, A, lda, c, i, w.Y, w.V, w.x, w.part);
        k_hs_w<<<1, 32, 0, st>>>(i, parts, w.part, w.T, w.wv);
        k_hs_apply<<<parts, kHRowThreads, 0, st>>>(n, A, lda, c, i, w.V, w.wv, w.x, w.part);
        k_hs_reflector<<<1, 32, 0, st>>>(n, A, lda, c, i, parts, w.part, w.x, w.V, w.T, w.sv,
                                         w.scal);
        k_hs_v<<<parts, kHRowThreads, 0, st>>>(n, A, lda, c, i, w.x, w.V, w.scal);
        k_hs_gemv<<<(unsigned)((n + 31) / 32), 32 * kGvWarps, 0, st>>>(n, A, lda, c, i, w.V,
                                                                     w.sv, w.Y, w.scal);
    }
    return 6 * b;
}

// Steps 2 and 3 for the panel at k (b columns), and Q <- Q (I - V T V^T):
// returns the kernels launched.  With a second stream qst (and two events)
// the Q chain runs there beside the A chain -- they share only V and T,
// which the panel wrote before the fork -- so that each fills the other's
// last partial wave; st waits for it before returning.
int hess_update(int64_t n, double *A, int64_t lda, double *Q, int64_t ldq, int64_t k, int b,
                double *ws, cudaStream_t st, cudaStream_t qst, cudaEvent_t fork,
                cudaEvent_t join) {
    const HessWs w = hess_ws(n, ws);
    const int64_t p_cap = (int64_t)kHSplits * n * kHb;
    int ng = 0;
    const int64_t j0 = k + b;            // first trailing column
    const int nt = (int)(n - j0);
    const int rows = (int)(n - k - 1);   // rows k+1 .. n-1 (V is zero above)
    const bool side = Q && qst && fork && join;
    if (Q) {   // Q[:, k+1:n] -= (Q[:, k+1:n] V[k+1:n, :]) T V[k+1:n, :]^T
        cudaStream_t s = st;
        if (side) {
            cudaEventRecord(fork, st);
            cudaStreamWaitEvent(qst, fork, 0);
            s = qst;
        }
        gemm_splitk<false, false>((int)n, b, rows, 1.0, Q + (k + 1) * ldq, ldq, w.V + (k + 1), n,
                                  0.0, w.W, n, w.Pq, p_cap, s);
        gemm(false, false, (int)n, b, b, 1.0, w.W, n, w.T, kHb, 0.0, w.VTq, n, s);
        gemm(false, true, (int)n, rows, b, -1.0, w.VTq, n, w.V + (k + 1), n, 1.0,
             Q + (k + 1) * ldq, ldq, s);
        if (side) cudaEventRecord(join, qst);
        ng += 3;
    }
    if (nt > 0) {
        // A[:, j0:n] -= Y V[j0:n, :]^T (every row: the top part and the rest)
        gemm(false, true, (int)n, nt, b, -1.0, w.Y, n, w.V + j0, n, 1.0, A + j0 * lda, lda, st);
        // rows k+1 ..: A <- A - (V T^T) (V^T A), with Zt = A^T V (nt x b,
        // the long dimension on the tile's rows)
        gemm_splitk<true, false>(nt, b, rows, 1.0, A + (k + 1) + j0 * lda, lda, w.V + (k + 1), n,
                                 0.0, w.Z, n, w.P, p_cap, st);
        gemm(false, true, rows, b, b, 1.0, w.V + (k + 1), n, w.T, kHb, 0.0, w.VT, n, st);
        gemm(false, true, rows, nt, b, -1.0, w.VT, n, w.Z, n, 1.0, A + (k + 1) + j0 * lda, lda,
             st);
        ng += 4;
    }
    if (side) cudaStreamWaitEvent(st, join, 0);
    return ng;
}

// ---------------------------------------------------------------------------
// split-precision updates (evec_hessenberg with EVEC_SPLIT)
// ---------------------------------------------------------------------------

cudaError_t split_gemm_rows(const double *A, int64_t lda, int M, int K, int S,
                            __nv_bfloat16 *sa, unsigned long long *rowmax, int *ea,
                            cudaStream_t st);
cudaError_t split_slice_cols(const double *B, int64_t ldb, int K, int N, int S, int Npad,
                             __nv_bfloat16 *sb, unsigned long long *colmax, int *eb,
                             cudaStream_t st);
cudaError_t split_gemm_sliced(const __nv_bfloat16 *sa, int Mpad, const __nv_bfloat16 *sb,
                              int Npad, int M, int N, int K, int S, const int *kend,
                              const int *ea, const int *eb, double *C, int64_t ldc, int *err,
                              cudaStream_t st, int acc, int ksplit, double *part);
int split_pad_m(int M);
int split_pad_n(int N);
int split_pad_k(int K);

// The same updates as hess_update with the five large products through the
// split GEMM (BF16 digit slices with row / column power-of-two scales, FP64
// results; the operands are sliced before each product, so a product may
// update its own input): the two long products with the panel's columns
// (W = Q V and Z = A^T V, K = the rows below the panel) and the three
// rank-b updates (Q -= (W T) V^T, A -= Y V^T, A -= (V T^T) Z^T).  A
// transposed operand is sliced from the stored matrix directly: the row
// slices of M^T are the column slices of M and the other way round.  The
// two b x b products with T stay FP64.  sw: the slice buffers of both
// chains (HessSplitWs).  *status receives the first launch error.
int hess_update_split(int64_t n, double *A, int64_t lda, double *Q, int64_t ldq, int64_t k,
                      int b, double *ws, const HessSplitWs &sw, int S, int *err, int nsm,
                      cudaStream_t st, cudaStream_t qst, cudaEvent_t fork, cudaEvent_t join,
                      cudaError_t *status) {
    const HessWs w = hess_ws(n, ws);
    int ng = 0;
    const int64_t j0 = k + b;            // first trailing column
    const int nt = (int)(n - j0);
    const int rows = (int)(n - k - 1);   // rows k+1 .. n-1 (V is zero above)
    const int ni = (int)n;
    const bool side = Q && qst && fork && join;
    cudaError_t ce = cudaSuccess;
    auto ok = [&](cudaError_t e) {
        if (ce == cudaSuccess) ce = e;
        return ce == cudaSuccess;
    };
    // the long products (b output columns, K = rows) have one 128-row band
    // per CTA: their K steps are shared by up to kHSplitMax CTAs per band
    // so that the GPU fills, at least four 32-deep K steps each
    auto ksplit = [&](int M, int K) {
        const int bands = split_pad_m(M) / 128;
        int ks = std::min(kHSplitMax, std::max(1, (nsm + bands - 1) / bands));
        return std::max(1, std::min(ks, split_pad_k(K) / 128));
    };
    if (Q) {
        cudaStream_t s = st;
        if (side) {
            cudaEventRecord(fork, st);
            cudaStreamWaitEvent(qst, fork, 0);
            s = qst;
        }
        double *Qc = Q + (k + 1) * ldq;
        const double *V1 = w.V + (k + 1);
        // W = Q[:, k+1:n] V (n x b, K = rows)
        if (ok(split_gemm_rows(Qc, ldq, ni, rows, S, sw.qa, sw.qam, sw.qae, s)) &&
            ok(split_slice_cols(V1, n, rows, b, S, split_pad_n(b), sw.qb, sw.qbm, sw.qbe, s)))
            ok(split_gemm_sliced(sw.qa, split_pad_m(ni), sw.qb, split_pad_n(b), ni, b, rows, S,
                                 nullptr, sw.qae, sw.qbe, w.W, n, err, s, 0, ksplit(ni, rows),
                                 sw.qp));
        gemm(false, false, ni, b, b, 1.0, w.W, n, w.T, kHb, 0.0, w.VTq, n, s);
        // Q[:, k+1:n] -= VTq V^T: V^T's columns are V's rows
        if (ok(split_gemm_rows(w.VTq, n, ni, b, S, sw.qa, sw.qam, sw.qae, s)) &&
            ok(split_gemm_rows(V1, n, rows, b, S, sw.qb, sw.qbm, sw.qbe, s)))
            ok(split_gemm_sliced(sw.qa, split_pad_m(ni), sw.qb, split_pad_m(rows), ni, rows, b, S,
                                 nullptr, sw.qae, sw.qbe, Qc, ldq, err, s, -1, 1, nullptr));
        if (side) cudaEventRecord(join, qst);
        ng += 11;
    }
    if (nt > 0 && ce == cudaSuccess) {
        double *Aj = A + j0 * lda;
        double *As = A + (k + 1) + j0 * lda;
        // A[:, j0:n] -= Y V[j0:n, :]^T (every row)
        if (ok(split_gemm_rows(w.Y, n, ni, b, S, sw.ta, sw.tam, sw.tae, st)) &&
            ok(split_gemm_rows(w.V + j0, n, nt, b, S, sw.tb, sw.tbm, sw.tbe, st)))
            ok(split_gemm_sliced(sw.ta, split_pad_m(ni), sw.tb, split_pad_m(nt), ni, nt, b, S,
                                 nullptr, sw.tae, sw.tbe, Aj, lda, err, st, -1, 1, nullptr));
        // Z = A[k+1:n, j0:n]^T V[k+1:n, :] (nt x b, K = rows): A^T's rows are
        // the columns of A
        if (ok(split_slice_cols(As, lda, rows, nt, S, split_pad_m(nt), sw.ta, sw.tam, sw.tae,
                                st)) &&
            ok(split_slice_cols(w.V + (k + 1), n, rows, b, S, split_pad_n(b), sw.tb, sw.tbm,
                                sw.tbe, st)))
            ok(split_gemm_sliced(sw.ta, split_pad_m(nt), sw.tb, split_pad_n(b), nt, b, rows, S,
                                 nullptr, sw.tae, sw.tbe, w.Z, n, err, st, 0, ksplit(nt, rows),
                                 sw.tp));
        gemm(false, true, rows, b, b, 1.0, w.V + (k + 1), n, w.T, kHb, 0.0, w.VT, n, st);
        // A[k+1:n, j0:n] -= VT Z^T: Z^T's columns are Z's rows
        if (ok(split_gemm_rows(w.VT, n, rows, b, S, sw.ta, sw.tam, sw.tae, st)) &&
            ok(split_gemm_rows(w.Z, n, nt, b, S, sw.tb, sw.tbm, sw.tbe, st)))
            ok(split_gemm_sliced(sw.ta, split_pad_m(rows), sw.tb, split_pad_m(nt), rows, nt, b, S,
                                 nullptr, sw.tae, sw.tbe, As, lda, err, st, -1, 1, nullptr));
        ng += 16;
    }
    if (side) cudaStreamWaitEvent(st, join, 0);
    if (status) *status = ce;
    return ng;
}

}  // namespace evec
