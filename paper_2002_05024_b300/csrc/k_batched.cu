// k_batched.cu -- many independent Schur forms in one persistent launch.
//
// Each CTA (4 warps) takes the next matrix from a device work queue (an
// atomic counter over the matrices, which the host orders by decreasing
// estimated work, so the longest solves start first) and runs the whole
// tiled robust solve of Sec. 3.3 for it on its own: tile norms and input
// validation, then for s = N-1 .. 0 the diagonal-tile solves of every
// active unit (the same device code as the per-step kernel, in chunks of
// 16 real or 8 complex units) followed by the updates Y_r <- 2^dy Y_r -
// 2^dx T_rs X_s for all r < s, and finally the consolidation into canonical
// form.  CTAs never wait on one another; the queue is the only shared state.
// Matrices of this workload are small (n <= 1024), so one SM per matrix
// keeps each solve's data in L1/L2 and the device busy across the batch.
//
// Split precision (S > 0): the updates run as BF16 digit-slice products on
// the tensor cores, the same arithmetic as the single-matrix split update
// (balanced 7-bit digits after power-of-two row / column normalisation,
// one TMEM accumulator per digit diagonal, FP64 recombination) at CTA
// scope: per 128-row block of the rows above tile s and 32-column chunk of
// the active columns, the CTA slices T's rows and X_s's columns straight
// into shared memory (K-major, 64-byte swizzle), one thread issues the
// concatenated MMAs, and the 4 warps drain their TMEM lane quarters.  Each
// CTA holds 256 TMEM columns (8 diagonals x 32 columns); two CTAs per SM.
#include "diag_tile.cuh"
#include "split_common.cuh"

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

// tau[r N + s] = |M_rs|_inf for r < s, the in-tile block column norms, and
// validation of every referenced entry (upper part, and with `lower` the
// first subdiagonal of the diagonal tiles), errors at base + i + j ld.
// M is the quasi-triangular matrix, or a pencil's upper triangular T.
// smem: kBThreads doubles.
__device__ void cta_tile_norms(const Plan &P, const double *M, int64_t ld, int64_t base,
                               double *tau_out, double *blk_tau_out, bool lower, double *red,
                               DevStatus *status) {
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
                    const double v = M[i + (int64_t)j * ld];
                    check_entry_b(v, base + i + (int64_t)j * ld, status);
                    rs += fabs(v);
                }
                sum = fmax(sum, rs);
            }
            sum = bwarp_max(sum);
            if (lane == 0) red[warp] = sum;
            __syncthreads();
            if (tid == 0)
                tau_out[(int64_t)r * N + s] = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
            __syncthreads();
        }
        for (int j = c0; j < c1; j++)
            for (int i = c0 + tid; i < c1 && i <= j + (lower ? 1 : 0); i += kBThreads)
                check_entry_b(M[i + (int64_t)j * ld], base + i + (int64_t)j * ld, status);
        for (int k = P.tile_blk[s] + warp; k < P.tile_blk[s + 1]; k += kBThreads / 32) {
            const int q = P.blk_start[k];
            const int bs = P.blk_size[k];
            double mx = 0.0;
            for (int i = c0 + lane; i < q; i += 32) {
                double a = fabs(M[i + (int64_t)q * ld]);
                if (bs == 2) a += fabs(M[i + (int64_t)(q + 1) * ld]);
                mx = fmax(mx, a);
            }
            mx = bwarp_max(mx);
            if (lane == 0) blk_tau_out[k] = mx;
        }
    }
}

// Updates of step s: for every 64-column block of the active columns and
// every tile r < s, Y_r <- 2^dy Y_r - T_rs (2^dx X_s) with the new column
// maxima (GEN: Y_r <- 2^dy Y_r - [S_rs (beta X~) - T_rs (alpha X~)] with
// X~ = 2^dx X_s, two accumulation passes over the same registers; alpha
// mixes a pair's (Re, Im) columns, (alpha x)_re = ar xr - ai xi,
// (alpha x)_im = ar xi + ai xr).  Thread (tx, ty) = (tid % 16, tid / 16) owns rows ty + 8 i
// (i < 8) and columns tx + 16 j (j < 4) of the 64 x 64 block.  X_s is
// staged scaled by 2^dx[r, j] before the product (exact): the protection
// decisions bound the product of the scaled operands, not of the unscaled
// ones, which may overflow.
// smem: Bs [64][65], As [64][64], red [8][64] doubles, sdx / sdy [64] ints.
template <bool GEN>
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
            double acc[8][4];
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
            // pass 0: A = T_rs (S_rs for a pencil); pass 1 (pencils): A = T2_rs
            for (int pass = 0; pass < (GEN ? 2 : 1); pass++) {
                const double *A = pass == 0 ? B.T : B.T2;
                const int64_t lda = pass == 0 ? B.ldt : B.ldt2;
                if (pass == 1) __syncthreads();   // the first pass's readers are done
                for (int e = tid; e < 64 * 64; e += kBThreads) {
                    const int i = e % 64, k = e / 64;
                    As[k * 64 + i] =
                        (i < rows && k < K) ? A[(r0 + i) + (int64_t)(k0 + k) * lda] : 0.0;
                }
                __syncthreads();   // sdx is read by the staging of X_s below
                for (int e = tid; e < 64 * 64; e += kBThreads) {
                    const int k = e % 64, j = e / 64;
                    double v = 0.0;
                    if (k < K && j < nc) {
                        const int64_t c = j0 + j;
                        v = scale2(Y[(k0 + k) + c * ldy], sdx[j]);
                        if constexpr (GEN) {
                            const int u = P.col_unit[c];
                            const double ar = P.unit_lam[2 * u], ai = P.unit_lam[2 * u + 1];
                            if (pass == 0) {
                                v *= P.unit_beta[u];
                            } else {
                                double ax = ar * v;
                                if (ai != 0.0) {   // the pair partner, same scale
                                    const bool re = c == P.unit_col[u];
                                    const double xp =
                                        scale2(Y[(k0 + k) + (re ? c + 1 : c - 1) * ldy], sdx[j]);
                                    ax = re ? fma(ar, v, -ai * xp) : fma(ar, v, ai * xp);
                                }
                                v = -ax;
                            }
                        }
                    }
                    Bs[k * 65 + j] = v;
                }
                __syncthreads();
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

// ---------------------------------------------------------------------------
// split-precision update of step s (S > 0)
// ---------------------------------------------------------------------------
constexpr int kBSN = 32;                          // columns per chunk
constexpr int kBSBoxA = kTM * kTK * 2;            // 8 KB: 128 rows x 32 K (one slice)
constexpr int kBSBoxB = kBSN * kTK * 2;           // 2 KB: 32 columns x 32 K
constexpr int kBSSlots = 10;                      // tiles met by 128 rows (tiles >= 15 rows)
constexpr int kBSTmemCols = kSplitMaxS * kBSN;    // 256
// dynamic smem of the split update, from a 1024-byte aligned base
constexpr size_t kBSOffB = (size_t)kSplitMaxS * kBSBoxA;              // 64 KB
constexpr size_t kBSOffTab = kBSOffB + (size_t)kSplitMaxS * kBSBoxB;  // + 16 KB
// tables: nu [slots][32] u64, dx / dy [slots][32], ea / rt [128], eb [32]
constexpr size_t kBSTabBytes =
    (size_t)kBSSlots * kBSN * 8 + 2 * kBSSlots * kBSN * 4 + 2 * kTM * 4 + kBSN * 4;
constexpr size_t kBSBytes = 1024 + kBSOffTab + kBSTabBytes;

__device__ __forceinline__ void bsum2_add(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// byte offset of element (row, k) (k < 32) in a K-major, 64-byte swizzled box
// of 64-byte rows: 16-byte chunk c of row r sits at chunk c ^ ((r >> 1) & 3)
__device__ __forceinline__ int sw64_off(int r, int c) { return r * 64 + ((c ^ ((r >> 1) & 3)) << 4); }

// 8 values -> S slices of 8 BF16 digits each, stored as one 16-byte chunk
// per slice at dst + p * stride
__device__ __forceinline__ void slice8_store(const double (&x)[8], int e, int S,
                                             unsigned char *dst, int stride) {
    uint32_t w[kSplitMaxS][4];
#pragma unroll
    for (int p = 0; p < kSplitMaxS; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) w[p][q] = 0u;
#pragma unroll
    for (int t = 0; t < 8; t++) {
        int d[kSplitMaxS];
#pragma unroll
        for (int p = 0; p < kSplitMaxS; p++) d[p] = 0;
        digits7(x[t], e, S, d);
#pragma unroll
        for (int p = 0; p < kSplitMaxS; p++) {
            const uint32_t h = (uint32_t)__bfloat16_as_ushort(digit_bf16(d[p], p));
            w[p][t >> 1] |= (t & 1) ? (h << 16) : h;
        }
    }
#pragma unroll
    for (int p = 0; p < kSplitMaxS; p++)
        if (p < S)
            *(uint4 *)(dst + (size_t)p * stride) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// Y_r <- 2^dy Y_r - T_rs (2^dx X_s) for all r < s, as split products.
// Pencils (GEN): Y_r <- 2^dy Y_r - [S_rs T_rs] 2^dx W with the 2K x nc
// right-hand side W = [beta X_s; -alpha X_s] (alpha mixes a pair's columns,
// as in cta_tile_update<true>), so the product's K is twice the tile's;
// the row exponents cover both matrices' rows, the column exponents W's.
// Returns false if a bounded wait gave up (status->timeout is set).
template <bool GEN>
__device__ bool cta_split_update(const BatchItem &B, int s, int S, unsigned char *sm,
                                 uint32_t tmem, uint64_t *bar, uint32_t &phase, int *err) {
    const Plan &P = B.P;
    const int64_t m = P.m;
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *sA = sm;
    unsigned char *sB = sm + kBSOffB;
    unsigned long long *snu = (unsigned long long *)(sm + kBSOffTab);   // [slots][32]
    int *sdx = (int *)(snu + kBSSlots * kBSN);                           // [slots][32]
    int *sdy = sdx + kBSSlots * kBSN;
    int *sea = sdy + kBSSlots * kBSN;                                    // [128]
    int *srt = sea + kTM;                                                // [128]
    int *seb = srt + kTM;                                                // [32]
    const int k0 = P.tile_start[s], K = P.tile_start[s + 1] - k0;
    const int K2 = GEN ? 2 * K : K;   // the product's K: [S T] against W
    const int halves = (K2 + kTK - 1) / kTK;
    const int t0 = k0;   // rows above tile s
    double *Y = B.X;
    const int64_t ldy = B.ldx;
    // A entry (row, kk): S (or T) for kk < K, the pencil's T for K <= kk < 2K
    auto a_at = [&](int row, int kk) -> double {
        if (GEN && kk >= K) return B.T2[row + (int64_t)(k0 + kk - K) * B.ldt2];
        return B.T[row + (int64_t)(k0 + kk) * B.ldt];
    };
    // W entry (kk, column c): X_s for a standard problem; beta x, then
    // -(alpha x) (a pair's partner column at the same scale) for a pencil
    auto w_at = [&](int kk, int64_t c) -> double {
        if constexpr (!GEN) {
            return Y[(k0 + kk) + c * ldy];
        } else {
            const int u = P.col_unit[c];
            const int k = kk < K ? kk : kk - K;
            const double v = Y[(k0 + k) + c * ldy];
            if (kk < K) return v * P.unit_beta[u];
            const double ar = P.unit_lam[2 * u], ai = P.unit_lam[2 * u + 1];
            double ax = ar * v;
            if (ai != 0.0) {
                const bool re = c == P.unit_col[u];
                const double xp = Y[(k0 + k) + (re ? c + 1 : c - 1) * ldy];
                ax = re ? fma(ar, v, -ai * xp) : fma(ar, v, ai * xp);
            }
            return -ax;
        }
    };
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTM >> 4) << 24);
    for (int rb0 = 0; rb0 < t0; rb0 += kTM) {
        const int rows = min(kTM, t0 - rb0);
        const int row = rb0 + tid;
        const bool rv = tid < rows;
        // row tile and row exponent over the tile's K columns
        {
            int r = 0;
            if (rv) {
                int lo = 0, hi = s - 1;   // tile_start[lo] <= row < tile_start[hi + 1]
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (P.tile_start[mid] <= row) lo = mid;
                    else hi = mid - 1;
                }
                r = lo;
            }
            long long mb = 0;
            if (rv)
                for (int kk = 0; kk < K2; kk++) mb = max(mb, abs_bits(a_at(row, kk)));
            srt[tid] = rv ? r : -1;
            sea[tid] = exp_from_max((unsigned long long)mb);
        }
        __syncthreads();
        const int rfirst = srt[0];
        const int nslots = srt[rows - 1] - rfirst + 1;
        const int myslot = rv ? srt[tid] - rfirst : 0;
        const int er = sea[tid];
        for (int64_t j0 = P.tile_col[s]; j0 < m; j0 += kBSN) {
            const int nc = (int)min((int64_t)kBSN, m - j0);
            // column exponents of X_s and the chunk's tables
            if (tid < kBSN) {
                long long mb = 0;
                if (tid < nc)
                    for (int kk = 0; kk < K2; kk++) mb = max(mb, abs_bits(w_at(kk, j0 + tid)));
                seb[tid] = exp_from_max((unsigned long long)mb);
            }
            for (int idx = tid; idx < nslots * kBSN; idx += kBThreads) {
                const int sl = idx / kBSN, j = idx % kBSN;
                const int64_t at = (int64_t)(rfirst + sl) * m + j0 + j;
                sdx[idx] = j < nc ? B.seg_dx[at] : 0;
                sdy[idx] = j < nc ? B.seg_dy[at] : kFresh;
                snu[idx] = 0ull;
            }
            __syncthreads();
            for (int h = 0; h < halves; h++) {
                // A: thread = row, four 8-K chunks; B: thread = (column, chunk)
                for (int c = 0; c < 4; c++) {
                    double x[8];
#pragma unroll
                    for (int t = 0; t < 8; t++) {
                        const int kk = h * kTK + c * 8 + t;
                        x[t] = (rv && kk < K2) ? a_at(row, kk) : 0.0;
                    }
                    slice8_store(x, er, S, sA + sw64_off(tid, c), kBSBoxA);
                }
                {
                    const int j = tid >> 2, c = tid & 3;
                    double x[8];
#pragma unroll
                    for (int t = 0; t < 8; t++) {
                        const int kk = h * kTK + c * 8 + t;
                        x[t] = (j < nc && kk < K2) ? w_at(kk, j0 + j) : 0.0;
                    }
                    slice8_store(x, seb[j], S, sB + sw64_off(j, c), kBSBoxB);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    // the B slices lie one after another (slice q at rows 32 q):
                    // A_p against slices 0 .. S-1-p (N = 32 (S - p)) at TMEM
                    // column 32 p adds A_p B_q to diagonal p + q for every q
                    for (int kin = 0; kin < 2; kin++) {
                        const uint64_t bd = desc_sw64(saddr(sB) + kin * 32);
                        for (int p = 0; p < S; p++) {
                            const uint32_t id =
                                idesc | ((uint32_t)(((S - p) * kBSN) >> 3) << 17);
                            const uint64_t ad = desc_sw64(saddr(sA + p * kBSBoxA) + kin * 32);
                            const int acc = (h == 0 && kin == 0 && p == 0) ? 0 : 1;
                            asm volatile(
                                "{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n" ::"r"(
                                    tmem + (uint32_t)(p * kBSN)),
                                "l"(ad), "l"(bd), "r"(id), "r"(acc));
                        }
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
                        "[%0];" ::"r"(saddr(bar)));
                }
                const bool ok = mbar_wait(saddr(bar), phase, err);
                phase ^= 1u;
                if (__syncthreads_or(!ok)) return false;
            }
            // epilogue: thread = row (TMEM lane), 4 groups of 8 columns
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
            for (int g = 0; g < 4; g++) {
                if (g * 8 >= nc) break;   // block-uniform
                float hi[8], lo[8], sum5[8];
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    hi[q] = 0.0f;
                    lo[q] = 0.0f;
                    sum5[q] = 0.0f;
                }
                // diagonals 0-4 through the two-sum, 5.. summed in FP32 first
#pragma unroll
                for (int d0 = 0; d0 < kSplitMaxS; d0 += 2) {
                    if (d0 < S) {
                        uint32_t v[2][8];
                        TMEM_LD8(tl + (uint32_t)(d0 * kBSN + g * 8), v[0]);
                        if (d0 + 1 < S) TMEM_LD8(tl + (uint32_t)((d0 + 1) * kBSN + g * 8), v[1]);
                        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                        for (int e = 0; e < 2; e++) {
                            const int d = d0 + e;
                            if (d < S) {
#pragma unroll
                                for (int q = 0; q < 8; q++) {
                                    const float xv = __uint_as_float(v[e][q]);
                                    if (d == 0) hi[q] = xv;
                                    else if (d < 5) bsum2_add(hi[q], lo[q], xv);
                                    else sum5[q] += xv;
                                }
                            }
                        }
                    }
                }
                if (S > 5)
#pragma unroll
                    for (int q = 0; q < 8; q++) bsum2_add(hi[q], lo[q], sum5[q]);
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int jl = g * 8 + q;
                    if (!rv || jl >= nc) continue;
                    const int dx = sdx[myslot * kBSN + jl], dy = sdy[myslot * kBSN + jl];
                    const float h2 = hi[q] + lo[q];
                    const float l2 = lo[q] - (h2 - hi[q]);
                    const double Pv = df_to_double(h2, l2, er + seb[jl] + dx);
                    double *yp = Y + row + (j0 + jl) * ldy;
                    double y;
                    if (dy == kFresh) y = -Pv;
                    else if (dy >= -1022 && dy <= 1023) y = fma(*yp, pow2_normal(dy), -Pv);
                    else y = scale2(*yp, dy) - Pv;
                    *yp = y;
                    atomicMax(&snu[myslot * kBSN + jl], (unsigned long long)abs_bits(y));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            for (int idx = tid; idx < nslots * kBSN; idx += kBThreads) {
                const int sl = idx / kBSN, j = idx % kBSN;
                if (j < nc && snu[idx])
                    atomicMax((unsigned long long *)&B.seg_nu[(int64_t)(rfirst + sl) * m + j0 + j],
                              snu[idx]);
            }
            __syncthreads();
        }
    }
    return true;
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

// Back-transformation Xout = Q Y of a solved matrix (Y canonical, zero
// below each column's block), in 64 x 64 blocks of Xout with the thread
// layout of cta_tile_update: K runs to the block end of the last column of
// the column block (the rows below are zero in every column of it).  Then
// the canonical form of every unit's columns (max_i |x_i|, a pair's
// |re| + |im|, brought into [1, 2); the exponent adjusted by the same
// power of two).  Y is canonical, so |Q Y|_inf <= 2 sqrt(n): no overflow.
// smem: As [64][64], Bs [64][65] doubles; red [4] doubles.
__device__ void cta_backtransform(const BatchItem &B, double *smem, double *red) {
    const Plan &P = B.P;
    const int64_t m = P.m, n = P.n;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int lane = tid & 31, warp = tid >> 5;
    double *Bs = smem;                  // [k][65]
    double *As = Bs + 64 * 65;          // [k][64]
    for (int64_t j0 = 0; j0 < m; j0 += 64) {
        const int nc = (int)min((int64_t)64, m - j0);
        const int ul = P.col_unit[j0 + nc - 1];
        const int kb = P.unit_blk[ul];
        const int kend = P.blk_start[kb] + P.blk_size[kb];
        for (int64_t i0 = 0; i0 < n; i0 += 64) {
            const int rows = (int)min((int64_t)64, n - i0);
            double acc[8][4];
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
            for (int k0 = 0; k0 < kend; k0 += 64) {
                const int K = min(64, kend - k0);
                __syncthreads();   // the previous chunk's readers are done
                for (int e = tid; e < 64 * 64; e += kBThreads) {
                    const int i = e % 64, k = e / 64;
                    As[k * 64 + i] = (i < rows && k < K) ? B.Q[(i0 + i) + (int64_t)(k0 + k) * B.ldq]
                                                         : 0.0;
                }
                for (int e = tid; e < 64 * 64; e += kBThreads) {
                    const int k = e % 64, j = e / 64;
                    Bs[k * 65 + j] = (k < K && j < nc) ? B.X[(k0 + k) + (j0 + j) * B.ldx] : 0.0;
                }
                __syncthreads();
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
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int jl = tx + 16 * j;
                if (jl >= nc) continue;
                double *c = B.Xout + (j0 + jl) * B.ldxo + i0;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int row = ty + 8 * i;
                    if (row < rows) c[row] = acc[i][j];
                }
            }
        }
    }
    __syncthreads();   // every column of Xout is written
    constexpr int kW = kBThreads / 32;
    for (int u = 0; u < P.nunits; u++) {
        const int col = P.unit_col[u];
        const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
        double *xr = B.Xout + (int64_t)col * B.ldxo;
        double *xi = B.Xout + (int64_t)(col + 1) * B.ldxo;
        double mx = 0.0;
        for (int64_t i = tid; i < n; i += kBThreads) {
            double v = fabs(xr[i]);
            if (cplx) v += fabs(xi[i]);
            mx = fmax(mx, v);
        }
        mx = bwarp_max(mx);
        if (lane == 0) red[warp] = mx;
        __syncthreads();
        mx = 0.0;
#pragma unroll
        for (int w = 0; w < kW; w++) mx = fmax(mx, red[w]);
        __syncthreads();   // red is reused by the next unit
        if (mx == 0.0) continue;
        const int t2 = ilog2_abs(mx);
        for (int64_t i = tid; i < n; i += kBThreads) {
            xr[i] = scale2(xr[i], -t2);
            if (cplx) xi[i] = scale2(xi[i], -t2);
        }
        if (tid == 0) {
            B.scale_exp[col] -= t2;
            if (cplx) B.scale_exp[col + 1] -= t2;
        }
    }
}

}  // namespace

// GEN: every item is a pencil (beta S - alpha T), FP64 updates only.
template <bool SPLIT, bool GEN>
__global__ void __launch_bounds__(kBThreads)
    k_batched(const BatchItem *__restrict__ items, int count, int *queue, DevStatus *status,
              int S) {
    extern __shared__ double smem[];
    __shared__ int next;
    __shared__ int sbest[kBThreads / 32];
    __shared__ double sred[kBThreads / 32];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_holder;
    uint32_t tmem = 0, phase = 0;
    unsigned char *sbase = (unsigned char *)(((uintptr_t)smem + 1023) & ~(uintptr_t)1023);
    if constexpr (SPLIT) {
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             saddr(&tmem_holder)),
                         "r"(kBSTmemCols));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&mbar)), "r"(1));
            asm volatile("fence.mbarrier_init.release.cluster;");
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        tmem = tmem_holder;
    }
    bool alive = true;
    while (alive) {
        if (threadIdx.x == 0) next = atomicAdd(queue, 1);
        __syncthreads();
        const int k = next;
        __syncthreads();
        if (k >= count) break;
        const BatchItem B = items[k];
        const Plan &P = B.P;
        cta_tile_norms(P, B.T, B.ldt, B.t_base, B.tau, B.blk_tau, true, smem, status);
        __syncthreads();
        Pencil pen;
        if constexpr (GEN) {
            cta_tile_norms(P, B.T2, B.ldt2, B.t2_base, B.tau2, B.blk_tau2, false, smem, status);
            __syncthreads();
            pen.T = B.T2;
            pen.ldt = B.ldt2;
            pen.tau = B.tau2;
            pen.blk_tau = B.blk_tau2;
        }
        for (int s = P.ntiles - 1; s >= 0; s--) {
            for (int pos = P.tile_real[s]; pos < P.nreal; pos += Lanes<false>::U * 4) {
                diag_tile<4, false, GEN>(s, pos, B.T, B.ldt, P, B.tau, B.blk_tau, B.X, B.ldx,
                                         B.seg_e, B.seg_nu, B.seg_dx, B.seg_dy, smem, pen);
                __syncthreads();
            }
            for (int pos = P.tile_cplx[s]; pos < P.ncplx; pos += Lanes<true>::U * 4) {
                diag_tile<4, true, GEN>(s, pos, B.T, B.ldt, P, B.tau, B.blk_tau, B.X, B.ldx,
                                        B.seg_e, B.seg_nu, B.seg_dx, B.seg_dy, smem, pen);
                __syncthreads();
            }
            if (s > 0 && P.tile_col[s] < P.m) {
                if constexpr (SPLIT) {
                    if (!cta_split_update<GEN>(B, s, S, sbase, tmem, &mbar, phase,
                                          &status->timeout)) {
                        alive = false;
                        break;
                    }
                } else {
                    cta_tile_update<GEN>(B, s, smem);
                }
                __syncthreads();
            }
        }
        if (!alive) break;
        for (int u = 0; u < P.nunits; u++) cta_finalize_unit(B, u, sbest);
        __syncthreads();
        if constexpr (!GEN) {
            if (B.lam_re || B.lam_im)
                for (int u = threadIdx.x; u < P.nunits; u += kBThreads) {
                    const int col = P.unit_col[u];
                    const double re = P.unit_lam[2 * u], im = P.unit_lam[2 * u + 1];
                    if (B.lam_re) B.lam_re[col] = re;
                    if (B.lam_im) B.lam_im[col] = im;
                    if (im != 0.0) {
                        if (B.lam_re) B.lam_re[col + 1] = re;
                        if (B.lam_im) B.lam_im[col + 1] = -im;
                    }
                }
        }
        if (B.Q) {   // X = Q Y (pencils: Z Y) and the canonical form
            cta_backtransform(B, smem, sred);
            __syncthreads();
        }
    }
    if constexpr (SPLIT) {
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (threadIdx.x < 32)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(kBSTmemCols));
    }
}

// gen_tile > 0: a batch of pencils whose tiles have at most gen_tile rows
// (the diagonal-tile solver also holds T's tile)
size_t batched_smem_bytes(bool split, int gen_tile) {
    const size_t upd = sizeof(double) * (64 * 65 + 64 * 64 + 8 * 64) + sizeof(int) * 128;
    // the split variant aligns its operand tiles to 1024 bytes; its size
    // also keeps at most two CTAs (2 x 256 TMEM columns) on an SM
    const size_t base =
        gen_tile > 0 ? std::max(diag_smem<4, true>(gen_tile), upd) : std::max(diag_smem<4>(64), upd);
    return split ? std::max(base + 1024, kBSBytes) : base;
}

// One persistent launch: grid = SMs x CTAs per SM (occupancy query); S > 0
// runs the split-precision updates (S digit slices); gen_tile > 0 the
// pencil variant (tiles of at most gen_tile rows).
cudaError_t launch_batched(const BatchItem *items, int count, int *queue, DevStatus *status,
                           int nsm, cudaStream_t st, int S, int gen_tile) {
    const bool split = S > 0;
    const size_t smem = batched_smem_bytes(split, gen_tile);
    auto kern = gen_tile > 0 ? (split ? k_batched<true, true> : k_batched<false, true>)
                             : (split ? k_batched<true, false> : k_batched<false, false>);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    if (split) per_sm = std::min(per_sm, kTmemCols / kBSTmemCols);
    // Standard batches: at most two CTAs per SM.  Their time is the chain of
    // the largest matrices, each on one CTA, and a third CTA on its SM slows
    // that CTA more than it adds (B300, the 2000-matrix batch: 61.7 ms at two
    // CTAs per SM, 79.4 at three).  Pencil batches, whose steps carry twice
    // the update work, gain from the third (142.7 -> 113.3 ms).
    if (gen_tile <= 0) per_sm = std::min(per_sm, 2);
    const int grid = std::min(count, nsm * per_sm);
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, kBThreads, smem, st>>>(items, count, queue, status, S);
    return cudaGetLastError();
}

size_t batch_item_bytes() { return sizeof(BatchItem); }

}  // namespace evec
