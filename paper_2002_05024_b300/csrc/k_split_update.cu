// k_split_update.cu -- the tile update of one step of the tiled
// backsubstitution (Sec. 3.3: Y_r <- 2^dy Y_r - T_rs (2^dx X_s) for every
// tile row r above the diagonal tile s, with the column maxima of the new
// segments) as split-precision products on the BF16 tensor cores.
//
// The update's K is one tile (<= 64), so per output element the tensor-core
// work (S (S + 1) / 2 slice products of K) and the epilogue (drain 8 digit
// diagonals from TMEM, recombine, one FP64 read-modify-write of Y) cost about
// the same.  The kernel therefore overlaps them: each CTA keeps one 128-row
// block of the panel T[0:t0, tile s] resident in shared memory as its S
// slices (up to 128 KB), streams 32-column tiles of X_s through a two-stage
// TMA ring, and alternates two TMEM accumulators (2 x 8 diagonals x 32
// columns = 512 columns), so the MMAs of column tile j + 1 run while the
// epilogue warps finish tile j.  The grid is one wave: M blocks x column
// groups <= the SM count, one CTA per SM.
//
// Warps 0-15: epilogue (TMEM lane quarter w % 4, 8 of the 32 columns);
// warp 16: TMEM allocation + MMA issue; warp 17: TMA producer (lane 0) and
// the per-tile exponent tables (all lanes, into shared memory).  Every
// mbarrier wait is bounded and gives up by setting *err.
#include "split_common.cuh"

namespace evec {

constexpr int kUN = 32;                               // columns per tile
constexpr int kUBoxA = kTM * kTK * 2;                 // 8 KB: 128 rows x 32 K
constexpr int kUBoxB = kUN * kTK * 2;                 // 2 KB: 32 rows x 32 K
constexpr int kUPanelBytes = kSplitMaxS * 2 * kUBoxA; // 128 KB (K = 64)
constexpr int kUStageBytes = kSplitMaxS * 2 * kUBoxB; // 32 KB
constexpr int kUEpiWarps = 16;                        // lane quarter w % 4, 8 columns each
constexpr int kUMmaWarp = kUEpiWarps, kUProdWarp = kUEpiWarps + 1;
constexpr int kUThreads = 32 * (kUEpiWarps + 2);
constexpr int kUAccCols = kSplitMaxS * kUN;           // 256 TMEM columns per buffer
constexpr int kUSlots = 12;                           // tile rows met by 128 rows (tiles >= 15)
// per stage: dx, dy [kUSlots][kUN] and eb [kUN] (int)
constexpr int kUTableInts = 2 * kUSlots * kUN + kUN;

size_t split_update_smem_bytes() {
    return 1024 + kUPanelBytes + 2 * kUStageBytes + 2 * kUTableInts * 4 + 256;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect(uint64_t *b, int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)),
                 "r"(bytes));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *b) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            saddr(b)));
}

// max of non-negative 64-bit patterns over the lanes with member set, via two
// 32-bit warp reductions (high word, then low word among the high-word max)
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long b, bool member) {
    const unsigned h = member ? (unsigned)(b >> 32) : 0u;
    const unsigned hm = __reduce_max_sync(0xffffffffu, h);
    const unsigned l = (member && h == hm) ? (unsigned)b : 0u;
    const unsigned lm = __reduce_max_sync(0xffffffffu, l);
    return ((unsigned long long)hm << 32) | lm;
}

// two-sum accumulation of x into (hi, lo): hi takes the rounded sum, lo
// collects the exact rounding errors (renormalised once at the end)
__device__ __forceinline__ void sum2_add(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// Y (column-major, ldy) rows [0, M) x columns [col0, col0 + N) updated in
// place; A = panel slices at rows aRow0 + p aMpad of tmA; B = column slices
// at rows q Npad of tmB (32-row boxes); K (32 or 64) = the tile's rows
// rounded up to 32; ea = row exponents of the panel rows, eb = column
// exponents of X_s; row_tile maps a row to its tile; dx / dy / nu are the
// [ntiles][m] segment arrays (nu as bit patterns, merged with atomicMax).
__global__ void __launch_bounds__(kUThreads, 1)
    k_split_update(const __grid_constant__ CUtensorMap tmA,
                   const __grid_constant__ CUtensorMap tmB, int S, int M, int N, int aRow0,
                   int aMpad, int Npad, int K, const int *__restrict__ ea,
                   const int *__restrict__ eb, double *__restrict__ Y, int64_t ldy,
                   const int32_t *__restrict__ row_tile, const int32_t *__restrict__ dx,
                   const int32_t *__restrict__ dy, unsigned long long *__restrict__ nu, int64_t m,
                   int col0, int *err, int by0) {
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + kUPanelBytes;
    int *tab = (int *)(sB + 2 * kUStageBytes);   // [2][kUTableInts]
    uint64_t *bars = (uint64_t *)(tab + 2 * kUTableInts);
    uint64_t *a_full = bars, *b_full = bars + 1, *b_empty = bars + 3, *acc_full = bars + 5,
             *acc_empty = bars + 7, *t_full = bars + 9, *t_empty = bars + 11;
    uint32_t *tmem_holder = (uint32_t *)(bars + 13);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = ((int)blockIdx.y + by0) * kTM;   // row blocks by0, by0 + 1, ...
    const int ntN = (N + kUN - 1) / kUN;
    const int nmine = (int)blockIdx.x < ntN ? (ntN - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int khalves = K / kTK;
    const int rlo = row_tile[m0], rhi = row_tile[min(m0 + kTM, M) - 1];

    if (warp == kUMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tmem_holder)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(a_full, 1);
        for (int b = 0; b < 2; b++) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], 1);
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kUEpiWarps);
            mbar_init(&t_full[b], 32);
            mbar_init(&t_empty[b], kUEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("fence.proxy.async.shared::cta;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_holder;

    if (warp == kUProdWarp) {
        // lane 0: TMA of the panel once, then of the column tiles; all lanes:
        // the tile's exponent tables (dx, dy per tile row and column, eb)
        if (lane == 0 && nmine > 0) {
            mbar_expect(a_full, S * khalves * kUBoxA);
            for (int h = 0; h < khalves; h++)
                for (int p = 0; p < S; p++)
                    tma2d(saddr(sA + (h * kSplitMaxS + p) * kUBoxA), &tmA, h * kTK,
                          aRow0 + p * aMpad + m0, saddr(a_full));
        }
        int issued = 0;
        for (int j = 0; j < nmine; j++) {
            const int st = j & 1;
            const uint32_t ph = ((uint32_t)(j >> 1) & 1) ^ 1;
            int ok = 1;
            if (lane == 0) {
                ok = mbar_wait(saddr(&b_empty[st]), ph, err) &&
                     mbar_wait(saddr(&t_empty[st]), ph, err);
                if (ok) {
                    const int n0 = ((int)blockIdx.x + j * (int)gridDim.x) * kUN;
                    mbar_expect(&b_full[st], S * khalves * kUBoxB);
                    unsigned char *dst = sB + st * kUStageBytes;
                    for (int h = 0; h < khalves; h++)
                        for (int q = 0; q < S; q++)
                            tma2d(saddr(dst + (h * kSplitMaxS + q) * kUBoxB), &tmB, h * kTK,
                                  q * Npad + n0, saddr(&b_full[st]));
                    issued = j + 1;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            const int n0 = ((int)blockIdx.x + j * (int)gridDim.x) * kUN;
            int *t = tab + st * kUTableInts;
            const int col = n0 + lane;
            const bool cv = col < N;
            for (int sl = 0; sl <= rhi - rlo; sl++) {
                const int64_t at = (int64_t)(rlo + sl) * m + col0 + col;
                t[sl * kUN + lane] = cv ? dx[at] : 0;
                t[(kUSlots + sl) * kUN + lane] = cv ? dy[at] : kFresh;
            }
            t[2 * kUSlots * kUN + lane] = cv ? eb[col] : 0;
            mbar_arrive(&t_full[st]);
        }
        if (lane == 0) {   // the copies in flight have landed before the CTA ends
            if (nmine > 0) mbar_wait(saddr(a_full), 0, err);
            for (int j = max(0, issued - 2); j < issued; j++)
                mbar_wait(saddr(&b_full[j & 1]), (uint32_t)(j >> 1) & 1, err);
        }
    } else if (warp == kUMmaWarp) {
        if (lane == 0 && nmine > 0) {   // MMA issue
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTM >> 4) << 24);
            bool ok = mbar_wait(saddr(a_full), 0, err);
            const uint32_t a0 = saddr(sA);
            for (int j = 0; ok && j < nmine; j++) {
                const int st = j & 1, ab = j & 1;
                const uint32_t ph = (uint32_t)(j >> 1) & 1;
                if (!mbar_wait(saddr(&acc_empty[ab]), ph ^ 1, err)) break;
                if (!mbar_wait(saddr(&b_full[st]), ph, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t b0 = saddr(sB + st * kUStageBytes);
                const uint32_t acc0 = tmem + (uint32_t)(ab * kUAccCols);
                // The B slices of the tile lie one after another (slice q at
                // rows 32 q), so one MMA of A_p against slices 0 .. S-1-p
                // (N = 32 (S - p)) written at column 32 p adds A_p B_q to
                // diagonal p + q for every q at once.  Narrow MMAs into one
                // accumulator complete one at a time; these wide ones keep
                // the tensor pipe busy.
                for (int kk = 0; kk < 2 * khalves; kk++) {
                    const int h = kk >> 1, kin = kk & 1;
                    const uint64_t bd = desc_sw64(b0 + h * kSplitMaxS * kUBoxB + kin * 32);
                    for (int p = 0; p < S; p++) {
                        const uint32_t id = idesc | ((uint32_t)(((S - p) * kUN) >> 3) << 17);
                        const uint64_t ad = desc_sw64(a0 + (h * kSplitMaxS + p) * kUBoxA + kin * 32);
                        // the first product (p = 0, first K step) overwrites
                        const int acc = (p == 0 && kk == 0) ? 0 : 1;
                        asm volatile(
                            "{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n" ::"r"(
                                acc0 + (uint32_t)(p * kUN)),
                            "l"(ad), "l"(bd), "r"(id), "r"(acc));
                    }
                }
                umma_commit(&b_empty[st]);
                umma_commit(&acc_full[ab]);
            }
        }
    } else {   // epilogue warps
        const int quarter = warp & 3, cg = warp >> 2;   // lane quarter, 8-column group
        const int row = m0 + quarter * 32 + lane;
        const bool rv = row < M;
        const int r = rv ? row_tile[row] : -1;
        const int slot = rv ? r - rlo : 0;
        const int er = rv ? ea[row] : 0;
        // the warp's 32 rows fall into at most four tile rows (tiles above
        // the last have >= 15 rows: 1 + 15 + 15 + 1): group g = index of the
        // lane's tile row among them
        const unsigned vmask = __ballot_sync(0xffffffffu, rv);
        int gr[4] = {-1, -1, -1, -1};
        int ng = 0, grp = -1;
        {
            unsigned left = vmask;
            while (left && ng < 4) {
                const int rl = __shfl_sync(0xffffffffu, r, __ffs(left) - 1);
                const unsigned in = __ballot_sync(0xffffffffu, rv && r == rl);
                if (rv && r == rl) grp = ng;
                gr[ng++] = rl;
                left &= ~in;
            }
        }
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cg * 8);
        for (int j = 0; j < nmine; j++) {
            const int ab = j & 1;
            const uint32_t ph = (uint32_t)(j >> 1) & 1;
            const int cl0 = cg * 8;   // first local column of this warp
            const int c0 = ((int)blockIdx.x + j * (int)gridDim.x) * kUN + cl0;
            if (!mbar_wait(saddr(&t_full[ab]), ph, err)) break;
            const int *t = tab + ab * kUTableInts;
            const int *tdx = t + slot * kUN + cl0;
            const int *tdy = t + (kUSlots + slot) * kUN + cl0;
            const int *teb = t + 2 * kUSlots * kUN + cl0;
            // operands that do not wait for the accumulator
            double *ycol = Y + row + ((int64_t)col0 + c0) * ldy;
            double oldv[8];
            int dyv[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                dyv[q] = tdy[q];
                oldv[q] = (rv && c0 + q < N && dyv[q] != kFresh) ? ycol[q * ldy] : 0.0;
            }
            if (!mbar_wait(saddr(&acc_full[ab]), ph, err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ta = tl + (uint32_t)(ab * kUAccCols);
            float hi[8], lo[8], sm[8];
            // diagonal D is below about 2^(-7D) of diagonal 0: diagonals 0-4
            // enter the two-sum accumulator one by one, 5.. are summed in FP32
            // first (rounding near 2^-58 of the leading term).  Loads go in
            // pairs of diagonals, one wait per pair.
#pragma unroll
            for (int q = 0; q < 8; q++) {
                hi[q] = 0.0f;
                lo[q] = 0.0f;
                sm[q] = 0.0f;
            }
#pragma unroll
            for (int d0 = 0; d0 < kSplitMaxS; d0 += 2) {
                if (d0 < S) {
                    uint32_t v[2][8];
                    TMEM_LD8(ta + (uint32_t)(d0 * kUN), v[0]);
                    if (d0 + 1 < S) TMEM_LD8(ta + (uint32_t)((d0 + 1) * kUN), v[1]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const int d = d0 + e;
                        if (d < S) {
#pragma unroll
                            for (int q = 0; q < 8; q++) {
                                const float x = __uint_as_float(v[e][q]);
                                if (d == 0) hi[q] = x;
                                else if (d < 5) sum2_add(hi[q], lo[q], x);
                                else sm[q] += x;
                            }
                        }
                    }
                }
            }
            if (S > 5)
#pragma unroll
                for (int q = 0; q < 8; q++) sum2_add(hi[q], lo[q], sm[q]);
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int c = c0 + q;
                if (c >= N) break;   // warp-uniform
                unsigned long long b = 0ull;
                if (rv) {
                    // renormalise the two-sum pair: |lo| <= ulp(hi) / 2
                    const float h2 = hi[q] + lo[q];
                    const float l2 = lo[q] - (h2 - hi[q]);
                    const double P = df_to_double(h2, l2, er + teb[q] + tdx[q]);
                    double y;
                    if (dyv[q] == kFresh)
                        y = __longlong_as_double(__double_as_longlong(P) ^ (1ll << 63));
                    else if (dyv[q] >= -1022 && dyv[q] <= 1023)   // old 2^dy exact in the FMA
                        y = fma(oldv[q], pow2_normal(dyv[q]), -P);
                    else y = scale2(oldv[q], dyv[q]) - P;
                    ycol[q * ldy] = y;
                    b = (unsigned long long)abs_bits(y);
                }
                for (int g = 0; g < ng; g++) {
                    const unsigned long long mx = warp_max_u64(b, grp == g);
                    if (lane == 0 && mx) atomicMax(&nu[(int64_t)gr[g] * m + col0 + c], mx);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[ab]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == kUMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

// X_s slices for the update: one warp per column j of the K x N block B
// (K <= 64, column-major, ldb): column maximum by shuffles, exponent eb_j,
// then S slices [S][Npad][64] (K contiguous, zero beyond K and N)
__global__ void __launch_bounds__(256)
    k_slice_xs(const double *__restrict__ B, int64_t ldb, int K, int N, int Nr, int S,
               __nv_bfloat16 *__restrict__ out, int Npad, int *__restrict__ eb) {
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= Nr) return;
    double x0 = 0.0, x1 = 0.0;
    if (j < N) {
        if (lane < K) x0 = B[lane + (int64_t)j * ldb];
        if (lane + 32 < K) x1 = B[lane + 32 + (int64_t)j * ldb];
    }
    long long b = max(abs_bits(x0), abs_bits(x1));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    const int e = exp_from_max((unsigned long long)b);
    int d0[kSplitMaxS], d1[kSplitMaxS];
#pragma unroll
    for (int p = 0; p < kSplitMaxS; p++) d0[p] = d1[p] = 0;
    digits7(x0, e, S, d0);
    digits7(x1, e, S, d1);
    for (int p = 0; p < S; p++) {
        __nv_bfloat16 *o = out + ((size_t)p * Npad + j) * 64;
        o[lane] = digit_bf16(d0[p], p);
        o[lane + 32] = digit_bf16(d1[p], p);
    }
    if (lane == 0) eb[j] = e;
}

// Step s of the split tile updates, panel-resident form (tiles <= 64 rows),
// in two parts: split_slice_xs slices X_s = Y[t0 : t0 + ts, col0 : m] (or
// the pencil right-hand side), split_update_rows updates the 128-row
// blocks [rb0, rb1) of the rows above tile s on at most `cap` CTAs (one
// per SM).  rhs (pencils, 2 |tile| <= 64): the right-hand side
// [beta X_s; -(alpha X_s)] (ld ldr) replaces X_s, and split_update_rows
// then takes pencil = true (K = 2 |tile|).
cudaError_t split_slice_xs(const SplitUpdateCtx &ctx, int t0, int ts, int col0, int m,
                           const double *Y, int64_t ldy, __nv_bfloat16 *sb, int *eb,
                           cudaStream_t st, const double *rhs, int64_t ldr) {
    const int N = m - col0;
    if (N <= 0 || t0 <= 0) return cudaSuccess;
    const int Nr = (N + kUN - 1) / kUN * kUN;
    const int K = rhs ? 2 * ts : ts;
    k_slice_xs<<<Nr / 8, 256, 0, st>>>(rhs ? rhs : Y + t0 + (int64_t)col0 * ldy, rhs ? ldr : ldy,
                                       K, N, Nr, ctx.S, sb, ctx.Npad, eb);
    return cudaGetLastError();
}

cudaError_t split_update_rows(const SplitUpdateCtx &ctx, int t0, int ts, int prow0, int pea,
                              int col0, int m, double *Y, int64_t ldy, const int *ea_panels,
                              const int *eb, const int32_t *row_tile, const int32_t *dx,
                              const int32_t *dy, double *seg_nu, int *err, int rb0, int rb1,
                              int cap, cudaStream_t st, bool pencil) {
    const int N = m - col0;
    if (N <= 0 || t0 <= 0 || rb1 <= rb0) return cudaSuccess;
    const int Nr = (N + kUN - 1) / kUN * kUN;
    const int K = pencil ? 2 * ts : ts;   // the pencil right-hand side has 2 |tile| rows
    const int mpad = (t0 + kTM - 1) / kTM * kTM;
    const int gy = rb1 - rb0;
    const int ntN = Nr / kUN;
    const int gx = std::max(1, std::min(ntN, cap / gy));
    const size_t smem = split_update_smem_bytes();
    cudaFuncSetAttribute(k_split_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_split_update<<<dim3(gx, gy), kUThreads, smem, st>>>(
        ctx.tmA, ctx.tmB32, ctx.S, t0, N, prow0, mpad, ctx.Npad, (K + kTK - 1) / kTK * kTK,
        ea_panels + pea, eb, Y, ldy, row_tile, dx, dy, (unsigned long long *)seg_nu, m, col0,
        err, rb0);
    return cudaGetLastError();
}

cudaError_t split_update_step_resident(const SplitUpdateCtx &ctx, int t0, int ts, int prow0,
                                       int pea, int col0, int m, double *Y, int64_t ldy,
                                       const int *ea_panels, __nv_bfloat16 *sb, int *eb,
                                       const int32_t *row_tile, const int32_t *dx,
                                       const int32_t *dy, double *seg_nu, int *err, int nsm,
                                       cudaStream_t st, const double *rhs, int64_t ldr) {
    cudaError_t e = split_slice_xs(ctx, t0, ts, col0, m, Y, ldy, sb, eb, st, rhs, ldr);
    if (e != cudaSuccess) return e;
    return split_update_rows(ctx, t0, ts, prow0, pea, col0, m, Y, ldy, ea_panels, eb, row_tile,
                             dx, dy, seg_nu, err, 0, (t0 + kTM - 1) / kTM, nsm, st,
                             rhs != nullptr);
}

}  // namespace evec
