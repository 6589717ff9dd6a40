// k_split.cu -- split-precision FP64 GEMM on the BF16 tensor cores (tcgen05).
//
// C = A B with FP64 operands, computed as in the Ozaki scheme (error-free
// splitting of the operands into small-integer slices whose products are
// exact in FP32): every row of A is normalised by a power of two 2^ea_i so
// |a~| < 1/2, every column of B by 2^eb_j; each normalised value is written
// in balanced base 2^7 with S <= 8 digits, x~ = sum_p d_p 2^(-7(p+1)),
// |d_p| <= 64, and slice p holds d_p 2^(-7(p+1)) as an exact BF16 number.
// Only the digit diagonals D = p + q < S are formed (S (S + 1) / 2 slice
// products).  A diagonal's products are multiples of 2^(-7(D+2)) bounded by
// 2^12 of those units; a diagonal has at most 8 terms, so its sum over
// K = 512 stays within 2^24 units and is exact in the FP32 tensor-core
// accumulator.  Each diagonal has its own TMEM accumulator; every 512 of K
// the epilogue warps drain them into a double-float (hi, lo) FP32
// accumulator, and at the end C_ij = 2^(ea_i + eb_j) (hi + lo) in FP64.
// The digits and the dropped diagonals leave about 2^(1 - 7S) of the row /
// column maxima per product term (2^-48 at S = 7, 2^-55 at S = 8); the
// double-float accumulator keeps 48 bits of the running sum.
//
// Kernel layout: CTA tile 128 x 64, K staged 32 at a time (SWIZZLE_64B TMA
// boxes; 2 stages x (8 tiles of A + 8 tiles of B) = 2 x 96 KB), 512 TMEM
// columns (8 diagonals x 64).  Warps 0-7: epilogue (TMEM lane quarter
// w % 4, column half w / 4); warp 8: TMEM allocation + MMA issue (one
// thread); warp 9: TMA producer (one thread).  Every mbarrier wait is
// bounded; a wait that gives up sets *err and the roles stop issuing work.
//
// Two epilogues: the back-transformation writes C = 2^(ea + eb) (A B); the
// tile update of step s (Sec. 3.3, Z <- Y - T X) applies, per row i (tile
// row r) and column j, Y_ij <- 2^dy[r, j] Y_ij - 2^(ea_i + eb_j + dx[r, j])
// (A~ B~)_ij and merges |Y_ij| into the column maximum of segment (r, j)
// (shared-memory maxima per output tile, one global atomicMax per (r, j)
// and tile, before the CTA takes its next tile).
#include <math.h>

#include <algorithm>
#include <mutex>

#include "split_common.cuh"

namespace evec {

constexpr int kTN = 64;
constexpr int kStageA = kTM * kTK * 2;             // 8 KB per slice tile
constexpr int kStageB = kTN * kTK * 2;             // 4 KB per slice tile
constexpr int kStageBytes = kSplitMaxS * (kStageA + kStageB);
constexpr int kChunkStages = 16;                   // 512 of K per exact drain
constexpr int kSplitThreads = 320;

// stage buffers, barriers, then the update epilogue's tables: column maxima
// red[12][64] (u64), scale exponents sdx / sdy [12][64] and eb [64] (int)
size_t split_smem_bytes() {
    return 1024 + 2 * (size_t)kStageBytes + 128 + 12 * 64 * 8 + 2 * 12 * 64 * 4 + 64 * 4;
}

// ---------------------------------------------------------------------------
// slicing kernels
// ---------------------------------------------------------------------------

// row maxima of the column-major M x K matrix A (bit patterns, atomicMax),
// kc columns per CTA row
__global__ void k_row_max(const double *__restrict__ A, int64_t lda, int M, int K, int kc,
                          unsigned long long *__restrict__ rowmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int k0 = blockIdx.y * kc, k1 = min(K, k0 + kc);
    long long b = 0;
    for (int k = k0; k < k1; k++) b = max(b, abs_bits(A[i + (int64_t)k * lda]));
    if (b) atomicMax(&rowmax[i], (unsigned long long)b);
}

// A slices: S x [Mpad][Kpad] BF16, K contiguous; 32 rows x 64 K per CTA,
// transposed through shared memory (reads coalesced along rows, writes
// along K); padding rows / columns are written as zeros
__global__ void __launch_bounds__(256) k_slice_rows(const double *__restrict__ A, int64_t lda,
                                                    int M, int K, int S,
                                                    const unsigned long long *__restrict__ rowmax,
                                                    __nv_bfloat16 *__restrict__ out, int Mpad,
                                                    int Kpad, int *__restrict__ ea) {
    __shared__ __nv_bfloat16 sd[kSplitMaxS][32][64 + 2];
    const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
    const int tid = threadIdx.x;
    for (int e = tid; e < 32 * 64; e += 256) {
        const int r = e % 32, c = e / 32;
        const int i = i0 + r, k = k0 + c;
        int d[kSplitMaxS] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (i < M && k < K) {
            const int ex = exp_from_max(rowmax[i]);
            digits7(A[i + (int64_t)k * lda], ex, S, d);
        }
        for (int p = 0; p < S; p++) sd[p][r][c] = digit_bf16(d[p], p);
    }
    if (blockIdx.x == 0 && tid < 32 && i0 + tid < Mpad)
        ea[i0 + tid] = (i0 + tid < M) ? exp_from_max(rowmax[i0 + tid]) : 0;
    __syncthreads();
    for (int e = tid; e < 32 * 64; e += 256) {
        const int r = e / 64, c = e % 64;
        const int i = i0 + r, k = k0 + c;
        if (i < Mpad && k < Kpad)
            for (int p = 0; p < S; p++)
                out[((size_t)p * Mpad + i) * Kpad + k] = sd[p][r][c];
    }
}

// B slices from the columns of the column-major K x N matrix B:
// S x [Npad][Kpad] BF16 (column j's K entries contiguous); one warp per
// column for the maximum, then one thread per (j, k)
__global__ void k_col_max(const double *__restrict__ B, int64_t ldb, int K, int N,
                          unsigned long long *__restrict__ colmax) {
    const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (j >= N) return;
    long long b = 0;
    for (int k = lane; k < K; k += 32) b = max(b, abs_bits(B[k + (int64_t)j * ldb]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if (lane == 0) colmax[j] = (unsigned long long)b;
}

__global__ void k_slice_cols(const double *__restrict__ B, int64_t ldb, int K, int N, int S,
                             const unsigned long long *__restrict__ colmax,
                             __nv_bfloat16 *__restrict__ out, int Npad, int Kpad,
                             int *__restrict__ eb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (k >= Kpad) return;
    int d[kSplitMaxS] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (j < N && k < K) digits7(B[k + (int64_t)j * ldb], exp_from_max(colmax[j]), S, d);
    for (int p = 0; p < S; p++) out[((size_t)p * Npad + j) * Kpad + k] = digit_bf16(d[p], p);
    if (k == 0) eb[j] = (j < N) ? exp_from_max(colmax[j]) : 0;
}

// ---------------------------------------------------------------------------
// tcgen05 GEMM
// ---------------------------------------------------------------------------

struct SplitUpd {
    const int32_t *row_tile;     // global row -> tile index
    const int32_t *dx, *dy;      // [ntiles][m] scale exponents of the step
    unsigned long long *nu;      // [ntiles][m] column maxima (bit patterns)
    int64_t m;                   // row length of the segment arrays
    int col0;                    // global column of local column 0
    int acc;                     // plain product: 0 C = P, +1 C += P, -1 C -= P
    int64_t zstride;             // plain product split over K (gridDim.z > 1):
                                 // CTA z writes its partial product at C + z zstride
};
constexpr int kMaxSlots = 12;    // tile rows met by one 128-row CTA tile (tiles >= 15 rows)

// barrier 1 over the 256 threads of the epilogue warps, returning the AND of
// their predicates
__device__ __forceinline__ bool epi_bar_and(bool p) {
    int r;
    asm volatile(
        "{\n.reg .pred pi, po;\nsetp.ne.b32 pi, %1, 0;\n"
        "bar.red.and.pred po, 1, 256, pi;\nselp.b32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((int)p)
        : "memory");
    return r != 0;
}

// C[i, j] (FP64, column-major, rows < M, cols < N) = 2^(ea_i + eb_j) *
// sum_k A~_ik B~_kj over k < K (kend[N tile], or kuni when kend is null);
// with UPD the tile-update epilogue instead.  A slice p of this product
// starts at row aRow0 + p * aMpad of the A tensor map.
template <bool UPD>
__global__ void __launch_bounds__(kSplitThreads, 1)
    k_split_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 int S, int M, int N, int aRow0, int aMpad, int Npad, const int *__restrict__ kend,
                 int kuni, const int *__restrict__ ea, const int *__restrict__ eb,
                 double *__restrict__ C, int64_t ldc, SplitUpd upd, int *err, int ntiles_n,
                 int gw, int mtiles) {
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(base + 2 * kStageBytes);
    // bars[0..1] full, bars[2..3] empty, bars[4] acc_full, bars[5] acc_empty
    uint32_t *tmem_holder = (uint32_t *)(bars + 8);
    unsigned long long *red = (unsigned long long *)(bars + 16);   // [kMaxSlots][kTN]
    int *sdx = (int *)(red + kMaxSlots * kTN);                        // [kMaxSlots][kTN]
    int *sdy = sdx + kMaxSlots * kTN;                                 // [kMaxSlots][kTN]
    int *seb = sdy + kMaxSlots * kTN;                                 // [kTN]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Tile order: groups of gw column tiles; within a group the row bands
    // in turn, the group's column tiles fastest, so the tiles in flight at
    // one time cover about (148 / gw) row bands x gw column tiles and share
    // their operand slices through L2; heaviest column tiles first.  A CTA
    // takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... (persistent: the
    // next tile's loads and MMAs run while the epilogue writes the last
    // one's results); the tile-update epilogue (UPD) merges each tile's
    // column maxima before it takes the next tile.
    const int ntiles_total = mtiles * ntiles_n;
    auto tile_of = [&](int t, int &m0_, int &n0_, int &nt_) {
        const int per = gw * mtiles;
        const int grp = t / per;
        const int rem = t - grp * per;
        const int w = min(gw, ntiles_n - grp * gw);
        nt_ = ntiles_n - 1 - (grp * gw + rem % w);
        n0_ = nt_ * kTN;
        m0_ = (rem / w) * kTM;
    };
    // the K steps of a tile for this CTA: all of them, or its share of a K
    // split over gridDim.z
    auto ksteps = [&](int nt_, int &s0_) {
        const int nst_all = (kend ? kend[nt_] : kuni) / kTK;
        const int zper = ((int)gridDim.z > 1) ? (nst_all + (int)gridDim.z - 1) / (int)gridDim.z
                                             : nst_all;
        s0_ = (int)blockIdx.z * zper;
        return max(0, min(nst_all, s0_ + zper) - s0_);
    };
    if (!UPD && gridDim.z > 1) C += (int64_t)blockIdx.z * upd.zstride;
    if (UPD)
        for (int i = tid; i < kMaxSlots * kTN; i += kSplitThreads) red[i] = 0ull;

    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tmem_holder)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < 4; b++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&bars[b])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&bars[4])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&bars[5])), "r"(8));
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("fence.proxy.async.shared::cta;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_holder;

    if (warp == 9) {
        if (lane == 0) {   // TMA producer
            int gi = 0;   // K steps issued over all of this CTA's tiles
            bool run = true;
            for (int t = (int)blockIdx.x; run && t < ntiles_total; t += (int)gridDim.x) {
                int m0, n0, nt, s0;
                tile_of(t, m0, n0, nt);
                const int nst = ksteps(nt, s0);
            for (int it = 0; it < nst; it++, gi++) {
                const int st = gi & 1;
                const uint32_t ph = (uint32_t)(gi >> 1) & 1;
                if (!mbar_wait(saddr(&bars[2 + st]), ph ^ 1, err)) {
                    run = false;
                    break;
                }
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                 saddr(&bars[st])),
                             "r"(S * (kStageA + kStageB)));
                unsigned char *sa = base + st * kStageBytes;
                unsigned char *sb = sa + kSplitMaxS * kStageA;
                for (int p = 0; p < S; p++)
                    tma2d(saddr(sa + p * kStageA), &tmA, (s0 + it) * kTK, aRow0 + p * aMpad + m0,
                          saddr(&bars[st]));
                // B as [column half c][slice q] boxes of 32 rows, so the
                // slices of one half lie one after another
                for (int c = 0; c < 2; c++)
                    for (int q = 0; q < S; q++)
                        tma2d(saddr(sb + (c * kSplitMaxS + q) * (kStageB / 2)), &tmB,
                              (s0 + it) * kTK,
                              q * Npad + n0 + c * 32, saddr(&bars[st]));
            }
            }
            // the copies of the last stages have landed before the CTA ends
            for (int it = max(0, gi - 2); it < gi; it++)
                mbar_wait(saddr(&bars[it & 1]), (uint32_t)(it >> 1) & 1, err);
        }
    } else if (warp == 8) {
        if (lane == 0) {   // MMA issue
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTM >> 4) << 24);
            int gi = 0, gc = 0;   // K steps and accumulator chunks over all tiles
            bool run = true;
            for (int t = (int)blockIdx.x; run && t < ntiles_total; t += (int)gridDim.x) {
                int m0, n0, nt, s0;
                tile_of(t, m0, n0, nt);
                const int nst = ksteps(nt, s0);
            for (int it = 0; it < nst; it++, gi++) {
                const int st = gi & 1;
                const int sic = it % kChunkStages;
                // before a chunk overwrites TMEM, the epilogue has drained
                // the previous one (of this tile or the last)
                if (sic == 0 && gc > 0 &&
                    !mbar_wait(saddr(&bars[5]), (uint32_t)(gc - 1) & 1, err)) {
                    run = false;
                    break;
                }
                if (!mbar_wait(saddr(&bars[st]), (uint32_t)(gi >> 1) & 1, err)) {
                    run = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = saddr(base + st * kStageBytes);
                const uint32_t sb = sa + kSplitMaxS * kStageA;
                // One MMA of A_p against the S - p slices of a column half
                // (N = 32 (S - p)), written at column 32 p of the half's 256,
                // adds A_p B_q to diagonal p + q for every q: 2 S wide MMAs
                // per K step instead of S (S + 1) narrow ones (narrow MMAs
                // complete one at a time).
                for (int kk = 0; kk < kTK / 16; kk++)
                    for (int hf = 0; hf < 2; hf++) {
                        const uint64_t bd =
                            desc_sw64(sb + hf * kSplitMaxS * (kStageB / 2) + kk * 32);
                        for (int p = 0; p < S; p++) {
                            const uint32_t id = idesc | ((uint32_t)(((S - p) * 32) >> 3) << 17);
                            const uint64_t ad = desc_sw64(sa + p * kStageA + kk * 32);
                            // the first K step of a chunk overwrites (p = 0
                            // covers every diagonal of the half)
                            const int acc = (sic == 0 && kk == 0 && p == 0) ? 0 : 1;
                            asm volatile(
                                "{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n" ::"r"(
                                    tmem + (uint32_t)(hf * 256 + p * 32)),
                                "l"(ad), "l"(bd), "r"(id), "r"(acc));
                        }
                    }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        saddr(&bars[2 + st])));
                if (sic == kChunkStages - 1 || it == nst - 1) {
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
                        "[%0];" ::"r"(saddr(&bars[4])));
                    gc++;
                }
            }
            }
        }
    } else {   // epilogue warps 0-7
        const int quarter = warp & 3, half = warp >> 2;
        const int cb0 = half * 32;
        int gc = 0;   // accumulator chunks drained over all tiles
        bool ok = true;
        for (int t = (int)blockIdx.x; ok && t < ntiles_total; t += (int)gridDim.x) {
        int m0, n0, nt, s0;
        tile_of(t, m0, n0, nt);
        const int chunks = (ksteps(nt, s0) + kChunkStages - 1) / kChunkStages;
        const int row = m0 + quarter * 32 + lane;
        if (UPD) {   // exponent tables of this CTA's (tile row, column) pairs
            const int rlo = upd.row_tile[m0], rhi = upd.row_tile[min(m0 + kTM, M) - 1];
            const int cnt = (rhi - rlo + 1) * kTN;
            for (int i = tid; i < cnt; i += 256) {
                const int sl = i / kTN, c = i % kTN, col = n0 + c;
                int dxv = 0, dyv = kFresh;
                if (col < N) {
                    const int64_t at = (int64_t)(rlo + sl) * upd.m + upd.col0 + col;
                    dxv = upd.dx[at];
                    dyv = upd.dy[at];
                }
                sdx[i] = dxv;
                sdy[i] = dyv;
            }
            if (tid < kTN) seb[tid] = (n0 + tid < N) ? eb[n0 + tid] : 0;
            asm volatile("bar.sync 1, 256;" ::: "memory");
        }
        float hi[32], lo[32];
#pragma unroll
        for (int j = 0; j < 32; j++) { hi[j] = 0.0f; lo[j] = 0.0f; }
        for (int c = 0; c < chunks && ok; c++, gc++) {
            ok = mbar_wait(saddr(&bars[4]), (uint32_t)gc & 1, err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int cb = 0; cb < 4; cb++) {
                uint32_t v[kSplitMaxS][8];
#pragma unroll
                for (int dgl = 0; dgl < kSplitMaxS; dgl++) {
                    if (dgl < S) {
                        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) +
                                            (uint32_t)(half * 256 + dgl * 32 + cb * 8);
                        TMEM_LD8(ta, v[dgl]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; j++) v[dgl][j] = 0u;
                    }
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    // diagonal D is below about 2^(-7D) of diagonal 0:
                    // diagonals 5.. are summed in FP32 (rounding near 2^-58
                    // of the leading term), diagonals 0-4 and that sum are
                    // added to the double-float accumulator one by one
                    float small = 0.0f;
#pragma unroll
                    for (int dgl = kSplitMaxS - 1; dgl >= 5; dgl--)
                        small += __uint_as_float(v[dgl][j]);
                    const int jj = cb * 8 + j;
#pragma unroll
                    for (int dgl = 0; dgl < 5; dgl++)
                        df_add(hi[jj], lo[jj], __uint_as_float(v[dgl][j]));
                    df_add(hi[jj], lo[jj], small);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&bars[5])));
        }
        if (!UPD && row < M) {
            const int er = ea[row];
            if (upd.acc == 0) {
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const int col = n0 + cb0 + j;
                    if (col < N)
                        C[row + (int64_t)col * ldc] = df_to_double(hi[j], lo[j], er + eb[col]);
                }
            } else {   // C +- P: eight old values loaded, then eight updates
#pragma unroll
                for (int g = 0; g < 4; g++) {
                    double oldv[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int col = n0 + cb0 + g * 8 + q;
                        oldv[q] = col < N ? C[row + (int64_t)col * ldc] : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int j = g * 8 + q, col = n0 + cb0 + j;
                        if (col >= N) break;
                        const double p = df_to_double(hi[j], lo[j], er + eb[col]);
                        C[row + (int64_t)col * ldc] = upd.acc > 0 ? oldv[q] + p : oldv[q] - p;
                    }
                }
            }
        }
        if (UPD) {
            // rows of one tile row r are a contiguous run of lanes: the
            // column maximum of each run is a segmented suffix max over
            // shuffles, and the run's first lane merges it into red[]
            const bool rv = row < M;
            const int slot = rv ? upd.row_tile[row] - upd.row_tile[m0] : kMaxSlots;
            const int er = rv ? ea[row] : 0;
            unsigned same = 0;   // bit k: lane + 2^k lies in the same run
#pragma unroll
            for (int k = 0; k < 5; k++) {
                const int o = __shfl_down_sync(0xffffffffu, slot, 1 << k);
                if (lane + (1 << k) < 32 && o == slot) same |= 1u << k;
            }
            const int up = __shfl_up_sync(0xffffffffu, slot, 1);
            const bool head = rv && (lane == 0 || up != slot);
            const int sbase = rv ? slot * kTN : 0;
            double *crow = C + row + (int64_t)upd.col0 * ldc;
#pragma unroll
            for (int g = 0; g < 4; g++) {   // 8 columns: loads first, then the updates
                double oldv[8];
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int c = cb0 + g * 8 + q;
                    oldv[q] = 0.0;
                    if (rv && n0 + c < N && sdy[sbase + c] != kFresh)
                        oldv[q] = crow[(int64_t)(n0 + c) * ldc];
                }
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int j = g * 8 + q, c = cb0 + j;
                    if (n0 + c >= N) break;   // warp-uniform
                    unsigned long long b = 0ull;
                    if (rv) {
                        const int dyv = sdy[sbase + c];
                        const double prod =
                            df_to_double(hi[j], lo[j], er + seb[c] + sdx[sbase + c]);
                        double v;
                        if (dyv == kFresh) v = -prod;
                        else if (dyv >= -1022 && dyv <= 1023)   // old 2^dy exact in the FMA
                            v = fma(oldv[q], pow2_normal(dyv), -prod);
                        else v = scale2(oldv[q], dyv) - prod;
                        crow[(int64_t)(n0 + c) * ldc] = v;
                        b = (unsigned long long)abs_bits(v);
                    }
#pragma unroll
                    for (int k = 0; k < 5; k++) {
                        const unsigned long long o = __shfl_down_sync(0xffffffffu, b, 1 << k);
                        if ((same >> k) & 1u) b = max(b, o);
                    }
                    if (head && b) atomicMax(&red[slot * kTN + c], b);
                }
            }
            // the tile's column maxima into the segment maxima, red[] cleared
            // for the next tile of this CTA; the eight warps agree on ok, so
            // a warp whose wait gave up never leaves the others at a barrier
            ok = epi_bar_and(ok);
            const int r0 = upd.row_tile[m0];
            for (int i = tid; i < kMaxSlots * kTN; i += 256) {
                const unsigned long long v = red[i];
                const int col = n0 + i % kTN;
                if (v != 0ull && col < N)
                    atomicMax(&upd.nu[(int64_t)(r0 + i / kTN) * upd.m + upd.col0 + col], v);
                red[i] = 0ull;
            }
            ok = epi_bar_and(ok);
        }
        }   // tiles
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 8)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

bool get_encoder() {
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        else
            cudaGetLastError();
    });
    return g_encode != nullptr;
}

bool make_map(CUtensorMap *tm, void *ptr, int rows, int kpad, int box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int split_pad_m(int M) { return (M + kTM - 1) / kTM * kTM; }
int split_pad_n(int N) { return (N + kTN - 1) / kTN * kTN; }
int split_pad_k(int K) { return (K + 63) / 64 * 64; }
// K columns of the panel slices of the split tile updates: 64 for the
// panel-resident kernel (K <= 64), else the largest tile rounded up to 64
int split_update_kp(int k) { return k <= 64 ? 64 : (k + 63) / 64 * 64; }

// Slices of A (rows) and B (columns) into the caller's buffers, then the
// GEMM.  Buffers: sa [S][Mpad][Kpad], sb [S][Npad][Kpad] BF16; rowmax
// [Mpad], colmax [Npad] u64; ea [Mpad], eb [Npad] int; kend [N tiles]
// (device, multiples of 32, <= Kpad) or null for the whole K range.  Returns cudaErrorInvalidValue when
// a tensor map cannot be encoded.
// C = A B split in two parts, so that B's columns can be taken in chunks:
// the row slices of A (once), then per chunk the column slices of B and
// the product.
cudaError_t split_gemm_rows(const double *A, int64_t lda, int M, int K, int S,
                            __nv_bfloat16 *sa, unsigned long long *rowmax, int *ea,
                            cudaStream_t st) {
    const int Mpad = split_pad_m(M), Kpad = split_pad_k(K);
    cudaMemsetAsync(rowmax, 0, sizeof(unsigned long long) * Mpad, st);
    // short rows (the window products, K <= 256): chunks of 32 columns, so
    // that a few hundred rows still fill the GPU; long rows: 256
    const int kc = K <= 512 ? 32 : 256;
    k_row_max<<<dim3((M + 255) / 256, (K + kc - 1) / kc), 256, 0, st>>>(A, lda, M, K, kc,
                                                                        rowmax);
    k_slice_rows<<<dim3(Kpad / 64, Mpad / 32), 256, 0, st>>>(A, lda, M, K, S, rowmax, sa, Mpad,
                                                              Kpad, ea);
    return cudaGetLastError();
}

// Column slices of the K x N matrix B into sb [S][Npad][Kpad] (Npad >=
// split_pad_n(N), a multiple of kTN: a larger Npad lets the same slices
// serve as the row slices of B^T with Npad = split_pad_m(N)), exponents eb.
cudaError_t split_slice_cols(const double *B, int64_t ldb, int K, int N, int S, int Npad,
                             __nv_bfloat16 *sb, unsigned long long *colmax, int *eb,
                             cudaStream_t st) {
    const int Kpad = split_pad_k(K);
    k_col_max<<<(N + 7) / 8, 256, 0, st>>>(B, ldb, K, N, colmax);
    k_slice_cols<<<dim3((Kpad + 255) / 256, Npad), 256, 0, st>>>(B, ldb, K, N, S, colmax, sb,
                                                                  Npad, Kpad, eb);
    return cudaGetLastError();
}

// C (+ or -)= sum over z of the ksplit partial products at part + z M N
// (leading dimension M), summed in FP64 in the order of z.
__global__ void __launch_bounds__(256)
    k_sum_partials(const double *__restrict__ part, int ksplit, int M, int N,
                   double *__restrict__ C, int64_t ldc, int acc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t MN = (int64_t)M * N;
    if (e >= MN) return;
    double v = part[e];
    for (int z = 1; z < ksplit; z++) v += part[(int64_t)z * MN + e];
    const int64_t i = e % M, j = e / M;
    double *c = C + i + j * ldc;
    *c = acc == 0 ? v : (acc > 0 ? *c + v : *c - v);
}

// C = A B (acc 0), C += A B (+1) or C -= A B (-1) from the slices of A (sa
// [S][Mpad][Kpad], exponents ea) and of B (sb [S][Npad][Kpad], exponents
// eb), over K < kend[N tile] (or the whole padded K when kend is null).
// ksplit > 1 (kend null): the K steps are shared by ksplit CTAs per output
// tile, each writing its partial product to part (ksplit M N doubles),
// then summed into C -- for products with few output tiles and a long K.
cudaError_t split_gemm_sliced(const __nv_bfloat16 *sa, int Mpad, const __nv_bfloat16 *sb,
                              int Npad, int M, int N, int K, int S, const int *kend,
                              const int *ea, const int *eb, double *C, int64_t ldc, int *err,
                              cudaStream_t st, int acc, int ksplit, double *part) {
    if (!get_encoder()) return cudaErrorInvalidValue;
    const int Kpad = split_pad_k(K);
    CUtensorMap tmA, tmB;
    if (!make_map(&tmA, (void *)sa, S * Mpad, Kpad, kTM) ||
        !make_map(&tmB, (void *)sb, S * Npad, Kpad, 32))
        return cudaErrorInvalidValue;
    const size_t smem = split_smem_bytes();
    cudaFuncSetAttribute(k_split_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (ksplit > 1 && (kend || !part)) return cudaErrorInvalidValue;
    SplitUpd none = {};
    none.acc = ksplit > 1 ? 0 : acc;
    none.zstride = (int64_t)M * N;
    // column tiles per group: gw about sqrt(CTAs in flight x (row band
    // bytes / column tile bytes)), so one wave's row bands and column tiles
    // cost about the same DRAM traffic (a band of Q's slices holds twice
    // the rows of a column tile of Y's)
    const int ntn = split_pad_n(N) / kTN, mtn = split_pad_m(M) / kTM;
    int nsm = 148, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        nsm = 148;
    }
    const int gw = std::max(1, std::min(ntn, (int)lround(sqrt(2.0 * nsm))));
    if (ksplit > 1) {
        k_split_gemm<false><<<dim3(ntn * mtn, 1, ksplit), kSplitThreads, smem, st>>>(
            tmA, tmB, S, M, N, 0, Mpad, Npad, nullptr, Kpad, ea, eb, part, M, none, err, ntn, gw,
            mtn);
        const int64_t MN = (int64_t)M * N;
        k_sum_partials<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(part, ksplit, M, N, C, ldc,
                                                                     acc);
        return cudaGetLastError();
    }
    // Products with one or two K steps (the rank-32 updates) run persistent,
    // one CTA per SM taking every gridDim.x-th tile, so that a CTA's fixed
    // cost (TMEM allocation, barrier set-up, the first loads) is paid once
    // and the next tile's MMAs run under the last one's epilogue: the
    // Hessenberg updates 108 -> 98 ms at n = 4096.  Longer products keep one
    // CTA per tile: there the scheduler hands each free SM the next tile, so
    // the tiles in flight stay a contiguous window that shares its operand
    // slices through L2 (persistent CTAs drift apart; the n = 16384
    // back-transformation went from 110 to 119 ms).
    const int grid = Kpad <= 64 ? std::min(ntn * mtn, nsm) : ntn * mtn;
    k_split_gemm<false><<<grid, kSplitThreads, smem, st>>>(
        tmA, tmB, S, M, N, 0, Mpad, Npad, kend, kend ? 0 : Kpad, ea, eb, C, ldc, none, err, ntn,
        gw, mtn);
    return cudaGetLastError();
}

cudaError_t split_gemm_cols(const double *B, int64_t ldb, int M, int N, int K, int S,
                            const int *kend, double *C, int64_t ldc, const __nv_bfloat16 *sa,
                            __nv_bfloat16 *sb, unsigned long long *colmax, const int *ea,
                            int *eb, int *err, cudaStream_t st) {
    if (!get_encoder()) return cudaErrorInvalidValue;
    const int Mpad = split_pad_m(M), Npad = split_pad_n(N);
    cudaError_t e = split_slice_cols(B, ldb, K, N, S, Npad, sb, colmax, eb, st);
    if (e != cudaSuccess) return e;
    return split_gemm_sliced(sa, Mpad, sb, Npad, M, N, K, S, kend, ea, eb, C, ldc, err, st, 0, 1,
                             nullptr);
}

cudaError_t launch_split_gemm(const double *A, int64_t lda, const double *B, int64_t ldb, int M,
                              int N, int K, int S, const int *kend, double *C, int64_t ldc,
                              __nv_bfloat16 *sa, __nv_bfloat16 *sb, unsigned long long *rowmax,
                              unsigned long long *colmax, int *ea, int *eb, int *err,
                              cudaStream_t st) {
    if (!get_encoder()) return cudaErrorInvalidValue;
    cudaError_t e = split_gemm_rows(A, lda, M, K, S, sa, rowmax, ea, st);
    if (e != cudaSuccess) return e;
    return split_gemm_cols(B, ldb, M, N, K, S, kend, C, ldc, sa, sb, colmax, ea, eb, err, st);
}

// ---------------------------------------------------------------------------
// tile updates in split precision
// ---------------------------------------------------------------------------

// Slices of every panel T[0:t0_s, tile s] (s >= 1) at once: panel s holds
// S slices of Mpad_s = roundup(t0_s, 128) rows x Kp columns starting at row
// prow0[s] of the buffer; row exponents (per panel row) at pea[s] + i.
// One CTA per 32 rows of one panel; 256 threads.
__global__ void __launch_bounds__(256)
    k_slice_panels(const double *__restrict__ T, int64_t ldt, const double *__restrict__ T2,
                   int64_t ldt2, const int32_t *__restrict__ tstart,
                   const int32_t *__restrict__ prow0, const int32_t *__restrict__ pea, int S,
                   int Kp, __nv_bfloat16 *__restrict__ out, int *__restrict__ ea) {
    const int s = blockIdx.y + 1;
    const int t0 = tstart[s], ts = tstart[s + 1] - t0;
    // panel row i: T[i, tile s], then (pencils) T2[i, tile s]
    const int kw = T2 ? 2 * ts : ts;
    auto at = [&](int i, int k) -> double {
        return k < ts ? T[i + (int64_t)(t0 + k) * ldt] : T2[i + (int64_t)(t0 + k - ts) * ldt2];
    };
    const int mpad = (t0 + kTM - 1) / kTM * kTM;
    const int i0 = blockIdx.x * 32;
    if (i0 >= mpad) return;
    __shared__ long long rm[32][9];
    __shared__ int rex[32];
    __shared__ __nv_bfloat16 sd[kSplitMaxS][32][64 + 2];
    const int tid = threadIdx.x;
    {   // row maxima over the panel's columns: 8 threads per row
        const int r = tid / 8, part = tid % 8;
        const int i = i0 + r;
        long long b = 0;
        if (i < t0)
            for (int k = part; k < kw; k += 8) b = max(b, abs_bits(at(i, k)));
        rm[r][part] = b;
    }
    __syncthreads();
    if (tid < 32) {
        long long b = 0;
        for (int q = 0; q < 8; q++) b = max(b, rm[tid][q]);
        rex[tid] = exp_from_max((unsigned long long)b);
        ea[pea[s] + i0 + tid] = rex[tid];
    }
    __syncthreads();
    for (int kh = 0; kh < Kp; kh += 64) {   // 64 columns at a time
        for (int e = tid; e < 32 * 64; e += 256) {
            const int r = e % 32, c = e / 32;
            const int i = i0 + r, k = kh + c;
            int d[kSplitMaxS] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (i < t0 && k < kw) digits7(at(i, k), rex[r], S, d);
            for (int p = 0; p < S; p++) sd[p][r][c] = digit_bf16(d[p], p);
        }
        __syncthreads();
        for (int e = tid; e < 32 * 64; e += 256) {
            const int r = e / 64, c = e % 64;
            for (int p = 0; p < S; p++)
                out[((size_t)prow0[s] + (size_t)p * mpad + i0 + r) * Kp + kh + c] = sd[p][r][c];
        }
        __syncthreads();
    }
}

// Once per call: slice every panel of T (pencils: of [S T], K = 2 |tile|);
// encode the two tensor maps.
cudaError_t split_update_prepare(const double *T, int64_t ldt, const double *T2, int64_t ldt2,
                                 int n, int ntiles, int maxtile,
                                 const int32_t *tstart_d, const int32_t *prow0_d,
                                 const int32_t *pea_d, int total_rows, int S, int m,
                                 __nv_bfloat16 *panels, int *ea_panels, __nv_bfloat16 *sb,
                                 SplitUpdateCtx *ctx, cudaStream_t st) {
    if (!get_encoder()) return cudaErrorInvalidValue;
    ctx->S = S;
    ctx->Kp = split_update_kp(T2 ? 2 * maxtile : maxtile);
    ctx->Npad = split_pad_n(m);
    if (ntiles > 1) {
        const int maxblocks = split_pad_m(n) / 32;   // >= roundup(t0_s, 128) / 32 for all s
        k_slice_panels<<<dim3(maxblocks, ntiles - 1), 256, 0, st>>>(
            T, ldt, T2, ldt2, tstart_d, prow0_d, pea_d, S, ctx->Kp, panels, ea_panels);
    }
    if (!make_map(&ctx->tmA, panels, total_rows > 0 ? total_rows : kTM, ctx->Kp, kTM) ||
        !make_map(&ctx->tmB32, sb, S * ctx->Npad, ctx->Kp, 32))
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// Step s: slice X_s = Y[t0_s:t1_s, col0:m], then Y_r -= T_rs X_s for all rows
// above tile s with the robust epilogue.
// rhs (pencils): the right-hand side [beta X_s; -(alpha X_s)] (2 |tile| rows,
// ld ldr) replaces X_s = Y[t0 : t0 + ts, col0 : m].
cudaError_t split_update_step(const SplitUpdateCtx &ctx, int t0, int ts, int prow0, int pea,
                              int col0, int m, double *Y, int64_t ldy, const int *ea_panels,
                              __nv_bfloat16 *sb, unsigned long long *colmax, int *eb,
                              const int32_t *row_tile, const int32_t *dx, const int32_t *dy,
                              double *seg_nu, int *err, cudaStream_t st, const double *rhs,
                              int64_t ldr) {
    const int N = m - col0;
    if (N <= 0 || t0 <= 0) return cudaSuccess;
    const double *B = rhs ? rhs : Y + t0 + (int64_t)col0 * ldy;
    const int64_t ldb = rhs ? ldr : ldy;
    const int K = rhs ? 2 * ts : ts;
    k_col_max<<<(N + 7) / 8, 256, 0, st>>>(B, ldb, K, N, colmax);
    k_slice_cols<<<dim3((ctx.Kp + 255) / 256, split_pad_n(N)), 256, 0, st>>>(
        B, ldb, K, N, ctx.S, colmax, sb, ctx.Npad, ctx.Kp, eb);
    const int mpad = (t0 + kTM - 1) / kTM * kTM;
    const size_t smem = split_smem_bytes();
    cudaFuncSetAttribute(k_split_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    SplitUpd upd = {};
    upd.row_tile = row_tile;
    upd.dx = dx;
    upd.dy = dy;
    upd.nu = (unsigned long long *)seg_nu;
    upd.m = m;
    upd.col0 = col0;
    const int ntn = split_pad_n(N) / kTN;
    // persistent, one CTA per SM over every gridDim.x-th tile: once a tile's
    // accumulators are drained, the next tile's loads and MMAs run under the
    // rest of its epilogue (the FP64 read-modify-write of Y and the column
    // maxima), which with one CTA per tile left the tensor pipe idle
    int nsm = 148, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        nsm = 148;
    }
    const int tiles = ntn * (mpad / kTM);
    k_split_gemm<true><<<std::min(tiles, nsm), kSplitThreads, smem, st>>>(
        ctx.tmA, ctx.tmB32, ctx.S, t0, N, prow0, mpad, ctx.Npad, nullptr, (K + kTK - 1) / kTK * kTK,
        ea_panels + pea, eb, Y, ldy, upd, err, ntn, ntn, mpad / kTM);
    return cudaGetLastError();
}

}  // namespace evec
