// k_split.cu -- split-precision FP64 GEMM on the BF16 tensor cores (tcgen05).
//
// C = A B with FP64 operands, computed as in the Ozaki scheme (error-free
// splitting of the operands into small-integer slices whose products are
// exact in FP32): every row of A is normalised by a power of two 2^ea_i so
// |a~| < 1/2, every column of B by 2^eb_j; each normalised value is written
// in balanced base 2^7 with S digits, x~ = sum_p d_p 2^(-7p), |d_p| <= 64,
// and slice p holds d_p 2^(-7p) as an exact BF16 number.  For every digit
// diagonal D = p + q (p + q <= S + 1 in 1-based terms) the products
// A_p B_q are multiples of 2^(-7D) bounded by 2^12 2^(-7D); a diagonal
// has at most 7 terms, so its sum over K = 512 stays below 2^24 units and
// is exact in the FP32 tensor-core accumulator.  Each diagonal has its own
// TMEM accumulator; every 512 of K the epilogue warps drain them into a
// double-float (hi, lo) FP32 accumulator, and at the end
// C_ij = 2^(ea_i + eb_j) (hi + lo) in FP64.  Truncation after S = 7
// slices leaves 2^-49 of the row / column maxima; the double-float sum
// keeps 48 bits.
//
// Kernel layout: CTA tile 128 x 64, K staged 32 at a time (SWIZZLE_64B TMA
// boxes; 2 stages x (S tiles of A + S tiles of B) = 2 x 84 KB), 512 TMEM
// columns (7 diagonals x 64).  Warps 0-7: epilogue (TMEM lane quarter
// w % 4, column half w / 4); warp 8: TMEM allocation + MMA issue (one
// thread); warp 9: TMA producer (one thread).  Every mbarrier wait is
// bounded; a wait that gives up sets *err and the roles stop issuing work.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "evec_internal.cuh"

namespace evec {

constexpr int kSplitMaxS = 7;
constexpr int kTM = 128, kTN = 64, kTK = 32;
constexpr int kStageA = kTM * kTK * 2;             // 8 KB per slice tile
constexpr int kStageB = kTN * kTK * 2;             // 4 KB per slice tile
constexpr int kStageBytes = kSplitMaxS * (kStageA + kStageB);
constexpr int kChunkStages = 16;                   // 512 of K per exact drain
constexpr int kSplitThreads = 320;
constexpr int kTmemCols = 512;
constexpr long kWaitLimit = 1L << 26;

size_t split_smem_bytes() { return 1024 + 2 * (size_t)kStageBytes + 128; }

// ---------------------------------------------------------------------------
// slicing
// ---------------------------------------------------------------------------

// balanced base-2^7 digits of x * 2^-e (|x| < 2^(e-1)), most significant
// first, by integer arithmetic on the IEEE encoding
__device__ __forceinline__ void digits7(double x, int e, int S, int *d) {
    const long long bits = __double_as_longlong(x);
    const int E = (int)((bits >> 52) & 0x7ff);
    long long mant = bits & ((1LL << 52) - 1);
    if (E) mant |= (1LL << 52);
    const int shift = (E ? E : 1) - 1075 + 7 * S - e;   // x 2^(7S - e) = mant 2^shift
    long long I;
    if (mant == 0) I = 0;
    else if (shift >= 0) I = mant << shift;             // |I| < 2^(7S-1): no overflow
    else if (shift > -62) I = (mant + (1LL << (-shift - 1))) >> (-shift);
    else I = 0;
    if (bits < 0) I = -I;
    for (int p = S - 1; p >= 1; p--) {
        long long r = I & 127;
        if (r >= 64) r -= 128;
        d[p] = (int)r;
        I = (I - r) >> 7;
    }
    d[0] = (int)I;                                      // |d_0| <= 64
}

__device__ __forceinline__ __nv_bfloat16 digit_bf16(int d, int p) {
    // d 2^(-7(p+1)) is exact in BF16 (|d| <= 64)
    return __float2bfloat16_rn((float)d * __int_as_float((127 - 7 * (p + 1)) << 23));
}

__device__ __forceinline__ int exp_from_max(unsigned long long mb) {
    // |x| <= max < 2^(ilog2(max) + 1)  ->  e = ilog2(max) + 2 gives |x 2^-e| < 1/2
    if (mb == 0) return 0;
    return ilog2_abs(__longlong_as_double((long long)mb)) + 2;
}

// row maxima of the column-major M x K matrix A (bit patterns, atomicMax)
__global__ void k_row_max(const double *__restrict__ A, int64_t lda, int M, int K,
                          unsigned long long *__restrict__ rowmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int k0 = blockIdx.y * 256, k1 = min(K, k0 + 256);
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
        int d[kSplitMaxS] = {0, 0, 0, 0, 0, 0, 0};
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
    int d[kSplitMaxS] = {0, 0, 0, 0, 0, 0, 0};
    if (j < N && k < K) digits7(B[k + (int64_t)j * ldb], exp_from_max(colmax[j]), S, d);
    for (int p = 0; p < S; p++) out[((size_t)p * Npad + j) * Kpad + k] = digit_bf16(d[p], p);
    if (k == 0) eb[j] = (j < N) ? exp_from_max(colmax[j]) : 0;
}

// ---------------------------------------------------------------------------
// tcgen05 GEMM
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err) {
    for (long it = 0; it < kWaitLimit; it++) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
            "selp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023) == 1023 && *(volatile int *)err) return false;
    }
    atomicExch(err, 1);
    return false;
}

// K-major, 64-byte swizzle: 8-row atoms of 64 B, atoms 512 B apart
__device__ __forceinline__ uint64_t desc_sw64(uint32_t a) {
    uint64_t d = 0;
    d |= (uint64_t)((a & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

__device__ __forceinline__ void tma2d(uint32_t dst, const CUtensorMap *tm, int x, int y,
                                      uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    lo = lo + e;
    const float h2 = s + lo;
    lo = lo - (h2 - s);
    hi = h2;
}

#define TMEM_LD8(taddr, r)                                                                   \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"     \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),     \
                   "=r"(r[6]), "=r"(r[7])                                                      \
                 : "r"(taddr))

// C[i, j] (FP64, column-major, rows < M, cols < N) = 2^(ea_i + eb_j) *
// sum_k A~_ik B~_kj over k < kend[N tile]
__global__ void __launch_bounds__(kSplitThreads, 1)
    k_split_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 int S, int M, int N, int Mpad, int Npad, const int *__restrict__ kend,
                 const int *__restrict__ ea, const int *__restrict__ eb,
                 double *__restrict__ C, int64_t ldc, int *err) {
    extern __shared__ unsigned char smraw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(base + 2 * kStageBytes);
    // bars[0..1] full, bars[2..3] empty, bars[4] acc_full, bars[5] acc_empty
    uint32_t *tmem_holder = (uint32_t *)(bars + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = gridDim.x - 1 - blockIdx.x;   // heaviest column tiles first
    const int mt = blockIdx.y;
    const int n0 = nt * kTN, m0 = mt * kTM;
    const int K = kend[nt];
    const int nst = K / kTK;
    const int chunks = (nst + kChunkStages - 1) / kChunkStages;

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
            int issued = 0;
            for (int it = 0; it < nst; it++) {
                const int st = it & 1;
                const uint32_t ph = (uint32_t)(it >> 1) & 1;
                if (!mbar_wait(saddr(&bars[2 + st]), ph ^ 1, err)) break;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                 saddr(&bars[st])),
                             "r"(S * (kStageA + kStageB)));
                unsigned char *sa = base + st * kStageBytes;
                unsigned char *sb = sa + kSplitMaxS * kStageA;
                for (int p = 0; p < S; p++)
                    tma2d(saddr(sa + p * kStageA), &tmA, it * kTK, p * Mpad + m0, saddr(&bars[st]));
                for (int q = 0; q < S; q++)
                    tma2d(saddr(sb + q * kStageB), &tmB, it * kTK, q * Npad + n0, saddr(&bars[st]));
                issued = it + 1;
            }
            // the copies of the last stages have landed before the CTA ends
            for (int it = max(0, issued - 2); it < issued; it++)
                mbar_wait(saddr(&bars[it & 1]), (uint32_t)(it >> 1) & 1, err);
        }
    } else if (warp == 8) {
        if (lane == 0) {   // MMA issue
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                   ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
            for (int it = 0; it < nst; it++) {
                const int st = it & 1;
                const int c = it / kChunkStages, sic = it % kChunkStages;
                if (sic == 0 && c > 0 && !mbar_wait(saddr(&bars[5]), (uint32_t)(c - 1) & 1, err))
                    break;
                if (!mbar_wait(saddr(&bars[st]), (uint32_t)(it >> 1) & 1, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = saddr(base + st * kStageBytes);
                const uint32_t sb = sa + kSplitMaxS * kStageA;
                for (int p = 0; p < S; p++)
                    for (int q = 0; p + q < S; q++) {
                        const int dgl = p + q;
                        for (int kk = 0; kk < kTK / 16; kk++) {
                            // the first product of a diagonal in a chunk overwrites it
                            const int acc = (sic == 0 && kk == 0 && p == 0) ? 0 : 1;
                            const uint64_t ad = desc_sw64(sa + p * kStageA + kk * 32);
                            const uint64_t bd = desc_sw64(sb + q * kStageB + kk * 32);
                            asm volatile(
                                "{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n" ::"r"(
                                    tmem + dgl * kTN),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                        }
                    }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        saddr(&bars[2 + st])));
                if (sic == kChunkStages - 1 || it == nst - 1)
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
                        "[%0];" ::"r"(saddr(&bars[4])));
            }
        }
    } else {   // epilogue warps 0-7
        const int quarter = warp & 3, half = warp >> 2;
        const int row = m0 + quarter * 32 + lane;
        const int cb0 = half * 32;
        float hi[32], lo[32];
#pragma unroll
        for (int j = 0; j < 32; j++) { hi[j] = 0.0f; lo[j] = 0.0f; }
        bool ok = true;
        for (int c = 0; c < chunks && ok; c++) {
            ok = mbar_wait(saddr(&bars[4]), (uint32_t)c & 1, err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int cb = 0; cb < 4; cb++) {
                uint32_t v[kSplitMaxS][8];
#pragma unroll
                for (int dgl = 0; dgl < kSplitMaxS; dgl++) {
                    if (dgl < S) {
                        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) +
                                            (uint32_t)(dgl * kTN + cb0 + cb * 8);
                        TMEM_LD8(ta, v[dgl]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; j++) v[dgl][j] = 0u;
                    }
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    // diagonals 3.. (small) summed in FP32 first, then the
                    // leading three and that sum added exactly
                    float small = 0.0f;
#pragma unroll
                    for (int dgl = kSplitMaxS - 1; dgl >= 3; dgl--)
                        small += __uint_as_float(v[dgl][j]);
                    const int jj = cb * 8 + j;
                    df_add(hi[jj], lo[jj], __uint_as_float(v[0][j]));
                    df_add(hi[jj], lo[jj], __uint_as_float(v[1][j]));
                    df_add(hi[jj], lo[jj], __uint_as_float(v[2][j]));
                    df_add(hi[jj], lo[jj], small);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&bars[5])));
        }
        if (row < M) {
            const int er = ea[row];
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int col = n0 + cb0 + j;
                if (col < N)
                    C[row + (int64_t)col * ldc] =
                        scale2((double)hi[j] + (double)lo[j], er + eb[col]);
            }
        }
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

static bool get_encoder() {
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

static bool make_map(CUtensorMap *tm, void *ptr, int rows, int kpad, int box_rows) {
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

// Slices of A (rows) and B (columns) into the caller's buffers, then the
// GEMM.  Buffers: sa [S][Mpad][Kpad], sb [S][Npad][Kpad] BF16; rowmax
// [Mpad], colmax [Npad] u64; ea [Mpad], eb [Npad] int; kend [N tiles]
// (device, multiples of 32, <= Kpad).  Returns cudaErrorInvalidValue when
// a tensor map cannot be encoded.
cudaError_t launch_split_gemm(const double *A, int64_t lda, const double *B, int64_t ldb, int M,
                              int N, int K, int S, const int *kend, double *C, int64_t ldc,
                              __nv_bfloat16 *sa, __nv_bfloat16 *sb, unsigned long long *rowmax,
                              unsigned long long *colmax, int *ea, int *eb, int *err,
                              cudaStream_t st) {
    if (!get_encoder()) return cudaErrorInvalidValue;
    const int Mpad = split_pad_m(M), Npad = split_pad_n(N), Kpad = split_pad_k(K);
    cudaMemsetAsync(rowmax, 0, sizeof(unsigned long long) * Mpad, st);
    k_row_max<<<dim3((M + 255) / 256, (K + 255) / 256), 256, 0, st>>>(A, lda, M, K, rowmax);
    k_slice_rows<<<dim3(Kpad / 64, Mpad / 32), 256, 0, st>>>(A, lda, M, K, S, rowmax, sa, Mpad,
                                                              Kpad, ea);
    k_col_max<<<(N + 7) / 8, 256, 0, st>>>(B, ldb, K, N, colmax);
    k_slice_cols<<<dim3((Kpad + 255) / 256, Npad), 256, 0, st>>>(B, ldb, K, N, S, colmax, sb,
                                                                  Npad, Kpad, eb);
    CUtensorMap tmA, tmB;
    if (!make_map(&tmA, sa, S * Mpad, Kpad, kTM) || !make_map(&tmB, sb, S * Npad, Kpad, kTN))
        return cudaErrorInvalidValue;
    const size_t smem = split_smem_bytes();
    cudaFuncSetAttribute(k_split_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_split_gemm<<<dim3(Npad / kTN, Mpad / kTM), kSplitThreads, smem, st>>>(
        tmA, tmB, S, M, N, Mpad, Npad, kend, ea, eb, C, ldc, err);
    return cudaGetLastError();
}

}  // namespace evec
