// split_common.cuh -- pieces shared by the split-precision kernels: digit
// slicing of FP64 values (balanced base 2^7, exact BF16 slices), the
// mbarrier / TMA / UMMA-descriptor helpers of the tcgen05 pipelines, the
// double-float accumulator and its exact conversion to FP64, and the host
// side tensor-map encoder.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "evec_internal.cuh"

namespace evec {

constexpr int kSplitMaxS = 8;       // digit slices per operand
constexpr int kTM = 128, kTK = 32;  // MMA rows; K per TMA box (64 bytes of BF16)
constexpr int kTmemCols = 512;
constexpr long kWaitLimit = 1L << 26;

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
    // unrolled over the largest S with a predicate, so d stays in registers
#pragma unroll
    for (int p = kSplitMaxS - 1; p >= 1; p--) {
        if (p < S) {
            long long r = I & 127;
            if (r >= 64) r -= 128;
            d[p] = (int)r;
            I = (I - r) >> 7;
        }
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

// f 2^k as a double, built from f's fields with integer operations (the FP64
// pipe is the scarce unit): exact when f is zero or normal and the result is
// a normal double; otherwise clears ok and the caller takes scale2
__device__ __forceinline__ double f2d_pow2(float f, int k, bool &ok) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t a = u & 0x7fffffffu;
    if (a == 0u) return 0.0;
    const int fe = (int)(a >> 23);
    const int e = fe - 127 + k;
    ok = ok && fe != 0 && e >= -1022 && e <= 1023;
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                    ((unsigned long long)(unsigned)(e + 1023) << 52) |
                                    ((unsigned long long)(a & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// (hi + lo) 2^k in FP64 for a normalised double-float pair (|lo| <= ulp(hi)
// / 2): both parts scaled exactly, then one FP64 add, exact (48 bits)
__device__ __forceinline__ double df_to_double(float hi, float lo, int k) {
    bool ok = true;
    const double h = f2d_pow2(hi, k, ok), l = f2d_pow2(lo, k, ok);
    return ok ? h + l : scale2((double)hi + (double)lo, k);
}

#define TMEM_LD8(taddr, r)                                                                   \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"     \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),     \
                   "=r"(r[6]), "=r"(r[7])                                                      \
                 : "r"(taddr))

#define TMEM_LD16(taddr, r)                                                                  \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,"   \
                 "%11,%12,%13,%14,%15}, [%16];"                                                 \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),     \
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),   \
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])                          \
                 : "r"(taddr))

// host side: the driver's tensor-map encoder (resolved once) and a 2D BF16
// map over a [rows][kpad] K-contiguous slice buffer with SWIZZLE_64B boxes
// of {32 K, box_rows}
bool get_encoder();
bool make_map(CUtensorMap *tm, void *ptr, int rows, int kpad, int box_rows);

// per-call state of the split tile updates: the tensor maps of the panel
// slices (A, 128-row boxes) and of one step's column slices (B, 32-row boxes)
struct SplitUpdateCtx {
    CUtensorMap tmA, tmB32;
    int S, Kp, Npad;
};

}  // namespace evec
