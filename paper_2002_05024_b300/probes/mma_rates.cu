// mma_rates.cu -- cost of tcgen05.mma (kind::f16, BF16 in, FP32 accumulate,
// M = 128, cta_group::1) as issued by the split-precision GEMMs: cycles per
// MMA for N = 16 .. 256 into one accumulator, round-robin over eight
// accumulators, identical operands, and the concatenated-slice group the
// kernels use (8 MMAs, N = 32 (8 - p) at TMEM column 32 p).  One CTA per SM;
// thread 0 issues R MMAs on fixed shared-memory operands, commits, waits
// (bounded), and reports cycles per MMA.  Standalone:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o mma_rates mma_rates.cu && ./mma_rates
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t a, int sw128) {
    uint64_t d = 0;
    d |= (uint64_t)((a & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((sw128 ? 1024 : 512) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(sw128 ? 2 : 4) << 61;
    return d;
}

// mode 0: one accumulator, N for all; 1: concatenated slices, N = (8 - p) 32
// at column 32 p, 8 MMAs per group; 2: eight accumulators round-robin;
// 3: one accumulator, identical operands
__global__ void __launch_bounds__(128, 1) k(int R, int N, int sw128, int mode, long long *out, int *err) {
    extern __shared__ unsigned char sm[];
    unsigned char *base = (unsigned char *)(((uintptr_t)sm + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;              // 8 x 16 KB (128 rows x 128 B)
    unsigned char *sB = base + 8 * 16384;  // 64 KB (256 rows x 128 B... as needed)
    __shared__ uint64_t bar;
    __shared__ uint32_t th;
    const int tid = threadIdx.x;
    for (int i = tid; i < (8 * 16384 + 65536) / 4; i += blockDim.x)
        ((uint32_t *)base)[i] = 0x3f803f80u ^ (i * 2654435761u & 0x00ff00ffu);
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&th)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = th;
    if (tid == 0) {
        const int rowb = sw128 ? 128 : 64;
        long long t0 = clock64();
        int issued = 0;
        for (int r = 0; r < R; r++) {
            if (mode == 2) {   // N columns, 8 accumulators round-robin (8 N <= 512)
                const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24);
                const int kk = (r >> 3) & 3;
                const int p = r & 7;
                const uint64_t ad = desc(saddr(sA + p * 16384) + (kk * 32) % rowb, sw128);
                const uint64_t bd = desc(saddr(sB) + (kk * 32) % rowb, sw128);
                asm volatile("{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n"
                             ::"r"(tmem + (r & 7) * N), "l"(ad), "l"(bd), "r"(idesc), "r"(r >= 8 ? 1 : 0));
                issued++;
            } else if (mode == 3) {   // same accumulator, same A and B every time
                const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24);
                const uint64_t ad = desc(saddr(sA), sw128);
                const uint64_t bd = desc(saddr(sB), sw128);
                asm volatile("{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(r > 0 ? 1 : 0));
                issued++;
            } else if (mode == 0) {
                const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24);
                const int kk = r & 3;
                const int p = (r >> 2) & 7;
                const uint64_t ad = desc(saddr(sA + p * 16384) + (kk * 32) % rowb, sw128);
                const uint64_t bd = desc(saddr(sB) + (kk * 32) % rowb, sw128);
                asm volatile("{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(r > 0 ? 1 : 0));
                issued++;
            } else {
                const int kk = r & 3;
                for (int p = 0; p < 8; p++) {
                    const int n = (8 - p) * 32;
                    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | (8u << 24);
                    const uint64_t ad = desc(saddr(sA + p * 16384) + (kk * 32) % rowb, sw128);
                    const uint64_t bd = desc(saddr(sB) + (kk * 32) % rowb, sw128);
                    asm volatile("{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n"
                                 ::"r"(tmem + p * 32), "l"(ad), "l"(bd), "r"(idesc), "r"(r > 0 || p > 0 ? 1 : 0));
                    issued++;
                }
            }
        }
        long long t1 = clock64();
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&bar)));
        uint32_t done = 0;
        for (long it = 0; it < (1L << 28) && !done; it++)
            asm volatile("{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
                         : "=r"(done) : "r"(saddr(&bar)), "r"(0) : "memory");
        if (!done) atomicExch(err, 1);
        long long t2 = clock64();
        out[blockIdx.x * 4 + 0] = t1 - t0;
        out[blockIdx.x * 4 + 1] = t2 - t0;
        out[blockIdx.x * 4 + 2] = issued;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

int main() {
    long long *out; int *err;
    cudaMalloc(&out, 148 * 4 * 8); cudaMalloc(&err, 4); cudaMemset(err, 0, 4);
    const int smem = 1024 + 8 * 16384 + 65536;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    long long h[148 * 4];
    for (int mode : {2, 3}) {
        for (int N : {16, 32, 64}) {
            k<<<148, 128, smem>>>(2048, N, 0, mode, out, err);
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return 1; }
            cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
            double issue = 0, tot = 0;
            for (int b = 0; b < 148; b++) { issue += h[b * 4]; tot += h[b * 4 + 1]; }
            issue /= 148; tot /= 148;
            printf("mode %d SW64 N=%3d: %.1f cycles/MMA (issue %.1f)\n", mode, N, tot / 2048, issue / 2048);
        }
    }
    for (int sw = 0; sw < 1; sw++) {
        for (int N : {16, 32, 64, 128, 256}) {
            k<<<148, 128, smem>>>(2048, N, sw, 0, out, err);
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return 1; }
            cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
            double issue = 0, tot = 0;
            for (int b = 0; b < 148; b++) { issue += h[b * 4]; tot += h[b * 4 + 1]; }
            issue /= 148; tot /= 148;
            printf("%s N=%3d: %.1f cycles/MMA (issue %.1f), %.0f MAC/clk/SM\n", sw ? "SW128" : "SW64 ", N,
                   tot / 2048, issue / 2048, 128.0 * N * 16 * 2048 / tot);
        }
        k<<<148, 128, smem>>>(512, 0, sw, 1, out, err);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return 1; }
        cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
        double tot = 0;
        for (int b = 0; b < 148; b++) tot += h[b * 4 + 1];
        tot /= 148;
        // per group of 8 MMAs: sum of N = 36 * 32 columns
        printf("%s concat (8 MMAs, N=(8-p)*32): %.1f cycles/group, %.0f MAC/clk/SM\n", sw ? "SW128" : "SW64 ",
               tot / 512, 128.0 * 36 * 32 * 16 * 512 / tot);
    }
    int herr; cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
    printf("err %d\n", herr);
    return 0;
}
