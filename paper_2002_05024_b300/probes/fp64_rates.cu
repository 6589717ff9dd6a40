// fp64_rates.cu -- measures the FP64 rates the roofline of the FP64 path is
// built on: DFMA throughput (many independent chains), FP64 mma.sync
// throughput, and the dependent-chain latency of the FP64 primitives the
// diagonal-tile solver uses.  Standalone:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_rates fp64_rates.cu && ./fp64_rates
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
    printf("CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); return 1; } } while (0)

__global__ void dfma_rate(double *out, int iters, double a, double b) {
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; c++) acc[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 8; c++) acc[c] = fma(acc[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dmma_rate(double *out, int iters) {
    double a0 = threadIdx.x * 1e-3, a1 = a0 + 1e-5, b = 1.0 - threadIdx.x * 1e-4;
    double c[4][4] = {};
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 4; k++)
            asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
                         : "+d"(c[k][0]), "+d"(c[k][1]), "+d"(c[k][2]), "+d"(c[k][3])
                         : "d"(a0), "d"(a1), "d"(b));
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// dependent chains, one warp: cycles per operation
__global__ void latency(double *out, long long *cyc, double a) {
    const int N = 2048;
    double x = a + threadIdx.x * 1e-12;
    long long t0, t1;
    t0 = clock64(); for (int i = 0; i < N; i++) x = fma(x, 0.999999, 1e-7); t1 = clock64(); cyc[0] = t1 - t0;
    t0 = clock64(); for (int i = 0; i < N; i++) x = (x > 1.5) ? x - 0.25 : x + 0.5; t1 = clock64(); cyc[1] = t1 - t0;
    t0 = clock64();
    for (int i = 0; i < N; i++) { double r; asm volatile("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x)); x = r + 1.0; }
    t1 = clock64(); cyc[2] = t1 - t0;
    t0 = clock64(); for (int i = 0; i < N / 8; i++) x = 3.0 / x; t1 = clock64(); cyc[3] = (t1 - t0) * 8;
    out[threadIdx.x] = x;
}

// DFMA rate when only `act` lanes of each warp are active
__global__ void masked_rate(double *out, int iters, int act, double a, double b) {
    const int lane = threadIdx.x & 31;
    double acc[8];
    for (int c = 0; c < 8; c++) acc[c] = lane * 1e-3 + c;
    if (lane < act)
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int c = 0; c < 8; c++) acc[c] = fma(acc[c], a, b);
        }
    double s = 0;
    for (int c = 0; c < 8; c++) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, 0));
    const int sms = p.multiProcessorCount;
    double *d;
    long long *c;
    CK(cudaMalloc(&d, sizeof(double) * sms * 8 * 256));
    CK(cudaMalloc(&c, sizeof(long long) * 8));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms;
    const int blocks = sms * 8, threads = 256;
    dfma_rate<<<blocks, threads>>>(d, 16, 1.0000001, 1e-9);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    dfma_rate<<<blocks, threads>>>(d, 4096, 1.0000001, 1e-9);
    cudaEventRecord(e1);
    CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    printf("%s, %d SMs\n", p.name, sms);
    printf("DFMA throughput          %.3f TFLOP/s\n", 2.0 * 8 * 4096 * (double)blocks * threads / ms / 1e9);
    dmma_rate<<<blocks, threads>>>(d, 16);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    dmma_rate<<<blocks, threads>>>(d, 1024);
    cudaEventRecord(e1);
    CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    printf("mma.sync m16n8k4 f64     %.3f TFLOP/s\n",
           2.0 * 16 * 8 * 4 * 4 * 1024.0 * blocks * (threads / 32) / ms / 1e9);
    for (int act : {32, 8, 1}) {
        masked_rate<<<blocks, threads>>>(d, 16, act, 1.0000001, 1e-9);
        CK(cudaDeviceSynchronize());
        cudaEventRecord(e0);
        masked_rate<<<blocks, threads>>>(d, 2048, act, 1.0000001, 1e-9);
        cudaEventRecord(e1);
        CK(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms, e0, e1);
        const double winstr = (double)blocks * (threads / 32) * 2048 * 8;
        printf("DFMA, %2d active lanes    %.2f ns per warp-instruction per SM\n", act, ms * 1e6 / (winstr / sms));
    }
    latency<<<1, 32>>>(d, c, 1.25);
    CK(cudaDeviceSynchronize());
    long long h[4];
    CK(cudaMemcpy(h, c, sizeof(h), cudaMemcpyDeviceToHost));
    printf("latency DFMA             %.1f cycles\n", h[0] / 2048.0);
    printf("latency DSETP+select+DADD %.1f cycles\n", h[1] / 2048.0);
    printf("latency rcp.approx+DADD  %.1f cycles\n", h[2] / 2048.0);
    printf("latency FP64 division    %.1f cycles\n", h[3] / 2048.0);
    return 0;
}
