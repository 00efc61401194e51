// Peak-rate probe used by bench.py for the ALU roofline of the pair kernels:
// MUFU.RSQ (rsqrt.approx.ftz.f32) results, FFMA results, the attraction
// pair mix (1 rsqrt + 5 FP32 ops), DFMA results and the attraction pair with
// plain FP64 accumulation, per SM per clock.  Each thread runs
// kChains independent dependency chains; every thread writes one float so
// nothing is eliminated.  The cycle count is the largest clock64() interval
// over the CTAs.  Output: one line per kernel, "<name> ops/SM/clk = <x> ...".
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kChains = 8;

__global__ void rsq_kernel(float *out, int iters, long long *cycles)
{
    float v[kChains];
    for (int c = 0; c < kChains; ++c) v[c] = 1.0f + (threadIdx.x + c) * 1e-3f;
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[c]));
            v[c] = y;
        }
    }
    long long t1 = clock64();
    float s = 0;
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void ffma_kernel(float *out, int iters, long long *cycles)
{
    float v[kChains];
    for (int c = 0; c < kChains; ++c) v[c] = 1.0f + (threadIdx.x + c) * 1e-3f;
    const float a = 0.999f, b = 1e-4f;
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    long long t1 = clock64();
    float s = 0;
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// rsqrt and 5 FP32 ops interleaved (the attraction pair mix).
__global__ void mix_kernel(float *out, int iters, long long *cycles)
{
    float v[kChains], acc[kChains];
    for (int c = 0; c < kChains; ++c) { v[c] = 1.0f + (threadIdx.x + c) * 1e-3f; acc[c] = 0; }
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float dx = v[c] - 0.25f;
            float r2 = fmaf(dx, dx, 0.5f);
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
            float w = y * 0.75f;
            acc[c] += w;
            v[c] = fmaf(w, dx, v[c]);
        }
    }
    long long t1 = clock64();
    float s = 0;
    for (int c = 0; c < kChains; ++c) s += v[c] + acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// FP64 fused multiply-add results (GB300's FP64 pipe).
__global__ void dfma_kernel(float *out, int iters, long long *cycles)
{
    double v[kChains];
    for (int c = 0; c < kChains; ++c) v[c] = 1.0 + (threadIdx.x + c) * 1e-3;
    const double a = 0.999, b = 1e-4;
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
    long long t1 = clock64();
    double s = 0;
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// The attraction pair with the plain FP64-accumulate form: the pair term in
// FP32 (difference, squared distance, SFU rsqrt, weight), the sums of the
// force component and of the weights in FP64 for every pair.
__global__ void fp64acc_kernel(float *out, int iters, long long *cycles)
{
    float v[kChains];
    double ax[kChains], aw[kChains];
    for (int c = 0; c < kChains; ++c) {
        v[c] = 1.0f + (threadIdx.x + c) * 1e-3f;
        ax[c] = 0.0;
        aw[c] = 0.0;
    }
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const float dx = v[c] - 0.25f;
            const float r2 = fmaf(dx, dx, 0.5f);
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
            const float w = y * 0.75f;
            aw[c] += (double)w;
            ax[c] = fma((double)w, (double)dx, ax[c]);
            v[c] += 1e-7f;
        }
    }
    long long t1 = clock64();
    double s = 0;
    for (int c = 0; c < kChains; ++c) s += v[c] + ax[c] + aw[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

int main()
{
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    const int threads = 512, bps = 2, iters = 1 << 16;
    const int blocks = sms * bps;
    float *out;
    long long *cyc;
    cudaMalloc(&out, sizeof(float) * blocks * threads);
    cudaMalloc(&cyc, sizeof(long long) * blocks);
    long long *hc = new long long[blocks];
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const char *names[5] = {"rsqrt", "ffma", "attr_mix(1 rsqrt + 5 fp32)", "dfma",
                            "fp64acc(pair, fp64 sums)"};
    for (int k = 0; k < 5; ++k) {
        // the FP64 kernels run far slower: fewer iterations keep them short
        const int it = k >= 3 ? iters / 16 : iters;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(a);
            if (k == 0) rsq_kernel<<<blocks, threads>>>(out, it, cyc);
            else if (k == 1) ffma_kernel<<<blocks, threads>>>(out, it, cyc);
            else if (k == 2) mix_kernel<<<blocks, threads>>>(out, it, cyc);
            else if (k == 3) dfma_kernel<<<blocks, threads>>>(out, it, cyc);
            else fp64acc_kernel<<<blocks, threads>>>(out, it, cyc);
            cudaEventRecord(b);
            cudaEventSynchronize(b);
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaMemcpy(hc, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
        double maxc = 0;
        for (int i = 0; i < blocks; ++i) maxc = hc[i] > maxc ? hc[i] : maxc;
        const double ops = (double)blocks * threads * it * kChains;
        const double per_sm_clk = ops / sms / maxc;
        const double eff_ghz = maxc / (ms * 1e-3) / 1e9;
        printf("%-28s ops/SM/clk = %.2f  (%.3f ms, %.0f cycles, implied clock %.3f GHz, %.3e ops/s)\n",
               names[k], per_sm_clk, ms, maxc, eff_ghz, ops / (ms * 1e-3));
    }
    printf("sms %d, max clock attr %d kHz, err %s\n", sms, clk, cudaGetErrorString(cudaGetLastError()));
    return 0;
}
