// fp32_rate.cu -- measures the FP32 fused multiply-add rate of the GPU (the denominator of the
// ALU roofline the benchmark reports for the literal-curvature data term).  Not part of the
// estimator: a separate probe library, built beside libfm.so.
//
// Every thread runs 8 independent FMA chains x = x * a + b (a = 0.999, b = 0.001 keep the
// values normal and bounded), 16 steps per loop trip, so each SM sub-partition always has
// independent work to issue.  The grid holds 4 blocks of 256 threads per SM.  Block 0 also
// reads the SM cycle counter and the global nanosecond timer at the start and the end, which
// gives the clock the measurement ran at.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8, kUnroll = 16, kBlock = 256, kBlocksPerSm = 4;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kBlock) k_ffma(float* sink, long long* clk, int iters, float a, float b) {
    long long c0 = 0;
    uint64_t t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        t0 = global_ns();
    }
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) sink[blockIdx.x] = s;  // never true; keeps the chains live
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = clock64() - c0;
        clk[1] = (long long)(global_ns() - t0);
    }
}

}  // namespace

// FP32 rate of `device`: tflops = measured FMA flops (2 per FMA) per second over the whole
// GPU, per_sm_clk = FMA lane-operations per SM per clock, mhz = the SM clock during the run.
// Returns 0, or -1 on a CUDA error.
extern "C" __attribute__((visibility("default"))) int fmprobe_fp32_rate(int device, double* tflops,
                                                                         double* per_sm_clk, double* mhz) {
    if (cudaSetDevice(device) != cudaSuccess) return -1;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    float* sink = nullptr;
    long long* clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = -1;
    const int grid = nsm * kBlocksPerSm, iters = 4096;
    if (cudaMalloc(&sink, grid * sizeof(float)) == cudaSuccess && cudaMalloc(&clk, 2 * sizeof(long long)) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        k_ffma<<<grid, kBlock>>>(sink, clk, 256, 0.999f, 0.001f);  // warm-up
        cudaEventRecord(e0);
        k_ffma<<<grid, kBlock>>>(sink, clk, iters, 0.999f, 0.001f);
        cudaEventRecord(e1);
        long long h[2] = {0, 0};
        float ms = 0.f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess && ms > 0.f && h[1] > 0) {
            const double fmas = (double)grid * kBlock * kChains * kUnroll * (double)iters;
            const double sec = ms * 1e-3;
            const double f_mhz = (double)h[0] / (double)h[1] * 1e3;
            *tflops = 2.0 * fmas / sec / 1e12;
            *mhz = f_mhz;
            *per_sm_clk = fmas / sec / (f_mhz * 1e6) / nsm;
            rc = 0;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(clk);
    return rc;
}
