// Micro-benchmarks of the pipes the LOO kernels are bound by: FP32 FMA lanes
// and MUFU ex2 results per SM per clock, measured with many independent
// chains per thread and the SM clock taken from clock64() over the same
// launch.  These rates are the roofline denominators for the pair kernels.
#include "cde_internal.h"

namespace cde {

__global__ void k_peak_ffma(float* out, int iters, float s, long long* cyc) {
    long long c0 = clock64();
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) a[i] = fmaf(a[i], s, 0.999f);
    }
    float r = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) r += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - c0;
}

__global__ void k_peak_ex2(float* out, int iters, long long* cyc) {
    long long c0 = clock64();
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = threadIdx.x * 1e-3f + i * 0.01f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float r;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-a[i]));
            a[i] = r;
        }
    }
    float r = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) r += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - c0;
}

int measure_peaks(cde_ctx* ctx, cde_peaks* o) {
    const int S = ctx->sm_count, blocks = S * 8, threads = 256;
    float* out = nullptr;
    long long* cyc = nullptr;
    CDE_CUDA(cudaMalloc((void**)&out, sizeof(float) * blocks * threads));
    CDE_CUDA(cudaMalloc((void**)&cyc, sizeof(long long) * blocks));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaStream_t st = ctx->stream;
    std::vector<long long> hc(blocks);
    double res[2][2];  // [kind][ops_per_s, clock_hz]
    for (int kind = 0; kind < 2; ++kind) {
        const int iters = kind == 0 ? 20000 : 10000;
        double best = 1e30;
        double clk = 0;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            if (kind == 0) k_peak_ffma<<<blocks, threads, 0, st>>>(out, iters, 0.9999f, cyc);
            else k_peak_ex2<<<blocks, threads, 0, st>>>(out, iters, cyc);
            cudaEventRecord(e1, st);
            CDE_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            CDE_CUDA(cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost));
            long long mx = 0;
            for (auto v : hc) mx = v > mx ? v : mx;
            if (rep > 0 && ms < best) {
                best = ms;
                clk = (double)mx / (ms * 1e-3);
            }
        }
        const double ops = 16.0 * iters * (double)blocks * threads;
        res[kind][0] = ops / (best * 1e-3);
        res[kind][1] = clk;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    const double f = res[0][1] > 0 ? res[0][1] : 1.9e9;
    o->sm_count = S;
    o->sm_clock_mhz = f / 1e6;
    o->ffma_tops = res[0][0] / 1e12;
    o->ex2_tops = res[1][0] / 1e12;
    o->ffma_per_clk_sm = res[0][0] / S / f;
    o->ex2_per_clk_sm = res[1][0] / S / (res[1][1] > 0 ? res[1][1] : f);
    return CDE_OK;
}

}  // namespace cde

extern "C" int cde_measure_peaks(cde_ctx* ctx, cde_peaks* out) {
    if (!ctx || !out) return cde::set_error(CDE_EINVAL, "cde_measure_peaks: null argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    return cde::measure_peaks(ctx, out);
}
