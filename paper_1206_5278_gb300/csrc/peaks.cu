// Micro-benchmarks of the pipes the kernels are bound by: FP32 FMA lanes and
// MUFU ex2 results per SM per clock, measured with many independent chains
// per thread and the SM clock taken from clock64() over the same launch, and
// the 5th-generation tensor core's BF16 rate for the density kernel's MMA
// shape (tcgen05, M = 128, N = 256, K = 16, issued back to back by one thread).
#include <algorithm>
#include <vector>

#include "cde_internal.h"
#include "tc_util.cuh"

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

// One CTA per SM (the shared-memory request keeps a second one off the SM):
// R accumulating BF16 MMAs of 128 x 256 x 16 from shared-memory operands
// (values irrelevant), cycles from the first issue to the commit's arrival.
constexpr int kPeakUmmaSmem = 120 * 1024;

template <int KIND>   // 0: kind::f16 BF16 (K = 16), 1: kind::tf32 (K = 8); M = 128, N = 256
__global__ void __launch_bounds__(128) k_peak_umma(int R, long long* cyc, int* err) {
    extern __shared__ float4 pk_dyn[];
    unsigned char* A = reinterpret_cast<unsigned char*>(pk_dyn);   // 128 x 32 bf16
    unsigned char* B = A + 8192;                                  // 256 x 32 bf16
    __shared__ unsigned long long bar;
    __shared__ uint32_t tb;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (8192 + 16384) / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(A)[i] = 0x3f803f80u;
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&tb), 256);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t t = tb;
    if (tid == 0) {
        const uint32_t idesc = KIND == 0 ? tc_idesc_bf16(128, 256) : tc_idesc_tf32(128, 256);
        const uint64_t ad = tc_sdesc(smem_u32(A), 128, 512), bd = tc_sdesc(smem_u32(B), 128, 512);
        const long long c0 = clock64();
        for (int r = 0; r < R; ++r) {
            if constexpr (KIND == 0) tc_mma_bf16(t, ad, bd, idesc, r > 0 ? 1u : 0u);
            else tc_mma_tf32(t, ad, bd, idesc, r > 0 ? 1u : 0u);
        }
        tc_commit(smem_u32(&bar));
        mbar_wait(smem_u32(&bar), 0, &abort_flag, err, 1);
        cyc[blockIdx.x] = clock64() - c0;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(t, 256);
    }
}

// Legacy warp-level MMAs (the LOO tile and d >= 16 gradient kernels): eight
// independent accumulator chains per warp, 8 warps per CTA, 2 CTAs per SM.
template <int KIND>   // 0: m16n8k8 TF32, 1: m16n8k16 BF16
__global__ void __launch_bounds__(256) k_peak_mma(int iters, float* out, long long* cyc) {
    const long long c0 = clock64();
    float d[8][4];
#pragma unroll
    for (int c = 0; c < 8; ++c) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0.f;
    const uint32_t a0 = 0x3c003c00u ^ threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, b0 = a0 + 5, b1 = a0 + 7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if constexpr (KIND == 0)
                asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                             "{%8,%9}, {%0,%1,%2,%3};"
                             : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                             : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            else
                asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                             "{%8,%9}, {%0,%1,%2,%3};"
                             : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                             : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    float r = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) r += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - c0;
}

static int measure_mma(cde_ctx* ctx, int kind, double* mac_per_clk) {
    const int S = ctx->sm_count, blocks = 2 * S, threads = 256, iters = 2000;
    float* out = nullptr;
    long long* cyc = nullptr;
    CDE_CUDA(cudaMalloc((void**)&out, sizeof(float) * blocks * threads));
    CDE_CUDA(cudaMalloc((void**)&cyc, sizeof(long long) * blocks));
    std::vector<long long> hc(blocks);
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        if (kind == 0) k_peak_mma<0><<<blocks, threads, 0, ctx->stream>>>(iters, out, cyc);
        else k_peak_mma<1><<<blocks, threads, 0, ctx->stream>>>(iters, out, cyc);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            cudaFree(out);
            cudaFree(cyc);
            return cuda_error(e, "cde_measure_peaks: mma.sync probe");
        }
        long long mx = 0;
        for (auto v : hc) mx = v > mx ? v : mx;
        // MACs of one MMA: 16 x 8 x 8 (TF32) or 16 x 8 x 16 (BF16); 2 CTAs x 8 warps per SM
        const double macs = (kind == 0 ? 1024.0 : 2048.0) * 8 * iters * 8 * 2;
        const double r = macs / (double)mx;
        if (r > best) best = r;
    }
    cudaFree(out);
    cudaFree(cyc);
    *mac_per_clk = best;
    return CDE_OK;
}

static int measure_umma(cde_ctx* ctx, int kind, double* mac_per_clk) {
    const int S = ctx->sm_count, R = 4096;
    long long* cyc = nullptr;
    int* err = ctx->d_err + kErrTensorWait;
    CDE_CUDA(cudaMalloc((void**)&cyc, sizeof(long long) * S));
    auto kern = kind == 0 ? k_peak_umma<0> : k_peak_umma<1>;
    CDE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeakUmmaSmem));
    std::vector<long long> hc(S);
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        kern<<<S, 128, kPeakUmmaSmem, ctx->stream>>>(R, cyc, err);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, sizeof(long long) * S, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            cudaFree(cyc);
            return cuda_error(e, "cde_measure_peaks: tensor-core probe");
        }
        std::vector<long long> srt(hc);
        std::sort(srt.begin(), srt.end());
        const double med = (double)srt[S / 2];
        const double r = (double)R * 128 * 256 * (kind == 0 ? 16 : 8) / med;
        if (r > best) best = r;
    }
    cudaFree(cyc);
    int tw = 0;
    CDE_CUDA(cudaMemcpy(&tw, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (tw) return set_error(CDE_ETIMEOUT, "cde_measure_peaks: tensor-core probe wait ran out");
    *mac_per_clk = best;
    return CDE_OK;
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
    double umma = 0, umma32 = 0;
    int rc = measure_umma(ctx, 0, &umma);
    if (rc == CDE_OK) rc = measure_umma(ctx, 1, &umma32);
    if (rc != CDE_OK) return rc;
    o->umma_bf16_mac_per_clk_sm = umma;
    o->umma_bf16_tflops = 2.0 * umma * S * f / 1e12;
    o->umma_tf32_mac_per_clk_sm = umma32;
    double m0 = 0, m1 = 0;
    int rc2 = measure_mma(ctx, 0, &m0);
    if (rc2 == CDE_OK) rc2 = measure_mma(ctx, 1, &m1);
    if (rc2 != CDE_OK) return rc2;
    o->mma_tf32_mac_per_clk_sm = m0;
    o->mma_bf16_mac_per_clk_sm = m1;
    return CDE_OK;
}

}  // namespace cde

extern "C" int cde_measure_peaks(cde_ctx* ctx, cde_peaks* out) {
    if (!ctx || !out) return cde::set_error(CDE_EINVAL, "cde_measure_peaks: null argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    return cde::measure_peaks(ctx, out);
}
