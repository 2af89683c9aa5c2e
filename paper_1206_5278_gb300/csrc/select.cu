// Bandwidth selection as the paper runs it, on top of the exact grid kernel.
//
// Random search (Sec. 3.5, Sec. 4): bandwidths are drawn uniformly from
// (0, h_max] and the best pair by the likelihood score is kept.  Here every
// round draws G1 values of h1 and G2 values of h2 and scores all G1 x G2 pairs
// exactly in one grid launch (the same cost as G1 x G2 / 1024 of a 32 x 32
// grid), so one launch yields G1 G2 uniformly distributed candidates.
//
// Reference rule (Sec. 4.2, after Silverman): each kernel gets the bandwidth
// that minimises the asymptotic mean integrated squared error of an
// unconditional KDE of a normal density with the data's spread,
//   h = A(K, d) sigma n^{-1/(d+4)},   A^{d+4} = d R(K) / (mu2(K)^2 J_d),
// with J_d = int (Laplacian phi)^2 = d (d + 2) / (2^{d+2} pi^{d/2}) for the
// standard normal phi in d dimensions, and for the radial kernels
//   Gaussian:      R = (4 pi)^{-d/2},             mu2 = 1         -> A^{d+4} = 4 / (d + 2)
//   Epanechnikov:  R = 2 (d + 2) / (V_d (d + 4)), mu2 = 1/(d + 4)  -> A^{d+4} = 8 (d + 4) (2 sqrt(pi))^d / V_d
// (V_d the unit-ball volume).  x uses its d dimensions with sigma^2 the mean
// marginal variance (1 on standardised data); y uses d = 1 and its own sd.
#include <cmath>
#include <vector>

#include "cde_internal.h"

namespace cde {

__global__ void k_col_stats(const float* __restrict__ x, int64_t N, int d, double* stats);

// SplitMix64 (Steele, Lea & Flood, 2014) as a counter-based stream: the k-th
// value of the stream with seed s is mix(s + (k + 1) * gamma).
static uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform draw in (0, h_max]: h_max (1 - u), u = 53 random bits / 2^53, raised
// to at least 1e-6 h_max (so every draw is a valid bandwidth).
static double draw_bandwidth(uint64_t seed, uint64_t k, double h_max) {
    const double u = (double)(splitmix64_at(seed, k) >> 11) * 0x1p-53;
    const double h = h_max * (1.0 - u);
    return h > 1e-6 * h_max ? h : 1e-6 * h_max;
}

static double log_ball_volume(int d) {
    double lv = (d % 2) ? std::log(2.0) : 0.0;
    for (int k = 2 + d % 2; k <= d; k += 2) lv += std::log(2.0 * M_PI / k);
    return lv;
}

// ln A(K, d) of the normal-reference rule
static double log_rule_constant(int kernel, int d) {
    const double p = 1.0 / (d + 4.0);
    if (kernel == CDE_KERNEL_EPAN)
        return p * (std::log(8.0 * (d + 4.0)) + d * std::log(2.0 * std::sqrt(M_PI)) - log_ball_volume(d));
    return p * std::log(4.0 / (d + 2.0));
}

}  // namespace cde

using namespace cde;

extern "C" int cde_reference_rule(cde_ctx* ctx, cde_dataset ds, double* h1, double* h2) {
    CDE_NVTX("cde_reference_rule");
    if (!ctx || !h1 || !h2) return set_error(CDE_EINVAL, "cde_reference_rule: null argument");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_reference_rule: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int d = D->d;
    double* dstats = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&dstats, (size_t)2 * (d + 1) * sizeof(double), st));
    // column statistics of the stored (possibly standardised) x and of y
    for (int c = 0; c <= d; ++c) {
        const float* col = c < d ? D->xs + (int64_t)c * D->Np : D->y;
        k_col_stats<<<1, 1024, 0, st>>>(col, D->N, 1, dstats + 2 * c);
    }
    cudaError_t e = cudaGetLastError();
    std::vector<double> stats(2 * (d + 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(stats.data(), dstats, stats.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dstats, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "cde_reference_rule");
    double var = 0.0;
    for (int c = 0; c < d; ++c) var += stats[2 * c + 1] * stats[2 * c + 1];
    const double sx = std::sqrt(var / d), sy = stats[2 * d + 1];
    if (!(sx > 0.0) || !(sy > 0.0)) return set_error(CDE_EINVAL, "cde_reference_rule: zero spread");
    const double n = (double)D->N;
    *h1 = std::exp(log_rule_constant(D->kernel, d)) * sx * std::pow(n, -1.0 / (d + 4.0));
    *h2 = std::exp(log_rule_constant(D->kernel, 1)) * sy * std::pow(n, -1.0 / 5.0);
    return CDE_OK;
}

extern "C" int cde_select_random(cde_ctx* ctx, cde_dataset ds, double h1_max, double h2_max, int rounds,
                                 int G1, int G2, uint64_t seed, int objective, double* best,
                                 double* h1_out, double* h2_out, double* Lc_out, double* Le_out) {
    CDE_NVTX("cde_select_random");
    if (!ctx || !best) return set_error(CDE_EINVAL, "cde_select_random: null argument");
    if (!std::isfinite(h1_max) || !std::isfinite(h2_max) || h1_max < 1e-6 || h2_max < 1e-6 ||
        h1_max > 1e6 || h2_max > 1e6)
        return set_error(CDE_EINVAL, "cde_select_random: h_max must be finite in [1e-6, 1e6]");
    if (rounds < 1 || G1 < 1 || G2 < 1 || G1 > 32 || G2 > 32)
        return set_error(CDE_EINVAL, "cde_select_random: need rounds >= 1 and 1 <= G1, G2 <= 32");
    if (objective != CDE_L_COND && objective != CDE_L_EQ3)
        return set_error(CDE_EINVAL, "cde_select_random: objective must be CDE_L_COND or CDE_L_EQ3");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_select_random: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int GG = G1 * G2;
    double* dout = nullptr;
    double* hout = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&dout, (size_t)2 * GG * sizeof(double), st));
    if (cudaMallocHost((void**)&hout, (size_t)2 * GG * sizeof(double)) != cudaSuccess) {
        cudaFreeAsync(dout, st);
        return set_error(CDE_ENOMEM, "cde_select_random: pinned buffer");
    }
    std::vector<double> h1(G1), h2(G2);
    bool have = false;
    double bv = -INFINITY;
    int rc = CDE_OK;
    for (int r = 0; r < rounds && rc == CDE_OK; ++r) {
        const uint64_t k0 = (uint64_t)r * (G1 + G2);
        for (int k = 0; k < G1; ++k) h1[k] = draw_bandwidth(seed, k0 + k, h1_max);
        for (int l = 0; l < G2; ++l) h2[l] = draw_bandwidth(seed, k0 + G1 + l, h2_max);
        rc = loo_grid_enqueue(ctx, *D, h1.data(), G1, h2.data(), G2, nullptr, 0, dout, dout + GG, nullptr, st);
        if (rc != CDE_OK) break;
        cudaError_t e = cudaMemcpyAsync(hout, dout, (size_t)2 * GG * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "cde_select_random");
            break;
        }
        for (int c = 0; c < GG; ++c) {
            const double v = hout[(objective == CDE_L_COND ? 0 : GG) + c];
            if (v > bv) {  // first strict maximum in (round, k, l) order; -inf and NaN never win
                bv = v;
                have = true;
                best[0] = h1[c / G2];
                best[1] = h2[c % G2];
                best[2] = hout[c];
                best[3] = hout[GG + c];
            }
        }
        if (h1_out) for (int k = 0; k < G1; ++k) h1_out[(size_t)r * G1 + k] = h1[k];
        if (h2_out) for (int l = 0; l < G2; ++l) h2_out[(size_t)r * G2 + l] = h2[l];
        if (Lc_out) for (int c = 0; c < GG; ++c) Lc_out[(size_t)r * GG + c] = hout[c];
        if (Le_out) for (int c = 0; c < GG; ++c) Le_out[(size_t)r * GG + c] = hout[GG + c];
    }
    cudaFreeAsync(dout, st);
    cudaStreamSynchronize(st);
    cudaFreeHost(hout);
    if (rc != CDE_OK) return rc;
    if (!have) {
        best[0] = best[1] = NAN;
        best[2] = best[3] = -INFINITY;
    }
    return CDE_OK;
}
