// A variant of the LOO grid launch that allocates no device memory.
//
// cde_loo_loglik keeps its FP64 tile partials and its tile counter in memory
// taken from the stream-ordered allocator on every call.  This variant keeps
// them in one file-scope device array of fixed size instead, for callers that
// must not allocate device memory (see cde_loo_loglik_noalloc in cde.h).  The
// array's device address is looked up once per device with
// cudaGetSymbolAddress: in host code the array's name is only a host-side
// stand-in and must never be handed to a kernel.
#include <cmath>
#include <mutex>

#include "cde_internal.h"
#include "loo_common.cuh"

namespace cde {

__global__ void k_loo_final(const double* __restrict__ part, int n_tiles, int GG, int G2T, int G1r,
                            int G2r, int ld, double N, double* Lc, double* Le);

// Scratch: tile partials (2 x G1 x G2 doubles per tile) followed by the tile
// counter.  16 MiB in total; every GPU that loads the library holds it until exit.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
constexpr size_t kNoAllocCounterBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
static int noalloc_scratch(int device, void** out) {
    if (device < 0 || device >= kNoAllocMaxDevices)
        return set_error(CDE_EINVAL, "cde_loo_loglik_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cde_loo_loglik_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return CDE_OK;
}


}  // namespace cde

using namespace cde;

extern "C" int cde_loo_loglik_noalloc(cde_ctx* ctx, cde_dataset ds, const double* h1, int G1,
                                      const double* h2, int G2, double* d_L_cond, double* d_L_eq3,
                                      void* stream) {
    CDE_NVTX("cde_loo_loglik_noalloc");
    if (!ctx || !h1 || !h2) return set_error(CDE_EINVAL, "cde_loo_loglik_noalloc: null argument");
    if (G1 < 1 || G2 < 1 || G1 > 32 || G2 > 32)
        return set_error(CDE_EINVAL,
                         "cde_loo_loglik_noalloc: grids are limited to 1..32 bandwidths per axis "
                         "(the fixed 16 MiB scratch holds one grid block)");
    for (int k = 0; k < G1; ++k)
        if (!std::isfinite(h1[k]) || h1[k] < 1e-12 || h1[k] > 1e12)
            return set_error(CDE_EINVAL, "cde_loo_loglik_noalloc: h1 must be finite in [1e-12, 1e12]");
    for (int l = 0; l < G2; ++l)
        if (!std::isfinite(h2[l]) || h2[l] < 1e-12 || h2[l] > 1e12)
            return set_error(CDE_EINVAL, "cde_loo_loglik_noalloc: h2 must be finite in [1e-12, 1e12]");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_loo_loglik_noalloc: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    void* scratch = nullptr;
    int rc = noalloc_scratch(ctx->device, &scratch);
    if (rc != CDE_OK) return rc;
    cudaStream_t st = pick_stream(ctx, stream);

    const int T1 = loo_pad1(G1), T2 = loo_pad2(G2);
    LooArgs a{};
    fill_loo_args(a, *D, h1, G1, h2, G2, T1, T2);
    const int JW = 1024 / (T1 * T2);
    a.rows = nullptr;
    a.n_rows = D->N;
    a.n_units = (int)((D->N + JW - 1) / JW);
    // the tile partition of cde_loo_loglik (at most 3 slots per CTA once N is large);
    // where its small tiles need more slots than the scratch holds, they grow to fit
    const size_t slot_bytes = (size_t)2 * T1 * T2 * sizeof(double);
    const int max_tiles = (int)((kNoAllocScratchBytes - kNoAllocCounterBytes) / slot_bytes);
    const int cmax = loo_grid_ctas(ctx, T1, T2);
    int upt = loo_units_per_tile(ctx, T1, T2, D->N);
    LooTiles tp = loo_tiles(a.n_units, upt, cmax);
    if (tp.n_tiles > max_tiles) {
        upt = (a.n_units + max_tiles - 1) / max_tiles;
        tp = LooTiles{0, 0, 0, (a.n_units + upt - 1) / upt};
    }
    a.units_per_tile = upt;
    a.n_tiles = tp.n_tiles;
    a.big_g = tp.big_g;
    a.big_levels = tp.big_levels;
    a.big_s0 = tp.big_s0;
    a.win0 = 0;
    a.win1 = INT_MAX;
    a.ell_rows = nullptr;
    a.G1r = G1;
    a.G2r = G2;
    a.part = static_cast<double*>(scratch);
    a.tile_base = 0;
    a.work = reinterpret_cast<int*>(static_cast<char*>(scratch) + kNoAllocScratchBytes - kNoAllocCounterBytes);
    // the array keeps the previous call's contents: the tile counter must start at zero
    CDE_CUDA(cudaMemsetAsync(a.work, 0, sizeof(int), st));
    const int grid = a.n_tiles < cmax ? a.n_tiles : cmax;
    // kernel timing (cde_timing_last) covers this call's tile kernel, as in cde_loo_loglik
    timing_reset(ctx);
    timing_begin(ctx, st);
    rc = launch_loo_tile_kernel(T1, T2, a, grid, st);
    timing_end(ctx, st);
    if (rc != CDE_OK) return rc;
    if (d_L_cond || d_L_eq3) {
        const int GG = T1 * T2;
        k_loo_final<<<(GG * 32 + 255) / 256, 256, 0, st>>>(a.part, a.n_tiles, GG, T2, G1, G2, G2,
                                                          (double)D->N, d_L_cond, d_L_eq3);
        CDE_CUDA(cudaGetLastError());
    }
    return CDE_OK;
}
