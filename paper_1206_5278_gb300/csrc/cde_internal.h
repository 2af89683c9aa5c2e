// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cde.h"

namespace cde {

// Thread-local error text; set_error returns the status for `return set_error(...)`.
int set_error(int status, const std::string& msg);
int cuda_error(cudaError_t e, const char* where);

// NVTX range over an entry point (visible to profilers that inject NVTX; a
// few nanoseconds otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define CDE_NVTX(name) ::cde::NvtxRange cde_nvtx_range_(name)

// Checked builds (compiled with -DCDE_CHECKS: libcde_checked.so): CDE_CK(i, n,
// code) tests 0 <= i < n, records the first failing code in this translation
// unit's g_cde_check and returns 0 instead (the access stays inside the
// buffer; nothing traps).  cde_check_status reads and clears the codes of all
// translation units.  Normal builds: CDE_CK(i, n, code) is i.
#if defined(CDE_CHECKS) && defined(__CUDACC__)
static __device__ unsigned int g_cde_check;
__device__ __forceinline__ int64_t cde_ck(int64_t i, int64_t n, unsigned int code) {
    if (i < 0 || i >= n) {
        atomicCAS(&g_cde_check, 0u, code);
        return 0;
    }
    return i;
}
#define CDE_CK(i, n, code) ::cde::cde_ck((int64_t)(i), (int64_t)(n), (code))
// read and clear this translation unit's code (host side)
#define CDE_CHECK_READER(name)                                                   \
    int name(unsigned int* code) {                                               \
        unsigned int v = 0;                                                      \
        CDE_CUDA(cudaMemcpyFromSymbol(&v, g_cde_check, sizeof(v)));              \
        if (v) {                                                                 \
            const unsigned int z = 0;                                            \
            CDE_CUDA(cudaMemcpyToSymbol(g_cde_check, &z, sizeof(z)));            \
        }                                                                        \
        *code = v;                                                               \
        return CDE_OK;                                                           \
    }
#else
#define CDE_CK(i, n, code) (i)
#endif

#define CDE_CUDA(call)                                         \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return ::cde::cuda_error(_e, #call); \
    } while (0)

// Device-resident dataset.  x is stored structure-of-arrays, x[c][i] at
// xs[c * Np + i], padded to Np (a multiple of kPadRows) with zeros.
struct Dataset {
    int64_t id = 0;
    int64_t N = 0, Np = 0;
    int d = 0;
    int standardized = 0;
    int kernel = 0;        // CDE_KERNEL_GAUSS or CDE_KERNEL_EPAN
    float* xs = nullptr;   // [d][Np]
    float* y = nullptr;    // [Np]
    float* mx = nullptr;   // [N] min_{i!=j} |x_j - x_i|^2 (FP32, same formula as the kernels);
                           //     zeros for Epanechnikov datasets (no shift)
    float* my = nullptr;   // [N] min_{i!=j} (y_j - y_i)^2 (zeros for Epanechnikov)
    // [N] each row's nearest neighbours seen from the other coordinate (Gaussian only;
    // they bound where the joint minimum of a1 dx^2 + a2 dy^2 can lie):
    float* qx = nullptr;   //     dx^2 to the y-nearest point (the smallest, if several are y-nearest)
    float* qy = nullptr;   //     dy^2 to the x-nearest point (the smallest, if several are x-nearest)
    std::vector<double> mean, sd;  // per-dimension (identity when not standardised)
    size_t bytes = 0;
    std::atomic<int> users{0};     // jobs currently reading it (serving)
};

constexpr int kPadRows = 256;
constexpr int kMaxD = 64;          // largest d_x handled by the SIMT kernels
// word of cde_ctx::d_err set by a tensor-core kernel whose bounded mbarrier wait ran out
constexpr int kErrTensorWait = 16;

struct Server;  // serve.cpp

}  // namespace cde

struct cde_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    cudaStream_t stream = nullptr;
    std::recursive_mutex mu;  // serialises the synchronous API
    std::mutex ds_mu;         // guards the dataset map
    std::map<int64_t, std::shared_ptr<cde::Dataset>> datasets;
    int64_t next_id = 1;
    cde::Server* server = nullptr;
    int* d_err = nullptr;     // device-side error flag (bounded waits, checks)

    int tune_upt[3][3] = {};  // autotuned units per tile by grid shape (8/16/32), 0 = default
    int tune_ctas[3][3] = {}; // autotuned resident CTAs per SM, 0 = default (2)
    bool tuned[3][3] = {};    // shape class tuned (autotuner, cde_tuning_set*, cde_tuning_load)
    bool autotune_batch = true;  // cde_loo_loglik_batch tunes the untuned shape classes it meets
    void* batch_plan = nullptr;  // cached batched launch (graph), batch.cu
    // workspace of the synchronous host-output calls (they hold `mu` until their
    // stream has drained, so one call uses it at a time): device scratch and a
    // pinned host buffer, grown on demand up to kWorkspaceMax, freed at shutdown
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* ws_host = nullptr;
    size_t ws_host_bytes = 0;
    // kernel timing (cde_timing_enable): events around the dominant kernel of
    // the latest timed call, on that call's stream
    bool timing = false;
    bool tev_open = false;    // tev0 recorded in the current call
    bool tev_set = false;     // a complete pair exists
    cudaEvent_t tev0 = nullptr, tev1 = nullptr;
};

namespace cde {

// Dominant-kernel timing: a call resets, the first dominant launch records
// the start event, every dominant launch re-records the end event.  Threads
// that set t_untimed (the request-queue worker) never touch the events.
inline thread_local bool t_untimed = false;

// A kernel's dynamic shared-memory limit is a per-device attribute: set it once
// per device (the current one) and call site; `done` marks devices 0..63.
template <class Kernel>
inline cudaError_t smem_attr_once(std::atomic<uint64_t>& done, Kernel kern, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}
inline void timing_reset(cde_ctx* c) {
    if (!t_untimed) c->tev_open = false;
}
inline void timing_begin(cde_ctx* c, cudaStream_t st) {
    if (c->timing && !t_untimed && !c->tev_open) {
        cudaEventRecord(c->tev0, st);
        c->tev_open = true;
    }
}
inline void timing_end(cde_ctx* c, cudaStream_t st) {
    if (c->timing && !t_untimed && c->tev_open) {
        cudaEventRecord(c->tev1, st);
        c->tev_set = true;
    }
}

std::shared_ptr<Dataset> find_dataset(cde_ctx* ctx, cde_dataset ds);

// ln c_d of the radial Epanechnikov kernel in d dimensions (loo_grid.cu)
double epan_log_norm(int d);
cudaStream_t pick_stream(cde_ctx* ctx, void* s);

// ---- LOO grid (loo_grid.cu) ----
// Enqueue the LOO score for one dataset over a bandwidth grid (any G1, G2):
// d_Lc / d_Le are device arrays G1 x G2 (either may be null); d_ell_rows
// (n_rows x G1 x G2) is written when rows != null.
// `scratch` (optional, stream-ordered exclusive use): device memory for the tile
// partials and counters; when it is null or smaller than loo_grid_scratch_bytes
// the call allocates from the stream-ordered pool instead.
int loo_grid_enqueue(cde_ctx* ctx, const Dataset& D, const double* h1, int G1, const double* h2,
                     int G2, const int64_t* d_rows, int64_t n_rows, double* d_Lc, double* d_Le,
                     double* d_ell_rows, cudaStream_t st, void* scratch = nullptr,
                     size_t scratch_bytes = 0);
size_t loo_grid_scratch_bytes(cde_ctx* ctx, const Dataset& D, int G1, int G2, int64_t n_rows);

// One grid block (G1, G2 <= 32) launched in parts, each its own launch: windows
// of units of the large tiles, then ranges of the small tiles.  Every tile adds
// its units to a fixed partial slot in unit order and the final reduction is
// loo_grid_enqueue's, so the result is bitwise that of one launch (the request
// loop runs selection grids this way, so queued density jobs run in between).
// Scratch: loo_chunked_scratch_bytes, stream-ordered, the caller's for the whole sequence.
struct LooChunked;
int loo_chunked_create(cde_ctx* ctx, const Dataset& D, const double* h1, int G1, const double* h2, int G2,
                       LooChunked** out);
void loo_chunked_destroy(LooChunked* c);
size_t loo_chunked_scratch_bytes(const LooChunked* c);
// the next part, about `pair_evals` pair evaluations (at least one unit per large
// tile, or one small tile per CTA); *done = 1 once every unit has been launched
int loo_chunked_next(LooChunked* c, void* scratch, double pair_evals, cudaStream_t st, int* done);
int loo_chunked_final(const LooChunked* c, const void* scratch, double* d_Lc, double* d_Le, cudaStream_t st);

constexpr size_t kWorkspaceMax = (size_t)64 << 20;
// Make ctx->ws at least `dev` bytes and ctx->ws_host at least `host` bytes
// (synchronous growth; callers hold ctx->mu and no work of theirs is in flight).
int workspace_reserve(cde_ctx* ctx, size_t dev, size_t host);

// Nearest squared distances per row (cached at dataset creation).
int nn_shift_enqueue(const Dataset& D, cudaStream_t st, int sm_count);

// Standardise / pack raw row-major x into the SoA layout (device input).
int pack_enqueue(Dataset& D, const float* d_x_rowmajor, const float* d_y, cudaStream_t st,
                 double* d_stats);

// ---- gradient (loo_grad.cu) ----
// d_rowv (optional, N x 3 doubles) receives per-row {ell_j, d ell_j/d ln h1, d ell_j/d ln h2}.
// A gradient evaluation in launches over ranges of row blocks (bitwise the
// single launch's result): create (scratch, stream-ordered), next until *done,
// then finish (per-row merge, sums into d_out3 if given; frees the sequence) or
// free on an error.
struct GradChunked;
int grad_chunked_create(cde_ctx* ctx, const Dataset& D, double h1, double h2, cudaStream_t st, double* d_rowv_ext,
                        GradChunked** out);
int grad_chunked_next(GradChunked* c, double pair_evals, cudaStream_t st, int* done);
int grad_chunked_finish(cde_ctx* ctx, GradChunked* c, double* d_out3, cudaStream_t st);
void grad_chunked_free(GradChunked* c, cudaStream_t st);
int loo_grad_enqueue(cde_ctx* ctx, const Dataset& D, double h1, double h2, double* d_out3,
                     cudaStream_t st, double* d_rowv);

// ---- density (density.cu) ----
// per-query nearest squared distances m_q (FP32, pair-kernel formula) of
// packed queries xq [d][Qp]; mq holds Q floats
int query_shift_enqueue(int sm_count, const Dataset& D, const float* xq, int64_t Q, int64_t Qp, float* mq,
                        cudaStream_t st);
int density_enqueue(cde_ctx* ctx, const Dataset& D, double h1, double h2, const float* d_xq,
                    int64_t Q, const float* d_yg, int G, float* d_f, cudaStream_t st);

// ---- batched (batch.cu) ----
struct BatchItem {
    const Dataset* D;
    const double* h1; int G1;
    const double* h2; int G2;
    double* d_Lc;   // device G1 x G2 (may be null)
    double* d_Le;
};
// Run (building and capturing on first use) the batched launch; host outputs.
int loo_batch_run(cde_ctx* ctx, const std::vector<BatchItem>& items, std::vector<double*>& Lc,
                  std::vector<double*>& Le, cudaStream_t st);
void batch_plan_free(cde_ctx* ctx);

// ---- peaks (peaks.cu) ----
int measure_peaks(cde_ctx* ctx, cde_peaks* out);

}  // namespace cde
