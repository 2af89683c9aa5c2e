// C ABI: context, errors, datasets and the synchronous entry points.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "cde_internal.h"

namespace cde {

static thread_local std::string g_err;

int set_error(int status, const std::string& msg) {
    g_err = msg;
    return status;
}

int cuda_error(cudaError_t e, const char* where) {
    const int st = (e == cudaErrorMemoryAllocation) ? CDE_ENOMEM : CDE_ECUDA;
    return set_error(st, std::string(where) + ": " + cudaGetErrorString(e));
}

std::shared_ptr<Dataset> find_dataset(cde_ctx* ctx, cde_dataset ds) {
    std::lock_guard<std::mutex> g(ctx->ds_mu);
    auto it = ctx->datasets.find(ds);
    return it == ctx->datasets.end() ? nullptr : it->second;
}

cudaStream_t pick_stream(cde_ctx* ctx, void* s) {
    return s ? reinterpret_cast<cudaStream_t>(s) : ctx->stream;
}

static bool bandwidth_ok(double h) { return std::isfinite(h) && h >= 1e-12 && h <= 1e12; }

static int check_grid(const double* h, int G, const char* name) {
    if (!h || G < 1) return set_error(CDE_EINVAL, std::string(name) + ": empty bandwidth grid");
    for (int k = 0; k < G; ++k)
        if (!bandwidth_ok(h[k]))
            return set_error(CDE_EINVAL, std::string(name) + ": bandwidth must be finite in [1e-12, 1e12]");
    return CDE_OK;
}

static void free_dataset(Dataset* D) {
    cudaFree(D->xs);
    cudaFree(D->y);
    cudaFree(D->mx);
    cudaFree(D->my);
    cudaFree(D->qx);
    cudaFree(D->qy);
    D->xs = D->y = D->mx = D->my = D->qx = D->qy = nullptr;
}

__global__ void k_finite_check(const float* a, int64_t n, int* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[i])) atomicOr(flag, 1);
}

}  // namespace cde

namespace cde {
int workspace_reserve(cde_ctx* ctx, size_t dev, size_t host) {
    if (dev > ctx->ws_bytes) {
        if (ctx->ws) CDE_CUDA(cudaFree(ctx->ws));
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        CDE_CUDA(cudaMalloc(&ctx->ws, dev));
        ctx->ws_bytes = dev;
    }
    if (host > ctx->ws_host_bytes) {
        if (ctx->ws_host) CDE_CUDA(cudaFreeHost(ctx->ws_host));
        ctx->ws_host = nullptr;
        ctx->ws_host_bytes = 0;
        CDE_CUDA(cudaMallocHost(&ctx->ws_host, host));
        ctx->ws_host_bytes = host;
    }
    return CDE_OK;
}
}  // namespace cde

#ifdef CDE_CHECKS
namespace cde {
int check_status_loo(unsigned int*);
int check_status_batch(unsigned int*);
int check_status_density(unsigned int*);
int check_status_products(unsigned int*);
int check_status_grad(unsigned int*);
int check_status_gram(unsigned int*);
}  // namespace cde
#endif

using namespace cde;

extern "C" {

const char* cde_version(void) { return "cde-gb300 0.1 (sm_103a)"; }

const char* cde_last_error(void) { return g_err.c_str(); }

int cde_init(cde_ctx** out, int device, size_t budget) {
    if (!out) return set_error(CDE_EINVAL, "cde_init: null output");
    *out = nullptr;
    int n = 0;
    CDE_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return set_error(CDE_EINVAL, "cde_init: no such device");
    CDE_CUDA(cudaSetDevice(device));
    cudaDeviceProp p;
    CDE_CUDA(cudaGetDeviceProperties(&p, device));
    if (p.major * 10 + p.minor < 100)
        return set_error(CDE_EINVAL, "cde_init: device is not a Blackwell-class GPU");
    auto* ctx = new cde_ctx();
    ctx->device = device;
    ctx->sm_count = p.multiProcessorCount;
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        delete ctx;
        return cuda_error(e, "cudaMemGetInfo");
    }
    ctx->budget = budget ? budget : (size_t)(0.9 * (double)fr);
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_err, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, 64 * sizeof(int));
    if (e != cudaSuccess) {
        if (ctx->stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return cuda_error(e, "cde_init");
    }
    // CDE_AUTOTUNE=0: the batched call runs untuned shape classes with the defaults
    if (const char* at = getenv("CDE_AUTOTUNE")) ctx->autotune_batch = strcmp(at, "0") != 0;
    // a tuning cache named by the environment is applied when it matches this device
    if (const char* tc = getenv("CDE_TUNING_CACHE")) {
        if (cde_tuning_load(ctx, tc) != CDE_OK) set_error(CDE_OK, "");
    }
    *out = ctx;
    return CDE_OK;
}

void cde_server_stop_internal(cde_ctx* ctx);

void cde_shutdown(cde_ctx* ctx) {
    if (!ctx) return;
    cde_server_stop_internal(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    batch_plan_free(ctx);
    {
        std::lock_guard<std::mutex> g(ctx->ds_mu);
        for (auto& kv : ctx->datasets) free_dataset(kv.second.get());
        ctx->datasets.clear();
    }
    cudaFree(ctx->d_err);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->ws_host) cudaFreeHost(ctx->ws_host);
    if (ctx->tev0) cudaEventDestroy(ctx->tev0);
    if (ctx->tev1) cudaEventDestroy(ctx->tev1);
    cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int cde_create_dataset(cde_ctx* ctx, const float* x, const float* y, int64_t N, int d, int standardize,
                       int flags, cde_dataset* out) {
    CDE_NVTX("cde_create_dataset");
    if (!ctx || !x || !y || !out) return set_error(CDE_EINVAL, "cde_create_dataset: null argument");
    if (N < 2) return set_error(CDE_EINVAL, "cde_create_dataset: need N >= 2");
    if (N > (int64_t)1 << 30) return set_error(CDE_EINVAL, "cde_create_dataset: N too large");
    if (d < 1 || d > kMaxD) return set_error(CDE_EINVAL, "cde_create_dataset: d_x must be in [1, 64]");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    const bool in_dev = flags & CDE_IN_DEVICE;
    if (!in_dev) {
        for (int64_t i = 0; i < N * d; ++i)
            if (!std::isfinite(x[i])) return set_error(CDE_EINVAL, "cde_create_dataset: non-finite x");
        for (int64_t i = 0; i < N; ++i)
            if (!std::isfinite(y[i])) return set_error(CDE_EINVAL, "cde_create_dataset: non-finite y");
    }
    auto D = std::make_shared<Dataset>();
    D->N = N;
    D->d = d;
    D->Np = (N + kPadRows - 1) / kPadRows * kPadRows;
    D->standardized = standardize ? 1 : 0;
    D->kernel = (flags & CDE_KERNEL_EPANECHNIKOV) ? CDE_KERNEL_EPAN : CDE_KERNEL_GAUSS;
    D->bytes = (size_t)D->Np * (d + 1) * 4 + (size_t)N * 16;
    if (ctx->used.load() + D->bytes > ctx->budget)
        return set_error(CDE_ENOMEM, "cde_create_dataset: memory budget exceeded");
    cudaStream_t st = ctx->stream;
    float *dx = nullptr, *dy = nullptr;
    double* dstats = nullptr;
    int rc = CDE_OK;
    auto fail = [&](int r) {
        cudaStreamSynchronize(st);
        if (!in_dev) {
            cudaFree(dx);
            cudaFree(dy);
        }
        cudaFree(dstats);
        free_dataset(D.get());
        return r;
    };
    cudaError_t e = cudaMalloc((void**)&D->xs, (size_t)D->Np * d * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D->y, (size_t)D->Np * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D->mx, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D->my, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D->qx, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D->qy, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dstats, (size_t)2 * d * sizeof(double) + 64);
    if (e != cudaSuccess) return fail(cuda_error(e, "cde_create_dataset: cudaMalloc"));
    if (in_dev) {
        dx = const_cast<float*>(x);
        dy = const_cast<float*>(y);
        int* flag = ctx->d_err + 8;
        e = cudaMemsetAsync(flag, 0, sizeof(int), st);
        if (e == cudaSuccess) {
            k_finite_check<<<256, 256, 0, st>>>(dx, N * d, flag);
            k_finite_check<<<64, 256, 0, st>>>(dy, N, flag);
            int h = 0;
            e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && h) return fail(set_error(CDE_EINVAL, "cde_create_dataset: non-finite input"));
        }
        if (e != cudaSuccess) return fail(cuda_error(e, "cde_create_dataset: finite check"));
    } else {
        e = cudaMalloc((void**)&dx, (size_t)N * d * 4);
        if (e == cudaSuccess) e = cudaMalloc((void**)&dy, (size_t)N * 4);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, (size_t)N * d * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, (size_t)N * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(cuda_error(e, "cde_create_dataset: upload"));
    }
    rc = pack_enqueue(*D, dx, dy, st, dstats);
    if (rc != CDE_OK) return fail(rc);
    std::vector<double> stats(2 * d, 0.0);
    if (standardize) {
        e = cudaMemcpyAsync(stats.data(), dstats, 2 * d * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(cuda_error(e, "cde_create_dataset: stats"));
        for (int c = 0; c < d; ++c)
            if (!(stats[2 * c + 1] > 0.0))
                return fail(set_error(CDE_EINVAL, "cde_create_dataset: zero spread in a dimension"));
    }
    if (D->kernel == CDE_KERNEL_GAUSS) {
        rc = nn_shift_enqueue(*D, st, ctx->sm_count);
        if (rc != CDE_OK) return fail(rc);
    } else {
        e = cudaMemsetAsync(D->mx, 0, (size_t)N * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(D->my, 0, (size_t)N * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(D->qx, 0, (size_t)N * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(D->qy, 0, (size_t)N * 4, st);
        if (e != cudaSuccess) return fail(cuda_error(e, "cde_create_dataset: shifts"));
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_error(e, "cde_create_dataset: kernels"));
    if (!in_dev) {
        cudaFree(dx);
        cudaFree(dy);
    }
    cudaFree(dstats);
    D->mean.resize(d);
    D->sd.resize(d);
    for (int c = 0; c < d; ++c) {
        D->mean[c] = standardize ? stats[2 * c] : 0.0;
        D->sd[c] = standardize ? stats[2 * c + 1] : 1.0;
    }
    ctx->used += D->bytes;
    {
        std::lock_guard<std::mutex> g(ctx->ds_mu);
        D->id = ctx->next_id++;
        ctx->datasets[D->id] = D;
    }
    *out = D->id;
    return CDE_OK;
}

int cde_destroy_dataset(cde_ctx* ctx, cde_dataset ds) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_destroy_dataset: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    std::shared_ptr<Dataset> D;
    {
        std::lock_guard<std::mutex> g(ctx->ds_mu);
        auto it = ctx->datasets.find(ds);
        if (it == ctx->datasets.end()) return set_error(CDE_ENOTFOUND, "cde_destroy_dataset: unknown dataset");
        if (it->second->users.load() > 0) return set_error(CDE_EBUSY, "cde_destroy_dataset: dataset in use");
        D = it->second;
        ctx->datasets.erase(it);
    }
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaDeviceSynchronize();
    batch_plan_free(ctx);  // a captured batch may reference this dataset
    free_dataset(D.get());
    ctx->used -= D->bytes;
    return CDE_OK;
}

int cde_dataset_info(cde_ctx* ctx, cde_dataset ds, int64_t* N, int* d, double* mean, double* sd) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_dataset_info: null context");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_dataset_info: unknown dataset");
    if (N) *N = D->N;
    if (d) *d = D->d;
    for (int c = 0; c < D->d; ++c) {
        if (mean) mean[c] = D->mean[c];
        if (sd) sd[c] = D->sd[c];
    }
    return CDE_OK;
}

int cde_check_status(cde_ctx* ctx, unsigned int* code, int* enabled) {
    if (!ctx || !code) return set_error(CDE_EINVAL, "cde_check_status: null argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    *code = 0;
#ifdef CDE_CHECKS
    if (enabled) *enabled = 1;
    CDE_CUDA(cudaDeviceSynchronize());
    int (*readers[])(unsigned int*) = {check_status_loo, check_status_batch, check_status_density,
                                       check_status_products, check_status_grad, check_status_gram};
    for (auto rd : readers) {
        unsigned int c = 0;
        const int rc = rd(&c);
        if (rc != CDE_OK) return rc;
        if (!*code && c) *code = c;
    }
#else
    if (enabled) *enabled = 0;
    CDE_CUDA(cudaDeviceSynchronize());
#endif
    int tw = 0;
    CDE_CUDA(cudaMemcpy(&tw, ctx->d_err + kErrTensorWait, sizeof(int), cudaMemcpyDeviceToHost));
    if (tw) {
        CDE_CUDA(cudaMemset(ctx->d_err + kErrTensorWait, 0, sizeof(int)));
        if (!*code) *code = CDE_CHECK_TENSOR_WAIT | (unsigned int)tw;
    }
    return CDE_OK;
}

int cde_timing_enable(cde_ctx* ctx, int on) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_timing_enable: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    if (on && !ctx->tev0) {
        CDE_CUDA(cudaEventCreate(&ctx->tev0));
        CDE_CUDA(cudaEventCreate(&ctx->tev1));
    }
    ctx->timing = on != 0;
    ctx->tev_open = ctx->tev_set = false;
    return CDE_OK;
}

int cde_timing_last(cde_ctx* ctx, double* ms) {
    if (!ctx || !ms) return set_error(CDE_EINVAL, "cde_timing_last: null argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!ctx->tev_set) return set_error(CDE_EINVAL, "cde_timing_last: no timed kernel yet");
    CDE_CUDA(cudaSetDevice(ctx->device));
    CDE_CUDA(cudaEventSynchronize(ctx->tev1));
    float f = 0.f;
    CDE_CUDA(cudaEventElapsedTime(&f, ctx->tev0, ctx->tev1));
    *ms = f;
    return CDE_OK;
}

int cde_dataset_nn(cde_ctx* ctx, cde_dataset ds, float* nn_x2, float* nn_y2) {
    if (!ctx || (!nn_x2 && !nn_y2)) return set_error(CDE_EINVAL, "cde_dataset_nn: null argument");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_dataset_nn: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    if (nn_x2) CDE_CUDA(cudaMemcpyAsync(nn_x2, D->mx, (size_t)D->N * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (nn_y2) CDE_CUDA(cudaMemcpyAsync(nn_y2, D->my, (size_t)D->N * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CDE_CUDA(cudaStreamSynchronize(ctx->stream));
    return CDE_OK;
}

int cde_dataset_nn_other(cde_ctx* ctx, cde_dataset ds, float* other_x2, float* other_y2) {
    if (!ctx || (!other_x2 && !other_y2)) return set_error(CDE_EINVAL, "cde_dataset_nn_other: null argument");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_dataset_nn_other: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    if (other_x2) CDE_CUDA(cudaMemcpyAsync(other_x2, D->qx, (size_t)D->N * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (other_y2) CDE_CUDA(cudaMemcpyAsync(other_y2, D->qy, (size_t)D->N * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CDE_CUDA(cudaStreamSynchronize(ctx->stream));
    return CDE_OK;
}

int cde_dataset_kernel(cde_ctx* ctx, cde_dataset ds, int* kernel) {
    if (!ctx || !kernel) return set_error(CDE_EINVAL, "cde_dataset_kernel: null argument");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_dataset_kernel: unknown dataset");
    *kernel = D->kernel;
    return CDE_OK;
}

int cde_loo_loglik(cde_ctx* ctx, cde_dataset ds, const double* h1, int G1, const double* h2, int G2,
                   double* Lc, double* Le, int flags, void* stream) {
    CDE_NVTX("cde_loo_loglik");
    if (!ctx) return set_error(CDE_EINVAL, "cde_loo_loglik: null context");
    int rc = check_grid(h1, G1, "h1");
    if (rc == CDE_OK) rc = check_grid(h2, G2, "h2");
    if (rc != CDE_OK) return rc;
    if ((int64_t)G1 * G2 > (1 << 24)) return set_error(CDE_EINVAL, "cde_loo_loglik: grid too large");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_loo_loglik: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    if (flags & CDE_OUT_DEVICE) return loo_grid_enqueue(ctx, *D, h1, G1, h2, G2, nullptr, 0, Lc, Le, nullptr, st);
    const size_t n = (size_t)G1 * G2;
    // small calls: the context workspace (no per-call allocation, one copy into pinned memory)
    const size_t out_bytes = (2 * n * sizeof(double) + 255) & ~(size_t)255;
    const size_t scr = loo_grid_scratch_bytes(ctx, *D, G1, G2, D->N);
    if (out_bytes + scr <= kWorkspaceMax && workspace_reserve(ctx, out_bytes + scr, 2 * n * sizeof(double)) == CDE_OK) {
        double* dout = static_cast<double*>(ctx->ws);
        rc = loo_grid_enqueue(ctx, *D, h1, G1, h2, G2, nullptr, 0, dout, dout + n, nullptr, st,
                              static_cast<char*>(ctx->ws) + out_bytes, ctx->ws_bytes - out_bytes);
        cudaError_t e = cudaSuccess;
        if (rc == CDE_OK) e = cudaMemcpyAsync(ctx->ws_host, dout, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (rc != CDE_OK) return rc;
        if (e != cudaSuccess) return cuda_error(e, "cde_loo_loglik: copy");
        if (e2 != cudaSuccess) return cuda_error(e2, "cde_loo_loglik: kernels");
        const double* hb = static_cast<const double*>(ctx->ws_host);
        if (Lc) memcpy(Lc, hb, n * sizeof(double));
        if (Le) memcpy(Le, hb + n, n * sizeof(double));
        return CDE_OK;
    }
    double* dbuf = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&dbuf, 2 * n * sizeof(double), st));
    rc = loo_grid_enqueue(ctx, *D, h1, G1, h2, G2, nullptr, 0, Lc ? dbuf : nullptr, Le ? dbuf + n : nullptr,
                          nullptr, st);
    cudaError_t e = cudaSuccess;
    if (rc == CDE_OK && Lc) e = cudaMemcpyAsync(Lc, dbuf, n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (rc == CDE_OK && e == cudaSuccess && Le)
        e = cudaMemcpyAsync(Le, dbuf + n, n * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dbuf, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (rc != CDE_OK) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cde_loo_loglik: copy");
    if (e2 != cudaSuccess) return cuda_error(e2, "cde_loo_loglik: kernels");
    return CDE_OK;
}

int cde_loo_rows(cde_ctx* ctx, cde_dataset ds, const double* h1, int G1, const double* h2, int G2,
                 const int64_t* rows, int64_t n_rows, double* ell_out, void* stream) {
    CDE_NVTX("cde_loo_rows");
    if (!ctx || !rows || !ell_out) return set_error(CDE_EINVAL, "cde_loo_rows: null argument");
    int rc = check_grid(h1, G1, "h1");
    if (rc == CDE_OK) rc = check_grid(h2, G2, "h2");
    if (rc != CDE_OK) return rc;
    if (n_rows < 1) return set_error(CDE_EINVAL, "cde_loo_rows: need n_rows >= 1");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_loo_rows: unknown dataset");
    for (int64_t r = 0; r < n_rows; ++r)
        if (rows[r] < 0 || rows[r] >= D->N) return set_error(CDE_EINVAL, "cde_loo_rows: row out of range");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    const size_t n = (size_t)n_rows * G1 * G2;
    int64_t* drows = nullptr;
    double* dell = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&drows, n_rows * sizeof(int64_t), st));
    CDE_CUDA(cudaMallocAsync((void**)&dell, n * sizeof(double), st));
    cudaError_t e = cudaMemcpyAsync(drows, rows, n_rows * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        rc = loo_grid_enqueue(ctx, *D, h1, G1, h2, G2, drows, n_rows, nullptr, nullptr, dell, st);
    if (e == cudaSuccess && rc == CDE_OK)
        e = cudaMemcpyAsync(ell_out, dell, n * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(drows, st);
    cudaFreeAsync(dell, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (rc != CDE_OK) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cde_loo_rows");
    if (e2 != cudaSuccess) return cuda_error(e2, "cde_loo_rows: kernels");
    return CDE_OK;
}

}  // extern "C"
