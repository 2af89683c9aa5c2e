// Many datasets, one persistent launch per grid shape, inside a captured
// CUDA graph; plus the autotuner of the per-shape tile parameters.
//
// Every dataset contributes (dataset, tile) work items -- the same tiles the
// single-dataset launch forms (loo_units_per_tile) -- to one queue ordered
// longest-first (cost N^2 per tile row).  Persistent CTAs take items from an
// atomic counter; when a CTA switches dataset it copies that dataset's
// argument block (coefficients included) into shared memory and runs the
// shared tile body.  Tile partials land in per-dataset slots and are reduced
// by the same fixed-order cell reduction as the single launch, so each
// dataset's scores are bitwise identical to cde_loo_loglik on it alone.
//
// The launch sequence (counter reset, one persistent kernel per shape, the
// final reductions and the copy of all scores to pinned host memory) is
// captured once into a CUDA graph and replayed while the batch (datasets and
// bandwidth grids) stays the same.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "cde_internal.h"
#include "loo_common.cuh"
#include "loo_mma.cuh"

namespace cde {

template <int G1, int G2, int KERN>
__global__ void __launch_bounds__(256, 2) k_loo_batch(const LooArgs* __restrict__ items,
                                                      const int2* __restrict__ work, int n_work,
                                                      int* counter) {
    extern __shared__ float4 sm4[];
    __shared__ LooArgs A;
    __shared__ int next_w, need, cur;
    if (threadIdx.x == 0) cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const int w = atomicAdd(counter, 1);
            next_w = w;
            need = 0;
            if (w < n_work && work[w].x != cur) {
                need = 1;
                cur = work[w].x;
            }
        }
        __syncthreads();
        const int w = next_w;
        if (w >= n_work) break;
        if (need) {
            const int* src = reinterpret_cast<const int*>(items + work[w].x);
            int* dst = reinterpret_cast<int*>(&A);
            for (int e = threadIdx.x; e < (int)(sizeof(LooArgs) / sizeof(int)); e += blockDim.x)
                dst[e] = src[e];
            __syncthreads();
        }
        const CoefSmem cf{A.a1, A.a2};
        loo_tile_mma<G1, G2, KERN>(A, cf, work[w].y, reinterpret_cast<float*>(sm4));
    }
}

// one warp per (item, cell); same reduction as the single launch
__global__ void k_loo_final_batch(const LooArgs* __restrict__ items, const int* __restrict__ item_cell0,
                                  int n_items, int GG, int G2T, const int64_t* __restrict__ out_off,
                                  double* __restrict__ out) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    // locate the item: cells are numbered item-major
    int lo = 0, hi = n_items;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (item_cell0[mid] <= gw) lo = mid;
        else hi = mid;
    }
    if (gw >= item_cell0[n_items]) return;
    const int it = lo, cell = gw - item_cell0[it];
    const LooArgs& a = items[it];
    double sc, se;
    loo_final_cell(a.part, a.n_tiles, GG, cell, lane, sc, se);
    const int k = cell / G2T, l = cell % G2T;
    if (lane == 0 && k < a.G1r && l < a.G2r) {
        const int n = a.G1r * a.G2r;
        double* o = out + out_off[it];
        o[k * a.G2r + l] = sc;
        o[n + k * a.G2r + l] = se / (double)a.N - log((double)a.N - 1.0);
    }
}

template <int G1, int G2, int KERN>
static int launch_batch_shape_k(const LooArgs* d_items, const int2* d_work, int n_work, int* counter,
                                int grid, cudaStream_t st, int dmax) {
    using C = MmaCfg<G1, G2>;
    static std::atomic<uint64_t> attr{0};
    CDE_CUDA(smem_attr_once(attr, k_loo_batch<G1, G2, KERN>, (int)C::smem_bytes(kMaxD)));
    k_loo_batch<G1, G2, KERN><<<grid, C::kThreads, C::smem_bytes(dmax), st>>>(d_items, d_work, n_work, counter);
    CDE_CUDA(cudaGetLastError());
    return CDE_OK;
}

template <int G1, int G2>
static int launch_batch_shape(int kern, const LooArgs* d_items, const int2* d_work, int n_work,
                              int* counter, int grid, cudaStream_t st, int dmax) {
    return kern == CDE_KERNEL_EPAN
               ? launch_batch_shape_k<G1, G2, 1>(d_items, d_work, n_work, counter, grid, st, dmax)
               : launch_batch_shape_k<G1, G2, 0>(d_items, d_work, n_work, counter, grid, st, dmax);
}

// work groups are keyed by kern * 4096 + T1 * 64 + T2
static int shape_t1(int key) { return (key % 4096) / 64; }
static int shape_t2(int key) { return key % 64; }
static int shape_kern(int key) { return key / 4096; }

static int launch_batch(int T1, int T2, int kern, const LooArgs* d_items, const int2* d_work, int n_work,
                        int* counter, int grid, cudaStream_t st, int dmax) {
#define CDE_BSHAPE(A, B) \
    if (T1 == A && T2 == B) return launch_batch_shape<A, B>(kern, d_items, d_work, n_work, counter, grid, st, dmax);
    CDE_BSHAPE(16, 8) CDE_BSHAPE(16, 16) CDE_BSHAPE(16, 32)
    CDE_BSHAPE(32, 8) CDE_BSHAPE(32, 16) CDE_BSHAPE(32, 32)
#undef CDE_BSHAPE
    return set_error(CDE_EINVAL, "batch: unsupported grid shape");
}



// A captured batched launch and the device memory it references.
struct BatchPlan {
    std::vector<int64_t> key_ids;
    std::vector<double> key_h;
    std::vector<int> key_g;
    int tune_stamp = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* dmem = nullptr;        // items, work, counters, partials, outputs
    double* hout = nullptr;      // pinned copy of all outputs
    size_t out_doubles = 0;
    std::vector<int64_t> out_off;
    std::vector<int> gsz;        // G1*G2 per item
    cudaStream_t stream = nullptr;
    int kernel_launches = 0;
    ~BatchPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (dmem) cudaFree(dmem);
        if (hout) cudaFreeHost(hout);
        if (stream) cudaStreamDestroy(stream);
    }
};

static int tune_stamp_of(cde_ctx* ctx) {
    int s = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s = s * 31 + ctx->tune_upt[a][b] * 7 + ctx->tune_ctas[a][b];
    return s;
}

static int build_plan(cde_ctx* ctx, const std::vector<BatchItem>& items, BatchPlan& P) {
    const int n = (int)items.size();
    // group by padded shape
    std::vector<LooArgs> args(n);
    std::vector<int> shape(n);
    size_t part_doubles = 0;
    P.out_off.resize(n);
    P.gsz.resize(n);
    size_t out = 0;
    int dmax = 1;
    for (int b = 0; b < n; ++b) {
        const BatchItem& it = items[b];
        const int T1 = loo_pad1(it.G1), T2 = loo_pad2(it.G2);
        shape[b] = it.D->kernel * 4096 + T1 * 64 + T2;
        LooArgs& a = args[b];
        memset(&a, 0, sizeof(a));
        fill_loo_args(a, *it.D, it.h1, it.G1, it.h2, it.G2, T1, T2);
        const int JW = 1024 / (T1 * T2);
        a.rows = nullptr;
        a.n_rows = it.D->N;
        a.n_units = (int)((it.D->N + JW - 1) / JW);
        a.units_per_tile = loo_units_per_tile(ctx, T1, T2, it.D->N);
        // the single launch's partition (its grid size), so that the partials agree
        const LooTiles tp = loo_tiles(a.n_units, a.units_per_tile, loo_grid_ctas(ctx, T1, T2));
        a.n_tiles = tp.n_tiles;
        a.big_g = tp.big_g;
        a.big_levels = tp.big_levels;
        a.big_s0 = tp.big_s0;
        a.win0 = 0;
        a.win1 = INT_MAX;
        a.G1r = it.G1;
        a.G2r = it.G2;
        a.ell_rows = nullptr;
        part_doubles += (size_t)a.n_tiles * 2 * T1 * T2;
        P.out_off[b] = (int64_t)out;
        P.gsz[b] = it.G1 * it.G2;
        out += 2 * (size_t)it.G1 * it.G2;
        dmax = std::max(dmax, it.D->d);
    }
    P.out_doubles = out;
    std::vector<int> shapes(shape);
    std::sort(shapes.begin(), shapes.end());
    shapes.erase(std::unique(shapes.begin(), shapes.end()), shapes.end());
    // work lists per shape, longest datasets first
    std::vector<std::vector<int2>> work(shapes.size());
    std::vector<std::vector<int>> members(shapes.size());
    for (size_t s = 0; s < shapes.size(); ++s) {
        for (int b = 0; b < n; ++b)
            if (shape[b] == shapes[s]) members[s].push_back(b);
        std::stable_sort(members[s].begin(), members[s].end(),
                         [&](int x, int y) { return items[x].D->N > items[y].D->N; });
        for (int b : members[s])
            for (int t = 0; t < args[b].n_tiles; ++t) work[s].push_back(make_int2(b, t));
    }
    // one device allocation
    size_t work_n = 0;
    for (auto& w : work) work_n += w.size();
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t off_items = 0;
    const size_t off_work = al(off_items + sizeof(LooArgs) * n);
    const size_t off_cnt = al(off_work + sizeof(int2) * work_n);
    const size_t off_cell0 = al(off_cnt + sizeof(int) * 2 * shapes.size());
    const size_t off_ooff = al(off_cell0 + sizeof(int) * (n + 1) * shapes.size());
    const size_t off_part = al(off_ooff + sizeof(int64_t) * n);
    const size_t off_out = al(off_part + sizeof(double) * part_doubles);
    const size_t total = al(off_out + sizeof(double) * out);
    CDE_CUDA(cudaMalloc(&P.dmem, total));
    char* base = static_cast<char*>(P.dmem);
    double* dpart = reinterpret_cast<double*>(base + off_part);
    size_t po = 0;
    for (int b = 0; b < n; ++b) {
        args[b].part = dpart + po;
        const int GG = shape_t1(shape[b]) * shape_t2(shape[b]);
        po += (size_t)args[b].n_tiles * 2 * GG;
    }
    CDE_CUDA(cudaMallocHost((void**)&P.hout, sizeof(double) * std::max<size_t>(out, 1)));
    CDE_CUDA(cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking));
    cudaStream_t st = P.stream;
    LooArgs* d_items = reinterpret_cast<LooArgs*>(base + off_items);
    CDE_CUDA(cudaMemcpy(d_items, args.data(), sizeof(LooArgs) * n, cudaMemcpyHostToDevice));
    int2* d_work = reinterpret_cast<int2*>(base + off_work);
    std::vector<size_t> woff(shapes.size());
    size_t wo = 0;
    for (size_t s = 0; s < shapes.size(); ++s) {
        woff[s] = wo;
        if (!work[s].empty())
            CDE_CUDA(cudaMemcpy(d_work + wo, work[s].data(), sizeof(int2) * work[s].size(),
                                cudaMemcpyHostToDevice));
        wo += work[s].size();
    }
    int* d_cnt = reinterpret_cast<int*>(base + off_cnt);
    int* d_cell0 = reinterpret_cast<int*>(base + off_cell0);
    int64_t* d_ooff = reinterpret_cast<int64_t*>(base + off_ooff);
    CDE_CUDA(cudaMemcpy(d_ooff, P.out_off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
    double* d_out = reinterpret_cast<double*>(base + off_out);
    // per shape: a LooArgs sub-array view in member order for the final kernel
    std::vector<std::vector<int>> cell0(shapes.size());
    for (size_t s = 0; s < shapes.size(); ++s) {
        const int T1 = shape_t1(shapes[s]), T2 = shape_t2(shapes[s]);
        cell0[s].resize(n + 1, 0);
        // item-major cell numbering over all n items; items of other shapes get 0 cells
        int acc = 0;
        for (int b = 0; b < n; ++b) {
            cell0[s][b] = acc;
            if (shape[b] == shapes[s]) acc += T1 * T2;
        }
        cell0[s][n] = acc;
        CDE_CUDA(cudaMemcpy(d_cell0 + (size_t)s * (n + 1), cell0[s].data(), sizeof(int) * (n + 1),
                            cudaMemcpyHostToDevice));
    }
    // capture
    P.kernel_launches = 0;
    CDE_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = CDE_OK;
    cudaError_t e = cudaMemsetAsync(d_cnt, 0, sizeof(int) * 2 * shapes.size(), st);
    for (size_t s = 0; s < shapes.size() && rc == CDE_OK && e == cudaSuccess; ++s) {
        const int T1 = shape_t1(shapes[s]), T2 = shape_t2(shapes[s]);
        const int n_work = (int)work[s].size();
        const int cmax = loo_grid_ctas(ctx, T1, T2);
        const int grid = std::max(1, std::min(n_work, cmax));
        rc = launch_batch(T1, T2, shape_kern(shapes[s]), d_items, d_work + woff[s], n_work, d_cnt + s,
                          grid, st, dmax);
        if (rc != CDE_OK) break;
        const int GG = T1 * T2;
        const int cells = cell0[s][n];
        k_loo_final_batch<<<(cells * 32 + 255) / 256, 256, 0, st>>>(
            d_items, d_cell0 + (size_t)s * (n + 1), n, GG, T2, d_ooff, d_out);
        e = cudaGetLastError();
        P.kernel_launches += 2;
    }
    if (e == cudaSuccess && rc == CDE_OK && out)
        e = cudaMemcpyAsync(P.hout, d_out, sizeof(double) * out, cudaMemcpyDeviceToHost, st);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (rc != CDE_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_error(e, "batch: capture");
    }
    if (e2 != cudaSuccess) return cuda_error(e2, "batch: end capture");
    P.graph = g;
    CDE_CUDA(cudaGraphInstantiate(&P.exec, g, 0));
    return CDE_OK;
}

int loo_batch_run(cde_ctx* ctx, const std::vector<BatchItem>& items, std::vector<double*>& Lc,
                  std::vector<double*>& Le, cudaStream_t user_st) {
    // key of the batch: datasets, grids and tuning state
    std::vector<int64_t> ids;
    std::vector<double> hs;
    std::vector<int> gs;
    for (const auto& it : items) {
        ids.push_back(it.D->id);
        gs.push_back(it.G1);
        gs.push_back(it.G2);
        hs.insert(hs.end(), it.h1, it.h1 + it.G1);
        hs.insert(hs.end(), it.h2, it.h2 + it.G2);
    }
    BatchPlan* P = static_cast<BatchPlan*>(ctx->batch_plan);
    const int stamp = tune_stamp_of(ctx);
    if (!P || P->key_ids != ids || P->key_h != hs || P->key_g != gs || P->tune_stamp != stamp) {
        delete P;
        ctx->batch_plan = nullptr;
        P = new BatchPlan();
        int rc = build_plan(ctx, items, *P);
        if (rc != CDE_OK) {
            delete P;
            return rc;
        }
        P->key_ids = ids;
        P->key_h = hs;
        P->key_g = gs;
        P->tune_stamp = stamp;
        ctx->batch_plan = P;
    }
    // order after the caller's stream, replay, wait
    cudaEvent_t ev;
    CDE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, user_st);
    cudaStreamWaitEvent(P->stream, ev, 0);
    cudaEventDestroy(ev);
    timing_reset(ctx);
    timing_begin(ctx, P->stream);
    CDE_CUDA(cudaGraphLaunch(P->exec, P->stream));
    timing_end(ctx, P->stream);
    CDE_CUDA(cudaStreamSynchronize(P->stream));
    for (size_t b = 0; b < items.size(); ++b) {
        const int n = P->gsz[b];
        if (Lc[b]) memcpy(Lc[b], P->hout + P->out_off[b], sizeof(double) * n);
        if (Le[b]) memcpy(Le[b], P->hout + P->out_off[b] + n, sizeof(double) * n);
    }
    return CDE_OK;
}

void batch_plan_free(cde_ctx* ctx) {
    delete static_cast<BatchPlan*>(ctx->batch_plan);
    ctx->batch_plan = nullptr;
}

// ---------------------------------------------------------------------------
// Autotuner: for one grid shape class, time the single-dataset launch on a
// representative dataset over every tile configuration -- units per tile and
// resident CTAs per SM -- and keep the fastest in the context.  Both launch
// paths read the kept configuration, so their results stay bitwise identical.
// ---------------------------------------------------------------------------
static int shape_class(int T) { return T <= 8 ? 0 : T <= 16 ? 1 : 2; }

int autotune_shape(cde_ctx* ctx, const Dataset& D, const double* h1, int G1, const double* h2, int G2,
                   int* best_upt, int* best_ctas, double* best_ms) {
    const int T1 = loo_pad1(G1), T2 = loo_pad2(G2);
    const int a = shape_class(T1), b = shape_class(T2);
    const int JW = 1024 / (T1 * T2);
    std::vector<int> upts;
    for (int u : {1, 2, 4, 8, 16})
        if (u * JW >= 2 && u * JW <= 64) upts.push_back(u);
    cudaStream_t st = ctx->stream;
    double* dout = nullptr;
    CDE_CUDA(cudaMalloc((void**)&dout, 2 * sizeof(double) * G1 * G2));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    int bu = 0, bc = 0;
    int rc = CDE_OK;
    struct Cand {
        int u, c;
        double ms;
    };
    std::vector<Cand> timed;
    for (int u : upts)
            for (int c : {1, 2}) {
                tuning_candidate(T1, T2, u, c);
                // one untimed launch, then the fastest of three
                float tmin = 1e30f;
                for (int rep = 0; rep < 4 && rc == CDE_OK; ++rep) {
                    cudaEventRecord(e0, st);
                    rc = loo_grid_enqueue(ctx, D, h1, G1, h2, G2, nullptr, 0, dout, dout + G1 * G2, nullptr, st);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess && rc == CDE_OK) rc = cuda_error(cudaGetLastError(), "autotune");
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) tmin = std::min(tmin, ms);
                }
                if (rc != CDE_OK) break;
                timed.push_back({u, c, tmin});
                best = std::min(best, (double)tmin);
            }
    // the configuration to keep: among those within 3% of the fastest (the timed launches
    // are a few ms, and in a batch the tile size hardly matters: the queue spans datasets),
    // the most units per tile (fewest FP64 partial slots to write and reduce), then
    // two CTAs per SM
    double kept = best;
    for (const Cand& k : timed)
        if (k.ms <= 1.03 * best && (k.u > bu || (k.u == bu && k.c > bc))) {
            bu = k.u;
            bc = k.c;
            kept = k.ms;
        }
    tuning_candidate_clear();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dout);
    if (rc != CDE_OK) return rc;
    ctx->tune_upt[a][b] = bu;
    ctx->tune_ctas[a][b] = bc;
    ctx->tuned[a][b] = true;
    if (best_upt) *best_upt = bu;
    if (best_ctas) *best_ctas = bc;
    if (best_ms) *best_ms = kept;
    return CDE_OK;
}

// Tune every shape class of the batch that has no configuration yet, each on
// its largest dataset, and store the result in the tuning cache named by
// CDE_TUNING_CACHE when there is one.
static int autotune_batch_shapes(cde_ctx* ctx, const std::vector<BatchItem>& items) {
    if (!ctx->autotune_batch) return CDE_OK;
    int pick[3][3];
    for (auto& r : pick)
        for (int& v : r) v = -1;
    for (int i = 0; i < (int)items.size(); ++i) {
        const int a = shape_class(loo_pad1(items[i].G1)), b = shape_class(loo_pad2(items[i].G2));
        if (ctx->tuned[a][b]) continue;
        if (pick[a][b] < 0 || items[i].D->N > items[pick[a][b]].D->N) pick[a][b] = i;
    }
    bool any = false;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            if (pick[a][b] < 0) continue;
            const BatchItem& it = items[pick[a][b]];
            const int rc = autotune_shape(ctx, *it.D, it.h1, it.G1, it.h2, it.G2, nullptr, nullptr, nullptr);
            if (rc != CDE_OK) return rc;
            any = true;
        }
    if (any)
        if (const char* tc = getenv("CDE_TUNING_CACHE"))
            if (cde_tuning_save(ctx, tc) != CDE_OK) set_error(CDE_OK, "");
    return CDE_OK;
}

#ifdef CDE_CHECKS
CDE_CHECK_READER(check_status_batch)
#endif

}  // namespace cde

using namespace cde;

extern "C" int cde_loo_loglik_batch(cde_ctx* ctx, int n, const cde_dataset* ds, const double* const* h1,
                                    const int* G1, const double* const* h2, const int* G2,
                                    double* const* L_cond_out, double* const* L_eq3_out, void* stream) {
    CDE_NVTX("cde_loo_loglik_batch");
    if (!ctx || n < 0 || (n > 0 && (!ds || !h1 || !G1 || !h2 || !G2)))
        return set_error(CDE_EINVAL, "cde_loo_loglik_batch: bad arguments");
    if (n == 0) return CDE_OK;
    std::vector<BatchItem> items(n);
    std::vector<std::shared_ptr<Dataset>> keep(n);
    std::vector<double*> Lc(n), Le(n);
    for (int b = 0; b < n; ++b) {
        if (G1[b] < 1 || G1[b] > 32 || G2[b] < 1 || G2[b] > 32 || !h1[b] || !h2[b])
            return set_error(CDE_EINVAL, "cde_loo_loglik_batch: each grid must have 1..32 bandwidths per axis");
        for (int k = 0; k < G1[b]; ++k)
            if (!std::isfinite(h1[b][k]) || h1[b][k] < 1e-12 || h1[b][k] > 1e12)
                return set_error(CDE_EINVAL, "cde_loo_loglik_batch: bad h1");
        for (int k = 0; k < G2[b]; ++k)
            if (!std::isfinite(h2[b][k]) || h2[b][k] < 1e-12 || h2[b][k] > 1e12)
                return set_error(CDE_EINVAL, "cde_loo_loglik_batch: bad h2");
        keep[b] = find_dataset(ctx, ds[b]);
        if (!keep[b]) return set_error(CDE_ENOTFOUND, "cde_loo_loglik_batch: unknown dataset");
        items[b] = BatchItem{keep[b].get(), h1[b], G1[b], h2[b], G2[b], nullptr, nullptr};
        Lc[b] = L_cond_out ? L_cond_out[b] : nullptr;
        Le[b] = L_eq3_out ? L_eq3_out[b] : nullptr;
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    // Datasets whose single launch runs on the d >= 16 kernel (Gram-form distances)
    // take that launch, one per dataset, so that their results stay those of
    // cde_loo_loglik; the others share the batched graph of the direct tile body.
    std::vector<BatchItem> bitems;
    std::vector<double*> bLc, bLe;
    for (int b = 0; b < n; ++b) {
        if (loo_use_gram(*items[b].D, loo_pad1(G1[b]), loo_pad2(G2[b]))) {
            const int rc = cde_loo_loglik(ctx, ds[b], h1[b], G1[b], h2[b], G2[b], Lc[b], Le[b], 0, stream);
            if (rc != CDE_OK) return rc;
        } else {
            bitems.push_back(items[b]);
            bLc.push_back(Lc[b]);
            bLe.push_back(Le[b]);
        }
    }
    if (bitems.empty()) return CDE_OK;
    const int rc = autotune_batch_shapes(ctx, bitems);
    if (rc != CDE_OK) return rc;
    return loo_batch_run(ctx, bitems, bLc, bLe, pick_stream(ctx, stream));
}

extern "C" int cde_autotune(cde_ctx* ctx, cde_dataset ds, const double* h1, int G1, const double* h2, int G2,
                            int* units_per_tile, int* ctas_per_sm, double* best_ms) {
    CDE_NVTX("cde_autotune");
    if (!ctx || !h1 || !h2 || G1 < 1 || G1 > 32 || G2 < 1 || G2 > 32)
        return set_error(CDE_EINVAL, "cde_autotune: bad arguments (grids of 1..32 per axis)");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_autotune: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    return autotune_shape(ctx, *D, h1, G1, h2, G2, units_per_tile, ctas_per_sm, best_ms);
}

extern "C" int cde_tuning_get_ex(cde_ctx* ctx, int G1, int G2, int* units_per_tile, int* ctas_per_sm, int* tuned) {
    if (!ctx || G1 < 1 || G1 > 32 || G2 < 1 || G2 > 32) return set_error(CDE_EINVAL, "cde_tuning_get: bad arguments");
    const int T1 = loo_pad1(G1), T2 = loo_pad2(G2);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (units_per_tile) *units_per_tile = loo_units_per_tile(ctx, T1, T2, 0);
    if (ctas_per_sm) *ctas_per_sm = loo_grid_ctas(ctx, T1, T2) / ctx->sm_count;
    if (tuned) *tuned = ctx->tuned[shape_class(T1)][shape_class(T2)] ? 1 : 0;
    return CDE_OK;
}

extern "C" int cde_tuning_get(cde_ctx* ctx, int G1, int G2, int* units_per_tile, int* ctas_per_sm) {
    return cde_tuning_get_ex(ctx, G1, G2, units_per_tile, ctas_per_sm, nullptr);
}

extern "C" int cde_autotune_enable(cde_ctx* ctx, int on) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_autotune_enable: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->autotune_batch = on != 0;
    return CDE_OK;
}

// Tuning cache file: a header line with the device it was tuned on, then one
// line "a b units_per_tile ctas_per_sm tuned" per shape class (a, b in 0..2
// for padded sizes 8|16|32 of G1 and G2).
static std::string tuning_device_key(cde_ctx* ctx) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, ctx->device) != cudaSuccess) return "unknown";
    char buf[400];
    snprintf(buf, sizeof(buf), "%s sm_%d%d sms=%d", p.name, p.major, p.minor, p.multiProcessorCount);
    for (char* c = buf; *c; ++c)
        if (*c == '\n') *c = ' ';
    return buf;
}

extern "C" int cde_tuning_save(cde_ctx* ctx, const char* path) {
    if (!ctx || !path) return set_error(CDE_EINVAL, "cde_tuning_save: null argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return set_error(CDE_EINVAL, std::string("cde_tuning_save: cannot write ") + path);
    fprintf(f, "cde-tuning 2 %s\n", tuning_device_key(ctx).c_str());
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            fprintf(f, "%d %d %d %d %d\n", a, b, ctx->tune_upt[a][b], ctx->tune_ctas[a][b], ctx->tuned[a][b] ? 1 : 0);
    const bool ok = fclose(f) == 0 && rename(tmp.c_str(), path) == 0;
    if (!ok) return set_error(CDE_EINVAL, std::string("cde_tuning_save: cannot write ") + path);
    return CDE_OK;
}

extern "C" int cde_tuning_load(cde_ctx* ctx, const char* path) {
    if (!ctx || !path) return set_error(CDE_EINVAL, "cde_tuning_load: null argument");
    FILE* f = fopen(path, "r");
    if (!f) return set_error(CDE_ENOTFOUND, std::string("cde_tuning_load: cannot read ") + path);
    char line[512];
    int upt[3][3], ctas[3][3], tuned[3][3], seen = 0;
    bool ok = fgets(line, sizeof(line), f) != nullptr;
    if (ok) {
        std::string h(line);
        while (!h.empty() && (h.back() == '\n' || h.back() == '\r')) h.pop_back();
        ok = h == "cde-tuning 2 " + tuning_device_key(ctx);
        if (!ok) {
            fclose(f);
            return set_error(CDE_EINVAL, "cde_tuning_load: file was tuned on another device or version");
        }
    }
    int a, b, u, c, t;
    while (ok && fgets(line, sizeof(line), f)) {
        if (sscanf(line, "%d %d %d %d %d", &a, &b, &u, &c, &t) != 5 || a < 0 || a > 2 || b < 0 || b > 2 || u < 0 ||
            u > 64 || c < 0 || c > 2 || t < 0 || t > 1 || (seen & (1 << (3 * a + b)))) {
            ok = false;
            break;
        }
        upt[a][b] = u;
        ctas[a][b] = c;
        tuned[a][b] = t;
        seen |= 1 << (3 * a + b);
    }
    fclose(f);
    if (!ok || seen != 0x1ff) return set_error(CDE_EINVAL, "cde_tuning_load: malformed file");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) {
            ctx->tune_upt[a][b] = upt[a][b];
            ctx->tune_ctas[a][b] = ctas[a][b];
            ctx->tuned[a][b] = tuned[a][b] != 0;
        }
    return CDE_OK;
}

extern "C" int cde_tuning_set(cde_ctx* ctx, int G1, int G2, int units_per_tile, int ctas_per_sm) {
    if (!ctx || G1 < 1 || G1 > 32 || G2 < 1 || G2 > 32 || units_per_tile < 0 || units_per_tile > 64 ||
        ctas_per_sm < 0 || ctas_per_sm > 2)
        return set_error(CDE_EINVAL, "cde_tuning_set: bad arguments");
    // the classes the kernels read: G1 padded to 16 | 32, G2 to 8 | 16 | 32
    const int a = shape_class(loo_pad1(G1)), b = shape_class(loo_pad2(G2));
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->tune_upt[a][b] = units_per_tile;
    ctx->tune_ctas[a][b] = ctas_per_sm;
    // an explicit configuration counts as tuned; both defaults make the class untuned again
    ctx->tuned[a][b] = units_per_tile || ctas_per_sm;
    return CDE_OK;
}
