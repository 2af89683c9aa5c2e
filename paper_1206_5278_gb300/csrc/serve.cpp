// Request loop with continuous batching over resident datasets.
//
// Clients submit density jobs (Eq. 1 at Q query points x a y grid) and
// bandwidth-selection jobs (LOO grid search, then Adam ascent on
// (ln h1, ln h2) driven by the adjoint kernel).  One scheduler thread admits
// queued jobs while a stream slot and the job-memory budget allow (a job that
// does not fit waits; smaller later jobs may pass it; selection jobs take at
// most half of the slots and never the last free one, run their grid and
// their gradient steps as ~10 ms launches, and run on low-priority streams, so
// density queries are not held up by long selections), enqueues their kernels
// on the slot's stream so admitted jobs overlap on the device, and polls
// completion events.  A selection job is a small state machine: every part
// of its grid and of each gradient step is one enqueue (each writes fixed
// partial slots, so the result is bitwise that of one launch); the host update between
// steps happens when its event completes, so the device keeps running other
// jobs meanwhile.  Every kernel is deterministic and partitions work by the
// job's own sizes only, so a job's result is the same alone and in the mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "cde_internal.h"

namespace cde {

using Clock = std::chrono::steady_clock;

// pair evaluations (N^2 G1 G2 units) per launch of a selection job's grid: about
// 10 ms of the grid kernel, the longest a density job waits behind it
constexpr double kSelChunk = 2.5e11;
// pairs per launch of a gradient step (about 10 ms of the gradient kernel at d = 8)
constexpr double kGradChunk = 1.2e10;

struct Job {
    int64_t ticket = 0;
    cde_request req{};
    std::shared_ptr<Dataset> D;
    Clock::time_point t_submit, t_done;
    size_t mem = 0;
    int status = CDE_OK;
    bool done = false;
    // running state
    int slot = -1;
    int phase = 0;          // selection: 0 grid, 1.. gradient steps
    // selection grid in tile ranges (one launch per scheduling step)
    LooChunked* gc = nullptr;
    void* d_grid = nullptr; // the grid's partials and counters
    bool grid_init = false;
    bool grid_final = false;  // the final reduction has been enqueued
    // the running gradient step in ranges of row blocks (one launch per scheduling step)
    GradChunked* gr = nullptr;
    bool step_final = false;  // the step's per-row merge and sums have been enqueued
    cudaEvent_t ev = nullptr;
    // device / pinned buffers
    float* d_xq = nullptr;
    float* d_yg = nullptr;
    float* d_f = nullptr;
    double* d_small = nullptr;     // selection: grid L (G1 G2) + 3 doubles
    float* h_f = nullptr;          // pinned density output
    float* h_in = nullptr;         // pinned density inputs
    double* h_small = nullptr;     // pinned selection values
    // selection state (Adam on ln h)
    double th[2] = {0, 0}, m[2] = {0, 0}, v[2] = {0, 0};
    double best[3] = {0, 0, -INFINITY}, grid_best[3] = {0, 0, -INFINITY};
    int step = 0;
};

struct Server {
    cde_ctx* ctx = nullptr;
    cde_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<int64_t, std::shared_ptr<Job>> jobs;   // all not-yet-forgotten tickets
    std::vector<std::shared_ptr<Job>> running;
    std::vector<cudaStream_t> streams;      // per slot: selection jobs (lowest priority)
    std::vector<cudaStream_t> streams_hi;   // per slot: density jobs (highest priority)
    std::vector<int> slot_busy;
    std::vector<char*> pin;          // per-slot pinned staging (grows, reused)
    std::vector<size_t> pin_cap;
    std::vector<char*> pin_retired;  // outgrown staging, freed at stop (cudaFreeHost waits for the device)
    size_t mem_used = 0, mem_budget = 0;
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    // stats
    std::vector<double> lat_all, lat_den, lat_sel;
    int64_t completed = 0, cancelled = 0, failed = 0, peak = 0, peak_sel = 0;
    double busy_s = 0;
    Clock::time_point busy_since;
};

static double pct(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p / 100.0 * (v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - lo);
}

static size_t job_mem(const Job& J, int sm_count) {
    const cde_request& r = J.req;
    if (r.kind == CDE_REQ_DENSITY) {
        const int64_t qt = (r.Q + 31) / 32;
        const int64_t ns = std::max<int64_t>(1, (4LL * sm_count + qt - 1) / std::max<int64_t>(qt, 1));
        return (size_t)r.Q * J.D->d * 8 + (size_t)r.G_y * 4 + (size_t)r.Q * r.G_y * 4 * (2 + ns) +
               (size_t)r.Q * 16 + 4096;
    }
    const size_t tiles = (size_t)(J.D->N / 8 + 2);
    return tiles * 2 * 1024 * 8 + (size_t)J.D->N * (6 * 4 * 16 + 24) + 65536;
}

// A job's stream: density jobs run on their slot's high-priority stream, so the
// device dispatches their blocks ahead of the waiting blocks of selection kernels.
static cudaStream_t job_stream(const Server& S, const Job& J) {
    if (J.slot < 0) return nullptr;
    return J.req.kind == CDE_REQ_DENSITY ? S.streams_hi[J.slot] : S.streams[J.slot];
}

static void release(Server& S, Job& J) {
    if (J.ev) cudaEventDestroy(J.ev);
    J.ev = nullptr;
    cudaStream_t st = job_stream(S, J);
    if (J.d_xq) cudaFreeAsync(J.d_xq, st);
    if (J.d_f) cudaFreeAsync(J.d_f, st);
    if (J.d_small) cudaFreeAsync(J.d_small, st);
    if (J.d_grid) cudaFreeAsync(J.d_grid, st);
    J.d_grid = nullptr;
    if (J.gc) loo_chunked_destroy(J.gc);
    J.gc = nullptr;
    if (J.gr) grad_chunked_free(J.gr, st);
    J.gr = nullptr;
    J.d_xq = J.d_yg = J.d_f = nullptr;
    J.d_small = nullptr;
    J.h_f = J.h_in = nullptr;
    J.h_small = nullptr;
}

static int slot_pinned(Server& S, int slot, size_t bytes, char** out) {
    if (S.pin_cap[slot] < bytes) {
        // the outgrown buffer is only retired here: freeing pinned memory waits for
        // the whole device, which would stall every job behind a long selection kernel
        if (S.pin[slot]) S.pin_retired.push_back(S.pin[slot]);
        S.pin[slot] = nullptr;
        S.pin_cap[slot] = 0;
        const size_t cap = std::max<size_t>(bytes + bytes / 2, 1 << 20);
        CDE_CUDA(cudaMallocHost((void**)&S.pin[slot], cap));
        S.pin_cap[slot] = cap;
    }
    *out = S.pin[slot];
    return CDE_OK;
}

// Enqueue the next piece of work of a running job on its stream and record its event.
static int advance(Server& S, Job& J) {
    cudaStream_t st = job_stream(S, J);
    const cde_request& r = J.req;
    const Dataset& D = *J.D;
    if (r.kind == CDE_REQ_DENSITY) {
        const size_t nq = (size_t)r.Q * D.d, nf = (size_t)r.Q * r.G_y;
        char* pb = nullptr;
        int prc = slot_pinned(S, J.slot, (nq + r.G_y + nf) * sizeof(float), &pb);
        if (prc != CDE_OK) return prc;
        J.h_in = reinterpret_cast<float*>(pb);
        J.h_f = J.h_in + nq + r.G_y;
        memcpy(J.h_in, r.xq, nq * sizeof(float));
        memcpy(J.h_in + nq, r.ygrid, r.G_y * sizeof(float));
        CDE_CUDA(cudaMallocAsync((void**)&J.d_xq, (nq + r.G_y) * sizeof(float), st));
        J.d_yg = J.d_xq + nq;
        CDE_CUDA(cudaMallocAsync((void**)&J.d_f, std::max<size_t>(nf, 1) * sizeof(float), st));
        CDE_CUDA(cudaMemcpyAsync(J.d_xq, J.h_in, (nq + r.G_y) * sizeof(float), cudaMemcpyHostToDevice, st));
        int rc = density_enqueue(S.ctx, D, r.h1, r.h2, J.d_xq, r.Q, J.d_yg, r.G_y, J.d_f, st);
        if (rc != CDE_OK) return rc;
        CDE_CUDA(cudaMemcpyAsync(J.h_f, J.d_f, nf * sizeof(float), cudaMemcpyDeviceToHost, st));
    } else if (J.phase == 0) {
        const size_t g = (size_t)r.G1 * r.G2;
        if (!J.grid_init) {
            char* pb = nullptr;
            int prc = slot_pinned(S, J.slot, (g + 4) * sizeof(double), &pb);
            if (prc != CDE_OK) return prc;
            J.h_small = reinterpret_cast<double*>(pb);
            CDE_CUDA(cudaMallocAsync((void**)&J.d_small, (g + 4) * sizeof(double), st));
            J.grid_init = true;
            if (r.G1 <= 32 && r.G2 <= 32) {
                int rc = loo_chunked_create(S.ctx, D, r.h1_grid, r.G1, r.h2_grid, r.G2, &J.gc);
                if (rc != CDE_OK) return rc;
                CDE_CUDA(cudaMallocAsync(&J.d_grid, loo_chunked_scratch_bytes(J.gc), st));
            } else {
                // wider grids: one enqueue of all its blocks
                int rc = loo_grid_enqueue(S.ctx, D, r.h1_grid, r.G1, r.h2_grid, r.G2, nullptr, 0, J.d_small,
                                          nullptr, nullptr, st);
                if (rc != CDE_OK) return rc;
                J.grid_final = true;
            }
        }
        if (!J.grid_final) {
            // the next part: about kSelChunk pair evaluations, so that density jobs
            // queued meanwhile run between two launches of a long grid
            int done = 0;
            int rc = loo_chunked_next(J.gc, J.d_grid, kSelChunk, st, &done);
            if (rc != CDE_OK) return rc;
            if (done) {
                rc = loo_chunked_final(J.gc, J.d_grid, J.d_small, nullptr, st);
                if (rc != CDE_OK) return rc;
                J.grid_final = true;
            }
        }
        if (J.grid_final)
            CDE_CUDA(cudaMemcpyAsync(J.h_small, J.d_small, g * sizeof(double), cudaMemcpyDeviceToHost, st));
    } else {
        // a gradient step in ranges of row blocks of about kGradChunk pairs each
        const size_t g = (size_t)r.G1 * r.G2;
        if (!J.gr) {
            int rc = grad_chunked_create(S.ctx, D, std::exp(J.th[0]), std::exp(J.th[1]), st, nullptr, &J.gr);
            if (rc != CDE_OK) return rc;
            J.step_final = false;
        }
        int done = 0;
        int rc = grad_chunked_next(J.gr, kGradChunk, st, &done);
        if (rc != CDE_OK) return rc;
        if (done) {
            GradChunked* c = J.gr;
            J.gr = nullptr;
            rc = grad_chunked_finish(S.ctx, c, J.d_small + g, st);
            if (rc != CDE_OK) return rc;
            J.step_final = true;
            CDE_CUDA(cudaMemcpyAsync(J.h_small + g, J.d_small + g, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
    }
    CDE_CUDA(cudaEventCreateWithFlags(&J.ev, cudaEventDisableTiming));
    CDE_CUDA(cudaEventRecord(J.ev, st));
    return CDE_OK;
}

// Called when the job's event completed.  Returns true when the job is finished.
static bool on_event(Server& S, Job& J) {
    const cde_request& r = J.req;
    cudaEventDestroy(J.ev);
    J.ev = nullptr;
    if (r.kind == CDE_REQ_DENSITY) {
        memcpy(r.f_out, J.h_f, (size_t)r.Q * r.G_y * sizeof(float));
        return true;
    }
    const size_t g = (size_t)r.G1 * r.G2;
    const double N = (double)J.D->N;
    if (J.phase == 0 && !J.grid_final) return false;   // more ranges of the grid to launch
    if (J.phase > 0 && !J.step_final) return false;    // more row blocks of the gradient step
    if (J.phase == 0) {
        int bk = 0;
        for (size_t c = 1; c < g; ++c)
            if (J.h_small[c] > J.h_small[bk]) bk = (int)c;
        if (r.L_grid_out) memcpy(r.L_grid_out, J.h_small, g * sizeof(double));
        J.grid_best[0] = r.h1_grid[bk / r.G2];
        J.grid_best[1] = r.h2_grid[bk % r.G2];
        J.grid_best[2] = J.h_small[bk];
        for (int q = 0; q < 3; ++q) J.best[q] = J.grid_best[q];
        J.th[0] = std::log(J.grid_best[0]);
        J.th[1] = std::log(J.grid_best[1]);
    } else {
        const double* o = J.h_small + g;  // L, dL/dln h1, dL/dln h2 at th
        if (o[0] > J.best[2]) {
            J.best[0] = std::exp(J.th[0]);
            J.best[1] = std::exp(J.th[1]);
            J.best[2] = o[0];
        }
        // Adam ascent on L/N in log-bandwidth space
        const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
        ++J.step;
        for (int q = 0; q < 2; ++q) {
            const double gq = o[1 + q] / N;
            J.m[q] = b1 * J.m[q] + (1 - b1) * gq;
            J.v[q] = b2 * J.v[q] + (1 - b2) * gq * gq;
            const double mh = J.m[q] / (1 - std::pow(b1, J.step)), vh = J.v[q] / (1 - std::pow(b2, J.step));
            J.th[q] += r.lr * mh / (std::sqrt(vh) + eps);
            J.th[q] = std::min(std::max(J.th[q], std::log(1e-6)), std::log(1e6));
        }
    }
    ++J.phase;
    if (J.phase > r.n_steps) {
        r.sel_out[0] = J.best[0];
        r.sel_out[1] = J.best[1];
        r.sel_out[2] = J.best[2];
        r.sel_out[3] = J.grid_best[2];
        return true;
    }
    return false;
}

static void finish(Server& S, const std::shared_ptr<Job>& J, int status) {
    // S.mu held
    J->status = status;
    J->done = true;
    J->t_done = Clock::now();
    const double ms = std::chrono::duration<double, std::milli>(J->t_done - J->t_submit).count();
    if (status == CDE_OK) {
        ++S.completed;
        S.lat_all.push_back(ms);
        (J->req.kind == CDE_REQ_DENSITY ? S.lat_den : S.lat_sel).push_back(ms);
    } else if (status == CDE_ECANCELED) {
        ++S.cancelled;
    } else {
        ++S.failed;
    }
    J->D->users--;
    J->D.reset();
    S.cv_done.notify_all();
}

static void loop(Server* Sp) {
    t_untimed = true;   // jobs are not timed by cde_timing_enable
    Server& S = *Sp;
    cudaSetDevice(S.ctx->device);
    std::unique_lock<std::mutex> lk(S.mu);
    while (true) {
        // 1) completions
        for (size_t k = 0; k < S.running.size();) {
            auto J = S.running[k];
            const cudaError_t q = cudaEventQuery(J->ev);
            if (q == cudaErrorNotReady) {
                ++k;
                continue;
            }
            int status = CDE_OK;
            bool fin = true;
            if (q != cudaSuccess) {
                status = cuda_error(q, "serve: job");
            } else {
                fin = on_event(S, *J);
                if (!fin) {
                    const int rc = advance(S, *J);
                    if (rc != CDE_OK) {
                        status = rc;
                        fin = true;
                    }
                }
            }
            if (fin) {
                release(S, *J);
                S.slot_busy[J->slot] = 0;
                S.mem_used -= J->mem;
                finish(S, J, status);
                S.running.erase(S.running.begin() + k);
                if (S.running.empty())
                    S.busy_s += std::chrono::duration<double>(Clock::now() - S.busy_since).count();
            } else {
                ++k;
            }
        }
        // 2) admissions (by free slot and job memory).  Selection jobs take at most
        //    half of the slots (at least one): they are GPU-bound for seconds and gain
        //    little from running side by side, while density jobs arriving meanwhile
        //    then find a slot, and several of them can run at once
        const int sel_cap = std::max<int>(1, (int)S.slot_busy.size() / 2);
        for (auto it = S.queue.begin(); it != S.queue.end();) {
            int slot = -1, n_free = 0;
            for (size_t s = 0; s < S.slot_busy.size(); ++s)
                if (!S.slot_busy[s]) {
                    if (slot < 0) slot = (int)s;
                    ++n_free;
                }
            if (slot < 0) break;
            auto J = *it;
            if (J->req.kind != CDE_REQ_DENSITY) {
                int n_sel = 0;
                for (const auto& R : S.running) n_sel += R->req.kind != CDE_REQ_DENSITY;
                if (n_sel >= sel_cap || (n_free == 1 && S.slot_busy.size() > 1)) {
                    ++it;  // a density job behind it may take the slot
                    continue;
                }
            }
            if (S.mem_used + J->mem > S.mem_budget && !S.running.empty()) {
                ++it;  // does not fit now; a smaller job behind it may
                continue;
            }
            it = S.queue.erase(it);
            J->slot = slot;
            S.slot_busy[slot] = 1;
            S.mem_used += J->mem;
            if (S.running.empty()) S.busy_since = Clock::now();
            const int rc = advance(S, *J);
            if (rc != CDE_OK) {
                release(S, *J);
                S.slot_busy[slot] = 0;
                S.mem_used -= J->mem;
                finish(S, J, rc);
                if (S.running.empty())
                    S.busy_s += std::chrono::duration<double>(Clock::now() - S.busy_since).count();
                continue;
            }
            S.running.push_back(J);
            S.peak = std::max<int64_t>(S.peak, (int64_t)S.running.size());
            int64_t n_sel = 0;
            for (const auto& R : S.running) n_sel += R->req.kind != CDE_REQ_DENSITY;
            S.peak_sel = std::max(S.peak_sel, n_sel);
        }
        if (S.stop && S.running.empty()) break;
        // 3) wait: briefly when jobs run (poll their events), else for work
        if (S.running.empty())
            S.cv_work.wait_for(lk, std::chrono::milliseconds(50));
        else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace cde

using namespace cde;

extern "C" {

int cde_server_start(cde_ctx* ctx, const cde_server_config* cfg) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_server_start: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (ctx->server) return set_error(CDE_EBUSY, "cde_server_start: already running");
    auto* S = new Server();
    S->ctx = ctx;
    S->cfg.n_streams = cfg && cfg->n_streams > 0 ? cfg->n_streams : 4;
    S->cfg.queue_capacity = cfg && cfg->queue_capacity > 0 ? cfg->queue_capacity : 1024;
    S->cfg.job_mem_budget = cfg ? cfg->job_mem_budget : 0;
    if (S->cfg.n_streams > 64) S->cfg.n_streams = 64;
    const size_t avail = ctx->budget > ctx->used.load() ? ctx->budget - ctx->used.load() : 0;
    S->mem_budget = S->cfg.job_mem_budget ? S->cfg.job_mem_budget : avail;
    cudaError_t e = cudaSetDevice(ctx->device);
    int prio_lo = 0, prio_hi = 0;   // numerically: least and greatest priority
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (int s = 0; s < S->cfg.n_streams && e == cudaSuccess; ++s) {
        cudaStream_t st = nullptr, sh = nullptr;
        e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_lo);
        if (e == cudaSuccess) S->streams.push_back(st);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sh, cudaStreamNonBlocking, prio_hi);
        if (e == cudaSuccess) S->streams_hi.push_back(sh);
    }
    if (e != cudaSuccess) {
        for (auto st : S->streams) cudaStreamDestroy(st);
        for (auto st : S->streams_hi) cudaStreamDestroy(st);
        delete S;
        return cuda_error(e, "cde_server_start");
    }
    S->slot_busy.assign(S->streams.size(), 0);
    S->pin.assign(S->streams.size(), nullptr);
    S->pin_cap.assign(S->streams.size(), 0);
    S->th = std::thread(loop, S);
    ctx->server = S;
    return CDE_OK;
}

void cde_server_stop_internal(cde_ctx* ctx) {
    Server* S = ctx ? ctx->server : nullptr;
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        for (auto& J : S->queue) finish(*S, J, CDE_ECANCELED);
        S->queue.clear();
        S->cv_work.notify_all();
    }
    S->th.join();
    for (auto st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto st : S->streams_hi) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto p : S->pin)
        if (p) cudaFreeHost(p);
    for (auto p : S->pin_retired) cudaFreeHost(p);
    ctx->server = nullptr;
    delete S;
}

int cde_server_stop(cde_ctx* ctx) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_server_stop: null context");
    if (!ctx->server) return set_error(CDE_EINVAL, "cde_server_stop: not running");
    cde_server_stop_internal(ctx);
    return CDE_OK;
}

int cde_submit(cde_ctx* ctx, const cde_request* req, int64_t* ticket) {
    if (!ctx || !req || !ticket) return set_error(CDE_EINVAL, "cde_submit: null argument");
    Server* S = ctx->server;
    if (!S) return set_error(CDE_EINVAL, "cde_submit: server not running");
    auto J = std::make_shared<Job>();
    J->req = *req;
    const cde_request& r = J->req;
    J->D = find_dataset(ctx, r.ds);
    if (!J->D) return set_error(CDE_ENOTFOUND, "cde_submit: unknown dataset");
    auto bw = [](double h) { return std::isfinite(h) && h >= 1e-12 && h <= 1e12; };
    if (r.kind == CDE_REQ_DENSITY) {
        if (r.Q < 1 || r.G_y < 1 || !r.xq || !r.ygrid || !r.f_out || !bw(r.h1) || !bw(r.h2) ||
            r.Q * (int64_t)r.G_y > ((int64_t)1 << 32))
            return set_error(CDE_EINVAL, "cde_submit: bad density request");
    } else if (r.kind == CDE_REQ_SELECT) {
        if (!r.h1_grid || !r.h2_grid || r.G1 < 1 || r.G2 < 1 || r.G1 * (int64_t)r.G2 > 4096 || r.n_steps < 0 ||
            r.n_steps > 10000 || !r.sel_out || !(r.lr > 0) || !std::isfinite(r.lr))
            return set_error(CDE_EINVAL, "cde_submit: bad selection request");
        for (int k = 0; k < r.G1; ++k)
            if (!bw(r.h1_grid[k])) return set_error(CDE_EINVAL, "cde_submit: bad h1 grid");
        for (int k = 0; k < r.G2; ++k)
            if (!bw(r.h2_grid[k])) return set_error(CDE_EINVAL, "cde_submit: bad h2 grid");
    } else {
        return set_error(CDE_EINVAL, "cde_submit: unknown request kind");
    }
    J->mem = job_mem(*J, ctx->sm_count);
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) return set_error(CDE_EINVAL, "cde_submit: server stopping");
    if ((int)S->queue.size() >= S->cfg.queue_capacity) return set_error(CDE_EBUSY, "cde_submit: queue full");
    if (J->mem > S->mem_budget) return set_error(CDE_ENOMEM, "cde_submit: job larger than the memory budget");
    J->ticket = S->next_ticket++;
    J->t_submit = Clock::now();
    J->D->users++;
    S->queue.push_back(J);
    S->jobs[J->ticket] = J;
    *ticket = J->ticket;
    S->cv_work.notify_all();
    return CDE_OK;
}

int cde_poll(cde_ctx* ctx, int64_t ticket, int* done, int* status) {
    if (!ctx || !done) return set_error(CDE_EINVAL, "cde_poll: null argument");
    Server* S = ctx->server;
    if (!S) return set_error(CDE_EINVAL, "cde_poll: server not running");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return set_error(CDE_ENOTFOUND, "cde_poll: unknown ticket");
    *done = it->second->done ? 1 : 0;
    if (status) *status = it->second->done ? it->second->status : CDE_OK;
    return CDE_OK;
}

int cde_wait(cde_ctx* ctx, int64_t ticket, int64_t timeout_us) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_wait: null context");
    Server* S = ctx->server;
    if (!S) return set_error(CDE_EINVAL, "cde_wait: server not running");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return set_error(CDE_ENOTFOUND, "cde_wait: unknown ticket");
    auto J = it->second;
    if (timeout_us < 0) {
        S->cv_done.wait(lk, [&] { return J->done; });
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return J->done; })) {
        return set_error(CDE_ETIMEOUT, "cde_wait: not finished");
    }
    if (J->status != CDE_OK) return set_error(J->status, "cde_wait: job failed or was cancelled");
    return CDE_OK;
}

int cde_cancel(cde_ctx* ctx, int64_t ticket) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_cancel: null context");
    Server* S = ctx->server;
    if (!S) return set_error(CDE_EINVAL, "cde_cancel: server not running");
    std::lock_guard<std::mutex> g(S->mu);
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
        if ((*it)->ticket == ticket) {
            auto J = *it;
            S->queue.erase(it);
            finish(*S, J, CDE_ECANCELED);
            return CDE_OK;
        }
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return set_error(CDE_ENOTFOUND, "cde_cancel: unknown ticket");
    return set_error(CDE_EBUSY, it->second->done ? "cde_cancel: already finished" : "cde_cancel: running");
}

int cde_server_stats_get(cde_ctx* ctx, cde_server_stats* out) {
    if (!ctx || !out) return set_error(CDE_EINVAL, "cde_server_stats_get: null argument");
    Server* S = ctx->server;
    if (!S) return set_error(CDE_EINVAL, "cde_server_stats_get: server not running");
    std::lock_guard<std::mutex> g(S->mu);
    out->completed = S->completed;
    out->cancelled = S->cancelled;
    out->failed = S->failed;
    out->p50_ms = pct(S->lat_all, 50);
    out->p99_ms = pct(S->lat_all, 99);
    double m = 0;
    for (double v : S->lat_all) m += v;
    out->mean_ms = S->lat_all.empty() ? 0 : m / S->lat_all.size();
    out->p50_density_ms = pct(S->lat_den, 50);
    out->p99_density_ms = pct(S->lat_den, 99);
    out->p50_select_ms = pct(S->lat_sel, 50);
    out->p99_select_ms = pct(S->lat_sel, 99);
    double busy = S->busy_s;
    if (!S->running.empty()) busy += std::chrono::duration<double>(Clock::now() - S->busy_since).count();
    out->busy_s = busy;
    out->peak_concurrent = S->peak;
    out->peak_selection = S->peak_sel;
    return CDE_OK;
}

int cde_server_stats_reset(cde_ctx* ctx) {
    if (!ctx) return set_error(CDE_EINVAL, "cde_server_stats_reset: null context");
    Server* S = ctx->server;
    if (!S) return set_error(CDE_EINVAL, "cde_server_stats_reset: server not running");
    std::lock_guard<std::mutex> g(S->mu);
    S->lat_all.clear();
    S->lat_den.clear();
    S->lat_sel.clear();
    S->completed = S->cancelled = S->failed = S->peak = S->peak_sel = 0;
    S->busy_s = 0;
    if (!S->running.empty()) S->busy_since = Clock::now();
    // forget finished tickets
    for (auto it = S->jobs.begin(); it != S->jobs.end();) {
        if (it->second->done) it = S->jobs.erase(it);
        else ++it;
    }
    return CDE_OK;
}

}  // extern "C"
