// Products of the conditional density estimate at query points, as the
// paper's evaluation uses them (Sec. 4, Sec. 4.2):
//
//   E[y | x_q]      = sum_i u_qi y_i / sum_i u_qi   (the y kernel is symmetric)
//   fhat(y_q | x_q) = sum_i u_qi K_h2(y_q - y_i) / sum_i u_qi   (Eq. 1 at one point)
//   prediction interval: the narrowest window holding a fraction 1 - alpha of
//   S draws from fhat(. | x_q) (Sec. 4).
//
// u_qi are the x weights of Eq. 1 (Gaussian: 2^{a1 (m_q - |x_q - x_i|^2)} with
// the query's nearest squared distance m_q; Epanechnikov: (1 - |x_q - x_i|^2/h1^2)_+).
//
// k_cond_stats: the three sums per query, queries in registers (four per
// thread up to d = 8, two up to 16, else one), data points staged through
// shared memory point-major, the data range split
// over gridDim.y; split partials are summed in FP64 in split order.
//
// k_cond_sample: one CTA per query.  A draw from fhat(.|x_q) is a mixture
// draw: an index i with probability u_qi / sum u (inverse CDF over the
// cumulative weights), then y_i + h2 e with e from the y kernel (inverse CDF:
// Phi^{-1} for the Gaussian, 2 sin(asin(2V - 1)/3) for the Epanechnikov kernel,
// whose CDF is (2 + 3t - t^3)/4).  The cumulative weights come from a block
// scan over chunks of 256 points in a fixed order, computed twice (total, then
// the search) with identical results; the S index targets are sorted so the
// second pass resolves them chunk by chunk.  The S values are then sorted and
// the narrowest window of ceil((1 - alpha) S) consecutive values is taken.
// Random numbers: value k of the SplitMix64 stream of the seed, k = 2 (q S + s)
// for the index draw of sample s of query q and k + 1 for its kernel offset;
// 24 random bits give u = (bits + 1/2) 2^-24 in (0, 1).
#include <cmath>

#include "cde_internal.h"

namespace cde {

__global__ void k_query_pack(const float* __restrict__ xq, int64_t Q, int64_t Qp, int d,
                             const double* __restrict__ mean, const double* __restrict__ sd,
                             float* __restrict__ out);

__device__ __forceinline__ float ex2p(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float fma_sat_p(float a, float b, float c) {
    float r;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// x weight from the squared distance (Gaussian: shifted by the query's m_q)
template <int KERN>
__device__ __forceinline__ float xweight(float dx2, float a1, float mq) {
    if constexpr (KERN == 0) return ex2p(a1 * (mq - dx2));
    else return fma_sat_p(-a1, dx2, 1.f);
}

// y kernel profile at squared distance t2 (constant applied in the epilogue)
template <int KERN>
__device__ __forceinline__ float yprofile(float t2, float a2) {
    if constexpr (KERN == 0) return ex2p(-a2 * t2);
    else return fma_sat_p(-a2, t2, 1.f);
}

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t k) {
    return ((float)(splitmix64_dev(seed, k) >> 40) + 0.5f) * 0x1p-24f;
}

// --------------------------------------------------------------------------
// Per-query sums
// --------------------------------------------------------------------------
constexpr int kCSThreads = 128;

struct StatArgs {
    const float* xs;   // [d][Np]
    const float* y;    // [Np]
    const float* xq;   // [d][Qp] standardised like the data
    const float* yq;   // [Q] or null
    const float* mq;   // [Q] (Gaussian)
    int64_t N, Np, Q, Qp;
    int d;
    float a1, a2;
    int64_t i_per_split;
    float* part;       // [splits][Q][3]: sum u, sum u y, sum u w
};

template <int KERN, int DREG, int kCSJB>
__global__ void __launch_bounds__(kCSThreads) k_cond_stats(const StatArgs a) {
    __shared__ __align__(16) float xt[kCSThreads][DREG];  // point-major: 128-bit broadcast loads
    __shared__ float yt[kCSThreads];
    const int tid = threadIdx.x;
    const int64_t qbase = (int64_t)blockIdx.x * kCSThreads * kCSJB + tid;
    const int64_t i0 = (int64_t)blockIdx.y * a.i_per_split;
    const int64_t i1 = min(a.N, i0 + a.i_per_split);
    const int d = a.d;
    const bool has_yq = a.yq != nullptr;
    float xq[kCSJB][DREG], yq[kCSJB], mq[kCSJB], amq[kCSJB], S0[kCSJB], S1[kCSJB], S2[kCSJB];
#pragma unroll
    for (int b = 0; b < kCSJB; ++b) {
        const int64_t q = qbase + (int64_t)b * kCSThreads;
        const int64_t qc = q < a.Q ? q : 0;
#pragma unroll
        for (int c = 0; c < DREG; ++c) xq[b][c] = c < d ? a.xq[(int64_t)c * a.Qp + qc] : 0.f;
        yq[b] = has_yq ? a.yq[qc] : 0.f;
        mq[b] = KERN == 0 ? a.mq[qc] : 0.f;
        amq[b] = a.a1 * mq[b];
        S0[b] = S1[b] = S2[b] = 0.f;
    }
    for (int64_t t0 = i0; t0 < i1; t0 += kCSThreads) {
        __syncthreads();
        const int64_t it = CDE_CK(t0 + tid, a.Np, 301);  // < Np: splits and Np are multiples of 128
#pragma unroll
        for (int c = 0; c < DREG; ++c) xt[tid][c] = c < d ? a.xs[(int64_t)c * a.Np + it] : 0.f;
        yt[tid] = a.y[it];
        __syncthreads();
        const int n = (int)min((int64_t)kCSThreads, i1 - t0);
        for (int t = 0; t < n; ++t) {
            const float yi = yt[t];
            float xi[DREG];
#pragma unroll
            for (int c = 0; c < DREG; c += 4) {
                const float4 v4 = *reinterpret_cast<const float4*>(&xt[t][c]);
                xi[c] = v4.x;
                xi[c + 1] = v4.y;
                xi[c + 2] = v4.z;
                xi[c + 3] = v4.w;
            }
            if constexpr (kCSJB % 2 == 0) {
                // two queries per packed FP32x2 instruction (xq - x_i as fma(x_i, -1, xq),
                // the scalar subtraction's rounding; the x argument a1 m_q - a1 dx2 as one FMA)
                const float2 m1 = make_float2(-1.f, -1.f), yi2 = make_float2(yi, yi);
#pragma unroll
                for (int b = 0; b < kCSJB; b += 2) {
                    float2 dx2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < DREG; ++c) {
                        const float2 v = __ffma2_rn(make_float2(xi[c], xi[c]), m1, make_float2(xq[b][c], xq[b + 1][c]));
                        dx2 = __ffma2_rn(v, v, dx2);
                    }
                    float2 u;
                    if constexpr (KERN == 0) {
                        const float2 arg = __ffma2_rn(dx2, make_float2(-a.a1, -a.a1), make_float2(amq[b], amq[b + 1]));
                        u = make_float2(ex2p(arg.x), ex2p(arg.y));
                    } else {
                        u = make_float2(fma_sat_p(-a.a1, dx2.x, 1.f), fma_sat_p(-a.a1, dx2.y, 1.f));
                    }
                    const float2 s0 = __fadd2_rn(make_float2(S0[b], S0[b + 1]), u);
                    const float2 s1 = __ffma2_rn(u, yi2, make_float2(S1[b], S1[b + 1]));
                    S0[b] = s0.x;
                    S0[b + 1] = s0.y;
                    S1[b] = s1.x;
                    S1[b + 1] = s1.y;
                    if (has_yq) {
                        const float2 dy = __ffma2_rn(yi2, m1, make_float2(yq[b], yq[b + 1]));
                        const float2 t2 = __fmul2_rn(dy, dy);
                        float2 w;
                        if constexpr (KERN == 0) {
                            const float2 arg = __fmul2_rn(make_float2(-a.a2, -a.a2), t2);
                            w = make_float2(ex2p(arg.x), ex2p(arg.y));
                        } else {
                            w = make_float2(fma_sat_p(-a.a2, t2.x, 1.f), fma_sat_p(-a.a2, t2.y, 1.f));
                        }
                        const float2 s2 = __ffma2_rn(u, w, make_float2(S2[b], S2[b + 1]));
                        S2[b] = s2.x;
                        S2[b + 1] = s2.y;
                    }
                }
            } else {
#pragma unroll
                for (int b = 0; b < kCSJB; ++b) {
                    float dx2 = 0.f;
#pragma unroll
                    for (int c = 0; c < DREG; ++c) {
                        const float v = xq[b][c] - xi[c];
                        dx2 = fmaf(v, v, dx2);
                    }
                    const float u = xweight<KERN>(dx2, a.a1, mq[b]);
                    S0[b] += u;
                    S1[b] = fmaf(u, yi, S1[b]);
                    if (has_yq) {
                        const float dy = yq[b] - yi;
                        S2[b] = fmaf(u, yprofile<KERN>(dy * dy, a.a2), S2[b]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int b = 0; b < kCSJB; ++b) {
        const int64_t q = qbase + (int64_t)b * kCSThreads;
        if (q >= a.Q) continue;
        float* p = a.part + ((int64_t)blockIdx.y * a.Q + q) * 3;
        p[0] = S0[b];
        p[1] = S1[b];
        p[2] = S2[b];
    }
}

// mean = sum u y / sum u (NaN when sum u = 0), fat = norm * sum u w / sum u (0 then)
__global__ void k_cond_stats_final(const float* __restrict__ part, int n_split, int64_t Q, double norm,
                                   double* __restrict__ mean, double* __restrict__ fat) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int s = 0; s < n_split; ++s) {
        const float* p = part + ((int64_t)s * Q + q) * 3;
        s0 += p[0];
        s1 += p[1];
        s2 += p[2];
    }
    if (mean) mean[q] = s1 / s0;
    if (fat) fat[q] = s0 > 0.0 ? norm * s2 / s0 : 0.0;
}

// --------------------------------------------------------------------------
// Sampling and the narrowest interval: one CTA (256 threads) per query
// --------------------------------------------------------------------------
constexpr int kSmpThreads = 256, kSmpMax = 4096;

struct SampleArgs {
    const float* xs;
    const float* y;
    const float* xq;   // [d][Qp]
    const float* mq;   // [Q] (Gaussian)
    int64_t N, Np, Q, Qp;
    int d, S, SP, m_keep;   // samples, padded power of two, window size ceil((1-alpha) S)
    float a1, h2;
    uint64_t seed;
    float* lo;         // [Q]
    float* hi;         // [Q]
    float* samples;    // [Q][S] sorted, or null
};

struct SampleSmem {
    float val[kSmpMax];   // targets, then sample values
    int idx[kSmpMax];     // resolved data index per target
    float P[kSmpThreads]; // inclusive scan of the chunk's weights
    float wsum[kSmpThreads / 32];
    int wpos[kSmpThreads / 32];
    float xq[kMaxD];
    float total, base;
    int last, chunk_last, p, p2;
    float best_w[kSmpThreads / 32];
    int best_k[kSmpThreads / 32];
};

// inclusive scan of v over the CTA in a fixed order (warp shuffles, then the
// warp totals); returns this thread's prefix and leaves the total in P[255]
__device__ __forceinline__ float block_scan(float v, SampleSmem& S) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    if (lane == 31) S.wsum[warp] = v;
    __syncthreads();
    if (tid == 0)
        for (int w = 1; w < kSmpThreads / 32; ++w) S.wsum[w] += S.wsum[w - 1];
    __syncthreads();
    if (warp > 0) v += S.wsum[warp - 1];
    S.P[tid] = v;
    __syncthreads();
    return v;
}

__device__ __forceinline__ void bitonic_sort(float* v, int n) {
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const float x = v[i], z = v[ixj];
                    if ((x > z) == up) {
                        v[i] = z;
                        v[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
}

template <int KERN>
__device__ __forceinline__ float weight_at(const SampleArgs& a, const SampleSmem& S, int64_t i, float mq) {
    if (i >= a.N) return 0.f;
    float dx2 = 0.f;
    for (int c = 0; c < a.d; ++c) {
        const float v = S.xq[c] - a.xs[(int64_t)c * a.Np + i];
        dx2 = fmaf(v, v, dx2);
    }
    return xweight<KERN>(dx2, a.a1, mq);
}

template <int KERN>
__global__ void __launch_bounds__(kSmpThreads) k_cond_sample(const SampleArgs a) {
    extern __shared__ float4 smp4[];
    SampleSmem& S = *reinterpret_cast<SampleSmem*>(smp4);
    const int tid = threadIdx.x;
    const int64_t q = blockIdx.x;
    for (int c = tid; c < a.d; c += kSmpThreads) S.xq[c] = a.xq[(int64_t)c * a.Qp + q];
    const float mq = KERN == 0 ? a.mq[q] : 0.f;
    if (tid == 0) {
        S.total = 0.f;
        S.last = -1;
    }
    __syncthreads();
    const int64_t n_chunks = (a.N + kSmpThreads - 1) / kSmpThreads;
    // pass 1: the total weight, chunk by chunk in the order of pass 2
    for (int64_t k = 0; k < n_chunks; ++k) {
        const int64_t i = k * kSmpThreads + tid;
        const float u = weight_at<KERN>(a, S, i, mq);
        block_scan(u, S);
        if (u > 0.f) atomicMax(&S.last, (int)i);
        if (tid == 0) S.total = S.total + S.P[kSmpThreads - 1];
        __syncthreads();
    }
    const float total = S.total;
    const int last = S.last;
    if (last < 0 || !(total > 0.f)) {  // no weight (Epanechnikov: no x-neighbour)
        if (tid == 0) {
            a.lo[q] = NAN;
            a.hi[q] = NAN;
        }
        if (a.samples)
            for (int s = tid; s < a.S; s += kSmpThreads) a.samples[q * a.S + s] = NAN;
        return;
    }
    // sorted index targets
    for (int s = tid; s < a.SP; s += kSmpThreads)
        S.val[s] = s < a.S ? uniform24(a.seed, 2 * ((uint64_t)q * a.S + s)) * total : INFINITY;
    __syncthreads();
    bitonic_sort(S.val, a.SP);
    // pass 2: resolve the targets against the cumulative weights
    if (tid == 0) {
        S.base = 0.f;
        S.p = 0;
    }
    __syncthreads();
    for (int64_t k = 0; k < n_chunks; ++k) {
        const int64_t i = k * kSmpThreads + tid;
        const float u = weight_at<KERN>(a, S, i, mq);
        if (tid == 0) S.chunk_last = -1;
        block_scan(u, S);
        if (u > 0.f) atomicMax(&S.chunk_last, tid);
        if (tid == 0) {
            const float end = S.base + S.P[kSmpThreads - 1];
            int lo = S.p, hi = a.S;  // first target >= end
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (S.val[mid] < end) lo = mid + 1;
                else hi = mid;
            }
            S.p2 = lo;
        }
        __syncthreads();
        if (S.chunk_last >= 0)
            for (int s = S.p + tid; s < S.p2; s += kSmpThreads) {
                const float t = S.val[s] - S.base;
                int lo = 0, hi = kSmpThreads;  // first prefix above t
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (S.P[mid] <= t) lo = mid + 1;
                    else hi = mid;
                }
                if (lo > S.chunk_last) lo = S.chunk_last;  // rounding at the chunk's end
                S.idx[s] = (int)(k * kSmpThreads + lo);
            }
        __syncthreads();
        if (tid == 0) {
            S.base = S.base + S.P[kSmpThreads - 1];
            if (S.chunk_last >= 0) S.p = S.p2;
        }
        __syncthreads();
    }
    for (int s = S.p + tid; s < a.S; s += kSmpThreads) S.idx[s] = last;  // targets at the very top
    __syncthreads();
    // sample values, sorted
    for (int s = tid; s < a.SP; s += kSmpThreads) {
        float v = INFINITY;
        if (s < a.S) {
            const float V = uniform24(a.seed, 2 * ((uint64_t)q * a.S + s) + 1);
            const float e = KERN == 0 ? normcdfinvf(V) : 2.f * sinf(asinf(2.f * V - 1.f) * (1.f / 3.f));
            v = a.y[CDE_CK(S.idx[s], a.N, 302)] + a.h2 * e;
        }
        S.val[s] = v;
    }
    __syncthreads();
    bitonic_sort(S.val, a.SP);
    // narrowest window of m_keep consecutive values (first minimum)
    const int m = a.m_keep;
    float bw = INFINITY;
    int bk = 0x7fffffff;
    for (int k = tid; k + m - 1 < a.S; k += kSmpThreads) {
        const float w = S.val[k + m - 1] - S.val[k];
        if (w < bw) {
            bw = w;
            bk = k;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ow = __shfl_xor_sync(0xffffffffu, bw, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (ow < bw || (ow == bw && ok < bk)) {
            bw = ow;
            bk = ok;
        }
    }
    if ((tid & 31) == 0) {
        S.best_w[tid >> 5] = bw;
        S.best_k[tid >> 5] = bk;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kSmpThreads / 32; ++w)
            if (S.best_w[w] < bw || (S.best_w[w] == bw && S.best_k[w] < bk)) {
                bw = S.best_w[w];
                bk = S.best_k[w];
            }
        a.lo[q] = S.val[bk];
        a.hi[q] = S.val[bk + m - 1];
    }
    if (a.samples)
        for (int s = tid; s < a.S; s += kSmpThreads) a.samples[q * a.S + s] = S.val[s];
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
// Standardised SoA queries (and the Gaussian shifts) on the stream; caller frees.
static int prep_queries(cde_ctx* ctx, const Dataset& D, const float* d_xq, int64_t Q, int64_t Qp,
                        float** xq_out, float** mq_out, cudaStream_t st) {
    float *xq = nullptr, *mq = nullptr;
    double* stats = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&xq, (size_t)Qp * D.d * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&mq, (size_t)Q * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&stats, (size_t)2 * D.d * sizeof(double), st));
    CDE_CUDA(cudaMemcpyAsync(stats, D.mean.data(), D.d * sizeof(double), cudaMemcpyHostToDevice, st));
    CDE_CUDA(cudaMemcpyAsync(stats + D.d, D.sd.data(), D.d * sizeof(double), cudaMemcpyHostToDevice, st));
    k_query_pack<<<(unsigned)((Qp + 255) / 256), 256, 0, st>>>(d_xq, Q, Qp, D.d, stats, stats + D.d, xq);
    CDE_CUDA(cudaGetLastError());
    if (D.kernel == CDE_KERNEL_GAUSS) {
        const int rc = query_shift_enqueue(ctx->sm_count, D, xq, Q, Qp, mq, st);
        if (rc != CDE_OK) return rc;
    }
    CDE_CUDA(cudaFreeAsync(stats, st));
    *xq_out = xq;
    *mq_out = mq;
    return CDE_OK;
}

// queries per thread: more while the coordinates fit in registers
static int stats_jb(int d) { return d <= 8 ? 4 : d <= 16 ? 2 : 1; }

template <int KERN>
static void launch_stats_d(const StatArgs& a, dim3 grid, cudaStream_t st) {
    if (a.d <= 4) k_cond_stats<KERN, 4, 4><<<grid, kCSThreads, 0, st>>>(a);
    else if (a.d <= 8) k_cond_stats<KERN, 8, 4><<<grid, kCSThreads, 0, st>>>(a);
    else if (a.d <= 16) k_cond_stats<KERN, 16, 2><<<grid, kCSThreads, 0, st>>>(a);
    else k_cond_stats<KERN, 64, 1><<<grid, kCSThreads, 0, st>>>(a);
}

static int cond_stats_enqueue(cde_ctx* ctx, const Dataset& D, double h1, double h2, const float* d_xq,
                              const float* d_yq, int64_t Q, double* d_mean, double* d_fat, cudaStream_t st) {
    timing_reset(ctx);
    const int64_t Qp = (Q + 255) / 256 * 256;
    float *xq = nullptr, *mq = nullptr, *part = nullptr;
    int rc = prep_queries(ctx, D, d_xq, Q, Qp, &xq, &mq, st);
    if (rc != CDE_OK) return rc;
    const bool epan = D.kernel == CDE_KERNEL_EPAN;
    StatArgs a{};
    a.xs = D.xs;
    a.y = D.y;
    a.xq = xq;
    a.yq = d_yq;
    a.mq = mq;
    a.N = D.N;
    a.Np = D.Np;
    a.Q = Q;
    a.Qp = Qp;
    a.d = D.d;
    const double L2E = 1.4426950408889634074;
    a.a1 = (float)(epan ? 1.0 / (h1 * h1) : L2E / (2 * h1 * h1));
    a.a2 = (float)(epan ? 1.0 / (h2 * h2) : L2E / (2 * h2 * h2));
    const int64_t per_cta = (int64_t)kCSThreads * stats_jb(D.d);
    const int64_t gx = (Q + per_cta - 1) / per_cta;
    const int64_t tiles = (D.N + kCSThreads - 1) / kCSThreads;
    int64_t ns = (8LL * ctx->sm_count + gx - 1) / gx;
    if (ns > tiles) ns = tiles;
    if (ns < 1) ns = 1;
    const int64_t tps = (tiles + ns - 1) / ns;
    ns = (tiles + tps - 1) / tps;
    a.i_per_split = tps * kCSThreads;
    CDE_CUDA(cudaMallocAsync((void**)&part, (size_t)ns * Q * 3 * sizeof(float), st));
    a.part = part;
    const dim3 grid((unsigned)gx, (unsigned)ns);
    timing_begin(ctx, st);
    if (epan) launch_stats_d<1>(a, grid, st);
    else launch_stats_d<0>(a, grid, st);
    timing_end(ctx, st);
    CDE_CUDA(cudaGetLastError());
    const double norm = epan ? std::exp(epan_log_norm(1)) / h2 : 1.0 / (2.5066282746310002 * h2);
    k_cond_stats_final<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(part, (int)ns, Q, norm, d_mean,
                                                                   d_yq ? d_fat : nullptr);
    CDE_CUDA(cudaGetLastError());
    cudaFreeAsync(part, st);
    cudaFreeAsync(xq, st);
    cudaFreeAsync(mq, st);
    return CDE_OK;
}

static int cond_interval_enqueue(cde_ctx* ctx, const Dataset& D, double h1, double h2, const float* d_xq,
                                 int64_t Q, int S, double alpha, uint64_t seed, float* d_lo, float* d_hi,
                                 float* d_samples, cudaStream_t st) {
    const int64_t Qp = (Q + 255) / 256 * 256;
    float *xq = nullptr, *mq = nullptr;
    int rc = prep_queries(ctx, D, d_xq, Q, Qp, &xq, &mq, st);
    if (rc != CDE_OK) return rc;
    const bool epan = D.kernel == CDE_KERNEL_EPAN;
    SampleArgs a{};
    a.xs = D.xs;
    a.y = D.y;
    a.xq = xq;
    a.mq = mq;
    a.N = D.N;
    a.Np = D.Np;
    a.Q = Q;
    a.Qp = Qp;
    a.d = D.d;
    a.S = S;
    int sp = 1;
    while (sp < S) sp <<= 1;
    a.SP = sp;
    a.m_keep = (int)std::ceil((1.0 - alpha) * S - 1e-9);
    if (a.m_keep < 1) a.m_keep = 1;
    if (a.m_keep > S) a.m_keep = S;
    const double L2E = 1.4426950408889634074;
    a.a1 = (float)(epan ? 1.0 / (h1 * h1) : L2E / (2 * h1 * h1));
    a.h2 = (float)h2;
    a.seed = seed;
    a.lo = d_lo;
    a.hi = d_hi;
    a.samples = d_samples;
    static std::atomic<uint64_t> attr0{0}, attr1{0};
    CDE_CUDA(smem_attr_once(attr0, k_cond_sample<0>, (int)sizeof(SampleSmem)));
    CDE_CUDA(smem_attr_once(attr1, k_cond_sample<1>, (int)sizeof(SampleSmem)));
    // one CTA per query (grid.x allows 2^31 - 1)
    if (epan) k_cond_sample<1><<<(unsigned)Q, kSmpThreads, sizeof(SampleSmem), st>>>(a);
    else k_cond_sample<0><<<(unsigned)Q, kSmpThreads, sizeof(SampleSmem), st>>>(a);
    CDE_CUDA(cudaGetLastError());
    cudaFreeAsync(xq, st);
    cudaFreeAsync(mq, st);
    return CDE_OK;
}

#ifdef CDE_CHECKS
CDE_CHECK_READER(check_status_products)
#endif

}  // namespace cde

using namespace cde;

static int check_bw(double h1, double h2, const char* who) {
    if (!std::isfinite(h1) || !std::isfinite(h2) || h1 < 1e-12 || h2 < 1e-12 || h1 > 1e12 || h2 > 1e12)
        return set_error(CDE_EINVAL, std::string(who) + ": bandwidth must be finite in [1e-12, 1e12]");
    return CDE_OK;
}

extern "C" int cde_cond_stats(cde_ctx* ctx, cde_dataset ds, double h1, double h2, const float* xq,
                              const float* yq, int64_t Q, double* mean_out, double* fat_out, int flags,
                              void* stream) {
    CDE_NVTX("cde_cond_stats");
    if (!ctx) return set_error(CDE_EINVAL, "cde_cond_stats: null context");
    int rc = check_bw(h1, h2, "cde_cond_stats");
    if (rc != CDE_OK) return rc;
    if (Q < 0 || (Q > 0 && (!xq || (!mean_out && !fat_out) || (fat_out && !yq))))
        return set_error(CDE_EINVAL, "cde_cond_stats: bad sizes or null pointers");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_cond_stats: unknown dataset");
    if (Q == 0) return CDE_OK;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    const bool in_dev = flags & CDE_IN_DEVICE, out_dev = flags & CDE_OUT_DEVICE;
    const float* dq = xq;
    const float* dy = yq;
    float *dxq = nullptr, *dyq = nullptr;
    double *dmean = out_dev ? mean_out : nullptr, *dfat = out_dev ? fat_out : nullptr;
    if (!in_dev) {
        for (int64_t e = 0; e < Q * D->d; ++e)
            if (!std::isfinite(xq[e])) return set_error(CDE_EINVAL, "cde_cond_stats: non-finite query");
        CDE_CUDA(cudaMallocAsync((void**)&dxq, (size_t)Q * D->d * sizeof(float), st));
        CDE_CUDA(cudaMemcpyAsync(dxq, xq, (size_t)Q * D->d * sizeof(float), cudaMemcpyHostToDevice, st));
        dq = dxq;
        if (yq) {
            CDE_CUDA(cudaMallocAsync((void**)&dyq, (size_t)Q * sizeof(float), st));
            CDE_CUDA(cudaMemcpyAsync(dyq, yq, (size_t)Q * sizeof(float), cudaMemcpyHostToDevice, st));
            dy = dyq;
        }
    }
    if (!out_dev) {
        if (mean_out) CDE_CUDA(cudaMallocAsync((void**)&dmean, (size_t)Q * sizeof(double), st));
        if (fat_out) CDE_CUDA(cudaMallocAsync((void**)&dfat, (size_t)Q * sizeof(double), st));
    }
    rc = cond_stats_enqueue(ctx, *D, h1, h2, dq, fat_out ? dy : nullptr, Q, dmean, dfat, st);
    cudaError_t e = cudaSuccess;
    if (rc == CDE_OK && !out_dev) {
        if (mean_out) e = cudaMemcpyAsync(mean_out, dmean, (size_t)Q * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && fat_out)
            e = cudaMemcpyAsync(fat_out, dfat, (size_t)Q * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    if (dxq) cudaFreeAsync(dxq, st);
    if (dyq) cudaFreeAsync(dyq, st);
    if (!out_dev) {
        if (dmean) cudaFreeAsync(dmean, st);
        if (dfat) cudaFreeAsync(dfat, st);
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (rc == CDE_OK && e == cudaSuccess && e2 != cudaSuccess) e = e2;
    }
    if (rc != CDE_OK) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cde_cond_stats");
    return CDE_OK;
}

extern "C" int cde_cond_interval(cde_ctx* ctx, cde_dataset ds, double h1, double h2, const float* xq,
                                 int64_t Q, int S, double alpha, uint64_t seed, float* lo_out, float* hi_out,
                                 float* samples_out, int flags, void* stream) {
    CDE_NVTX("cde_cond_interval");
    if (!ctx) return set_error(CDE_EINVAL, "cde_cond_interval: null context");
    int rc = check_bw(h1, h2, "cde_cond_interval");
    if (rc != CDE_OK) return rc;
    if (Q < 0 || S < 1 || S > kSmpMax || !(alpha > 0.0 && alpha < 1.0) ||
        (Q > 0 && (!xq || !lo_out || !hi_out)))
        return set_error(CDE_EINVAL, "cde_cond_interval: need 1 <= S <= 4096, 0 < alpha < 1, non-null pointers");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_cond_interval: unknown dataset");
    if (Q == 0) return CDE_OK;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    const bool in_dev = flags & CDE_IN_DEVICE, out_dev = flags & CDE_OUT_DEVICE;
    const float* dq = xq;
    float* dxq = nullptr;
    float *dlo = out_dev ? lo_out : nullptr, *dhi = out_dev ? hi_out : nullptr;
    float* dsm = out_dev ? samples_out : nullptr;
    if (!in_dev) {
        for (int64_t e = 0; e < Q * D->d; ++e)
            if (!std::isfinite(xq[e])) return set_error(CDE_EINVAL, "cde_cond_interval: non-finite query");
        CDE_CUDA(cudaMallocAsync((void**)&dxq, (size_t)Q * D->d * sizeof(float), st));
        CDE_CUDA(cudaMemcpyAsync(dxq, xq, (size_t)Q * D->d * sizeof(float), cudaMemcpyHostToDevice, st));
        dq = dxq;
    }
    if (!out_dev) {
        CDE_CUDA(cudaMallocAsync((void**)&dlo, (size_t)Q * sizeof(float), st));
        CDE_CUDA(cudaMallocAsync((void**)&dhi, (size_t)Q * sizeof(float), st));
        if (samples_out) CDE_CUDA(cudaMallocAsync((void**)&dsm, (size_t)Q * S * sizeof(float), st));
    }
    rc = cond_interval_enqueue(ctx, *D, h1, h2, dq, Q, S, alpha, seed, dlo, dhi, dsm, st);
    cudaError_t e = cudaSuccess;
    if (rc == CDE_OK && !out_dev) {
        e = cudaMemcpyAsync(lo_out, dlo, (size_t)Q * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hi_out, dhi, (size_t)Q * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && samples_out)
            e = cudaMemcpyAsync(samples_out, dsm, (size_t)Q * S * sizeof(float), cudaMemcpyDeviceToHost, st);
    }
    if (dxq) cudaFreeAsync(dxq, st);
    if (!out_dev) {
        cudaFreeAsync(dlo, st);
        cudaFreeAsync(dhi, st);
        if (dsm) cudaFreeAsync(dsm, st);
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (rc == CDE_OK && e == cudaSuccess && e2 != cudaSuccess) e = e2;
    }
    if (rc != CDE_OK) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cde_cond_interval");
    return CDE_OK;
}
