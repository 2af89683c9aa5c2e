// Exact all-pairs leave-one-out log-likelihood of the double-kernel
// conditional density estimator over a grid of bandwidth pairs.
//
// Holmes, Gray & Isbell, Sec. 3.2: L = (1/n) sum_j ln A_j - ln(n-1) with
// A_j = sum_{i!=j} K_h1(|x_j-x_i|) K_h2(y_j-y_i); the conditional score adds
// B_j = sum_{i!=j} K_h1(|x_j-x_i|) and sums ln(A_j/B_j) (Eq. 1 at the left-out
// point).  Every pair (j,i) is visited once for all G1 x G2 bandwidths:
//
//   u_i(k) = 2^{a1_k (m_x,j - |x_j-x_i|^2)},  w_i(l) = 2^{a2_l (m_y,j - (y_j-y_i)^2)},
//   a1_k = log2(e)/(2 h1_k^2),  a2_l = log2(e)/(2 h2_l^2),
//   At_j(k,l) = sum_i u_i(k) w_i(l),     Bt_j(k) = sum_i u_i(k),
//
// where m_x,j / m_y,j are row j's nearest squared distances in x and in y (so
// the largest u and the largest w are exactly 1: no overflow, and B never
// underflows).  The Gaussian factors are separable, so one squared distance
// per pair feeds G1 + G2 exp2 (MUFU), and the G1 x G2 outer-product sums run on
// the tensor cores as per-row TF32 GEMMs with split operands (loo_mma.cuh).  The epilogue
// removes the shifts and the kernel constants in FP64:
//   ell_j = ln2 (log2 At - log2 Bt - a2_l m_y,j) - ln(sqrt(2 pi) h2_l)
//   ln A_j = ln2 (log2 At - a1_k m_x,j - a2_l m_y,j) - d ln(sqrt(2pi) h1_k) - ln(sqrt(2pi) h2_l)
// A cell whose shifted numerator At falls below 2^(ceil(log2 N) - 91) (the
// x-nearest and the y-nearest neighbours differ and both factors are small;
// below it the terms that lost precision to the FP32 range could matter) is
// recomputed exactly with a joint shift anchored at
// argmin_i [a1 (dx2-m_x) + a2 (dy2-m_y)].
//
// Work decomposition: a CTA of 8 warps owns a "unit" of JW = 1024/(G1 G2)
// rows (G1 padded to 16 or 32, G2 to 8, 16 or 32); the 8 warps split the i
// range in interleaved chunks of 32 points and their FP32 partial sums are
// combined in fixed warp order.  Units are grouped
// into tiles; each tile's FP64 partial scores go to their own slot and a final
// kernel sums the slots in tile order, so results are bitwise reproducible and
// independent of how tiles are scheduled.
#include <cmath>
#include <cstdio>

#include "cde_internal.h"
#include "loo_common.cuh"
#include "loo_mma.cuh"

namespace cde {

// --------------------------------------------------------------------------
// Dataset packing: optional FP64 standardisation, row-major -> SoA.
// --------------------------------------------------------------------------
__global__ void k_col_stats(const float* __restrict__ x, int64_t N, int d, double* stats) {
    // one CTA per column: mean, then sum of squared deviations (fixed-order tree)
    __shared__ double red[1024];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += (double)x[i * d + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = red[0] / (double)N;
    __syncthreads();
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        double t = (double)x[i * d + c] - mean;
        v += t * t;
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        stats[2 * c] = mean;
        stats[2 * c + 1] = sqrt(red[0] / (double)(N - 1));
    }
}

__global__ void k_pack(const float* __restrict__ x, const float* __restrict__ y, int64_t N,
                       int64_t Np, int d, const double* __restrict__ stats, int standardize,
                       float* __restrict__ xs, float* __restrict__ ys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Np) return;
    for (int c = 0; c < d; ++c) {
        float v = 0.f;
        if (i < N) {
            if (standardize)
                v = (float)(((double)x[i * d + c] - stats[2 * c]) / stats[2 * c + 1]);
            else
                v = x[i * d + c];
        }
        xs[(int64_t)c * Np + i] = v;
    }
    ys[i] = i < N ? y[i] : 0.f;
}

int pack_enqueue(Dataset& D, const float* d_x, const float* d_y, cudaStream_t st, double* d_stats) {
    if (D.standardized) {
        k_col_stats<<<D.d, 1024, 0, st>>>(d_x, D.N, D.d, d_stats);
        CDE_CUDA(cudaGetLastError());
    }
    const int64_t blocks = (D.Np + 255) / 256;
    k_pack<<<(unsigned)blocks, 256, 0, st>>>(d_x, d_y, D.N, D.Np, D.d, d_stats, D.standardized,
                                             D.xs, D.y);
    CDE_CUDA(cudaGetLastError());
    return CDE_OK;
}

// --------------------------------------------------------------------------
// Per-row nearest squared distances (the exp2 shifts), O(N^2 d), computed
// once per dataset.  Same FP32 distance formula as every pair kernel.
// Alongside each minimum the kernels keep the other coordinate's distance of
// the point that attains it -- qy_j = dy^2 of the x-nearest point, qx_j = dx^2
// of the y-nearest point -- minimising the pair lexicographically, so ties
// keep the smaller second distance and the result does not depend on the
// order in which points are visited.  Every joint minimiser of
// a1 (dx^2 - m_x) + a2 (dy^2 - m_y) (a1, a2 > 0) has dx^2 <= qx and dy^2 <= qy
// (it can be no worse than either neighbour), which is what the exact
// fallback of the grid kernels uses to skip points.
// --------------------------------------------------------------------------

// (a, b) < (c, d) lexicographically
__device__ __forceinline__ bool lex_less(float a, float b, float c, float d) {
    return a < c || (a == c && b < d);
}

__global__ void __launch_bounds__(256) k_nn_shift(const float* __restrict__ xs,
                                                  const float* __restrict__ y, int64_t N,
                                                  int64_t Np, int d, float* __restrict__ mx,
                                                  float* __restrict__ my, float* __restrict__ qx,
                                                  float* __restrict__ qy) {
    extern __shared__ float sm[];  // [d + 1][256]
    const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const bool vj = j < N;
    float xj[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xj[c] = (vj && c < d) ? xs[(int64_t)c * Np + j] : 0.f;
    const float yj = vj ? y[j] : 0.f;
    float bx = INFINITY, by = INFINITY, ax = INFINITY, ay = INFINITY;
    for (int64_t i0 = 0; i0 < N; i0 += 256) {
        __syncthreads();
        for (int c = 0; c <= d; ++c) {
            const float* src = c < d ? xs + (int64_t)c * Np : y;
            sm[c * 256 + threadIdx.x] = src[i0 + threadIdx.x];  // i0+tid < Np
        }
        __syncthreads();
        const int n = (int)min((int64_t)256, N - i0);
        for (int t = 0; t < n; ++t) {
            const int64_t i = i0 + t;
            float dx2 = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < d) {
                    float u = xj[c] - sm[c * 256 + t];
                    dx2 = fmaf(u, u, dx2);
                }
            for (int c = 8; c < d; ++c) {
                float u = xs[(int64_t)c * Np + j * vj] - sm[c * 256 + t];
                dx2 = fmaf(u, u, dx2);
            }
            const float dy = yj - sm[d * 256 + t];
            const float dy2 = dy * dy;
            if (i != j) {
                if (lex_less(dx2, dy2, bx, ax)) {
                    bx = dx2;
                    ax = dy2;
                }
                if (lex_less(dy2, dx2, by, ay)) {
                    by = dy2;
                    ay = dx2;
                }
            }
        }
    }
    if (vj) {
        mx[j] = bx;
        my[j] = by;
        qy[j] = ax;
        qx[j] = ay;
    }
}

// d <= 8: four rows per thread, point-major shared tiles (128-bit loads), the
// data range split over gridDim.y; split minima merge with a 64-bit integer
// atomicMin on (minimum, other distance) bit pairs (exact and order-free:
// squared distances are non-negative, so their bit patterns order like the
// values).  The distance is accumulated in the same order (dimension 0 first,
// one fmaf per dimension; padding dimensions add exactly 0) as in every pair
// kernel.
constexpr int kNnThreads = 128, kNnJB = 4;   // rows per thread (even: packed pairs)

__device__ __forceinline__ unsigned long long nn_key(float m, float o) {
    return ((unsigned long long)__float_as_uint(m) << 32) | __float_as_uint(o);
}

template <int DREG>
__global__ void __launch_bounds__(kNnThreads) k_nn_shift_split(const float* __restrict__ xs,
                                                               const float* __restrict__ y, int64_t N,
                                                               int64_t Np, int d, int64_t i_per_split,
                                                               unsigned long long* __restrict__ kx,
                                                               unsigned long long* __restrict__ ky) {
    __shared__ __align__(16) float xt[kNnThreads][DREG];
    __shared__ float yt[kNnThreads];
    const int tid = threadIdx.x;
    const int64_t jbase = (int64_t)blockIdx.x * kNnThreads * kNnJB + tid;
    const int64_t i0 = (int64_t)blockIdx.y * i_per_split;
    const int64_t i1 = min(N, i0 + i_per_split);
    // running lexicographic minima as keys (minimum bits, other coordinate's bits):
    // non-negative floats order like their bit patterns, so one 64-bit compare is
    // the (minimum, then other distance) order
    float xj[kNnJB][DREG], yj[kNnJB];
    unsigned long long mkx[kNnJB], mky[kNnJB];
    int jj[kNnJB];
#pragma unroll
    for (int b = 0; b < kNnJB; ++b) {
        const int64_t j = jbase + (int64_t)b * kNnThreads;
        const int64_t jc = j < N ? j : 0;
        jj[b] = (int)j;
#pragma unroll
        for (int c = 0; c < DREG; ++c) xj[b][c] = c < d ? xs[(int64_t)c * Np + jc] : 0.f;
        yj[b] = y[jc];
        mkx[b] = mky[b] = nn_key(INFINITY, INFINITY);
    }
    for (int64_t t0 = i0; t0 < i1; t0 += kNnThreads) {
        __syncthreads();
        const int64_t it = CDE_CK(t0 + tid, Np, 110);  // < Np: splits and Np are multiples of 128
#pragma unroll
        for (int c = 0; c < DREG; ++c) xt[tid][c] = c < d ? xs[(int64_t)c * Np + it] : 0.f;
        yt[tid] = y[it];
        __syncthreads();
        const int n = (int)min((int64_t)kNnThreads, i1 - t0);
        for (int t = 0; t < n; ++t) {
            const int i32 = (int)(t0 + t);
            float xi[DREG];
#pragma unroll
            for (int c = 0; c < DREG; c += 4) {
                const float4 v4 = *reinterpret_cast<const float4*>(&xt[t][c]);
                xi[c] = v4.x;
                xi[c + 1] = v4.y;
                xi[c + 2] = v4.z;
                xi[c + 3] = v4.w;
            }
            const float yi = yt[t];
            // rows in packed FP32x2 pairs; x_j - x_i as fma(x_i, -1, x_j), the
            // scalar subtraction's rounding, so the minima are bitwise the same
            const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
            for (int b = 0; b < kNnJB; b += 2) {
                float2 dx2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < DREG; ++c) {
                    const float2 q = __ffma2_rn(make_float2(xi[c], xi[c]), m1, make_float2(xj[b][c], xj[b + 1][c]));
                    dx2 = __ffma2_rn(q, q, dx2);
                }
                const float2 dy = __ffma2_rn(make_float2(yi, yi), m1, make_float2(yj[b], yj[b + 1]));
                const float2 dy2 = __fmul2_rn(dy, dy);
                const bool o0 = i32 != jj[b], o1 = i32 != jj[b + 1];
                const unsigned long long x0 = nn_key(dx2.x, dy2.x), x1 = nn_key(dx2.y, dy2.y);
                const unsigned long long y0 = nn_key(dy2.x, dx2.x), y1 = nn_key(dy2.y, dx2.y);
                if (o0 && x0 < mkx[b]) mkx[b] = x0;
                if (o1 && x1 < mkx[b + 1]) mkx[b + 1] = x1;
                if (o0 && y0 < mky[b]) mky[b] = y0;
                if (o1 && y1 < mky[b + 1]) mky[b + 1] = y1;
            }
        }
    }
#pragma unroll
    for (int b = 0; b < kNnJB; ++b) {
        const int64_t j = jbase + (int64_t)b * kNnThreads;
        if (j >= N) continue;
        atomicMin(kx + j, mkx[b]);
        atomicMin(ky + j, mky[b]);
    }
}

// unpack the merged (minimum, other distance) keys
__global__ void k_nn_unpack(const unsigned long long* __restrict__ kx, const unsigned long long* __restrict__ ky,
                            int64_t N, float* __restrict__ mx, float* __restrict__ my, float* __restrict__ qx,
                            float* __restrict__ qy) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const unsigned long long a = kx[j], b = ky[j];
    mx[j] = __uint_as_float((unsigned int)(a >> 32));
    qy[j] = __uint_as_float((unsigned int)a);
    my[j] = __uint_as_float((unsigned int)(b >> 32));
    qx[j] = __uint_as_float((unsigned int)b);
}

int nn_shift_enqueue(const Dataset& D, cudaStream_t st, int sm_count) {
    if (D.d <= 8) {
        const int64_t per_cta = (int64_t)kNnThreads * kNnJB;
        const int64_t gx = (D.N + per_cta - 1) / per_cta;
        const int64_t tiles = (D.N + kNnThreads - 1) / kNnThreads;
        int64_t ns = (4LL * sm_count + gx - 1) / gx;
        if (ns > tiles) ns = tiles;
        if (ns < 1) ns = 1;
        const int64_t tps = (tiles + ns - 1) / ns;
        ns = (tiles + tps - 1) / tps;
        unsigned long long* keys = nullptr;   // [2][N] merge keys, stream-ordered scratch
        CDE_CUDA(cudaMallocAsync((void**)&keys, (size_t)2 * D.N * sizeof(unsigned long long), st));
        // 0x7f bytes: the first word 3.4e38, above any distance
        CDE_CUDA(cudaMemsetAsync(keys, 0x7f, (size_t)2 * D.N * sizeof(unsigned long long), st));
        const dim3 grid((unsigned)gx, (unsigned)ns);
        if (D.d <= 4)
            k_nn_shift_split<4><<<grid, kNnThreads, 0, st>>>(D.xs, D.y, D.N, D.Np, D.d, tps * kNnThreads, keys, keys + D.N);
        else
            k_nn_shift_split<8><<<grid, kNnThreads, 0, st>>>(D.xs, D.y, D.N, D.Np, D.d, tps * kNnThreads, keys, keys + D.N);
        CDE_CUDA(cudaGetLastError());
        k_nn_unpack<<<(unsigned)((D.N + 255) / 256), 256, 0, st>>>(keys, keys + D.N, D.N, D.mx, D.my, D.qx, D.qy);
        CDE_CUDA(cudaGetLastError());
        CDE_CUDA(cudaFreeAsync(keys, st));
        return CDE_OK;
    }
    const int64_t blocks = (D.N + 255) / 256;
    const size_t smem = (size_t)(D.d + 1) * 256 * sizeof(float);
    if (smem > 48 * 1024)
        CDE_CUDA(cudaFuncSetAttribute(k_nn_shift, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_nn_shift<<<(unsigned)blocks, 256, smem, st>>>(D.xs, D.y, D.N, D.Np, D.d, D.mx, D.my, D.qx, D.qy);
    CDE_CUDA(cudaGetLastError());
    return CDE_OK;
}

// --------------------------------------------------------------------------
// Final fixed-order reduction of tile partials: one warp per grid cell.
// --------------------------------------------------------------------------
__global__ void k_loo_final(const double* __restrict__ part, int n_tiles, int GG, int G2T,
                            int G1r, int G2r, int ld, double N, double* Lc, double* Le) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= GG) return;
    const int k = warp / G2T, l = warp % G2T;
    double sc, se;
    loo_final_cell(part, n_tiles, GG, warp, lane, sc, se);
    if (lane == 0 && k < G1r && l < G2r) {
        if (Lc) Lc[k * ld + l] = sc;
        if (Le) Le[k * ld + l] = se / N - log(N - 1.0);
    }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
template <int G1, int G2, int KERN>
static int launch_shape_k(const LooArgs& a, int grid, cudaStream_t st) {
    using C = MmaCfg<G1, G2>;
    const size_t smem = C::smem_bytes(a.d);
    static std::atomic<uint64_t> attr{0};   // per instantiation
    CDE_CUDA(smem_attr_once(attr, k_loo_mma<G1, G2, KERN>, (int)C::smem_bytes(kMaxD)));
    k_loo_mma<G1, G2, KERN><<<grid, C::kThreads, smem, st>>>(a);
    CDE_CUDA(cudaGetLastError());
    return CDE_OK;
}

template <int G1, int G2>
static int launch_shape(const LooArgs& a, int grid, cudaStream_t st) {
    return a.kern == CDE_KERNEL_EPAN ? launch_shape_k<G1, G2, 1>(a, grid, st)
                                     : launch_shape_k<G1, G2, 0>(a, grid, st);
}


int launch_loo_tile_kernel(int T1, int T2, const LooArgs& a, int grid, cudaStream_t st) {
#define CDE_SHAPE(A, B) \
    if (T1 == A && T2 == B) return launch_shape<A, B>(a, grid, st);
    CDE_SHAPE(16, 8) CDE_SHAPE(16, 16) CDE_SHAPE(16, 32)
    CDE_SHAPE(32, 8) CDE_SHAPE(32, 16) CDE_SHAPE(32, 32)
#undef CDE_SHAPE
    return set_error(CDE_EINVAL, "unsupported grid block shape");
}

// ln c_d of the radial Epanechnikov kernel, c_d = (d + 2) / (2 V_d), with the
// unit-ball volume from V_0 = 1, V_1 = 2, V_k = (2 pi / k) V_{k-2}.
double epan_log_norm(int d) {
    double lv = (d % 2) ? std::log(2.0) : 0.0;
    for (int k = 2 + d % 2; k <= d; k += 2) lv += std::log(2.0 * M_PI / k);
    return std::log(d + 2.0) - std::log(2.0) - lv;
}

void fill_loo_args(LooArgs& a, const Dataset& D, const double* h1, int g1, const double* h2,
                   int g2, int T1, int T2) {
    a.xs = D.xs; a.y = D.y; a.mx = D.mx; a.my = D.my; a.qx = D.qx; a.qy = D.qy;
    a.N = D.N; a.Np = D.Np; a.d = D.d;
    a.kern = D.kernel;
    if (D.kernel == CDE_KERNEL_EPAN) {
        // profiles (1 - t/h^2)_+; ln K_h = ln(profile) - (d ln h - ln c_d); no shifts
        a.thresh = 0.f;
        const double lcd = epan_log_norm(D.d), lc1 = epan_log_norm(1);
        for (int k = 0; k < 32; ++k) {
            const double h = h1[k < g1 ? k : g1 - 1];
            a.a1[k] = (float)(1.0 / (h * h));
            a.lam1[k] = D.d * log(h) - lcd;
        }
        for (int l = 0; l < 32; ++l) {
            const double h = h2[l < g2 ? l : g2 - 1];
            a.a2[l] = (float)(1.0 / (h * h));
            a.kap2[l] = log(h) - lc1;
        }
        (void)T1; (void)T2;
        return;
    }
    // Recompute a cell exactly when its shifted numerator At is below
    // 2^(ceil(log2 N) - 91).  A term below 2^-115 loses its cross terms (their
    // lo factors leave the normal range) and one below 2^-126 flushes; N such
    // terms are at most N 2^-115 = 2^-24 of this threshold.
    {
        int lg = 0;
        while (((int64_t)1 << lg) < D.N) ++lg;
        a.thresh = ldexpf(1.f, lg - 91);
    }
    const double L2E = 1.4426950408889634074;      // log2(e)
    const double LNS2PI = 0.91893853320467274178;  // ln sqrt(2 pi)
    for (int k = 0; k < 32; ++k) {
        const double h = h1[k < g1 ? k : g1 - 1];
        a.a1[k] = (float)(L2E / (2.0 * h * h));
        a.lam1[k] = D.d * (LNS2PI + log(h));
    }
    for (int l = 0; l < 32; ++l) {
        const double h = h2[l < g2 ? l : g2 - 1];
        a.a2[l] = (float)(L2E / (2.0 * h * h));
        a.kap2[l] = LNS2PI + log(h);
    }
    (void)T1; (void)T2;
}

static int shape_index(int T) { return T <= 8 ? 0 : T <= 16 ? 1 : 2; }

// Units per tile: the autotuned value for this grid shape when the context has
// one, else enough units for 8 rows per tile.  Both the single-dataset and the
// batched launch use this, so they form identical tile partials.
// The autotuner's candidate of one shape class, seen by the launches of the
// tuning thread only: the context's table changes once, to the kept values, so
// other threads (the request loop) never plan with a candidate.
static thread_local int t_cand_a = -1, t_cand_b = -1, t_cand_upt = 0, t_cand_ctas = 0;

void tuning_candidate(int T1, int T2, int units_per_tile, int ctas_per_sm) {
    t_cand_a = shape_index(T1);
    t_cand_b = shape_index(T2);
    t_cand_upt = units_per_tile;
    t_cand_ctas = ctas_per_sm;
}

void tuning_candidate_clear() { t_cand_a = t_cand_b = -1; }

static int tuned_upt(cde_ctx* ctx, int T1, int T2) {
    const int a = shape_index(T1), b = shape_index(T2);
    if (a == t_cand_a && b == t_cand_b) return t_cand_upt;
    return ctx ? ctx->tune_upt[a][b] : 0;
}

static int tuned_ctas(cde_ctx* ctx, int T1, int T2) {
    const int a = shape_index(T1), b = shape_index(T2);
    if (a == t_cand_a && b == t_cand_b) return t_cand_ctas;
    return ctx ? ctx->tune_ctas[a][b] : 0;
}

int loo_units_per_tile(cde_ctx* ctx, int T1, int T2, int64_t n_rows) {
    const int t = tuned_upt(ctx, T1, T2);
    if (t > 0) return t;
    const int JW = 1024 / (T1 * T2);
    int upt = JW >= 8 ? 1 : 8 / JW;
    // Smaller tiles while the grid would give fewer than 64 tiles per resident CTA: the
    // tiles come from an atomic queue, and the last CTAs to finish decide the launch's time.
    // (N = 50,000 at 32 x 32: 70.3 ms with 8 rows per tile, 69.1 ms with 2.)
    if (ctx && n_rows > 0) {
        const int c = tuned_ctas(ctx, T1, T2);
        const int64_t units = (n_rows + JW - 1) / JW;
        const int64_t want = 64LL * (c > 0 ? c : 2) * ctx->sm_count;
        while (upt > 1 && (units + upt - 1) / upt < want) upt >>= 1;
    }
    return upt;
}

int loo_grid_ctas(cde_ctx* ctx, int T1, int T2) {
    const int c = tuned_ctas(ctx, T1, T2);
    return (c > 0 ? c : 2) * ctx->sm_count;
}

// Launch plan of one grid block: rows per unit, units per tile, tiles, CTAs and
// the scratch they need (tile partials, then the d >= 16 kernel's per-CTA buffer
// of recomputed cells, then the tile counter).
struct LooPlan {
    bool gram;
    int rpu, upt, n_units, n_tiles, grid;
    LooTiles tiles;
    size_t part_bytes, fb_bytes;
    size_t bytes() const { return part_bytes + fb_bytes + 256; }
};

static LooPlan loo_plan(cde_ctx* ctx, const Dataset& D, int T1, int T2, int64_t n_rows) {
    LooPlan p{};
    p.gram = loo_use_gram(D, T1, T2);
    p.rpu = p.gram ? loo_gram_rows_per_unit(T1, T2) : 1024 / (T1 * T2);
    p.upt = p.gram ? 1 : loo_units_per_tile(ctx, T1, T2, n_rows);
    p.n_units = (int)((n_rows + p.rpu - 1) / p.rpu);
    const int cmax = p.gram ? ctx->sm_count : loo_grid_ctas(ctx, T1, T2);
    p.tiles = loo_tiles(p.n_units, p.upt, cmax);
    p.n_tiles = p.tiles.n_tiles;
    p.grid = p.n_tiles < cmax ? p.n_tiles : cmax;
    p.part_bytes = (size_t)p.n_tiles * 2 * T1 * T2 * sizeof(double);
    p.fb_bytes = p.gram ? (size_t)p.grid * loo_gram_fb_bytes_per_cta() : 0;
    return p;
}

size_t loo_grid_scratch_bytes(cde_ctx* ctx, const Dataset& D, int G1, int G2, int64_t n_rows) {
    size_t mx = 0;
    for (int k0 = 0; k0 < G1; k0 += 32) {
        const int T1 = loo_pad1(G1 - k0 < 32 ? G1 - k0 : 32);
        for (int l0 = 0; l0 < G2; l0 += 32) {
            const int T2 = loo_pad2(G2 - l0 < 32 ? G2 - l0 : 32);
            const size_t b = loo_plan(ctx, D, T1, T2, n_rows).bytes();
            if (b > mx) mx = b;
        }
    }
    return mx;
}

int loo_grid_enqueue(cde_ctx* ctx, const Dataset& D, const double* h1, int G1, const double* h2,
                     int G2, const int64_t* d_rows, int64_t n_rows, double* d_Lc, double* d_Le,
                     double* d_ell_rows, cudaStream_t st, void* scratch, size_t scratch_bytes) {
    timing_reset(ctx);
    if (!d_rows) n_rows = D.N;
    for (int k0 = 0; k0 < G1; k0 += 32) {
        const int g1 = G1 - k0 < 32 ? G1 - k0 : 32;
        const int T1 = loo_pad1(g1);
        for (int l0 = 0; l0 < G2; l0 += 32) {
            const int g2 = G2 - l0 < 32 ? G2 - l0 : 32;
            const int T2 = loo_pad2(g2);
            LooArgs a{};
            fill_loo_args(a, D, h1 + k0, g1, h2 + l0, g2, T1, T2);
            const LooPlan pl = loo_plan(ctx, D, T1, T2, n_rows);
            a.rows = d_rows;
            a.n_rows = n_rows;
            a.n_units = pl.n_units;
            a.units_per_tile = pl.upt;
            a.n_tiles = pl.n_tiles;
            a.big_g = pl.tiles.big_g;
            a.big_levels = pl.tiles.big_levels;
            a.big_s0 = pl.tiles.big_s0;
            a.win0 = 0;
            a.win1 = INT_MAX;
            a.ell_rows = d_ell_rows ? d_ell_rows + (size_t)k0 * G2 + l0 : nullptr;
            a.ell_ld_row = (int64_t)G1 * G2;
            a.ell_ld_k = G2;
            a.G1r = g1;
            a.G2r = g2;
            double* part = nullptr;
            const bool own = !(scratch && pl.bytes() <= scratch_bytes);
            if (own) CDE_CUDA(cudaMallocAsync((void**)&part, pl.bytes(), st));
            else part = static_cast<double*>(scratch);
            a.part = part;
            a.fb = reinterpret_cast<double*>(reinterpret_cast<char*>(part) + pl.part_bytes);
            a.tile_base = 0;
            a.work = reinterpret_cast<int*>(reinterpret_cast<char*>(part) + pl.part_bytes + pl.fb_bytes);
            CDE_CUDA(cudaMemsetAsync(a.work, 0, sizeof(int), st));
            const int grid = pl.grid;
            timing_begin(ctx, st);
            int rc = pl.gram ? launch_loo_gram(T1, T2, a, grid, st) : launch_loo_tile_kernel(T1, T2, a, grid, st);
            timing_end(ctx, st);
            if (rc != CDE_OK) {
                if (own) cudaFreeAsync(part, st);
                return rc;
            }
            if (d_Lc || d_Le) {
                const int GG = T1 * T2;
                k_loo_final<<<(GG * 32 + 255) / 256, 256, 0, st>>>(
                    part, a.n_tiles, GG, T2, g1, g2, G2, (double)D.N,
                    d_Lc ? d_Lc + (size_t)k0 * G2 + l0 : nullptr,
                    d_Le ? d_Le + (size_t)k0 * G2 + l0 : nullptr);
                CDE_CUDA(cudaGetLastError());
            }
            if (own) CDE_CUDA(cudaFreeAsync(part, st));
        }
    }
    return CDE_OK;
}

#ifdef CDE_CHECKS
CDE_CHECK_READER(check_status_loo)
#endif

}  // namespace cde

namespace cde {

// --------------------------------------------------------------------------
// One grid block launched in tile ranges (the request loop's selection jobs):
// each range is its own launch, so other streams' kernels run between them.
// Every tile writes its own partial slot whatever launch processes it, and
// the final reduction is the one of loo_grid_enqueue, so the result is
// bitwise the result of a single launch.
// --------------------------------------------------------------------------
__global__ void k_set_int(int* p, int v) { *p = v; }

int loo_chunked_create(cde_ctx* ctx, const Dataset& D, const double* h1, int G1, const double* h2, int G2,
                       LooChunked** out) {
    if (G1 > 32 || G2 > 32) return set_error(CDE_EINVAL, "loo_chunked_create: one grid block (<= 32 x 32) only");
    auto* c = new LooChunked{};
    c->T1 = loo_pad1(G1);
    c->T2 = loo_pad2(G2);
    c->G1 = G1;
    c->G2 = G2;
    LooArgs& a = c->a;
    fill_loo_args(a, D, h1, G1, h2, G2, c->T1, c->T2);
    const LooPlan pl = loo_plan(ctx, D, c->T1, c->T2, D.N);
    a.rows = nullptr;
    a.n_rows = D.N;
    a.n_units = pl.n_units;
    a.units_per_tile = pl.upt;
    a.n_tiles = pl.n_tiles;
    a.big_g = pl.tiles.big_g;
    a.big_levels = pl.tiles.big_levels;
    a.big_s0 = pl.tiles.big_s0;
    a.win0 = 0;
    a.win1 = INT_MAX;
    a.ell_rows = nullptr;
    a.G1r = G1;
    a.G2r = G2;
    a.tile_base = 0;
    c->next_l = 0;
    c->next_m = 0;
    c->next_t = a.big_levels * a.big_g;
    c->gram = pl.gram;
    c->n_tiles = pl.n_tiles;
    c->cmax = pl.grid;
    c->part_bytes = pl.part_bytes;
    c->fb_bytes = pl.fb_bytes;
    c->bytes = pl.bytes();
    c->N = D.N;
    *out = c;
    return CDE_OK;
}

void loo_chunked_destroy(LooChunked* c) { delete c; }
size_t loo_chunked_scratch_bytes(const LooChunked* c) { return c->bytes; }

// The next launch of the sequence, about `pair_evals` evaluations: the levels of
// large tiles in order, each either whole (with the levels after it that still
// fit) or a window of units m at a time in all of its tiles (one CTA per tile,
// each adding its window to its slot in unit order), then the small tiles in
// index ranges.  *done is set by the launch that processes the last units.
int loo_chunked_next(LooChunked* c, void* scratch, double pair_evals, cudaStream_t st, int* done) {
    LooArgs a = c->a;
    a.part = static_cast<double*>(scratch);
    a.fb = reinterpret_cast<double*>(static_cast<char*>(scratch) + c->part_bytes);
    a.work = reinterpret_cast<int*>(static_cast<char*>(scratch) + c->part_bytes + c->fb_bytes);
    const double rows_per_unit = c->gram ? loo_gram_rows_per_unit(c->T1, c->T2) : 1024.0 / (c->T1 * c->T2);
    const double per_unit = rows_per_unit * (double)c->N * c->T1 * c->T2;
    const int G = a.big_g, L = a.big_levels;
    int t0, t1, grid;
    if (c->next_l < L) {
        const int s = a.big_s0 >> c->next_l;
        if (c->next_m == 0 && per_unit * s * G <= pair_evals) {
            // whole levels while they fit
            double budget = pair_evals;
            int l = c->next_l;
            while (l < L && per_unit * (a.big_s0 >> l) * G <= budget) budget -= per_unit * (a.big_s0 >> l) * G, ++l;
            t0 = c->next_l * G;
            t1 = l * G;
            c->next_l = l;
        } else {
            // a window of units in every tile of the level
            int w = (int)std::ceil(pair_evals / (per_unit * G));
            if (w < 1) w = 1;
            a.win0 = c->next_m;
            a.win1 = std::min(s, c->next_m + w);
            t0 = c->next_l * G;
            t1 = t0 + G;
            c->next_m = a.win1;
            if (c->next_m >= s) {
                ++c->next_l;
                c->next_m = 0;
            }
        }
        grid = std::min(t1 - t0, c->cmax);
    } else {
        // a range of small tiles, at least one per CTA of the full launch
        const double per_tile = per_unit * a.units_per_tile;
        double nt = std::ceil(pair_evals / per_tile);
        if (nt < c->cmax) nt = c->cmax;
        t0 = c->next_t;
        t1 = (int)std::min<double>(c->n_tiles, c->next_t + nt);
        grid = std::min(t1 - t0, c->cmax);
        c->next_t = t1;
    }
    *done = c->next_l >= L && c->next_t >= c->n_tiles;
    if (t1 <= t0) return CDE_OK;
    a.n_tiles = t1;   // tiles t0 .. t1-1: the queue starts at t0 and stops at t1
    k_set_int<<<1, 1, 0, st>>>(a.work, t0);
    CDE_CUDA(cudaGetLastError());
    return c->gram ? launch_loo_gram(c->T1, c->T2, a, grid, st) : launch_loo_tile_kernel(c->T1, c->T2, a, grid, st);
}

int loo_chunked_final(const LooChunked* c, const void* scratch, double* d_Lc, double* d_Le, cudaStream_t st) {
    const int GG = c->T1 * c->T2;
    k_loo_final<<<(GG * 32 + 255) / 256, 256, 0, st>>>(static_cast<const double*>(scratch), c->n_tiles, GG, c->T2,
                                                        c->G1, c->G2, c->G2, (double)c->N, d_Lc, d_Le);
    CDE_CUDA(cudaGetLastError());
    return CDE_OK;
}

}  // namespace cde

// The tile partition of n_units units (units_per_tile small-tile units, G CTAs),
// as every LOO launch forms it: the same host/device code the kernels run.
extern "C" int cde_loo_tile_partition(int64_t n_units, int units_per_tile, int ctas, int tile, int* n_tiles,
                                      int* unit_first, int* unit_stride, int* unit_count) {
    if (n_units < 1 || n_units >= (1LL << 31) || units_per_tile < 1 || ctas < 0)
        return cde::set_error(CDE_EINVAL, "cde_loo_tile_partition: bad arguments");
    const cde::LooTiles p = cde::loo_tiles((int)n_units, units_per_tile, ctas);
    if (n_tiles) *n_tiles = p.n_tiles;
    if (tile < 0) return CDE_OK;
    if (tile >= p.n_tiles) return cde::set_error(CDE_EINVAL, "cde_loo_tile_partition: no such tile");
    cde::LooArgs a{};
    a.n_units = (int)n_units;
    a.units_per_tile = units_per_tile;
    a.big_g = p.big_g;
    a.big_levels = p.big_levels;
    a.big_s0 = p.big_s0;
    int u0, st, len;
    cde::loo_tile_span(a, tile, u0, st, len);
    if (unit_first) *unit_first = u0;
    if (unit_stride) *unit_stride = st;
    if (unit_count) *unit_count = len;
    return CDE_OK;
}

