// Pieces of the leave-one-out grid kernel shared by the single-dataset launch
// (loo_grid.cu), the persistent batched launch (batch.cu) and the
// allocation-free launch (noalloc.cu): the argument block, coefficient access,
// the exact joint-shift fallback and the FP64 per-unit epilogue.  The tile
// body (tensor-core outer product) is in loo_mma.cuh; loo_grid.cu describes
// the method.
#pragma once

#include <cstdint>

#include "cde_internal.h"

namespace cde {

struct LooArgs {
    const float* xs;        // [d][Np] structure-of-arrays x (standardised if asked)
    const float* y;         // [Np]
    const float* mx;        // [N] nearest squared x distance per row
    const float* my;        // [N] nearest squared y distance per row
    const int64_t* rows;    // optional list of rows (null: rows 0..n_rows-1)
    double* part;           // [n_tiles][2][T1*T2] FP64 tile partials (L_cond, sum ln A)
    double* ell_rows;       // optional per-row ell output
    int64_t ell_ld_row;     // row stride of ell_rows (doubles)
    int ell_ld_k;           // k stride of ell_rows
    int G1r, G2r;           // real (unpadded) sizes of this grid block
    int64_t N, Np, n_rows;
    int d;
    int n_units, units_per_tile, n_tiles;
    int tile_base;          // batched launch: first global tile of this item
    int* work;              // batched launch: queue counter
    int kern;               // CDE_KERNEL_GAUSS or CDE_KERNEL_EPAN
    float thresh;           // cells with shifted numerator below this are recomputed
    // per-bandwidth coefficients, padded by repeating the last bandwidth:
    //   Gaussian:     a = log2(e)/(2 h^2), lam1 = d ln(sqrt(2 pi) h1), kap2 = ln(sqrt(2 pi) h2)
    //   Epanechnikov: a = 1/h^2,           lam1 = d ln h1 - ln c_d,     kap2 = ln h2 - ln c_1
    float a1[32], a2[32];
    double lam1[32];
    double kap2[32];
};

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a * b + c clamped to [0, 1] in the same instruction (NaN -> 0)
__device__ __forceinline__ float fma_sat(float a, float b, float c) {
    float r;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Kernel factors of two values that share nothing but the family.
//   Gaussian (KERN 0):     t = shifted negative squared distance, factor 2^{c t}
//   Epanechnikov (KERN 1): t = squared distance, factor (1 - c t)_+ (c = 1/h^2;
//                          t = +inf gives exactly 0)
template <int KERN>
__device__ __forceinline__ float2 kernel_factor2(float2 c, float2 t) {
    if constexpr (KERN == 0) {
        const float2 a = __fmul2_rn(c, t);
        return make_float2(ex2_approx(a.x), ex2_approx(a.y));
    } else {
        return make_float2(fma_sat(-c.x, t.x, 1.f), fma_sat(-c.y, t.y, 1.f));
    }
}

// log2 of a positive normal float, returned in FP64: exact exponent plus the
// FP32 log2 of the mantissa in [1, 2) (absolute error below 1e-7).
__device__ __forceinline__ double log2_wide(float v) {
    int e;
    const float m = frexpf(v, &e);
    return (double)(e - 1) + (double)log2f(2.0f * m);
}

// Fixed-order reduction of one grid cell over tile partials (one warp):
// lane t sums tiles t, t+32, ... in order, then a fixed xor tree.
__device__ __forceinline__ void loo_final_cell(const double* __restrict__ part, int n_tiles, int GG,
                                               int cell, int lane, double& sc, double& se) {
    sc = 0.0;
    se = 0.0;
    for (int t = lane; t < n_tiles; t += 32) {
        sc += part[(int64_t)t * 2 * GG + cell];
        se += part[(int64_t)t * 2 * GG + GG + cell];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        se += __shfl_xor_sync(0xffffffffu, se, o);
    }
}

// Coefficient access from shared memory (batched launch: one item at a time).
struct CoefSmem {
    const float* a1s;
    const float* a2s;
    __device__ __forceinline__ float a1(int k) const { return a1s[k]; }
    __device__ __forceinline__ float a2(int l) const { return a2s[l]; }
};

// Coefficient access straight from the kernel's parameter block.
struct CoefParam {
    const LooArgs& a;
    __device__ __forceinline__ float a1(int k) const { return a.a1[k]; }
    __device__ __forceinline__ float a2(int l) const { return a.a2[l]; }
};

// Exact joint-shift recomputation of the flagged cells of one unit (whole
// CTA).  For a cell (row j, k, l) with e_i = a1_k (dx2_i - m_x,j) + a2_l (dy2_i - m_y,j):
// pass 1 finds i* = argmin e_i, pass 2 sums 2^{-(a1_k (dx2_i - dx2_*) + a2_l (dy2_i - dy2_*))},
// so the dominant term is exactly 1 and log2 At = -e_* + log2 S.  Cells are
// sorted, grouped by row and processed FB at a time, each pass visiting every
// point once for the whole group.
template <class C, class Coef>
__device__ __forceinline__ void loo_fallback(const LooArgs& a, const Coef& cf, float* sm, int nfl) {
    constexpr int GG = C::GG, FB = C::FB, G2 = C::G2v;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = a.d;
    const int64_t N = a.N, Np = a.Np;
    float* xj_s = sm + C::off_xj(d);
    float* yj_s = sm + C::off_yj(d);
    float* mx_s = sm + C::off_mx(d);
    float* my_s = sm + C::off_my(d);
    const long long* ji_s = reinterpret_cast<const long long*>(sm + C::off_ji(d));
    int* flag_s = reinterpret_cast<int*>(sm + C::off_flag(d));
    float* redf = sm + C::off_red(d);
    int* redi = reinterpret_cast<int*>(sm + C::off_red(d) + C::kWarps * FB);
    int* fbi = reinterpret_cast<int*>(sm + C::off_fb(d));
    double* la2 = reinterpret_cast<double*>(sm);

    // sort the (distinct) flagged cell ids in place: each thread ranks its entries
    int mine[4], rank[4];
    int nm = 0;
    for (int q = tid; q < nfl; q += C::kThreads) {
        const int v = flag_s[q];
        int r = 0;
        for (int t = 0; t < nfl; ++t) r += flag_s[t] < v;
        mine[nm] = v;
        rank[nm] = r;
        ++nm;
    }
    __syncthreads();
    for (int m = 0; m < nm; ++m) flag_s[rank[m]] = mine[m];
    __syncthreads();

    int q0 = 0;
    while (q0 < nfl) {
        // group: up to FB consecutive cells of the same row
        const int jl = flag_s[q0] / GG;
        int nb = 0;
        while (nb < FB && q0 + nb < nfl && flag_s[q0 + nb] / GG == jl) ++nb;
        float A[FB], B[FB];
#pragma unroll
        for (int f = 0; f < FB; ++f) {
            const int c = flag_s[q0 + (f < nb ? f : 0)];
            const int kl = c - jl * GG, k = kl / G2, l = kl - k * G2;
            A[f] = cf.a1(k);
            B[f] = cf.a2(l);
        }
        const float mxj = mx_s[jl], myj = my_s[jl], yj = yj_s[jl];
        const long long j = ji_s[jl];
        const float* xjr = xj_s + jl * d;
        // pass 1: argmin over i of e_i for each cell
        float best[FB];
        int bi[FB];
#pragma unroll
        for (int f = 0; f < FB; ++f) {
            best[f] = INFINITY;
            bi[f] = 0x7fffffff;
        }
        for (int64_t i = tid; i < N; i += C::kThreads) {
            if (i == j) continue;
            float dx2 = 0.f;
            for (int cc = 0; cc < d; ++cc) {
                const float t = xjr[cc] - a.xs[(int64_t)cc * Np + i];
                dx2 = fmaf(t, t, dx2);
            }
            const float dy = yj - a.y[i];
            const float ex = dx2 - mxj, ey = dy * dy - myj;
#pragma unroll
            for (int f = 0; f < FB; ++f) {
                const float e = A[f] * ex + B[f] * ey;
                if (e < best[f]) {   // i increases: first minimum kept
                    best[f] = e;
                    bi[f] = (int)i;
                }
            }
        }
#pragma unroll
        for (int f = 0; f < FB; ++f) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best[f], o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi[f], o);
                if (ob < best[f] || (ob == best[f] && oi < bi[f])) {
                    best[f] = ob;
                    bi[f] = oi;
                }
            }
            if (lane == 0) {
                redf[warp * FB + f] = best[f];
                redi[warp * FB + f] = bi[f];
            }
        }
        __syncthreads();
        if (tid < FB) {
            float b = redf[tid];
            int ix = redi[tid];
            for (int w = 1; w < C::kWarps; ++w) {
                const float ob = redf[w * FB + tid];
                const int oi = redi[w * FB + tid];
                if (ob < b || (ob == b && oi < ix)) {
                    b = ob;
                    ix = oi;
                }
            }
            if (ix < 0 || (int64_t)ix >= N) ix = (j == 0) ? 1 : 0;  // every e infinite
            fbi[tid] = ix;
        }
        __syncthreads();
        float dxs[FB], dys[FB];
#pragma unroll
        for (int f = 0; f < FB; ++f) {
            const int is = (int)CDE_CK(fbi[f], N, 108);
            float t2 = 0.f;
            for (int cc = 0; cc < d; ++cc) {
                const float t = xjr[cc] - a.xs[(int64_t)cc * Np + is];
                t2 = fmaf(t, t, t2);
            }
            dxs[f] = t2;
            const float t = yj - a.y[is];
            dys[f] = t * t;
        }
        // pass 2: shifted sums
        float S[FB];
#pragma unroll
        for (int f = 0; f < FB; ++f) S[f] = 0.f;
        for (int64_t i = tid; i < N; i += C::kThreads) {
            if (i == j) continue;
            float dx2 = 0.f;
            for (int cc = 0; cc < d; ++cc) {
                const float t = xjr[cc] - a.xs[(int64_t)cc * Np + i];
                dx2 = fmaf(t, t, dx2);
            }
            const float dy = yj - a.y[i];
            const float dy2 = dy * dy;
#pragma unroll
            for (int f = 0; f < FB; ++f)
                S[f] += ex2_approx(-(A[f] * (dx2 - dxs[f]) + B[f] * (dy2 - dys[f])));
        }
        __syncthreads();
#pragma unroll
        for (int f = 0; f < FB; ++f) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S[f] += __shfl_xor_sync(0xffffffffu, S[f], o);
            if (lane == 0) redf[warp * FB + f] = S[f];
        }
        __syncthreads();
#pragma unroll
        for (int f = 0; f < FB; ++f)
            if (tid == f && f < nb) {
                float tot = 0.f;
                for (int w = 0; w < C::kWarps; ++w) tot += redf[w * FB + f];
                const double es = (double)A[f] * ((double)dxs[f] - (double)mxj) +
                                  (double)B[f] * ((double)dys[f] - (double)myj);
                la2[flag_s[q0 + f]] = -es + log2_wide(tot);
            }
        __syncthreads();
        q0 += nb;
    }
}

// Per-unit epilogue shared by the tile bodies.  On entry At[m] holds the
// warp-combined shifted numerator of cell tid + 256 m and btl_s the FP64 log2
// of the shifted denominators; `big` (the first BIG floats of shared memory)
// is free.  Flags cells below the threshold, recomputes them exactly, and adds
// the FP64 log-ratios of the unit's rows into the tile partial (thread-owned
// cells, rows in order).
template <class C, int KERN, class Coef>
__device__ __forceinline__ void loo_unit_epilogue(const LooArgs& a, const Coef& cf, float* sm, int u,
                                                  int u_begin, int tile, const float (&At)[4]) {
    constexpr int JW = C::JW, GG = C::GG, G1 = C::G1v, G2 = C::G2v;
    constexpr double LN2 = 0.69314718055994530942;
    const int tid = threadIdx.x;
    const int d = a.d;
    float* big = sm;
    float* mx_s = sm + C::off_mx(d);
    float* my_s = sm + C::off_my(d);
    int* vr_s = reinterpret_cast<int*>(sm + C::off_vr(d));
    double* btl_s = reinterpret_cast<double*>(sm + C::off_btl(d));
    int* flag_s = reinterpret_cast<int*>(sm + C::off_flag(d));
    int* nflag_s = reinterpret_cast<int*>(sm + C::off_nflag(d));
        // ---- shifted log numerators; flag cells that lost range ----
        double* la2 = reinterpret_cast<double*>(big);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int c = tid + 256 * m;
            const int jl = c / GG;
            if (!vr_s[jl]) continue;
            const float v = At[m];
            if (v >= a.thresh) {
                la2[c] = log2_wide(v);
            } else {
                const int q = atomicAdd(nflag_s, 1);
                flag_s[q] = c;
            }
        }
        __syncthreads();
        if constexpr (KERN == 0) {
            // (Epanechnikov sums need no shift: their threshold is 0, nothing is flagged)
            const int nfl = *nflag_s;
            if (nfl > 0) loo_fallback<C>(a, cf, sm, nfl);
        }
        __syncthreads();

        // ---- FP64 log-ratio; each thread owns whole grid cells (all rows of
        //      the unit, in row order) and adds them to the tile partial ----
        {
            const bool first = (u == u_begin);
            double* part = a.part + CDE_CK(tile, a.n_tiles, 106) * 2 * GG;
            constexpr int NOWN = GG >= 256 ? GG / 256 : 1;
#pragma unroll
            for (int s = 0; s < NOWN; ++s) {
                const int kl = tid + 256 * s;
                if (kl >= GG) continue;
                const int k = kl / G2, l = kl - k * G2;
                const double a1k = (double)cf.a1(k), a2l = (double)cf.a2(l);
                const double lam = a.lam1[k], kap = a.kap2[l];
                double sc = 0.0, se = 0.0;
                for (int jl = 0; jl < JW; ++jl) {
                    if (!vr_s[jl]) continue;
                    const int c = jl * GG + kl;
                    const double shy = a2l * (double)my_s[jl];
                    const double lA = la2[c];
                    // a zero numerator (Epanechnikov: empty support, also when
                    // the denominator is zero) is ell = -inf, never NaN
                    const double ell = lA == -INFINITY ? -INFINITY : LN2 * (lA - btl_s[jl * G1 + k] - shy) - kap;
                    const double lnA = LN2 * (lA - a1k * (double)mx_s[jl] - shy) - lam - kap;
                    sc += ell;
                    se += lnA;
                    if (a.ell_rows && k < a.G1r && l < a.G2r) {
                        const int64_t r = CDE_CK((int64_t)u * JW + jl, a.n_rows, 107);
                        a.ell_rows[r * a.ell_ld_row + (int64_t)k * a.ell_ld_k + l] = ell;
                    }
                }
                if (first) {
                    part[kl] = sc;
                    part[GG + kl] = se;
                } else {
                    part[kl] += sc;
                    part[GG + kl] += se;
                }
            }
        }
}

// Grid shapes of the tile kernels: k (h1) padded to an M-tile multiple of 16,
// l (h2) to 8, 16 or 32.
inline int loo_pad1(int g) { return g <= 16 ? 16 : 32; }
inline int loo_pad2(int g) { return g <= 8 ? 8 : (g <= 16 ? 16 : 32); }

int launch_loo_tile_kernel(int T1, int T2, const LooArgs& a, int grid, cudaStream_t st);
void fill_loo_args(LooArgs& a, const Dataset& D, const double* h1, int g1, const double* h2,
                   int g2, int T1, int T2);
// units per tile of a grid block shape over n_rows rows (the tuned value when set; n_rows = 0:
// the per-shape default without the small-grid reduction)
int loo_units_per_tile(cde_ctx* ctx, int T1, int T2, int64_t n_rows);
int loo_grid_ctas(cde_ctx* ctx, int T1, int T2);

}  // namespace cde
