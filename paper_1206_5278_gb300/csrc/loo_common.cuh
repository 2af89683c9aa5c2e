// Pieces of the leave-one-out grid kernel shared by the single-dataset launch
// (loo_grid.cu), the persistent batched launch (batch.cu) and the
// allocation-free launch (noalloc.cu): the argument block, coefficient access,
// the exact joint-shift fallback and the FP64 per-unit epilogue.  The tile
// body (tensor-core outer product) is in loo_mma.cuh; loo_grid.cu describes
// the method.
#pragma once

#include <climits>
#include <cstdint>

#include "cde_internal.h"

namespace cde {

struct LooArgs {
    const float* xs;        // [d][Np] structure-of-arrays x (standardised if asked)
    const float* y;         // [Np]
    const float* mx;        // [N] nearest squared x distance per row
    const float* my;        // [N] nearest squared y distance per row
    const float* qx;        // [N] dx^2 of each row's y-nearest point (fallback bounds)
    const float* qy;        // [N] dy^2 of each row's x-nearest point
    const int64_t* rows;    // optional list of rows (null: rows 0..n_rows-1)
    double* part;           // [n_tiles][2][T1*T2] FP64 tile partials (L_cond, sum ln A)
    double* fb;             // d >= 16 kernel: [grid][16384] per-CTA recomputed log2 At
    double* ell_rows;       // optional per-row ell output
    int64_t ell_ld_row;     // row stride of ell_rows (doubles)
    int ell_ld_k;           // k stride of ell_rows
    int G1r, G2r;           // real (unpadded) sizes of this grid block
    int64_t N, Np, n_rows;
    int d;
    int n_units, units_per_tile, n_tiles;
    // tile partition (LooTiles): big_levels levels of big_g tiles each, the tiles of
    // level l holding big_s0 >> l units; the rest hold units_per_tile consecutive
    // units.  big_levels = 0: all tiles are small.
    int big_g, big_levels, big_s0;
    int win0, win1;         // units m of each tile processed by this launch: [win0, win1)
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

// Tile partition of a launch's units.  One partial slot per tile; a tile's units
// are added to its slot in order, and the slots are reduced in a fixed order, so
// the result depends on the partition only, not on which CTA runs which tile or
// in which launch.  With enough work the tiles shrink as the launch proceeds
// (guided self-scheduling): level l holds G tiles (one per resident CTA) of
// s0 >> l units, s0 = n_units / 2G, interleaved with stride G inside the level's
// range so that every tile samples the whole dataset; levels stop before the
// size falls under 2 units_per_tile, and small tiles of units_per_tile
// consecutive units take the rest.  The atomic queue hands tiles out in index
// order, so the launch ends on small tiles as with uniform ones, with
// G log2(n_units / G) + 2G slots instead of one per small tile.
struct LooTiles {
    int big_g, big_levels, big_s0, n_tiles;
};

__host__ __device__ inline LooTiles loo_tiles(int n_units, int upt, int G) {
    LooTiles p{0, 0, 0, 0};
    if (G > 0 && (int64_t)n_units >= 8LL * G * upt) {
        p.big_g = G;
        p.big_s0 = n_units / (2 * G);
        while (p.big_levels < 16 && (p.big_s0 >> p.big_levels) >= 2 * upt) ++p.big_levels;
        int64_t covered = 0;
        for (int l = 0; l < p.big_levels; ++l) covered += p.big_s0 >> l;
        const int rest = n_units - (int)(covered * G);
        p.n_tiles = p.big_levels * G + (rest + upt - 1) / upt;
    } else {
        p.n_tiles = (n_units + upt - 1) / upt;
    }
    return p;
}

// first unit of level l (the units of levels 0 .. l-1 come before it)
__host__ __device__ __forceinline__ int loo_level_base(const LooArgs& a, int l) {
    int s = 0;
    for (int i = 0; i < l; ++i) s += a.big_s0 >> i;
    return s * a.big_g;
}

// tile t's units: u0 + m stride for m < len
__host__ __device__ __forceinline__ void loo_tile_span(const LooArgs& a, int t, int& u0, int& stride, int& len) {
    const int nb = a.big_levels * a.big_g;
    if (t < nb) {
        const int l = t / a.big_g;
        u0 = loo_level_base(a, l) + (t - l * a.big_g);
        stride = a.big_g;
        len = a.big_s0 >> l;
    } else {
        u0 = loo_level_base(a, a.big_levels) + (t - nb) * a.units_per_tile;
        stride = 1;
        len = a.units_per_tile < a.n_units - u0 ? a.units_per_tile : a.n_units - u0;
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

// log2(1 + 5.12e-8): ex2.approx.ftz.f32 is low by 5.12e-8 relative on average
// (measured on sm_103a); the fallback's terms carry it in their exponent, as
// the tile body's factors do
constexpr float kFbEx2Fix = 7.39e-8f;

// Exact joint-shift recomputation of the flagged cells of one unit (whole
// CTA).  For a cell (row j, k, l) let X_i = dx2_i - m_x,j, Y_i = dy2_i - m_y,j and
// e_i = a1_k X_i + a2_l Y_i.  Then At = sum_i 2^{-e_i} = 2^{-e_*} S with
// S = sum_i 2^{-(a1_k (dx2_i - dx2_*) + a2_l (dy2_i - dy2_*))} for the minimiser
// i* (its term is exactly 1), and log2 At = -e_* + log2 S.  All flagged cells
// of the unit are processed together in two passes over the points:
//  1. the minimiser of every cell.  It is no worse than the x-nearest point
//     (X = 0, Y = Yh) and the y-nearest point (X = Xh, Y = 0), so
//     e_* <= min(a2 Yh, a1 Xh): only points with dx2 <= qx and dy2 <= qy
//     (qx, qy: the dataset's stored other-coordinate distances of the two
//     neighbours), and inside the union over the row's cells of those
//     triangles, are candidates.  A cell keeps the smallest key (e bits, i):
//     the smallest e, ties to the smallest index, whatever the order of visits.
//  2. the sums.  A point with e_i > e_* + T adds less than 2^-T; with
//     T = 32 + ceil(log2 N) all of them together add less than 2^-32 of S.
//     So only points with X <= max_f (e_*f + T)/a1_f and Y <= max_f (e_*f + T)/a2_f
//     (the row's box) are candidates.
// Each warp takes chunks of 32 consecutive points (lane = point: distances to
// every flagged row, candidate tests) and compacts a row's candidates into a
// shared list; then lane = cell: each lane runs its cells over the list.
// Pass 1 folds the list into the lane's (e, i) minimum and merges it with a
// 64-bit shared atomicMin; pass 2 sums the list's terms in FP32 (list order)
// and adds the chunk sum as an integer in units of 2^-(62 - ceil(log2 N))
// (64-bit shared atomicAdd: exact, so the cell's sum is the same whatever the
// order in which warps finish, and it cannot overflow).  Both passes compute
// dx2 and dy2 with the tile body's FP32 formula.
template <class C, class Coef>
__device__ __forceinline__ void loo_fallback(const LooArgs& a, const Coef& cf, float* sm, int nfl) {
    constexpr int GG = C::GG, G2 = C::G2v, JW = C::JW, NT = C::kThreads, NW = C::kWarps;
    constexpr int LG2 = G2 == 8 ? 3 : (G2 == 16 ? 4 : 5);
    constexpr int JG = JW * GG;
    static_assert(8 * JG <= C::COMB, "fallback scratch must fit in the combine buffer");
    static_assert(JW <= 8, "per-row fallback parameters hold 8 rows");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = a.d;
    const int64_t N = a.N, Np = a.Np;
    const float* xj_s = sm + C::off_xj(d);
    const float* yj_s = sm + C::off_yj(d);
    const float* mx_s = sm + C::off_mx(d);
    const float* my_s = sm + C::off_my(d);
    const long long* ji_s = reinterpret_cast<const long long*>(sm + C::off_ji(d));
    int* flag_s = reinterpret_cast<int*>(sm + C::off_flag(d));
    double* la2 = reinterpret_cast<double*>(sm);
    // per flagged cell f (after la2): the pass-1 key, reused for the pass-2 sum;
    // the minimiser's distances; the cell's coefficients
    unsigned long long* best = reinterpret_cast<unsigned long long*>(sm + 2 * JG);
    unsigned long long* acc = best;
    float* dxs = sm + 4 * JG;
    float* dys = sm + 5 * JG;
    float* As = sm + 6 * JG;
    float* Bs = sm + 7 * JG;
    // per warp: the candidate list of one (chunk, row); per row: bounds and cell range
    float* fbw = sm + C::off_fbw(d);
    float* lx = fbw + warp * 96;
    float* ly = lx + 32;
    int* li = reinterpret_cast<int*>(ly + 32);
    float* rqx = fbw + NW * 96;
    float* rqy = rqx + 8;
    int* rlo_b = reinterpret_cast<int*>(rqy + 8);   // float bits of positive values (0: none)
    int* rhi_b = rlo_b + 8;
    int* rx_b = rhi_b + 8;
    int* ry_b = rx_b + 8;
    int* rs = ry_b + 8;                              // cells [rs, re) of the row in flag_s
    int* re = rs + 8;

    // sort the (distinct) flagged cell ids in place: each thread ranks its entries
    int mine[4], rank[4];
    int nm = 0;
    for (int q = tid; q < nfl; q += NT) {
        const int v = flag_s[q];
        int r = 0;
        for (int t = 0; t < nfl; ++t) r += flag_s[t] < v;
        mine[nm] = v;
        rank[nm] = r;
        ++nm;
    }
    if (tid < JW) {
        rs[tid] = re[tid] = 0;
        rlo_b[tid] = 0;
        rhi_b[tid] = __float_as_int(INFINITY);
        rx_b[tid] = ry_b[tid] = 0;
        const long long j = ji_s[tid];
        rqx[tid] = a.qx[j];
        rqy[tid] = a.qy[j];
    }
    __syncthreads();
    for (int m = 0; m < nm; ++m) flag_s[rank[m]] = mine[m];
    __syncthreads();

    int lg = 0;
    while (((int64_t)1 << lg) < N) ++lg;
    const float T = (float)(32 + lg);
    const int SC = 62 - lg;            // fixed-point scale of the sums
    const float scale = ldexpf(1.f, SC), inv_scale_f = ldexpf(1.f, -SC);

    // cells: coefficients, row ranges, and the triangles of the argmin region --
    // cells with rho = a2/a1 <= Xh/Yh are bounded by the x-nearest point
    // (X + rho Y <= rho Yh; the largest rho covers the others), the rest by the
    // y-nearest point (X + rho Y <= Xh; the smallest rho)
    for (int f = tid; f < nfl; f += NT) {
        const int c = flag_s[f], r = c / GG, kl = c - r * GG, k = kl >> LG2, l = kl & (G2 - 1);
        const float A = cf.a1(k), B = cf.a2(l);
        As[f] = A;
        Bs[f] = B;
        best[f] = ~0ull;
        if (f == 0 || flag_s[f - 1] / GG != r) rs[r] = f;
        if (f == nfl - 1 || flag_s[f + 1] / GG != r) re[r] = f + 1;
        const float Xh = rqx[r] - mx_s[r], Yh = rqy[r] - my_s[r];
        const float rho = B / A;
        if (rho * Yh <= Xh) atomicMax(rlo_b + r, __float_as_int(rho));
        else atomicMin(rhi_b + r, __float_as_int(rho));
    }
    __syncthreads();

    // squared distances of a chunk's point (lane) to row r, the tile body's formula
    const auto dist = [&](int r, const float (&xi)[8], int64_t i, float yi, float& dx2, float& dy2) {
        const float* xjr = xj_s + r * d;
        float s = 0.f;
#pragma unroll
        for (int cc = 0; cc < 8; ++cc)
            if (cc < d) {
                const float t = xjr[cc] - xi[cc];
                s = fmaf(t, t, s);
            }
        for (int cc = 8; cc < d; ++cc) {
            const float t = xjr[cc] - a.xs[(int64_t)cc * Np + i];
            s = fmaf(t, t, s);
        }
        dx2 = s;
        const float dy = yj_s[r] - yi;
        dy2 = dy * dy;
    };

    // ---- pass 1: the minimiser of every flagged cell ----
    for (int64_t base = (int64_t)warp * 32; base < N; base += NW * 32) {
        const int64_t i = base + lane;
        const bool v = i < N;
        const int64_t ic = v ? i : base;
        float xi[8];
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) xi[cc] = cc < d ? a.xs[(int64_t)cc * Np + CDE_CK(ic, N, 108)] : 0.f;
        const float yi = a.y[ic];
        for (int r = 0; r < JW; ++r) {
            const int f0 = rs[r], f1 = re[r];
            if (f0 == f1) continue;
            float dx2, dy2;
            dist(r, xi, ic, yi, dx2, dy2);
            const float mxr = mx_s[r], myr = my_s[r];
            const float X = dx2 - mxr, Y = dy2 - myr;
            const float Xh = rqx[r] - mxr, Yh = rqy[r] - myr;
            const float rlo = __int_as_float(rlo_b[r]), rhi = __int_as_float(rhi_b[r]);
            const bool in = v && i != ji_s[r] && dx2 <= rqx[r] && dy2 <= rqy[r] &&
                            ((rlo > 0.f && fmaf(rlo, Y, X) <= rlo * Yh) || (rhi < INFINITY && fmaf(rhi, Y, X) <= Xh));
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (m == 0u) continue;
            if (in) {
                const int p = __popc(m & ((1u << lane) - 1u));
                lx[p] = X;
                ly[p] = Y;
                li[p] = (int)i;
            }
            __syncwarp();
            const int nc = __popc(m);
            for (int f = f0 + lane; f < f1; f += 32) {
                const float A = As[f], B = Bs[f];
                float emin = INFINITY;
                int imin = 0;
                for (int q = 0; q < nc; ++q) {
                    const float e = fmaxf(fmaf(A, lx[q], B * ly[q]), 0.f);
                    if (e < emin) {
                        emin = e;
                        imin = li[q];
                    }
                }
                const unsigned long long key = ((unsigned long long)__float_as_uint(emin) << 32) | (unsigned int)imin;
                if (key < best[f]) atomicMin(best + f, key);
            }
            __syncwarp();
        }
    }
    __syncthreads();

    // ---- the minimisers' distances; the rows' boxes of pass 2 ----
    for (int f = tid; f < nfl; f += NT) {
        const int r = flag_s[f] / GG;
        const long long j = ji_s[r];
        const unsigned long long b = best[f];
        // no point in the region (cannot happen: the two neighbours are in it):
        // anchor at the x-nearest bound
        const bool none = b == ~0ull;
        const int64_t is = none ? (j == 0 ? 1 : 0) : (int64_t)(unsigned int)b;
        const float* xjr = xj_s + r * d;
        float t2 = 0.f;
        for (int cc = 0; cc < d; ++cc) {
            const float t = xjr[cc] - a.xs[(int64_t)cc * Np + CDE_CK(is, N, 108)];
            t2 = fmaf(t, t, t2);
        }
        const float t = yj_s[r] - a.y[is];
        dxs[f] = t2;
        dys[f] = t * t;
        const float A = As[f], B = Bs[f];
        const float es = fmaxf(fmaf(A, t2 - mx_s[r], B * (t * t - my_s[r])), 0.f);
        atomicMax(rx_b + r, __float_as_int((es + T) / A));
        atomicMax(ry_b + r, __float_as_int((es + T) / B));
        acc[f] = 0ull;   // the key of this cell has been read
    }
    __syncthreads();

    // ---- pass 2: the shifted sums over the points that can matter ----
    for (int64_t base = (int64_t)warp * 32; base < N; base += NW * 32) {
        const int64_t i = base + lane;
        const bool v = i < N;
        const int64_t ic = v ? i : base;
        float xi[8];
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) xi[cc] = cc < d ? a.xs[(int64_t)cc * Np + CDE_CK(ic, N, 108)] : 0.f;
        const float yi = a.y[ic];
        for (int r = 0; r < JW; ++r) {
            const int f0 = rs[r], f1 = re[r];
            if (f0 == f1) continue;
            float dx2, dy2;
            dist(r, xi, ic, yi, dx2, dy2);
            const float RXd = mx_s[r] + __int_as_float(rx_b[r]), RYd = my_s[r] + __int_as_float(ry_b[r]);
            const bool in = v && i != ji_s[r] && dx2 <= RXd && dy2 <= RYd;
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (m == 0u) continue;
            if (in) {
                const int p = __popc(m & ((1u << lane) - 1u));
                lx[p] = dx2;
                ly[p] = dy2;
            }
            __syncwarp();
            const int nc = __popc(m);
            for (int f = f0 + lane; f < f1; f += 32) {
                const float A = As[f], B = Bs[f], dxf = dxs[f], dyf = dys[f];
                float s = 0.f;
                for (int q = 0; q < nc; ++q)
                    s += ex2_approx(kFbEx2Fix - (A * (lx[q] - dxf) + B * (ly[q] - dyf)));
                const unsigned long long qv = __float2ull_rn(s * scale);
                if (qv) atomicAdd(acc + f, qv);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int f = tid; f < nfl; f += NT) {
        const int c = flag_s[f], r = c / GG;
        const float tot = (float)((double)acc[f] * (double)inv_scale_f);
        const double es = (double)As[f] * ((double)dxs[f] - (double)mx_s[r]) +
                          (double)Bs[f] * ((double)dys[f] - (double)my_s[r]);
        la2[c] = -es + log2_wide(tot);
    }
    __syncthreads();
}

// Per-unit epilogue shared by the tile bodies.  On entry At[m] holds the
// warp-combined shifted numerator of cell tid + 256 m and btl_s the FP64 log2
// of the shifted denominators; `big` (the first BIG floats of shared memory)
// is free.  Flags cells below the threshold, recomputes them exactly, and adds
// the FP64 log-ratios of the unit's rows into the tile partial (thread-owned
// cells, rows in order; `first`: the tile's first unit, which stores instead).
template <class C, int KERN, class Coef>
__device__ __forceinline__ void loo_unit_epilogue(const LooArgs& a, const Coef& cf, float* sm, int u,
                                                  bool first, int tile, const float (&At)[4]) {
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
            // cells of the padded grid (the last bandwidth repeated) are never
            // output: they are not recomputed either
            const int kl = c - jl * GG;
            const bool padded = kl / G2 >= a.G1r || kl % G2 >= a.G2r;
            if (v >= a.thresh || padded) {
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
// d_x >= 16: the kernel with the x cross-term on the tensor cores (loo_gram.cu)
constexpr int kGramMinD = 16;
int launch_loo_gram(int T1, int T2, const LooArgs& a, int grid, cudaStream_t st);
int loo_gram_rows_per_unit(int T1, int T2);
size_t loo_gram_fb_bytes_per_cta();
size_t loo_gram_smem_bytes(int T1, int T2, int d);
// whether a grid block of this shape over this dataset runs on the d >= 16 kernel
bool loo_use_gram(const Dataset& D, int T1, int T2);
void fill_loo_args(LooArgs& a, const Dataset& D, const double* h1, int g1, const double* h2,
                   int g2, int T1, int T2);
// units per tile of a grid block shape over n_rows rows (the tuned value when set; n_rows = 0:
// the per-shape default without the small-grid reduction)
int loo_units_per_tile(cde_ctx* ctx, int T1, int T2, int64_t n_rows);
// the autotuner's candidate for a shape class, used by this thread's launches only
void tuning_candidate(int T1, int T2, int units_per_tile, int ctas_per_sm);
void tuning_candidate_clear();

// (the launch plan behind the opaque LooChunked of cde_internal.h)
struct LooChunked {
    LooArgs a;
    int T1, T2, G1, G2;
    bool gram;
    int n_tiles, cmax;
    size_t part_bytes, fb_bytes, bytes;
    int64_t N;
    int next_l;     // levels < next_l are done
    int next_m;     // level next_l: units m < next_m of its tiles are done
    int next_t;     // small tiles: tiles < next_t are done
};
int loo_grid_ctas(cde_ctx* ctx, int T1, int T2);

}  // namespace cde
