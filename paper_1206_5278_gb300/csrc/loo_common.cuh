// The leave-one-out pair kernel, shared by the single-dataset launch
// (loo_grid.cu) and the persistent batched launch (batch.cu).
// See loo_grid.cu for the method; this file holds the tile body.
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
    float thresh;           // cells with shifted numerator below this are recomputed
    float a1[32], a2[32];   // log2(e)/(2 h^2), padded by repeating the last bandwidth
    double lam1[32];        // d ln(sqrt(2 pi) h1_k)
    double kap2[32];        // ln(sqrt(2 pi) h2_l)
};

template <int G1, int G2>
struct LooCfg {
    static constexpr int kThreads = 256, kWarps = 8;
    static constexpr int G1v = G1, G2v = G2;
    static constexpr int GG = G1 * G2;
    static constexpr int JW = 1024 / GG;               // rows per unit
    static constexpr int IC = (32 / JW) > 8 ? 32 / JW : 8;  // i per warp chunk
    static constexpr int PPL = IC * JW / 32;           // phase-1 pairs per lane
    static constexpr int NKQ = G1 / 4, NLQ = G2 / 8;   // phase-2 lane tile: 4 k x 8 l
    static constexpr int LPJ = NKQ * NLQ;              // lanes per row in phase 2
    static constexpr int UCH = JW * G1 / 4;            // 16-B chunks of a u row
    static constexpr int WCH = JW * G2 / 4;            // 16-B chunks of a w row
    static constexpr int UROW = UCH * 4 + 4;           // floats per u row (+16 B pad: no bank conflicts)
    static constexpr int WROW = WCH * 4 + 4;
    static constexpr int STAGE = IC * (UROW + WROW);   // floats per warp
    static constexpr int COMB = kWarps * 1024 + kWarps * 32 * 4;
    static constexpr int BIG0 = kWarps * STAGE > COMB ? kWarps * STAGE : COMB;
    static constexpr int BIG = BIG0 > 2048 ? BIG0 : 2048;  // also holds 1024 doubles
    static constexpr int NKL = GG >= 256 ? GG / 256 : 1;
    static_assert(LPJ * JW == 32, "lane tiling");
    static_assert(UCH >= 8 && WCH >= 8, "row chunks");
    static constexpr int FB = 8;                       // flagged cells per fallback pass

    __host__ __device__ static int dpad(int d) { return (d * JW + 3) & ~3; }
    // float offsets of the per-unit area
    __host__ __device__ static int off_xj() { return BIG; }
    __host__ __device__ static int off_xj(int) { return BIG; }
    __host__ __device__ static int off_yj(int d) { return BIG + dpad(d); }
    __host__ __device__ static int off_mx(int d) { return off_yj(d) + 16; }
    __host__ __device__ static int off_my(int d) { return off_yj(d) + 32; }
    __host__ __device__ static int off_ji(int d) { return off_yj(d) + 48; }    // 16 int64
    __host__ __device__ static int off_vr(int d) { return off_yj(d) + 80; }    // 16 int
    __host__ __device__ static int off_btl(int d) { return off_yj(d) + 96; }   // JW*G1 doubles
    __host__ __device__ static int off_flag(int d) { return off_btl(d) + 2 * JW * G1; }  // 1024 int
    __host__ __device__ static int off_nflag(int d) { return off_flag(d) + 1024; }
    __host__ __device__ static int off_red(int d) { return off_nflag(d) + 4; }   // 8 warps x FB x 2 words
    __host__ __device__ static int off_fb(int d) { return off_red(d) + 2 * kWarps * FB; }  // FB x 2 words
    static size_t smem_bytes(int d) { return (size_t)(off_fb(d) + 2 * FB + 8) * sizeof(float); }
};

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
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
            const int is = fbi[f];
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
template <class C, class Coef>
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
        const int nfl = *nflag_s;
        if (nfl > 0) loo_fallback<C>(a, cf, sm, nfl);
        __syncthreads();

        // ---- FP64 log-ratio; each thread owns whole grid cells (all rows of
        //      the unit, in row order) and adds them to the tile partial ----
        {
            const bool first = (u == u_begin);
            double* part = a.part + (int64_t)tile * 2 * GG;
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
                    const double ell = LN2 * (lA - btl_s[jl * G1 + k] - shy) - kap;
                    const double lnA = LN2 * (lA - a1k * (double)mx_s[jl] - shy) - lam - kap;
                    sc += ell;
                    se += lnA;
                    if (a.ell_rows && k < a.G1r && l < a.G2r) {
                        const int64_t r = (int64_t)u * JW + jl;
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

// One tile of units: units [tile*UPT, min(n_units, (tile+1)*UPT)).
template <int G1, int G2, class Coef>
__device__ __forceinline__ void loo_tile(const LooArgs& a, const Coef& cf, int tile, float* sm) {
    using C = LooCfg<G1, G2>;
    constexpr int JW = C::JW, IC = C::IC, PPL = C::PPL, NKQ = C::NKQ, NLQ = C::NLQ;
    constexpr int LPJ = C::LPJ, GG = C::GG, UROW = C::UROW, WROW = C::WROW;
    constexpr int WH = C::WCH / 2;
    constexpr double LN2 = 0.69314718055994530942;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = a.d;
    float* big = sm;
    float* xj_s = sm + C::off_xj();
    float* yj_s = sm + C::off_yj(d);
    float* mx_s = sm + C::off_mx(d);
    float* my_s = sm + C::off_my(d);
    long long* ji_s = reinterpret_cast<long long*>(sm + C::off_ji(d));
    int* vr_s = reinterpret_cast<int*>(sm + C::off_vr(d));
    double* btl_s = reinterpret_cast<double*>(sm + C::off_btl(d));
    int* flag_s = reinterpret_cast<int*>(sm + C::off_flag(d));
    int* nflag_s = reinterpret_cast<int*>(sm + C::off_nflag(d));
    const int u_begin = tile * a.units_per_tile;
    const int u_end = min(a.n_units, u_begin + a.units_per_tile);
    const int64_t N = a.N, Np = a.Np;
    const int64_t n_chunks = (N + IC - 1) / IC;

    // phase-2 lane tile
    const int jl2 = lane / LPJ, rr = lane % LPJ, kq2 = rr / NLQ, lq2 = rr % NLQ;
    float* ust = big + warp * C::STAGE;
    float* wst = ust + IC * UROW;
    const float* urd = ust + 4 * (jl2 * NKQ + kq2);
    const float* wrd = wst + 4 * (jl2 * NLQ + lq2);
    const int il = lane % IC;

    for (int u = u_begin; u < u_end; ++u) {
        // ---- unit set-up ----
        __syncthreads();
        if (tid < JW) {
            const int64_t r = (int64_t)u * JW + tid;
            const bool v = r < a.n_rows;
            const int64_t r0 = v ? r : 0;
            const int64_t j = a.rows ? a.rows[r0] : r0;
            ji_s[tid] = j;
            vr_s[tid] = v;
            yj_s[tid] = a.y[j];
            mx_s[tid] = a.mx[j];
            my_s[tid] = a.my[j];
        }
        if (tid == 0) *nflag_s = 0;
        __syncthreads();
        for (int e = tid; e < JW * d; e += C::kThreads) {
            const int jl = e / d, c = e - jl * d;
            xj_s[e] = a.xs[(int64_t)c * Np + ji_s[jl]];
        }
        __syncthreads();

        float2 acc[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] = make_float2(0.f, 0.f);
        // B partial sums: lane (jl2, kq2, lq2) owns k = 4 kq2 + lq2 * NBT + q, q < NBT
        constexpr int NBT = 4 / NLQ;
        float bt[NBT];
#pragma unroll
        for (int q = 0; q < NBT; ++q) bt[q] = 0.f;

        // per-pair row constants (fixed for the unit)
        float pmx[PPL], pmy[PPL], pyj[PPL];
        long long pj[PPL];
        int pjl[PPL];
#pragma unroll
        for (int r = 0; r < PPL; ++r) {
            const int jl = (lane + 32 * r) / IC;
            pjl[r] = jl;
            pmx[r] = mx_s[jl];
            pmy[r] = my_s[jl];
            pyj[r] = yj_s[jl];
            pj[r] = ji_s[jl];
        }

        float xin[8], yin = 0.f;
        int64_t ch = warp;
        if (ch < n_chunks) {
            const int64_t i = ch * IC + il;
#pragma unroll
            for (int c = 0; c < 8; ++c) xin[c] = c < d ? a.xs[(int64_t)c * Np + i] : 0.f;
            yin = a.y[i];
        }
        for (; ch < n_chunks; ch += C::kWarps) {
            const int64_t i = ch * IC + il;
            float xi[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) xi[c] = xin[c];
            const float yi = yin;
            // ---- phase 1: distances and exp2 factors for this lane's pairs ----
#pragma unroll
            for (int r = 0; r < PPL; ++r) {
                const int jl = pjl[r];
                const float* xjr = xj_s + jl * d;
                float dx2 = 0.f;
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < d) {
                        const float t = xjr[c] - xi[c];
                        dx2 = fmaf(t, t, dx2);
                    }
                for (int c = 8; c < d; ++c) {
                    const float t = xjr[c] - a.xs[(int64_t)c * Np + i];
                    dx2 = fmaf(t, t, dx2);
                }
                const float dy = pyj[r] - yi;
                const float dy2 = dy * dy;
                const bool ok = (i < N) && (i != pj[r]);
                const float t1 = ok ? pmx[r] - dx2 : -INFINITY;
                const float t2 = pmy[r] - dy2;
                float* ub = ust + il * UROW + 4 * jl * NKQ;
#pragma unroll
                for (int kq = 0; kq < NKQ; ++kq) {
                    const float u0 = ex2_approx(cf.a1(4 * kq + 0) * t1);
                    const float u1 = ex2_approx(cf.a1(4 * kq + 1) * t1);
                    const float u2 = ex2_approx(cf.a1(4 * kq + 2) * t1);
                    const float u3 = ex2_approx(cf.a1(4 * kq + 3) * t1);
                    *reinterpret_cast<float4*>(ub + 4 * kq) = make_float4(u0, u1, u2, u3);
                }
                float* wb = wst + il * WROW + 4 * jl * NLQ;
#pragma unroll
                for (int lq = 0; lq < NLQ; ++lq) {
                    float w[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) w[q] = ex2_approx(cf.a2(8 * lq + q) * t2);
                    *reinterpret_cast<float4*>(wb + 4 * lq) = make_float4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<float4*>(wb + 4 * (WH + lq)) =
                        make_float4(w[4], w[5], w[6], w[7]);
                }
            }
            // prefetch the next chunk's point
            if (ch + C::kWarps < n_chunks) {
                const int64_t i2 = (ch + C::kWarps) * IC + il;
#pragma unroll
                for (int c = 0; c < 8; ++c) xin[c] = c < d ? a.xs[(int64_t)c * Np + i2] : 0.f;
                yin = a.y[i2];
            }
            __syncwarp();
            // ---- phase 2: outer-product accumulation, 4 k x 8 l per lane ----
#pragma unroll
            for (int ii = 0; ii < IC; ++ii) {
                const float4 ua = *reinterpret_cast<const float4*>(urd + ii * UROW);
                const float4 wa = *reinterpret_cast<const float4*>(wrd + ii * WROW);
                const float4 wb = *reinterpret_cast<const float4*>(wrd + ii * WROW + 4 * WH);
                const float2 U[4] = {make_float2(ua.x, ua.x), make_float2(ua.y, ua.y),
                                     make_float2(ua.z, ua.z), make_float2(ua.w, ua.w)};
                const float2 W[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w),
                                     make_float2(wb.x, wb.y), make_float2(wb.z, wb.w)};
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[p][q] = __ffma2_rn(U[p], W[q], acc[p][q]);
                if constexpr (NLQ == 1) {
                    bt[0] += ua.x;
                    bt[1] += ua.y;
                    bt[2] += ua.z;
                    bt[3] += ua.w;
                } else if constexpr (NLQ == 2) {
                    bt[0] += lq2 ? ua.z : ua.x;
                    bt[1] += lq2 ? ua.w : ua.y;
                } else {
                    const float lo = (lq2 & 1) ? ua.y : ua.x;
                    const float hi = (lq2 & 1) ? ua.w : ua.z;
                    bt[0] += (lq2 & 2) ? hi : lo;
                }
            }
            __syncwarp();
        }

        // ---- combine the 8 warps' partial sums in fixed order ----
        __syncthreads();
        float* accS = big;
        float* bpS = big + C::kWarps * 1024;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                *reinterpret_cast<float2*>(accS + warp * 1024 + jl2 * GG + (4 * kq2 + p) * G2 +
                                           8 * lq2 + 2 * q) = acc[p][q];
#pragma unroll
        for (int q = 0; q < NBT; ++q) bpS[(warp * 32 + lane) * 4 + q] = bt[q];
        __syncthreads();
        float At[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int c = tid + 256 * m;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < C::kWarps; ++w) s += accS[w * 1024 + c];
            At[m] = s;
        }
        for (int e = tid; e < JW * G1; e += C::kThreads) {
            // owner lane of (jl, k): kq = k/4, lq = (k%4)/NBT, q = (k%4)%NBT
            const int jl = e / G1, k = e - jl * G1;
            const int kq = k >> 2, lq = (k & 3) / NBT, q = (k & 3) % NBT;
            const int ln = jl * LPJ + kq * NLQ + lq;
            float s = 0.f;
            for (int w = 0; w < C::kWarps; ++w) s += bpS[(w * 32 + ln) * 4 + q];
            btl_s[e] = log2_wide(s);
        }
        __syncthreads();

        loo_unit_epilogue<C>(a, cf, sm, u, u_begin, tile, At);
    }
}

// Tiles are taken from a counter (a.work, zeroed before the launch) so that
// units needing the exact fallback do not leave other SMs idle; each tile's
// partial has its own slot, so the schedule does not change the result.
template <int G1, int G2>
__global__ void __launch_bounds__(256, 2) k_loo_grid(const LooArgs a) {
    extern __shared__ float4 sm4[];
    __shared__ int next_tile;
    const CoefParam cf{a};
    for (int t0 = blockIdx.x;; t0 += gridDim.x) {
        if (threadIdx.x == 0) next_tile = a.work ? atomicAdd(a.work, 1) : t0;
        __syncthreads();
        const int t = next_tile;
        if (t >= a.n_tiles) break;
        loo_tile<G1, G2>(a, cf, t, reinterpret_cast<float*>(sm4));
    }
}

// Grid shapes of the tile kernels: k (h1) padded to an M-tile multiple of 16,
// l (h2) to 8, 16 or 32.
inline int loo_pad1(int g) { return g <= 16 ? 16 : 32; }
inline int loo_pad2(int g) { return g <= 8 ? 8 : (g <= 16 ? 16 : 32); }

int launch_loo_tile_kernel(int T1, int T2, const LooArgs& a, int grid, cudaStream_t st);
void fill_loo_args(LooArgs& a, const Dataset& D, const double* h1, int g1, const double* h2,
                   int g2, int T1, int T2);
int loo_units_per_tile(cde_ctx* ctx, int T1, int T2);
int loo_grid_ctas(cde_ctx* ctx, int T1, int T2);

}  // namespace cde
