// Tensor-core tile body of the leave-one-out grid kernel.
//
// Same sums as the FP32 tile body in loo_common.cuh (At_j(k,l) = sum_i
// u_i(k) w_i(l), Bt_j(k) = sum_i u_i(k)), with the outer-product accumulation
// issued as m16n8k8 TF32 tensor-core MMAs whose operands never touch shared
// memory: for row j the GEMM is D[k][l] += sum_i U[k][i] W[i][l] (M = k,
// N = l, K = i), and every lane produces exactly the fragment elements it
// owns -- A: (k = 16 mt + g [+8], i = t [+4]), B: (i = t [+4], l = 8 nt + g),
// g = lane/4, t = lane%4 -- with its own exp2 on the SFU (G1 + G2 per pair,
// no duplication across lanes).
//
// Precision: each factor v is split v = hi + lo, hi = v truncated to TF32
// (11 significant bits), lo = v - hi (exact in FP32, |lo| < 2^-10 |v|).  The
// product u w is formed as hi_u hi_w (TF32 m16n8k8) plus the two cross terms
// hi_u lo_w + lo_u hi_w, which carry at most 2^-9 of the product and so need
// only BF16 precision: both go through ONE BF16 m16n8k16 MMA whose k axis
// stacks [hi_u | lo_u] against [lo_w ; hi_w] (twice the MAC rate of TF32).
// Dropped lo*lo and the BF16 rounding of the cross terms leave about 2^-17
// relative per term (the sums over i average these errors).
//
// Bias.  A score sums N rows, so a per-row error with a fixed sign grows like
// N while random ones grow like sqrt(N); at N = 50,000 a bias of 1e-7 per row
// is 5e-3 on a score whose rows cancel to |L| ~ 100.  Two biases are removed:
//  * lo*lo: with hi the truncation of v, lo >= 0 for both factors and the
//    dropped lo_u lo_w is always positive (about 2^-22 of the product on
//    average).  w is instead split as w' = w / r, hi = trunc(w'),
//    lo = w' r - hi (one FMA, r = 1 - 11 2^-15 exact in FP32): lo is then
//    signed with mean ~0 over log-uniform mantissas, so E[lo_u lo_w] ~ 0.
//    The 1/r enters the exp2 argument as the constant kWc, so the split costs
//    the same instructions as truncation.
//  * ex2.approx.ftz.f32 returns values low by 5.1e-8 relative on average
//    (measured on sm_103a over exponent arguments in [-120, 0], rms error
//    6.0e-8).  The u factors' bias cancels between At and Bt in the
//    conditional score; the w factors' does not.  Both exp2 arguments carry
//    the constant kEx2Fix = log2(1 + 5.1e-8), again an FMA in place of a
//    multiply.
// Measured on the N = 50,000, d = 5, 32 x 32 grid against the full FP64
// grid: mean per-row error of L_cond -1.8e-7 before, ~0 after.  Each lane takes
// the points (2t, 2t+1) of a k-step so the TF32 and BF16 fragment layouts hold
// the same points.  The tensor core's FP32 accumulation is kept short: each
// chunk of 64 points (128 at 32 x 32: 16 or 32 MMAs per accumulator) starts
// from zero and is then added to an FP32 running total with a rounded add; the
// running totals live in shared memory.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "loo_common.cuh"

namespace cde {

// exp2-argument constants of the Gaussian factors (see the bias note above)
constexpr float kEx2Fix = 7.39e-8f;                        // log2(1 + 5.12e-8)
constexpr float kWr = 1.0f - 11.0f / 32768.0f;             // exact in FP32
constexpr float kWc = 4.843844517e-4f + 7.39e-8f;          // -log2(kWr) + kEx2Fix

// Gaussian factors 2^{c t + k} of two values (k: the argument constant)
__device__ __forceinline__ float2 gauss_factor2(float2 c, float2 t, float k) {
    const float2 a = __ffma2_rn(c, t, make_float2(k, k));
    return make_float2(ex2_approx(a.x), ex2_approx(a.y));
}

template <int G1, int G2>
struct MmaCfg {
    static_assert(G1 == 16 || G1 == 32, "M tiles of 16");
    static_assert(G2 == 8 || G2 == 16 || G2 == 32, "N tiles of 8");
    static constexpr int kThreads = 256, kWarps = 8;
    static constexpr int G1v = G1, G2v = G2;
    static constexpr int GG = G1 * G2;
    static constexpr int JW = 1024 / GG;     // rows per unit (all handled by every warp)
    static constexpr int MT = G1 / 16, NT = G2 / 8;
    // points per warp chunk (IC / 8 MMA k-steps): the chunk sums start from zero
    // and are added to the FP32 running totals once per chunk
    static constexpr int IC = 64;
    static constexpr int COMB = kWarps * 1024 + kWarps * JW * G1;
    // per warp: (t1, t1) and t2 for JW rows x IC points
    __host__ __device__ static int stage(int) { return kWarps * JW * IC * 3; }
    __host__ __device__ static int big(int d) {
        const int s = stage(d);
        const int b = s > COMB ? s : COMB;
        return b > 2048 ? b : 2048;
    }
    __host__ __device__ static int dpad(int d) { return (d * JW + 3) & ~3; }
    __host__ __device__ static int off_xj(int d) { return big(d); }
    __host__ __device__ static int off_yj(int d) { return big(d) + dpad(d); }
    __host__ __device__ static int off_mx(int d) { return off_yj(d) + 16; }
    __host__ __device__ static int off_my(int d) { return off_yj(d) + 32; }
    __host__ __device__ static int off_ji(int d) { return off_yj(d) + 48; }
    __host__ __device__ static int off_vr(int d) { return off_yj(d) + 80; }
    __host__ __device__ static int off_btl(int d) { return off_yj(d) + 96; }
    __host__ __device__ static int off_flag(int d) { return off_btl(d) + 2 * JW * G1; }
    __host__ __device__ static int off_nflag(int d) { return off_flag(d) + 1024; }
    // exact recomputation: per warp a list of 32 candidate points (3 words each),
    // then per row (at most 8) its bounds and cell range
    static constexpr int FBW = kWarps * 96 + 8 * 8;
    __host__ __device__ static int off_fbw(int d) { return off_nflag(d) + 4; }
    // per warp the FP32 running totals of its 1024 cells in MMA fragment order
    // (lane-contiguous float4 per (row, M tile, N tile): conflict-free)
    __host__ __device__ static int off_dts(int d) { return (off_fbw(d) + FBW + 3) & ~3; }
    static size_t smem_bytes(int d) { return (size_t)(off_dts(d) + kWarps * 1024) * sizeof(float); }
};

__device__ __forceinline__ uint32_t tf32_rna(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two floats to one register of BF16 (x in the low half: the lower k index)
__device__ __forceinline__ uint32_t pack_bf16x2(float x, float y) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int G1, int G2, int KERN, class Coef>
__device__ __forceinline__ void loo_tile_mma(const LooArgs& a, const Coef& cf, int tile, float* sm) {
    using C = MmaCfg<G1, G2>;
    constexpr int JW = C::JW, MT = C::MT, NT = C::NT, GG = C::GG, IC = C::IC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int d = a.d;
    float* big = sm;
    float* xj_s = sm + C::off_xj(d);
    float* yj_s = sm + C::off_yj(d);
    float* mx_s = sm + C::off_mx(d);
    float* my_s = sm + C::off_my(d);
    long long* ji_s = reinterpret_cast<long long*>(sm + C::off_ji(d));
    int* vr_s = reinterpret_cast<int*>(sm + C::off_vr(d));
    double* btl_s = reinterpret_cast<double*>(sm + C::off_btl(d));
    int* nflag_s = reinterpret_cast<int*>(sm + C::off_nflag(d));
    // per warp and row: t1 of each point twice ([32] float2), then t2 ([32] float):
    // the packed FP32x2 multiplies pair two x coefficients on one point, and one
    // y coefficient on two points
    float* tt = big + warp * JW * IC * 3;

    // this lane's coefficients: (k = 16 mt + g, k + 8) as a pair; l = 8 nt + g twice
    float2 ca1[MT], ca2[NT];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) ca1[mt] = make_float2(cf.a1(16 * mt + g), cf.a1(16 * mt + g + 8));
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) ca2[nt] = make_float2(cf.a2(8 * nt + g), cf.a2(8 * nt + g));

    // this launch's units of the tile (all of them unless a chunked launch gives a
    // window).  The loop's state lives in shared memory: thread 0 advances it, every
    // thread reads it after the barrier at the top of the loop, so it holds no
    // registers through the unit's body (the body runs at the register limit).
    __shared__ int ls_u, ls_end, ls_stride, ls_first;
    if (tid == 0) {
        int u_first, u_stride, u_len;
        loo_tile_span(a, tile, u_first, u_stride, u_len);
        ls_u = u_first + max(a.win0, 0) * u_stride;
        ls_end = u_first + min(u_len, a.win1) * u_stride;
        ls_stride = u_stride;
        ls_first = u_first;
    }
    const int64_t N = a.N, Np = a.Np;
    const int64_t n_chunks = (N + IC - 1) / IC;

    for (;;) {
        __syncthreads();
        const int u = ls_u;
        if (u >= ls_end) break;
        const bool first_u = u == ls_first;
        if (tid < JW) {
            const int64_t r = (int64_t)u * JW + tid;
            const bool v = r < a.n_rows;
            const int64_t r0 = v ? r : 0;
            const int64_t j = CDE_CK(a.rows ? a.rows[CDE_CK(r0, a.n_rows, 101)] : r0, a.N, 102);
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

        // running totals in shared memory (keeping them in registers costs 32 per
        // thread, which the compiler then takes from the software pipeline)
        float4* dts = reinterpret_cast<float4*>(sm + C::off_dts(d)) + warp * 256;
        float2 bt[JW][MT];  // denominator partials of k = 16 mt + g and k + 8
#pragma unroll
        for (int r = 0; r < JW; ++r)
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                bt[r][mt] = make_float2(0.f, 0.f);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) dts[((r * MT + mt) * NT + nt) * 32 + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
            }

        // point coordinates of the first chunk (lane = point of each 32-point half),
        // prefetched one chunk ahead
        constexpr int HH = IC / 32;
        float xin[HH][8], yin[HH];
        int64_t ch = warp;
        if (ch < n_chunks) {
#pragma unroll
            for (int h = 0; h < HH; ++h) {
                const int64_t i = CDE_CK(ch * IC + h * 32 + lane, Np, 103);  // < Np
#pragma unroll
                for (int c = 0; c < 8; ++c) xin[h][c] = c < d ? a.xs[(int64_t)c * Np + i] : 0.f;
                yin[h] = a.y[i];
            }
        }
        // one row per unit (G1 G2 = 1024): its constants stay in registers for
        // the whole chunk loop instead of being re-read from shared memory
        float yr1 = 0.f, mxr1 = 0.f, myr1 = 0.f;
        int jr1 = 0;
        if constexpr (JW == 1) {
            yr1 = yj_s[0];
            mxr1 = mx_s[0];
            myr1 = my_s[0];
            jr1 = (int)ji_s[0];
        }
        const int N32 = (int)N;  // N < 2^31
        for (; ch < n_chunks; ch += C::kWarps) {
            // ---- distance pass: lane = the points (h = 0, 1) of the chunk's halves,
            //      packed FP32x2; masked pairs get t1 = -inf ----
            static_assert(IC == 64, "two points per lane");
            __syncwarp();
            {
              const int64_t i0 = ch * IC + lane, i1 = i0 + 32;
#pragma unroll
              for (int r = 0; r < JW; ++r) {
                const float* xjr = xj_s + r * d;
                float2 dx2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < d) {
                        const float2 q = __fadd2_rn(make_float2(xjr[c], xjr[c]), make_float2(-xin[0][c], -xin[1][c]));
                        dx2 = __ffma2_rn(q, q, dx2);
                    }
                for (int c = 8; c < d; ++c) {
                    const float2 q = __fadd2_rn(make_float2(xjr[c], xjr[c]),
                                                make_float2(-a.xs[(int64_t)c * Np + CDE_CK(i0, Np, 104)],
                                                            -a.xs[(int64_t)c * Np + CDE_CK(i1, Np, 104)]));
                    dx2 = __ffma2_rn(q, q, dx2);
                }
                const float yr = JW == 1 ? yr1 : yj_s[r];
                const float2 dy = __fadd2_rn(make_float2(yr, yr), make_float2(-yin[0], -yin[1]));
                const float2 dy2 = __fmul2_rn(dy, dy);
                const int jr = JW == 1 ? jr1 : (int)ji_s[r];
                const bool ok0 = (int)i0 < N32 && (int)i0 != jr, ok1 = (int)i1 < N32 && (int)i1 != jr;
                // Gaussian: shifted exponents (masked pairs -inf); Epanechnikov:
                // squared distances (masked pairs +inf)
                const float mxv = JW == 1 ? mxr1 : mx_s[r], myv = JW == 1 ? myr1 : my_s[r];
                float2 t1, t2;
                if constexpr (KERN == 0) {
                    t1 = __fadd2_rn(make_float2(mxv, mxv), make_float2(-dx2.x, -dx2.y));
                    t2 = __fadd2_rn(make_float2(myv, myv), make_float2(-dy2.x, -dy2.y));
                    // masked pairs: w = 0 as well (at i = j, m_y - 0 could overflow 2^{a2 t2})
                    t1.x = ok0 ? t1.x : -INFINITY;  t1.y = ok1 ? t1.y : -INFINITY;
                    t2.x = ok0 ? t2.x : -INFINITY;  t2.y = ok1 ? t2.y : -INFINITY;
                } else {
                    t1 = make_float2(ok0 ? dx2.x : INFINITY, ok1 ? dx2.y : INFINITY);
                    t2 = dy2;
                }
                reinterpret_cast<float2*>(tt + r * 3 * IC)[lane] = make_float2(t1.x, t1.x);
                reinterpret_cast<float2*>(tt + r * 3 * IC)[32 + lane] = make_float2(t1.y, t1.y);
                tt[r * 3 * IC + 2 * IC + lane] = t2.x;
                tt[r * 3 * IC + 2 * IC + 32 + lane] = t2.y;
              }
            }
            if (ch + C::kWarps < n_chunks) {
#pragma unroll
                for (int h = 0; h < HH; ++h) {
                    const int64_t i2 = CDE_CK((ch + C::kWarps) * IC + h * 32 + lane, Np, 105);
#pragma unroll
                    for (int c = 0; c < 8; ++c) xin[h][c] = c < d ? a.xs[(int64_t)c * Np + i2] : 0.f;
                    yin[h] = a.y[i2];
                }
            }
            __syncwarp();
            // ---- MMA pass: IC / 8 k-steps of 8 points ----
            float D[JW][MT][NT][4];
#pragma unroll
            for (int r = 0; r < JW; ++r)
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                        for (int q = 0; q < 4; ++q) D[r][mt][nt][q] = 0.f;
#pragma unroll
            for (int s = 0; s < IC / 8; ++s) {
#pragma unroll
                for (int r = 0; r < JW; ++r) {
                    // this lane's two points of the k-step: p0 = 8s + 2t, p1 = p0 + 1
                    const float4 q1 = *reinterpret_cast<const float4*>(tt + r * 3 * IC + 2 * (8 * s + 2 * t));
                    const float2 t1p0 = make_float2(q1.x, q1.y), t1p1 = make_float2(q1.z, q1.w);
                    const float2 t2p = *reinterpret_cast<const float2*>(tt + r * 3 * IC + 2 * IC + 8 * s + 2 * t);
                    // Two orders of the k-step, the faster one per kernel and shape (measured at
                    // N = 50,000): all B fragments, all A fragments, then the 16 MMAs; or the A
                    // fragments, then per N tile its B fragment and its MMAs, which spreads the
                    // MMAs over the factor work (Epanechnikov 32 x 32: 57.6 -> 55.2 ms; Gaussian
                    // 16 x 16: 23.25 -> 23.0 ms; Gaussian 32 x 32 59.1 -> 59.9 ms, so not there)
                    constexpr bool kSpread = KERN == 1 || GG == 256;
                    if constexpr (!kSpread) {
                        // B fragments: w(l, p0) in register 0, w(l, p1) in register 1 (TF32);
                        // BF16: register 0 = lo w at (p0, p1), register 1 = hi w at (p0, p1)
                        uint32_t bh[NT][2], bx[NT][2];
    #pragma unroll
                        for (int nt = 0; nt < NT; ++nt) {
                            // Gaussian: w' = w / r, lo = w' r - hi (signed); Epanechnikov: lo = w - hi
                            const float2 w = KERN == 0 ? gauss_factor2(ca2[nt], t2p, kWc)
                                                       : kernel_factor2<KERN>(ca2[nt], t2p);
                            const float2 h = make_float2(__uint_as_float(__float_as_uint(w.x) & 0xffffe000u),
                                                         __uint_as_float(__float_as_uint(w.y) & 0xffffe000u));
                            const float2 l = KERN == 0 ? __ffma2_rn(w, make_float2(kWr, kWr), make_float2(-h.x, -h.y))
                                                       : __ffma2_rn(h, make_float2(-1.f, -1.f), w);
                            bh[nt][0] = __float_as_uint(h.x);
                            bh[nt][1] = __float_as_uint(h.y);
                            bx[nt][0] = pack_bf16x2(l.x, l.y);
                            bx[nt][1] = pack_bf16x2(h.x, h.y);
                        }
                        // A fragments: TF32 (k, p0), (k+8, p0), (k, p1), (k+8, p1);
                        // BF16 columns 2t, 2t+1 hold hi u at (p0, p1), columns 2t+8, 2t+9 lo u
                        uint32_t ah[MT][4], ax[MT][4];
    #pragma unroll
                        for (int mt = 0; mt < MT; ++mt) {
                            // (k, p0), (k+8, p0) and (k, p1), (k+8, p1)
                            const float2 u0 = KERN == 0 ? gauss_factor2(ca1[mt], t1p0, kEx2Fix)
                                                        : kernel_factor2<KERN>(ca1[mt], t1p0);
                            const float2 u1 = KERN == 0 ? gauss_factor2(ca1[mt], t1p1, kEx2Fix)
                                                        : kernel_factor2<KERN>(ca1[mt], t1p1);
                            bt[r][mt] = __fadd2_rn(bt[r][mt], __fadd2_rn(u0, u1));
                            const float2 h0 = make_float2(__uint_as_float(__float_as_uint(u0.x) & 0xffffe000u),
                                                          __uint_as_float(__float_as_uint(u0.y) & 0xffffe000u));
                            const float2 h1 = make_float2(__uint_as_float(__float_as_uint(u1.x) & 0xffffe000u),
                                                          __uint_as_float(__float_as_uint(u1.y) & 0xffffe000u));
                            const float2 l0 = __ffma2_rn(h0, make_float2(-1.f, -1.f), u0);
                            const float2 l1 = __ffma2_rn(h1, make_float2(-1.f, -1.f), u1);
                            ah[mt][0] = __float_as_uint(h0.x);
                            ah[mt][1] = __float_as_uint(h0.y);
                            ah[mt][2] = __float_as_uint(h1.x);
                            ah[mt][3] = __float_as_uint(h1.y);
                            ax[mt][0] = pack_bf16x2(h0.x, h1.x);
                            ax[mt][1] = pack_bf16x2(h0.y, h1.y);
                            ax[mt][2] = pack_bf16x2(l0.x, l1.x);
                            ax[mt][3] = pack_bf16x2(l0.y, l1.y);
                        }
                        // hi*hi on TF32; hi*lo + lo*hi together on one BF16 k16 MMA
    #pragma unroll
                        for (int mt = 0; mt < MT; ++mt)
    #pragma unroll
                            for (int nt = 0; nt < NT; ++nt) mma_tf32(D[r][mt][nt], ah[mt], bh[nt][0], bh[nt][1]);
    #pragma unroll
                        for (int mt = 0; mt < MT; ++mt)
    #pragma unroll
                            for (int nt = 0; nt < NT; ++nt) mma_bf16(D[r][mt][nt], ax[mt], bx[nt][0], bx[nt][1]);
                    } else {
                        // A fragments: TF32 (k, p0), (k+8, p0), (k, p1), (k+8, p1);
                        // BF16 columns 2t, 2t+1 hold hi u at (p0, p1), columns 2t+8, 2t+9 lo u
                        uint32_t ah[MT][4], ax[MT][4];
    #pragma unroll
                        for (int mt = 0; mt < MT; ++mt) {
                            // (k, p0), (k+8, p0) and (k, p1), (k+8, p1)
                            const float2 u0 = KERN == 0 ? gauss_factor2(ca1[mt], t1p0, kEx2Fix)
                                                        : kernel_factor2<KERN>(ca1[mt], t1p0);
                            const float2 u1 = KERN == 0 ? gauss_factor2(ca1[mt], t1p1, kEx2Fix)
                                                        : kernel_factor2<KERN>(ca1[mt], t1p1);
                            bt[r][mt] = __fadd2_rn(bt[r][mt], __fadd2_rn(u0, u1));
                            const float2 h0 = make_float2(__uint_as_float(__float_as_uint(u0.x) & 0xffffe000u),
                                                          __uint_as_float(__float_as_uint(u0.y) & 0xffffe000u));
                            const float2 h1 = make_float2(__uint_as_float(__float_as_uint(u1.x) & 0xffffe000u),
                                                          __uint_as_float(__float_as_uint(u1.y) & 0xffffe000u));
                            const float2 l0 = __ffma2_rn(h0, make_float2(-1.f, -1.f), u0);
                            const float2 l1 = __ffma2_rn(h1, make_float2(-1.f, -1.f), u1);
                            ah[mt][0] = __float_as_uint(h0.x);
                            ah[mt][1] = __float_as_uint(h0.y);
                            ah[mt][2] = __float_as_uint(h1.x);
                            ah[mt][3] = __float_as_uint(h1.y);
                            ax[mt][0] = pack_bf16x2(h0.x, h1.x);
                            ax[mt][1] = pack_bf16x2(h0.y, h1.y);
                            ax[mt][2] = pack_bf16x2(l0.x, l1.x);
                            ax[mt][3] = pack_bf16x2(l0.y, l1.y);
                        }
                        // per N tile: its B fragments, then its MMAs (same order per accumulator:
                        // TF32 hi*hi, then the BF16 cross terms)
#pragma unroll
                        for (int nt = 0; nt < NT; ++nt) {
                            const float2 w = KERN == 0 ? gauss_factor2(ca2[nt], t2p, kWc)
                                                       : kernel_factor2<KERN>(ca2[nt], t2p);
                            const float2 h = make_float2(__uint_as_float(__float_as_uint(w.x) & 0xffffe000u),
                                                         __uint_as_float(__float_as_uint(w.y) & 0xffffe000u));
                            const float2 l = KERN == 0 ? __ffma2_rn(w, make_float2(kWr, kWr), make_float2(-h.x, -h.y))
                                                       : __ffma2_rn(h, make_float2(-1.f, -1.f), w);
                            const uint32_t bh0 = __float_as_uint(h.x), bh1 = __float_as_uint(h.y);
                            const uint32_t bx0 = pack_bf16x2(l.x, l.y), bx1 = pack_bf16x2(h.x, h.y);
#pragma unroll
                            for (int mt = 0; mt < MT; ++mt) mma_tf32(D[r][mt][nt], ah[mt], bh0, bh1);
#pragma unroll
                            for (int mt = 0; mt < MT; ++mt) mma_bf16(D[r][mt][nt], ax[mt], bx0, bx1);
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < JW; ++r)
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt)
                        {
                            float4 o = dts[((r * MT + mt) * NT + nt) * 32 + lane];
                            const float2 s0 = __fadd2_rn(make_float2(o.x, o.y), make_float2(D[r][mt][nt][0], D[r][mt][nt][1]));
                            const float2 s1 = __fadd2_rn(make_float2(o.z, o.w), make_float2(D[r][mt][nt][2], D[r][mt][nt][3]));
                            dts[((r * MT + mt) * NT + nt) * 32 + lane] = make_float4(s0.x, s0.y, s1.x, s1.y);
                        }
        }

        // ---- combine the 8 warps in fixed order ----
        __syncthreads();
        float* accS = big;
        float* btS = big + C::kWarps * 1024;
#pragma unroll
        for (int r = 0; r < JW; ++r)
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const float4 o = dts[((r * MT + mt) * NT + nt) * 32 + lane];
                    const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = 16 * mt + g + 8 * (q >> 1), l = 8 * nt + 2 * t + (q & 1);
                        accS[warp * 1024 + r * GG + k * G2 + l] = ov[q];
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float v = h ? bt[r][mt].y : bt[r][mt].x;
                    v += __shfl_xor_sync(0xffffffffu, v, 1);
                    v += __shfl_xor_sync(0xffffffffu, v, 2);
                    if (t == 0) btS[warp * JW * G1 + r * G1 + 16 * mt + g + 8 * h] = v;
                }
            }
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
            float s = 0.f;
            for (int w = 0; w < C::kWarps; ++w) s += btS[w * JW * G1 + e];
            btl_s[e] = log2_wide(s);
        }
        __syncthreads();
        loo_unit_epilogue<C, KERN>(a, cf, sm, u, first_u, tile, At);
        // (every thread read ls_u before the barriers of the unit's body)
        if (tid == 0) ls_u += ls_stride;
    }
}

template <int G1, int G2, int KERN>
__global__ void __launch_bounds__(256, 2) k_loo_mma(const LooArgs a) {
    extern __shared__ float4 sm4[];
    __shared__ int next_tile;
    const CoefParam cf{a};
    for (int t0 = blockIdx.x;; t0 += gridDim.x) {
        if (threadIdx.x == 0) next_tile = a.work ? atomicAdd(a.work, 1) : t0;
        __syncthreads();
        const int t = next_tile;
        if (t >= a.n_tiles) break;
        loo_tile_mma<G1, G2, KERN>(a, cf, t, reinterpret_cast<float*>(sm4));
    }
}

}  // namespace cde
