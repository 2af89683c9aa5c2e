// Gradient of the conditional LOO log-likelihood with respect to
// (ln h1, ln h2) at one bandwidth pair, plus the score itself.
//
// For the Gaussian kernels of Sec. 2, d ln K_h1(r)/d ln h1 = r^2/h1^2 - d and
// d ln K_h2(t)/d ln h2 = t^2/h2^2 - 1, so with the Sec. 3.2 sums A_j, B_j:
//   d ell_j/d ln h1 = (E_Aj[dx2] - E_Bj[dx2]) / h1^2,
//   d ell_j/d ln h2 = E_Aj[dy2] / h2^2 - 1,
// E_Aj weighting i by K_h1 K_h2 and E_Bj by K_h1 (i != j).  Per row five
// shifted sums are needed:
//   S_A = sum v_i, S_Ax = sum v_i dx2_i, S_Ay = sum v_i dy2_i,
//   S_B = sum u_i, S_Bx = sum u_i dx2_i,
// with the separable per-row shifts of the grid kernel:
//   u_i = 2^{-a1 (dx2_i - m_x)}  (<= 1, the x-nearest neighbour gives 1),
//   w_i = 2^{-a2 (dy2_i - m_y)},  v_i = u_i w_i,
// two exp2 per pair.  S_B >= 1 never underflows; a row whose S_A falls below
// 2^-40 (its x-near and y-near neighbours differ and both factors are small) is
// recomputed exactly by k_grad_fallback with a joint shift: v_i = 2^{M - e_i},
// e_i = a1 (dx2_i - m_x) + a2 (dy2_i - m_y), M the running minimum of e_i
// (online rescaling: when a smaller e arrives the sums are multiplied by
// 2^{e - M}).
//
// Epanechnikov datasets (profiles u = (1 - dx2/h1^2)_+, w = (1 - dy2/h2^2)_+):
// d K_h1/d ln h1 = c_d h1^{-d} (v - d u) with v = 2 dx2/h1^2 inside the support,
// d K_h2/d ln h2 = c_1 h2^{-1} (z - w) with z = 2 dy2/h2^2 inside, so
//   d ell_j/d ln h1 = sum v w / sum u w - sum v / sum u,
//   d ell_j/d ln h2 = sum u z / sum u w - 1,
// and the same five slots hold sum u w, sum v w, sum u z, sum u, sum v (no
// shift: M = 0).  A row with sum u w = 0 has ell_j = -inf and adds 0 to both
// derivatives.
//
// The i range is split over gridDim.y CTAs; split partials (M, S_A, S_Ax,
// S_Ay, S_B, S_Bx) are merged per row in FP64 in split order, the per-row
// log-ratio and derivatives are formed in FP64, and rows are summed in a
// fixed order, so the result is bitwise reproducible.
#include <cmath>
#include <string>
#include <type_traits>

#include "cde_internal.h"
#include "tc_util.cuh"

namespace cde {

struct GradArgs {
    const float* xs;
    const float* y;
    const float* mx;
    const float* my;
    int64_t N, Np;
    int d;
    float a1, a2;          // Gaussian log2(e)/(2 h^2); Epanechnikov 1/h^2
    int64_t i_per_split;   // multiple of the tile
    float* part;           // [n_split][N][6]
    const uint32_t* xsplit;   // d >= 16: TF32 hi words [Np][DK] in the MMA core-matrix layout, then lo
    const float* xnorm;       // d >= 16: |x_i|^2 [Np]
    int* err;                 // the context's device-wait word (k_grad_tc)
    int64_t bx0;              // first row block of this launch (grid x covers row blocks bx0 ...)
};

constexpr int kGradThreads = 128;

__device__ __forceinline__ float ex2g(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float fma_sat_g(float a, float b, float c) {
    float r;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// One pair's contribution with the online joint shift, without branches: when
// e does not lower the running minimum the rescale factor is exactly 2^0 = 1
// (M = +inf at the start: r = 0, the sums are 0).  Gaussian fallback rows only.
__device__ __forceinline__ void grad_accumulate_joint(bool ok, float dx2, float dy2, float mx, float my,
                                                      float a1, float a2, float& M, float& SA, float& SAx,
                                                      float& SAy, float& SB, float& SBx) {
    const float ex = dx2 - mx, ey = dy2 - my;
    const float e = fmaf(a1, ex, a2 * ey);
    const bool lower = ok && e < M;
    const float Mn = lower ? e : M;
    const float r = lower ? ex2g(e - M) : 1.f;
    SA *= r;
    SAx *= r;
    SAy *= r;
    M = Mn;
    const float u = ok ? ex2g(-a1 * ex) : 0.f;
    const float v = ok ? ex2g(M - e) : 0.f;
    SB += u;
    SBx = fmaf(u, dx2, SBx);
    SA += v;
    SAx = fmaf(v, dx2, SAx);
    SAy = fmaf(v, dy2, SAy);
}

// Two rows' contributions from one point through the packed FP32x2 pipe (rows
// in .x and .y; Gaussian: am = a1 m_x, bm = a2 m_y of the rows).  Gaussian:
// the separable shifted factors u = 2^{a1 m_x - a1 dx2}, w = 2^{a2 m_y - a2 dy2}
// (one FMA each), v = u w, and S_B += u, S_Bx += u dx2, S_A += v,
// S_Ax += v dx2, S_Ay += v dy2.  Epanechnikov: plain sums of the profiles and
// their log-derivative weights (the support test is the profile itself being
// positive).
template <int KERN>
__device__ __forceinline__ void grad_accumulate2(bool ok0, bool ok1, float2 dx2, float2 dy2, float2 am,
                                                 float2 bm, float a1, float a2, float2& SA, float2& SAx,
                                                 float2& SAy, float2& SB, float2& SBx) {
    if constexpr (KERN == 1) {
        const float2 u = make_float2(ok0 ? fma_sat_g(-a1, dx2.x, 1.f) : 0.f, ok1 ? fma_sat_g(-a1, dx2.y, 1.f) : 0.f);
        const float2 w = make_float2(fma_sat_g(-a2, dy2.x, 1.f), fma_sat_g(-a2, dy2.y, 1.f));
        const float ta1 = 2.f * a1, ta2 = 2.f * a2;
        const float2 vx = __fmul2_rn(make_float2(ta1, ta1), dx2), zy = __fmul2_rn(make_float2(ta2, ta2), dy2);
        const float2 v = make_float2(u.x > 0.f ? vx.x : 0.f, u.y > 0.f ? vx.y : 0.f);
        const float2 z = make_float2(w.x > 0.f ? zy.x : 0.f, w.y > 0.f ? zy.y : 0.f);
        SA = __ffma2_rn(u, w, SA);
        SAx = __ffma2_rn(v, w, SAx);
        SAy = __ffma2_rn(u, z, SAy);
        SB = __fadd2_rn(SB, u);
        SBx = __fadd2_rn(SBx, v);
        return;
    }
    const float2 au = __ffma2_rn(dx2, make_float2(-a1, -a1), am);   // a1 m_x - a1 dx2
    const float2 aw = __ffma2_rn(dy2, make_float2(-a2, -a2), bm);   // a2 m_y - a2 dy2
    const float2 u = make_float2(ok0 ? ex2g(au.x) : 0.f, ok1 ? ex2g(au.y) : 0.f);
    const float2 v = __fmul2_rn(u, make_float2(ex2g(aw.x), ex2g(aw.y)));
    SB = __fadd2_rn(SB, u);
    SBx = __ffma2_rn(u, dx2, SBx);
    SA = __fadd2_rn(SA, v);
    SAx = __ffma2_rn(v, dx2, SAx);
    SAy = __ffma2_rn(v, dy2, SAy);
}

// d < 16: JB rows per thread (processed as JB / 2 packed pairs), points
// point-major in shared memory (128-bit broadcast loads), 32-bit index masks.
template <int JB, int DREG, int KERN>
__global__ void __launch_bounds__(kGradThreads) k_loo_grad(const GradArgs g) {
    static_assert(JB % 2 == 0, "rows go through the packed pipe in pairs");
    constexpr int JP = JB / 2;
    __shared__ __align__(16) float xt[kGradThreads][DREG];  // point-major: 128-bit broadcast loads
    __shared__ float yt[kGradThreads];
    const int tid = threadIdx.x;
    const int64_t jbase = ((int64_t)blockIdx.x + g.bx0) * kGradThreads * JB + tid;
    const int64_t i0 = (int64_t)blockIdx.y * g.i_per_split;
    const int64_t i1 = min(g.N, i0 + g.i_per_split);
    const int d = g.d;
    float2 xj[JP][DREG], yj[JP], am[JP], bm[JP];
    float2 SA[JP], SAx[JP], SAy[JP], SB[JP], SBx[JP];
    int jj[JB];
#pragma unroll
    for (int b = 0; b < JB; ++b) {
        const int64_t j = jbase + (int64_t)b * kGradThreads;
        const int64_t jc = j < g.N ? j : 0;
        jj[b] = (int)j;   // N < 2^31
        const int p = b >> 1;
        float* xr = reinterpret_cast<float*>(&xj[p][0]) + (b & 1);
#pragma unroll
        for (int c = 0; c < DREG; ++c) xr[2 * c] = c < d ? g.xs[(int64_t)c * g.Np + jc] : 0.f;
        reinterpret_cast<float*>(&yj[p])[b & 1] = g.y[jc];
        reinterpret_cast<float*>(&am[p])[b & 1] = g.a1 * g.mx[jc];   // a1 m_x (Gaussian; unused otherwise)
        reinterpret_cast<float*>(&bm[p])[b & 1] = g.a2 * g.my[jc];   // a2 m_y
    }
#pragma unroll
    for (int p = 0; p < JP; ++p) SA[p] = SAx[p] = SAy[p] = SB[p] = SBx[p] = make_float2(0.f, 0.f);
    const float a1 = g.a1, a2 = g.a2;
    const float2 m1 = make_float2(-1.f, -1.f);
    for (int64_t t0 = i0; t0 < i1; t0 += kGradThreads) {
        __syncthreads();
        const int64_t it = CDE_CK(t0 + tid, g.Np, 401);  // < Np: i_per_split and Np are multiples of 128
#pragma unroll
        for (int c = 0; c < DREG; ++c) xt[tid][c] = c < d ? g.xs[(int64_t)c * g.Np + it] : 0.f;
        yt[tid] = g.y[it];
        __syncthreads();
        const int n = (int)min((int64_t)kGradThreads, i1 - t0);
        // the leave-one-out test is needed only where the tile meets this CTA's rows
        const int64_t r0 = ((int64_t)blockIdx.x + g.bx0) * kGradThreads * JB;
        const auto body = [&](auto masked) {
            for (int t = 0; t < n; ++t) {
                const int i32 = (int)(t0 + t);  // N < 2^31
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
#pragma unroll
                for (int p = 0; p < JP; ++p) {
                    // x_j - x_i as fma(x_i, -1, x_j): the scalar subtraction's rounding
                    float2 dx2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < DREG; ++c) {
                        const float2 q = __ffma2_rn(make_float2(xi[c], xi[c]), m1, xj[p][c]);
                        dx2 = __ffma2_rn(q, q, dx2);
                    }
                    const float2 dy = __ffma2_rn(make_float2(yi, yi), m1, yj[p]);
                    const float2 dy2 = __fmul2_rn(dy, dy);
                    const bool ok0 = !decltype(masked)::value || i32 != jj[2 * p];
                    const bool ok1 = !decltype(masked)::value || i32 != jj[2 * p + 1];
                    grad_accumulate2<KERN>(ok0, ok1, dx2, dy2, am[p], bm[p], a1, a2, SA[p], SAx[p], SAy[p], SB[p],
                                           SBx[p]);
                }
            }
        };
        if (t0 < r0 + kGradThreads * JB && t0 + kGradThreads > r0) body(std::true_type{});
        else body(std::false_type{});
    }
#pragma unroll
    for (int b = 0; b < JB; ++b) {
        const int64_t j = jbase + (int64_t)b * kGradThreads;
        if (j >= g.N) continue;
        const int p = b >> 1;
        float* q = g.part + ((int64_t)blockIdx.y * g.N + j) * 6;
        const auto pick = [b](float2 v) { return (b & 1) ? v.y : v.x; };
        q[0] = 0.f;  // no running shift on this path
        q[1] = pick(SA[p]);
        q[2] = pick(SAx[p]);
        q[3] = pick(SAy[p]);
        q[4] = pick(SB[p]);
        q[5] = pick(SBx[p]);
    }
}

// Two adjacent points' contributions to one row (the row's a1 m_x, a2 m_y in
// both lanes) through the packed FP32x2 pipe; the operations of grad_accumulate2.
template <int KERN>
__device__ __forceinline__ void grad_accumulate_pts(bool ok0, bool ok1, float2 dx2, float2 dy2, float am, float bm,
                                                    float a1, float a2, float2& SA, float2& SAx, float2& SAy,
                                                    float2& SB, float2& SBx) {
    grad_accumulate2<KERN>(ok0, ok1, dx2, dy2, make_float2(am, am), make_float2(bm, bm), a1, a2, SA, SAx, SAy,
                           SB, SBx);
}

// ---- d >= 16 on the 5th-generation tensor cores (k_grad_tc) ------------------
//
// The cross term x_j . x_i of |x_j - x_i|^2 = n_j + n_i - 2 x_j . x_i is a
// true contraction over the dimensions with rows j and points i as the two
// free indices, so it runs as tcgen05 MMAs (kind::tf32, M = 128 rows, N = PT
// points, K = 8 per instruction) with the accumulator in tensor memory, on
// split operands x = hi + lo (hi the TF32 truncation, lo the exact FP32
// remainder): hi hi + hi lo + lo hi, FP32 accumulation, about 2^-20 of
// sum_k |x_jk x_ik| per dot product; the norms n are FP32 and the distance is
// clamped at 0.  Warp 0 copies the CTA's 128 split rows once and each point
// tile (split rows, norms, y) by bulk copies into a two-stage ring, and one
// thread issues the MMAs into one of two TMEM buffers.  Sixteen epilogue warps
// (four per TMEM lane quadrant, one quarter of the tile's columns each) read
// their dot products with tcgen05.ld, release the TMEM buffer, and form the
// per-pair sums of grad_accumulate_pts from the stage's norms and y; a stage
// is refilled once its MMAs and all epilogue warps are done with it (warp 0
// refills one tile behind, after queueing the next MMAs).  Per-pair
// leave-one-out and split-end tests run only in the column blocks that need
// them.  Every wait is bounded.

constexpr int kGTRows = 128;                      // rows per CTA: the TMEM lanes, MMA M
constexpr int kGTEpi = 16;                        // epilogue warps
constexpr int kGTThreads = 32 * (1 + kGTEpi);     // warp 0: copies and MMA issue

template <int DK>
struct GradTc {
    static constexpr int PT = DK <= 32 ? 256 : 128;   // points per tile (MMA N)
    static constexpr int COLS = PT / 4;               // columns per epilogue warp
    static constexpr int A_WORDS = kGTRows * DK;      // one split (hi or lo) of the rows
    static constexpr int B_WORDS = PT * DK;           // one split of a point tile
    static constexpr uint32_t SBO = DK * 32;          // bytes between 8-row groups: DK / 4 core matrices
};

template <int DK>
struct GradTcSmem {
    uint32_t ah[GradTc<DK>::A_WORDS], al[GradTc<DK>::A_WORDS];
    uint32_t bh[2][GradTc<DK>::B_WORDS], bl[2][GradTc<DK>::B_WORDS];
    float ny[2][2][GradTc<DK>::PT];   // the tile's norms and y, per stage
    float red[kGTEpi][5][32];
    unsigned long long full[2], empty[2], tfull[2], tempty[2], afull;
    uint32_t tmem_base;
    int abort;
};

// Once per call: every point's x split into TF32 hi + lo in the K-major,
// no-swizzle core-matrix layout of the MMA operands (word (p, k) at
// (p / 8) 8 DK + (k / 4) 32 + (p % 8) 4 + k % 4: a tile of points starting at
// a multiple of 8 is one contiguous block), and its squared norm.  A block
// handles 32 points.
template <int DK>
__global__ void __launch_bounds__(256) k_grad_split_tc(const float* __restrict__ xs, int64_t Np, int d,
                                                       uint32_t* __restrict__ xsplit, float* __restrict__ xnorm) {
    __shared__ float v[32][DK + 1];
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    for (int e = threadIdx.x; e < 32 * DK; e += 256) {
        const int c = e / 32, pp = e % 32;
        v[pp][c] = c < d ? xs[(int64_t)c * Np + p0 + pp] : 0.f;   // p0 + pp < Np (a multiple of 256)
    }
    __syncthreads();
    uint32_t* hi = xsplit + p0 * DK;
    uint32_t* lo = xsplit + Np * DK + p0 * DK;
    for (int w = threadIdx.x; w < 32 * DK; w += 256) {
        const int grp = w / (8 * DK), rem = w % (8 * DK);
        const int kc = rem / 32, r8 = (rem % 32) / 4, k4 = rem % 4;
        const float x = v[8 * grp + r8][4 * kc + k4];
        const uint32_t h = __float_as_uint(x) & 0xffffe000u;
        hi[w] = h;
        lo[w] = __float_as_uint(x - __uint_as_float(h));
    }
    if (threadIdx.x < 32) {
        float n = 0.f;
        for (int c = 0; c < d; ++c) n = fmaf(v[threadIdx.x][c], v[threadIdx.x][c], n);
        xnorm[p0 + threadIdx.x] = n;
    }
}

// One epilogue pass over NC columns already in registers (point p0 + c for
// column c, its norm and y at ns[c], ys[c]; the caller's row j): distances from
// the dot products and the norms,
// then the sums of grad_accumulate_pts.  MASKED: some column is past the split's
// end or is one of the warp's own rows (the leave-one-out exclusion); otherwise
// every pair counts and no per-pair test is made.
template <int KERN, int NC, bool MASKED>
__device__ __forceinline__ void grad_tc_columns(const GradArgs& g, const float (&dot)[NC], const float* ns,
                                                const float* ys, int64_t p0, int64_t i1, int j, float nj, float yj,
                                                float am, float bm, float2& SA, float2& SAx, float2& SAy, float2& SB,
                                                float2& SBx) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float a1 = g.a1, a2 = g.a2;
#pragma unroll
    for (int c = 0; c < NC; c += 4) {
        const int64_t p = p0 + c;
        const float4 n4 = *reinterpret_cast<const float4*>(ns + c);   // shared memory, broadcast
        const float4 y4 = *reinterpret_cast<const float4*>(ys + c);
        const int ip = (int)p;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 dd = make_float2(dot[c + 2 * h], dot[c + 2 * h + 1]);
            const float2 nip = h ? make_float2(n4.z, n4.w) : make_float2(n4.x, n4.y);
            const float2 yip = h ? make_float2(y4.z, y4.w) : make_float2(y4.x, y4.y);
            const float2 s2 = __ffma2_rn(dd, make_float2(-2.f, -2.f), __fadd2_rn(make_float2(nj, nj), nip));
            const float2 dx2 = make_float2(fmaxf(s2.x, 0.f), fmaxf(s2.y, 0.f));
            const float2 dy = __ffma2_rn(yip, m1, make_float2(yj, yj));
            const float2 dy2 = __fmul2_rn(dy, dy);
            const int ia = ip + 2 * h;
            const bool ok0 = !MASKED || (ia < i1 && ia != j), ok1 = !MASKED || (ia + 1 < i1 && ia + 1 != j);
            grad_accumulate_pts<KERN>(ok0, ok1, dx2, dy2, am, bm, a1, a2, SA, SAx, SAy, SB, SBx);
        }
    }
}

// Bulk-copy point tile t0 (hi and lo split rows, norms, y) into stage s,
// completing on full[s]; one thread.
template <int DK>
__device__ __forceinline__ void grad_tc_load(const GradArgs& g, GradTcSmem<DK>& S, int s, int64_t t0) {
    using C = GradTc<DK>;
    const uint32_t fb = smem_u32(&S.full[s]);
    mbar_arrive_expect_tx(fb, 2u * C::B_WORDS * 4u + 2u * C::PT * 4u);
    const int64_t tc = CDE_CK(t0, g.Np - C::PT + 1, 412);   // t0 + PT <= Np
    bulk_g2s(smem_u32(S.bh[s]), g.xsplit + tc * DK, C::B_WORDS * 4u, fb);
    bulk_g2s(smem_u32(S.bl[s]), g.xsplit + (g.Np + tc) * DK, C::B_WORDS * 4u, fb);
    bulk_g2s(smem_u32(S.ny[s][0]), g.xnorm + tc, C::PT * 4u, fb);
    bulk_g2s(smem_u32(S.ny[s][1]), g.y + tc, C::PT * 4u, fb);
}

template <int DK, int KERN>
__global__ void __launch_bounds__(kGTThreads, 1) k_grad_tc(const GradArgs g) {
    using C = GradTc<DK>;
    extern __shared__ float4 gt_dyn[];
    GradTcSmem<DK>& S = *reinterpret_cast<GradTcSmem<DK>*>(gt_dyn);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t N = g.N, Np = g.Np;
    const int64_t r0 = ((int64_t)blockIdx.x + g.bx0) * kGTRows;
    const int64_t i0 = (int64_t)blockIdx.y * g.i_per_split, i1 = min(N, i0 + g.i_per_split);
    const int ntiles = i0 < i1 ? (int)((i1 - i0 + C::PT - 1) / C::PT) : 0;
    const uint32_t* xh = g.xsplit;
    const uint32_t* xl = g.xsplit + Np * DK;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&S.full[s]), 1);
            mbar_init(smem_u32(&S.empty[s]), 1 + kGTEpi);   // its MMAs and every epilogue warp
            mbar_init(smem_u32(&S.tfull[s]), 1);
            mbar_init(smem_u32(&S.tempty[s]), kGTEpi);
        }
        mbar_init(smem_u32(&S.afull), 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&S.tmem_base), 2 * C::PT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = S.tmem_base;
    volatile int* abort_flag = &S.abort;

    if (warp == 0) {
        if (lane == 0) {
            // the CTA's rows, then the first two point tiles
            const uint32_t ab = smem_u32(&S.afull);
            mbar_arrive_expect_tx(ab, 2u * C::A_WORDS * 4u);
            bulk_g2s(smem_u32(S.ah), xh + CDE_CK(r0, Np - kGTRows + 1, 411) * DK, C::A_WORDS * 4u, ab);
            bulk_g2s(smem_u32(S.al), xl + r0 * DK, C::A_WORDS * 4u, ab);
            for (int k = 0; k < 2 && k < ntiles; ++k) grad_tc_load<DK>(g, S, k, i0 + (int64_t)k * C::PT);
            constexpr uint32_t idesc = tc_idesc_tf32(kGTRows, C::PT);
            bool ok = mbar_wait(ab, 0, abort_flag, g.err, 0x100);
            for (int k = 0; k < ntiles && ok; ++k) {
                const int s = k & 1, b = k & 1;
                const uint32_t ph = (uint32_t)(k >> 1) & 1u;
                ok = mbar_wait(smem_u32(&S.full[s]), ph, abort_flag, g.err, 0x200) &&
                     mbar_wait(smem_u32(&S.tempty[b]), ph ^ 1u, abort_flag, g.err, 0x400);
                if (!ok) break;
                tc_fence_after();
                const uint32_t dt = tbase + (uint32_t)(b * C::PT);
#pragma unroll
                for (int ks = 0; ks < DK / 8; ++ks) {
                    const uint64_t dah = tc_sdesc(smem_u32(S.ah) + 256 * ks, 128, C::SBO);
                    const uint64_t dal = tc_sdesc(smem_u32(S.al) + 256 * ks, 128, C::SBO);
                    const uint64_t dbh = tc_sdesc(smem_u32(S.bh[s]) + 256 * ks, 128, C::SBO);
                    const uint64_t dbl = tc_sdesc(smem_u32(S.bl[s]) + 256 * ks, 128, C::SBO);
                    tc_mma_tf32(dt, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                    tc_mma_tf32(dt, dah, dbl, idesc, 1u);
                    tc_mma_tf32(dt, dal, dbh, idesc, 1u);
                }
                tc_commit(smem_u32(&S.empty[s]));
                tc_commit(smem_u32(&S.tfull[b]));
                // tile k + 1 into the other stage once tile k - 1's MMAs and epilogue are done
                // with it (MMA k is already queued, so the tensor cores do not wait on this)
                if (k >= 1 && k + 1 < ntiles) {
                    const int sp = (k - 1) & 1;
                    ok = mbar_wait(smem_u32(&S.empty[sp]), (uint32_t)((k - 1) >> 1) & 1u, abort_flag, g.err, 0x800);
                    if (!ok) break;
                    grad_tc_load<DK>(g, S, sp, i0 + (int64_t)(k + 1) * C::PT);
                }
            }
            // every copy this thread started has been waited for (full) or was never
            // started; the last two tiles' stage releases (their MMAs and epilogues)
            if (ok && ntiles > 0) {
                for (int k = ntiles - 2 < 0 ? 0 : ntiles - 2; k < ntiles; ++k)
                    mbar_wait(smem_u32(&S.empty[k & 1]), (uint32_t)(k >> 1) & 1u, abort_flag, g.err, 0x800);
            }
        }
        __syncwarp();
    } else {
        // epilogue: TMEM lane quadrant q (its 32 rows), column block cb of every tile
        const int e = warp - 1, q = warp & 3, cb = e >> 2;
        const int64_t jr = r0 + 32 * q + lane;
        const int j = (int)jr;   // N < 2^31
        const int64_t jc = jr < N ? jr : 0;
        const float nj = g.xnorm[jc], yj = g.y[jc];
        const float am = g.a1 * g.mx[jc], bm = g.a2 * g.my[jc];
        float2 SA = make_float2(0.f, 0.f), SAx = SA, SAy = SA, SB = SA, SBx = SA;
        for (int k = 0; k < ntiles; ++k) {
            const int b = k & 1;
            if (!mbar_wait(smem_u32(&S.tfull[b]), (uint32_t)(k >> 1) & 1u, abort_flag, g.err, 0x1000)) break;
            tc_fence_after();
            const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * C::PT + cb * C::COLS);
            const int64_t p0 = i0 + (int64_t)k * C::PT + cb * C::COLS;
            const float* ns = &S.ny[k & 1][0][cb * C::COLS];
            const float* ys = &S.ny[k & 1][1][cb * C::COLS];
#pragma unroll
            for (int h = 0; h < C::COLS / 32; ++h) {
                float dot[32];
                tmem_ld32(ta + 32 * h, dot);
                tmem_wait_ld();
                if (h == C::COLS / 32 - 1) {   // all of this warp's columns are in registers: release the buffer
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&S.tempty[b]));
                }
                const int64_t pb = p0 + 32 * h, jlo = r0 + 32 * q;   // warp-uniform
                if (pb + 32 > i1 || (pb < jlo + 32 && pb + 32 > jlo))
                    grad_tc_columns<KERN, 32, true>(g, dot, ns + 32 * h, ys + 32 * h, pb, i1, j, nj, yj, am, bm, SA,
                                                    SAx, SAy, SB, SBx);
                else
                    grad_tc_columns<KERN, 32, false>(g, dot, ns + 32 * h, ys + 32 * h, pb, i1, j, nj, yj, am, bm, SA,
                                                     SAx, SAy, SB, SBx);
            }
            __syncwarp();   // this warp is done with the stage's norms and y
            if (lane == 0) mbar_arrive(smem_u32(&S.empty[k & 1]));
        }
        S.red[e][0][lane] = SA.x + SA.y;
        S.red[e][1][lane] = SAx.x + SAx.y;
        S.red[e][2][lane] = SAy.x + SAy.y;
        S.red[e][3][lane] = SB.x + SB.y;
        S.red[e][4][lane] = SBx.x + SBx.y;
        asm volatile("bar.sync 1, %0;" ::"r"(kGTEpi * 32) : "memory");   // the epilogue warps only
        if (cb == 0 && jr < N) {
            float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 4; ++c) {   // column blocks in order
                const int ee = 4 * c + (e & 3);
#pragma unroll
                for (int m = 0; m < 5; ++m) v[m] += S.red[ee][m][lane];
            }
            float* pp = g.part + ((int64_t)blockIdx.y * N + jr) * 6;
            pp[0] = 0.f;
            pp[1] = v[0];
            pp[2] = v[1];
            pp[3] = v[2];
            pp[4] = v[3];
            pp[5] = v[4];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 2 * C::PT);
    }
}

// Per row: merge split partials (FP64, split order), then
// rowv[j] = {ell_j, d ell_j/d ln h1, d ell_j/d ln h2}.  Gaussian rows whose
// numerator sum fell below 2^-40 are listed for k_grad_fallback instead.
__global__ void k_grad_rows(const float* __restrict__ part, int n_split, int64_t N,
                            const float* __restrict__ my, float a2f, double h1, double h2,
                            int epan, double lnc1, double* __restrict__ rowv, int* __restrict__ fb_count,
                            int* __restrict__ fb_rows) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double SA = 0, SAx = 0, SAy = 0, SB = 0, SBx = 0;
    for (int s = 0; s < n_split; ++s) {
        const float* p = part + ((int64_t)s * N + j) * 6;
        SA += p[1];
        SAx += p[2];
        SAy += p[3];
        SB += p[4];
        SBx += p[5];
    }
    const double LN2 = 0.69314718055994530942, LNS2PI = 0.91893853320467274178;
    double ell, g1, g2;
    if (epan) {
        // slots: sum u w, sum v w, sum u z, sum u, sum v
        const bool live = SA > 0.0;
        ell = live ? log(SA) - log(SB) - (log(h2) - lnc1) : -INFINITY;
        g1 = live ? SAx / SA - SBx / SB : 0.0;
        g2 = live ? SAy / SA - 1.0 : 0.0;
    } else {
        if (!(SA >= 0x1p-40)) {
            fb_rows[CDE_CK(atomicAdd(fb_count, 1), N, 404)] = (int)j;
            return;
        }
        ell = log(SA) - log(SB) - LN2 * (double)a2f * (double)my[j] - (LNS2PI + log(h2));
        g1 = (SAx / SA - SBx / SB) / (h1 * h1);
        g2 = (SAy / SA) / (h2 * h2) - 1.0;
    }
    rowv[3 * j] = ell;
    rowv[3 * j + 1] = g1;
    rowv[3 * j + 2] = g2;
}

// Exact recomputation of the listed Gaussian rows (one CTA per row, rows
// strided over the grid): every i with the online joint shift, thread partials
// merged with a common shift in a fixed order.
constexpr int kFbThreads = 256;

__device__ __forceinline__ void merge_shifted(float& M, float (&S)[5], float Mo, const float (&So)[5]) {
    const float Mm = fminf(M, Mo);
    const float r = (M == Mm) ? 1.f : ex2g(Mm - M);    // the side at the minimum keeps its scale
    const float ro = (Mo == Mm) ? 1.f : ex2g(Mm - Mo);
#pragma unroll
    for (int q = 0; q < 3; ++q) S[q] = S[q] * r + So[q] * ro;
    S[3] += So[3];  // the denominator sums carry no joint shift
    S[4] += So[4];
    M = Mm;
}

__global__ void __launch_bounds__(kFbThreads) k_grad_fallback(const GradArgs g, const int* __restrict__ fb_count,
                                                               const int* __restrict__ fb_rows, double h1,
                                                               double h2, double* __restrict__ rowv) {
    __shared__ float xj_s[kMaxD];
    __shared__ float redM[kFbThreads / 32], redS[kFbThreads / 32][5];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = *fb_count;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        const int j = (int)CDE_CK(fb_rows[r], g.N, 403);
        __syncthreads();
        for (int c = tid; c < g.d; c += kFbThreads) xj_s[c] = g.xs[(int64_t)c * g.Np + j];
        __syncthreads();
        const float yj = g.y[j], mx = g.mx[j], my = g.my[j];
        float M = INFINITY, S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int64_t i = tid; i < g.N; i += kFbThreads) {
            float dx2 = 0.f;
            for (int c = 0; c < g.d; ++c) {
                const float q = xj_s[c] - g.xs[(int64_t)c * g.Np + i];
                dx2 = fmaf(q, q, dx2);
            }
            const float dy = yj - g.y[i];
            grad_accumulate_joint(i != j, dx2, dy * dy, mx, my, g.a1, g.a2, M, S[0], S[1], S[2], S[3], S[4]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float So[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) So[q] = __shfl_xor_sync(0xffffffffu, S[q], o);
            merge_shifted(M, S, __shfl_xor_sync(0xffffffffu, M, o), So);
        }
        if (lane == 0) {
            redM[warp] = M;
#pragma unroll
            for (int q = 0; q < 5; ++q) redS[warp][q] = S[q];
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kFbThreads / 32; ++w) {
                float So[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) So[q] = redS[w][q];
                merge_shifted(M, S, redM[w], So);
            }
            const double LN2 = 0.69314718055994530942, LNS2PI = 0.91893853320467274178;
            const double SA = S[0], SAx = S[1], SAy = S[2], SB = S[3], SBx = S[4];
            rowv[3 * (int64_t)j] = log(SA) - log(SB) - LN2 * ((double)M + (double)g.a2 * (double)my) -
                                   (LNS2PI + log(h2));
            rowv[3 * (int64_t)j + 1] = (SAx / SA - SBx / SB) / (h1 * h1);
            rowv[3 * (int64_t)j + 2] = (SAy / SA) / (h2 * h2) - 1.0;
        }
    }
}

// Fixed-order sum of the per-row triples: one CTA of 1024 threads.
__global__ void k_sum_rows3(const double* __restrict__ rowv, int64_t N, double* __restrict__ out3) {
    __shared__ double red[3][1024];
    double s0 = 0, s1 = 0, s2 = 0;
    for (int64_t j = threadIdx.x; j < N; j += 1024) {
        s0 += rowv[3 * j];
        s1 += rowv[3 * j + 1];
        s2 += rowv[3 * j + 2];
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) out3[threadIdx.x] = red[threadIdx.x][0];
}

template <int JB, int DREG>
static void launch_grad(const GradArgs& g, dim3 grid, cudaStream_t st, bool epan) {
    if (epan) k_loo_grad<JB, DREG, 1><<<grid, kGradThreads, 0, st>>>(g);
    else k_loo_grad<JB, DREG, 0><<<grid, kGradThreads, 0, st>>>(g);
}

template <int DK>
static int launch_grad_tc(const GradArgs& g, dim3 grid, cudaStream_t st, bool epan) {
    const size_t smem = sizeof(GradTcSmem<DK>);
    static std::atomic<uint64_t> attr0{0}, attr1{0};   // per instantiation
    CDE_CUDA(smem_attr_once(attr0, k_grad_tc<DK, 0>, (int)smem));
    CDE_CUDA(smem_attr_once(attr1, k_grad_tc<DK, 1>, (int)smem));
    if (epan) k_grad_tc<DK, 1><<<grid, kGTThreads, smem, st>>>(g);
    else k_grad_tc<DK, 0><<<grid, kGTThreads, smem, st>>>(g);
    return CDE_OK;
}

// Resident CTAs per SM of the SIMT gradient kernel (the Gaussian instantiation;
// the Epanechnikov one uses no more registers), queried once per instantiation.
template <int JB, int DREG>
static int grad_simt_ctas_per_sm() {
    static std::atomic<int> n{0};
    int v = n.load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_loo_grad<JB, DREG, 0>, kGradThreads, 0) !=
                cudaSuccess || v < 1)
            v = 1;
        n.store(v, std::memory_order_relaxed);
    }
    return v;
}

// Point splits: the count, among those that leave every CTA at least 8 point
// tiles, whose CTAs fill the last wave of `slots` resident CTAs best (one CTA
// per SM for k_grad_tc; the occupancy of k_loo_grad).
static int64_t grad_splits(int64_t row_ctas, int64_t tiles, int64_t slots) {
    int64_t best = 1;
    double best_eff = -1.0;
    for (int64_t ns = 1; ns <= 16; ++ns) {
        const int64_t per = (tiles + ns - 1) / ns;
        if (ns > 1 && per < 8) break;
        const int64_t n_eff = (tiles + per - 1) / per, ctas = row_ctas * n_eff;
        const int64_t waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = ns;
        }
    }
    return best;
}

// A gradient evaluation as a sequence of launches over ranges of row blocks.
// Every (row block, point split) writes its own partial and the per-row
// merge and the sums run once at the end, so the result does not depend on
// how the row blocks are split over launches (the request loop runs
// gradient steps this way, so queued density jobs run in between).
struct GradChunked {
    GradArgs g;
    bool tc, epan;
    int DREG, DK;
    int64_t gx, ns, next_bx;
    int64_t slots;     // resident CTAs of the GPU for this kernel
    double h1, h2;
    double* rowv;
    bool own_rowv;
    int* fb;
};

int grad_chunked_create(cde_ctx* ctx, const Dataset& D, double h1, double h2, cudaStream_t st, double* d_rowv_ext,
                        GradChunked** out) {
    auto* c = new GradChunked{};
    GradArgs& g = c->g;
    g.xs = D.xs;
    g.y = D.y;
    g.mx = D.mx;
    g.my = D.my;
    g.N = D.N;
    g.Np = D.Np;
    g.d = D.d;
    const double L2E = 1.4426950408889634074;
    c->epan = D.kernel == CDE_KERNEL_EPAN;
    c->h1 = h1;
    c->h2 = h2;
    g.a1 = (float)(c->epan ? 1.0 / (h1 * h1) : L2E / (2 * h1 * h1));
    g.a2 = (float)(c->epan ? 1.0 / (h2 * h2) : L2E / (2 * h2 * h2));
    c->tc = D.d >= 16;   // tensor-core cross term
    c->DREG = D.d <= 4 ? 4 : D.d <= 8 ? 8 : D.d <= 16 ? 16 : D.d <= 32 ? 32 : 64;
    c->DK = D.d <= 16 ? 16 : D.d <= 32 ? 32 : 64;
    const int JB = c->DREG <= 8 ? 4 : c->DREG <= 32 ? 2 : 1;
    const int64_t rows_per_cta = c->tc ? (int64_t)kGTRows : (int64_t)kGradThreads * JB;
    const int tile = c->tc ? (c->DK <= 32 ? 256 : 128) : kGradThreads;
    c->gx = (D.N + rows_per_cta - 1) / rows_per_cta;
    const int64_t tiles = (D.N + tile - 1) / tile;
    int64_t ns;
    if (c->tc) {
        c->slots = ctx->sm_count;
    } else {
        const int per_sm = c->DREG == 4 ? grad_simt_ctas_per_sm<4, 4>()
                           : c->DREG == 8 ? grad_simt_ctas_per_sm<4, 8>() : grad_simt_ctas_per_sm<2, 16>();
        c->slots = (int64_t)per_sm * ctx->sm_count;
    }
    ns = grad_splits(c->gx, tiles, c->slots);
    if (ns > tiles) ns = tiles;
    if (ns < 1) ns = 1;
    const int64_t tiles_per = (tiles + ns - 1) / ns;
    g.i_per_split = tiles_per * tile;
    c->ns = (tiles + tiles_per - 1) / tiles_per;
    c->next_bx = 0;
    c->rowv = d_rowv_ext;
    c->own_rowv = d_rowv_ext == nullptr;
    int rc = CDE_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        rc = cuda_error(e, what);
        return rc;
    };
    cudaError_t e = cudaMallocAsync((void**)&g.part, (size_t)c->ns * D.N * 6 * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&c->fb, (size_t)(D.N + 1) * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->fb, 0, sizeof(int), st);
    if (e == cudaSuccess && c->own_rowv) e = cudaMallocAsync((void**)&c->rowv, (size_t)D.N * 3 * sizeof(double), st);
    if (e == cudaSuccess && c->tc) {
        uint32_t* xsplit = nullptr;
        float* xnorm = nullptr;
        e = cudaMallocAsync((void**)&xsplit, (size_t)2 * D.Np * c->DK * sizeof(uint32_t), st);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&xnorm, (size_t)D.Np * sizeof(float), st);
        g.xsplit = xsplit;
        g.xnorm = xnorm;
        g.err = ctx->d_err + kErrTensorWait;
        if (e == cudaSuccess) {
            const unsigned sb = (unsigned)(D.Np / 32);
            if (c->DK == 16) k_grad_split_tc<16><<<sb, 256, 0, st>>>(D.xs, D.Np, D.d, xsplit, xnorm);
            else if (c->DK == 32) k_grad_split_tc<32><<<sb, 256, 0, st>>>(D.xs, D.Np, D.d, xsplit, xnorm);
            else k_grad_split_tc<64><<<sb, 256, 0, st>>>(D.xs, D.Np, D.d, xsplit, xnorm);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        fail(e, "gradient: scratch");
        grad_chunked_free(c, st);
        return rc;
    }
    *out = c;
    return CDE_OK;
}

// Launch the next range of row blocks: about `pair_evals` pairs, and at least
// enough row blocks to fill the GPU with their point splits; pair_evals <= 0:
// all the rest.  *done once every row block has been launched.
int grad_chunked_next(GradChunked* c, double pair_evals, cudaStream_t st, int* done) {
    const int64_t rows_per_block = c->tc ? (int64_t)kGTRows : (int64_t)kGradThreads * (c->DREG <= 8 ? 4 : c->DREG <= 32 ? 2 : 1);
    const double per_block = (double)rows_per_block * (double)c->g.N;
    int64_t nb = c->gx - c->next_bx;
    if (pair_evals > 0 && pair_evals < per_block * (double)nb) {
        const int64_t fill = (c->slots + c->ns - 1) / c->ns;
        nb = std::max<int64_t>((int64_t)std::ceil(pair_evals / per_block), fill);
        nb = std::min(nb, c->gx - c->next_bx);
    }
    GradArgs g = c->g;
    g.bx0 = c->next_bx;
    const dim3 grid((unsigned)nb, (unsigned)c->ns);
    if (c->tc) {
        const int rl = c->DK == 16 ? launch_grad_tc<16>(g, grid, st, c->epan)
                       : c->DK == 32 ? launch_grad_tc<32>(g, grid, st, c->epan)
                                     : launch_grad_tc<64>(g, grid, st, c->epan);
        if (rl != CDE_OK) return rl;
    } else {
        if (c->DREG == 4) launch_grad<4, 4>(g, grid, st, c->epan);
        else if (c->DREG == 8) launch_grad<4, 8>(g, grid, st, c->epan);
        else launch_grad<2, 16>(g, grid, st, c->epan);
    }
    CDE_CUDA(cudaGetLastError());
    c->next_bx += nb;
    *done = c->next_bx >= c->gx;
    return CDE_OK;
}

void grad_chunked_free(GradChunked* c, cudaStream_t st) {
    if (!c) return;
    if (c->g.part) cudaFreeAsync(c->g.part, st);
    if (c->fb) cudaFreeAsync(c->fb, st);
    if (c->g.xsplit) cudaFreeAsync(const_cast<uint32_t*>(c->g.xsplit), st);
    if (c->g.xnorm) cudaFreeAsync(const_cast<float*>(c->g.xnorm), st);
    if (c->own_rowv && c->rowv) cudaFreeAsync(c->rowv, st);
    delete c;
}

// After the last range: the per-row merge, the exact recomputation of listed
// rows, and (d_out3) the fixed-order sums; frees the sequence.
int grad_chunked_finish(cde_ctx* ctx, GradChunked* c, double* d_out3, cudaStream_t st) {
    const GradArgs& g = c->g;
    k_grad_rows<<<(unsigned)((g.N + 255) / 256), 256, 0, st>>>(g.part, (int)c->ns, g.N, g.my, g.a2, c->h1, c->h2,
                                                             c->epan ? 1 : 0, epan_log_norm(1), c->rowv, c->fb,
                                                             c->fb + 1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !c->epan) {
        // listed rows only; exits at once when the list is empty
        k_grad_fallback<<<2 * ctx->sm_count, kFbThreads, 0, st>>>(g, c->fb, c->fb + 1, c->h1, c->h2, c->rowv);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && d_out3) {
        k_sum_rows3<<<1, 1024, 0, st>>>(c->rowv, g.N, d_out3);
        e = cudaGetLastError();
    }
    grad_chunked_free(c, st);
    if (e != cudaSuccess) return cuda_error(e, "gradient: final kernels");
    return CDE_OK;
}

int loo_grad_enqueue(cde_ctx* ctx, const Dataset& D, double h1, double h2, double* d_out3,
                     cudaStream_t st, double* d_rowv_ext) {
    timing_reset(ctx);
    GradChunked* c = nullptr;
    int rc = grad_chunked_create(ctx, D, h1, h2, st, d_rowv_ext, &c);
    if (rc != CDE_OK) return rc;
    int done = 0;
    timing_begin(ctx, st);
    rc = grad_chunked_next(c, 0.0, st, &done);   // all row blocks in one launch
    timing_end(ctx, st);
    if (rc != CDE_OK) {
        grad_chunked_free(c, st);
        return rc;
    }
    return grad_chunked_finish(ctx, c, d_out3, st);
}

#ifdef CDE_CHECKS
CDE_CHECK_READER(check_status_grad)
#endif

}  // namespace cde

using namespace cde;

// After a synchronous d >= 16 call: a bounded tensor-core wait that ran out on
// the device (k_grad_tc) becomes CDE_ETIMEOUT, and the report is cleared.
static int grad_wait_status(cde_ctx* ctx, const Dataset& D, cudaStream_t st, const char* who) {
    if (D.d < 16) return CDE_OK;
    int tw = 0;
    CDE_CUDA(cudaMemcpyAsync(&tw, ctx->d_err + kErrTensorWait, sizeof(int), cudaMemcpyDeviceToHost, st));
    CDE_CUDA(cudaStreamSynchronize(st));
    if (!tw) return CDE_OK;
    CDE_CUDA(cudaMemsetAsync(ctx->d_err + kErrTensorWait, 0, sizeof(int), st));
    return set_error(CDE_ETIMEOUT, std::string(who) + ": a tensor-core wait ran out on the device");
}

extern "C" int cde_loo_grad(cde_ctx* ctx, cde_dataset ds, double h1, double h2, double* out3,
                            int flags, void* stream) {
    CDE_NVTX("cde_loo_grad");
    if (!ctx || !out3) return set_error(CDE_EINVAL, "cde_loo_grad: null argument");
    if (!std::isfinite(h1) || !std::isfinite(h2) || h1 < 1e-12 || h2 < 1e-12 || h1 > 1e12 || h2 > 1e12)
        return set_error(CDE_EINVAL, "cde_loo_grad: bandwidth must be finite in [1e-12, 1e12]");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_loo_grad: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    if (flags & CDE_OUT_DEVICE) return loo_grad_enqueue(ctx, *D, h1, h2, out3, st, nullptr);
    double* dout = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&dout, 3 * sizeof(double), st));
    int rc = loo_grad_enqueue(ctx, *D, h1, h2, dout, st, nullptr);
    cudaError_t e = cudaSuccess;
    if (rc == CDE_OK) e = cudaMemcpyAsync(out3, dout, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dout, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (rc != CDE_OK) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cde_loo_grad: copy");
    if (e2 != cudaSuccess) return cuda_error(e2, "cde_loo_grad: kernels");
    return grad_wait_status(ctx, *D, st, "cde_loo_grad");
}

extern "C" int cde_loo_grad_rows(cde_ctx* ctx, cde_dataset ds, double h1, double h2, double* rows_out,
                                 void* stream) {
    CDE_NVTX("cde_loo_grad_rows");
    if (!ctx || !rows_out) return set_error(CDE_EINVAL, "cde_loo_grad_rows: null argument");
    if (!std::isfinite(h1) || !std::isfinite(h2) || h1 < 1e-12 || h2 < 1e-12 || h1 > 1e12 || h2 > 1e12)
        return set_error(CDE_EINVAL, "cde_loo_grad_rows: bandwidth must be finite in [1e-12, 1e12]");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_loo_grad_rows: unknown dataset");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    double* rowv = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&rowv, (size_t)D->N * 3 * sizeof(double), st));
    int rc = loo_grad_enqueue(ctx, *D, h1, h2, nullptr, st, rowv);
    cudaError_t e = cudaSuccess;
    if (rc == CDE_OK)
        e = cudaMemcpyAsync(rows_out, rowv, (size_t)D->N * 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(rowv, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (rc != CDE_OK) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cde_loo_grad_rows: copy");
    if (e2 != cudaSuccess) return cuda_error(e2, "cde_loo_grad_rows: kernels");
    return grad_wait_status(ctx, *D, st, "cde_loo_grad_rows");
}
