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

#include "cde_internal.h"

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

// One pair's contribution.  Gaussian: the separable shifted factors u, w and
// v = u w.  Epanechnikov: plain sums of the profiles and their log-derivative
// weights (the support test is the profile itself being positive).
template <int KERN>
__device__ __forceinline__ void grad_accumulate(bool ok, float dx2, float dy2, float mx, float my,
                                                float a1, float a2, float& SA, float& SAx,
                                                float& SAy, float& SB, float& SBx) {
    if constexpr (KERN == 1) {
        const float u = ok ? fma_sat_g(-a1, dx2, 1.f) : 0.f;
        const float w = fma_sat_g(-a2, dy2, 1.f);
        const float v = u > 0.f ? 2.f * a1 * dx2 : 0.f;
        const float z = w > 0.f ? 2.f * a2 * dy2 : 0.f;
        SA = fmaf(u, w, SA);
        SAx = fmaf(v, w, SAx);
        SAy = fmaf(u, z, SAy);
        SB += u;
        SBx += v;
        return;
    }
    const float u = ok ? ex2g(-a1 * (dx2 - mx)) : 0.f;
    const float v = u * ex2g(-a2 * (dy2 - my));
    SB += u;
    SBx = fmaf(u, dx2, SBx);
    SA += v;
    SAx = fmaf(v, dx2, SAx);
    SAy = fmaf(v, dy2, SAy);
}

template <int JB, int DREG, int KERN>
__global__ void __launch_bounds__(kGradThreads) k_loo_grad(const GradArgs g) {
    __shared__ __align__(16) float xt[kGradThreads][DREG];  // point-major: 128-bit broadcast loads
    __shared__ float yt[kGradThreads];
    const int tid = threadIdx.x;
    const int64_t jbase = (int64_t)blockIdx.x * kGradThreads * JB + tid;
    const int64_t i0 = (int64_t)blockIdx.y * g.i_per_split;
    const int64_t i1 = min(g.N, i0 + g.i_per_split);
    const int d = g.d;
    float xj[JB][DREG], yj[JB], mxj[JB], myj[JB];
    float SA[JB], SAx[JB], SAy[JB], SB[JB], SBx[JB];
    int64_t jj[JB];
#pragma unroll
    for (int b = 0; b < JB; ++b) {
        const int64_t j = jbase + (int64_t)b * kGradThreads;
        const int64_t jc = j < g.N ? j : 0;
        jj[b] = j;
#pragma unroll
        for (int c = 0; c < DREG; ++c) xj[b][c] = c < d ? g.xs[(int64_t)c * g.Np + jc] : 0.f;
        yj[b] = g.y[jc];
        mxj[b] = g.mx[jc];
        myj[b] = g.my[jc];
        SA[b] = SAx[b] = SAy[b] = SB[b] = SBx[b] = 0.f;
    }
    const float a1 = g.a1, a2 = g.a2;
    for (int64_t t0 = i0; t0 < i1; t0 += kGradThreads) {
        __syncthreads();
        const int64_t it = CDE_CK(t0 + tid, g.Np, 401);  // < Np: i_per_split and Np are multiples of 128
#pragma unroll
        for (int c = 0; c < DREG; ++c) xt[tid][c] = c < d ? g.xs[(int64_t)c * g.Np + it] : 0.f;
        yt[tid] = g.y[it];
        __syncthreads();
        const int n = (int)min((int64_t)kGradThreads, i1 - t0);
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
            for (int b = 0; b < JB; ++b) {
                float dx2 = 0.f;
#pragma unroll
                for (int c = 0; c < DREG; ++c) {
                    const float q = xj[b][c] - xi[c];
                    dx2 = fmaf(q, q, dx2);
                }
                const float dy = yj[b] - yi;
                const float dy2 = dy * dy;
                grad_accumulate<KERN>(i32 != (int)jj[b], dx2, dy2, mxj[b], myj[b], a1, a2, SA[b], SAx[b],
                                      SAy[b], SB[b], SBx[b]);
            }
        }
    }
#pragma unroll
    for (int b = 0; b < JB; ++b) {
        if (jj[b] >= g.N) continue;
        float* p = g.part + ((int64_t)blockIdx.y * g.N + jj[b]) * 6;
        p[0] = 0.f;  // no running shift on this path
        p[1] = SA[b];
        p[2] = SAx[b];
        p[3] = SAy[b];
        p[4] = SB[b];
        p[5] = SBx[b];
    }
}

// ---------------------------------------------------------------------------
// d >= 16: the x cross-term on the tensor cores.  |x_j - x_i|^2 =
// n_j + n_i - 2 x_j.x_i with the dot products of a 16-row x 8-point tile from
// m16n8k8 TF32 MMAs on split operands (x = hi + lo, products hi*hi + hi*lo +
// lo*hi, FP32 accumulation), norms n in FP32, the result clamped at 0.  Each
// warp owns 16 rows (their split fragments stay in registers); the CTA stages
// 64 points at a time, already split, in shared memory.
// ---------------------------------------------------------------------------
constexpr int kGMWarps = 4, kGMTile = 64;

__device__ __forceinline__ void split_tf32_g(float v, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(v) & 0xffffe000u;
    lo = __float_as_uint(v - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32_g(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int DK, int KERN>
__global__ void __launch_bounds__(kGMWarps * 32) k_loo_grad_mma(const GradArgs g) {
    constexpr int KK = DK / 8, RS = DK + 4;  // padded smem row (bank spread)
    __shared__ uint32_t xh[kGMTile * RS], xl[kGMTile * RS];
    __shared__ float ni_s[kGMTile], yi_s[kGMTile];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gq = lane >> 2, t = lane & 3;
    const int d = g.d;
    const int64_t N = g.N, Np = g.Np;
    const int64_t i0 = (int64_t)blockIdx.y * g.i_per_split;
    const int64_t i1 = min(N, i0 + g.i_per_split);
    int64_t jr[2];
    float nj[2], yj[2], mxj[2], myj[2];
    uint32_t ah[KK][4], al[KK][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t j = (int64_t)blockIdx.x * (kGMWarps * 16) + warp * 16 + gq + 8 * h;
        jr[h] = j;
        const int64_t jc = j < N ? j : 0;
        float n = 0.f;
        for (int c = 0; c < d; ++c) {
            const float v = g.xs[(int64_t)c * Np + jc];
            n = fmaf(v, v, n);
        }
        nj[h] = n;
        yj[h] = g.y[jc];
        mxj[h] = g.mx[jc];
        myj[h] = g.my[jc];
#pragma unroll
        for (int kk = 0; kk < KK; ++kk) {
            const int c0 = 8 * kk + t, c1 = c0 + 4;
            const float v0 = c0 < d ? g.xs[(int64_t)c0 * Np + jc] : 0.f;
            const float v1 = c1 < d ? g.xs[(int64_t)c1 * Np + jc] : 0.f;
            split_tf32_g(v0, ah[kk][h], al[kk][h]);        // a0 / a1: (row g [+8], k t)
            split_tf32_g(v1, ah[kk][2 + h], al[kk][2 + h]); // a2 / a3: (row g [+8], k t+4)
        }
    }
    const float a1 = g.a1, a2 = g.a2;
    float SA[2] = {0, 0}, SAx[2] = {0, 0}, SAy[2] = {0, 0}, SB[2] = {0, 0},
          SBx[2] = {0, 0};
    for (int64_t t0 = i0; t0 < i1; t0 += kGMTile) {
        __syncthreads();
        for (int e = tid; e < DK * kGMTile; e += kGMWarps * 32) {
            const int c = e / kGMTile, p = e - c * kGMTile;
            const float v = c < d ? g.xs[(int64_t)c * Np + CDE_CK(t0 + p, Np, 402)] : 0.f;  // t0 + p < Np
            uint32_t hv, lv;
            split_tf32_g(v, hv, lv);
            xh[p * RS + c] = hv;
            xl[p * RS + c] = lv;
        }
        if (tid < kGMTile) {
            float n = 0.f;
            for (int c = 0; c < d; ++c) {
                const float v = g.xs[(int64_t)c * Np + t0 + tid];
                n = fmaf(v, v, n);
            }
            ni_s[tid] = n;
            yi_s[tid] = g.y[t0 + tid];
        }
        __syncthreads();
        // 4 n-tiles (32 points) at a time: independent accumulators hide the MMA latency
#pragma unroll 1
        for (int n4 = 0; n4 < kGMTile / 32; ++n4) {
            float D[4][4];
#pragma unroll
            for (int n = 0; n < 4; ++n) D[n][0] = D[n][1] = D[n][2] = D[n][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < KK; ++kk) {
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    const int pr = (32 * n4 + 8 * n + gq) * RS + 8 * kk + t;
                    const uint32_t bh0 = xh[pr], bh1 = xh[pr + 4], bl0 = xl[pr], bl1 = xl[pr + 4];
                    mma_tf32_g(D[n], ah[kk], bh0, bh1);
                    mma_tf32_g(D[n], ah[kk], bl0, bl1);
                    mma_tf32_g(D[n], al[kk], bh0, bh1);
                }
            }
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int h = q >> 1, p = 32 * n4 + 8 * n + 2 * t + (q & 1);
                    const int64_t i = t0 + p;
                    const float dx2 = fmaxf(nj[h] + ni_s[p] - 2.f * D[n][q], 0.f);
                    const float dy = yj[h] - yi_s[p];
                    grad_accumulate<KERN>(i < i1 && i != jr[h], dx2, dy * dy, mxj[h], myj[h], a1, a2,
                                          SA[h], SAx[h], SAy[h], SB[h], SBx[h]);
                }
        }
    }
    // combine the 4 lanes that share a row (t = 0..3), fixed xor order
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[5] = {SA[h], SAx[h], SAy[h], SB[h], SBx[h]};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            v[q] += __shfl_xor_sync(0xffffffffu, v[q], 1);
            v[q] += __shfl_xor_sync(0xffffffffu, v[q], 2);
        }
        if (t == 0 && jr[h] < N) {
            float* pp = g.part + ((int64_t)blockIdx.y * N + jr[h]) * 6;
            pp[0] = 0.f;
            pp[1] = v[0];
            pp[2] = v[1];
            pp[3] = v[2];
            pp[4] = v[3];
            pp[5] = v[4];
        }
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
static void launch_grad_mma(const GradArgs& g, dim3 grid, cudaStream_t st, bool epan) {
    if (epan) k_loo_grad_mma<DK, 1><<<grid, kGMWarps * 32, 0, st>>>(g);
    else k_loo_grad_mma<DK, 0><<<grid, kGMWarps * 32, 0, st>>>(g);
}

int loo_grad_enqueue(cde_ctx* ctx, const Dataset& D, double h1, double h2, double* d_out3,
                     cudaStream_t st, double* d_rowv_ext) {
    GradArgs g{};
    g.xs = D.xs;
    g.y = D.y;
    g.mx = D.mx;
    g.my = D.my;
    g.N = D.N;
    g.Np = D.Np;
    g.d = D.d;
    const double L2E = 1.4426950408889634074;
    const bool epan = D.kernel == CDE_KERNEL_EPAN;
    g.a1 = (float)(epan ? 1.0 / (h1 * h1) : L2E / (2 * h1 * h1));
    g.a2 = (float)(epan ? 1.0 / (h2 * h2) : L2E / (2 * h2 * h2));
    const bool tc = D.d >= 16;   // tensor-core cross term
    const int DREG = D.d <= 4 ? 4 : D.d <= 8 ? 8 : D.d <= 16 ? 16 : D.d <= 32 ? 32 : 64;
    const int JB = DREG <= 8 ? 4 : DREG <= 32 ? 2 : 1;
    const int64_t rows_per_cta = tc ? (int64_t)kGMWarps * 16 : (int64_t)kGradThreads * JB;
    const int tile = tc ? kGMTile : kGradThreads;
    const int64_t gx = (D.N + rows_per_cta - 1) / rows_per_cta;
    // split i so that the launch has about 8 CTAs per SM
    int64_t want = (tc ? 16LL : 8LL) * ctx->sm_count;
    int64_t ns = (want + gx - 1) / gx;
    const int64_t tiles = (D.N + tile - 1) / tile;
    if (ns > tiles) ns = tiles;
    if (ns < 1) ns = 1;
    const int64_t tiles_per = (tiles + ns - 1) / ns;
    g.i_per_split = tiles_per * tile;
    ns = (tiles + tiles_per - 1) / tiles_per;
    float* part = nullptr;
    double* rowv = d_rowv_ext;
    int* fb = nullptr;  // [0] count, then the listed rows
    CDE_CUDA(cudaMallocAsync((void**)&part, (size_t)ns * D.N * 6 * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&fb, (size_t)(D.N + 1) * sizeof(int), st));
    CDE_CUDA(cudaMemsetAsync(fb, 0, sizeof(int), st));
    if (!rowv) CDE_CUDA(cudaMallocAsync((void**)&rowv, (size_t)D.N * 3 * sizeof(double), st));
    g.part = part;
    dim3 grid((unsigned)gx, (unsigned)ns);
    if (tc) {
        if (D.d <= 16) launch_grad_mma<16>(g, grid, st, epan);
        else if (D.d <= 32) launch_grad_mma<32>(g, grid, st, epan);
        else launch_grad_mma<64>(g, grid, st, epan);
    } else if (DREG == 4) launch_grad<4, 4>(g, grid, st, epan);
    else if (DREG == 8) launch_grad<4, 8>(g, grid, st, epan);
    else launch_grad<2, 16>(g, grid, st, epan);
    CDE_CUDA(cudaGetLastError());
    k_grad_rows<<<(unsigned)((D.N + 255) / 256), 256, 0, st>>>(part, (int)ns, D.N, D.my, g.a2, h1, h2,
                                                             epan ? 1 : 0, epan_log_norm(1), rowv, fb, fb + 1);
    CDE_CUDA(cudaGetLastError());
    if (!epan) {
        // listed rows only; exits at once when the list is empty
        k_grad_fallback<<<2 * ctx->sm_count, kFbThreads, 0, st>>>(g, fb, fb + 1, h1, h2, rowv);
        CDE_CUDA(cudaGetLastError());
    }
    if (d_out3) {
        k_sum_rows3<<<1, 1024, 0, st>>>(rowv, D.N, d_out3);
        CDE_CUDA(cudaGetLastError());
    }
    CDE_CUDA(cudaFreeAsync(part, st));
    CDE_CUDA(cudaFreeAsync(fb, st));
    if (!d_rowv_ext) CDE_CUDA(cudaFreeAsync(rowv, st));
    return CDE_OK;
}

#ifdef CDE_CHECKS
CDE_CHECK_READER(check_status_grad)
#endif

}  // namespace cde

using namespace cde;

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
    return CDE_OK;
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
    return CDE_OK;
}
