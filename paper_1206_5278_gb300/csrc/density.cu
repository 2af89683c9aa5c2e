// Conditional density fhat(y|x) of Eq. 1 (Holmes, Gray & Isbell, Sec. 2) at
// Q query points x_q and a G-point y grid, over all N data points:
//
//   fhat(y_g | x_q) = sum_i K_h1(x_q - x_i) K_h2(y_g - y_i) / sum_i K_h1(x_q - x_i)
//                   = [sum_i u_qi w_ig] / [sum_i u_qi] / (sqrt(2 pi) h2)
//   u_qi = 2^{a1 (m_q - |x_q - x_i|^2)},  w_ig = 2^{-a2 (y_g - y_i)^2},
//
// m_q the query's nearest squared distance (so max_i u_qi = 1 and neither sum
// underflows), a = log2(e)/(2 h^2).  Epanechnikov datasets use the profiles
// u_qi = (1 - |x_q - x_i|^2/h1^2)_+ and w_ig = (1 - (y_g - y_i)^2/h2^2)_+ (no
// shift; a = 1/h^2) and the constant c_1/h2 = 3/(4 h2); a query with no
// x-neighbour inside h1 (0/0) gets f = 0.  The numerator is a (Q x N) x (N x G)
// product whose factors are generated on the fly; each CTA owns 32 queries x
// 256 grid points and runs the product on the tensor cores (k_density).  Small
// Q splits the data range across CTAs; split partials are summed in split
// order.
#include <cmath>

#include <cuda_bf16.h>

#include <cstdint>

#include "cde_internal.h"

namespace cde {

constexpr int kDQ = 32;    // queries per CTA
constexpr int kDG = 256;   // grid points per CTA
constexpr int kDIC = 32;   // data points per chunk

struct DensArgs {
    const float* xs;   // dataset [d][Np]
    const float* y;    // [Np]
    const float* xq;   // queries [d][Qp] (standardised like the data)
    const float* mq;   // [Q]
    const float* yg;   // [G]
    int64_t N, Np, Q, Qp;
    int d, G;
    float a1, a2;
    int64_t i_per_split;   // multiple of kDIC
    float* num;            // [n_split][Q][G]
    float* den;            // [n_split][Q]
};

__device__ __forceinline__ float ex2d(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a * b + c clamped to [0, 1] (the Epanechnikov profile in one instruction)
__device__ __forceinline__ float fma_sat_d(float a, float b, float c) {
    float r;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// x factor from its shared-memory argument: Gaussian 2^T (T = a1 (m_q - dx2),
// -inf masked), Epanechnikov (1 - a1 T)_+ (T = dx2, +inf masked)
template <int KERN>
__device__ __forceinline__ float dens_ufac(float T, float a1) {
    if constexpr (KERN == 0) return ex2d(T);
    else return fma_sat_d(-a1, T, 1.f);
}

// y factor at squared distance t2
template <int KERN>
__device__ __forceinline__ float dens_wfac(float t2, float a2) {
    if constexpr (KERN == 0) return ex2d(-a2 * t2);
    else return fma_sat_d(-a2, t2, 1.f);
}

__global__ void k_query_pack(const float* __restrict__ xq, int64_t Q, int64_t Qp, int d,
                             const double* __restrict__ mean, const double* __restrict__ sd,
                             float* __restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Qp) return;
    for (int c = 0; c < d; ++c)
        out[(int64_t)c * Qp + q] = q < Q ? (float)(((double)xq[q * d + c] - mean[c]) / sd[c]) : 0.f;
}

// per-query nearest squared distance to the data (same FP32 formula as the
// main kernel).  The data range is split over gridDim.y; split minima are
// merged with an integer atomicMin on the float bits (exact and order-free:
// squared distances are non-negative, so their bit patterns order like ints).
__global__ void __launch_bounds__(256) k_query_shift(const float* __restrict__ xs, int64_t N,
                                                     int64_t Np, int d, const float* __restrict__ xq,
                                                     int64_t Q, int64_t Qp, int64_t i_per_split,
                                                     unsigned int* __restrict__ mq_bits) {
    extern __shared__ float sm[];  // [d][256]
    const int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t ib = (int64_t)blockIdx.y * i_per_split;
    const int64_t ie = min(N, ib + i_per_split);
    float xqr[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xqr[c] = (q < Qp && c < d) ? xq[(int64_t)c * Qp + q] : 0.f;
    float best = INFINITY;
    for (int64_t i0 = ib; i0 < ie; i0 += 256) {
        __syncthreads();
        for (int c = 0; c < d; ++c) sm[c * 256 + threadIdx.x] = xs[(int64_t)c * Np + i0 + threadIdx.x];
        __syncthreads();
        const int n = (int)min((int64_t)256, ie - i0);
        if (q < Q)
            for (int tt = 0; tt < n; ++tt) {
                float dx2 = 0.f;
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < d) {
                        const float u = xqr[c] - sm[c * 256 + tt];
                        dx2 = fmaf(u, u, dx2);
                    }
                for (int c = 8; c < d; ++c) {
                    const float u = xq[(int64_t)c * Qp + q] - sm[c * 256 + tt];
                    dx2 = fmaf(u, u, dx2);
                }
                best = fminf(best, dx2);
            }
    }
    if (q < Q) atomicMin(mq_bits + q, __float_as_uint(best));
}

struct DensSmem {
    float T[kDQ][kDIC + 4];     // x factor argument (dens_ufac), masked points give 0
    uint4 Af[kDIC / 8][2][32];  // per chunk, k-step, m-tile, lane: TF32 A fragment (hi u)
    uint4 Ax[kDIC / 8][2][32];  //   and the BF16 cross-term A fragment [hi u | lo u]
    float yis[kDIC];
    float xqs[kMaxD][kDQ];
    float xis[kMaxD][kDIC];
    float dens[kDQ];
};

__device__ __forceinline__ void split_tf32_d(float v, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(v) & 0xffffe000u;
    lo = __float_as_uint(v - __uint_as_float(hi));
}

__device__ __forceinline__ uint32_t pack_bf16x2_d(float x, float y) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(x, y);  // x in the low half
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_d(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_tf32_d(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Numerator tile F[32 queries][256 grid points] += U[32 x IC] W[IC x 256] on
// the tensor cores with split operands v = hi + lo: hi*hi as TF32 m16n8k8, the
// two cross terms together as one BF16 m16n8k16 (about 2^-17 per term),
// A (u, M = queries) and B (w, N = grid points) operands; warp w owns grid
// points [32 w, 32 w + 32) and makes its B fragments in-lane with exp2.  Per chunk the 32 x IC
// arguments of u go to shared memory, then one thread per (k-step, m-tile,
// lane) slot turns them into the split A fragments (TF32 hi, BF16 [hi | lo])
// that every warp loads, so each u is evaluated once per CTA.  Each 32-point
// chunk accumulates from zero and is added to an FP32 running total.
template <int KERN>
__global__ void __launch_bounds__(256, 2) k_density(const DensArgs a) {
    extern __shared__ float4 dsm4[];
    DensSmem& S = *reinterpret_cast<DensSmem*>(dsm4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t q0 = (int64_t)blockIdx.x * kDQ;
    const int g0 = blockIdx.y * kDG;
    const int64_t s = blockIdx.z;
    const int64_t i_begin = s * a.i_per_split;
    const int64_t i_end = min(a.N, i_begin + a.i_per_split);
    const int d = a.d;
    for (int e = tid; e < d * kDQ; e += 256) {
        const int c = e / kDQ, qq = e % kDQ;
        S.xqs[c][qq] = (q0 + qq < a.Qp) ? a.xq[(int64_t)c * a.Qp + q0 + qq] : 0.f;
    }
    // distance-pass role: query dq, points dp..dp+3
    const int dq = tid >> 3, dp = (tid & 7) * 4;
    const float mqv = (KERN == 0 && q0 + dq < a.Q) ? a.mq[q0 + dq] : 0.f;
    float ygv[4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int gg = g0 + 32 * warp + 8 * nt + g;
        ygv[nt] = a.yg[gg < a.G ? gg : a.G - 1];
    }
    float Dt[2][4][4];
    // fragment-pass role (one thread per k-step, m-tile and lane slot): its two
    // queries' denominator partials, summed over its points of every chunk
    const int fks = tid >> 6, fmt = (tid >> 5) & 1;
    float bq0 = 0.f, bq1 = 0.f;
    float2 yg2[4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) yg2[nt] = make_float2(ygv[nt], ygv[nt]);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) Dt[mt][nt][0] = Dt[mt][nt][1] = Dt[mt][nt][2] = Dt[mt][nt][3] = 0.f;
    const float a1 = a.a1, a2 = a.a2;
    for (int64_t c0 = i_begin; c0 < i_end; c0 += kDIC) {
        __syncthreads();
        for (int e = tid; e < (d + 1) * kDIC; e += 256) {
            const int c = e / kDIC, ii = e % kDIC;
            const int64_t i = CDE_CK(c0 + ii, a.Np, 201);  // < Np
            if (c < d) S.xis[c][ii] = a.xs[(int64_t)c * a.Np + i];
            else S.yis[ii] = a.y[i];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int ii = dp + r;
            float dx2 = 0.f;
            for (int c = 0; c < d; ++c) {
                const float u = S.xqs[c][dq] - S.xis[c][ii];
                dx2 = fmaf(u, u, dx2);
            }
            if constexpr (KERN == 0) S.T[dq][ii] = (c0 + ii < i_end) ? a1 * (mqv - dx2) : -INFINITY;
            else S.T[dq][ii] = (c0 + ii < i_end) ? dx2 : INFINITY;
        }
        __syncthreads();
        // fragment pass: every x factor of the chunk once (not once per warp),
        // split hi + lo and packed into the A fragments the MMA pass loads
        {
            const int pa = 8 * fks + 2 * t, pb = pa + 1, r0 = 16 * fmt + g, r1 = r0 + 8;
            const float u0 = dens_ufac<KERN>(S.T[r0][pa], a1);   // (q, p0)
            const float u1 = dens_ufac<KERN>(S.T[r1][pa], a1);   // (q + 8, p0)
            const float u2 = dens_ufac<KERN>(S.T[r0][pb], a1);   // (q, p1)
            const float u3 = dens_ufac<KERN>(S.T[r1][pb], a1);   // (q + 8, p1)
            bq0 += u0 + u2;
            bq1 += u1 + u3;
            uint32_t h0, h1, h2, h3, l0, l1, l2, l3;
            split_tf32_d(u0, h0, l0);
            split_tf32_d(u1, h1, l1);
            split_tf32_d(u2, h2, l2);
            split_tf32_d(u3, h3, l3);
            S.Af[fks][fmt][lane] = make_uint4(h0, h1, h2, h3);
            S.Ax[fks][fmt][lane] = make_uint4(pack_bf16x2_d(__uint_as_float(h0), __uint_as_float(h2)),
                                              pack_bf16x2_d(__uint_as_float(h1), __uint_as_float(h3)),
                                              pack_bf16x2_d(__uint_as_float(l0), __uint_as_float(l2)),
                                              pack_bf16x2_d(__uint_as_float(l1), __uint_as_float(l3)));
        }
        __syncthreads();
        float D[2][4][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) D[mt][nt][0] = D[mt][nt][1] = D[mt][nt][2] = D[mt][nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < kDIC / 8; ++ks) {
            // this lane's two points of the k-step: p0 = 8 ks + 2t, p1 = p0 + 1
            const int pa = 8 * ks + 2 * t;
            uint32_t ah[2][4], ax[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const uint4 f = S.Af[ks][mt][lane], x = S.Ax[ks][mt][lane];
                ah[mt][0] = f.x;
                ah[mt][1] = f.y;
                ah[mt][2] = f.z;
                ah[mt][3] = f.w;
                ax[mt][0] = x.x;
                ax[mt][1] = x.y;
                ax[mt][2] = x.z;
                ax[mt][3] = x.w;
            }
            const float2 yab = *reinterpret_cast<const float2*>(&S.yis[pa]);
            const float2 nyab = make_float2(-yab.x, -yab.y);
            uint32_t bh[4][2], bx[4][2];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const float2 tt = __fadd2_rn(yg2[nt], nyab);   // (y_g - y_p0, y_g - y_p1)
                const float2 t2 = __fmul2_rn(tt, tt);
                const float w0 = dens_wfac<KERN>(t2.x, a2), w1 = dens_wfac<KERN>(t2.y, a2);
                const float2 h = make_float2(__uint_as_float(__float_as_uint(w0) & 0xffffe000u),
                                             __uint_as_float(__float_as_uint(w1) & 0xffffe000u));
                const float2 l = __ffma2_rn(h, make_float2(-1.f, -1.f), make_float2(w0, w1));  // exact
                bh[nt][0] = __float_as_uint(h.x);
                bh[nt][1] = __float_as_uint(h.y);
                bx[nt][0] = pack_bf16x2_d(l.x, l.y);
                bx[nt][1] = pack_bf16x2_d(h.x, h.y);
            }
            // hi*hi on TF32; both cross terms in one BF16 k16 MMA
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_tf32_d(D[mt][nt], ah[mt], bh[nt][0], bh[nt][1]);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16_d(D[mt][nt], ax[mt], bx[nt][0], bx[nt][1]);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) Dt[mt][nt][q] += D[mt][nt][q];
    }
    // denominators: a query's partials sit in the 4 lanes (t) of 4 warps (k-steps)
    // of its m-tile; sum t by shuffles, then the k-steps in order
    bq0 += __shfl_xor_sync(0xffffffffu, bq0, 1);
    bq0 += __shfl_xor_sync(0xffffffffu, bq0, 2);
    bq1 += __shfl_xor_sync(0xffffffffu, bq1, 1);
    bq1 += __shfl_xor_sync(0xffffffffu, bq1, 2);
    __syncthreads();                      // the last chunk's fragments are no longer read
    float* red = reinterpret_cast<float*>(&S.Af[0][0][0]);   // [k-step][query]
    if (t == 0) {
        red[fks * kDQ + 16 * fmt + g] = bq0;
        red[fks * kDQ + 16 * fmt + g + 8] = bq1;
    }
    __syncthreads();
    if (tid < kDQ) S.dens[tid] = ((red[tid] + red[kDQ + tid]) + red[2 * kDQ + tid]) + red[3 * kDQ + tid];
    __syncthreads();
    float* num = a.num + s * a.Q * a.G;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t qq = q0 + 16 * mt + g + 8 * (q >> 1);
                const int gg = g0 + 32 * warp + 8 * nt + 2 * t + (q & 1);
                if (qq < a.Q && gg < a.G) num[qq * a.G + gg] = Dt[mt][nt][q];
            }
    if (blockIdx.y == 0 && tid < kDQ && q0 + tid < a.Q) a.den[s * a.Q + q0 + tid] = S.dens[tid];
}

// f[q][g] = (sum_s num) / (sum_s den) * norm, splits in order (norm the y
// kernel's constant; a zero denominator -- no x-neighbour -- gives 0)
__global__ void k_density_final(const float* __restrict__ num, const float* __restrict__ den,
                                int n_split, int64_t Q, int G, float norm, float* __restrict__ f) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Q * G) return;
    const int64_t q = e / G;
    float sn = 0.f, sd = 0.f;
    for (int s = 0; s < n_split; ++s) {
        sn += num[(int64_t)s * Q * G + e];
        sd += den[(int64_t)s * Q + q];
    }
    f[e] = sd > 0.f ? sn / sd * norm : 0.f;
}

int density_enqueue(cde_ctx* ctx, const Dataset& D, double h1, double h2, const float* d_xq,
                    int64_t Q, const float* d_yg, int G, float* d_f, cudaStream_t st) {
    if (Q == 0) return CDE_OK;
    const int64_t Qp = (Q + kDQ - 1) / kDQ * kDQ;
    float *xq = nullptr, *mq = nullptr, *num = nullptr, *den = nullptr;
    double* stats = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&xq, (size_t)Qp * D.d * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&mq, (size_t)Q * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&stats, (size_t)2 * D.d * sizeof(double), st));
    CDE_CUDA(cudaMemcpyAsync(stats, D.mean.data(), D.d * sizeof(double), cudaMemcpyHostToDevice, st));
    CDE_CUDA(cudaMemcpyAsync(stats + D.d, D.sd.data(), D.d * sizeof(double), cudaMemcpyHostToDevice, st));
    k_query_pack<<<(unsigned)((Qp + 255) / 256), 256, 0, st>>>(d_xq, Q, Qp, D.d, stats, stats + D.d, xq);
    CDE_CUDA(cudaGetLastError());
    const size_t sm = (size_t)D.d * 256 * sizeof(float);
    if (sm > 48 * 1024)
        CDE_CUDA(cudaFuncSetAttribute(k_query_shift, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const bool epan = D.kernel == CDE_KERNEL_EPAN;
    if (!epan) {
        const int64_t qb = (Q + 255) / 256;
        const int64_t tiles = (D.N + 255) / 256;
        int64_t sy = (4LL * ctx->sm_count + qb - 1) / qb;
        if (sy > tiles) sy = tiles;
        if (sy < 1) sy = 1;
        const int64_t tps = (tiles + sy - 1) / sy;
        sy = (tiles + tps - 1) / tps;
        CDE_CUDA(cudaMemsetAsync(mq, 0x7f, (size_t)Q * sizeof(float), st));  // 3.4e38: above any distance
        k_query_shift<<<dim3((unsigned)qb, (unsigned)sy), 256, sm, st>>>(
            D.xs, D.N, D.Np, D.d, xq, Q, Qp, tps * 256, reinterpret_cast<unsigned int*>(mq));
        CDE_CUDA(cudaGetLastError());
    }
    DensArgs a{};
    a.xs = D.xs;
    a.y = D.y;
    a.xq = xq;
    a.mq = mq;
    a.yg = d_yg;
    a.N = D.N;
    a.Np = D.Np;
    a.Q = Q;
    a.Qp = Qp;
    a.d = D.d;
    a.G = G;
    const double L2E = 1.4426950408889634074;
    a.a1 = (float)(epan ? 1.0 / (h1 * h1) : L2E / (2 * h1 * h1));
    a.a2 = (float)(epan ? 1.0 / (h2 * h2) : L2E / (2 * h2 * h2));
    const int64_t qt = Qp / kDQ;
    const int gt = (G + kDG - 1) / kDG;
    const int64_t chunks = (D.N + kDIC - 1) / kDIC;
    int64_t ns = (4LL * ctx->sm_count + qt * gt - 1) / (qt * gt);
    if (ns > chunks) ns = chunks;
    if (ns < 1) ns = 1;
    const int64_t cps = (chunks + ns - 1) / ns;
    a.i_per_split = cps * kDIC;
    ns = (chunks + cps - 1) / cps;
    CDE_CUDA(cudaMallocAsync((void**)&num, (size_t)ns * Q * G * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&den, (size_t)ns * Q * sizeof(float), st));
    a.num = num;
    a.den = den;
    static bool attr = false;
    if (!attr) {
        CDE_CUDA(cudaFuncSetAttribute(k_density<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(DensSmem)));
        CDE_CUDA(cudaFuncSetAttribute(k_density<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(DensSmem)));
        attr = true;
    }
    const dim3 dgrid((unsigned)qt, (unsigned)gt, (unsigned)ns);
    if (epan) k_density<1><<<dgrid, 256, sizeof(DensSmem), st>>>(a);
    else k_density<0><<<dgrid, 256, sizeof(DensSmem), st>>>(a);
    CDE_CUDA(cudaGetLastError());
    const float norm = (float)(epan ? std::exp(epan_log_norm(1)) / h2 : 1.0 / (2.5066282746310002 * h2));
    k_density_final<<<(unsigned)((Q * G + 255) / 256), 256, 0, st>>>(num, den, (int)ns, Q, G, norm, d_f);
    CDE_CUDA(cudaGetLastError());
    cudaFreeAsync(xq, st);
    cudaFreeAsync(mq, st);
    cudaFreeAsync(stats, st);
    cudaFreeAsync(num, st);
    cudaFreeAsync(den, st);
    return CDE_OK;
}

#ifdef CDE_CHECKS
CDE_CHECK_READER(check_status_density)
#endif

}  // namespace cde

using namespace cde;

extern "C" int cde_density(cde_ctx* ctx, cde_dataset ds, double h1, double h2, const float* xq,
                           int64_t Q, const float* ygrid, int G, float* f_out, int flags, void* stream) {
    CDE_NVTX("cde_density");
    if (!ctx) return set_error(CDE_EINVAL, "cde_density: null context");
    if (Q < 0 || G < 1 || (Q > 0 && (!xq || !ygrid || !f_out)))
        return set_error(CDE_EINVAL, "cde_density: bad sizes or null pointers");
    if (!std::isfinite(h1) || !std::isfinite(h2) || h1 < 1e-12 || h2 < 1e-12 || h1 > 1e12 || h2 > 1e12)
        return set_error(CDE_EINVAL, "cde_density: bandwidth must be finite in [1e-12, 1e12]");
    if (Q * (int64_t)G > ((int64_t)1 << 34)) return set_error(CDE_EINVAL, "cde_density: output too large");
    auto D = find_dataset(ctx, ds);
    if (!D) return set_error(CDE_ENOTFOUND, "cde_density: unknown dataset");
    if (Q == 0) return CDE_OK;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    const bool in_dev = flags & CDE_IN_DEVICE, out_dev = flags & CDE_OUT_DEVICE;
    const float *dq = xq, *dg = ygrid;
    float* dxq = nullptr;
    float* dyg = nullptr;
    float* df = out_dev ? f_out : nullptr;
    if (!in_dev) {
        for (int64_t e = 0; e < Q * D->d; ++e)
            if (!std::isfinite(xq[e])) return set_error(CDE_EINVAL, "cde_density: non-finite query");
        for (int g = 0; g < G; ++g)
            if (!std::isfinite(ygrid[g])) return set_error(CDE_EINVAL, "cde_density: non-finite y grid");
        CDE_CUDA(cudaMallocAsync((void**)&dxq, (size_t)Q * D->d * sizeof(float), st));
        CDE_CUDA(cudaMallocAsync((void**)&dyg, (size_t)G * sizeof(float), st));
        CDE_CUDA(cudaMemcpyAsync(dxq, xq, (size_t)Q * D->d * sizeof(float), cudaMemcpyHostToDevice, st));
        CDE_CUDA(cudaMemcpyAsync(dyg, ygrid, (size_t)G * sizeof(float), cudaMemcpyHostToDevice, st));
        dq = dxq;
        dg = dyg;
    }
    if (!out_dev) CDE_CUDA(cudaMallocAsync((void**)&df, (size_t)Q * G * sizeof(float), st));
    int rc = density_enqueue(ctx, *D, h1, h2, dq, Q, dg, G, df, st);
    cudaError_t e = cudaSuccess;
    if (rc == CDE_OK && !out_dev)
        e = cudaMemcpyAsync(f_out, df, (size_t)Q * G * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (dxq) cudaFreeAsync(dxq, st);
    if (dyg) cudaFreeAsync(dyg, st);
    if (!out_dev) cudaFreeAsync(df, st);
    if (!out_dev) {
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (rc == CDE_OK && e2 != cudaSuccess) return cuda_error(e2, "cde_density: kernels");
    }
    if (rc != CDE_OK) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cde_density: copy");
    return CDE_OK;
}
