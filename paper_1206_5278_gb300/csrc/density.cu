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
// x-neighbour inside h1 (0/0) gets f = 0.
//
// The numerator is a (Q x N) x (N x G) matrix product whose factors are made
// on the fly, so it runs on the 5th-generation tensor cores (k_density_tc):
// a tile is 128 queries x up to 256 grid points, accumulated in tensor memory
// over the data points in chunks of 32.  Sixteen warps evaluate the chunk's u
// (A operand, 128 x 32) and w (B operand, 256 x 32), split each value
// v = hi + lo into two BF16 numbers (round to nearest, |lo| <= 2^-9 v, lo
// rounded again: about 2^-17 v left out) and store them in shared memory;
// thread 0 issues hi*hi + hi*lo + lo*hi as BF16 MMAs with FP32 accumulation
// (about 2^-16 relative per product).  (Streaming precomputed w blocks
// instead was measured slower: 32 KB per chunk from L2 per SM.)  The tensor
// cores' own accumulation is kept to 16 chunks (96 MMAs); the warps then add
// the accumulator into FP32 register totals while the MMAs continue in a
// second TMEM buffer.  Work is split evenly over one CTA per SM in (tile,
// chunk) units; the partial tiles of each CTA are summed in CTA order
// afterwards (bitwise reproducible).
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include <cstdint>

#include "cde_internal.h"
#include "tc_util.cuh"

namespace cde {

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

// d <= 8: the same minima with JB queries per thread (two per packed FP32x2
// instruction; JB = 8, or 2 for few queries), point-major shared tiles of
// data points (128-bit loads) and the data range split over gridDim.y; split
// minima merge with an integer atomicMin on the float bits as above.  Same
// distance formula: dimension 0 first, one fused multiply-add per dimension
// on xq - x_i.
constexpr int kQsThreads = 128;

template <int DREG, int kQsJB>
__global__ void __launch_bounds__(kQsThreads) k_query_shift_split(const float* __restrict__ xs, int64_t N,
                                                                  int64_t Np, int d, const float* __restrict__ xq,
                                                                  int64_t Q, int64_t Qp, int64_t i_per_split,
                                                                  unsigned int* __restrict__ mq_bits) {
    __shared__ __align__(16) float xt[kQsThreads][DREG];
    const int tid = threadIdx.x;
    const int64_t qbase = (int64_t)blockIdx.x * kQsThreads * kQsJB + tid;
    const int64_t i0 = (int64_t)blockIdx.y * i_per_split;
    const int64_t i1 = min(N, i0 + i_per_split);
    float2 q2[kQsJB / 2][DREG];
    float best[kQsJB];
#pragma unroll
    for (int p = 0; p < kQsJB / 2; ++p) {
        const int64_t qa = qbase + (int64_t)(2 * p) * kQsThreads, qb = qa + kQsThreads;
#pragma unroll
        for (int c = 0; c < DREG; ++c)
            q2[p][c] = make_float2(c < d && qa < Qp ? xq[(int64_t)c * Qp + qa] : 0.f,
                                   c < d && qb < Qp ? xq[(int64_t)c * Qp + qb] : 0.f);
        best[2 * p] = best[2 * p + 1] = INFINITY;
    }
    const float2 m1 = make_float2(-1.f, -1.f);
    for (int64_t t0 = i0; t0 < i1; t0 += kQsThreads) {
        __syncthreads();
        const int64_t it = CDE_CK(t0 + tid, Np, 202);  // < Np: splits and Np are multiples of 128
#pragma unroll
        for (int c = 0; c < DREG; ++c) xt[tid][c] = c < d ? xs[(int64_t)c * Np + it] : 0.f;
        __syncthreads();
        const int n = (int)min((int64_t)kQsThreads, i1 - t0);
        for (int t = 0; t < n; ++t) {
            float xi[DREG];
#pragma unroll
            for (int c = 0; c < DREG; c += 4) {
                const float4 v4 = *reinterpret_cast<const float4*>(&xt[t][c]);
                xi[c] = v4.x;
                xi[c + 1] = v4.y;
                xi[c + 2] = v4.z;
                xi[c + 3] = v4.w;
            }
#pragma unroll
            for (int p = 0; p < kQsJB / 2; ++p) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < DREG; ++c) {
                    const float2 tq = __ffma2_rn(make_float2(xi[c], xi[c]), m1, q2[p][c]);
                    acc = __ffma2_rn(tq, tq, acc);
                }
                best[2 * p] = fminf(best[2 * p], acc.x);
                best[2 * p + 1] = fminf(best[2 * p + 1], acc.y);
            }
        }
    }
#pragma unroll
    for (int b = 0; b < kQsJB; ++b) {
        const int64_t q = qbase + (int64_t)b * kQsThreads;
        if (q < Q) atomicMin(mq_bits + q, __float_as_uint(best[b]));
    }
}

// m_q = min_i |x_q - x_i|^2 for the packed queries xq [d][Qp] (Gaussian datasets)
int query_shift_enqueue(int sm_count, const Dataset& D, const float* xq, int64_t Q, int64_t Qp, float* mq,
                        cudaStream_t st) {
    if (Q == 0) return CDE_OK;
    CDE_CUDA(cudaMemsetAsync(mq, 0x7f, (size_t)Q * sizeof(float), st));  // 3.4e38: above any distance
    auto* mqb = reinterpret_cast<unsigned int*>(mq);
    if (D.d <= 8) {
        const int jb = Q >= 4096 ? 8 : 2;
        const int64_t per_cta = (int64_t)kQsThreads * jb;
        const int64_t gx = (Q + per_cta - 1) / per_cta;
        const int64_t tiles = (D.N + kQsThreads - 1) / kQsThreads;
        int64_t ns = (4LL * sm_count + gx - 1) / gx;
        if (ns > tiles) ns = tiles;
        if (ns < 1) ns = 1;
        const int64_t tps = (tiles + ns - 1) / ns;
        ns = (tiles + tps - 1) / tps;
        const dim3 grid((unsigned)gx, (unsigned)ns);
        const int64_t ips = tps * kQsThreads;
        if (D.d <= 4 && jb == 8)
            k_query_shift_split<4, 8><<<grid, kQsThreads, 0, st>>>(D.xs, D.N, D.Np, D.d, xq, Q, Qp, ips, mqb);
        else if (D.d <= 4)
            k_query_shift_split<4, 2><<<grid, kQsThreads, 0, st>>>(D.xs, D.N, D.Np, D.d, xq, Q, Qp, ips, mqb);
        else if (jb == 8)
            k_query_shift_split<8, 8><<<grid, kQsThreads, 0, st>>>(D.xs, D.N, D.Np, D.d, xq, Q, Qp, ips, mqb);
        else
            k_query_shift_split<8, 2><<<grid, kQsThreads, 0, st>>>(D.xs, D.N, D.Np, D.d, xq, Q, Qp, ips, mqb);
        CDE_CUDA(cudaGetLastError());
        return CDE_OK;
    }
    const size_t sm = (size_t)D.d * 256 * sizeof(float);
    if (sm > 48 * 1024)
        CDE_CUDA(cudaFuncSetAttribute(k_query_shift, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t qb = (Q + 255) / 256;
    const int64_t tiles = (D.N + 255) / 256;
    int64_t sy = (4LL * sm_count + qb - 1) / qb;
    if (sy > tiles) sy = tiles;
    if (sy < 1) sy = 1;
    const int64_t tps = (tiles + sy - 1) / sy;
    sy = (tiles + tps - 1) / tps;
    k_query_shift<<<dim3((unsigned)qb, (unsigned)sy), 256, sm, st>>>(D.xs, D.N, D.Np, D.d, xq, Q, Qp, tps * 256, mqb);
    CDE_CUDA(cudaGetLastError());
    return CDE_OK;
}

constexpr int kTcM = 128;        // queries per tile (TMEM lanes)
constexpr int kTcN = 256;        // grid points per tile (largest MMA N)
constexpr int kTcKC = 32;        // data points per chunk (two k16 MMA steps)
constexpr int kTcStages = 3;     // operand ring depth
constexpr int kTcF = 16;         // chunks accumulated in TMEM before a flush
constexpr int kTcProd = 512;     // threads: all make operands; thread 0 also issues the MMAs
constexpr int kTcCols = kTcN / (kTcProd / 128);  // accumulator columns per thread (its warp's TMEM lanes)
constexpr uint32_t kTcSBO = (kTcKC / 8) * 128;   // 8-row group stride of an operand tile

struct DensTcArgs {
    const float* xs;   // dataset [d][Np]
    const float* y;    // [Np]
    const float* xq;   // queries [d][Qp] (standardised like the data)
    const float* mq;   // [Q] nearest squared distances (Gaussian)
    const float* yg;   // [G]
    int64_t N, Np, Q, Qp;
    int d, G, GT;      // GT: grid tiles of 256
    float a1, a2;
    int64_t C;         // chunks per tile
    int64_t U;         // units = tiles * C
    int P;             // CTAs
    int MT;            // partial slots per CTA
    float* part;       // [P * MT][128][256]
    float* dpart;      // [P * MT][128]
    int* err;          // timeout word
};

struct TcSmem {
    unsigned char A[kTcStages][2][kTcM * kTcKC * 2];   // u: hi, lo (BF16, K-major core matrices)
    unsigned char B[kTcStages][2][kTcN * kTcKC * 2];   // w: hi, lo
    float pt[3][kMaxD + 1][kTcKC];                     // chunk's x (d rows) and y: ring of 3 chunks
    float xq[kMaxD][kTcM];                             // the tile's query coordinates
    float den[3][kTcM];
    unsigned long long empty[kTcStages], accfull[2];
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t pack_bf16x2_d(float lo_elem, float hi_elem) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);  // first argument in the low half
    return *reinterpret_cast<const uint32_t*>(&v);
}

// v = hi + lo for two adjacent K elements (k even in the low half): the BF16
// roundings of v and of the exact remainder v - hi
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    hi = pack_bf16x2_d(v0, v1);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16x2_d(v0 - h0, v1 - h1);
}

// One chunk's place in the CTA's unit range: tile t, chunk c, and the
// accumulation period it belongs to.  Periods are runs of at most kTcF chunks
// of one tile; a tile's run inside the CTA's range is its segment.
struct TcPeriod {
    int64_t t, c;
    int len;
    bool first, last;   // first / last period of its segment
};

__device__ __forceinline__ TcPeriod tc_period(int64_t u, int64_t u0, int64_t u1, int64_t C) {
    TcPeriod p;
    p.t = u / C;
    p.c = u - p.t * C;
    int64_t ce = min(C, p.c + kTcF);
    if (p.t * C + ce > u1) ce = u1 - p.t * C;
    p.len = (int)(ce - p.c);
    p.first = p.c == 0 || u == u0;
    p.last = ce == C || p.t * C + ce == u1;
    return p;
}

// MMA N of grid tile gt (a multiple of 16)
__device__ __forceinline__ int tc_ntile(int G, int gt) { return min(kTcN, (G - gt * kTcN + 15) / 16 * 16); }

// Issue the MMAs of the chunk in stage s (thread 0, after the barrier that
// ends the chunk): hi*hi + hi*lo + lo*hi for both k16 steps into TMEM buffer
// b, then release the stage; the last chunk of a period also signals the flush.
__device__ __forceinline__ void tc_issue(TcSmem& S, uint32_t tbase, int s, int b, bool first, bool last,
                                         uint32_t idesc) {
    const uint32_t dt = tbase + (uint32_t)(b * kTcN);
    tc_fence_after();
#pragma unroll
    for (int ks = 0; ks < kTcKC / 16; ++ks) {
        const uint64_t ah = tc_sdesc(smem_u32(&S.A[s][0][0]) + 256 * ks, 128, kTcSBO);
        const uint64_t al = tc_sdesc(smem_u32(&S.A[s][1][0]) + 256 * ks, 128, kTcSBO);
        const uint64_t bh = tc_sdesc(smem_u32(&S.B[s][0][0]) + 256 * ks, 128, kTcSBO);
        const uint64_t bl = tc_sdesc(smem_u32(&S.B[s][1][0]) + 256 * ks, 128, kTcSBO);
        tc_mma_bf16(dt, ah, bh, idesc, (!first || ks > 0) ? 1u : 0u);
        tc_mma_bf16(dt, ah, bl, idesc, 1u);
        tc_mma_bf16(dt, al, bh, idesc, 1u);
    }
    tc_commit(smem_u32(&S.empty[s]));
    if (last) tc_commit(smem_u32(&S.accfull[b]));
}

// Start the asynchronous copy of one chunk's points (x rows, then y) into
// point buffer `slot`; i0 < 0: no chunk (the group is still committed, so
// every thread's group count stays in step).
__device__ __forceinline__ void tc_fetch_points(const DensTcArgs& a, TcSmem& S, int slot, int64_t i0) {
    if (i0 >= 0) {
        const int nel = (a.d + 1) * kTcKC;
        for (int e = threadIdx.x; e < nel; e += kTcProd) {
            const int row = e / kTcKC, p = e % kTcKC;
            const float* src = (row < a.d ? a.xs + (int64_t)row * a.Np : a.y) + CDE_CK(i0 + p, a.Np, 211);
            cp_async4(smem_u32(&S.pt[slot][row][p]), src);
        }
    }
    cp_async_commit();
}

// Make the chunk's operands: u (A, 128 queries x 32 points) and w (B, up to
// 256 grid points x 32 points), each split into BF16 hi and lo, in operand
// stage s from the points in buffer pb; then publish the next chunk's points
// (copied asynchronously two chunks ahead) with the closing barrier.  Thread
// roles: A (query tid % 128, points 8 (tid / 128) ... + 8, one core-matrix
// column), B (grid row tid % 256, points 16 (tid / 256) ... + 16).  Pairs of
// points go through the packed FP32x2 pipe; xq - x is formed as
// fma(x, -1, xq), the same rounding as the scalar subtraction of every other
// pair kernel.
template <int KERN>
__device__ __forceinline__ void tc_produce(const DensTcArgs& a, TcSmem& S, int s, uint32_t empty_parity, int pb,
                                           int nvalid, int ntile, float mqv, float ygv, float& den, float& denc,
                                           volatile int* abort_flag) {
    const int tid = threadIdx.x;
    const int d = a.d;
    const float2 m1 = make_float2(-1.f, -1.f);
    // the MMAs that read this stage last time are done
    mbar_wait(smem_u32(&S.empty[s]), empty_parity, abort_flag, a.err, 1);
    const int q = tid & (kTcM - 1), qr = tid >> 7;
    float2 v2[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v2[e] = make_float2(0.f, 0.f);
    for (int cd = 0; cd < d; ++cd) {
        const float xqc = S.xq[cd][q];
        const float2 xq2 = make_float2(xqc, xqc);
        const float4* xp = reinterpret_cast<const float4*>(&S.pt[pb][cd][8 * qr]);
        const float4 xa = xp[0], xb = xp[1];
        float2 t;
        t = __ffma2_rn(make_float2(xa.x, xa.y), m1, xq2);
        v2[0] = __ffma2_rn(t, t, v2[0]);
        t = __ffma2_rn(make_float2(xa.z, xa.w), m1, xq2);
        v2[1] = __ffma2_rn(t, t, v2[1]);
        t = __ffma2_rn(make_float2(xb.x, xb.y), m1, xq2);
        v2[2] = __ffma2_rn(t, t, v2[2]);
        t = __ffma2_rn(make_float2(xb.z, xb.w), m1, xq2);
        v2[3] = __ffma2_rn(t, t, v2[3]);
    }
    float u[8];
    if constexpr (KERN == 0) {
        // 2^{a1 (m_q - dx2)} as 2^{a1 m_q - a1 dx2}
        const float a1 = a.a1, am = a1 * mqv;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 arg = __ffma2_rn(make_float2(-a1, -a1), v2[e], make_float2(am, am));
            u[2 * e] = ex2d(arg.x);
            u[2 * e + 1] = ex2d(arg.y);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            u[2 * e] = fma_sat_d(-a.a1, v2[e].x, 1.f);
            u[2 * e + 1] = fma_sat_d(-a.a1, v2[e].y, 1.f);
        }
    }
    if (nvalid < kTcKC) {   // the data's last, partial chunk: points past N get u = 0
        const int nv = nvalid - 8 * qr;
#pragma unroll
        for (int p = 0; p < 8; ++p) u[p] = p < nv ? u[p] : 0.f;
    }
    float cs = 0.f;
#pragma unroll
    for (int p = 0; p < 8; ++p) cs += u[p];
    // compensated running sum of the denominator
    const float yk = cs - denc, tk = den + yk;
    denc = (tk - den) - yk;
    den = tk;
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) split_pair(u[2 * e], u[2 * e + 1], h[e], l[e]);
    const uint32_t off = (uint32_t)(q >> 3) * kTcSBO + (uint32_t)(q & 7) * 16 + (uint32_t)qr * 128;
    *reinterpret_cast<uint4*>(&S.A[s][0][off]) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(&S.A[s][1][off]) = make_uint4(l[0], l[1], l[2], l[3]);
    // ---- B: w for grid row g and points 16 gh ... 16 gh + 15 (two core-matrix columns)
    {
        const int g = tid & (kTcN - 1), gh = tid >> 8;
        if (g < ntile) {
            const uint32_t rowoff = (uint32_t)(g >> 3) * kTcSBO + (uint32_t)(g & 7) * 16;
            const float2 yg2 = make_float2(ygv, ygv);
            const float4* yp = reinterpret_cast<const float4*>(&S.pt[pb][d][16 * gh]);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const float4 ya = yp[2 * kk], yb = yp[2 * kk + 1];
                const float2 yy[4] = {make_float2(ya.x, ya.y), make_float2(ya.z, ya.w), make_float2(yb.x, yb.y),
                                      make_float2(yb.z, yb.w)};
                uint32_t hb[4], lb[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 t = __ffma2_rn(yy[e], m1, yg2);
                    const float2 t2 = __fmul2_rn(t, t);
                    float w0, w1;
                    if constexpr (KERN == 0) {
                        const float2 arg = __fmul2_rn(t2, make_float2(-a.a2, -a.a2));
                        w0 = ex2d(arg.x);
                        w1 = ex2d(arg.y);
                    } else {
                        w0 = fma_sat_d(-a.a2, t2.x, 1.f);
                        w1 = fma_sat_d(-a.a2, t2.y, 1.f);
                    }
                    split_pair(w0, w1, hb[e], lb[e]);
                }
                const uint32_t boff = rowoff + (uint32_t)(2 * gh + kk) * 128;
                *reinterpret_cast<uint4*>(&S.B[s][0][boff]) = make_uint4(hb[0], hb[1], hb[2], hb[3]);
                *reinterpret_cast<uint4*>(&S.B[s][1][boff]) = make_uint4(lb[0], lb[1], lb[2], lb[3]);
            }
        }
    }
    fence_async_smem();   // the tensor cores read these after the barrier
    cp_async_wait_1();    // this thread's copies of the next chunk have landed
    __syncthreads();
}

// Add accumulation period pq's TMEM buffer into the register totals (the
// warp's 32 TMEM lanes = queries, columns 64 (warp / 4) ... + 64); at the end
// of a segment write the totals and the denominator as a partial tile.  The
// TMEM reads are ordered before the next MMA into the buffer by the fence
// and the barrier that ends the next chunk.
__device__ __forceinline__ void tc_flush(const DensTcArgs& a, TcSmem& S, uint32_t tbase, int pq, int64_t tq,
                                         bool lastq, float den_seg, int64_t t_first, float (&tot)[kTcCols],
                                         volatile int* abort_flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = pq & 1;
    const bool ok = mbar_wait(smem_u32(&S.accfull[b]), (uint32_t)(pq >> 1) & 1, abort_flag, a.err, 2);
    tc_fence_after();
    if (ok) {
        const uint32_t ta =
            tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * kTcN + (warp >> 2) * kTcCols);
#pragma unroll
        for (int cb = 0; cb < kTcCols / 32; ++cb) {
            float v[32];
            tmem_ld32(ta + 32 * cb, v);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) tot[32 * cb + j] += v[j];
        }
    }
    tc_fence_before();
    if (lastq) {
        const int64_t slot = (int64_t)blockIdx.x * a.MT + (tq - t_first);
        const int row = 32 * (warp & 3) + lane;
        float4* dst = reinterpret_cast<float4*>(a.part + (slot * kTcM + row) * kTcN + (warp >> 2) * kTcCols);
#pragma unroll
        for (int v4 = 0; v4 < kTcCols / 4; ++v4) {
            dst[v4] = make_float4(tot[4 * v4], tot[4 * v4 + 1], tot[4 * v4 + 2], tot[4 * v4 + 3]);
            tot[4 * v4] = tot[4 * v4 + 1] = tot[4 * v4 + 2] = tot[4 * v4 + 3] = 0.f;
        }
        // a query's four denominator parts (point quarters), summed in order
        const int q = tid & (kTcM - 1), qr = tid >> 7;
        if (qr > 0) S.den[qr - 1][q] = den_seg;
        __syncthreads();
        if (qr == 0) a.dpart[slot * kTcM + q] = ((den_seg + S.den[0][q]) + S.den[1][q]) + S.den[2][q];
        __syncthreads();
    }
}

template <int KERN>
__global__ void __launch_bounds__(kTcProd, 1) k_density_tc(const DensTcArgs a) {
    extern __shared__ float4 tc_dyn[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_dyn);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t u0 = (int64_t)blockIdx.x * a.U / a.P, u1 = ((int64_t)blockIdx.x + 1) * a.U / a.P;
    const int64_t t_first = u0 / a.C;
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) mbar_init(smem_u32(&S.empty[s]), 1);
        for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&S.accfull[b]), 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&S.tmem_base), 2 * kTcN);
    {
        // the first two chunks' points (units u0 and u0 + 1)
        const int64_t c0 = u0 % a.C, c1 = c0 + 1 == a.C ? 0 : c0 + 1;
        tc_fetch_points(a, S, 0, c0 * kTcKC);
        tc_fetch_points(a, S, 1, u0 + 1 < u1 ? c1 * kTcKC : -1);
        cp_async_wait_1();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = S.tmem_base;
    volatile int* abort_flag = &S.abort;

    float tot[kTcCols];
#pragma unroll
    for (int j = 0; j < kTcCols; ++j) tot[j] = 0.f;
    float den = 0.f, denc = 0.f, den_done = 0.f;
    int s = 0, pb = 0;   // operand stage, point buffer of the current chunk
    uint32_t empty_parity = 1;
    int64_t u = u0, cur_t = -1, prev_t = -1;
    bool prev_last = false;
    int pi = 0, ntile = kTcN;
    uint32_t idesc = 0;
    float mqv = 0.f, ygv = 0.f;
    while (u < u1) {
        const TcPeriod P = tc_period(u, u0, u1, a.C);
        if (P.t != cur_t) {   // a new tile: its queries, shift and grid row
            cur_t = P.t;
            const int64_t qt = P.t / a.GT;
            const int gt = (int)(P.t % a.GT);
            for (int e = tid; e < a.d * kTcM; e += kTcProd) {
                const int cd = e / kTcM, qq = e % kTcM;
                S.xq[cd][qq] = a.xq[(int64_t)cd * a.Qp + CDE_CK(qt * kTcM + qq, a.Qp, 213)];
            }
            const int64_t qg = qt * kTcM + (tid & (kTcM - 1));
            mqv = (KERN == 0 && qg < a.Q) ? a.mq[qg] : 0.f;
            const int gg = gt * kTcN + (tid & (kTcN - 1));
            ygv = a.yg[gg < a.G ? gg : a.G - 1];
            ntile = tc_ntile(a.G, gt);
            idesc = tc_idesc_bf16(kTcM, ntile);
            __syncthreads();
        }
        if (P.first && pi > 0) {
            den_done = den;
            den = denc = 0.f;
        }
        for (int j = 0; j < P.len; ++j) {
            const int64_t c = P.c + j;
            const int nvalid = (int)min((int64_t)kTcKC, a.N - c * kTcKC);
            // the unit two ahead: units run through a tile's chunks, then to chunk 0 of the next tile
            const int64_t c1 = c + 1 == a.C ? 0 : c + 1, c2 = c1 + 1 == a.C ? 0 : c1 + 1;
            tc_fetch_points(a, S, pb == 0 ? 2 : pb - 1, u + j + 2 < u1 ? c2 * kTcKC : -1);
            tc_produce<KERN>(a, S, s, empty_parity, pb, nvalid, ntile, mqv, ygv, den, denc, abort_flag);
            if (tid == 0 && !*abort_flag) tc_issue(S, tbase, s, pi & 1, j == 0, j == P.len - 1, idesc);
            pb = pb == 2 ? 0 : pb + 1;
            if (++s == kTcStages) {
                s = 0;
                empty_parity ^= 1;
            }
        }
        if (pi >= 1) tc_flush(a, S, tbase, pi - 1, prev_t, prev_last, den_done, t_first, tot, abort_flag);
        prev_t = P.t;
        prev_last = P.last;
        u += P.len;
        ++pi;
    }
    if (pi >= 1) tc_flush(a, S, tbase, pi - 1, prev_t, prev_last, den, t_first, tot, abort_flag);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 2 * kTcN);
    }
}

// CTA owning unit u under the even split of U units over P CTAs
// (u0(c) = floor(c U / P)): the largest c with u0(c) <= u
__device__ __forceinline__ int64_t tc_owner(int64_t u, int64_t U, int64_t P) { return ((u + 1) * P - 1) / U; }

// f[q][g] = (sum over the CTAs covering the tile of the partial numerators) /
// (same for the denominators) * norm; a zero denominator (no x-neighbour)
// gives 0.  A block is 32 grid points x 8 slots; a slot is one of `parts`
// consecutive pieces of the covering CTAs' range (parts = 1, 2, 4 or 8) of one
// query row.  Pieces are summed in CTA order, then the pieces in order.  f
// has row stride ldf (the caller's full grid when this pass covers part of it).
__global__ void __launch_bounds__(256) k_density_final(const DensTcArgs a, float norm, int parts_log2,
                                                       float* __restrict__ f, int64_t ldf) {
    __shared__ float rn[8][32], rd[8][32];
    const int lane = threadIdx.x & 31, slot = threadIdx.x >> 5;
    const int parts = 1 << parts_log2, part = slot & (parts - 1);
    const int64_t gb_n = (a.G + 31) / 32, qb = (int64_t)blockIdx.x / gb_n;
    const int gb = (int)((int64_t)blockIdx.x - qb * gb_n);
    const int64_t q = qb * (8 >> parts_log2) + (slot >> parts_log2);
    const int g = gb * 32 + lane;
    float sn = 0.f, sd = 0.f;
    if (q < a.Q) {
        const int64_t t = (q / kTcM) * a.GT + (gb * 32) / kTcN;
        const int64_t c0 = tc_owner(t * a.C, a.U, a.P), c1 = tc_owner(t * a.C + a.C - 1, a.U, a.P);
        const int64_t per = (c1 - c0 + parts) / parts;
        const int64_t cb = c0 + part * per, ce = min(c1 + 1, cb + per);
        for (int64_t c = cb; c < ce; ++c) {
            const int64_t ub = c * a.U / a.P, ue = (c + 1) * a.U / a.P;
            if (ub >= ue) continue;
            const int64_t sl = c * a.MT + (t - ub / a.C);
            if (g < a.G) sn += a.part[(sl * kTcM + (q % kTcM)) * kTcN + g % kTcN];
            sd += a.dpart[sl * kTcM + (q % kTcM)];
        }
    }
    rn[slot][lane] = sn;
    rd[slot][lane] = sd;
    __syncthreads();
    if (part == 0 && q < a.Q && g < a.G) {
        for (int p = 1; p < parts; ++p) {
            sn += rn[slot + p][lane];
            sd += rd[slot + p][lane];
        }
        f[q * ldf + g] = sd > 0.f ? sn / sd * norm : 0.f;
    }
}

int density_enqueue(cde_ctx* ctx, const Dataset& D, double h1, double h2, const float* d_xq,
                    int64_t Q, const float* d_yg, int G, float* d_f, cudaStream_t st) {
    timing_reset(ctx);
    if (Q == 0) return CDE_OK;
    const int64_t Qp = (Q + kTcM - 1) / kTcM * kTcM;
    float *xq = nullptr, *mq = nullptr, *part = nullptr, *dpart = nullptr;
    double* stats = nullptr;
    CDE_CUDA(cudaMallocAsync((void**)&xq, (size_t)Qp * D.d * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&mq, (size_t)Q * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&stats, (size_t)2 * D.d * sizeof(double), st));
    CDE_CUDA(cudaMemcpyAsync(stats, D.mean.data(), D.d * sizeof(double), cudaMemcpyHostToDevice, st));
    CDE_CUDA(cudaMemcpyAsync(stats + D.d, D.sd.data(), D.d * sizeof(double), cudaMemcpyHostToDevice, st));
    k_query_pack<<<(unsigned)((Qp + 255) / 256), 256, 0, st>>>(d_xq, Q, Qp, D.d, stats, stats + D.d, xq);
    CDE_CUDA(cudaGetLastError());
    const bool epan = D.kernel == CDE_KERNEL_EPAN;
    if (!epan) {
        const int rc = query_shift_enqueue(ctx->sm_count, D, xq, Q, Qp, mq, st);
        if (rc != CDE_OK) return rc;
    }
    const double L2E = 1.4426950408889634074;
    DensTcArgs a{};
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
    a.GT = (G + kTcN - 1) / kTcN;
    a.a1 = (float)(epan ? 1.0 / (h1 * h1) : L2E / (2 * h1 * h1));
    a.a2 = (float)(epan ? 1.0 / (h2 * h2) : L2E / (2 * h2 * h2));
    a.C = (D.N + kTcKC - 1) / kTcKC;
    a.U = (Qp / kTcM) * a.GT * a.C;
    a.P = (int)std::min<int64_t>(ctx->sm_count, a.U);
    a.MT = (int)(((a.U + a.P - 1) / a.P + a.C - 1) / a.C + 1);
    a.err = ctx->d_err + kErrTensorWait;
    CDE_CUDA(cudaMallocAsync((void**)&part, (size_t)a.P * a.MT * kTcM * kTcN * sizeof(float), st));
    CDE_CUDA(cudaMallocAsync((void**)&dpart, (size_t)a.P * a.MT * kTcM * sizeof(float), st));
    a.part = part;
    a.dpart = dpart;
    static std::atomic<uint64_t> attr0{0}, attr1{0};
    CDE_CUDA(smem_attr_once(attr0, k_density_tc<0>, (int)sizeof(TcSmem)));
    CDE_CUDA(smem_attr_once(attr1, k_density_tc<1>, (int)sizeof(TcSmem)));
    timing_begin(ctx, st);
    if (epan) k_density_tc<1><<<a.P, kTcProd, sizeof(TcSmem), st>>>(a);
    else k_density_tc<0><<<a.P, kTcProd, sizeof(TcSmem), st>>>(a);
    timing_end(ctx, st);
    CDE_CUDA(cudaGetLastError());
    const float norm = (float)(epan ? std::exp(epan_log_norm(1)) / h2 : 1.0 / (2.5066282746310002 * h2));
    // CTAs covering one tile: at most ceil(C / per-CTA units) + 1
    const int64_t ncta = (a.C + a.U / a.P - 1) / (a.U / a.P) + 1;
    const int plog = ncta > 16 ? 3 : ncta > 8 ? 2 : ncta > 4 ? 1 : 0;
    const int64_t fblocks = (Q + (8 >> plog) - 1) / (8 >> plog) * ((G + 31) / 32);
    k_density_final<<<(unsigned)fblocks, 256, 0, st>>>(a, norm, plog, d_f, G);
    CDE_CUDA(cudaGetLastError());
    cudaFreeAsync(xq, st);
    cudaFreeAsync(mq, st);
    cudaFreeAsync(stats, st);
    cudaFreeAsync(part, st);
    cudaFreeAsync(dpart, st);
    return CDE_OK;
}

// Self-test of the bounded on-device wait: one thread waits on an mbarrier
// that nothing arrives on, exactly as the tensor-core kernel's waits do; the
// wait gives up after its limit (about a second), records `code` in the
// context's wait word and returns normally.
__global__ void k_wait_selftest(int* err, int code) {
    __shared__ unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait(smem_u32(&bar), 0, &abort_flag, err, code);
    }
}

#ifdef CDE_CHECKS
CDE_CHECK_READER(check_status_density)
#endif

}  // namespace cde

using namespace cde;

extern "C" int cde_selftest_wait(cde_ctx* ctx) {
    CDE_NVTX("cde_selftest_wait");
    if (!ctx) return set_error(CDE_EINVAL, "cde_selftest_wait: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CDE_CUDA(cudaSetDevice(ctx->device));
    k_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->d_err + kErrTensorWait, 64);
    CDE_CUDA(cudaGetLastError());
    CDE_CUDA(cudaStreamSynchronize(ctx->stream));
    return CDE_OK;
}

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
    if (!out_dev) {
        const int rw = workspace_reserve(ctx, 0, 64);
        if (rw != CDE_OK) {
            if (dxq) cudaFreeAsync(dxq, st);
            if (dyg) cudaFreeAsync(dyg, st);
            return rw;
        }
        CDE_CUDA(cudaMallocAsync((void**)&df, (size_t)Q * G * sizeof(float), st));
    }
    int rc = density_enqueue(ctx, *D, h1, h2, dq, Q, dg, G, df, st);
    cudaError_t e = cudaSuccess;
    int* tw_host = static_cast<int*>(ctx->ws_host);   // pinned; the context lock is held
    if (rc == CDE_OK && !out_dev) {
        e = cudaMemcpyAsync(f_out, df, (size_t)Q * G * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && tw_host)
            e = cudaMemcpyAsync(tw_host, ctx->d_err + kErrTensorWait, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    if (dxq) cudaFreeAsync(dxq, st);
    if (dyg) cudaFreeAsync(dyg, st);
    if (!out_dev) cudaFreeAsync(df, st);
    if (!out_dev) {
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (rc == CDE_OK && e2 != cudaSuccess) return cuda_error(e2, "cde_density: kernels");
    }
    if (rc != CDE_OK) return rc;
    if (e != cudaSuccess) return cuda_error(e, "cde_density: copy");
    if (!out_dev && tw_host && *tw_host) {
        cudaMemsetAsync(ctx->d_err + kErrTensorWait, 0, sizeof(int), st);
        return set_error(CDE_ETIMEOUT, "cde_density: a tensor-core wait ran out on the device");
    }
    return CDE_OK;
}
