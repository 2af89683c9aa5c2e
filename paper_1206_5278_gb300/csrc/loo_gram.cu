// Leave-one-out grid kernel for d_x >= 16: squared distances from the x
// cross-term on the tensor cores (Sec. 3.2 sums A_j, B_j over all pairs).
//
// At d_x >= 16 the direct distance pass of the tile body (loo_mma.cuh) reads
// d_x coordinates of every point once per row, 128 bytes per pair at d = 32,
// and spends 2 d_x FP32 operations on it.  Here a CTA of 16 warps owns a unit
// of R = 16 JW rows and every warp walks all points for its own JW rows
// (JW = 1024/(G1 G2): the tile body's rows per unit), so each tile of P points
// is read once for all R rows, and the R x P block of dot products x_j . x_i
// is one small GEMM (K = d_x):
//
//   |x_j - x_i|^2 = n_j + n_i - 2 x_j . x_i,   n = |x|^2 (FP32),
//
// with the dot products as 3xTF32 mma.sync m16n8k8 (x = hi + lo with hi the
// TF32 rounding: lo hi + hi lo + hi hi, FP32 accumulate), clamped at 0.  Its
// error, about 2^-19 (n_j + n_i), is large next to the distances that decide
// the weights at small h1, so pairs with |x_j - x_i|^2 - m_x,j < (n_j + n_i)/32
// are recomputed with the tile body's direct FP32 formula (bitwise the value
// the nearest-neighbour shifts were taken from; a few per mille of the pairs
// on the benchmark data).  A pair beyond that limit weighs at most
// exp(-(n_j + n_i)/(64 h1^2)) of the nearest one, which bounds what its Gram
// error can move a row's log-sum to about 2^-19 32/e ~ 2e-5 of one term.
//
// Per step of P points the warps first form the distance block of the next
// step (double-buffered in shared memory: t1 = m_x,j - d2, t2 = m_y,j - dy2,
// masked pairs t1 = -inf) and then run the tile body's exp2 / split /
// outer-product MMAs on the current block; one CTA barrier per step.
//
// The epilogue flags cells below the recompute threshold (as the tile body
// does) and recomputes them exactly in two passes over the points that reuse
// the distance blocks: points whose Gram distance, widened by 2^-16 (n_j + n_i)
// (four times the Gram error bound), can lie in a cell's argmin region or sum
// box get their distance recomputed directly, and everything after that is the
// direct fallback's arithmetic (loo_common.cuh), so the recomputed cells are
// those of the direct path.  Their log-numerators go to a per-CTA FP64 buffer;
// the unit's FP64 log-ratios are then summed over its rows in row order into
// the unit's partial slot, and k_loo_final sums the slots in order: results are
// bitwise reproducible.
#include <cmath>

#include "cde_internal.h"
#include "loo_common.cuh"
#include "loo_mma.cuh"

namespace cde {

template <int G1, int G2>
struct GramCfg {
    static constexpr int kWarps = 16, kThreads = 512;
    static constexpr int GG = G1 * G2, JW = 1024 / GG, R = 16 * JW;
    static constexpr int MT = G1 / 16, NT = G2 / 8;
    // points per step: one CTA barrier per step, and fewer barriers keep the
    // warps' exp2 and MMA phases from lining up (512 vs 128 points: 0.83x time)
    static constexpr int P = 512 / JW;
    static constexpr int PS = P + 8;                                 // row stride of the blocks
    static constexpr int CPS = P / 32;                               // 32-point chunks per step
    static constexpr int GT = (R / 16) * (P / 8);                    // Gram output tiles per step
    static constexpr int TPW = GT / kWarps;                          // per warp
    static constexpr int CELLS = R * GG;                             // 16384: one bit per thread-word
    static constexpr int FMAX = 1024;                                // flagged cells per fallback round
    static_assert(CELLS == 32 * kThreads, "one flag word per thread");
    static_assert(TPW * kWarps == GT, "whole Gram tiles per warp");
    // shared memory layout in 4-byte words (KS: row stride of the staged row coordinates)
    __host__ __device__ static int ks(int d) { return ((d + 7) & ~7) + 4; }
    __host__ __device__ static int o_rows() { return 0; }
    __host__ __device__ static int o_blk(int d) { return (R * ks(d) + 3) & ~3; }                // [2][R][PS] t1
    __host__ __device__ static int o_np(int d) { return o_blk(d) + 2 * R * PS; }                // [2][P] norms
    __host__ __device__ static int o_y(int d) { return o_np(d) + 2 * P; }                       // [2][P] y
    __host__ __device__ static int o_rc(int d) { return o_y(d) + 2 * P; }                       // [8][R]
    __host__ __device__ static int o_at(int d) { return o_rc(d) + 8 * R; }                      // [R][GG]
    __host__ __device__ static int o_btl(int d) { return o_at(d) + CELLS; }                     // [R][G1] f64
    __host__ __device__ static int o_flag(int d) { return o_btl(d) + 2 * R * G1; }              // [512]
    __host__ __device__ static int o_pos(int d) { return o_flag(d) + kThreads; }                // [512]
    __host__ __device__ static int o_misc(int d) { return o_pos(d) + kThreads; }                // [64]
    __host__ __device__ static int o_list(int d) { return o_misc(d) + 64; }                     // [FMAX]
    __host__ __device__ static int o_best(int d) { return o_list(d) + FMAX; }                   // [FMAX] u64
    __host__ __device__ static int o_acc(int d) { return o_best(d) + 2 * FMAX; }                // [FMAX] u64
    __host__ __device__ static int o_dxs(int d) { return o_acc(d) + 2 * FMAX; }                 // [FMAX]
    __host__ __device__ static int o_dys(int d) { return o_dxs(d) + FMAX; }                     // [FMAX]
    __host__ __device__ static int o_sx(int d) { return o_dys(d) + FMAX; }                      // [FMAX] staircase X
    __host__ __device__ static int o_sy(int d) { return o_sx(d) + FMAX; }                       // [FMAX] staircase Y
    __host__ __device__ static int o_cf(int d) { return o_sy(d) + FMAX; }   // a1[32], a2[32], lam1[32], kap2[32] (f64)
    __host__ __device__ static int o_rp(int d) { return o_cf(d) + 192; }                        // [8][R]
    static size_t smem_bytes(int d) { return (size_t)(o_rp(d) + 8 * R) * 4; }
};

constexpr int kGramMaxKSteps = kMaxD / 8;     // k-steps of 8 dimensions at the largest d_x
constexpr float kGramNear = 1.0f / 32.0f;     // direct recomputation below this share of n_j + n_i
constexpr float kGramSlack = 1.0f / 65536.0f; // pre-test widening, times n_j + n_i

// direct FP32 squared distance, the tile body's order (dimension 0 first, fmaf)
__device__ __forceinline__ float direct_d2(const float* __restrict__ xr, const float* __restrict__ xs,
                                           int64_t p, int d, int64_t Np) {
    float d2 = 0.f;
#pragma unroll 4
    for (int c = 0; c < d; ++c) {
        const float q = xr[c] - xs[(int64_t)c * Np + p];
        d2 = fmaf(q, q, d2);
    }
    return d2;
}

// TF32 split with hi the round-to-nearest TF32 value (lo = x - hi exact)
__device__ __forceinline__ void split_rn(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna(x);
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// Distance block of one step: t1 of every (row, point) of the unit, the
// points' norms and y, into buffer `buf`.  NEAR: recompute the near pairs
// directly (the main pass; the fallback's passes work with the Gram values and
// recompute the few points they keep).
template <int G1, int G2, int KERN, bool NEAR>
__device__ __forceinline__ void gram_block(const LooArgs& a, float* sm, int64_t p0, int buf) {
    using C = GramCfg<G1, G2>;
    constexpr int R = C::R, P = C::P, PS = C::PS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int d = a.d, KS = C::ks(d), KSTEPS = (d + 7) >> 3;
    const int64_t N = a.N, Np = a.Np;
    const float* rows_s = sm + C::o_rows();
    float* T1 = sm + C::o_blk(d) + buf * R * PS;
    float* NPs = sm + C::o_np(d) + buf * P;
    float* Ys = sm + C::o_y(d) + buf * P;
    const float* rc = sm + C::o_rc(d);
    const float *mxr_s = rc + R, *nr_s = rc + 3 * R;
    const int* jr_s = reinterpret_cast<const int*>(rc + 6 * R);
#pragma unroll
    for (int tt = 0; tt < C::TPW; ++tt) {
        const int ti = warp + C::kWarps * tt;
        const int mtg = ti / (P / 8), ntg = ti - mtg * (P / 8);
        // this lane's B point (steps may run past the padded length: those points are
        // masked, and their loads are clamped to the last stored point)
        const int64_t pg = CDE_CK(min(p0 + 8 * ntg + g, Np - 1), Np, 121);
        const int r0 = 16 * mtg + g, r1 = r0 + 8;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        float np = 0.f;
        // all of the tile's point coordinates first (one round trip to L2, not one per k-step)
        float xb0[kGramMaxKSteps], xb1[kGramMaxKSteps];
#pragma unroll
        for (int s = 0; s < kGramMaxKSteps; ++s) {
            const int c0 = 8 * s + t, c1 = c0 + 4;
            xb0[s] = (s < KSTEPS && c0 < d) ? a.xs[(int64_t)c0 * Np + pg] : 0.f;
            xb1[s] = (s < KSTEPS && c1 < d) ? a.xs[(int64_t)c1 * Np + pg] : 0.f;
        }
#pragma unroll
        for (int s = 0; s < kGramMaxKSteps; ++s) {
            if (s >= KSTEPS) break;
            const int c0 = 8 * s + t, c1 = c0 + 4;
            const float x0 = xb0[s], x1 = xb1[s];
            np = fmaf(x0, x0, fmaf(x1, x1, np));
            uint32_t bh0, bl0, bh1, bl1;
            split_rn(x0, bh0, bl0);
            split_rn(x1, bh1, bl1);
            uint32_t ah[4], al[4];
            split_rn(rows_s[r0 * KS + c0], ah[0], al[0]);
            split_rn(rows_s[r1 * KS + c0], ah[1], al[1]);
            split_rn(rows_s[r0 * KS + c1], ah[2], al[2]);
            split_rn(rows_s[r1 * KS + c1], ah[3], al[3]);
            mma_tf32(acc, al, bh0, bh1);
            mma_tf32(acc, ah, bl0, bl1);
            mma_tf32(acc, ah, bh0, bh1);
        }
        // point norms: lanes 4g .. 4g+3 hold point g's dimensions
        np += __shfl_xor_sync(0xffffffffu, np, 1);
        np += __shfl_xor_sync(0xffffffffu, np, 2);
        const float npa = __shfl_sync(0xffffffffu, np, 8 * t), npb = __shfl_sync(0xffffffffu, np, 8 * t + 4);
        if (t == 0 && mtg == 0) {
            NPs[8 * ntg + g] = np;
            Ys[8 * ntg + g] = a.y[pg];
        }
        // outputs: rows r0, r1 x points 2t, 2t+1 of the tile
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rl = q < 2 ? r0 : r1;
            const int pl = 8 * ntg + 2 * t + (q & 1);
            const int64_t p = p0 + pl;
            const float nr = nr_s[rl], nsum = nr + ((q & 1) ? npb : npa);
            const float mxv = mxr_s[rl];
            const bool ok = p < N && (int)p != jr_s[rl];
            float d2 = fmaxf(fmaf(-2.f, acc[q], nsum), 0.f);
            if (NEAR && ok && d2 - mxv < kGramNear * nsum) d2 = direct_d2(rows_s + rl * KS, a.xs, p, d, Np);
            T1[rl * PS + pl] = KERN == 0 ? (ok ? mxv - d2 : -INFINITY) : (ok ? d2 : INFINITY);
        }
    }
}

// The tile body's exp2 / split / outer-product MMAs on one step's block, for
// this warp's JW rows (same arithmetic as loo_tile_mma).
template <int G1, int G2, int KERN, int JW, int MT, int NT>
__device__ __forceinline__ void gram_consume(const float* sm, int d, int buf, const float2 (&ca1)[MT],
                                             const float2 (&ca2)[NT], float (&Dt)[JW][MT][NT][4],
                                             float2 (&bt)[JW][MT]) {
    using C = GramCfg<G1, G2>;
    constexpr int R = C::R, PS = C::PS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = lane & 3;
    const float* T1 = sm + C::o_blk(d) + buf * R * PS;
    const float* Ys = sm + C::o_y(d) + buf * C::P;
    const float* rc = sm + C::o_rc(d);
    // this warp's rows' y and y shift
    float yrw[JW], myw[JW];
#pragma unroll
    for (int r = 0; r < JW; ++r) {
        yrw[r] = rc[warp * JW + r];
        myw[r] = rc[2 * R + warp * JW + r];
    }
#pragma unroll 1
    for (int c = 0; c < C::CPS; ++c) {
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
        for (int s = 0; s < 4; ++s) {
#pragma unroll
            for (int r = 0; r < JW; ++r) {
                const int pl = 32 * c + 8 * s + 2 * t;
                const float2 q1 = *reinterpret_cast<const float2*>(T1 + (warp * JW + r) * PS + pl);
                const float2 t1p0 = make_float2(q1.x, q1.x), t1p1 = make_float2(q1.y, q1.y);
                // t2 = m_y - dy^2, at most 0: the left-out point (dy = 0) and padding
                // (their u is 0) then get w <= 1, never an overflow
                const float2 yp = *reinterpret_cast<const float2*>(Ys + pl);
                const float2 dyp = __ffma2_rn(yp, make_float2(-1.f, -1.f), make_float2(yrw[r], yrw[r]));
                float2 t2p;
                if (KERN == 0) {
                    // dy^2 rounded as in the stored shift, so the y-nearest point has t2 = 0 exactly
                    const float2 dy2 = __fmul2_rn(dyp, dyp);
                    t2p = __ffma2_rn(dy2, make_float2(-1.f, -1.f), make_float2(myw[r], myw[r]));
                    t2p = make_float2(fminf(t2p.x, 0.f), fminf(t2p.y, 0.f));
                } else {
                    t2p = __fmul2_rn(dyp, dyp);
                }
                uint32_t bh[NT][2], bx[NT][2];
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const float2 w = KERN == 0 ? gauss_factor2(ca2[nt], t2p, kWc) : kernel_factor2<KERN>(ca2[nt], t2p);
                    const float2 h = make_float2(__uint_as_float(__float_as_uint(w.x) & 0xffffe000u),
                                                 __uint_as_float(__float_as_uint(w.y) & 0xffffe000u));
                    const float2 l = KERN == 0 ? __ffma2_rn(w, make_float2(kWr, kWr), make_float2(-h.x, -h.y))
                                               : __ffma2_rn(h, make_float2(-1.f, -1.f), w);
                    bh[nt][0] = __float_as_uint(h.x);
                    bh[nt][1] = __float_as_uint(h.y);
                    bx[nt][0] = pack_bf16x2(l.x, l.y);
                    bx[nt][1] = pack_bf16x2(h.x, h.y);
                }
                uint32_t ah[MT][4], ax[MT][4];
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const float2 u0 = KERN == 0 ? gauss_factor2(ca1[mt], t1p0, kEx2Fix) : kernel_factor2<KERN>(ca1[mt], t1p0);
                    const float2 u1 = KERN == 0 ? gauss_factor2(ca1[mt], t1p1, kEx2Fix) : kernel_factor2<KERN>(ca1[mt], t1p1);
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
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) mma_tf32(D[r][mt][nt], ah[mt], bh[nt][0], bh[nt][1]);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) mma_bf16(D[r][mt][nt], ax[mt], bx[nt][0], bx[nt][1]);
            }
        }
#pragma unroll
        for (int r = 0; r < JW; ++r)
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; q += 2) {
                        const float2 s2 = __fadd2_rn(make_float2(Dt[r][mt][nt][q], Dt[r][mt][nt][q + 1]),
                                                     make_float2(D[r][mt][nt][q], D[r][mt][nt][q + 1]));
                        Dt[r][mt][nt][q] = s2.x;
                        Dt[r][mt][nt][q + 1] = s2.y;
                    }
    }
}

// Block-wide exclusive scan of one int per thread (512 threads); returns the total.
__device__ __forceinline__ int gram_scan(int v, int* pos, int* misc) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) misc[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < 16 ? misc[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < 16) misc[16 + lane] = wi - w;   // exclusive warp offsets
        if (lane == 15) misc[32] = wi;             // total
    }
    __syncthreads();
    pos[tid] = misc[16 + warp] + incl - v;
    const int total = misc[32];
    __syncthreads();
    return total;
}

// Whether (X, Y) lies in the union of boxes [0, sx[i]] x [0, sy'[i]], given the
// boxes' X extents sorted ascending (sx) and the suffix maxima of their Y
// extents (sy): the first box reaching X decides.
__device__ __forceinline__ bool stair_in(const float* sx, const float* sy, int n, float X, float Y) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (sx[m] < X) lo = m + 1;
        else hi = m;
    }
    return lo < n && Y <= sy[lo];
}

// One fallback pass over a step's block for this warp's rows with flagged cells
// of the current round.  Lanes first take the points (the region tests), then
// the row's cells: each point that passes is broadcast to all lanes, and lane
// f % 32 updates cell f, which only it owns (no atomics; each cell sees the
// points in step, chunk and lane order, so the sums are reproducible).
//   PASS 1: argmin keys (e bits, point) on the block's distances;
//   PASS 2: the shifted sums over the points inside the row's box, with their
//           distances recomputed directly.
template <int G1, int G2, int PASS, int JW>
__device__ __forceinline__ void gram_fb_scan(const LooArgs& a, float* sm, int64_t p0, int buf, float (&fx)[JW],
                                             float (&fy)[JW], unsigned int (&fp)[JW]) {
    using C = GramCfg<G1, G2>;
    constexpr int R = C::R, PS = C::PS, GG = C::GG;
    static_assert(JW == C::JW, "rows per warp");
    constexpr int LG2 = G2 == 8 ? 3 : (G2 == 16 ? 4 : 5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d, KS = C::ks(d);
    const int64_t Np = a.Np;
    const float* rows_s = sm + C::o_rows();
    const float* T1 = sm + C::o_blk(d) + buf * R * PS;
    const float* NPs = sm + C::o_np(d) + buf * C::P;
    const float* Ys = sm + C::o_y(d) + buf * C::P;
    const float* rc = sm + C::o_rc(d);
    const float *yr_s = rc, *mxr_s = rc + R, *myr_s = rc + 2 * R, *nr_s = rc + 3 * R;
    const float *qxr_s = rc + 4 * R, *qyr_s = rc + 5 * R;
    const int* list = reinterpret_cast<const int*>(sm + C::o_list(d));
    unsigned long long* best = reinterpret_cast<unsigned long long*>(sm + C::o_best(d));
    float* sum = sm + C::o_acc(d);
    const float* dxs = sm + C::o_dxs(d);
    const float* dys = sm + C::o_dys(d);
    const float* rp = sm + C::o_rp(d);   // rlo, rhi (per row), rb, rn (ints)
    const int* rbn = reinterpret_cast<const int*>(rp + 4 * R);
    const float* sx = sm + C::o_sx(d);
    const float* sy = sm + C::o_sy(d);
    // the grid's coefficients in shared memory: 32 entries each, one per bank, so
    // lanes reading different cells' coefficients never serialise
    const float* a1s = sm + C::o_cf(d);
    const float* a2s = a1s + 32;
#pragma unroll
    for (int r = 0; r < JW; ++r) {   // unrolled: fx[r], fy[r], fp[r] stay in registers
        const int rl = warp * JW + r;
        const int fb = rbn[rl], fn = rbn[R + rl];
        if (fn == 0) continue;
        const float mxv = mxr_s[rl], myv = myr_s[rl], yv = yr_s[rl], nr = nr_s[rl];
        const float Xh = qxr_s[rl] - mxv, Yh = qyr_s[rl] - myv;
        const float rlo = rp[rl], rhi = rp[R + rl];
        const float rloY = rlo * Yh;
#pragma unroll 1
        for (int c = 0; c < C::CPS; ++c) {
            const int pl = 32 * c + lane;
            const int64_t p = p0 + pl;
            const float t1v = T1[rl * PS + pl];
            const bool live = t1v > -INFINITY;                       // not a masked pair
            const float Xb = -t1v;                                   // the block's X (Gram, or direct if near)
            const float Xg = Xb - kGramSlack * (nr + NPs[pl]);      // lowest the exact X can be
            const float dy = yv - Ys[pl];
            const float dy2 = __fmul_rn(dy, dy);
            const float Y = dy2 - myv;
            if (PASS == 1) {
                // argmin keys on the block's distances: a key that is not the exact
                // minimiser is within 2 a1 times the Gram error of it, which is all the
                // anchor of pass 2 needs (its own distances are then taken directly)
                const bool in = live && Xg <= Xh && Y <= Yh &&
                                ((rlo >= 0.f && fmaf(rlo, Y, Xg) <= rloY) || (rhi < INFINITY && fmaf(rhi, Y, Xg) <= Xh));
                // Every cell's minimiser is on the region's Pareto front (no other point
                // has both a smaller X and a smaller Y): the warp keeps the row's front,
                // one entry per lane (free entries hold +inf), and the cells are scored on
                // it once the pass is done.  A point that finds the front full updates
                // the cells directly instead.
                unsigned int m = __ballot_sync(0xffffffffu, in);
                const float X = fmaxf(Xb, 0.f);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const float Xq = __shfl_sync(0xffffffffu, X, src), Yq = __shfl_sync(0xffffffffu, Y, src);
                    const unsigned int pq = (unsigned int)(p0 + 32 * c + src);
                    if (__ballot_sync(0xffffffffu, fx[r] <= Xq && fy[r] <= Yq)) continue;   // dominated
                    if (Xq <= fx[r] && Yq <= fy[r]) fx[r] = fy[r] = INFINITY;               // entries it dominates
                    const unsigned int fr = __ballot_sync(0xffffffffu, fx[r] == INFINITY);
                    if (fr) {
                        if (lane == __ffs(fr) - 1) {
                            fx[r] = Xq;
                            fy[r] = Yq;
                            fp[r] = pq;
                        }
                    } else {
                        for (int f = fb + lane; f < fb + fn; f += 32) {
                            const int kl = list[f] - rl * GG, k = kl >> LG2, l = kl & (G2 - 1);
                            const float e = fmaxf(fmaf(a1s[k], Xq, a2s[l] * Yq), 0.f);
                            const unsigned long long key = ((unsigned long long)__float_as_uint(e) << 32) | pq;
                            if (key < best[f]) best[f] = key;
                        }
                    }
                }
            } else {
                (void)fx; (void)fy; (void)fp;
                // the region's points with their distances recomputed directly (few: each
                // lane recomputes its own point; the result is then broadcast to the cells)
                const bool pre = live && stair_in(sx + fb, sy + fb, fn, Xg, Y);
                float d2 = 0.f;
                if (pre) d2 = direct_d2(rows_s + rl * KS, a.xs, p, d, Np);
                const bool in = pre && stair_in(sx + fb, sy + fb, fn, d2 - mxv, Y);
                unsigned int m = __ballot_sync(0xffffffffu, in);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const float d2q = __shfl_sync(0xffffffffu, d2, src), dy2q = __shfl_sync(0xffffffffu, dy2, src);
                    for (int f = fb + lane; f < fb + fn; f += 32) {
                        const int kl = list[f] - rl * GG, k = kl >> LG2, l = kl & (G2 - 1);
                        sum[f] += ex2_approx(kFbEx2Fix - (a1s[k] * (d2q - dxs[f]) + a2s[l] * (dy2q - dys[f])));
                    }
                }
            }
        }
    }
}

template <int G1, int G2, int KERN, class Coef>
__device__ __forceinline__ void gram_unit(const LooArgs& a, const Coef& cf, int u, int tile, bool first,
                                          float* sm) {
    using C = GramCfg<G1, G2>;
    constexpr int R = C::R, P = C::P, JW = C::JW, MT = C::MT, NT = C::NT, GG = C::GG, NTH = C::kThreads;
    constexpr int LG2 = G2 == 8 ? 3 : (G2 == 16 ? 4 : 5);
    constexpr double LN2 = 0.69314718055994530942;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int d = a.d, KS = C::ks(d), KP = KS - 4;
    const int64_t N = a.N, Np = a.Np;
    float* rows_s = sm + C::o_rows();
    float* rc = sm + C::o_rc(d);
    float *yr_s = rc, *mxr_s = rc + R, *myr_s = rc + 2 * R, *nr_s = rc + 3 * R;
    float *qxr_s = rc + 4 * R, *qyr_s = rc + 5 * R;
    int* jr_s = reinterpret_cast<int*>(rc + 6 * R);
    int* vr_s = reinterpret_cast<int*>(rc + 7 * R);
    float* At_s = sm + C::o_at(d);
    double* btl_s = reinterpret_cast<double*>(sm + C::o_btl(d));
    unsigned int* flag = reinterpret_cast<unsigned int*>(sm + C::o_flag(d));
    int* pos = reinterpret_cast<int*>(sm + C::o_pos(d));
    int* misc = reinterpret_cast<int*>(sm + C::o_misc(d));

    // ---- the unit's rows ----
    __syncthreads();
    for (int r = tid; r < R; r += NTH) {
        const int64_t rr = (int64_t)u * R + r;
        const bool v = rr < a.n_rows;
        const int64_t r0 = v ? rr : 0;
        const int64_t j = CDE_CK(a.rows ? a.rows[CDE_CK(r0, a.n_rows, 122)] : r0, N, 123);
        jr_s[r] = (int)j;
        vr_s[r] = v;
        yr_s[r] = a.y[j];
        mxr_s[r] = a.mx[j];
        myr_s[r] = a.my[j];
        qxr_s[r] = KERN == 0 ? a.qx[j] : 0.f;
        qyr_s[r] = KERN == 0 ? a.qy[j] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < R * KP; e += NTH) {
        const int r = e / KP, c = e - r * KP;
        rows_s[r * KS + c] = c < d ? a.xs[(int64_t)c * Np + jr_s[r]] : 0.f;
    }
    __syncthreads();
    for (int r = tid; r < R; r += NTH) {
        float n = 0.f;
        for (int c = 0; c < d; ++c) n = fmaf(rows_s[r * KS + c], rows_s[r * KS + c], n);
        nr_s[r] = n;
    }
    // the grid's coefficients in shared memory (read below with a different cell per
    // thread: from the parameter block such reads would serialise)
    float* a1s = sm + C::o_cf(d);
    float* a2s = a1s + 32;
    double* lam1s = reinterpret_cast<double*>(a1s + 64);
    double* kap2s = lam1s + 32;
    if (tid < 32) {
        a1s[tid] = cf.a1(tid);
        a2s[tid] = cf.a2(tid);
        lam1s[tid] = a.lam1[tid];
        kap2s[tid] = a.kap2[tid];
    }

    float2 ca1[MT], ca2[NT];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) ca1[mt] = make_float2(cf.a1(16 * mt + g), cf.a1(16 * mt + g + 8));
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) ca2[nt] = make_float2(cf.a2(8 * nt + g), cf.a2(8 * nt + g));
    float Dt[JW][MT][NT][4];
    float2 bt[JW][MT];
#pragma unroll
    for (int r = 0; r < JW; ++r)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            bt[r][mt] = make_float2(0.f, 0.f);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) Dt[r][mt][nt][q] = 0.f;
        }
    __syncthreads();

    // ---- main pass over the points ----
    const int64_t n_steps = (N + P - 1) / P;
    gram_block<G1, G2, KERN, true>(a, sm, 0, 0);
    __syncthreads();
    for (int64_t s = 0; s < n_steps; ++s) {
        const int b = (int)(s & 1);
        if (s + 1 < n_steps) gram_block<G1, G2, KERN, true>(a, sm, (s + 1) * P, b ^ 1);
        gram_consume<G1, G2, KERN, JW, MT, NT>(sm, d, b, ca1, ca2, Dt, bt);
        __syncthreads();
    }

    // ---- per-row totals to shared memory ----
#pragma unroll
    for (int r = 0; r < JW; ++r) {
        const int rl = warp * JW + r;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = 16 * mt + g + 8 * (q >> 1), l = 8 * nt + 2 * t + (q & 1);
                    At_s[rl * GG + k * G2 + l] = Dt[r][mt][nt][q];
                }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v = h ? bt[r][mt].y : bt[r][mt].x;
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                if (t == 0) btl_s[rl * G1 + 16 * mt + g + 8 * h] = log2_wide(v);
            }
        }
    }
    __syncthreads();

    // ---- cells below the recompute threshold: exact two-pass recomputation ----
    double* fbv = a.fb + (size_t)blockIdx.x * C::CELLS;   // this CTA's recomputed log2 At
    unsigned int fw = 0;
    if (KERN == 0) {
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
            const int cell = 32 * tid + b, kl = cell % GG;
            // cells of the padded grid (the last bandwidth repeated) are never output
            const bool real = (kl >> LG2) < a.G1r && (kl & (G2 - 1)) < a.G2r;
            if (vr_s[cell / GG] && real && At_s[cell] < a.thresh) fw |= 1u << b;
        }
    }
    flag[tid] = fw;
    const int total = gram_scan(__popc(fw), pos, misc);
    if (KERN == 0 && total > 0) {
        int* list = reinterpret_cast<int*>(sm + C::o_list(d));
        unsigned long long* best = reinterpret_cast<unsigned long long*>(sm + C::o_best(d));
        float* sum = sm + C::o_acc(d);
        float* dxs = sm + C::o_dxs(d);
        float* dys = sm + C::o_dys(d);
        float* rp = sm + C::o_rp(d);
        int* rbn = reinterpret_cast<int*>(rp + 4 * R);
        int lg = 0;
        while (((int64_t)1 << lg) < N) ++lg;
        const float T = (float)(32 + lg);
        for (int base = 0; base < total; base += C::FMAX) {
            const int n = min(C::FMAX, total - base);
            {   // the round's cells, in (row, k, l) order
                unsigned int bits = flag[tid];
                int q = pos[tid];
                while (bits) {
                    const int bb = __ffs(bits) - 1;
                    bits &= bits - 1;
                    if (q >= base && q < base + n) list[q - base] = 32 * tid + bb;
                    ++q;
                }
            }
            for (int f = tid; f < n; f += NTH) {
                best[f] = ~0ull;
                sum[f] = 0.f;
            }
            __syncthreads();
            // per row: its range of the list, and the argmin region's triangles
            for (int rl = tid; rl < R; rl += NTH) {
                int lo = 0, hi = n;   // first entry of row rl
                while (lo < hi) {
                    const int m = (lo + hi) >> 1;
                    if (list[m] / GG < rl) lo = m + 1;
                    else hi = m;
                }
                int e = lo;
                while (e < n && list[e] / GG == rl) ++e;
                rbn[rl] = lo;
                rbn[R + rl] = e - lo;
                const float Xh = qxr_s[rl] - mxr_s[rl], Yh = qyr_s[rl] - myr_s[rl];
                float rlo = -1.f, rhi = INFINITY;
                for (int f = lo; f < e; ++f) {
                    const int kl = list[f] - rl * GG;
                    const float rho = a2s[kl & (G2 - 1)] / a1s[kl >> LG2];
                    if (rho * Yh <= Xh) rlo = fmaxf(rlo, rho);
                    else rhi = fminf(rhi, rho);
                }
                rp[rl] = rlo;
                rp[R + rl] = rhi;
            }
            __syncthreads();
            // pass 1: argmin keys (via each row's Pareto front)
            float fx[JW], fy[JW];
            unsigned int fp[JW];
#pragma unroll
            for (int r = 0; r < JW; ++r) {
                fx[r] = fy[r] = INFINITY;
                fp[r] = 0u;
            }
            gram_block<G1, G2, KERN, false>(a, sm, 0, 0);
            __syncthreads();
            for (int64_t s = 0; s < n_steps; ++s) {
                const int b = (int)(s & 1);
                if (s + 1 < n_steps) gram_block<G1, G2, KERN, false>(a, sm, (s + 1) * P, b ^ 1);
                gram_fb_scan<G1, G2, 1, JW>(a, sm, s * P, b, fx, fy, fp);
                __syncthreads();
            }
            // score the cells on their row's front (lane = cell)
#pragma unroll
            for (int r = 0; r < JW; ++r) {
                const int rl = warp * JW + r;
                const int fb = rbn[rl], fn = rbn[R + rl];
                if (fn == 0) continue;
                const unsigned int valid = __ballot_sync(0xffffffffu, fx[r] < INFINITY);
                for (int f0 = fb; f0 < fb + fn; f0 += 32) {
                    const int f = f0 + lane;
                    const bool own = f < fb + fn;
                    const int kl = own ? list[f] - rl * GG : 0, k = kl >> LG2, l = kl & (G2 - 1);
                    unsigned long long bk = own ? best[f] : ~0ull;
                    unsigned int vm = valid;
                    while (vm) {
                        const int src = __ffs(vm) - 1;
                        vm &= vm - 1;
                        const float Xq = __shfl_sync(0xffffffffu, fx[r], src), Yq = __shfl_sync(0xffffffffu, fy[r], src);
                        const unsigned int pq = __shfl_sync(0xffffffffu, fp[r], src);
                        const float e = fmaxf(fmaf(a1s[k], Xq, a2s[l] * Yq), 0.f);
                        const unsigned long long key = ((unsigned long long)__float_as_uint(e) << 32) | pq;
                        bk = key < bk ? key : bk;
                    }
                    if (own) best[f] = bk;
                }
            }
            __syncthreads();
            // the anchors' direct distances (a cell with no key, which the x- and the
            // y-nearest points rule out, is anchored at the x-nearest bound: X = 0, Y = Yh)
            for (int f = tid; f < n; f += NTH) {
                const int rl = list[f] / GG;
                const unsigned long long bk = best[f];
                if (bk == ~0ull) {
                    dxs[f] = mxr_s[rl];
                    dys[f] = qyr_s[rl];
                } else {
                    const int64_t ps = CDE_CK((int64_t)(unsigned int)bk, N, 124);
                    dxs[f] = direct_d2(rows_s + rl * KS, a.xs, ps, d, Np);
                    const float dy = yr_s[rl] - a.y[ps];
                    dys[f] = __fmul_rn(dy, dy);
                }
            }
            __syncthreads();
            // the region of pass 2: a cell's terms exceed 2^-T only at X <= (e_* + T)/a1,
            // Y <= (e_* + T)/a2; a row's region is the union of its cells' boxes, kept
            // as a staircase: the boxes sorted by X extent (ties by position) with the
            // largest Y extent at or beyond each (a point is in the union iff its
            // Y <= that of the first box reaching its X)
            float* sx = sm + C::o_sx(d);
            float* sy = sm + C::o_sy(d);
            for (int f = tid; f < n; f += NTH) {
                const int rl = list[f] / GG, kl = list[f] - rl * GG, k = kl >> LG2, l = kl & (G2 - 1);
                const float es = fmaxf(fmaf(a1s[k], dxs[f] - mxr_s[rl], a2s[l] * (dys[f] - myr_s[rl])), 0.f);
                const float rx = (es + T) / a1s[k], ry = (es + T) / a2s[l];
                int rank = rbn[rl];
                for (int g2 = rbn[rl]; g2 < rbn[rl] + rbn[R + rl]; ++g2) {
                    if (g2 == f) continue;
                    const int kl2 = list[g2] - rl * GG, k2 = kl2 >> LG2, l2 = kl2 & (G2 - 1);
                    const float es2 = fmaxf(fmaf(a1s[k2], dxs[g2] - mxr_s[rl], a2s[l2] * (dys[g2] - myr_s[rl])), 0.f);
                    const float rx2 = (es2 + T) / a1s[k2];
                    rank += (rx2 < rx || (rx2 == rx && g2 < f));
                }
                sx[rank] = rx;
                sy[rank] = ry;
            }
            __syncthreads();
            for (int rl = tid; rl < R; rl += NTH) {
                float m = -1.f;
                for (int f = rbn[rl] + rbn[R + rl] - 1; f >= rbn[rl]; --f) {
                    m = fmaxf(m, sy[f]);
                    sy[f] = m;
                }
            }
            __syncthreads();
            // pass 2: the sums
            gram_block<G1, G2, KERN, false>(a, sm, 0, 0);
            __syncthreads();
            for (int64_t s = 0; s < n_steps; ++s) {
                const int b = (int)(s & 1);
                if (s + 1 < n_steps) gram_block<G1, G2, KERN, false>(a, sm, (s + 1) * P, b ^ 1);
                gram_fb_scan<G1, G2, 2, JW>(a, sm, s * P, b, fx, fy, fp);
                __syncthreads();
            }
            for (int f = tid; f < n; f += NTH) {
                const int cell = list[f], rl = cell / GG, kl = cell - rl * GG, k = kl >> LG2, l = kl & (G2 - 1);
                const float tot = sum[f];
                const double es = (double)a1s[k] * ((double)dxs[f] - (double)mxr_s[rl]) +
                                  (double)a2s[l] * ((double)dys[f] - (double)myr_s[rl]);
                fbv[cell] = -es + log2_wide(tot);
            }
            __syncthreads();
        }
    }

    // ---- FP64 log-ratios, summed over the unit's rows in row order ----
    __threadfence_block();
    __syncthreads();
    constexpr int NOWN = GG > NTH ? GG / NTH : 1;
    double sc[NOWN], se[NOWN];
#pragma unroll
    for (int s = 0; s < NOWN; ++s) sc[s] = se[s] = 0.0;
    for (int rl = 0; rl < R; ++rl) {
        if (!vr_s[rl]) continue;
        const double shy_m = (double)myr_s[rl], shx_m = (double)mxr_s[rl];
#pragma unroll
        for (int s = 0; s < NOWN; ++s) {
            const int kl = tid + NTH * s;
            if (kl >= GG) continue;
            const int k = kl >> LG2, l = kl & (G2 - 1);
            const int cell = rl * GG + kl;
            const bool fl = (flag[cell >> 5] >> (cell & 31)) & 1u;
            const double lA = fl ? fbv[cell] : log2_wide(At_s[cell]);
            const double a1k = (double)a1s[k], a2l = (double)a2s[l];
            const double shy = a2l * shy_m;
            const double ell = lA == -INFINITY ? -INFINITY : LN2 * (lA - btl_s[rl * G1 + k] - shy) - kap2s[l];
            const double lnA = LN2 * (lA - a1k * shx_m - shy) - lam1s[k] - kap2s[l];
            sc[s] += ell;
            se[s] += lnA;
            if (a.ell_rows && k < a.G1r && l < a.G2r) {
                const int64_t r = CDE_CK((int64_t)u * R + rl, a.n_rows, 125);
                a.ell_rows[r * a.ell_ld_row + (int64_t)k * a.ell_ld_k + l] = ell;
            }
        }
    }
    // the tile's partial slot: its first unit stores, the others add in order
    double* part = a.part + (size_t)CDE_CK(tile, a.n_tiles, 126) * 2 * GG;
#pragma unroll
    for (int s = 0; s < NOWN; ++s) {
        const int kl = tid + NTH * s;
        if (kl >= GG) continue;
        if (first) {
            part[kl] = sc[s];
            part[GG + kl] = se[s];
        } else {
            part[kl] += sc[s];
            part[GG + kl] += se[s];
        }
    }
}

template <int G1, int G2, int KERN>
__global__ void __launch_bounds__(512, 1) k_loo_gram(const LooArgs a) {
    extern __shared__ float4 sm4[];
    __shared__ int next_tile;
    __shared__ int ls_u, ls_end, ls_stride, ls_first;
    const CoefParam cf{a};
    for (int t0 = blockIdx.x;; t0 += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) next_tile = a.work ? atomicAdd(a.work, 1) : t0;
        __syncthreads();
        const int t = next_tile;
        if (t >= a.n_tiles) break;
        // the tile's units; the loop state lives in shared memory (thread 0 advances
        // it, every thread reads it after a barrier), not in registers through the body
        if (threadIdx.x == 0) {
            int u_first, u_stride, u_len;
            loo_tile_span(a, t, u_first, u_stride, u_len);
            ls_u = u_first + max(a.win0, 0) * u_stride;
            ls_end = u_first + min(u_len, a.win1) * u_stride;
            ls_stride = u_stride;
            ls_first = u_first;
        }
        for (;;) {
            __syncthreads();
            const int u = ls_u;
            if (u >= ls_end) break;
            gram_unit<G1, G2, KERN>(a, cf, u, next_tile, u == ls_first, reinterpret_cast<float*>(sm4));
            // (every thread read ls_u before the barriers of the unit's body)
            if (threadIdx.x == 0) ls_u += ls_stride;
        }
    }
}

// 227 KB: the opt-in shared memory of a CTA, less room for the static part
constexpr int kSmemOptin = 232448 - 1024;

template <int G1, int G2, int KERN>
static int launch_gram_k(const LooArgs& a, int grid, cudaStream_t st) {
    using C = GramCfg<G1, G2>;
    static std::atomic<uint64_t> attr{0};
    const size_t big = C::smem_bytes(kMaxD) < (size_t)kSmemOptin ? C::smem_bytes(kMaxD) : (size_t)kSmemOptin;
    CDE_CUDA(smem_attr_once(attr, k_loo_gram<G1, G2, KERN>, (int)big));
    k_loo_gram<G1, G2, KERN><<<grid, C::kThreads, C::smem_bytes(a.d), st>>>(a);
    CDE_CUDA(cudaGetLastError());
    return CDE_OK;
}

int loo_gram_rows_per_unit(int T1, int T2) { return 16 * (1024 / (T1 * T2)); }

size_t loo_gram_smem_bytes(int T1, int T2, int d) {
#define CDE_GSHAPE(A, B) \
    if (T1 == A && T2 == B) return GramCfg<A, B>::smem_bytes(d);
    CDE_GSHAPE(16, 8) CDE_GSHAPE(16, 16) CDE_GSHAPE(16, 32)
    CDE_GSHAPE(32, 8) CDE_GSHAPE(32, 16) CDE_GSHAPE(32, 32)
#undef CDE_GSHAPE
    return (size_t)1 << 30;
}

bool loo_use_gram(const Dataset& D, int T1, int T2) {
    return D.d >= kGramMinD && loo_gram_smem_bytes(T1, T2, D.d) <= (size_t)kSmemOptin;
}

size_t loo_gram_fb_bytes_per_cta() { return (size_t)16384 * sizeof(double); }

int launch_loo_gram(int T1, int T2, const LooArgs& a, int grid, cudaStream_t st) {
#define CDE_GSHAPE(A, B)                                                                     \
    if (T1 == A && T2 == B)                                                                  \
        return a.kern == CDE_KERNEL_EPAN ? launch_gram_k<A, B, 1>(a, grid, st)               \
                                         : launch_gram_k<A, B, 0>(a, grid, st);
    CDE_GSHAPE(16, 8) CDE_GSHAPE(16, 16) CDE_GSHAPE(16, 32)
    CDE_GSHAPE(32, 8) CDE_GSHAPE(32, 16) CDE_GSHAPE(32, 32)
#undef CDE_GSHAPE
    return set_error(CDE_EINVAL, "unsupported grid block shape");
}

#ifdef CDE_CHECKS
CDE_CHECK_READER(check_status_gram)
#endif

}  // namespace cde
