// Element contraction on the tensor cores, error-free (WQ_PREC_TC).
//
// The element blocks of Eqs. 9, 11, 12 and S,
//     K_e[a][b] = sum_{t, q} s^t_{aq} T^t_{qb}
// (s: weights times coefficient, or Gauss weight times coefficient times test
// function; T: trial table), are small dense products: 16 x 16 tiles with K =
// (terms) x (points of e) mostly 16..32.  They go to the tensor cores through an
// error-free splitting of the operands (the idea of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines of
// matrix multiplication and its applications", Numer. Algorithms 59, 2012):
//  * the trial side of element e, component c, is scaled by 2^(8 - f), 2^f > max|T|
//    over the element, and rounded into 5 slices of 8 bits, T 2^(8-f) =
//    sum_l b_l 2^(-8 l) with integers |b_0| <= 256, |b_l| <= 128 (exact bf16), to
//    2^-33 of 256 (set-up, from the FP64 table);
//  * the test side of row a is scaled by 2^(f_t + 8 - E_a), 2^E_a > max_{t,q} |s^t_aq|
//    2^(f_t) (the bound from per-function maxima of the weights and the largest
//    coefficient of the element), and sliced the same way at run time from the split
//    (hi, lo) products;
//  * every product a_k b_l of bf16 integers is exact, and a level sum
//    D_d = sum_{k + l = d} sum_K a_k b_l has |D_d| <= 114,816 K < 2^24 for K <= 128, so
//    the FP32 accumulation of the MMA adds integers exactly;
//  * K_e[a][b] = 2^(E_a - 16) sum_{d <= 4} 2^(-8 d) D_d, the pairs with k + l > 4
//    dropped (below 2^-40 of the tile's product scale).
// The error is relative to the tile's largest |s| |T| K, not to each entry: the weights
// of ill-conditioned rows span several decades with cancelling signs.  Five slices, and
// a fold that keeps D_0 + 2^-8 D_1 as an exact TwoSum pair, put the 24,576-element
// sphere bilaplacian at the FP32 rounding of the values (four slices with a plain FP32
// fold: 1e-5 normwise).  The SIMT work is per (row, point, term) -- split product and 5
// slices, ~24 instructions -- instead of per (row, column, point, term).
//
// Persistent warps, one 16 x 16 tile at a time (the FP32 path's tiles and slot map; the
// next tile's descriptors are prefetched).  K is walked in quarter-chunks of 4 points
// of one term (each term's points padded to a multiple of 4), two quarters per
// m16n8k8 step: lane (g, t4) = (lane / 4, lane % 4) takes the quarter t4 / 2 selects
// and builds the A fragments of its rows g, g + 8 at that quarter's points
// 2 (t4 % 2), 2 (t4 % 2) + 1, loads the trial fragments precomputed in that order (one
// 8-byte load per slice), and runs 15 slice pairs x 2 n-tiles of mma.sync into 5 level
// accumulators; the next half-chunk's loads are in flight meanwhile.  Every 16
// half-chunks (K = 128) the levels are added to the tile's slots (a TwoSum against the
// earlier segments), so any K is exact.
#include <algorithm>

#include <cuda_bf16.h>

#include "kernels.h"

namespace wqd {

constexpr int TC_NWARP = 4;     // warps per block
constexpr int TC_PMAX = 64;     // points per element (WQ side^2, Gauss 16 nsub)
constexpr int TC_NS = WQ_TC_SLICES;        // slices per operand
constexpr int TC_QW = WQ_TC_QUARTER_WORDS; // trial-slice words per (quarter-chunk, column block)
constexpr int TC_SEGH = 16;                // half-chunks per exact segment: K <= 128
constexpr int TC_BLOCKS_PER_SM = 4;   // resident blocks at the register budget (no spills)

__device__ __forceinline__ float tc_warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void tc_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// 2^e as a float (0 below the normal range, clamped above).
__device__ __forceinline__ float exp2i(int e) {
    e = min(e, 127);
    return e < -126 ? 0.0f : __int_as_float((e + 127) << 23);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// Five 8-bit slices of y = yh + yl (|y| <= 256, |yl| <= ulp(yh) / 2): integers k_s with
// y = k0 + 2^-8 k1 + ... + 2^-32 k4 to 2^-33.  Rounding to an integer adds and subtracts
// 1.5 2^23 (FMA pipe; rintf runs on the slower conversion pipe).  The remainders
// yh - k0 and r 2^8 - k1 are exact; yl enters at the third slice (|k2| <= 129) and the
// remainder after it, (t - k2) + yl, is kept to 2^-24 of itself, far below k4's unit.
__device__ __forceinline__ void slice5(float yh, float yl, float (&k)[TC_NS]) {
    const float M = 12582912.0f;
    k[0] = __fsub_rn(__fadd_rn(yh, M), M);
    float r = yh - k[0];
    k[1] = __fsub_rn(__fmaf_rn(r, 256.0f, M), M);
    r = __fmaf_rn(r, 256.0f, -k[1]);
    const float t = r * 256.0f, yl2 = yl * 65536.0f;
    k[2] = __fsub_rn(__fadd_rn(t + yl2, M), M);
    r = (t - k[2]) + yl2;
    k[3] = __fsub_rn(__fmaf_rn(r, 256.0f, M), M);
    r = __fmaf_rn(r, 256.0f, -k[3]);
    k[4] = __fsub_rn(__fmaf_rn(r, 256.0f, M), M);
}

// Two integers |k| <= 256 as a bf16x2 word (low = first): their FP32 encodings have
// zero low halves, so the bf16 encodings are the high halves (one byte permute).
__device__ __forceinline__ uint32_t pack_int_bf16x2(float lo, float hi) {
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// Smallest E with 2^E > x (x > 0, finite): the frexp exponent, from the encoding for
// normal x.
__device__ __forceinline__ int exp_above(float x) {
    const unsigned e = (__float_as_uint(x) >> 23) & 255u;
    if (e != 0u) return (int)e - 126;
    int ex;
    frexpf(x, &ex);
    return ex;
}

__device__ __forceinline__ void tc_cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}

// Operands of one half-chunk (8 points of one term): this lane's test-side values
// (rows g, g + 8 at points 2 t4, 2 t4 + 1) and its trial-side fragment words.
struct Half {
    float2 v[4];     // [row][point]
    uint2 b[TC_NS];  // per slice: the words of n-tiles 0 and 1
    int t, q;        // this lane's term and first point (t < 0: beyond the last quarter)
};

// Per-tile constants of the test-side loads: element base, row strides, validity.
struct TileV {
    const float2* base;
    int r0, r1;          // offsets of rows g, g + 8 (-1: beyond m)
    int qs, cs;          // stride of a point, of a column / component
};

// This lane's quarter-chunk (term t, quarter qq) of a half-chunk: its trial fragment
// words and test-side values.
__device__ __forceinline__ void load_half(Half& H, const TileV& tv, const int (*sT)[2], int t, int qq, int P,
                                          int t4, const uint32_t* __restrict__ bsl) {
    H.t = t;
    H.q = 4 * qq + 2 * (t4 & 1);
    const float2 z = make_float2(0.0f, 0.0f);
    if (t < 0) {
#pragma unroll
        for (int l = 0; l < TC_NS; ++l) H.b[l] = make_uint2(0u, 0u);
#pragma unroll
        for (int x = 0; x < 4; ++x) H.v[x] = z;
        return;
    }
    const uint32_t* bp = bsl + sT[t][1] + qq * TC_QW;
#pragma unroll
    for (int l = 0; l < TC_NS; ++l) H.b[l] = __ldg(reinterpret_cast<const uint2*>(bp + l * 32));
    const int q = H.q;
    const float2* vb = tv.base + q * tv.qs + sT[t][0] * tv.cs;
    const bool q0 = q < P, q1 = q + 1 < P;
    H.v[0] = (tv.r0 >= 0 && q0) ? __ldg(vb + tv.r0) : z;
    H.v[1] = (tv.r0 >= 0 && q1) ? __ldg(vb + tv.qs + tv.r0) : z;
    H.v[2] = (tv.r1 >= 0 && q0) ? __ldg(vb + tv.r1) : z;
    H.v[3] = (tv.r1 >= 0 && q1) ? __ldg(vb + tv.qs + tv.r1) : z;
}

template <int NT, bool GAUSS>
__global__ void __launch_bounds__(TC_NWARP * 32, TC_BLOCKS_PER_SM)
    k_elem_tc(TcItems it, TcSrc src, const double* __restrict__ coef, TermsF tm) {
    __shared__ __align__(16) float2 sMul[TC_NWARP][NT][TC_PMAX];   // per-term multipliers at the points
    __shared__ int sTerm[TC_NWARP][NT][2];                          // test column, slice block
    __shared__ float sSg[TC_NWARP][NT][2][32];                      // per (term, row, lane) slice scale
    __shared__ int sSlot[TC_NWARP][8][32];                          // destination slots per (entry, lane)
    __shared__ int sItem[TC_NWARP][2][12];                          // tile descriptors, double-buffered
    __shared__ __align__(16) float2 sCr[TC_NWARP][4][TC_PMAX];      // split coefficient rows at the points
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * TC_NWARP;
    int64_t k = (int64_t)blockIdx.x * TC_NWARP + wib;
    if (k >= it.n) return;
    // persistent warps: tiles k, k + nw, ...; the next tile's descriptors are copied in
    // the background while this one is processed
    auto fetch_item = [&](int64_t kk, int b) {
        if (lane < 4) tc_cp_async4(&sItem[wib][b][lane], reinterpret_cast<const int*>(it.item + kk) + lane);
        else if (lane < 8) tc_cp_async4(&sItem[wib][b][lane], reinterpret_cast<const int*>(it.it2 + kk) + lane - 4);
        else if (lane == 8) tc_cp_async4(&sItem[wib][b][8], it.kb + kk);
    };
    fetch_item(k, 0);
    for (int buf = 0; k < it.n; k += nw, buf ^= 1) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncwarp();
        const int* si = sItem[wib][buf];
        const int4 d = make_int4(si[0], si[1], si[2], si[3]);
        const int4 d2 = make_int4(si[4], si[5], si[6], si[7]);
        const int kb = si[8];
        if (k + nw < it.n) fetch_item(k + nw, buf ^ 1);
        const int m = d.z & 255, P = (d.z >> 8) & 255, a0 = ((d.z >> 16) & 15) * 16, b0 = ((d.z >> 20) & 15) * 16;
        const int qpt = d2.w >> 2, ncb = (m + 15) >> 4;   // quarter-chunks per term
        const int g = lane >> 2, t4 = lane & 3, ra = a0 + g;
        const int nt = tm.nt, nc = src.nc, nv = GAUSS ? src.nc : src.nwc;
        int(*sT)[2] = sTerm[wib];
        int f8[NT];   // f_t + 8 per term (uniform)
        if (lane < nt) {
#pragma unroll
            for (int t = 0; t < NT; ++t)
                if (t == lane) {
                    sT[t][0] = GAUSS ? tm.sc[t] : tm.wc[t];
                    sT[t][1] = (tm.tc[t] * ncb + (b0 >> 4)) * qpt * TC_QW;
                }
        }
        __syncwarp();
        TileV tv;
        tv.base = GAUSS ? src.vsrc + d.x : src.vsrc + (int64_t)d.w * nv;
        tv.r0 = ra < m ? (GAUSS ? ra : ra * nv) : -1;
        tv.r1 = ra + 8 < m ? (GAUSS ? ra + 8 : (ra + 8) * nv) : -1;
        tv.qs = GAUSS ? nc * m : m * nv;
        tv.cs = GAUSS ? m : 1;
        const uint32_t* __restrict__ bsl = src.bs + d2.y + ((t4 & 1) * 8 + g) * 2;
        // quarter-chunks: lanes t4 < 2 take the even quarter of a half-chunk, t4 >= 2 the
        // odd one; (tq, qq) = this lane's quarter, advanced by two per half-chunk
        const int nq = nt * qpt;
        int tq = 0, qq = t4 >> 1;
        auto advance = [&]() {
            qq += 2;
            while (qq >= qpt && tq < nt) qq -= qpt, ++tq;
        };
        if (qq >= qpt) qq -= qpt, ++tq;
        // first half-chunk's operands in flight while the scales are set up
        Half h0;
        load_half(h0, tv, sT, tq < nt ? tq : -1, qq, P, t4, bsl);
        // destination slots of this lane's 8 entries (rows g, g + 8; columns 2 t4, 2 t4 + 1
        // of both n-tiles), copied to shared memory in the background
        {
            const int32_t* sp = src.scat + kb + ra * m + b0 + 2 * t4;
            const int bc = b0 + 2 * t4;
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const int dr = 8 * (x >> 2), dc = 8 * ((x >> 1) & 1) + (x & 1);
                if (ra + dr < m && bc + dc < m) tc_cp_async4(&sSlot[wib][x][lane], sp + dr * m + dc);
                else sSlot[wib][x][lane] = -1;
            }
        }
        float vm[2][NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            f8[t] = t < nt ? __ldg(src.fexp + (int64_t)d2.z * nc + tm.tc[t]) + 8 : 0;
            const int vc = GAUSS ? tm.sc[t] : tm.wc[t];
            const float* vr = src.vmax + (int64_t)(d2.x + ra) * nv + vc;
            vm[0][t] = (t < nt && ra < m) ? __ldg(vr) : 0.0f;
            vm[1][t] = (t < nt && ra + 8 < m) ? __ldg(vr + 8 * nv) : 0.0f;
        }
        // per-term multipliers (split pairs) at the element's points, zero up to P4
        float2(*M)[TC_PMAX] = sMul[wib];
        float cmax[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) cmax[t] = 0.0f;
        // the coefficient rows split once per point (a runtime loop over the rows used)
        float2(*CR)[TC_PMAX] = sCr[wib];
#pragma unroll 1
        for (int r = 0; r < tm.ncrow; ++r)
            for (int q = lane; q < 4 * qpt; q += 32) {
                float2 c = make_float2(0.0f, 0.0f);
                if (q < P) c = coef ? split_double(coef[r * tm.cstride + d.y + q]) : make_float2(1.0f, 0.0f);
                CR[r][q] = c;
            }
        __syncwarp();
        for (int q = lane; q < 4 * qpt; q += 32) {
            const bool in = q < P;
            const float2 gq = GAUSS && in ? src.gw2[d.y + q] : make_float2(1.0f, 0.0f);
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int c = tm.crow[t];
                float2 v = c >= 0 ? CR[c][q] : make_float2(tm.shi[t], tm.slo[t]);
                if (GAUSS) {
                    const float ph = v.x * gq.x;
                    v = make_float2(ph, fmaf(v.x, gq.x, -ph) + fmaf(v.x, gq.y, v.y * gq.x));
                }
                if (!in) v = make_float2(0.0f, 0.0f);
                M[t][q] = v;
                cmax[t] = fmaxf(cmax[t], fabsf(v.x));
            }
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) cmax[t] = tc_warp_max(cmax[t]);
        // row exponents 2^E > max_t vmax[row][v_t] cmax_t 2^f_t, the slice scales
        // 2^(f_t + 8 - E) per (term, row) and the entries' scales 2^(E - 16)
        float esc[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            float bound = 0.0f;
#pragma unroll
            for (int t = 0; t < NT; ++t)
                if (t < nt) bound = fmaxf(bound, vm[rr][t] * cmax[t] * exp2i(f8[t] - 8));
            const int E = bound > 0.0f ? exp_above(bound * (1.0f + 0x1p-20f)) : 0;
#pragma unroll
            for (int t = 0; t < NT; ++t) sSg[wib][t][rr][lane] = exp2i(f8[t] - E);
            esc[rr] = exp2i(E - 16);
        }
        __syncwarp();

        float acc[TC_NS][2][4];
#pragma unroll
        for (int l = 0; l < TC_NS; ++l)
#pragma unroll
            for (int n = 0; n < 2; ++n)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[l][n][j] = 0.0f;

        // slices of one half-chunk's test side into A fragments, then the 30 MMAs
        auto step = [&](const Half& H) {
            const int t = H.t < 0 ? 0 : H.t, q = H.t < 0 ? 0 : H.q;   // zero operands beyond the last quarter
            const float2 mu0 = M[t][q], mu1 = M[t][q + 1];
            uint32_t A[TC_NS][2];
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const float sg = sSg[wib][t][rr][lane];
                float ks[2][TC_NS];
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const float2 v = H.v[rr * 2 + pp];
                    const float2 mu = pp ? mu1 : mu0;
                    const float ph = v.x * mu.x;
                    const float pl = fmaf(v.x, mu.x, -ph) + fmaf(v.x, mu.y, v.y * mu.x);
                    slice5(ph * sg, pl * sg, ks[pp]);
                }
#pragma unroll
                for (int s = 0; s < TC_NS; ++s) A[s][rr] = pack_int_bf16x2(ks[0][s], ks[1][s]);
            }
#pragma unroll
            for (int n = 0; n < 2; ++n)
#pragma unroll
                for (int ka = 0; ka < TC_NS; ++ka)
#pragma unroll
                    for (int lb = 0; lb < TC_NS - ka; ++lb)
                        mma_k8(acc[ka + lb][n], A[ka][0], A[ka][1], n ? H.b[lb].y : H.b[lb].x);
        };
        // write the level sums of this segment to the slots (adding to the earlier
        // segments' values, which only this lane writes) and clear them
        auto flush = [&](bool first) {
            asm volatile("cp.async.wait_all;\n" ::: "memory");
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const int sl = sSlot[wib][x][lane];
                const int n = (x >> 1) & 1, j = (x >> 2) * 2 + (x & 1);
                const float sc = esc[x >> 2];
                // D0 and 2^-8 D1 are exact floats (integers below 2^24); their TwoSum plus
                // the lower levels (rounded at 2^-24 of a 2^-16 part) keep the pair to
                // ~2^-40 of the tile scale
                float rest = acc[TC_NS - 1][n][j];
#pragma unroll
                for (int l = TC_NS - 2; l >= 2; --l) rest = rest * 0x1p-8f + acc[l][n][j];
                float hs, he;
                tc_two_sum(acc[0][n][j], acc[1][n][j] * 0x1p-8f, hs, he);
                const float hi = hs * sc;
                const float lo = (he + rest * 0x1p-16f) * sc;
                if (sl >= 0) {
                    if (!first) {
                        const float2 o = src.kscr[sl];
                        float s2, e2;
                        tc_two_sum(o.x, hi, s2, e2);
                        src.kscr[sl] = make_float2(s2, o.y + lo + e2);
                    } else {
                        src.kscr[sl] = make_float2(hi, lo);
                    }
                }
            }
#pragma unroll
            for (int l = 0; l < TC_NS; ++l)
#pragma unroll
                for (int n = 0; n < 2; ++n)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[l][n][j] = 0.0f;
        };

        // walk the half-chunks two at a time, the next one's operands in flight
        const int nhalf = (nq + 1) >> 1;
        int seg = 0;
        bool first = true;
        Half h1;
        for (int h = 0; h < nhalf; h += 2) {
            advance();
            if (h + 1 < nhalf) load_half(h1, tv, sT, tq < nt ? tq : -1, qq, P, t4, bsl);
            step(h0);
            advance();
            if (h + 2 < nhalf) load_half(h0, tv, sT, tq < nt ? tq : -1, qq, P, t4, bsl);
            if (h + 1 < nhalf) step(h1);
            seg += 2;
            if (seg == TC_SEGH && h + 2 < nhalf) {
                flush(first);
                first = false;
                seg = 0;
            }
        }
        flush(first);
        __syncwarp();   // the per-warp shared arrays are rewritten by the next tile
    }
}

cudaError_t launch_elem_tc(const TcItems& it, const TcSrc& src, const Terms& tm, int gauss, const double* coef,
                           float* vals, cudaStream_t st, cudaEvent_t* evs) {
    if (evs) cudaEventRecord(evs[0], st);
    cudaError_t e = cudaSuccess;
    if (src.nnz > 0 && it.n > 0) {
        const int ntk = tm.nt <= 4 ? tm.nt : 8;
        const TermsF tf = make_terms_f(tm, ntk);
        // persistent grid: the resident blocks
        const unsigned eb = (unsigned)std::min<int64_t>((it.n + TC_NWARP - 1) / TC_NWARP,
                                                        (int64_t)std::max(it.n_sm, 1) * TC_BLOCKS_PER_SM);
#define WQ_TC_CASE(N)                                                                                    \
    do {                                                                                                 \
        if (gauss)                                                                                       \
            k_elem_tc<N, true><<<eb, TC_NWARP * 32, 0, st>>>(it, src, coef, tf);                         \
        else                                                                                             \
            k_elem_tc<N, false><<<eb, TC_NWARP * 32, 0, st>>>(it, src, coef, tf);                        \
    } while (0)
        switch (ntk) {
            case 1: WQ_TC_CASE(1); break;
            case 2: WQ_TC_CASE(2); break;
            case 3: WQ_TC_CASE(3); break;
            case 4: WQ_TC_CASE(4); break;
            default: WQ_TC_CASE(8); break;
        }
#undef WQ_TC_CASE
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (evs) cudaEventRecord(evs[1], st);
        ElemSrc gs{};
        gs.ep = ElemPlan{src.scat, src.gptr, src.kscr};
        gs.nnz = src.nnz;
        e = launch_gather_f32(gs, vals, true, st);
    } else if (evs) {
        cudaEventRecord(evs[1], st);
    }
    if (evs) cudaEventRecord(evs[2], st);
    return e;
}

// ------------------------------------------------------------------ set-up
// One block per element: exponents f_c of the table components, the trial-side
// slices in fragment order, and the test-side bounds (weights for WQ, table for Gauss).
__global__ void __launch_bounds__(128) k_tc_prep(int nc, int nwc, const int32_t* __restrict__ m_arr,
                                                 const double* __restrict__ table, const double* __restrict__ We,
                                                 TcPrep pr) {
    __shared__ double smax[4][8];
    __shared__ int sf[8];
    const int64_t e = blockIdx.x;
    const int4 el = pr.el[e];
    const int m = m_arr[e], P = el.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double* tb = table + el.x;
    double mx[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) mx[c] = 0.0;
    for (int x = threadIdx.x; x < P * m; x += blockDim.x) {
        const int q = x / m, b = x - q * m;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < nc) mx[c] = fmax(mx[c], fabs(tb[((int64_t)q * nc + c) * m + b]));
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        double v = mx[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) smax[w][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        const int c = threadIdx.x;
        const double v = fmax(fmax(smax[0][c], smax[1][c]), fmax(smax[2][c], smax[3][c]));
        int f = 0;
        if (v > 0.0) frexp(v, &f);   // 2^f > v
        sf[c] = f;
        pr.fexp[e * nc + c] = f;
    }
    __syncthreads();
    // trial-side slices, per (component, column block, quarter-chunk, point pair p, column g)
    const int ncb = (m + 15) >> 4, qpt = (P + 3) >> 2;
    const int nitem = nc * ncb * qpt * 16;
    uint32_t* out = pr.bs + pr.bs_ptr[e];
    for (int x = threadIdx.x; x < nitem; x += blockDim.x) {
        const int pg = x & 15, p = pg >> 3, g = pg & 7;
        int r = x >> 4;
        const int qq = r % qpt;
        r /= qpt;
        const int cb = r % ncb, c = r / ncb;
        float kk[2][2][TC_NS];   // [n-tile][point][slice]
#pragma unroll
        for (int n = 0; n < 2; ++n) {
            const int b = cb * 16 + n * 8 + g;
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const int q = qq * 4 + 2 * p + pp;
                double y = (q < P && b < m) ? ldexp(tb[((int64_t)q * nc + c) * m + b], 8 - sf[c]) : 0.0;
#pragma unroll
                for (int l = 0; l < TC_NS; ++l) {
                    const double v = rint(y);
                    kk[n][pp][l] = (float)v;
                    y = (y - v) * 256.0;
                }
            }
        }
        uint32_t* o = out + ((int64_t)(c * ncb + cb) * qpt + qq) * TC_QW + pg * 2;
#pragma unroll
        for (int l = 0; l < TC_NS; ++l)
            *reinterpret_cast<uint2*>(o + l * 32) =
                make_uint2(pack_bf16x2(kk[0][0][l], kk[0][1][l]), pack_bf16x2(kk[1][0][l], kk[1][1][l]));
    }
    // test-side bounds per (function, column)
    const int nv = We ? nwc : nc;
    for (int x = threadIdx.x; x < m * nv; x += blockDim.x) {
        const int a = x / nv, v = x - a * nv;
        double mv = 0.0;
        for (int q = 0; q < P; ++q)
            mv = fmax(mv, fabs(We ? We[((int64_t)el.z + (int64_t)q * m + a) * nwc + v]
                                  : tb[((int64_t)q * nc + v) * m + a]));
        pr.vmax[((int64_t)el.w + a) * nv + v] = __double2float_ru(mv);
    }
}

cudaError_t launch_tc_prep(int64_t E, int nc, int nwc, const int32_t* m, const double* table, const double* We,
                           const TcPrep& pr, cudaStream_t st) {
    if (E == 0) return cudaSuccess;
    if (nc > 8) return cudaErrorInvalidValue;
    k_tc_prep<<<(unsigned)E, 128, 0, st>>>(nc, nwc, m, table, We, pr);
    return cudaGetLastError();
}

}  // namespace wqd
