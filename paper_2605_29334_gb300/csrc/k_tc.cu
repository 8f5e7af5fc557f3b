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
//  * the trial side of element e, component c, is scaled by 2^(8 - f), 2^f >= max|T|
//    over the element, and rounded into 4 slices of 8 bits, T 2^(8-f) =
//    sum_l b_l 2^(-8 l) with integers |b_0| <= 256, |b_l| <= 128 (exact bf16), to
//    2^-25 of 256 (set-up, from the FP64 table);
//  * the test side of row a is scaled by 2^(f_t + 8 - E_a), 2^E_a >= max_{t,q} |s^t_aq|
//    2^(f_t) (the bound from per-function maxima of the weights and the largest
//    coefficient of the element), and sliced the same way at run time from the split
//    (hi, lo) products;
//  * every product a_k b_l of bf16 integers is exact, and a level sum
//    D_d = sum_{k + l = d} sum_K a_k b_l has |D_d| < 2^24 for K <= 160, so the FP32
//    accumulation of the MMA is exact (integers below 2^24);
//  * K_e[a][b] = 2^(E_a - 16) sum_{d <= 3} 2^(-8 d) D_d, the pairs with k + l > 3
//    dropped (below 2^-32 of the tile's product scale).
// On the 10,240-element Poisson workload this gives ~1e-8 normwise against FP64 (the
// level-3 cut and the final FP32 rounding), the compensated SIMT path's accuracy at a
// fraction of its instructions: the SIMT work is per (row, point, term) -- split
// product and 4 slices, ~25 instructions -- instead of per (row, column, point, term).
//
// One warp per 16 x 16 tile (the FP32 path's tiles and slot map).  The K range is
// walked in half-chunks of 8 points of one term (each term's points padded to a
// multiple of 8).  Lane (g, t4) = (lane / 4, lane % 4) builds the m16n8k8 A fragments
// of its rows g, g + 8 at the points 2 t4, 2 t4 + 1, loads the trial fragments
// precomputed in that order (two 16-byte loads), and runs 10 slice pairs x 2 n-tiles
// of mma.sync into 4 level accumulators; the next half-chunk's loads are in flight
// meanwhile.  Slicing uses FMA-pipe rounding (add and subtract 1.5 2^23) and a byte
// permute for the bf16 packing.  Every 20 half-chunks (K = 160) the levels are added
// to the tile's slots (a TwoSum against the earlier segments), so any K is exact.
#include <algorithm>

#include <cuda_bf16.h>

#include "kernels.h"

namespace wqd {

constexpr int TC_NWARP = 4;     // warps per block
constexpr int TC_PMAX = 64;     // points per element (WQ side^2, Gauss 16 nsub)
constexpr int TC_SEG = 10;      // chunks per exact segment: K <= 160
constexpr int TC_BLOCKS_PER_SM = 5;

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

// Four 8-bit slices of y = yh + yl (|y| <= 256, |yl| <= ulp(yh) / 2): integers k_s with
// y = k0 + 2^-8 k1 + 2^-16 k2 + 2^-24 k3 to 2^-25.  Rounding to an integer adds and
// subtracts 1.5 2^23 (FMA pipe; rintf runs on the slower conversion pipe).  Every
// remainder yh - k0, r 2^8 - k1, t - k2 is exact; yl enters at the third slice
// (|k2| <= 129), so 14 FP32 instructions.
__device__ __forceinline__ void slice4(float yh, float yl, float (&k)[4]) {
    const float M = 12582912.0f;
    k[0] = __fsub_rn(__fadd_rn(yh, M), M);
    float r = yh - k[0];
    k[1] = __fsub_rn(__fmaf_rn(r, 256.0f, M), M);
    r = __fmaf_rn(r, 256.0f, -k[1]);
    const float t = __fmaf_rn(r, 256.0f, yl * 65536.0f);
    k[2] = __fsub_rn(__fadd_rn(t, M), M);
    r = t - k[2];
    k[3] = __fsub_rn(__fmaf_rn(r, 256.0f, M), M);
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

// Operands of one half-chunk (8 points of one term) for one n-tile: this lane's
// test-side values (rows g, g + 8 at points 2 t4, 2 t4 + 1), the term's multipliers at
// those points, and the trial-side fragment words (slices 0..3).
struct Half {
    float2 v[4];     // [row][point]
    float2 mu[2];    // [point]
    uint4 b;
};

// Per-tile constants of the loads.
struct TileV {
    const float2* base;  // test side of the element
    int r0, r1;          // offsets of rows g, g + 8 (-1: beyond m)
    int qs, cs;          // stride of a point, of a column / component
    int p0, P;           // first point, points
};

// Per-term constants (warp-uniform, in shared memory).
struct TermC {
    int vc;              // test-side column (weight column, or table component)
    int boff;            // trial slices of (component, column block), words
    int mrow;            // multiplier row in cp2 (-1: constant)
    float shi, slo;      // constant multiplier (split)
};

template <bool GAUSS>
__device__ __forceinline__ void load_half(Half& H, const TileV& tv, const TermC& tc, int hh, int n, int t4,
                                          const uint32_t* __restrict__ bsl, const float2* __restrict__ cp2,
                                          int64_t npts, const float2* __restrict__ gw2) {
    H.b = __ldg(reinterpret_cast<const uint4*>(bsl + tc.boff + hh * 256) + n);
    const int q = hh * 8 + 2 * t4;
    const float2* vb = tv.base + q * tv.qs + tc.vc * tv.cs;
    const bool q0 = q < tv.P, q1 = q + 1 < tv.P;
    const float2 z = make_float2(0.0f, 0.0f);
    H.v[0] = (tv.r0 >= 0 && q0) ? __ldg(vb + tv.r0) : z;
    H.v[1] = (tv.r0 >= 0 && q1) ? __ldg(vb + tv.qs + tv.r0) : z;
    H.v[2] = (tv.r1 >= 0 && q0) ? __ldg(vb + tv.r1) : z;
    H.v[3] = (tv.r1 >= 0 && q1) ? __ldg(vb + tv.qs + tv.r1) : z;
    if (tc.mrow >= 0) {
        const float2* mp = cp2 + tc.mrow * npts + tv.p0 + q;
        H.mu[0] = q0 ? __ldg(mp) : z;
        H.mu[1] = q1 ? __ldg(mp + 1) : z;
    } else if (GAUSS) {   // Gauss weight times the constant
        const float2 c = make_float2(tc.shi, tc.slo);
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
            const float2 g = (pp ? q1 : q0) ? __ldg(gw2 + tv.p0 + q + pp) : z;
            const float ph = g.x * c.x;
            H.mu[pp] = make_float2(ph, fmaf(g.x, c.x, -ph) + fmaf(g.x, c.y, g.y * c.x));
        }
    } else {
        H.mu[0] = H.mu[1] = make_float2(tc.shi, tc.slo);
    }
}

template <int NT, bool GAUSS>
__global__ void __launch_bounds__(TC_NWARP * 32, TC_BLOCKS_PER_SM)
    k_elem_tc(TcItems it, TcSrc src, TermsF tm) {
    __shared__ TermC sTerm[TC_NWARP][NT];
    __shared__ float sSg[TC_NWARP][NT][2][32];     // per (term, row, lane) slice scale
    __shared__ int sSlot[TC_NWARP][8][32];         // destination slots per (entry, lane)
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * TC_NWARP + wib;
    if (k >= it.n) return;
    const int4 d = it.item[k];
    const int4 d2 = it.it2[k];
    const int kb = it.kb[k];
    const int m = d.z & 255, P = (d.z >> 8) & 255, a0 = ((d.z >> 16) & 15) * 16, b0 = ((d.z >> 20) & 15) * 16;
    const int hpt = d2.w >> 3, ncb = (m + 15) >> 4;
    const int g = lane >> 2, t4 = lane & 3, ra = a0 + g;
    const int nt = tm.nt, nc = src.nc, nv = GAUSS ? src.nc : src.nwc;
    TermC* sT = sTerm[wib];
    if (lane < nt) {
#pragma unroll
        for (int t = 0; t < NT; ++t)
            if (t == lane) {
                TermC c;
                c.vc = GAUSS ? tm.sc[t] : tm.wc[t];
                c.boff = (tm.tc[t] * ncb + (b0 >> 4)) * hpt * 256;
                c.mrow = tm.crow[t];
                c.shi = tm.shi[t];
                c.slo = tm.slo[t];
                sT[t] = c;
            }
    }
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
    __syncwarp();
    TileV tv;
    tv.base = GAUSS ? src.vsrc + d.x : src.vsrc + (int64_t)d.w * nv;
    tv.r0 = ra < m ? (GAUSS ? ra : ra * nv) : -1;
    tv.r1 = ra + 8 < m ? (GAUSS ? ra + 8 : (ra + 8) * nv) : -1;
    tv.qs = GAUSS ? nc * m : m * nv;
    tv.cs = GAUSS ? m : 1;
    tv.p0 = d.y;
    tv.P = P;
    const uint32_t* __restrict__ bsl = src.bs + d2.y + lane * 8;
    // exponents and bounds (independent of the coefficients)
    float vm[2][NT], fsc[NT];
    int f8[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        f8[t] = t < nt ? __ldg(src.fexp + (int64_t)d2.z * nc + tm.tc[t]) + 8 : 0;
        const int vc = GAUSS ? tm.sc[t] : tm.wc[t];
        const float* vr = src.vmax + (int64_t)(d2.x + ra) * nv + vc;
        vm[0][t] = (t < nt && ra < m) ? __ldg(vr) : 0.0f;
        vm[1][t] = (t < nt && ra + 8 < m) ? __ldg(vr + 8 * nv) : 0.0f;
    }
    // the split coefficients and their per-element maxima come from the preceding kernel
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    const float* cm = src.cmx + (int64_t)d2.z * 5;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int c = tm.crow[t];
        const float sabs = fabsf(tm.shi[t]) * (1.0f + 0x1p-22f);
        fsc[t] = t >= nt ? 0.0f : (c >= 0 ? __ldg(cm + c) : (GAUSS ? __ldg(cm + 4) * sabs : sabs));
    }
    // row exponents 2^E > max_t vmax[row][v_t] cmax_t 2^f_t, the slice scales
    // 2^(f_t + 8 - E) per (term, row) and the entries' scales 2^(E - 16)
    float esc[2];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        float bound = 0.0f;
#pragma unroll
        for (int t = 0; t < NT; ++t)
            if (t < nt) bound = fmaxf(bound, vm[rr][t] * fsc[t] * exp2i(f8[t] - 8));
        const int E = bound > 0.0f ? exp_above(bound * (1.0f + 0x1p-20f)) : 0;
#pragma unroll
        for (int t = 0; t < NT; ++t) sSg[wib][t][rr][lane] = exp2i(f8[t] - E);
        esc[rr] = exp2i(E - 16);
    }

    // slices of one half-chunk's test side into A fragments, then 10 MMAs
    float acc[4][4];
    auto step = [&](const Half& H, int t) {
        uint32_t A[4][2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const float sg = sSg[wib][t][rr][lane];
            float ks[2][4];
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const float2 v = H.v[rr * 2 + pp];
                const float2 mu = H.mu[pp];
                const float ph = v.x * mu.x;
                const float pl = fmaf(v.x, mu.x, -ph) + fmaf(v.x, mu.y, v.y * mu.x);
                slice4(ph * sg, pl * sg, ks[pp]);
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) A[s][rr] = pack_int_bf16x2(ks[0][s], ks[1][s]);
        }
        const uint32_t bw[4] = {H.b.x, H.b.y, H.b.z, H.b.w};
#pragma unroll
        for (int ka = 0; ka < 4; ++ka)
#pragma unroll
            for (int lb = 0; lb < 4 - ka; ++lb) mma_k8(acc[ka + lb], A[ka][0], A[ka][1], bw[lb]);
    };
    // write the level sums of n-tile n to the slots (adding to the earlier segments'
    // values, which only this lane writes) and clear them
    auto flush = [&](int n, bool first) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int sl = sSlot[wib][(j >> 1) * 4 + n * 2 + (j & 1)][lane];
            const float sc = esc[j >> 1];
            const float hi = acc[0][j] * sc;
            const float lo = ((acc[3][j] * 0x1p-8f + acc[2][j]) * 0x1p-8f + acc[1][j]) * (0x1p-8f * sc);
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
    };

    // the two n-tiles one after the other (the second is empty for m <= b0 + 8); the
    // half-chunks two per trip, the next one's operands in flight
    const int nhalf = nt * hpt;
    for (int n = 0; n < 2; ++n) {
        if (b0 + 8 * n >= m) break;
#pragma unroll
        for (int l = 0; l < 4; ++l)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[l][j] = 0.0f;
        int t = 0, hh = 0, seg = 0;
        bool first = true;
        Half h0, h1;
        load_half<GAUSS>(h0, tv, sT[0], 0, n, t4, bsl, src.cp2, src.npts, src.gw2);
        for (int h = 0; h < nhalf; h += 2) {
            int t1 = t, hh1 = hh + 1;
            if (hh1 == hpt) hh1 = 0, ++t1;
            if (h + 1 < nhalf) load_half<GAUSS>(h1, tv, sT[t1], hh1, n, t4, bsl, src.cp2, src.npts, src.gw2);
            step(h0, t);
            int t2 = t1, hh2 = hh1 + 1;
            if (hh2 == hpt) hh2 = 0, ++t2;
            if (h + 2 < nhalf) load_half<GAUSS>(h0, tv, sT[t2], hh2, n, t4, bsl, src.cp2, src.npts, src.gw2);
            if (h + 1 < nhalf) step(h1, t1);
            t = t2, hh = hh2;
            seg += 2;
            if (seg == 2 * TC_SEG && h + 2 < nhalf) {
                flush(n, first);
#pragma unroll
                for (int l = 0; l < 4; ++l)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[l][j] = 0.0f;
                first = false;
                seg = 0;
            }
        }
        flush(n, first);
    }
}

// Split coefficients at the points (one warp per element): cp2[r][p] = (hi, lo) of
// coefficient row r (times the Gauss weight for Gauss points), cmx[e][r] = the
// element's largest |hi|; cmx[e][4] = the largest Gauss weight (Gauss points).
__global__ void __launch_bounds__(256) k_tc_coef(int64_t E, const int64_t* __restrict__ pptr,
                                                 const double* __restrict__ coef, int ncrow, int64_t cstride,
                                                 const float2* __restrict__ gw2, float2* __restrict__ cp2,
                                                 float* __restrict__ cmx, int64_t npts) {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (e >= E) return;
    const int64_t p0 = pptr[e];
    const int P = (int)(pptr[e + 1] - p0);
    for (int r = 0; r < ncrow; ++r) {
        float mx = 0.0f;
        for (int q = lane; q < P; q += 32) {
            const double v = coef ? coef[r * cstride + p0 + q] : 1.0;
            const float h = __double2float_rn(v);
            float2 c = make_float2(h, __double2float_rn(v - (double)h));
            if (gw2) {
                const float2 gq = gw2[p0 + q];
                const float ph = c.x * gq.x;
                c = make_float2(ph, fmaf(c.x, gq.x, -ph) + fmaf(c.x, gq.y, c.y * gq.x));
            }
            cp2[r * npts + p0 + q] = c;
            mx = fmaxf(mx, fabsf(c.x));
        }
        mx = tc_warp_max(mx);
        if (lane == 0) cmx[e * 5 + r] = mx * (1.0f + 0x1p-22f);
    }
    if (gw2) {
        float mx = 0.0f;
        for (int q = lane; q < P; q += 32) mx = fmaxf(mx, fabsf(gw2[p0 + q].x));
        mx = tc_warp_max(mx);
        if (lane == 0) cmx[e * 5 + 4] = mx * (1.0f + 0x1p-22f);
    }
}

cudaError_t launch_elem_tc(const TcItems& it, const TcSrc& src, const Terms& tm, int gauss, const double* coef,
                           float* vals, cudaStream_t st, cudaEvent_t* evs) {
    if (evs) cudaEventRecord(evs[0], st);
    cudaError_t e = cudaSuccess;
    if (src.nnz > 0 && it.n > 0) {
        const int ntk = tm.nt <= 4 ? tm.nt : 8;
        const TermsF tf = make_terms_f(tm, ntk);
        if (tf.ncrow > 4) return cudaErrorInvalidValue;
        k_tc_coef<<<(unsigned)((src.E + 7) / 8), 256, 0, st>>>(src.E, src.pptr, coef, tf.ncrow, tm.cstride,
                                                                gauss ? src.gw2 : nullptr, src.cp2, src.cmx,
                                                                src.npts);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)((it.n + TC_NWARP - 1) / TC_NWARP));
        cfg.blockDim = dim3(TC_NWARP * 32);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
#define WQ_TC_CASE(N)                                                                                    \
    do {                                                                                                 \
        if (gauss)                                                                                       \
            e = cudaLaunchKernelEx(&cfg, k_elem_tc<N, true>, it, src, tf);                               \
        else                                                                                             \
            e = cudaLaunchKernelEx(&cfg, k_elem_tc<N, false>, it, src, tf);                              \
    } while (0)
        switch (ntk) {
            case 1: WQ_TC_CASE(1); break;
            case 2: WQ_TC_CASE(2); break;
            case 3: WQ_TC_CASE(3); break;
            case 4: WQ_TC_CASE(4); break;
            default: WQ_TC_CASE(8); break;
        }
#undef WQ_TC_CASE
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
    // trial-side slices
    const int ncb = (m + 15) >> 4, hpt = (P + 7) >> 3;
    const int nitem = nc * ncb * hpt * 32;
    uint32_t* out = pr.bs + pr.bs_ptr[e];
    for (int x = threadIdx.x; x < nitem; x += blockDim.x) {
        const int ln = x & 31;
        int r = x >> 5;
        const int hh = r % hpt;
        r /= hpt;
        const int cb = r % ncb, c = r / ncb;
        const int g = ln >> 2, t4 = ln & 3;
        uint32_t wd[8];
#pragma unroll
        for (int n = 0; n < 2; ++n) {
            const int b = cb * 16 + n * 8 + g;
            float kk[2][4];
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const int q = hh * 8 + 2 * t4 + pp;
                double y = (q < P && b < m) ? ldexp(tb[((int64_t)q * nc + c) * m + b], 8 - sf[c]) : 0.0;
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const double v = rint(y);
                    kk[pp][l] = (float)v;
                    y = (y - v) * 256.0;
                }
            }
#pragma unroll
            for (int l = 0; l < 4; ++l) wd[n * 4 + l] = pack_bf16x2(kk[0][l], kk[1][l]);
        }
        uint4* o4 = reinterpret_cast<uint4*>(out + ((int64_t)(c * ncb + cb) * hpt + hh) * 256 + ln * 8);
        o4[0] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        o4[1] = make_uint4(wd[4], wd[5], wd[6], wd[7]);
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
