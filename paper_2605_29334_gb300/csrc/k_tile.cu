// Element blocks staged by the bulk-copy (TMA) engine, then per-row sums.
//
// The operators of Eqs. 9, 11, 12 and S (and the exact heat tangent) are sums over
// the support elements of a row:
//     A_ij = sum_{e in supp N_i cap supp N_j} K_e[a(i)][b(j)],
//     K_e[a][b] = sum_{q, t} s^t_{aq} T^t_{qb},   s^t_{aq} = S^{c_t}_{aq} mult_t(x_q),
// with S the test side (WQ: the weights w^{c}_{iq} of the row's function at the
// element's points, Sec. 4.3; Gauss: w_g |J_g| D_c N_a(x_g)), T the trial side (the
// basis table D_c N_b(x_q), Sec. 4.1) and mult_t a coefficient row at the points or a
// constant.  Two kernels:
//
//  * k_tile_f32: persistent warps, one 16 x 16 tile of K_e at a time, K walked in
//    chunks of at most QC points.  Every element's test and trial data sit in
//    element-major packs built at rule set-up ([component][point][16-row block][16],
//    zero-padded beyond m_e), so the data of one tile and chunk are one contiguous
//    block per component (m_e <= 16) or one 128-byte row per (component, point).  Each
//    warp has three stages: one lane issues cp.async.bulk copies two chunks ahead of the
//    one the warp computes, and an mbarrier with the expected byte count signals each
//    stage's arrival.  The arithmetic per tile is the compensated FP32 scheme of
//    k_elem_f32 (split (hi, lo) products, extraction against a power-of-two constant,
//    6 FP32 instructions per product), in the same order, so the element blocks are
//    bitwise those of the slot-map kernel.  Row a of the block goes straight to the
//    slot block of (row of function a, this element) in a row-major slot layout: one
//    128-byte store per tile row and column block, no slot map.
//  * k_rowsum_f32: one half-warp per CSR row; the row's slots are one contiguous range
//    (its support entries in support order), added 16 at a time with TwoSum into the
//    row's entries in shared memory (positions from a table of the same layout), then
//    the row is written once.  The sum order per entry is the support order, as in the
//    slot-map path.  Launched as a programmatic dependent of k_tile_f32.
#include <algorithm>

#include "kernels.h"

namespace wqd {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned tl_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tl_mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tl_smem(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void tl_fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void tl_fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tl_mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tl_smem(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool tl_mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tl_smem(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16),
// completion counted on the mbarrier in bytes
__device__ __forceinline__ void tl_bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     tl_smem(dst)),
                 "l"(src), "r"(bytes), "r"(tl_smem(bar))
                 : "memory");
}
__device__ __forceinline__ uint64_t tl_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

// Bounded wait of the whole warp for a stage: every lane polls the mbarrier (each
// lane's own completed wait makes the bulk-copied data visible to it), sleeping
// 16..64 ns between polls, for at most ~200 ms; false for all lanes if any lane ran out
// of time (the status word then gets ST_TIMEOUT and the caller leaves the kernel).
__device__ __forceinline__ bool tl_wait(uint64_t* b, unsigned parity, unsigned* status) {
    bool ok = tl_mbar_try_wait(b, parity);
    if (!ok) {
        // back off between polls so that waiting warps leave the issue slots to the others
        const uint64_t t0 = tl_globaltimer();
        unsigned ns = 16;
        for (;;) {
            __nanosleep(ns);
            if (tl_mbar_try_wait(b, parity)) {
                ok = true;
                break;
            }
            if (ns < 64) ns <<= 1;
            if (tl_globaltimer() - t0 > 200000000ull) break;
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && status && (threadIdx.x & 31) == 0) atomicOr(status, (unsigned)ST_TIMEOUT);
    return ok;
}

__device__ __forceinline__ void tl_two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}
__device__ __forceinline__ void tl_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ float tl_warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Smallest power of two >= 4 x (a non-negative finite float x).
__device__ __forceinline__ float tl_pow2_above_4x(float x) {
    const unsigned bits = __float_as_uint(x * 4.0f);
    return __uint_as_float(((bits >> 23) + 1u) << 23);
}

// ------------------------------------------------------------------ phase 1
// Chunk length and warps per block: variant 0 stages chunks of up to 12 / 8 / 4 points
// (terms <= 2 / <= 4 / 8, the chunks of the slot-map kernel), variant 1 up to 16 points
// for <= 2 terms (one chunk per tile for 4 x 4 points).  Every warp has NSTAGE stages
// (variant 0: 2, so that more warps fit an SM; variant 1: 3) and keeps NSTAGE - 1 chunks
// in flight ahead of the one it computes.
template <int NT, int V>
struct TileCfg {
    static constexpr int QC0 = NT <= 2 ? 12 : (NT <= 4 ? 8 : 4);
    static constexpr int QC = (V == 1 && NT <= 2) ? 16 : QC0;         // most points per chunk
    static constexpr int CM = NT < 4 ? NT : 4;                      // staged components per side
    static constexpr int NSTAGE = V == 0 ? 2 : 3;
    static constexpr int STAGE = 2 * CM * QC * 16;                   // float2: test comps, trial comps
    static constexpr int PROD = NT * QC * 16;                        // float2: products s per term
    static constexpr int MULT = QC * NT;                             // float2: multipliers per (point, term)
    static constexpr int WARP_F2 = ((NSTAGE * STAGE + PROD + MULT + NSTAGE) + 15) / 16 * 16;   // + mbarriers
    static constexpr int SMEM_BUDGET = 200 * 1024;
    static constexpr int WPB_RAW = SMEM_BUDGET / (WARP_F2 * 8);
    static constexpr int WPB = WPB_RAW > 16 ? 16 : WPB_RAW;         // warps per block (one block per SM)
    static constexpr int SMEM = WPB * WARP_F2 * 8;
};

// One chunk of one tile: the item's descriptor and the chunk's points.
struct TileJobItem {
    int4 d;          // test pack base, trial pack base, first point, first function (kdst)
    int m, P, a0, b0, ncb, rule, tmx;
    int c, nch, q0, nq;
    bool valid;
};

template <int NT, int V, bool COMP, bool BATCH, int NP>
__global__ void __launch_bounds__(TileCfg<NT, V>::WPB * 32, 1)
    k_tile_f32(TileJob job, const __grid_constant__ PtrTable<NP> pt, TileTerms tm) {
    using Cfg = TileCfg<NT, V>;
    constexpr int QC = Cfg::QC, CM = Cfg::CM, WPB = Cfg::WPB, NS = Cfg::NSTAGE;
    extern __shared__ __align__(128) float2 tl_dyn[];
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * WPB + wib, GW = (int64_t)gridDim.x * WPB;
    const int64_t n_mine = gw < job.n_items ? (job.n_items - 1 - gw) / GW + 1 : 0;
    if (n_mine == 0) return;
    float2* wsm = tl_dyn + (int64_t)wib * Cfg::WARP_F2;
    float2* const stg0 = wsm;
    float2* const prod = wsm + NS * Cfg::STAGE;
    float2* const mult = prod + Cfg::PROD;
    uint64_t* const bar = reinterpret_cast<uint64_t*>(mult + Cfg::MULT);
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) tl_mbar_init(bar + s, 1);
        tl_fence_mbar_init();
    }
    __syncwarp();
    const int bl = lane & 15, half = lane >> 4, rbase = 8 * half;

    // descriptors of 32 of this warp's items at a time: lane x holds item dbase + x
    int4 dsc = make_int4(0, 0, 0, 0);
    int4 mta = make_int4(0, 0, 0, 0);
    int64_t dbase = -64;
    auto fetch_item = [&](int64_t x, TileJobItem& J) {
        if (x < dbase || x >= dbase + 32) {   // warp-uniform
            dbase = x & ~(int64_t)31;
            const int64_t xx = dbase + lane;
            if (xx < n_mine) {
                const int64_t kk = gw + xx * GW;
                dsc = job.item[kk];
                mta = job.meta[kk];
            }
        }
        const int s = (int)(x - dbase);
        J.d = make_int4(__shfl_sync(0xffffffffu, dsc.x, s), __shfl_sync(0xffffffffu, dsc.y, s),
                        __shfl_sync(0xffffffffu, dsc.z, s), __shfl_sync(0xffffffffu, dsc.w, s));
        const int mt = __shfl_sync(0xffffffffu, mta.x, s);
        J.rule = __shfl_sync(0xffffffffu, mta.y, s);
        J.tmx = __shfl_sync(0xffffffffu, mta.z, s);
        J.m = mt & 255;
        J.P = (mt >> 8) & 255;
        J.a0 = ((mt >> 16) & 15) * 16;
        J.b0 = ((mt >> 20) & 15) * 16;
        J.ncb = (mt >> 24) & 15;
        J.nch = (J.P + QC - 1) / QC;
        J.c = 0;
        J.q0 = 0;
        J.nq = min((J.P + J.nch - 1) / J.nch, J.P);
        J.valid = true;
    };
    // the job after J: its next chunk, else the next item's first chunk
    auto advance = [&](TileJobItem& J, int64_t& x) {
        if (J.c + 1 < J.nch) {
            const int qc = (J.P + J.nch - 1) / J.nch;
            ++J.c;
            J.q0 = J.c * qc;
            J.nq = min(qc, J.P - J.q0);
        } else if (x + 1 < n_mine) {
            ++x;
            fetch_item(x, J);
        } else {
            J.valid = false;
        }
    };
    // bulk copies of job J's chunk into stage s: the staged components of each side at a
    // stride of nq points.  A tile of one chunk takes one copy per side (its components
    // are contiguous in the pack), a tile of several chunks one copy per component.
    auto issue = [&](const TileJobItem& J, int s) {
        const TileSrc& src = BATCH ? job.srcs[J.rule] : job.one;
        float2* stg = stg0 + s * Cfg::STAGE;
        const int ncomp = tm.s_n + tm.r_n;
        if (lane == 0) {
            tl_fence_proxy_async();
            tl_mbar_expect_tx(bar + s, (unsigned)(ncomp * J.nq * 128));
        }
        __syncwarp();
        const float2* gs = src.S0 + J.d.x + ((int64_t)((J.a0 >> 4) * src.n_test + tm.s_lo) * J.P + J.q0) * 16;
        const float2* gt = src.T0 + J.d.y + ((int64_t)((J.b0 >> 4) * src.n_trial + tm.r_lo) * J.P + J.q0) * 16;
        if (J.nch == 1) {
            if (lane == 0) tl_bulk_g2s(stg, gs, (unsigned)(tm.s_n * J.nq * 128), bar + s);
            if (lane == 1) tl_bulk_g2s(stg + CM * QC * 16, gt, (unsigned)(tm.r_n * J.nq * 128), bar + s);
        } else if (lane < ncomp) {
            const bool test = lane < tm.s_n;
            const int ci = test ? lane : lane - tm.s_n;
            const float2* g = (test ? gs : gt) + (int64_t)ci * J.P * 16;
            float2* d = stg + (test ? 0 : CM * QC * 16) + ci * J.nq * 16;
            tl_bulk_g2s(d, g, (unsigned)(J.nq * 128), bar + s);
        }
    };
    // coefficient rows of job J at its chunk's points (lane q < nq holds point q), and
    // the bound on |T_hi| over the terms' trial components (max of the set-up table)
    auto load_coef = [&](const TileJobItem& J, double (&cv)[4], float& tb) {
        const TileSrc& src = BATCH ? job.srcs[J.rule] : job.one;
        const double* cf = pt.coef[BATCH ? J.rule : 0];
#pragma unroll
        for (int cr = 0; cr < 4; ++cr) {
            cv[cr] = 0.0;
            if (cf && cr < tm.ncrow && lane < J.nq) cv[cr] = __ldg(cf + cr * tm.cstride + J.d.z + J.q0 + lane);
        }
        tb = 0.0f;
        if (COMP) {
            const float* tx = src.tmx + J.tmx + (J.b0 >> 4) * src.n_trial + tm.r_lo;
#pragma unroll
            for (int t = 0; t < NT; ++t)
                if (t < tm.nt) tb = fmaxf(tb, __ldg(tx + tm.rcomp[t]));
        }
    };

    TileJobItem jc, j1, j2;
    int64_t xc = 0, x1, x2;
    fetch_item(0, jc);
    j1 = jc;
    x1 = xc;
    advance(j1, x1);
    j2 = j1;
    x2 = x1;
    if (j1.valid) advance(j2, x2);
    issue(jc, 0);
    if (NS == 3 && j1.valid) issue(j1, 1);
    double cc[4];
    float tmx_c;
    load_coef(jc, cc, tmx_c);
    unsigned phase = 0u;               // bit s: parity of stage s's next completion
    int s = 0;                         // stage of jc
    float acc[8], lo[8];
    float cst = 0.0f;
    int kd_l = 0;                      // lanes 0..15: slot block of tile row a0 + lane
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = lo[r] = 0.0f;
    for (;;) {
        // NS - 1 jobs ahead are in flight: issue the last of them, fetch the next one's
        // coefficients
        if (NS == 3 && j2.valid) issue(j2, s >= NS - 2 ? s + 2 - NS : s + 2);
        if (NS == 2 && j1.valid) issue(j1, s ^ 1);
        double cn[4] = {0.0, 0.0, 0.0, 0.0};
        float tmx_n = 0.0f;
        if (j1.valid) load_coef(j1, cn, tmx_n);
        const TileSrc& src = BATCH ? job.srcs[jc.rule] : job.one;
        const int m = jc.m, a0 = jc.a0, b0 = jc.b0, nq = jc.nq;
        if (jc.c == 0) kd_l = bl + a0 < m && lane < 16 ? __ldg(src.kdst + jc.d.w + a0 + bl) : 0;
        if (!tl_wait(bar + s, (phase >> s) & 1u, job.status)) {
            // copies did not arrive: leave after a bounded wait for those still in flight
            const int s1 = s + 1 == NS ? 0 : s + 1, s2 = s1 + 1 == NS ? 0 : s1 + 1;
            if (j1.valid) tl_wait(bar + s1, (phase >> s1) & 1u, nullptr);
            if (NS == 3 && j2.valid) tl_wait(bar + s2, (phase >> s2) & 1u, nullptr);
            return;
        }
        phase ^= 1u << s;
        // ---- compute chunk jc.c of tile jc from stage s
        const float2* Sst = stg0 + s * Cfg::STAGE;
        const float2* Tst = Sst + CM * QC * 16;
        const int b = b0 + bl;
        const bool bok = b < m, aok = a0 + bl < m;
        const int nj = (nq + 1 - half) >> 1;       // this half-warp's points in the chunk
        if (lane < nq) {
            const bool has_coef = pt.coef[BATCH ? jc.rule : 0] != nullptr;
            if (tm.ncrow <= 1) {
                const float2 cs = has_coef ? split_double(cc[0]) : make_float2(1.0f, 0.0f);
#pragma unroll
                for (int t = 0; t < NT; ++t)
                    mult[lane * NT + t] = tm.crow[t] >= 0 ? cs : make_float2(tm.shi[t], tm.slo[t]);
            } else {
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const int cr = tm.crow[t];
                    double cv = cc[0];
                    if (cr == 1) cv = cc[1];
                    if (cr == 2) cv = cc[2];
                    if (cr == 3) cv = cc[3];
                    mult[lane * NT + t] = cr < 0 ? make_float2(tm.shi[t], tm.slo[t])
                                                 : (has_coef ? split_double(cv) : make_float2(1.0f, 0.0f));
                }
            }
        }
        __syncwarp();
        // products s (rows beyond m zeroed), with the largest |s_hi| of the chunk and a bound
        // on |T_hi| over the element's points and the tile's columns (set-up table) for the
        // accumulation bound
        float smax = 0.0f, tmax = 0.0f;
#pragma unroll
        for (int jj = 0; jj < (QC + 1) / 2; ++jj) {
            const int qq = half + 2 * jj;
            if (jj < nj) {
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    float2 v = make_float2(0.0f, 0.0f);
                    if (aok) {
                        const float2 w = Sst[(tm.tcomp[t] * nq + qq) * 16 + bl], c = mult[qq * NT + t];
                        float ph, pe;
                        tl_two_prod(w.x, c.x, ph, pe);
                        v = make_float2(ph, pe + fmaf(w.x, c.y, w.y * c.x));
                    }
                    prod[(t * QC + qq) * 16 + bl] = v;
                    if (COMP) smax = fmaxf(smax, fabsf(v.x));
                }
            }
        }
        if (COMP) tmax = tmx_c;
        if (COMP) {
            smax = tl_warp_max(smax);
            if (jc.c == 0) {
                cst = tl_pow2_above_4x((float)(nq * NT) * smax * tmax * 1.0001f);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    acc[r] = cst;
                    lo[r] = 0.0f;
                }
            } else {
                float vmax = 0.0f;
#pragma unroll
                for (int r = 0; r < 8; ++r) vmax = fmaxf(vmax, fabsf(acc[r] - cst));
                vmax = tl_warp_max(vmax);
                const float cnw = tl_pow2_above_4x(vmax + (float)(nq * NT) * smax * tmax * 1.0001f);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    float s2, e2;
                    tl_two_sum(cnw, acc[r] - cst, s2, e2);
                    acc[r] = s2;
                    lo[r] += e2;
                }
                cst = cnw;
            }
        } else if (jc.c == 0) {
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r] = lo[r] = 0.0f;
        }
        __syncwarp();
        if (bok) {
#pragma unroll 2
            for (int qq = 0; qq < nq; ++qq) {
                float2 T[NT];
                const float4* srow[NT];
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    T[t] = Tst[(tm.rcomp[t] * nq + qq) * 16 + bl];
                    srow[t] = reinterpret_cast<const float4*>(prod + (t * QC + qq) * 16 + rbase);
                }
#pragma unroll
                for (int t = 0; t < NT; ++t) {
#pragma unroll
                    for (int r2 = 0; r2 < 4; ++r2) {
                        const float4 sv = srow[t][r2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float sx = h ? sv.z : sv.x, sy = h ? sv.w : sv.y;
                            const int r = 2 * r2 + h;
                            if (COMP) {
                                const float an = fmaf(sx, T[t].x, acc[r]);
                                const float e = fmaf(sx, T[t].x, acc[r] - an);
                                acc[r] = an;
                                lo[r] += e;
                            } else {
                                acc[r] = fmaf(sx, T[t].x, acc[r]);
                            }
                            lo[r] = fmaf(sx, T[t].y, lo[r]);
                            lo[r] = fmaf(sy, T[t].x, lo[r]);
                        }
                    }
                }
            }
        }
        if (jc.c + 1 == jc.nch) {
            // tile row a goes to its CSR row's slot block, column block b0 / 16; every lane
            // writes (zeros beyond m), so each row is one 128-byte store
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int kd = __shfl_sync(0xffffffffu, kd_l, rbase + r);
                if (a0 + rbase + r < m)
                    src.kslot[(int64_t)kd + b0 + bl] = make_float2(COMP ? acc[r] - cst : acc[r], lo[r]);
            }
        }
        __syncwarp();   // this stage is read completely before a later issue reuses it
        if (!j1.valid) break;
        jc = j1;
        xc = x1;
        j1 = j2;
        x1 = x2;
        if (j2.valid) advance(j2, x2);
#pragma unroll
        for (int cr = 0; cr < 4; ++cr) cc[cr] = cn[cr];
        tmx_c = tmx_n;
        s = s + 1 == NS ? 0 : s + 1;
    }
    (void)xc;
}

// ------------------------------------------------------------------ phase 2
// One TwoSum (or plain) update of a row entry in shared memory.
template <bool COMP>
__device__ __forceinline__ void rs_add(float2* acc, int p, float2 v) {
    float2 a = acc[p];
    if (COMP) {
        float s3, e3;
        tl_two_sum(a.x, v.x, s3, e3);
        a = make_float2(s3, a.y + (v.y + e3));
    } else {
        a = make_float2(a.x + v.x, a.y + v.y);
    }
    acc[p] = a;
}

// Row i's slots are one contiguous range [rowslot[i], rowslot[i+1]): its support
// entries in support order, each a block of 16-slot column blocks holding the element
// block row of the row's function (written by the element kernel), with the entries'
// positions in the row at the same indices of pos (0xFFFF: padding).  Within one 16-slot
// block the positions are distinct, so a half-warp adds a block at a time.
template <bool COMP, bool BATCH, int NP>
__global__ void __launch_bounds__(256) k_rowsum_f32(RowSrc one, RowBatch rb, const __grid_constant__ PtrTable<NP> pt) {
    extern __shared__ __align__(16) float2 rs_acc[];
    const int lane = threadIdx.x & 31, hw = threadIdx.x >> 4, bl = threadIdx.x & 15;
    const unsigned hmask = 0xFFFFu << (lane & 16);
    const int ri = BATCH ? rb.blk_rule[blockIdx.x] : 0;
    const RowSrc& src = BATCH ? rb.src[ri] : one;
    const int64_t i = (BATCH ? rb.blk_row[blockIdx.x] : (int64_t)blockIdx.x * 16) + hw;
    float* __restrict__ vals = pt.vals[BATCH ? ri : 0];
    float2* acc = rs_acc + (int64_t)hw * (BATCH ? rb.max_n_i : src.max_n_i);
    // the row plan does not depend on the element kernel: read it before waiting for it
    int r0 = 0, ni = 0, x0 = 0, x1 = 0;
    const bool live = i < src.n;
    if (live) {
        r0 = src.row_ptr[i];
        ni = src.row_ptr[i + 1] - r0;
        x0 = src.rowslot[i];
        x1 = src.rowslot[i + 1];
    }
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (!live) return;
    for (int x = bl; x < ni; x += 16) acc[x] = make_float2(0.0f, 0.0f);
    __syncwarp(hmask);
    // all of the row's slot blocks (up to 16 at a time) are loaded before the dependent
    // shared-memory updates, so that a row waits for one memory latency, not one per block
    for (int x = x0; x < x1; x += 256) {
        float2 v[16];
        int p[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int xx = x + 16 * u + bl;
            v[u] = make_float2(0.0f, 0.0f);
            p[u] = 0xFFFF;
            if (xx < x1) {
                v[u] = src.kslot[xx];
                p[u] = src.pos[xx];
            }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (x + 16 * u >= x1) break;   // uniform over the half-warp
            if (p[u] != 0xFFFF) rs_add<COMP>(acc, p[u], v[u]);
            __syncwarp(hmask);
        }
    }
    for (int x = bl; x < ni; x += 16) {
        const float2 a = acc[x];
        vals[r0 + x] = a.x + a.y;
    }
}

// ------------------------------------------------------------------ launchers
template <int NT, int V, bool COMP, bool BATCH, int NP>
static cudaError_t launch_tile_nt(const TileJob& job, const PtrTable<NP>& pt, const TileTerms& tm, int n_sm,
                                  cudaStream_t st) {
    using Cfg = TileCfg<NT, V>;
    int blocks = (int)std::min<int64_t>((job.n_items + Cfg::WPB - 1) / Cfg::WPB, (int64_t)std::max(n_sm, 1));
    if (blocks < 1) blocks = 1;
    k_tile_f32<NT, V, COMP, BATCH, NP><<<blocks, Cfg::WPB * 32, Cfg::SMEM, st>>>(job, pt, tm);
    return cudaGetLastError();
}

template <int NT, int V>
static cudaError_t prepare_nt() {
    const int smem = TileCfg<NT, V>::SMEM;
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    };
    set(k_tile_f32<NT, V, true, false, 1>);
    set(k_tile_f32<NT, V, false, false, 1>);
    set(k_tile_f32<NT, V, true, true, WQ_BATCH_MAX>);
    set(k_tile_f32<NT, V, false, true, WQ_BATCH_MAX>);
    return e;
}

// Shared-memory size of every tile-kernel instance on the current device (once per
// device, before any launch or stream capture).
cudaError_t prepare_tile_kernels() {
    cudaError_t e = prepare_nt<1, 0>();
    if (e == cudaSuccess) e = prepare_nt<2, 0>();
    if (e == cudaSuccess) e = prepare_nt<3, 0>();
    if (e == cudaSuccess) e = prepare_nt<4, 0>();
    if (e == cudaSuccess) e = prepare_nt<8, 0>();
    if (e == cudaSuccess) e = prepare_nt<1, 1>();
    if (e == cudaSuccess) e = prepare_nt<2, 1>();
    if (e == cudaSuccess) e = prepare_nt<3, 1>();
    if (e == cudaSuccess) e = prepare_nt<4, 1>();
    if (e == cudaSuccess) e = prepare_nt<8, 1>();
    return e;
}

template <bool BATCH, int NP>
static cudaError_t launch_tile_pair(const TileJob& job, const RowSrc& rs, const RowBatch& rb, const PtrTable<NP>& pt,
                                    const TileTerms& tm, bool comp, int variant, int n_sm, int64_t n_rowblocks,
                                    int max_n_i, cudaStream_t st, cudaEvent_t* evs) {
    cudaError_t e = cudaSuccess;
    if (job.n_items > 0) {
        const int ntk = tm.nt <= 4 ? tm.nt : 8;
#define WQ_TL_CASE(N)                                                                                        \
    e = variant == 1 ? (comp ? launch_tile_nt<N, 1, true, BATCH, NP>(job, pt, tm, n_sm, st)                  \
                             : launch_tile_nt<N, 1, false, BATCH, NP>(job, pt, tm, n_sm, st))                \
                     : (comp ? launch_tile_nt<N, 0, true, BATCH, NP>(job, pt, tm, n_sm, st)                  \
                             : launch_tile_nt<N, 0, false, BATCH, NP>(job, pt, tm, n_sm, st))
        switch (ntk) {
            case 1: WQ_TL_CASE(1); break;
            case 2: WQ_TL_CASE(2); break;
            case 3: WQ_TL_CASE(3); break;
            case 4: WQ_TL_CASE(4); break;
            default: WQ_TL_CASE(8); break;
        }
#undef WQ_TL_CASE
        if (e != cudaSuccess) return e;
    }
    if (evs) cudaEventRecord(evs[1], st);
    if (n_rowblocks == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)n_rowblocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = (size_t)16 * max_n_i * sizeof(float2);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cfg.dynamicSmemBytes > 48 * 1024) return cudaErrorInvalidValue;   // rows longer than 384 entries
    if (comp)
        e = cudaLaunchKernelEx(&cfg, k_rowsum_f32<true, BATCH, NP>, rs, rb, pt);
    else
        e = cudaLaunchKernelEx(&cfg, k_rowsum_f32<false, BATCH, NP>, rs, rb, pt);
    return e;
}

cudaError_t launch_tile_f32(const TileJob& job, const RowSrc& rs, const TileTerms& tm, const double* coef,
                            float* vals, bool compensated, int variant, int n_sm, cudaStream_t st, cudaEvent_t* evs) {
    if (evs) cudaEventRecord(evs[0], st);
    PtrTable<1> pt;
    pt.coef[0] = coef;
    pt.vals[0] = vals;
    cudaError_t e = launch_tile_pair<false, 1>(job, rs, RowBatch{}, pt, tm, compensated, variant, n_sm,
                                               (rs.n + 15) / 16, rs.max_n_i, st, evs);
    if (evs) cudaEventRecord(evs[2], st);
    return e;
}

cudaError_t launch_tile_batch(const TileJob& job, const RowBatch& rb, const double* const* coefs, float* const* vals,
                              int k, const TileTerms& tm, bool compensated, int variant, int n_sm, cudaStream_t st) {
    if (k < 1 || k > WQ_BATCH_MAX) return cudaErrorInvalidValue;
    PtrTable<WQ_BATCH_MAX> pt{};
    for (int r = 0; r < k; ++r) {
        pt.coef[r] = coefs[r];
        pt.vals[r] = vals[r];
    }
    return launch_tile_pair<true, WQ_BATCH_MAX>(job, RowSrc{}, rb, pt, tm, compensated, variant, n_sm, rb.n_blocks,
                                                rb.max_n_i, st, nullptr);
}

// ------------------------------------------------------------------ packs (rule set-up)
// Element-major packs: out[off_e + ((cb ncomp + c) P_e + q) 16 + r] = value of element e,
// component c, point q, local function cb 16 + r (0 beyond m_e): the data of one
// 16-function block of the element are contiguous, components after one another.  Sources:
//   PK_TABLE2  split table [src_e + (q nc + c) m_e + j] (float2)
//   PK_W2E     element-major split weights [(src_e + q m_e + j) nwc + c] (float2)
//   PK_GAUSS   FP64 Gauss table times the Gauss weight, split: gt[src_e + (q nc + c) m_e + j] gw[pt_e + q]
__global__ void k_pack(PackJob pj) {
    const int64_t e = blockIdx.x;
    if (e >= pj.E) return;
    const int m = pj.m[e], P = pj.P[e], ncb = (m + 15) / 16;
    const int64_t src = pj.src_off[e], off = pj.out_off[e], p0 = pj.pt0 ? pj.pt0[e] : 0;
    const int64_t total = (int64_t)pj.ncomp * P * ncb * 16;
    for (int64_t x = threadIdx.x; x < total; x += blockDim.x) {
        const int r = (int)(x & 15);
        int64_t y = x >> 4;
        const int q = (int)(y % P);
        y /= P;
        const int c = (int)(y % pj.ncomp);
        const int cb = (int)(y / pj.ncomp);
        const int j = cb * 16 + r;
        float2 v = make_float2(0.0f, 0.0f);
        if (j < m) {
            if (pj.kind == PK_TABLE2) {
                v = pj.f2[src + ((int64_t)q * pj.nc + c) * m + j];
            } else if (pj.kind == PK_W2E) {
                v = pj.f2[(src + (int64_t)q * m + j) * pj.nwc + c];
            } else {
                const double d = pj.f64[src + ((int64_t)q * pj.nc + c) * m + j] * pj.gw[p0 + q];
                const float h = __double2float_rn(d);
                v = make_float2(h, __double2float_rn(d - (double)h));
            }
        }
        pj.out[off + x] = v;
    }
}

// Bound table of a trial pack: tmx[tmx_off_e + cb ncomp + c] = max |hi| over the points and
// the 16 functions of block cb, component c of element e.
__global__ void k_pack_max(PackJob pj, const int64_t* __restrict__ tmx_off, float* __restrict__ tmx) {
    const int64_t e = blockIdx.x;
    if (e >= pj.E) return;
    const int m = pj.m[e], P = pj.P[e], ncb = (m + 15) / 16;
    const float2* blk = pj.out + pj.out_off[e];
    for (int x = threadIdx.x; x < ncb * pj.ncomp; x += blockDim.x) {
        float v = 0.0f;
        for (int y = 0; y < P * 16; ++y) v = fmaxf(v, fabsf(blk[(int64_t)x * P * 16 + y].x));
        tmx[tmx_off[e] + x] = v;
    }
}

cudaError_t launch_pack_max(const PackJob& pj, const int64_t* tmx_off, float* tmx, cudaStream_t st) {
    if (pj.E == 0) return cudaSuccess;
    k_pack_max<<<(unsigned)pj.E, 32, 0, st>>>(pj, tmx_off, tmx);
    return cudaGetLastError();
}

cudaError_t launch_pack(const PackJob& pj, cudaStream_t st) {
    if (pj.E == 0) return cudaSuccess;
    k_pack<<<(unsigned)pj.E, 128, 0, st>>>(pj);
    return cudaGetLastError();
}

}  // namespace wqd
