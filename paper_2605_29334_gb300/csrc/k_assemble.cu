// Assembly kernels.
//  * k_moments_f64 (rule build): the Gauss component matrices G^c (c = 1) that are
//    the moments b of the weight systems (Sec. 2, Sec. 4.3), row-wise: one warp per
//    test function i, the row's n_i values accumulated in shared memory and written
//    once; per support element the products w_g |J_g| D_c N_i(x_g) are formed once,
//    lane-parallel, and broadcast by shuffles; for m_e <= 16 the two half-warps take
//    alternate points.
//  * k_elem_f32 / k_gather_f32 and k_elem_f64 / k_gather_f64: WQ and Gauss operators
//    (Eqs. 9, 11, 12, S and the exact heat tangent) element-major (see below).
#include <algorithm>

#include "kernels.h"

namespace wqd {

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// ------------------------------------------------------------------ Gauss moments
__global__ void __launch_bounds__(128, 6) k_moments_f64(Rows rw, const int4* __restrict__ desc, int tc, int nc,
                                                        const double* __restrict__ table,
                                                        const double* __restrict__ gw, double* __restrict__ vals,
                                                        int max_n_i) {
    extern __shared__ double sh_acc[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (k >= rw.n) return;
    const int64_t i = rw.order ? rw.order[k] : k;
    double* acc = sh_acc + (int64_t)wib * max_n_i;
    const int r0 = rw.row_ptr[i], n_i = rw.row_ptr[i + 1] - r0;
    for (int x = lane; x < n_i; x += 32) acc[x] = 0.0;
    __syncwarp();
    for (int64_t s = rw.supp_ptr[i]; s < rw.supp_ptr[i + 1]; ++s) {
        const int4 d = desc[s];
        const int m = d.z & 255, P = (d.z >> 8) & 255, il = (d.z >> 16) & 255;
        const double* tb = table + d.x;
        const uint16_t* pos = rw.pos + d.w;
        const bool half = m <= 16;
        const int jl0 = half ? (lane & 15) : lane, hs = half ? (lane >> 4) : 0;
        double a0 = 0.0, a1 = 0.0;   // lanes own function jl0 (and jl0 + 32)
        for (int q0 = 0; q0 < P; q0 += 32) {
            const int nq = min(32, P - q0);
            double sv = 0.0;
            if (lane < nq) sv = gw[d.y + q0 + lane] * tb[((int64_t)(q0 + lane) * nc + tc) * m + il];
            if (half) {
                for (int qq = 0; qq < nq; qq += 2) {
                    const int q = qq + hs;
                    const double sq = __shfl_sync(0xffffffffu, sv, q & 31);
                    if (q < nq && jl0 < m) a0 = fma(sq, tb[((int64_t)(q0 + q) * nc + tc) * m + jl0], a0);
                }
            } else {
                for (int q = 0; q < nq; ++q) {
                    const double sq = __shfl_sync(0xffffffffu, sv, q);
                    const double* tq = tb + ((int64_t)(q0 + q) * nc + tc) * m;
                    if (jl0 < m) a0 = fma(sq, tq[jl0], a0);
                    if (jl0 + 32 < m) a1 = fma(sq, tq[jl0 + 32], a1);
                }
            }
        }
        if (half) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, 16);
            if (hs == 0 && jl0 < m) acc[pos[jl0]] += a0;
        } else {
            if (jl0 < m) acc[pos[jl0]] += a0;
            if (jl0 + 32 < m) acc[pos[jl0 + 32]] += a1;
            for (int j = jl0 + 64; j < m; j += 32) {   // m > 64: rare, recompute per function
                double a2 = 0.0;
                for (int q = 0; q < P; ++q) {
                    const double* tq = tb + ((int64_t)q * nc + tc) * m;
                    a2 = fma(gw[d.y + q] * tq[il], tq[j], a2);
                }
                acc[pos[j]] += a2;
            }
        }
        __syncwarp();
    }
    for (int x = lane; x < n_i; x += 32) vals[r0 + x] = acc[x];
}

cudaError_t launch_moments_f64(const Rows& rw, const int4* desc, int tc, int nc, const double* table,
                               const double* gw, double* vals, int max_n_i, cudaStream_t st) {
    if (rw.n == 0) return cudaSuccess;
    const int threads = 128, wpb = threads / 32;
    const unsigned blocks = (unsigned)((rw.n + wpb - 1) / wpb);
    const size_t smem = (size_t)wpb * max_n_i * sizeof(double);
    k_moments_f64<<<blocks, threads, smem, st>>>(rw, desc, tc, nc, table, gw, vals, max_n_i);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32
// Split products: weights, table values and coefficients are (hi, lo) float
// pairs with hi = fl32(v), lo = fl32(v - hi), and s * T ~ s_hi T_hi + (s_hi T_lo +
// s_lo T_hi).  The weighted terms of one entry cancel heavily, so plain FP32 sums
// of the s_hi T_hi lose digits (~1.5e-6 normwise on the 10,240-element Poisson
// workload, F32_FAST).  The compensated mode accumulates them without error
// growth by extraction against a power-of-two constant (the splitting idea of
// Rump, Ogita and Oishi, "Accurate floating-point summation", SIAM J. Sci.
// Comput. 31, 2008): with C = 2^k >= 4 B, B a bound on every partial sum of the
// entry, the accumulator acc = C + partial sum stays in [3C/4, 5C/4], so
//     acc' = fma(s_hi, T_hi, acc),  d = acc - acc'  (exact, Sterbenz),
//     e = fma(s_hi, T_hi, d)        (the rounding error of acc', to 2^-24 of itself)
// and the errors e, together with the cross terms, go to a correction sum lo.  The
// entry is (acc - C) + lo: 6 FP32 instructions per product, and errors of order
// N^2 2^-48 C for N products, far below the final FP32 rounding.  B is taken per
// tile and chunk as (products in the chunk) x max|s_hi| x max|T_hi|; on the next
// chunk the accumulator is moved to a new constant with TwoSum.
//
// Element-major form.  Phase 1 computes the dense block of every element's
// test x trial pairs
//     K_e[a][b] = sum_{q, t} s^t_{a q} T^t_{q b},  T^t_{q b} = D_{c_t} N_b(x_q),
//     s^t_{a q} = w^{c_t}_{i_a q} a_t(x_q)                     (WQ: weights of row i_a)
//     s^t_{a q} = w_q |J_q| a_t(x_q) D_{c_t} N_a(x_q)           (Gauss: test function)
// (a, b over the m_e functions of e, q over its points).  One warp computes one
// 16 x 16 tile of one block: a regular element (m_e = 16) is one tile; larger
// elements are several and are listed first, so their longer point loops start
// in the first wave.  Per chunk of points, the tile's trial table columns,
// test-side rows (weights or table values), coefficients and Gauss weights are
// copied to shared memory with cp.async in one batch; the products s are then
// formed in place and every lane accumulates one column b over 8 rows (two
// half-warps), reading its table value once per (point, term) and the row values
// as broadcasts.  Each entry goes to its slot in kscr, where the contributions to
// one CSR entry are contiguous and in the order of the elements in supp N_i.
// Phase 2, one thread per CSR entry, sums its slots with TwoSum.  No atomics: the
// result is bitwise reproducible.
constexpr int EL_NWARP = 4;     // warps per block

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Smallest power of two >= 4 x (a non-negative finite float x).
__device__ __forceinline__ float pow2_above_4x(float x) {
    const unsigned bits = __float_as_uint(x * 4.0f);
    return __uint_as_float(((bits >> 23) + 1u) << 23);
}

template <int NT, bool COMP, bool GAUSS, bool BATCH, int NP>
__global__ void __launch_bounds__(EL_NWARP * 32, 6)
    k_elem_f32(ElemItems it, ElemSrc one, BatchPlan bp, const __grid_constant__ PtrTable<NP> pt, TermsF tm) {
    constexpr int QC = NT <= 2 ? 12 : (NT <= 4 ? 8 : 4);   // most points per staged chunk
    __shared__ __align__(16) float2 sT[EL_NWARP][QC * NT * 16];   // trial side [point][term][column]
    __shared__ __align__(16) float2 sS[EL_NWARP][QC * NT * 16];   // test side, then the products s
    __shared__ __align__(16) double sD[EL_NWARP][5 * QC];         // coefficient rows 0..3, Gauss weights
    __shared__ __align__(16) float2 sC[EL_NWARP][QC * NT];        // split multipliers per (point, term)
    __shared__ __align__(16) int32_t sSlot[EL_NWARP][256];        // destination slots of the tile
    // every block of this grid has started once the last wave runs: from then on the
    // per-entry sums (a programmatic dependent) may be scheduled into freed slots
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * EL_NWARP + wib;
    if (k >= (BATCH ? bp.n_items : it.n)) return;
    const int4 d = BATCH ? bp.item[k] : it.item[k];
    const int kb = BATCH ? bp.kb[k] : it.kb[k];
    const int ri = BATCH ? bp.item_rule[k] : 0;
    const ElemSrc src = BATCH ? bp.src[ri] : one;
    const ElemPlan ep = src.ep;
    const int nc = src.nc, nwc = src.nwc;
    const float2* __restrict__ table2 = src.table2;
    const float2* __restrict__ W2e = src.W2e;
    const double* __restrict__ gw = src.gw;
    const double* __restrict__ coef = pt.coef[BATCH ? ri : 0];
    const int m = d.z & 255, P = (d.z >> 8) & 255, a0 = ((d.z >> 16) & 15) * 16, b0 = ((d.z >> 20) & 15) * 16;
    float2* T_ = sT[wib];
    float2* S_ = sS[wib];
    double* D_ = sD[wib];
    float2* C_ = sC[wib];
    const int bl = lane & 15, half = lane >> 4, rbase = 8 * half;
    const int b = b0 + bl;
    const bool bok = b < m, aok = a0 + bl < m;      // this lane's column; the row it stages
    int32_t* SL = sSlot[wib];
    // destination slots of the tile's entries, copied with the first chunk
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int a = a0 + rbase + r;
        if (bok && a < m) cp_async4(SL + (rbase + r) * 16 + bl, ep.scat + kb + a * m + b);
    }
    float acc[8], lo[8];
    float cst = 0.0f;                               // the extraction constant C
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = lo[r] = 0.0f;
    const int nch = (P + QC - 1) / QC;
    const int qc = (P + nch - 1) / nch;            // balanced chunks of at most QC points
    // staging offsets (32-bit: tables and weights are below 2^31 entries): lane (half, bl)
    // copies points q0 + half + 2 j, column / row bl
    const float2* tb = table2 + d.x;
    const int ncm = nc * m;
    const int tcol = half * ncm + b0 + bl, trow = half * ncm + a0 + bl;
    const float2* wb = W2e + (int64_t)d.w * nwc;
    const int wrow = (half * m + a0 + bl) * nwc, mnwc = m * nwc;
    for (int q0 = 0; q0 < P; q0 += qc) {
        const int nq = min(qc, P - q0);
        const int nj = (nq + 1 - half) >> 1;       // this half-warp's points in the chunk
        __syncwarp();
        for (int j = 0; j < nj; ++j) {
            const int qq = half + 2 * j;
            const int qo = (q0 + 2 * j) * ncm;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (bok) cp_async8(T_ + (qq * NT + t) * 16 + bl, tb + (tcol + qo + tm.tc[t] * m));
                if (aok) {
                    if (GAUSS)
                        cp_async8(S_ + (qq * NT + t) * 16 + bl, tb + (trow + qo + tm.sc[t] * m));
                    else
                        cp_async8(S_ + (qq * NT + t) * 16 + bl, wb + (wrow + (q0 + 2 * j) * mnwc + tm.wc[t]));
                }
            }
        }
        if (lane < nq) {
            if (coef)
                for (int cr = 0; cr < tm.ncrow; ++cr)
                    cp_async8(D_ + cr * QC + lane, coef + cr * tm.cstride + d.y + q0 + lane);
            if (GAUSS) cp_async8(D_ + 4 * QC + lane, gw + d.y + q0 + lane);
        }
        cp_async_wait_all();
        __syncwarp();
        if (lane < nq) {
            if (GAUSS) {
                const double g = D_[4 * QC + lane];
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const int cr = tm.crow[t];
                    C_[lane * NT + t] = split_double(g * (cr < 0 ? tm.scale[t] : (coef ? D_[cr * QC + lane] : 1.0)));
                }
            } else if (tm.ncrow <= 1) {
                const float2 cs = coef ? split_double(D_[lane]) : make_float2(1.0f, 0.0f);   // once per point
#pragma unroll
                for (int t = 0; t < NT; ++t)
                    C_[lane * NT + t] = tm.crow[t] >= 0 ? cs : make_float2(tm.shi[t], tm.slo[t]);
            } else {
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const int cr = tm.crow[t];
                    if (cr < 0)
                        C_[lane * NT + t] = make_float2(tm.shi[t], tm.slo[t]);
                    else
                        C_[lane * NT + t] = coef ? split_double(D_[cr * QC + lane]) : make_float2(1.0f, 0.0f);
                }
            }
        }
        __syncwarp();
        // products s in place (rows beyond m are zeroed), with the largest |s_hi| and
        // |T_hi| of the chunk for the accumulation bound
        float smax = 0.0f, tmax = 0.0f;
        for (int j = 0; j < nj; ++j) {
            const int qq = half + 2 * j;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                float2* sp = S_ + (qq * NT + t) * 16 + bl;
                float2 v = make_float2(0.0f, 0.0f);
                if (aok) {
                    const float2 w = *sp, c = C_[qq * NT + t];
                    float ph, pe;
                    two_prod(w.x, c.x, ph, pe);
                    v = make_float2(ph, pe + fmaf(w.x, c.y, w.y * c.x));
                }
                *sp = v;
                if (COMP) {
                    smax = fmaxf(smax, fabsf(v.x));
                    if (bok) tmax = fmaxf(tmax, fabsf(T_[(qq * NT + t) * 16 + bl].x));
                }
            }
        }
        if (COMP) {
            // constant for this chunk: C >= 4 (|value so far| + N max|s| max|T|)
            smax = warp_max(smax);
            tmax = warp_max(tmax);
            if (q0 == 0) {
                cst = pow2_above_4x((float)(nq * NT) * smax * tmax * 1.0001f);
#pragma unroll
                for (int r = 0; r < 8; ++r) acc[r] = cst;
            } else {
                float vmax = 0.0f;
#pragma unroll
                for (int r = 0; r < 8; ++r) vmax = fmaxf(vmax, fabsf(acc[r] - cst));
                vmax = warp_max(vmax);
                const float cn = pow2_above_4x(vmax + (float)(nq * NT) * smax * tmax * 1.0001f);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    float s2, e2;
                    two_sum(cn, acc[r] - cst, s2, e2);
                    acc[r] = s2;
                    lo[r] += e2;
                }
                cst = cn;
            }
        }
        __syncwarp();
        if (bok) {
#pragma unroll 2
            for (int qq = 0; qq < nq; ++qq) {
                float2 T[NT];
                const float4* srow[NT];
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    T[t] = T_[(qq * NT + t) * 16 + bl];
                    srow[t] = reinterpret_cast<const float4*>(S_ + (qq * NT + t) * 16 + rbase);
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
    }
    cp_async_wait_all();
    __syncwarp();
    if (bok) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (a0 + rbase + r < m) ep.kscr[SL[(rbase + r) * 16 + bl]] = make_float2(acc[r] - cst, lo[r]);
    }
}

// Phase 2: one thread per two consecutive CSR entries.  Their slots are contiguous;
// they are fetched 8 at a time, all loads in flight together, and each is added
// with TwoSum to the entry it belongs to (in slot order, i.e. support order).
template <bool COMP, bool BATCH, int NP>
__global__ void __launch_bounds__(256) k_gather_f32(ElemSrc one, BatchPlan bp, const __grid_constant__ PtrTable<NP> pt) {
    // launched as a programmatic dependent of the element kernel (see the wait below)
    const int ri = BATCH ? bp.gblk_rule[blockIdx.x] : 0;
    const int64_t base = BATCH ? bp.gblk_start[blockIdx.x] : (int64_t)blockIdx.x * 512;
    const ElemSrc src = BATCH ? bp.src[ri] : one;
    const int64_t nnz = src.nnz;
    const int32_t* __restrict__ gptr = src.ep.gptr;
    const float2* __restrict__ kscr = src.ep.kscr;
    float* __restrict__ vals = pt.vals[BATCH ? ri : 0];
    const int64_t n = base + 2 * threadIdx.x;
    // the slot ranges do not depend on the element kernel: read them before waiting for it
    int c0 = 0, c1 = 0, c2 = 0;
    if (n < nnz) {
        c0 = gptr[n];
        c1 = gptr[n + 1];
        c2 = gptr[min(n + 2, nnz)];
    }
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (n >= nnz) return;
    float hi0 = 0.0f, lo0 = 0.0f, hi1 = 0.0f, lo1 = 0.0f;
    for (int cb = c0; cb < c2; cb += 8) {
        float2 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = cb + j < c2 ? kscr[cb + j] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool first = cb + j < c1;
            float h = first ? hi0 : hi1, l = first ? lo0 : lo1;
            if (COMP) {
                float s3, e3;
                two_sum(h, v[j].x, s3, e3);
                h = s3;
                l += v[j].y + e3;
            } else {
                h += v[j].x;
                l += v[j].y;
            }
            if (first) hi0 = h, lo0 = l;
            else hi1 = h, lo1 = l;
        }
    }
    // n is even: one 8-byte store per pair where the output is 8-byte aligned (a warp
    // then writes 256 contiguous bytes in one instruction, also to mapped host memory)
    if (n + 1 < nnz && (reinterpret_cast<uintptr_t>(vals) & 7) == 0) {
        *reinterpret_cast<float2*>(vals + n) = make_float2(hi0 + lo0, hi1 + lo1);
    } else {
        vals[n] = hi0 + lo0;
        if (n + 1 < nnz) vals[n + 1] = hi1 + lo1;
    }
}

// Element kernel, then the per-entry sums as a programmatic dependent launch (its
// grid is set up while the element kernel drains and waits with griddepcontrol.wait).
template <bool BATCH, int NP>
static cudaError_t launch_elem_pair(const ElemItems& it, const ElemSrc& one, const BatchPlan& bp,
                                    const PtrTable<NP>& pt, const Terms& tm, int gauss, bool compensated,
                                    int64_t n_items, int64_t n_gblocks, cudaStream_t st, cudaEvent_t* evs) {
    const int ntk = tm.nt <= 4 ? tm.nt : 8;         // more than 4 terms run as 8 (zero padding)
    const TermsF tf = make_terms_f(tm, ntk);
    const unsigned eb = (unsigned)((n_items + EL_NWARP - 1) / EL_NWARP);
#define WQ_EL_CASE(N, C)                                                                                  \
    do {                                                                                                  \
        if (gauss)                                                                                        \
            k_elem_f32<N, C, true, BATCH, NP><<<eb, EL_NWARP * 32, 0, st>>>(it, one, bp, pt, tf);         \
        else                                                                                              \
            k_elem_f32<N, C, false, BATCH, NP><<<eb, EL_NWARP * 32, 0, st>>>(it, one, bp, pt, tf);        \
    } while (0)
    if (n_items > 0) {
        switch (ntk * 2 + (compensated ? 1 : 0)) {
            case 2: WQ_EL_CASE(1, false); break;
            case 3: WQ_EL_CASE(1, true); break;
            case 4: WQ_EL_CASE(2, false); break;
            case 5: WQ_EL_CASE(2, true); break;
            case 6: WQ_EL_CASE(3, false); break;
            case 7: WQ_EL_CASE(3, true); break;
            case 8: WQ_EL_CASE(4, false); break;
            case 9: WQ_EL_CASE(4, true); break;
            case 16: WQ_EL_CASE(8, false); break;
            default: WQ_EL_CASE(8, true); break;
        }
    }
#undef WQ_EL_CASE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (evs) cudaEventRecord(evs[1], st);
    if (n_gblocks == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)n_gblocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (compensated)
        e = cudaLaunchKernelEx(&cfg, k_gather_f32<true, BATCH, NP>, one, bp, pt);
    else
        e = cudaLaunchKernelEx(&cfg, k_gather_f32<false, BATCH, NP>, one, bp, pt);
    return e;
}

cudaError_t launch_elem_f32(const ElemItems& it, const ElemSrc& src, const Terms& tm, int gauss, const double* coef,
                            float* vals, bool compensated, cudaStream_t st, cudaEvent_t* evs) {
    if (evs) cudaEventRecord(evs[0], st);
    cudaError_t e = cudaSuccess;
    if (src.nnz > 0) {
        PtrTable<1> pt;
        pt.coef[0] = coef;
        pt.vals[0] = vals;
        e = launch_elem_pair<false, 1>(it, src, BatchPlan{}, pt, tm, gauss, compensated, it.n, (src.nnz + 511) / 512,
                                       st, evs);
    } else if (evs) {
        cudaEventRecord(evs[1], st);
    }
    if (evs) cudaEventRecord(evs[2], st);
    return e;
}

cudaError_t launch_gather_f32(const ElemSrc& src, float* vals, bool compensated, cudaStream_t st) {
    if (src.nnz == 0) return cudaSuccess;
    PtrTable<1> pt;
    pt.coef[0] = nullptr;
    pt.vals[0] = vals;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((src.nnz + 511) / 512));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (compensated) return cudaLaunchKernelEx(&cfg, k_gather_f32<true, false, 1>, src, BatchPlan{}, pt);
    return cudaLaunchKernelEx(&cfg, k_gather_f32<false, false, 1>, src, BatchPlan{}, pt);
}

cudaError_t launch_elem_batch(const BatchPlan& bp, const double* const* coefs, float* const* vals, int k,
                              const Terms& tm, bool compensated, cudaStream_t st) {
    if (k < 1 || k > WQ_BATCH_MAX) return cudaErrorInvalidValue;
    PtrTable<WQ_BATCH_MAX> pt{};
    for (int r = 0; r < k; ++r) {
        pt.coef[r] = coefs[r];
        pt.vals[r] = vals[r];
    }
    return launch_elem_pair<true, WQ_BATCH_MAX>(ElemItems{}, ElemSrc{}, bp, pt, tm, 0, compensated, bp.n_items,
                                                bp.n_gblocks, st, nullptr);
}

// ------------------------------------------------------------------ FP64 element-major
// The same tiles and slot map in FP64: K_e[a][b] = sum_{q,t} s^t_aq T^t_qb with
// s = w c (WQ) or w_q |J_q| c D N_a (Gauss), one FMA per product, no compensation
// (FP64 sums of a few tens of products), the block entries in the slot buffer as
// doubles, then one plain per-entry sum in support order.  Bound by the FP64 pipes
// (2 FMA per cycle per SM on this GPU).
template <int NT, bool GAUSS>
__global__ void __launch_bounds__(EL_NWARP * 32, 6)
    k_elem_f64(ElemItems it, ElemSrc64 src, const double* __restrict__ coef, Terms tm) {
    constexpr int QC = NT <= 2 ? 12 : (NT <= 4 ? 8 : 4);
    __shared__ __align__(16) double sT[EL_NWARP][QC * NT * 16];
    __shared__ __align__(16) double sS[EL_NWARP][QC * NT * 16];
    __shared__ __align__(16) double sD[EL_NWARP][5 * QC];
    __shared__ __align__(16) int32_t sSlot[EL_NWARP][256];
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * EL_NWARP + wib;
    if (k >= it.n) return;
    const int4 d = it.item[k];
    const int kb = it.kb[k];
    const int m = d.z & 255, P = (d.z >> 8) & 255, a0 = ((d.z >> 16) & 15) * 16, b0 = ((d.z >> 20) & 15) * 16;
    double* T_ = sT[wib];
    double* S_ = sS[wib];
    double* D_ = sD[wib];
    int32_t* SL = sSlot[wib];
    const int bl = lane & 15, half = lane >> 4, rbase = 8 * half;
    const int b = b0 + bl;
    const bool bok = b < m, aok = a0 + bl < m;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int a = a0 + rbase + r;
        if (bok && a < m) cp_async4(SL + (rbase + r) * 16 + bl, src.scat + kb + a * m + b);
    }
    int ncrow = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) ncrow = max(ncrow, tm.t[t].crow + 1);
    double acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.0;
    const int nch = (P + QC - 1) / QC;
    const int qc = (P + nch - 1) / nch;
    const double* tb = src.table + d.x;
    const int ncm = src.nc * m;
    const int tcol = half * ncm + b0 + bl, trow = half * ncm + a0 + bl;
    const double* wb = src.We + (int64_t)d.w * src.nwc;
    const int wrow = (half * m + a0 + bl) * src.nwc, mnwc = m * src.nwc;
    for (int q0 = 0; q0 < P; q0 += qc) {
        const int nq = min(qc, P - q0);
        const int nj = (nq + 1 - half) >> 1;
        __syncwarp();
        for (int j = 0; j < nj; ++j) {
            const int qq = half + 2 * j;
            const int qo = (q0 + 2 * j) * ncm;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (bok) cp_async8(T_ + (qq * NT + t) * 16 + bl, tb + (tcol + qo + tm.t[t].tc * m));
                if (aok) {
                    if (GAUSS)
                        cp_async8(S_ + (qq * NT + t) * 16 + bl, tb + (trow + qo + tm.t[t].sc * m));
                    else
                        cp_async8(S_ + (qq * NT + t) * 16 + bl, wb + (wrow + (q0 + 2 * j) * mnwc + tm.t[t].wc));
                }
            }
        }
        if (lane < nq) {
            if (coef)
                for (int cr = 0; cr < ncrow; ++cr)
                    cp_async8(D_ + cr * QC + lane, coef + cr * tm.cstride + d.y + q0 + lane);
            if (GAUSS) cp_async8(D_ + 4 * QC + lane, src.gw + d.y + q0 + lane);
        }
        cp_async_wait_all();
        __syncwarp();
        // products s in place (rows beyond m are zeroed)
        for (int j = 0; j < nj; ++j) {
            const int qq = half + 2 * j;
            const double g = GAUSS ? D_[4 * QC + qq] : 1.0;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                double* sp = S_ + (qq * NT + t) * 16 + bl;
                const int cr = tm.t[t].crow;
                const double c = cr < 0 ? tm.t[t].scale : (coef ? D_[cr * QC + qq] : 1.0);
                *sp = aok ? *sp * (g * c) : 0.0;
            }
        }
        __syncwarp();
        if (bok) {
#pragma unroll 2
            for (int qq = 0; qq < nq; ++qq) {
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const double T = T_[(qq * NT + t) * 16 + bl];
                    const double2* srow = reinterpret_cast<const double2*>(S_ + (qq * NT + t) * 16 + rbase);
#pragma unroll
                    for (int r2 = 0; r2 < 4; ++r2) {
                        const double2 sv = srow[r2];
                        acc[2 * r2] = fma(sv.x, T, acc[2 * r2]);
                        acc[2 * r2 + 1] = fma(sv.y, T, acc[2 * r2 + 1]);
                    }
                }
            }
        }
    }
    cp_async_wait_all();
    __syncwarp();
    if (bok) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (a0 + rbase + r < m) src.kscr[SL[(rbase + r) * 16 + bl]] = acc[r];
    }
}

__global__ void __launch_bounds__(256) k_gather_f64(int64_t nnz, const int32_t* __restrict__ gptr,
                                                    const double* __restrict__ kscr, double* __restrict__ vals) {
    const int64_t n = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    int c0 = 0, c1 = 0, c2 = 0;
    if (n < nnz) {
        c0 = gptr[n];
        c1 = gptr[n + 1];
        c2 = gptr[min(n + 2, nnz)];
    }
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (n >= nnz) return;
    double s0 = 0.0, s1 = 0.0;
    for (int c = c0; c < c1; ++c) s0 += kscr[c];
    for (int c = c1; c < c2; ++c) s1 += kscr[c];
    if (n + 1 < nnz && (reinterpret_cast<uintptr_t>(vals) & 15) == 0) {
        *reinterpret_cast<double2*>(vals + n) = make_double2(s0, s1);
    } else {
        vals[n] = s0;
        if (n + 1 < nnz) vals[n + 1] = s1;
    }
}

cudaError_t launch_elem_f64(const ElemItems& it, const ElemSrc64& src, const Terms& tm, int gauss,
                            const double* coef, double* vals, cudaStream_t st, cudaEvent_t* evs) {
    if (evs) cudaEventRecord(evs[0], st);
    cudaError_t e = cudaSuccess;
    if (src.nnz > 0 && it.n > 0) {
        Terms tp = tm;
        const int ntk = tm.nt <= 4 ? tm.nt : 8;
        for (int t = tm.nt; t < ntk; ++t) tp.t[t] = {0, 0, 0, -1, 0.0};
        const unsigned eb = (unsigned)((it.n + EL_NWARP - 1) / EL_NWARP);
#define WQ_E64_CASE(N)                                                                                   \
    do {                                                                                                 \
        if (gauss)                                                                                       \
            k_elem_f64<N, true><<<eb, EL_NWARP * 32, 0, st>>>(it, src, coef, tp);                        \
        else                                                                                             \
            k_elem_f64<N, false><<<eb, EL_NWARP * 32, 0, st>>>(it, src, coef, tp);                       \
    } while (0)
        switch (ntk) {
            case 1: WQ_E64_CASE(1); break;
            case 2: WQ_E64_CASE(2); break;
            case 3: WQ_E64_CASE(3); break;
            case 4: WQ_E64_CASE(4); break;
            default: WQ_E64_CASE(8); break;
        }
#undef WQ_E64_CASE
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (evs) cudaEventRecord(evs[1], st);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)((src.nnz + 511) / 512));
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_gather_f64, src.nnz, src.gptr, (const double*)src.kscr, vals);
    } else if (evs) {
        cudaEventRecord(evs[1], st);
    }
    if (evs) cudaEventRecord(evs[2], st);
    return e;
}

// Element-major copy of the FP64 weights (We[dst[r]] = W[r], nwc columns).
__global__ void k_copy_rows(const double* __restrict__ W, const int32_t* __restrict__ dst, double* __restrict__ We,
                            int64_t rows, int nwc) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < rows * nwc;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = x / nwc, c = x - r * nwc;
        We[(int64_t)dst[r] * nwc + c] = W[x];
    }
}

cudaError_t launch_copy_rows(const double* W, const int32_t* dst, double* We, int64_t rows, int nwc, int n_sm,
                             cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((rows * nwc + 255) / 256, (int64_t)std::max(n_sm, 1) * 16);
    k_copy_rows<<<blocks, 256, 0, st>>>(W, dst, We, rows, nwc);
    return cudaGetLastError();
}

// Element-major split copy of the weights: row r of W (test function i, point q
// of element e) goes to W2e row dst[r] = wbase_e + q m_e + a(i, e).
__global__ void k_split_rows(const double* __restrict__ W, const int32_t* __restrict__ dst, float2* __restrict__ W2e,
                             int64_t rows, int nwc) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < rows * nwc;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = x / nwc, c = x - r * nwc;
        const double v = W[x];
        const float h = (float)v;
        W2e[(int64_t)dst[r] * nwc + c] = make_float2(h, (float)(v - (double)h));
    }
}

cudaError_t launch_split_rows(const double* W, const int32_t* dst, float2* W2e, int64_t rows, int nwc, int n_sm,
                              cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((rows * nwc + 255) / 256, (int64_t)std::max(n_sm, 1) * 16);
    k_split_rows<<<blocks, 256, 0, st>>>(W, dst, W2e, rows, nwc);
    return cudaGetLastError();
}

}  // namespace wqd
