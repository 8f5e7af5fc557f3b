// Row-wise assembly (paper Eqs. 9, 11, 12 and the WQ form of Eq. S):
//     A_ij = sum_{q in pts(supp N_i)} sum_t w^{c_t}_iq * a_t(x_q) * D_{c_t} N_j(x_q),
// one warp per test function (row) i, the row's n_i values accumulated in
// shared memory and written once (no atomics, deterministic).  The warp walks
// the elements of supp N_i in ascending order; lane jl handles local function
// jl of the element and adds its contribution at the row position pos[jl]
// (positions of one element are distinct, so the lanes never collide).
//
// The same engine runs element-wise Gauss quadrature row by row (the paper's
// reference, Table 2 right column): the "weight" of test function i at Gauss
// point g is w_g |J_g| D_c N_i(x_g), read from the Gauss table.
#include <algorithm>

#include "kernels.h"

namespace wqd {

template <int GAUSS, int NT>
__global__ void __launch_bounds__(128) k_rowasm_f64(Elems el, Rows rw, Terms tm, const double* __restrict__ table,
                                                    const double* __restrict__ W, int nwc,
                                                    const double* __restrict__ gw, const double* __restrict__ coef,
                                                    double* __restrict__ vals, int max_n_i) {
    extern __shared__ double sh_acc[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= rw.n) return;
    double* acc = sh_acc + (int64_t)wib * max_n_i;
    const int r0 = rw.row_ptr[i], n_i = rw.row_ptr[i + 1] - r0;
    for (int k = lane; k < n_i; k += 32) acc[k] = 0.0;
    __syncwarp();
    const int nc = el.nc;
    int64_t woff = GAUSS ? 0 : rw.w_ptr[i];
    for (int64_t s = rw.supp_ptr[i]; s < rw.supp_ptr[i + 1]; ++s) {
        const int e = rw.supp[s];
        const int m = el.m[e];
        const uint16_t* pos = rw.pos + rw.pos_ptr[s];
        if (!GAUSS) {
            const int side = el.side[e], P = side * side;
            const double* tb = table + el.bt_ptr[e];
            const int64_t pp = el.pt_ptr[e];
            for (int jl = lane; jl < m; jl += 32) {
                double v = 0.0;
                for (int q = 0; q < P; ++q) {
                    const double* wrow = W + (woff + q) * nwc;
                    const double cq = coef ? coef[pp + q] : 1.0;
                    const double* tq = tb + (int64_t)q * nc * m + jl;
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const double a = tm.t[t].use_coef ? cq : tm.t[t].scale;
                        v += (wrow[tm.t[t].wc] * a) * tq[tm.t[t].tc * m];
                    }
                }
                acc[pos[jl]] += v;
            }
            woff += P;
        } else {
            const int il = rw.il[s];
            const int P = 16 * el.nsub[e];
            const double* tb = table + el.gbt_ptr[e];
            const int64_t pp = el.gp_ptr[e];
            for (int jl = lane; jl < m; jl += 32) {
                double v = 0.0;
                for (int g = 0; g < P; ++g) {
                    const double wg = gw[pp + g] * (coef ? coef[pp + g] : 1.0);
                    const double* tq = tb + (int64_t)g * nc * m;
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const double a = tm.t[t].use_coef ? wg : gw[pp + g] * tm.t[t].scale;
                        v += (a * tq[tm.t[t].tc * m + il]) * tq[tm.t[t].tc * m + jl];
                    }
                }
                acc[pos[jl]] += v;
            }
        }
        __syncwarp();
    }
    for (int k = lane; k < n_i; k += 32) vals[r0 + k] = acc[k];
}

cudaError_t launch_rowasm_f64(const Elems& el, const Rows& rw, const Terms& tm, int gauss, const double* table,
                              const double* W, int nwc, const double* gw, const double* coef, double* vals,
                              int max_n_i, cudaStream_t st) {
    if (rw.n == 0) return cudaSuccess;
    const int threads = 128, wpb = threads / 32;
    const unsigned blocks = (unsigned)((rw.n + wpb - 1) / wpb);
    const size_t smem = (size_t)wpb * max_n_i * sizeof(double);
#define WQ_F64_CASE(G, N) \
    k_rowasm_f64<G, N><<<blocks, threads, smem, st>>>(el, rw, tm, table, W, nwc, gw, coef, vals, max_n_i)
    switch (tm.nt + 4 * (gauss ? 1 : 0)) {
        case 1: WQ_F64_CASE(0, 1); break;
        case 2: WQ_F64_CASE(0, 2); break;
        case 3: WQ_F64_CASE(0, 3); break;
        case 4: WQ_F64_CASE(0, 4); break;
        case 5: WQ_F64_CASE(1, 1); break;
        case 6: WQ_F64_CASE(1, 2); break;
        case 7: WQ_F64_CASE(1, 3); break;
        default: WQ_F64_CASE(1, 4); break;
    }
#undef WQ_F64_CASE
    return cudaGetLastError();
}

// ---------------------------------------------------------------- FP32 path
// Split products: every FP64 weight and table value is stored as a pair of
// floats (hi, lo) with hi = fl32(v), lo = fl32(v - hi); the coefficient is split
// on the fly.  One term contributes
//     s = (w_hi + w_lo)(c_hi + c_lo) ~ s_hi + s_lo  (exact product of the his by FMA),
//     s * T ~ s_hi T_hi + (s_hi T_lo + s_lo T_hi),
// and the large parts are summed with an error-free transformation (Knuth's
// TwoSum), whose rounding errors join the correction sum.  The weighted terms
// cancel heavily (stiffness rows sum to zero), so a plain FP32 sum of the large
// parts would lose several digits.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// One CTA per SM walks a contiguous chunk of rows of the spatially sorted row
// order (rows that share elements run on the same SM, so the element tables
// stay in L1).  Per support element, lane q first forms the split product
// s_q = w_iq * a_t(x_q) for point q of the chunk; lanes then take functions:
// for m <= 16 the two half-warps take alternate points and are merged at the
// end, otherwise one lane per function.  Point products are broadcast with
// shuffles.
template <int NT>
__global__ void __launch_bounds__(1024, 1) k_rowasm_f32(Elems el, Rows rw, TermsF tm, const float2* __restrict__ table2,
                                                      const float2* __restrict__ W2, int nwc,
                                                      const double* __restrict__ coef, float* __restrict__ vals,
                                                      int max_n_i, int64_t rows_per_cta) {
    extern __shared__ float sh_accf[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float* acc = sh_accf + (int64_t)wib * 2 * max_n_i;
    const int64_t k0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t k1 = min(rw.n, k0 + rows_per_cta);
    const int nc = el.nc;
    for (int64_t k = k0 + wib; k < k1; k += nw) {
        const int64_t i = rw.order ? rw.order[k] : k;
        const int r0 = rw.row_ptr[i], n_i = rw.row_ptr[i + 1] - r0;
        for (int x = lane; x < 2 * n_i; x += 32) acc[x] = 0.0f;
        __syncwarp();
        int64_t woff = rw.w_ptr[i];
        for (int64_t s = rw.supp_ptr[i]; s < rw.supp_ptr[i + 1]; ++s) {
            const int e = rw.supp[s];
            const int m = el.m[e];
            const uint16_t* pos = rw.pos + rw.pos_ptr[s];
            const int side = el.side[e], P = side * side;
            const float2* tb = table2 + el.bt_ptr[e];
            const int64_t pp = el.pt_ptr[e];
            const bool half = m <= 16;
            for (int q0 = 0; q0 < P; q0 += 32) {
                const int nq = min(32, P - q0);
                float shi[NT], slo[NT];
                if (lane < nq) {
                    const double cd = coef ? coef[pp + q0 + lane] : 1.0;
                    const float chi = __double2float_rn(cd);
                    const float clo = __double2float_rn(cd - (double)chi);
                    const float2* wrow = W2 + (woff + q0 + lane) * nwc;
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const float ahi = tm.use_coef[t] ? chi : tm.shi[t];
                        const float alo = tm.use_coef[t] ? clo : tm.slo[t];
                        const float2 w = wrow[tm.wc[t]];
                        float ph, pe;
                        two_prod(w.x, ahi, ph, pe);
                        shi[t] = ph;
                        slo[t] = pe + fmaf(w.x, alo, w.y * ahi);
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < NT; ++t) shi[t] = slo[t] = 0.0f;
                }
                if (half) {
                    const int jl = lane & 15, hs = lane >> 4;
                    float hi = 0.0f, lo = 0.0f;
                    for (int qq = 0; qq < nq; qq += 2) {
                        const int q = qq + hs;
                        const bool ok = (q < nq) && (jl < m);
                        const float2* tq = tb + (int64_t)(q0 + q) * nc * m + jl;
#pragma unroll
                        for (int t = 0; t < NT; ++t) {
                            const float ah = __shfl_sync(0xffffffffu, shi[t], q & 31);
                            const float al = __shfl_sync(0xffffffffu, slo[t], q & 31);
                            if (ok) {
                                const float2 T = tq[tm.tc[t] * m];
                                float ph, pe, s2, e2;
                                two_prod(ah, T.x, ph, pe);
                                two_sum(hi, ph, s2, e2);
                                hi = s2;
                                lo += e2 + pe + fmaf(ah, T.y, al * T.x);
                            }
                        }
                    }
                    // merge the two half-warps (alternate points)
                    const float ohi = __shfl_xor_sync(0xffffffffu, hi, 16);
                    const float olo = __shfl_xor_sync(0xffffffffu, lo, 16);
                    if (hs == 0 && jl < m) {
                        float s2, e2;
                        two_sum(hi, ohi, s2, e2);
                        const int p = pos[jl];
                        float s3, e3;
                        two_sum(acc[2 * p], s2, s3, e3);
                        acc[2 * p] = s3;
                        acc[2 * p + 1] += lo + olo + e2 + e3;
                    }
                } else {
                    for (int j0 = 0; j0 < m; j0 += 32) {
                        const int jl = j0 + lane;
                        float hi = 0.0f, lo = 0.0f;
                        for (int q = 0; q < nq; ++q) {
                            const float2* tq = tb + (int64_t)(q0 + q) * nc * m + jl;
#pragma unroll
                            for (int t = 0; t < NT; ++t) {
                                const float ah = __shfl_sync(0xffffffffu, shi[t], q);
                                const float al = __shfl_sync(0xffffffffu, slo[t], q);
                                if (jl < m) {
                                    const float2 T = tq[tm.tc[t] * m];
                                    float ph, pe, s2, e2;
                                    two_prod(ah, T.x, ph, pe);
                                    two_sum(hi, ph, s2, e2);
                                    hi = s2;
                                    lo += e2 + pe + fmaf(ah, T.y, al * T.x);
                                }
                            }
                        }
                        if (jl < m) {
                            const int p = pos[jl];
                            float s3, e3;
                            two_sum(acc[2 * p], hi, s3, e3);
                            acc[2 * p] = s3;
                            acc[2 * p + 1] += lo + e3;
                        }
                    }
                }
                __syncwarp();
            }
            woff += P;
        }
        for (int x = lane; x < n_i; x += 32) vals[r0 + x] = acc[2 * x] + acc[2 * x + 1];
        __syncwarp();
    }
}

cudaError_t launch_rowasm_f32(const Elems& el, const Rows& rw, const Terms& tm, const float2* table2,
                              const float2* W2, int nwc, const double* coef, float* vals, int max_n_i,
                              cudaStream_t st) {
    if (rw.n == 0) return cudaSuccess;
    TermsF tf{};
    for (int t = 0; t < tm.nt; ++t) {
        tf.wc[t] = tm.t[t].wc;
        tf.tc[t] = tm.t[t].tc;
        tf.use_coef[t] = tm.t[t].use_coef;
        tf.shi[t] = (float)tm.t[t].scale;
        tf.slo[t] = (float)(tm.t[t].scale - (double)tf.shi[t]);
    }
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 1024;
    const int64_t n_cta = std::min<int64_t>(std::max(n_sm, 1), (rw.n + 31) / 32);
    const int64_t rpc = (rw.n + n_cta - 1) / n_cta;
    const size_t smem = (size_t)(threads / 32) * 2 * max_n_i * sizeof(float);
    switch (tm.nt) {
        case 1: k_rowasm_f32<1><<<(unsigned)n_cta, threads, smem, st>>>(el, rw, tf, table2, W2, nwc, coef, vals, max_n_i, rpc); break;
        case 2: k_rowasm_f32<2><<<(unsigned)n_cta, threads, smem, st>>>(el, rw, tf, table2, W2, nwc, coef, vals, max_n_i, rpc); break;
        case 3: k_rowasm_f32<3><<<(unsigned)n_cta, threads, smem, st>>>(el, rw, tf, table2, W2, nwc, coef, vals, max_n_i, rpc); break;
        default: k_rowasm_f32<4><<<(unsigned)n_cta, threads, smem, st>>>(el, rw, tf, table2, W2, nwc, coef, vals, max_n_i, rpc); break;
    }
    return cudaGetLastError();
}

}  // namespace wqd
