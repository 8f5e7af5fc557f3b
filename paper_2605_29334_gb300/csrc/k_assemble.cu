// Row-wise assembly (paper Eqs. 9, 11, 12 and the WQ form of Eq. S):
//     A_ij = sum_{q in pts(supp N_i)} sum_t  s^t_iq * D_{c_t} N_j(x_q),
//     s^t_iq = w^{c_t}_iq * a_t(x_q)                    (WQ: weights of row i)
//     s^t_ig = w_g |J_g| a_t(x_g) * D_{c_t} N_i(x_g)     (Gauss: test function value)
// One warp per test function (row) i; the row's n_i values are accumulated in
// shared memory and written once (no atomics, deterministic).  The warp walks
// the elements of supp N_i; for each element the per-point products s^t are
// formed once, lane-parallel (lane q <-> point q), and broadcast by shuffles.
// Functions go to lanes: for m_e <= 16 the two half-warps take alternate points
// and are merged at the end of the element (all 32 lanes busy), otherwise one
// lane per function.  Positions of one element's functions in row i are
// distinct, so lanes never collide in the row accumulator.
//
// Per support entry a packed descriptor {table offset, first point, m | P << 8 |
// il << 16, position offset} replaces the chain of dependent index loads.
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

// ------------------------------------------------------------------ FP64
template <int GAUSS, int NT>
__global__ void __launch_bounds__(128, 6) k_rowasm_f64(Rows rw, const int4* __restrict__ desc, Terms tm, int nc,
                                                       const double* __restrict__ table,
                                                       const double* __restrict__ W, int nwc,
                                                       const double* __restrict__ gw,
                                                       const double* __restrict__ coef,
                                                       double* __restrict__ vals, int max_n_i) {
    extern __shared__ double sh_acc[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (k >= rw.n) return;
    const int64_t i = rw.order ? rw.order[k] : k;
    double* acc = sh_acc + (int64_t)wib * max_n_i;
    const int r0 = rw.row_ptr[i], n_i = rw.row_ptr[i + 1] - r0;
    for (int x = lane; x < n_i; x += 32) acc[x] = 0.0;
    __syncwarp();
    int64_t woff = GAUSS ? 0 : rw.w_ptr[i];
    const int64_t s0 = rw.supp_ptr[i], s1 = rw.supp_ptr[i + 1];
    for (int64_t s = s0; s < s1; ++s) {
        const int4 d = desc[s];
        const int m = d.z & 255, P = (d.z >> 8) & 255, il = (d.z >> 16) & 255;
        const double* tb = table + d.x;
        const uint16_t* pos = rw.pos + d.w;
        const bool half = m <= 16;
        const int jl0 = half ? (lane & 15) : lane, hs = half ? (lane >> 4) : 0;
        double a0 = 0.0, a1 = 0.0;   // lanes own function jl0 (and jl0 + 32)
        for (int q0 = 0; q0 < P; q0 += 32) {
            const int nq = min(32, P - q0);
            double sv[NT];
            if (lane < nq) {
                const int q = q0 + lane;
                const double c = coef ? coef[d.y + q] : 1.0;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const double a = tm.t[t].use_coef ? c : tm.t[t].scale;
                    if (GAUSS)
                        sv[t] = gw[d.y + q] * a * tb[((int64_t)q * nc + tm.t[t].tc) * m + il];
                    else
                        sv[t] = W[(woff + q) * nwc + tm.t[t].wc] * a;
                }
            } else {
#pragma unroll
                for (int t = 0; t < NT; ++t) sv[t] = 0.0;
            }
            if (half) {
                for (int qq = 0; qq < nq; qq += 2) {
                    const int q = qq + hs;
                    const bool ok = q < nq && jl0 < m;
                    const double* tq = tb + (int64_t)(q0 + q) * nc * m + jl0;
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const double sq = __shfl_sync(0xffffffffu, sv[t], q & 31);
                        if (ok) a0 = fma(sq, tq[tm.t[t].tc * m], a0);
                    }
                }
            } else {
                for (int q = 0; q < nq; ++q) {
                    const double* tq = tb + (int64_t)(q0 + q) * nc * m;
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const double sq = __shfl_sync(0xffffffffu, sv[t], q);
                        if (jl0 < m) a0 = fma(sq, tq[tm.t[t].tc * m + jl0], a0);
                        if (jl0 + 32 < m) a1 = fma(sq, tq[tm.t[t].tc * m + jl0 + 32], a1);
                    }
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
                    const double* tq = tb + (int64_t)q * nc * m;
                    const double c = coef ? coef[d.y + q] : 1.0;
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const double a = tm.t[t].use_coef ? c : tm.t[t].scale;
                        const double sq = GAUSS ? gw[d.y + q] * a * tq[tm.t[t].tc * m + il]
                                                : W[(woff + q) * nwc + tm.t[t].wc] * a;
                        a2 = fma(sq, tq[tm.t[t].tc * m + j], a2);
                    }
                }
                acc[pos[j]] += a2;
            }
        }
        if (!GAUSS) woff += P;
        __syncwarp();
    }
    for (int x = lane; x < n_i; x += 32) vals[r0 + x] = acc[x];
}

cudaError_t launch_rowasm_f64(const Rows& rw, const int4* desc, const Terms& tm, int nc, int gauss,
                              const double* table, const double* W, int nwc, const double* gw, const double* coef,
                              double* vals, int max_n_i, cudaStream_t st) {
    if (rw.n == 0) return cudaSuccess;
    const int threads = 128, wpb = threads / 32;
    const unsigned blocks = (unsigned)((rw.n + wpb - 1) / wpb);
    const size_t smem = (size_t)wpb * max_n_i * sizeof(double);
#define WQ_F64_CASE(G, N) \
    k_rowasm_f64<G, N><<<blocks, threads, smem, st>>>(rw, desc, tm, nc, table, W, nwc, gw, coef, vals, max_n_i)
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

// ------------------------------------------------------------------ FP32
// Split products: weights, table values and coefficients are (hi, lo) float
// pairs with hi = fl32(v), lo = fl32(v - hi).  Per point, lane q forms
//     s = (w_hi + w_lo)(a_hi + a_lo) ~ s_hi + s_lo   (exact product of the his by FMA);
// per function, s * T ~ s_hi T_hi + (s_hi T_lo + s_lo T_hi), the large parts summed
// with Knuth's TwoSum (error-free) and every rounding error collected in the
// correction sum.  The weighted terms of one entry cancel heavily, so plain FP32
// sums would lose several digits (measured ~2e-6 normwise without TwoSum).
//
// CTAs walk contiguous chunks of the Morton-sorted rows, so rows that share
// elements run on the same SM and their element tables stay in L1.  Per row, a
// warp stages a window of up to 32 support entries in shared memory in three
// coalesced steps -- descriptors, the split products s^t of all their points
// (weights and coefficients are read once, lane-parallel), the position block --
// and then runs the element loop with only the (independent, pipelined) table
// loads left in global memory.
constexpr int F32_WIN_PTS = 64;     // points per staged window
constexpr int F32_WIN_POS = 512;    // positions per staged window
constexpr int F32_WARPS = 16;

template <int NT>
__global__ void __launch_bounds__(F32_WARPS * 32, 2) k_rowasm_f32(Rows rw, const int4* __restrict__ desc, TermsF tm,
                                                               int nc, const float2* __restrict__ table2,
                                                               const float2* __restrict__ W2, int nwc,
                                                               const float2* __restrict__ coef2,
                                                               float* __restrict__ vals, int max_n_i,
                                                               int64_t rows_per_cta) {
    extern __shared__ __align__(16) unsigned char sh_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // per-warp shared layout
    const size_t per_warp = 32 * sizeof(int4) + 2 * 33 * sizeof(int) + F32_WIN_PTS * NT * sizeof(float2) +
                            F32_WIN_POS * sizeof(uint16_t) + 2 * (size_t)max_n_i * sizeof(float);
    unsigned char* base = sh_raw + (size_t)wib * ((per_warp + 15) & ~(size_t)15);
    int4* sdesc = reinterpret_cast<int4*>(base);
    int* pbase = reinterpret_cast<int*>(sdesc + 32);      // [33] point offsets of the window's elements
    int* mbase = pbase + 33;                               // [33] position offsets
    float2* sval = reinterpret_cast<float2*>(mbase + 33);  // [F32_WIN_PTS][NT]
    uint16_t* spos = reinterpret_cast<uint16_t*>(sval + F32_WIN_PTS * NT);
    float* acc = reinterpret_cast<float*>(spos + F32_WIN_POS);
    const int64_t k0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t k1 = min(rw.n, k0 + rows_per_cta);
    for (int64_t k = k0 + wib; k < k1; k += F32_WARPS) {
        const int64_t i = rw.order ? rw.order[k] : k;
        const int r0 = rw.row_ptr[i], n_i = rw.row_ptr[i + 1] - r0;
        for (int x = lane; x < 2 * n_i; x += 32) acc[x] = 0.0f;
        int64_t woff = rw.w_ptr[i];
        int64_t sb = rw.supp_ptr[i];
        const int64_t s1 = rw.supp_ptr[i + 1];
        while (sb < s1) {
            // ---- window of support entries: descriptors, prefix sums
            const int nd = (int)min((int64_t)32, s1 - sb);
            const int4 dl = lane < nd ? desc[sb + lane] : make_int4(0, 0, 0, 0);
            const int Pl = (dl.z >> 8) & 255, ml = dl.z & 255;
            int sp = Pl, sm = ml;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int a = __shfl_up_sync(0xffffffffu, sp, off), b = __shfl_up_sync(0xffffffffu, sm, off);
                if (lane >= off) {
                    sp += a;
                    sm += b;
                }
            }
            const bool fits = lane < nd && ((sp <= F32_WIN_PTS && sm <= F32_WIN_POS) || lane == 0);
            const int nwin = __popc(__ballot_sync(0xffffffffu, fits));
            const int Wp = __shfl_sync(0xffffffffu, sp, nwin - 1), Wm = __shfl_sync(0xffffffffu, sm, nwin - 1);
            __syncwarp();
            if (lane < nwin) {
                sdesc[lane] = dl;
                pbase[lane + 1] = sp;
                mbase[lane + 1] = sm;
            }
            if (lane == 0) {
                pbase[0] = 0;
                mbase[0] = 0;
            }
            __syncwarp();
            // ---- split products of every point of the window
            for (int kq = lane; kq < Wp; kq += 32) {
                int j = 0;
                while (pbase[j + 1] <= kq) ++j;
                const int q = kq - pbase[j];
                const float2 c = coef2 ? coef2[sdesc[j].y + q] : make_float2(1.0f, 0.0f);
                const float2* wrow = W2 + (woff + kq) * nwc;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const float ahi = tm.use_coef[t] ? c.x : tm.shi[t];
                    const float alo = tm.use_coef[t] ? c.y : tm.slo[t];
                    const float2 w = wrow[tm.wc[t]];
                    float ph, pe;
                    two_prod(w.x, ahi, ph, pe);
                    sval[kq * NT + t] = make_float2(ph, pe + fmaf(w.x, alo, w.y * ahi));
                }
            }
            // ---- positions (contiguous over consecutive support entries of a row)
            const uint16_t* gpos = rw.pos + sdesc[0].w;
            for (int x = lane; x < Wm; x += 32) spos[x] = gpos[x];
            __syncwarp();
            // ---- element loop
            for (int j = 0; j < nwin; ++j) {
                const int4 d = sdesc[j];
                const int m = d.z & 255, P = (d.z >> 8) & 255;
                const float2* tb = table2 + d.x;
                const float2* sv = sval + pbase[j] * NT;
                const uint16_t* pos = spos + mbase[j];
                if (m <= 16) {
                    const int jl = lane & 15, hs = lane >> 4;
                    float hi = 0.0f, lo = 0.0f;
#pragma unroll 2
                    for (int qq = 0; qq < P; qq += 2) {
                        const int q = qq + hs;
                        if (q < P && jl < m) {
                            const float2* tq = tb + (int64_t)q * nc * m + jl;
#pragma unroll
                            for (int t = 0; t < NT; ++t) {
                                const float2 T = tq[tm.tc[t] * m];
                                const float2 a = sv[q * NT + t];
                                float ph, pe, s2, e2;
                                two_prod(a.x, T.x, ph, pe);
                                two_sum(hi, ph, s2, e2);
                                hi = s2;
                                lo += e2 + pe + fmaf(a.x, T.y, a.y * T.x);
                            }
                        }
                    }
                    const float ohi = __shfl_xor_sync(0xffffffffu, hi, 16);
                    const float olo = __shfl_xor_sync(0xffffffffu, lo, 16);
                    if (hs == 0 && jl < m) {
                        float s2, e2, s3, e3;
                        two_sum(hi, ohi, s2, e2);
                        const int p = pos[jl];
                        two_sum(acc[2 * p], s2, s3, e3);
                        acc[2 * p] = s3;
                        acc[2 * p + 1] += lo + olo + e2 + e3;
                    }
                } else {
                    for (int jl = lane; jl < m; jl += 32) {
                        float hi = 0.0f, lo = 0.0f;
                        const float2* tq = tb + jl;
#pragma unroll 2
                        for (int q = 0; q < P; ++q) {
#pragma unroll
                            for (int t = 0; t < NT; ++t) {
                                const float2 T = tq[((int64_t)q * nc + tm.tc[t]) * m];
                                const float2 a = sv[q * NT + t];
                                float ph, pe, s2, e2;
                                two_prod(a.x, T.x, ph, pe);
                                two_sum(hi, ph, s2, e2);
                                hi = s2;
                                lo += e2 + pe + fmaf(a.x, T.y, a.y * T.x);
                            }
                        }
                        float s3, e3;
                        const int p = pos[jl];
                        two_sum(acc[2 * p], hi, s3, e3);
                        acc[2 * p] = s3;
                        acc[2 * p + 1] += lo + e3;
                    }
                }
                __syncwarp();
            }
            woff += Wp;
            sb += nwin;
        }
        __syncwarp();
        for (int x = lane; x < n_i; x += 32) vals[r0 + x] = acc[2 * x] + acc[2 * x + 1];
        __syncwarp();
    }
}

__global__ void k_split_coef(const double* __restrict__ c, float2* __restrict__ c2, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = c[i];
        const float hi = __double2float_rn(v);
        c2[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

cudaError_t launch_rowasm_f32(const Rows& rw, const int4* desc, const Terms& tm, int nc, const float2* table2,
                              const float2* W2, int nwc, const double* coef, float2* coef2_buf, int64_t n_points,
                              float* vals, int max_n_i, int n_sm, cudaStream_t st) {
    if (rw.n == 0) return cudaSuccess;
    TermsF tf{};
    for (int t = 0; t < tm.nt; ++t) {
        tf.wc[t] = tm.t[t].wc;
        tf.tc[t] = tm.t[t].tc;
        tf.use_coef[t] = tm.t[t].use_coef;
        tf.shi[t] = (float)tm.t[t].scale;
        tf.slo[t] = (float)(tm.t[t].scale - (double)tf.shi[t]);
    }
    if (coef) {
        const int blocks = (int)std::min<int64_t>((n_points + 255) / 256, (int64_t)std::max(n_sm, 1) * 8);
        k_split_coef<<<std::max(blocks, 1), 256, 0, st>>>(coef, coef2_buf, n_points);
    }
    const int threads = F32_WARPS * 32;
    const int64_t n_cta = std::min<int64_t>((int64_t)std::max(n_sm, 1) * 2, (rw.n + F32_WARPS - 1) / F32_WARPS);
    const int64_t rpc = (rw.n + n_cta - 1) / n_cta;
    const size_t per_warp = 32 * sizeof(int4) + 2 * 33 * sizeof(int) + F32_WIN_PTS * std::max(tm.nt, 1) * sizeof(float2) +
                            F32_WIN_POS * sizeof(uint16_t) + 2 * (size_t)max_n_i * sizeof(float);
    const size_t smem = (size_t)F32_WARPS * ((per_warp + 15) & ~(size_t)15);
    const float2* c2 = coef ? coef2_buf : nullptr;
#define WQ_F32_CASE(N)                                                                                      \
    cudaFuncSetAttribute(k_rowasm_f32<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
    k_rowasm_f32<N><<<(unsigned)n_cta, threads, smem, st>>>(rw, desc, tf, nc, table2, W2, nwc, c2, vals, max_n_i, rpc)
    switch (tm.nt) {
        case 1: WQ_F32_CASE(1); break;
        case 2: WQ_F32_CASE(2); break;
        case 3: WQ_F32_CASE(3); break;
        default: WQ_F32_CASE(4); break;
    }
#undef WQ_F32_CASE
    return cudaGetLastError();
}

}  // namespace wqd
