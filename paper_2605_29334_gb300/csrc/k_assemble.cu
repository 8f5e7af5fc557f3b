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

// ------------------------------------------------------------ FP32 staged
// One CTA per chunk of Morton-consecutive rows.  Phase A stages everything the
// chunk needs into shared memory with many loads in flight: the tables of the
// union of the rows' support elements (cp.async, only the components of the
// operator's terms, laid out [point][term][function]), the split products s of
// every (row, point), the position blocks and the union-local element indices.
// Phase B runs the same arithmetic as k_rowasm_f32 from shared memory only.
// Used for operators with at most two terms.
constexpr int CH_WARPS = 16;

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

template <int NT, bool COMP>
__global__ void __launch_bounds__(CH_WARPS * 32, 2) k_chunk_f32(Chunks ch, Rows rw, const int4* __restrict__ desc,
                                                              TermsF tm, int nc, const float2* __restrict__ table2,
                                                              const float2* __restrict__ W2, int nwc,
                                                              const float2* __restrict__ coef2,
                                                              float* __restrict__ vals, int max_n_i) {
    extern __shared__ __align__(16) unsigned char sh_ch[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int c = blockIdx.x;
    const int4 info = ch.info[c];
    const int u0 = ch.u_ptr[c], nu = ch.u_ptr[c + 1] - u0;
    int4* sunion = reinterpret_cast<int4*>(sh_ch);
    float2* stab = reinterpret_cast<float2*>(sunion + nu);
    float2* sval = stab + info.x;
    uint16_t* sloc = reinterpret_cast<uint16_t*>(sval + info.y);
    uint16_t* spos = sloc + info.z;
    float* acc = reinterpret_cast<float*>(sh_ch + ch.data_bytes) + (int64_t)wib * 2 * max_n_i;
    const int k0 = ch.row_ptr[c], k1 = ch.row_ptr[c + 1];
    const int tc0 = tm.tc[0], tc1 = NT > 1 ? tm.tc[1] : 0;

    // ---- phase A1: union info and element tables ([point][term][function])
    for (int x = threadIdx.x; x < nu; x += blockDim.x) sunion[x] = ch.u[u0 + x];
    for (int u = wib; u < nu; u += CH_WARPS) {
        const int4 ud = ch.u[u0 + u];
        const int m = ud.y & 255, P = (ud.y >> 8) & 255;
        const float2* src = table2 + ud.x;
        float2* dst = stab + ud.z;
        const int R = P * NT;
        if (m <= 16) {
            const int jl = lane & 15;
            if (jl < m)
                for (int r = lane >> 4; r < R; r += 2) {
                    const int q = NT == 1 ? r : (r >> 1), t = NT == 1 ? 0 : (r & 1);
                    cp_async8(dst + r * m + jl, src + ((int64_t)q * nc + (t ? tc1 : tc0)) * m + jl);
                }
        } else {
            for (int r = 0; r < R; ++r) {
                const int q = NT == 1 ? r : (r >> 1), t = NT == 1 ? 0 : (r & 1);
                for (int jl = lane; jl < m; jl += 32)
                    cp_async8(dst + r * m + jl, src + ((int64_t)q * nc + (t ? tc1 : tc0)) * m + jl);
            }
        }
    }
    // ---- phase A2: per row: local indices, positions, split products of its points
    for (int k = k0 + wib; k < k1; k += CH_WARPS) {
        const int4 ri = ch.rows[k];
        const int i = ri.x;
        const int64_t s0 = rw.supp_ptr[i], s1 = rw.supp_ptr[i + 1];
        const int ns = (int)(s1 - s0);
        for (int x = lane; x < ns; x += 32) sloc[ri.w + x] = ch.sloc[s0 + x];
        const int4 dfirst = desc[s0];
        const int4 dlast = desc[s1 - 1];
        const int npos = dlast.w + (dlast.z & 255) - dfirst.w;
        const uint16_t* gpos = rw.pos + dfirst.w;
        for (int x = lane; x < npos; x += 32) spos[ri.z + x] = gpos[x];
        const float2* wrow0 = W2 + rw.w_ptr[i] * nwc;
        float2* svr = sval + ri.y;
        int pb = 0;
        for (int64_t sb = s0; sb < s1; sb += 32) {
            const int nd = (int)min((int64_t)32, s1 - sb);
            const int4 dl = lane < nd ? desc[sb + lane] : make_int4(0, 0, 0, 0);
            for (int jj = 0; jj < nd; ++jj) {
                const int pz = __shfl_sync(0xffffffffu, dl.z, jj), pty = __shfl_sync(0xffffffffu, dl.y, jj);
                const int P = (pz >> 8) & 255;
                for (int q = lane; q < P; q += 32) {
                    const float2 cc = coef2 ? coef2[pty + q] : make_float2(1.0f, 0.0f);
                    const float2* wrow = wrow0 + (int64_t)(pb + q) * nwc;
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const float ahi = tm.use_coef[t] ? cc.x : tm.shi[t];
                        const float alo = tm.use_coef[t] ? cc.y : tm.slo[t];
                        const float2 w = wrow[tm.wc[t]];
                        float ph, pe;
                        two_prod(w.x, ahi, ph, pe);
                        svr[(pb + q) * NT + t] = make_float2(ph, pe + fmaf(w.x, alo, w.y * ahi));
                    }
                }
                pb += P;
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // ---- phase B: rows from shared memory
    for (int k = k0 + wib; k < k1; k += CH_WARPS) {
        const int4 ri = ch.rows[k];
        const int i = ri.x;
        const int r0 = rw.row_ptr[i], n_i = rw.row_ptr[i + 1] - r0;
        const int ns = (int)(rw.supp_ptr[i + 1] - rw.supp_ptr[i]);
        for (int x = lane; x < 2 * n_i; x += 32) acc[x] = 0.0f;
        __syncwarp();
        const float2* sv = sval + ri.y;
        const uint16_t* pos = spos + ri.z;
        const uint16_t* loc = sloc + ri.w;
        for (int x = 0; x < ns; ++x) {
            const int4 ud = sunion[loc[x]];
            const int m = ud.y & 255, P = (ud.y >> 8) & 255;
            const float2* tb = stab + ud.z;
            if (m <= 16) {
                const int jl = lane & 15, hs = lane >> 4;
                float hi = 0.0f, lo = 0.0f;
                const bool jok = jl < m;
                const float2* tq = tb + hs * NT * m + jl;
                const float2* aq = sv + hs * NT;
                for (int q = hs; q < P; q += 2, tq += 2 * NT * m, aq += 2 * NT) {
                    if (jok) {
#pragma unroll
                        for (int t = 0; t < NT; ++t) {
                            const float2 T = tq[t * m];
                            const float2 a = aq[t];
                            if (COMP) {
                                float ph, pe, s2, e2;
                                two_prod(a.x, T.x, ph, pe);
                                two_sum(hi, ph, s2, e2);
                                hi = s2;
                                lo += e2 + pe + fmaf(a.x, T.y, a.y * T.x);
                            } else {
                                hi = fmaf(a.x, T.x, hi);
                                lo = fmaf(a.x, T.y, lo);
                                lo = fmaf(a.y, T.x, lo);
                            }
                        }
                    }
                }
                const float ohi = __shfl_xor_sync(0xffffffffu, hi, 16);
                const float olo = __shfl_xor_sync(0xffffffffu, lo, 16);
                if (hs == 0 && jok) {
                    const int p = pos[jl];
                    if (COMP) {
                        float s2, e2, s3, e3;
                        two_sum(hi, ohi, s2, e2);
                        two_sum(acc[2 * p], s2, s3, e3);
                        acc[2 * p] = s3;
                        acc[2 * p + 1] += lo + olo + e2 + e3;
                    } else {
                        acc[2 * p] += hi + ohi;
                        acc[2 * p + 1] += lo + olo;
                    }
                }
            } else {
                for (int jl = lane; jl < m; jl += 32) {
                    float hi = 0.0f, lo = 0.0f;
                    const float2* tq = tb + jl;
                    for (int q = 0; q < P; ++q, tq += NT * m) {
#pragma unroll
                        for (int t = 0; t < NT; ++t) {
                            const float2 T = tq[t * m];
                            const float2 a = sv[q * NT + t];
                            if (COMP) {
                                float ph, pe, s2, e2;
                                two_prod(a.x, T.x, ph, pe);
                                two_sum(hi, ph, s2, e2);
                                hi = s2;
                                lo += e2 + pe + fmaf(a.x, T.y, a.y * T.x);
                            } else {
                                hi = fmaf(a.x, T.x, hi);
                                lo = fmaf(a.x, T.y, lo);
                                lo = fmaf(a.y, T.x, lo);
                            }
                        }
                    }
                    const int p = pos[jl];
                    if (COMP) {
                        float s3, e3;
                        two_sum(acc[2 * p], hi, s3, e3);
                        acc[2 * p] = s3;
                        acc[2 * p + 1] += lo + e3;
                    } else {
                        acc[2 * p] += hi;
                        acc[2 * p + 1] += lo;
                    }
                }
            }
            sv += P * NT;
            pos += m;
            __syncwarp();
        }
        for (int x = lane; x < n_i; x += 32) vals[r0 + x] = acc[2 * x] + acc[2 * x + 1];
        __syncwarp();
    }
}

// ------------------------------------------------------- FP32 element-major
// Phase 1: the dense block of every element's test x trial pairs
//     K_e[a][b] = sum_{q, t} s^t_{a q} T^t_{q b},   s^t_{a q} = w^{c_t}_{i_a q} a_t(x_q),
// (a, b over the m_e functions of e, q over its points) with split products and
// TwoSum accumulation.  One warp computes one 16 x 16 tile of one block (a
// regular element, m_e = 16, is one tile; larger elements are several, listed
// first so that their longer point loops start in the first wave).  Points are
// taken EL_QC at a time: the tile's table columns are copied to shared memory
// with cp.async, the weights of its 16 rows are loaded into registers all at
// once, multiplied by the split coefficient and stored to shared memory; then a
// lane accumulates column b over 8 rows (two half-warps), reading its table
// value once per (point, term) and the row values as broadcasts.  Each entry is
// stored at its slot in kscr, where the contributions to one CSR entry are
// contiguous and in the order of the elements in supp N_i.
// Phase 2, one thread per CSR entry: the compensated sum of its slots.  No
// atomics: the result is bitwise reproducible.
constexpr int EL_QC = 8;        // points per staged chunk
constexpr int EL_NWARP = 8;     // warps per block

template <int NT, bool COMP>
__global__ void __launch_bounds__(EL_NWARP * 32)
    k_elem_f32(ElemPlan ep, TermsF tm, int nc, const float2* __restrict__ table2, const float2* __restrict__ W2,
               int nwc, const double* __restrict__ coef) {
    constexpr int IT = 16 * EL_QC / 32;             // staged (row, point) items per lane and term
    __shared__ __align__(16) float2 sT[EL_NWARP][EL_QC * NT * 16];
    __shared__ __align__(16) float2 sS[EL_NWARP][EL_QC * NT * 16];
    __shared__ float2 sC[EL_NWARP][EL_QC];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * EL_NWARP + wib;
    if (k >= ep.n_items) return;
    const int4 d = ep.item[k];
    const int kb = ep.item_k[k];
    const int m = d.z & 255, P = (d.z >> 8) & 255, a0 = ((d.z >> 16) & 15) * 16, b0 = ((d.z >> 20) & 15) * 16;
    const float2* tb = table2 + d.x;
    float2* T_ = sT[wib];
    float2* S_ = sS[wib];
    const int bl = lane & 15, rbase = 8 * (lane >> 4);
    const int b = b0 + bl;
    // destination slots of this lane's entries (independent of the arithmetic: loaded first)
    int slot[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int a = a0 + rbase + r;
        slot[r] = (a < m && b < m) ? ep.scat[kb + a * m + b] : 0;
    }
    const int ewv = (lane < 16 && a0 + lane < m) ? ep.ew_off[d.w + a0 + lane] : 0;
    float hi[8], lo[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) hi[r] = lo[r] = 0.0f;
    for (int q0 = 0; q0 < P; q0 += EL_QC) {
        const int nq = min(EL_QC, P - q0);
        __syncwarp();
        // the tile's table columns at the chunk's points, [point][term][column]
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int tc = tm.tc[t];
            for (int x = lane; x < nq * 16; x += 32) {
                const int qq = x >> 4, c = x & 15;
                if (b0 + c < m)
                    cp_async8(T_ + (qq * NT + t) * 16 + c, tb + ((int64_t)(q0 + qq) * nc + tc) * m + b0 + c);
            }
        }
        if (lane < nq) {
            const double c = coef ? coef[d.y + q0 + lane] : 1.0;
            const float chi = (float)c;
            sC[wib][lane] = make_float2(chi, (float)(c - (double)chi));
        }
        // weights of the tile's rows at the chunk's points, all loads in flight together
        float2 wv[NT][IT];
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const int x = lane + 32 * j, qq = x % EL_QC, ar = x / EL_QC;
            const int ea = __shfl_sync(0xffffffffu, ewv, ar);
            const bool ok = qq < nq && a0 + ar < m;
            const float2* wrow = W2 + ((int64_t)ea + q0 + qq) * nwc;
#pragma unroll
            for (int t = 0; t < NT; ++t) wv[t][j] = ok ? wrow[tm.wc[t]] : make_float2(0.0f, 0.0f);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const int x = lane + 32 * j, qq = x % EL_QC, ar = x / EL_QC;
            const float2 c = sC[wib][qq];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const float ahi = tm.use_coef[t] ? c.x : tm.shi[t];
                const float alo = tm.use_coef[t] ? c.y : tm.slo[t];
                const float2 w = wv[t][j];
                float ph, pe;
                two_prod(w.x, ahi, ph, pe);
                S_[(qq * NT + t) * 16 + ar] = make_float2(ph, pe + fmaf(w.x, alo, w.y * ahi));
            }
        }
        cp_async_wait_all();
        __syncwarp();
        if (b < m) {
            for (int qq = 0; qq < nq; ++qq) {
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const float2 T = T_[(qq * NT + t) * 16 + bl];
                    const float4* srow = reinterpret_cast<const float4*>(S_ + (qq * NT + t) * 16 + rbase);
#pragma unroll
                    for (int r2 = 0; r2 < 4; ++r2) {
                        const float4 sv = srow[r2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float sx = h ? sv.z : sv.x, sy = h ? sv.w : sv.y;
                            const int r = 2 * r2 + h;
                            if (COMP) {
                                float ph, pe, s2, e2;
                                two_prod(sx, T.x, ph, pe);
                                two_sum(hi[r], ph, s2, e2);
                                hi[r] = s2;
                                lo[r] += e2;
                                lo[r] += pe;
                                lo[r] = fmaf(sx, T.y, lo[r]);
                                lo[r] = fmaf(sy, T.x, lo[r]);
                            } else {
                                hi[r] = fmaf(sx, T.x, hi[r]);
                                lo[r] = fmaf(sx, T.y, lo[r]);
                                lo[r] = fmaf(sy, T.x, lo[r]);
                            }
                        }
                    }
                }
            }
        }
    }
    if (b < m) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (a0 + rbase + r < m) ep.kscr[slot[r]] = make_float2(hi[r], lo[r]);
    }
}

template <bool COMP>
__global__ void __launch_bounds__(256) k_gather_f32(int64_t nnz, const int32_t* __restrict__ gptr,
                                                    const float2* __restrict__ kscr, float* __restrict__ vals) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nnz) return;
    const int c0 = gptr[n], c1 = gptr[n + 1];
    float hi = 0.0f, lo = 0.0f;
    for (int cb = c0; cb < c1; cb += 8) {
        float2 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = cb + j < c1 ? kscr[cb + j] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (COMP) {
                float s3, e3;
                two_sum(hi, v[j].x, s3, e3);
                hi = s3;
                lo += v[j].y + e3;
            } else {
                hi += v[j].x;
                lo += v[j].y;
            }
        }
    }
    vals[n] = hi + lo;
}

cudaError_t launch_elem_f32(const ElemPlan& ep, int64_t nnz, const Terms& tm, int nc, const float2* table2,
                            const float2* W2, int nwc, const double* coef, float* vals, bool compensated,
                            cudaStream_t st) {
    if (nnz == 0) return cudaSuccess;
    TermsF tf{};
    for (int t = 0; t < tm.nt; ++t) {
        tf.wc[t] = tm.t[t].wc;
        tf.tc[t] = tm.t[t].tc;
        tf.use_coef[t] = tm.t[t].use_coef;
        tf.shi[t] = (float)tm.t[t].scale;
        tf.slo[t] = (float)(tm.t[t].scale - (double)tf.shi[t]);
    }
    const unsigned eb = (unsigned)((ep.n_items + EL_NWARP - 1) / EL_NWARP);
#define WQ_EL_CASE(N, C) k_elem_f32<N, C><<<eb, EL_NWARP * 32, 0, st>>>(ep, tf, nc, table2, W2, nwc, coef)
    if (ep.n_items > 0) {
        switch (tm.nt * 2 + (compensated ? 1 : 0)) {
            case 2: WQ_EL_CASE(1, false); break;
            case 3: WQ_EL_CASE(1, true); break;
            case 4: WQ_EL_CASE(2, false); break;
            case 5: WQ_EL_CASE(2, true); break;
            case 6: WQ_EL_CASE(3, false); break;
            case 7: WQ_EL_CASE(3, true); break;
            case 8: WQ_EL_CASE(4, false); break;
            default: WQ_EL_CASE(4, true); break;
        }
    }
#undef WQ_EL_CASE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned gb = (unsigned)((nnz + 255) / 256);
    if (compensated)
        k_gather_f32<true><<<gb, 256, 0, st>>>(nnz, ep.gptr, ep.kscr, vals);
    else
        k_gather_f32<false><<<gb, 256, 0, st>>>(nnz, ep.gptr, ep.kscr, vals);
    return cudaGetLastError();
}

cudaError_t launch_rowasm_f32(const Rows& rw, const int4* desc, const Chunks* ch, const Terms& tm, int nc,
                              const float2* table2, const float2* W2, int nwc, const double* coef, float2* coef2_buf,
                              int64_t n_points, float* vals, int max_n_i, int n_sm, bool compensated,
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
    if (coef) {
        const int blocks = (int)std::min<int64_t>((n_points + 255) / 256, (int64_t)std::max(n_sm, 1) * 8);
        k_split_coef<<<std::max(blocks, 1), 256, 0, st>>>(coef, coef2_buf, n_points);
    }
    const float2* c2 = coef ? coef2_buf : nullptr;
    if (ch && ch->n_chunks > 0 && tm.nt <= 2) {
        const size_t smem = (size_t)ch->data_bytes + (size_t)CH_WARPS * 2 * max_n_i * sizeof(float);
#define WQ_CH_CASE(N, C)                                                                                     \
    cudaFuncSetAttribute(k_chunk_f32<N, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
    k_chunk_f32<N, C><<<(unsigned)ch->n_chunks, CH_WARPS * 32, smem, st>>>(*ch, rw, desc, tf, nc, table2, W2, nwc, \
                                                                          c2, vals, max_n_i)
        if (tm.nt == 1) {
            if (compensated) { WQ_CH_CASE(1, true); } else { WQ_CH_CASE(1, false); }
        } else {
            if (compensated) { WQ_CH_CASE(2, true); } else { WQ_CH_CASE(2, false); }
        }
#undef WQ_CH_CASE
        return cudaGetLastError();
    }
    if (!compensated) return cudaErrorNotSupported;   // the fast mode exists for <= 2 terms only
    const int threads = F32_WARPS * 32;
    const int64_t n_cta = std::min<int64_t>((int64_t)std::max(n_sm, 1) * 2, (rw.n + F32_WARPS - 1) / F32_WARPS);
    const int64_t rpc = (rw.n + n_cta - 1) / n_cta;
    const size_t per_warp = 32 * sizeof(int4) + 2 * 33 * sizeof(int) + F32_WIN_PTS * std::max(tm.nt, 1) * sizeof(float2) +
                            F32_WIN_POS * sizeof(uint16_t) + 2 * (size_t)max_n_i * sizeof(float);
    const size_t smem = (size_t)F32_WARPS * ((per_warp + 15) & ~(size_t)15);
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
