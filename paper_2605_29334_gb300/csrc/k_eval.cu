// Placement of the quadrature points and evaluation of the spline functions
// with their physical derivatives (paper Sec. 4.1, Eqs. 13-17).
//
// One warp per point.  Lanes 0..15 each own one Bezier control point of the
// geometry net and the warp reduces x, x_u, x_v, x_uu, x_uv, x_vv by butterfly
// shuffles; then every lane evaluates the functions jl = lane, lane + 32, ...
// of the element:
//   a_alpha = dx/dxi^alpha, a^1 = (a_2 x n)/|n|^2, a^2 = (n x a_1)/|n|^2 with
//   n = a_1 x a_2 (the contravariant basis, |n|^2 = det a_ab), a^ab = a^a.a^b,
//   grad N = (a^1b N_,b) a_1 + (a^2b N_,b) a_2,
//   lap N  = a^ab (N_,ab - Gamma^g_ab N_,g),  Gamma^g_ab = a^g . x_,ab,
// and writes table[(point * nc + comp) * m + jl] (comp: N, d_x, d_y, [d_z], lap).
// WQ points sit at cell centres ((k+1/2)/s, (l+1/2)/s) of the element's
// parametric domain (split elements: sub-element (theta >= 1/2), xi = 2 theta - sub);
// Gauss points are the 4 x 4 Gauss-Legendre points of every (sub-)element.
#include <algorithm>

#include "kernels.h"

namespace wqd {

__constant__ double c_gauss_x[4];
__constant__ double c_gauss_w[4];

void set_gauss_constants(const double x[4], const double w[4]) {
    cudaMemcpyToSymbol(c_gauss_x, x, 4 * sizeof(double));
    cudaMemcpyToSymbol(c_gauss_w, w, 4 * sizeof(double));
}

__device__ __forceinline__ void bern3(double t, double* B, double* dB, double* ddB) {
    const double s = 1.0 - t;
    B[0] = s * s * s;
    B[1] = 3.0 * t * s * s;
    B[2] = 3.0 * t * t * s;
    B[3] = t * t * t;
    dB[0] = -3.0 * s * s;
    dB[1] = 3.0 * s * s - 6.0 * t * s;
    dB[2] = 6.0 * t * s - 3.0 * t * t;
    dB[3] = 3.0 * t * t;
    ddB[0] = 6.0 * s;
    ddB[1] = -12.0 + 18.0 * t;
    ddB[2] = 6.0 - 18.0 * t;
    ddB[3] = 6.0 * t;
}

__global__ void __launch_bounds__(256) k_eval(Elems el, const int32_t* __restrict__ pt_elem, int64_t npts,
                                              int gauss, double* __restrict__ table, double* __restrict__ xout,
                                              double* __restrict__ wout, unsigned* status) {
    const int lane = threadIdx.x & 31;
    const int64_t pt = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pt >= npts) return;
    const int e = pt_elem[pt];
    if (e < 0 || e >= el.E) {
        if (lane == 0) atomicOr(status, ST_BAD_INDEX);
        return;
    }
    const int64_t p0 = gauss ? el.gp_ptr[e] : el.pt_ptr[e];
    const int local = (int)(pt - p0);
    const int ns = el.nsub[e];
    int sub;
    double xu, xv, wq = 0.0;
    if (gauss) {
        sub = local >> 4;
        const int g = local & 15;
        xu = c_gauss_x[g & 3];
        xv = c_gauss_x[g >> 2];
        wq = c_gauss_w[g & 3] * c_gauss_w[g >> 2];
    } else {
        const int s = el.side[e];
        const int k = local % s, l = local / s;
        const double tu = (k + 0.5) / s, tv = (l + 0.5) / s;
        if (ns == 4) {
            const int su = tu >= 0.5, sv = tv >= 0.5;
            sub = su + 2 * sv;
            xu = 2.0 * tu - su;
            xv = 2.0 * tv - sv;
        } else {
            sub = 0;
            xu = tu;
            xv = tv;
        }
    }
    double Bu[4], dBu[4], ddBu[4], Bv[4], dBv[4], ddBv[4];
    bern3(xu, Bu, dBu, ddBu);
    bern3(xv, Bv, dBv, ddBv);

    // geometry derivatives by a warp reduction over the 16 control points
    double g[18];
    {
        const int i = (lane >> 2) & 3, j = lane & 3;
        const double* P = el.geom + 48 * (el.sub_ptr[e] + sub) + (i * 4 + j) * 3;
        const double on = lane < 16 ? 1.0 : 0.0;
        const double w[6] = {on * Bu[i] * Bv[j], on * dBu[i] * Bv[j], on * Bu[i] * dBv[j],
                             on * ddBu[i] * Bv[j], on * dBu[i] * dBv[j], on * Bu[i] * ddBv[j]};
        const double px = P[0], py = P[1], pz = P[2];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            g[3 * a + 0] = w[a] * px;
            g[3 * a + 1] = w[a] * py;
            g[3 * a + 2] = w[a] * pz;
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
            for (int a = 0; a < 18; ++a) g[a] += __shfl_xor_sync(0xffffffffu, g[a], off);
        // every lane uses lane 0's sums (butterfly orders differ in the last bit)
#pragma unroll
        for (int a = 0; a < 18; ++a) g[a] = __shfl_sync(0xffffffffu, g[a], 0);
    }
    const double *a1 = g + 3, *a2 = g + 6, *xuu = g + 9, *xuv = g + 12, *xvv = g + 15;
    // contravariant base vectors through the normal n = a1 x a2 (|n|^2 = det a_ab):
    // a^1 = (a2 x n)/|n|^2, a^2 = (n x a1)/|n|^2 -- no cancellation in a11 a22 - a12^2
    const double nx = a1[1] * a2[2] - a1[2] * a2[1];
    const double ny = a1[2] * a2[0] - a1[0] * a2[2];
    const double nz = a1[0] * a2[1] - a1[1] * a2[0];
    const double det = nx * nx + ny * ny + nz * nz;
    if (!(det > 0.0) || !isfinite(det)) {
        if (lane == 0) atomicOr(status, ST_GEOMETRY);
        return;
    }
    double A1[3], A2[3];
    A1[0] = (a2[1] * nz - a2[2] * ny) / det;
    A1[1] = (a2[2] * nx - a2[0] * nz) / det;
    A1[2] = (a2[0] * ny - a2[1] * nx) / det;
    A2[0] = (ny * a1[2] - nz * a1[1]) / det;
    A2[1] = (nz * a1[0] - nx * a1[2]) / det;
    A2[2] = (nx * a1[1] - ny * a1[0]) / det;
    const double i11 = A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2];
    const double i12 = A1[0] * A2[0] + A1[1] * A2[1] + A1[2] * A2[2];
    const double i22 = A2[0] * A2[0] + A2[1] * A2[1] + A2[2] * A2[2];
    const double G1uu = A1[0] * xuu[0] + A1[1] * xuu[1] + A1[2] * xuu[2];
    const double G1uv = A1[0] * xuv[0] + A1[1] * xuv[1] + A1[2] * xuv[2];
    const double G1vv = A1[0] * xvv[0] + A1[1] * xvv[1] + A1[2] * xvv[2];
    const double G2uu = A2[0] * xuu[0] + A2[1] * xuu[1] + A2[2] * xuu[2];
    const double G2uv = A2[0] * xuv[0] + A2[1] * xuv[1] + A2[2] * xuv[2];
    const double G2vv = A2[0] * xvv[0] + A2[1] * xvv[1] + A2[2] * xvv[2];

    const int m = el.m[e];
    const int nc = el.nc;
    const double* C = el.coef + el.coef_ptr[e];
    double* T = table + (gauss ? el.gbt_ptr[e] : el.bt_ptr[e]) + (int64_t)local * nc * m;
    for (int jl = lane; jl < m; jl += 32) {
        const double* c = C + ((int64_t)jl * ns + sub) * 16;
        double N = 0, Nu = 0, Nv = 0, Nuu = 0, Nuv = 0, Nvv = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            double r0 = 0, r1 = 0, r2 = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double cij = c[i * 4 + j];
                r0 += cij * Bv[j];
                r1 += cij * dBv[j];
                r2 += cij * ddBv[j];
            }
            N += Bu[i] * r0;
            Nu += dBu[i] * r0;
            Nv += Bu[i] * r1;
            Nuu += ddBu[i] * r0;
            Nuv += dBu[i] * r1;
            Nvv += Bu[i] * r2;
        }
        const double luu = Nuu - G1uu * Nu - G2uu * Nv;
        const double luv = Nuv - G1uv * Nu - G2uv * Nv;
        const double lvv = Nvv - G1vv * Nu - G2vv * Nv;
        const double lap = i11 * luu + 2.0 * i12 * luv + i22 * lvv;
        T[jl] = N;
        T[m + jl] = Nu * A1[0] + Nv * A2[0];
        T[2 * m + jl] = Nu * A1[1] + Nv * A2[1];
        if (nc == 5) T[3 * m + jl] = Nu * A1[2] + Nv * A2[2];
        T[(nc - 1) * m + jl] = lap;
    }
    if (lane == 0) {
        const double* ref = el.geom_ref + 3 * (int64_t)e;
        xout[pt * 3 + 0] = ref[0] + g[0];
        xout[pt * 3 + 1] = ref[1] + g[1];
        xout[pt * 3 + 2] = ref[2] + g[2];
        if (gauss) wout[pt] = wq * sqrt(det);
    }
}

cudaError_t launch_eval(const Elems& el, const int32_t* pt_elem, int64_t npts, int gauss, double* table,
                        double* xout, double* wout, unsigned* status, cudaStream_t st) {
    if (npts == 0) return cudaSuccess;
    const int threads = 256, wpb = threads / 32;
    const int64_t blocks = (npts + wpb - 1) / wpb;
    k_eval<<<(unsigned)blocks, threads, 0, st>>>(el, pt_elem, npts, gauss, table, xout, wout, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- interp
// One thread per point: u_q = sum_j N_j(x_q) u_j and its gradient, summed over the
// m_e functions of the point's element in local order (no cross-lane reductions:
// FP64 adds are scarce on this GPU).
__global__ void __launch_bounds__(256) k_interp(Elems el, const int32_t* __restrict__ pt_elem,
                                                const int32_t* __restrict__ fns, const int64_t* __restrict__ fn_ptr,
                                                int64_t Q, const double* __restrict__ table,
                                                const double* __restrict__ u, double* __restrict__ uq,
                                                double* __restrict__ grad) {
    const int64_t pt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pt >= Q) return;
    const int e = pt_elem[pt];
    const int m = el.m[e], nc = el.nc;
    const double* T = table + el.bt_ptr[e] + (pt - el.pt_ptr[e]) * nc * m;
    const int32_t* f = fns + fn_ptr[e];
    double v = 0, gx = 0, gy = 0, gz = 0;
    for (int jl = 0; jl < m; ++jl) {
        const double uj = u[f[jl]];
        v = fma(uj, T[jl], v);
        gx = fma(uj, T[m + jl], gx);
        gy = fma(uj, T[2 * m + jl], gy);
        if (nc == 5) gz = fma(uj, T[3 * m + jl], gz);
    }
    uq[pt] = v;
    if (grad) {
        grad[pt * 3 + 0] = gx;
        grad[pt * 3 + 1] = gy;
        grad[pt * 3 + 2] = gz;
    }
}

cudaError_t launch_interp(const Elems& el, const int32_t* pt_elem, const int32_t* fns, const int64_t* fn_ptr,
                          int64_t Q, const double* table, const double* u, double* uq, double* grad,
                          cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    k_interp<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(el, pt_elem, fns, fn_ptr, Q, table, u, uq, grad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- hi/lo split
__global__ void k_split_f32(const double* __restrict__ src, float2* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[i];
        const float hi = __double2float_rn(v);
        const float lo = __double2float_rn(v - (double)hi);
        dst[i] = make_float2(hi, lo);
    }
}

cudaError_t launch_split_f32(const double* src, float2* dst, int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_split_f32<<<blocks, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace wqd

namespace wqd {

// ---------------------------------------------------------------- heat fields
// Point data of the nonlinear heat problem (paper Sec. 5, theta = 1):
//   u_q = sum_j N_j(x_q) u_j, grad u_q likewise, uo_q from u_old;
//   kappa_q = k0 + k2 u_q^2 (coefficient of the tangent S, Eq. S),
//   g[0][q] = (u_q - uo_q) / dt - f,   g[1 + d][q] = kappa_q d_d u_q,
//   and (jacobian) kappa[1 + d][q] = k'(u_q) d_d u_q for the exact tangent
// (the residual R_A = Q_A((u - u_old)/dt - f) + sum_d Q^d_A(kappa d_d u)).
__global__ void __launch_bounds__(256) k_heat_fields(Elems el, const int32_t* __restrict__ pt_elem,
                                                     const int32_t* __restrict__ fns,
                                                     const int64_t* __restrict__ fn_ptr, int64_t Q,
                                                     const double* __restrict__ table, const double* __restrict__ u,
                                                     const double* __restrict__ uo, double dt, double k0, double k2,
                                                     double f, bool jacobian, double* __restrict__ kappa,
                                                     double* __restrict__ g) {
    const int64_t pt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pt >= Q) return;
    const int e = pt_elem[pt];
    const int m = el.m[e], nc = el.nc;
    const double* T = table + el.bt_ptr[e] + (pt - el.pt_ptr[e]) * nc * m;
    const int32_t* fl = fns + fn_ptr[e];
    double v = 0, vo = 0, gx = 0, gy = 0, gz = 0;
    for (int jl = 0; jl < m; ++jl) {
        const int j = fl[jl];
        const double uj = u[j], nj = T[jl];
        v = fma(uj, nj, v);
        vo = fma(uo[j], nj, vo);
        gx = fma(uj, T[m + jl], gx);
        gy = fma(uj, T[2 * m + jl], gy);
        if (nc == 5) gz = fma(uj, T[3 * m + jl], gz);
    }
    const double k = k0 + k2 * v * v;
    kappa[pt] = k;
    if (jacobian) {   // k'(u) d_d u, the coefficient rows of the exact tangent
        const double dk = 2.0 * k2 * v;
        kappa[Q + pt] = dk * gx;
        kappa[2 * Q + pt] = dk * gy;
        if (nc == 5) kappa[3 * Q + pt] = dk * gz;
    }
    g[pt] = (v - vo) / dt - f;
    g[Q + pt] = k * gx;
    g[2 * Q + pt] = k * gy;
    if (nc == 5) g[3 * Q + pt] = k * gz;
}

cudaError_t launch_heat_fields(const Elems& el, const int32_t* pt_elem, const int32_t* fns, const int64_t* fn_ptr,
                               int64_t Q, const double* table, const double* u, const double* uo, double dt, double k0,
                               double k2, double f, bool jacobian, double* kappa, double* g, cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    k_heat_fields<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(el, pt_elem, fns, fn_ptr, Q, table, u, uo, dt, k0, k2,
                                                              f, jacobian, kappa, g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- WQ apply
// Matrix-free WQ functional: y_i = sum_t sum_{q in pts(supp N_i)} w^{c_t}_iq g_t(x_q).
// One warp per row; the row's weight rows [w_ptr[i], w_ptr[i+1]) are contiguous, so
// lanes stride over them (coalesced), each with its point index pt_of_w[x]; one warp
// reduction per row.
__global__ void __launch_bounds__(256) k_apply(Rows rw, const int32_t* __restrict__ pt_of_w, int nt, int4 wc4,
                                               const double* __restrict__ W, int nwc, const double* __restrict__ g,
                                               int64_t Q, double* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= rw.n) return;
    const int wc[4] = {wc4.x, wc4.y, wc4.z, wc4.w};
    double acc = 0.0;
    for (int64_t x = rw.w_ptr[i] + lane; x < rw.w_ptr[i + 1]; x += 32) {
        const double* wrow = W + x * nwc;
        const int64_t q = pt_of_w[x];
        for (int t = 0; t < nt; ++t) acc = fma(wrow[wc[t]], g[t * Q + q], acc);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) y[i] = acc;
}

cudaError_t launch_apply(const Rows& rw, const int32_t* pt_of_w, int nt, int4 wc4, const double* W, int nwc,
                         const double* g, int64_t Q, double* y, cudaStream_t st) {
    if (rw.n == 0) return cudaSuccess;
    const int threads = 256, wpb = threads / 32;
    k_apply<<<(unsigned)((rw.n + wpb - 1) / wpb), threads, 0, st>>>(rw, pt_of_w, nt, wc4, W, nwc, g, Q, y);
    return cudaGetLastError();
}

}  // namespace wqd
