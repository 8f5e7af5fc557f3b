// Placement of the quadrature points and evaluation of the spline functions
// with their physical derivatives (paper Sec. 4.1, Eqs. 13-17).
//
// One warp per point.  Lanes 0..15 each own one Bezier control point of the
// geometry net and the warp reduces x, x_u, x_v, x_uu, x_uv, x_vv by butterfly
// shuffles; then every lane evaluates the functions jl = lane, lane + 32, ...
// of the element:
//   a_alpha = dx/dxi^alpha, a_ab = a_a.a_b, a^ab = inverse,
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
    const double g11 = a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2];
    const double g12 = a1[0] * a2[0] + a1[1] * a2[1] + a1[2] * a2[2];
    const double g22 = a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2];
    const double det = g11 * g22 - g12 * g12;
    if (!(det > 0.0) || !isfinite(det)) {
        if (lane == 0) atomicOr(status, ST_GEOMETRY);
        return;
    }
    const double i11 = g22 / det, i12 = -g12 / det, i22 = g11 / det;
    double A1[3], A2[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        A1[d] = i11 * a1[d] + i12 * a2[d];
        A2[d] = i12 * a1[d] + i22 * a2[d];
    }
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
        xout[pt * 3 + 0] = g[0];
        xout[pt * 3 + 1] = g[1];
        xout[pt * 3 + 2] = g[2];
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
__global__ void __launch_bounds__(256) k_interp(Elems el, const int32_t* __restrict__ pt_elem,
                                                const int32_t* __restrict__ fns, const int64_t* __restrict__ fn_ptr,
                                                int64_t Q, const double* __restrict__ table,
                                                const double* __restrict__ u, double* __restrict__ uq,
                                                double* __restrict__ grad) {
    const int lane = threadIdx.x & 31;
    const int64_t pt = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pt >= Q) return;
    const int e = pt_elem[pt];
    const int m = el.m[e], nc = el.nc;
    const double* T = table + el.bt_ptr[e] + (pt - el.pt_ptr[e]) * nc * m;
    double v = 0, gx = 0, gy = 0, gz = 0;
    for (int jl = lane; jl < m; jl += 32) {
        const double uj = u[fns[fn_ptr[e] + jl]];
        v += uj * T[jl];
        gx += uj * T[m + jl];
        gy += uj * T[2 * m + jl];
        if (nc == 5) gz += uj * T[3 * m + jl];
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, off);
        gx += __shfl_xor_sync(0xffffffffu, gx, off);
        gy += __shfl_xor_sync(0xffffffffu, gy, off);
        gz += __shfl_xor_sync(0xffffffffu, gz, off);
    }
    if (lane == 0) {
        uq[pt] = v;
        if (grad) {
            grad[pt * 3 + 0] = gx;
            grad[pt * 3 + 1] = gy;
            grad[pt * 3 + 2] = gz;
        }
    }
}

cudaError_t launch_interp(const Elems& el, const int32_t* pt_elem, const int32_t* fns, const int64_t* fn_ptr,
                          int64_t Q, const double* table, const double* u, double* uq, double* grad,
                          cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    const int threads = 256, wpb = threads / 32;
    k_interp<<<(unsigned)((Q + wpb - 1) / wpb), threads, 0, st>>>(el, pt_elem, fns, fn_ptr, Q, table, u, uq, grad);
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
