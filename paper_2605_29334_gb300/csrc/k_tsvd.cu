// Truncated-SVD weights of every test function (paper Sec. 4.3):
//     A = [D_c N_j(x_q)]  (j in S_i, q in the points of supp N_i),  A = U S V^T,
//     keep s_k >= tol * s_max,
//     w = Z^2 V_t (V_t^T Z^2 V_t)^{-1} S_t^{-1} U_t^T b,   Z = diag(N_i(x_q)).
//
// One CTA per system (persistent grid over rows), FP64, matrices in a per-CTA
// global scratch slice:
//  1. gather A row-major by function (At[a][q]) and z from the point tables;
//  2. Householder QR with column pivoting of A^T (r_i x n_i): A^T P = Q R;
//  3. one-sided (Hestenes) Jacobi on the n_i rows of R (length n_i), round-robin
//     pairs, four lanes per pair, accumulating the rotations in Jt (J^T R = S Y^T,
//     so A = (P Y) S (Q J)^T): FP32 sweeps on a float copy first, then FP64 sweeps
//     from the re-orthogonalised FP32 rotations;  a sweep cap ends it with a status flag;
//  4. s_k = |row k of the rotated R|, keep s_k >= tol s_max;  g = S_t^{-1} U_t^T b;
//  5. G = Z V_t (columns z * Q j_k), Householder QR G = Q' R', then
//     w = Z Q' R'^{-T} g  -- the inverse of G^T G = V_t^T Z^2 V_t applied through
//     the QR factor, as the paper does for the full-rank case (Sec. 2, Eq. QR).
//  The pivoted QR is Drmac and Veselic's preconditioning of one-sided Jacobi (SIAM J.
//  Matrix Anal. Appl. 29, 2008): the same SVD, in about half the sweeps.
//  If N_i vanishes at one of its points (z_q == 0, V_t^T Z^2 V_t singular) the
//  row uses Z = I and is flagged.  rank_out / zid_out may be null.
#include "kernels.h"

namespace wqd {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return __shfl_sync(0xffffffffu, v, 0);
}

// One-sided Jacobi on the n rows (length n) of A, rotations accumulated in the rows of J,
// by the whole CTA: groups of JG lanes per rotation pair (8 pairs per warp), round-robin
// pairs, at most max_sweeps sweeps; returns whether a sweep found nothing to rotate.
// FP64: zeta = (be - al) / (2 ga) in FP64, the tangent from it in FP32 (hypotf; t =
// 1/(2 zeta) beyond 1e30), cos/sin in FP64 from that tangent (c = (1 + t^2)^-1/2 by two
// Newton steps from an FP32 seed, s = c t): every applied rotation is orthogonal to FP64
// rounding, the FP32 angle only costs convergence speed.  FP32: all in FP32.
template <typename T>
__device__ __forceinline__ bool jacobi_rows(T* __restrict__ A, T* __restrict__ J, int n, int max_sweeps, int& nchk,
                                            int& nrot) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    constexpr bool F64 = sizeof(T) == 8;
    const int np = (n + 1) & ~1;
    const T tolJ = F64 ? (T)fmax(2.220446049250313e-16 * sqrt((double)n), 1e-15)
                       : (T)fmaxf(1.1920929e-7f * sqrtf((float)n), 1e-7f);
    const T tol2 = tolJ * tolJ;
    constexpr int JG = 4;
    const int gl = lane & (JG - 1), grp = lane / JG;
    const int per_pass = nwarp * (32 / JG);
    const int npairs = np / 2;
    int converged = (n < 2);
    for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        int rotated = 0;
        for (int rnd = 0; rnd < np - 1; ++rnd) {
            for (int kb = 0; kb < npairs; kb += per_pass) {
                const int k = kb + warp * (32 / JG) + grp;
                int p = 0, q = 0;
                if (k == 0) {
                    p = rnd;
                    q = np - 1;
                } else {
                    p = (rnd + k) % (np - 1);
                    q = (rnd - k + (np - 1)) % (np - 1);
                }
                const bool valid = k < npairs && p < n && q < n;
                T* ap = A + (int64_t)(valid ? p : 0) * n;
                T* aq = A + (int64_t)(valid ? q : 0) * n;
                T al = 0, be = 0, ga = 0;
                if (valid)
                    for (int x = gl; x < n; x += JG) {
                        const T u = ap[x], w = aq[x];
                        al = fma(u, u, al);
                        be = fma(w, w, be);
                        ga = fma(u, w, ga);
                    }
#pragma unroll
                for (int o = JG / 2; o >= 1; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                nchk += valid && gl == 0;
                if (valid && al > (T)0 && be > (T)0 && ga * ga > tol2 * (al * be)) {
                    nrot += gl == 0;
                    T c, sn;
                    if (F64) {
                        const double z = ((double)be - (double)al) / (2.0 * (double)ga);
                        double t;
                        if (fabs(z) < 1e30) {
                            const float zf = (float)z;
                            t = (double)(copysignf(1.0f, zf) / (fabsf(zf) + hypotf(1.0f, zf)));
                        } else {
                            t = 0.5 / z;
                        }
                        const double qq = fma(t, t, 1.0);
                        double cd = (double)rsqrtf((float)qq);
                        cd = cd * fma(-0.5 * qq, cd * cd, 1.5);
                        cd = cd * fma(-0.5 * qq, cd * cd, 1.5);
                        c = (T)cd;
                        sn = (T)(cd * t);
                    } else {
                        const float z = ((float)be - (float)al) / (2.0f * (float)ga);
                        const float t = fabsf(z) < 1e18f ? copysignf(1.0f, z) / (fabsf(z) + hypotf(1.0f, z)) : 0.5f / z;
                        const float cf = rsqrtf(fmaf(t, t, 1.0f));
                        c = (T)cf;
                        sn = (T)(cf * t);
                    }
                    for (int x = gl; x < n; x += JG) {
                        const T u = ap[x], w = aq[x];
                        ap[x] = fma(c, u, -sn * w);
                        aq[x] = fma(sn, u, c * w);
                    }
                    T* jp = J + (int64_t)p * n;
                    T* jq = J + (int64_t)q * n;
                    for (int x = gl; x < n; x += JG) {
                        const T u = jp[x], w = jq[x];
                        jp[x] = fma(c, u, -sn * w);
                        jq[x] = fma(sn, u, c * w);
                    }
                    rotated = 1;
                }
            }
            __syncthreads();
        }
        converged = !__syncthreads_or(rotated);
    }
    return converged != 0;
}

// One system (row i of one component), solved by the whole CTA in the scratch slice S
// (2 n r + 4 n^2 + 2 r + 7 n doubles).  Returns this thread's share of the FP64
// operation count: ~4 (n - k)(r - k) per pivoted-QR step, 10 n^3 for the
// re-orthogonalisation, 6 n per pair check and 12 n + 20 per rotation in the FP64 sweeps, ~2 r t^2 + 8 r t + 4 r n t for V_t, the
// QR of G and the solves.  Every row's result depends on its own data only, so the weights do not
// depend on which CTA solves which row or in what order.
__device__ __forceinline__ double tsvd_system(const Elems& el, const Rows& rw, const double* __restrict__ table,
                                              int tc, const double* __restrict__ mom, double* __restrict__ W,
                                              int nwc, int wc, double tol, int max_sweeps, int64_t i,
                                              double* __restrict__ S, int32_t* __restrict__ rank_out,
                                              uint8_t* __restrict__ zid_out, unsigned* status, int* sh_t_ptr) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5, bd = blockDim.x;
    int& sh_t = *sh_t_ptr;
    double fl = 0.0;
    const int nc = el.nc;
    {
        const int n = rw.row_ptr[i + 1] - rw.row_ptr[i];
        const int r = (int)(rw.w_ptr[i + 1] - rw.w_ptr[i]);
        double* At = S;                      // [n][r]  A by rows, then the reflectors and R of A^T P = Q R
        double* G = At + (int64_t)n * r;     // [n][r]  (t columns of Z V_t, then Householder data)
        double* Jt = G + (int64_t)n * r;     // [n][n]
        double* Rb = Jt + (int64_t)n * n;    // [n][n]  R by rows, rotated by the Jacobi sweeps
        double* z = Rb + (int64_t)n * n;     // [r]
        double* v = z + r;                   // [r]
        double* b = v + r;                   // [n]
        double* sig = b + n;                 // [n]
        double* g = sig + n;                 // [n]
        double* tau = g + n;                 // [n]  reflectors of G
        double* htau = tau + n;              // [n]  reflectors of A^T
        int* keep = (int*)(htau + n);        // [n]
        int* perm = keep + n;                // [n]  column pivots of A^T (function order)
        double* Tm = htau + 2 * n;           // [n][n]  products of the re-orthogonalisation, followed
                                             //         by the float copies of R and J ([n][n] each)
        for (int64_t k = tid; k < (int64_t)n * r; k += bd) At[k] = 0.0;
        for (int64_t k = tid; k < (int64_t)n * n; k += bd) Jt[k] = (k / n == k % n) ? 1.0 : 0.0;
        for (int k = tid; k < n; k += bd) {
            b[k] = mom[rw.row_ptr[i] + k];
            perm[k] = k;
        }
        __syncthreads();
        // 1. gather
        int qoff = 0;
        for (int64_t s = rw.supp_ptr[i]; s < rw.supp_ptr[i + 1]; ++s) {
            const int e = rw.supp[s];
            const int m = el.m[e], P = el.side[e] * el.side[e];
            const double* tb = table + el.bt_ptr[e];
            const uint16_t* pos = rw.pos + rw.pos_ptr[s];
            const int il = rw.il[s];
            for (int k = tid; k < P * m; k += bd) {
                const int q = k / m, jl = k - q * m;
                At[(int64_t)pos[jl] * r + qoff + q] = tb[((int64_t)q * nc + tc) * m + jl];
            }
            for (int q = tid; q < P; q += bd) z[qoff + q] = tb[(int64_t)q * nc * m + il];
            qoff += P;
        }
        __syncthreads();
        int zero_z = 0;
        for (int q = tid; q < r; q += bd) zero_z |= (z[q] == 0.0);
        zero_z = __syncthreads_or(zero_z);
        if (zero_z)
            for (int q = tid; q < r; q += bd) z[q] = 1.0;
        // 2. Householder QR with column pivoting of A^T (r x n; its columns are the rows
        //    of At): A^T P = Q R, the reflectors kept below R in At (At[k][k+1..r) is
        //    reflector k, At[j][k] = R[k][j] for j >= k).  The one-sided Jacobi then runs
        //    on the rows of the n x n factor R: pivoting grades R so that its rows are far
        //    closer to orthogonal than those of A (about half the sweeps, each on rows of
        //    length n instead of r), and A = (P Y) S (Q J)^T with R = J S Y^T.
        // squared norms of the columns of A^T (the pivot choice), downdated after every
        // step by the entry that moves into R; the pivots only steer the convergence,
        // every choice gives the same factorisation A^T P = Q R of its own P
        for (int j = warp; j < n; j += nwarp) {
            double s2 = 0.0;
            for (int x = lane; x < r; x += 32) s2 = fma(At[(int64_t)j * r + x], At[(int64_t)j * r + x], s2);
            s2 = warp_sum(s2);
            if (lane == 0) sig[j] = s2;
        }
        __syncthreads();
        for (int k = 0; k < n; ++k) {
            if (tid == 0) {
                int pv = k;
                for (int j = k + 1; j < n; ++j)
                    if (sig[j] > sig[pv]) pv = j;
                sh_t = pv;
                fl += 4.0 * (double)(n - k) * (double)(r - k);
            }
            __syncthreads();
            const int pv = sh_t;
            if (pv != k) {
                for (int x = tid; x < r; x += bd) {
                    const double t0 = At[(int64_t)k * r + x];
                    At[(int64_t)k * r + x] = At[(int64_t)pv * r + x];
                    At[(int64_t)pv * r + x] = t0;
                }
                if (tid == 0) {
                    const int t1 = perm[k];
                    perm[k] = perm[pv];
                    perm[pv] = t1;
                    const double t2 = sig[k];
                    sig[k] = sig[pv];
                    sig[pv] = t2;
                }
            }
            __syncthreads();
            double* hk = At + (int64_t)k * r;
            if (warp == 0) {
                double xn2 = 0.0;
                for (int x = k + 1 + lane; x < r; x += 32) xn2 = fma(hk[x], hk[x], xn2);
                xn2 = warp_sum(xn2);
                const double alpha = hk[k];
                double tk = 0.0, beta = alpha, scale = 0.0;
                if (xn2 > 0.0) {
                    beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
                    tk = (beta - alpha) / beta;
                    scale = 1.0 / (alpha - beta);
                }
                __syncwarp();
                if (xn2 > 0.0)
                    for (int x = k + 1 + lane; x < r; x += 32) hk[x] *= scale;
                if (lane == 0) {
                    hk[k] = beta;
                    htau[k] = tk;
                }
            }
            __syncthreads();
            const double tk = htau[k];
            for (int j = k + 1 + warp; j < n; j += nwarp) {
                double* aj = At + (int64_t)j * r;
                double d = 0.0;
                for (int x = k + 1 + lane; x < r; x += 32) d = fma(hk[x], aj[x], d);
                d = warp_sum(d);
                d = tk * (aj[k] + d);
                for (int x = k + 1 + lane; x < r; x += 32) aj[x] -= d * hk[x];
                __syncwarp();
                if (lane == 0) {
                    aj[k] -= d;
                    sig[j] = fmax(sig[j] - aj[k] * aj[k], 0.0);
                }
            }
            __syncthreads();
        }
        for (int64_t k = tid; k < (int64_t)n * n; k += bd) {
            const int rr = (int)(k / n), cc = (int)(k - (int64_t)rr * n);
            Rb[k] = cc >= rr ? At[(int64_t)cc * r + rr] : 0.0;
        }
        __syncthreads();
        // 3. one-sided Jacobi on the rows of R, first in FP32 on a float copy (its rotations
        //    accumulated in Jf), then in FP64 from Jt = the polar factor of Jf (two
        //    Newton-Schulz steps, Higham, "Functions of Matrices", 2008, Sec. 8.3) and
        //    R <- Jt R: the FP32 sweeps do most of the rotations at the FP32 pipe's rate,
        //    the FP64 sweeps (about half as many as from R itself) take the rows to FP64
        //    orthogonality, and every applied transformation stays orthogonal to FP64
        //    rounding, so the result is the FP64 SVD of R.
        float* Rf = reinterpret_cast<float*>(Tm + (int64_t)n * n);   // [n][n]
        float* Jf = Rf + (int64_t)n * n;                              // [n][n]
        for (int64_t k = tid; k < (int64_t)n * n; k += bd) {
            Rf[k] = (float)Rb[k];
            Jf[k] = (k / n == k % n) ? 1.0f : 0.0f;
        }
        __syncthreads();
        int nchk = 0, nrot = 0;   // FP64 pair checks and rotations of this lane group
        {
            int c32 = 0, r32 = 0;
            jacobi_rows<float>(Rf, Jf, n, max_sweeps, c32, r32);
        }
        for (int64_t k = tid; k < (int64_t)n * n; k += bd) Jt[k] = (double)Jf[k];
        __syncthreads();
        for (int it = 0; it < 2; ++it) {            // Jt <- (3 I - Jt Jt^T) Jt / 2
            for (int64_t k = tid; k < (int64_t)n * n; k += bd) {
                const int a = (int)(k / n), c = (int)(k - (int64_t)a * n);
                double d = 0.0;
                for (int x = 0; x < n; ++x) d = fma(Jt[(int64_t)a * n + x], Jt[(int64_t)c * n + x], d);
                G[k] = d;
            }
            __syncthreads();
            for (int64_t k = tid; k < (int64_t)n * n; k += bd) {
                const int a = (int)(k / n), c = (int)(k - (int64_t)a * n);
                double d = 0.0;
                for (int x = 0; x < n; ++x) d = fma(G[(int64_t)a * n + x], Jt[(int64_t)x * n + c], d);
                Tm[k] = 0.5 * fma(3.0, Jt[k], -d);
            }
            __syncthreads();
            for (int64_t k = tid; k < (int64_t)n * n; k += bd) Jt[k] = Tm[k];
            __syncthreads();
        }
        for (int64_t k = tid; k < (int64_t)n * n; k += bd) {   // R <- Jt R
            const int a = (int)(k / n), c = (int)(k - (int64_t)a * n);
            double d = 0.0;
            for (int x = 0; x <= c; ++x) d = fma(Jt[(int64_t)a * n + x], Rb[(int64_t)x * n + c], d);   // R upper
            Tm[k] = d;
        }
        __syncthreads();
        for (int64_t k = tid; k < (int64_t)n * n; k += bd) Rb[k] = Tm[k];
        __syncthreads();
        if (tid == 0) fl += 10.0 * (double)n * n * n;
        const bool converged = jacobi_rows<double>(Rb, Jt, n, max_sweeps, nchk, nrot);
        if (!converged && tid == 0) atomicOr(status, ST_NOT_CONVERGED);
        fl += 6.0 * n * nchk + (12.0 * n + 20.0) * nrot;
        // 4. singular values, kept set, g = S_t^-1 U_t^T b with U = P Y (row a of the
        //    rotated R is s_a y_a^T, and (P y)[perm[j]] = y[j])
        for (int a = warp; a < n; a += nwarp) {
            double s2 = 0.0;
            for (int x = lane; x < n; x += 32) s2 += Rb[(int64_t)a * n + x] * Rb[(int64_t)a * n + x];
            s2 = warp_sum(s2);
            if (lane == 0) sig[a] = sqrt(s2);
        }
        __syncthreads();
        if (tid == 0) {
            double smax = 0.0;
            for (int a = 0; a < n; ++a) smax = fmax(smax, sig[a]);
            int t = 0;
            if (smax > 0.0)
                for (int a = 0; a < n; ++a)
                    if (sig[a] >= tol * smax) keep[t++] = a;
            sh_t = t;
        }
        __syncthreads();
        const int t = sh_t;
        if (tid == 0) fl += 2.0 * r * (double)t * t + 8.0 * r * t + 4.0 * (double)r * n * t;
        for (int k = warp; k < t; k += nwarp) {
            const int a = keep[k];
            double d = 0.0;
            for (int x = lane; x < n; x += 32) d += Rb[(int64_t)a * n + x] * b[perm[x]];
            d = warp_sum(d);
            if (lane == 0) g[k] = d / (sig[a] * sig[a]);
        }
        // 5. G = Z V_t with V = Q J: column c = Z Q [j_a; 0] (j_a = row a of Jt), the
        //    reflectors of A^T applied last to first
        for (int c = warp; c < t; c += nwarp) {
            const int a = keep[c];
            double* gc = G + (int64_t)c * r;
            for (int x = lane; x < r; x += 32) gc[x] = x < n ? Jt[(int64_t)a * n + x] : 0.0;
            __syncwarp();
            for (int kk = n - 1; kk >= 0; --kk) {
                const double* hk = At + (int64_t)kk * r;
                double d = 0.0;
                for (int x = kk + 1 + lane; x < r; x += 32) d = fma(hk[x], gc[x], d);
                d = warp_sum(d);
                d = htau[kk] * (gc[kk] + d);
                for (int x = kk + 1 + lane; x < r; x += 32) gc[x] -= d * hk[x];
                __syncwarp();
                if (lane == 0) gc[kk] -= d;
                __syncwarp();
            }
            for (int x = lane; x < r; x += 32) gc[x] *= z[x];
        }
        __syncthreads();
        // Householder QR of G (r x t, column c stored at G + c*r)
        for (int c = 0; c < t; ++c) {
            double* gc = G + (int64_t)c * r;
            if (warp == 0) {
                double xn2 = 0.0;
                for (int x = c + 1 + lane; x < r; x += 32) xn2 += gc[x] * gc[x];
                xn2 = warp_sum(xn2);
                const double alpha = gc[c];
                double tk = 0.0, beta = alpha, scale = 0.0;
                if (xn2 > 0.0) {
                    beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
                    tk = (beta - alpha) / beta;
                    scale = 1.0 / (alpha - beta);
                }
                __syncwarp();
                if (xn2 > 0.0)
                    for (int x = c + 1 + lane; x < r; x += 32) gc[x] *= scale;
                if (lane == 0) {
                    gc[c] = beta;
                    tau[c] = tk;
                }
            }
            __syncthreads();
            const double tk = tau[c];
            for (int l = c + 1 + warp; l < t; l += nwarp) {
                double* gl = G + (int64_t)l * r;
                double d = 0.0;
                for (int x = c + 1 + lane; x < r; x += 32) d += gc[x] * gl[x];
                d = warp_sum(d);
                d = tk * (gl[c] + d);
                for (int x = c + 1 + lane; x < r; x += 32) gl[x] -= d * gc[x];
                __syncwarp();
                if (lane == 0) gl[c] -= d;
            }
            __syncthreads();
        }
        // solve R^T y = g (R[l][c] = G[c*r + l]), then v = Q [y; 0], w = z v
        if (warp == 0) {
            for (int x = lane; x < r; x += 32) v[x] = 0.0;
            __syncwarp();
            for (int c = 0; c < t; ++c) {
                const double* gc = G + (int64_t)c * r;
                double d = 0.0;
                for (int l = lane; l < c; l += 32) d += gc[l] * v[l];
                d = warp_sum(d);
                const double y = (g[c] - d) / gc[c];
                __syncwarp();
                if (lane == 0) v[c] = y;
                __syncwarp();
            }
            for (int c = t - 1; c >= 0; --c) {
                const double* gc = G + (int64_t)c * r;
                double d = 0.0;
                for (int x = c + 1 + lane; x < r; x += 32) d += gc[x] * v[x];
                d = warp_sum(d);
                d = tau[c] * (v[c] + d);
                __syncwarp();
                for (int x = c + 1 + lane; x < r; x += 32) v[x] -= d * gc[x];
                if (lane == 0) v[c] -= d;
                __syncwarp();
            }
            int bad = 0;
            double* wout = W + rw.w_ptr[i] * nwc + wc;
            for (int x = lane; x < r; x += 32) {
                const double wv = z[x] * v[x];
                bad |= !isfinite(wv);
                wout[(int64_t)x * nwc] = wv;
            }
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) {
                if (rank_out) rank_out[i] = t;
                if (zid_out) zid_out[i] = (uint8_t)zero_z;
                if (bad) atomicOr(status, ST_NONFINITE);
            }
        }
        __syncthreads();
    }
    return fl;
}

__device__ __forceinline__ void add_flops(double fl, double* flops) {
    __shared__ double sh_fl[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    if (flops) {
        for (int o = 16; o >= 1; o >>= 1) fl += __shfl_xor_sync(0xffffffffu, fl, o);
        if (lane == 0) sh_fl[warp] = fl;
        __syncthreads();
        if (tid == 0) {
            double f = 0.0;
            for (int w = 0; w < nwarp; ++w) f += sh_fl[w];
            atomicAdd(flops, f);
        }
    }
}

__global__ void __launch_bounds__(128, 6) k_tsvd(Elems el, Rows rw, const double* __restrict__ table, int tc,
                                              const double* __restrict__ mom, double* __restrict__ W, int nwc,
                                              int wc, double tol, int max_sweeps, double* __restrict__ scratch,
                                              int64_t per_cta, int32_t* __restrict__ rank_out,
                                              uint8_t* __restrict__ zid_out, unsigned* status,
                                              double* __restrict__ flops) {
    __shared__ int sh_t;
    double fl = 0.0;
    double* S = scratch + (int64_t)blockIdx.x * per_cta;
    for (int64_t i = blockIdx.x; i < rw.n; i += gridDim.x)
        fl += tsvd_system(el, rw, table, tc, mom, W, nwc, wc, tol, max_sweeps, i, S, rank_out, zid_out, status, &sh_t);
    add_flops(fl, flops);
}

// Every system of several rules and components in one persistent launch: CTAs take
// jobs {system set, row} from a queue ordered by estimated cost (largest first), so
// that the uneven systems near extraordinary points spread over the grid.
__global__ void __launch_bounds__(128, 6) k_tsvd_batch(const TsvdSet* __restrict__ sets, const int2* __restrict__ jobs,
                                                    int64_t n_jobs, unsigned long long* __restrict__ next,
                                                    double tol, int max_sweeps, double* __restrict__ scratch,
                                                    int64_t per_cta, double* __restrict__ flops) {
    __shared__ int sh_t, sh_row;
    __shared__ long long sh_job;
    __shared__ TsvdSet ts;   // the job's rule and component, read from shared memory by every loop
    double fl = 0.0;
    double* S = scratch + (int64_t)blockIdx.x * per_cta;
    for (;;) {
        if (threadIdx.x == 0) {
            sh_job = (long long)atomicAdd(next, 1ull);
            if (sh_job < n_jobs) {
                const int2 jb = jobs[sh_job];
                sh_row = jb.y;
                ts = sets[jb.x];
            }
        }
        __syncthreads();
        if (sh_job >= n_jobs) break;
        // tsvd_system ends with a barrier, so thread 0 refills sh_job / ts only after
        // every thread is done with them
        fl += tsvd_system(ts.el, ts.rw, ts.table, ts.tc, ts.mom, ts.W, ts.nwc, ts.wc, tol, max_sweeps, sh_row, S,
                          ts.rank, ts.zid, ts.status, &sh_t);
    }
    add_flops(fl, flops);
}

cudaError_t launch_tsvd_batch(const TsvdSet* sets, const int2* jobs, int64_t n_jobs, unsigned long long* next,
                              double tol, int max_sweeps, double* scratch, int64_t per_cta, int n_cta, double* flops,
                              cudaStream_t st) {
    if (n_jobs == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_tsvd_batch<<<n_cta, 128, 0, st>>>(sets, jobs, n_jobs, next, tol, max_sweeps, scratch, per_cta, flops);
    return cudaGetLastError();
}

cudaError_t launch_tsvd(const Elems& el, const Rows& rw, const double* table, int tc, const double* mom, double* W,
                        int nwc, int wc, double tol, int max_sweeps, double* scratch, int64_t per_cta, int n_cta,
                        int32_t* rank, uint8_t* zid, unsigned* status, double* flops, cudaStream_t st) {
    if (rw.n == 0) return cudaSuccess;
    k_tsvd<<<n_cta, 128, 0, st>>>(el, rw, table, tc, mom, W, nwc, wc, tol, max_sweeps, scratch, per_cta, rank, zid,
                                  status, flops);
    return cudaGetLastError();
}

}  // namespace wqd
