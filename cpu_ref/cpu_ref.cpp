// cpu_ref: a multi-core CPU baseline of the assembly, FP64, OpenMP.
//
// Given precomputed inputs -- the truncated-SVD weights of every test function (Sec. 4.3),
// the basis values and derivatives at the WQ and Gauss points (Sec. 4.1) and the
// coefficient at the points -- it assembles
//   WQ (row-wise, Sec. 4.1 eqs. WQ_define / diff):
//       A_ij = sum_t sum_{q in pts(supp N_i)} w^{c_t}_iq coef(x_q) D_{c_t} N_j(x_q)
//   Gauss (element-wise, the textbook way): per element e the block
//       K_e[a][b] = sum_t sum_g gw_g coef(x_g) D_{c_t} N_a(x_g) D_{c_t} N_b(x_g),
//   then every row adds the blocks of its support elements.
// Rows (and, for the Gauss blocks, elements) are distributed over OpenMP threads;
// every output value is written by one thread, so the result does not depend on the
// thread count.  This is a timing baseline for the host cores; it shares no code with
// the GPU library.
#include <omp.h>

#include <algorithm>
#include <cstdint>
#include <vector>

namespace {

// Positions of the m (ascending) function ids fns in the ascending column list of a row.
inline void positions(const int32_t* cols, int n_i, const int32_t* fns, int m, int* pos) {
    int k = 0;
    for (int b = 0; b < m; ++b) {
        while (k < n_i && cols[k] < fns[b]) ++k;
        pos[b] = k;
    }
}

}  // namespace

extern "C" {

int cpu_ref_threads() { return omp_get_max_threads(); }
void cpu_ref_set_threads(int t) { omp_set_num_threads(t > 0 ? t : 1); }

// WQ, row-wise.  Element e: functions fns[fn_ptr[e] .. fn_ptr[e+1]) (ascending), points
// [pt_ptr[e], pt_ptr[e+1]), table block at table + tab_ptr[e] laid out [point][comp][m]
// with nc components.  Row i: columns col[row_ptr[i] .. row_ptr[i+1]) (ascending), support
// elements supp[supp_ptr[i] ..] (ascending), weights at w[(w_ptr[i] + k) * nwc + wc], k
// running over the support elements' points in order.  Terms t: weight column wc[t],
// table component tc[t], coefficient row crow[t] (-1: constant scale[t]) of coef
// ([rows][Q], rows cstride apart; null means 1).  vals [nnz] out.
void cpu_ref_wq(int64_t n, const int64_t* row_ptr, const int32_t* col, const int64_t* supp_ptr, const int32_t* supp,
                const int64_t* w_ptr, const double* w, int nwc, const int64_t* fn_ptr, const int32_t* fns,
                const int64_t* pt_ptr, const int64_t* tab_ptr, const double* table, int nc, int nt, const int* wc,
                const int* tc, const int* crow, const double* scale, const double* coef, int64_t cstride,
                double* vals) {
#pragma omp parallel
    {
        std::vector<int> pos;
        std::vector<double> acc;
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            const int64_t r0 = row_ptr[i];
            const int n_i = (int)(row_ptr[i + 1] - r0);
            acc.assign(n_i, 0.0);
            int64_t k = w_ptr[i];
            for (int64_t s = supp_ptr[i]; s < supp_ptr[i + 1]; ++s) {
                const int32_t e = supp[s];
                const int m = (int)(fn_ptr[e + 1] - fn_ptr[e]);
                const int64_t p0 = pt_ptr[e], P = pt_ptr[e + 1] - p0;
                pos.resize(m);
                positions(col + r0, n_i, fns + fn_ptr[e], m, pos.data());
                const double* tb = table + tab_ptr[e];
                for (int64_t q = 0; q < P; ++q, ++k) {
                    for (int t = 0; t < nt; ++t) {
                        const double c = crow[t] < 0 ? scale[t] : (coef ? coef[crow[t] * cstride + p0 + q] : 1.0);
                        const double sv = w[k * nwc + wc[t]] * c;
                        const double* tq = tb + (q * nc + tc[t]) * m;
                        for (int b = 0; b < m; ++b) acc[pos[b]] += sv * tq[b];
                    }
                }
            }
            std::copy(acc.begin(), acc.end(), vals + r0);
        }
    }
}

// Gauss, element-wise blocks (kbuf [sum_e m_e^2], at kb_ptr[e]) then row sums.  Gauss
// table blocks at gtable + gtab_ptr[e] ([point][comp][m]), points [gp_ptr[e], gp_ptr[e+1]),
// Gauss weights (times the area element) gw; il[s] = local index of function i in
// element supp[s].  Terms: test component sc[t], trial component tc[t], coefficient row
// crow[t] (-1: constant scale[t]).
void cpu_ref_gq(int64_t n, int64_t E, const int64_t* row_ptr, const int32_t* col, const int64_t* supp_ptr,
                const int32_t* supp, const uint8_t* il, const int64_t* fn_ptr, const int32_t* fns,
                const int64_t* gp_ptr, const int64_t* gtab_ptr, const double* gtable, const double* gw, int nc, int nt,
                const int* sc, const int* tc, const int* crow, const double* scale, const double* coef,
                int64_t cstride, const int64_t* kb_ptr, double* kbuf, double* vals) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < E; ++e) {
        const int m = (int)(fn_ptr[e + 1] - fn_ptr[e]);
        const int64_t g0 = gp_ptr[e], G = gp_ptr[e + 1] - g0;
        double* K = kbuf + kb_ptr[e];
        std::fill(K, K + (int64_t)m * m, 0.0);
        const double* tb = gtable + gtab_ptr[e];
        for (int64_t g = 0; g < G; ++g)
            for (int t = 0; t < nt; ++t) {
                const double c = crow[t] < 0 ? scale[t] : (coef ? coef[crow[t] * cstride + g0 + g] : 1.0);
                const double f = gw[g0 + g] * c;
                const double* ta = tb + (g * nc + sc[t]) * m;
                const double* tt = tb + (g * nc + tc[t]) * m;
                for (int a = 0; a < m; ++a) {
                    const double sa = f * ta[a];
                    double* Ka = K + (int64_t)a * m;
                    for (int b = 0; b < m; ++b) Ka[b] += sa * tt[b];
                }
            }
    }
#pragma omp parallel
    {
        std::vector<int> pos;
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            const int64_t r0 = row_ptr[i];
            const int n_i = (int)(row_ptr[i + 1] - r0);
            double* out = vals + r0;
            std::fill(out, out + n_i, 0.0);
            for (int64_t s = supp_ptr[i]; s < supp_ptr[i + 1]; ++s) {
                const int32_t e = supp[s];
                const int m = (int)(fn_ptr[e + 1] - fn_ptr[e]);
                pos.resize(m);
                positions(col + r0, n_i, fns + fn_ptr[e], m, pos.data());
                const double* Ka = kbuf + kb_ptr[e] + (int64_t)il[s] * m;
                for (int b = 0; b < m; ++b) out[pos[b]] += Ka[b];
            }
        }
    }
}

}  // extern "C"
