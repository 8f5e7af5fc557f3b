// Launchers of the WQ device kernels (implemented in k_*.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dev.cuh"

namespace wqd {

// One assembly term: WQ weight column wc / Gauss test table component sc on the
// test side, trial table component tc, multiplied by coefficient row crow of the
// caller's coefficient array (rows cstride apart; -1: the constant scale).
constexpr int WQ_MAX_TERMS = 8;
struct Term {
    int wc, tc, sc, crow;
    double scale;
};
struct Terms {
    int nt;
    Term t[WQ_MAX_TERMS];
    int64_t cstride;   // entries between coefficient rows (the number of points)
};
// The same terms for the FP32 kernels (constant scales also split into (hi, lo)).
struct TermsF {
    int wc[WQ_MAX_TERMS], tc[WQ_MAX_TERMS], sc[WQ_MAX_TERMS], crow[WQ_MAX_TERMS];
    double scale[WQ_MAX_TERMS];
    float shi[WQ_MAX_TERMS], slo[WQ_MAX_TERMS];
    int ncrow;         // coefficient rows read (max crow + 1)
    int nt;            // real terms (the rest are zero padding)
    int64_t cstride;
};
inline TermsF make_terms_f(const Terms& tm, int ntk) {
    TermsF tf{};
    tf.cstride = tm.cstride;
    tf.nt = tm.nt;
    for (int t = 0; t < ntk; ++t) {
        const bool real = t < tm.nt;
        tf.wc[t] = real ? tm.t[t].wc : 0;
        tf.tc[t] = real ? tm.t[t].tc : 0;
        tf.sc[t] = real ? tm.t[t].sc : 0;
        tf.crow[t] = real ? tm.t[t].crow : -1;
        tf.scale[t] = real ? tm.t[t].scale : 0.0;   // padding terms contribute zero
        tf.shi[t] = (float)tf.scale[t];
        tf.slo[t] = (float)(tf.scale[t] - (double)tf.shi[t]);
        tf.ncrow = tf.ncrow > tf.crow[t] + 1 ? tf.ncrow : tf.crow[t] + 1;
    }
    return tf;
}

// Placement + basis evaluation at WQ (gauss = 0) or Gauss (gauss = 1) points:
// table [pts][nc][m_e] per element, coordinates xout [pts][3], Gauss weights
// (w * area element) wout [pts] (Gauss only).
cudaError_t launch_eval(const Elems& el, const int32_t* pt_elem, int64_t npts, int gauss,
                        double* table, double* xout, double* wout, unsigned* status, cudaStream_t st);

// Gauss component matrices G^c (c = 1) row-wise: the moments b of the weight
// systems, table component tc, Gauss weights gw (area element included).
cudaError_t launch_moments_f64(const Rows& rw, const int4* desc, int tc, int nc, const double* table,
                               const double* gw, double* vals, int max_n_i, cudaStream_t st);

// FP32 element-major assembly (split products; compensated = TwoSum sums):
// element tiles into the slot buffer, then one sum per CSR entry.  WQ items
// (gauss = 0) read the test side from the element-major weights W2e; Gauss items
// (gauss = 1) from the table, times the Gauss weights gw.  1..4 terms; float CSR values.
cudaError_t launch_elem_f32(const ElemItems& it, const ElemSrc& src, const Terms& tm, int gauss, const double* coef,
                            float* vals, bool compensated, cudaStream_t st, cudaEvent_t* evs = nullptr);

// The same for k <= WQ_BATCH_MAX rules with one launch of each kernel (WQ items;
// the rules share their weight components and dimension, so one TermsF serves all).
cudaError_t launch_elem_batch(const BatchPlan& bp, const double* const* coefs, float* const* vals, int k,
                              const Terms& tm, bool compensated, cudaStream_t st);

// Tensor-core contraction: slices per operand, and trial-slice words per (quarter-chunk
// of 4 points of one component, 16-column block): per slice, 2 point pairs x 8
// columns x 2 n-tiles.
constexpr int WQ_TC_SLICES = 5;
constexpr int WQ_TC_QUARTER_WORDS = 32 * WQ_TC_SLICES;

// Per-entry sums of the slot buffer (FP32 pairs, TwoSum) as a programmatic dependent
// of the element kernel just launched on st.
cudaError_t launch_gather_f32(const ElemSrc& src, float* vals, bool compensated, cudaStream_t st);

// Tensor-core element contraction (bf16 slices, exact FP32 integer sums; 1..8 terms),
// then the per-entry sums; float CSR values.  Trial-side slices from launch_tc_prep.
cudaError_t launch_elem_tc(const TcItems& it, const TcSrc& src, const Terms& tm, int gauss, const double* coef,
                           float* vals, cudaStream_t st, cudaEvent_t* evs = nullptr);
// Trial-side slices, exponents and test-side bounds of every element (rule set-up):
// table [E blocks][P][nc][m]; We element-major FP64 weights (WQ) or null (Gauss).
cudaError_t launch_tc_prep(int64_t E, int nc, int nwc, const int32_t* m, const double* table, const double* We,
                           const TcPrep& pr, cudaStream_t st);

// FP64 element-major assembly (same tiles and slot map; FMA sums; double CSR values).
cudaError_t launch_elem_f64(const ElemItems& it, const ElemSrc64& src, const Terms& tm, int gauss,
                            const double* coef, double* vals, cudaStream_t st, cudaEvent_t* evs = nullptr);
// Element-major copy of the FP64 weights (We[dst[r]] = W[r], nwc columns).
cudaError_t launch_copy_rows(const double* W, const int32_t* dst, double* We, int64_t rows, int nwc, int n_sm,
                             cudaStream_t st);

// Element-major split copy of the weights (W2e[dst[r]] = split(W[r]), nwc columns).
cudaError_t launch_split_rows(const double* W, const int32_t* dst, float2* W2e, int64_t rows, int nwc, int n_sm,
                              cudaStream_t st);

// Truncated-SVD weights of every row for one component (Sec. 4.3):
//   table comp tc gives A, table comp 0 gives Z, mom [nnz] gives b;
//   writes W[(w_ptr[i] + q) * nwc + wc].  scratch holds `per_cta` doubles per CTA.
//   Per-row rank written to rank[i], Z = I fallback flagged in zid[i]; the FP64
//   operation count is added to *flops (may be null).
// Scratch of one truncated-SVD system (doubles) for rows of at most max_n functions and
// max_r points, and the CTAs per SM the solver kernels are built for.
inline int64_t tsvd_scratch_doubles(int64_t max_n, int64_t max_r) {
    return 2 * max_n * max_r + 4 * max_n * max_n + 2 * max_r + 7 * max_n + 8;
}
constexpr int TSVD_CTAS_PER_SM = 6;
cudaError_t launch_tsvd(const Elems& el, const Rows& rw, const double* table, int tc,
                        const double* mom, double* W, int nwc, int wc, double tol, int max_sweeps,
                        double* scratch, int64_t per_cta, int n_cta, int32_t* rank, uint8_t* zid,
                        unsigned* status, double* flops, cudaStream_t st);

// The same solves for many rules and components in one persistent launch (n_cta CTAs,
// per_cta doubles of scratch each): jobs[j] = {index into sets, row}, taken in order
// through the counter *next (zeroed on `st` before the launch).
cudaError_t launch_tsvd_batch(const TsvdSet* sets, const int2* jobs, int64_t n_jobs, unsigned long long* next,
                              double tol, int max_sweeps, double* scratch, int64_t per_cta, int n_cta, double* flops,
                              cudaStream_t st);

// u_h and grad u_h at WQ points (Sec. 5 interpolation).
cudaError_t launch_interp(const Elems& el, const int32_t* pt_elem, const int32_t* fns,
                          const int64_t* fn_ptr, int64_t Q, const double* table, const double* u,
                          double* uq, double* grad, cudaStream_t st);

// Heat point fields (Sec. 5): kappa [Q] = k0 + k2 u^2; g [1 + dim][Q] residual data.
cudaError_t launch_heat_fields(const Elems& el, const int32_t* pt_elem, const int32_t* fns, const int64_t* fn_ptr,
                               int64_t Q, const double* table, const double* u, const double* uo, double dt, double k0,
                               double k2, double f, bool jacobian, double* kappa, double* g, cudaStream_t st);

// Matrix-free WQ functional y_i = sum_t sum_q w^{wc_t}_iq g[t][q] (weight columns in wc4, nt <= 4).
cudaError_t launch_apply(const Rows& rw, const int32_t* pt_of_w, int nt, int4 wc4, const double* W, int nwc,
                         const double* g, int64_t Q, double* y, cudaStream_t st);

// Tile engine (k_tile.cu): element blocks staged by bulk copies, then per-row sums
// (programmatic dependent launch); float CSR values.  variant 0 / 1: chunks of up to
// 12 / 6 points (2 terms).  n_sm = multiprocessors (persistent grid).  evs: 3 events
// (before, between, after) or null.  prepare_tile_kernels() sets the kernels' shared
// memory size on the current device (once, before any launch or capture).
cudaError_t prepare_tile_kernels();
cudaError_t launch_tile_f32(const TileJob& job, const RowSrc& rs, const TileTerms& tm, const double* coef,
                            float* vals, bool compensated, int variant, int n_sm, cudaStream_t st,
                            cudaEvent_t* evs = nullptr);
// The same for k <= WQ_BATCH_MAX rules (items carry their rule; rows in RowBatch blocks).
cudaError_t launch_tile_batch(const TileJob& job, const RowBatch& rb, const double* const* coefs, float* const* vals,
                              int k, const TileTerms& tm, bool compensated, int variant, int n_sm, cudaStream_t st);
// Element-major pack of a table or of the weights (rule set-up), and the bound table of a
// trial pack (max |hi| per element, 16-function block and component).
cudaError_t launch_pack(const PackJob& pj, cudaStream_t st);
cudaError_t launch_pack_max(const PackJob& pj, const int64_t* tmx_off, float* tmx, cudaStream_t st);

// Convert double arrays to (hi, lo) float pairs.
cudaError_t launch_split_f32(const double* src, float2* dst, int64_t n, cudaStream_t st);

void set_gauss_constants(const double x[4], const double w[4]);

}  // namespace wqd
