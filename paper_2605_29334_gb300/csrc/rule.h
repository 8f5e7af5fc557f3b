// Handle types of the WQ library (shared by the C-ABI translation units).
#pragma once

#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.h"
#include "wq_internal.h"

// noalloc.cu: look up the no-allocation entry point's scratch on device `dev` (current).
bool wqi_noalloc_bind(int dev, std::string& err);

constexpr int WQ_TUNE_MAX = 7;   // autotune candidates: TC, and 2 SIMT modes x 3 kernel variants

struct wq_ctx {
    int device = -1;
    std::string err;
};

struct wq_basis {
    wq_ctx* ctx = nullptr;
    wqi::BasisHost B;
};

namespace wqi {
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};
}  // namespace wqi

struct wq_rule {
    wq_ctx* ctx = nullptr;
    int device = -1;                       // the context's device, kept for destruction
    const wq_basis* basis = nullptr;
    int dim = 2, nc = 4;
    uint32_t comps = 0;
    int nwc = 0;
    int wcidx[5] = {-1, -1, -1, -1, -1};
    int64_t n = 0, E = 0, Q = 0, G = 0, nnz = 0, sum_r = 0, nsupp = 0;
    int max_n_i = 0, max_r = 0;
    double tol = 1e-12;
    int max_sweeps = 40;
    int count_mode = 0;
    int32_t auto_prec[5][2] = {{1, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}};   // WQ_PREC_AUTO per (op, gauss)
    int32_t auto_var[5][2] = {{2, 2}, {2, 2}, {2, 2}, {2, 2}, {2, 2}};    // float-mode kernel variant chosen
    // the last autotune's candidates per (op, gauss): mode, variant, error, time
    struct TuneRow {
        int32_t mode, variant;
        double err;
        float ms;
    };
    TuneRow tune[5][2][WQ_TUNE_MAX] = {};
    int32_t ntune[5][2] = {};
    int32_t set_var[5][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};   // wq_rule_set_variant (-1: auto)
    std::vector<wqi::DevBuf> bufs;
    // device arrays
    int32_t *d_m = nullptr, *d_nsub = nullptr, *d_side = nullptr, *d_pt_elem = nullptr, *d_gp_elem = nullptr;
    int64_t *d_coef_ptr = nullptr, *d_sub_ptr = nullptr, *d_pt_ptr = nullptr, *d_gp_ptr = nullptr;
    int64_t *d_bt_ptr = nullptr, *d_gbt_ptr = nullptr, *d_fn_ptr = nullptr;
    double *d_coef = nullptr, *d_geom = nullptr, *d_geom_ref = nullptr, *d_table = nullptr, *d_gtable = nullptr;
    double *d_x = nullptr, *d_gx = nullptr, *d_gw = nullptr;
    int32_t *d_row_ptr = nullptr, *d_col = nullptr, *d_supp = nullptr, *d_fns = nullptr;
    int64_t *d_supp_ptr = nullptr, *d_pos_ptr = nullptr, *d_w_ptr = nullptr;
    int32_t* d_order = nullptr;
    int4* d_desc_gq = nullptr;            // per (row, support element): Gauss table offset, points, m/P/il, positions

    // element-major FP32 assembly
    int4 *d_it_wq = nullptr, *d_it_gq = nullptr;
    int32_t *d_kb_wq = nullptr, *d_kb_gq = nullptr, *d_wrow_dst = nullptr, *d_scat = nullptr, *d_gptr = nullptr;
    int32_t* d_pt_of_w = nullptr;          // point index of every weight row
    float2* d_kscr = nullptr;
    int64_t kscr_len = 0;
    wqd::ElemItems it_wq{}, it_gq{};
    wqd::ElemPlan ep{};
    wqd::ElemSrc src_wq{}, src_gq{};
    wqd::ElemSrc64 src64_wq{}, src64_gq{};
    double* d_We = nullptr;                // element-major FP64 weights [wbase_e + q m_e + a][nwc]
    // tensor-core contraction (WQ_PREC_TC): per-element layout, trial-side slices,
    // exponents, test-side bounds, per-tile extras, split Gauss weights
    bool tc_ok = false;                    // every element has at most 64 points
    int4 *d_tcel_wq = nullptr, *d_tcel_gq = nullptr, *d_it2_wq = nullptr, *d_it2_gq = nullptr;
    int64_t *d_bsp_wq = nullptr, *d_bsp_gq = nullptr;
    int64_t bs_words_wq = 0, bs_words_gq = 0;
    uint32_t *d_bs_wq = nullptr, *d_bs_gq = nullptr;
    int32_t *d_fexp_wq = nullptr, *d_fexp_gq = nullptr;
    float *d_vmax_wq = nullptr, *d_vmax_gq = nullptr;
    float2* d_gw2 = nullptr;
    wqd::TcItems tit_wq{}, tit_gq{};
    wqd::TcSrc tc_wq{}, tc_gq{};
    std::vector<int4> h_it_wq;          // host copies of the WQ tiles (batched assembly)
    std::vector<int32_t> h_kb_wq;
    int n_sm = 1;
    uint16_t* d_pos = nullptr;
    uint8_t* d_il = nullptr;
    double* d_W = nullptr;                 // [sum_r][nwc]
    double* d_mom[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    float2 *d_table2 = nullptr, *d_gtable2 = nullptr;
    float2* d_W2 = nullptr;                // element-major split weights [wbase_e + q m_e + a][nwc]
    unsigned* d_status = nullptr;
    // staging for wq_assemble_host
    double* d_coef_stage = nullptr;
    double* d_vals_stage = nullptr;
    // kernel timing (wq_rule_set_timing): 3 events per recorded call
    mutable std::vector<cudaEvent_t> tev;
    mutable int tcount = 0;
    int tcap = 0;
    cudaEvent_t* next_timing_events() const {
        if (tcount >= tcap) return nullptr;
        return tev.data() + 3 * (tcount++);
    }
    // tile engine (k_tile.cu): element-major packs (WQ test / trial, Gauss test / trial),
    // 16 x 16 tiles per quadrature, the per-row sum plan
    bool tile_ok = false;
    float2 *d_pk_sw = nullptr, *d_pk_tw = nullptr, *d_pk_sg = nullptr, *d_pk_tg = nullptr;
    int4 *d_ti_wq = nullptr, *d_ti_gq = nullptr;
    int4 *d_tm_wq = nullptr, *d_tm_gq = nullptr;
    float *d_tmx_wq = nullptr, *d_tmx_gq = nullptr;
    int32_t *d_rowslot = nullptr, *d_kdst = nullptr;
    uint16_t* d_pos2 = nullptr;
    float2* d_kslot = nullptr;
    int64_t kslot_len = 0;
    wqd::TileJob tj_wq{}, tj_gq{};
    wqd::RowSrc rsrc{};
    std::vector<int4> h_ti_wq;            // host copies of the WQ tiles (batched assembly)
    std::vector<int4> h_tm_wq;
    wqd::Elems el{};
    wqd::Rows rw{};
    wq_rule_info info{};

    ~wq_rule() {
        for (auto ev : tev) cudaEventDestroy(ev);
        for (auto& b : bufs)
            if (b.p) cudaFree(b.p);
    }
};

// Several rules assembled together (wq_batch_create / wq_assemble_batched).
struct wq_batch {
    wq_ctx* ctx = nullptr;
    int device = -1;
    std::vector<const wq_rule*> rules;
    std::vector<wqi::DevBuf> bufs;
    wqd::BatchPlan plan{};
    bool tile_ok = false;                 // every rule has the tile engine's plan
    wqd::TileJob tj{};
    wqd::RowBatch rb{};
    ~wq_batch() {
        for (auto& b : bufs)
            if (b.p) cudaFree(b.p);
    }
};

