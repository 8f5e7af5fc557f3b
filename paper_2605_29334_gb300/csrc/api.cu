// C ABI of the WQ library (include/wq.h): handles, the device rule build
// (placement, basis tables, Gauss moments, truncated-SVD weights) and the
// assembly entry points.  Host set-up lives in host.cpp, kernels in k_*.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "rule.h"
#include "wq_internal.h"

namespace {

wq_status fail(wq_ctx* ctx, wq_status code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

template <class T>
bool dalloc(wq_rule* R, T*& p, size_t count, wq_status& st) {
    void* q = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        st = fail(R->ctx, WQ_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                                          cudaGetErrorString(e));
        return false;
    }
    R->bufs.push_back({q, bytes});
    p = static_cast<T*>(q);
    return true;
}

template <class T>
bool upload(wq_rule* R, T*& p, const std::vector<T>& v, wq_status& st) {
    if (!dalloc(R, p, v.size(), st)) return false;
    if (v.empty()) return true;
    cudaError_t e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        st = fail(R->ctx, WQ_ERR_CUDA, std::string("upload failed: ") + cudaGetErrorString(e));
        return false;
    }
    return true;
}

#define CUDA_TRY(ctx, call)                                                                        \
    do {                                                                                           \
        cudaError_t _e = (call);                                                                   \
        if (_e != cudaSuccess)                                                                     \
            return fail(ctx, WQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e));    \
    } while (0)

wq_status status_to_error(wq_ctx* ctx, unsigned s) {
    if (s & wqd::ST_BAD_INDEX) return fail(ctx, WQ_ERR_CUDA, "device index check failed");
    if (s & wqd::ST_GEOMETRY) return fail(ctx, WQ_ERR_MESH, "folded or degenerate geometry map at a quadrature point");
    if (s & wqd::ST_NOT_CONVERGED) return fail(ctx, WQ_ERR_NOT_CONVERGED, "Jacobi SVD reached its sweep cap");
    if (s & wqd::ST_NONFINITE) return fail(ctx, WQ_ERR_NONFINITE, "non-finite value in the weight solve");
    if (s & wqd::ST_ILLPOSED) return fail(ctx, WQ_ERR_ILLPOSED, "ill-posed weight system");
    return WQ_OK;
}

int table_comp(const wq_rule* R, int comp) {
    switch (comp) {
        case WQ_COMP_N: return 0;
        case WQ_COMP_X: return 1;
        case WQ_COMP_Y: return 2;
        case WQ_COMP_Z: return R->dim == 3 ? 3 : -1;
        case WQ_COMP_LAP: return R->nc - 1;
        default: return -1;
    }
}

// Terms of an operator; returns false if a needed weight set is missing.  Each term
// pairs a test component (WQ weight set / Gauss test table) with a trial table
// component and a coefficient row (-1: the constant scale); npts = the number of
// points of the coefficient rows (WQ or Gauss).
bool op_terms(const wq_rule* R, int op, double alpha, bool need_weights, wqd::Terms& tm, int64_t npts) {
    tm.nt = 0;
    tm.cstride = npts;
    auto add = [&](int test, int trial, int crow, double scale) -> bool {
        const int sc = table_comp(R, test), tc = table_comp(R, trial);
        if (sc < 0 || tc < 0) return false;
        const int wc = R->wcidx[test];
        if (need_weights && wc < 0) return false;
        tm.t[tm.nt++] = {wc < 0 ? 0 : wc, tc, sc, crow, scale};
        return true;
    };
    const int grads[3] = {WQ_COMP_X, WQ_COMP_Y, WQ_COMP_Z};
    const int nd = R->dim == 3 ? 3 : 2;
    switch (op) {
        case WQ_OP_MASS: return add(WQ_COMP_N, WQ_COMP_N, 0, 1.0);
        case WQ_OP_STIFF:
            for (int d = 0; d < nd; ++d)
                if (!add(grads[d], grads[d], 0, 1.0)) return false;
            return true;
        case WQ_OP_BIHARM: return add(WQ_COMP_LAP, WQ_COMP_LAP, 0, 1.0);
        case WQ_OP_HEAT_S:
            if (!add(WQ_COMP_N, WQ_COMP_N, -1, alpha)) return false;
            for (int d = 0; d < nd; ++d)
                if (!add(grads[d], grads[d], 0, 1.0)) return false;
            return true;
        case WQ_OP_HEAT_J:
            if (!add(WQ_COMP_N, WQ_COMP_N, -1, alpha)) return false;
            for (int d = 0; d < nd; ++d)
                if (!add(grads[d], grads[d], 0, 1.0)) return false;
            for (int d = 0; d < nd; ++d)
                if (!add(grads[d], WQ_COMP_N, 1 + d, 1.0)) return false;
            return true;
        default: return false;
    }
}

// Terms of the tile kernels (k_tile.cu) from an operator's terms: test components
// (weight columns for WQ, table components of the Gauss test pack) and trial table
// components as indices into the staged ranges.  False if a range is wider than the
// kernel stages (min(terms, 4) components per side).
bool tile_terms(const wqd::Terms& tm, bool gauss, wqd::TileTerms& tt) {
    const int ntk = tm.nt <= 4 ? tm.nt : 8;
    const int cm = ntk < 4 ? ntk : 4;
    int slo = 1 << 20, shi = -1, rlo = 1 << 20, rhi = -1;
    for (int t = 0; t < tm.nt; ++t) {
        const int sc = gauss ? tm.t[t].sc : tm.t[t].wc, rc = tm.t[t].tc;
        slo = std::min(slo, sc);
        shi = std::max(shi, sc);
        rlo = std::min(rlo, rc);
        rhi = std::max(rhi, rc);
    }
    if (tm.nt < 1 || shi - slo + 1 > cm || rhi - rlo + 1 > cm) return false;
    tt = wqd::TileTerms{};
    tt.nt = tm.nt;
    tt.s_lo = slo;
    tt.s_n = shi - slo + 1;
    tt.r_lo = rlo;
    tt.r_n = rhi - rlo + 1;
    tt.cstride = tm.cstride;
    tt.ncrow = 0;
    for (int t = 0; t < ntk; ++t) {
        const bool real = t < tm.nt;
        tt.tcomp[t] = real ? (gauss ? tm.t[t].sc : tm.t[t].wc) - slo : 0;
        tt.rcomp[t] = real ? tm.t[t].tc - rlo : 0;
        tt.crow[t] = real ? tm.t[t].crow : -1;
        const double sc = real ? tm.t[t].scale : 0.0;   // padding terms contribute zero
        tt.shi[t] = (float)sc;
        tt.slo[t] = (float)(sc - (double)tt.shi[t]);
        tt.ncrow = std::max(tt.ncrow, tt.crow[t] + 1);
    }
    return tt.ncrow <= 4;
}

// Kernel variant of the float modes for (op, gauss): wq_rule_set_variant's, else the
// autotuner's choice (WQ_VARIANT_TILE12 until it has run).
int float_variant(const wq_rule* R, int op, int gauss) {
    const int v = R->set_var[op][gauss];
    return v >= 0 ? v : R->auto_var[op][gauss];
}

}  // namespace



extern "C" {

wq_status wq_create(int device, wq_ctx** out) {
    if (!out) return WQ_ERR_ARG;
    *out = nullptr;
    wq_ctx* c = new (std::nothrow) wq_ctx();
    if (!c) return WQ_ERR_OOM;
    if (device >= 0) {
        int nd = 0;
        cudaError_t e = cudaGetDeviceCount(&nd);
        if (e != cudaSuccess || device >= nd) {
            cudaGetLastError();
            delete c;
            return WQ_ERR_NO_DEVICE;
        }
        e = cudaSetDevice(device);
        if (e != cudaSuccess) {
            delete c;
            return WQ_ERR_CUDA;
        }
        // the no-allocation entry point's fixed scratch: its device address is looked up
        // (and its memory committed) now, with the device current
        std::string nerr;
        if (!wqi_noalloc_bind(device, nerr)) {
            cudaGetLastError();
            delete c;
            return WQ_ERR_CUDA;
        }
    }
    c->device = device;
    *out = c;
    return WQ_OK;
}

void wq_destroy(wq_ctx* ctx) { delete ctx; }

const char* wq_last_error(const wq_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

wq_status wq_build_basis(wq_ctx* ctx, const wq_mesh_desc* mesh, wq_basis** out) {
    if (!ctx || !mesh || !out) return fail(ctx, WQ_ERR_ARG, "null argument");
    *out = nullptr;
    if (mesh->dim != 2 && mesh->dim != 3) return fail(ctx, WQ_ERR_ARG, "dim must be 2 or 3");
    if (mesh->n_vertices <= 0 || mesh->n_faces <= 0 || !mesh->xyz || !mesh->quads)
        return fail(ctx, WQ_ERR_ARG, "empty mesh");
    if (mesh->n_vertices > INT32_MAX || mesh->n_faces > INT32_MAX / 4)
        return fail(ctx, WQ_ERR_ARG, "mesh too large for 32-bit indices");
    wq_basis* b = new (std::nothrow) wq_basis();
    if (!b) return fail(ctx, WQ_ERR_OOM, "host allocation failed");
    b->ctx = ctx;
    wqi::Error err{WQ_OK, ""};
    bool ok = false;
    try {
        ok = wqi::build_basis(*mesh, b->B, err);
    } catch (const std::bad_alloc&) {
        err = {WQ_ERR_OOM, "host allocation failed"};
    }
    if (!ok) {
        delete b;
        return fail(ctx, err.code, err.msg);
    }
    if (b->B.E == 0) {
        delete b;
        return fail(ctx, WQ_ERR_MESH, "mesh has no active element");
    }
    *out = b;
    return WQ_OK;
}

void wq_basis_destroy(wq_basis* basis) { delete basis; }

wq_status wq_basis_info_get(const wq_basis* basis, wq_basis_info* info) {
    if (!basis || !info) return WQ_ERR_ARG;
    const wqi::BasisHost& B = basis->B;
    info->n_functions = B.n;
    info->n_elements = B.E;
    info->n_irregular = B.n_irregular;
    info->nnz = B.row_ptr.empty() ? 0 : B.row_ptr[B.n];
    info->max_m = B.max_m;
    info->max_n_i = B.max_n_i;
    for (int k = 0; k < 7; ++k) info->type_count[k] = B.type_count[k];
    return WQ_OK;
}

wq_status wq_basis_element(const wq_basis* basis, int64_t e, int32_t* face, int32_t* type, int32_t* m,
                           int32_t* nsub, int32_t* h_fns, double* h_coef) {
    if (!basis) return WQ_ERR_ARG;
    const wqi::BasisHost& B = basis->B;
    if (e < 0 || e >= B.E) return fail(basis->ctx, WQ_ERR_ARG, "element index out of range");
    if (face) *face = B.elem_face[e];
    if (type) *type = B.etype[e];
    if (m) *m = B.m(e);
    if (nsub) *nsub = B.nsub[e];
    if (h_fns) std::copy(B.fns.begin() + B.fn_ptr[e], B.fns.begin() + B.fn_ptr[e + 1], h_fns);
    if (h_coef) std::copy(B.coef.begin() + B.coef_ptr[e], B.coef.begin() + B.coef_ptr[e + 1], h_coef);
    return WQ_OK;
}

wq_status wq_basis_ctrl(const wq_basis* basis, double* h_xyz) {
    if (!basis || !h_xyz) return WQ_ERR_ARG;
    std::copy(basis->B.ctrl.begin(), basis->B.ctrl.end(), h_xyz);
    return WQ_OK;
}

wq_status wq_basis_pattern(const wq_basis* basis, int64_t* h_row_ptr, int32_t* h_col) {
    if (!basis) return WQ_ERR_ARG;
    if (h_row_ptr) std::copy(basis->B.row_ptr.begin(), basis->B.row_ptr.end(), h_row_ptr);
    if (h_col) std::copy(basis->B.col.begin(), basis->B.col.end(), h_col);
    return WQ_OK;
}

wq_status wq_point_counts(const wq_basis* basis, int32_t count_mode, int32_t* h_side) {
    if (!basis || !h_side) return WQ_ERR_ARG;
    std::vector<int32_t> side;
    wqi::Error err{WQ_OK, ""};
    if (!wqi::point_counts(basis->B, count_mode, side, err)) return fail(basis->ctx, err.code, err.msg);
    std::copy(side.begin(), side.end(), h_side);
    return WQ_OK;
}

namespace {
// Weights, moments and weight statistics of a saved rule (wq_rule_save / wq_rule_load).
struct SavedRule {
    std::vector<double> W;                 // [sum_r][nwc]
    std::vector<std::vector<double>> mom;  // per built component, [nnz]
    int32_t n_truncated[5], n_z_identity[5];
    float setup_ms;
};

constexpr char kRuleMagic[8] = {'W', 'Q', 'R', 'U', 'L', 'E', '0', '1'};
struct RuleFileHeader {
    char magic[8];
    uint32_t version, comps;
    int32_t count_mode, max_sweeps;
    double tol;
    int64_t n, E, nnz, Q, G, sum_r;
    int32_t nwc, dim;
    uint64_t fingerprint;
    int32_t n_truncated[5], n_z_identity[5];
    float setup_ms;
    int32_t pad;
};

// FNV-1a over the mesh that defines the spline space (coordinates and quads).
uint64_t basis_fingerprint(const wqi::BasisHost& B) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t bytes) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t k = 0; k < bytes; ++k) {
            h ^= c[k];
            h *= 1099511628211ull;
        }
    };
    mix(&B.dim, sizeof(B.dim));
    mix(&B.n, sizeof(B.n));
    mix(&B.E, sizeof(B.E));
    mix(B.xyz.data(), B.xyz.size() * sizeof(double));
    mix(B.topo.quads.data(), B.topo.quads.size() * sizeof(int32_t));
    return h;
}

// What a rule build carries from its first device phase (plan, uploads, point tables,
// moments) through the weight solves to its last phase (split copies, packs,
// tensor-core plan).  The device arrays belong to the rule.
struct BuildState {
    cudaStream_t st = nullptr;
    double tol = 1e-12;
    int sweeps = 40;
    const SavedRule* saved = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int32_t* d_rank = nullptr;      // [nwc][n] rank of every system
    uint8_t* d_zid = nullptr;       // [nwc][n] Z = I flags
    double* d_flops = nullptr;
    int32_t *d_Pw = nullptr, *d_Pg = nullptr;
    int64_t *d_sw_off = nullptr, *d_tw_off = nullptr, *d_sg_off = nullptr, *d_tg_off = nullptr;
    int64_t *d_wbase = nullptr, *d_tmx_off = nullptr;
    int64_t bt_E = 0, gbt_E = 0;
    int64_t per_cta = 0;            // weight-solve scratch per CTA (doubles)
    std::vector<double> row_cost;   // n_i^2 r_i: the Jacobi work of each row's system
    BuildState() = default;
    BuildState(const BuildState&) = delete;
    BuildState& operator=(const BuildState&) = delete;
    ~BuildState() {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};
}  // namespace

// A CUDA error left pending by another caller (or by a teardown) must not be reported
// by this library's next launch check: entry points that launch work drop it first.
static inline void drop_stale_error() { (void)cudaGetLastError(); }

// First phase of a rule build: host plan, uploads, placement, basis tables and Gauss
// moments (queued on the build stream, not waited for).  On failure the rule is freed.
static wq_status rule_prepare(wq_basis* basis, const wq_rule_opts* opts, const SavedRule* saved, wq_rule** out,
                              BuildState& bs) {
    if (!basis || !opts || !out) return WQ_ERR_ARG;
    *out = nullptr;
    wq_ctx* ctx = basis->ctx;
    if (ctx->device < 0) return fail(ctx, WQ_ERR_NO_DEVICE, "context has no device");
    if ((opts->comps & ~31u) || opts->comps == 0) return fail(ctx, WQ_ERR_ARG, "bad component mask");
    const wqi::BasisHost& B = basis->B;
    if (B.dim == 2 && (opts->comps & (1u << WQ_COMP_Z)))
        return fail(ctx, WQ_ERR_ARG, "d_z weights requested on a planar domain");
    double tol = opts->tsvd_rel_tol > 0 ? opts->tsvd_rel_tol : 1e-12;
    int sweeps = opts->max_sweeps > 0 ? opts->max_sweeps : 40;
    cudaStream_t st = (cudaStream_t)opts->stream;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    drop_stale_error();

    wq_rule* R = new (std::nothrow) wq_rule();
    if (!R) return fail(ctx, WQ_ERR_OOM, "host allocation failed");
    R->ctx = ctx;
    R->device = ctx->device;
    R->basis = basis;
    R->dim = B.dim;
    R->nc = B.dim + 2;
    R->comps = opts->comps;
    for (int c = 0; c < 5; ++c)
        if (opts->comps & (1u << c)) R->wcidx[c] = R->nwc++;
    R->n = B.n;
    R->E = B.E;
    R->nnz = B.row_ptr[B.n];
    R->max_n_i = B.max_n_i;
    R->tol = tol;
    R->max_sweeps = sweeps;
    R->count_mode = opts->count_mode;
    wq_status sst = WQ_OK;
    auto bail = [&](wq_status s) {
        delete R;
        return s;
    };

    // a1: point counts (host)
    std::vector<int32_t> side;
    wqi::Error err{WQ_OK, ""};
    if (!wqi::point_counts(B, opts->count_mode, side, err)) return bail(fail(ctx, err.code, err.msg));
    const int64_t E = B.E, n = B.n;
    const int nc = R->nc;
    std::vector<int32_t> m(E), nsub(B.nsub.begin(), B.nsub.end());
    std::vector<int64_t> pt_ptr(E + 1, 0), gp_ptr(E + 1, 0), bt_ptr(E + 1, 0), gbt_ptr(E + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        m[e] = B.m(e);
        const int64_t P = (int64_t)side[e] * side[e];
        pt_ptr[e + 1] = pt_ptr[e] + P;
        gp_ptr[e + 1] = gp_ptr[e] + 16 * nsub[e];
        bt_ptr[e + 1] = bt_ptr[e] + P * nc * m[e];
        gbt_ptr[e + 1] = gbt_ptr[e] + 16LL * nsub[e] * nc * m[e];
    }
    R->Q = pt_ptr[E];
    R->G = gp_ptr[E];
    std::vector<int32_t> pt_elem(R->Q), gp_elem(R->G);
    for (int64_t e = 0; e < E; ++e) {
        for (int64_t p = pt_ptr[e]; p < pt_ptr[e + 1]; ++p) pt_elem[p] = (int32_t)e;
        for (int64_t p = gp_ptr[e]; p < gp_ptr[e + 1]; ++p) gp_elem[p] = (int32_t)e;
    }
    // row plan: positions of each support element's functions in row i
    R->nsupp = B.supp_ptr[n];
    std::vector<int64_t> pos_ptr(R->nsupp + 1, 0), w_ptr(n + 1, 0);
    std::vector<uint8_t> il(R->nsupp);
    for (int64_t s = 0; s < R->nsupp; ++s) pos_ptr[s + 1] = pos_ptr[s] + m[B.supp[s]];
    std::vector<uint16_t> pos(pos_ptr[R->nsupp]);
    bs.row_cost.assign(n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* c0 = B.col.data() + B.row_ptr[i];
        const int32_t* c1 = B.col.data() + B.row_ptr[i + 1];
        if (c1 - c0 > 65535) return bail(fail(ctx, WQ_ERR_ARG, "row longer than 65535 entries"));
        int64_t r = 0;
        for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
            const int32_t e = B.supp[s];
            r += (int64_t)side[e] * side[e];
            int found = -1;
            for (int64_t p = B.fn_ptr[e]; p < B.fn_ptr[e + 1]; ++p) {
                const int32_t j = B.fns[p];
                pos[pos_ptr[s] + (p - B.fn_ptr[e])] = (uint16_t)(std::lower_bound(c0, c1, j) - c0);
                if (j == (int32_t)i) found = (int)(p - B.fn_ptr[e]);
            }
            if (found < 0 || found > 255) return bail(fail(ctx, WQ_ERR_ARG, "support bookkeeping failed"));
            il[s] = (uint8_t)found;
        }
        w_ptr[i + 1] = w_ptr[i] + r;
        R->max_r = std::max<int>(R->max_r, (int)r);
        const double ni = (double)(B.row_ptr[i + 1] - B.row_ptr[i]);
        bs.row_cost[i] = ni * ni * (double)r;
        if (r < B.row_ptr[i + 1] - B.row_ptr[i])
            return bail(fail(ctx, WQ_ERR_ILLPOSED, "r_i < n_i for test function " + std::to_string(i)));
    }
    R->sum_r = w_ptr[n];
    // processing order of the rows: Morton order of the functions' control points
    std::vector<int32_t> order(n);
    {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], B.ctrl[3 * i + d]);
                hi[d] = std::max(hi[d], B.ctrl[3 * i + d]);
            }
        std::vector<uint64_t> key(n);
        for (int64_t i = 0; i < n; ++i) {
            uint64_t k = 0;
            uint32_t c[3];
            for (int d = 0; d < 3; ++d) {
                double t = hi[d] > lo[d] ? (B.ctrl[3 * i + d] - lo[d]) / (hi[d] - lo[d]) : 0.0;
                c[d] = (uint32_t)std::min(2097151.0, std::max(0.0, t * 2097151.0));
            }
            for (int b = 20; b >= 0; --b)
                for (int d = 0; d < 3; ++d) k = (k << 1) | ((c[d] >> b) & 1u);
            key[i] = k;
        }
        for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    }
    // packed per-(row, support element) descriptors of the Gauss moment kernel
    if (bt_ptr[E] > INT32_MAX || gbt_ptr[E] > INT32_MAX || pos_ptr[R->nsupp] > INT32_MAX || R->G > INT32_MAX)
        return bail(fail(ctx, WQ_ERR_ARG, "mesh too large for 32-bit table offsets"));
    std::vector<int4> desc_gq(R->nsupp);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
            const int32_t e = B.supp[s];
            if (m[e] > 255 || side[e] * side[e] > 255)
                return bail(fail(ctx, WQ_ERR_ARG, "element with more than 255 functions or points"));
            desc_gq[s] = make_int4((int)gbt_ptr[e], (int)gp_ptr[e], m[e] | (16 * nsub[e]) << 8 | il[s] << 16,
                                   (int)pos_ptr[s]);
        }
    // element-major FP32 plan: 16 x 16 tiles of the element blocks (elements with
    // more chunks of points first), the element-major row of every weight row, and
    // the slot of every block entry, grouped by CSR entry in support order
    std::vector<int64_t> kptr(E + 1, 0), wbase(E + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        kptr[e + 1] = kptr[e] + (int64_t)m[e] * m[e];
        wbase[e + 1] = wbase[e] + (int64_t)m[e] * side[e] * side[e];
    }
    if (kptr[E] > INT32_MAX || wbase[E] > INT32_MAX)
        return bail(fail(ctx, WQ_ERR_ARG, "mesh too large for 32-bit element block offsets"));
    std::vector<int4> it_wq, it_gq;
    std::vector<int32_t> kb_wq, kb_gq, ie_wq, ie_gq;
    auto make_items = [&](bool gauss, std::vector<int4>& item, std::vector<int32_t>& kb, std::vector<int32_t>& ie) {
        auto npts = [&](int64_t e) { return gauss ? 16 * nsub[e] : side[e] * side[e]; };
        auto chunks = [&](int64_t e) { return (npts(e) + 7) / 8; };
        std::vector<int32_t> by_work(E);
        for (int64_t e = 0; e < E; ++e) by_work[e] = (int32_t)e;
        std::stable_sort(by_work.begin(), by_work.end(), [&](int32_t x, int32_t y) {
            return chunks(x) * ((m[x] + 15) / 16) > chunks(y) * ((m[y] + 15) / 16);
        });
        for (int32_t e : by_work)
            for (int a0 = 0; a0 < m[e]; a0 += 16)
                for (int b0 = 0; b0 < m[e]; b0 += 16) {
                    item.push_back(make_int4(gauss ? (int)gbt_ptr[e] : (int)bt_ptr[e],
                                             gauss ? (int)gp_ptr[e] : (int)pt_ptr[e],
                                             m[e] | npts(e) << 8 | (a0 / 16) << 16 | (b0 / 16) << 20,
                                             (int)wbase[e]));
                    kb.push_back((int32_t)kptr[e]);
                    ie.push_back(e);
                }
    };
    make_items(false, it_wq, kb_wq, ie_wq);
    make_items(true, it_gq, kb_gq, ie_gq);
    // tensor-core contraction: per element {table offset, points, weight row, first
    // function} and the offsets of its trial-side slices (nc components x column
    // blocks x quarter-chunks x WQ_TC_QUARTER_WORDS words); per tile {first function,
    // slice offset, element, points rounded up to 4}
    std::vector<int4> tcel_wq(E), tcel_gq(E), it2_wq(it_wq.size()), it2_gq(it_gq.size());
    std::vector<int64_t> bsp_wq(E + 1, 0), bsp_gq(E + 1, 0);
    R->tc_ok = true;
    for (int64_t e = 0; e < E; ++e) {
        const int pw = side[e] * side[e], pg = 16 * nsub[e], ncb = (m[e] + 15) / 16;
        if (pw > 64 || pg > 64) R->tc_ok = false;
        tcel_wq[e] = make_int4((int)bt_ptr[e], pw, (int)wbase[e], (int)B.fn_ptr[e]);
        tcel_gq[e] = make_int4((int)gbt_ptr[e], pg, (int)wbase[e], (int)B.fn_ptr[e]);
        bsp_wq[e + 1] = bsp_wq[e] + (int64_t)nc * ncb * ((pw + 3) / 4) * wqd::WQ_TC_QUARTER_WORDS;
        bsp_gq[e + 1] = bsp_gq[e] + (int64_t)nc * ncb * ((pg + 3) / 4) * wqd::WQ_TC_QUARTER_WORDS;
    }
    if (bsp_wq[E] > INT32_MAX || bsp_gq[E] > INT32_MAX || B.fn_ptr[E] > INT32_MAX) R->tc_ok = false;
    if (opts->skip_plans & WQ_PLAN_NO_TC) R->tc_ok = false;
    for (size_t x = 0; x < it_wq.size(); ++x) {
        const int32_t e = ie_wq[x];
        it2_wq[x] = make_int4((int)B.fn_ptr[e], (int)bsp_wq[e], e, (side[e] * side[e] + 3) / 4 * 4);
    }
    for (size_t x = 0; x < it_gq.size(); ++x) {
        const int32_t e = ie_gq[x];
        it2_gq[x] = make_int4((int)B.fn_ptr[e], (int)bsp_gq[e], e, (16 * nsub[e] + 3) / 4 * 4);
    }
    R->bs_words_wq = bsp_wq[E];
    R->bs_words_gq = bsp_gq[E];
    if (R->Q > INT32_MAX) return bail(fail(ctx, WQ_ERR_ARG, "too many points for 32-bit point indices"));
    std::vector<int32_t> wrow_dst(w_ptr[n]), pt_of_w(w_ptr[n]), scat(kptr[E]), gptr(R->nnz + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = w_ptr[i];
        for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
            const int32_t e = B.supp[s];
            for (int q = 0; q < side[e] * side[e]; ++q) {
                pt_of_w[r] = (int32_t)(pt_ptr[e] + q);
                wrow_dst[r++] = (int32_t)(wbase[e] + (int64_t)q * m[e] + il[s]);
            }
            for (int b = 0; b < m[e]; ++b) ++gptr[B.row_ptr[i] + pos[pos_ptr[s] + b] + 1];
        }
    }
    for (int64_t x = 0; x < R->nnz; ++x) gptr[x + 1] += gptr[x];
    {
        std::vector<int32_t> cur(gptr.begin(), gptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
                const int32_t e = B.supp[s];
                for (int b = 0; b < m[e]; ++b)
                    scat[kptr[e] + (int64_t)il[s] * m[e] + b] = cur[B.row_ptr[i] + pos[pos_ptr[s] + b]]++;
            }
    }
    R->kscr_len = kptr[E];
    // tile engine (k_tile.cu): element-major packs [component][point][16-row block][16]
    // per element (WQ test = split weights, WQ trial = split table, Gauss test = Gauss
    // weight x table, Gauss trial = split Gauss table), 16 x 16 tiles of every element
    // block (elements with more points and column blocks first), and the per-row sum plan
    std::vector<int32_t> Pw(E), Pg(E), rowslot(n + 1, 0), kdst(B.fn_ptr[E], 0);
    std::vector<uint16_t> pos2;
    std::vector<int64_t> sw_off(E + 1, 0), tw_off(E + 1, 0), sg_off(E + 1, 0), tg_off(E + 1, 0);
    std::vector<int4> ti_wq, ti_gq, tm_wq, tm_gq;
    std::vector<int64_t> tmx_off(E + 1, 0);
    R->tile_ok = true;
    for (int64_t e = 0; e < E; ++e) {
        const int ncb = (m[e] + 15) / 16;
        Pw[e] = side[e] * side[e];
        Pg[e] = 16 * nsub[e];
        if (ncb > 15 || Pw[e] > 255 || Pg[e] > 255) R->tile_ok = false;
        sw_off[e + 1] = sw_off[e] + (int64_t)R->nwc * Pw[e] * ncb * 16;
        tw_off[e + 1] = tw_off[e] + (int64_t)nc * Pw[e] * ncb * 16;
        sg_off[e + 1] = sg_off[e] + (int64_t)nc * Pg[e] * ncb * 16;
        tg_off[e + 1] = tg_off[e] + (int64_t)nc * Pg[e] * ncb * 16;
        tmx_off[e + 1] = tmx_off[e] + (int64_t)nc * ncb;
    }
    if (std::max({sw_off[E], tw_off[E], sg_off[E], tg_off[E]}) > INT32_MAX) R->tile_ok = false;
    if (opts->skip_plans & WQ_PLAN_NO_TILE) R->tile_ok = false;
    // row-major slot layout of the element blocks: row i's support entries in support
    // order, each ceil(m_e / 16) blocks of 16 slots; the slot block of (row i, element e)
    // receives element e's block row of function i (kdst), pos2 the positions in row i
    {
        int64_t ns = 0;
        for (int64_t i = 0; i < n && R->tile_ok; ++i) {
            rowslot[i] = (int32_t)ns;
            for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) ns += 16 * ((m[B.supp[s]] + 15) / 16);
            if (ns > INT32_MAX) R->tile_ok = false;
        }
        rowslot[n] = (int32_t)ns;
        R->kslot_len = ns;
        if (R->tile_ok) {
            pos2.assign((size_t)ns, (uint16_t)0xFFFF);
            for (int64_t i = 0; i < n; ++i) {
                int64_t x = rowslot[i];
                for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
                    const int32_t e = B.supp[s];
                    kdst[B.fn_ptr[e] + il[s]] = (int32_t)x;
                    for (int b = 0; b < m[e]; ++b) pos2[x + b] = pos[pos_ptr[s] + b];
                    x += 16 * ((m[e] + 15) / 16);
                }
            }
        }
    }
    if (R->tile_ok) {
        auto make_tiles = [&](bool gauss, std::vector<int4>& item, std::vector<int4>& meta) {
            const std::vector<int32_t>& P = gauss ? Pg : Pw;
            std::vector<int32_t> ord(E);
            for (int64_t e = 0; e < E; ++e) ord[e] = (int32_t)e;
            std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
                const int cx = (m[x] + 15) / 16, cy = (m[y] + 15) / 16;
                return (int64_t)P[x] * cx * cx > (int64_t)P[y] * cy * cy;
            });
            for (int32_t e : ord) {
                const int ncb = (m[e] + 15) / 16;
                for (int ta = 0; ta < ncb; ++ta)
                    for (int tb = 0; tb < ncb; ++tb) {
                        item.push_back(make_int4((int)(gauss ? sg_off[e] : sw_off[e]), (int)(gauss ? tg_off[e] : tw_off[e]),
                                                 (int)(gauss ? gp_ptr[e] : pt_ptr[e]), (int)B.fn_ptr[e]));
                        meta.push_back(make_int4(m[e] | P[e] << 8 | ta << 16 | tb << 20 | ncb << 24, 0,
                                                 (int)tmx_off[e], 0));
                    }
            }
        };
        make_tiles(false, ti_wq, tm_wq);
        make_tiles(true, ti_gq, tm_gq);
    }
    std::vector<int32_t> row_ptr32(n + 1);
    for (int64_t i = 0; i <= n; ++i) row_ptr32[i] = (int32_t)B.row_ptr[i];
    if (B.row_ptr[n] > INT32_MAX) return bail(fail(ctx, WQ_ERR_ARG, "nnz exceeds 32-bit row pointers"));

    // uploads
    if (!upload(R, R->d_m, m, sst) || !upload(R, R->d_nsub, nsub, sst) || !upload(R, R->d_side, side, sst) ||
        !upload(R, R->d_coef_ptr, B.coef_ptr, sst) || !upload(R, R->d_coef, B.coef, sst) ||
        !upload(R, R->d_sub_ptr, B.sub_ptr, sst) || !upload(R, R->d_geom, B.geom, sst) ||
        !upload(R, R->d_geom_ref, B.geom_ref, sst) ||
        !upload(R, R->d_pt_ptr, pt_ptr, sst) || !upload(R, R->d_gp_ptr, gp_ptr, sst) ||
        !upload(R, R->d_bt_ptr, bt_ptr, sst) || !upload(R, R->d_gbt_ptr, gbt_ptr, sst) ||
        !upload(R, R->d_pt_elem, pt_elem, sst) || !upload(R, R->d_gp_elem, gp_elem, sst) ||
        !upload(R, R->d_row_ptr, row_ptr32, sst) || !upload(R, R->d_col, B.col, sst) ||
        !upload(R, R->d_supp_ptr, B.supp_ptr, sst) || !upload(R, R->d_supp, B.supp, sst) ||
        !upload(R, R->d_pos_ptr, pos_ptr, sst) || !upload(R, R->d_pos, pos, sst) || !upload(R, R->d_il, il, sst) ||
        !upload(R, R->d_w_ptr, w_ptr, sst) || !upload(R, R->d_fn_ptr, B.fn_ptr, sst) ||
        !upload(R, R->d_order, order, sst) ||
        !upload(R, R->d_desc_gq, desc_gq, sst) || !upload(R, R->d_fns, B.fns, sst) ||
        !upload(R, R->d_it_wq, it_wq, sst) || !upload(R, R->d_kb_wq, kb_wq, sst) ||
        !upload(R, R->d_it_gq, it_gq, sst) || !upload(R, R->d_kb_gq, kb_gq, sst) ||
        !upload(R, R->d_wrow_dst, wrow_dst, sst) || !upload(R, R->d_scat, scat, sst) ||
        !upload(R, R->d_pt_of_w, pt_of_w, sst) ||
        !upload(R, R->d_gptr, gptr, sst) || !upload(R, R->d_tcel_wq, tcel_wq, sst) ||
        !upload(R, R->d_tcel_gq, tcel_gq, sst) || !upload(R, R->d_bsp_wq, bsp_wq, sst) ||
        !upload(R, R->d_bsp_gq, bsp_gq, sst) || !upload(R, R->d_it2_wq, it2_wq, sst) ||
        !upload(R, R->d_it2_gq, it2_gq, sst))
        return bail(sst);
    int32_t *d_Pw = nullptr, *d_Pg = nullptr;
    int64_t *d_sw_off = nullptr, *d_tw_off = nullptr, *d_sg_off = nullptr, *d_tg_off = nullptr, *d_wbase = nullptr;
    int64_t* d_tmx_off = nullptr;
    if (R->tile_ok &&
        (!upload(R, R->d_ti_wq, ti_wq, sst) || !upload(R, R->d_tm_wq, tm_wq, sst) ||
         !upload(R, R->d_ti_gq, ti_gq, sst) || !upload(R, R->d_tm_gq, tm_gq, sst) ||
         !upload(R, R->d_rowslot, rowslot, sst) || !upload(R, R->d_kdst, kdst, sst) ||
         !upload(R, R->d_pos2, pos2, sst) || !dalloc(R, R->d_kslot, (size_t)std::max<int64_t>(R->kslot_len, 1), sst) ||
         !upload(R, d_Pw, Pw, sst) || !upload(R, d_Pg, Pg, sst) || !upload(R, d_sw_off, sw_off, sst) ||
         !upload(R, d_tw_off, tw_off, sst) || !upload(R, d_sg_off, sg_off, sst) || !upload(R, d_tg_off, tg_off, sst) ||
         !upload(R, d_wbase, wbase, sst) || !upload(R, d_tmx_off, tmx_off, sst) ||
         !dalloc(R, R->d_tmx_wq, (size_t)tmx_off[E], sst) || !dalloc(R, R->d_tmx_gq, (size_t)tmx_off[E], sst) ||
         !dalloc(R, R->d_pk_sw, (size_t)sw_off[E], sst) ||
         !dalloc(R, R->d_pk_tw, (size_t)tw_off[E], sst) || !dalloc(R, R->d_pk_sg, (size_t)sg_off[E], sst) ||
         !dalloc(R, R->d_pk_tg, (size_t)tg_off[E], sst)))
        return bail(sst);
    if (R->tc_ok &&
        (!dalloc(R, R->d_bs_wq, (size_t)bsp_wq[E], sst) || !dalloc(R, R->d_bs_gq, (size_t)bsp_gq[E], sst) ||
         !dalloc(R, R->d_fexp_wq, (size_t)E * nc, sst) || !dalloc(R, R->d_fexp_gq, (size_t)E * nc, sst) ||
         !dalloc(R, R->d_vmax_wq, (size_t)B.fn_ptr[E] * R->nwc, sst) ||
         !dalloc(R, R->d_vmax_gq, (size_t)B.fn_ptr[E] * nc, sst) || !dalloc(R, R->d_gw2, (size_t)R->G, sst)))
        return bail(sst);
    if (!dalloc(R, R->d_table, (size_t)bt_ptr[E], sst) || !dalloc(R, R->d_gtable, (size_t)gbt_ptr[E], sst) ||
        !dalloc(R, R->d_x, (size_t)R->Q * 3, sst) || !dalloc(R, R->d_gx, (size_t)R->G * 3, sst) ||
        !dalloc(R, R->d_gw, (size_t)R->G, sst) || !dalloc(R, R->d_W, (size_t)R->sum_r * R->nwc, sst) ||
        !dalloc(R, R->d_status, 1, sst) || !dalloc(R, R->d_table2, (size_t)bt_ptr[E], sst) ||
        !dalloc(R, R->d_gtable2, (size_t)gbt_ptr[E], sst) ||
        !dalloc(R, R->d_W2, (size_t)R->sum_r * R->nwc, sst) || !dalloc(R, R->d_We, (size_t)R->sum_r * R->nwc, sst) ||
        !dalloc(R, R->d_coef_stage, (size_t)R->Q, sst) ||
        !dalloc(R, R->d_vals_stage, (size_t)R->nnz, sst) ||
        !dalloc(R, R->d_kscr, (size_t)std::max<int64_t>(R->kscr_len, 1), sst))
        return bail(sst);
    for (int c = 0; c < 5; ++c)
        if (R->wcidx[c] >= 0 && !dalloc(R, R->d_mom[c], (size_t)R->nnz, sst)) return bail(sst);
    const int64_t nw = std::max(R->nwc, 1);
    if (!dalloc(R, bs.d_rank, (size_t)(n * nw), sst) || !dalloc(R, bs.d_zid, (size_t)(n * nw), sst) ||
        !dalloc(R, bs.d_flops, 1, sst))
        return bail(sst);
    // weight-solve scratch per CTA (allocated by the solve, freed after it)
    const int64_t mn = R->max_n_i, mr = R->max_r;
    bs.per_cta = wqd::tsvd_scratch_doubles(mn, mr);
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
    R->n_sm = std::max(n_sm, 1);
    bs.st = st;
    bs.tol = tol;
    bs.sweeps = sweeps;
    bs.saved = saved;
    bs.d_Pw = d_Pw;
    bs.d_Pg = d_Pg;
    bs.d_sw_off = d_sw_off;
    bs.d_tw_off = d_tw_off;
    bs.d_sg_off = d_sg_off;
    bs.d_tg_off = d_tg_off;
    bs.d_wbase = d_wbase;
    bs.d_tmx_off = d_tmx_off;
    bs.bt_E = bt_ptr[E];
    bs.gbt_E = gbt_ptr[E];

    wqd::Elems& el = R->el;
    el.dim = B.dim;
    el.nc = nc;
    el.E = E;
    el.m = R->d_m;
    el.nsub = R->d_nsub;
    el.side = R->d_side;
    el.coef_ptr = R->d_coef_ptr;
    el.coef = R->d_coef;
    el.sub_ptr = R->d_sub_ptr;
    el.geom = R->d_geom;
    el.geom_ref = R->d_geom_ref;
    el.pt_ptr = R->d_pt_ptr;
    el.gp_ptr = R->d_gp_ptr;
    el.bt_ptr = R->d_bt_ptr;
    el.gbt_ptr = R->d_gbt_ptr;
    wqd::Rows& rw = R->rw;
    rw.n = n;
    rw.row_ptr = R->d_row_ptr;
    rw.supp_ptr = R->d_supp_ptr;
    rw.supp = R->d_supp;
    rw.pos_ptr = R->d_pos_ptr;
    rw.pos = R->d_pos;
    rw.il = R->d_il;
    rw.w_ptr = R->d_w_ptr;
    rw.order = R->d_order;
    R->it_wq = {(int64_t)it_wq.size(), R->d_it_wq, R->d_kb_wq};
    R->it_gq = {(int64_t)it_gq.size(), R->d_it_gq, R->d_kb_gq};
    R->ep = {R->d_scat, R->d_gptr, R->d_kscr};
    R->src_wq = {R->ep, R->d_table2, R->d_W2, nullptr, R->nnz, nc, R->nwc};
    R->src_gq = {R->ep, R->d_gtable2, nullptr, R->d_gw, R->nnz, nc, R->nwc};
    R->src64_wq = {R->d_scat, R->d_gptr, reinterpret_cast<double*>(R->d_kscr), R->d_table, R->d_We, nullptr, R->nnz,
                   nc, R->nwc};
    R->src64_gq = {R->d_scat, R->d_gptr, reinterpret_cast<double*>(R->d_kscr), R->d_gtable, nullptr, R->d_gw, R->nnz,
                   nc, R->nwc};
    R->tc_wq = {R->d_scat, R->d_kscr, R->d_gptr, R->d_W2, nullptr, R->d_bs_wq, R->d_fexp_wq, R->d_vmax_wq,
                R->nnz, nc, R->nwc};
    R->tc_gq = {R->d_scat, R->d_kscr, R->d_gptr, R->d_gtable2, R->d_gw2, R->d_bs_gq, R->d_fexp_gq, R->d_vmax_gq,
                R->nnz, nc, R->nwc};
    R->tit_wq = {(int64_t)it_wq.size(), R->d_it_wq, R->d_kb_wq, R->d_it2_wq, R->n_sm};
    R->tit_gq = {(int64_t)it_gq.size(), R->d_it_gq, R->d_kb_gq, R->d_it2_gq, R->n_sm};
    R->h_it_wq = it_wq;
    R->h_kb_wq = kb_wq;
    if (R->tile_ok) {
        R->tj_wq = {(int64_t)ti_wq.size(), R->d_ti_wq, R->d_tm_wq, {R->d_pk_sw, R->d_pk_tw, R->d_kslot, R->d_kdst, R->d_tmx_wq, R->nwc, nc},
                    nullptr, R->d_status};
        R->tj_gq = {(int64_t)ti_gq.size(), R->d_ti_gq, R->d_tm_gq, {R->d_pk_sg, R->d_pk_tg, R->d_kslot, R->d_kdst, R->d_tmx_gq, nc, nc},
                    nullptr, R->d_status};
        R->rsrc = {n, R->d_row_ptr, R->d_rowslot, R->d_pos2, R->d_kslot, R->max_n_i};
        R->h_ti_wq = ti_wq;
        R->h_tm_wq = tm_wq;
    }

    // Gauss-Legendre 4-point rule on [0, 1] (closed form)
    {
        const double s = 2.0 / 7.0 * std::sqrt(6.0 / 5.0);
        const double t[4] = {-std::sqrt(3.0 / 7.0 + s), -std::sqrt(3.0 / 7.0 - s), std::sqrt(3.0 / 7.0 - s),
                             std::sqrt(3.0 / 7.0 + s)};
        const double w[4] = {(18 - std::sqrt(30.0)) / 36, (18 + std::sqrt(30.0)) / 36, (18 + std::sqrt(30.0)) / 36,
                             (18 - std::sqrt(30.0)) / 36};
        double x[4], ww[4];
        for (int k = 0; k < 4; ++k) {
            x[k] = 0.5 * (t[k] + 1.0);
            ww[k] = 0.5 * w[k];
        }
        wqd::set_gauss_constants(x, ww);
    }
    if (R->tile_ok) {
        cudaError_t pe = wqd::prepare_tile_kernels();
        if (pe != cudaSuccess) return bail(fail(ctx, WQ_ERR_CUDA, std::string("tile kernels: ") + cudaGetErrorString(pe)));
    }
    if (cudaEventCreate(&bs.ev0) != cudaSuccess || cudaEventCreate(&bs.ev1) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(ctx, WQ_ERR_CUDA, "rule build: event creation failed"));
    }
    cudaError_t ce = cudaEventRecord(bs.ev0, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(R->d_status, 0, sizeof(unsigned), st);
    // a2 + a3: placement and basis tables at WQ and Gauss points
    if (ce == cudaSuccess)
        ce = wqd::launch_eval(el, R->d_pt_elem, R->Q, 0, R->d_table, R->d_x, nullptr, R->d_status, st);
    if (ce == cudaSuccess)
        ce = wqd::launch_eval(el, R->d_gp_elem, R->G, 1, R->d_gtable, R->d_gx, R->d_gw, R->d_status, st);
    // a4: Gauss moments per component (c = 1)
    for (int c = 0; c < 5 && ce == cudaSuccess && !saved; ++c) {
        if (R->wcidx[c] < 0) continue;
        ce = wqd::launch_moments_f64(rw, R->d_desc_gq, table_comp(R, c), nc, R->d_gtable, R->d_gw, R->d_mom[c],
                                     R->max_n_i, st);
    }
    if (ce != cudaSuccess) return bail(fail(ctx, WQ_ERR_CUDA, std::string("rule build: ") + cudaGetErrorString(ce)));
    *out = R;
    return WQ_OK;
}

// Weight statistics (truncated systems, Z = I fallbacks) of every built component from
// the per-row ranks and flags the solves wrote; waits for the build stream.
static cudaError_t weight_stats(wq_rule* R, BuildState& bs) {
    const int64_t n = R->n;
    const wqi::BasisHost& B = R->basis->B;
    std::vector<int32_t> rank(n);
    std::vector<uint8_t> zid(n);
    for (int c = 0; c < 5; ++c) {
        if (R->wcidx[c] < 0) continue;
        const int64_t k = R->wcidx[c];
        cudaError_t ce = cudaSuccess;
        if (n > 0) {
            ce = cudaMemcpyAsync(rank.data(), bs.d_rank + k * n, n * sizeof(int32_t), cudaMemcpyDeviceToHost, bs.st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(zid.data(), bs.d_zid + k * n, n, cudaMemcpyDeviceToHost, bs.st);
        }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(bs.st);
        if (ce != cudaSuccess) return ce;
        int trunc = 0, zcount = 0;
        for (int64_t i = 0; i < n; ++i) {
            trunc += rank[i] < (B.row_ptr[i + 1] - B.row_ptr[i]);
            zcount += zid[i];
        }
        R->info.n_truncated[c] = trunc;
        R->info.n_z_identity[c] = zcount;
    }
    return cudaSuccess;
}

// a5 for one rule: the truncated-SVD weights of every built component, one launch per
// component (timed, FP64 operations counted); the scratch lives for the solves only.
static wq_status rule_weights_single(wq_rule* R, BuildState& bs) {
    wq_ctx* ctx = R->ctx;
    const int n_cta = (int)std::min<int64_t>(R->n, (int64_t)R->n_sm * wqd::TSVD_CTAS_PER_SM);
    double* d_scratch = nullptr;
    if (n_cta > 0 && cudaMalloc(&d_scratch, (size_t)bs.per_cta * n_cta * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, WQ_ERR_OOM, "weight-solve scratch allocation failed");
    }
    cudaEvent_t evt0 = nullptr, evt1 = nullptr;
    cudaError_t ce = cudaMemsetAsync(bs.d_flops, 0, sizeof(double), bs.st);
    if (ce == cudaSuccess) ce = cudaEventCreate(&evt0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&evt1);
    if (ce == cudaSuccess) ce = cudaEventRecord(evt0, bs.st);
    for (int c = 0; c < 5 && ce == cudaSuccess; ++c) {
        if (R->wcidx[c] < 0) continue;
        const int64_t k = R->wcidx[c];
        ce = wqd::launch_tsvd(R->el, R->rw, R->d_table, table_comp(R, c), R->d_mom[c], R->d_W, R->nwc, (int)k, bs.tol,
                              bs.sweeps, d_scratch, bs.per_cta, n_cta, bs.d_rank + k * R->n, bs.d_zid + k * R->n,
                              R->d_status, bs.d_flops, bs.st);
    }
    double fl = 0.0;
    float tms = 0.0f;
    if (ce == cudaSuccess) ce = cudaEventRecord(evt1, bs.st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&fl, bs.d_flops, sizeof(double), cudaMemcpyDeviceToHost, bs.st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(bs.st);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&tms, evt0, evt1);
    if (evt0) cudaEventDestroy(evt0);
    if (evt1) cudaEventDestroy(evt1);
    if (d_scratch) cudaFree(d_scratch);   // after the synchronisation (cudaFree waits itself otherwise)
    if (ce == cudaSuccess) ce = weight_stats(R, bs);
    if (ce != cudaSuccess) return fail(ctx, WQ_ERR_CUDA, std::string("weight solves: ") + cudaGetErrorString(ce));
    R->info.tsvd_ms = tms;
    R->info.tsvd_gflop = fl * 1e-9;
    return WQ_OK;
}

// Last phase: saved weights (loaded rule), FP32 split copies, element-major packs,
// tensor-core plan; waits for the build stream and reads the device status.
static wq_status rule_finish(wq_rule* R, BuildState& bs) {
    wq_ctx* ctx = R->ctx;
    const SavedRule* saved = bs.saved;
    cudaStream_t st = bs.st;
    const int64_t E = R->E;
    const int nc = R->nc;
    cudaError_t ce = cudaSuccess;
    if (saved) {
        // weights and moments from the file (host buffers live until the synchronisation below)
        ce = cudaMemcpyAsync(R->d_W, saved->W.data(), saved->W.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        int k = 0;
        for (int c = 0; c < 5 && ce == cudaSuccess; ++c) {
            if (R->wcidx[c] < 0) continue;
            ce = cudaMemcpyAsync(R->d_mom[c], saved->mom[k].data(), saved->mom[k].size() * sizeof(double),
                                 cudaMemcpyHostToDevice, st);
            ++k;
        }
        for (int c = 0; c < 5; ++c) {
            R->info.n_truncated[c] = saved->n_truncated[c];
            R->info.n_z_identity[c] = saved->n_z_identity[c];
        }
    }
    // FP32 split copies for the mixed-precision assembly
    if (ce == cudaSuccess) ce = wqd::launch_split_f32(R->d_table, R->d_table2, bs.bt_E, st);
    if (ce == cudaSuccess) ce = wqd::launch_split_f32(R->d_gtable, R->d_gtable2, bs.gbt_E, st);
    if (ce == cudaSuccess) ce = wqd::launch_split_rows(R->d_W, R->d_wrow_dst, R->d_W2, R->sum_r, R->nwc, R->n_sm, st);
    if (ce == cudaSuccess) ce = wqd::launch_copy_rows(R->d_W, R->d_wrow_dst, R->d_We, R->sum_r, R->nwc, R->n_sm, st);
    // element-major packs of the tile engine
    if (R->tile_ok) {
        wqd::PackJob pj{};
        pj.E = E;
        pj.m = R->d_m;
        pj.nc = nc;
        pj.nwc = R->nwc;
        pj.kind = wqd::PK_W2E;   // WQ test side: the split weights
        pj.ncomp = R->nwc;
        pj.P = bs.d_Pw;
        pj.src_off = bs.d_wbase;
        pj.out_off = bs.d_sw_off;
        pj.f2 = R->d_W2;
        pj.out = R->d_pk_sw;
        if (ce == cudaSuccess) ce = wqd::launch_pack(pj, st);
        pj.kind = wqd::PK_TABLE2;   // WQ trial side: the split table
        pj.ncomp = nc;
        pj.src_off = R->d_bt_ptr;
        pj.out_off = bs.d_tw_off;
        pj.f2 = R->d_table2;
        pj.out = R->d_pk_tw;
        if (ce == cudaSuccess) ce = wqd::launch_pack(pj, st);
        if (ce == cudaSuccess) ce = wqd::launch_pack_max(pj, bs.d_tmx_off, R->d_tmx_wq, st);
        pj.kind = wqd::PK_GAUSS;   // Gauss test side: Gauss weight x table, split
        pj.P = bs.d_Pg;
        pj.src_off = R->d_gbt_ptr;
        pj.out_off = bs.d_sg_off;
        pj.f64 = R->d_gtable;
        pj.gw = R->d_gw;
        pj.pt0 = R->d_gp_ptr;
        pj.out = R->d_pk_sg;
        if (ce == cudaSuccess) ce = wqd::launch_pack(pj, st);
        pj.kind = wqd::PK_TABLE2;   // Gauss trial side: the split Gauss table
        pj.pt0 = nullptr;
        pj.out_off = bs.d_tg_off;
        pj.f2 = R->d_gtable2;
        pj.out = R->d_pk_tg;
        if (ce == cudaSuccess) ce = wqd::launch_pack(pj, st);
        if (ce == cudaSuccess) ce = wqd::launch_pack_max(pj, bs.d_tmx_off, R->d_tmx_gq, st);
    }
    // trial-side slices and test-side bounds of the tensor-core contraction
    if (R->tc_ok) {
        if (ce == cudaSuccess) ce = wqd::launch_split_f32(R->d_gw, R->d_gw2, R->G, st);
        if (ce == cudaSuccess)
            ce = wqd::launch_tc_prep(E, nc, R->nwc, R->d_m, R->d_table, R->d_We,
                                     {R->d_tcel_wq, R->d_bsp_wq, R->d_bs_wq, R->d_fexp_wq, R->d_vmax_wq}, st);
        if (ce == cudaSuccess)
            ce = wqd::launch_tc_prep(E, nc, R->nwc, R->d_m, R->d_gtable, nullptr,
                                     {R->d_tcel_gq, R->d_bsp_gq, R->d_bs_gq, R->d_fexp_gq, R->d_vmax_gq}, st);
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(bs.ev1, st);
    unsigned hstat = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hstat, R->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return fail(ctx, WQ_ERR_CUDA, std::string("rule build: ") + cudaGetErrorString(ce));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, bs.ev0, bs.ev1);
    wq_status s2 = status_to_error(ctx, hstat);
    if (s2 != WQ_OK) return s2;
    R->info.n_points = R->Q;
    R->info.n_gauss = R->G;
    R->info.sum_r = R->sum_r;
    R->info.max_r = R->max_r;
    R->info.setup_ms = ms;
    return WQ_OK;
}

static wq_status rule_build_impl(wq_basis* basis, const wq_rule_opts* opts, const SavedRule* saved, wq_rule** out) {
    BuildState bs;
    wq_rule* R = nullptr;
    wq_status s = rule_prepare(basis, opts, saved, &R, bs);
    if (s != WQ_OK) return s;
    if (!saved) s = rule_weights_single(R, bs);
    if (s == WQ_OK) s = rule_finish(R, bs);
    if (s != WQ_OK) {
        delete R;
        return s;
    }
    *out = R;
    return WQ_OK;
}

wq_status wq_rule_build(wq_basis* basis, const wq_rule_opts* opts, wq_rule** out) {
    return rule_build_impl(basis, opts, nullptr, out);
}

wq_status wq_rule_build_batched(int32_t k, wq_basis* const* bases, const wq_rule_opts* opts, wq_rule** out) {
    drop_stale_error();
    if (!bases || !opts || !out || k < 1) return WQ_ERR_ARG;
    for (int r = 0; r < k; ++r) out[r] = nullptr;
    for (int r = 0; r < k; ++r)
        if (!bases[r]) return WQ_ERR_ARG;
    wq_ctx* ctx = bases[0]->ctx;
    for (int r = 0; r < k; ++r)
        if (bases[r]->ctx->device != ctx->device)
            return fail(ctx, WQ_ERR_ARG, "batched rule build: the bases must share the device");
    std::vector<BuildState> bs(k);
    std::vector<wq_rule*> R(k, nullptr);
    auto release = [&](wq_status s) {
        for (wq_rule*& x : R) {
            delete x;
            x = nullptr;
        }
        return s;
    };
    for (int r = 0; r < k; ++r) {
        wq_status s = rule_prepare(bases[r], opts, nullptr, &R[r], bs[r]);
        if (s != WQ_OK) return release(s);
    }
    // one job per (rule, built component, row), the rows with the most Jacobi work first
    std::vector<wqd::TsvdSet> sets;
    std::vector<int2> jobs;
    std::vector<double> cost;
    int64_t per_cta = 1;
    for (int r = 0; r < k; ++r) {
        wq_rule* Q = R[r];
        if (Q->n > INT32_MAX) return release(fail(ctx, WQ_ERR_ARG, "batched rule build: too many rows in one rule"));
        per_cta = std::max(per_cta, bs[r].per_cta);
        for (int c = 0; c < 5; ++c) {
            if (Q->wcidx[c] < 0) continue;
            const int64_t kk = Q->wcidx[c];
            const int set = (int)sets.size();
            sets.push_back({Q->el, Q->rw, Q->d_table, table_comp(Q, c), Q->d_mom[c], Q->d_W, Q->nwc, (int)kk,
                            bs[r].d_rank + kk * Q->n, bs[r].d_zid + kk * Q->n, Q->d_status});
            for (int64_t i = 0; i < Q->n; ++i) {
                jobs.push_back(make_int2(set, (int)i));
                cost.push_back(bs[r].row_cost[i]);
            }
        }
    }
    {
        std::vector<int64_t> ord(jobs.size());
        for (size_t j = 0; j < ord.size(); ++j) ord[j] = (int64_t)j;
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
        std::vector<int2> sorted(jobs.size());
        for (size_t j = 0; j < ord.size(); ++j) sorted[j] = jobs[ord[j]];
        jobs.swap(sorted);
    }
    cudaStream_t st = (cudaStream_t)opts->stream;
    const int n_sm = R[0]->n_sm;
    const int n_cta = (int)std::min<int64_t>((int64_t)jobs.size(), (int64_t)n_sm * wqd::TSVD_CTAS_PER_SM);
    wqd::TsvdSet* d_sets = nullptr;
    int2* d_jobs = nullptr;
    unsigned long long* d_next = nullptr;
    double *d_flops = nullptr, *d_scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto free_tmp = [&]() {
        if (d_sets) cudaFree(d_sets);
        if (d_jobs) cudaFree(d_jobs);
        if (d_next) cudaFree(d_next);
        if (d_flops) cudaFree(d_flops);
        if (d_scratch) cudaFree(d_scratch);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&d_sets, std::max<size_t>(sets.size(), 1) * sizeof(wqd::TsvdSet)) != cudaSuccess ||
        cudaMalloc(&d_jobs, std::max<size_t>(jobs.size(), 1) * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&d_next, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&d_flops, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d_scratch, (size_t)per_cta * std::max(n_cta, 1) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        free_tmp();
        return release(fail(ctx, WQ_ERR_OOM, "batched rule build: weight-solve buffers"));
    }
    double fl = 0.0;
    float tms = 0.0f;
    cudaError_t ce = cudaMemcpyAsync(d_sets, sets.data(), sets.size() * sizeof(wqd::TsvdSet), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess && !jobs.empty())
        ce = cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(d_flops, 0, sizeof(double), st);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, st);
    if (ce == cudaSuccess)
        ce = wqd::launch_tsvd_batch(d_sets, d_jobs, (int64_t)jobs.size(), d_next, bs[0].tol, bs[0].sweeps, d_scratch,
                                    per_cta, n_cta, d_flops, st);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&fl, d_flops, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&tms, e0, e1);
    free_tmp();
    if (ce != cudaSuccess)
        return release(fail(ctx, WQ_ERR_CUDA, std::string("batched weight solves: ") + cudaGetErrorString(ce)));
    for (int r = 0; r < k; ++r) {
        R[r]->info.tsvd_ms = tms;
        R[r]->info.tsvd_gflop = fl * 1e-9;
        ce = weight_stats(R[r], bs[r]);
        if (ce != cudaSuccess)
            return release(fail(ctx, WQ_ERR_CUDA, std::string("batched weight solves: ") + cudaGetErrorString(ce)));
        wq_status s = rule_finish(R[r], bs[r]);
        if (s != WQ_OK) return release(s);
    }
    for (int r = 0; r < k; ++r) out[r] = R[r];
    return WQ_OK;
}

wq_status wq_rule_save(const wq_rule* rule, const char* path) {
    if (!rule || !path) return WQ_ERR_ARG;
    wq_ctx* ctx = rule->ctx;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    RuleFileHeader h{};
    std::memcpy(h.magic, kRuleMagic, 8);
    h.version = 1;
    h.comps = rule->comps;
    h.count_mode = rule->count_mode;
    h.max_sweeps = rule->max_sweeps;
    h.tol = rule->tol;
    h.n = rule->n;
    h.E = rule->E;
    h.nnz = rule->nnz;
    h.Q = rule->Q;
    h.G = rule->G;
    h.sum_r = rule->sum_r;
    h.nwc = rule->nwc;
    h.dim = rule->dim;
    h.fingerprint = basis_fingerprint(rule->basis->B);
    for (int c = 0; c < 5; ++c) {
        h.n_truncated[c] = rule->info.n_truncated[c];
        h.n_z_identity[c] = rule->info.n_z_identity[c];
    }
    h.setup_ms = rule->info.setup_ms;
    std::vector<double> buf((size_t)rule->sum_r * rule->nwc);
    CUDA_TRY(ctx, cudaMemcpy(buf.data(), rule->d_W, buf.size() * sizeof(double), cudaMemcpyDeviceToHost));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(ctx, WQ_ERR_ARG, std::string("cannot open for writing: ") + path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
    std::vector<double> mb((size_t)rule->nnz);
    for (int c = 0; c < 5 && ok; ++c) {
        if (rule->wcidx[c] < 0) continue;
        if (cudaMemcpy(mb.data(), rule->d_mom[c], mb.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(f);
            return fail(ctx, WQ_ERR_CUDA, "copying the moments failed");
        }
        ok = std::fwrite(mb.data(), sizeof(double), mb.size(), f) == mb.size();
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(ctx, WQ_ERR_ARG, std::string("write failed: ") + path);
    return WQ_OK;
}

wq_status wq_rule_load(wq_basis* basis, const char* path, wq_rule** out) {
    if (!basis || !path || !out) return WQ_ERR_ARG;
    *out = nullptr;
    wq_ctx* ctx = basis->ctx;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ctx, WQ_ERR_ARG, std::string("cannot open: ") + path);
    RuleFileHeader h{};
    auto close_fail = [&](const std::string& msg) {
        std::fclose(f);
        return fail(ctx, WQ_ERR_ARG, msg);
    };
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kRuleMagic, 8) != 0 || h.version != 1)
        return close_fail("not a WQ rule file (version 1)");
    const wqi::BasisHost& B = basis->B;
    if (h.fingerprint != basis_fingerprint(B) || h.n != B.n || h.E != B.E || h.dim != B.dim ||
        h.nnz != B.row_ptr[B.n])
        return close_fail("rule file was saved for a different mesh");
    if ((h.comps & ~31u) || h.comps == 0 || h.nwc < 1 || h.nwc > 5 || h.sum_r < 0)
        return close_fail("corrupt rule file header");
    SavedRule sv;
    sv.W.resize((size_t)h.sum_r * h.nwc);
    if (std::fread(sv.W.data(), sizeof(double), sv.W.size(), f) != sv.W.size()) return close_fail("truncated rule file");
    for (int c = 0; c < 5; ++c)
        if (h.comps & (1u << c)) {
            sv.mom.emplace_back((size_t)h.nnz);
            if (std::fread(sv.mom.back().data(), sizeof(double), (size_t)h.nnz, f) != (size_t)h.nnz)
                return close_fail("truncated rule file");
        }
    std::fclose(f);
    for (int c = 0; c < 5; ++c) {
        sv.n_truncated[c] = h.n_truncated[c];
        sv.n_z_identity[c] = h.n_z_identity[c];
    }
    sv.setup_ms = h.setup_ms;
    wq_rule_opts opts{};
    opts.comps = h.comps;
    opts.count_mode = h.count_mode;
    opts.tsvd_rel_tol = h.tol;
    opts.max_sweeps = h.max_sweeps;
    opts.stream = nullptr;
    wq_rule* R = nullptr;
    wq_status s = rule_build_impl(basis, &opts, &sv, &R);
    if (s != WQ_OK) return s;
    if (R->sum_r != h.sum_r || R->Q != h.Q || R->G != h.G) {
        wq_rule_destroy(R);
        return fail(ctx, WQ_ERR_ARG, "rule file does not match the rebuilt point plan");
    }
    *out = R;
    return WQ_OK;
}

void wq_rule_destroy(wq_rule* rule) {
    // the rule keeps its device id: its context may already be gone (any destruction order)
    if (!rule) return;
    if (rule->device >= 0 && cudaSetDevice(rule->device) != cudaSuccess) cudaGetLastError();
    delete rule;
    cudaGetLastError();   // nothing of a teardown is reported through a later call
}

wq_status wq_rule_info_get(const wq_rule* rule, wq_rule_info* info) {
    if (!rule || !info) return WQ_ERR_ARG;
    *info = rule->info;
    return WQ_OK;
}

wq_status wq_rule_points(const wq_rule* rule, const double** d_x, int64_t* n_points) {
    if (!rule) return WQ_ERR_ARG;
    if (d_x) *d_x = rule->d_x;
    if (n_points) *n_points = rule->Q;
    return WQ_OK;
}

wq_status wq_rule_gauss_points(const wq_rule* rule, const double** d_x, int64_t* n_gauss) {
    if (!rule) return WQ_ERR_ARG;
    if (d_x) *d_x = rule->d_gx;
    if (n_gauss) *n_gauss = rule->G;
    return WQ_OK;
}

wq_status wq_pattern(const wq_rule* rule, int64_t* n, int64_t* nnz, const int32_t** d_row_ptr, const int32_t** d_col) {
    if (!rule) return WQ_ERR_ARG;
    if (n) *n = rule->n;
    if (nnz) *nnz = rule->nnz;
    if (d_row_ptr) *d_row_ptr = rule->d_row_ptr;
    if (d_col) *d_col = rule->d_col;
    return WQ_OK;
}

wq_status wq_rule_weights(const wq_rule* rule, int32_t comp, const double** d_w, const int64_t** d_w_ptr) {
    if (!rule || comp < 0 || comp > 4 || rule->wcidx[comp] < 0)
        return fail(rule ? rule->ctx : nullptr, WQ_ERR_ARG, "component not built");
    // the weights of all components are interleaved; expose the base of this one (stride nwc)
    if (d_w) *d_w = rule->d_W + rule->wcidx[comp];
    if (d_w_ptr) *d_w_ptr = rule->d_w_ptr;
    return WQ_OK;
}

wq_status wq_rule_table(const wq_rule* rule, int32_t gauss, const double** d_table, const int64_t** d_off,
                        const int64_t** d_pt_ptr, const double** d_gw, int32_t* ncomp) {
    if (!rule) return WQ_ERR_ARG;
    if (d_table) *d_table = gauss ? rule->d_gtable : rule->d_table;
    if (d_off) *d_off = gauss ? rule->d_gbt_ptr : rule->d_bt_ptr;
    if (d_pt_ptr) *d_pt_ptr = gauss ? rule->d_gp_ptr : rule->d_pt_ptr;
    if (d_gw) *d_gw = gauss ? rule->d_gw : nullptr;
    if (ncomp) *ncomp = rule->nc;
    return WQ_OK;
}

wq_status wq_moments(const wq_rule* rule, int32_t comp, double* d_vals, void* stream) {
    drop_stale_error();
    if (!rule || !d_vals || comp < 0 || comp > 4 || !rule->d_mom[comp])
        return fail(rule ? rule->ctx : nullptr, WQ_ERR_ARG, "component not built");
    CUDA_TRY(rule->ctx, cudaMemcpyAsync(d_vals, rule->d_mom[comp], rule->nnz * sizeof(double),
                                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return WQ_OK;
}

wq_status wq_assemble(const wq_rule* rule, int32_t op, const void* d_coef, double alpha, int32_t prec, void* d_vals,
                      void* stream) {
    drop_stale_error();
    if (!rule || !d_vals) return WQ_ERR_ARG;
    wqd::Terms tm;
    if (!op_terms(rule, op, alpha, true, tm, rule->Q))
        return fail(rule->ctx, WQ_ERR_ARG, "operator needs weight sets that this rule did not build");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (prec == WQ_PREC_AUTO) prec = rule->auto_prec[op][0];
    if (prec != WQ_PREC_F64 && prec != WQ_PREC_F32 && prec != WQ_PREC_F32_FAST && prec != WQ_PREC_TC)
        return fail(rule->ctx, WQ_ERR_ARG, "unknown precision");
    if (prec == WQ_PREC_TC && !rule->tc_ok)
        return fail(rule->ctx, WQ_ERR_ARG, "WQ_PREC_TC: this rule has no tensor-core plan (an element with more than 64 points, or WQ_PLAN_NO_TC)");
    cudaEvent_t* evs = rule->next_timing_events();
    if (prec == WQ_PREC_F64)
        e = wqd::launch_elem_f64(rule->it_wq, rule->src64_wq, tm, 0, (const double*)d_coef, (double*)d_vals, st, evs);
    else if (prec == WQ_PREC_TC)
        e = wqd::launch_elem_tc(rule->tit_wq, rule->tc_wq, tm, 0, (const double*)d_coef, (float*)d_vals, st, evs);
    else if (wqd::TileTerms tt; float_variant(rule, op, 0) != WQ_VARIANT_SLOTMAP && rule->tile_ok &&
                                    tile_terms(tm, false, tt))
        e = wqd::launch_tile_f32(rule->tj_wq, rule->rsrc, tt, (const double*)d_coef, (float*)d_vals,
                                 prec == WQ_PREC_F32, float_variant(rule, op, 0), rule->n_sm, st, evs);
    else
        e = wqd::launch_elem_f32(rule->it_wq, rule->src_wq, tm, 0, (const double*)d_coef, (float*)d_vals,
                                 prec == WQ_PREC_F32, st, evs);
    if (e != cudaSuccess) return fail(rule->ctx, WQ_ERR_CUDA, std::string("assembly launch: ") + cudaGetErrorString(e));
    return WQ_OK;
}

wq_status wq_gq_assemble(const wq_rule* rule, int32_t op, const void* d_coef, double alpha, int32_t prec,
                         void* d_vals, void* stream) {
    drop_stale_error();
    if (!rule || !d_vals) return WQ_ERR_ARG;
    wqd::Terms tm;
    if (!op_terms(rule, op, alpha, false, tm, rule->G)) return fail(rule->ctx, WQ_ERR_ARG, "unknown operator");
    cudaError_t e;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == WQ_PREC_AUTO) prec = rule->auto_prec[op][1];
    if (prec != WQ_PREC_F64 && prec != WQ_PREC_F32 && prec != WQ_PREC_F32_FAST && prec != WQ_PREC_TC)
        return fail(rule->ctx, WQ_ERR_ARG, "unknown precision");
    if (prec == WQ_PREC_TC && !rule->tc_ok)
        return fail(rule->ctx, WQ_ERR_ARG, "WQ_PREC_TC: this rule has no tensor-core plan (an element with more than 64 points, or WQ_PLAN_NO_TC)");
    cudaEvent_t* evs = rule->next_timing_events();
    if (prec == WQ_PREC_F64)
        e = wqd::launch_elem_f64(rule->it_gq, rule->src64_gq, tm, 1, (const double*)d_coef, (double*)d_vals, st, evs);
    else if (prec == WQ_PREC_TC)
        e = wqd::launch_elem_tc(rule->tit_gq, rule->tc_gq, tm, 1, (const double*)d_coef, (float*)d_vals, st, evs);
    else if (wqd::TileTerms tt; float_variant(rule, op, 1) != WQ_VARIANT_SLOTMAP && rule->tile_ok &&
                                    tile_terms(tm, true, tt))
        e = wqd::launch_tile_f32(rule->tj_gq, rule->rsrc, tt, (const double*)d_coef, (float*)d_vals,
                                 prec == WQ_PREC_F32, float_variant(rule, op, 1), rule->n_sm, st, evs);
    else
        e = wqd::launch_elem_f32(rule->it_gq, rule->src_gq, tm, 1, (const double*)d_coef, (float*)d_vals,
                                 prec == WQ_PREC_F32, st, evs);
    if (e != cudaSuccess) return fail(rule->ctx, WQ_ERR_CUDA, std::string("assembly launch: ") + cudaGetErrorString(e));
    return WQ_OK;
}

wq_status wq_interp(const wq_rule* rule, const double* d_u, double* d_uq, double* d_grad, void* stream) {
    drop_stale_error();
    if (!rule || !d_u || !d_uq) return WQ_ERR_ARG;
    cudaError_t e = wqd::launch_interp(rule->el, rule->d_pt_elem, rule->d_fns, rule->d_fn_ptr, rule->Q,
                                       rule->d_table, d_u, d_uq, d_grad, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(rule->ctx, WQ_ERR_CUDA, std::string("interp launch: ") + cudaGetErrorString(e));
    return WQ_OK;
}

wq_status wq_apply(const wq_rule* rule, int32_t n_terms, const int32_t* h_comps, const double* d_g, double* d_y,
                   void* stream) {
    drop_stale_error();
    if (!rule || !h_comps || !d_g || !d_y || n_terms < 1 || n_terms > 4) return WQ_ERR_ARG;
    int wc[4] = {0, 0, 0, 0};
    for (int t = 0; t < n_terms; ++t) {
        if (h_comps[t] < 0 || h_comps[t] > 4 || rule->wcidx[h_comps[t]] < 0)
            return fail(rule->ctx, WQ_ERR_ARG, "wq_apply: weight component not built into this rule");
        wc[t] = rule->wcidx[h_comps[t]];
    }
    cudaError_t e = wqd::launch_apply(rule->rw, rule->d_pt_of_w, n_terms, make_int4(wc[0], wc[1], wc[2], wc[3]),
                                      rule->d_W, rule->nwc, d_g, rule->Q, d_y, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(rule->ctx, WQ_ERR_CUDA, std::string("apply launch: ") + cudaGetErrorString(e));
    return WQ_OK;
}

wq_status wq_heat_fields(const wq_rule* rule, const double* d_u, const double* d_u_old, double dt, double k0, double k2,
                         double f, int32_t jacobian, double* d_kappa, double* d_g, void* stream) {
    drop_stale_error();
    if (!rule || !d_u || !d_u_old || !d_kappa || !d_g || !(dt > 0)) return WQ_ERR_ARG;
    cudaError_t e = wqd::launch_heat_fields(rule->el, rule->d_pt_elem, rule->d_fns, rule->d_fn_ptr, rule->Q,
                                            rule->d_table, d_u, d_u_old, dt, k0, k2, f, jacobian != 0, d_kappa, d_g,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(rule->ctx, WQ_ERR_CUDA, std::string("heat fields launch: ") + cudaGetErrorString(e));
    return WQ_OK;
}

wq_status wq_batch_create(int32_t k, const wq_rule* const* rules, wq_batch** out) {
    drop_stale_error();
    if (!rules || !out || k < 1 || k > wqd::WQ_BATCH_MAX || !rules[0]) return WQ_ERR_ARG;
    *out = nullptr;
    wq_ctx* ctx = rules[0]->ctx;
    for (int r = 0; r < k; ++r) {
        if (!rules[r]) return fail(ctx, WQ_ERR_ARG, "null rule in batch");
        if (rules[r]->ctx->device != ctx->device || rules[r]->comps != rules[0]->comps ||
            rules[r]->dim != rules[0]->dim)
            return fail(ctx, WQ_ERR_ARG, "batched rules must share the device, weight components and dimension");
    }
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    wq_batch* Bt = new (std::nothrow) wq_batch();
    if (!Bt) return fail(ctx, WQ_ERR_OOM, "host allocation failed");
    Bt->ctx = ctx;
    Bt->device = ctx->device;
    Bt->rules.assign(rules, rules + k);
    // all tiles, ordered by their number of point chunks (long ones first), then by rule
    struct T {
        int4 it;
        int32_t kb, r;
    };
    std::vector<T> all;
    for (int r = 0; r < k; ++r)
        for (size_t x = 0; x < rules[r]->h_it_wq.size(); ++x)
            all.push_back({rules[r]->h_it_wq[x], rules[r]->h_kb_wq[x], r});
    std::stable_sort(all.begin(), all.end(), [](const T& a, const T& b) {
        return (((a.it.z >> 8) & 255) + 7) / 8 > (((b.it.z >> 8) & 255) + 7) / 8;
    });
    std::vector<int4> item(all.size());
    std::vector<int32_t> kb(all.size()), irule(all.size());
    for (size_t x = 0; x < all.size(); ++x) {
        item[x] = all[x].it;
        kb[x] = all[x].kb;
        irule[x] = all[x].r;
    }
    std::vector<wqd::ElemSrc> src(k);
    std::vector<int32_t> gr;
    std::vector<int64_t> gs;
    for (int r = 0; r < k; ++r) {
        src[r] = rules[r]->src_wq;
        for (int64_t b0 = 0; b0 < rules[r]->nnz; b0 += 512) {
            gr.push_back(r);
            gs.push_back(b0);
        }
    }
    auto up = [&](auto*& d, const auto& v) {
        using E = typename std::decay<decltype(v[0])>::type;
        void* p = nullptr;
        const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(E);
        if (cudaMalloc(&p, bytes) != cudaSuccess) return false;
        Bt->bufs.push_back({p, bytes});
        if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice) != cudaSuccess)
            return false;
        d = static_cast<E*>(p);
        return true;
    };
    int4* d_item = nullptr;
    int32_t *d_kb = nullptr, *d_irule = nullptr, *d_gr = nullptr;
    int64_t* d_gs = nullptr;
    wqd::ElemSrc* d_src = nullptr;
    if (!up(d_item, item) || !up(d_kb, kb) || !up(d_irule, irule) || !up(d_src, src) || !up(d_gr, gr) ||
        !up(d_gs, gs)) {
        delete Bt;
        return fail(ctx, WQ_ERR_OOM, "batch plan upload failed");
    }
    Bt->plan = {(int64_t)item.size(), d_item, d_kb, d_irule, d_src, (int64_t)gr.size(), d_gr, d_gs};
    *out = Bt;
    return WQ_OK;
}

void wq_batch_destroy(wq_batch* batch) {
    if (!batch) return;
    if (batch->device >= 0 && cudaSetDevice(batch->device) != cudaSuccess) cudaGetLastError();
    delete batch;
    cudaGetLastError();
}

wq_status wq_assemble_batched(const wq_batch* batch, int32_t op, const void* const* h_coefs, double alpha,
                              int32_t prec, void* const* h_vals, void* stream) {
    drop_stale_error();
    if (!batch || !h_vals) return WQ_ERR_ARG;
    const int k = (int)batch->rules.size();
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == WQ_PREC_AUTO) {   // the first rule's choice (the rules share their operators)
        if (op < 0 || op > 4) return fail(batch->ctx, WQ_ERR_ARG, "unknown operator");
        prec = batch->rules[0]->auto_prec[op][0];
    }
    if (prec == WQ_PREC_F64 || prec == WQ_PREC_TC) {   // one launch pair per rule
        for (int r = 0; r < k; ++r) {
            wq_status s = wq_assemble(batch->rules[r], op, h_coefs ? h_coefs[r] : nullptr, alpha, prec, h_vals[r],
                                      stream);
            if (s != WQ_OK) return s;
        }
        return WQ_OK;
    }
    if (prec != WQ_PREC_F32 && prec != WQ_PREC_F32_FAST) return fail(batch->ctx, WQ_ERR_ARG, "unknown precision");
    wqd::Terms tm;
    if (!op_terms(batch->rules[0], op, alpha, true, tm, 0))
        return fail(batch->ctx, WQ_ERR_ARG, "operator needs weight sets that these rules did not build");
    for (int t = 0; t < tm.nt; ++t)
        if (tm.t[t].crow > 0)
            return fail(batch->ctx, WQ_ERR_ARG, "batched assembly takes operators with one coefficient row");
    const double* coefs[wqd::WQ_BATCH_MAX];
    float* vals[wqd::WQ_BATCH_MAX];
    for (int r = 0; r < k; ++r) {
        coefs[r] = h_coefs ? (const double*)h_coefs[r] : nullptr;
        vals[r] = (float*)h_vals[r];
        if (!vals[r]) return fail(batch->ctx, WQ_ERR_ARG, "null output in batch");
    }
    cudaError_t e = wqd::launch_elem_batch(batch->plan, coefs, vals, k, tm, prec == WQ_PREC_F32, st);
    if (e != cudaSuccess) return fail(batch->ctx, WQ_ERR_CUDA, std::string("batched assembly: ") + cudaGetErrorString(e));
    return WQ_OK;
}

wq_status wq_rule_autotune(wq_rule* rule, int32_t op, const void* d_coef, double alpha, int32_t gauss, double tol,
                           int32_t reps, void* stream, int32_t* chosen, double* h_err, float* h_ms) {
    drop_stale_error();
    if (!rule || op < 0 || op > 4 || (gauss != 0 && gauss != 1) || reps < 1 || !(tol >= 0.0))
        return fail(rule ? rule->ctx : nullptr, WQ_ERR_ARG, "autotune: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nnz = rule->nnz;
    double* d64 = nullptr;
    float* d32 = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int32_t saved_var = rule->set_var[op][gauss];
    auto release = [&]() {
        if (d64) cudaFree(d64);
        if (d32) cudaFree(d32);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        rule->set_var[op][gauss] = saved_var;
    };
    if (cudaMalloc(&d64, std::max<int64_t>(nnz, 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d32, std::max<int64_t>(nnz, 1) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(rule->ctx, WQ_ERR_OOM, "autotune: scratch allocation failed");
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        release();
        return fail(rule->ctx, WQ_ERR_CUDA, "autotune: event creation failed");
    }
    auto run = [&](int32_t prec, void* out) {
        return gauss ? wq_gq_assemble(rule, op, d_coef, alpha, prec, out, stream)
                     : wq_assemble(rule, op, d_coef, alpha, prec, out, stream);
    };
    wq_status s = run(WQ_PREC_F64, d64);
    std::vector<double> a64(nnz);
    std::vector<float> a32(nnz);
    if (s == WQ_OK && nnz > 0 &&
        (cudaMemcpyAsync(a64.data(), d64, nnz * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
        s = fail(rule->ctx, WQ_ERR_CUDA, "autotune: copy failed");
    if (s != WQ_OK) {
        release();
        return s;
    }
    double amax = 0.0;
    for (double v : a64) amax = std::max(amax, std::fabs(v));
    // candidates: the tensor-core slices, then each SIMT mode with each kernel variant
    struct Cand {
        int32_t mode, variant;
    };
    const Cand cand[WQ_TUNE_MAX] = {{WQ_PREC_TC, -1},
                                    {WQ_PREC_F32, WQ_VARIANT_SLOTMAP},
                                    {WQ_PREC_F32, WQ_VARIANT_TILE12},
                                    {WQ_PREC_F32, WQ_VARIANT_TILE16},
                                    {WQ_PREC_F32_FAST, WQ_VARIANT_SLOTMAP},
                                    {WQ_PREC_F32_FAST, WQ_VARIANT_TILE12},
                                    {WQ_PREC_F32_FAST, WQ_VARIANT_TILE16}};
    int32_t best = -1, best_var = WQ_VARIANT_SLOTMAP;
    float best_ms = 0.0f;
    double mode_err[3] = {-1.0, -1.0, -1.0};
    float mode_ms[3] = {-1.0f, -1.0f, -1.0f};
    wq_rule::TuneRow* tab = rule->tune[op][gauss];
    int nt = 0;
    for (const Cand& c : cand) {
        if (c.variant >= 0 && c.variant != WQ_VARIANT_SLOTMAP && !rule->tile_ok) continue;
        rule->set_var[op][gauss] = c.variant >= 0 ? c.variant : saved_var;
        double err = -1.0;
        float ms = -1.0f;
        if (run(c.mode, d32) == WQ_OK) {   // a mode this rule or operator does not take is skipped
            if (nnz > 0 && (cudaMemcpyAsync(a32.data(), d32, nnz * sizeof(float), cudaMemcpyDeviceToHost, st) !=
                                cudaSuccess ||
                            cudaStreamSynchronize(st) != cudaSuccess)) {
                release();
                return fail(rule->ctx, WQ_ERR_CUDA, "autotune: copy failed");
            }
            double dmax = 0.0;
            for (int64_t x = 0; x < nnz; ++x) dmax = std::max(dmax, std::fabs((double)a32[x] - a64[x]));
            err = amax > 0.0 ? dmax / amax : dmax;
            if (err <= tol) {
                for (int w = 0; w < 2; ++w) run(c.mode, d32);
                cudaEventRecord(e0, st);
                for (int r = 0; r < reps; ++r) run(c.mode, d32);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    release();
                    return fail(rule->ctx, WQ_ERR_CUDA, "autotune: timing failed");
                }
                ms /= (float)reps;
                if (best < 0 || ms < best_ms) {
                    best = c.mode;
                    best_var = c.variant >= 0 ? c.variant : best_var;
                    best_ms = ms;
                }
            }
        } else {
            rule->ctx->err.clear();
        }
        const int k = c.mode == WQ_PREC_TC ? 0 : (c.mode == WQ_PREC_F32 ? 1 : 2);
        if (err >= 0.0 && (mode_err[k] < 0.0 || (ms >= 0.0f && (mode_ms[k] < 0.0f || ms < mode_ms[k])))) {
            mode_err[k] = err;
            if (ms >= 0.0f) mode_ms[k] = ms;
        }
        tab[nt++] = {c.mode, c.variant, err, ms};
    }
    rule->ntune[op][gauss] = nt;
    release();
    rule->auto_prec[op][gauss] = best >= 0 ? best : WQ_PREC_F32;
    rule->auto_var[op][gauss] = best >= 0 ? best_var : WQ_VARIANT_SLOTMAP;
    if (chosen) *chosen = best;
    for (int k = 0; k < 3; ++k) {
        if (h_err) h_err[k] = mode_err[k];
        if (h_ms) h_ms[k] = mode_ms[k];
    }
    return WQ_OK;
}

wq_status wq_rule_autotune_report(const wq_rule* rule, int32_t op, int32_t gauss, int32_t capacity, int32_t* n,
                                  int32_t* h_mode, int32_t* h_variant, double* h_err, float* h_ms) {
    if (!rule || op < 0 || op > 4 || (gauss != 0 && gauss != 1) || capacity < 0 || !n) return WQ_ERR_ARG;
    const int nt = rule->ntune[op][gauss];
    *n = nt;
    for (int k = 0; k < std::min(nt, (int)capacity); ++k) {
        const wq_rule::TuneRow& t = rule->tune[op][gauss][k];
        if (h_mode) h_mode[k] = t.mode;
        if (h_variant) h_variant[k] = t.variant;
        if (h_err) h_err[k] = t.err;
        if (h_ms) h_ms[k] = t.ms;
    }
    return WQ_OK;
}

wq_status wq_rule_set_variant(wq_rule* rule, int32_t op, int32_t gauss, int32_t variant) {
    if (!rule || op < 0 || op > 4 || (gauss != 0 && gauss != 1) || variant < -1 || variant > WQ_VARIANT_SLOTMAP)
        return fail(rule ? rule->ctx : nullptr, WQ_ERR_ARG, "set_variant: bad argument");
    if (variant >= 0 && variant != WQ_VARIANT_SLOTMAP && !rule->tile_ok)
        return fail(rule->ctx, WQ_ERR_ARG, "set_variant: this rule has no tile-engine plan");
    rule->set_var[op][gauss] = variant;
    return WQ_OK;
}

wq_status wq_rule_get_variant(const wq_rule* rule, int32_t op, int32_t gauss, int32_t* variant) {
    if (!rule || op < 0 || op > 4 || (gauss != 0 && gauss != 1) || !variant) return WQ_ERR_ARG;
    *variant = float_variant(rule, op, gauss);
    return WQ_OK;
}

wq_status wq_rule_set_timing(wq_rule* rule, int32_t capacity) {
    if (!rule || capacity < 0) return WQ_ERR_ARG;
    CUDA_TRY(rule->ctx, cudaSetDevice(rule->ctx->device));
    for (auto ev : rule->tev) cudaEventDestroy(ev);
    rule->tev.clear();
    rule->tcap = 0;
    rule->tcount = 0;
    rule->tev.resize((size_t)capacity * 3, nullptr);
    for (auto& ev : rule->tev) {
        if (cudaEventCreate(&ev) != cudaSuccess) {
            ev = nullptr;
            for (auto e2 : rule->tev)
                if (e2) cudaEventDestroy(e2);
            rule->tev.clear();
            return fail(rule->ctx, WQ_ERR_CUDA, "event creation failed");
        }
    }
    rule->tcap = capacity;
    return WQ_OK;
}

wq_status wq_rule_kernel_times(wq_rule* rule, int32_t max_calls, float* h_ms, int32_t* n_calls) {
    if (!rule || max_calls < 0 || (max_calls > 0 && !h_ms)) return WQ_ERR_ARG;
    const int n = std::min(rule->tcount, max_calls);
    for (int k = 0; k < n; ++k) {
        cudaEvent_t* ev = rule->tev.data() + 3 * k;
        CUDA_TRY(rule->ctx, cudaEventSynchronize(ev[2]));
        CUDA_TRY(rule->ctx, cudaEventElapsedTime(&h_ms[2 * k], ev[0], ev[1]));
        CUDA_TRY(rule->ctx, cudaEventElapsedTime(&h_ms[2 * k + 1], ev[1], ev[2]));
    }
    if (n_calls) *n_calls = n;
    rule->tcount = 0;
    return WQ_OK;
}

wq_status wq_basis_functions(const wq_basis* basis, int64_t* h_raw_ids) {
    if (!basis || !h_raw_ids) return WQ_ERR_ARG;
    std::copy(basis->B.raw_ids.begin(), basis->B.raw_ids.end(), h_raw_ids);
    return WQ_OK;
}

wq_status wq_assemble_host(const wq_rule* rule, int32_t op, const double* h_coef, double alpha, int32_t prec,
                           void* h_vals, void* stream) {
    drop_stale_error();
    if (!rule || !h_coef || !h_vals) return WQ_ERR_ARG;
    if (op == WQ_OP_HEAT_J) return fail(rule->ctx, WQ_ERR_ARG, "wq_assemble_host takes one coefficient row");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(rule->ctx, cudaMemcpyAsync(rule->d_coef_stage, h_coef, rule->Q * sizeof(double), cudaMemcpyHostToDevice, st));
    // page-locked host memory mapped into the device's address space: the per-entry
    // sums write it directly (the values cross the host link once, no staging copy)
    void* out = rule->d_vals_stage;
    bool direct = false;
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, h_vals) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer != nullptr) {
        out = pa.devicePointer;
        direct = true;
    } else {
        cudaGetLastError();
    }
    wq_status s = wq_assemble(rule, op, rule->d_coef_stage, alpha, prec, out, stream);
    if (s != WQ_OK) return s;
    if (!direct) {
        const size_t vb = rule->nnz * (prec == WQ_PREC_F64 ? sizeof(double) : sizeof(float));
        CUDA_TRY(rule->ctx, cudaMemcpyAsync(h_vals, rule->d_vals_stage, vb, cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(rule->ctx, cudaStreamSynchronize(st));
    return WQ_OK;
}

}  // extern "C"
