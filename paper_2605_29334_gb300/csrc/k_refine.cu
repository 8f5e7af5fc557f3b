// One global refinement of a bicubic ASUTS control mesh on the device (Sec. 3):
// the knot-insertion stencils of the vertex-based control points and the
// de Casteljau split of the enriched faces' Bezier nets for the face-based ones.
// The plan (fine topology, stencils, element coefficients) is built on the host
// (refine_host.cpp); this file holds the kernels and the wq_refine_* C ABI.
//
// k_refine: one launch, one warp per work item.  The de Casteljau split is linear, so
//   at set-up it is folded into the element's Bezier coefficients: every inner point of
//   the four children of a coarse enriched face is a fixed combination of the coarse
//   control points, of which only the non-zero terms are kept (about a seventh of the
//   dense m x 16 coefficients on the benchmark mesh).  A face is then 16 short dot
//   products, a group of 32 fine vertices 32 knot-insertion stencils (at most 9 coarse
//   vertices each).
#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "rule.h"
#include "wq_internal.h"

// A coarse enriched face on the device: the 16 inner points of its children as a padded
// (ELL) list of non-zero terms, K per point, stored term-major ([k][16]) at ell_off,
// each a coefficient and the raw control-variable id of its function.
struct FaceJobDev {
    int64_t ell_off;
    int32_t K;       // terms per point (even: the two half-warps take alternate terms)
    int32_t nsub;    // 1 or 4 (2 x 2-split irregular element)
    int32_t out;     // first fine face-based point written (16 per job)
    int32_t pad;
};

struct wq_refine {
    wq_ctx* ctx = nullptr;
    int device = -1;
    wqi::RefinePlan plan;
    int64_t n_terms = 0;                   // non-zero coefficients over all face jobs
    int64_t n_ell = 0;                     // their padded (ELL) entries
    std::vector<wqi::DevBuf> bufs;
    int32_t* d_st_src = nullptr;           // stencils per group of 32 fine vertices, [group][RF_SLOTS][32]
    double* d_st_w = nullptr;
    uint8_t* d_st_K = nullptr;             // the group's longest stencil
    FaceJobDev* d_jobs = nullptr;
    int32_t* d_ell_id = nullptr;           // raw control-variable id of every (padded) term
    double* d_ell_c = nullptr;             // its coefficient (0 for padding)
    int n_sm = 1;
    ~wq_refine() {
        for (auto& b : bufs)
            if (b.p) cudaFree(b.p);
    }
};

namespace {

constexpr int RF_SLOTS = 9;   // longest stencil: the 3 x 3 vertex rule

constexpr int RF_WARPS = 8;   // warps per block of the refinement kernel

// de Casteljau at 1/2 of a cubic: control point x of the two halves (x = 0..6) as a
// combination of the four of the whole (rows 1/2^k binomial weights, exact in FP64).
constexpr double kHalfSplit[7][4] = {{1.0, 0.0, 0.0, 0.0},       {0.5, 0.5, 0.0, 0.0},
                                     {0.25, 0.5, 0.25, 0.0},     {0.125, 0.375, 0.375, 0.125},
                                     {0.0, 0.25, 0.5, 0.25},     {0.0, 0.0, 0.5, 0.5},
                                     {0.0, 0.0, 0.0, 1.0}};

// Both parts of one refinement in one launch, one warp per work item, taken in a
// grid-stride loop: first the coarse enriched faces, then the fine vertices in groups
// of 32.  No shared memory and no barrier: every item is a padded (ELL) list of
// (control point, coefficient) terms per output point.
//   Face: slot t = lane & 15 is inner point t of the four children (child t / 4 at
//   coarse corner t / 4, its corner t % 4); its terms are the non-zero coefficients of
//   the element's functions in that point -- for a plain face the de Casteljau split at
//   1/2 folded into the Bezier coefficients at set-up, for a 2 x 2-split irregular
//   element the coefficients of the sub-net point itself.  The two half-warps take
//   alternate terms, then add.
//   Vertex group: lane l is fine vertex 32 g + l; its knot-insertion stencil, padded to
//   the group's longest (K_g <= RF_SLOTS) and stored [g][k][32], so that the loads of a
//   lane are in flight together.
__global__ void __launch_bounds__(RF_WARPS * 32) k_refine(int64_t n_jobs, const FaceJobDev* __restrict__ jobs,
                                                          const int32_t* __restrict__ ell_id,
                                                          const double* __restrict__ ell_c, int64_t Vc,
                                                          const double* __restrict__ xyz,
                                                          const double* __restrict__ fxyz,
                                                          double* __restrict__ out_f, int64_t nv,
                                                          const uint8_t* __restrict__ vK,
                                                          const int32_t* __restrict__ src,
                                                          const double* __restrict__ w,
                                                          double* __restrict__ out_v) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t n_vchunks = (nv + 31) / 32;
    const int64_t total = n_jobs + n_vchunks;
    const int64_t stride = (int64_t)gridDim.x * RF_WARPS;
    for (int64_t item = (int64_t)blockIdx.x * RF_WARPS + wib; item < total; item += stride) {
        if (item >= n_jobs) {
            const int64_t g = item - n_jobs, v = g * 32 + lane;
            const int K = vK[g];
            const int32_t* sg = src + g * (RF_SLOTS * 32) + lane;
            const double* wg = w + g * (RF_SLOTS * 32) + lane;
            int32_t sidx[RF_SLOTS];
            double c[RF_SLOTS];
#pragma unroll
            for (int k = 0; k < RF_SLOTS; ++k)
                if (k < K) {
                    sidx[k] = sg[k * 32];
                    c[k] = wg[k * 32];
                }
            double x = 0.0, y = 0.0, z = 0.0;
#pragma unroll
            for (int k = 0; k < RF_SLOTS; ++k)
                if (k < K) {
                    const double* p = xyz + 3 * (int64_t)sidx[k];
                    x = fma(c[k], p[0], x);
                    y = fma(c[k], p[1], y);
                    z = fma(c[k], p[2], z);
                }
            if (v < nv) {
                out_v[3 * v] = x;
                out_v[3 * v + 1] = y;
                out_v[3 * v + 2] = z;
            }
            continue;
        }
        const FaceJobDev jb = jobs[item];
        const int t = lane & 15, half = lane >> 4;
        const int32_t* ids = ell_id + jb.ell_off;
        const double* cs = ell_c + jb.ell_off;
        double x = 0.0, y = 0.0, z = 0.0;
#pragma unroll 4
        for (int k = half; k < jb.K; k += 2) {
            const int64_t r = ids[k * 16 + t];
            const double c = cs[k * 16 + t];
            const double* q = r < Vc ? xyz + 3 * r : fxyz + 3 * (r - Vc);
            x = fma(c, q[0], x);
            y = fma(c, q[1], y);
            z = fma(c, q[2], z);
        }
        x += __shfl_down_sync(0xffffffffu, x, 16);
        y += __shfl_down_sync(0xffffffffu, y, 16);
        z += __shfl_down_sync(0xffffffffu, z, 16);
        if (lane < 16) {
            double* o = out_f + 3 * ((int64_t)jb.out + t);
            o[0] = x;
            o[1] = y;
            o[2] = z;
        }
    }
}

wq_status rfail(wq_ctx* ctx, wq_status code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

template <class T>
wq_status rupload(wq_refine* R, T*& p, const std::vector<T>& v) {
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return rfail(R->ctx, WQ_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed");
    }
    R->bufs.push_back({q, bytes});
    p = static_cast<T*>(q);
    if (!v.empty()) {
        e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return rfail(R->ctx, WQ_ERR_CUDA, std::string("upload failed: ") + cudaGetErrorString(e));
    }
    return WQ_OK;
}

}  // namespace

extern "C" {

wq_status wq_refine_create(const wq_basis* basis, wq_refine** out) {
    if (!basis || !out) return WQ_ERR_ARG;
    *out = nullptr;
    (void)cudaGetLastError();
    wq_refine* R = new (std::nothrow) wq_refine();
    if (!R) return rfail(basis->ctx, WQ_ERR_OOM, "host allocation failed");
    R->ctx = basis->ctx;
    R->device = basis->ctx ? basis->ctx->device : -1;
    wqi::Error err{WQ_OK, ""};
    bool ok = false;
    try {
        ok = wqi::build_refine(basis->B, R->plan, err);
    } catch (const std::bad_alloc&) {
        err = {WQ_ERR_OOM, "host allocation failed"};
    }
    if (!ok) {
        delete R;
        return rfail(basis->ctx, err.code, err.msg);
    }
    // face jobs: for each of the 16 children's inner points the non-zero coefficients of
    // the element's functions in it (zero terms would add exactly nothing), in function
    // order, padded to an even count K per job with zero terms on the job's first function
    std::vector<FaceJobDev> fj;
    std::vector<int32_t> ell_id;
    std::vector<double> ell_c;
    try {
        fj.resize(R->plan.jobs.size());
        std::vector<std::vector<std::pair<int32_t, double>>> terms(16);
        for (size_t x = 0; x < R->plan.jobs.size(); ++x) {
            const wqi::RefineJob& J = R->plan.jobs[x];
            const int np = 16 * J.nsub;
            int K = 0;
            for (int t = 0; t < 16; ++t) {
                    const int k = t >> 2, c2 = t & 3;            // child (coarse corner), its corner
                const int cu = (k == 1 || k == 2), cv = (k >= 2), du = (c2 == 1 || c2 == 2), dv = (c2 >= 2);
                terms[t].clear();
                for (int a = 0; a < J.m; ++a) {
                    const double* ca = R->plan.coef.data() + J.coef_off + (int64_t)a * np;
                    double c = 0.0;
                    if (J.nsub != 1) {
                        c = ca[(cu + 2 * cv) * 16 + (1 + du) * 4 + (1 + dv)];   // the sub-net's point
                    } else {
                        // de Casteljau at 1/2 folded in: row xx of the u-split, column yy of
                        // the v-split of the 4 x 4 net
                        const int xx = 3 * cu + 1 + du, yy = 3 * cv + 1 + dv;
                        for (int i = 0; i < 4; ++i)
                            for (int j = 0; j < 4; ++j) c += kHalfSplit[xx][i] * kHalfSplit[yy][j] * ca[i * 4 + j];
                    }
                    if (c != 0.0) terms[t].push_back({R->plan.fn_raw[(size_t)J.fn_off + a], c});
                }
                K = std::max(K, (int)terms[t].size());
                R->n_terms += (int64_t)terms[t].size();
            }
            K = (K + 1) & ~1;
            fj[x] = {(int64_t)ell_id.size(), K, J.nsub, J.out, 0};
            const int32_t pad_id = J.m > 0 ? R->plan.fn_raw[(size_t)J.fn_off] : 0;
            for (int k = 0; k < K; ++k)
                for (int t = 0; t < 16; ++t) {
                    const bool real = k < (int)terms[t].size();
                    ell_id.push_back(real ? terms[t][k].first : pad_id);
                    ell_c.push_back(real ? terms[t][k].second : 0.0);
                }
        }
    } catch (const std::bad_alloc&) {
        delete R;
        return rfail(basis->ctx, WQ_ERR_OOM, "host allocation failed");
    }
    R->n_ell = (int64_t)ell_id.size();
    if (R->device >= 0) {
        if (cudaSetDevice(R->device) != cudaSuccess) {
            cudaGetLastError();
            delete R;
            return rfail(basis->ctx, WQ_ERR_CUDA, "cudaSetDevice failed");
        }
        int n_sm = 0;
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, R->device) == cudaSuccess && n_sm > 0)
            R->n_sm = n_sm;
        cudaGetLastError();
        const wqi::RefinePlan& P = R->plan;
        // stencils per group of 32 fine vertices, padded to the group's longest (weight 0,
        // source 0), [group][RF_SLOTS][32]
        const int64_t ng = (P.Vf + 31) / 32;
        std::vector<int32_t> ell_src((size_t)ng * RF_SLOTS * 32, 0);
        std::vector<double> ell_w((size_t)ng * RF_SLOTS * 32, 0.0);
        std::vector<uint8_t> gK((size_t)std::max<int64_t>(ng, 1), 0);
        for (int64_t v = 0; v < P.Vf; ++v) {
            const int64_t len = P.st_ptr[v + 1] - P.st_ptr[v];
            if (len > RF_SLOTS) {
                delete R;
                return rfail(basis->ctx, WQ_ERR_MESH, "refinement stencil longer than 9 entries");
            }
            const int64_t g = v / 32, l = v % 32;
            gK[g] = (uint8_t)std::max<int64_t>(gK[g], len);
            for (int64_t k = 0; k < len; ++k) {
                ell_src[(size_t)((g * RF_SLOTS + k) * 32 + l)] = P.st_src[P.st_ptr[v] + k];
                ell_w[(size_t)((g * RF_SLOTS + k) * 32 + l)] = P.st_w[P.st_ptr[v] + k];
            }
        }
        wq_status s = WQ_OK;
        if (s == WQ_OK) s = rupload(R, R->d_st_src, ell_src);
        if (s == WQ_OK) s = rupload(R, R->d_st_w, ell_w);
        if (s == WQ_OK) s = rupload(R, R->d_st_K, gK);
        if (s == WQ_OK) s = rupload(R, R->d_jobs, fj);
        if (s == WQ_OK) s = rupload(R, R->d_ell_id, ell_id);
        if (s == WQ_OK) s = rupload(R, R->d_ell_c, ell_c);
        if (s != WQ_OK) {
            delete R;
            return s;
        }
    }
    *out = R;
    return WQ_OK;
}

void wq_refine_destroy(wq_refine* r) {
    if (!r) return;
    if (r->device >= 0 && cudaSetDevice(r->device) != cudaSuccess) cudaGetLastError();
    delete r;
}

wq_status wq_refine_info_get(const wq_refine* r, wq_refine_info* info) {
    if (!r || !info) return WQ_ERR_ARG;
    const wqi::RefinePlan& P = r->plan;
    info->n_vertices = P.Vf;
    info->n_faces = P.Ff;
    info->n_face_xyz = P.n_fx_f;
    info->n_coarse_vertices = P.Vc;
    info->n_coarse_face_xyz = P.n_fx_c;
    info->n_stencil = (int64_t)P.st_src.size();
    info->n_face_jobs = (int64_t)P.jobs.size();
    info->n_face_fns = (int64_t)P.fn_raw.size();
    info->n_face_coef = (int64_t)P.coef.size();
    info->n_face_terms = r->n_terms;
    info->n_face_ell = r->n_ell;
    return WQ_OK;
}

wq_status wq_refine_mesh(const wq_refine* r, int32_t* h_quads, int32_t* h_level0_face) {
    if (!r) return WQ_ERR_ARG;
    if (h_quads) std::copy(r->plan.quads.begin(), r->plan.quads.end(), h_quads);
    if (h_level0_face) std::copy(r->plan.level0.begin(), r->plan.level0.end(), h_level0_face);
    return WQ_OK;
}

wq_status wq_refine_stencils(const wq_refine* r, int64_t* h_ptr, int32_t* h_src, double* h_w) {
    if (!r) return WQ_ERR_ARG;
    if (h_ptr) std::copy(r->plan.st_ptr.begin(), r->plan.st_ptr.end(), h_ptr);
    if (h_src) std::copy(r->plan.st_src.begin(), r->plan.st_src.end(), h_src);
    if (h_w) std::copy(r->plan.st_w.begin(), r->plan.st_w.end(), h_w);
    return WQ_OK;
}

wq_status wq_refine_apply(const wq_refine* r, const double* d_xyz, const double* d_face_xyz, double* d_xyz_fine,
                          double* d_face_xyz_fine, void* stream) {
    if (!r) return WQ_ERR_ARG;
    (void)cudaGetLastError();
    if (r->device < 0) return rfail(r->ctx, WQ_ERR_NO_DEVICE, "context has no device");
    const wqi::RefinePlan& P = r->plan;
    if (!d_xyz || !d_xyz_fine || (P.n_fx_c > 0 && (!d_face_xyz || !d_face_xyz_fine)))
        return rfail(r->ctx, WQ_ERR_ARG, "null control-point array");
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != r->device) e = cudaSetDevice(r->device);   // no call when already current
    if (e != cudaSuccess) return rfail(r->ctx, WQ_ERR_CUDA, std::string("device selection: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nj = (int64_t)P.jobs.size();
    const int64_t items = nj + (P.Vf + 31) / 32;
    if (items > 0) {
        // one warp per item, up to eight resident blocks of eight warps per SM
        const int64_t blocks = std::min<int64_t>((items + RF_WARPS - 1) / RF_WARPS, (int64_t)r->n_sm * 8);
        k_refine<<<(unsigned)blocks, RF_WARPS * 32, 0, st>>>(nj, r->d_jobs, r->d_ell_id, r->d_ell_c, P.Vc, d_xyz,
                                                             d_face_xyz, d_face_xyz_fine, P.Vf, r->d_st_K,
                                                             r->d_st_src, r->d_st_w, d_xyz_fine);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return rfail(r->ctx, WQ_ERR_CUDA, std::string("refine launch: ") + cudaGetErrorString(e));
    return WQ_OK;
}

wq_status wq_basis_face_ctrl(const wq_basis* basis, int64_t* n_face_xyz, double* h_face_xyz) {
    if (!basis) return WQ_ERR_ARG;
    if (n_face_xyz) *n_face_xyz = (int64_t)basis->B.face_xyz.size() / 3;
    if (h_face_xyz) std::copy(basis->B.face_xyz.begin(), basis->B.face_xyz.end(), h_face_xyz);
    return WQ_OK;
}

}  // extern "C"
