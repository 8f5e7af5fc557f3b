// One global refinement of a bicubic ASUTS control mesh on the device (Sec. 3):
// the knot-insertion stencils of the vertex-based control points and the
// de Casteljau split of the enriched faces' Bezier nets for the face-based ones.
// The plan (fine topology, stencils, element coefficients) is built on the host
// (refine_host.cpp); this file holds the kernels and the wq_refine_* C ABI.
//
// k_refine_vertices: one thread per fine vertex, x_w = sum_k w_k x_{src_k} over
//   its stencil (at most 9 coarse vertices, padded to 9 and stored slot-major so
//   that all of a thread's loads are in flight together; gathers of 24-byte points).
// k_refine_faces: one block of 64 threads per coarse enriched face.  The block
//   gathers the coarse control points of the element's functions into shared
//   memory (64 at a time, all loads in flight together); thread p then contracts
//   Bezier coefficient p of every function with them into net point p (16 points,
//   or 4 x 16 for a 2 x 2-split irregular element); a plain face's net is split at 1/2 along
//   u and v by de Casteljau's algorithm in shared memory (4 x 4 -> 7 x 7), and
//   16 threads write the inner points of the four children (for a split element
//   the sub-nets are the children's nets).
#include <string>
#include <vector>

#include "rule.h"
#include "wq_internal.h"

struct wq_refine {
    wq_ctx* ctx = nullptr;
    int device = -1;
    wqi::RefinePlan plan;
    std::vector<wqi::DevBuf> bufs;
    int32_t* d_st_src = nullptr;           // stencils padded to RF_SLOTS, slot-major [RF_SLOTS][Vf]
    double* d_st_w = nullptr;
    wqi::RefineJob* d_jobs = nullptr;
    int32_t* d_fn_raw = nullptr;
    double* d_coef = nullptr;
    ~wq_refine() {
        for (auto& b : bufs)
            if (b.p) cudaFree(b.p);
    }
};

namespace {

constexpr int RF_SLOTS = 9;   // longest stencil: the 3 x 3 vertex rule

// Stencils padded to RF_SLOTS entries (weight 0, source 0), slot-major: entry k of
// vertex v at k * nv + v, so that a warp reads each slot contiguously and every
// load of a thread is issued before the first one is used.
__global__ void __launch_bounds__(256) k_refine_vertices(int64_t nv, const int32_t* __restrict__ src,
                                                         const double* __restrict__ w,
                                                         const double* __restrict__ xyz, double* __restrict__ out) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int32_t s[RF_SLOTS];
    double c[RF_SLOTS];
#pragma unroll
    for (int k = 0; k < RF_SLOTS; ++k) {
        s[k] = src[k * nv + v];
        c[k] = w[k * nv + v];
    }
    double x = 0.0, y = 0.0, z = 0.0;
#pragma unroll
    for (int k = 0; k < RF_SLOTS; ++k) {
        const double* p = xyz + 3 * (int64_t)s[k];
        x = fma(c[k], p[0], x);
        y = fma(c[k], p[1], y);
        z = fma(c[k], p[2], z);
    }
    out[3 * v] = x;
    out[3 * v + 1] = y;
    out[3 * v + 2] = z;
}

__device__ __forceinline__ void split_half(const double* b, int stride_in, double* o, int stride_out) {
    // de Casteljau at 1/2: 4 control points -> the 7 of the two halves
    const double b0 = b[0], b1 = b[stride_in], b2 = b[2 * stride_in], b3 = b[3 * stride_in];
    const double b01 = 0.5 * (b0 + b1), b12 = 0.5 * (b1 + b2), b23 = 0.5 * (b2 + b3);
    const double b012 = 0.5 * (b01 + b12), b123 = 0.5 * (b12 + b23);
    o[0] = b0;
    o[stride_out] = b01;
    o[2 * stride_out] = b012;
    o[3 * stride_out] = 0.5 * (b012 + b123);
    o[4 * stride_out] = b123;
    o[5 * stride_out] = b23;
    o[6 * stride_out] = b3;
}

__global__ void __launch_bounds__(64) k_refine_faces(int64_t n_jobs, const wqi::RefineJob* __restrict__ jobs,
                                                     const int32_t* __restrict__ fn_raw,
                                                     const double* __restrict__ coef, int64_t Vc,
                                                     const double* __restrict__ xyz,
                                                     const double* __restrict__ fxyz, double* __restrict__ out) {
    __shared__ double sP[3][64];         // control points of the functions being contracted
    __shared__ double net[3][64];        // [coord][sub*16 + i*4 + j]
    __shared__ double half[3][7 * 4];    // u-split rows: [coord][x*4 + j]
    __shared__ double full[3][7 * 7];    // [coord][x*7 + y]
    const int64_t b = blockIdx.x;
    if (b >= n_jobs) return;
    const wqi::RefineJob jb = jobs[b];
    const int t = threadIdx.x;
    const int np = 16 * jb.nsub;
    double x = 0.0, y = 0.0, z = 0.0;
    const double* c = coef + jb.coef_off + t;
    for (int a0 = 0; a0 < jb.m; a0 += 64) {
        // the control points of up to 64 functions, gathered by all threads at once
        const int na = min(64, jb.m - a0);
        if (t < na) {
            const int64_t r = fn_raw[jb.fn_off + a0 + t];
            const double* p = r < Vc ? xyz + 3 * r : fxyz + 3 * (r - Vc);
            sP[0][t] = p[0];
            sP[1][t] = p[1];
            sP[2][t] = p[2];
        }
        __syncthreads();
        if (t < np) {
#pragma unroll 8
            for (int a = 0; a < na; ++a) {
                const double w = c[(int64_t)(a0 + a) * np];
                x = fma(w, sP[0][a], x);
                y = fma(w, sP[1][a], y);
                z = fma(w, sP[2][a], z);
            }
        }
        __syncthreads();
    }
    if (t < np) {
        net[0][t] = x;
        net[1][t] = y;
        net[2][t] = z;
    }
    __syncthreads();
    const int k = t >> 2, c2 = t & 3;                       // child (coarse corner), its corner
    const int cu = (k == 1 || k == 2), cv = (k >= 2);
    const int du = (c2 == 1 || c2 == 2), dv = (c2 >= 2);
    if (jb.nsub == 1) {
        if (t < 12) {                                       // 4 rows j x 3 coordinates, along u
            const int j = t / 3, d = t % 3;
            split_half(&net[d][j], 4, &half[d][j], 4);
        }
        __syncthreads();
        if (t < 21) {                                       // 7 columns x 3 coordinates, along v
            const int x = t / 3, d = t % 3;
            split_half(&half[d][x * 4], 1, &full[d][x * 7], 1);
        }
        __syncthreads();
        if (t < 16) {
            const int x = 3 * cu + 1 + du, y = 3 * cv + 1 + dv;
            double* o = out + 3 * ((int64_t)jb.out + t);
            o[0] = full[0][x * 7 + y];
            o[1] = full[1][x * 7 + y];
            o[2] = full[2][x * 7 + y];
        }
    } else if (t < 16) {
        const int s = cu + 2 * cv;                          // the child is sub-element s
        const int p = s * 16 + (1 + du) * 4 + (1 + dv);
        double* o = out + 3 * ((int64_t)jb.out + t);
        o[0] = net[0][p];
        o[1] = net[1][p];
        o[2] = net[2][p];
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
    if (R->device >= 0) {
        if (cudaSetDevice(R->device) != cudaSuccess) {
            cudaGetLastError();
            delete R;
            return rfail(basis->ctx, WQ_ERR_CUDA, "cudaSetDevice failed");
        }
        const wqi::RefinePlan& P = R->plan;
        std::vector<int32_t> ell_src((size_t)RF_SLOTS * P.Vf, 0);
        std::vector<double> ell_w((size_t)RF_SLOTS * P.Vf, 0.0);
        for (int64_t v = 0; v < P.Vf; ++v) {
            if (P.st_ptr[v + 1] - P.st_ptr[v] > RF_SLOTS) {
                delete R;
                return rfail(basis->ctx, WQ_ERR_MESH, "refinement stencil longer than 9 entries");
            }
            for (int64_t k = P.st_ptr[v]; k < P.st_ptr[v + 1]; ++k) {
                ell_src[(size_t)(k - P.st_ptr[v]) * P.Vf + v] = P.st_src[k];
                ell_w[(size_t)(k - P.st_ptr[v]) * P.Vf + v] = P.st_w[k];
            }
        }
        wq_status s = WQ_OK;
        if (s == WQ_OK) s = rupload(R, R->d_st_src, ell_src);
        if (s == WQ_OK) s = rupload(R, R->d_st_w, ell_w);
        if (s == WQ_OK) s = rupload(R, R->d_jobs, P.jobs);
        if (s == WQ_OK) s = rupload(R, R->d_fn_raw, P.fn_raw);
        if (s == WQ_OK) s = rupload(R, R->d_coef, P.coef);
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
    if (P.Vf > 0) {
        const unsigned g = (unsigned)((P.Vf + 255) / 256);
        k_refine_vertices<<<g, 256, 0, st>>>(P.Vf, r->d_st_src, r->d_st_w, d_xyz, d_xyz_fine);
    }
    const int64_t nj = (int64_t)P.jobs.size();
    if (nj > 0)
        k_refine_faces<<<(unsigned)nj, 64, 0, st>>>(nj, r->d_jobs, r->d_fn_raw, r->d_coef, P.Vc, d_xyz, d_face_xyz,
                                                    d_face_xyz_fine);
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
