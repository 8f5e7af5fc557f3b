// wq_rule_weights_noalloc: the truncated-SVD weight solve of an existing rule,
// run with a scratch area that is compiled into the library instead of one the
// library allocates.
//
// Who needs it: callers that must not allocate device memory while they run --
// for instance a host application that has handed all free device memory to
// its own pool allocator, or a time-critical loop in which the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable.  The weight solve
// of wq_rule_build needs a per-CTA workspace of 2 n r + 4 n^2 + 2 r + 7 n doubles
// (n = #S_i, r = #points of N_i); here it comes from the fixed array below.
//
// The array g_noalloc_scratch is a file-scope __device__ object: every device
// that loads the library holds its 32 MiB until the process exits.  Host code
// may not use its name as a device address, so its device address is looked up
// with cudaGetSymbolAddress, with the device current, when wq_create binds a
// context to the device (noalloc_bind below).  Under lazy module loading that lookup
// is also what commits the array's memory on the device, so the commitment happens
// at context creation and not inside a later call that must not allocate.  All calls
// share the array and it keeps the last call's contents: the status word is cleared
// at the start of every call, and calls that overlap on the GPU (another stream,
// another host thread) race on the array.  The call reads its status back and
// synchronises on the caller's stream.
#include <mutex>
#include <string>

#include "rule.h"

namespace {

constexpr int64_t kScratchDoubles = 4 * 1024 * 1024;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];
__device__ __align__(256) unsigned g_noalloc_status;

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned* g_status_ptr[kMaxDevices] = {nullptr};

wq_status set_err(wq_ctx* ctx, wq_status code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

// Look up (once per device, with that device current) the device addresses of the
// scratch array and status word; false with a message if the runtime refuses.
bool lookup(int dev, std::string& err) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_ptr[dev]) return true;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
        return false;
    }
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_noalloc_status);
    if (e != cudaSuccess) {
        err = std::string("cudaGetSymbolAddress(status): ") + cudaGetErrorString(e);
        return false;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
    g_status_ptr[dev] = static_cast<unsigned*>(q);
    return true;
}

}  // namespace

// Called by wq_create with `dev` current.
bool wqi_noalloc_bind(int dev, std::string& err) {
    if (dev < 0 || dev >= kMaxDevices) return true;   // the entry point reports it
    return lookup(dev, err);
}

extern "C" wq_status wq_rule_weights_noalloc(const wq_rule* rule, int32_t comp, double* d_w, void* stream) {
    if (!rule || !d_w || comp < 0 || comp > 4) return WQ_ERR_ARG;
    wq_ctx* ctx = rule->ctx;
    if (rule->wcidx[comp] < 0 || !rule->d_mom[comp])
        return set_err(ctx, WQ_ERR_ARG, "component not built into this rule");
    const int dev = ctx->device;
    if (dev < 0 || dev >= kMaxDevices) return set_err(ctx, WQ_ERR_NO_DEVICE, "context has no usable device");
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return set_err(ctx, WQ_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    (void)cudaGetLastError();   // an error pending from another caller is not this call's
    cudaStream_t st = (cudaStream_t)stream;
    std::string lerr;
    if (!lookup(dev, lerr)) return set_err(ctx, WQ_ERR_CUDA, lerr);   // normally done by wq_create already
    double* scratch = g_scratch_ptr[dev];
    unsigned* status = g_status_ptr[dev];
    const int64_t mn = rule->max_n_i, mr = rule->max_r;
    const int64_t per_cta = wqd::tsvd_scratch_doubles(mn, mr);
    if (per_cta > kScratchDoubles)
        return set_err(ctx, WQ_ERR_ARG,
                       "weight system too large for the fixed scratch: needs " + std::to_string(per_cta * 8) +
                           " bytes per system, the library holds " + std::to_string(kScratchDoubles * 8));
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    int64_t n_cta = kScratchDoubles / per_cta;
    n_cta = std::min<int64_t>(n_cta, (int64_t)std::max(n_sm, 1) * wqd::TSVD_CTAS_PER_SM);
    n_cta = std::min<int64_t>(n_cta, std::max<int64_t>(rule->n, 1));
    e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = wqd::launch_tsvd(rule->el, rule->rw, rule->d_table, comp == WQ_COMP_LAP ? rule->nc - 1 : comp,
                             rule->d_mom[comp], d_w, 1, 0, rule->tol, rule->max_sweeps, scratch, per_cta, (int)n_cta,
                             nullptr, nullptr, status, nullptr, st);
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_err(ctx, WQ_ERR_CUDA, std::string("no-alloc weight solve: ") + cudaGetErrorString(e));
    if (h & wqd::ST_NOT_CONVERGED) return set_err(ctx, WQ_ERR_NOT_CONVERGED, "Jacobi SVD reached its sweep cap");
    if (h & wqd::ST_NONFINITE) return set_err(ctx, WQ_ERR_NONFINITE, "non-finite value in the weight solve");
    return WQ_OK;
}
