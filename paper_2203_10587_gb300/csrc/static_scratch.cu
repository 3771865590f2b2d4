// exago_eval_all_static: the batched evaluation of exago_eval_all with its scratch in a fixed,
// file-scope device array instead of a workspace the caller or the library allocates.
//
// Who needs it: callers that may not allocate device memory themselves once they are running,
// for example a solver whose device memory is owned by a pooling allocator (raw cudaMalloc /
// cudaFree would bypass its accounting, and cudaFree synchronises the whole device), or a serving
// loop that reserves all memory at start-up and must not block on an allocation later.  Such a
// caller still passes its own inputs and outputs; only the per-call scratch moves here.
//
// Limits: the array holds EXAGO_STATIC_SCRATCH_BYTES (16 MiB).  Every GPU that loads this library
// reserves it for the life of the process.  A batch whose scratch (exago_eval_workspace_size)
// exceeds it is rejected with EXAGO_EINVAL.  All calls share the one array per device: calls that
// overlap on the GPU (different streams, or different host threads without ordering) race on it.
// Nothing in it has to start at zero: each call writes every scratch entry it later reads.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr size_t kStaticBytes = EXAGO_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) double g_static_scratch[kStaticBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device, looked up once per device.  In host
// code the array's name only stands for the device symbol, so the address must come from
// cudaGetSymbolAddress with that device current.
cudaError_t static_scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" exago_status exago_eval_all_static(exago_net_t net, const exago_batch *bt, double *f,
                                              double *grad, double *gh, double *jval,
                                              double *hval) {
    using namespace exago;
    const HostPlan *plan = nullptr;
    const DevNet *dev = nullptr;
    int net_device = -1;
    if (!net_internal_view(net, &plan, &dev, &net_device))
        return set_last_error(net ? EXAGO_ESTATE : EXAGO_EINVAL,
                              net ? "net was planned without a device" : "net is NULL");
    if (!bt) return set_last_error(EXAGO_EINVAL, "batch is NULL");
    if (bt->B < 0) return set_last_error(EXAGO_EINVAL, "batch B < 0");
    if (bt->B == 0) return EXAGO_OK;
    if (!bt->x) return set_last_error(EXAGO_EINVAL, "batch x is NULL");
    if (hval && !bt->lambda)
        return set_last_error(EXAGO_EINVAL, "batch lambda is NULL (needed by the Hessian)");
    const size_t need = workspace_bytes(*plan, bt->B);
    if (need > kStaticBytes) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "batch of %d states needs %zu bytes of scratch; the static scratch holds %zu "
                 "bytes: split the batch", bt->B, need, kStaticBytes);
        return set_last_error(EXAGO_EINVAL, msg);
    }
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
    if (cur != net_device || cur < 0 || cur >= kMaxDevices)
        return set_last_error(EXAGO_EINVAL, "make the net's device current before the call");
    void *base = nullptr;
    e = static_scratch_address(cur, &base);
    if (e != cudaSuccess)
        return set_last_error(EXAGO_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                               cudaGetErrorString(e));
    EvalReq R{};
    R.B = bt->B;
    R.x = bt->x; R.lam = bt->lambda; R.mask = bt->mask; R.gen_mask = bt->gen_mask;
    R.pd_scale = bt->pd_scale; R.obj_weight = bt->obj_weight; R.sigma = bt->obj_factor;
    R.f = f; R.grad = grad; R.gh = gh; R.jval = jval; R.hval = hval;
    R.scratch = (double *)base;
    R.stage_cap = multi_kernel_stage_cap(net);   // as the multi-kernel schedule stages its rows
    int le = launch_eval(*dev, R, bt->stream);
    if (le != 0) return set_last_error(EXAGO_ECUDA, cudaGetErrorString((cudaError_t)le));
    return EXAGO_OK;
}
