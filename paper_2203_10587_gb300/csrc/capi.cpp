// C ABI of the evaluator (declared in include/exago.h): network lifetime, pattern queries and the
// evaluation entry points of the polar AC-OPF model (ExaGO, Sec. III, eqs. (7)-(10)).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace exago;

namespace {

thread_local std::string g_err;

exago_status fail(exago_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

exago_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? EXAGO_ENOMEM : EXAGO_ECUDA, m);
}

}  // namespace

struct exago_net {
    HostPlan plan;
    bool on_device = false;
    int device = -1;
    DevNet dev{};
    std::vector<void *> allocs;
    int *status_host = nullptr;   // host-mapped device status word
    void *ws = nullptr;           // internal workspace
    size_t ws_bytes = 0;
    std::mutex mu;                // guards workspace growth
};

namespace {

template <typename T>
exago_status upload(exago_net *net, const std::vector<T> &v, const T **out) {
    *out = nullptr;
    if (v.empty()) return EXAGO_OK;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, v.size() * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (network arrays)");
    net->allocs.push_back(p);
    e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (network arrays)");
    *out = (const T *)p;
    return EXAGO_OK;
}

exago_status alloc_dev(exago_net *net, size_t bytes, double **out) {
    *out = nullptr;
    if (bytes == 0) return EXAGO_OK;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (admittances)");
    net->allocs.push_back(p);
    *out = (double *)p;
    return EXAGO_OK;
}

void free_device(exago_net *net) {
    for (void *p : net->allocs) cudaFree(p);
    net->allocs.clear();
    if (net->ws) cudaFree(net->ws);
    net->ws = nullptr;
    net->ws_bytes = 0;
    if (net->status_host) cudaFreeHost(net->status_host);
    net->status_host = nullptr;
    net->on_device = false;
}

exago_status do_upload(exago_net *net) {
    const HostPlan &p = net->plan;
    DevNet &d = net->dev;
    exago_status s;
    cudaError_t e = cudaGetDevice(&net->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    d = DevNet{};
    d.nb = p.nb; d.nl = p.nl; d.ng = p.ng; d.n = p.n; d.m = p.m;
    d.nslot = p.nslot;
    d.nslot_pad = (p.nslot + 31) / 32 * 32;
    d.nshared = p.nshared;
    d.nfix = (int)p.fix_dst.size();
    d.nnzJ = p.nnzJ; d.nnzJg = p.nnzJg; d.nnzH = p.nnzH;
    d.baseMVA = p.baseMVA;
#define UP(field, vec) if ((s = upload(net, p.vec, &d.field)) != EXAGO_OK) return s
    UP(f, f); UP(t, t);
    UP(br_off, br_off); UP(br_slot, br_slot); UP(br_shared, br_shared);
    UP(slot_ptr, slot_ptr);
    UP(bus_jP, bus_jP); UP(bus_jQ, bus_jQ); UP(bus_k, bus_k); UP(bus_h, bus_h);
    UP(Gs, Gs); UP(Bs, Bs); UP(Pd, Pd); UP(Qd, Qd);
    UP(gen_ptr, gen_ptr); UP(gen_ord, gen_ord); UP(gen_bus, gbus);
    UP(gen_jP, gen_jP); UP(gen_jQ, gen_jQ); UP(gen_h, gen_h);
    UP(c2, c2); UP(c1, c1); UP(c0, c0);
    UP(fix_ptr, fix_ptr); UP(fix_src, fix_src); UP(fix_dst, fix_dst); UP(fix_isH, fix_isH);
#undef UP
    // branch parameters, then the pi-model admittances evaluated on the device
    const double *r = nullptr, *x = nullptr, *b = nullptr, *tap = nullptr;
    if ((s = upload(net, p.r, &r)) != EXAGO_OK) return s;
    if ((s = upload(net, p.x, &x)) != EXAGO_OK) return s;
    if ((s = upload(net, p.b, &b)) != EXAGO_OK) return s;
    if ((s = upload(net, p.tap, &tap)) != EXAGO_OK) return s;
    double *Y[6];
    for (int k = 0; k < 6; k++)
        if ((s = alloc_dev(net, (size_t)p.nl * sizeof(double), &Y[k])) != EXAGO_OK) return s;
    d.Gff = Y[0]; d.Bff = Y[1]; d.Gtt = Y[2]; d.Btt = Y[3]; d.Gft = Y[4]; d.Bft = Y[5];
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    int le = launch_admittance(r, x, b, tap, p.nl, Y[0], Y[1], Y[2], Y[3], Y[4], Y[5], st);
    e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (le != 0) return cuda_fail((cudaError_t)le, "admittance kernel launch");
    if (e != cudaSuccess) return cuda_fail(e, "admittance kernel");
    e = cudaHostAlloc((void **)&net->status_host, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc (status word)");
    *net->status_host = 0;
    e = cudaHostGetDevicePointer((void **)&d.status, net->status_host, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostGetDevicePointer (status word)");
    net->on_device = true;
    return EXAGO_OK;
}

exago_status plan_only(int nb, const double *Gs, const double *Bs, const double *Pd,
                       const double *Qd, int nl, const int *f, const int *t, const double *r,
                       const double *x, const double *b, const double *tap, const double *rateA,
                       int ng, const int *gbus, const double *c2, const double *c1,
                       const double *c0, double baseMVA, exago_net_t *out) {
    if (!out) return fail(EXAGO_EINVAL, "out is NULL");
    *out = nullptr;
    exago_net *net = new (std::nothrow) exago_net();
    if (!net) return fail(EXAGO_ENOMEM, "host allocation failed");
    std::string err;
    exago_status s;
    try {
        s = build_plan(net->plan, nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus,
                       c2, c1, c0, baseMVA, err);
    } catch (const std::bad_alloc &) {
        s = EXAGO_ENOMEM;
        err = "host allocation failed while planning";
    }
    if (s != EXAGO_OK) {
        delete net;
        return fail(s, err);
    }
    *out = net;
    return EXAGO_OK;
}

exago_status check_batch(exago_net *net, const exago_batch *bt, bool need_lam) {
    if (!net) return fail(EXAGO_EINVAL, "net is NULL");
    if (!net->on_device) return fail(EXAGO_ESTATE, "net was planned without a device (exago_net_plan)");
    if (!bt) return fail(EXAGO_EINVAL, "batch is NULL");
    if (bt->B < 0) return fail(EXAGO_EINVAL, "batch B < 0");
    if (bt->B == 0) return EXAGO_OK;
    if (!bt->x) return fail(EXAGO_EINVAL, "batch x is NULL");
    if (need_lam && !bt->lambda) return fail(EXAGO_EINVAL, "batch lambda is NULL (needed by the Hessian)");
    if (bt->workspace) {
        if (((uintptr_t)bt->workspace & 255) != 0) return fail(EXAGO_EINVAL, "workspace not 256-byte aligned");
        if (bt->workspace_bytes < workspace_bytes(net->plan, bt->B))
            return fail(EXAGO_EINVAL, "workspace smaller than exago_eval_workspace_size");
    }
    return EXAGO_OK;
}

exago_status ensure_workspace(exago_net *net, int B) {
    size_t need = workspace_bytes(net->plan, B);
    std::lock_guard<std::mutex> lk(net->mu);
    if (net->ws_bytes >= need) return EXAGO_OK;
    if (net->ws) {
        cudaError_t e = cudaDeviceSynchronize();   // earlier work may still use the old buffer
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize (workspace growth)");
        cudaFree(net->ws);
        net->ws = nullptr;
        net->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&net->ws, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (workspace)");
    net->ws_bytes = need;
    return EXAGO_OK;
}

exago_status eval(exago_net *net, const exago_batch *bt, double *f, double *grad, double *gh,
                  double *jval, double *hval, ProfileHook *hook = nullptr) {
    exago_status s = check_batch(net, bt, hval != nullptr);
    if (s != EXAGO_OK || bt->B == 0) return s;
    void *ws = bt->workspace;
    if (!ws && (gh || jval || hval)) {
        if ((s = ensure_workspace(net, bt->B)) != EXAGO_OK) return s;
        ws = net->ws;
    }
    const HostPlan &p = net->plan;
    EvalReq R{};
    R.B = bt->B;
    R.x = bt->x; R.lam = bt->lambda; R.mask = bt->mask;
    R.pd_scale = bt->pd_scale; R.obj_weight = bt->obj_weight; R.sigma = bt->obj_factor;
    R.f = f; R.grad = grad; R.gh = gh; R.jval = jval; R.hval = hval;
    if (ws) {
        char *w = (char *)ws;
        const size_t pad = (size_t)net->dev.nslot_pad;
        R.scratch = (double *)w;
        w += ((size_t)bt->B * NCOMP * pad * sizeof(double) + 255) / 256 * 256;
        R.offscratch = (double *)w;
    }
    int e = launch_eval(net->dev, R, bt->stream, hook);
    if (e != 0) return cuda_fail((cudaError_t)e, "evaluation kernel launch");
    return EXAGO_OK;
}

}  // namespace

namespace exago {

bool net_internal_view(exago_net_t net, const HostPlan **plan, const DevNet **dev, int *device) {
    if (!net || !net->on_device) return false;
    *plan = &net->plan;
    *dev = &net->dev;
    *device = net->device;
    return true;
}

exago_status set_last_error(exago_status s, const std::string &msg) { return fail(s, msg); }

}  // namespace exago

extern "C" {

const char *exago_last_error(void) { return g_err.c_str(); }

const char *exago_status_name(exago_status s) {
    switch (s) {
        case EXAGO_OK: return "EXAGO_OK";
        case EXAGO_EINVAL: return "EXAGO_EINVAL";
        case EXAGO_ENOMEM: return "EXAGO_ENOMEM";
        case EXAGO_ECUDA: return "EXAGO_ECUDA";
        case EXAGO_ETIMEOUT: return "EXAGO_ETIMEOUT";
        case EXAGO_EBUSY: return "EXAGO_EBUSY";
        case EXAGO_ESTATE: return "EXAGO_ESTATE";
    }
    return "EXAGO_UNKNOWN";
}

exago_status exago_net_plan(int nb, const double *Gs, const double *Bs, const double *Pd,
                            const double *Qd, int nl, const int *f, const int *t,
                            const double *r, const double *x, const double *b,
                            const double *tap, const double *rateA, int ng, const int *gbus,
                            const double *c2, const double *c1, const double *c0,
                            double baseMVA, exago_net_t *out) {
    return plan_only(nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus, c2, c1, c0,
                     baseMVA, out);
}

exago_status exago_net_create(int nb, const double *Gs, const double *Bs, const double *Pd,
                              const double *Qd, int nl, const int *f, const int *t,
                              const double *r, const double *x, const double *b,
                              const double *tap, const double *rateA, int ng, const int *gbus,
                              const double *c2, const double *c1, const double *c0,
                              double baseMVA, exago_net_t *out) {
    exago_status s = plan_only(nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus, c2,
                               c1, c0, baseMVA, out);
    if (s != EXAGO_OK) return s;
    s = do_upload(*out);
    if (s != EXAGO_OK) {
        std::string keep = g_err;
        free_device(*out);
        delete *out;
        *out = nullptr;
        g_err = keep;
    }
    return s;
}

exago_status exago_net_destroy(exago_net_t net) {
    if (!net) return EXAGO_OK;
    free_device(net);
    delete net;
    return EXAGO_OK;
}

exago_status exago_net_dims(exago_net_t net, int *n, int *m_eq, int *m_ineq, int64_t *nnzJ,
                            int64_t *nnzH) {
    if (!net) return fail(EXAGO_EINVAL, "net is NULL");
    if (n) *n = net->plan.n;
    if (m_eq) *m_eq = 2 * net->plan.nb;
    if (m_ineq) *m_ineq = 2 * net->plan.nl;
    if (nnzJ) *nnzJ = net->plan.nnzJ;
    if (nnzH) *nnzH = net->plan.nnzH;
    return EXAGO_OK;
}

exago_status exago_net_jac_pattern(exago_net_t net, int64_t *rowptr, int *col) {
    if (!net || !rowptr || (!col && net->plan.nnzJ > 0)) return fail(EXAGO_EINVAL, "null argument");
    std::memcpy(rowptr, net->plan.Jrowptr.data(), net->plan.Jrowptr.size() * sizeof(int64_t));
    if (net->plan.nnzJ) std::memcpy(col, net->plan.Jcol.data(), net->plan.Jcol.size() * sizeof(int));
    return EXAGO_OK;
}

exago_status exago_net_hess_pattern(exago_net_t net, int64_t *rowptr, int *col) {
    if (!net || !rowptr || (!col && net->plan.nnzH > 0)) return fail(EXAGO_EINVAL, "null argument");
    std::memcpy(rowptr, net->plan.Hrowptr.data(), net->plan.Hrowptr.size() * sizeof(int64_t));
    if (net->plan.nnzH) std::memcpy(col, net->plan.Hcol.data(), net->plan.Hcol.size() * sizeof(int));
    return EXAGO_OK;
}

exago_status exago_net_ineq_bounds(exago_net_t net, double *hlo, double *hhi) {
    if (!net || (net->plan.nl > 0 && (!hlo || !hhi))) return fail(EXAGO_EINVAL, "null argument");
    const int nl = net->plan.nl;
    for (int l = 0; l < nl; l++) {
        double ra = net->plan.rateA[l];
        double hi = ra == 0.0 ? HUGE_VAL : ra * ra;
        hlo[l] = hlo[nl + l] = 0.0;
        hhi[l] = hhi[nl + l] = hi;
    }
    return EXAGO_OK;
}

exago_status exago_net_plan_array(exago_net_t net, const char *name, void *dst, size_t bytes,
                                  size_t *needed) {
    if (!net || !name) return fail(EXAGO_EINVAL, "null argument");
    const HostPlan &p = net->plan;
    const void *src = nullptr;
    size_t n = 0;
#define ARR(key, vec) if (!std::strcmp(name, key)) { src = p.vec.data(); n = p.vec.size() * sizeof(p.vec[0]); }
    ARR("br_off", br_off) else ARR("br_slot", br_slot) else ARR("br_shared", br_shared)
    else ARR("slot_ptr", slot_ptr) else ARR("bus_jP", bus_jP) else ARR("bus_jQ", bus_jQ)
    else ARR("bus_k", bus_k) else ARR("bus_h", bus_h) else ARR("gen_ptr", gen_ptr)
    else ARR("gen_ord", gen_ord) else ARR("gen_jP", gen_jP) else ARR("gen_jQ", gen_jQ)
    else ARR("gen_h", gen_h) else ARR("fix_ptr", fix_ptr) else ARR("fix_src", fix_src)
    else ARR("fix_dst", fix_dst) else ARR("fix_isH", fix_isH)
    else return fail(EXAGO_EINVAL, std::string("unknown plan array ") + name);
#undef ARR
    if (needed) *needed = n;
    if (dst) {
        if (bytes < n) return fail(EXAGO_EINVAL, "destination too small");
        if (n) std::memcpy(dst, src, n);
    }
    return EXAGO_OK;
}

exago_status exago_eval_workspace_size(exago_net_t net, int B, size_t *bytes) {
    if (!net || !bytes || B < 0) return fail(EXAGO_EINVAL, "bad argument");
    *bytes = workspace_bytes(net->plan, B);
    return EXAGO_OK;
}

exago_status exago_net_reserve(exago_net_t net, int B) {
    if (!net || B < 0) return fail(EXAGO_EINVAL, "bad argument");
    if (!net->on_device) return fail(EXAGO_ESTATE, "net was planned without a device");
    return ensure_workspace(net, B);
}

exago_status exago_eval_obj(exago_net_t net, const exago_batch *bt, double *f) {
    if (!f) return fail(EXAGO_EINVAL, "f is NULL");
    return eval(net, bt, f, nullptr, nullptr, nullptr, nullptr);
}

exago_status exago_eval_grad(exago_net_t net, const exago_batch *bt, double *grad) {
    if (!grad) return fail(EXAGO_EINVAL, "grad is NULL");
    return eval(net, bt, nullptr, grad, nullptr, nullptr, nullptr);
}

exago_status exago_eval_cons(exago_net_t net, const exago_batch *bt, double *gh) {
    if (!gh) return fail(EXAGO_EINVAL, "gh is NULL");
    return eval(net, bt, nullptr, nullptr, gh, nullptr, nullptr);
}

exago_status exago_eval_jac(exago_net_t net, const exago_batch *bt, double *jval) {
    if (!jval) return fail(EXAGO_EINVAL, "jval is NULL");
    return eval(net, bt, nullptr, nullptr, nullptr, jval, nullptr);
}

exago_status exago_eval_hess(exago_net_t net, const exago_batch *bt, double *hval) {
    if (!hval) return fail(EXAGO_EINVAL, "hval is NULL");
    return eval(net, bt, nullptr, nullptr, nullptr, nullptr, hval);
}

exago_status exago_eval_all(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                            double *gh, double *jval, double *hval) {
    return eval(net, bt, f, grad, gh, jval, hval);
}

exago_status exago_eval_profile(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                                double *gh, double *jval, double *hval, int reps, int *nkernels,
                                const char **names, double *ms) {
    if (reps < 1 || !nkernels || !names || !ms) return fail(EXAGO_EINVAL, "bad profile arguments");
    exago_status s = check_batch(net, bt, hval != nullptr);
    if (s != EXAGO_OK) return s;
    *nkernels = 0;
    if (bt->B == 0) return EXAGO_OK;
    ProfileHook hk;
    for (int i = 0; i < ProfileHook::MAX; i++) {
        cudaError_t e = cudaEventCreate(&hk.ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; j++) cudaEventDestroy(hk.ev[j]);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    double acc[ProfileHook::MAX] = {0};
    int nk = 0;
    for (int r = 0; r < reps && s == EXAGO_OK; r++) {
        hk.n = 0;
        s = eval(net, bt, f, grad, gh, jval, hval, &hk);
        if (s != EXAGO_OK) break;
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)bt->stream);
        if (e != cudaSuccess) { s = cuda_fail(e, "cudaStreamSynchronize (profile)"); break; }
        nk = hk.n - 1;
        for (int k = 0; k < nk; k++) {
            float t = 0.f;
            cudaEventElapsedTime(&t, hk.ev[k], hk.ev[k + 1]);
            acc[k] += t;
            names[k] = hk.name[k];
        }
    }
    for (int i = 0; i < ProfileHook::MAX; i++) cudaEventDestroy(hk.ev[i]);
    if (s != EXAGO_OK) return s;
    *nkernels = nk;
    for (int k = 0; k < nk; k++) ms[k] = acc[k] / reps;
    return EXAGO_OK;
}

exago_status exago_net_check(exago_net_t net, void *stream) {
    if (!net) return fail(EXAGO_EINVAL, "net is NULL");
    if (!net->on_device) return fail(EXAGO_ESTATE, "net was planned without a device");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int v = *(volatile int *)net->status_host;
    if (v != 0) {
        *(volatile int *)net->status_host = 0;
        char msg[128];
        snprintf(msg, sizeof msg, "a bounded device-side wait gave up (code %d)", v);
        return fail(EXAGO_ETIMEOUT, msg);
    }
    return EXAGO_OK;
}

}  // extern "C"
