// Coupling (ramp) rows between the states of a batch: the linear constraints that tie the
// subproblems of ExaGO's multi-stage problems together -- consecutive periods (Sec. IV, eq. (15)),
// each contingency to the base case (Sec. V-A, eq. (20)), each scenario to the base scenario
// (Sec. VI-A, eq. (31)), and any tree of them (the general form, Sec. I, eqs. (5)-(6)).  Each state
// b has a parent p(b) in the same batch (-1 for none), and the generators' real power is the
// ramp-limited quantity, one row per (b, k):
//     r[b][k] = Pg_k(x_b) - Pg_k(x_p(b)).
// The rows are linear, so C x is also their Jacobian-vector product, their Jacobian values are the
// constants +1 / -1, and they add nothing to the Lagrangian Hessian.  The transpose product is a
// gather over each state's children, in a fixed order (no atomics):
//     (C^T nu)[b][Pg_k] = [p(b) >= 0] nu[b][k] - sum over children c of b of nu[c][k].
// States with few children are summed by one thread per (state, generator); a state with many
// children (the base case of a contingency or scenario batch) is summed by blocks of 8 generators
// whose 32 rows of threads take every 32nd child of the list staged in shared memory and then
// reduce in a fixed tree.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

struct exago_coupling {
    int B = 0, nb = 0, ng = 0, n = 0;
    bool on_device = false;
    int device = -1;
    std::vector<int> parent, child_ptr, child_idx, light, heavy;
    int *d_parent = nullptr, *d_child_ptr = nullptr, *d_child_idx = nullptr;
    int *d_light = nullptr, *d_heavy = nullptr;
    void *d_mem = nullptr;
};

namespace {

using exago::set_last_error;

// A state with more children than this is reduced by blocks of (8 generators x 32 child lanes).
constexpr int kHeavyChildren = 8;
constexpr int kMaxGridY = 65535;
// Children of a heavy state staged in shared memory per pass.
constexpr int kStageChildren = 2048;

// Values per thread along a row: every load of a thread is issued before its first store.
constexpr int kUnroll = 4;
constexpr int kRowSpan = 256 * kUnroll;   // values of one row per block

// Block (256 threads) per (state b0 + blockIdx.y, kRowSpan generators): one subtraction per value.
// The state and its parent are uniform over the block.
__global__ void __launch_bounds__(256) k_coupling(const int *__restrict__ parent, int b0, int n,
                                                  int nb, int ng, const double *__restrict__ x,
                                                  double *__restrict__ r) {
    const int b = b0 + blockIdx.y;
    const int p = __ldg(parent + b);
    const double *xb = x + (int64_t)b * n + 2 * nb;
    const double *xp = x + (int64_t)(p < 0 ? b : p) * n + 2 * nb;
    double *rb = r + (int64_t)b * ng;
    const int k0 = blockIdx.x * kRowSpan + threadIdx.x;
    double own[kUnroll], par[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
        const int k = k0 + u * 256;
        own[u] = k < ng && p >= 0 ? __ldg(xb + k) : 0.0;
        par[u] = k < ng && p >= 0 ? __ldg(xp + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
        const int k = k0 + u * 256;
        if (k < ng) rb[k] = p < 0 ? 0.0 : own[u] - par[u];
    }
}

__device__ __forceinline__ void put(double *o, double v, int accumulate) {
    *o = accumulate ? *o + v : v;
}

// Block (256 threads) per (listed state, kRowSpan generators): its own row's multiplier minus its
// children's, the children in ascending order.  The state's child range is uniform over the block.
__global__ void __launch_bounds__(256) k_coupling_jtv_light(
    const int *__restrict__ light, int j0, const int *__restrict__ parent,
    const int *__restrict__ cptr, const int *__restrict__ cidx, int ng,
    const double *__restrict__ nu, double *out, int64_t ldo, int accumulate) {
    const int s = __ldg(light + j0 + blockIdx.y);
    const bool own = __ldg(parent + s) >= 0;
    const int c0 = __ldg(cptr + s), c1 = __ldg(cptr + s + 1);
    const double *ns = nu + (int64_t)s * ng;
    double *os = out + (int64_t)s * ldo;
    const int k0 = blockIdx.x * kRowSpan + threadIdx.x;
    double v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
        const int k = k0 + u * 256;
        v[u] = own && k < ng ? __ldg(ns + k) : 0.0;
    }
    for (int c = c0; c < c1; c++) {
        const double *nc = nu + (int64_t)__ldg(cidx + c) * ng;
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int k = k0 + u * 256;
            if (k < ng) v[u] -= __ldg(nc + k);
        }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
        const int k = k0 + u * 256;
        if (k < ng) put(os + k, v[u], accumulate);
    }
}

// Block (8 x 32) per (listed state, 8 generators): the state's children are staged in shared
// memory, thread row ty sums children ty, ty + 32, ... (independent loads), and the 32 partial
// sums are reduced by a fixed halving tree.
__global__ void __launch_bounds__(256) k_coupling_jtv_heavy(
    const int *__restrict__ heavy, int h0, const int *__restrict__ parent,
    const int *__restrict__ cptr, const int *__restrict__ cidx, int ng,
    const double *__restrict__ nu, double *out, int64_t ldo, int accumulate) {
    __shared__ int kids[kStageChildren];
    __shared__ double part[32][9];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 8 + tx;
    const int s = __ldg(heavy + h0 + blockIdx.y);
    const int k = blockIdx.x * 8 + tx;
    const int c0 = __ldg(cptr + s), c1 = __ldg(cptr + s + 1);
    double acc = 0.0;
    for (int base = c0; base < c1; base += kStageChildren) {
        const int cnt = min(kStageChildren, c1 - base);
        __syncthreads();   // the previous pass is done with kids
        for (int j = tid; j < cnt; j += 256) kids[j] = __ldg(cidx + base + j);
        __syncthreads();
        if (k < ng) {
#pragma unroll 8
            for (int j = ty; j < cnt; j += 32) acc += __ldg(nu + (int64_t)kids[j] * ng + k);
        }
    }
    part[ty][tx] = acc;
    __syncthreads();
    for (int h = 16; h >= 1; h >>= 1) {
        if (ty < h) part[ty][tx] += part[ty + h][tx];
        __syncthreads();
    }
    if (ty == 0 && k < ng) {
        const double own = __ldg(parent + s) >= 0 ? __ldg(nu + (int64_t)s * ng + k) : 0.0;
        put(out + (int64_t)s * ldo + k, own - part[0][tx], accumulate);
    }
}

exago_status check_call(exago_coupling_t c) {
    if (!c) return set_last_error(EXAGO_EINVAL, "coupling is NULL");
    if (!c->on_device)
        return set_last_error(EXAGO_ESTATE, "coupling was built on a net planned without a device");
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
    if (cur != c->device)
        return set_last_error(EXAGO_EINVAL, "make the coupling's device current before the call");
    return EXAGO_OK;
}

// Blocks along a row of ng values: one 256-thread block per kRowSpan values.
unsigned row_blocks(int ng) { return (unsigned)((ng + kRowSpan - 1) / kRowSpan); }

}  // namespace

extern "C" {

exago_status exago_coupling_create(exago_net_t net, int B, const int *parent,
                                   exago_coupling_t *out) {
    if (!out) return set_last_error(EXAGO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!net) return set_last_error(EXAGO_EINVAL, "net is NULL");
    if (B < 0) return set_last_error(EXAGO_EINVAL, "B < 0");
    if (B > 0 && !parent) return set_last_error(EXAGO_EINVAL, "parent is NULL");
    int n = 0, meq = 0, mineq = 0;
    int64_t nnzJ = 0, nnzH = 0;
    exago_status st = exago_net_dims(net, &n, &meq, &mineq, &nnzJ, &nnzH);
    if (st != EXAGO_OK) return st;
    for (int b = 0; b < B; b++) {
        const int p = parent[b];
        if (p < -1 || p >= B || p == b)
            return set_last_error(EXAGO_EINVAL, "parent[" + std::to_string(b) + "] = " +
                                                    std::to_string(p) +
                                                    ": must be -1 or another state of the batch");
    }
    exago_coupling *c = new (std::nothrow) exago_coupling;
    if (!c) return set_last_error(EXAGO_ENOMEM, "host allocation");
    c->B = B;
    c->nb = meq / 2;
    c->n = n;
    c->ng = (n - meq) / 2;   // n = 2 nb + 2 ng, m_eq = 2 nb
    c->parent.assign(parent, parent + B);
    c->child_ptr.assign(B + 1, 0);
    for (int b = 0; b < B; b++)
        if (parent[b] >= 0) c->child_ptr[parent[b] + 1]++;
    for (int b = 0; b < B; b++) c->child_ptr[b + 1] += c->child_ptr[b];
    c->child_idx.resize(c->child_ptr[B]);
    {
        std::vector<int> fill(c->child_ptr.begin(), c->child_ptr.end() - 1);
        for (int b = 0; b < B; b++)   // ascending child order
            if (parent[b] >= 0) c->child_idx[fill[parent[b]]++] = b;
    }
    for (int b = 0; b < B; b++)
        (c->child_ptr[b + 1] - c->child_ptr[b] > kHeavyChildren ? c->heavy : c->light).push_back(b);

    const exago::HostPlan *plan = nullptr;
    const exago::DevNet *dev = nullptr;
    if (exago::net_internal_view(net, &plan, &dev, &c->device)) {
        c->on_device = true;
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess || cur != c->device) {
            delete c;
            return set_last_error(e != cudaSuccess ? EXAGO_ECUDA : EXAGO_EINVAL,
                                  e != cudaSuccess ? cudaGetErrorString(e)
                                                   : "make the net's device current before the call");
        }
        // one allocation: parent [B], child_ptr [B + 1], child_idx, light, heavy
        const size_t ints = (size_t)B + (B + 1) + c->child_idx.size() + c->light.size() + c->heavy.size();
        e = exago::dev_malloc(&c->d_mem, std::max<size_t>(ints, 1) * sizeof(int));
        if (e != cudaSuccess) {
            delete c;
            return set_last_error(EXAGO_ENOMEM, "cudaMalloc (coupling tables)");
        }
        std::vector<int> all;
        all.reserve(ints);
        all.insert(all.end(), c->parent.begin(), c->parent.end());
        all.insert(all.end(), c->child_ptr.begin(), c->child_ptr.end());
        all.insert(all.end(), c->child_idx.begin(), c->child_idx.end());
        all.insert(all.end(), c->light.begin(), c->light.end());
        all.insert(all.end(), c->heavy.begin(), c->heavy.end());
        if (!all.empty()) {
            e = cudaMemcpy(c->d_mem, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(c->d_mem);
                delete c;
                return set_last_error(EXAGO_ECUDA, std::string("cudaMemcpy (coupling tables): ") +
                                                       cudaGetErrorString(e));
            }
        }
        int *p = (int *)c->d_mem;
        c->d_parent = p;
        p += B;
        c->d_child_ptr = p;
        p += B + 1;
        c->d_child_idx = p;
        p += c->child_idx.size();
        c->d_light = p;
        p += c->light.size();
        c->d_heavy = p;
    }
    *out = c;
    return EXAGO_OK;
}

exago_status exago_coupling_destroy(exago_coupling_t c) {
    if (!c) return EXAGO_OK;
    if (c->d_mem) cudaFree(c->d_mem);
    delete c;
    return EXAGO_OK;
}

exago_status exago_coupling_dims(exago_coupling_t c, int *B, int64_t *rows, int64_t *nnz) {
    if (!c) return set_last_error(EXAGO_EINVAL, "coupling is NULL");
    int64_t coupled = 0;
    for (int p : c->parent) coupled += p >= 0;
    if (B) *B = c->B;
    if (rows) *rows = (int64_t)c->B * c->ng;
    if (nnz) *nnz = 2 * coupled * c->ng;
    return EXAGO_OK;
}

exago_status exago_coupling_jac_pattern(exago_coupling_t c, int64_t *rowptr, int64_t *col,
                                        double *val) {
    if (!c) return set_last_error(EXAGO_EINVAL, "coupling is NULL");
    if (!rowptr || !col) return set_last_error(EXAGO_EINVAL, "rowptr or col is NULL");
    int64_t q = 0;
    rowptr[0] = 0;
    for (int b = 0; b < c->B; b++) {
        const int p = c->parent[b];
        for (int k = 0; k < c->ng; k++) {
            if (p >= 0) {
                const int64_t cb = (int64_t)b * c->n + 2 * c->nb + k;
                const int64_t cp = (int64_t)p * c->n + 2 * c->nb + k;
                const bool self_first = cb < cp;
                col[q] = self_first ? cb : cp;
                col[q + 1] = self_first ? cp : cb;
                if (val) {
                    val[q] = self_first ? 1.0 : -1.0;
                    val[q + 1] = self_first ? -1.0 : 1.0;
                }
                q += 2;
            }
            rowptr[(int64_t)b * c->ng + k + 1] = q;
        }
    }
    return EXAGO_OK;
}

exago_status exago_eval_coupling(exago_coupling_t c, const double *x, double *r, void *stream) {
    exago_status st = check_call(c);
    if (st != EXAGO_OK) return st;
    if (c->B == 0 || c->ng == 0) return EXAGO_OK;
    if (!x || !r) return set_last_error(EXAGO_EINVAL, "x or r is NULL");
    for (int b0 = 0; b0 < c->B; b0 += kMaxGridY) {
        const int nbk = std::min(kMaxGridY, c->B - b0);
        k_coupling<<<dim3(row_blocks(c->ng), nbk), 256, 0, (cudaStream_t)stream>>>(
            c->d_parent, b0, c->n, c->nb, c->ng, x, r);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_last_error(EXAGO_ECUDA, std::string("coupling launch: ") + cudaGetErrorString(e));
    return EXAGO_OK;
}

exago_status exago_eval_coupling_jtv(exago_coupling_t c, const double *nu, double *out,
                                     int64_t ldo, int accumulate, void *stream) {
    exago_status st = check_call(c);
    if (st != EXAGO_OK) return st;
    if (c->B == 0 || c->ng == 0) return EXAGO_OK;
    if (!nu || !out) return set_last_error(EXAGO_EINVAL, "nu or out is NULL");
    if (ldo < c->ng) return set_last_error(EXAGO_EINVAL, "ldo < ng");
    cudaStream_t s = (cudaStream_t)stream;
    const int nlight = (int)c->light.size(), nheavy = (int)c->heavy.size();
    for (int j0 = 0; j0 < nlight; j0 += kMaxGridY) {
        const int nj = std::min(kMaxGridY, nlight - j0);
        k_coupling_jtv_light<<<dim3(row_blocks(c->ng), nj), 256, 0, s>>>(
            c->d_light, j0, c->d_parent, c->d_child_ptr, c->d_child_idx, c->ng, nu, out, ldo,
            accumulate ? 1 : 0);
    }
    for (int h0 = 0; h0 < nheavy; h0 += kMaxGridY) {
        const int nh = std::min(kMaxGridY, nheavy - h0);
        k_coupling_jtv_heavy<<<dim3((c->ng + 7) / 8, nh), dim3(8, 32), 0, s>>>(
            c->d_heavy, h0, c->d_parent, c->d_child_ptr, c->d_child_idx, c->ng, nu, out, ldo,
            accumulate ? 1 : 0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_last_error(EXAGO_ECUDA, std::string("coupling transpose launch: ") +
                                               cudaGetErrorString(e));
    return EXAGO_OK;
}

}  // extern "C"
