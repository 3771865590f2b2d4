// Feasibility slacks of the AC-OPF model: load loss and power imbalance (ExaGO, arXiv 2203.10587,
// Sec. III, Fig. 2).  Each slack z_k >= 0 sits at one bus, in the P or the Q balance, with sign
// +1 or -1 and a linear cost: it adds sign z_k to that balance and w cost_k z_k to the objective;
// its Jacobian column is the constant sign in that row and the Hessian gets nothing.  The terms
// are applied to a finished evaluation (exago_eval_* outputs) by three small kernels:
//   * rows: one thread per (balance row with slacks, group of 8 states) adds the row's slacks in
//     ascending slack order to each state's value (the same additions, in the same order, as the
//     definition);
//   * objective: one block per state sums cost_k z_k (four partial sums per thread, then a fixed
//     256-lane tree) and adds w times the sum to f; the gradient w cost_k by its own kernel;
//   * transpose: one thread per (state, slack) gathers sign_k v[row_k].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

struct exago_slack {
    int nb = 0, nz = 0;
    bool on_device = false;
    int device = -1;
    std::vector<int> bus, row, sign;
    std::vector<double> cost;
    std::vector<int> grow;              // [nz] balance row of each slack: row nb + bus
    std::vector<int> rptr, rlist, used; // CSR of the slacks by balance row; rows that have some
    int *d_int = nullptr;               // grow, sign, rptr, rlist, used
    double *d_cost = nullptr;
    void *d_mem = nullptr;
};

namespace {

using exago::set_last_error;

constexpr int kLanes = 256;
constexpr int kMaxGridY = 65535;

// Balance rows: one thread per (balance row with slacks, group of kGroup states).  The row's slack
// list is read once for the group; each state's value gets the row's slacks in ascending order
// (the definition's additions in the definition's order), the group's loads issued together.
constexpr int kGroup = 8;
__global__ void __launch_bounds__(128) k_slack_rows(const int *__restrict__ used, int nused,
                                                    const int *__restrict__ rptr,
                                                    const int *__restrict__ rlist,
                                                    const int *__restrict__ sign, int nz, int b0,
                                                    int nB, const double *__restrict__ z,
                                                    double *gh, int64_t ldgh) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nused) return;
    const int g0 = b0 + blockIdx.y * kGroup;
    const int ns = min(kGroup, b0 + nB - g0);
    const int r = __ldg(used + j);
    double v[kGroup];
#pragma unroll
    for (int t = 0; t < kGroup; t++)
        if (t < ns) v[t] = gh[(int64_t)(g0 + t) * ldgh + r];
    for (int q = __ldg(rptr + r), q1 = __ldg(rptr + r + 1); q < q1; q++) {
        const int k = __ldg(rlist + q);
        const double sk = __ldg(sign + k);
#pragma unroll
        for (int t = 0; t < kGroup; t++)
            if (t < ns) v[t] += sk * __ldg(z + (int64_t)(g0 + t) * nz + k);
    }
#pragma unroll
    for (int t = 0; t < kGroup; t++)
        if (t < ns) gh[(int64_t)(g0 + t) * ldgh + r] = v[t];
}

// Objective: one block per state; each thread keeps four partial sums over slacks t, t + 256,
// t + 512, t + 768, then t + 1024, ... (independent loads in flight), combined in a fixed order
// and then over a fixed 256-lane tree.
__global__ void __launch_bounds__(kLanes) k_slack_obj(const double *__restrict__ cost, int nz,
                                                      int b0, const double *__restrict__ z,
                                                      const double *__restrict__ obj_weight,
                                                      double *f) {
    __shared__ double part[kLanes];
    const int b = b0 + blockIdx.x;
    const double *zb = z + (int64_t)b * nz;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int k = threadIdx.x;
    for (; k + 3 * kLanes < nz; k += 4 * kLanes) {
        a0 = fma(__ldg(cost + k), __ldg(zb + k), a0);
        a1 = fma(__ldg(cost + k + kLanes), __ldg(zb + k + kLanes), a1);
        a2 = fma(__ldg(cost + k + 2 * kLanes), __ldg(zb + k + 2 * kLanes), a2);
        a3 = fma(__ldg(cost + k + 3 * kLanes), __ldg(zb + k + 3 * kLanes), a3);
    }
    for (; k < nz; k += kLanes) a0 = fma(__ldg(cost + k), __ldg(zb + k), a0);
    part[threadIdx.x] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    for (int h = kLanes / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) f[b] = fma(obj_weight ? __ldg(obj_weight + b) : 1.0, part[0], f[b]);
}

// Gradient w cost_k: blocks of 256 threads along each state's slacks, four values per thread.
__global__ void __launch_bounds__(256) k_slack_grad(const double *__restrict__ cost, int nz,
                                                    int b0, const double *__restrict__ obj_weight,
                                                    double *__restrict__ grad_z) {
    const int b = b0 + blockIdx.y;
    const double w = obj_weight ? __ldg(obj_weight + b) : 1.0;
    double *gb = grad_z + (int64_t)b * nz;
    const int k0 = blockIdx.x * 1024 + threadIdx.x;
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int k = k0 + u * 256;
        if (k < nz) gb[k] = w * __ldg(cost + k);
    }
}

__global__ void __launch_bounds__(256) k_slack_jtv(const int *__restrict__ grow,
                                                   const int *__restrict__ sign, int nz, int b0,
                                                   const double *__restrict__ v, int64_t ldv,
                                                   double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz) return;
    const int b = b0 + blockIdx.y;
    out[(int64_t)b * nz + k] = __ldg(sign + k) * __ldg(v + (int64_t)b * ldv + __ldg(grow + k));
}

exago_status check_call(exago_slack_t s, const exago_batch *bt) {
    if (!s) return set_last_error(EXAGO_EINVAL, "slack set is NULL");
    if (!s->on_device)
        return set_last_error(EXAGO_ESTATE, "slack set was built on a net planned without a device");
    if (!bt) return set_last_error(EXAGO_EINVAL, "batch is NULL");
    if (bt->B < 0) return set_last_error(EXAGO_EINVAL, "batch B < 0");
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
    if (cur != s->device)
        return set_last_error(EXAGO_EINVAL, "make the slack set's device current before the call");
    return EXAGO_OK;
}

}  // namespace

extern "C" {

exago_status exago_slack_create(exago_net_t net, int nz, const int *bus, const int *row,
                                const int *sign, const double *cost, exago_slack_t *out) {
    if (!out) return set_last_error(EXAGO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!net) return set_last_error(EXAGO_EINVAL, "net is NULL");
    if (nz < 0) return set_last_error(EXAGO_EINVAL, "nz < 0");
    if (nz > 0 && (!bus || !row || !sign || !cost))
        return set_last_error(EXAGO_EINVAL, "bus, row, sign or cost is NULL");
    int n = 0, meq = 0, mineq = 0;
    int64_t nnzJ = 0, nnzH = 0;
    exago_status st = exago_net_dims(net, &n, &meq, &mineq, &nnzJ, &nnzH);
    if (st != EXAGO_OK) return st;
    const int nb = meq / 2;
    for (int k = 0; k < nz; k++) {
        if (bus[k] < 0 || bus[k] >= nb || (row[k] != 0 && row[k] != 1) ||
            (sign[k] != 1 && sign[k] != -1) || !std::isfinite(cost[k]))
            return set_last_error(EXAGO_EINVAL, "slack " + std::to_string(k) +
                                                    ": bus out of range, row not 0 or 1, sign "
                                                    "not +1 or -1, or cost not finite");
    }
    exago_slack *s = new (std::nothrow) exago_slack;
    if (!s) return set_last_error(EXAGO_ENOMEM, "host allocation");
    s->nb = nb;
    s->nz = nz;
    s->bus.assign(bus, bus + nz);
    s->row.assign(row, row + nz);
    s->sign.assign(sign, sign + nz);
    s->cost.assign(cost, cost + nz);
    s->grow.resize(nz);
    s->rptr.assign(2 * nb + 1, 0);
    for (int k = 0; k < nz; k++) {
        s->grow[k] = row[k] * nb + bus[k];
        s->rptr[s->grow[k] + 1]++;
    }
    for (int r = 0; r < 2 * nb; r++) s->rptr[r + 1] += s->rptr[r];
    s->rlist.resize(nz);
    {
        std::vector<int> fill(s->rptr.begin(), s->rptr.end() - 1);
        for (int k = 0; k < nz; k++) s->rlist[fill[s->grow[k]]++] = k;   // ascending k per row
    }
    for (int r = 0; r < 2 * nb; r++)
        if (s->rptr[r + 1] > s->rptr[r]) s->used.push_back(r);

    const exago::HostPlan *plan = nullptr;
    const exago::DevNet *dev = nullptr;
    if (exago::net_internal_view(net, &plan, &dev, &s->device)) {
        s->on_device = true;
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess || cur != s->device) {
            delete s;
            return set_last_error(e != cudaSuccess ? EXAGO_ECUDA : EXAGO_EINVAL,
                                  e != cudaSuccess ? cudaGetErrorString(e)
                                                   : "make the net's device current before the call");
        }
        std::vector<int> ints;
        ints.insert(ints.end(), s->grow.begin(), s->grow.end());
        ints.insert(ints.end(), s->sign.begin(), s->sign.end());
        ints.insert(ints.end(), s->rptr.begin(), s->rptr.end());
        ints.insert(ints.end(), s->rlist.begin(), s->rlist.end());
        ints.insert(ints.end(), s->used.begin(), s->used.end());
        const size_t ibytes = (ints.size() * sizeof(int) + 255) / 256 * 256;
        const size_t bytes = ibytes + std::max<size_t>((size_t)nz, 1) * sizeof(double);
        e = exago::dev_malloc(&s->d_mem, bytes);
        if (e != cudaSuccess) {
            delete s;
            return set_last_error(EXAGO_ENOMEM, "cudaMalloc (slack tables)");
        }
        s->d_int = (int *)s->d_mem;
        s->d_cost = (double *)((char *)s->d_mem + ibytes);
        e = cudaMemcpy(s->d_int, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && nz > 0)
            e = cudaMemcpy(s->d_cost, s->cost.data(), nz * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(s->d_mem);
            delete s;
            return set_last_error(EXAGO_ECUDA, std::string("cudaMemcpy (slack tables): ") +
                                                   cudaGetErrorString(e));
        }
    }
    *out = s;
    return EXAGO_OK;
}

exago_status exago_slack_destroy(exago_slack_t s) {
    if (!s) return EXAGO_OK;
    if (s->d_mem) cudaFree(s->d_mem);
    delete s;
    return EXAGO_OK;
}

exago_status exago_slack_pattern(exago_slack_t s, int64_t *rows, double *vals) {
    if (!s) return set_last_error(EXAGO_EINVAL, "slack set is NULL");
    if (s->nz > 0 && (!rows || !vals)) return set_last_error(EXAGO_EINVAL, "rows or vals is NULL");
    for (int k = 0; k < s->nz; k++) {
        rows[k] = s->grow[k];
        vals[k] = s->sign[k];
    }
    return EXAGO_OK;
}

exago_status exago_eval_slack(exago_slack_t s, const exago_batch *bt, const double *z, double *gh,
                              int64_t ldgh, double *f, double *grad_z) {
    exago_status st = check_call(s, bt);
    if (st != EXAGO_OK || bt->B == 0 || s->nz == 0) return st;
    if (!z) return set_last_error(EXAGO_EINVAL, "z is NULL");
    if (gh && ldgh < 2 * s->nb) return set_last_error(EXAGO_EINVAL, "ldgh < 2 nb");
    cudaStream_t stream = (cudaStream_t)bt->stream;
    const int nused = (int)s->used.size();
    const int *grow = s->d_int, *sign = grow + s->nz, *rptr = sign + s->nz;
    const int *rlist = rptr + 2 * s->nb + 1, *used = rlist + s->nz;
    for (int b0 = 0; b0 < bt->B; b0 += kMaxGridY) {
        const int nB = std::min(kMaxGridY, bt->B - b0);
        if (gh && nused > 0)
            k_slack_rows<<<dim3((nused + 127) / 128, (nB + kGroup - 1) / kGroup), 128, 0, stream>>>(
                used, nused, rptr, rlist, sign, s->nz, b0, nB, z, gh, ldgh);
        if (f) k_slack_obj<<<nB, kLanes, 0, stream>>>(s->d_cost, s->nz, b0, z, bt->obj_weight, f);
        if (grad_z)
            k_slack_grad<<<dim3((s->nz + 1023) / 1024, nB), 256, 0, stream>>>(
                s->d_cost, s->nz, b0, bt->obj_weight, grad_z);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_last_error(EXAGO_ECUDA, std::string("slack launch: ") + cudaGetErrorString(e));
    return EXAGO_OK;
}

exago_status exago_eval_all_slack(exago_net_t net, const exago_batch *bt, exago_slack_t s,
                                  const double *z, double *f, double *grad, double *gh,
                                  double *jval, double *hval, double *grad_z) {
    exago_status st = check_call(s, bt);
    if (st != EXAGO_OK || bt->B == 0) return st;
    int n = 0, meq = 0, mineq = 0;
    if ((st = exago_net_dims(net, &n, &meq, &mineq, nullptr, nullptr)) != EXAGO_OK) return st;
    if (meq / 2 != s->nb) return set_last_error(EXAGO_EINVAL, "slack set of another grid");
    // the evaluation, then the slack kernels on the same stream (bit for bit the two calls)
    if ((st = exago_eval_all(net, bt, f, grad, gh, jval, hval)) != EXAGO_OK) return st;
    return exago_eval_slack(s, bt, z, gh, meq + mineq, f, grad_z);
}

exago_status exago_eval_slack_jtv(exago_slack_t s, const exago_batch *bt, const double *v,
                                  int64_t ldv, double *out) {
    exago_status st = check_call(s, bt);
    if (st != EXAGO_OK || bt->B == 0 || s->nz == 0) return st;
    if (!v || !out) return set_last_error(EXAGO_EINVAL, "v or out is NULL");
    if (ldv < 2 * s->nb) return set_last_error(EXAGO_EINVAL, "ldv < 2 nb");
    const int *grow = s->d_int, *sign = grow + s->nz;
    for (int b0 = 0; b0 < bt->B; b0 += kMaxGridY) {
        const int nB = std::min(kMaxGridY, bt->B - b0);
        k_slack_jtv<<<dim3((s->nz + 255) / 256, nB), 256, 0, (cudaStream_t)bt->stream>>>(
            grow, sign, s->nz, b0, v, ldv, out);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_last_error(EXAGO_ECUDA, std::string("slack transpose launch: ") +
                                               cudaGetErrorString(e));
    return EXAGO_OK;
}

}  // extern "C"
