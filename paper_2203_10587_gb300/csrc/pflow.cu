// Batched power-flow Newton step on the device (exago_pf_*), the power-flow application (PFLOW)
// of the paper: for every state b, J_pf(x_b) d = -g_pf(x_b) and x_b + d, where g_pf are the P
// balances of the non-slack buses and the Q balances of the PQ buses (Sec. III, eq. (8)), and
// the unknowns Va of the non-slack and Vm of the PQ buses.  g and J are the evaluation's own
// (exago_eval_all on the batch, into this step's workspace).
//
// The system is kept at 2 x 2 blocks per bus (rows P_u, Q_u; columns Va_v, Vm_v) on the bus
// graph: a fixed unknown (Va and Vm of the slack bus, Vm of a PV bus) gets an identity row in
// place of its bus's inactive balance (P <-> Va, Q <-> Vm) and a zero column, so its step is
// exactly 0 and the other unknowns solve the reduced system.  The block matrix is not symmetric:
// it is factored A = L D U without pivoting (blockfact.cu) on the same minimum-degree order of
// the bus graph as the KKT step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "blockfact.h"
#include "internal.h"

namespace exago {
namespace {

constexpr int PNT = 128;
constexpr double kPfTiny = 1e-13;

// Entry sources: q >= 0 the Jacobian value q, -1 zero, -2 one (an identity row of a fixed
// unknown).
struct PfDev {
    int nb, n, m;
    int64_t nnzJ;
    const int *src_lo, *src_up;   // [nblk * 4]: block (I, J) and its transposed position (J, I)
    const int *col_of_bus;        // [nb]
    const int *active;            // [nb] bit 0: P row active (non-slack), bit 1: Q row (PQ)
};

__device__ __forceinline__ double pf_src(int s, const double *jv) {
    return s >= 0 ? __ldg(jv + s) : s == -2 ? 1.0 : 0.0;
}

__global__ void __launch_bounds__(PNT) k_pf_assemble(const PfDev P, int B, int64_t nblk,
                                                     const double *__restrict__ jval, double *T,
                                                     double *TU) {
    const int b = blockIdx.y * PNT + threadIdx.x;
    if (b >= B) return;
    const int64_t p = blockIdx.x;
    const double *jv = jval + (size_t)b * P.nnzJ;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        T[((size_t)p * 4 + e) * B + b] = pf_src(__ldg(P.src_lo + p * 4 + e), jv);
        TU[((size_t)p * 4 + e) * B + b] = pf_src(__ldg(P.src_up + p * 4 + e), jv);
    }
}

// Right-hand side -g_pf (0 on the identity rows) into x [col][2][B], and the largest |g_pf| of
// each state (atomicMax on the bits of a nonnegative double, whose order is the numeric order).
__global__ void __launch_bounds__(PNT) k_pf_rhs(const PfDev P, int B, const double *__restrict__ gh,
                                                double *x, unsigned long long *mis) {
    const int b = blockIdx.y * PNT + threadIdx.x;
    if (b >= B) return;
    const int u = blockIdx.x;
    const int act = __ldg(P.active + u);
    const double *g = gh + (size_t)b * P.m;
    const double gP = (act & 1) ? __ldg(g + u) : 0.0, gQ = (act & 2) ? __ldg(g + P.nb + u) : 0.0;
    const int c = __ldg(P.col_of_bus + u);
    x[((size_t)c * 2) * B + b] = -gP;
    x[((size_t)c * 2 + 1) * B + b] = -gQ;
    const double a = fmax(fabs(gP), fabs(gQ));
    if (a > 0.0 || a != a) atomicMax(mis + b, (unsigned long long)__double_as_longlong(a));
}

__global__ void __launch_bounds__(PNT) k_pf_update(const PfDev P, int B, const double *__restrict__ x0,
                                                   const double *__restrict__ d, double *x1) {
    const int b = blockIdx.y * PNT + threadIdx.x;
    if (b >= B) return;
    const int j = blockIdx.x;   // variable index of x = [Va | Vm | Pg | Qg]
    const double *xb = x0 + (size_t)b * P.n;
    double v = __ldg(xb + j);
    if (j < 2 * P.nb) {
        const int u = j < P.nb ? j : j - P.nb, a = j < P.nb ? 0 : 1;
        v += __ldcg(d + ((size_t)__ldg(P.col_of_bus + u) * 2 + a) * B + b);
    }
    x1[(size_t)b * P.n + j] = v;
}

__global__ void k_pf_mismatch(const unsigned long long *mis, double *out, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) out[b] = __longlong_as_double((long long)mis[b]);
}

size_t r256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace exago

using namespace exago;

struct exago_pf {
    exago_net_t net = nullptr;
    BlockSym S;
    DevSym D;
    PfDev P{};
    std::vector<void *> allocs;
    std::mutex mu;
    void *ws = nullptr;
    size_t ws_bytes = 0;
};

namespace {

struct PfLayout {
    size_t gh, jv, blk, x, cnt, total;
};

PfLayout pf_layout(const exago_pf *pf, int B) {
    PfLayout L;
    L.gh = r256((size_t)B * pf->P.m * sizeof(double));
    L.jv = r256((size_t)B * pf->P.nnzJ * sizeof(double));
    L.blk = r256((size_t)pf->S.nblk * 4 * B * sizeof(double));
    L.x = r256((size_t)pf->S.nb * 2 * B * sizeof(double));
    L.cnt = r256((size_t)B * (2 * sizeof(int) + sizeof(unsigned long long)));
    L.total = L.gh + L.jv + 4 * L.blk + L.x + L.cnt;
    return L;
}

void free_pf(exago_pf *pf) {
    if (!pf) return;
    if (pf->ws || !pf->allocs.empty()) cudaDeviceSynchronize();
    for (void *p : pf->allocs) cudaFree(p);
    pf->allocs.clear();
    if (pf->ws) cudaFree(pf->ws);
    pf->ws = nullptr;
}

template <typename T>
exago_status pf_upload(exago_pf *pf, const std::vector<T> &v, const T **out) {
    *out = nullptr;
    if (v.empty()) return EXAGO_OK;
    void *p = nullptr;
    cudaError_t e = dev_malloc(&p, v.size() * sizeof(T));
    if (e != cudaSuccess)
        return set_last_error(e == cudaErrorMemoryAllocation ? EXAGO_ENOMEM : EXAGO_ECUDA,
                              std::string("power-flow tables: ") + cudaGetErrorString(e));
    pf->allocs.push_back(p);
    e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
    *out = (const T *)p;
    return EXAGO_OK;
}

int64_t find_pos(const std::vector<int64_t> &rp, const std::vector<int> &ci, int row, int col) {
    auto b = ci.begin() + rp[row], e = ci.begin() + rp[row + 1];
    auto it = std::lower_bound(b, e, col);
    return it != e && *it == col ? (int64_t)(it - ci.begin()) : -1;
}

}  // namespace

extern "C" {

exago_status exago_pf_create(exago_net_t net, const int *bus_type, exago_pf_t *out) {
    const HostPlan *P = nullptr;
    const DevNet *dev = nullptr;
    int device = -1;
    if (!out) return set_last_error(EXAGO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!net_internal_view(net, &P, &dev, &device))
        return set_last_error(net ? EXAGO_ESTATE : EXAGO_EINVAL,
                              net ? "net was planned without a device" : "net is NULL");
    if (!bus_type) return set_last_error(EXAGO_EINVAL, "bus_type is NULL");
    const int nb = P->nb, nl = P->nl;
    int nslack = 0;
    for (int i = 0; i < nb; i++) {
        if (bus_type[i] < 1 || bus_type[i] > 3)
            return set_last_error(EXAGO_EINVAL, "bus_type must be 1 (PQ), 2 (PV) or 3 (slack)");
        nslack += bus_type[i] == 3;
    }
    if (nslack < 1) return set_last_error(EXAGO_EINVAL, "no slack bus");
    exago_pf *pf = new (std::nothrow) exago_pf();
    if (!pf) return set_last_error(EXAGO_ENOMEM, "host allocation failed");
    pf->net = net;
    std::string err;
    try {
        std::vector<int> aptr(nb + 1, 0), adj;
        for (int l = 0; l < nl; l++) aptr[P->f[l] + 1]++;
        for (int i = 0; i < nb; i++) aptr[i + 1] += aptr[i];
        adj.resize(aptr[nb]);
        {
            std::vector<int> fill(aptr.begin(), aptr.end() - 1);
            for (int l = 0; l < nl; l++) adj[fill[P->f[l]]++] = P->t[l];
        }
        if (!build_block_sym(nb, aptr.data(), adj.data(), pf->S, err)) {
            delete pf;
            return set_last_error(EXAGO_EINVAL, "power-flow symbolic factorisation: " + err);
        }
        const BlockSym &S = pf->S;
        auto row_active = [&](int u, int a) { return a == 0 ? bus_type[u] != 3 : bus_type[u] == 1; };
        // source of entry (equation a of bus u, unknown c of bus v)
        auto src = [&](int u, int a, int v, int c) -> int {
            if (!row_active(u, a) || !row_active(v, c)) return u == v && a == c ? -2 : -1;
            const int64_t q = find_pos(P->Jrowptr, P->Jcol, a == 0 ? u : nb + u, c == 0 ? v : nb + v);
            return (int)q;   // -1 where the pattern has no entry
        };
        std::vector<int> lo((size_t)S.nblk * 4), up((size_t)S.nblk * 4);
        for (int J = 0; J < nb; J++) {
            const int v = S.perm[J];
            for (int64_t p = S.colptr[J]; p < S.colptr[J + 1]; p++) {
                const int u = S.perm[S.rowidx[p]];
                for (int a = 0; a < 2; a++)
                    for (int c = 0; c < 2; c++) {
                        lo[(size_t)p * 4 + a * 2 + c] = src(u, a, v, c);   // rows of I, columns of J
                        up[(size_t)p * 4 + a * 2 + c] = src(v, a, u, c);   // rows of J, columns of I
                    }
            }
        }
        std::vector<int> active(nb);
        for (int u = 0; u < nb; u++) active[u] = (row_active(u, 0) ? 1 : 0) | (row_active(u, 1) ? 2 : 0);
        exago_status s = EXAGO_OK;
        if (upload_block_sym(pf->S, pf->D, pf->allocs) != 0) s = set_last_error(EXAGO_ENOMEM, "power-flow symbolic tables");
        pf->D.k.status = dev->status;   // the net's status word (debug-build index checks)
        PfDev &D = pf->P;
        D.nb = nb; D.n = P->n; D.m = P->m; D.nnzJ = P->nnzJ;
        if (P->nnzJ >= (1ll << 31)) s = set_last_error(EXAGO_EINVAL, "grid too large");
        if (s == EXAGO_OK) s = pf_upload(pf, lo, &D.src_lo);
        if (s == EXAGO_OK) s = pf_upload(pf, up, &D.src_up);
        if (s == EXAGO_OK) s = pf_upload(pf, S.iperm, &D.col_of_bus);
        if (s == EXAGO_OK) s = pf_upload(pf, active, &D.active);
        if (s != EXAGO_OK) {
            free_pf(pf);
            delete pf;
            return s;
        }
    } catch (const std::bad_alloc &) {
        free_pf(pf);
        delete pf;
        return set_last_error(EXAGO_ENOMEM, "host allocation failed (power-flow analysis)");
    }
    *out = pf;
    return EXAGO_OK;
}

exago_status exago_pf_destroy(exago_pf_t pf) {
    if (!pf) return EXAGO_OK;
    free_pf(pf);
    delete pf;
    return EXAGO_OK;
}

exago_status exago_pf_workspace_size(exago_pf_t pf, int B, size_t *bytes) {
    if (!pf || !bytes) return set_last_error(EXAGO_EINVAL, "null argument");
    if (B < 0) return set_last_error(EXAGO_EINVAL, "B < 0");
    *bytes = B == 0 ? 0 : pf_layout(pf, B).total;
    return EXAGO_OK;
}

exago_status exago_pf_step(exago_pf_t pf, const exago_batch *batch, double *x_new,
                           double *mismatch) {
    if (!pf || !batch) return set_last_error(EXAGO_EINVAL, "null argument");
    const int B = batch->B;
    if (B < 0) return set_last_error(EXAGO_EINVAL, "batch B < 0");
    if (B == 0) return EXAGO_OK;
    if (B > 65535 * PNT) return set_last_error(EXAGO_EINVAL, "B too large for one call");
    if (!batch->x || !x_new) return set_last_error(EXAGO_EINVAL, "x or x_new is NULL");
    const PfLayout Lw = pf_layout(pf, B);
    cudaStream_t st = (cudaStream_t)batch->stream;
    std::unique_lock<std::mutex> lk(pf->mu, std::defer_lock);
    char *w = (char *)batch->workspace;
    if (w) {
        if (((uintptr_t)w & 255) != 0) return set_last_error(EXAGO_EINVAL, "workspace not 256-byte aligned");
        if (batch->workspace_bytes < Lw.total)
            return set_last_error(EXAGO_EINVAL, "workspace smaller than exago_pf_workspace_size");
    } else {
        lk.lock();
        if (pf->ws_bytes < Lw.total) {
            if (pf->ws) {
                cudaError_t e = cudaDeviceSynchronize();
                if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
                cudaFree(pf->ws);
                pf->ws = nullptr;
                pf->ws_bytes = 0;
            }
            cudaError_t e = dev_malloc(&pf->ws, Lw.total);
            if (e != cudaSuccess) {
                pf->ws = nullptr;
                return set_last_error(e == cudaErrorMemoryAllocation ? EXAGO_ENOMEM : EXAGO_ECUDA,
                                      "power-flow workspace");
            }
            pf->ws_bytes = Lw.total;
        }
        w = (char *)pf->ws;
    }
    double *gh = (double *)w;
    double *jv = (double *)(w + Lw.gh);
    char *fw = w + Lw.gh + Lw.jv;
    double *T = (double *)fw, *TU = (double *)(fw + Lw.blk);
    double *L = (double *)(fw + 2 * Lw.blk), *U = (double *)(fw + 3 * Lw.blk);
    double *x = (double *)(fw + 4 * Lw.blk);
    int *neg = (int *)(fw + 4 * Lw.blk + Lw.x);
    int *bad = neg + B;
    unsigned long long *mis = (unsigned long long *)(bad + B);
    // g and J at x (the evaluation of the batch's states; its own scratch is the net's)
    exago_batch eb = *batch;
    eb.workspace = nullptr;
    eb.workspace_bytes = 0;
    eb.lambda = nullptr;
    exago_status s = exago_eval_all(pf->net, &eb, nullptr, nullptr, gh, jv, nullptr);
    if (s != EXAGO_OK) return s;
    cudaError_t e = cudaMemsetAsync(neg, 0, Lw.cnt, st);
    if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
    const PfDev &D = pf->P;
    const unsigned gy = (unsigned)((B + PNT - 1) / PNT);
    k_pf_assemble<<<dim3((unsigned)pf->S.nblk, gy), PNT, 0, st>>>(D, B, pf->S.nblk, jv, T, TU);
    k_pf_rhs<<<dim3((unsigned)D.nb, gy), PNT, 0, st>>>(D, B, gh, x, mis);
    int le = launch_block_factor<2, false>(pf->D, B, T, TU, L, U, neg, bad, kPfTiny, st);
    if (le == 0) le = launch_block_solve<2, false>(pf->D, B, T, L, U, x, st);
    if (le == 0) {
        k_pf_update<<<dim3((unsigned)D.n, gy), PNT, 0, st>>>(D, B, batch->x, x, x_new);
        if (mismatch) k_pf_mismatch<<<(B + 255) / 256, 256, 0, st>>>(mis, mismatch, B);
        le = (int)cudaGetLastError();
    }
    if (le != 0)
        return set_last_error(EXAGO_ECUDA, std::string("power-flow kernels: ") +
                                               cudaGetErrorString((cudaError_t)le));
    return EXAGO_OK;
}

}  // extern "C"
