// Batched interior-point KKT step on the device (exago_kkt_*): for every state b of a batch,
//     K_b [dx; dlam] = r_b,   K_b = [[W_b + diag(dx_b), J_b'], [J_b, -diag(dc_b)]],
// the augmented primal-dual system the paper's interior-point solvers (Ipopt, HiOp; Sec. II-III)
// factor once per iteration, for each contingency or scenario subproblem under EMPAR (Sec. V-A,
// eqs. (16)-(20); Sec. VI-A).  W and J are the values exago_eval_all writes (Lagrangian Hessian,
// lower triangle, and the Jacobian of [g; h], in the exported CSR patterns).
//
// Elimination plan (fixed per grid; exact algebra, no approximation):
//   1. each flow row h (pivot -dc < 0) couples only the four voltage variables of its branch, whose
//      Hessian block is already dense, so eliminating it adds j j' / dc to that block and creates
//      no fill;
//   2. each generator's Pg (pivot W_kk + dx_k) and Qg (pivot dx) couples only its bus's P or Q
//      row: eliminating it subtracts a^2 / pivot from that row's diagonal;
//   3. what remains is one 4 x 4 block per bus, unknowns (Va, Vm, lamP, lamQ), on the bus graph:
//      factored by the batched block L D L' (blockfact.cu) on a minimum-degree order;
//   4. the eliminated unknowns are recovered from the reduced solution.
// Per state the factor's negative pivots (1. to 3.) are counted: the inertia an interior-point
// method checks (m negative pivots for a correct step).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "blockfact.h"
#include "internal.h"

namespace exago {
namespace {

constexpr int KNT = 128;
constexpr double kTiny = 1e-13;   // relative size of a pivot treated as zero

// Where an entry of the reduced 4 x 4 block matrix comes from: src = 2 q (Hessian value q) or
// 2 q + 1 (Jacobian value q), or -1; diag = 2 i (+ dx_i) or 2 r + 1 (- dc_r), or -1.
struct KktDev {
    int nb, nl, ng, n, m;
    int64_t nnzJ, nnzH, nnzJg, hpg;
    const int *asm_src, *asm_diag;     // [nblk * 16]
    const int *bus_of_col;             // [nb] perm: bus of elimination index k
    const int *col_of_bus;             // [nb] iperm
    const int64_t *blk_br_ptr;         // [nblk + 1] branches whose flow rows touch the block
    const int *blk_br;                 // branch l << 2 | (row bus is the lower end) << 1 |
                                       //   (column bus is the lower end)
    const int *bus_br_ptr, *bus_br;    // [nb + 1] incident branches, l << 1 | (bus is lower end)
    const int *gen_ptr, *gen_ord;      // generators of each bus
    const int *gen_jP, *gen_jQ;        // [ng] Jacobian positions of (P_bus, Pg_k), (Q_bus, Qg_k)
    const int *br_f, *br_t;
};

// Flow row r of branch l: from row (side 0) or to row (side 1); its four Jacobian values in the
// order (Va_lo, Va_hi, Vm_lo, Vm_hi), lo = min(f, t).
__device__ __forceinline__ const double *hrow(const KktDev &K, const double *jv, int l, int side) {
    return jv + K.nnzJg + 4 * ((size_t)side * K.nl + l);
}

// Assembly of the reduced matrix: one thread per (state, block).
__global__ void __launch_bounds__(KNT) k_kkt_assemble(const KktDev K, const DevSymK S, int B,
                                                      const double *__restrict__ jval,
                                                      const double *__restrict__ hval,
                                                      const double *__restrict__ dx,
                                                      const double *__restrict__ dc, double *T) {
    const int b = blockIdx.y * KNT + threadIdx.x;
    if (b >= B) return;
    const int p = blockIdx.x;
    const double *jv = jval + (size_t)b * K.nnzJ, *hv = hval + (size_t)b * K.nnzH;
    const double *dxb = dx + (size_t)b * K.n, *dcb = dc + (size_t)b * K.m;
    double v[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const int s = __ldg(K.asm_src + (size_t)p * 16 + e), d = __ldg(K.asm_diag + (size_t)p * 16 + e);
        double a = s < 0 ? 0.0 : (s & 1) ? __ldg(jv + (s >> 1)) : __ldg(hv + (s >> 1));
        if (d >= 0) a += (d & 1) ? -__ldg(dcb + (d >> 1)) : __ldg(dxb + (d >> 1));
        v[e] = a;
    }
    // flow rows eliminated: + j j' / dc on the (Va, Vm) x (Va, Vm) part, in branch order, the
    // from row before the to row
    for (int64_t q = __ldg(K.blk_br_ptr + p); q < __ldg(K.blk_br_ptr + p + 1); q++) {
        const int code = __ldg(K.blk_br + q);
        const int l = code >> 2, ulo = (code >> 1) & 1, vlo = code & 1;
        const int ua = ulo ? 0 : 1, um = ulo ? 2 : 3, va = vlo ? 0 : 1, vm = vlo ? 2 : 3;
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const double *j = hrow(K, jv, l, side);
            const double rdc = 1.0 / __ldg(dcb + 2 * K.nb + side * K.nl + l);
            const double ja = __ldg(j + ua) * rdc, jm = __ldg(j + um) * rdc;
            const double ka = __ldg(j + va), km = __ldg(j + vm);
            v[0] = fma(ja, ka, v[0]);   // (Va_u, Va_v)
            v[1] = fma(ja, km, v[1]);   // (Va_u, Vm_v)
            v[4] = fma(jm, ka, v[4]);   // (Vm_u, Va_v)
            v[5] = fma(jm, km, v[5]);   // (Vm_u, Vm_v)
        }
    }
    // generators eliminated (diagonal blocks): - a^2 / pivot on the bus's lamP and lamQ diagonal
    const int col = __ldg(S.rowidx + p);
    if (__ldg(S.colptr + col) == p) {
        const int u = __ldg(K.bus_of_col + col);
        for (int g = __ldg(K.gen_ptr + u); g < __ldg(K.gen_ptr + u + 1); g++) {
            const int k = __ldg(K.gen_ord + g);
            const double aP = __ldg(jv + __ldg(K.gen_jP + k)), aQ = __ldg(jv + __ldg(K.gen_jQ + k));
            const double pP = __ldg(hv + K.hpg + k) + __ldg(dxb + 2 * K.nb + k);
            const double pQ = __ldg(dxb + 2 * K.nb + K.ng + k);
            v[10] = fma(-aP, aP / pP, v[10]);
            v[15] = fma(-aQ, aQ / pQ, v[15]);
        }
    }
#pragma unroll
    for (int e = 0; e < 16; e++) T[((size_t)p * 16 + e) * B + b] = v[e];
}

// Reduced right-hand side, one thread per (state, bus), into x [col][4][B]; also counts the
// generators' negative pivots.
__global__ void __launch_bounds__(KNT) k_kkt_rhs(const KktDev K, int B, const double *__restrict__ jval,
                                                 const double *__restrict__ hval,
                                                 const double *__restrict__ dx,
                                                 const double *__restrict__ dc,
                                                 const double *__restrict__ rhs, double *x, int *neg) {
    const int b = blockIdx.y * KNT + threadIdx.x;
    if (b >= B) return;
    const int u = blockIdx.x;
    const double *jv = jval + (size_t)b * K.nnzJ, *hv = hval + (size_t)b * K.nnzH;
    const double *dxb = dx + (size_t)b * K.n, *dcb = dc + (size_t)b * K.m;
    const double *rb = rhs + (size_t)b * (K.n + K.m);
    double ra = __ldg(rb + u), rm = __ldg(rb + K.nb + u);
    double rP = __ldg(rb + K.n + u), rQ = __ldg(rb + K.n + K.nb + u);
    for (int q = __ldg(K.bus_br_ptr + u); q < __ldg(K.bus_br_ptr + u + 1); q++) {
        const int code = __ldg(K.bus_br + q);
        const int l = code >> 1, lo = code & 1;
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const double *j = hrow(K, jv, l, side);
            const int row = 2 * K.nb + side * K.nl + l;
            const double w = __ldg(rb + K.n + row) / __ldg(dcb + row);
            ra = fma(__ldg(j + (lo ? 0 : 1)), w, ra);
            rm = fma(__ldg(j + (lo ? 2 : 3)), w, rm);
        }
    }
    int nn = 0;
    for (int g = __ldg(K.gen_ptr + u); g < __ldg(K.gen_ptr + u + 1); g++) {
        const int k = __ldg(K.gen_ord + g);
        const double aP = __ldg(jv + __ldg(K.gen_jP + k)), aQ = __ldg(jv + __ldg(K.gen_jQ + k));
        const double pP = __ldg(hv + K.hpg + k) + __ldg(dxb + 2 * K.nb + k);
        const double pQ = __ldg(dxb + 2 * K.nb + K.ng + k);
        rP = fma(-aP, __ldg(rb + 2 * K.nb + k) / pP, rP);
        rQ = fma(-aQ, __ldg(rb + 2 * K.nb + K.ng + k) / pQ, rQ);
        nn += (pP < 0.0) + (pQ < 0.0);
    }
    if (nn) atomicAdd(neg + b, nn);
    const int c = __ldg(K.col_of_bus + u);
    double *xc = x + (size_t)c * 4 * B + b;
    xc[0] = ra;
    xc[(size_t)B] = rm;
    xc[2 * (size_t)B] = rP;
    xc[3 * (size_t)B] = rQ;
}

// Recovery, one thread per (state, bus): Va, Vm, lamP, lamQ of the bus and Pg, Qg of its
// generators into sol [B][n + m].
__global__ void __launch_bounds__(KNT) k_kkt_recover_bus(const KktDev K, int B,
                                                         const double *__restrict__ jval,
                                                         const double *__restrict__ hval,
                                                         const double *__restrict__ dx,
                                                         const double *__restrict__ rhs,
                                                         const double *__restrict__ x,
                                                         double *sol) {
    const int b = blockIdx.y * KNT + threadIdx.x;
    if (b >= B) return;
    const int u = blockIdx.x;
    const int c = __ldg(K.col_of_bus + u);
    const double *xc = x + (size_t)c * 4 * B + b;
    const double va = __ldcg(xc), vm = __ldcg(xc + (size_t)B);
    const double lP = __ldcg(xc + 2 * (size_t)B), lQ = __ldcg(xc + 3 * (size_t)B);
    double *s = sol + (size_t)b * (K.n + K.m);
    s[u] = va;
    s[K.nb + u] = vm;
    s[K.n + u] = lP;
    s[K.n + K.nb + u] = lQ;
    const double *jv = jval + (size_t)b * K.nnzJ, *hv = hval + (size_t)b * K.nnzH;
    const double *dxb = dx + (size_t)b * K.n, *rb = rhs + (size_t)b * (K.n + K.m);
    for (int g = __ldg(K.gen_ptr + u); g < __ldg(K.gen_ptr + u + 1); g++) {
        const int k = __ldg(K.gen_ord + g);
        const double aP = __ldg(jv + __ldg(K.gen_jP + k)), aQ = __ldg(jv + __ldg(K.gen_jQ + k));
        const double pP = __ldg(hv + K.hpg + k) + __ldg(dxb + 2 * K.nb + k);
        const double pQ = __ldg(dxb + 2 * K.nb + K.ng + k);
        s[2 * K.nb + k] = fma(-aP, lP, __ldg(rb + 2 * K.nb + k)) / pP;
        s[2 * K.nb + K.ng + k] = fma(-aQ, lQ, __ldg(rb + 2 * K.nb + K.ng + k)) / pQ;
    }
}

// Recovery of the flow rows' multipliers, one thread per (state, branch):
// dlam_r = (j_r . dx_branch - r_r) / dc_r; also counts their pivots -dc_r < 0.
__global__ void __launch_bounds__(KNT) k_kkt_recover_branch(const KktDev K, int B,
                                                            const double *__restrict__ jval,
                                                            const double *__restrict__ dc,
                                                            const double *__restrict__ rhs,
                                                            const double *__restrict__ x,
                                                            double *sol, int *neg) {
    const int b = blockIdx.y * KNT + threadIdx.x;
    if (b >= B) return;
    const int l = blockIdx.x;
    const int f = __ldg(K.br_f + l), t = __ldg(K.br_t + l);
    const int lo = f < t ? f : t, hi = f < t ? t : f;
    const double *xl = x + (size_t)__ldg(K.col_of_bus + lo) * 4 * B + b;
    const double *xh = x + (size_t)__ldg(K.col_of_bus + hi) * 4 * B + b;
    const double d0 = __ldcg(xl), d1 = __ldcg(xh);
    const double d2 = __ldcg(xl + (size_t)B), d3 = __ldcg(xh + (size_t)B);
    const double *jv = jval + (size_t)b * K.nnzJ, *dcb = dc + (size_t)b * K.m;
    const double *rb = rhs + (size_t)b * (K.n + K.m);
    double *s = sol + (size_t)b * (K.n + K.m);
    int nn = 0;
#pragma unroll
    for (int side = 0; side < 2; side++) {
        const double *j = hrow(K, jv, l, side);
        const int row = 2 * K.nb + side * K.nl + l;
        double a = __ldg(j) * d0;
        a = fma(__ldg(j + 1), d1, a);
        a = fma(__ldg(j + 2), d2, a);
        a = fma(__ldg(j + 3), d3, a);
        const double d = __ldg(dcb + row);
        s[K.n + row] = (a - __ldg(rb + K.n + row)) / d;
        nn += d > 0.0;
    }
    if (nn) atomicAdd(neg + b, nn);
}

__global__ void k_kkt_counts(const int *neg, const int *bad, int *out, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) { out[2 * b] = neg[b]; out[2 * b + 1] = bad[b]; }
}

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace exago

using namespace exago;

struct exago_kkt {
    exago_net_t net = nullptr;
    int device = -1;
    bool on_device = false;
    BlockSym S;
    DevSym D;
    KktDev K{};
    std::vector<void *> allocs;
    std::mutex mu;            // the internal workspace
    void *ws = nullptr;
    size_t ws_bytes = 0;
};

namespace {

size_t kkt_ws_bytes(const exago_kkt *k, int B) {
    const size_t blk = (size_t)k->S.nblk * 16 * (size_t)B * sizeof(double);
    return 2 * round256(blk) + round256((size_t)k->S.nb * 4 * B * sizeof(double)) +
           round256(2 * (size_t)B * sizeof(int));
}

template <typename T>
exago_status upload_vec(exago_kkt *k, const std::vector<T> &v, const T **out) {
    *out = nullptr;
    if (v.empty()) return EXAGO_OK;
    void *p = nullptr;
    cudaError_t e = dev_malloc(&p, v.size() * sizeof(T));
    if (e != cudaSuccess)
        return set_last_error(e == cudaErrorMemoryAllocation ? EXAGO_ENOMEM : EXAGO_ECUDA,
                              std::string("KKT tables: ") + cudaGetErrorString(e));
    k->allocs.push_back(p);
    e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
    *out = (const T *)p;
    return EXAGO_OK;
}

// Position of (row, col) in a CSR pattern with ascending columns, or -1.
int64_t csr_find(const std::vector<int64_t> &rp, const std::vector<int> &ci, int row, int col) {
    auto b = ci.begin() + rp[row], e = ci.begin() + rp[row + 1];
    auto it = std::lower_bound(b, e, col);
    return it != e && *it == col ? (int64_t)(it - ci.begin()) : -1;
}

void free_kkt(exago_kkt *k) {
    if (!k) return;
    if (k->ws || !k->allocs.empty()) cudaDeviceSynchronize();
    for (void *p : k->allocs) cudaFree(p);
    k->allocs.clear();
    if (k->ws) cudaFree(k->ws);
    k->ws = nullptr;
}

}  // namespace

extern "C" {

exago_status exago_kkt_create(exago_net_t net, exago_kkt_t *out) {
    const HostPlan *P = nullptr;
    const DevNet *dev = nullptr;
    int device = -1;
    if (!out) return set_last_error(EXAGO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!net_plan_view(net, &P)) return set_last_error(EXAGO_EINVAL, "net is NULL");
    const bool on_device = net_internal_view(net, &P, &dev, &device);
    exago_kkt *k = new (std::nothrow) exago_kkt();
    if (!k) return set_last_error(EXAGO_ENOMEM, "host allocation failed");
    k->net = net;
    k->device = device;
    k->on_device = on_device;
    const int nb = P->nb, nl = P->nl, ng = P->ng, n = P->n, m = P->m;
    std::string err;
    try {
        // bus graph from the branches
        std::vector<int> aptr(nb + 1, 0), adj;
        for (int l = 0; l < nl; l++) { aptr[P->f[l] + 1]++; }
        for (int i = 0; i < nb; i++) aptr[i + 1] += aptr[i];
        adj.resize(aptr[nb]);
        {
            std::vector<int> fill(aptr.begin(), aptr.end() - 1);
            for (int l = 0; l < nl; l++) adj[fill[P->f[l]]++] = P->t[l];
        }
        if (!build_block_sym(nb, aptr.data(), adj.data(), k->S, err)) {
            delete k;
            return set_last_error(EXAGO_EINVAL, "KKT symbolic factorisation: " + err);
        }
        const BlockSym &S = k->S;
        // variable / row index of entry a (0..3) of bus u: Va, Vm (x) or lamP, lamQ (rows)
        auto var = [&](int u, int a) { return a == 0 ? u : a == 1 ? nb + u : a == 2 ? u : nb + u; };
        std::vector<int> asrc((size_t)S.nblk * 16, -1), adiag((size_t)S.nblk * 16, -1);
        std::vector<int64_t> bbp(S.nblk + 1, 0);
        std::vector<int> bb;
        // branches between each bus pair (sorted by the pair's lower bus) and incident to each bus
        std::vector<std::vector<int>> inc(nb);
        for (int l = 0; l < nl; l++) { inc[P->f[l]].push_back(l); inc[P->t[l]].push_back(l); }
        for (int J = 0; J < nb; J++) {
            const int v = S.perm[J];
            for (int64_t p = S.colptr[J]; p < S.colptr[J + 1]; p++) {
                const int u = S.perm[S.rowidx[p]];
                for (int a = 0; a < 4; a++)
                    for (int c = 0; c < 4; c++) {
                        const size_t e = (size_t)p * 16 + a * 4 + c;
                        const bool ax = a < 2, cx = c < 2;
                        int64_t q = -1;
                        if (ax && cx) {
                            const int i = var(u, a), j = var(v, c);
                            q = csr_find(P->Hrowptr, P->Hcol, std::max(i, j), std::min(i, j));
                            if (q >= 0) asrc[e] = (int)(2 * q);
                            if (i == j) adiag[e] = 2 * i;
                        } else if (!ax && cx) {
                            q = csr_find(P->Jrowptr, P->Jcol, var(u, a), var(v, c));
                            if (q >= 0) asrc[e] = (int)(2 * q + 1);
                        } else if (ax && !cx) {
                            q = csr_find(P->Jrowptr, P->Jcol, var(v, c), var(u, a));
                            if (q >= 0) asrc[e] = (int)(2 * q + 1);
                        } else if (u == v && a == c) {
                            adiag[e] = 2 * var(u, a) + 1;
                        }
                    }
                // branches whose flow rows touch block (u, v)
                for (int l : inc[u]) {
                    const int f = P->f[l], t = P->t[l];
                    if (!(u == v || (f == u && t == v) || (f == v && t == u))) continue;
                    const int lo = std::min(f, t);
                    bb.push_back((l << 2) | ((u == lo) << 1) | (v == lo));
                }
                bbp[p + 1] = (int64_t)bb.size();
            }
        }
        if ((int64_t)P->nnzJ > (1ll << 30) || (int64_t)P->nnzH > (1ll << 30) || nl >= (1 << 29)) {
            delete k;
            return set_last_error(EXAGO_EINVAL, "grid too large for the KKT tables");
        }
        std::vector<int> busbr_ptr(nb + 1, 0), busbr;
        for (int u = 0; u < nb; u++) {
            for (int l : inc[u]) busbr.push_back((l << 1) | (u == std::min(P->f[l], P->t[l])));
            busbr_ptr[u + 1] = (int)busbr.size();
        }
        std::vector<int> gjP(ng), gjQ(ng);
        for (int g = 0; g < ng; g++) {
            const int u = P->gbus[g];
            gjP[g] = (int)csr_find(P->Jrowptr, P->Jcol, u, 2 * nb + g);
            gjQ[g] = (int)csr_find(P->Jrowptr, P->Jcol, nb + u, 2 * nb + ng + g);
            if (gjP[g] < 0 || gjQ[g] < 0) {
                delete k;
                return set_last_error(EXAGO_EINVAL, "generator Jacobian entry missing");
            }
        }
        if (!on_device) {   // a plan-only net: the symbolic analysis alone
            *out = k;
            return EXAGO_OK;
        }
        exago_status s = EXAGO_OK;
        if (upload_block_sym(k->S, k->D, k->allocs) != 0) s = set_last_error(EXAGO_ENOMEM, "KKT symbolic tables");
        k->D.k.status = dev->status;   // the net's status word (debug-build index checks)
        KktDev &K = k->K;
        K.nb = nb; K.nl = nl; K.ng = ng; K.n = n; K.m = m;
        K.nnzJ = P->nnzJ; K.nnzH = P->nnzH; K.nnzJg = P->nnzJg; K.hpg = P->Hrowptr[2 * nb];
        if (s == EXAGO_OK) s = upload_vec(k, asrc, &K.asm_src);
        if (s == EXAGO_OK) s = upload_vec(k, adiag, &K.asm_diag);
        if (s == EXAGO_OK) s = upload_vec(k, S.perm, &K.bus_of_col);
        if (s == EXAGO_OK) s = upload_vec(k, S.iperm, &K.col_of_bus);
        if (s == EXAGO_OK) s = upload_vec(k, bbp, &K.blk_br_ptr);
        if (s == EXAGO_OK) s = upload_vec(k, bb, &K.blk_br);
        if (s == EXAGO_OK) s = upload_vec(k, busbr_ptr, &K.bus_br_ptr);
        if (s == EXAGO_OK) s = upload_vec(k, busbr, &K.bus_br);
        if (s == EXAGO_OK) s = upload_vec(k, P->gen_ptr, &K.gen_ptr);
        if (s == EXAGO_OK) s = upload_vec(k, P->gen_ord, &K.gen_ord);
        if (s == EXAGO_OK) s = upload_vec(k, gjP, &K.gen_jP);
        if (s == EXAGO_OK) s = upload_vec(k, gjQ, &K.gen_jQ);
        if (s == EXAGO_OK) s = upload_vec(k, P->f, &K.br_f);
        if (s == EXAGO_OK) s = upload_vec(k, P->t, &K.br_t);
        if (s != EXAGO_OK) {
            free_kkt(k);
            delete k;
            return s;
        }
    } catch (const std::bad_alloc &) {
        free_kkt(k);
        delete k;
        return set_last_error(EXAGO_ENOMEM, "host allocation failed (KKT analysis)");
    }
    *out = k;
    return EXAGO_OK;
}

exago_status exago_kkt_destroy(exago_kkt_t kkt) {
    if (!kkt) return EXAGO_OK;
    free_kkt(kkt);
    delete kkt;
    return EXAGO_OK;
}

exago_status exago_kkt_info(exago_kkt_t kkt, int64_t *blocks, int64_t *pairs, int *levels,
                            double *flops) {
    if (!kkt) return set_last_error(EXAGO_EINVAL, "kkt is NULL");
    const BlockSym &S = kkt->S;
    if (blocks) *blocks = S.nblk;
    if (pairs) *pairs = (int64_t)S.pairs.size();
    if (levels) *levels = S.nlevels;
    if (flops) {
        // FP64 flops of one state: block products (64 FMA each), pivot inverses and scalings
        // (4 x 4: about 100 + 64 FMA per block), both sweeps (16 FMA per block each way)
        *flops = 2.0 * (64.0 * (double)S.pairs.size() + 164.0 * (double)S.nblk + 32.0 * (double)S.nblk);
    }
    return EXAGO_OK;
}

exago_status exago_kkt_order(exago_kkt_t kkt, int *perm, int *parent, int *level) {
    if (!kkt) return set_last_error(EXAGO_EINVAL, "kkt is NULL");
    const BlockSym &S = kkt->S;
    if (perm) std::copy(S.perm.begin(), S.perm.end(), perm);
    if (parent) std::copy(S.parent.begin(), S.parent.end(), parent);
    if (level) std::copy(S.level.begin(), S.level.end(), level);
    return EXAGO_OK;
}

exago_status exago_kkt_workspace_size(exago_kkt_t kkt, int B, size_t *bytes) {
    if (!kkt || !bytes) return set_last_error(EXAGO_EINVAL, "null argument");
    if (B < 0) return set_last_error(EXAGO_EINVAL, "B < 0");
    *bytes = B == 0 ? 0 : kkt_ws_bytes(kkt, B);
    return EXAGO_OK;
}

exago_status exago_kkt_solve(exago_kkt_t kkt, int B, const double *jval, const double *hval,
                             const double *dx, const double *dc, const double *rhs, double *sol,
                             int *inertia, void *workspace, size_t workspace_bytes, void *stream) {
    if (!kkt) return set_last_error(EXAGO_EINVAL, "kkt is NULL");
    if (!kkt->on_device) return set_last_error(EXAGO_ESTATE, "KKT analysis of a net without a device");
    if (B < 0) return set_last_error(EXAGO_EINVAL, "B < 0");
    if (B == 0) return EXAGO_OK;
    if (B > 65535 * KNT) return set_last_error(EXAGO_EINVAL, "B too large for one call");
    if (!jval || !hval || !dx || !dc || !rhs || !sol)
        return set_last_error(EXAGO_EINVAL, "null input or output");
    const size_t need = kkt_ws_bytes(kkt, B);
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_lock<std::mutex> lk(kkt->mu, std::defer_lock);
    char *w = (char *)workspace;
    if (w) {
        if (((uintptr_t)w & 255) != 0) return set_last_error(EXAGO_EINVAL, "workspace not 256-byte aligned");
        if (workspace_bytes < need) return set_last_error(EXAGO_EINVAL, "workspace smaller than exago_kkt_workspace_size");
    } else {
        lk.lock();
        if (kkt->ws_bytes < need) {
            if (kkt->ws) {
                cudaError_t e = cudaDeviceSynchronize();
                if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
                cudaFree(kkt->ws);
                kkt->ws = nullptr;
                kkt->ws_bytes = 0;
            }
            cudaError_t e = dev_malloc(&kkt->ws, need);
            if (e != cudaSuccess) {
                kkt->ws = nullptr;
                return set_last_error(e == cudaErrorMemoryAllocation ? EXAGO_ENOMEM : EXAGO_ECUDA,
                                      "KKT workspace");
            }
            kkt->ws_bytes = need;
        }
        w = (char *)kkt->ws;
    }
    const size_t blk = round256((size_t)kkt->S.nblk * 16 * (size_t)B * sizeof(double));
    double *T = (double *)w;
    double *L = (double *)(w + blk);
    double *x = (double *)(w + 2 * blk);
    int *neg = (int *)(w + 2 * blk + round256((size_t)kkt->S.nb * 4 * B * sizeof(double)));
    int *bad = neg + B;
    const KktDev &K = kkt->K;
    const unsigned gy = (unsigned)((B + KNT - 1) / KNT);
    cudaError_t e = cudaMemsetAsync(neg, 0, 2 * (size_t)B * sizeof(int), st);
    if (e != cudaSuccess) return set_last_error(EXAGO_ECUDA, cudaGetErrorString(e));
    k_kkt_assemble<<<dim3((unsigned)kkt->S.nblk, gy), KNT, 0, st>>>(K, kkt->D.k, B, jval, hval, dx,
                                                                    dc, T);
    k_kkt_rhs<<<dim3((unsigned)K.nb, gy), KNT, 0, st>>>(K, B, jval, hval, dx, dc, rhs, x, neg);
    int le = launch_block_factor<4, true>(kkt->D, B, T, nullptr, L, nullptr, neg, bad, kTiny, st);
    if (le == 0) le = launch_block_solve<4, true>(kkt->D, B, T, L, nullptr, x, st);
    if (le == 0) {
        k_kkt_recover_bus<<<dim3((unsigned)K.nb, gy), KNT, 0, st>>>(K, B, jval, hval, dx, rhs, x, sol);
        if (K.nl > 0)
            k_kkt_recover_branch<<<dim3((unsigned)K.nl, gy), KNT, 0, st>>>(K, B, jval, dc, rhs, x, sol, neg);
        if (inertia) k_kkt_counts<<<(B + 255) / 256, 256, 0, st>>>(neg, bad, inertia, B);
        le = (int)cudaGetLastError();
    }
    if (le != 0) return set_last_error(EXAGO_ECUDA, std::string("KKT kernels: ") +
                                                        cudaGetErrorString((cudaError_t)le));
    return EXAGO_OK;
}

}  // extern "C"
