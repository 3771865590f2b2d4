// Internal structures of the evaluator: the host plan built once per grid and the device view
// the kernels read.  Not part of the public ABI (include/exago.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/exago.h"

namespace exago {

// Per-(branch, end) partial sums handed from the branch kernel to the bus kernel.  Component k of
// slot s of state b lives at scratch[(b * NCOMP + k) * nslot_pad + s].
enum SlotComp {
    SC_P = 0,    // active injection of this end at its own bus
    SC_Q = 1,    // reactive injection
    SC_PA = 2,   // dP/dVa_u   (u = this end's bus)
    SC_PU = 3,   // dP/dVm_u
    SC_QA = 4,   // dQ/dVa_u
    SC_QU = 5,   // dQ/dVm_u
    SC_HAA = 6,  // Lagrangian Hessian (Va_u, Va_u)
    SC_HUA = 7,  // (Vm_u, Va_u)
    SC_HUU = 8,  // (Vm_u, Vm_u)
    NCOMP = 9
};

// Off-diagonal outputs of one branch (written directly unless the branch has a parallel twin).
enum OffComp {
    OJ_PF_VAT = 0, OJ_PF_VMT, OJ_QF_VAT, OJ_QF_VMT,   // rows of the from bus, columns of the to bus
    OJ_PT_VAF, OJ_PT_VMF, OJ_QT_VAF, OJ_QT_VMF,       // rows of the to bus, columns of the from bus
    OH_AA, OH_MM, OH_MF_AT, OH_MT_AF,                 // (Va_f,Va_t), (Vm_f,Vm_t), (Vm_f,Va_t), (Vm_t,Va_f)
    NOFF
};

// Host plan of one grid: validated copies of the inputs, both sparsity patterns, and the output
// position of every value each kernel writes.
struct HostPlan {
    int nb = 0, nl = 0, ng = 0, n = 0, m = 0;
    int64_t nnzJ = 0, nnzJg = 0, nnzH = 0;
    double baseMVA = 100.0;
    std::vector<double> Gs, Bs, Pd, Qd, r, x, b, tap, rateA, c2, c1, c0;
    std::vector<int> f, t, gbus;

    std::vector<int64_t> Jrowptr, Hrowptr;
    std::vector<int> Jcol, Hcol;

    std::vector<int> br_off;      // [NOFF][nl] output positions (J for 0..7, H for 8..11)
    std::vector<int> br_slot;     // [2][nl] slot of the from end and of the to end
    std::vector<int> br_shared;   // [nl] -1, or index among branches with a parallel twin
    int nshared = 0;

    std::vector<int> slot_ptr;    // [nb + 1] slots of bus i are [slot_ptr[i], slot_ptr[i+1])
    int nslot = 0;                // 2 nl

    std::vector<int> bus_jP, bus_jQ, bus_k;   // [nb] J positions of (P_i, Va_i), (Q_i, Va_i);
                                              // k_i = columns per block, so Vm_i is at +k_i
    std::vector<int> bus_h;       // [3][nb] H positions (Va_i,Va_i), (Vm_i,Va_i), (Vm_i,Vm_i)
    std::vector<int> gen_ptr;     // [nb + 1] generators of bus i: gen_ord[gen_ptr[i] .. )
    std::vector<int> gen_ord;     // [ng] generator ids sorted by (bus, id)
    std::vector<int> gen_jP, gen_jQ, gen_h;   // [ng] positions of (P_bus, Pg_k), (Q_bus, Qg_k), (Pg_k, Pg_k)

    // Parallel-branch fixups: entry e sums fix_src[fix_ptr[e] .. fix_ptr[e+1]) into position
    // fix_dst[e] of J (fix_isH[e] == 0) or H.  A source is comp * nshared + shared index.
    std::vector<int> fix_ptr, fix_src, fix_dst;
    std::vector<uint8_t> fix_isH;
};

// Device view handed to the kernels by value.
struct DevNet {
    int nb, nl, ng, n, m, nslot, nslot_pad, nshared, nfix;
    int64_t nnzJ, nnzJg, nnzH;
    double baseMVA;
    const int *f, *t;
    const double *Gff, *Bff, *Gtt, *Btt, *Gft, *Bft;   // pi-model admittances (no phase shift: ft == tf)
    const int *br_off, *br_slot, *br_shared;
    const int *slot_ptr;
    const int *bus_jP, *bus_jQ, *bus_k, *bus_h;
    const double *Gs, *Bs, *Pd, *Qd;
    const int *gen_ptr, *gen_ord, *gen_bus, *gen_jP, *gen_jQ, *gen_h;
    const double *c2, *c1, *c0;
    const int *fix_ptr, *fix_src, *fix_dst;
    const uint8_t *fix_isH;
    int *status;                // device status word (host-mapped)
};

// What one evaluation call asks for.
struct EvalReq {
    int B;
    const double *x, *lam;
    const uint8_t *mask;
    const double *pd_scale, *obj_weight;
    double sigma;
    double *f, *grad, *gh, *jval, *hval;
    double *scratch;            // [B][NCOMP][nslot_pad] slot partial sums
    double *offscratch;         // [B][NOFF][nshared] off-diagonal values of parallel branches
};

// One adjoint-product call (adjoint.cu): JVP u -> J u, JTV v -> J^T v, HVP u -> (grad^2 L) u.
enum AdjMode : int { ADJ_JVP = 0, ADJ_JTV = 1, ADJ_HVP = 2 };
struct AdjReq {
    int B;
    const double *x, *lam;          // lam: HVP multipliers [B][m]
    const uint8_t *mask;
    const double *obj_weight;
    double sigma;
    const double *v;                // JVP / HVP: [B][n]; JTV: [B][m]
    double *out;                    // JVP: [B][m]; JTV / HVP: [B][n]
    double *scratch;                // [B][2][nslot_pad]
};
int launch_adjoint(const DevNet &net, const AdjReq &req, int mode, void *stream);

size_t workspace_bytes(const HostPlan &p, int B);

// Builds the plan; returns EXAGO_OK or EXAGO_EINVAL with a message in err.
exago_status build_plan(HostPlan &p, int nb, const double *Gs, const double *Bs, const double *Pd,
                        const double *Qd, int nl, const int *f, const int *t, const double *r,
                        const double *x, const double *b, const double *tap,
                        const double *rateA, int ng, const int *gbus, const double *c2,
                        const double *c1, const double *c0, double baseMVA, std::string &err);

// Optional per-kernel timing: an event is recorded on the launching stream before each kernel
// and after the last one; name[i] labels the interval ev[i] .. ev[i+1].
struct ProfileHook {
    static constexpr int MAX = 16;
    cudaEvent_t ev[MAX];
    const char *name[MAX];
    int n = 0;
};

// Kernel launchers (kernels.cu).  Each returns the launch's cudaError_t as int.
int launch_admittance(const double *r, const double *x, const double *b, const double *tap,
                      int nl, double *Gff, double *Bff, double *Gtt, double *Btt, double *Gft,
                      double *Bft, void *stream);
int launch_eval(const DevNet &net, const EvalReq &req, void *stream, ProfileHook *hook = nullptr);

// Persistent schedule (one launch; see kernels.cu).  counters: 1 + 2B ints of the workspace;
// req.scratch / req.offscratch hold `ring` state slots.
struct PersistLaunch {
    int block;              // 64, 128 or 256 threads
    int occ_warps;          // 0, 24 or 32: resident warps per SM the registers must allow
    int grid;               // CTAs (SM count x resident CTAs per SM)
    int lag, ring;          // bus tiles trail branch tiles by `lag` states; ring > lag slots
    long long spin_limit;   // polls before a bounded wait gives up
    int force_timeout;      // testing only
    int *counters;
};
int launch_eval_persistent(const DevNet &net, const EvalReq &req, const PersistLaunch &pl,
                           void *stream, ProfileHook *hook = nullptr);
int persist_blocks_per_sm(int block, int occ_warps);

// Read-only view of a net's plan and device tables (false for NULL or a plan-only net), and the
// thread-local error setter of the C ABI.  Used by entry points defined outside capi.cpp.
bool net_internal_view(exago_net_t net, const HostPlan **plan, const DevNet **dev, int *device);
exago_status set_last_error(exago_status s, const std::string &msg);

}  // namespace exago
