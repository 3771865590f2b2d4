// Internal structures of the evaluator: the host plan built once per grid and the device view
// the kernels read.  Not part of the public ABI (include/exago.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/exago.h"

namespace exago {

// Per-(branch, end) record handed from the branch phase to the bus phase: NCOMP doubles at
// scratch[(b * nslot + slot) * NCOMP + k] for state b, where slot is the end's position in its
// bus's slot list.  A bus tile's records are therefore one contiguous range, which the bus phase
// can copy to shared memory in one coalesced pass; the branch phase writes each 80-byte record
// as five 16-byte pairs.  The end's injections P and Q are not carried: a bus's balances follow
// from its sums of dP/dVm_u, dQ/dVm_u, dP/dVa_u and dQ/dVa_u (bus_tail).  For the end at bus u
// towards bus v:
enum SlotComp {
    SC_PA = 0,   // dP/dVa_u            (dP/dVa_v = -dP/dVa_u)
    SC_PU = 1,   // dP/dVm_u
    SC_PV = 2,   // dP/dVm_v
    SC_QA = 3,   // dQ/dVa_u
    SC_QU = 4,   // dQ/dVm_u
    SC_QV = 5,   // dQ/dVm_v
    SC_HAA = 6,  // Lagrangian Hessian of the branch: (Va_u, Va_u) = -(Va_u, Va_v)
    SC_HUA = 7,  // (Vm_u, Va_u) = -(Vm_u, Va_v)
    SC_HUU = 8,  // (Vm_u, Vm_u)
    SC_HUV = 9,  // (Vm_u, Vm_v)
    NCOMP = 10
};

// Host plan of one grid: validated copies of the inputs, both sparsity patterns, and what each
// kernel needs to write its outputs.
struct HostPlan {
    int nb = 0, nl = 0, ng = 0, n = 0, m = 0;
    int64_t nnzJ = 0, nnzJg = 0, nnzH = 0;
    double baseMVA = 100.0;
    std::vector<double> Gs, Bs, Pd, Qd, r, x, b, tap, rateA, c2, c1, c0;
    std::vector<double> c2g, c1g;   // 2 c2 baseMVA^2 and c1 baseMVA
    std::vector<double> shift;      // [nl] phase shift (rad) per branch, or empty: none
    std::vector<int> f, t, gbus;

    std::vector<int64_t> Jrowptr, Hrowptr;
    std::vector<int> Jcol, Hcol;

    // Slots: one per (branch, end), grouped by the end's bus, ordered by (bus, other bus,
    // branch).  A bus's slots therefore visit its row columns in ascending order, and parallel
    // branches are adjacent.
    int nslot = 0;                // 2 nl
    std::vector<int> slot_ptr;    // [nb + 1] slots of bus i are [slot_ptr[i], slot_ptr[i+1])
    std::vector<int> slot_nbr;    // [nslot] the other bus of the slot's branch
    std::vector<int> slot_ref;    // [nslot] 2 l + end of the slot (adjoint records by branch)
    std::vector<int> br_slot;     // [2][nl] slot of the from end and of the to end
    std::vector<int> slot_bus;    // [nslot] the bus of the slot
    std::vector<int> slot_pos;    // [nslot] column of the neighbour among the bus's row columns,
                                  // or -1 for a later branch of a parallel group

    // Row starts of bus i: J rows P_i and Q_i, H rows Va_i and Vm_i; k_i = neighbours + 1 (Va
    // columns of a J row, Vm columns follow); nlow_i = neighbours below i (position of the
    // diagonal among the Va columns).
    std::vector<int> bus_jP, bus_jQ, bus_hA, bus_hM, bus_k, bus_nlow;
    // bus_perm: [4][nb]; row t holds, within every aligned tile of 32 << t buses, the tile's buses
    // by descending degree (then id), so that a warp of the bus phase walks slot lists of similar
    // length
    std::vector<int> bus_perm;
    std::vector<int> gen_ptr;     // [nb + 1] generators of bus i: gen_ord[gen_ptr[i] .. )
    std::vector<int> gen_ord;     // [ng] generator ids sorted by (bus, id)
};

// Device view handed to the kernels by value.
struct DevNet {
    int nb, nl, ng, n, m, nslot;
    int64_t nnzJ, nnzJg, nnzH, hpg;          // hpg: H position of (Pg_0, Pg_0)
    int jP_end, jQ_end, hA_end, hM_end;      // ends of the four row blocks of the bus rows
    int stage_cap_rows[4];                   // shared-memory doubles of a bus tile of 32/64/128/256
    int stage_cap_all[4];                    // buses: its row segments, or components plus rows
    int stage_cap_bulk[4];                   // ... or its whole records plus rows
    double baseMVA;
    const int *f, *t;
    const double *Gff, *Bff, *Gtt, *Btt, *Gft, *Bft;   // pi-model admittances (Gft, Bft: from end's)
    const double *Gtf, *Btf;     // to end's mutual admittances where they differ (phase-shifting
                                 // transformers), else nullptr: Gtf = Gft and Btf = Bft
    const double *Gff2, *Bff2, *Gtt2, *Btt2;            // 2 Gff, 2 Bff, 2 Gtt, 2 Btt (exact)
    const double *Kft;                                  // Gft^2 + Bft^2
    const int *slot_ptr, *slot_nbr, *slot_ref, *br_slot, *slot_bus, *slot_pos;
    const int *bus_jP, *bus_jQ, *bus_hA, *bus_hM, *bus_k, *bus_nlow, *bus_perm;
    const double *Gs, *Bs, *Pd, *Qd;
    const int *gen_ptr, *gen_ord;
    const double *c2, *c1, *c0;
    const double *c2g, *c1g;    // 2 c2 baseMVA^2 and c1 baseMVA (cost derivatives in p.u.)
    int *status;                // device status word (host-mapped)
    int chk_nslot;              // bound of slot indices for the debug build's checks (nslot)
};

// Device status word bits.  The bounded waits store their timeout codes (1, 2); the debug build's
// index checks (EXAGO_DEBUG) OR in ST_BOUNDS and skip the access they guard.
enum : int { ST_BOUNDS = 16 };
#if defined(__CUDACC__)
__device__ __forceinline__ bool debug_fail(int *status) {
    if (status) atomicOr(status, ST_BOUNDS);
    return false;
}
#endif
#ifdef EXAGO_DEBUG
#define EXAGO_DCHECK(N, cond) ((cond) ? true : ::exago::debug_fail((N).status))
#else
#define EXAGO_DCHECK(N, cond) true
#endif

// One state of a gathered batch (serving: states of several requests in one launch): where its
// inputs and outputs live.  Absent inputs are nullptr (no mask, unit load scale, weight 1).
struct StateTab {
    const double *x, *lam;
    const uint8_t *mask;
    const double *pd_scale, *obj_weight;   // obj_weight: this state's weight
    double sigma;
    double *f, *grad, *gh, *jval, *hval;   // this state's outputs (f: one value)
    const uint8_t *gen_mask;               // [ng], or nullptr (all in service)
};

// What one evaluation call asks for.  With tab, state b's inputs and outputs are tab[b]'s, and the
// batch pointers below only say which outputs are wanted (non-null) and which inputs exist.
struct EvalReq {
    const double *x, *lam;
    const uint8_t *mask;        // [B][nl]; NULL = all in service
    const double *pd_scale, *obj_weight;
    double sigma;
    double *f, *grad, *gh, *jval, *hval;
    double *scratch;            // [B][nslot][NCOMP] branch-end records (or ring slots)
    int scr_b0;                 // state b's records are at scratch + (b - scr_b0) * nslot * NCOMP
                                // in the multi-kernel and pipelined schedules
    int stage_recs;             // 1: bus tiles read their records slot-parallel into shared
                                // memory; 2: in one bulk copy (persistent kernel)
    int stage_cap;              // shared-memory doubles of one bus tile (records and rows)
    int B;
    const StateTab *tab;        // device table of B states, or nullptr
    const uint8_t *gen_mask;    // [B][ng] generator status; NULL = all in service
};
// The persistent kernel takes this struct by value beside DevNet and its own parameters; its
// size (128 bytes, no padding) is kept so that adding a field does not shift the kernel's other
// parameters (which measurably changed the generated code of the persistent kernel).
static_assert(sizeof(EvalReq) == 128, "EvalReq layout");

// Pipelined schedule (kernels.cu): the batch in chunks; the branch kernel of a chunk runs on the
// caller's stream while the bus kernel of the previous chunk runs on `side`, ordered by events
// only.  Records of `ring` chunks rotate through the workspace.
struct PipeLaunch {
    int chunk, ring;
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    cudaEvent_t ev_br[8], ev_bu[8];   // ring + 1 <= 8
};

// One adjoint-product call (adjoint.cu): JVP u -> J u, JTV v -> J^T v, HVP u -> (grad^2 L) u.
enum AdjMode : int { ADJ_JVP = 0, ADJ_JTV = 1, ADJ_HVP = 2 };
struct AdjReq {
    int B;
    const double *x, *lam;          // lam: HVP multipliers [B][m]
    const uint8_t *mask, *gen_mask;
    const double *obj_weight;
    double sigma;
    const double *v;                // JVP / HVP: [B][n]; JTV: [B][m]
    double *out;                    // JVP: [B][m]; JTV / HVP: [B][n]
    double *scratch;                // [B][2 nl][2] branch-end records
};
int launch_adjoint(const DevNet &net, const AdjReq &req, int mode, void *stream);

size_t workspace_bytes(const HostPlan &p, int B);

// Builds the plan; returns EXAGO_OK or EXAGO_EINVAL with a message in err.
exago_status build_plan(HostPlan &p, int nb, const double *Gs, const double *Bs, const double *Pd,
                        const double *Qd, int nl, const int *f, const int *t, const double *r,
                        const double *x, const double *b, const double *tap,
                        const double *rateA, int ng, const int *gbus, const double *c2,
                        const double *c1, const double *c0, double baseMVA,
                        const double *shift, std::string &err);

// Optional per-kernel timing: an event is recorded on the launching stream before each kernel
// and after the last one; name[i] labels the interval ev[i] .. ev[i+1].
// phase: a device array of 16 u64 for the persistent kernel's phase timestamps (earliest and
// latest global-timer ns of each PhaseSlot event, persist_kernel.cuh), or null.
struct ProfileHook {
    static constexpr int MAX = 16;
    cudaEvent_t ev[MAX];
    const char *name[MAX];
    int n = 0;
    unsigned long long *phase = nullptr;
};

// Kernel launchers (kernels.cu).  Each returns the launch's cudaError_t as int.
// Y[0..10] = Gff, Bff, Gtt, Btt, Gft, Bft, 2 Gff, 2 Bff, 2 Gtt, 2 Btt, Gft^2 + Bft^2; with a
// phase shift per branch (shift non-null), Y[11], Y[12] = Gtf, Btf as well.
int launch_admittance(const double *r, const double *x, const double *b, const double *tap,
                      const double *shift, int nl, double *const Y[13], void *stream);
int launch_eval(const DevNet &net, const EvalReq &req, void *stream, ProfileHook *hook = nullptr);
int launch_eval_pipelined(const DevNet &net, const EvalReq &req, const PipeLaunch &pl,
                          void *stream, ProfileHook *hook = nullptr);

// Persistent schedule (one launch; see persist.cu).  counters: 1 + 2B + 256 ints of the workspace;
// req.scratch holds `ring` state slots.
struct PersistLaunch {
    int block;              // 64, 128 or 256 threads
    int occ_warps;          // 16 or 24: resident warps per SM the registers must allow; 8: the
                            // compiler's choice
    int grid;               // CTAs (SM count x resident CTAs per SM)
    int lag, ring;          // bus tiles trail branch tiles by `lag` states; ring > lag slots
    int group;              // tiles of one kind and state per work item
    long long spin_limit;   // polls before a bounded wait gives up
    int force_timeout;      // testing only
    int sm_count;           // SMs of the device
    int *counters;          // 1 + 2B + 256 ints
};
int launch_eval_persistent(const DevNet &net, const EvalReq &req, const PersistLaunch &pl,
                           void *stream, ProfileHook *hook = nullptr);
int persist_blocks_per_sm(int block, int occ_warps, size_t smem_bytes);
// Warp-tiled persistent schedule (persist_warp.cu): a warp takes one branch or bus, its lanes 32
// states.  pl.block is 64 or 128; pl.lag and pl.ring count groups of 32 states; req.scratch holds
// `ring` group slots (persist_w_slot_doubles each); occ_warps 8 or 16; req.stage_cap is the
// doubles of one lane's shared-memory staging row (odd, at most kStageMaxDoubles / 32; 0 = none).
int launch_eval_persistent_w(const DevNet &net, const EvalReq &req, const PersistLaunch &pl,
                             void *stream, ProfileHook *hook = nullptr);
int persist_w_blocks_per_sm(int block, int occ_warps, int stage_cap);
int persist_w_allow_stage();

// Shared memory of a bus tile (eval_items.cuh, bus_tile): its records and its row segments.  The
// largest tile's need in doubles, capped at kStageMaxDoubles; a tile above the cap reads its
// records from global memory and writes its rows directly.
constexpr int kStageMaxDoubles = 9216;   // 72 KB
// The persistent schedule's ring slot of one state: NCOMP x nslot doubles of branch-end records,
// then the kObjLanes partial sums of the state's objective (256 virtual lanes).
constexpr int kObjLanes = 256;
constexpr int kDiagComps = 7;            // record components summed into a bus's diagonal
// One ring slot of the warp-tiled schedule: 32 states' lane-interleaved records, then their
// objective partials.
inline size_t persist_w_slot_doubles(int nslot) { return ((size_t)NCOMP * nslot + kObjLanes) * 32; }
__host__ __device__ inline int stage_index(int block) {
    return block == 32 ? 0 : block == 64 ? 1 : block == 256 ? 3 : 2;
}
int persist_allow_stage();   // persist.cu
int cart_allow_stage();      // cartesian.cu: the cartesian persistent kernel
int bus_allow_stage();       // kernels.cu
int bus_blocks_per_sm(size_t smem_bytes);   // k_bus blocks of 128 threads per SM (kernels.cu)

// Read-only view of a net's plan and device tables (false for NULL or a plan-only net), and the
// thread-local error setter of the C ABI.  Used by entry points defined outside capi.cpp.
bool net_internal_view(exago_net_t net, const HostPlan **plan, const DevNet **dev, int *device);
// The host plan of any net, with or without a device (false for NULL).
bool net_plan_view(exago_net_t net, const HostPlan **plan);
exago_status set_last_error(exago_status s, const std::string &msg);
// Shared-memory doubles of a bus tile of the multi-kernel schedule's bus kernel (128 threads),
// within the budget that keeps its register-limited residency, as exago_eval_all launches it.
int multi_kernel_stage_cap(exago_net_t net);
// Runs fn(ws, pl) with the net's lock held from the workspace lookup until fn returns, so that no
// other host thread can grow (and free) the workspace before fn's kernels are queued.  ws is
// caller_ws when given (or when bytes is 0), else the net's internal workspace grown to at least
// `bytes`, and then fn's work on `st` is ordered after the workspace's last use on another stream
// (as in the evaluations).  pl: the net's two-stream pipeline resources when `pipeline`, else null.
exago_status with_net_workspace(exago_net_t net, void *caller_ws, size_t bytes, cudaStream_t st,
                                bool pipeline,
                                const std::function<exago_status(void *, const PipeLaunch *)> &fn);
// The net's user configuration (exago_net_set_config; zeros = automatic).
exago_config net_config(exago_net_t net);
// Launches `launch`'s work through the net's cache of instantiated CUDA graphs, keyed by every
// argument the work bakes in (key[0] names the schedule).  Only inside with_net_workspace's fn
// (the net's lock held) and on a stream that is not being captured.
exago_status net_graph_launch_locked(exago_net_t net, const std::vector<uint64_t> &key,
                                     const std::function<int(cudaStream_t)> &launch,
                                     cudaStream_t stream);
// exago_eval_cart without the graph cache (serving: every request has its own buffers).
exago_status eval_cart_direct(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                              double *gh, double *jval, double *hval);
// cudaMalloc for every device allocation of the library (honours exago_test_fail_allocations).
cudaError_t dev_malloc(void **p, size_t bytes);
// exago_eval_all without the graph cache (serving: every request has its own buffers).  With
// tab (a device table of bt->B states), state b's inputs and outputs are tab[b]'s; bt and the
// output pointers then only say which inputs exist and which outputs are wanted.
exago_status eval_direct(exago_net_t net, const exago_batch *bt, double *f, double *grad,
                         double *gh, double *jval, double *hval, const StateTab *tab = nullptr);

}  // namespace exago
