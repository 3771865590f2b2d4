// The persistent fused kernel of the polar AC-OPF model evaluation (ExaGO, arXiv 2203.10587,
// Sec. III, eqs. (7)-(10)) and its launch helpers, templated on the outputs and on W_GM (per-state
// generator masks).  Included by persist.cu (launches without generator masks) and persist_gm.cu
// (launches with them), so that the two sets of instantiations compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "eval_items.cuh"

namespace exago {

// ---------------------------------------------------------------------------------------------
// Persistent schedule: one launch of numSMs x (resident CTAs per SM) blocks that claim work items
// from a ticket counter until the list is empty.  A work item is `group` consecutive tiles of
// one kind and one state (blockDim branches or buses each), so that the items' claims, waits and
// signals are shared by several tiles.  For each state b there are Tbr branch items and Tbu bus
// items.  The list is ordered
//     Br(0) .. Br(L-1), [Br(L) Bu(0)], [Br(L+1) Bu(1)], ..., Bu(B-L) .. Bu(B-1)
// so that bus tiles trail branch tiles by L states.  The branch partials of state b live in ring
// slot b mod Rg of the workspace (Rg > L slots, sized to stay in L2), which keeps the
// branch -> bus hand-off on chip.  Two waits order the work:
//   * a bus tile of b waits until all Tbr branch tiles of b have signalled;
//   * a branch tile of b >= Rg waits until all Tbu bus tiles of b - Rg have signalled (ring reuse).
// Both wait only on items with smaller tickets, which are held by running CTAs and wait only on
// smaller tickets still; the smallest unfinished ticket never waits, so the launch cannot
// deadlock.  Every wait is bounded: after spin_limit polls it records a timeout in the status
// word, skips its work and still signals, so the launch always ends.  The objective is split
// over the state's last branch items, which write the partial sums of its 256 virtual lanes into
// the ring slot (after the records), and bus tile 0 adds them up with obj_block's tree (it does
// the whole objective on a net without branches); every bus tile writes the gradient entries of
// its buses.
struct PersistParams {
    int B, Tbr, Tbu, lag, ring, total, group;
    int *ctr;               // [1 + 2B]: ticket, branch tiles done per state, bus tiles done
    long long spin_limit;
    int force_timeout;      // testing: bus tiles wait for one branch tile more than exists
    // exago_eval_profile only (else null): phase times in ns of the global timer, earliest
    // [0 .. PH_N) and latest [PH_N .. 2 PH_N) over the launch's CTAs (PhaseSlot)
    unsigned long long *times;
    // Small launches (a few items per SM): 0 = off.  Otherwise the CTAs rank themselves on their
    // SM (ctr[1 + 2B + smid]); rank >= spread exits at once, and rank k claims its first item
    // after k x kSpreadNs and claims one item at a time, so that consecutive tickets land on
    // different SMs instead of piling onto the CTAs that start first.
    int spread;
};
constexpr int kSpreadSMs = 256;        // per-SM rank counters after the per-state counters
constexpr unsigned kSpreadNs = 400;    // a claim round: about the time all SMs' first CTAs claim

// Phase timestamps of a profiled persistent launch: slot k holds the earliest (times[k]) and the
// latest (times[PH_N + k]) time that event k was reached.
enum PhaseSlot : int {
    PH_ENTRY = 0,      // a CTA starts
    PH_BR_START = 1,   // a branch item starts its work (after its ring wait)
    PH_BR_END = 2,     // a branch item has finished
    PH_BU_START = 3,   // a bus item starts its work (after its wait for the state's branches)
    PH_BU_END = 4,     // a bus item has finished
    PH_OBJ_START = 5,  // the objective of a state starts
    PH_OBJ_END = 6,    // and ends
    PH_EXIT = 7,       // a CTA exits
    PH_N = 8
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 of a profiled launch records event k (earliest and latest).
__device__ __forceinline__ void phase_mark(unsigned long long *times, int k) {
    if (times && threadIdx.x == 0) {
        const unsigned long long t = global_ns();
        atomicMin(times + k, t);
        atomicMax(times + PH_N + k, t);
    }
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Signals one finished tile: a release add at GPU scope.  Called by thread 0 after a
// __syncthreads, so it publishes the whole block's writes (release is cumulative).
__device__ __forceinline__ void red_release_add(int *p) {
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(p) : "memory");
}

// Polls *p until it reaches target; false (and a timeout code in the status word) after
// spin_limit polls.
static __device__ bool bounded_wait(const int *p, int target, long long limit, int *status, int code) {
    long long it = 0;
    while (ld_acquire(p) < target) {
        if (++it > limit) {
            if (status) *(volatile int *)status = code;
            return false;
        }
        __nanosleep(100);
    }
    return true;
}

// (code 3: a bus tile's bulk copy of its records did not complete, bulk_wait in eval_items.cuh)
enum : int { ST_TIMEOUT_BUS = 1, ST_TIMEOUT_RING = 2 };

// Invalidates in L2, without write-back, every whole 128-byte line of [p, q): branch-end records
// of a ring slot that its bus tiles have consumed.  Nothing reads them again; the ring slot's
// next writer (a branch tile of state b + ring, which waits for this tile's signal) overwrites
// them, so writing them back to DRAM would be wasted traffic.  PTX treats a discard as a weak
// write of indeterminate values, so the release of the tile's signal orders it before that next
// writer.  Lines shared with a neighbouring tile's range are kept.
// Called by the 32 lanes of one warp, which take every 32nd line.
__device__ __forceinline__ void discard_lines(const void *p, const void *q, int lane) {
    uintptr_t a = (((uintptr_t)p + 127) & ~(uintptr_t)127) + 128 * (uintptr_t)lane;
    const uintptr_t e = (uintptr_t)q & ~(uintptr_t)127;
    for (; a < e; a += 32 * 128) asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
}

__host__ __device__ __forceinline__ void decode_item(const PersistParams &P, int t, bool *is_branch,
                                                     int *b, int *tile) {
    const int L = P.lag, Tbr = P.Tbr, Tbu = P.Tbu;
    const int head = L * Tbr;
    if (t < head) {
        *is_branch = true; *b = t / Tbr; *tile = t % Tbr;
        return;
    }
    const int u = t - head, grp = Tbr + Tbu, ngroups = P.B - L;
    if (u < ngroups * grp) {
        const int g = u / grp, r = u % grp;
        if (r < Tbr) { *is_branch = true; *b = L + g; *tile = r; }
        else { *is_branch = false; *b = g; *tile = r - Tbr; }
        return;
    }
    const int v = u - ngroups * grp;
    *is_branch = false; *b = ngroups + v / Tbu; *tile = v % Tbu;
}

// MINB: resident CTAs per SM the register allocation must allow (1 = compiler's choice).
// WANT may carry W_GM: the variant that honours per-state generator masks.
template <int WANT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_persist(const DevNet N, const EvalReq R,
                                                      const PersistParams P) {
    __shared__ int s_item, s_ok;
    __shared__ double s_part[OBJ_LANES];
    __shared__ unsigned long long s_mbar;   // bulk copies of bus tiles' records (stage_recs 2)
    extern __shared__ __align__(16) double stage[];
    int *done_br = P.ctr + 1, *done_bu = P.ctr + 1 + P.B;
    static_assert(OBJ_LANES == kObjLanes && OBJ_LANES % NT == 0, "objective lanes");
    const size_t rec_doubles = (size_t)NCOMP * N.nslot;
    const size_t slot_doubles = rec_doubles + kObjLanes;   // records, then objective partials
    const int cap = R.stage_cap;
    // Thread 0 claims the next ticket while the block works on the current one.  The smallest
    // unfinished ticket is always some block's current item (a block's prefetched ticket is
    // larger than its current one), so the argument above still holds.  In a spread launch a
    // block claims one ticket at a time (and late-ranked blocks claim none): the argument holds
    // as well, since tickets are still claimed in order by running blocks.
    int next = 0;
    unsigned bulk_phase = 0;
    const BulkCtx bk{&s_mbar, P.spin_limit};
    if (R.stage_recs == 2 && threadIdx.x == 0) {
        const unsigned m = (unsigned)__cvta_generic_to_shared(&s_mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    phase_mark(P.times, PH_ENTRY);
    if (threadIdx.x == 0) {
        if (P.spread > 0) {
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            const int k = smid < kSpreadSMs ? atomicAdd(P.ctr + 1 + 2 * P.B + smid, 1) : 0;
            if (k >= P.spread) next = P.total;                   // enough blocks on this SM
            else {
                if (k > 0) __nanosleep(k * kSpreadNs);
                next = atomicAdd(P.ctr, 1);
            }
        } else {
            next = atomicAdd(P.ctr, 1);
        }
    }
    for (bool first = true;; first = false) {
        if (threadIdx.x == 0) {
            if (P.spread > 0) {
                if (!first && next < P.total) next = atomicAdd(P.ctr, 1);
                s_item = next;
            } else {
                s_item = next;
                if (next < P.total) next = atomicAdd(P.ctr, 1);
            }
        }
        __syncthreads();
        const int t = s_item;
        if (t >= P.total) {
            phase_mark(P.times, PH_EXIT);
            return;
        }
        bool is_branch;
        int b, tile;
        decode_item(P, t, &is_branch, &b, &tile);
        const int slot = b % P.ring;
        double *scr = R.scratch + (size_t)slot * slot_doubles;
        if (is_branch) {
            if (threadIdx.x == 0)
                s_ok = b < P.ring || bounded_wait(done_bu + (b - P.ring), P.Tbu, P.spin_limit,
                                                  N.status, ST_TIMEOUT_RING);
            __syncthreads();
            phase_mark(P.times, PH_BR_START);
            if (s_ok && R.f) {
                // the objective's lane groups q = 0 .. 256/NT - 1, group q by the state's branch
                // item Tbr - 1 - (q mod Tbr) (the last items, the ragged tail among them), into
                // the slot's partials; bus item 0 adds them up
                constexpr int G = OBJ_LANES / NT;
                for (int q = P.Tbr - 1 - tile; q < G; q += P.Tbr) {
                    phase_mark(P.times, PH_OBJ_START);
                    obj_lanes<(WANT & W_GM) != 0, NT>(N, R, b, q, scr + rec_doubles);
                }
            }
            if (s_ok)
                for (int l = tile * P.group * NT + threadIdx.x; l < N.nl && l < (tile + 1) * P.group * NT;
                     l += NT)
                    branch_item<WANT>(N, R, b, l, scr);
            __syncthreads();
            if (threadIdx.x == 0) red_release_add(done_br + b);
            phase_mark(P.times, PH_BR_END);
        } else {
            if (threadIdx.x == 0)
                s_ok = bounded_wait(done_br + b, P.Tbr + P.force_timeout, P.spin_limit, N.status,
                                    ST_TIMEOUT_BUS);
            __syncthreads();
            phase_mark(P.times, PH_BU_START);
            if (s_ok) {
                for (int k = 0; k < P.group; k++) {
                    const int i0 = (tile * P.group + k) * NT;
                    if (i0 >= N.nb) break;
                    if (WANT & (W_G | W_J | W_H))
                        bus_tile<WANT, BlockGroup>(N, R, b, i0, scr, stage, cap,
                                                   R.stage_recs == 2 ? &bk : nullptr, &bulk_phase);
                    if (i0 + (int)threadIdx.x < N.nb && R.grad)
                        grad_bus<(WANT & W_GM) != 0>(N, R, b, i0 + threadIdx.x);
                }
                if (tile == 0 && R.f) {
                    if (P.Tbr == 0) {   // no branch items: the whole objective here
                        obj_block<(WANT & W_GM) != 0, NT>(N, R, b, s_part);
                    } else if (threadIdx.x < 32) {
                        obj_tree_warp(R, b, scr + rec_doubles);
                    }
                    phase_mark(P.times, PH_OBJ_END);
                }
            }
            __syncthreads();
            phase_mark(P.times, PH_BU_END);
            if (threadIdx.x < 32) {
                if (s_ok && (WANT & (W_G | W_J | W_H))) {   // this item's records are consumed
                    const int i0 = tile * P.group * NT;
                    const int i1 = min(N.nb, (tile + 1) * P.group * NT);
                    discard_lines(scr + (size_t)__ldg(N.slot_ptr + i0) * NCOMP,
                                  scr + (size_t)__ldg(N.slot_ptr + i1) * NCOMP, threadIdx.x);
                    __syncwarp();   // the lanes' discards before lane 0's release
                }
                if (threadIdx.x == 0) red_release_add(done_bu + b);
            }
        }
    }
}

// CTAs per SM for a target of occ_warps resident warps (0: the compiler's register choice).
constexpr int minb(int nt, int occ_warps) {
    return occ_warps <= 0 ? 1 : (occ_warps / (nt / 32) > 0 ? occ_warps / (nt / 32) : 1);
}

template <int WANT, int NT, int MINB>
static void launch_one(const DevNet &N, const EvalReq &R, const PersistParams &P, int grid,
                       size_t smem, cudaStream_t st) {
    k_persist<WANT, NT, MINB><<<grid, NT, smem, st>>>(N, R, P);
}

// Opts every persistent variant in to kStageMaxDoubles of dynamic shared memory (above the
// default 48 KB once the static part is added).  Called once per device, outside any capture.
template <int NT, int X>
static int allow_stage_nt() {
    const int bytes = kStageMaxDoubles * (int)sizeof(double);
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *k) {
        cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (r != cudaSuccess) e = r;
    };
    constexpr int ALL = W_G | W_J | W_H;
    set((const void *)k_persist<X, NT, 1>); set((const void *)k_persist<W_G | X, NT, 1>);
    set((const void *)k_persist<W_J | X, NT, 1>); set((const void *)k_persist<W_G | W_J | X, NT, 1>);
    set((const void *)k_persist<W_H | X, NT, 1>); set((const void *)k_persist<W_G | W_H | X, NT, 1>);
    set((const void *)k_persist<W_J | W_H | X, NT, 1>); set((const void *)k_persist<ALL | X, NT, 1>);
    set((const void *)k_persist<ALL | X, NT, minb(NT, 24)>);
    set((const void *)k_persist<ALL | X, NT, minb(NT, 16)>);
    return (int)e;
}


// Launches the variant for the requested outputs (plus X = 0 or W_GM).
template <int NT, int X>
static int launch_persist_nt(const DevNet &N, const EvalReq &R, const PersistParams &P, int grid,
                             int occ_warps, cudaStream_t st) {
    const int want = (R.gh ? W_G : 0) | (R.jval ? W_J : 0) | (R.hval ? W_H : 0);
    const size_t smem = (size_t)R.stage_cap * sizeof(double);
    constexpr int ALL = W_G | W_J | W_H;
    if (want == ALL && occ_warps == 24) launch_one<ALL | X, NT, minb(NT, 24)>(N, R, P, grid, smem, st);
    else if (want == ALL && occ_warps == 16) launch_one<ALL | X, NT, minb(NT, 16)>(N, R, P, grid, smem, st);
    else switch (want) {
        case 0: launch_one<X, NT, 1>(N, R, P, grid, smem, st); break;
        case W_G: launch_one<W_G | X, NT, 1>(N, R, P, grid, smem, st); break;
        case W_J: launch_one<W_J | X, NT, 1>(N, R, P, grid, smem, st); break;
        case W_G | W_J: launch_one<W_G | W_J | X, NT, 1>(N, R, P, grid, smem, st); break;
        case W_H: launch_one<W_H | X, NT, 1>(N, R, P, grid, smem, st); break;
        case W_G | W_H: launch_one<W_G | W_H | X, NT, 1>(N, R, P, grid, smem, st); break;
        case W_J | W_H: launch_one<W_J | W_H | X, NT, 1>(N, R, P, grid, smem, st); break;
        default: launch_one<ALL | X, NT, 1>(N, R, P, grid, smem, st); break;
    }
    return (int)cudaGetLastError();
}


// Launch of the persistent variants with generator masks (persist_gm.cu).
int launch_persist_gm(int block, const DevNet &N, const EvalReq &R, const PersistParams &P,
                      int grid, int occ_warps, cudaStream_t st);
int persist_allow_stage_gm();

}  // namespace exago
