// The warp-tiled ("branch per warp") persistent kernel of the polar AC-OPF model evaluation
// (ExaGO, arXiv 2203.10587, Sec. III, eqs. (7)-(10)) over a batch of independent states
// (SCOPFLOW contingencies, Sec. V-A; SOPFLOW scenarios, Sec. VI-A).  Included by persist_warp.cu
// (launches without generator masks) and persist_warp_gm.cu (with them, or phase shifters).
//
// The per-thread tiling (k_persist) gives each lane its own branch or bus of one state.  Here a
// warp takes one branch (or one bus) and its 32 lanes take 32 consecutive states of the batch:
//   * a bus's slot walk has the same length on every lane, so the walk runs converged (with a
//     branch or bus per lane, lanes of a warp walk buses of different degrees);
//   * the per-branch tables (admittances, slots, end buses) are one broadcast load per warp;
//   * records are interleaved by lane ([group][slot][NCOMP / 2][32][2]), so that a warp's record
//     stores and loads are 512-byte runs.
// The per-state inputs and outputs are the same rows as before, so those loads and stores are
// scattered across states instead.  Every (state, branch) and (state, bus) runs the same item
// functions in the same order as the per-thread tiling, so the outputs are bitwise equal.
//
// The work list is k_persist's with "state" replaced by "group of 32 states": for group g there
// are Tbr branch items and Tbu bus items of `group` x (NT / 32) branches or buses each, ordered
//     Br(0) .. Br(L-1), [Br(L) Bu(0)], ..., Bu(G-L) .. Bu(G-1),
// group g's records live in ring slot g mod ring, and the two bounded waits (a bus item for its
// group's branch items; a branch item for the bus items of the group that last used its ring
// slot) point to smaller tickets, as in k_persist, so the launch cannot deadlock.
#pragma once

#include <cuda_runtime.h>

#include "persist_kernel.cuh"

namespace exago {

constexpr int kLanes = 32;   // states per group (one per lane)

// Objective partial sums of one group for obj_block's virtual lanes [32 c, 32 c + 32), lane =
// state: virtual lane v sums the terms of generators v, v + 256, ... in increasing order (an
// out-of-service generator adds +0.0, as in obj_block), into part[v * 32 + lane].
template <bool GM>
__device__ __forceinline__ void obj_chunk_w(const DevNet &N, const EvalReq &R, int b, int c,
                                            double *part, int lane) {
    const double *Pg = st_x(N, R, b) + 2 * N.nb;
    [[maybe_unused]] const uint8_t *gm = nullptr;
    if constexpr (GM) gm = st_gmask(N, R, b);
    for (int v = 32 * c; v < 32 * c + 32; v++) {
        double acc = 0.0;
        for (int k = v; k < N.ng; k += OBJ_LANES) {
            double t = 0.0;
            bool on = true;
            if constexpr (GM) on = gen_on(gm, k);
            if (on) {
                const double MW = N.baseMVA * __ldg(Pg + k);
                t = fma(fma(__ldg(N.c2 + k), MW, __ldg(N.c1 + k)), MW, __ldg(N.c0 + k));
            }
            acc = acc + t;
        }
        part[(size_t)v * kLanes + lane] = acc;
    }
}

// obj_block's pairwise tree over the 256 partials of the lane's state (part[v * 32 + lane],
// written by other CTAs of the launch: read through L2): levels 128, 64 and 32 as in
// obj_tree_warp, the 32 results in tree[v * 32 + lane] (shared memory, 1024 doubles), then
// levels 16 .. 1 there.  Writes f of state b.
__device__ __forceinline__ void obj_tree_w(const EvalReq &R, int b, const double *part,
                                           double *tree, int lane) {
    for (int v = 0; v < 32; v++) {
        double p[8];
#pragma unroll
        for (int j = 0; j < 8; j++) p[j] = __ldcg(part + (size_t)(v + 32 * j) * kLanes + lane);
#pragma unroll
        for (int j = 0; j < 4; j++) p[j] += p[j + 4];
        p[0] += p[2];
        p[1] += p[3];
        tree[v * kLanes + lane] = p[0] + p[1];
    }
    for (int w = 16; w > 0; w >>= 1)
        for (int v = 0; v < w; v++) tree[v * kLanes + lane] += tree[(v + w) * kLanes + lane];
    *st_f(R, b) = st_w(R, b) * tree[lane];
}

// Where bus i of state b writes its rows: straight into the state's J and H values.
template <int WANT>
__device__ __forceinline__ BusRows rows_w(const DevNet &N, const EvalReq &R, int b, int i) {
    BusRows W{};
    if (WANT & W_J) {
        double *Jb = st_jval(N, R, b);
        W.JP = Jb + __ldg(N.bus_jP + i);
        W.JQ = Jb + __ldg(N.bus_jQ + i);
    }
    if (WANT & W_H) {
        double *Hb = st_hval(N, R, b);
        W.HA = Hb + __ldg(N.bus_hA + i);
        W.HM = Hb + __ldg(N.bus_hM + i);
    }
    return W;
}

// Copies the staged rows of the item's live states out of shared memory: state s (lane s) has
// `len` doubles at stage[s * lstr ..], of which [0, n0) go to dst(s, 0) + e, then n1 to dst(s, 1),
// n2 to dst(s, 2) and the rest to dst(s, 3) (each dst(s, k) a row segment of state s, offset so
// that element e of the staging row lands at dst + e).  Warp w takes states w, w + NW, ..., its
// lanes consecutive doubles of one state's segments.
template <int NW, class Dst>
__device__ __forceinline__ void copy_out_w(const double *stage, int lstr, int nlive, int len,
                                           int n0, int n1, int n2, const Dst &dst, int wid,
                                           int lane) {
    const int e1 = n0, e2 = n0 + n1, e3 = n0 + n1 + n2;
    for (int s = wid; s < nlive; s += NW) {
        const double *src = stage + (size_t)s * lstr;
        double *const d0 = dst(s, 0), *const d1 = dst(s, 1), *const d2 = dst(s, 2),
                      *const d3 = dst(s, 3);
        for (int e = lane; e < len; e += 32) {
            double *d = e < e1 ? d0 : e < e2 ? d1 : e < e3 ? d2 : d3;
            d[e] = src[e];
        }
    }
}

// P.B is the number of groups here; R.B the number of states.  R.stage_cap: doubles of one
// lane's staging row (odd; 0 = no staging); the dynamic shared memory holds 32 such rows, and
// at least the 1024 doubles of the objective tree.
template <int WANT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_persist_w(const DevNet N, const EvalReq R,
                                                        const PersistParams P) {
    static_assert(NT % 32 == 0 && NT >= 32, "whole warps");
    constexpr int NW = NT / 32;                                  // warps: branches per tile
    constexpr bool GM = (WANT & W_GM) != 0;
    constexpr bool WG = WANT & W_G, WJ = WANT & W_J, WH = WANT & W_H;
    __shared__ int s_item, s_ok;
    extern __shared__ double wstage[];
    int *done_br = P.ctr + 1, *done_bu = P.ctr + 1 + P.B;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t rec_doubles = (size_t)NCOMP * N.nslot * kLanes;
    const size_t slot_doubles = rec_doubles + (size_t)kObjLanes * kLanes;
    const int lstr = R.stage_cap;
    double *myrow = wstage + (size_t)lane * lstr;                // this lane's staging row
    // claiming as in k_persist: thread 0 claims the next ticket while the block works
    int next = 0;
    phase_mark(P.times, PH_ENTRY);
    if (threadIdx.x == 0) {
        if (P.spread > 0) {
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            const int k = smid < kSpreadSMs ? atomicAdd(P.ctr + 1 + 2 * P.B + smid, 1) : 0;
            if (k >= P.spread) next = P.total;
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
        __syncthreads();   // also: the previous item's staged rows are copied out
        const int t = s_item;
        if (t >= P.total) {
            phase_mark(P.times, PH_EXIT);
            return;
        }
        bool is_branch;
        int g, tile;
        decode_item(P, t, &is_branch, &g, &tile);
        const int b = g * kLanes + lane;                         // this lane's state
        const bool live = b < R.B;
        const int nlive = min(kLanes, R.B - g * kLanes);
        double *scr = R.scratch + (size_t)(g % P.ring) * slot_doubles;
        const int per_item = P.group * NW;                       // branches (buses) per item
        if (is_branch) {
            if (threadIdx.x == 0)
                s_ok = g < P.ring || bounded_wait(done_bu + (g - P.ring), P.Tbu, P.spin_limit,
                                                  N.status, ST_TIMEOUT_RING);
            __syncthreads();
            phase_mark(P.times, PH_BR_START);
            const int l0 = tile * per_item, cnt = min(N.nl, l0 + per_item) - l0;
            // the item's h rows, staged per lane as [J from rows | J to rows | h from | h to]
            const bool staged = (WJ || (WG && R.gh)) && 10 * per_item <= lstr;
            if (s_ok && live) {
                if (R.f) {
                    // obj_block's 256 virtual lanes in 8 chunks of 32; chunk c by warp c mod
                    // (Tbr NW) counted from the group's last branch item backwards
                    for (int c = (P.Tbr - 1 - tile) * NW + wid; c < OBJ_LANES / 32; c += P.Tbr * NW) {
                        phase_mark(P.times, PH_OBJ_START);
                        obj_chunk_w<GM>(N, R, b, c, scr + rec_doubles, lane);
                    }
                }
                for (int k = 0; k < P.group; k++) {
                    const int l = (tile * P.group + k) * NW + wid;
                    if (l >= N.nl) continue;
                    BranchOut O{};
                    if (staged) {
                        const int q = l - l0;
                        O.Jf = myrow + 4 * q;
                        O.Jt = myrow + 4 * per_item + 4 * q;
                        O.hf = myrow + 8 * per_item + q;
                        O.ht = myrow + 9 * per_item + q;
                    }
                    branch_item<WANT, kLanes>(N, R, b, l, scr + 2 * lane, O);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) red_release_add(done_br + g);
            phase_mark(P.times, PH_BR_END);
            if (staged && s_ok) {
                // a lane's staging row holds [J from rows | J to rows | h from | h to] at offsets
                // 0, 4 per_item, 8 per_item, 9 per_item; the item's 4 cnt, 4 cnt, cnt and cnt of
                // them go to four contiguous segments of the state's rows
                const int nj = WJ ? 4 * cnt : 0, nh = (WG && R.gh) ? cnt : 0;
                const int gbase = g * kLanes;
                for (int s = wid; s < nlive; s += NW) {
                    const double *src = wstage + (size_t)s * lstr;
                    double *Jb = WJ ? st_jval(N, R, gbase + s) + N.nnzJg + 4 * (size_t)l0 : nullptr;
                    double *hb = nh ? st_gh(N, R, gbase + s) + 2 * N.nb + l0 : nullptr;
                    for (int e = lane; e < 2 * nj + 2 * nh; e += 32) {
                        double *d;
                        int o;
                        if (e < nj) { d = Jb + e; o = e; }
                        else if (e < 2 * nj) { d = Jb + 4 * (size_t)N.nl + (e - nj); o = 4 * per_item + (e - nj); }
                        else if (e < 2 * nj + nh) { d = hb + (e - 2 * nj); o = 8 * per_item + (e - 2 * nj); }
                        else { d = hb + N.nl + (e - 2 * nj - nh); o = 9 * per_item + (e - 2 * nj - nh); }
                        *d = src[o];
                    }
                }
            }
        } else {
            if (threadIdx.x == 0)
                s_ok = bounded_wait(done_br + g, P.Tbr + P.force_timeout, P.spin_limit, N.status,
                                    ST_TIMEOUT_BUS);
            __syncthreads();
            phase_mark(P.times, PH_BU_START);
            const int i0 = tile * per_item, i1 = min(N.nb, i0 + per_item);
            const int nb = N.nb;
            const int p0 = row_start(N.bus_jP, i0, nb, N.jP_end), p1 = row_start(N.bus_jP, i1, nb, N.jP_end);
            const int q0 = row_start(N.bus_jQ, i0, nb, N.jQ_end);
            const int a0 = row_start(N.bus_hA, i0, nb, N.hA_end), a1 = row_start(N.bus_hA, i1, nb, N.hA_end);
            const int m0 = row_start(N.bus_hM, i0, nb, N.hM_end), m1 = row_start(N.bus_hM, i1, nb, N.hM_end);
            const int LP = WJ ? p1 - p0 : 0, LA = WH ? a1 - a0 : 0, LM = WH ? m1 - m0 : 0;
            const int LROWS = 2 * LP + LA + LM;
            const bool staged = (WJ || WH) && LROWS <= lstr;
            if (s_ok && live) {
                for (int k = 0; k < P.group; k++) {
                    const int i = (tile * P.group + k) * NW + wid;
                    if (i >= N.nb) break;
                    if (WANT & (W_G | W_J | W_H)) {
                        BusRows W;
                        if (staged) {
                            W.JP = myrow + (__ldg(N.bus_jP + i) - p0);
                            W.JQ = myrow + LP + (__ldg(N.bus_jQ + i) - q0);
                            W.HA = myrow + 2 * LP + (__ldg(N.bus_hA + i) - a0);
                            W.HM = myrow + 2 * LP + LA + (__ldg(N.bus_hM + i) - m0);
                        } else {
                            W = rows_w<WANT>(N, R, b, i);
                        }
                        bus_item<WANT, false, kLanes>(N, R, b, i, scr + 2 * lane, 0, W);
                    }
                    if (R.grad) grad_bus<GM>(N, R, b, i);
                }
            }
            if (tile == 0 && R.f && s_ok) {
                if (P.Tbr == 0) {   // no branch items: the partials here, by this item's warps
                    if (live)
                        for (int c = wid; c < OBJ_LANES / 32; c += NW)
                            obj_chunk_w<GM>(N, R, b, c, scr + rec_doubles, lane);
                }
            }
            __syncthreads();
            if (staged && s_ok) {
                const int gbase = g * kLanes;
                // element e of a lane's staging row: P rows [0, LP), Q rows [LP, 2 LP), Va rows
                // [2 LP, 2 LP + LA), Vm rows after; each base is offset by its segment's start
                auto dst = [&](int s, int k) -> double * {
                    if (k < 2) {
                        if (!WJ) return nullptr;
                        double *Jb = st_jval(N, R, gbase + s);
                        return k == 0 ? Jb + p0 : Jb + (q0 - LP);
                    }
                    if (!WH) return nullptr;
                    double *Hb = st_hval(N, R, gbase + s);
                    return k == 2 ? Hb + (a0 - 2 * LP) : Hb + (m0 - 2 * LP - LA);
                };
                copy_out_w<NW>(wstage, lstr, nlive, LROWS, LP, LP, LA, dst, wid, lane);
            }
            if (tile == 0 && R.f && s_ok) {
                // the tree in the staging space, once the rows are out
                if (staged) __syncthreads();
                if (wid == 0 && live) obj_tree_w(R, b, scr + rec_doubles, wstage, lane);
                phase_mark(P.times, PH_OBJ_END);
            }
            __syncthreads();
            phase_mark(P.times, PH_BU_END);
            if (threadIdx.x < 32) {
                if (s_ok && (WANT & (W_G | W_J | W_H))) {   // this item's records are consumed
                    discard_lines(scr + (size_t)__ldg(N.slot_ptr + i0) * (NCOMP * kLanes),
                                  scr + (size_t)__ldg(N.slot_ptr + i1) * (NCOMP * kLanes), lane);
                    __syncwarp();   // the lanes' discards before lane 0's release
                }
                if (threadIdx.x == 0) red_release_add(done_bu + g);
            }
        }
    }
}

// Dynamic shared memory of a launch: 32 staging rows of R.stage_cap doubles, and at least the
// objective tree's 1024 doubles.
inline size_t persist_w_smem(int stage_cap) {
    const size_t d = (size_t)kLanes * (stage_cap > 0 ? stage_cap : 0);
    return (d > 1024 ? d : 1024) * sizeof(double);
}

template <int WANT, int NT, int MINB>
static void launch_one_w(const DevNet &N, const EvalReq &R, const PersistParams &P, int grid,
                         cudaStream_t st) {
    k_persist_w<WANT, NT, MINB><<<grid, NT, persist_w_smem(R.stage_cap), st>>>(N, R, P);
}

// Launches the warp-tiled variant for the requested outputs (plus X = 0 or W_GM | W_PS): all
// outputs at 8 (compiler's registers) or 16 resident warps per SM, any other set of outputs with
// the compiler's registers.
template <int NT, int X>
static int launch_persist_w_nt(const DevNet &N, const EvalReq &R, const PersistParams &P,
                               int grid, int occ_warps, cudaStream_t st) {
    const int want = (R.gh ? W_G : 0) | (R.jval ? W_J : 0) | (R.hval ? W_H : 0);
    constexpr int ALL = W_G | W_J | W_H;
    if (want == ALL && occ_warps == 16) launch_one_w<ALL | X, NT, minb(NT, 16)>(N, R, P, grid, st);
    else switch (want) {
        case 0: launch_one_w<X, NT, 1>(N, R, P, grid, st); break;
        case W_G: launch_one_w<W_G | X, NT, 1>(N, R, P, grid, st); break;
        case W_J: launch_one_w<W_J | X, NT, 1>(N, R, P, grid, st); break;
        case W_G | W_J: launch_one_w<W_G | W_J | X, NT, 1>(N, R, P, grid, st); break;
        case W_H: launch_one_w<W_H | X, NT, 1>(N, R, P, grid, st); break;
        case W_G | W_H: launch_one_w<W_G | W_H | X, NT, 1>(N, R, P, grid, st); break;
        case W_J | W_H: launch_one_w<W_J | W_H | X, NT, 1>(N, R, P, grid, st); break;
        default: launch_one_w<ALL | X, NT, 1>(N, R, P, grid, st); break;
    }
    return (int)cudaGetLastError();
}

template <int NT, int X>
static int occupancy_w_nt(int occ_warps, size_t smem) {
    constexpr int ALL = W_G | W_J | W_H;
    int per_sm = 0;
    cudaError_t e = occ_warps == 16
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist_w<ALL | X, NT, minb(NT, 16)>, NT, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist_w<ALL | X, NT, 1>, NT, smem);
    return e == cudaSuccess && per_sm > 0 ? per_sm : 1;
}

// Opts every warp-tiled variant in to kStageMaxDoubles of dynamic shared memory.
template <int NT, int X>
static int allow_stage_w_nt() {
    const int bytes = kStageMaxDoubles * (int)sizeof(double);
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *k) {
        cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (r != cudaSuccess) e = r;
    };
    constexpr int ALL = W_G | W_J | W_H;
    set((const void *)k_persist_w<X, NT, 1>); set((const void *)k_persist_w<W_G | X, NT, 1>);
    set((const void *)k_persist_w<W_J | X, NT, 1>); set((const void *)k_persist_w<W_G | W_J | X, NT, 1>);
    set((const void *)k_persist_w<W_H | X, NT, 1>); set((const void *)k_persist_w<W_G | W_H | X, NT, 1>);
    set((const void *)k_persist_w<W_J | W_H | X, NT, 1>); set((const void *)k_persist_w<ALL | X, NT, 1>);
    set((const void *)k_persist_w<ALL | X, NT, minb(NT, 16)>);
    return (int)e;
}

// persist_warp_gm.cu: the variants with generator masks and phase shifters.
int launch_persist_w_gm(int block, const DevNet &N, const EvalReq &R, const PersistParams &P,
                        int grid, int occ_warps, cudaStream_t st);
int persist_w_allow_stage_gm();

}  // namespace exago
