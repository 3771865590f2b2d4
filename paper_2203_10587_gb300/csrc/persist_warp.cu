// Warp-tiled persistent schedule of the polar AC-OPF model evaluation (ExaGO, arXiv 2203.10587,
// Sec. III, eqs. (7)-(10)): one launch over a batch of independent states (contingencies,
// Sec. V-A; scenarios, Sec. VI-A) in which a warp takes one branch or bus and its lanes take 32
// states (persist_warp.cuh).
#include <cuda_runtime.h>

#include "persist_warp.cuh"

namespace exago {

int persist_w_blocks_per_sm(int block, int occ_warps, int stage_cap) {
    const size_t smem = persist_w_smem(stage_cap);
    if (block == 128) return occupancy_w_nt<128, 0>(occ_warps, smem);
    return occupancy_w_nt<64, 0>(occ_warps, smem);
}

int persist_w_allow_stage() {
    int e = allow_stage_w_nt<64, 0>();
    if (e == 0) e = allow_stage_w_nt<128, 0>();
    if (e == 0) e = persist_w_allow_stage_gm();
    return e;
}

int launch_eval_persistent_w(const DevNet &N, const EvalReq &R, const PersistLaunch &L,
                             void *stream, ProfileHook *hk) {
    cudaStream_t st = (cudaStream_t)stream;
    if (R.B <= 0) return 0;
    const int block = L.block == 128 ? 128 : 64;
    const int per_item = (block / 32) * (L.group >= 1 ? L.group : 1);
    PersistParams P;
    P.B = (R.B + kLanes - 1) / kLanes;                       // groups of 32 states
    P.group = L.group >= 1 ? L.group : 1;
    P.Tbr = (N.nl + per_item - 1) / per_item;
    P.Tbu = (N.nb + per_item - 1) / per_item;
    P.lag = L.lag < P.B ? L.lag : P.B;
    P.ring = L.ring;
    P.total = P.B * (P.Tbr + P.Tbu);
    P.ctr = L.counters;
    P.spin_limit = L.spin_limit;
    P.force_timeout = L.force_timeout;
    P.times = hk ? hk->phase : nullptr;
    // every wait must point to a smaller ticket: ring slots must outnumber the lag
    if (P.lag < 1 || P.ring <= P.lag) return (int)cudaErrorInvalidValue;
    mark(hk, st, "persistent");
    cudaError_t e = cudaMemsetAsync(L.counters, 0, (size_t)(1 + 2 * P.B + kSpreadSMs) * sizeof(int),
                                    st);
    if (e != cudaSuccess) return (int)e;
    const int grid = L.grid < P.total ? L.grid : P.total;
    P.spread = L.sm_count > 0 && P.total <= 2 * grid ? (P.total + L.sm_count - 1) / L.sm_count : 0;
    int rc;
    if (R.gen_mask || R.tab || N.Gtf) rc = launch_persist_w_gm(block, N, R, P, grid, L.occ_warps, st);
    else if (block == 128) rc = launch_persist_w_nt<128, 0>(N, R, P, grid, L.occ_warps, st);
    else rc = launch_persist_w_nt<64, 0>(N, R, P, grid, L.occ_warps, st);
    mark(hk, st, "end");
    return rc;
}

}  // namespace exago
