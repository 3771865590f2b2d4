// Persistent fused schedule of the polar AC-OPF model evaluation (ExaGO, arXiv 2203.10587,
// Sec. III, eqs. (7)-(10)) over a batch of independent states (SCOPFLOW contingencies,
// Sec. V-A; SOPFLOW scenarios, Sec. VI-A; EMPAR subproblems, Sec. V-A): one launch whose CTAs
// claim branch and bus tiles of every state from a work list.
#include <cuda_runtime.h>

#include "persist_kernel.cuh"

namespace exago {

int persist_allow_stage() {
    int e = allow_stage_nt<32, 0>();
    if (e == 0) e = allow_stage_nt<64, 0>();
    if (e == 0) e = allow_stage_nt<128, 0>();
    if (e == 0) e = allow_stage_nt<256, 0>();
    if (e == 0) e = persist_allow_stage_gm();
    return e;
}

template <int NT, int MINB>
static int occupancy_of(size_t smem) {
    auto kern = k_persist<W_G | W_J | W_H, NT, MINB>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    return e == cudaSuccess && per_sm > 0 ? per_sm : 1;
}

template <int NT>
static int occupancy_nt(int occ_warps, size_t smem) {
    if (occ_warps == 24) return occupancy_of<NT, minb(NT, 24)>(smem);
    if (occ_warps == 16) return occupancy_of<NT, minb(NT, 16)>(smem);
    return occupancy_of<NT, 1>(smem);
}

int persist_blocks_per_sm(int block, int occ_warps, size_t smem_bytes) {
    if (block == 32) return occupancy_nt<32>(occ_warps, smem_bytes);
    if (block == 256) return occupancy_nt<256>(occ_warps, smem_bytes);
    if (block == 64) return occupancy_nt<64>(occ_warps, smem_bytes);
    return occupancy_nt<128>(occ_warps, smem_bytes);
}

int launch_eval_persistent(const DevNet &N, const EvalReq &R, const PersistLaunch &L,
                           void *stream, ProfileHook *hk) {
    cudaStream_t st = (cudaStream_t)stream;
    if (R.B <= 0) return 0;
    PersistParams P;
    P.B = R.B;
    P.group = L.group >= 1 ? L.group : 1;
    P.Tbr = (N.nl + L.block * P.group - 1) / (L.block * P.group);
    P.Tbu = (N.nb + L.block * P.group - 1) / (L.block * P.group);
    P.lag = L.lag < R.B ? L.lag : R.B;
    P.ring = L.ring;
    P.total = R.B * (P.Tbr + P.Tbu);
    P.ctr = L.counters;
    P.spin_limit = L.spin_limit;
    P.force_timeout = L.force_timeout;
    P.times = hk ? hk->phase : nullptr;
    // every wait must point to a smaller ticket: ring slots must outnumber the lag
    if (P.lag < 1 || P.ring <= P.lag) return (int)cudaErrorInvalidValue;
    mark(hk, st, "persistent");
    cudaError_t e = cudaMemsetAsync(L.counters, 0, (size_t)(1 + 2 * R.B + kSpreadSMs) * sizeof(int),
                                    st);
    if (e != cudaSuccess) return (int)e;
    int grid = L.grid < P.total ? L.grid : P.total;
    // a launch of at most two items per CTA spreads its items over the SMs (PersistParams::spread):
    // the first ceil(total / SMs) CTAs of each SM take part
    P.spread = L.sm_count > 0 && P.total <= 2 * grid ? (P.total + L.sm_count - 1) / L.sm_count : 0;
    int rc;
    if (R.gen_mask || R.tab || N.Gtf) {
        // generator masks (a gathered batch's states may carry their own) or phase shifters
        rc = launch_persist_gm(L.block, N, R, P, grid, L.occ_warps, st);
    } else if (L.block == 32) rc = launch_persist_nt<32, 0>(N, R, P, grid, L.occ_warps, st);
    else if (L.block == 256) rc = launch_persist_nt<256, 0>(N, R, P, grid, L.occ_warps, st);
    else if (L.block == 64) rc = launch_persist_nt<64, 0>(N, R, P, grid, L.occ_warps, st);
    else rc = launch_persist_nt<128, 0>(N, R, P, grid, L.occ_warps, st);
    mark(hk, st, "end");
    return rc;
}

}  // namespace exago

extern "C" exago_status exago_test_work_list(int B, int Tbr, int Tbu, int lag, int *kind,
                                             int *state, int *tile) {
    if (B < 1 || Tbr < 0 || Tbu < 1 || lag < 1 || lag > B || !kind || !state || !tile ||
        (long long)B * (Tbr + Tbu) > 2147483647ll)
        return exago::set_last_error(EXAGO_EINVAL, "bad work-list arguments");
    exago::PersistParams P{};
    P.B = B;
    P.Tbr = Tbr;
    P.Tbu = Tbu;
    P.lag = lag;
    P.total = B * (Tbr + Tbu);
    for (int t = 0; t < P.total; t++) {
        bool br = false;
        int b = 0, tl = 0;
        exago::decode_item(P, t, &br, &b, &tl);
        kind[t] = br ? 1 : 0;
        state[t] = b;
        tile[t] = tl;
    }
    return EXAGO_OK;
}
