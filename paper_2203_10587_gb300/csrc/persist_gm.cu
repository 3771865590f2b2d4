// The persistent kernel's general variants: they honour per-state generator masks (a contingency
// may be a generator outage, Sec. V-A) and phase-shifting transformers (W_PS), and are compiled
// apart from the variants without them (persist.cu).
#include <cuda_runtime.h>

#include "persist_kernel.cuh"

namespace exago {

int launch_persist_gm(int block, const DevNet &N, const EvalReq &R, const PersistParams &P,
                      int grid, int occ_warps, cudaStream_t st) {
    if (block == 32) return launch_persist_nt<32, W_GM | W_PS>(N, R, P, grid, occ_warps, st);
    if (block == 256) return launch_persist_nt<256, W_GM | W_PS>(N, R, P, grid, occ_warps, st);
    if (block == 64) return launch_persist_nt<64, W_GM | W_PS>(N, R, P, grid, occ_warps, st);
    return launch_persist_nt<128, W_GM | W_PS>(N, R, P, grid, occ_warps, st);
}

int persist_allow_stage_gm() {
    int e = allow_stage_nt<32, W_GM | W_PS>();
    if (e == 0) e = allow_stage_nt<64, W_GM | W_PS>();
    if (e == 0) e = allow_stage_nt<128, W_GM | W_PS>();
    if (e == 0) e = allow_stage_nt<256, W_GM | W_PS>();
    return e;
}

}  // namespace exago
