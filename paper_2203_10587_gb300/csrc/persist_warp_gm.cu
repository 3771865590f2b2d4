// The warp-tiled persistent kernel's general variants: they honour per-state generator masks
// (Sec. V-A) and phase-shifting transformers (W_PS), compiled apart from the variants without
// them (persist_warp.cu).
#include <cuda_runtime.h>

#include "persist_warp.cuh"

namespace exago {

int launch_persist_w_gm(int block, const DevNet &N, const EvalReq &R, const PersistParams &P,
                        int grid, int occ_warps, cudaStream_t st) {
    if (block == 128) return launch_persist_w_nt<128, W_GM | W_PS>(N, R, P, grid, occ_warps, st);
    return launch_persist_w_nt<64, W_GM | W_PS>(N, R, P, grid, occ_warps, st);
}

int persist_w_allow_stage_gm() {
    int e = allow_stage_w_nt<64, W_GM | W_PS>();
    if (e == 0) e = allow_stage_w_nt<128, W_GM | W_PS>();
    return e;
}

}  // namespace exago
