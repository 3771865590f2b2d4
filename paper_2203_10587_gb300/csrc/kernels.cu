// CUDA kernels (sm_103a, FP64) of the polar AC-OPF model evaluation: ExaGO (arXiv 2203.10587),
// Sec. III, eqs. (7)-(10), batched over independent states (contingencies, Sec. V-A; scenarios,
// Sec. VI-A).
//
// GB300 executes FP64 at 1/64 of the FP32 rate (about 600 G FP64 instructions/s for the whole
// GPU), so the branch arithmetic, not HBM, bounds this path.  The kernels are therefore written
// to issue as few FP64 instructions as possible:
//   * one sincos per branch, shared by both ends; B cos and B sin serve both ends' flows and
//     each A, C term is one fma (without phase shift the mutual admittances are equal; a net
//     with phase-shifting transformers takes the to end's own pair in the variants that allow it);
//   * P and dP/dVm of an end come from one product Gss Vu + Vv A; the angle derivatives are
//     products of the magnitude derivatives;
//   * the Lagrangian Hessian block of an end, lamP grad^2 P + lamQ grad^2 Q + mu grad^2 (P^2+Q^2),
//     has only six distinct values, because every angle derivative is antisymmetric in
//     (Va_from, Va_to); A^2 + C^2 = G^2 + B^2 is a per-branch constant;
//   * out-of-service branches take a predicated path that only stores zeros;
//   * assembly sums each bus's branch-end records in a fixed slot order (by the other bus, then
//     branch), with no atomics, so results do not depend on the launch shape.
#include <cuda_runtime.h>

#include "eval_items.cuh"

namespace exago {

// ---------------------------------------------------------------------------------------------
// pi-model admittances (once per network).  ys = 1/(r + jx); Yff = (ys + jb/2)/tau^2,
// Ytt = ys + jb/2; tap 0 means tau = 1.  Without phase shift Yft = Ytf = -ys/tau.  A phase-shifting
// transformer has the complex ratio T = tau e^{j phi} on the from side: Yft = -ys/conj(T) =
// -ys e^{j phi}/tau and Ytf = -ys/T = -ys e^{-j phi}/tau (shift non-null; Y[11], Y[12] = Gtf, Btf).
struct AdmittanceOut {
    double *Y[13];   // Gff, Bff, Gtt, Btt, Gft, Bft, 2 Gff, 2 Bff, 2 Gtt, 2 Btt, Gft^2 + Bft^2,
                     // Gtf, Btf
};

__global__ void k_admittance(const double *__restrict__ r, const double *__restrict__ x,
                             const double *__restrict__ b, const double *__restrict__ tap,
                             const double *__restrict__ shift, int nl, AdmittanceOut out) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    double rl = r[l], xl = x[l];
    double z2 = rl * rl + xl * xl;
    double gs = rl / z2, bs = -xl / z2;
    double tau = tap[l] == 0.0 ? 1.0 : tap[l];
    double bc = bs + 0.5 * b[l];
    const double Gff = gs / (tau * tau), Bff = bc / (tau * tau);
    out.Y[0][l] = Gff;
    out.Y[1][l] = Bff;
    out.Y[2][l] = gs;
    out.Y[3][l] = bc;
    double Gft = -gs / tau, Bft = -bs / tau;
    if (shift) {
        double sp, cp;
        sincos(shift[l], &sp, &cp);
        Gft = -(gs * cp - bs * sp) / tau;        // -(gs + j bs)(cp + j sp) / tau
        Bft = -(gs * sp + bs * cp) / tau;
        out.Y[11][l] = -(gs * cp + bs * sp) / tau;   // -(gs + j bs)(cp - j sp) / tau
        out.Y[12][l] = -(bs * cp - gs * sp) / tau;
    }
    out.Y[4][l] = Gft;
    out.Y[5][l] = Bft;
    out.Y[10][l] = fma(Gft, Gft, Bft * Bft);     // |Yft|^2 = |Ytf|^2
    out.Y[6][l] = 2.0 * Gff;     // doubling is exact
    out.Y[7][l] = 2.0 * Bff;
    out.Y[8][l] = 2.0 * gs;
    out.Y[9][l] = 2.0 * bc;
}

int launch_admittance(const double *r, const double *x, const double *b, const double *tap,
                      const double *shift, int nl, double *const Y[13], void *stream) {
    if (nl <= 0) return 0;
    AdmittanceOut out;
    for (int k = 0; k < 13; k++) out.Y[k] = Y[k];
    k_admittance<<<(nl + 127) / 128, 128, 0, (cudaStream_t)stream>>>(r, x, b, tap, shift, nl, out);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Multi-kernel schedule: branch, bus, gradient and objective launches over the batch.
template <int WANT>
__global__ void __launch_bounds__(128) k_branch(const DevNet N, const EvalReq R, int b0) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = b0 + blockIdx.y;
    // this schedule always honours phase-shifting transformers (W_PS)
    if (l < N.nl) branch_item<WANT | W_PS>(N, R, b, l, R.scratch + (size_t)(b - R.scr_b0) * N.nslot * NCOMP);
}

template <int WANT>
__global__ void __launch_bounds__(128) k_bus(const DevNet N, const EvalReq R, int b0) {
    extern __shared__ double stage[];
    const int b = b0 + blockIdx.y;
    // this schedule always honours generator masks (W_GM)
    bus_tile<WANT | W_GM, BlockGroup>(N, R, b, blockIdx.x * blockDim.x,
                               R.scratch + (size_t)(b - R.scr_b0) * N.nslot * NCOMP, stage, R.stage_cap);
}

// Gradient of the objective: w (2 c2 base^2 Pg + c1 base) on Pg entries, 0 elsewhere.
__global__ void k_grad(const DevNet N, const EvalReq R, int b0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N.n) return;
    const int b = b0 + blockIdx.y;
    const int k = j - 2 * N.nb;
    st_grad(N, R, b)[j] = (k >= 0 && k < N.ng) ? grad_pg<true>(N, R, b, k) : 0.0;
}

__global__ void __launch_bounds__(OBJ_LANES) k_obj(const DevNet N, const EvalReq R, int b0) {
    __shared__ double part[OBJ_LANES];
    obj_block<true, OBJ_LANES>(N, R, b0 + blockIdx.x, part);
}

template <int WANT>
static void launch_branch_bus(const DevNet &N, const EvalReq &R, int b0, int nB, cudaStream_t st,
                              ProfileHook *hk) {
    if (N.nl > 0) {
        mark(hk, st, "branch");
        k_branch<WANT><<<dim3((N.nl + 127) / 128, nB), 128, 0, st>>>(N, R, b0);
    }
    mark(hk, st, "bus");
    const size_t smem = (size_t)R.stage_cap * sizeof(double);
    k_bus<WANT><<<dim3((N.nb + 127) / 128, nB), 128, smem, st>>>(N, R, b0);
}

// Opts the bus kernels in to kStageMaxDoubles of dynamic shared memory (once per device).
int bus_allow_stage() {
    const int bytes = kStageMaxDoubles * (int)sizeof(double);
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *k) {
        cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (r != cudaSuccess) e = r;
    };
    set((const void *)k_bus<W_G>); set((const void *)k_bus<W_J>); set((const void *)k_bus<W_G | W_J>);
    set((const void *)k_bus<W_H>); set((const void *)k_bus<W_G | W_H>);
    set((const void *)k_bus<W_J | W_H>); set((const void *)k_bus<W_G | W_J | W_H>);
    return (int)e;
}

int bus_blocks_per_sm(size_t smem_bytes) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bus<W_G | W_J | W_H>,
                                                                  128, smem_bytes);
    return e == cudaSuccess && per_sm > 0 ? per_sm : 1;
}

int launch_eval(const DevNet &N, const EvalReq &R, void *stream, ProfileHook *hk) {
    cudaStream_t st = (cudaStream_t)stream;
    const int want = (R.gh ? W_G : 0) | (R.jval ? W_J : 0) | (R.hval ? W_H : 0);
    const int maxY = 65535;
    for (int b0 = 0; b0 < R.B; b0 += maxY) {
        const int nB = R.B - b0 < maxY ? R.B - b0 : maxY;
        switch (want) {
            case 0: break;
            case W_G: launch_branch_bus<W_G>(N, R, b0, nB, st, hk); break;
            case W_J: launch_branch_bus<W_J>(N, R, b0, nB, st, hk); break;
            case W_G | W_J: launch_branch_bus<W_G | W_J>(N, R, b0, nB, st, hk); break;
            case W_H: launch_branch_bus<W_H>(N, R, b0, nB, st, hk); break;
            case W_G | W_H: launch_branch_bus<W_G | W_H>(N, R, b0, nB, st, hk); break;
            case W_J | W_H: launch_branch_bus<W_J | W_H>(N, R, b0, nB, st, hk); break;
            default: launch_branch_bus<W_G | W_J | W_H>(N, R, b0, nB, st, hk); break;
        }
        if (R.grad) {
            mark(hk, st, "grad");
            k_grad<<<dim3((N.n + 255) / 256, nB), 256, 0, st>>>(N, R, b0);
        }
    }
    if (R.f && R.B > 0) {
        mark(hk, st, "obj");
        k_obj<<<R.B, OBJ_LANES, 0, st>>>(N, R, 0);
    }
    mark(hk, st, "end");
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Pipelined schedule.  For chunk k of `chunk` states: the branch kernel runs on the caller's
// stream, then the bus and gradient kernels run on the side stream after an event from it, so
// the FP64-bound branch work of chunk k + 1 overlaps the latency-bound bus work of chunk k on the
// same SMs (each kernel keeps its own register allocation).  The branch kernel of chunk k waits
// for the bus kernel of chunk k - ring before it overwrites that chunk's ring slot.  All ordering
// is by events between launches; nothing waits inside a kernel.
template <int WANT>
static void pipe_chunk(const DevNet &N, const EvalReq &Rk, int b0, int nB, cudaStream_t main,
                       cudaStream_t side, cudaEvent_t ev_br, cudaEvent_t ev_bu) {
    if (N.nl > 0) k_branch<WANT><<<dim3((N.nl + 127) / 128, nB), 128, 0, main>>>(N, Rk, b0);
    cudaEventRecord(ev_br, main);
    cudaStreamWaitEvent(side, ev_br, 0);
    const size_t smem = (size_t)Rk.stage_cap * sizeof(double);
    if constexpr (WANT != 0) k_bus<WANT><<<dim3((N.nb + 127) / 128, nB), 128, smem, side>>>(N, Rk, b0);
    if (Rk.grad) k_grad<<<dim3((N.n + 255) / 256, nB), 256, 0, side>>>(N, Rk, b0);
    cudaEventRecord(ev_bu, side);
}

int launch_eval_pipelined(const DevNet &N, const EvalReq &R, const PipeLaunch &P, void *stream,
                          ProfileHook *hk) {
    cudaStream_t main = (cudaStream_t)stream;
    if (R.B <= 0) return 0;
    if (P.chunk < 1 || P.ring < 1 || P.ring + 1 > 8) return (int)cudaErrorInvalidValue;
    const int want = (R.gh ? W_G : 0) | (R.jval ? W_J : 0) | (R.hval ? W_H : 0);
    const size_t chunk_doubles = (size_t)P.chunk * N.nslot * NCOMP;
    mark(hk, main, "pipelined");
    cudaEventRecord(P.ev_fork, main);
    cudaStreamWaitEvent(P.side, P.ev_fork, 0);
    if (R.f) k_obj<<<R.B, OBJ_LANES, 0, main>>>(N, R, 0);
    const int nchunks = (R.B + P.chunk - 1) / P.chunk;
    for (int k = 0; k < nchunks; k++) {
        const int b0 = k * P.chunk;
        const int nB = R.B - b0 < P.chunk ? R.B - b0 : P.chunk;
        if (k >= P.ring) cudaStreamWaitEvent(main, P.ev_bu[(k - P.ring) % (P.ring + 1)], 0);
        EvalReq Rk = R;
        Rk.scratch = R.scratch + (size_t)(k % P.ring) * chunk_doubles;
        Rk.scr_b0 = b0;
        cudaEvent_t eb = P.ev_br[k % (P.ring + 1)], eu = P.ev_bu[k % (P.ring + 1)];
        switch (want) {
            case 0: pipe_chunk<0>(N, Rk, b0, nB, main, P.side, eb, eu); break;
            case W_G: pipe_chunk<W_G>(N, Rk, b0, nB, main, P.side, eb, eu); break;
            case W_J: pipe_chunk<W_J>(N, Rk, b0, nB, main, P.side, eb, eu); break;
            case W_G | W_J: pipe_chunk<W_G | W_J>(N, Rk, b0, nB, main, P.side, eb, eu); break;
            case W_H: pipe_chunk<W_H>(N, Rk, b0, nB, main, P.side, eb, eu); break;
            case W_G | W_H: pipe_chunk<W_G | W_H>(N, Rk, b0, nB, main, P.side, eb, eu); break;
            case W_J | W_H: pipe_chunk<W_J | W_H>(N, Rk, b0, nB, main, P.side, eb, eu); break;
            default: pipe_chunk<W_G | W_J | W_H>(N, Rk, b0, nB, main, P.side, eb, eu); break;
        }
    }
    cudaEventRecord(P.ev_join, P.side);
    cudaStreamWaitEvent(main, P.ev_join, 0);
    mark(hk, main, "end");
    return (int)cudaGetLastError();
}

}  // namespace exago
