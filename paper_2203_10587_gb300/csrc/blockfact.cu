// Batched numeric block factorisation and solve (blockfact.h), one thread per (state, target
// block) per level of the elimination tree.
//
// Factor, per level: every target (I, J) of the level's columns accumulates its left-looking
// update T_IJ = A_IJ - sum_K F_IK U_KJ (SYM: U_KJ = L_JK') in registers, in the pair order the
// host fixed (ascending K), and stores it; then every target rescales by the inverse of its
// column's pivot block D_J = T_JJ (L_IJ = T_IJ D_J^-1; LU: U_JI = D_J^-1 T'_JI; the diagonal
// position of L receives D_J^-1).  The pivot block is inverted by Gauss-Jordan elimination
// without pivoting, in the same order by every thread of its column, so all of them use bitwise
// the same inverse.  Solve: forward y_J = r_J - sum_K F_JK z_K, z_J = D_J^-1 y_J over ascending
// levels (F = L D is what the factor kept in T), then backward x_J = z_J - sum_I U_JI x_I over
// descending levels.
// A warp holds 32 consecutive states of one target, so every value load is one coalesced
// 256-byte access and every index load is uniform across the warp.
#include <cuda_runtime.h>

#include "blockfact.h"
#include "internal.h"

namespace exago {

namespace {

constexpr int kNT = 128;   // states per block

template <int BS>
__device__ __forceinline__ void load_blk(const double *A, int64_t p, int B, int b, double *v) {
    constexpr int BB = BS * BS;
    const double *a = A + (size_t)p * BB * B + b;
#pragma unroll
    for (int e = 0; e < BB; e++) v[e] = __ldg(a + (size_t)e * B);
}

template <int BS>
__device__ __forceinline__ void load_blk_cg(const double *A, int64_t p, int B, int b, double *v) {
    // values written earlier in the same factorisation by other blocks: through L2
    constexpr int BB = BS * BS;
    const double *a = A + (size_t)p * BB * B + b;
#pragma unroll
    for (int e = 0; e < BB; e++) v[e] = __ldcg(a + (size_t)e * B);
}

template <int BS>
__device__ __forceinline__ void store_blk(double *A, int64_t p, int B, int b, const double *v) {
    constexpr int BB = BS * BS;
    double *a = A + (size_t)p * BB * B + b;
#pragma unroll
    for (int e = 0; e < BB; e++) a[(size_t)e * B] = v[e];
}

// acc -= X Y  (X, Y, acc BS x BS row-major), or acc -= X Y' with TY.
template <int BS, bool TY>
__device__ __forceinline__ void sub_mul(double *acc, const double *X, const double *Y) {
#pragma unroll
    for (int i = 0; i < BS; i++)
#pragma unroll
        for (int j = 0; j < BS; j++) {
            double s = acc[i * BS + j];
#pragma unroll
            for (int k = 0; k < BS; k++) s = fma(-X[i * BS + k], TY ? Y[j * BS + k] : Y[k * BS + j], s);
            acc[i * BS + j] = s;
        }
}

// out = X Y
template <int BS>
__device__ __forceinline__ void mul(const double *X, const double *Y, double *out) {
#pragma unroll
    for (int i = 0; i < BS; i++)
#pragma unroll
        for (int j = 0; j < BS; j++) {
            double s = X[i * BS] * Y[j];
#pragma unroll
            for (int k = 1; k < BS; k++) s = fma(X[i * BS + k], Y[k * BS + j], s);
            out[i * BS + j] = s;
        }
}

// Inverse of the pivot block by Gauss-Jordan elimination without pivoting.  neg: pivots below
// zero (for a symmetric block, its negative eigenvalues: the pivots are the D of its LDL');
// bad: pivots with |d| <= tiny * max |entry| (the block is numerically singular).
template <int BS>
__device__ __forceinline__ void invert(const double *D, double *inv, int *neg, int *bad, double tiny) {
    double a[BS][2 * BS];
    double amax = 0.0;
#pragma unroll
    for (int i = 0; i < BS; i++)
#pragma unroll
        for (int j = 0; j < BS; j++) {
            a[i][j] = D[i * BS + j];
            a[i][BS + j] = i == j ? 1.0 : 0.0;
            amax = fmax(amax, fabs(D[i * BS + j]));
        }
    int nneg = 0, nbad = 0;
#pragma unroll
    for (int k = 0; k < BS; k++) {
        const double piv = a[k][k];
        nneg += piv < 0.0;
        nbad += !(fabs(piv) > tiny * amax);
        const double r = 1.0 / piv;
#pragma unroll
        for (int j = 0; j < 2 * BS; j++) a[k][j] *= r;
#pragma unroll
        for (int i = 0; i < BS; i++) {
            if (i == k) continue;
            const double f = a[i][k];
#pragma unroll
            for (int j = 0; j < 2 * BS; j++) a[i][j] = fma(-f, a[k][j], a[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < BS; i++)
#pragma unroll
        for (int j = 0; j < BS; j++) inv[i * BS + j] = a[i][BS + j];
    *neg = nneg;
    *bad = nbad;
}

// Update phase of one level: targets [t0, t0 + gridDim.x).
template <int BS, bool SYM>
__global__ void __launch_bounds__(kNT) k_bf_update(const DevSymK S, int B, double *T, double *TU,
                                                   const double *L, const double *U, int t0) {
    constexpr int BB = BS * BS;
    const int b = blockIdx.y * kNT + threadIdx.x;
    if (b >= B) return;
    const int t = t0 + blockIdx.x;
    const int p = __ldg(S.tgt_blk + t);
    const bool diag = p == __ldg(S.tgt_diag + t);
    const int64_t q0 = __ldg(S.tptr + t), q1 = __ldg(S.tptr + t + 1);
    if (q0 == q1) return;   // nothing to subtract: T already holds A_IJ
    double acc[BB], accU[BB];
    load_blk_cg<BS>(T, p, B, b, acc);
    if (!SYM && !diag) load_blk_cg<BS>(TU, p, B, b, accU);
    for (int64_t q = q0; q < q1; q++) {
        const int2 pr = __ldg(S.pairs + q);   // (I, K), (J, K)
        if (!EXAGO_DCHECK(S, pr.x >= 0 && pr.x < S.nblk && pr.y >= 0 && pr.y < S.nblk)) continue;
        double X[BB], Y[BB];
        load_blk_cg<BS>(T, pr.x, B, b, X);                      // F_IK
        if (SYM) {
            load_blk_cg<BS>(L, pr.y, B, b, Y);                  // L_JK
            sub_mul<BS, true>(acc, X, Y);
        } else {
            load_blk_cg<BS>(U, pr.y, B, b, Y);                  // U_KJ
            sub_mul<BS, false>(acc, X, Y);
            if (!diag) {
                load_blk_cg<BS>(T, pr.y, B, b, X);              // F_JK
                load_blk_cg<BS>(U, pr.x, B, b, Y);              // U_KI
                sub_mul<BS, false>(accU, X, Y);
            }
        }
    }
    store_blk<BS>(T, p, B, b, acc);
    if (!SYM && !diag) store_blk<BS>(TU, p, B, b, accU);
}

// Scale phase of one level.
template <int BS, bool SYM>
__global__ void __launch_bounds__(kNT) k_bf_scale(const DevSymK S, int B, const double *T,
                                                  const double *TU, double *L, double *U,
                                                  int *neg, int *bad, double tiny, int t0) {
    constexpr int BB = BS * BS;
    const int b = blockIdx.y * kNT + threadIdx.x;
    if (b >= B) return;
    const int t = t0 + blockIdx.x;
    const int p = __ldg(S.tgt_blk + t), pd = __ldg(S.tgt_diag + t);
    double D[BB], Di[BB];
    load_blk_cg<BS>(T, pd, B, b, D);
    int nn, nbad;
    invert<BS>(D, Di, &nn, &nbad, tiny);
    if (p == pd) {
        store_blk<BS>(L, p, B, b, Di);
        if (nn) atomicAdd(neg + b, nn);
        if (nbad) atomicAdd(bad + b, nbad);
        return;
    }
    double X[BB], Y[BB];
    load_blk_cg<BS>(T, p, B, b, X);
    mul<BS>(X, Di, Y);                                          // L_IJ = T_IJ D_J^-1
    store_blk<BS>(L, p, B, b, Y);
    if (!SYM) {
        load_blk_cg<BS>(TU, p, B, b, X);
        mul<BS>(Di, X, Y);                                      // U_JI = D_J^-1 T'_JI
        store_blk<BS>(U, p, B, b, Y);
    }
}

// ---- split variants: the terms of one target (or one column's sweep) divided among kSlices
// (kSweepSlices) warps of a block that holds 32 states; slice w takes every kSlices-th term from
// the w-th, and
// warp 0 adds the slices' partial sums in slice order.  Used where a level has few targets, so
// that the long sums of the dense top of the elimination tree are not one thread's latency
// chain.  The split is fixed by the structure alone (never by the batch size), so every state's
// result is the same whatever the batch it belongs to.
constexpr int kSlices = 8;
constexpr int kSweepSlices = 32;   // the sweeps carry less per term, so they split wider

template <int BS, bool SYM>
__global__ void __launch_bounds__(32 * kSlices) k_bf_update_split(const DevSymK S, int B, double *T,
                                                                  double *TU, const double *L,
                                                                  const double *U, int t0) {
    constexpr int BB = BS * BS, NP = SYM ? BB : 2 * BB;   // partial sums: lower (and upper)
    __shared__ double part[kSlices][NP][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane;
    const bool live = b < B;
    const int t = t0 + blockIdx.x;
    const int p = __ldg(S.tgt_blk + t);
    const bool diag = p == __ldg(S.tgt_diag + t);
    const int64_t q0 = __ldg(S.tptr + t), q1 = __ldg(S.tptr + t + 1);
    if (q0 == q1) return;   // uniform over the block
    double acc[BB], accU[BB];
#pragma unroll
    for (int e = 0; e < BB; e++) { acc[e] = 0.0; accU[e] = 0.0; }
    if (live)
        for (int64_t q = q0 + w; q < q1; q += kSlices) {
            const int2 pr = __ldg(S.pairs + q);
            if (!EXAGO_DCHECK(S, pr.x >= 0 && pr.x < S.nblk && pr.y >= 0 && pr.y < S.nblk)) continue;
            double X[BB], Y[BB];
            load_blk_cg<BS>(T, pr.x, B, b, X);
            if (SYM) {
                load_blk_cg<BS>(L, pr.y, B, b, Y);
                sub_mul<BS, true>(acc, X, Y);
            } else {
                load_blk_cg<BS>(U, pr.y, B, b, Y);
                sub_mul<BS, false>(acc, X, Y);
                if (!diag) {
                    load_blk_cg<BS>(T, pr.y, B, b, X);
                    load_blk_cg<BS>(U, pr.x, B, b, Y);
                    sub_mul<BS, false>(accU, X, Y);
                }
            }
        }
#pragma unroll
    for (int e = 0; e < BB; e++) {
        part[w][e][lane] = acc[e];
        if (!SYM) part[w][(NP - BB) + e][lane] = accU[e];
    }
    __syncthreads();
    if (w != 0 || !live) return;
    load_blk_cg<BS>(T, p, B, b, acc);
    if (!SYM && !diag) load_blk_cg<BS>(TU, p, B, b, accU);
#pragma unroll
    for (int e = 0; e < BB; e++) {
        double s = part[0][e][lane];
#pragma unroll
        for (int v = 1; v < kSlices; v++) s += part[v][e][lane];
        acc[e] += s;
        if (!SYM) {
            double su = part[0][(NP - BB) + e][lane];
#pragma unroll
            for (int v = 1; v < kSlices; v++) su += part[v][(NP - BB) + e][lane];
            accU[e] += su;
        }
    }
    store_blk<BS>(T, p, B, b, acc);
    if (!SYM && !diag) store_blk<BS>(TU, p, B, b, accU);
}

// Forward sweep of one level's columns, split: y_J = r_J + (the slices' sums of -F_JK z_K);
// z_J = D_J^-1 y_J.
template <int BS>
__global__ void __launch_bounds__(32 * kSweepSlices) k_bf_forward_split(const DevSymK S, int B,
                                                                   const double *T,
                                                                   const double *L, double *x,
                                                                   int c0) {
    __shared__ double part[kSweepSlices][BS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane;
    const bool live = b < B;
    const int J = __ldg(S.lvl_cols + c0 + blockIdx.x);
    double y[BS];
#pragma unroll
    for (int i = 0; i < BS; i++) y[i] = 0.0;
    const int64_t r0 = __ldg(S.rowptr + J), r1 = __ldg(S.rowptr + J + 1);
    if (live)
        for (int64_t r = r0 + w; r < r1; r += kSweepSlices) {
            const int K = __ldg(S.rowcol + r), p = __ldg(S.rowblk + r);
            if (!EXAGO_DCHECK(S, K >= 0 && K < S.nb && p >= 0 && p < S.nblk)) continue;
            double F[BS * BS], z[BS];
            load_blk<BS>(T, p, B, b, F);
#pragma unroll
            for (int i = 0; i < BS; i++) z[i] = __ldcg(x + ((size_t)K * BS + i) * B + b);
#pragma unroll
            for (int i = 0; i < BS; i++)
#pragma unroll
                for (int k = 0; k < BS; k++) y[i] = fma(-F[i * BS + k], z[k], y[i]);
        }
#pragma unroll
    for (int i = 0; i < BS; i++) part[w][i][lane] = y[i];
    __syncthreads();
    if (w != 0 || !live) return;
#pragma unroll
    for (int i = 0; i < BS; i++) {
        double s = part[0][i][lane];
#pragma unroll
        for (int v = 1; v < kSweepSlices; v++) s += part[v][i][lane];
        y[i] = __ldcg(x + ((size_t)J * BS + i) * B + b) + s;
    }
    double Di[BS * BS];
    load_blk<BS>(L, __ldg(S.colptr + J), B, b, Di);
#pragma unroll
    for (int i = 0; i < BS; i++) {
        double s = Di[i * BS] * y[0];
#pragma unroll
        for (int k = 1; k < BS; k++) s = fma(Di[i * BS + k], y[k], s);
        x[((size_t)J * BS + i) * B + b] = s;
    }
}

// Backward sweep of one level's columns, split: x_J = z_J + (the slices' sums of -U_JI x_I).
template <int BS, bool SYM>
__global__ void __launch_bounds__(32 * kSweepSlices) k_bf_backward_split(const DevSymK S, int B,
                                                                    const double *L,
                                                                    const double *U, double *x,
                                                                    int c0) {
    __shared__ double part[kSweepSlices][BS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane;
    const bool live = b < B;
    const int J = __ldg(S.lvl_cols + c0 + blockIdx.x);
    double v[BS];
#pragma unroll
    for (int i = 0; i < BS; i++) v[i] = 0.0;
    const int64_t p0 = __ldg(S.colptr + J), p1 = __ldg(S.colptr + J + 1);
    if (live)
        for (int64_t p = p0 + 1 + w; p < p1; p += kSweepSlices) {
            const int I = __ldg(S.rowidx + p);
            if (!EXAGO_DCHECK(S, I >= 0 && I < S.nb)) continue;
            double M[BS * BS], xi[BS];
            load_blk<BS>(SYM ? L : U, p, B, b, M);
#pragma unroll
            for (int i = 0; i < BS; i++) xi[i] = __ldcg(x + ((size_t)I * BS + i) * B + b);
#pragma unroll
            for (int i = 0; i < BS; i++)
#pragma unroll
                for (int k = 0; k < BS; k++)
                    v[i] = fma(-(SYM ? M[k * BS + i] : M[i * BS + k]), xi[k], v[i]);
        }
#pragma unroll
    for (int i = 0; i < BS; i++) part[w][i][lane] = v[i];
    __syncthreads();
    if (w != 0 || !live) return;
#pragma unroll
    for (int i = 0; i < BS; i++) {
        double s = part[0][i][lane];
#pragma unroll
        for (int u = 1; u < kSweepSlices; u++) s += part[u][i][lane];
        x[((size_t)J * BS + i) * B + b] = __ldcg(x + ((size_t)J * BS + i) * B + b) + s;
    }
}

// Forward sweep of one level's columns: y_J = r_J - sum_K F_JK z_K; z_J = D_J^-1 y_J.
template <int BS>
__global__ void __launch_bounds__(kNT) k_bf_forward(const DevSymK S, int B, const double *T,
                                                    const double *L, double *x, int c0) {
    const int b = blockIdx.y * kNT + threadIdx.x;
    if (b >= B) return;
    const int J = __ldg(S.lvl_cols + c0 + blockIdx.x);
    double y[BS];
#pragma unroll
    for (int i = 0; i < BS; i++) y[i] = __ldcg(x + ((size_t)J * BS + i) * B + b);
    const int64_t r0 = __ldg(S.rowptr + J), r1 = __ldg(S.rowptr + J + 1);
    for (int64_t r = r0; r < r1; r++) {
        const int K = __ldg(S.rowcol + r), p = __ldg(S.rowblk + r);
        if (!EXAGO_DCHECK(S, K >= 0 && K < S.nb && p >= 0 && p < S.nblk)) continue;
        double F[BS * BS], z[BS];
        load_blk<BS>(T, p, B, b, F);
#pragma unroll
        for (int i = 0; i < BS; i++) z[i] = __ldcg(x + ((size_t)K * BS + i) * B + b);
#pragma unroll
        for (int i = 0; i < BS; i++)
#pragma unroll
            for (int k = 0; k < BS; k++) y[i] = fma(-F[i * BS + k], z[k], y[i]);
    }
    double Di[BS * BS];
    load_blk<BS>(L, __ldg(S.colptr + J), B, b, Di);
#pragma unroll
    for (int i = 0; i < BS; i++) {
        double s = Di[i * BS] * y[0];
#pragma unroll
        for (int k = 1; k < BS; k++) s = fma(Di[i * BS + k], y[k], s);
        x[((size_t)J * BS + i) * B + b] = s;
    }
}

// Backward sweep of one level's columns: x_J = z_J - sum_{I in colstruct(J)} U_JI x_I
// (SYM: U_JI = L_IJ').
template <int BS, bool SYM>
__global__ void __launch_bounds__(kNT) k_bf_backward(const DevSymK S, int B, const double *L,
                                                     const double *U, double *x, int c0) {
    const int b = blockIdx.y * kNT + threadIdx.x;
    if (b >= B) return;
    const int J = __ldg(S.lvl_cols + c0 + blockIdx.x);
    double v[BS];
#pragma unroll
    for (int i = 0; i < BS; i++) v[i] = __ldcg(x + ((size_t)J * BS + i) * B + b);
    const int64_t p0 = __ldg(S.colptr + J), p1 = __ldg(S.colptr + J + 1);
    for (int64_t p = p0 + 1; p < p1; p++) {
        const int I = __ldg(S.rowidx + p);
        if (!EXAGO_DCHECK(S, I >= 0 && I < S.nb)) continue;
        double M[BS * BS], xi[BS];
        load_blk<BS>(SYM ? L : U, p, B, b, M);
#pragma unroll
        for (int i = 0; i < BS; i++) xi[i] = __ldcg(x + ((size_t)I * BS + i) * B + b);
#pragma unroll
        for (int i = 0; i < BS; i++)
#pragma unroll
            for (int k = 0; k < BS; k++)
                v[i] = fma(-(SYM ? M[k * BS + i] : M[i * BS + k]), xi[k], v[i]);
    }
#pragma unroll
    for (int i = 0; i < BS; i++) x[((size_t)J * BS + i) * B + b] = v[i];
}

}  // namespace

// A level is split when it has fewer than this many targets (factor) or columns (sweeps): a
// property of the structure, not of the batch.
constexpr int kSplitBelow = 64;

template <int BS, bool SYM>
int launch_block_factor(const DevSym &S, int B, double *T, double *TU, double *L, double *U,
                        int *neg, int *bad, double tiny, cudaStream_t st) {
    if (B <= 0) return 0;
    const unsigned gy = (unsigned)((B + kNT - 1) / kNT), gy32 = (unsigned)((B + 31) / 32);
    for (int l = 0; l < S.nlevels; l++) {
        const int t0 = S.lvl_tptr[l], nt = S.lvl_tptr[l + 1] - t0;
        if (nt <= 0) continue;
        const dim3 grid((unsigned)nt, gy);
        if (nt < kSplitBelow)
            k_bf_update_split<BS, SYM><<<dim3((unsigned)nt, gy32), 32 * kSlices, 0, st>>>(
                S.k, B, T, TU, L, U, t0);
        else
            k_bf_update<BS, SYM><<<grid, kNT, 0, st>>>(S.k, B, T, TU, L, U, t0);
        k_bf_scale<BS, SYM><<<grid, kNT, 0, st>>>(S.k, B, T, TU, L, U, neg, bad, tiny, t0);
    }
    return (int)cudaGetLastError();
}

template <int BS, bool SYM>
int launch_block_solve(const DevSym &S, int B, const double *T, const double *L, const double *U,
                       double *x, cudaStream_t st) {
    if (B <= 0) return 0;
    const unsigned gy = (unsigned)((B + kNT - 1) / kNT), gy32 = (unsigned)((B + 31) / 32);
    for (int l = 0; l < S.nlevels; l++) {
        const int c0 = S.lvl_colptr[l], nc = S.lvl_colptr[l + 1] - c0;
        if (nc <= 0) continue;
        if (nc < kSplitBelow)
            k_bf_forward_split<BS><<<dim3((unsigned)nc, gy32), 32 * kSweepSlices, 0, st>>>(
                S.k, B, T, L, x, c0);
        else
            k_bf_forward<BS><<<dim3((unsigned)nc, gy), kNT, 0, st>>>(S.k, B, T, L, x, c0);
    }
    for (int l = S.nlevels - 1; l >= 0; l--) {
        const int c0 = S.lvl_colptr[l], nc = S.lvl_colptr[l + 1] - c0;
        if (nc <= 0) continue;
        if (nc < kSplitBelow)
            k_bf_backward_split<BS, SYM><<<dim3((unsigned)nc, gy32), 32 * kSweepSlices, 0, st>>>(
                S.k, B, L, U, x, c0);
        else
            k_bf_backward<BS, SYM><<<dim3((unsigned)nc, gy), kNT, 0, st>>>(S.k, B, L, U, x, c0);
    }
    return (int)cudaGetLastError();
}

int upload_block_sym(const BlockSym &S, DevSym &D, std::vector<void *> &allocs) {
    D = DevSym();
    D.k.nb = S.nb;
    D.k.nlevels = D.nlevels = S.nlevels;
    D.k.nblk = S.nblk;
    D.k.ntgt = (int64_t)S.tgt_blk.size();
    D.k.npairs = (int64_t)S.pairs.size();
    D.lvl_colptr = S.lvl_colptr;
    D.lvl_tptr = S.lvl_tptr;
    auto up = [&](const void *src, size_t bytes, const void **dst) -> int {
        *dst = nullptr;
        if (bytes == 0) return 0;
        void *p = nullptr;
        cudaError_t e = dev_malloc(&p, bytes);
        if (e != cudaSuccess) return (int)e;
        allocs.push_back(p);
        e = cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice);
        *dst = p;
        return (int)e;
    };
    int e = 0;
#define UPV(field, vec) \
    if (!e) e = up(S.vec.data(), S.vec.size() * sizeof(S.vec[0]), (const void **)&D.k.field)
    UPV(colptr, colptr); UPV(rowidx, rowidx); UPV(rowptr, rowptr); UPV(rowblk, rowblk);
    UPV(rowcol, rowcol); UPV(lvl_cols, lvl_cols); UPV(tgt_blk, tgt_blk); UPV(tgt_diag, tgt_diag);
    UPV(tptr, tptr); UPV(pairs, pairs);
#undef UPV
    return e;
}

template int launch_block_factor<4, true>(const DevSym &, int, double *, double *, double *,
                                          double *, int *, int *, double, cudaStream_t);
template int launch_block_factor<2, false>(const DevSym &, int, double *, double *, double *,
                                           double *, int *, int *, double, cudaStream_t);
template int launch_block_solve<4, true>(const DevSym &, int, const double *, const double *,
                                         const double *, double *, cudaStream_t);
template int launch_block_solve<2, false>(const DevSym &, int, const double *, const double *,
                                          const double *, double *, cudaStream_t);

}  // namespace exago
