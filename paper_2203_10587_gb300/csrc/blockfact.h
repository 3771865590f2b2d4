// Batched sparse block factorisation on one fixed pattern: the linear algebra of an interior-point
// KKT step and of a power-flow Newton step, for a batch of independent states (SCOPFLOW
// contingencies with EMPAR, Sec. V-A; SOPFLOW scenarios, Sec. VI-A).  Internal to the library.
//
// The matrix is BS x BS blocks on the bus graph (block (u, v) is structurally nonzero when u = v
// or a branch joins u and v).  The host computes one symbolic factorisation for all states:
//   * a minimum-degree elimination order of the bus graph (ties to the lowest bus index);
//   * the block structure of the factor: column k (the k-th eliminated bus) holds its diagonal
//     block and the blocks of the rows in colstruct(k), the buses adjacent to k in the
//     elimination graph when k is eliminated (all later in the order);
//   * the elimination tree and its levels (level = 1 + the highest level of a child, leaves 0):
//     the columns of one level do not depend on each other;
//   * for every target block (I, J) with I in {J} + colstruct(J), the list of pairs
//     (position of (I, K), position of (J, K)) over the earlier columns K with both blocks
//     nonzero: the terms of its left-looking update.
// The device factors A = L D L' (SYM, symmetric: the KKT step) or A = L D U (the power flow),
// with unit block-triangular L, U and block-diagonal D, level by level:
//   T_IJ = A_IJ - sum_K F_IK U_KJ  with F_IK = L_IK D_K  (= the stored T_IK), U_KJ = L_JK' (SYM);
//   D_J = T_JJ;  L_IJ = T_IJ D_J^-1;  U_JI = D_J^-1 T'_JI (upper targets, LU only).
// Every value array is batch-interleaved: entry e of block p of state b is at [(p BS^2 + e) B + b],
// so the threads of a warp (consecutive states) read consecutive doubles.  No atomics on values.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace exago {

struct BlockSym {
    int nb = 0;                      // block rows / columns (buses)
    std::vector<int> perm, iperm;    // perm[k] = bus eliminated k-th; iperm[bus] = k
    // factor structure, column by column (elimination index space): blocks colptr[k] ..
    // colptr[k+1]-1, the first the diagonal, then the rows of colstruct(k) ascending
    std::vector<int64_t> colptr;
    std::vector<int> rowidx;         // [nblk] elimination index of each block's row
    int64_t nblk = 0;
    // row structure: for row i, the blocks (i, K), K < i, ascending K: rowptr[i] .. rowptr[i+1]-1
    std::vector<int64_t> rowptr;
    std::vector<int> rowblk;         // block position of (i, K)
    std::vector<int> rowcol;         // K
    std::vector<int> parent;         // elimination tree (elimination index), -1 at a root
    std::vector<int> level;          // level of each column
    int nlevels = 0;
    // columns by level: lvl_cols[lvl_colptr[l] .. lvl_colptr[l+1]) are level l's columns
    std::vector<int> lvl_colptr, lvl_cols;
    // targets = every block position, grouped by level of its column (lvl_tptr), each with its
    // update pairs pairs[tptr[t] .. tptr[t+1]) (two block positions each: (I, K) and (J, K))
    std::vector<int> lvl_tptr;       // [nlevels + 1] into targets
    std::vector<int> tgt_blk;        // block position of each target
    std::vector<int> tgt_diag;       // block position of the target column's diagonal
    std::vector<int64_t> tptr;       // [ntargets + 1]
    std::vector<int2> pairs;         // (position of (I, K), position of (J, K))
    // solve schedule: for each column, in the level order of lvl_cols
    double flops_factor_per_block = 0;   // sum over pairs of one block product (BS^3 FMA units)
};

// Builds the symbolic factorisation of the bus graph given as adjacency lists (adj_ptr [nb + 1],
// adj [..]; duplicates and self loops are ignored).  Returns false with a message on an
// inconsistent graph.
bool build_block_sym(int nb, const int *adj_ptr, const int *adj, BlockSym &S, std::string &err);

// Device tables of a symbolic factorisation (handed to the kernels by value).
struct DevSymK {
    int nb, nlevels;
    int64_t nblk, ntgt, npairs;
    const int64_t *colptr;   // [nb + 1]
    const int *rowidx;       // [nblk]
    const int64_t *rowptr;   // [nb + 1]
    const int *rowblk, *rowcol;
    const int *lvl_cols;     // [nb]
    const int *tgt_blk, *tgt_diag;
    const int64_t *tptr;
    const int2 *pairs;
    int *status;             // the owning net's device status word (debug-build index checks)
};

// The device tables and the host copies of the launch ranges.
struct DevSym {
    DevSymK k{};
    int nlevels = 0;
    std::vector<int> lvl_colptr, lvl_tptr;
};

// Uploads S (cudaMalloc through dev_malloc; the pointers go to `allocs` for the owner to free).
int upload_block_sym(const BlockSym &S, DevSym &D, std::vector<void *> &allocs);

// Batched numeric factorisation and solve on DevSym.  T: the assembled matrix A, lower blocks
// (and TU the upper blocks, the transposed positions, for LU), [nblk][BS*BS][B]; overwritten by
// F = L D (and U D).  L: [nblk][BS*BS][B] receives L (off-diagonal) and D^-1 (diagonal
// positions); U likewise for LU.  neg [B] counts the negative pivots of the diagonal blocks'
// in-block elimination (SYM), bad [B] the pivots with |d| below tiny * the block's largest entry.
template <int BS, bool SYM>
int launch_block_factor(const DevSym &S, int B, double *T, double *TU, double *L, double *U,
                        int *neg, int *bad, double tiny, cudaStream_t st);
// x [nb][BS][B] (elimination index order): on entry the right-hand side, on return the solution.
// T, L, U as the factorisation left them.
template <int BS, bool SYM>
int launch_block_solve(const DevSym &S, int B, const double *T, const double *L, const double *U,
                       double *x, cudaStream_t st);

}  // namespace exago
