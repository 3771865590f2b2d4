// Host symbolic factorisation of the bus graph for the batched block factorisation (blockfact.h).
//
// Ordering: minimum degree on the elimination graph.  Repeatedly the uneliminated bus of least
// current degree (lowest index on ties) is eliminated and its neighbours become a clique; the
// neighbour set at elimination is the block structure of its factor column.  The graphs here are
// sparse (degree <= 8 before fill), so plain sorted adjacency vectors merged on each elimination
// are enough.  Plain host code (no CUDA calls): the host tests build it with the address and
// undefined-behaviour sanitizers.
#include <algorithm>
#include <cstdio>
#include <set>

#include "blockfact.h"

namespace exago {

namespace {

// out = (a U b) \ {x, y}, a and b sorted ascending without duplicates.
void merge_without(const std::vector<int> &a, const std::vector<int> &b, int x, int y,
                   std::vector<int> &out) {
    out.clear();
    out.reserve(a.size() + b.size());
    size_t i = 0, j = 0;
    while (i < a.size() || j < b.size()) {
        int v;
        if (j >= b.size() || (i < a.size() && a[i] < b[j])) v = a[i++];
        else if (i >= a.size() || b[j] < a[i]) v = b[j++];
        else { v = a[i]; i++; j++; }
        if (v != x && v != y) out.push_back(v);
    }
}

}  // namespace

bool build_block_sym(int nb, const int *adj_ptr, const int *adj, BlockSym &S, std::string &err) {
    S = BlockSym();
    if (nb < 1) { err = "empty graph"; return false; }
    S.nb = nb;
    std::vector<std::vector<int>> g(nb);
    for (int v = 0; v < nb; v++) {
        for (int q = adj_ptr[v]; q < adj_ptr[v + 1]; q++) {
            const int u = adj[q];
            if (u < 0 || u >= nb) { err = "adjacency index out of range"; return false; }
            if (u != v) { g[v].push_back(u); g[u].push_back(v); }
        }
    }
    for (auto &a : g) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    // minimum degree, lowest index on ties
    std::set<std::pair<int, int>> queue;
    for (int v = 0; v < nb; v++) queue.insert({(int)g[v].size(), v});
    std::vector<std::vector<int>> colbus(nb);   // neighbour buses of the k-th eliminated bus
    S.perm.resize(nb);
    S.iperm.assign(nb, -1);
    std::vector<int> tmp;
    for (int k = 0; k < nb; k++) {
        const int v = queue.begin()->second;
        queue.erase(queue.begin());
        S.perm[k] = v;
        S.iperm[v] = k;
        const std::vector<int> N = g[v];
        for (int u : N) {
            queue.erase({(int)g[u].size(), u});
            merge_without(g[u], N, u, v, tmp);
            g[u].swap(tmp);
            queue.insert({(int)g[u].size(), u});
        }
        colbus[k] = N;
        g[v].clear();
        g[v].shrink_to_fit();
    }
    // factor structure in elimination index space
    S.colptr.assign(nb + 1, 0);
    for (int k = 0; k < nb; k++) S.colptr[k + 1] = S.colptr[k] + 1 + (int64_t)colbus[k].size();
    S.nblk = S.colptr[nb];
    if (S.nblk > 0x7fffffff) { err = "factor too large"; return false; }
    S.rowidx.resize(S.nblk);
    std::vector<int64_t> rowcount(nb + 1, 0);
    for (int k = 0; k < nb; k++) {
        std::vector<int> rows;
        rows.reserve(colbus[k].size());
        for (int u : colbus[k]) rows.push_back(S.iperm[u]);
        std::sort(rows.begin(), rows.end());
        int64_t p = S.colptr[k];
        S.rowidx[p++] = k;
        for (int i : rows) {
            if (i <= k) { err = "elimination order inconsistent"; return false; }
            S.rowidx[p++] = i;
            rowcount[i + 1]++;
        }
        colbus[k].clear();
        colbus[k].shrink_to_fit();
    }
    // row structure (ascending K within each row: columns are visited in order)
    S.rowptr.assign(nb + 1, 0);
    for (int i = 0; i < nb; i++) S.rowptr[i + 1] = S.rowptr[i] + rowcount[i + 1];
    S.rowblk.resize(S.rowptr[nb]);
    S.rowcol.resize(S.rowptr[nb]);
    {
        std::vector<int64_t> fill(S.rowptr.begin(), S.rowptr.end() - 1);
        for (int k = 0; k < nb; k++)
            for (int64_t p = S.colptr[k] + 1; p < S.colptr[k + 1]; p++) {
                const int i = S.rowidx[p];
                S.rowblk[fill[i]] = (int)p;
                S.rowcol[fill[i]] = k;
                fill[i]++;
            }
    }
    // elimination tree and levels (a child precedes its parent in the order)
    S.parent.assign(nb, -1);
    S.level.assign(nb, 0);
    for (int k = 0; k < nb; k++) {
        if (S.colptr[k + 1] - S.colptr[k] > 1) S.parent[k] = S.rowidx[S.colptr[k] + 1];
        const int p = S.parent[k];
        if (p >= 0 && S.level[p] < S.level[k] + 1) S.level[p] = S.level[k] + 1;
    }
    S.nlevels = 0;
    for (int k = 0; k < nb; k++) S.nlevels = std::max(S.nlevels, S.level[k] + 1);
    S.lvl_colptr.assign(S.nlevels + 1, 0);
    for (int k = 0; k < nb; k++) S.lvl_colptr[S.level[k] + 1]++;
    for (int l = 0; l < S.nlevels; l++) S.lvl_colptr[l + 1] += S.lvl_colptr[l];
    S.lvl_cols.resize(nb);
    {
        std::vector<int> fill(S.lvl_colptr.begin(), S.lvl_colptr.end() - 1);
        for (int k = 0; k < nb; k++) S.lvl_cols[fill[S.level[k]]++] = k;
    }
    // targets (every block), grouped by level, and their update pairs (two passes: count, fill)
    S.lvl_tptr.assign(S.nlevels + 1, 0);
    S.tgt_blk.clear();
    S.tgt_diag.clear();
    S.tgt_blk.reserve(S.nblk);
    S.tgt_diag.reserve(S.nblk);
    for (int l = 0; l < S.nlevels; l++) {
        for (int c = S.lvl_colptr[l]; c < S.lvl_colptr[l + 1]; c++) {
            const int J = S.lvl_cols[c];
            for (int64_t p = S.colptr[J]; p < S.colptr[J + 1]; p++) {
                S.tgt_blk.push_back((int)p);
                S.tgt_diag.push_back((int)S.colptr[J]);
            }
        }
        S.lvl_tptr[l + 1] = (int)S.tgt_blk.size();
    }
    const int64_t ntgt = (int64_t)S.tgt_blk.size();
    std::vector<int> tgt_of_blk(S.nblk);
    for (int64_t t = 0; t < ntgt; t++) tgt_of_blk[S.tgt_blk[t]] = (int)t;
    std::vector<int64_t> count(ntgt + 1, 0);
    std::vector<int64_t> pos_of_row(nb, -1);
    auto for_pairs = [&](auto &&emit) {
        for (int J = 0; J < nb; J++) {
            for (int64_t p = S.colptr[J]; p < S.colptr[J + 1]; p++) pos_of_row[S.rowidx[p]] = p;
            for (int64_t r = S.rowptr[J]; r < S.rowptr[J + 1]; r++) {
                const int K = S.rowcol[r];
                const int pJK = S.rowblk[r];
                // blocks (I, K) of column K with I >= J: from (J, K) on
                for (int64_t q = pJK; q < S.colptr[K + 1]; q++) {
                    const int64_t pIJ = pos_of_row[S.rowidx[q]];
                    if (pIJ < 0) return false;   // would be a fill the structure lacks
                    emit(tgt_of_blk[pIJ], (int)q, pJK);
                }
            }
            for (int64_t p = S.colptr[J]; p < S.colptr[J + 1]; p++) pos_of_row[S.rowidx[p]] = -1;
        }
        return true;
    };
    if (!for_pairs([&](int64_t t, int, int) { count[t + 1]++; })) {
        err = "symbolic factorisation missed a fill block";
        return false;
    }
    S.tptr.assign(ntgt + 1, 0);
    for (int64_t t = 0; t < ntgt; t++) S.tptr[t + 1] = S.tptr[t] + count[t + 1];
    S.pairs.resize(S.tptr[ntgt]);
    {
        std::vector<int64_t> fill(S.tptr.begin(), S.tptr.end() - 1);
        for_pairs([&](int64_t t, int q, int pJK) {
            S.pairs[fill[t]++] = make_int2(q, pJK);
        });
    }
    S.flops_factor_per_block = (double)S.pairs.size();
    return true;
}

}  // namespace exago
