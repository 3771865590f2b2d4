// Sanitizer test driver for the library's host code: for each grid file it runs the plan's
// validation and construction (plan.cpp) and, for valid grids, the symbolic analysis of the
// batched block factorisation (blockfact_sym.cpp), and checks the structures' invariants.  Built
// with -fsanitize=address,undefined by tests/test_host_sanitizers.py; exits nonzero on any
// failed check.
#include <cstdio>
#include <string>
#include <vector>

#include "../../paper_2203_10587_gb300/csrc/blockfact.h"
#include "../../paper_2203_10587_gb300/csrc/internal.h"
#include "grid_io.h"

using namespace exago;

#define CHECK(c) do { if (!(c)) { fprintf(stderr, "%s: check failed: %s\n", path, #c); return 1; } } while (0)

static int run(const char *path) {
    grid_file g{};
    read_grid(path, &g);
    HostPlan P;
    std::string err;
    const exago_status s = build_plan(P, g.nb, g.Gs, g.Bs, g.Pd, g.Qd, g.nl, g.f, g.t, g.r, g.x,
                                      g.b, g.tap, g.rateA, g.ng, g.gbus, g.c2, g.c1, g.c0,
                                      g.baseMVA, g.shift, err);
    if (g.expect != 0) {
        CHECK(s == EXAGO_EINVAL && !err.empty());
        free_grid(&g);
        return 0;
    }
    CHECK(s == EXAGO_OK);
    CHECK((int)P.Jrowptr.size() == P.m + 1 && P.Jrowptr[P.m] == P.nnzJ);
    for (int r = 0; r < P.m; r++)
        for (int64_t q = P.Jrowptr[r]; q < P.Jrowptr[r + 1]; q++) {
            CHECK(P.Jcol[q] >= 0 && P.Jcol[q] < P.n);
            if (q > P.Jrowptr[r]) CHECK(P.Jcol[q] > P.Jcol[q - 1]);
        }
    for (int r = 0; r < P.n; r++)
        for (int64_t q = P.Hrowptr[r]; q < P.Hrowptr[r + 1]; q++) CHECK(P.Hcol[q] >= 0 && P.Hcol[q] <= r);
    CHECK(P.slot_ptr[P.nb] == P.nslot);
    // symbolic analysis of the bus graph
    std::vector<int> aptr(P.nb + 1, 0), adj;
    for (int l = 0; l < P.nl; l++) aptr[P.f[l] + 1]++;
    for (int i = 0; i < P.nb; i++) aptr[i + 1] += aptr[i];
    adj.resize(aptr[P.nb]);
    std::vector<int> fill(aptr.begin(), aptr.end() - 1);
    for (int l = 0; l < P.nl; l++) adj[fill[P.f[l]]++] = P.t[l];
    BlockSym S;
    CHECK(build_block_sym(P.nb, aptr.data(), adj.data(), S, err));
    std::vector<int> seen(P.nb, 0);
    for (int v : S.perm) { CHECK(v >= 0 && v < P.nb); seen[v]++; }
    for (int c : seen) CHECK(c == 1);
    for (int k = 0; k < P.nb; k++) {
        CHECK(S.colptr[k + 1] > S.colptr[k] && S.rowidx[S.colptr[k]] == k);
        for (int64_t p = S.colptr[k] + 1; p < S.colptr[k + 1]; p++) CHECK(S.rowidx[p] > S.rowidx[p - 1]);
    }
    for (size_t t = 0; t + 1 < S.tptr.size(); t++) CHECK(S.tptr[t + 1] >= S.tptr[t]);
    for (const int2 &pr : S.pairs) CHECK(pr.x >= 0 && pr.x < S.nblk && pr.y >= 0 && pr.y < S.nblk);
    printf("%s: nb %d nnzJ %lld blocks %lld pairs %zu levels %d\n", path, P.nb,
           (long long)P.nnzJ, (long long)S.nblk, S.pairs.size(), S.nlevels);
    free_grid(&g);
    return 0;
}

int main(int argc, char **argv) {
    for (int i = 1; i < argc; i++)
        if (run(argv[i])) return 1;
    return 0;
}
