// Host planning of one grid: validation, the Jacobian and Lagrangian-Hessian sparsity patterns
// of the polar AC-OPF model (ExaGO, Sec. III, eqs. (7)-(10)), and the output position of every
// value the kernels write.  Runs once per grid; nothing here is on the per-iteration path.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <utility>

#include "internal.h"

namespace exago {

namespace {

bool finite_all(const double *a, int n) {
    for (int i = 0; i < n; i++)
        if (!std::isfinite(a[i])) return false;
    return true;
}

std::vector<double> copy_or(const double *a, int n, double dflt) {
    std::vector<double> v(n, dflt);
    if (a)
        for (int i = 0; i < n; i++) v[i] = a[i];
    return v;
}

}  // namespace

size_t workspace_bytes(const HostPlan &p, int B) {
    return ((size_t)B * (size_t)p.nslot * NCOMP * sizeof(double) + 255) / 256 * 256;
}

exago_status build_plan(HostPlan &p, int nb, const double *Gs, const double *Bs, const double *Pd,
                        const double *Qd, int nl, const int *f, const int *t, const double *r,
                        const double *x, const double *b, const double *tap,
                        const double *rateA, int ng, const int *gbus, const double *c2,
                        const double *c1, const double *c0, double baseMVA,
                        const double *shift, std::string &err) {
    char msg[256];
    if (nb < 1 || nl < 0 || ng < 0) {
        err = "need nb >= 1, nl >= 0, ng >= 0";
        return EXAGO_EINVAL;
    }
    if (nl > 0 && (!f || !t || !r || !x || !b)) {
        err = "branch arrays f, t, r, x, b must be non-null when nl > 0";
        return EXAGO_EINVAL;
    }
    if (ng > 0 && (!gbus || !c2 || !c1)) {
        err = "generator arrays gbus, c2, c1 must be non-null when ng > 0";
        return EXAGO_EINVAL;
    }
    if (!(baseMVA > 0.0) || !std::isfinite(baseMVA)) {
        err = "baseMVA must be positive and finite";
        return EXAGO_EINVAL;
    }
    p = HostPlan();
    p.nb = nb; p.nl = nl; p.ng = ng;
    p.n = 2 * nb + 2 * ng;
    p.m = 2 * nb + 2 * nl;
    p.baseMVA = baseMVA;
    p.Gs = copy_or(Gs, nb, 0.0); p.Bs = copy_or(Bs, nb, 0.0);
    p.Pd = copy_or(Pd, nb, 0.0); p.Qd = copy_or(Qd, nb, 0.0);
    p.r = copy_or(r, nl, 0.0); p.x = copy_or(x, nl, 0.0); p.b = copy_or(b, nl, 0.0);
    p.tap = copy_or(tap, nl, 0.0); p.rateA = copy_or(rateA, nl, 0.0);
    p.c2 = copy_or(c2, ng, 0.0); p.c1 = copy_or(c1, ng, 0.0); p.c0 = copy_or(c0, ng, 0.0);
    // cost derivatives per p.u. of Pg: d/dPg of c2 (base Pg)^2 + c1 base Pg
    p.c2g.resize(ng);
    p.c1g.resize(ng);
    for (int k = 0; k < ng; k++) {
        p.c2g[k] = 2.0 * p.c2[k] * baseMVA * baseMVA;
        p.c1g[k] = p.c1[k] * baseMVA;
    }
    p.f.assign(f ? f : nullptr, f ? f + nl : nullptr);
    p.t.assign(t ? t : nullptr, t ? t + nl : nullptr);
    p.gbus.assign(gbus ? gbus : nullptr, gbus ? gbus + ng : nullptr);

    for (auto *v : {&p.Gs, &p.Bs, &p.Pd, &p.Qd})
        if (!finite_all(v->data(), nb)) { err = "non-finite bus data"; return EXAGO_EINVAL; }
    for (auto *v : {&p.r, &p.x, &p.b, &p.tap, &p.rateA})
        if (!finite_all(v->data(), nl)) { err = "non-finite branch data"; return EXAGO_EINVAL; }
    if (shift && nl > 0) {
        p.shift.assign(shift, shift + nl);
        if (!finite_all(p.shift.data(), nl)) { err = "non-finite phase shift"; return EXAGO_EINVAL; }
    }
    for (auto *v : {&p.c2, &p.c1, &p.c0})
        if (!finite_all(v->data(), ng)) { err = "non-finite generator data"; return EXAGO_EINVAL; }
    for (int l = 0; l < nl; l++) {
        if (p.f[l] < 0 || p.f[l] >= nb || p.t[l] < 0 || p.t[l] >= nb) {
            snprintf(msg, sizeof msg, "branch %d: bus index out of range (f=%d, t=%d, nb=%d)", l, p.f[l], p.t[l], nb);
            err = msg;
            return EXAGO_EINVAL;
        }
        if (p.f[l] == p.t[l]) {
            snprintf(msg, sizeof msg, "branch %d: from and to bus are both %d", l, p.f[l]);
            err = msg;
            return EXAGO_EINVAL;
        }
        if (p.r[l] == 0.0 && p.x[l] == 0.0) {
            snprintf(msg, sizeof msg, "branch %d: zero series impedance (r = x = 0)", l);
            err = msg;
            return EXAGO_EINVAL;
        }
        if (p.tap[l] < 0.0) {
            snprintf(msg, sizeof msg, "branch %d: negative tap ratio", l);
            err = msg;
            return EXAGO_EINVAL;
        }
    }
    for (int k = 0; k < ng; k++)
        if (p.gbus[k] < 0 || p.gbus[k] >= nb) {
            snprintf(msg, sizeof msg, "generator %d: bus index %d out of range", k, p.gbus[k]);
            err = msg;
            return EXAGO_EINVAL;
        }

    // adjacency: sorted distinct neighbours; cols_i = nbr(i) + {i}, sorted
    std::vector<std::vector<int>> nbr(nb), cols(nb);
    for (int l = 0; l < nl; l++) {
        nbr[p.f[l]].push_back(p.t[l]);
        nbr[p.t[l]].push_back(p.f[l]);
    }
    for (int i = 0; i < nb; i++) {
        auto &v = nbr[i];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        cols[i] = v;
        cols[i].insert(std::lower_bound(cols[i].begin(), cols[i].end(), i), i);
    }
    auto rank = [&](int i, int j) {  // position of bus j among cols_i
        return (int)(std::lower_bound(cols[i].begin(), cols[i].end(), j) - cols[i].begin());
    };
    auto lowrank = [&](int i, int j) {  // position of j among the neighbours of i below i
        return (int)(std::lower_bound(nbr[i].begin(), nbr[i].end(), j) - nbr[i].begin());
    };

    // generators by bus
    p.gen_ptr.assign(nb + 1, 0);
    for (int k = 0; k < ng; k++) p.gen_ptr[p.gbus[k] + 1]++;
    for (int i = 0; i < nb; i++) p.gen_ptr[i + 1] += p.gen_ptr[i];
    p.gen_ord.assign(ng, 0);
    {
        std::vector<int> fill(p.gen_ptr.begin(), p.gen_ptr.end() - 1);
        for (int k = 0; k < ng; k++) p.gen_ord[fill[p.gbus[k]]++] = k;  // ascending id within a bus
    }

    // ---- Jacobian pattern: P rows, Q rows (eq. (8)), then from / to flow rows (eq. (9))
    const int mrows = p.m;
    p.Jrowptr.assign(mrows + 1, 0);
    for (int i = 0; i < nb; i++) {
        int len = 2 * (int)cols[i].size() + (p.gen_ptr[i + 1] - p.gen_ptr[i]);
        p.Jrowptr[i + 1] = len;
        p.Jrowptr[nb + i + 1] = len;
    }
    for (int r2 = 0; r2 < 2 * nl; r2++) p.Jrowptr[2 * nb + r2 + 1] = 4;
    for (int i = 0; i < mrows; i++) p.Jrowptr[i + 1] += p.Jrowptr[i];
    p.nnzJ = p.Jrowptr[mrows];
    p.nnzJg = p.Jrowptr[2 * nb];
    if (p.nnzJ >= INT32_MAX) { err = "Jacobian too large for 32-bit positions"; return EXAGO_EINVAL; }
    p.Jcol.assign(p.nnzJ, 0);
    for (int i = 0; i < nb; i++) {
        for (int rowblk = 0; rowblk < 2; rowblk++) {
            int64_t q = p.Jrowptr[rowblk * nb + i];
            for (int j : cols[i]) p.Jcol[q++] = j;
            for (int j : cols[i]) p.Jcol[q++] = nb + j;
            for (int s = p.gen_ptr[i]; s < p.gen_ptr[i + 1]; s++)
                p.Jcol[q++] = 2 * nb + rowblk * ng + p.gen_ord[s];
        }
    }
    for (int l = 0; l < nl; l++) {
        int lo = std::min(p.f[l], p.t[l]), hi = std::max(p.f[l], p.t[l]);
        for (int side = 0; side < 2; side++) {
            int64_t q = p.Jrowptr[2 * nb + side * nl + l];
            p.Jcol[q + 0] = lo;
            p.Jcol[q + 1] = hi;
            p.Jcol[q + 2] = nb + lo;
            p.Jcol[q + 3] = nb + hi;
        }
    }

    // ---- lower-triangle Lagrangian Hessian pattern
    p.Hrowptr.assign(p.n + 1, 0);
    for (int i = 0; i < nb; i++) {
        int nlow = lowrank(i, i);  // neighbours below i
        p.Hrowptr[i + 1] = nlow + 1;
        p.Hrowptr[nb + i + 1] = (int)cols[i].size() + nlow + 1;
    }
    for (int k = 0; k < ng; k++) p.Hrowptr[2 * nb + k + 1] = 1;
    for (int i = 0; i < p.n; i++) p.Hrowptr[i + 1] += p.Hrowptr[i];
    p.nnzH = p.Hrowptr[p.n];
    if (p.nnzH >= INT32_MAX) { err = "Hessian too large for 32-bit positions"; return EXAGO_EINVAL; }
    p.Hcol.assign(p.nnzH, 0);
    for (int i = 0; i < nb; i++) {
        int64_t q = p.Hrowptr[i];
        for (int j : nbr[i]) if (j < i) p.Hcol[q++] = j;
        p.Hcol[q++] = i;
        q = p.Hrowptr[nb + i];
        for (int j : cols[i]) p.Hcol[q++] = j;
        for (int j : nbr[i]) if (j < i) p.Hcol[q++] = nb + j;
        p.Hcol[q++] = nb + i;
    }
    for (int k = 0; k < ng; k++) p.Hcol[p.Hrowptr[2 * nb + k]] = 2 * nb + k;

    // ---- per-bus row starts
    p.bus_jP.assign(nb, 0); p.bus_jQ.assign(nb, 0); p.bus_hA.assign(nb, 0); p.bus_hM.assign(nb, 0);
    p.bus_k.assign(nb, 0); p.bus_nlow.assign(nb, 0);
    for (int i = 0; i < nb; i++) {
        p.bus_jP[i] = (int)p.Jrowptr[i];
        p.bus_jQ[i] = (int)p.Jrowptr[nb + i];
        p.bus_hA[i] = (int)p.Hrowptr[i];
        p.bus_hM[i] = (int)p.Hrowptr[nb + i];
        p.bus_k[i] = (int)cols[i].size();
        p.bus_nlow[i] = rank(i, i);
    }

    // ---- degree-sorted bus order inside every aligned bus tile of 32, 64, 128 and 256 buses
    // (degree = branch ends at the bus, the trip count of its slot loop), so that each warp of a
    // tile holds buses of similar degree
    std::vector<int> ends_at(nb, 0);
    for (int l = 0; l < nl; l++) { ends_at[p.f[l]]++; ends_at[p.t[l]]++; }
    p.bus_perm.resize(4 * (size_t)nb);
    for (int t = 0; t < 4; t++) {
        const int T = 32 << t;
        auto perm = p.bus_perm.begin() + (size_t)t * nb;
        for (int i = 0; i < nb; i++) perm[i] = i;
        for (int g0 = 0; g0 < nb; g0 += T) {
            const int g1 = g0 + T < nb ? g0 + T : nb;
            std::stable_sort(perm + g0, perm + g1,
                             [&](int a, int c) { return ends_at[a] > ends_at[c]; });
        }
    }

    // ---- slots: (bus, other bus, branch); each bus's slots walk its row columns in order
    p.nslot = 2 * nl;
    p.slot_ptr.assign(nb + 1, 0);
    for (int l = 0; l < nl; l++) { p.slot_ptr[p.f[l] + 1]++; p.slot_ptr[p.t[l] + 1]++; }
    for (int i = 0; i < nb; i++) p.slot_ptr[i + 1] += p.slot_ptr[i];
    std::vector<std::pair<int, int>> ends;   // (other bus, 2 * branch + end) of one bus
    std::vector<std::vector<std::pair<int, int>>> at(nb);
    for (int l = 0; l < nl; l++) {
        at[p.f[l]].push_back({p.t[l], 2 * l});
        at[p.t[l]].push_back({p.f[l], 2 * l + 1});
    }
    p.slot_nbr.assign(p.nslot, 0);
    p.slot_ref.assign(p.nslot, 0);
    p.br_slot.assign(2 * (size_t)nl, 0);
    for (int i = 0; i < nb; i++) {
        std::sort(at[i].begin(), at[i].end());
        int s2 = p.slot_ptr[i];
        for (auto &e : at[i]) {
            p.slot_nbr[s2] = e.first;
            p.slot_ref[s2] = e.second;   // 2 l + end
            p.br_slot[(size_t)(e.second & 1) * nl + (e.second >> 1)] = s2;
            s2++;
        }
    }
    // slot -> bus, and the column of the slot's neighbour among the bus's row columns (the
    // diagonal sits after the nlow lower neighbours); -1 for a later branch of a parallel group,
    // whose values the group's first slot sums
    p.slot_bus.assign(p.nslot, 0);
    p.slot_pos.assign(p.nslot, -1);
    for (int i = 0; i < nb; i++) {
        int pos = 0;
        for (int s = p.slot_ptr[i]; s < p.slot_ptr[i + 1]; s++) {
            p.slot_bus[s] = i;
            if (s > p.slot_ptr[i] && p.slot_nbr[s] == p.slot_nbr[s - 1]) continue;
            if (pos == p.bus_nlow[i]) pos++;
            p.slot_pos[s] = pos++;
        }
    }
    return EXAGO_OK;
}

}  // namespace exago
