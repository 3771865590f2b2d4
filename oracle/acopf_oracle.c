/*
 * Plain FP64 CPU oracle for the polar AC optimal power flow model evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the benchmark's CPU
 * baseline may load this file's library.  It shares no code, header, table or helper with the
 * CUDA evaluator; the two meet only in the seeded input generator.
 *
 * What it computes (ExaGO, arXiv 2203.10587, Sec. III, eqs. (7)-(10)): for one state x of the
 * compact model  min f(x)  s.t.  g(x) = 0,  h- <= h(x) <= h+,  x- <= x <= x+  it returns
 *   f(x), grad f(x), g(x) | h(x), the values of the Jacobian of [g; h], and the values of the
 *   lower triangle of the Lagrangian Hessian  sigma*grad^2 f + sum_i lam_i grad^2 g_i
 *   + sum_l mu_l grad^2 h_l.
 * The paper leaves the formulation to its references (Sec. III: the full formulation is omitted
 * for space); the model is the "power-balance-polar" one it names, written here as the textbook
 * pi-model in polar coordinates:
 *   variables      x = [Va (nb) | Vm (nb) | Pg (ng) | Qg (ng)]
 *   equalities     g = [P balance (nb) | Q balance (nb)]
 *   inequalities   h = [|S_from|^2 (nl) | |S_to|^2 (nl)]   (squared apparent power)
 *   multipliers    lam = [lamP (nb) | lamQ (nb) | muF (nl) | muT (nl)]
 * Contingencies (Sec. V-A, eqs. (16)-(20)) enter as a per-branch in-service mask: an out-of-service
 * branch contributes zero to every output, and its two h rows evaluate to zero.  Load scenarios
 * (Sec. VI-A, eqs. (27)-(31)) enter as a per-bus load scale, and the scenario weight pi_s as a
 * factor on the objective.
 *
 * The power-balance-cartesian formulation, which Sec. III names beside the polar one, is
 * oracle_eval_cart (voltages e + j f, voltage-magnitude rows e^2 + f^2); it shares the branch-end
 * rows (end_rows) and generator terms (gen_terms) with the polar evaluation.
 * The coupling (ramp) rows that tie the states of the multi-period, security-constrained and
 * stochastic problems together (Sec. I, eqs. (5)-(6); eqs. (15), (20), (31)) are at the end of
 * this file: oracle_coupling and its transpose product oracle_coupling_jtv.
 * Everything is evaluated directly, in plain loops, in the order: branches by ascending index
 * (from side, then to side), then bus shunts and loads, then generators.  Derivatives are the
 * chain rule through the branch angle theta = Va_u - Va_v, written out per side.  J and the
 * Hessian are produced as coordinate triplets (every structural dependency is emitted, even when
 * its value is zero) and summed into sorted CSR by oracle_coo_to_csr.
 * Compile with -ffp-contract=off so that every product and sum is rounded on its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nb, nl, ng;
    const double *Gs, *Bs, *Pd, *Qd;     /* per bus, p.u. */
    const int *f, *t;                    /* per branch, bus indices */
    const double *r, *x, *b, *tap;       /* per branch, p.u.; tap 0 means 1 */
    const int *gbus;                     /* per generator */
    const double *c2, *c1, *c0;          /* cost in MW terms: c2*MW^2 + c1*MW + c0 */
    double baseMVA;
    const double *shift;                 /* per branch, rad: phase shift of the from-side tap
                                            (phase-shifting transformer); NULL = all 0 */
} oracle_net;

typedef struct {
    int64_t n;        /* triplets written */
    int64_t cap;      /* capacity of the arrays */
    int *row, *col;
    double *val;
} oracle_coo;

/* ---- pi-model two-port of one branch (textbook; MATPOWER's branch model) ----
 * series admittance ys = 1/(r + j x) = gs + j bs, line charging b split half per end, and on the
 * from side an ideal transformer of complex ratio T = tau e^{j phi}: off-nominal tap tau and phase
 * shift phi (rad; a phase-shifting transformer).  The from-side series terminal sees V_f / T and
 * the from current is the series current divided by conj(T), so
 *   Y = [[(ys + j b/2)/tau^2, -ys/conj(T)], [-ys/T, ys + j b/2]],
 * -ys/conj(T) = -ys e^{j phi}/tau and -ys/T = -ys e^{-j phi}/tau.  The two mutual admittances
 * differ unless phi = 0.
 * Out: Y[0..7] = Gff, Bff, Gft, Bft, Gtf, Btf, Gtt, Btt.  Returns 0, or -1 if r = x = 0. */
int oracle_pi_model_shift(double r, double x, double b, double tap, double phi, double *Y)
{
    double z2 = r * r + x * x;
    double tau = (tap == 0.0) ? 1.0 : tap;
    double gs, bs, cp, sp;
    if (z2 == 0.0) return -1;
    gs = r / z2;
    bs = -x / z2;
    cp = cos(phi);
    sp = sin(phi);
    Y[0] = gs / (tau * tau);
    Y[1] = (bs + 0.5 * b) / (tau * tau);
    /* -(gs + j bs)(cp + j sp) / tau */
    Y[2] = -(gs * cp - bs * sp) / tau;
    Y[3] = -(gs * sp + bs * cp) / tau;
    /* -(gs + j bs)(cp - j sp) / tau */
    Y[4] = -(gs * cp + bs * sp) / tau;
    Y[5] = -(bs * cp - gs * sp) / tau;
    Y[6] = gs;
    Y[7] = bs + 0.5 * b;
    return 0;
}

/* The same without phase shift (phi = 0). */
int oracle_pi_model(double r, double x, double b, double tap, double *Y)
{
    return oracle_pi_model_shift(r, x, b, tap, 0.0, Y);
}

static double branch_shift(const oracle_net *net, int l)
{
    return net->shift ? net->shift[l] : 0.0;
}

/* ---- one end of a branch, seen from its own bus u towards the other bus v ----
 *   P = Gss Vu^2 + Vu Vv (Gm cos th + Bm sin th)
 *   Q = -Bss Vu^2 + Vu Vv (Gm sin th - Bm cos th),      th = Va_u - Va_v
 * Local variable order (Va_u, Va_v, Vu, Vv).  dP[4], dQ[4] are gradients, HP[16], HQ[16] the full
 * symmetric Hessians (row-major 4x4).  The angle enters only through th, with d th / d Va_u = 1
 * and d th / d Va_v = -1, so every angle derivative is a th-derivative times those signs. */
static void side_terms(double Gss, double Bss, double Gm, double Bm,
                       double Vau, double Vav, double Vu, double Vv,
                       double *P, double *Q, double *dP, double *dQ, double *HP, double *HQ)
{
    const double e[2] = {1.0, -1.0};          /* d th / d (Va_u, Va_v) */
    double th = Vau - Vav;
    double cs = cos(th), sn = sin(th);
    double a = Gm * cs + Bm * sn;             /* d a / d th = -c */
    double c = Gm * sn - Bm * cs;             /* d c / d th =  a */
    double VV = Vu * Vv;
    int i, j;

    *P = Gss * Vu * Vu + VV * a;
    *Q = -Bss * Vu * Vu + VV * c;

    /* gradients */
    for (i = 0; i < 2; i++) {
        dP[i] = VV * (-c) * e[i];
        dQ[i] = VV * a * e[i];
    }
    dP[2] = 2.0 * Gss * Vu + Vv * a;
    dP[3] = Vu * a;
    dQ[2] = -2.0 * Bss * Vu + Vv * c;
    dQ[3] = Vu * c;

    /* Hessians */
    for (i = 0; i < 2; i++) {
        for (j = 0; j < 2; j++) {
            HP[i * 4 + j] = VV * (-a) * e[i] * e[j];   /* d2 a / d th2 = -a */
            HQ[i * 4 + j] = VV * (-c) * e[i] * e[j];   /* d2 c / d th2 = -c */
        }
        /* mixed angle / magnitude: d/dVu and d/dVv of the angle gradient */
        HP[i * 4 + 2] = HP[2 * 4 + i] = Vv * (-c) * e[i];
        HP[i * 4 + 3] = HP[3 * 4 + i] = Vu * (-c) * e[i];
        HQ[i * 4 + 2] = HQ[2 * 4 + i] = Vv * a * e[i];
        HQ[i * 4 + 3] = HQ[3 * 4 + i] = Vu * a * e[i];
    }
    HP[2 * 4 + 2] = 2.0 * Gss;
    HP[2 * 4 + 3] = HP[3 * 4 + 2] = a;
    HP[3 * 4 + 3] = 0.0;
    HQ[2 * 4 + 2] = -2.0 * Bss;
    HQ[2 * 4 + 3] = HQ[3 * 4 + 2] = c;
    HQ[3 * 4 + 3] = 0.0;
}

static int push(oracle_coo *c, int row, int col, double v)
{
    if (c->n >= c->cap) return -1;
    c->row[c->n] = row;
    c->col[c->n] = col;
    c->val[c->n] = v;
    c->n++;
    return 0;
}

/* Lower-triangle triplet (row >= col) of a symmetric entry. */
static int push_sym(oracle_coo *c, int gi, int gj, double v)
{
    return gi >= gj ? push(c, gi, gj, v) : push(c, gj, gi, v);
}

/* One branch end's rows, shared by both formulations: the end's injection into its bus's balances,
 * its h value |S|^2, its Jacobian entries (P, Q and h rows over the end's four variables gidx)
 * and its Lagrangian-Hessian block  lamP_u grad^2 P + lamQ_u grad^2 Q + mu grad^2 (P^2 + Q^2),
 * with grad^2 (P^2 + Q^2) = 2 (dP dP' + P HP + dQ dQ' + Q HQ).  m (0 or 1) is the branch's
 * in-service flag and multiplies every term.  Returns 0 or -2 when a triplet array is full. */
static int end_rows(int nb, int u, int hrow, double m, double lamPu, double lamQu, double mu,
                    double P0, double Q0, const double *dP0, const double *dQ0,
                    const double *HP0, const double *HQ0, const int *gidx,
                    double *gP, double *gQ, double *hval, oracle_coo *J, oracle_coo *H)
{
    double P = P0, Q = Q0, dP[4], dQ[4], HP[16], HQ[16], Hs[16];
    int a, bb;
    for (a = 0; a < 4; a++) { dP[a] = dP0[a]; dQ[a] = dQ0[a]; }
    for (a = 0; a < 16; a++) { HP[a] = HP0[a]; HQ[a] = HQ0[a]; }
    P *= m;
    Q *= m;
    for (a = 0; a < 4; a++) { dP[a] *= m; dQ[a] *= m; }
    for (a = 0; a < 16; a++) { HP[a] *= m; HQ[a] *= m; }

    /* g: this end's injection enters the balance of its own bus u */
    gP[u] += P;
    gQ[u] += Q;
    /* h: squared apparent power at this end */
    *hval = P * P + Q * Q;

    if (J) {
        for (a = 0; a < 4; a++) {
            if (push(J, u, gidx[a], dP[a])) return -2;
            if (push(J, nb + u, gidx[a], dQ[a])) return -2;
        }
        for (a = 0; a < 4; a++) /* grad |S|^2 = 2 P grad P + 2 Q grad Q */
            if (push(J, hrow, gidx[a], 2.0 * P * dP[a] + 2.0 * Q * dQ[a])) return -2;
    }
    if (H) {
        for (a = 0; a < 4; a++)
            for (bb = 0; bb < 4; bb++)
                Hs[a * 4 + bb] = lamPu * HP[a * 4 + bb] + lamQu * HQ[a * 4 + bb]
                    + mu * 2.0 * (dP[a] * dP[bb] + P * HP[a * 4 + bb]
                                  + dQ[a] * dQ[bb] + Q * HQ[a * 4 + bb]);
        for (a = 0; a < 4; a++)
            for (bb = a; bb < 4; bb++)
                if (push_sym(H, gidx[a], gidx[bb], Hs[a * 4 + bb])) return -2;
    }
    return 0;
}

/* Generators, shared by both formulations: injection -Pg, -Qg at their bus, cost in MW
 * (f = w sum c2 MW^2 + c1 MW + c0, MW = baseMVA Pg), its gradient and Hessian (sigma-weighted),
 * and the -1 Jacobian entries.  A generator out of service (gmask[k] = 0; a contingency may be a
 * generator outage, Sec. V-A) contributes nothing: no injection, no cost, and zero gradient,
 * Jacobian and Hessian entries (the pattern keeps them).  gmask NULL = all in service.
 * Returns 0, -1 on a bad bus index, -2 when a triplet array is full. */
static int gen_terms(const oracle_net *net, const double *Pg, const double *Qg,
                     const uint8_t *gmask, double w, double sigma, double *gP, double *gQ,
                     double *fval, double *grad, oracle_coo *J, oracle_coo *H)
{
    const int nb = net->nb, ng = net->ng;
    const double base = net->baseMVA;
    int k;
    *fval = 0.0;
    for (k = 0; k < ng; k++) {
        int gb = net->gbus[k];
        int on = gmask == NULL || gmask[k] != 0;
        double MW = base * Pg[k];
        if (gb < 0 || gb >= nb) return -1;
        if (on) {
            gP[gb] -= Pg[k];
            gQ[gb] -= Qg[k];
            *fval += w * (net->c2[k] * MW * MW + net->c1[k] * MW + net->c0[k]);
            grad[2 * nb + k] = w * (2.0 * net->c2[k] * base * base * Pg[k] + net->c1[k] * base);
        }
        if (J) {
            if (push(J, gb, 2 * nb + k, on ? -1.0 : 0.0)) return -2;
            if (push(J, nb + gb, 2 * nb + ng + k, on ? -1.0 : 0.0)) return -2;
        }
        if (H) {
            double hk = on ? sigma * w * 2.0 * net->c2[k] * base * base : 0.0;
            if (push(H, 2 * nb + k, 2 * nb + k, hk)) return -2;
        }
    }
    return 0;
}

/* Capacity the triplet arrays need for one evaluation. */
void oracle_coo_capacity(const oracle_net *net, int64_t *capJ, int64_t *capH)
{
    *capJ = 24 * (int64_t)net->nl + 4 * (int64_t)net->nb + 2 * (int64_t)net->ng;
    *capH = 20 * (int64_t)net->nl + 3 * (int64_t)net->nb + (int64_t)net->ng;
}

/*
 * One evaluation (Sec. III, eqs. (7)-(10); objective weight pi_s of eq. (27)).
 *   x[n], lam[m]; mask[nl] (1 in service, 0 out; NULL = all in service); gmask[ng] the same for
 *   generators;
 *   pd_scale[nb] (NULL = 1); w = objective weight; sigma = objective factor in the Hessian.
 * Outputs: *fval, grad[n], gh[m]; J and H triplets appended to *J, *H (either may be NULL).
 * Returns 0, -1 on a bad branch (r = x = 0) or bus index, -2 when a triplet array is full.
 */
int oracle_eval(const oracle_net *net, const double *x, const double *lam, const uint8_t *mask,
                const uint8_t *gmask, const double *pd_scale, double w, double sigma,
                double *fval, double *grad, double *gh, oracle_coo *J, oracle_coo *H)
{
    const int nb = net->nb, nl = net->nl, ng = net->ng;
    const int n = 2 * nb + 2 * ng;
    const double *Va = x, *Vm = x + nb, *Pg = x + 2 * nb, *Qg = x + 2 * nb + ng;
    const double *lamP = lam, *lamQ = lam + nb, *muF = lam + 2 * nb, *muT = lam + 2 * nb + nl;
    double *gP = gh, *gQ = gh + nb, *hF = gh + 2 * nb, *hT = gh + 2 * nb + nl;
    int i, l;

    for (i = 0; i < 2 * nb + 2 * nl; i++) gh[i] = 0.0;
    for (i = 0; i < n; i++) grad[i] = 0.0;

    /* branches */
    for (l = 0; l < nl; l++) {
        double Y[8];
        int fb = net->f[l], tb = net->t[l];
        double m = (mask == NULL || mask[l]) ? 1.0 : 0.0;
        double P[2], Q[2], dP[2][4], dQ[2][4], HP[2][16], HQ[2][16];
        int gidx[2][4];
        int s;
        if (fb < 0 || fb >= nb || tb < 0 || tb >= nb || fb == tb) return -1;
        if (oracle_pi_model_shift(net->r[l], net->x[l], net->b[l], net->tap[l],
                                  branch_shift(net, l), Y) != 0) return -1;
        /* from side: u = f, v = t; to side: u = t, v = f */
        side_terms(Y[0], Y[1], Y[2], Y[3], Va[fb], Va[tb], Vm[fb], Vm[tb],
                   &P[0], &Q[0], dP[0], dQ[0], HP[0], HQ[0]);
        side_terms(Y[6], Y[7], Y[4], Y[5], Va[tb], Va[fb], Vm[tb], Vm[fb],
                   &P[1], &Q[1], dP[1], dQ[1], HP[1], HQ[1]);
        gidx[0][0] = fb; gidx[0][1] = tb; gidx[0][2] = nb + fb; gidx[0][3] = nb + tb;
        gidx[1][0] = tb; gidx[1][1] = fb; gidx[1][2] = nb + tb; gidx[1][3] = nb + fb;

        for (s = 0; s < 2; s++) {
            int rc = end_rows(nb, s == 0 ? fb : tb, 2 * nb + (s == 0 ? l : nl + l), m,
                              lamP[s == 0 ? fb : tb], lamQ[s == 0 ? fb : tb],
                              s == 0 ? muF[l] : muT[l], P[s], Q[s], dP[s], dQ[s], HP[s], HQ[s],
                              gidx[s], gP, gQ, (s == 0 ? hF : hT) + l, J, H);
            if (rc) return rc;
        }
    }

    /* bus shunts and loads: Gs Vm^2 + Pd and -Bs Vm^2 + Qd */
    for (i = 0; i < nb; i++) {
        double sc = pd_scale ? pd_scale[i] : 1.0;
        gP[i] += net->Gs[i] * Vm[i] * Vm[i] + net->Pd[i] * sc;
        gQ[i] += -net->Bs[i] * Vm[i] * Vm[i] + net->Qd[i] * sc;
        if (J) {
            if (push(J, i, i, 0.0)) return -2;                              /* dP_i/dVa_i */
            if (push(J, i, nb + i, 2.0 * net->Gs[i] * Vm[i])) return -2;     /* dP_i/dVm_i */
            if (push(J, nb + i, i, 0.0)) return -2;                         /* dQ_i/dVa_i */
            if (push(J, nb + i, nb + i, -2.0 * net->Bs[i] * Vm[i])) return -2;
        }
        if (H) {
            if (push(H, i, i, 0.0)) return -2;
            if (push(H, nb + i, i, 0.0)) return -2;
            if (push(H, nb + i, nb + i,
                     lamP[i] * 2.0 * net->Gs[i] - lamQ[i] * 2.0 * net->Bs[i])) return -2;
        }
    }

    /* generators: injection -Pg, -Qg at their bus; cost in MW */
    return gen_terms(net, Pg, Qg, gmask, w, sigma, gP, gQ, fval, grad, J, H);
}

/* ---- sum duplicate triplets into CSR with ascending columns ---- */
typedef struct { int row, col; int64_t idx; } key_t_;

static int cmp_key(const void *pa, const void *pb)
{
    const key_t_ *a = (const key_t_ *)pa, *b = (const key_t_ *)pb;
    if (a->row != b->row) return a->row < b->row ? -1 : 1;
    if (a->col != b->col) return a->col < b->col ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* Sorts by (row, col, emission order) and sums duplicates in emission order.
 * rowptr[nrows+1]; col/val need room for c->n entries.  Returns nnz, or -1 on a bad row
 * or allocation failure. */
int64_t oracle_coo_to_csr(const oracle_coo *c, int nrows, int64_t *rowptr, int *col, double *val)
{
    key_t_ *keys;
    int64_t i, nnz = 0;
    int r;
    keys = (key_t_ *)malloc((size_t)(c->n > 0 ? c->n : 1) * sizeof(key_t_));
    if (!keys) return -1;
    for (i = 0; i < c->n; i++) {
        if (c->row[i] < 0 || c->row[i] >= nrows) { free(keys); return -1; }
        keys[i].row = c->row[i];
        keys[i].col = c->col[i];
        keys[i].idx = i;
    }
    qsort(keys, (size_t)c->n, sizeof(key_t_), cmp_key);
    for (r = 0; r <= nrows; r++) rowptr[r] = 0;
    for (i = 0; i < c->n; i++) {
        if (nnz > 0 && i > 0 && keys[i].row == keys[i - 1].row && keys[i].col == keys[i - 1].col) {
            val[nnz - 1] += c->val[keys[i].idx];
        } else {
            col[nnz] = keys[i].col;
            val[nnz] = c->val[keys[i].idx];
            rowptr[keys[i].row + 1]++;
            nnz++;
        }
    }
    for (r = 0; r < nrows; r++) rowptr[r + 1] += rowptr[r];
    free(keys);
    return nnz;
}

/* ---- Coupling (ramp) rows between the subproblems of the multi-stage problems ----
 * The general problem (Sec. I, eqs. (5)-(6)), the multi-period problem (Sec. IV, eq. (15)), the
 * security-constrained one (Sec. V-A, eq. (20)) and the stochastic one (Sec. VI-A, eq. (31)) tie
 * each subproblem state x_b to one other state x_p(b) -- the previous time step, the base case,
 * or the base scenario -- by a bounded difference  -delta <= x_b - x_p(b) <= delta.  The text
 * names the generators' real power output as the quantity that is ramp-limited, so there is one
 * row per (state b, generator k):
 *     r[b][k] = Pg_k(x_b) - Pg_k(x_p(b)),
 * with Pg_k(x_b) = x_b[2 nb + k].  A state with p(b) = -1 (the first period, the base case) has
 * no rows; its entries of r are 0.  The states are stacked: x is [B][n], r is [B][ng].
 * Returns 0, or -1 for a parent index outside [-1, B) or equal to b. */
int oracle_coupling(int B, int n, int nb, int ng, const int *parent, const double *x, double *r)
{
    for (int b = 0; b < B; b++) {
        int p = parent[b];
        if (p < -1 || p >= B || p == b) return -1;
        for (int k = 0; k < ng; k++)
            r[(int64_t)b * ng + k] =
                p < 0 ? 0.0 : x[(int64_t)b * n + 2 * nb + k] - x[(int64_t)p * n + 2 * nb + k];
    }
    return 0;
}

/* The transpose product  out = C^T nu  in the stacked variable layout [B][n], straight from the
 * rows: row (b, k) holds +1 at column (b, Pg_k) and -1 at column (p(b), Pg_k), so its multiplier
 * nu[b][k] is added to the first and subtracted from the second, rows taken in ascending (b, k).
 * Every other entry of out is zero.  Returns 0, or -1 as oracle_coupling. */
int oracle_coupling_jtv(int B, int n, int nb, int ng, const int *parent, const double *nu,
                        double *out)
{
    for (int64_t i = 0; i < (int64_t)B * n; i++) out[i] = 0.0;
    for (int b = 0; b < B; b++) {
        int p = parent[b];
        if (p < -1 || p >= B || p == b) return -1;
        if (p < 0) continue;
        for (int k = 0; k < ng; k++) {
            out[(int64_t)b * n + 2 * nb + k] += nu[(int64_t)b * ng + k];
            out[(int64_t)p * n + 2 * nb + k] -= nu[(int64_t)b * ng + k];
        }
    }
    return 0;
}

/* ---- Power-balance-cartesian formulation (Sec. III names it beside the polar one) ----
 * The same network, balances, flow limits and cost, with the bus voltage in rectangular form
 * V_i = e_i + j f_i:
 *   variables     x   = [e (nb) | f (nb) | Pg (ng) | Qg (ng)]
 *   equalities    g   = [P balance (nb) | Q balance (nb)]
 *   inequalities  h   = [|S_from|^2 (nl) | |S_to|^2 (nl) | e_i^2 + f_i^2 (nb)]
 *   multipliers   lam = [lamP (nb) | lamQ (nb) | muF (nl) | muT (nl) | muV (nb)]
 * The voltage-magnitude limits, simple bounds on Vm in the polar model, become the last nb rows:
 * Vmin^2 <= e^2 + f^2 <= Vmax^2.
 * One end of a branch, from its bus u towards v, with a = e_u e_v + f_u f_v (= Vu Vv cos th),
 * b = f_u e_v - e_u f_v (= Vu Vv sin th) and s = e_u^2 + f_u^2 (= Vu^2):
 *   P =  Gss s + Gm a + Bm b
 *   Q = -Bss s + Gm b - Bm a
 * Both are linear in (s, a, b), so their gradients and (constant) Hessians follow from those of
 * s, a and b in the local order (e_u, f_u, e_v, f_v). */
static void side_terms_cart(double Gss, double Bss, double Gm, double Bm,
                            double eu, double fu, double ev, double fv,
                            double *P, double *Q, double *dP, double *dQ, double *HP, double *HQ)
{
    const double da[4] = {ev, fv, eu, fu};
    const double db[4] = {-fv, ev, fu, -eu};
    const double ds[4] = {2.0 * eu, 2.0 * fu, 0.0, 0.0};
    static const double Ha[16] = {0, 0, 1, 0,  0, 0, 0, 1,  1, 0, 0, 0,  0, 1, 0, 0};
    static const double Hb[16] = {0, 0, 0, -1,  0, 0, 1, 0,  0, 1, 0, 0,  -1, 0, 0, 0};
    static const double Hs[16] = {2, 0, 0, 0,  0, 2, 0, 0,  0, 0, 0, 0,  0, 0, 0, 0};
    double a = eu * ev + fu * fv;
    double b = fu * ev - eu * fv;
    double s = eu * eu + fu * fu;
    int i;
    *P = Gss * s + Gm * a + Bm * b;
    *Q = -Bss * s + Gm * b - Bm * a;
    for (i = 0; i < 4; i++) {
        dP[i] = Gss * ds[i] + Gm * da[i] + Bm * db[i];
        dQ[i] = -Bss * ds[i] + Gm * db[i] - Bm * da[i];
    }
    for (i = 0; i < 16; i++) {
        HP[i] = Gss * Hs[i] + Gm * Ha[i] + Bm * Hb[i];
        HQ[i] = -Bss * Hs[i] + Gm * Hb[i] - Bm * Ha[i];
    }
}

/* Capacity the triplet arrays need for one cartesian evaluation. */
void oracle_coo_capacity_cart(const oracle_net *net, int64_t *capJ, int64_t *capH)
{
    *capJ = 24 * (int64_t)net->nl + 6 * (int64_t)net->nb + 2 * (int64_t)net->ng;
    *capH = 20 * (int64_t)net->nl + 5 * (int64_t)net->nb + (int64_t)net->ng;
}

/*
 * One cartesian evaluation: arguments and returns as oracle_eval, with x[n] = [e | f | Pg | Qg],
 * lam[m] and gh[m] of m = 3 nb + 2 nl (the voltage rows last).  Triplets are emitted for every
 * structural dependency: per branch end its P, Q and h rows over (e_u, f_u, e_v, f_v); per bus the
 * shunt entries of its P and Q rows, its voltage row over (e_i, f_i), and the Hessian diagonal
 * block (e_i, e_i), (f_i, e_i), (f_i, f_i); per generator as in the polar model.
 */
int oracle_eval_cart(const oracle_net *net, const double *x, const double *lam,
                     const uint8_t *mask, const uint8_t *gmask, const double *pd_scale, double w,
                     double sigma,
                     double *fval, double *grad, double *gh, oracle_coo *J, oracle_coo *H)
{
    const int nb = net->nb, nl = net->nl, ng = net->ng;
    const int n = 2 * nb + 2 * ng;
    const double *E = x, *F = x + nb, *Pg = x + 2 * nb, *Qg = x + 2 * nb + ng;
    const double *lamP = lam, *lamQ = lam + nb, *muF = lam + 2 * nb, *muT = lam + 2 * nb + nl;
    const double *muV = lam + 2 * nb + 2 * nl;
    double *gP = gh, *gQ = gh + nb, *hF = gh + 2 * nb, *hT = gh + 2 * nb + nl;
    double *hV = gh + 2 * nb + 2 * nl;
    int i, l;

    for (i = 0; i < 3 * nb + 2 * nl; i++) gh[i] = 0.0;
    for (i = 0; i < n; i++) grad[i] = 0.0;

    /* branches */
    for (l = 0; l < nl; l++) {
        double Y[8];
        int fb = net->f[l], tb = net->t[l];
        double m = (mask == NULL || mask[l]) ? 1.0 : 0.0;
        double P[2], Q[2], dP[2][4], dQ[2][4], HP[2][16], HQ[2][16];
        int gidx[2][4];
        int s;
        if (fb < 0 || fb >= nb || tb < 0 || tb >= nb || fb == tb) return -1;
        if (oracle_pi_model_shift(net->r[l], net->x[l], net->b[l], net->tap[l],
                                  branch_shift(net, l), Y) != 0) return -1;
        side_terms_cart(Y[0], Y[1], Y[2], Y[3], E[fb], F[fb], E[tb], F[tb],
                        &P[0], &Q[0], dP[0], dQ[0], HP[0], HQ[0]);
        side_terms_cart(Y[6], Y[7], Y[4], Y[5], E[tb], F[tb], E[fb], F[fb],
                        &P[1], &Q[1], dP[1], dQ[1], HP[1], HQ[1]);
        gidx[0][0] = fb; gidx[0][1] = nb + fb; gidx[0][2] = tb; gidx[0][3] = nb + tb;
        gidx[1][0] = tb; gidx[1][1] = nb + tb; gidx[1][2] = fb; gidx[1][3] = nb + fb;

        for (s = 0; s < 2; s++) {
            int rc = end_rows(nb, s == 0 ? fb : tb, 2 * nb + (s == 0 ? l : nl + l), m,
                              lamP[s == 0 ? fb : tb], lamQ[s == 0 ? fb : tb],
                              s == 0 ? muF[l] : muT[l], P[s], Q[s], dP[s], dQ[s], HP[s], HQ[s],
                              gidx[s], gP, gQ, (s == 0 ? hF : hT) + l, J, H);
            if (rc) return rc;
        }
    }

    /* bus shunts, loads and voltage rows: Gs |V|^2 + Pd, -Bs |V|^2 + Qd, |V|^2 = e^2 + f^2 */
    for (i = 0; i < nb; i++) {
        double sc = pd_scale ? pd_scale[i] : 1.0;
        double V2 = E[i] * E[i] + F[i] * F[i];
        gP[i] += net->Gs[i] * V2 + net->Pd[i] * sc;
        gQ[i] += -net->Bs[i] * V2 + net->Qd[i] * sc;
        hV[i] = V2;
        if (J) {
            int vrow = 2 * nb + 2 * nl + i;
            if (push(J, i, i, 2.0 * net->Gs[i] * E[i])) return -2;
            if (push(J, i, nb + i, 2.0 * net->Gs[i] * F[i])) return -2;
            if (push(J, nb + i, i, -2.0 * net->Bs[i] * E[i])) return -2;
            if (push(J, nb + i, nb + i, -2.0 * net->Bs[i] * F[i])) return -2;
            if (push(J, vrow, i, 2.0 * E[i])) return -2;
            if (push(J, vrow, nb + i, 2.0 * F[i])) return -2;
        }
        if (H) {
            /* lamP 2 Gs - lamQ 2 Bs + muV 2 on both diagonals; the (f_i, e_i) entry is 0 */
            double d = lamP[i] * 2.0 * net->Gs[i] - lamQ[i] * 2.0 * net->Bs[i] + muV[i] * 2.0;
            if (push(H, i, i, d)) return -2;
            if (push(H, nb + i, i, 0.0)) return -2;
            if (push(H, nb + i, nb + i, d)) return -2;
        }
    }

    /* generators, exactly as in the polar model */
    return gen_terms(net, Pg, Qg, gmask, w, sigma, gP, gQ, fval, grad, J, H);
}

/* ---- Feasibility slacks: load loss and power imbalance ----
 * The model's feasibility options (Sec. III, Fig. 2: load loss, power imbalance) add nonnegative
 * variables that enter the bus balances linearly and are penalised linearly in the objective.
 * Slack k sits at bus bus[k] in the P balance (row[k] = 0) or the Q balance (row[k] = 1), with
 * sign[k] = +1 or -1 and cost coefficient cost[k] (per p.u.):
 *     g_{row,bus}  +=  sign z_k,      f  +=  w cost z_k,      df/dz_k = w cost,
 * and the Jacobian column of z_k has the single entry sign[k] in that row; the Hessian gets
 * nothing.  Load loss at bus i is a slack with sign -1 (it lowers the load Pd_i); an imbalance is
 * a pair with signs -1 and +1.  For one state: z[nz], gh[m] and *f are added to, grad_z[nz]
 * written (either pointer may be NULL).  Returns 0, or -1 for a bus, row or sign out of range. */
int oracle_slack(int nb, int nz, const int *bus, const int *row, const int *sign,
                 const double *cost, const double *z, double w, double *gh, double *f,
                 double *grad_z)
{
    int k;
    for (k = 0; k < nz; k++) {
        if (bus[k] < 0 || bus[k] >= nb || (row[k] != 0 && row[k] != 1) ||
            (sign[k] != 1 && sign[k] != -1))
            return -1;
        if (gh) gh[row[k] * nb + bus[k]] += sign[k] * z[k];
        if (f) *f += w * cost[k] * z[k];
        if (grad_z) grad_z[k] = w * cost[k];
    }
    return 0;
}
