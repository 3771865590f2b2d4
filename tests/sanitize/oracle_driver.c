/* Sanitizer test driver for the plain C oracle: for each valid grid file it runs every oracle
 * entry point on the file's state (both formulations with and without Jacobian and Hessian, the
 * triplet summation, the feasibility slacks and the coupling rows) and checks that the results
 * are finite.  Built with -fsanitize=address,undefined together with oracle/acopf_oracle.c by
 * tests/test_host_sanitizers.py (test infrastructure); exits nonzero on any failure. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "grid_io.h"

typedef struct {
    int nb, nl, ng;
    const double *Gs, *Bs, *Pd, *Qd;
    const int *f, *t;
    const double *r, *x, *b, *tap;
    const int *gbus;
    const double *c2, *c1, *c0;
    double baseMVA;
    const double *shift;
} oracle_net;
typedef struct { int64_t n, cap; int *row, *col; double *val; } oracle_coo;

int oracle_eval(const oracle_net *, const double *, const double *, const uint8_t *,
                const uint8_t *, const double *, double, double, double *, double *, double *,
                oracle_coo *, oracle_coo *);
int oracle_eval_cart(const oracle_net *, const double *, const double *, const uint8_t *,
                     const uint8_t *, const double *, double, double, double *, double *,
                     double *, oracle_coo *, oracle_coo *);
void oracle_coo_capacity(const oracle_net *, int64_t *, int64_t *);
void oracle_coo_capacity_cart(const oracle_net *, int64_t *, int64_t *);
int64_t oracle_coo_to_csr(const oracle_coo *, int, int64_t *, int *, double *);
int oracle_slack(int, int, const int *, const int *, const int *, const double *, const double *,
                 double, double *, double *, double *);
int oracle_coupling(int, int, int, int, const int *, const double *, double *);
int oracle_coupling_jtv(int, int, int, int, const int *, const double *, double *);

static oracle_coo make_coo(int64_t cap) {
    oracle_coo c;
    c.n = 0; c.cap = cap;
    c.row = (int *)malloc(sizeof(int) * (cap > 0 ? cap : 1));
    c.col = (int *)malloc(sizeof(int) * (cap > 0 ? cap : 1));
    c.val = (double *)malloc(sizeof(double) * (cap > 0 ? cap : 1));
    return c;
}
static void free_coo(oracle_coo *c) { free(c->row); free(c->col); free(c->val); }

static int finite_all(const double *v, int64_t n) {
    for (int64_t i = 0; i < n; i++) if (!isfinite(v[i])) return 0;
    return 1;
}

static int run(const char *path) {
    grid_file g;
    read_grid(path, &g);
    if (g.expect != 0) { free_grid(&g); return 0; }
    oracle_net N = {g.nb, g.nl, g.ng, g.Gs, g.Bs, g.Pd, g.Qd, g.f, g.t, g.r, g.x, g.b, g.tap,
                    g.gbus, g.c2, g.c1, g.c0, g.baseMVA, g.shift};
    const int n = 2 * g.nb + 2 * g.ng, m = 2 * g.nb + 2 * g.nl, mc = m + g.nb;
    double f, *grad = malloc(sizeof(double) * n), *gh = malloc(sizeof(double) * mc);
    double *lamc = malloc(sizeof(double) * mc);
    for (int i = 0; i < mc; i++) lamc[i] = i < m ? g.lam[i] : 0.5;
    uint8_t *gm = malloc(g.ng > 0 ? g.ng : 1);
    for (int k = 0; k < g.ng; k++) gm[k] = (uint8_t)(k % 3 != 1);
    int64_t capJ, capH;
    for (int cart = 0; cart < 2; cart++) {
        if (cart) oracle_coo_capacity_cart(&N, &capJ, &capH);
        else oracle_coo_capacity(&N, &capJ, &capH);
        for (int want = 0; want < 2; want++) {
            oracle_coo J = make_coo(capJ), H = make_coo(capH);
            int rc = cart ? oracle_eval_cart(&N, g.xs, lamc, g.mask, gm, NULL, 0.7, 0.9, &f, grad,
                                             gh, want ? &J : NULL, want ? &H : NULL)
                          : oracle_eval(&N, g.xs, g.lam, g.mask, gm, NULL, 0.7, 0.9, &f, grad, gh,
                                        want ? &J : NULL, want ? &H : NULL);
            if (rc != 0 || !finite_all(gh, cart ? mc : m) || !finite_all(grad, n) || !isfinite(f)) {
                fprintf(stderr, "%s: evaluation failed (cart %d)\n", path, cart);
                return 1;
            }
            if (want) {
                int64_t *rp = malloc(sizeof(int64_t) * ((cart ? mc : m) + 1));
                int *col = malloc(sizeof(int) * (J.n > 0 ? J.n : 1));
                double *val = malloc(sizeof(double) * (J.n > 0 ? J.n : 1));
                if (oracle_coo_to_csr(&J, cart ? mc : m, rp, col, val) < 0 || !finite_all(val, rp[cart ? mc : m])) {
                    fprintf(stderr, "%s: J triplets\n", path);
                    return 1;
                }
                free(rp); free(col); free(val);
                rp = malloc(sizeof(int64_t) * (n + 1));
                col = malloc(sizeof(int) * (H.n > 0 ? H.n : 1));
                val = malloc(sizeof(double) * (H.n > 0 ? H.n : 1));
                if (oracle_coo_to_csr(&H, n, rp, col, val) < 0 || !finite_all(val, rp[n])) {
                    fprintf(stderr, "%s: H triplets\n", path);
                    return 1;
                }
                free(rp); free(col); free(val);
            }
            free_coo(&J); free_coo(&H);
        }
    }
    /* slacks: an imbalance pair on every P row */
    int nz = 2 * g.nb;
    int *bus = malloc(sizeof(int) * nz), *row = malloc(sizeof(int) * nz), *sg = malloc(sizeof(int) * nz);
    double *cost = malloc(sizeof(double) * nz), *z = malloc(sizeof(double) * nz), *gz = malloc(sizeof(double) * nz);
    for (int k = 0; k < nz; k++) { bus[k] = k % g.nb; row[k] = 0; sg[k] = k < g.nb ? -1 : 1; cost[k] = 10.0; z[k] = 0.01 * k; }
    double fs = f;
    if (oracle_slack(g.nb, nz, bus, row, sg, cost, z, 0.5, gh, &fs, gz) != 0) { fprintf(stderr, "slack\n"); return 1; }
    /* coupling rows over a three-state chain of this state */
    const int B = 3;
    int parent[3] = {-1, 0, 1};
    double *xb = malloc(sizeof(double) * B * n), *rr = malloc(sizeof(double) * B * (g.ng > 0 ? g.ng : 1));
    double *nu = malloc(sizeof(double) * B * (g.ng > 0 ? g.ng : 1)), *out = malloc(sizeof(double) * B * n);
    for (int s = 0; s < B; s++) for (int i = 0; i < n; i++) xb[s * n + i] = g.xs[i] + 0.1 * s;
    for (int i = 0; i < B * g.ng; i++) nu[i] = 1.0 + i;
    for (int i = 0; i < B * n; i++) out[i] = 0.0;
    if (oracle_coupling(B, n, g.nb, g.ng, parent, xb, rr) != 0 ||
        oracle_coupling_jtv(B, n, g.nb, g.ng, parent, nu, out) != 0) { fprintf(stderr, "coupling\n"); return 1; }
    printf("%s: ok (f %.6g)\n", path, f);
    free(bus); free(row); free(sg); free(cost); free(z); free(gz); free(xb); free(rr); free(nu); free(out);
    free(grad); free(gh); free(lamc); free(gm);
    free_grid(&g);
    return 0;
}

int main(int argc, char **argv) {
    for (int i = 1; i < argc; i++)
        if (run(argv[i])) return 1;
    return 0;
}
