/* Reading of the sanitizer tests' grid files (written by tests/test_host_sanitizers.py): one grid
 * per file, whitespace-separated numbers:
 *   expect nb nl ng baseMVA has_shift
 *   Gs Bs Pd Qd (nb each), f t (nl ints each), r x b tap rateA (nl each), gbus (ng ints),
 *   c2 c1 c0 (ng each), shift (nl, if has_shift), then one state: x (2 nb + 2 ng), lam (2 nb + 2 nl),
 *   mask (nl ints).
 * expect is 0 for a valid grid, 1 for one the library must reject. */
#ifndef SANITIZE_GRID_IO_H
#define SANITIZE_GRID_IO_H
#include <stdio.h>
#include <stdlib.h>

typedef struct {
    int expect, nb, nl, ng, has_shift;
    double baseMVA;
    double *Gs, *Bs, *Pd, *Qd, *r, *x, *b, *tap, *rateA, *c2, *c1, *c0, *shift;
    int *f, *t, *gbus;
    double *xs, *lam;
    unsigned char *mask;
} grid_file;

static double *read_d(FILE *fp, int n) {
    double *v = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int i = 0; i < n; i++)
        if (fscanf(fp, "%lf", &v[i]) != 1) { fprintf(stderr, "short file\n"); exit(2); }
    return v;
}
static int *read_i(FILE *fp, int n) {
    int *v = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; i++)
        if (fscanf(fp, "%d", &v[i]) != 1) { fprintf(stderr, "short file\n"); exit(2); }
    return v;
}
static void read_grid(const char *path, grid_file *g) {
    FILE *fp = fopen(path, "r");
    if (!fp) { perror(path); exit(2); }
    if (fscanf(fp, "%d %d %d %d %lf %d", &g->expect, &g->nb, &g->nl, &g->ng, &g->baseMVA,
               &g->has_shift) != 6) { fprintf(stderr, "bad header\n"); exit(2); }
    g->Gs = read_d(fp, g->nb); g->Bs = read_d(fp, g->nb); g->Pd = read_d(fp, g->nb);
    g->Qd = read_d(fp, g->nb);
    g->f = read_i(fp, g->nl); g->t = read_i(fp, g->nl);
    g->r = read_d(fp, g->nl); g->x = read_d(fp, g->nl); g->b = read_d(fp, g->nl);
    g->tap = read_d(fp, g->nl); g->rateA = read_d(fp, g->nl);
    g->gbus = read_i(fp, g->ng);
    g->c2 = read_d(fp, g->ng); g->c1 = read_d(fp, g->ng); g->c0 = read_d(fp, g->ng);
    g->shift = g->has_shift ? read_d(fp, g->nl) : NULL;
    g->xs = read_d(fp, 2 * g->nb + 2 * g->ng);
    g->lam = read_d(fp, 2 * g->nb + 2 * g->nl);
    int *m = read_i(fp, g->nl);
    g->mask = (unsigned char *)malloc(g->nl > 0 ? g->nl : 1);
    for (int i = 0; i < g->nl; i++) g->mask[i] = (unsigned char)m[i];
    free(m);
    fclose(fp);
}
static void free_grid(grid_file *g) {
    double *d[] = {g->Gs, g->Bs, g->Pd, g->Qd, g->r, g->x, g->b, g->tap, g->rateA, g->c2, g->c1,
                   g->c0, g->shift, g->xs, g->lam};
    for (unsigned i = 0; i < sizeof d / sizeof d[0]; i++) free(d[i]);
    free(g->f); free(g->t); free(g->gbus); free(g->mask);
}
#endif
