/*
 * exago.h -- C ABI of the GB300 batched evaluator of the polar AC optimal power flow model.
 *
 * The model is the compact ACOPF of ExaGO (arXiv 2203.10587), Sec. III, eqs. (7)-(10):
 *     min f(x)   s.t.   g(x) = 0,   h- <= h(x) <= h+,   x- <= x <= x+
 * in the "power-balance-polar" formulation named in Sec. III.  An interior-point solver (Ipopt,
 * HiOp, TAO; Sec. II-III) calls the model once per iteration for f, grad f, g, h, the Jacobian of
 * [g; h] and the Hessian of the Lagrangian; this library evaluates those callbacks for a batch of
 * B independent states on one GPU.  Independent states are the contingencies of SCOPFLOW
 * (Sec. V-A, eqs. (16)-(20)), the scenarios of SOPFLOW (Sec. VI-A, eqs. (27)-(31)) and the
 * subproblems of the embarrassingly parallel EMPAR solver (Sec. V-A).
 *
 * Conventions (all quantities per unit; angles in radians):
 *   variables     x      = [Va (nb) | Vm (nb) | Pg (ng) | Qg (ng)],            n = 2 nb + 2 ng
 *   constraints   g | h  = [P balance (nb) | Q balance (nb) | |S_from|^2 (nl) | |S_to|^2 (nl)],
 *                                                                                m = 2 nb + 2 nl
 *   multipliers   lambda = [lamP (nb) | lamQ (nb) | muF (nl) | muT (nl)]
 *   P balance of bus i:  sum of branch-end injections at i + Gs_i Vm_i^2 + Pd_i s_i - sum Pg at i
 *   Q balance of bus i:  sum of branch-end injections at i - Bs_i Vm_i^2 + Qd_i s_i - sum Qg at i
 *   branch model:        pi-model, series 1/(r + jx), charging b split half per end, tap on the
 *                        from end (tap 0 means 1), no phase shift (exago_net_create_shift
 *                        adds one per branch: phase-shifting transformers)
 *   objective:           f = w * sum_k (c2_k (baseMVA Pg_k)^2 + c1_k baseMVA Pg_k + c0_k)
 *   Lagrangian Hessian:  sigma grad^2 f + sum lam_i grad^2 g_i + sum mu_l grad^2 h_l, lower
 *                        triangle, row-major CSR, ascending columns
 *   Jacobian:            rows of g then h, row-major CSR, ascending columns
 *   out-of-service branch (mask 0): contributes nothing; its two h rows and their Jacobian and
 *                        Hessian entries evaluate to 0; the sparsity pattern is unchanged.
 *
 * Threading and streams: every function may be called from any host thread.  Evaluation calls
 * are asynchronous on the stream given in the batch; host-side argument errors return at once.
 * Calls that share one net and no caller workspace share the net's internal workspace; the
 * library orders them across streams and threads (exago_batch, `workspace`), except calls
 * captured into a caller's CUDA graph, which the caller orders.  Errors raised inside kernels (a bounded wait that
 * timed out) are recorded in a device status word and returned by exago_net_check.
 * Every function returns EXAGO_OK or an error code; exago_last_error() then describes it.
 */
#ifndef EXAGO_GB300_H
#define EXAGO_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EXAGO_OK = 0,
    EXAGO_EINVAL = 1,    /* bad argument: null pointer, out-of-range index, r = x = 0, ... */
    EXAGO_ENOMEM = 2,    /* device or host allocation failed */
    EXAGO_ECUDA = 3,     /* a CUDA runtime call failed */
    EXAGO_ETIMEOUT = 4,  /* a bounded device-side wait gave up, or a serve deadline passed */
    EXAGO_EBUSY = 5,     /* serve queue full */
    EXAGO_ESTATE = 6,    /* call not valid in the object's current state */
    EXAGO_EDEVICE = 7    /* a device-side index check failed (library built with EXAGO_DEBUG) */
} exago_status;

typedef struct exago_net *exago_net_t;

/* Thread-local description of the last non-OK status returned on this thread. */
const char *exago_last_error(void);

/* Name of a status code ("EXAGO_EINVAL", ...). */
const char *exago_status_name(exago_status s);

/*
 * Builds a network on the current CUDA device (Sec. III model data; the network build happens
 * once per grid, before the solver's iterations).  Copies every host array; the caller keeps
 * ownership of its arrays.  Validates indices (0 <= f, t < nb, f != t, 0 <= gbus < nb),
 * r = x = 0, negative taps, non-finite values and baseMVA <= 0 (EINVAL).  Builds the Jacobian and
 * Hessian patterns and every output position on the host, uploads them, and evaluates the
 * pi-model admittances on the device.
 *   nb, nl, ng >= 0 (nb >= 1).  Gs, Bs, Pd, Qd: [nb] or NULL (zeros).  f, t, r, x, b: [nl].
 *   tap: [nl] or NULL (all 1); 0 entries mean 1.  rateA: [nl] or NULL; flow limit in p.u., used
 *   only by exago_net_ineq_bounds (0 means unlimited).  gbus, c2, c1: [ng]; c0: [ng] or NULL.
 * On success *out owns device memory until exago_net_destroy.
 */
exago_status exago_net_create(int nb, const double *Gs, const double *Bs, const double *Pd,
                              const double *Qd, int nl, const int *f, const int *t,
                              const double *r, const double *x, const double *b,
                              const double *tap, const double *rateA, int ng, const int *gbus,
                              const double *c2, const double *c1, const double *c0,
                              double baseMVA, exago_net_t *out);

/*
 * exago_net_create for a network with phase-shifting transformers: the same arguments, plus
 * shift[nl] (host, rad; NULL = no phase shift anywhere), the phase angle of the ideal transformer
 * on each branch's from side.  Its complex ratio is T = tau e^{j shift} (tau = tap, 0 meaning 1),
 * so the mutual admittances become Yft = -ys/conj(T) and Ytf = -ys/T and differ between the two
 * ends (the textbook and MATPOWER branch model; Sec. III lists the network features the model
 * carries).  Every evaluation entry point of both formulations honours the shifts, through the
 * kernel variants that read each end's own mutual admittances; a net created with shift = NULL,
 * or by exago_net_create, runs the shift-free variants.  EINVAL for a non-finite shift.
 */
exago_status exago_net_create_shift(int nb, const double *Gs, const double *Bs, const double *Pd,
                                    const double *Qd, int nl, const int *f, const int *t,
                                    const double *r, const double *x, const double *b,
                                    const double *tap, const double *shift,
                                    const double *rateA, int ng, const int *gbus,
                                    const double *c2, const double *c1, const double *c0,
                                    double baseMVA, exago_net_t *out);

/*
 * Host-only planning with the same arguments and validation as exago_net_create, without
 * touching a GPU.  The handle answers exago_net_dims, the pattern, bound and plan-array queries
 * and exago_net_destroy; evaluation calls on it return EXAGO_ESTATE.  Useful to set up a solver's
 * symbolic factorisation before any device work, and to check the plan on a machine without GPU.
 */
exago_status exago_net_plan(int nb, const double *Gs, const double *Bs, const double *Pd,
                            const double *Qd, int nl, const int *f, const int *t,
                            const double *r, const double *x, const double *b,
                            const double *tap, const double *rateA, int ng, const int *gbus,
                            const double *c2, const double *c1, const double *c0,
                            double baseMVA, exago_net_t *out);

/* Frees the network's device and host memory.  NULL is accepted.  The caller must make sure no
 * work that uses the network is still queued on any stream. */
exago_status exago_net_destroy(exago_net_t net);

/* Problem dimensions: n variables, m_eq = 2 nb, m_ineq = 2 nl, nonzeros of J and of lower H. */
exago_status exago_net_dims(exago_net_t net, int *n, int *m_eq, int *m_ineq, int64_t *nnzJ,
                            int64_t *nnzH);

/* Jacobian pattern into caller host arrays: rowptr[m + 1], col[nnzJ] (eqs. (8)-(9) rows). */
exago_status exago_net_jac_pattern(exago_net_t net, int64_t *rowptr, int *col);

/* Lower-triangle Lagrangian Hessian pattern into caller host arrays: rowptr[n + 1], col[nnzH]. */
exago_status exago_net_hess_pattern(exago_net_t net, int64_t *rowptr, int *col);

/* Bounds h- and h+ of eq. (9) into caller host arrays [2 nl]: h- = 0, h+ = rateA^2 (or HUGE_VAL
 * where rateA = 0). */
exago_status exago_net_ineq_bounds(exago_net_t net, double *hlo, double *hhi);

/*
 * Copies one of the plan's int32 tables into a caller host buffer, for inspection and tests:
 * slot_ptr ([nb+1]), slot_nbr ([2 nl] other bus of each slot; slots are ordered by (bus, other
 * bus, branch)), slot_ref ([2 nl] record 2 l + end of each slot), bus_jP / bus_jQ (J row starts of
 * P_i / Q_i), bus_hA / bus_hM (H row starts of Va_i / Vm_i), bus_k (neighbours + 1), bus_nlow
 * (neighbours below i), bus_perm ([4][nb], the bus phase's thread order for tiles of 32, 64, 128
 * and 256 buses: each aligned tile sorted by descending degree), gen_ptr ([nb+1]) and gen_ord
 * ([ng]).
 * *needed receives the size in bytes;
 * dst may be NULL to query it.  EINVAL for an unknown name or a small buffer.
 */
exago_status exago_net_plan_array(exago_net_t net, const char *name, void *dst, size_t bytes,
                                  size_t *needed);

/*
 * One batch of B independent evaluation states.  Every pointer is a DEVICE pointer owned by the
 * caller that must stay valid until the work queued on `stream` completes.
 *   x          [B][n]    row-major
 *   lambda     [B][m]    multipliers (needed by the Hessian only; may be NULL otherwise)
 *   mask       [B][nl]   1 in service, 0 out of service (N-1 contingency, Sec. V-A); NULL = all 1
 *   pd_scale   [B][nb]   per-bus load scale of a scenario (Sec. VI-A); NULL = 1
 *   obj_weight [B]       scenario weight pi_s of eq. (27); NULL = 1
 *   obj_factor           sigma of the Lagrangian Hessian (Ipopt's obj_factor)
 *   stream               cudaStream_t to queue the work on (NULL = legacy default stream)
 *   workspace            optional device scratch of at least exago_eval_workspace_size bytes,
 *                        256-byte aligned; NULL = use the net's internal workspace, grown on
 *                        demand (a growth calls cudaMalloc; use exago_net_reserve before any
 *                        stream capture).  Calls that use the internal workspace are ordered by
 *                        the library: a call on another stream than the workspace's last user
 *                        first waits (on the device) for that use, and a growth waits for every
 *                        earlier use before it frees the old buffer, so such calls may come from
 *                        any stream and any host thread.  Calls captured into a caller's CUDA
 *                        graph are outside this ordering: the caller orders their replays against
 *                        other calls on the same net (and a growth after such a capture drains
 *                        the device).  Calls with their own `workspace` share nothing.
 *   gen_mask   [B][ng]   1 in service, 0 out of service (a generator outage, alone or with line
 *                        outages: SCOPFLOW contingencies, Sec. V-A); NULL = all 1.  An
 *                        out-of-service generator contributes nothing: no injection in its bus's
 *                        balances, no cost, and zero gradient, Jacobian (-1 entries) and cost
 *                        Hessian values; the sparsity pattern is unchanged.  Last in the struct,
 *                        so a caller that zero-initialises the batch gets NULL.
 */
typedef struct {
    int B;
    const double *x;
    const double *lambda;
    const uint8_t *mask;
    const double *pd_scale;
    const double *obj_weight;
    double obj_factor;
    void *stream;
    void *workspace;
    size_t workspace_bytes;
    const uint8_t *gen_mask;
} exago_batch;

/* Scratch bytes one evaluation of B states needs under the net's configuration (branch-end
 * values, and the persistent schedule's counters); enough for either schedule. */
exago_status exago_eval_workspace_size(exago_net_t net, int B, size_t *bytes);

/* Grows the net's internal workspace to hold B states now, so later calls allocate nothing. */
exago_status exago_net_reserve(exago_net_t net, int B);

/*
 * Evaluations (Sec. III, eqs. (7)-(10)).  Outputs are caller DEVICE buffers, row-major per state:
 *   f [B]; grad [B][n]; gh [B][m] (g then h); jval [B][nnzJ] in exago_net_jac_pattern order;
 *   hval [B][nnzH] in exago_net_hess_pattern order.
 * exago_eval_all computes any subset in one pass: NULL outputs are skipped.
 * Errors: EINVAL for a null net or batch, B < 0, a missing x (or lambda when hval is wanted), a
 * too-small or misaligned workspace; ECUDA if a launch fails.  B = 0 returns OK and does nothing.
 */
exago_status exago_eval_obj(exago_net_t net, const exago_batch *batch, double *f);
exago_status exago_eval_grad(exago_net_t net, const exago_batch *batch, double *grad);
exago_status exago_eval_cons(exago_net_t net, const exago_batch *batch, double *gh);
exago_status exago_eval_jac(exago_net_t net, const exago_batch *batch, double *jval);
exago_status exago_eval_hess(exago_net_t net, const exago_batch *batch, double *hval);
exago_status exago_eval_all(exago_net_t net, const exago_batch *batch, double *f, double *grad,
                            double *gh, double *jval, double *hval);

/*
 * Adjoint products of the constraint map c(x) = [g(x); h(x)] of eqs. (8)-(9), for solvers and
 * automatic differentiation, without forming J or the Hessian.  Batch inputs as for the
 * evaluations; vectors are caller DEVICE buffers, row-major per state.
 *   exago_eval_jvp:  out [B][m] = J(x) u,              u [B][n]
 *   exago_eval_jtv:  out [B][n] = J(x)^T v,            v [B][m]
 *   exago_eval_hvp:  out [B][n] = H u,  u [B][n], H = obj_factor w grad^2 f + sum_i lambda_i
 *                    grad^2 c_i -- the Lagrangian Hessian of exago_eval_hess (needs lambda).
 * Out-of-service branches contribute nothing.  EINVAL for null vectors or a missing lambda
 * (HVP); otherwise as exago_eval_all.  Results are deterministic (fixed summation order).
 */
exago_status exago_eval_jvp(exago_net_t net, const exago_batch *batch, const double *u, double *out);
exago_status exago_eval_jtv(exago_net_t net, const exago_batch *batch, const double *v, double *out);
exago_status exago_eval_hvp(exago_net_t net, const exago_batch *batch, const double *u, double *out);

/*
 * The power-balance-cartesian formulation (Sec. III names it beside the power-balance-polar one)
 * on the same net: bus voltages V_i = e_i + j f_i instead of (Va, Vm).
 *   variables     x      = [e (nb) | f (nb) | Pg (ng) | Qg (ng)]                 (n as polar)
 *   constraints   g | h  = [P balance | Q balance | |S_from|^2 | |S_to|^2 | e_i^2 + f_i^2 (nb)]
 *                 (m_c = 3 nb + 2 nl: the voltage-magnitude limits, bounds on Vm in the polar
 *                 model, become the last nb rows, Vmin^2 <= e^2 + f^2 <= Vmax^2)
 *   multipliers   lambda = [lamP | lamQ | muF | muT | muV]                        (m_c values)
 *   one branch end at bus u towards v, a = e_u e_v + f_u f_v, b = f_u e_v - e_u f_v:
 *                 P = Gss (e_u^2 + f_u^2) + G a + B b,   Q = -Bss (e_u^2 + f_u^2) + G b - B a
 * The balances, flow rows, masks, load scales, objective and generator terms are the polar model's.
 *   exago_net_dims_cart         n, m_eq = 2 nb, m_ineq = 2 nl + nb, nnzJ_c = nnzJ + 2 nb, nnzH.
 *   exago_net_jac_pattern_cart  HOST rowptr [m_c + 1], col [nnzJ_c]: the polar pattern with e in
 *                               place of Va and f in place of Vm, then voltage row i with columns
 *                               e_i, f_i.  The Hessian pattern is exago_net_hess_pattern's (same
 *                               substitution).  Works on a net made by exago_net_plan.
 *   exago_eval_cart_workspace_size  scratch bytes of exago_eval_cart for B states, enough for
 *                               either schedule (branch-end records of the persistent schedule's
 *                               ring, at most about 64 MB, and its counters, 8 B + 8 B per state;
 *                               or up to three chunks of records, at most about 75 MB).
 *   exago_eval_cart             f [B], grad [B][n], gh [B][m_c], jval [B][nnzJ_c], hval [B][nnzH]
 *                               (DEVICE buffers; any may be NULL) for the batch's states x [B][n]
 *                               and multipliers lambda [B][m_c].  batch->workspace as for
 *                               exago_eval_all (else the net's internal workspace, grown on
 *                               demand; a smaller batch->workspace that still holds two ring
 *                               slots and the counters is used with fewer slots).  Errors as
 *                               exago_eval_all.  The net's configuration picks the schedule:
 *                               EXAGO_SCHED_AUTO / PERSISTENT (the default) run the polar model's
 *                               persistent work list -- one launch whose CTAs claim branch and
 *                               bus items of 128 branches or buses of every state, bus items
 *                               waiting (bounded, EXAGO_ETIMEOUT in the status word) for their
 *                               state's branch items, records in an L2-resident ring of lag,
 *                               ring states (the configuration's lag and ring, else derived) --
 *                               through the net's graph cache (use_graph as for exago_eval_all).
 *                               EXAGO_SCHED_PIPELINED / KERNELS: per chunk of states a branch
 *                               kernel writes records and a bus kernel assembles the rows; the
 *                               bus kernel of a chunk runs on the net's side stream while the
 *                               next chunk's branch kernel runs on batch->stream (ordered by
 *                               events).  Both give bitwise equal results; the call returns with
 *                               all work ordered on batch->stream and may be captured in a CUDA
 *                               graph once a first call outside the capture has grown the
 *                               workspace, or with a batch->workspace.
 */
exago_status exago_net_dims_cart(exago_net_t net, int *n, int *m_eq, int *m_ineq, int64_t *nnzJ,
                                 int64_t *nnzH);
exago_status exago_net_jac_pattern_cart(exago_net_t net, int64_t *rowptr, int *col);
exago_status exago_eval_cart_workspace_size(exago_net_t net, int B, size_t *bytes);
exago_status exago_eval_cart(exago_net_t net, const exago_batch *batch, double *f, double *grad,
                             double *gh, double *jval, double *hval);
/* Adjoint products of the cartesian constraint map c = [g; h] (m_c rows), as exago_eval_jvp / jtv
 * / hvp for the polar one: out [B][m_c] = J u (u [B][n]); out [B][n] = J^T v (v [B][m_c]);
 * out [B][n] = H u with H = obj_factor w grad^2 f + sum_i lambda_i grad^2 c_i, the Hessian of
 * exago_eval_cart (needs lambda [B][m_c]).  A batch->workspace of exago_eval_cart_workspace_size
 * bytes is enough.  Errors as exago_eval_jvp. */
exago_status exago_eval_cart_jvp(exago_net_t net, const exago_batch *batch, const double *u,
                                 double *out);
exago_status exago_eval_cart_jtv(exago_net_t net, const exago_batch *batch, const double *v,
                                 double *out);
exago_status exago_eval_cart_hvp(exago_net_t net, const exago_batch *batch, const double *u,
                                 double *out);

/*
 * Feasibility slacks: load loss and power imbalance (Sec. III, Fig. 2).  Each slack z_k >= 0 sits
 * at bus bus[k] in the P balance (row[k] = 0) or the Q balance (row[k] = 1) with sign[k] = +1 or
 * -1 and a linear cost cost[k] per p.u.:  g_{row,bus} += sign z_k  and  f += w cost_k z_k, with
 * w the batch's obj_weight.  Load loss at a bus is a slack of sign -1 (it lowers the load); an
 * imbalance is a pair of signs -1 and +1.  The slack variables follow x in the solver's vector;
 * their Jacobian column is the single constant entry sign_k in balance row row_k nb + bus_k,
 * and they add nothing to the Lagrangian Hessian.
 *   exago_slack_create    HOST arrays [nz], copied.  EINVAL for a NULL net or out, nz < 0, NULL
 *                         arrays with nz > 0, a bus outside [0, nb), a row not 0 or 1, a sign not
 *                         +1 or -1, or a cost that is not finite.  A net made by exago_net_plan
 *                         gives a host-only set (pattern only; evaluations return ESTATE).
 *   exago_slack_pattern   HOST rows [nz] (the balance row of each slack's Jacobian entry) and
 *                         vals [nz] (its value, the sign).
 *   exago_eval_slack      adds the slacks to a finished evaluation of the same states, on
 *                         batch->stream (batch: B, obj_weight and stream are used): z [B][nz];
 *                         gh [B][ldgh] += the balance terms (rows 0 .. 2 nb of each state, in the
 *                         slacks' ascending order; ldgh = m for the polar model, m + nb for the
 *                         cartesian one); f [B] += w sum_k cost_k z_k; grad_z [B][nz] = w cost_k.
 *                         Any of gh, f, grad_z may be NULL.  All DEVICE buffers.
 *   exago_eval_slack_jtv  out [B][nz] = the slack columns' part of J^T v: sign_k v[row_k nb +
 *                         bus_k] for v [B][ldv] (ldv >= 2 nb); J u for the slack columns is
 *                         exago_eval_slack with z = u, gh the accumulator, f = grad_z = NULL.
 * Errors: EINVAL for NULL vectors (B > 0), ldgh or ldv below 2 nb or a different current device;
 * ECUDA if a launch fails.  B = 0 or nz = 0 does nothing.
 */
typedef struct exago_slack *exago_slack_t;
exago_status exago_slack_create(exago_net_t net, int nz, const int *bus, const int *row,
                                const int *sign, const double *cost, exago_slack_t *out);
exago_status exago_slack_destroy(exago_slack_t slack);
exago_status exago_slack_pattern(exago_slack_t slack, int64_t *rows, double *vals);
exago_status exago_eval_slack(exago_slack_t slack, const exago_batch *batch, const double *z,
                              double *gh, int64_t ldgh, double *f, double *grad_z);
/*
 * exago_eval_all and exago_eval_slack in one call, for the polar formulation: the evaluation's
 * outputs with the slacks' balance terms, cost and gradient grad_z [B][nz] (DEVICE) included, bit
 * for bit what the two calls give (it issues them in order on batch->stream).  Evaluating the
 * slacks inside the evaluation's launch was measured slower: the slacks' gathers land on the
 * latency-bound bus phase, while their own kernels run at HBM speed.  Errors as exago_eval_all
 * and exago_eval_slack; EINVAL for a slack set of another grid.
 */
exago_status exago_eval_all_slack(exago_net_t net, const exago_batch *batch, exago_slack_t slack,
                                  const double *z, double *f, double *grad, double *gh,
                                  double *jval, double *hval, double *grad_z);
exago_status exago_eval_slack_jtv(exago_slack_t slack, const exago_batch *batch, const double *v,
                                  int64_t ldv, double *out);

/*
 * Coupling (ramp) rows between the states of a batch.  ExaGO's multi-stage problems tie each
 * subproblem's state to one other state by a bounded difference: consecutive periods of the
 * multi-period problem (Sec. IV, eq. (15)), each contingency to the base case (Sec. V-A,
 * eq. (20)), each scenario to the base scenario (Sec. VI-A, eq. (31)), and trees of these (the
 * general form, Sec. I, eqs. (5)-(6)).  The ramp-limited quantity is the generators' real power, so
 * with parent p(b) of state b (-1: none) there is one row per (state b, generator k):
 *     r[b][k] = Pg_k(x_b) - Pg_k(x_p(b)),   bounds -delta_k <= r <= delta_k (solver data).
 * A state without a parent keeps its ng rows, which are zero and have no Jacobian entries.  The
 * rows are linear: exago_eval_coupling applied to a direction u is the Jacobian-vector product, the
 * Jacobian values are constants, and the rows add nothing to the Lagrangian Hessian.
 *
 *   exago_coupling_create   parent: HOST [B], each -1 or another state's index (not b itself);
 *                           copied, so the caller keeps its array.  Any parent structure is
 *                           accepted (chains, stars, trees, forests).  A net made by
 *                           exago_net_plan gives a host-only coupling (dims and pattern only;
 *                           evaluations return ESTATE).  The net's device must be current.
 *                           EINVAL for a NULL net or out, B < 0, a NULL parent with B > 0 or a
 *                           parent index outside [-1, B) or equal to its state; ENOMEM if the
 *                           device tables cannot be allocated.  The coupling does not refer to the
 *                           net after creation.
 *   exago_coupling_dims     B, rows = B ng, nnz = 2 ng x (states with a parent).
 *   exago_coupling_jac_pattern  HOST outputs: rowptr [rows + 1], col [nnz] and, if not NULL,
 *                           val [nnz] of the Jacobian with respect to the stacked variables of all
 *                           states: the column of (state b, Pg_k) is b n + 2 nb + k; +1 on the
 *                           row's own state, -1 on its parent's; columns ascending within a row.
 *   exago_eval_coupling     r [B][ng] from x [B][n] (DEVICE buffers, row-major per state), queued on
 *                           stream.  Bitwise the definition above (one subtraction per value).
 *   exago_eval_coupling_jtv out = C^T nu restricted to the Pg columns: for every state b and k,
 *                           out[b ldo + k] = [p(b) >= 0] nu[b][k] - sum over the children c of b
 *                           (states with p(c) = b) of nu[c][k];  (C^T nu) is zero in every other
 *                           column.  nu [B][ng]; out holds (B - 1) ldo + ng doubles and must not
 *                           overlap nu; ldo >= ng.  accumulate = 0 stores, 1 adds to out.  To add
 *                           C^T nu to a [B][n] gradient g, pass out = g + 2 nb and ldo = n.  The
 *                           children are summed in a fixed order (deterministic, no atomics).
 * Errors of the evaluations: EINVAL for NULL pointers (B > 0) or a different current device;
 * ECUDA if a launch fails.  B = 0 or ng = 0 does nothing.
 */
typedef struct exago_coupling *exago_coupling_t;
exago_status exago_coupling_create(exago_net_t net, int B, const int *parent,
                                   exago_coupling_t *out);
exago_status exago_coupling_destroy(exago_coupling_t cpl);
exago_status exago_coupling_dims(exago_coupling_t cpl, int *B, int64_t *rows, int64_t *nnz);
exago_status exago_coupling_jac_pattern(exago_coupling_t cpl, int64_t *rowptr, int64_t *col,
                                        double *val);
exago_status exago_eval_coupling(exago_coupling_t cpl, const double *x, double *r, void *stream);
exago_status exago_eval_coupling_jtv(exago_coupling_t cpl, const double *nu, double *out,
                                     int64_t ldo, int accumulate, void *stream);

/*
 * exago_eval_all without any allocation.  The paper has no counterpart: this serves callers that
 * may not allocate device memory once running -- for example a solver whose device memory belongs
 * to a pooling allocator (a raw cudaMalloc would bypass it, and cudaFree synchronises the device),
 * or a serving loop that reserves everything at start-up.  It takes the same batch and outputs as
 * exago_eval_all and gives the same results, but its scratch lives in one static device array of
 * EXAGO_STATIC_SCRATCH_BYTES per GPU, reserved by every GPU that loads the library until the
 * process exits; batch->workspace is ignored and nothing is allocated.
 *   - The net's device must be current.  The first call on a device looks up the array's device
 *     address (cudaGetSymbolAddress) once for that device; make that first call before any stream
 *     capture.
 *   - EINVAL if the batch's scratch exceeds the array: split the batch.  Each state needs
 *     10 x 2 nl doubles of branch-end records (80 bytes per branch end; the batch's total is
 *     rounded up to 256 bytes).
 *   - All calls share the array: calls that overlap on the GPU race on it, so order them (one
 *     stream, or events).  Nothing in it needs clearing; each call writes all the scratch it reads.
 */
#define EXAGO_STATIC_SCRATCH_BYTES ((size_t)16 << 20)
exago_status exago_eval_all_static(exago_net_t net, const exago_batch *batch, double *f,
                                   double *grad, double *gh, double *jval, double *hval);

/*
 * Per-kernel timing of exago_eval_all (tracing and benchmarks).  Runs the same evaluation `reps`
 * times on batch->stream with a CUDA event recorded on that stream before every kernel launch and
 * after the last one, waits for each repetition, and returns the mean duration in milliseconds of
 * each kernel of one evaluation: names[k] (static strings: "branch", "bus", "grad", "obj" for
 * the multi-kernel schedule, "persistent" for the fused one) and ms[k] for k < *nkernels.
 * After "persistent" come the fused kernel's phases, timed on the device's global timer by the
 * CTAs themselves in `reps` further evaluations (names starting "phase: "): kernel span, CTA entry to the first branch item,
 * the branch items, the last branch end to the first bus start (the wait of a single state),
 * the bus items, the objective, and the last bus end to the last CTA exit.  With several states
 * the phases overlap (a span can then exceed the sum, or be negative).  names and ms need room
 * for 16 entries.  Outputs are those of exago_eval_all.  EINVAL for reps < 1 or null
 * names/ms/nkernels.
 */
exago_status exago_eval_profile(exago_net_t net, const exago_batch *batch, double *f, double *grad,
                                double *gh, double *jval, double *hval, int reps, int *nkernels,
                                const char **names, double *ms);

/*
 * Launch configuration of a net (zero-initialised = automatic).
 *   schedule  EXAGO_SCHED_AUTO: the autotuned choice for the batch size if exago_net_autotune ran
 *             for it, else the persistent schedule.  EXAGO_SCHED_KERNELS: one launch per stage
 *             (branch, bus, fixup, gradient, objective) over the batch.  EXAGO_SCHED_PERSISTENT:
 *             one fused launch whose CTAs claim branch and bus tiles of all states from a work
 *             list (the batched evaluation of SCOPFLOW / SOPFLOW subproblems, Sec. V-A, VI-A).
 *   block     persistent: threads per CTA and items per tile (32, 64, 128, 256; 0 = 64).
 *   occupancy persistent: resident warps per SM the kernel's registers must allow (16 or 24;
 *             8 = the compiler's choice of registers; 0 = 16).  Higher occupancy can cost
 *             register spills.
 *   stage_records  EXAGO_STAGE_ON: a bus tile runs slot-parallel -- one thread per branch end
 *             reads its record (coalesced) and writes the neighbour's row entries, then one
 *             thread per bus sums its ends' diagonal terms from shared memory; DEFAULT / OFF:
 *             one thread per bus walks its ends, reading the records through L2.
 *             EXAGO_STAGE_BULK (persistent schedule, branch per thread; elsewhere OFF): one TMA
 *             bulk copy brings a bus tile's records into shared memory, and one thread per bus
 *             walks its ends there (tiles whose records do not fit read them through L2).
 *             EXAGO_SCHED_PIPELINED: the batch in chunks; the branch kernel of a chunk runs on
 *             the caller's stream while the bus kernel of the previous chunk runs on a
 *             high-priority net stream, ordered by events only (no device-side waits).
 *   lag       persistent: states by which bus tiles trail branch tiles (0 = derived).
 *   ring      persistent: scratch ring slots, > lag (0 = derived); pipelined: chunks of records
 *             in the ring (0 = 3, at most 7).
 *   chunk     pipelined: states per chunk (0 = as many as fit 48 MB of records in the ring).
 *   use_graph persistent and pipelined: EXAGO_GRAPH_DEFAULT / ON launch through a cached instantiated CUDA
 *             graph (one per distinct argument set, 8 kept).  An argument set is captured on its
 *             second use among the last 32 uncached calls, so a one-off set launches directly.
 *             OFF always launches directly.  A call on a stream that is being captured always
 *             launches directly.
 *   spin_limit  polls (about 0.4 us each) before a device-side wait gives up and records
 *             EXAGO_ETIMEOUT in the status word (0 = 2^22).
 *   test_force_timeout  testing only: bus tiles wait for a count that never arrives, so every
 *             wait times out; the launch still ends and exago_net_check reports it.
 *   tile_group  persistent: tiles of one kind and state per work item (1 to 4; 0 = 1), which
 *             divides the items' claims, waits and signals by that number.
 *   tiling    persistent: EXAGO_TILING_DEFAULT / THREAD: branch per thread -- each thread of a
 *             tile takes its own branch (bus) of one state.  EXAGO_TILING_WARP: branch per warp
 *             -- each warp takes one branch (bus) and its 32 lanes take 32 consecutive states,
 *             so every lane of a warp walks a bus of the same degree; blocks of 128 (0 = 128)
 *             or 64 threads, occupancy 8 or 16, tile_group branches (buses) per warp and work item,
 *             no record staging, and lag and ring count groups of 32 states (a ring slot then
 *             holds 32 states' records, so exago_eval_workspace_size grows accordingly).  Both
 *             tilings give bitwise equal outputs.  The power-balance-cartesian calls ignore it.
 */
enum { EXAGO_SCHED_AUTO = 0, EXAGO_SCHED_KERNELS = 1, EXAGO_SCHED_PERSISTENT = 2,
       EXAGO_SCHED_PIPELINED = 3 };
enum { EXAGO_GRAPH_DEFAULT = 0, EXAGO_GRAPH_ON = 1, EXAGO_GRAPH_OFF = 2 };
enum { EXAGO_STAGE_DEFAULT = 0, EXAGO_STAGE_ON = 1, EXAGO_STAGE_OFF = 2, EXAGO_STAGE_BULK = 3 };
enum { EXAGO_TILING_DEFAULT = 0, EXAGO_TILING_THREAD = 1, EXAGO_TILING_WARP = 2 };
typedef struct {
    int schedule;
    int block;
    int occupancy;
    int stage_records;
    int lag;
    int ring;
    int chunk;
    int use_graph;
    long long spin_limit;
    int test_force_timeout;
    int tile_group;
    int tiling;
} exago_config;

/* Sets the net's configuration (validated: EINVAL for unknown values or ring <= lag). */
exago_status exago_net_set_config(exago_net_t net, const exago_config *cfg);

/* The configuration a batch of B states would run with, every derived field filled in. */
exago_status exago_net_get_config(exago_net_t net, int B, exago_config *cfg);

/*
 * Autotuner: times the multi-kernel schedule, pipelined variants (three chunk sizes) and
 * persistent variants (block 32 / 64 / 128 / 256, occupancy 8 / 16 / 24 warps, 1 or 2 tiles per
 * work item), each with and without slot-parallel bus tiles, persistent variants with bulk-copied
 * bus tile records (block 64 / 128, occupancy 8 / 16), and the warp-tiled persistent
 * variants (branch per warp: block 64 / 128, occupancy 8 / 16, 1 or 2 branches per warp and
 * item), on this batch, `reps` evaluations each after one warm-up, on batch->stream, and records the
 * fastest for batches of this size (used by EXAGO_SCHED_AUTO).  Outputs are written as by
 * exago_eval_all.  *best (may be NULL) receives the choice.
 */
exago_status exago_net_autotune(exago_net_t net, const exago_batch *batch, double *f, double *grad,
                                double *gh, double *jval, double *hval, int reps,
                                exago_config *best);

/*
 * Serving: concurrent solver instances (grids of any sizes, each a registered net) submit
 * evaluation requests; network data and states stay on the device (ExaGO keeps model evaluation
 * on the GPU, Sec. II; independent subproblems as in EMPAR, Sec. V-A).  A scheduler thread admits
 * queued requests in arrival order whenever one of max_slots slots is free and the request's
 * workspace fits in the server's device arena (device_mem_budget bytes, allocated once here), and
 * launches each on one of n_streams streams, so requests overlap on the GPU and new ones join as
 * others finish.  An admission takes the oldest queued request together with later queued
 * requests for the same net and the same set of outputs, up to a number of states (32 by
 * default; exago_serve_set_merge), and evaluates all their states in one launch through a
 * device table of per-state pointers: each result is the one the request would get alone.
 * Serving allocates no device memory after exago_serve_create.
 *   exago_serve_create   EINVAL for max_slots, n_streams < 1 or a zero budget; ENOMEM if the
 *                        arena cannot be allocated.  The queue holds up to 4 max_slots requests.
 *   exago_serve_register the server uses (does not own) the net; it must outlive the server.
 *                        EINVAL for NULL or a net planned without a device.
 *   exago_serve_submit   request = an exago_batch (device inputs; workspace ignored) and device
 *                        outputs as for exago_eval_all; all must stay valid until the request
 *                        completes.  The request runs on a server stream after the work queued on
 *                        request->stream before the call (an event recorded there), so inputs
 *                        written on that stream need no synchronisation.  deadline_ms > 0: a request still queued after that
 *                        long completes with EXAGO_ETIMEOUT without running.  EBUSY when the
 *                        queue is full, ENOMEM when the request's workspace exceeds the whole
 *                        budget, EINVAL for bad arguments.  *ticket identifies the request.
 *   exago_serve_poll     *done = 1 once the request completed (successfully or not).
 *   exago_serve_wait     waits up to timeout_ms (<= 0: forever) and returns the request's status
 *                        (EXAGO_OK, or ETIMEOUT for an expired deadline, or the evaluation's
 *                        error), then forgets the ticket; EBUSY if it is still queued or running.
 *   exago_serve_stats    submit-to-completion latency quantiles (ms) and count of completed
 *                        requests so far.
 *   exago_serve_destroy  fails queued requests (ESTATE), waits for running ones, frees everything.
 */
typedef struct exago_server *exago_server_t;
exago_status exago_serve_create(size_t device_mem_budget, int max_slots, int n_streams,
                                exago_server_t *out);
exago_status exago_serve_register(exago_server_t server, exago_net_t net, int *net_id);
/* As exago_serve_register, for requests in the cartesian formulation: each is evaluated alone
 * (no merging) by exago_eval_cart's schedule without the graph cache, with outputs and
 * multipliers sized as exago_eval_cart's and a workspace of exago_eval_cart_workspace_size. */
exago_status exago_serve_register_cart(exago_server_t server, exago_net_t net, int *net_id);
exago_status exago_serve_submit(exago_server_t server, int net_id, const exago_batch *request,
                                double *f, double *grad, double *gh, double *jval, double *hval,
                                double deadline_ms, uint64_t *ticket);
/* States per merged admission (>= 1; 1 evaluates every request on its own).  EINVAL otherwise. */
exago_status exago_serve_set_merge(exago_server_t server, int max_states);
exago_status exago_serve_poll(exago_server_t server, uint64_t ticket, int *done);
exago_status exago_serve_wait(exago_server_t server, uint64_t ticket, double timeout_ms);
exago_status exago_serve_stats(exago_server_t server, double *p50_ms, double *p99_ms,
                               uint64_t *completed);
exago_status exago_serve_destroy(exago_server_t server);

/*
 * A native load generator for a server (benchmarks and tests; the paper has no counterpart):
 * drives `server` for `seconds` with n_clients simulated solver instances, each at most one
 * request outstanding, from the calling thread (no interpreter in the submission loop).
 *   clients[i]   the net id, request batch and DEVICE outputs of client i (kept valid by the
 *                caller); group[i] its grid group, 0 .. n_groups - 1;
 *   weight[g]    the share of arrivals that go to group g (need not sum to 1);
 *   rate <= 0    closed loop: every client resubmits as soon as its request completes;
 *   rate > 0     Poisson arrivals at `rate` requests/s (exponential gaps from a 64-bit Mersenne
 *                twister seeded by `seed`) until `seconds` of arrival time or of wall time have
 *                passed (a rate above what can be submitted falls behind the clock and still
 *                ends on time); each takes a free client of a group drawn by weight;
 *                when the group has none, its finished requests are collected, and failing
 *                that the oldest outstanding one is waited for (counted as deferred).
 *   result[5]    requests completed, seconds elapsed, server p50 and p99 latency (ms, over the
 *                server's whole life: create one server per run) and deferred arrivals.
 * Returns the first failing serve call's status; every request submitted is waited for.
 */
typedef struct {
    int net_id;
    const exago_batch *batch;
    double *f, *grad, *gh, *jval, *hval;
} exago_serve_client;
exago_status exago_serve_drive(exago_server_t server, const exago_serve_client *clients,
                               const int *group, int n_clients, const double *weight,
                               int n_groups, double rate, double seconds, uint64_t seed,
                               double *result);

/*
 * Batched interior-point KKT step (the linear solve the paper's solvers, Ipopt and HiOp, perform
 * once per iteration, Sec. II-III; one per contingency or scenario subproblem under EMPAR,
 * Sec. V-A, eqs. (16)-(20), and Sec. VI-A).  For every state b of a batch it solves
 *     K_b [dx; dlam] = r_b,    K_b = [[W_b + diag(dx_b), J_b'], [J_b, -diag(dc_b)]]
 * with W_b the Lagrangian Hessian and J_b the Jacobian of [g; h] exactly as exago_eval_all writes
 * them (hval [B][nnzH], the lower triangle; jval [B][nnzJ]).  The flow rows and the generator
 * variables are eliminated first (they create no fill), then the remaining 4 x 4 block per bus
 * (Va, Vm, lamP, lamQ) is factored by a batched block L D L' without pivoting on a minimum-degree
 * order of the bus graph computed once by exago_kkt_create.  K must be factorable without
 * pivoting: it is whenever W + diag(dx) is positive definite and dc > 0 (a quasi-definite K;
 * interior-point methods regularise to that), and dx of every Qg must be nonzero.
 *   exago_kkt_create      symbolic analysis on the host (ordering, factor structure, update
 *                         lists, levels) and upload.  On a net made by exago_net_plan it does the
 *                         analysis alone (info and order answer; solve returns ESTATE).  The
 *                         handle refers to the net, which must outlive it.
 *   exago_kkt_order       host arrays [nb] (each may be NULL): perm (the bus eliminated k-th),
 *                         parent (elimination tree over elimination indices, -1 at a root) and
 *                         level (0 at the leaves; columns of one level are factored together).
 *   exago_kkt_info        factor blocks, update pairs (4 x 4 block products per state), levels of
 *                         the elimination tree, and FP64 flops of one state's factor and solve.
 *   exago_kkt_workspace_size  scratch bytes for B states (two factor arrays of 16 blocks x 8 B x B
 *                         per factor block, the reduced vectors and counters).
 *   exago_kkt_solve       DEVICE pointers, row-major per state: jval [B][nnzJ], hval [B][nnzH],
 *                         dx [B][n], dc [B][m] (> 0), rhs [B][n + m]; sol [B][n + m] receives
 *                         [dx; dlam].  inertia [B][2] (or NULL) receives the number of negative
 *                         pivots of the whole factorisation (m for a correct interior-point step)
 *                         and of pivots below 1e-13 of their block (0 unless K is numerically
 *                         singular without pivoting).  workspace: at least exago_kkt_workspace_size
 *                         bytes, 256-byte aligned, or NULL for the handle's own (grown on demand;
 *                         a growth synchronises the device; calls using it must be ordered).
 *                         Asynchronous on `stream`.  EINVAL for null arguments or B too large.
 */
typedef struct exago_kkt *exago_kkt_t;
exago_status exago_kkt_create(exago_net_t net, exago_kkt_t *out);
exago_status exago_kkt_destroy(exago_kkt_t kkt);
exago_status exago_kkt_info(exago_kkt_t kkt, int64_t *blocks, int64_t *pairs, int *levels,
                            double *flops);
exago_status exago_kkt_order(exago_kkt_t kkt, int *perm, int *parent, int *level);
exago_status exago_kkt_workspace_size(exago_kkt_t kkt, int B, size_t *bytes);
exago_status exago_kkt_solve(exago_kkt_t kkt, int B, const double *jval, const double *hval,
                             const double *dx, const double *dc, const double *rhs, double *sol,
                             int *inertia, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Batched power-flow Newton step (PFLOW, the paper's power-flow application; balances of Sec. III,
 * eq. (8)).  Buses are PQ (type 1), PV (2) or slack (3); Pg, Qg and the PV and slack set points
 * are data in x.  For every state of the batch one step solves J_pf d = -g_pf, where g_pf holds the
 * P balances of the non-slack buses and the Q balances of the PQ buses and d the changes of Va
 * (non-slack buses) and Vm (PQ buses), and writes x + d.  g and J are exago_eval_all's at x
 * (batch->mask, gen_mask and pd_scale apply); J_pf is factored without pivoting on a minimum-degree
 * order of the bus graph (2 x 2 blocks per bus, the fixed unknowns' rows replaced by identity
 * rows, so they do not move).
 *   exago_pf_create          validates bus_type (host [nb], values 1..3, at least one slack) and
 *                            runs the symbolic analysis; the net must have a device and outlive
 *                            the handle.
 *   exago_pf_workspace_size  scratch bytes for B states (g, J, four factor arrays, vectors).
 *   exago_pf_step            x_new [B][n] (DEVICE; may equal batch->x) = x + d, Pg and Qg copied;
 *                            mismatch [B] (or NULL) = max |g_pf(x)| before the step.
 *                            batch->workspace: at least exago_pf_workspace_size bytes, or NULL for
 *                            the handle's own (grown on demand, synchronising the device; calls
 *                            using it must be ordered); the evaluation inside uses the net's
 *                            internal workspace.  batch->lambda is ignored.  Asynchronous on
 *                            batch->stream.
 */
typedef struct exago_pf *exago_pf_t;
exago_status exago_pf_create(exago_net_t net, const int *bus_type, exago_pf_t *out);
exago_status exago_pf_destroy(exago_pf_t pf);
exago_status exago_pf_workspace_size(exago_pf_t pf, int B, size_t *bytes);
exago_status exago_pf_step(exago_pf_t pf, const exago_batch *batch, double *x_new,
                           double *mismatch);

/*
 * Testing only: the next n device allocations made by the library (network tables, workspaces,
 * serving arenas) fail as if the device were out of memory, so that callers' ENOMEM paths can be
 * exercised without exhausting a GPU.  n <= 0 clears the hook.  The paper has no counterpart.
 */
void exago_test_fail_allocations(int n);

/*
 * Waits for `stream` and returns the device status word of the net: EXAGO_OK, EXAGO_EDEVICE if a
 * device-side index check of the debug build (EXAGO_DEBUG) failed, or EXAGO_ETIMEOUT if a bounded
 * device-side wait gave up, since the last check (the word is then cleared).
 */
exago_status exago_net_check(exago_net_t net, void *stream);

/*
 * Testing only: the bound on branch-end slot indices that the debug build's device-side checks
 * compare against (normally the net's slot count, 2 nl), lowered to `slots` (clamped to
 * [0, 2 nl]; a negative value restores it), so that the checks' failure path can be exercised
 * while every access the kernels still make stays in bounds.  Takes effect in launches made
 * after the call (not in CUDA graphs the net captured before).  Without EXAGO_DEBUG the checks,
 * and this bound, are compiled out.  The paper has no counterpart.
 */
exago_status exago_test_debug_bounds(exago_net_t net, int slots);

/*
 * Testing only: the persistent schedule's work list, decoded on the host by the kernels' own
 * decoder, for B states of Tbr branch items and Tbu bus items each, bus items trailing branch
 * items by `lag` states.  HOST arrays of B (Tbr + Tbu) entries receive, per ticket, kind
 * (1 branch, 0 bus), state and tile.  EINVAL unless B >= 1, Tbr >= 0, Tbu >= 1, 1 <= lag <= B
 * and B (Tbr + Tbu) fits an int.  The paper has no counterpart.
 */
exago_status exago_test_work_list(int B, int Tbr, int Tbu, int lag, int *kind, int *state,
                                  int *tile);

#ifdef __cplusplus
}
#endif

#endif /* EXAGO_GB300_H */
