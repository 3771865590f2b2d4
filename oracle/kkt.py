"""Plain CPU oracle of the linear algebra around the model evaluation: the interior-point KKT step
and the power-flow Newton step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline
are the only callers.  Nothing here touches the CUDA library; the model's values (J, the Lagrangian
Hessian, g) come from the plain C oracle (acopf_oracle.c) through ``oracle.acopf``.

KKT step.  The paper's solvers (Ipopt, HiOp; Sec. II-III) take one Newton step per interior-point
iteration on the primal-dual system of the model of eqs. (7)-(10); SCOPFLOW with EMPAR (Sec. V-A,
eqs. (16)-(20)) and SOPFLOW (Sec. VI-A) solve one such system per contingency or scenario.  With
the Lagrangian Hessian W (n x n), the constraint Jacobian J (m x n, rows g then h), the primal
diagonal dx (barrier term plus regularisation, n entries) and the dual diagonal dc (m entries: the
equality rows' regularisation and the inequality rows' slack term), the step solves
    K [dx_step; dlam] = r,     K = [[W + diag(dx), J'], [J, -diag(dc)]]
(the augmented system of Wachter and Biegler's interior-point method with the slacks eliminated).
``kkt_matrix`` writes K out entry by entry from the CSR values; ``kkt_solve`` solves it with a
library sparse direct solve.

Power-flow Newton step (PFLOW, the paper's power-flow application).  Buses are slack (type 3),
PV (2) or PQ (1); Pg and Qg are data.  The unknowns are Va at every non-slack bus and Vm at every
PQ bus, the equations the P balance at every non-slack bus and the Q balance at every PQ bus.  One
step solves J_pf d = -g_pf with the rows and columns of g and J (the model's own, from the C
oracle) that these select, and returns x with Va and Vm moved by d.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def kkt_matrix(n: int, m: int, J, H, dx, dc) -> sp.csr_matrix:
    """K of one state from J = (rowptr, col, val) (m rows) and the lower triangle of the
    Lagrangian Hessian H = (rowptr, col, val) (n rows), written entry by entry."""
    rows, cols, vals = [], [], []
    hp, hc, hv = H
    for i in range(n):                           # W, both triangles from the lower one
        for k in range(hp[i], hp[i + 1]):
            j = int(hc[k])
            rows.append(i); cols.append(j); vals.append(hv[k])
            if j != i:
                rows.append(j); cols.append(i); vals.append(hv[k])
    for i in range(n):                           # + diag(dx)
        rows.append(i); cols.append(i); vals.append(dx[i])
    jp, jc, jv = J
    for r in range(m):                           # J below, J' to the right
        for k in range(jp[r], jp[r + 1]):
            j = int(jc[k])
            rows.append(n + r); cols.append(j); vals.append(jv[k])
            rows.append(j); cols.append(n + r); vals.append(jv[k])
    for r in range(m):                           # - diag(dc)
        rows.append(n + r); cols.append(n + r); vals.append(-dc[r])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n + m, n + m))


def kkt_solve(n: int, m: int, J, H, dx, dc, rhs) -> np.ndarray:
    """[dx_step; dlam] of one state: K^{-1} rhs."""
    K = kkt_matrix(n, m, J, H, dx, dc)
    return sla.spsolve(K.tocsc(), np.asarray(rhs, dtype=np.float64))


def pf_sets(nb: int, bus_type):
    """Indices of the power-flow unknowns (Va of non-slack buses, then Vm of PQ buses) in
    x = [Va | Vm | Pg | Qg], and of its equations (P rows of non-slack buses, then Q rows of PQ
    buses) in g = [P | Q]."""
    bt = np.asarray(bus_type)
    ns = np.flatnonzero(bt != 3)
    pq = np.flatnonzero(bt == 1)
    return np.concatenate([ns, nb + pq]), np.concatenate([ns, nb + pq])


def pf_newton_step(om, net, x, bus_type, gen_mask=None, mask=None, pd_scale=None):
    """One power-flow Newton step: returns (x_new, mismatch), mismatch = max |g_pf(x)| before
    the step.  om is oracle.acopf; g and J are its evaluation at x (multipliers irrelevant;
    branch mask, generator mask and load scale as in the evaluation)."""
    nb = net.nb
    lam = np.zeros(net.m)
    r = om.evaluate(net, x, lam, mask, pd_scale, 1.0, 0.0, want_hess=False, gen_mask=gen_mask)
    cols, rows = pf_sets(nb, bus_type)
    jp, jc, jv = r["J"]
    Js = sp.csr_matrix((jv, jc, jp), shape=(net.m, net.n))
    Jpf = Js[rows][:, cols].tocsc()
    gpf = r["gh"][rows]
    d = sla.spsolve(Jpf, -gpf) if gpf.size else np.zeros(0)
    x_new = np.array(x, dtype=np.float64, copy=True)
    x_new[cols] += d
    return x_new, float(np.max(np.abs(gpf))) if gpf.size else 0.0
