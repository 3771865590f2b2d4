"""Pins of the CPU oracle against things other than itself (no GPU).

The paper prints no worked example (Sec. III leaves the ACOPF formulation to its references), so
the oracle is pinned by:
  * textbook closed forms: the lossless power-angle equations of a line, line charging b/2 at
    flat start, the objective with hand-computed numbers;
  * an independent formulation: bus injections S = V . conj(Ybus V) and branch flows
    S_f = V_f conj(I_f) in complex arithmetic (MATPOWER's nodal form), against the oracle's polar
    real-valued expansion;
  * the loss invariant: sum of net injections = sum over branches of gs |V_f e^{j Va_f}/tau - V_t e^{j Va_t}|^2;
  * central finite differences of g, h (Jacobian), f (gradient) and sigma grad f + J' lam (Hessian);
  * mask semantics: an out-of-service branch equals the branch removed from the grid;
  * symmetries: angle-shift invariance and the degree-2 (injections) and degree-4 (|S|^2)
    homogeneity in the voltage magnitudes, which tie J to g and H to J;
  * the nonzero counts 4nb + 16nl + 2ng (J) and 3nb + 4nl + ng (lower Hessian).
Each pin is chosen so that a dropped term, a sign error, a swapped from/to index or a transposed
operand in the oracle fails at least one of them; test_oracle_mutants.py plants such
mistakes in copies of the C oracle and checks that each one is caught.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth


def tiny_grid(nb, edges, params, gens, Pd=None, Qd=None, Gs=None, Bs=None):
    """Hand-built grid: edges [(f, t)], params [(r, x, b, tap)], gens [(bus, c2, c1)]."""
    nl = len(edges)
    arr = lambda v, n: np.asarray(v if v is not None else np.zeros(n), dtype=np.float64)
    return synth.Grid(
        nb=nb, Gs=arr(Gs, nb), Bs=arr(Bs, nb), Pd=arr(Pd, nb), Qd=arr(Qd, nb),
        f=np.array([e[0] for e in edges], np.int32), t=np.array([e[1] for e in edges], np.int32),
        r=np.array([p[0] for p in params]), x=np.array([p[1] for p in params]),
        b=np.array([p[2] for p in params]), tap=np.array([p[3] for p in params]),
        rateA=np.full(nl, 2.0), gbus=np.array([g[0] for g in gens], np.int32),
        c2=np.array([g[1] for g in gens], dtype=np.float64),
        c1=np.array([g[2] for g in gens], dtype=np.float64), c0=np.zeros(len(gens)))


def pack_x(g, Va, Vm, Pg=None, Qg=None):
    Pg = np.zeros(g.ng) if Pg is None else Pg
    Qg = np.zeros(g.ng) if Qg is None else Qg
    return np.concatenate([Va, Vm, Pg, Qg]).astype(np.float64)


# ---- independent complex-arithmetic formulation (nodal form, MATPOWER-style) -------------------

def complex_model(g, x, mask=None, pd_scale=None):
    """Branch flows and balances from complex voltages and currents (no polar expansion)."""
    nb, nl, ng = g.nb, g.nl, g.ng
    Va, Vm, Pg, Qg = x[:nb], x[nb:2 * nb], x[2 * nb:2 * nb + ng], x[2 * nb + ng:]
    V = Vm * np.exp(1j * Va)
    m = np.ones(nl) if mask is None else mask.astype(np.float64)
    ys = 1.0 / (g.r + 1j * g.x)
    tau = np.where(g.tap == 0.0, 1.0, g.tap)
    # complex ratio of the from-side ideal transformer: tap and phase shift (phase-shifting
    # transformers); the from current is the series current over conj(T)
    T = tau * np.exp(1j * (np.zeros(nl) if getattr(g, "shift", None) is None else g.shift))
    Yff = (ys + 0.5j * g.b) / (T * np.conj(T)) * m
    Yft = -ys / np.conj(T) * m
    Ytf = -ys / T * m
    Ytt = (ys + 0.5j * g.b) * m
    If = Yff * V[g.f] + Yft * V[g.t]
    It = Ytf * V[g.f] + Ytt * V[g.t]
    Sf = V[g.f] * np.conj(If)
    St = V[g.t] * np.conj(It)
    # nodal admittance matrix and injections S = V conj(Ybus V)
    Ybus = np.zeros((nb, nb), dtype=complex)
    np.add.at(Ybus, (g.f, g.f), Yff)
    np.add.at(Ybus, (g.f, g.t), Yft)
    np.add.at(Ybus, (g.t, g.f), Ytf)
    np.add.at(Ybus, (g.t, g.t), Ytt)
    Ybus[np.arange(nb), np.arange(nb)] += g.Gs + 1j * g.Bs
    Sbus = V * np.conj(Ybus @ V)
    sc = np.ones(nb) if pd_scale is None else pd_scale
    Sg = np.zeros(nb, dtype=complex)
    np.add.at(Sg, g.gbus, Pg + 1j * Qg)
    gP = Sbus.real + g.Pd * sc - Sg.real
    gQ = Sbus.imag + g.Qd * sc - Sg.imag
    return dict(Sf=Sf, St=St, gP=gP, gQ=gQ, V=V, ys=ys, tau=tau, T=T)


def gh_of(oracle_mod, net, x, lam, mask=None, pd_scale=None):
    return oracle_mod.evaluate(net, x, lam, mask, pd_scale, want_jac=False, want_hess=False)


# ---- textbook closed forms ----------------------------------------------------------------------

def test_power_angle_equations_lossless_line(oracle_mod):
    """r = 0, b = 0: Pf = V1 V2 sin(d)/x, Qf = (V1^2 - V1 V2 cos d)/x, Pt = -Pf (power-angle eqs.)."""
    xl, V1, V2, d = 0.1, 1.02, 0.97, 0.13
    g = tiny_grid(2, [(0, 1)], [(0.0, xl, 0.0, 0.0)], [(0, 0.01, 20.0)])
    net = oracle_mod.OracleNet(g)
    x = pack_x(g, np.array([d, 0.0]), np.array([V1, V2]))
    r = gh_of(oracle_mod, net, x, np.zeros(g.m))
    Pf = r["gh"][0]                      # bus 0 balance = Pf - Pg(=0)
    Pt = r["gh"][1]
    Qf = r["gh"][2]
    Qt = r["gh"][3]
    assert Pf == pytest.approx(V1 * V2 * np.sin(d) / xl, rel=1e-14)
    assert Pt == pytest.approx(-V1 * V2 * np.sin(d) / xl, rel=1e-14)
    assert Qf == pytest.approx((V1 ** 2 - V1 * V2 * np.cos(d)) / xl, rel=1e-13)
    assert Qt == pytest.approx((V2 ** 2 - V1 * V2 * np.cos(d)) / xl, rel=1e-13)
    # apparent power rows
    assert r["gh"][4] == pytest.approx(Pf ** 2 + Qf ** 2, rel=1e-14)
    assert r["gh"][5] == pytest.approx(Pt ** 2 + Qt ** 2, rel=1e-14)


def test_transformer_scales_from_voltage(oracle_mod):
    """Lossless transformer of ratio tau: Pf = (V1/tau) V2 sin(d) / x."""
    xl, V1, V2, d, tau = 0.2, 1.0, 1.01, -0.07, 0.97
    g = tiny_grid(2, [(0, 1)], [(0.0, xl, 0.0, tau)], [(0, 0.01, 20.0)])
    net = oracle_mod.OracleNet(g)
    r = gh_of(oracle_mod, net, pack_x(g, np.array([d, 0.0]), np.array([V1, V2])), np.zeros(g.m))
    assert r["gh"][0] == pytest.approx((V1 / tau) * V2 * np.sin(d) / xl, rel=1e-14)
    assert r["gh"][3] == pytest.approx((V2 ** 2 - (V1 / tau) * V2 * np.cos(d)) / xl, rel=1e-13)


def test_flat_start(oracle_mod):
    """Va = 0, Vm = 1, tap = 1: no flow for b = 0; with charging b, Qf = Qt = -b/2 exactly."""
    rng = np.random.default_rng(0)
    g = synth.make_grid(11, 12, 16, 3)
    g.tap[:] = 0.0
    net = oracle_mod.OracleNet(g)
    x = pack_x(g, np.zeros(g.nb), np.ones(g.nb), rng.uniform(0, 1, g.ng), rng.uniform(0, 1, g.ng))
    g0 = synth.Grid(**{**g.__dict__, "b": np.zeros(g.nl)})
    r0 = gh_of(oracle_mod, oracle_mod.OracleNet(g0), x, np.zeros(g.m))
    hP = r0["gh"][2 * g.nb:]
    assert np.all(np.abs(hP) < 1e-24)   # |S|^2 of zero flows
    Sg = np.zeros(g.nb)
    np.add.at(Sg, g.gbus, x[2 * g.nb:2 * g.nb + g.ng])
    np.testing.assert_allclose(r0["gh"][:g.nb], g.Pd - Sg, atol=1e-13)
    r = gh_of(oracle_mod, net, x, np.zeros(g.m))
    # h = Pf^2 + Qf^2 with Pf = 0, Qf = -b/2
    np.testing.assert_allclose(r["gh"][2 * g.nb:2 * g.nb + g.nl], (g.b / 2) ** 2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["gh"][2 * g.nb + g.nl:], (g.b / 2) ** 2, rtol=1e-12, atol=1e-15)


def test_objective_hand_numbers(oracle_mod):
    """c2 (100 Pg)^2 + c1 (100 Pg): 0.01*150^2 + 20*150 = 3225; d/dPg = 2300; d2 = 200 (x sigma w)."""
    g = tiny_grid(2, [(0, 1)], [(0.01, 0.1, 0.0, 0.0)], [(0, 0.01, 20.0), (1, 0.002, 35.0)])
    net = oracle_mod.OracleNet(g)
    x = pack_x(g, np.zeros(2), np.ones(2), np.array([1.5, -0.2]), np.zeros(2))
    r = oracle_mod.evaluate(net, x, np.zeros(g.m), obj_weight=0.5, sigma=3.0)
    # gen 2: 0.002*(-20)^2 + 35*(-20) = 0.8 - 700 = -699.2
    assert r["f"] == pytest.approx(0.5 * (3225.0 - 699.2), rel=1e-15)
    assert r["grad"][4] == pytest.approx(0.5 * 2300.0, rel=1e-15)
    assert r["grad"][5] == pytest.approx(0.5 * (2 * 0.002 * 1e4 * -0.2 + 3500.0), rel=1e-15)
    rowptr, col, val = r["H"]
    d = {(i, c): v for i in range(g.n) for c, v in zip(col[rowptr[i]:rowptr[i + 1]], val[rowptr[i]:rowptr[i + 1]])}
    assert d[(4, 4)] == pytest.approx(3.0 * 0.5 * 200.0, rel=1e-15)
    assert d[(5, 5)] == pytest.approx(3.0 * 0.5 * 40.0, rel=1e-15)


# ---- independent formulation --------------------------------------------------------------------

@pytest.mark.parametrize("seed,nb,nl,ng,shifters", [(21, 3, 3, 1, 0.0), (22, 30, 41, 6, 0.0),
                                                    (23, 200, 260, 50, 0.0),
                                                    (24, 60, 80, 12, 0.25)])
def test_matches_complex_nodal_form(oracle_mod, seed, nb, nl, ng, shifters):
    """The last case has phase-shifting transformers on a quarter of its branches: the nodal form
    then carries the complex tap ratio T = tau e^{j phi} of each."""
    g = synth.make_grid(seed, nb, nl, ng, shunts=True, shifter_frac=shifters)
    if nb == 3:
        g.tap[1] = 0.97   # 3-bus triangle with a transformer
    b = synth.random_batch(seed, g, 1, masks=True, pd_scale=True)
    net = oracle_mod.OracleNet(g)
    r = gh_of(oracle_mod, net, b.x[0], b.lam[0], b.mask[0], b.pd_scale[0])
    c = complex_model(g, b.x[0], b.mask[0], b.pd_scale[0])
    np.testing.assert_allclose(r["gh"][:nb], c["gP"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["gh"][nb:2 * nb], c["gQ"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["gh"][2 * nb:2 * nb + nl], np.abs(c["Sf"]) ** 2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["gh"][2 * nb + nl:], np.abs(c["St"]) ** 2, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("shifters", [0.0, 0.3])
def test_loss_invariant(oracle_mod, shifters):
    """Net injections sum to the series losses gs |V_f e^{j Va_f}/T - V_t e^{j Va_t}|^2 >= 0,
    T = tau e^{j phi} (an ideal phase-shifting transformer moves power without loss)."""
    g = synth.make_grid(31, 60, 80, 12, shunts=True, shifter_frac=shifters)
    b = synth.random_batch(31, g, 1, masks=True)
    x, mask = b.x[0], b.mask[0]
    r = gh_of(oracle_mod, oracle_mod.OracleNet(g), x, b.lam[0], mask)
    nb, ng = g.nb, g.ng
    Vm, Pg = x[nb:2 * nb], x[2 * nb:2 * nb + ng]
    lhs = r["gh"][:nb].sum() - g.Pd.sum() - (g.Gs * Vm ** 2).sum() + Pg.sum()
    V = Vm * np.exp(1j * x[:nb])
    gs = (1.0 / (g.r + 1j * g.x)).real
    tau = np.where(g.tap == 0.0, 1.0, g.tap)
    T = tau * np.exp(1j * (np.zeros(g.nl) if g.shift is None else g.shift))
    loss = mask * gs * np.abs(V[g.f] / T - V[g.t]) ** 2
    assert np.all(loss >= 0)
    assert lhs == pytest.approx(loss.sum(), rel=1e-11)


# ---- finite differences ---------------------------------------------------------------------

def _fd_check(oracle_mod, g, b, sigma=1.0, h=1e-6):
    net = oracle_mod.OracleNet(g)
    x, lam = b.x[0].copy(), b.lam[0]
    mask = None if b.mask is None else b.mask[0]
    ps = None if b.pd_scale is None else b.pd_scale[0]
    w = 1.0 if b.obj_weight is None else float(b.obj_weight[0])
    r = oracle_mod.evaluate(net, x, lam, mask, ps, w, sigma)
    n, m = g.n, g.m
    J = oracle_mod.csr_to_dense(r["J"], (m, n))
    Hl = oracle_mod.csr_to_dense(r["H"], (n, n))
    H = Hl + np.tril(Hl, -1).T
    Jfd = np.zeros((m, n))
    gfd = np.zeros(n)
    Hfd = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        rp = oracle_mod.evaluate(net, x + e, lam, mask, ps, w, sigma, want_hess=True)
        rm = oracle_mod.evaluate(net, x - e, lam, mask, ps, w, sigma, want_hess=True)
        Jfd[:, k] = (rp["gh"] - rm["gh"]) / (2 * h)
        gfd[k] = (rp["f"] - rm["f"]) / (2 * h)
        # gradient of the Lagrangian: sigma grad f + J' lam
        Lp = sigma * rp["grad"] + oracle_mod.csr_to_dense(rp["J"], (m, n)).T @ lam
        Lm = sigma * rm["grad"] + oracle_mod.csr_to_dense(rm["J"], (m, n)).T @ lam
        Hfd[:, k] = (Lp - Lm) / (2 * h)
    scale = lambda A: np.maximum(1.0, np.abs(A))
    assert np.max(np.abs(J - Jfd) / scale(J)) < 1e-6
    assert np.max(np.abs(r["grad"] - gfd) / scale(r["grad"])) < 1e-6
    assert np.max(np.abs(H - Hfd) / scale(H)) < 1e-5
    # the FD Hessian is symmetric, so the oracle's lower triangle stands for both halves
    assert np.max(np.abs(Hfd - Hfd.T) / scale(H)) < 1e-5
    return r


@pytest.mark.parametrize("seed", [41, 42])
def test_finite_differences(oracle_mod, seed):
    g = synth.make_grid(seed, 14, 20, 4, shunts=True)
    b = synth.random_batch(seed, g, 1, masks=True, pd_scale=True, obj_weight=True)
    _fd_check(oracle_mod, g, b, sigma=0.7)


def test_finite_differences_sigma_zero_and_transformers(oracle_mod):
    g = synth.make_grid(43, 10, 14, 3, transformer_frac=0.5, shunts=True)
    b = synth.random_batch(43, g, 1)
    _fd_check(oracle_mod, g, b, sigma=0.0)


def test_finite_differences_phase_shifters(oracle_mod):
    g = synth.make_grid(44, 12, 17, 3, shunts=True, shifter_frac=0.4)
    b = synth.random_batch(44, g, 1, masks=True, pd_scale=True)
    _fd_check(oracle_mod, g, b, sigma=0.9)


# ---- symmetries of the model ----------------------------------------------------------------

def test_homogeneity_and_angle_invariance(oracle_mod):
    """Two symmetries of the polar model (Sec. III, eqs. (8)-(9)) tie J and H together:
      * shifting every angle by one amount changes nothing, so every row of J and of H sums to
        zero over the angle columns;
      * the injections are homogeneous of degree 2 in the voltage magnitudes and |S|^2 of degree
        4, so (Euler) sum_k Vm_k dg_i/dVm_k = 2 (g_i less load and generation) and
        sum_k Vm_k dh_l/dVm_k = 4 h_l; differentiated once more, the Lagrangian Hessian's
        Vm-weighted rows are (1 lam_g + 3 lam_h) J on Vm rows and (2 lam_g + 4 lam_h) J on Va rows.
    The bus balances in the CUDA path rest on the degree-2 identity."""
    g = synth.make_grid(61, 40, 56, 9, transformer_frac=0.3, shunts=True)
    b = synth.random_batch(61, g, 1, masks=True, pd_scale=True, obj_weight=True, sigma=0.6)
    x, lam, mask, ps = b.x[0], b.lam[0], b.mask[0], b.pd_scale[0]
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), x, lam, mask, ps, float(b.obj_weight[0]), 0.6)
    nb, nl, n, m = g.nb, g.nl, g.n, g.m
    J = oracle_mod.csr_to_dense(r["J"], (m, n))
    Hl = oracle_mod.csr_to_dense(r["H"], (n, n))
    H = Hl + np.tril(Hl, -1).T
    Vm = x[nb:2 * nb]
    va, vm = slice(0, nb), slice(nb, 2 * nb)
    scale = np.abs(J[:, :2 * nb]).max(axis=1) * np.maximum(1.0, Vm.max())
    np.testing.assert_allclose(J[:, va].sum(axis=1), 0.0, atol=1e-12 * scale.max())
    Hs = np.abs(H[:2 * nb, :2 * nb]).max()
    np.testing.assert_allclose(H[:2 * nb, va].sum(axis=1), 0.0, atol=1e-12 * Hs)
    # injections: balances less load and generation
    Pg, Qg = x[2 * nb:2 * nb + g.ng], x[2 * nb + g.ng:]
    SgP = np.bincount(g.gbus, weights=Pg, minlength=nb)
    SgQ = np.bincount(g.gbus, weights=Qg, minlength=nb)
    inj = np.concatenate([r["gh"][:nb] - g.Pd * ps + SgP, r["gh"][nb:2 * nb] - g.Qd * ps + SgQ])
    deg = np.concatenate([2.0 * inj, 4.0 * r["gh"][2 * nb:]])
    np.testing.assert_allclose(J[:, vm] @ Vm, deg, rtol=1e-11, atol=1e-11 * scale.max())
    lg = lam.copy(); lg[2 * nb:] = 0.0
    lh = lam.copy(); lh[:2 * nb] = 0.0
    np.testing.assert_allclose(H[vm, vm] @ Vm, (J.T @ (lg + 3.0 * lh))[vm], rtol=1e-10, atol=1e-11 * Hs)
    np.testing.assert_allclose(H[va, vm] @ Vm, (J.T @ (2.0 * lg + 4.0 * lh))[va], rtol=1e-10,
                               atol=1e-11 * Hs)


# ---- masks, structure, batch --------------------------------------------------------------------

def test_mask_equals_branch_removed(oracle_mod):
    g = synth.make_grid(51, 20, 28, 5, shunts=True)
    b = synth.random_batch(51, g, 1)
    k = 7
    mask = np.ones(g.nl, np.uint8)
    mask[k] = 0
    keep = np.arange(g.nl) != k
    g2 = synth.Grid(**{**g.__dict__, "f": g.f[keep], "t": g.t[keep], "r": g.r[keep],
                       "x": g.x[keep], "b": g.b[keep], "tap": g.tap[keep], "rateA": g.rateA[keep]})
    nb, nl = g.nb, g.nl
    lam = b.lam[0]
    lam2 = np.concatenate([lam[:2 * nb], lam[2 * nb:2 * nb + nl][keep], lam[2 * nb + nl:][keep]])
    r1 = oracle_mod.evaluate(oracle_mod.OracleNet(g), b.x[0], lam, mask)
    r2 = oracle_mod.evaluate(oracle_mod.OracleNet(g2), b.x[0], lam2)
    rows = np.concatenate([np.arange(2 * nb), 2 * nb + np.flatnonzero(keep), 2 * nb + nl + np.flatnonzero(keep)])
    np.testing.assert_array_equal(r1["gh"][rows], r2["gh"])
    assert r1["gh"][2 * nb + k] == 0.0 and r1["gh"][2 * nb + nl + k] == 0.0
    J1 = oracle_mod.csr_to_dense(r1["J"], (g.m, g.n))
    J2 = oracle_mod.csr_to_dense(r2["J"], (g2.m, g2.n))
    np.testing.assert_allclose(J1[rows], J2, rtol=0, atol=1e-12)
    assert np.all(J1[[2 * nb + k, 2 * nb + nl + k]] == 0.0)
    np.testing.assert_allclose(oracle_mod.csr_to_dense(r1["H"], (g.n, g.n)),
                               oracle_mod.csr_to_dense(r2["H"], (g.n, g.n)), rtol=0, atol=1e-11)


def test_nonzero_counts(oracle_mod):
    g = synth.grid_30bus()
    b = synth.random_batch(1, g, 1)
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), b.x[0], b.lam[0])
    assert r["J"][0][-1] == 4 * g.nb + 16 * g.nl + 2 * g.ng == 788
    assert r["H"][0][-1] == 3 * g.nb + 4 * g.nl + g.ng == 260
    # lower triangle, ascending columns
    rowptr, col, _ = r["H"]
    for i in range(g.n):
        c = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(c <= i) and np.all(np.diff(c) > 0)


def test_parallel_branches_and_shared_gen_bus(oracle_mod):
    """Two parallel lines and two generators on one bus: duplicates merge into one nonzero."""
    g = tiny_grid(3, [(0, 1), (1, 0), (1, 2)],
                  [(0.01, 0.1, 0.02, 0.0), (0.02, 0.15, 0.01, 0.98), (0.015, 0.12, 0.0, 0.0)],
                  [(0, 0.01, 20.0), (0, 0.02, 25.0), (2, 0.005, 30.0)], Pd=[0.1, 0.5, 0.4],
                  Gs=[0.01, 0.0, 0.02], Bs=[0.0, 0.05, 0.0])
    b = synth.random_batch(3, g, 1, masks=False)
    r = _fd_check(oracle_mod, g, b)
    c = complex_model(g, b.x[0])
    np.testing.assert_allclose(r["gh"][:3], c["gP"], rtol=1e-12, atol=1e-12)
    # J: P0 row = Va0, Va1, Vm0, Vm1, Pg0, Pg1 (parallel lines share Va1, Vm1)
    rowptr, col, _ = r["J"]
    assert list(col[rowptr[0]:rowptr[1]]) == [0, 1, 3, 4, 6, 7]
