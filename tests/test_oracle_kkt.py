"""Pins of the KKT-step and power-flow Newton oracle (oracle/kkt.py; CPU only).

KKT step, K [dx; dlam] = r with K = [[W + diag(dx), J'], [J, -diag(dc)]]:
  * a one-variable, one-row system solved by hand (2 x 2 inverse);
  * K assembled densely as blocks from the dense J and W (no shared code with kkt_matrix) and
    solved with a dense LU, on a 30-bus grid;
  * the normal-equations form of the same step, dx = (W + Dx + J' Dc^-1 J)^-1 (r_x + J' Dc^-1 r_c)
    and dlam = Dc^-1 (J dx - r_c), on a 300-bus grid;
  * Sylvester's law of inertia: with W + Dx positive definite and dc > 0, K has exactly m negative
    eigenvalues.
Power-flow Newton step:
  * a two-bus case by hand (lossless line, flat start);
  * iterated from a flat start it converges quadratically to a point whose balances, recomputed
    in complex arithmetic (S = V conj(Ybus V)), vanish at every equation row;
  * the slack bus's Va and Vm and the PV buses' Vm stay fixed.
test_oracle_kkt_mutants below plants plausible mistakes in copies of the module and checks that
each one fails at least one of these pins.

Input recipe of the KKT cases: J and W from the model oracle at seeded states, dx_i = 1 + the
sum of |W_ij| over row i (so W + Dx is strictly diagonally dominant, hence positive definite),
dc ~ U(0.5, 2), r ~ N(0, 1).
"""
import importlib.util
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2203_10587_gb300 import synth
from test_oracle import complex_model, tiny_grid

KKT_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                       "kkt.py")


@pytest.fixture(scope="module")
def kkt():
    from oracle import kkt as K
    return K


def sym_dense(om, H, n):
    L = om.csr_to_dense(H, (n, n))
    return L + np.tril(L, -1).T


def kkt_inputs(om, g, seed, sigma=0.8):
    b = synth.random_batch(seed, g, 1, masks=True, sigma=sigma)
    r = om.evaluate(om.OracleNet(g), b.x[0], b.lam[0], b.mask[0], None, 1.0, sigma)
    W = sym_dense(om, r["H"], g.n)
    rng = np.random.default_rng(seed)
    dx = 1.0 + np.abs(W).sum(axis=1)
    dc = rng.uniform(0.5, 2.0, g.m)
    rhs = rng.normal(size=g.n + g.m)
    return r, W, dx, dc, rhs


def test_one_by_one_by_hand(kkt):
    """n = m = 1: [[w + dx, j], [j, -dc]] [a; l] = [r1; r2]; determinant -(w+dx) dc - j^2."""
    w, dx, j, dc, r1, r2 = 3.0, 0.5, 2.0, 0.25, 1.0, -2.0
    H = (np.array([0, 1]), np.array([0]), np.array([w]))
    J = (np.array([0, 1]), np.array([0]), np.array([j]))
    s = kkt.kkt_solve(1, 1, J, H, np.array([dx]), np.array([dc]), np.array([r1, r2]))
    det = -(w + dx) * dc - j * j
    assert s[0] == pytest.approx((-dc * r1 - j * r2) / det, rel=1e-14)
    assert s[1] == pytest.approx(((w + dx) * r2 - j * r1) / det, rel=1e-14)


def test_dense_block_solve_30bus(kkt, oracle_mod):
    g = synth.grid_30bus()
    r, W, dx, dc, rhs = kkt_inputs(oracle_mod, g, 1)
    Jd = oracle_mod.csr_to_dense(r["J"], (g.m, g.n))
    K = np.block([[W + np.diag(dx), Jd.T], [Jd, -np.diag(dc)]])
    want = np.linalg.solve(K, rhs)
    got = kkt.kkt_solve(g.n, g.m, r["J"], r["H"], dx, dc, rhs)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())


def test_normal_equations_form_300bus(kkt, oracle_mod):
    g = synth.make_grid(13, 300, 389, 77, transformer_frac=0.3, shunts=True)
    r, W, dx, dc, rhs = kkt_inputs(oracle_mod, g, 13)
    n, m = g.n, g.m
    jp, jc, jv = r["J"]
    Js = sp.csr_matrix((jv, jc, jp), shape=(m, n))
    rx, rc = rhs[:n], rhs[n:]
    S = sp.csr_matrix(W) + sp.diags(dx) + Js.T @ sp.diags(1.0 / dc) @ Js
    import scipy.sparse.linalg as sla
    ddx = sla.spsolve(S.tocsc(), rx + Js.T @ (rc / dc))
    dlam = (Js @ ddx - rc) / dc
    got = kkt.kkt_solve(n, m, r["J"], r["H"], dx, dc, rhs)
    scale = np.abs(got).max()
    np.testing.assert_allclose(got[:n], ddx, rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(got[n:], dlam, rtol=0, atol=1e-10 * scale)


def test_inertia_of_quasidefinite_kkt(kkt, oracle_mod):
    g = synth.make_grid(17, 40, 52, 9, shunts=True)
    r, W, dx, dc, rhs = kkt_inputs(oracle_mod, g, 17)
    K = kkt.kkt_matrix(g.n, g.m, r["J"], r["H"], dx, dc).toarray()
    np.testing.assert_array_equal(K, K.T)
    ev = np.linalg.eigvalsh(K)
    assert int((ev < 0).sum()) == g.m and int((ev > 0).sum()) == g.n


# ---- power flow -------------------------------------------------------------------------------

def test_pf_two_bus_by_hand(kkt, oracle_mod):
    """Slack bus 0 (V = 1, Va = 0), PQ bus 1 with load 0.5 + j 0.2 behind a lossless line x = 0.1:
    at flat start g = [0.5, 0.2] and J = diag(10, 10), so the step is (-0.05, -0.02)."""
    g = tiny_grid(2, [(0, 1)], [(0.0, 0.1, 0.0, 0.0)], [(0, 0.01, 20.0)], Pd=[0.0, 0.5],
                  Qd=[0.0, 0.2])
    x = np.array([0.0, 0.0, 1.0, 1.0, 0.0, 0.0])
    x1, mis = kkt.pf_newton_step(oracle_mod, oracle_mod.OracleNet(g), x, [3, 1])
    assert mis == pytest.approx(0.5, rel=1e-15)
    np.testing.assert_allclose(x1[[1, 3]], [-0.05, 0.98], rtol=1e-14)
    np.testing.assert_array_equal(x1[[0, 2, 4, 5]], x[[0, 2, 4, 5]])


def pf_case(seed, nb, nl, ng):
    g = synth.make_grid(seed, nb, nl, ng, transformer_frac=0.2, shunts=True)
    g.Pd *= 0.3
    g.Qd *= 0.3
    rng = np.random.default_rng(seed)
    bus_type = np.ones(g.nb, np.int32)
    bus_type[g.gbus] = 2
    bus_type[g.gbus[0]] = 3
    Pg = np.full(g.ng, g.Pd.sum() / g.ng)          # balanced dispatch, the slack takes the losses
    Qg = np.zeros(g.ng)
    Vm = np.ones(g.nb)
    Vm[g.gbus] = rng.uniform(0.98, 1.04, g.ng)     # PV set points
    x = np.concatenate([np.zeros(g.nb), Vm, Pg, Qg])
    return g, bus_type, x


@pytest.mark.parametrize("seed,nb,nl,ng", [(31, 30, 41, 6), (32, 300, 389, 60)])
def test_pf_converges_quadratically_to_a_power_flow_solution(kkt, oracle_mod, seed, nb, nl, ng):
    g, bt, x = pf_case(seed, nb, nl, ng)
    net = oracle_mod.OracleNet(g)
    x0 = x.copy()
    mis = []
    for _ in range(8):
        x, e = kkt.pf_newton_step(oracle_mod, net, x, bt)
        mis.append(e)
        if e < 1e-13:
            break
    assert mis[-1] < 1e-11, mis
    # quadratic rate once close: e_{k+1} <= C e_k^2
    for a, b in zip(mis[1:-1], mis[2:]):
        if a < 1e-2:
            assert b <= 50.0 * a * a + 1e-13, mis
    # the balances vanish at the solution, recomputed in complex arithmetic: P at every non-slack
    # bus, Q at every PQ bus (sets taken from the bus types here, not from the oracle)
    nb = g.nb
    rows = np.concatenate([np.flatnonzero(bt != 3), nb + np.flatnonzero(bt == 1)])
    cm = complex_model(g, x)
    gb = np.concatenate([cm["gP"], cm["gQ"]])
    np.testing.assert_allclose(gb[rows], 0.0, atol=1e-10)
    # the slack bus's Va and Vm, the PV buses' Vm, Pg and Qg did not move
    fixed = np.concatenate([np.flatnonzero(bt == 3), nb + np.flatnonzero(bt != 1),
                            np.arange(2 * nb, g.n)])
    np.testing.assert_array_equal(x[fixed], x0[fixed])


# ---- mutants ------------------------------------------------------------------------------------

MUTANTS = {
    "upper_W_dropped": ("            if j != i:\n                rows.append(j); cols.append(i); vals.append(hv[k])\n", ""),
    "dc_sign": ("vals.append(-dc[r])", "vals.append(dc[r])"),
    "transpose_dropped": ("            rows.append(j); cols.append(n + r); vals.append(jv[k])\n", ""),
    "dx_dropped": ("rows.append(i); cols.append(i); vals.append(dx[i])", "rows.append(i); cols.append(i); vals.append(0.0)"),
    "dx_on_constraints": ("rows.append(i); cols.append(i); vals.append(dx[i])", "rows.append(n + i); cols.append(n + i); vals.append(dx[i])"),
    "pf_step_sign": ("sla.spsolve(Jpf, -gpf)", "sla.spsolve(Jpf, gpf)"),
    "pf_pv_vm_free": ("pq = np.flatnonzero(bt == 1)", "pq = np.flatnonzero(bt != 3)"),
    "pf_slack_angle_free": ("ns = np.flatnonzero(bt != 3)", "ns = np.arange(bt.shape[0])"),
}


def load_copy(tmp_path, name, src):
    path = tmp_path / f"kkt_{name}.py"
    path.write_text(src)
    spec = importlib.util.spec_from_file_location(f"kkt_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PINS = [
    ("hand", lambda K, om: test_one_by_one_by_hand(K)),
    ("dense", lambda K, om: test_dense_block_solve_30bus(K, om)),
    ("normal", lambda K, om: test_normal_equations_form_300bus(K, om)),
    ("inertia", lambda K, om: test_inertia_of_quasidefinite_kkt(K, om)),
    ("pf_hand", lambda K, om: test_pf_two_bus_by_hand(K, om)),
    ("pf_converges", lambda K, om: test_pf_converges_quadratically_to_a_power_flow_solution(K, om, 31, 30, 41, 6)),
]


def test_unmutated_copy_passes_all_pins(tmp_path, oracle_mod):
    K = load_copy(tmp_path, "good", open(KKT_SRC).read())
    for _, pin in PINS:
        pin(K, oracle_mod)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_oracle_kkt_mutants(tmp_path, oracle_mod, name):
    old, new = MUTANTS[name]
    src = open(KKT_SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    K = load_copy(tmp_path, name, src.replace(old, new))
    caught = []
    for pname, pin in PINS:
        try:
            pin(K, oracle_mod)
        except (AssertionError, ValueError, np.linalg.LinAlgError, RuntimeError):
            caught.append(pname)
    assert caught, f"mutant {name} passed every pin"
