"""Pins of the oracle's power-balance-cartesian formulation (no GPU).

Sec. III names two representations of the ACOPF equations, power-balance-polar and
power-balance-cartesian.  The cartesian oracle (oracle_eval_cart) evaluates the same network with
V_i = e_i + j f_i and the voltage-magnitude rows e^2 + f^2.  Its pins:
  * the complex nodal form S = V conj(Ybus V) and the branch flows V_f conj(I_f), evaluated in
    complex arithmetic straight from e + j f (no oracle code);
  * the change of variables to the polar model: at e = Vm cos Va, f = Vm sin Va the constraint
    values equal the polar oracle's, the voltage rows equal Vm^2, the Jacobians satisfy
    J_polar = J_cart M with M = d(e, f) / d(Va, Vm), and the Lagrangian Hessians satisfy
    H_polar = M' H_cart M + sum_i (dL/de_i) grad^2 e_i + (dL/df_i) grad^2 f_i;
  * central finite differences: J against g | h, and the Hessian against sigma grad f + J' lam;
  * homogeneity: the branch and shunt terms are quadratic forms in (e, f), so J_ef (e, f) = 2 g
    and H_ef (e, f) = (J' lam)_ef when loads, generation, mu and sigma vanish;
  * rotating every voltage by one angle leaves g and h unchanged;
  * an out-of-service branch equals the branch removed from the grid;
  * the nonzero counts 6 nb + 16 nl + 2 ng (J) and 3 nb + 4 nl + ng (lower Hessian).
test_oracle_mutants.py plants sign, index and factor mistakes in the cartesian code and checks
that these pins catch each one.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from test_oracle import complex_model


def dense(om, csr, shape):
    return om.csr_to_dense(csr, shape)


def sym(L):
    return L + L.T - np.diag(np.diag(L))


def cart_state(g, rng, sigma_va=0.1):
    Va = rng.normal(0.0, sigma_va, g.nb)
    Vm = rng.uniform(0.95, 1.05, g.nb)
    Pg = rng.uniform(0.0, 2.0, g.ng)
    Qg = rng.uniform(-0.5, 0.5, g.ng)
    xp = np.concatenate([Va, Vm, Pg, Qg])
    xc = np.concatenate([Vm * np.cos(Va), Vm * np.sin(Va), Pg, Qg])
    return xp, xc


def grid_with_shunts(seed=51):
    return synth.make_grid(seed, 30, 41, 6, transformer_frac=0.3, shunts=True)


def test_matches_complex_nodal_form(oracle_mod):
    g = grid_with_shunts()
    rng = np.random.default_rng(52)
    xp, xc = cart_state(g, rng)
    ps = rng.uniform(0.8, 1.2, g.nb)
    mask = np.ones(g.nl, np.uint8)
    mask[[3, 17]] = 0
    net = oracle_mod.OracleNet(g)
    lam = np.zeros(g.m + g.nb)
    r = oracle_mod.evaluate(net, xc, lam, mask, ps, want_jac=False, want_hess=False,
                            cartesian=True)
    cm = complex_model(g, xp, mask, ps)
    nb, nl = g.nb, g.nl
    gh = r["gh"]
    np.testing.assert_allclose(gh[:nb], cm["gP"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(gh[nb:2 * nb], cm["gQ"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(gh[2 * nb:2 * nb + nl], np.abs(cm["Sf"]) ** 2, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(gh[2 * nb + nl:2 * nb + 2 * nl], np.abs(cm["St"]) ** 2, rtol=1e-12,
                               atol=1e-13)
    np.testing.assert_allclose(gh[2 * nb + 2 * nl:], np.abs(cm["V"]) ** 2, rtol=1e-14)


def change_of_variables(g, xp):
    """M = d(e, f, Pg, Qg) / d(Va, Vm, Pg, Qg) and the second derivatives of e_i, f_i."""
    nb, n = g.nb, g.n
    Va, Vm = xp[:nb], xp[nb:2 * nb]
    M = np.eye(n)
    i = np.arange(nb)
    M[i, i] = -Vm * np.sin(Va)            # de/dVa
    M[i, nb + i] = np.cos(Va)             # de/dVm
    M[nb + i, i] = Vm * np.cos(Va)        # df/dVa
    M[nb + i, nb + i] = np.sin(Va)        # df/dVm
    return M, Va, Vm


@pytest.mark.parametrize("seed", [53, 54])
def test_change_of_variables_to_polar(oracle_mod, seed):
    change_of_variables_check(oracle_mod, grid_with_shunts(seed), seed)


def change_of_variables_check(oracle_mod, g, seed):
    rng = np.random.default_rng(seed)
    xp, xc = cart_state(g, rng)
    lam_p = rng.normal(size=g.m)
    mask = np.ones(g.nl, np.uint8)
    mask[5] = 0
    sigma = 0.8
    net = oracle_mod.OracleNet(g)
    lam_c = np.concatenate([lam_p, np.zeros(g.nb)])     # no voltage rows in the polar model
    rp = oracle_mod.evaluate(net, xp, lam_p, mask, None, 1.3, sigma)
    rc = oracle_mod.evaluate(net, xc, lam_c, mask, None, 1.3, sigma, cartesian=True)
    nb, n, m = g.nb, g.n, g.m
    # values
    np.testing.assert_allclose(rc["gh"][:m], rp["gh"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(rc["gh"][m:], xp[nb:2 * nb] ** 2, rtol=1e-14)
    assert rc["f"] == rp["f"]
    np.testing.assert_array_equal(rc["grad"], rp["grad"])
    # Jacobian: chain rule
    Jc = dense(oracle_mod, rc["J"], (m + nb, n))
    Jp = dense(oracle_mod, rp["J"], (m, n))
    M, Va, Vm = change_of_variables(g, xp)
    np.testing.assert_allclose(Jc[:m] @ M, Jp, rtol=0, atol=1e-10)
    np.testing.assert_allclose((Jc[m:] @ M)[:, :nb], 0.0, atol=1e-14)                 # angle
    np.testing.assert_allclose((Jc[m:] @ M)[:, nb:2 * nb], np.diag(2 * Vm), atol=1e-13)
    # Lagrangian Hessian: second-order chain rule
    Hc = sym(dense(oracle_mod, rc["H"], (n, n)))
    Hp = sym(dense(oracle_mod, rp["H"], (n, n)))
    gL = Jc.T @ lam_c            # dL/d(e, f) (the objective has no voltage terms)
    extra = np.zeros((n, n))
    for i in range(nb):
        de, df = gL[i], gL[nb + i]
        a, v = i, nb + i         # (Va_i, Vm_i)
        # grad^2 e_i over (Va_i, Vm_i) = [[-Vm cos, -sin], [-sin, 0]];
        # grad^2 f_i = [[-Vm sin, cos], [cos, 0]]
        extra[a, a] += de * (-Vm[i] * np.cos(Va[i])) + df * (-Vm[i] * np.sin(Va[i]))
        extra[a, v] += de * (-np.sin(Va[i])) + df * np.cos(Va[i])
        extra[v, a] = extra[a, v]
    np.testing.assert_allclose(M.T @ Hc @ M + extra, Hp, rtol=0, atol=1e-9)


def test_finite_differences(oracle_mod):
    g = grid_with_shunts(55)
    rng = np.random.default_rng(55)
    _, x = cart_state(g, rng)
    m = g.m + g.nb
    lam = rng.normal(size=m)
    sigma = 0.7
    net = oracle_mod.OracleNet(g)
    r = oracle_mod.evaluate(net, x, lam, None, None, 1.0, sigma, cartesian=True)
    J = dense(oracle_mod, r["J"], (m, g.n))
    H = sym(dense(oracle_mod, r["H"], (g.n, g.n)))
    h = 1e-6
    for j in range(g.n):
        xp_, xm_ = x.copy(), x.copy()
        xp_[j] += h
        xm_[j] -= h
        rp = oracle_mod.evaluate(net, xp_, lam, None, None, 1.0, sigma, cartesian=True)
        rm = oracle_mod.evaluate(net, xm_, lam, None, None, 1.0, sigma, cartesian=True)
        col = (rp["gh"] - rm["gh"]) / (2 * h)
        np.testing.assert_allclose(J[:, j], col, rtol=1e-6, atol=1e-6)
        gLp = sigma * rp["grad"] + dense(oracle_mod, rp["J"], (m, g.n)).T @ lam
        gLm = sigma * rm["grad"] + dense(oracle_mod, rm["J"], (m, g.n)).T @ lam
        np.testing.assert_allclose(H[:, j], (gLp - gLm) / (2 * h), rtol=1e-6, atol=1e-5)


def test_homogeneity_and_rotation(oracle_mod):
    g = grid_with_shunts(56)
    g.Pd[:] = 0.0
    g.Qd[:] = 0.0
    rng = np.random.default_rng(56)
    _, x = cart_state(g, rng)
    x[2 * g.nb:] = 0.0                          # no generation
    nb, nl, m = g.nb, g.nl, g.m + g.nb
    lam = np.concatenate([rng.normal(size=2 * nb), np.zeros(2 * nl + nb)])   # lambda on g only
    net = oracle_mod.OracleNet(g)
    r = oracle_mod.evaluate(net, x, lam, None, None, 1.0, 0.0, cartesian=True)
    J = dense(oracle_mod, r["J"], (m, g.n))
    H = sym(dense(oracle_mod, r["H"], (g.n, g.n)))
    ef = x[:2 * nb]
    np.testing.assert_allclose(J[:2 * nb, :2 * nb] @ ef, 2 * r["gh"][:2 * nb], rtol=0, atol=1e-11)
    np.testing.assert_allclose(J[2 * nb + 2 * nl:, :2 * nb] @ ef, 2 * r["gh"][2 * nb + 2 * nl:],
                               rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(H[:2 * nb, :2 * nb] @ ef, (J.T @ lam)[:2 * nb], rtol=0, atol=1e-11)
    # rotate every voltage by phi
    phi = 0.37
    V = (x[:nb] + 1j * x[nb:2 * nb]) * np.exp(1j * phi)
    xr = x.copy()
    xr[:nb], xr[nb:2 * nb] = V.real, V.imag
    rr = oracle_mod.evaluate(net, xr, lam, None, None, 1.0, 0.0, want_jac=False, want_hess=False,
                             cartesian=True)
    np.testing.assert_allclose(rr["gh"], r["gh"], rtol=1e-12, atol=1e-12)


def test_mask_equals_branch_removed(oracle_mod):
    g = grid_with_shunts(57)
    rng = np.random.default_rng(57)
    _, x = cart_state(g, rng)
    off = [2, 9, 30]
    mask = np.ones(g.nl, np.uint8)
    mask[off] = 0
    keep = np.setdiff1d(np.arange(g.nl), off)
    g2 = synth.Grid(**{**g.__dict__, "f": g.f[keep], "t": g.t[keep], "r": g.r[keep],
                       "x": g.x[keep], "b": g.b[keep], "tap": g.tap[keep],
                       "rateA": g.rateA[keep]})
    m, m2 = g.m + g.nb, g2.m + g2.nb
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), x, np.zeros(m), mask, want_jac=False,
                            want_hess=False, cartesian=True)
    r2 = oracle_mod.evaluate(oracle_mod.OracleNet(g2), x, np.zeros(m2), want_jac=False,
                             want_hess=False, cartesian=True)
    nb, nl = g.nb, g.nl
    np.testing.assert_array_equal(r["gh"][:2 * nb], r2["gh"][:2 * nb])
    np.testing.assert_array_equal(r["gh"][2 * nb:2 * nb + nl][keep], r2["gh"][2 * nb:2 * nb + g2.nl])
    np.testing.assert_array_equal(r["gh"][2 * nb:2 * nb + nl][off], 0.0)
    np.testing.assert_array_equal(r["gh"][2 * nb + 2 * nl:], r2["gh"][2 * nb + 2 * g2.nl:])


def test_nonzero_counts(oracle_mod):
    g = synth.make_grid(58, 40, 55, 9)
    rng = np.random.default_rng(58)
    _, x = cart_state(g, rng)
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), x, rng.normal(size=g.m + g.nb),
                            cartesian=True)
    assert r["J"][0][-1] == 6 * g.nb + 16 * g.nl + 2 * g.ng
    assert r["H"][0][-1] == 3 * g.nb + 4 * g.nl + g.ng
