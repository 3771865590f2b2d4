"""Pins of the oracle's phase-shifting transformers (no GPU).

A phase-shifting transformer puts an ideal transformer of complex ratio T = tau e^{j phi} on the
from side of a branch's pi-model (the textbook and MATPOWER branch model), so the two mutual
admittances become -ys/conj(T) and -ys/T and differ.  Sec. III of the paper names the model's
network features without equations; these pins fix the oracle's reading against things other
than its own code:
  * the textbook flow of a lossless phase shifter, P = (V1/tau) V2 sin(d - phi) / x;
  * the physics of the ideal transformer: the branch's flows, and so every output of a one-branch
    grid (g, h, J, Lagrangian Hessian), equal those of the same branch without shift seen from a
    from-bus angle rotated by -phi;
  * zero shift reproduces the shift-free model bit for bit;
  * the complex nodal form, the loss invariant and central finite differences with shifts
    (test_oracle.py, parametrised), and the cartesian formulation's change of variables to the
    polar one on a grid with shifters.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from test_oracle import pack_x, tiny_grid


def one_branch(r, x, b, tau, phi):
    g = tiny_grid(2, [(0, 1)], [(r, x, b, tau)], [(0, 0.01, 20.0)], Gs=[0.02, 0.0], Bs=[0.0, -0.03],
                  Pd=[0.0, 0.4], Qd=[0.0, 0.1])
    g.shift = np.array([phi])
    return g


def test_lossless_phase_shifter_closed_form(oracle_mod):
    """r = 0, b = 0: Pf = (V1/tau) V2 sin(d - phi)/x, Pt = -Pf,
    Qf = ((V1/tau)^2 - (V1/tau) V2 cos(d - phi))/x, Qt = (V2^2 - (V1/tau) V2 cos(d - phi))/x."""
    xl, V1, V2, d = 0.15, 1.03, 0.98, 0.11
    for tau, phi in ((1.0, 0.3), (0.97, -0.25), (1.04, 0.5)):
        g = tiny_grid(2, [(0, 1)], [(0.0, xl, 0.0, tau)], [(0, 0.01, 20.0)])
        g.shift = np.array([phi])
        r = oracle_mod.evaluate(oracle_mod.OracleNet(g), pack_x(g, np.array([d, 0.0]),
                                np.array([V1, V2])), np.zeros(g.m), want_jac=False, want_hess=False)
        v1 = V1 / tau
        assert r["gh"][0] == pytest.approx(v1 * V2 * np.sin(d - phi) / xl, rel=1e-13)
        assert r["gh"][1] == pytest.approx(-v1 * V2 * np.sin(d - phi) / xl, rel=1e-13)
        assert r["gh"][2] == pytest.approx((v1 ** 2 - v1 * V2 * np.cos(d - phi)) / xl, rel=1e-12)
        assert r["gh"][3] == pytest.approx((V2 ** 2 - v1 * V2 * np.cos(d - phi)) / xl, rel=1e-12)


@pytest.mark.parametrize("r,x,b,tau,phi", [(0.02, 0.12, 0.05, 1.0, 0.35),
                                           (0.01, 0.2, 0.08, 0.96, -0.4),
                                           (0.03, 0.05, 0.0, 1.05, 0.05)])
def test_shift_equals_rotated_from_angle(oracle_mod, r, x, b, tau, phi):
    """The ideal transformer hands the series element V_f / T, and charging and the from-side
    self term depend on |V_f| only, so a one-branch grid with shift phi at (Va_f, Va_t) has the
    outputs of the unshifted grid at (Va_f - phi, Va_t): g, h, J and H (the rotation is a constant
    offset of one variable, so derivatives carry over)."""
    gs = one_branch(r, x, b, tau, phi)
    g0 = one_branch(r, x, b, tau, 0.0)
    g0.shift = None
    rng = np.random.default_rng(7)
    for _ in range(4):
        Va = rng.normal(0.0, 0.3, 2)
        Vm = rng.uniform(0.9, 1.1, 2)
        Pg, Qg = rng.uniform(0, 1, 1), rng.uniform(-0.5, 0.5, 1)
        lam = rng.normal(size=gs.m)
        xs = pack_x(gs, Va, Vm, Pg, Qg)
        x0 = pack_x(g0, Va - np.array([phi, 0.0]), Vm, Pg, Qg)
        rs = oracle_mod.evaluate(oracle_mod.OracleNet(gs), xs, lam, sigma=0.7)
        r0 = oracle_mod.evaluate(oracle_mod.OracleNet(g0), x0, lam, sigma=0.7)
        np.testing.assert_allclose(rs["gh"], r0["gh"], rtol=1e-12, atol=1e-13)
        for k in ("J", "H"):
            np.testing.assert_array_equal(rs[k][0], r0[k][0])
            np.testing.assert_array_equal(rs[k][1], r0[k][1])
            np.testing.assert_allclose(rs[k][2], r0[k][2], rtol=1e-11, atol=1e-12)
        assert rs["f"] == r0["f"]


def test_zero_shift_is_the_shift_free_model(oracle_mod):
    g = synth.make_grid(71, 40, 52, 9, transformer_frac=0.3, shunts=True)
    b = synth.random_batch(71, g, 1, masks=True, pd_scale=True, sigma=0.6)
    gz = synth.Grid(**{**g.__dict__, "shift": np.zeros(g.nl)})
    for cart in (False, True):
        lam = b.lam[0] if not cart else np.concatenate([b.lam[0], np.ones(g.nb)])
        r0 = oracle_mod.evaluate(oracle_mod.OracleNet(g), b.x[0], lam, b.mask[0], b.pd_scale[0],
                                 sigma=0.6, cartesian=cart)
        rz = oracle_mod.evaluate(oracle_mod.OracleNet(gz), b.x[0], lam, b.mask[0], b.pd_scale[0],
                                 sigma=0.6, cartesian=cart)
        np.testing.assert_array_equal(r0["gh"], rz["gh"])
        np.testing.assert_array_equal(r0["J"][2], rz["J"][2])
        np.testing.assert_array_equal(r0["H"][2], rz["H"][2])


def test_pi_model_mutual_admittances(oracle_mod):
    """Yft = -ys e^{j phi}/tau and Ytf = -ys e^{-j phi}/tau, in complex arithmetic."""
    r, x, b, tau, phi = 0.02, 0.13, 0.04, 0.97, 0.31
    Y = oracle_mod.pi_model(r, x, b, tau, shift=phi)
    ys = 1.0 / (r + 1j * x)
    yft = -ys * np.exp(1j * phi) / tau
    ytf = -ys * np.exp(-1j * phi) / tau
    np.testing.assert_allclose(Y[2:4], [yft.real, yft.imag], rtol=1e-14)
    np.testing.assert_allclose(Y[4:6], [ytf.real, ytf.imag], rtol=1e-14)
    np.testing.assert_allclose([Y[0], Y[1]], [ys.real / tau ** 2, (ys.imag + b / 2) / tau ** 2],
                               rtol=1e-14)


def test_cartesian_change_of_variables_with_shifters(oracle_mod):
    import test_oracle_cartesian as TK
    g = synth.make_grid(57, 30, 41, 6, transformer_frac=0.2, shunts=True, shifter_frac=0.3)
    TK.change_of_variables_check(oracle_mod, g, 57)
