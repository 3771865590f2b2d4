"""Pins of the oracle's feasibility slacks (load loss, power imbalance; Sec. III, Fig. 2) (no GPU).

A slack z_k >= 0 at bus i enters the P or Q balance with sign +1 or -1 and costs w cost_k z_k.
The pins: hand-computed values; load loss at a bus equals lowering that bus's load in the model
itself (the main oracle evaluated with Pd - z); an imbalance pair of equal values leaves the
balances unchanged and adds its cost; finite differences in z give the Jacobian column (sign in
the slack's row) to rounding, since the terms are linear; invalid slacks are refused.
test_oracle_mutants.py plants a dropped sign, a wrong row and a dropped weight.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth


def test_hand_values(oracle_mod):
    gh, f, grad = oracle_mod.slack(3, [0, 0, 2], [0, 0, 1], [-1, 1, -1], [10.0, 10.0, 5.0],
                                   [0.5, 0.25, 1.0], w=2.0)
    np.testing.assert_array_equal(gh, [-0.25, 0.0, 0.0, 0.0, 0.0, -1.0])
    assert f == 25.0                     # 2 (10 * 0.5 + 10 * 0.25 + 5 * 1)
    np.testing.assert_array_equal(grad, [20.0, 20.0, 10.0])


def test_load_loss_equals_lower_load(oracle_mod):
    g = synth.make_grid(101, 30, 41, 6, shunts=True)
    b = synth.random_batch(101, g, 1)
    load = np.flatnonzero(g.Pd > 0.2)
    rng = np.random.default_rng(101)
    zP = rng.uniform(0.0, 0.2, load.shape[0])
    zQ = 0.3 * zP
    net = oracle_mod.OracleNet(g)
    r = oracle_mod.evaluate(net, b.x[0], b.lam[0], want_jac=False, want_hess=False)
    bus = np.concatenate([load, load])
    row = np.concatenate([np.zeros_like(load), np.ones_like(load)])
    gh, f, _ = oracle_mod.slack(g.nb, bus, row, -np.ones(bus.shape[0]), np.full(bus.shape[0], 7.0),
                                np.concatenate([zP, zQ]), gh=r["gh"][:2 * g.nb])
    g2 = synth.Grid(**{**g.__dict__, "Pd": g.Pd.copy(), "Qd": g.Qd.copy()})
    g2.Pd[load] -= zP
    g2.Qd[load] -= zQ
    r2 = oracle_mod.evaluate(oracle_mod.OracleNet(g2), b.x[0], b.lam[0], want_jac=False,
                             want_hess=False)
    np.testing.assert_allclose(gh, r2["gh"][:2 * g.nb], rtol=0, atol=1e-13)
    assert f == pytest.approx(7.0 * (zP.sum() + zQ.sum()), rel=1e-14)


def test_imbalance_pair_cancels(oracle_mod):
    nb = 5
    gh0 = np.random.default_rng(102).normal(size=2 * nb)
    gh, f, grad = oracle_mod.slack(nb, [3, 3], [1, 1], [1, -1], [4.0, 4.0], [0.7, 0.7], w=0.5,
                                   gh=gh0, f=1.0)
    np.testing.assert_array_equal(gh, gh0)
    assert f == 1.0 + 0.5 * 4.0 * 1.4
    np.testing.assert_array_equal(grad, [2.0, 2.0])


def test_finite_differences_give_the_jacobian_column(oracle_mod):
    rng = np.random.default_rng(103)
    nb, nz = 7, 12
    bus = rng.integers(0, nb, nz)
    row = rng.integers(0, 2, nz)
    sign = rng.choice([-1, 1], nz)
    cost = rng.uniform(1.0, 9.0, nz)
    z = rng.uniform(0.0, 1.0, nz)
    base, _, _ = oracle_mod.slack(nb, bus, row, sign, cost, z)
    for k in range(nz):
        dz = z.copy()
        dz[k] += 0.5
        gh, _, _ = oracle_mod.slack(nb, bus, row, sign, cost, dz)
        col = (gh - base) / 0.5
        expect = np.zeros(2 * nb)
        expect[row[k] * nb + bus[k]] = sign[k]
        np.testing.assert_allclose(col, expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("bad", [dict(bus=[5]), dict(bus=[-1]), dict(row=[2]), dict(sign=[0])])
def test_invalid_slacks_refused(oracle_mod, bad):
    kw = dict(bus=[1], row=[0], sign=[1])
    kw.update(bad)
    with pytest.raises(ValueError):
        oracle_mod.slack(5, kw["bus"], kw["row"], kw["sign"], [1.0], [1.0])
