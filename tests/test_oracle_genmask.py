"""Pins of the oracle's generator outages (no GPU).

A contingency may be a generator outage, or a generator and a line together (Sec. V-A).  The
oracle takes a per-state generator mask; an out-of-service generator must act as if it were
removed from the grid, with its variables kept (zero gradient, Jacobian and Hessian entries).
The pins compare, in both formulations, the masked evaluation with the evaluation of the grid
without that generator (values, gradient, and every Jacobian and Hessian entry, mapped by
variable), and check a hand-built two-bus case.  test_oracle_mutants.py plants an ignored mask
and a kept -1 Jacobian entry and checks that these pins catch them.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from test_oracle import pack_x, tiny_grid


def drop_generators(g, off):
    keep = np.setdiff1d(np.arange(g.ng), off)
    return keep, synth.Grid(**{**g.__dict__, "gbus": g.gbus[keep], "c2": g.c2[keep],
                               "c1": g.c1[keep], "c0": g.c0[keep]})


def var_map(g, keep):
    """Columns of the grid without the dropped generators, in the full grid's variables."""
    nb, ng = g.nb, g.ng
    return np.concatenate([np.arange(2 * nb), 2 * nb + keep, 2 * nb + ng + keep])


@pytest.mark.parametrize("cartesian", [False, True])
def test_generator_out_equals_generator_removed(oracle_mod, cartesian):
    g = synth.make_grid(81, 40, 55, 12, shunts=True)
    g.c0[:] = np.linspace(1.0, 5.0, g.ng)              # a constant cost must vanish too
    rng = np.random.default_rng(81)
    x = rng.normal(size=g.n)
    x[g.nb:2 * g.nb] = rng.uniform(0.95, 1.05, g.nb)
    m = g.m + (g.nb if cartesian else 0)
    lam = rng.normal(size=m)
    off = np.array([2, 7, 11])
    gm = np.ones(g.ng, np.uint8)
    gm[off] = 0
    keep, g2 = drop_generators(g, off)
    cols = var_map(g, keep)
    kw = dict(obj_weight=0.7, sigma=0.9, cartesian=cartesian)
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), x, lam, gen_mask=gm, **kw)
    r2 = oracle_mod.evaluate(oracle_mod.OracleNet(g2), x[cols], lam, **kw)
    assert r["f"] == r2["f"]
    np.testing.assert_array_equal(r["gh"], r2["gh"])
    np.testing.assert_array_equal(r["grad"][cols], r2["grad"])
    dropped = np.concatenate([2 * g.nb + off, 2 * g.nb + g.ng + off])
    np.testing.assert_array_equal(r["grad"][dropped], 0.0)
    J = oracle_mod.csr_to_dense(r["J"], (m, g.n))
    J2 = oracle_mod.csr_to_dense(r2["J"], (m, g2.n))
    np.testing.assert_array_equal(J[:, cols], J2)
    np.testing.assert_array_equal(J[:, dropped], 0.0)
    H = oracle_mod.csr_to_dense(r["H"], (g.n, g.n))
    H2 = oracle_mod.csr_to_dense(r2["H"], (g2.n, g2.n))
    np.testing.assert_array_equal(H[np.ix_(cols, cols)], H2)
    np.testing.assert_array_equal(H[dropped][:, dropped], 0.0)
    # the pattern keeps the outaged generators' entries
    r1 = oracle_mod.evaluate(oracle_mod.OracleNet(g), x, lam, **kw)
    np.testing.assert_array_equal(r["J"][0], r1["J"][0])
    np.testing.assert_array_equal(r["H"][0], r1["H"][0])


def test_two_bus_generator_outage_by_hand(oracle_mod):
    """Flat start on a lossless line: the balances are Pd - Pg of the generators in service."""
    g = tiny_grid(2, [(0, 1)], [(0.0, 0.1, 0.0, 0.0)], [(0, 0.01, 20.0), (1, 0.02, 30.0)],
                  Pd=[0.4, 0.9], Qd=[0.1, 0.2])
    x = pack_x(g, np.zeros(2), np.ones(2), np.array([1.5, 0.25]), np.array([0.3, -0.1]))
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), x, np.zeros(g.m),
                            gen_mask=np.array([0, 1], np.uint8), want_jac=False,
                            want_hess=False)
    np.testing.assert_array_equal(r["gh"][:4], [0.4, 0.9 - 0.25, 0.1, 0.2 + 0.1])
    # cost of generator 1 only: 0.02 * 25^2 + 30 * 25 = 762.5
    assert r["f"] == pytest.approx(762.5, rel=1e-15)
