"""The live oracle reproduces its stored 30-bus snapshots, polar and cartesian (detects unintended
oracle drift).

Structure must match exactly; values to 1e-13, since libm sin/cos may differ by an ulp between
machines (e.g. FMA and non-FMA builds of the same routine)."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def test_oracle_reproduces_golden(oracle_mod):
    import make_golden
    g, b = make_golden.cases()
    stored = json.load(open(os.path.join(HERE, "golden", "c1_30bus.json")))["instances"]
    live = oracle_mod.evaluate_batch(oracle_mod.OracleNet(g), b)
    for s, r in zip(stored, live):
        close = lambda a, b: np.testing.assert_allclose(np.array(a), b, rtol=1e-13, atol=1e-13)
        close(s["f"], r["f"])
        close(s["gh"], r["gh"])
        close(s["grad"], r["grad"])
        np.testing.assert_array_equal(np.array(s["J_rowptr"]), r["J"][0])
        np.testing.assert_array_equal(np.array(s["J_col"]), r["J"][1])
        close(s["J_val"], r["J"][2])
        np.testing.assert_array_equal(np.array(s["H_rowptr"]), r["H"][0])
        np.testing.assert_array_equal(np.array(s["H_col"]), r["H"][1])
        close(s["H_val"], r["H"][2])


def test_cartesian_oracle_reproduces_golden(oracle_mod):
    import make_golden
    g, b, x, lam = make_golden.cartesian_cases()
    stored = json.load(open(os.path.join(HERE, "golden", "c1_30bus_cartesian.json")))["instances"]
    net = oracle_mod.OracleNet(g)
    for i, s in enumerate(stored):
        r = oracle_mod.evaluate(net, x[i], lam[i], b.mask[i], None, 1.0, b.sigma, cartesian=True)
        close = lambda a, c: np.testing.assert_allclose(np.array(a), c, rtol=1e-13, atol=1e-13)
        close(s["f"], r["f"])
        close(s["gh"], r["gh"])
        close(s["grad"], r["grad"])
        np.testing.assert_array_equal(np.array(s["J_rowptr"]), r["J"][0])
        np.testing.assert_array_equal(np.array(s["J_col"]), r["J"][1])
        close(s["J_val"], r["J"][2])
        np.testing.assert_array_equal(np.array(s["H_rowptr"]), r["H"][0])
        np.testing.assert_array_equal(np.array(s["H_col"]), r["H"][1])
        close(s["H_val"], r["H"][2])
