"""Writes tests/golden/c1_30bus.json and tests/golden/c1_30bus_cartesian.json from the CPU oracle
alone.

The paper prints no worked example, so the stored values come from the oracle (which its own pins
in test_oracle.py tie to closed forms, the complex nodal form, finite differences and the loss
invariant).  Workload: the 30-bus synthetic grid (seed 1, 41 branches, 6 generators) with two
states of seed 7, the second with a random outage mask, sigma = 0.8.
The cartesian snapshot evaluates the power-balance-cartesian formulation at the same operating
points (e = Vm cos Va, f = Vm sin Va) with voltage-row multipliers drawn from seed 8.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import acopf  # noqa: E402
from paper_2203_10587_gb300 import synth  # noqa: E402


def cases():
    g = synth.grid_30bus()
    b = synth.random_batch(7, g, 2, masks=True, sigma=0.8)
    b.mask[0, :] = 1
    return g, b


def cartesian_cases():
    """The same two states in rectangular voltages, with multipliers for the voltage rows."""
    g, b = cases()
    nb = g.nb
    x = b.x.copy()
    x[:, :nb] = b.x[:, nb:2 * nb] * np.cos(b.x[:, :nb])
    x[:, nb:2 * nb] = b.x[:, nb:2 * nb] * np.sin(b.x[:, :nb])
    muV = np.random.Generator(np.random.PCG64(8)).normal(size=(b.B, nb))
    lam = np.concatenate([b.lam, muV], axis=1)
    return g, b, x, lam


def snapshot(r):
    return {"f": r["f"], "grad": r["grad"].tolist(), "gh": r["gh"].tolist(),
            "J_rowptr": r["J"][0].tolist(), "J_col": r["J"][1].tolist(),
            "J_val": r["J"][2].tolist(), "H_rowptr": r["H"][0].tolist(),
            "H_col": r["H"][1].tolist(), "H_val": r["H"][2].tolist()}


def main_cartesian():
    g, b, x, lam = cartesian_cases()
    net = acopf.OracleNet(g)
    out = [snapshot(acopf.evaluate(net, x[i], lam[i], b.mask[i], None, 1.0, b.sigma,
                                   cartesian=True)) for i in range(b.B)]
    with open(os.path.join(HERE, "c1_30bus_cartesian.json"), "w") as fh:
        json.dump({"source": "oracle/acopf_oracle.c (oracle_eval_cart) via tests/golden/make_golden.py",
                   "workload": "30-bus synthetic grid seed 1; states seed 7 in rectangular "
                               "voltages; voltage-row multipliers seed 8; sigma 0.8",
                   "instances": out}, fh, indent=0)


def main():
    g, b = cases()
    net = acopf.OracleNet(g)
    out = []
    for i, r in enumerate(acopf.evaluate_batch(net, b)):
        out.append({"f": r["f"], "grad": r["grad"].tolist(), "gh": r["gh"].tolist(),
                    "J_rowptr": r["J"][0].tolist(), "J_col": r["J"][1].tolist(),
                    "J_val": r["J"][2].tolist(), "H_rowptr": r["H"][0].tolist(),
                    "H_col": r["H"][1].tolist(), "H_val": r["H"][2].tolist()})
    with open(os.path.join(HERE, "c1_30bus.json"), "w") as fh:
        json.dump({"source": "oracle/acopf_oracle.c via tests/golden/make_golden.py",
                   "workload": "30-bus synthetic grid seed 1; states seed 7; sigma 0.8",
                   "instances": out}, fh, indent=0)


if __name__ == "__main__":
    main()
    main_cartesian()
