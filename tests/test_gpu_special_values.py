"""GPU parity with multipliers and voltages at special floating-point values.

The kernels double values exactly on the integer pipe (2 mu for the flow rows' Hessian terms,
2 P and 2 Q for the h rows' Jacobian, 2 Vm, 2 Gs and 2 Bs): a normal value takes an exponent
increment, and zero, -0, subnormals and the values around the smallest normal take the general
path.  These states put the flow multipliers mu_f, mu_t (Sec. III, eqs. (9)-(10): the h rows'
multipliers) and some voltage magnitudes on those values, and compare every output with the
oracle element by element (|gpu - oracle| <= 1e-11 max(1, |oracle|)), and the persistent
tilings and the multi-kernel schedule with each other bit for bit.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import compare_instance, gpu_eval, oracle_eval

pytestmark = pytest.mark.gpu

SPECIAL = np.array([0.0, -0.0, 5e-324, -5e-324, 2.225073858507201e-308, -2.2250738585072014e-308,
                    2.2250738585072014e-308, 4.450147717014403e-308, 1e-300, -1e-300, 1e300, -1e300])


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def special_batch(g, B=8, seed=301):
    b = synth.random_batch(seed, g, B, masks=True, sigma=0.9)
    rng = np.random.default_rng(seed)
    nb, nl = g.nb, g.nl
    lam = b.lam.copy()
    x = b.x.copy()
    for s in range(B):
        # every flow multiplier of the state drawn from the special values
        lam[s, 2 * nb:2 * nb + 2 * nl] = rng.choice(SPECIAL, size=2 * nl)
        if s % 2:   # a few voltage magnitudes at zero or subnormal as well
            k = rng.choice(nb, size=5, replace=False)
            x[s, nb + k] = rng.choice([0.0, 5e-324, 2.225073858507201e-308], size=5)
    b.lam, b.x = lam, x
    return b


def test_special_multipliers_against_oracle(ex, oracle_mod):
    g = synth.make_grid(301, 300, 389, 77, transformer_frac=0.3, shunts=True)
    b = special_batch(g)
    net = ex.Net(g)
    outs = []
    for cfg in (dict(schedule=2), dict(schedule=2, tiling=2), dict(schedule=1)):
        ex.exago_net_set_config(net.h, **cfg)
        outs.append(gpu_eval(net, b))
    for o in outs[1:]:
        for k in outs[0]:
            np.testing.assert_array_equal(o[k], outs[0][k], err_msg=k)
    for i in range(b.B):
        compare_instance(outs[0], i, oracle_eval(oracle_mod, g, b, i), f"special [{i}]")
