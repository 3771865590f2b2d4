"""GPU: seeded random irregular grids against the oracle, under random launch configurations.

Each case draws a grid (1 to 700 buses, sizes off every tile boundary), then makes it irregular
-- parallel branches in both directions, several generators on one bus, generator-free and
branch-free buses, shunts, transformers -- and a batch with masks, load scales, weights and an
objective factor.  It picks a schedule and its options at random and compares every output of
every state with the oracle."""
import dataclasses

import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import compare_instance, gpu_eval, oracle_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def irregular_grid(rng, seed):
    nb = int(rng.choice([1, 2, 3, 31, 33, 65, 127, 129, 257, 700]))
    # a spanning tree plus extra edges, at most every pair once (duplicates are added below)
    nl = 0 if nb == 1 else int(rng.integers(nb - 1, min(2 * nb, nb * (nb - 1) // 2 + 1)))
    ng = int(rng.integers(0, nb + 1))
    if nb == 1:
        g = synth.make_grid(seed, 2, 1, 1, shunts=True)       # then cut to one bus below
        g = dataclasses.replace(g, nb=1, Gs=g.Gs[:1], Bs=g.Bs[:1], Pd=g.Pd[:1], Qd=g.Qd[:1],
                                f=g.f[:0], t=g.t[:0], r=g.r[:0], x=g.x[:0], b=g.b[:0],
                                tap=g.tap[:0], rateA=g.rateA[:0], gbus=np.zeros(1, np.int32))
        return g
    g = synth.make_grid(seed, nb, nl, min(ng, nb), shunts=bool(rng.integers(2)),
                        transformer_frac=float(rng.uniform(0, 0.5)))
    # parallel branches: copy some branches, half of them reversed
    k = int(rng.integers(0, max(1, g.nl // 4) + 1))
    if k:
        idx = rng.choice(g.nl, size=k)
        rev = rng.integers(0, 2, size=k).astype(bool)
        f2 = np.where(rev, g.t[idx], g.f[idx]).astype(np.int32)
        t2 = np.where(rev, g.f[idx], g.t[idx]).astype(np.int32)
        cat = lambda a, b: np.concatenate([a, b])
        g = dataclasses.replace(g, f=cat(g.f, f2), t=cat(g.t, t2), r=cat(g.r, g.r[idx] * 1.3),
                                x=cat(g.x, g.x[idx] * 0.9), b=cat(g.b, g.b[idx]),
                                tap=cat(g.tap, g.tap[idx]), rateA=cat(g.rateA, g.rateA[idx]))
    # several generators on some buses
    m = int(rng.integers(0, 6))
    if m and g.nb > 0:
        gb = rng.integers(0, g.nb, size=m).astype(np.int32)
        cat = lambda a, b: np.concatenate([a, b])
        g = dataclasses.replace(g, gbus=cat(g.gbus, gb), c2=cat(g.c2, rng.uniform(0.001, 0.01, m)),
                                c1=cat(g.c1, rng.uniform(10, 40, m)), c0=cat(g.c0, rng.uniform(0, 5, m)))
    return g


def random_config(rng):
    sched = int(rng.choice([1, 2, 2, 2, 3]))
    cfg = dict(schedule=sched, stage_records=int(rng.choice([1, 2])))
    if sched == 2:
        cfg.update(block=int(rng.choice([32, 64, 128, 256])), occupancy=int(rng.choice([8, 16, 24])),
                   tile_group=int(rng.integers(1, 5)))
        if rng.integers(2):
            lag = int(rng.integers(1, 4))
            cfg.update(lag=lag, ring=lag + int(rng.integers(1, 3)))
    if sched == 3:
        cfg.update(chunk=int(rng.integers(1, 6)), ring=int(rng.integers(1, 4)))
    cfg["use_graph"] = int(rng.choice([1, 2]))
    return cfg


@pytest.mark.parametrize("case", range(12))
def test_random_irregular_grid_and_configuration(ex, oracle_mod, case):
    rng = np.random.default_rng(1000 + case)
    g = irregular_grid(rng, 1000 + case)
    B = int(rng.integers(1, 12))
    b = synth.random_batch(2000 + case, g, B, masks=True, pd_scale=bool(rng.integers(2)),
                           obj_weight=bool(rng.integers(2)), sigma=float(rng.choice([0.0, 0.6, 1.0])))
    net = ex.Net(g)
    cfg = random_config(rng)
    ex.exago_net_set_config(net.h, **cfg)
    out = gpu_eval(net, b)
    for i in sorted({0, B - 1, int(rng.integers(B))}):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"case {case} {cfg} [{i}]")


@pytest.mark.parametrize("case", range(8))
def test_random_grids_with_generator_outages_both_formulations(ex, oracle_mod, case):
    """The same kind of irregular grids with random generator outages (about 20% of the
    generators out, a separate mask per state): the polar model under a random launch
    configuration, and the cartesian model at the same operating points, against the oracle."""
    from test_gpu_cartesian import oracle_cart, run_cart, to_cartesian
    rng = np.random.default_rng(3000 + case)
    g = irregular_grid(rng, 3000 + case)
    B = int(rng.integers(1, 12))
    b = synth.random_batch(4000 + case, g, B, masks=True, pd_scale=bool(rng.integers(2)),
                           obj_weight=bool(rng.integers(2)), sigma=float(rng.choice([0.0, 0.6, 1.0])),
                           gen_masks=True)
    net = ex.Net(g)
    cfg = random_config(rng)
    ex.exago_net_set_config(net.h, **cfg)
    out = gpu_eval(net, b)
    x, lam = to_cartesian(g, b, 5000 + case)
    cart = run_cart(ex, net, b, x, lam)
    for i in sorted({0, B - 1, int(rng.integers(B))}):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"case {case} {cfg} [{i}]")
        ref = oracle_cart(oracle_mod, g, b, x, lam, i)
        compare_instance(cart, i, ref, f"cartesian case {case} [{i}]")


@pytest.mark.parametrize("case", range(10))
def test_random_irregular_grids_warp_tiles(ex, oracle_mod, case):
    """The same irregular grids (a single bus without branches among them) under random
    branch-per-warp configurations, with batches that end inside or on a group of 32 states:
    bitwise equal to the branch-per-thread kernel, and sampled states against the oracle."""
    rng = np.random.default_rng(6000 + case)
    g = irregular_grid(rng, 6000 + case)
    B = int(rng.choice([1, 5, 31, 32, 33, 64, 70]))
    b = synth.random_batch(7000 + case, g, B, masks=True, pd_scale=bool(rng.integers(2)),
                           obj_weight=bool(rng.integers(2)), sigma=float(rng.choice([0.0, 0.6, 1.0])),
                           gen_masks=bool(rng.integers(2)))
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2)
    ref = gpu_eval(net, b)
    cfg = dict(schedule=2, tiling=2, block=int(rng.choice([64, 128])),
               occupancy=int(rng.choice([8, 16])), tile_group=int(rng.integers(1, 5)),
               use_graph=int(rng.choice([1, 2])))
    if rng.integers(2):
        lag = int(rng.integers(1, 4))
        cfg.update(lag=lag, ring=lag + int(rng.integers(1, 4)))
    ex.exago_net_set_config(net.h, **cfg)
    out = gpu_eval(net, b)
    for k in ref:
        np.testing.assert_array_equal(out[k], ref[k], err_msg=f"case {case} {cfg} {k}")
    for i in sorted({0, B - 1, int(rng.integers(B))}):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"warp case {case} {cfg} [{i}]")
