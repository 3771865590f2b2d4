"""GPU: feasibility slacks (load loss, power imbalance; Sec. III, Fig. 2) applied to a finished
evaluation through the C ABI, against the oracle's definition on the same seeded inputs: the
balance terms bit for bit (the same additions in the same order, checked on the GPU's own
evaluation), the gradient and the transpose product bit for bit, the objective within
|gpu - oracle| <= 1e-11 max(1, |oracle|) (a tree sum against the oracle's running sum).  The
full evaluation plus slacks is also compared with the oracle's model plus slacks.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import assert_close, oracle_eval, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def slack_set(g, seed):
    """An imbalance pair on every P and Q balance, and load loss (P and Q) at the loaded buses."""
    nb = g.nb
    load = np.flatnonzero(g.Pd > 0.3)
    bus = np.concatenate([np.tile(np.arange(nb), 4), load, load])
    row = np.concatenate([np.zeros(2 * nb), np.ones(2 * nb), np.zeros(load.shape[0]),
                          np.ones(load.shape[0])]).astype(np.int32)
    sign = np.concatenate([-np.ones(nb), np.ones(nb), -np.ones(nb), np.ones(nb),
                           -np.ones(2 * load.shape[0])]).astype(np.int32)
    cost = np.random.default_rng(seed).uniform(100.0, 1000.0, bus.shape[0])
    return bus.astype(np.int32), row, sign, cost


@pytest.mark.parametrize("case", ["300bus_x13", "2000bus_x512"])
def test_slacks_match_oracle(ex, oracle_mod, case):
    import torch
    if case == "300bus_x13":   # one full group of 8 states and a ragged one of 5
        g = synth.make_grid(111, 300, 389, 77, shunts=True)
        b = synth.random_batch(111, g, 13, masks=True, obj_weight=True, sigma=0.6)
        sample = range(13)
    else:
        g = synth.grid_2000()
        b = synth.contingency_batch(3, g, 512)
        b.obj_weight = np.random.default_rng(112).uniform(0.1, 1.0, 512)
        sample = (0, 1, 300, 511)
    bus, row, sign, cost = slack_set(g, 113)
    nz = bus.shape[0]
    z = np.random.default_rng(114).uniform(0.0, 0.2, (b.B, nz))
    net = ex.Net(g)
    sl = ex.Slack(net, bus, row, sign, cost)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], d["pd_scale"], d["obj_weight"], b.sigma)
    out = net.outputs(b.B, jac=False, hess=False)
    net.eval_all(bt, out)
    torch.cuda.synchronize()
    gh0, f0 = out["gh"].cpu().numpy(), out["f"].cpu().numpy()
    Z = torch.as_tensor(z, device="cuda")
    grad_z = torch.empty(b.B, nz, dtype=torch.float64, device="cuda")
    ex.exago_eval_slack(sl, bt, Z, out["gh"], g.m, out["f"], grad_z)
    v = np.random.default_rng(115).normal(size=(b.B, g.m))
    jt = torch.empty(b.B, nz, dtype=torch.float64, device="cuda")
    ex.exago_eval_slack_jtv(sl, bt, torch.as_tensor(v, device="cuda"), g.m, jt)
    torch.cuda.synchronize()
    gh, f, gz, jt = (out["gh"].cpu().numpy(), out["f"].cpu().numpy(), grad_z.cpu().numpy(),
                     jt.cpu().numpy())
    w = b.obj_weight
    for i in range(b.B):
        ref_gh, ref_f, ref_g = oracle_mod.slack(g.nb, bus, row, sign, cost, z[i], w[i],
                                                gh=gh0[i, :2 * g.nb], f=f0[i])
        np.testing.assert_array_equal(gh[i, :2 * g.nb], ref_gh)
        np.testing.assert_array_equal(gh[i, 2 * g.nb:], gh0[i, 2 * g.nb:])
        assert_close(f[i], ref_f, f"f + slack cost [{i}]")
        np.testing.assert_array_equal(gz[i], ref_g)
        np.testing.assert_array_equal(jt[i], sign * v[i, row * g.nb + bus])
    for i in sample:
        r = oracle_eval(oracle_mod, g, b, i)
        ref_gh, ref_f, _ = oracle_mod.slack(g.nb, bus, row, sign, cost, z[i], w[i],
                                            gh=r["gh"][:2 * g.nb], f=r["f"])
        assert_close(gh[i, :2 * g.nb], ref_gh, f"model + slacks g [{i}]")
        assert_close(f[i], ref_f, f"model + slacks f [{i}]")
    sl.close()
    net.close()


def test_slacks_on_cartesian_rows_and_empty(ex, oracle_mod):
    import torch
    from test_gpu_cartesian import run_cart, to_cartesian
    g = synth.make_grid(116, 120, 160, 30, shunts=True)
    b = synth.random_batch(116, g, 3)
    x, lam = to_cartesian(g, b, 116)
    net = ex.Net(g)
    base = run_cart(ex, net, b, x, lam, which=("gh",))["gh"]
    bus, row, sign, cost = slack_set(g, 117)
    z = np.random.default_rng(118).uniform(0.0, 0.2, (b.B, bus.shape[0]))
    sl = ex.Slack(net, bus, row, sign, cost)
    GH = torch.as_tensor(base.copy(), device="cuda")
    X = torch.as_tensor(x, device="cuda")
    bt = ex.make_batch(X)
    ex.exago_eval_slack(sl, bt, torch.as_tensor(z, device="cuda"), GH, g.m + g.nb)
    torch.cuda.synchronize()
    got = GH.cpu().numpy()
    for i in range(b.B):
        ref, _, _ = oracle_mod.slack(g.nb, bus, row, sign, cost, z[i], gh=base[i, :2 * g.nb])
        np.testing.assert_array_equal(got[i, :2 * g.nb], ref)
        np.testing.assert_array_equal(got[i, 2 * g.nb:], base[i, 2 * g.nb:])
    sl.close()
    empty = ex.Slack(net, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    ex.exago_eval_slack(empty, bt, torch.zeros(b.B, 0, dtype=torch.float64, device="cuda"), GH,
                        g.m + g.nb)
    with pytest.raises(ex.ExagoError):
        s2 = ex.Slack(net, bus, row, sign, cost)
        ex.exago_eval_slack(s2, bt, torch.as_tensor(z, device="cuda"), GH, 2 * g.nb - 1)
    empty.close()
    net.close()


def test_slacks_more_states_than_one_grid_row(ex, oracle_mod):
    """70,000 states on the 30-bus grid (several launches per call): balance terms, gradient and
    transpose bit for bit, the objective within the tolerance."""
    import torch
    g = synth.grid_30bus()
    B = 70_000
    bus, row, sign, cost = slack_set(g, 131)
    nz = bus.shape[0]
    rng = np.random.default_rng(132)
    z = rng.uniform(0.0, 0.2, (B, nz))
    gh0 = rng.normal(size=(B, g.m))
    f0 = rng.normal(size=B)
    net = ex.Net(g)
    sl = ex.Slack(net, bus, row, sign, cost)
    x = torch.zeros(B, g.n, dtype=torch.float64, device="cuda")
    bt = ex.make_batch(x)
    GH, F = torch.as_tensor(gh0.copy(), device="cuda"), torch.as_tensor(f0.copy(), device="cuda")
    GZ = torch.empty(B, nz, dtype=torch.float64, device="cuda")
    ex.exago_eval_slack(sl, bt, torch.as_tensor(z, device="cuda"), GH, g.m, F, GZ)
    JT = torch.empty(B, nz, dtype=torch.float64, device="cuda")
    ex.exago_eval_slack_jtv(sl, bt, torch.as_tensor(gh0, device="cuda"), g.m, JT)
    torch.cuda.synchronize()
    gh, f, gz, jt = GH.cpu().numpy(), F.cpu().numpy(), GZ.cpu().numpy(), JT.cpu().numpy()
    for i in (0, 65_534, 65_535, 65_536, B - 1):
        ref_gh, ref_f, ref_g = oracle_mod.slack(g.nb, bus, row, sign, cost, z[i],
                                                gh=gh0[i, :2 * g.nb], f=f0[i])
        np.testing.assert_array_equal(gh[i, :2 * g.nb], ref_gh)
        assert_close(f[i], ref_f, f"f [{i}]")
        np.testing.assert_array_equal(gz[i], ref_g)
        np.testing.assert_array_equal(jt[i], sign * gh0[i, row * g.nb + bus])
    sl.close()
    net.close()


@pytest.mark.parametrize("cfg", [
    dict(),                                                                  # persistent default
    dict(schedule=2, block=64, occupancy=16, stage_records=2, tile_group=1),  # the bench's
    dict(schedule=2, block=128, stage_records=1, tile_group=2),
    dict(schedule=2, block=32, occupancy=8),
    dict(schedule=1),                                                        # two calls (fallback)
])
def test_eval_all_slack_equals_the_two_calls(ex, cfg):
    """exago_eval_all_slack gives bitwise the results of exago_eval_all then exago_eval_slack, for
    every output (f, grad, g | h, J, H, grad_z), in every schedule."""
    import torch
    g = synth.make_grid(115, 300, 389, 77, shunts=True)
    b = synth.random_batch(115, g, 11, masks=True, pd_scale=True, obj_weight=True, sigma=0.7)
    bus, row, sign, cost = slack_set(g, 116)
    nz = bus.shape[0]
    z = torch.as_tensor(np.random.default_rng(117).uniform(0.0, 0.2, (b.B, nz)), device="cuda")
    net = ex.Net(g)
    if cfg:
        ex.exago_net_set_config(net.h, **cfg)
    sl = ex.Slack(net, bus, row, sign, cost)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], d["pd_scale"], d["obj_weight"], b.sigma)
    two = net.outputs(b.B)
    gz2 = torch.empty(b.B, nz, dtype=torch.float64, device="cuda")
    net.eval_all(bt, two)
    ex.exago_eval_slack(sl, bt, z, two["gh"], net.m, two["f"], gz2)
    one = net.outputs(b.B)
    gz1 = torch.full((b.B, nz), np.nan, dtype=torch.float64, device="cuda")
    for _ in range(2):   # the second call may replay a cached graph
        ex.exago_eval_all_slack(net.h, bt, sl, z, one["f"], one["grad"], one["gh"], one["jval"],
                                one["hval"], gz1)
    torch.cuda.synchronize()
    ex.exago_net_check(net.h)
    for k in two:
        np.testing.assert_array_equal(one[k].cpu().numpy(), two[k].cpu().numpy(), err_msg=k)
    np.testing.assert_array_equal(gz1.cpu().numpy(), gz2.cpu().numpy())


def test_eval_all_slack_2000_bus_512_against_oracle(ex, oracle_mod):
    """The one-call evaluation with slacks on the 2,000-bus x 512 batch in the benchmarked
    configuration, sampled against the oracle's model plus slacks."""
    import torch
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 512)
    b.obj_weight = np.random.default_rng(118).uniform(0.1, 1.0, 512)
    bus, row, sign, cost = slack_set(g, 119)
    nz = bus.shape[0]
    zh = np.random.default_rng(120).uniform(0.0, 0.2, (b.B, nz))
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, block=64, occupancy=16, stage_records=2,
                            tile_group=1)
    sl = ex.Slack(net, bus, row, sign, cost)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], None, d["obj_weight"], b.sigma)
    out = net.outputs(b.B)
    gz = torch.empty(b.B, nz, dtype=torch.float64, device="cuda")
    ex.exago_eval_all_slack(net.h, bt, sl, torch.as_tensor(zh, device="cuda"), out["f"],
                            out["grad"], out["gh"], out["jval"], out["hval"], gz)
    torch.cuda.synchronize()
    host = {k: v.cpu().numpy() for k, v in out.items()}
    for i in (0, 255, 511):
        ref = oracle_eval(oracle_mod, g, b, i)
        ghs, fs, gzs = oracle_mod.slack(g.nb, bus, row, sign, cost, zh[i], float(b.obj_weight[i]),
                                        gh=ref["gh"][:2 * g.nb], f=ref["f"])
        assert_close(host["gh"][i][:2 * g.nb], ghs, f"gh[{i}]")
        assert_close(host["gh"][i][2 * g.nb:], ref["gh"][2 * g.nb:], f"h[{i}]")
        assert_close(host["f"][i], fs, f"f[{i}]")
        assert_close(gz[i].cpu().numpy(), gzs, f"grad_z[{i}]")
        assert_close(host["jval"][i], ref["J"][2], f"J[{i}]")
        assert_close(host["hval"][i], ref["H"][2], f"H[{i}]")
