"""GPU: the warp-tiled persistent kernel (tiling = EXAGO_TILING_WARP: a warp takes one branch or
bus, its 32 lanes take 32 states) against the per-thread tiling and the oracle.

Both tilings run the same per-(state, branch) and per-(state, bus) arithmetic in the same order,
so every output must be bitwise equal to the per-thread persistent kernel's; sampled states are
also compared with the oracle element by element (|gpu - oracle| <= 1e-11 max(1, |oracle|)).
Batch sizes cover one partial group (B < 32), exact groups and a ragged last group.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import compare_instance, gpu_eval, oracle_eval, to_device

pytestmark = pytest.mark.gpu

WARP = 2


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


WARP_CONFIGS = [
    dict(schedule=2, tiling=WARP),                                     # derived lag / ring, graph
    dict(schedule=2, tiling=WARP, use_graph=2),                        # direct launch
    dict(schedule=2, tiling=WARP, block=128, occupancy=8, tile_group=2),
    dict(schedule=2, tiling=WARP, block=64, occupancy=16, tile_group=3),
    dict(schedule=2, tiling=WARP, lag=1, ring=2),                      # every group reuses a slot
]


@pytest.mark.parametrize("B", [1, 31, 32, 45, 97])
def test_warp_tiles_bitwise_equal_to_thread_tiles(ex, oracle_mod, B):
    g = synth.make_grid(201, 300, 389, 77, transformer_frac=0.3, shunts=True)
    b = synth.random_batch(202 + B, g, B, masks=True, pd_scale=True, obj_weight=True, sigma=0.9)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2)
    ref = gpu_eval(net, b)
    for cfg in WARP_CONFIGS:
        ex.exago_net_set_config(net.h, **cfg)
        for _ in range(2):                                             # cached graph, reused ring
            out = gpu_eval(net, b)
            for k in ref:
                np.testing.assert_array_equal(out[k], ref[k], err_msg=f"{cfg} {k}")
    for i in sorted({0, B // 2, B - 1}):
        compare_instance(ref, i, oracle_eval(oracle_mod, g, b, i), f"warp B={B}")


def test_benchmark_batch_2000bus_x512(ex, oracle_mod):
    """The 2,000-bus x 512 N-1 batch: warp tiles equal the per-thread kernel bit for bit, and
    states of every group position agree with the oracle."""
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 512)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, block=64, occupancy=16, stage_records=2, tile_group=1)
    ref = gpu_eval(net, b)
    ex.exago_net_set_config(net.h, schedule=2, tiling=WARP, block=64, occupancy=16, tile_group=1)
    out = gpu_eval(net, b)
    for k in ref:
        np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
    for i in (0, 31, 32, 255, 511):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), "warp 2000x512")


def test_meshed_grid_rows_beyond_the_staging_cap(ex, oracle_mod):
    """A meshed grid (mean bus degree 10, up to about 20): some items' rows exceed the shared-
    memory staging of either tiling and are written directly; both tilings still agree bit for
    bit and with the oracle."""
    g = synth.make_grid(261, 400, 2000, 100, max_degree=64, shunts=True)
    b = synth.random_batch(262, g, 40, masks=True, pd_scale=True, sigma=0.8)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2)
    ref = gpu_eval(net, b)
    for cfg in (dict(schedule=2, tiling=WARP, block=128, tile_group=2),
                dict(schedule=2, tiling=WARP, block=64), dict(schedule=1)):
        ex.exago_net_set_config(net.h, **cfg)
        out = gpu_eval(net, b)
        for k in ref:
            np.testing.assert_array_equal(out[k], ref[k], err_msg=f"{cfg} {k}")
    for i in (0, 31, 39):
        compare_instance(ref, i, oracle_eval(oracle_mod, g, b, i), "warp meshed")


def test_net_without_branches(ex, oracle_mod):
    """One bus, no branch: no branch items at all, so the first bus item of each group sums the
    objective's partials itself."""
    import dataclasses
    g = synth.make_grid(271, 2, 1, 1, shunts=True)
    g = dataclasses.replace(g, nb=1, Gs=g.Gs[:1], Bs=g.Bs[:1], Pd=g.Pd[:1], Qd=g.Qd[:1],
                            f=g.f[:0], t=g.t[:0], r=g.r[:0], x=g.x[:0], b=g.b[:0], tap=g.tap[:0],
                            rateA=g.rateA[:0], gbus=np.zeros(1, np.int32))
    b = synth.random_batch(272, g, 45, pd_scale=True, obj_weight=True, sigma=0.7)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2)
    ref = gpu_eval(net, b)
    for cfg in WARP_CONFIGS[:3]:
        ex.exago_net_set_config(net.h, **cfg)
        out = gpu_eval(net, b)
        for k in ref:
            np.testing.assert_array_equal(out[k], ref[k], err_msg=f"{cfg} {k}")
    for i in (0, 44):
        compare_instance(ref, i, oracle_eval(oracle_mod, g, b, i), "warp no branches")


def test_generator_outages_and_phase_shifters(ex, oracle_mod):
    """The general variant (generator masks, phase-shifting transformers)."""
    g = synth.make_grid(211, 300, 390, 75, transformer_frac=0.1, shunts=True, shifter_frac=0.2)
    b = synth.random_batch(212, g, 40, masks=True, pd_scale=True, obj_weight=True, sigma=0.7,
                           gen_masks=True)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2)
    ref = gpu_eval(net, b)
    for cfg in WARP_CONFIGS[:3]:
        ex.exago_net_set_config(net.h, **cfg)
        out = gpu_eval(net, b)
        for k in ref:
            np.testing.assert_array_equal(out[k], ref[k], err_msg=f"{cfg} {k}")
    for i in (0, 33, 39):
        compare_instance(ref, i, oracle_eval(oracle_mod, g, b, i), "warp shift+genmask")


@pytest.mark.parametrize("which", [("f",), ("grad",), ("gh",), ("jval",), ("hval",),
                                   ("f", "hval"), ("gh", "jval")])
def test_output_subsets(ex, which):
    g = synth.make_grid(221, 200, 260, 50, shunts=True)
    b = synth.random_batch(222, g, 37, masks=True, sigma=0.8)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, tiling=WARP)
    full = gpu_eval(net, b)
    part = gpu_eval(net, b, which=which)
    for k in which:
        np.testing.assert_array_equal(part[k], full[k], err_msg=str(which))


def test_reported_configuration(ex):
    g = synth.grid_2000()
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, tiling=WARP)
    c = ex.exago_net_get_config(net.h, 512)
    assert c["tiling"] == WARP and c["block"] in (64, 128) and c["occupancy"] in (8, 16)
    assert 1 <= c["lag"] < c["ring"] <= 512 // 32 + 1
    # the workspace holds the ring's groups of 32 states' records
    assert ex.exago_eval_workspace_size(net.h, 512) >= c["ring"] * 32 * 80 * 2 * g.nl
    for bad in (dict(tiling=3), dict(tiling=WARP, block=256), dict(tiling=WARP, occupancy=24)):
        with pytest.raises(ex.ExagoError):
            ex.exago_net_set_config(net.h, schedule=2, **bad)


def test_bounded_wait_timeout(ex):
    """Bus items wait for a branch count that never arrives: the launch ends, the status word
    says ETIMEOUT, and the next evaluation is correct."""
    g = synth.make_grid(231, 60, 80, 15)
    b = synth.random_batch(231, g, 40)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, tiling=WARP, use_graph=2, spin_limit=2000,
                            test_force_timeout=1)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"])
    out = net.outputs(b.B)
    net.eval_all(bt, out)
    with pytest.raises(ex.ExagoError) as ei:
        ex.exago_net_check(net.h)
    assert ei.value.name == "EXAGO_ETIMEOUT"
    ex.exago_net_set_config(net.h, schedule=2, tiling=WARP)
    good = gpu_eval(net, b)
    ex.exago_net_set_config(net.h, schedule=1)
    ref = gpu_eval(net, b)
    for k in ref:
        np.testing.assert_array_equal(good[k], ref[k])


def test_served_requests_on_a_warp_tiled_net(ex):
    """A server launches a net's requests with the net's configuration: with warp tiles (the
    gathered-batch variant) every result equals the request evaluated alone."""
    import torch
    g = synth.grid_2000()
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, tiling=WARP)
    srv = ex.exago_serve_create(1 << 30, max_slots=4, n_streams=2)
    try:
        ex.exago_serve_set_merge(srv, 32)
        nid = ex.exago_serve_register(srv, net.h)
        reqs = []
        for k in range(12):
            b = synth.random_batch(240 + k, g, 1 + k % 5, masks=True, sigma=0.8,
                                   gen_masks=k % 2 == 1)
            d = to_device(b)
            bt = ex.make_batch(d["x"], d["lam"], d["mask"], obj_factor=b.sigma,
                               gen_mask=d["gen_mask"])
            out = net.outputs(b.B)
            reqs.append((b, d, bt, out, ex.exago_serve_submit(srv, nid, bt, **out)))
        for *_, t in reqs:
            ex.exago_serve_wait(srv, t)
        torch.cuda.synchronize()
        ex.exago_net_set_config(net.h, schedule=2)
        for b, d, bt, out, _ in reqs:
            ref = net.outputs(b.B)
            net.eval_all(bt, ref)
            torch.cuda.synchronize()
            for k, v in ref.items():
                assert torch.equal(out[k], v), k
    finally:
        ex.exago_serve_destroy(srv)


def test_profile_phases(ex):
    g = synth.grid_2000()
    b = synth.random_batch(251, g, 64)
    net = ex.Net(g)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"])
    out = net.outputs(b.B)
    ex.exago_net_set_config(net.h, schedule=2, tiling=WARP)
    prof = ex.exago_eval_profile(net.h, bt, out["f"], out["grad"], out["gh"], out["jval"],
                                 out["hval"], reps=3)
    assert prof[0][0] == "persistent" and prof[0][1] > 0
    ph = dict(prof[1:])
    assert len(ph) == 7
