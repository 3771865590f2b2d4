"""GPU: the persistent fused schedule (one launch, work list, ring scratch, bounded waits, CUDA
graph) and the pipelined two-stream schedule against the multi-kernel schedule and the oracle;
fault injection of the bounded waits; the autotuner.
"""
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


CONFIGS = [
    dict(schedule=1),                                   # multi-kernel
    dict(schedule=2),                                   # persistent, derived lag/ring, graph
    dict(schedule=2, use_graph=2),                      # persistent, direct launch
    dict(schedule=2, block=64, lag=1, ring=2),          # tightest ring: every state reuses a slot
    dict(schedule=2, block=256, lag=3, ring=5),
    dict(schedule=2, occupancy=24),                     # register-capped variant
    dict(schedule=2, block=64, occupancy=16),
    dict(schedule=2, block=64, occupancy=16, tile_group=1),
    dict(schedule=2, block=32),
    dict(schedule=2, block=32, occupancy=8, stage_records=1),
    dict(schedule=2, block=256, occupancy=8),
    dict(schedule=2, block=128, tile_group=3, stage_records=1),
    dict(schedule=2, block=64, tile_group=4, lag=1, ring=2),       # smallest ring, grouped items
    dict(schedule=2, block=256, occupancy=16, stage_records=1),
    dict(schedule=3),                                   # pipelined, derived chunk, graph
    dict(schedule=3, chunk=7, ring=2, stage_records=1), # ring reuse from the third chunk on
    dict(schedule=3, chunk=5, use_graph=2),             # direct launches
    dict(schedule=1, stage_records=1),
    dict(schedule=2, tiling=2),                         # warp tiles: a warp per branch / bus
    dict(schedule=2, tiling=2, block=128, occupancy=8, tile_group=2),
    dict(schedule=2, tiling=2, lag=1, ring=2, use_graph=2),
    dict(schedule=2, stage_records=3),                  # bus tiles' records in one bulk copy each
    dict(schedule=2, block=128, stage_records=3, tile_group=2, lag=1, ring=2, use_graph=2),
    dict(schedule=2, block=32, occupancy=8, stage_records=3),
    dict(schedule=1, stage_records=3),                  # bulk copies only persistent: plain walk
]


def grids():
    from test_capi_host import parallel_grid
    return {
        "300bus": (synth.make_grid(71, 300, 389, 77, transformer_frac=0.3, shunts=True), 23),
        "parallel": (parallel_grid(), 9),
        "2000bus": (synth.grid_2000(), 40),
    }


@pytest.mark.parametrize("name", ["300bus", "parallel", "2000bus"])
def test_schedules_bitwise_equal_and_match_oracle(ex, oracle_mod, name):
    g, B = grids()[name]
    b = synth.random_batch(5, g, B, masks=True, pd_scale=True, obj_weight=True, sigma=0.9)
    net = ex.Net(g)
    outs = []
    for cfg in CONFIGS:
        ex.exago_net_set_config(net.h, **cfg)
        outs.append(gpu_eval(net, b))
        outs.append(gpu_eval(net, b))          # second call: cached graph / reused ring
    for o in outs[1:]:
        for k in outs[0]:
            np.testing.assert_array_equal(o[k], outs[0][k], err_msg=k)
    for i in (0, B // 2, B - 1):
        compare_instance(outs[0], i, oracle_eval(oracle_mod, g, b, i), name)


@pytest.mark.parametrize("cfg", [dict(block=64, occupancy=16), dict(block=128, occupancy=16),
                                 dict(block=64, occupancy=8, tile_group=3),
                                 dict(block=256, occupancy=16)])
def test_bulk_record_copies_on_the_benchmark_and_a_meshed_grid(ex, oracle_mod, cfg):
    """stage_records = BULK: each bus tile's records come into shared memory in one TMA bulk
    copy (tiles whose records do not fit walk them through L2).  On the 2,000-bus x 512 batch and
    on a meshed grid (larger tiles, some above the cap) every output equals the default
    schedule's bit for bit."""
    for g, b in ((synth.grid_2000(), None), (synth.make_grid(281, 500, 2500, 125, max_degree=64), None)):
        b = synth.contingency_batch(3, g, 512) if g.nb == 2000 else synth.random_batch(282, g, 70, masks=True)
        net = ex.Net(g)
        ex.exago_net_set_config(net.h, schedule=2, **cfg)
        ref = gpu_eval(net, b)
        ex.exago_net_set_config(net.h, schedule=2, stage_records=3, **cfg)
        assert ex.exago_net_get_config(net.h, b.B)["stage_records"] == 3
        for _ in range(2):
            out = gpu_eval(net, b)
            for key in ref:
                np.testing.assert_array_equal(out[key], ref[key], err_msg=f"{cfg} {g.nb} {key}")
        compare_instance(out, b.B - 1, oracle_eval(oracle_mod, g, b, b.B - 1), f"bulk {cfg} {g.nb}")


def test_graph_cache_under_many_argument_sets(ex):
    """More distinct argument sets than the graph cache holds, cycled three times with no
    synchronisation between calls: first uses launch directly, second uses are captured, the
    least recently used graphs are evicted while earlier launches may still be in flight.  Every
    result equals the direct launch of the same state."""
    import torch
    g = synth.make_grid(75, 120, 160, 30, shunts=True)
    b = synth.random_batch(75, g, 12, masks=True, sigma=0.7)
    net = ex.Net(g)
    from parity_util import to_device
    d = to_device(b)
    batches = [ex.make_batch(d["x"][i:i + 1], d["lam"][i:i + 1], d["mask"][i:i + 1], obj_factor=b.sigma)
               for i in range(b.B)]
    ex.exago_net_set_config(net.h, schedule=2, use_graph=2)
    ref = [net.eval_all(bt, net.outputs(1)) for bt in batches]
    ex.exago_net_set_config(net.h, schedule=2, use_graph=1)
    outs = [[net.outputs(1) for _ in range(3)] for _ in batches]
    for r in range(3):
        for i, bt in enumerate(batches):
            net.eval_all(bt, outs[i][r])
    torch.cuda.synchronize()
    ex.exago_net_check(net.h)
    for i in range(b.B):
        for r in range(3):
            for k, v in ref[i].items():
                assert torch.equal(outs[i][r][k], v), (i, r, k)


def test_single_state_and_subset_outputs(ex, oracle_mod):
    g = synth.grid_10k()
    b = synth.random_batch(8, g, 1)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2)
    out = gpu_eval(net, b)
    compare_instance(out, 0, oracle_eval(oracle_mod, g, b, 0), "10k persistent")
    # only some outputs requested: each must equal the full call
    for which in (("f",), ("grad",), ("gh",), ("jval",), ("hval",), ("f", "hval")):
        part = gpu_eval(net, b, which=which)
        for k in which:
            np.testing.assert_array_equal(part[k], out[k], err_msg=str(which))


def test_bounded_wait_timeout_is_reported_and_context_survives(ex):
    """Every bus tile waits for a branch count that never arrives; the launch still ends."""
    g = synth.make_grid(73, 60, 80, 15)
    b = synth.random_batch(73, g, 4)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, use_graph=2, spin_limit=2000, test_force_timeout=1)
    import torch
    from parity_util import to_device
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"])
    out = net.outputs(b.B)
    net.eval_all(bt, out)
    with pytest.raises(ex.ExagoError) as ei:
        ex.exago_net_check(net.h)
    assert ei.value.name == "EXAGO_ETIMEOUT"
    ex.exago_net_check(net.h)          # the word was cleared
    ex.exago_net_set_config(net.h, schedule=2)
    good = gpu_eval(net, b)            # the context is still usable
    ex.exago_net_set_config(net.h, schedule=1)
    ref = gpu_eval(net, b)
    for k in ref:
        np.testing.assert_array_equal(good[k], ref[k])


def test_autotune_picks_a_valid_configuration(ex):
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 64)
    net = ex.Net(g)
    from parity_util import to_device
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"])
    out = net.outputs(b.B)
    best = ex.exago_net_autotune(net.h, bt, out["f"], out["grad"], out["gh"], out["jval"],
                                 out["hval"], reps=3)
    assert best["schedule"] in (1, 2, 3)
    ex.exago_net_set_config(net.h)     # automatic: uses the tuned choice for B = 64
    got = ex.exago_net_get_config(net.h, 64)
    assert got["schedule"] == best["schedule"]
    a = gpu_eval(net, b)
    ex.exago_net_set_config(net.h, schedule=1)
    k = gpu_eval(net, b)
    for key in a:
        np.testing.assert_array_equal(a[key], k[key])


def test_profile_names_the_persistent_kernel(ex):
    g = synth.grid_30bus()
    b = synth.random_batch(1, g, 8)
    net = ex.Net(g)
    from parity_util import to_device
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"])
    out = net.outputs(b.B)
    ex.exago_net_set_config(net.h, schedule=2)
    prof = ex.exago_eval_profile(net.h, bt, out["f"], out["grad"], out["gh"], out["jval"],
                                 out["hval"], reps=3)
    assert prof[0][0] == "persistent" and prof[0][1] > 0
    ph = dict(prof[1:])
    assert len(ph) == 7 and all(n.startswith("phase: ") for n in ph)
    span = ph["phase: first CTA entry to last CTA exit"]
    # the device-timed span fits inside the event-timed interval (which adds the counters'
    # memset and the launch); phases of eight states overlap, but each lies within the span
    assert 0 <= span <= prof[0][1] * 1.05 + 2e-3
    for n in ("phase: first to last branch item (start to end)",
              "phase: first to last bus item (start to end)",
              "phase: objective (first start to last end)"):
        assert 0 <= ph[n] <= span, n
    # without the objective its phase is left out
    prof = ex.exago_eval_profile(net.h, bt, None, out["grad"], out["gh"], out["jval"],
                                 out["hval"], reps=2)
    assert "phase: objective (first start to last end)" not in dict(prof)
    ex.exago_net_set_config(net.h, schedule=1)
    prof = ex.exago_eval_profile(net.h, bt, out["f"], out["grad"], out["gh"], out["jval"],
                                 out["hval"], reps=3)
    assert [n for n, _ in prof] == ["branch", "bus", "grad", "obj"]
    ex.exago_net_set_config(net.h, schedule=3)
    prof = ex.exago_eval_profile(net.h, bt, out["f"], out["grad"], out["gh"], out["jval"],
                                 out["hval"], reps=3)
    assert [n for n, _ in prof] == ["pipelined"]
