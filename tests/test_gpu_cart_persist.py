"""GPU: the persistent schedule of the cartesian evaluation (exago_eval_cart's default).

One launch claims (state, 128 branches) and (state, 128 buses) items from the polar model's work
list; every item computes what the chunked two-stream schedule computes for it, so the two
schedules must agree bit for bit on every output.  Checked on grids with outages, shunts, load
scales, objective weights, generator masks, parallel branches and phase shifters; on the
2,000-bus N-1 batch with the ring of records reused many times over (default ring, a caller
workspace of two ring slots, a configured lag and ring); through the net's graph cache (repeated
calls, and calls after the arguments change); with the bounded waits forced to give up (the
timeout is reported and the context stays usable); and through the server, where a cartesian
request gives what the request gives alone.  Parity against the oracle runs in
test_gpu_cartesian.py and test_gpu_shift.py on the same default schedule.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import assert_close
from test_gpu_cartesian import oracle_cart, run_cart, to_cartesian

pytestmark = pytest.mark.gpu

PERSISTENT = dict(schedule=2)
CHUNKED = dict(schedule=3)


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def parallel_grid():
    from test_capi_host import parallel_grid as pg
    return pg()


CASES = {
    "30bus_outages": (lambda: synth.grid_30bus(), dict(B=4, masks=True, sigma=0.8)),
    "300bus_scales_weights_genmasks": (
        lambda: synth.make_grid(61, 300, 389, 77, transformer_frac=0.3, shunts=True),
        dict(B=7, masks=True, pd_scale=True, obj_weight=True, sigma=0.7, gen_masks=True)),
    "parallel_branches": (parallel_grid, dict(B=3, masks=True, sigma=1.0)),
    "shifters": (lambda: synth.make_grid(101, 300, 390, 75, transformer_frac=0.1, shunts=True,
                                         shifter_frac=0.3),
                 dict(B=6, masks=True, pd_scale=True, sigma=0.9)),
    "one_state": (lambda: synth.make_grid(5, 700, 910, 170, shunts=True), dict(B=1, sigma=1.0)),
}


def both(ex, net, b, x, lam, which=("f", "grad", "gh", "jval", "hval"), workspace=None, **cfg):
    ex.exago_net_set_config(net.h, **dict(PERSISTENT, **cfg))
    p = run_cart(ex, net, b, x, lam, which, workspace=workspace)
    ex.exago_net_check(net.h)
    ex.exago_net_set_config(net.h, **CHUNKED)
    c = run_cart(ex, net, b, x, lam, which)
    ex.exago_net_set_config(net.h)
    return p, c


@pytest.mark.parametrize("name", sorted(CASES))
def test_persistent_equals_chunked_and_oracle(ex, oracle_mod, name):
    mk, kw = CASES[name]
    g = mk()
    kw = dict(kw)
    B = kw.pop("B")
    b = synth.random_batch(81, g, B, **kw)
    x, lam = to_cartesian(g, b, 81)
    net = ex.Net(g)
    p, c = both(ex, net, b, x, lam)
    for k in c:
        np.testing.assert_array_equal(p[k], c[k], err_msg=f"{name} {k}")
    i = B - 1
    r = oracle_cart(oracle_mod, g, b, x, lam, i)
    assert_close(p["gh"][i], r["gh"], f"{name} gh[{i}]")
    assert_close(p["hval"][i], r["H"][2], f"{name} H[{i}]")
    # subsets of outputs: the objective rides on bus item 0 only when rows are wanted
    for which in (("f",), ("grad",), ("gh",), ("jval",), ("hval",), ("f", "gh"), ("grad", "hval")):
        ps, cs = both(ex, net, b, x, lam, which)
        for k in which:
            np.testing.assert_array_equal(ps[k], c[k], err_msg=f"{name} {which}")
            np.testing.assert_array_equal(cs[k], c[k], err_msg=f"{name} {which} chunked")
    net.close()


@pytest.mark.parametrize("shift", [0.0, 0.2])
@pytest.mark.parametrize("cfg", [dict(occupancy=8), dict(occupancy=24), dict(stage_records=2),
                                 dict(occupancy=24, stage_records=2)])
def test_launch_variants_equal_chunked(ex, cfg, shift):
    """Every register-occupancy variant, with rows staged in shared memory or stored directly,
    with and without phase shifters, equals the chunked schedule bit for bit."""
    g = synth.make_grid(87, 1200, 1560, 300, shunts=True, shifter_frac=shift)
    b = synth.random_batch(87, g, 37, masks=True, pd_scale=True, gen_masks=True, sigma=0.6)
    x, lam = to_cartesian(g, b, 87)
    net = ex.Net(g)
    p, c = both(ex, net, b, x, lam, **cfg)
    for k in c:
        np.testing.assert_array_equal(p[k], c[k], err_msg=f"{cfg} {k}")
    net.close()


def test_ring_reuse_small_workspace_and_configured_lag(ex, oracle_mod):
    """2,000-bus grid x 300 N-1 states: the default ring (fewer slots than states), a caller
    workspace that holds only two ring slots and the counters (lag 1), and a configured lag 3 and
    ring 5 all equal the chunked schedule bit for bit."""
    import torch
    g = synth.grid_2000()
    b = synth.contingency_batch(11, g, 300)
    x, lam = to_cartesian(g, b, 11)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, **CHUNKED)
    ref = run_cart(ex, net, b, x, lam)
    ex.exago_net_set_config(net.h)
    got = run_cart(ex, net, b, x, lam)
    ex.exago_net_check(net.h)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"default ring {k}")
    slot = 2 * g.nl * 14 * 8
    counters = (1 + 2 * b.B) * 4
    nbytes = ((2 * slot + 255) // 256 * 256 + (counters + 255) // 256 * 256)
    ws = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
    got = run_cart(ex, net, b, x, lam, workspace=ws)
    ex.exago_net_check(net.h)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"two slots {k}")
    small = torch.empty((nbytes - 512) // 8, dtype=torch.float64, device="cuda")
    with pytest.raises(ex.ExagoError) as ei:
        run_cart(ex, net, b, x, lam, workspace=small)
    assert ei.value.name == "EXAGO_EINVAL"
    ex.exago_net_set_config(net.h, schedule=2, lag=3, ring=5)
    got = run_cart(ex, net, b, x, lam)
    ex.exago_net_check(net.h)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"lag 3 ring 5 {k}")
    for i in (0, 299):
        r = oracle_cart(oracle_mod, g, b, x, lam, i)
        assert_close(got["jval"][i], r["J"][2], f"2000-bus J[{i}]")
    net.close()


def test_graph_cache_replays_and_follows_new_arguments(ex):
    """Repeated calls with the same arguments replay a captured graph (from the second call); a
    call with other buffers, or with another objective factor, launches anew.  Every result equals
    the uncached launch's bit for bit."""
    import torch
    from parity_util import to_device
    g = synth.make_grid(83, 900, 1170, 225, shunts=True)
    b = synth.random_batch(83, g, 40, masks=True, pd_scale=True)
    x, lam = to_cartesian(g, b, 83)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, use_graph=2)
    ref = run_cart(ex, net, b, x, lam)
    ex.exago_net_set_config(net.h, schedule=2, use_graph=1)
    d = to_device(b)
    X, LAM = torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")
    n, me, mi, nj, nh = ex.exago_net_dims_cart(net.h)
    outs = {"f": (b.B,), "grad": (b.B, n), "gh": (b.B, me + mi), "jval": (b.B, nj),
            "hval": (b.B, nh)}
    O = {k: torch.empty(s, dtype=torch.float64, device="cuda") for k, s in outs.items()}
    bt = ex.make_batch(X, LAM, d["mask"], d["pd_scale"], None, b.sigma)
    for rep in range(4):
        for t in O.values():
            t.fill_(np.nan)
        ex.exago_eval_cart(net.h, bt, O["f"], O["grad"], O["gh"], O["jval"], O["hval"])
        torch.cuda.synchronize()
        for k in outs:
            np.testing.assert_array_equal(O[k].cpu().numpy(), ref[k], err_msg=f"rep {rep} {k}")
    # the same buffers with another objective factor: the Hessian's generator entries change
    bt2 = ex.make_batch(X, LAM, d["mask"], d["pd_scale"], None, 0.25)
    ex.exago_eval_cart(net.h, bt2, None, None, None, None, O["hval"])
    torch.cuda.synchronize()
    ex.exago_net_set_config(net.h, schedule=3)
    b2 = synth.Batch(x=b.x, lam=b.lam, mask=b.mask, pd_scale=b.pd_scale, sigma=0.25)
    alt = run_cart(ex, net, b2, x, lam, ("hval",))
    np.testing.assert_array_equal(O["hval"].cpu().numpy(), alt["hval"])
    assert not np.array_equal(alt["hval"], ref["hval"])
    ex.exago_net_check(net.h)
    net.close()


def test_bounded_wait_timeout_is_reported_and_context_survives(ex):
    """Every bus item waits for a branch count that never arrives; the launch still ends, the
    status word reports EXAGO_ETIMEOUT once, and the next evaluation is clean."""
    g = synth.make_grid(73, 60, 80, 15)
    b = synth.random_batch(73, g, 4)
    x, lam = to_cartesian(g, b, 73)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, use_graph=2, spin_limit=2000, test_force_timeout=1)
    run_cart(ex, net, b, x, lam)
    with pytest.raises(ex.ExagoError) as ei:
        ex.exago_net_check(net.h)
    assert ei.value.name == "EXAGO_ETIMEOUT"
    ex.exago_net_check(net.h)          # the word was cleared
    ex.exago_net_set_config(net.h, schedule=2)
    good = run_cart(ex, net, b, x, lam)
    ex.exago_net_check(net.h)
    ex.exago_net_set_config(net.h, schedule=3)
    ref = run_cart(ex, net, b, x, lam)
    for k in ref:
        np.testing.assert_array_equal(good[k], ref[k])
    net.close()


def test_served_cartesian_requests_equal_requests_alone(ex):
    """Cartesian and polar requests on one server, several in flight: each cartesian result
    equals exago_eval_cart on the request alone, bit for bit, and each polar one exago_eval_all's."""
    import torch
    from parity_util import gpu_eval, to_device
    g = synth.make_grid(85, 500, 650, 125, shunts=True)
    net = ex.Net(g)
    srv = ex.exago_serve_create(1 << 30, 4, 3)
    try:
        cid = ex.exago_serve_register_cart(srv, net.h)
        pid = ex.exago_serve_register(srv, net.h)
        n, me, mi, nj, nh = ex.exago_net_dims_cart(net.h)
        reqs = []
        for k, B in enumerate((1, 3, 1, 8, 2, 1)):
            b = synth.random_batch(200 + k, g, B, masks=True, pd_scale=k % 2 == 0,
                                   obj_weight=k % 3 == 0, sigma=0.5 + 0.1 * k)
            x, lam = to_cartesian(g, b, 200 + k)
            d = to_device(b)
            X, LAM = torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")
            bt = ex.make_batch(X, LAM, d["mask"], d["pd_scale"], d["obj_weight"], b.sigma)
            O = {"f": torch.empty(B, dtype=torch.float64, device="cuda"),
                 "grad": torch.empty(B, n, dtype=torch.float64, device="cuda"),
                 "gh": torch.empty(B, me + mi, dtype=torch.float64, device="cuda"),
                 "jval": torch.empty(B, nj, dtype=torch.float64, device="cuda"),
                 "hval": torch.empty(B, nh, dtype=torch.float64, device="cuda")}
            t = ex.exago_serve_submit(srv, cid, bt, O["f"], O["grad"], O["gh"], O["jval"], O["hval"])
            pol = net.outputs(B)
            dp = ex.make_batch(d["x"], d["lam"], d["mask"], d["pd_scale"], d["obj_weight"], b.sigma)
            tp = ex.exago_serve_submit(srv, pid, dp, pol["f"], pol["grad"], pol["gh"], pol["jval"],
                                       pol["hval"])
            reqs.append((b, x, lam, O, t, pol, tp, (X, LAM, d, bt, dp)))
        for b, x, lam, O, t, pol, tp, _keep in reqs:
            ex.exago_serve_wait(srv, t, 60_000)
            ex.exago_serve_wait(srv, tp, 60_000)
        torch.cuda.synchronize()
        for b, x, lam, O, t, pol, tp, _keep in reqs:
            alone = run_cart(ex, net, b, x, lam)
            for k in alone:
                np.testing.assert_array_equal(O[k].cpu().numpy(), alone[k], err_msg=f"cart {k}")
            palone = gpu_eval(net, b)
            for k in palone:
                np.testing.assert_array_equal(pol[k].cpu().numpy(), palone[k], err_msg=f"polar {k}")
    finally:
        ex.exago_serve_destroy(srv)
    ex.exago_net_check(net.h)
    net.close()
