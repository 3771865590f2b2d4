"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Sizes span several 128-thread tiles with ragged tails; the paper-sized workloads (30-bus single,
10,000-bus single, 2,000-bus x 512 N-1 contingencies, 10,000-bus x 64 load scenarios) are
compared on sampled instances the oracle evaluates one by one.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import TOL, assert_close, compare_instance, gpu_eval, oracle_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def test_30bus_against_oracle_and_golden(ex, oracle_mod):
    import json, os
    g = synth.grid_30bus()
    b = synth.random_batch(7, g, 2, masks=True, sigma=0.8)
    b.mask[0, :] = 1
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in range(b.B):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), "30-bus")
    stored = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_30bus.json")))
    for i, s in enumerate(stored["instances"]):
        assert_close(out["gh"][i], s["gh"], "golden gh")
        assert_close(out["jval"][i], s["J_val"], "golden J")
        assert_close(out["hval"][i], s["H_val"], "golden H")
        assert_close(out["f"][i], s["f"], "golden f")


@pytest.mark.parametrize("sigma", [0.0, 0.7])
def test_ragged_batch_with_masks_scales_weights(ex, oracle_mod, sigma):
    g = synth.make_grid(13, 300, 389, 77, transformer_frac=0.3, shunts=True)
    b = synth.random_batch(13, g, 5, masks=True, pd_scale=True, obj_weight=True, sigma=sigma)
    b.mask[2, :] = 0          # every branch out of service
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in range(b.B):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"300-bus sigma={sigma}")


def test_signed_zero_and_subnormal_inputs(ex, oracle_mod):
    """Doubling on the integer pipe must equal 2 x for +-0 and subnormal multipliers, voltages and
    loads; flat angles give sin = 0 and cos = 1 exactly."""
    g = synth.make_grid(17, 200, 260, 50, shunts=True)
    b = synth.random_batch(17, g, 4, masks=True, sigma=0.5)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2e-308, 1e-310, -1e-310])
    rng = np.random.default_rng(17)
    for i in range(b.B):
        idx = rng.choice(g.m, size=64, replace=False)
        b.lam[i, idx] = rng.choice(special, size=64)
    b.x[1, :g.nb] = 0.0                      # flat angles
    b.x[2, g.nb:2 * g.nb][::7] = -0.0 * 1.0  # signed-zero voltages at some buses
    b.x[3, 2 * g.nb:] = rng.choice(special, size=2 * g.ng)
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in range(b.B):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"special inputs [{i}]")


def test_parallel_branches_and_shared_generator_bus(ex, oracle_mod):
    from test_capi_host import parallel_grid
    g = parallel_grid()
    b = synth.random_batch(5, g, 3, masks=True, pd_scale=True)
    b.mask[1] = [1, 0, 1, 1, 0, 1]
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in range(b.B):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), "parallel")


def test_isolated_and_zero_voltage_buses(ex, oracle_mod):
    """The bus balances come from the sums of the ends' derivatives (degree-2 homogeneity in the
    voltage magnitudes).  Cases where those sums are empty or degenerate: a bus whose every branch
    is out of service (its balance is shunt, load and generation only), a bus at zero or negative
    zero voltage, a bus with no branch at all, and very large shunts next to small flows."""
    g = synth.make_grid(81, 40, 52, 9, shunts=True)
    # one more bus, with a shunt, a load and a generator but no branch
    g = synth.Grid(**{**g.__dict__, "nb": g.nb + 1,
                      "Gs": np.append(g.Gs, 0.03), "Bs": np.append(g.Bs, -0.02),
                      "Pd": np.append(g.Pd, 0.4), "Qd": np.append(g.Qd, 0.1),
                      "gbus": np.append(g.gbus, g.nb).astype(np.int32), "c2": np.append(g.c2, 0.02),
                      "c1": np.append(g.c1, 15.0), "c0": np.append(g.c0, 1.0)})
    nb = g.nb
    g.Gs[3] = 250.0                          # large shunt: the balance must not lose its flow terms
    b = synth.random_batch(81, g, 6, masks=True, pd_scale=True, sigma=0.5)
    deg = np.bincount(np.concatenate([g.f, g.t]), minlength=nb)
    at = lambda i: np.flatnonzero((g.f == i) | (g.t == i))
    b.mask[0, :] = 1
    b.mask[0, at(7)] = 0                     # every branch of bus 7 out of service
    b.mask[1, :] = 0                         # every branch out: balances are shunts, loads, gens
    b.x[2, nb + 9] = 0.0                     # zero voltage
    b.x[3, nb + 11] = -0.0                   # negative zero
    b.x[4, nb:2 * nb] = 1.0
    b.x[4, :nb] = 0.0                        # flat start
    b.mask[5, at(int(np.argmax(deg)))] = 0   # the busiest bus loses all its branches
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in range(b.B):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"isolated/zero-V [{i}]")


def test_single_bus_no_branches(ex, oracle_mod):
    g = synth.Grid(nb=1, Gs=np.array([0.1]), Bs=np.array([0.2]), Pd=np.array([0.3]),
                   Qd=np.array([0.1]), f=np.zeros(0, np.int32), t=np.zeros(0, np.int32),
                   r=np.zeros(0), x=np.zeros(0), b=np.zeros(0), tap=np.zeros(0),
                   rateA=np.zeros(0), gbus=np.zeros(2, np.int32), c2=np.array([0.01, 0.02]),
                   c1=np.array([10.0, 12.0]), c0=np.array([1.0, 0.5]))
    b = synth.random_batch(2, g, 2)
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in range(b.B):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), "1-bus")


def test_entry_points_equal_fused_call(ex):
    import torch
    g = synth.make_grid(17, 200, 260, 50, shunts=True)
    b = synth.random_batch(17, g, 3, masks=True, pd_scale=True, obj_weight=True, sigma=0.5)
    net = ex.Net(g)
    full = gpu_eval(net, b)
    from parity_util import to_device
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], d["pd_scale"], d["obj_weight"], b.sigma)
    o = net.outputs(b.B)
    ex.exago_eval_obj(net.h, bt, o["f"])
    ex.exago_eval_grad(net.h, bt, o["grad"])
    ex.exago_eval_cons(net.h, bt, o["gh"])
    ex.exago_eval_jac(net.h, bt, o["jval"])
    ex.exago_eval_hess(net.h, bt, o["hval"])
    torch.cuda.synchronize()
    for k in full:
        np.testing.assert_array_equal(o[k].cpu().numpy(), full[k], err_msg=k)


def test_deterministic_and_batch_composition_invariant(ex):
    """Repeat calls are bitwise equal, and an instance gives the same bits alone or in a batch."""
    g = synth.make_grid(19, 500, 650, 120, shunts=True)
    b = synth.random_batch(19, g, 6, masks=True, pd_scale=True, obj_weight=True)
    net = ex.Net(g)
    a1 = gpu_eval(net, b)
    a2 = gpu_eval(net, b)
    for k in a1:
        np.testing.assert_array_equal(a1[k], a2[k])
    one = synth.Batch(x=b.x[3:4], lam=b.lam[3:4], mask=b.mask[3:4], pd_scale=b.pd_scale[3:4],
                      obj_weight=b.obj_weight[3:4], sigma=b.sigma)
    s = gpu_eval(net, one)
    for k in a1:
        np.testing.assert_array_equal(s[k][0], a1[k][3], err_msg=k)


def test_caller_workspace_equals_internal(ex):
    import torch
    g = synth.make_grid(23, 120, 160, 30)
    b = synth.random_batch(23, g, 4, masks=True)
    net = ex.Net(g)
    a = gpu_eval(net, b)
    nbytes = ex.exago_eval_workspace_size(net.h, b.B)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    c = gpu_eval(net, b, workspace=ws)
    for k in a:
        np.testing.assert_array_equal(a[k], c[k])


def test_more_states_than_one_grid_row(ex, oracle_mod):
    """B > 65535 exercises the launcher's chunking over the grid's y dimension."""
    g = synth.make_grid(29, 3, 3, 1)
    B = 65535 + 70
    rng = np.random.default_rng(29)
    base = synth.random_batch(29, g, 1, masks=False)
    x = base.x[0][None, :] + rng.normal(0, 0.02, (B, g.n))
    lam = base.lam[0][None, :] + rng.normal(0, 0.5, (B, g.m))
    mask = (rng.random((B, g.nl)) > 0.3).astype(np.uint8)
    b = synth.Batch(x=x, lam=lam, mask=mask, sigma=1.0)
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in [0, 1, 65534, 65535, 65536, B - 1]:
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), "chunked")


def test_empty_batch_is_a_noop(ex):
    import torch
    g = synth.grid_30bus()
    net = ex.Net(g)
    x = torch.zeros(0, net.n, dtype=torch.float64, device="cuda")
    bt = ex.make_batch(x, x, None)
    ex.exago_eval_all(net.h, bt)
    torch.cuda.synchronize()


def test_argument_errors(ex):
    import ctypes
    import torch
    g = synth.grid_30bus()
    net = ex.Net(g)
    x = torch.zeros(2, net.n, dtype=torch.float64, device="cuda")
    hv = torch.zeros(2, net.nnzH, dtype=torch.float64, device="cuda")
    bt = ex.make_batch(x, None, None)
    with pytest.raises(ex.ExagoError) as ei:   # the Hessian needs lambda
        ex.exago_eval_hess(net.h, bt, hv)
    assert ei.value.name == "EXAGO_EINVAL"
    bt2 = ex.make_batch(x, x, None)
    bt2.workspace = ctypes.c_void_p(hv.data_ptr())
    bt2.workspace_bytes = 8
    with pytest.raises(ex.ExagoError) as ei:
        ex.exago_eval_jac(net.h, bt2, hv)
    assert ei.value.name == "EXAGO_EINVAL"
    bt3 = ex.make_batch(x, x, None)
    bt3.x = None
    with pytest.raises(ex.ExagoError):
        ex.exago_eval_cons(net.h, bt3, hv)
    bt4 = ex.make_batch(x, x, None)
    bt4.B = -1
    with pytest.raises(ex.ExagoError):
        ex.exago_eval_cons(net.h, bt4, hv)
    for bad in (dict(tile_group=5), dict(block=48), dict(occupancy=12), dict(lag=4, ring=4)):
        with pytest.raises(ex.ExagoError) as ei:
            ex.exago_net_set_config(net.h, **bad)
        assert ei.value.name == "EXAGO_EINVAL"


# ---- paper-sized workloads, sampled ---------------------------------------------------------

def test_10k_bus_single_instance(ex, oracle_mod):
    g = synth.grid_10k()
    b = synth.random_batch(2, g, 1, sigma=1.0)
    net = ex.Net(g)
    out = gpu_eval(net, b)
    compare_instance(out, 0, oracle_eval(oracle_mod, g, b, 0), "10k")


def test_70k_bus_largest_serving_grid(ex, oracle_mod):
    """The largest grid of the serving mix (70,000 buses, 91,000 branches): two states, the
    second with masks and load scales, each against the oracle."""
    g = synth.grid_sized(53, 70_000)
    b = synth.random_batch(53, g, 2, masks=True, pd_scale=True, sigma=0.9)
    b.mask[0, :] = 1
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in range(2):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"70k [{i}]")


def test_2000_bus_512_contingencies_sampled(ex, oracle_mod):
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 512)
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in [0, 1, 137, 255, 256, 400, 510, 511]:
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), "N-1")
    # the outaged branch's h rows are exactly zero
    out_l = b.meta["outage"]
    assert np.all(out["gh"][np.arange(512), 2 * g.nb + out_l] == 0.0)
    assert np.all(out["gh"][np.arange(512), 2 * g.nb + g.nl + out_l] == 0.0)


def test_10k_bus_64_scenarios_sampled(ex, oracle_mod):
    g = synth.grid_10k()
    b = synth.scenario_batch(4, g, 64)
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in [0, 31, 63]:
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), "scenarios")


@pytest.mark.parametrize("grid,batch,cfg,sample", [
    # the launch configuration bench.py times on the 2,000-bus x 512 N-1 workload
    ("2000", "n1", dict(schedule=2, block=64, occupancy=16, stage_records=2, tile_group=1),
     [0, 255, 511]),
    # the configuration the autotuner picks for the 10,000-bus x 64 scenario workload
    ("10k", "scen", dict(schedule=2, block=128, occupancy=16, tile_group=1), [0, 63]),
])
def test_full_size_in_the_benchmarked_configuration(ex, oracle_mod, grid, batch, cfg, sample):
    g = synth.grid_2000() if grid == "2000" else synth.grid_10k()
    b = synth.contingency_batch(3, g, 512) if batch == "n1" else synth.scenario_batch(4, g, 64)
    net = ex.Net(g)
    default = gpu_eval(net, b)
    ex.exago_net_set_config(net.h, **cfg)
    out = gpu_eval(net, b)
    for k in default:
        np.testing.assert_array_equal(out[k], default[k], err_msg=k)
    for i in sample:
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"benchmarked config [{i}]")


def test_batch_keeps_its_tensors_alive(ex, oracle_mod):
    """make_batch holds references to the tensors whose device pointers it stores: a batch built
    from temporaries stays valid after the caller's references are gone and new allocations
    have been made."""
    import gc
    import torch
    g = synth.make_grid(131, 120, 160, 30, shunts=True)
    b = synth.random_batch(131, g, 3, masks=True, sigma=0.7)
    net = ex.Net(g)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    bt = ex.make_batch(t(b.x, torch.float64), t(b.lam, torch.float64), t(b.mask, torch.uint8),
                       obj_factor=b.sigma)
    gc.collect()
    junk = [torch.full((b.B, g.n), np.nan, dtype=torch.float64, device="cuda") for _ in range(8)]
    out = net.outputs(b.B)
    net.eval_all(bt, out)
    torch.cuda.synchronize()
    host = {k: v.cpu().numpy() for k, v in out.items()}
    for i in range(b.B):
        compare_instance(host, i, oracle_eval(oracle_mod, g, b, i), f"temporaries [{i}]")
    del junk
    net.close()
