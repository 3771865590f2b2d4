"""GPU parity with phase-shifting transformers (nets made by exago_net_create_shift).

A phase shifter gives the branch's two ends different mutual admittances (-ys/conj(T) and
-ys/T, T = tau e^{j phi}).  The kernels that allow it read the to end's own pair: the persistent
schedule's general variant, the multi-kernel and pipelined branch kernel, the adjoint kernels and
the cartesian kernels' phase-shifter variants.  Every output is compared with the oracle element
by element, |gpu - oracle| <= 1e-11 max(1, |oracle|), on grids with 10-30% shifters, up to the
2,000-bus x 512 N-1 batch in the benchmarked launch configuration.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import assert_close, compare_instance, gpu_eval, oracle_eval, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def shifted_grid(seed=101, nb=300, frac=0.3):
    return synth.make_grid(seed, nb, int(round(1.3 * nb)), nb // 4, transformer_frac=0.1,
                           shunts=True, shifter_frac=frac)


@pytest.mark.parametrize("cfg", [
    dict(schedule=2),                                                       # persistent
    dict(schedule=2, block=64, occupancy=16, stage_records=2, tile_group=1),
    dict(schedule=2, block=128, stage_records=1),
    dict(schedule=1),                                                       # multi-kernel
    dict(schedule=3, chunk=2),                                              # pipelined
])
def test_eval_all_against_oracle(ex, oracle_mod, cfg):
    g = shifted_grid()
    b = synth.random_batch(101, g, 5, masks=True, pd_scale=True, obj_weight=True, sigma=0.7,
                           gen_masks=True)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, **cfg)
    out = gpu_eval(net, b)
    for i in range(b.B):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"shift {cfg} [{i}]")


def test_schedules_bitwise_equal(ex):
    g = shifted_grid(103)
    b = synth.random_batch(103, g, 7, masks=True, sigma=0.9)
    net = ex.Net(g)
    outs = []
    for cfg in (dict(schedule=1), dict(schedule=2), dict(schedule=3, chunk=3)):
        ex.exago_net_set_config(net.h, **cfg)
        outs.append(gpu_eval(net, b))
    for o in outs[1:]:
        for k in outs[0]:
            np.testing.assert_array_equal(o[k], outs[0][k], err_msg=k)


def test_zero_shifts_equal_the_shift_free_net(ex):
    """A net created with all shifts 0 runs the phase-shifter variants; its to-end admittances
    equal the from end's, and every result equals the shift-free net's bit for bit."""
    g = synth.make_grid(105, 200, 260, 50, shunts=True)
    gz = synth.Grid(**{**g.__dict__, "shift": np.zeros(g.nl)})
    b = synth.random_batch(105, g, 6, masks=True, sigma=0.8)
    a = gpu_eval(ex.Net(g), b)
    z = gpu_eval(ex.Net(gz), b)
    for k in a:
        np.testing.assert_array_equal(z[k], a[k], err_msg=k)


def test_adjoint_products_against_oracle(ex, oracle_mod):
    import scipy.sparse as sp
    import torch
    g = shifted_grid(107)
    b = synth.random_batch(107, g, 4, masks=True, sigma=0.6)
    rng = np.random.default_rng(107)
    u = rng.normal(size=(b.B, g.n))
    v = rng.normal(size=(b.B, g.m))
    net = ex.Net(g)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], None, None, b.sigma)
    U, V = torch.as_tensor(u, device="cuda"), torch.as_tensor(v, device="cuda")
    jvp = torch.empty(b.B, net.m, dtype=torch.float64, device="cuda")
    jtv = torch.empty(b.B, net.n, dtype=torch.float64, device="cuda")
    hvp = torch.empty(b.B, net.n, dtype=torch.float64, device="cuda")
    ex.exago_eval_jvp(net.h, bt, U, jvp)
    ex.exago_eval_jtv(net.h, bt, V, jtv)
    ex.exago_eval_hvp(net.h, bt, U, hvp)
    torch.cuda.synchronize()
    jvp, jtv, hvp = jvp.cpu().numpy(), jtv.cpu().numpy(), hvp.cpu().numpy()
    for i in range(b.B):
        r = oracle_eval(oracle_mod, g, b, i)
        J = sp.csr_matrix((r["J"][2], r["J"][1], r["J"][0]), shape=(g.m, g.n))
        L = sp.csr_matrix((r["H"][2], r["H"][1], r["H"][0]), shape=(g.n, g.n))
        H = L + L.T - sp.diags(L.diagonal())
        assert_close(jvp[i], J @ u[i], f"shift J u [{i}]")
        assert_close(jtv[i], J.T @ v[i], f"shift J^T v [{i}]")
        assert_close(hvp[i], H @ u[i], f"shift H u [{i}]")


def test_cartesian_against_oracle(ex, oracle_mod):
    import scipy.sparse as sp
    import torch
    from test_gpu_cartesian import compare, oracle_cart, run_cart, to_cartesian
    g = shifted_grid(109, nb=200)
    b = synth.random_batch(109, g, 4, masks=True, pd_scale=True, sigma=0.8, gen_masks=True)
    x, lam = to_cartesian(g, b, 109)
    net = ex.Net(g)
    out = run_cart(ex, net, b, x, lam)
    refs = [oracle_cart(oracle_mod, g, b, x, lam, i) for i in range(b.B)]
    for i in range(b.B):
        compare(out, refs[i], i, "cartesian shift")
    # adjoint products against the oracle's cartesian J and H
    n, me, mi, nj, nh = ex.exago_net_dims_cart(net.h)
    mc = me + mi
    rng = np.random.default_rng(109)
    u = rng.normal(size=(b.B, n))
    v = rng.normal(size=(b.B, mc))
    d = to_device(b)
    X, LAM = torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")
    bt = ex.make_batch(X, LAM, d["mask"], None, None, b.sigma, gen_mask=d["gen_mask"])
    U, V = torch.as_tensor(u, device="cuda"), torch.as_tensor(v, device="cuda")
    jvp = torch.empty(b.B, mc, dtype=torch.float64, device="cuda")
    jtv = torch.empty(b.B, n, dtype=torch.float64, device="cuda")
    hvp = torch.empty(b.B, n, dtype=torch.float64, device="cuda")
    ex.exago_eval_cart_jvp(net.h, bt, U, jvp)
    ex.exago_eval_cart_jtv(net.h, bt, V, jtv)
    ex.exago_eval_cart_hvp(net.h, bt, U, hvp)
    torch.cuda.synchronize()
    jvp, jtv, hvp = jvp.cpu().numpy(), jtv.cpu().numpy(), hvp.cpu().numpy()
    for i in range(b.B):
        r = oracle_cart(oracle_mod, g, b, x, lam, i)
        J = sp.csr_matrix((r["J"][2], r["J"][1], r["J"][0]), shape=(mc, n))
        L = sp.csr_matrix((r["H"][2], r["H"][1], r["H"][0]), shape=(n, n))
        H = L + L.T - sp.diags(L.diagonal())
        assert_close(jvp[i], J @ u[i], f"cart shift J u [{i}]")
        assert_close(jtv[i], J.T @ v[i], f"cart shift J^T v [{i}]")
        assert_close(hvp[i], H @ u[i], f"cart shift H u [{i}]")


def test_served_request(ex, oracle_mod):
    import torch
    g = shifted_grid(111)
    b = synth.random_batch(111, g, 3, masks=True, sigma=0.9)
    net = ex.Net(g)
    alone = gpu_eval(net, b)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], None, None, b.sigma)
    out = net.outputs(b.B)
    srv = ex.exago_serve_create(1 << 28, max_slots=2, n_streams=2)
    try:
        nid = ex.exago_serve_register(srv, net.h)
        t = ex.exago_serve_submit(srv, nid, bt, **out)
        ex.exago_serve_wait(srv, t)
    finally:
        ex.exago_serve_destroy(srv)
    torch.cuda.synchronize()
    served = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    for k in alone:
        np.testing.assert_array_equal(served[k], alone[k], err_msg=k)
    compare_instance(served, 1, oracle_eval(oracle_mod, g, b, 1), "served shift")


def test_2000_bus_512_contingencies_with_shifters(ex, oracle_mod):
    """Full size: the 2,000-bus grid with 10% phase shifters, 512 N-1 states, in the benchmarked
    launch configuration, sampled against the oracle."""
    g = synth.make_grid(3, 2000, 2700, 500, shifter_frac=0.1)
    b = synth.contingency_batch(3, g, 512)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, block=64, occupancy=16, stage_records=2,
                            tile_group=1)
    out = gpu_eval(net, b)
    for i in [0, 200, 511]:
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"2000-bus shifters [{i}]")
