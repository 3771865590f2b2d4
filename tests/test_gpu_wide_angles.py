"""GPU parity at wide branch angles.

The branch kernels take the sine and cosine of theta = Va_f - Va_t from their own minimax
polynomials while |theta| <= pi/4 (the double nearest pi/4 included) and from the library sincos
beyond.  Normal states (Va ~ N(0, 0.1)) almost never leave the polynomial's interval, so these
states put matched branches exactly on the switch point and one ulp either side, on the quarter
and half turns and beyond, and draw whole grids from Va ~ U(-pi, pi)
(synth.wide_angle_batch).  The polar injections are Sec. III, eqs. (8)-(9); the comparison is
element by element against the oracle, |gpu - oracle| <= 1e-11 max(1, |oracle|).
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import TOL, assert_close, compare_instance, gpu_eval, oracle_eval, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def grid300():
    return synth.make_grid(13, 300, 389, 77, transformer_frac=0.3, shunts=True)


@pytest.mark.parametrize("cfg", [
    dict(schedule=2),                                                   # persistent (default)
    dict(schedule=2, block=64, occupancy=16, stage_records=2, tile_group=1),   # the bench's
    dict(schedule=1),                                                   # multi-kernel
    dict(schedule=1, stage_records=1),
    dict(schedule=3, chunk=2),                                          # pipelined
    dict(schedule=2, tiling=2),                                         # branch per warp
])
def test_eval_all_against_oracle(ex, oracle_mod, cfg):
    g = grid300()
    b = synth.wide_angle_batch(5, g, 6, masks=True, sigma=0.8)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, **cfg)
    out = gpu_eval(net, b)
    for i in range(b.B):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"wide {cfg} [{i}]")


def test_schedules_bitwise_equal_at_wide_angles(ex):
    g = grid300()
    b = synth.wide_angle_batch(7, g, 9, masks=True, sigma=0.6)
    net = ex.Net(g)
    outs = []
    for cfg in (dict(schedule=1), dict(schedule=2), dict(schedule=3, chunk=4)):
        ex.exago_net_set_config(net.h, **cfg)
        outs.append(gpu_eval(net, b))
    for o in outs[1:]:
        for k in outs[0]:
            np.testing.assert_array_equal(o[k], outs[0][k], err_msg=k)


def test_adjoint_products_against_oracle(ex, oracle_mod):
    import scipy.sparse as sp
    import torch
    g = grid300()
    b = synth.wide_angle_batch(11, g, 4, masks=True, sigma=0.7)
    rng = np.random.default_rng(11)
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
    ex.exago_net_check(net.h)
    jvp, jtv, hvp = jvp.cpu().numpy(), jtv.cpu().numpy(), hvp.cpu().numpy()
    for i in range(b.B):
        r = oracle_eval(oracle_mod, g, b, i)
        J = sp.csr_matrix((r["J"][2], r["J"][1], r["J"][0]), shape=(g.m, g.n))
        L = sp.csr_matrix((r["H"][2], r["H"][1], r["H"][0]), shape=(g.n, g.n))
        H = L + L.T - sp.diags(L.diagonal())
        assert_close(jvp[i], J @ u[i], f"wide J u [{i}]")
        assert_close(jtv[i], J.T @ v[i], f"wide J^T v [{i}]")
        assert_close(hvp[i], H @ u[i], f"wide H u [{i}]")


def test_served_request_at_wide_angles(ex, oracle_mod):
    import torch
    g = grid300()
    b = synth.wide_angle_batch(13, g, 3, masks=True, sigma=0.9)
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
    for i in range(b.B):
        compare_instance(served, i, oracle_eval(oracle_mod, g, b, i), f"served wide [{i}]")


def test_2000_bus_512_states_uniform_angles(ex, oracle_mod):
    """Full size, in the benchmarked launch configuration: 512 N-1 states whose angles are drawn
    from U(-pi, pi), sampled against the oracle."""
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 512)
    rng = np.random.default_rng(3)
    b.x[:, :g.nb] = rng.uniform(-np.pi, np.pi, (512, g.nb))
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=2, block=64, occupancy=16, stage_records=2,
                            tile_group=1)
    out = gpu_eval(net, b)
    for i in [0, 100, 255, 511]:
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"uniform angles [{i}]")
