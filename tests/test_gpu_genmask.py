"""GPU: generator outages (the batch's per-state generator mask; Sec. V-A: a contingency may be a
generator outage, alone or with a line) through every schedule, the adjoint products and the
cartesian formulation, against the oracle on the same seeded inputs, element by element, within
|gpu - oracle| <= 1e-11 max(1, |oracle|); every schedule bitwise equal to the others.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import assert_close, compare_instance, gpu_eval, oracle_eval, to_device
from test_gpu_schedules import CONFIGS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def test_generator_outages_every_schedule(ex, oracle_mod):
    g = synth.make_grid(91, 300, 389, 77, transformer_frac=0.3, shunts=True)
    b = synth.generator_contingency_batch(91, g, 23)
    b.pd_scale = np.exp(0.1 * np.random.default_rng(91).normal(size=(b.B, g.nb)))
    b.sigma = 0.8
    net = ex.Net(g)
    outs = []
    for cfg in CONFIGS:
        ex.exago_net_set_config(net.h, **cfg)
        outs.append(gpu_eval(net, b))
    for o in outs[1:]:
        for k in outs[0]:
            np.testing.assert_array_equal(o[k], outs[0][k], err_msg=k)
    for i in range(b.B):
        compare_instance(outs[0], i, oracle_eval(oracle_mod, g, b, i), f"gen outage [{i}]")
    net.close()


def test_generator_outages_full_size(ex, oracle_mod):
    """2,000-bus grid x 512 generator contingencies (every third with a line outage too), the
    default launch configuration; sampled states against the oracle."""
    g = synth.grid_2000()
    b = synth.generator_contingency_batch(92, g, 512)
    net = ex.Net(g)
    out = gpu_eval(net, b)
    for i in (0, 1, 2, 255, 499, 511):
        compare_instance(out, i, oracle_eval(oracle_mod, g, b, i), f"2000-bus gen outage [{i}]")
    net.close()


def test_generator_outages_adjoints(ex, oracle_mod):
    import scipy.sparse as sp
    import torch
    g = synth.make_grid(93, 200, 260, 50, shunts=True)
    b = synth.random_batch(93, g, 4, masks=True, obj_weight=True, sigma=0.7, gen_masks=True)
    rng = np.random.default_rng(93)
    u = rng.normal(size=(b.B, g.n))
    v = rng.normal(size=(b.B, g.m))
    net = ex.Net(g)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], None, d["obj_weight"], b.sigma,
                       gen_mask=d["gen_mask"])
    U, V = torch.as_tensor(u, device="cuda"), torch.as_tensor(v, device="cuda")
    jvp = torch.empty(b.B, g.m, dtype=torch.float64, device="cuda")
    jtv = torch.empty(b.B, g.n, dtype=torch.float64, device="cuda")
    hvp = torch.empty(b.B, g.n, dtype=torch.float64, device="cuda")
    ex.exago_eval_jvp(net.h, bt, U, jvp)
    ex.exago_eval_jtv(net.h, bt, V, jtv)
    ex.exago_eval_hvp(net.h, bt, U, hvp)
    torch.cuda.synchronize()
    for i in range(b.B):
        r = oracle_eval(oracle_mod, g, b, i)
        J = sp.csr_matrix((r["J"][2], r["J"][1], r["J"][0]), shape=(g.m, g.n))
        L = sp.csr_matrix((r["H"][2], r["H"][1], r["H"][0]), shape=(g.n, g.n))
        H = L + L.T - sp.diags(L.diagonal())
        assert_close(jvp[i].cpu().numpy(), J @ u[i], f"J u [{i}]")
        assert_close(jtv[i].cpu().numpy(), J.T @ v[i], f"J' v [{i}]")
        assert_close(hvp[i].cpu().numpy(), H @ u[i], f"H u [{i}]")
    net.close()


def test_generator_outages_cartesian(ex, oracle_mod):
    import scipy.sparse as sp
    import torch
    from test_gpu_cartesian import oracle_cart, run_cart, to_cartesian
    g = synth.make_grid(94, 200, 260, 50, shunts=True)
    b = synth.random_batch(94, g, 4, masks=True, obj_weight=True, sigma=0.6, gen_masks=True)
    x, lam = to_cartesian(g, b, 94)
    net = ex.Net(g)
    out = run_cart(ex, net, b, x, lam)
    mc = g.m + g.nb
    rng = np.random.default_rng(94)
    u = rng.normal(size=(b.B, g.n))
    v = rng.normal(size=(b.B, mc))
    d = to_device(b)
    # the batch holds raw device pointers: keep the tensors alive while it is used
    X, LAM = torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")
    bt = ex.make_batch(X, LAM, d["mask"], None, d["obj_weight"], b.sigma, gen_mask=d["gen_mask"])
    jtv = torch.empty(b.B, g.n, dtype=torch.float64, device="cuda")
    hvp = torch.empty(b.B, g.n, dtype=torch.float64, device="cuda")
    ex.exago_eval_cart_jtv(net.h, bt, torch.as_tensor(v, device="cuda"), jtv)
    ex.exago_eval_cart_hvp(net.h, bt, torch.as_tensor(u, device="cuda"), hvp)
    torch.cuda.synchronize()
    for i in range(b.B):
        r = oracle_cart(oracle_mod, g, b, x, lam, i)
        assert_close(out["f"][i], r["f"], f"cart f [{i}]")
        assert_close(out["grad"][i], r["grad"], f"cart grad [{i}]")
        assert_close(out["gh"][i], r["gh"], f"cart gh [{i}]")
        assert_close(out["jval"][i], r["J"][2], f"cart J [{i}]")
        assert_close(out["hval"][i], r["H"][2], f"cart H [{i}]")
        J = sp.csr_matrix((r["J"][2], r["J"][1], r["J"][0]), shape=(mc, g.n))
        L = sp.csr_matrix((r["H"][2], r["H"][1], r["H"][0]), shape=(g.n, g.n))
        H = L + L.T - sp.diags(L.diagonal())
        assert_close(jtv[i].cpu().numpy(), J.T @ v[i], f"cart J' v [{i}]")
        assert_close(hvp[i].cpu().numpy(), H @ u[i], f"cart H u [{i}]")
    net.close()
