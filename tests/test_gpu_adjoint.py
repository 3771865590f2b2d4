"""GPU: adjoint kernels (J u, J^T v, Hessian-vector products) and the torch.autograd.Function
wrappers, against the oracle's J and H (sparse matvecs) and central finite differences.
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


def oracle_mats(om, g, b, i):
    import scipy.sparse as sp
    r = oracle_eval(om, g, b, i)
    J = sp.csr_matrix((r["J"][2], r["J"][1], r["J"][0]), shape=(g.m, g.n))
    L = sp.csr_matrix((r["H"][2], r["H"][1], r["H"][0]), shape=(g.n, g.n))
    H = L + L.T - sp.diags(L.diagonal())
    return J, H


def run_adjoints(ex, net, b, u, v):
    import torch
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], d["pd_scale"], d["obj_weight"], b.sigma)
    U = torch.as_tensor(u, device="cuda")
    V = torch.as_tensor(v, device="cuda")
    jvp = torch.empty(b.B, net.m, dtype=torch.float64, device="cuda")
    jtv = torch.empty(b.B, net.n, dtype=torch.float64, device="cuda")
    hvp = torch.empty(b.B, net.n, dtype=torch.float64, device="cuda")
    ex.exago_eval_jvp(net.h, bt, U, jvp)
    ex.exago_eval_jtv(net.h, bt, V, jtv)
    ex.exago_eval_hvp(net.h, bt, U, hvp)
    torch.cuda.synchronize()
    return jvp.cpu().numpy(), jtv.cpu().numpy(), hvp.cpu().numpy()


@pytest.mark.parametrize("which", ["300bus", "parallel"])
def test_adjoints_match_oracle_matvecs(ex, oracle_mod, which):
    if which == "300bus":
        g = synth.make_grid(81, 300, 389, 77, transformer_frac=0.3, shunts=True)
    else:
        from test_capi_host import parallel_grid
        g = parallel_grid()
    b = synth.random_batch(81, g, 5, masks=True, pd_scale=True, obj_weight=True, sigma=0.7)
    rng = np.random.default_rng(81)
    u = rng.normal(size=(b.B, g.n))
    v = rng.normal(size=(b.B, g.m))
    net = ex.Net(g)
    jvp, jtv, hvp = run_adjoints(ex, net, b, u, v)
    for i in range(b.B):
        J, H = oracle_mats(oracle_mod, g, b, i)
        assert_close(jvp[i], J @ u[i], f"J u [{i}]")
        assert_close(jtv[i], J.T @ v[i], f"J^T v [{i}]")
        assert_close(hvp[i], H @ u[i], f"H u [{i}]")


def test_hvp_applies_the_evaluated_hessian(ex):
    """HVP equals the exago_eval_hess values (as a symmetric matrix) times u, state by state."""
    import scipy.sparse as sp
    import torch
    g = synth.make_grid(83, 200, 260, 50, shunts=True)
    b = synth.random_batch(83, g, 3, masks=True, obj_weight=True, sigma=1.3)
    net = ex.Net(g)
    from parity_util import gpu_eval
    hv = gpu_eval(net, b, which=("hval",))["hval"]
    rowptr, col = ex.exago_net_hess_pattern(net.h)
    u = np.random.default_rng(83).normal(size=(b.B, g.n))
    _, _, hvp = run_adjoints(ex, net, b, u, np.zeros((b.B, g.m)))
    for i in range(b.B):
        L = sp.csr_matrix((hv[i], col, rowptr), shape=(g.n, g.n))
        H = L + L.T - sp.diags(L.diagonal())
        assert_close(hvp[i], H @ u[i], f"hvp vs hess [{i}]")


def test_autograd_gradcheck_and_gradgradcheck(ex):
    import torch
    from paper_2203_10587_gb300 import autograd as ag
    g = synth.make_grid(85, 12, 16, 4, shunts=True)
    net = ex.Net(g)
    b = synth.random_batch(85, g, 2, masks=True)
    mask = torch.as_tensor(b.mask, device="cuda")
    x = torch.as_tensor(b.x, device="cuda").requires_grad_(True)
    f = lambda x: ag.cons(x, net, mask)
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-6, rtol=1e-5)
    assert torch.autograd.gradgradcheck(f, (x,), eps=1e-6, atol=1e-5, rtol=1e-4)
    w = torch.as_tensor([0.3, 0.7], dtype=torch.float64, device="cuda")
    fo = lambda x: ag.obj(x, net, w)
    assert torch.autograd.gradcheck(fo, (x,), eps=1e-6, atol=1e-5, rtol=1e-6)
    assert torch.autograd.gradgradcheck(fo, (x,), eps=1e-6, atol=1e-4, rtol=1e-5)


def test_10k_bus_64_scenarios_adjoint_against_finite_differences(ex, oracle_mod):
    """Config C4: forward g(x), J^T lambda and HVP in FP64 against central FD with h = 1e-6."""
    import torch
    from paper_2203_10587_gb300 import autograd as ag
    g = synth.grid_10k()
    b = synth.scenario_batch(4, g, 64)
    net = ex.Net(g)
    d = to_device(b)
    x = d["x"].clone().requires_grad_(True)
    lam = d["lam"]
    gh = ag.cons(x, net, None, d["pd_scale"])
    # J^T lambda through autograd, and J^T lambda checked against the oracle's J on samples
    (jtl,) = torch.autograd.grad(gh, x, grad_outputs=lam, create_graph=True)
    rng = np.random.default_rng(4)
    for i in (0, 63):
        J, H = oracle_mats(oracle_mod, g, b, i)
        assert_close(jtl[i].detach().cpu().numpy(), J.T @ b.lam[i], f"J^T lambda [{i}]")
    # directional FD of lambda^T g: (lambda^T g(x + h u) - lambda^T g(x - h u)) / 2h = (J^T lambda) . u
    h = 1e-6
    u = torch.as_tensor(rng.normal(size=(b.B, g.n)), device="cuda")
    with torch.no_grad():
        gp = ag.cons(x + h * u, net, None, d["pd_scale"])
        gm = ag.cons(x - h * u, net, None, d["pd_scale"])
        fd = ((lam * (gp - gm)).sum(1)) / (2 * h)
        an = (jtl * u).sum(1)
    rel = ((fd - an).abs() / an.abs().clamp_min(1.0)).max().item()
    assert rel < 1e-6, rel
    # HVP through double backward against FD of J^T lambda
    (hu,) = torch.autograd.grad(jtl, x, grad_outputs=u)
    with torch.no_grad():
        jp = torch.empty_like(jtl)
        jm = torch.empty_like(jtl)
        ex.exago_eval_jtv(net.h, ex.make_batch((x + h * u).contiguous()), lam, jp)
        ex.exago_eval_jtv(net.h, ex.make_batch((x - h * u).contiguous()), lam, jm)
        fdh = (jp - jm) / (2 * h)
    rel = ((fdh - hu).abs() / hu.abs().clamp_min(1.0)).max().item()
    assert rel < 1e-5, rel
