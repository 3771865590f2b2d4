"""GPU: the power-balance-cartesian evaluation (exago_eval_cart) through the C ABI against the
oracle's cartesian evaluator on the same seeded inputs, element by element, within
|gpu - oracle| <= 1e-11 max(1, |oracle|).

States are the seeded polar states of the synthetic generator mapped to e = Vm cos Va,
f = Vm sin Va, with multipliers for the voltage rows appended.  Cases: the 30-bus grid with
outages, a 300-bus grid with shunts, transformers, load scales and objective weights, a grid with
parallel branches and several generators on one bus, chunked batches (more states than one chunk
of branch-end records), subsets of outputs, a caller workspace, and the 2,000-bus x 512 N-1 batch
at full size (sampled states against the oracle, and every state against the polar GPU path at
the same point).
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import assert_close, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def to_cartesian(g, b, seed):
    """Cartesian copies of a polar synth.Batch: x -> [e | f | Pg | Qg], lambda + muV."""
    nb = g.nb
    Va, Vm = b.x[:, :nb], b.x[:, nb:2 * nb]
    x = b.x.copy()
    x[:, :nb] = Vm * np.cos(Va)
    x[:, nb:2 * nb] = Vm * np.sin(Va)
    muV = np.random.default_rng(seed).normal(size=(b.B, nb))
    lam = np.concatenate([b.lam, muV], axis=1)
    return x, lam


def run_cart(ex, net, b, x, lam, which=("f", "grad", "gh", "jval", "hval"), workspace=None):
    import torch
    d = to_device(b)
    X = torch.as_tensor(x, device="cuda")
    LAM = torch.as_tensor(lam, device="cuda")
    bt = ex.make_batch(X, LAM, d["mask"], d["pd_scale"], d["obj_weight"], b.sigma,
                       workspace=workspace, gen_mask=d["gen_mask"])
    n, me, mi, nj, nh = ex.exago_net_dims_cart(net.h)
    z = lambda *s: torch.full(s, np.nan, dtype=torch.float64, device="cuda")
    out = {"f": z(b.B), "grad": z(b.B, n), "gh": z(b.B, me + mi), "jval": z(b.B, nj),
           "hval": z(b.B, nh)}
    out = {k: (v if k in which else None) for k, v in out.items()}
    ex.exago_eval_cart(net.h, bt, out["f"], out["grad"], out["gh"], out["jval"], out["hval"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


def oracle_cart(om, g, b, x, lam, i):
    return om.evaluate(om.OracleNet(g), x[i], lam[i],
                       None if b.mask is None else b.mask[i],
                       None if b.pd_scale is None else b.pd_scale[i],
                       1.0 if b.obj_weight is None else float(b.obj_weight[i]), b.sigma,
                       cartesian=True,
                       gen_mask=None if b.gen_mask is None else b.gen_mask[i])


def compare(out, ref, i, what):
    if "f" in out:
        assert_close(out["f"][i], ref["f"], f"{what} f[{i}]")
    if "grad" in out:
        assert_close(out["grad"][i], ref["grad"], f"{what} grad[{i}]")
    if "gh" in out:
        assert_close(out["gh"][i], ref["gh"], f"{what} gh[{i}]")
    if "jval" in out:
        assert_close(out["jval"][i], ref["J"][2], f"{what} J[{i}]")
    if "hval" in out:
        assert_close(out["hval"][i], ref["H"][2], f"{what} H[{i}]")


def parallel_grid():
    from test_capi_host import parallel_grid as pg
    return pg()


CASES = {
    "30bus_outages": (lambda: synth.grid_30bus(),
                      dict(B=4, masks=True, sigma=0.8)),
    "300bus_shunts_scenarios": (lambda: synth.make_grid(61, 300, 389, 77, transformer_frac=0.3,
                                                        shunts=True),
                                dict(B=5, masks=True, pd_scale=True, obj_weight=True, sigma=0.7)),
    "parallel_branches": (parallel_grid, dict(B=3, masks=True, sigma=1.0)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_cartesian_matches_oracle(ex, oracle_mod, name):
    mk, kw = CASES[name]
    g = mk()
    B = kw.pop("B")
    b = synth.random_batch(62, g, B, **kw)
    x, lam = to_cartesian(g, b, 62)
    net = ex.Net(g)
    out = run_cart(ex, net, b, x, lam)
    for i in range(B):
        compare(out, oracle_cart(oracle_mod, g, b, x, lam, i), i, name)
    net.close()


def test_cartesian_output_subsets_and_workspace(ex, oracle_mod):
    """Every subset of outputs gives the full call's values bit for bit; a caller workspace
    gives the same values as the internal one."""
    import torch
    g = synth.make_grid(63, 120, 160, 30, shunts=True)
    b = synth.random_batch(63, g, 3, masks=True, sigma=0.9)
    x, lam = to_cartesian(g, b, 63)
    net = ex.Net(g)
    full = run_cart(ex, net, b, x, lam)
    for which in (("f",), ("grad",), ("gh",), ("jval",), ("hval",), ("gh", "hval")):
        part = run_cart(ex, net, b, x, lam, which)
        for k in which:
            np.testing.assert_array_equal(part[k], full[k], err_msg=str(which))
    ws_bytes = ex.exago_eval_cart_workspace_size(net.h, b.B)
    ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.float64, device="cuda")
    off = (-ws.data_ptr()) % 256 // 8
    wsa = ws[off:off + ws_bytes // 8]
    own = run_cart(ex, net, b, x, lam, workspace=wsa)
    for k in full:
        np.testing.assert_array_equal(own[k], full[k])
    compare(full, oracle_cart(oracle_mod, g, b, x, lam, 1), 1, "subset grid")
    net.close()


def test_cartesian_full_size_n1(ex, oracle_mod):
    """2,000-bus grid x 512 N-1 states (several chunks of records): sampled states against the
    oracle, and every state's g | h against the polar GPU path at the same point."""
    from parity_util import gpu_eval
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 512)
    x, lam = to_cartesian(g, b, 64)
    net = ex.Net(g)
    assert ex.exago_eval_cart_workspace_size(net.h, 512) < 512 * 2 * g.nl * 14 * 8
    out = run_cart(ex, net, b, x, lam)
    for i in (0, 1, 255, 511):
        compare(out, oracle_cart(oracle_mod, g, b, x, lam, i), i, "2000-bus")
    polar = gpu_eval(net, b, which=("gh",))
    assert_close(out["gh"][:, :g.m], polar["gh"], "cartesian vs polar g|h")
    np.testing.assert_allclose(out["gh"][:, g.m:], b.x[:, g.nb:2 * g.nb] ** 2, rtol=1e-14)
    net.close()


def test_cartesian_empty_batch(ex):
    import torch
    g = synth.grid_30bus()
    net = ex.Net(g)
    x = torch.zeros(0, g.n, dtype=torch.float64, device="cuda")
    ex.exago_eval_cart(net.h, ex.make_batch(x))
    assert ex.exago_eval_cart_workspace_size(net.h, 0) == 0
    net.close()


def test_cartesian_adjoints_match_oracle(ex, oracle_mod):
    """J u, J' v and (grad^2 L) u of the cartesian map against the oracle's J and H (sparse
    matrix-vector products), with outages, shunts, transformers and objective weights."""
    import scipy.sparse as sp
    import torch
    g = synth.make_grid(65, 300, 389, 77, transformer_frac=0.3, shunts=True)
    b = synth.random_batch(65, g, 4, masks=True, obj_weight=True, sigma=0.6)
    x, lam = to_cartesian(g, b, 65)
    mc = g.m + g.nb
    rng = np.random.default_rng(65)
    u = rng.normal(size=(b.B, g.n))
    v = rng.normal(size=(b.B, mc))
    net = ex.Net(g)
    d = to_device(b)
    X, LAM = torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")
    bt = ex.make_batch(X, LAM, d["mask"], None, d["obj_weight"], b.sigma)
    U, V = torch.as_tensor(u, device="cuda"), torch.as_tensor(v, device="cuda")
    jvp = torch.empty(b.B, mc, dtype=torch.float64, device="cuda")
    jtv = torch.empty(b.B, g.n, dtype=torch.float64, device="cuda")
    hvp = torch.empty(b.B, g.n, dtype=torch.float64, device="cuda")
    ex.exago_eval_cart_jvp(net.h, bt, U, jvp)
    ex.exago_eval_cart_jtv(net.h, bt, V, jtv)
    ex.exago_eval_cart_hvp(net.h, bt, U, hvp)
    torch.cuda.synchronize()
    jvp, jtv, hvp = jvp.cpu().numpy(), jtv.cpu().numpy(), hvp.cpu().numpy()
    for i in range(b.B):
        r = oracle_cart(oracle_mod, g, b, x, lam, i)
        J = sp.csr_matrix((r["J"][2], r["J"][1], r["J"][0]), shape=(mc, g.n))
        L = sp.csr_matrix((r["H"][2], r["H"][1], r["H"][0]), shape=(g.n, g.n))
        H = L + L.T - sp.diags(L.diagonal())
        assert_close(jvp[i], J @ u[i], f"cart J u [{i}]")
        assert_close(jtv[i], J.T @ v[i], f"cart J' v [{i}]")
        assert_close(hvp[i], H @ u[i], f"cart H u [{i}]")
    net.close()


def test_cartesian_autograd_double_backward(ex, oracle_mod):
    """torch.autograd over the cartesian map: grad of <v, c(x)> is J' v, and differentiating that
    again along w gives (sum_i v_i grad^2 c_i) w, both against the oracle."""
    import scipy.sparse as sp
    import torch
    from paper_2203_10587_gb300 import autograd
    g = synth.make_grid(66, 120, 160, 30, shunts=True)
    b = synth.random_batch(66, g, 3)
    x, _ = to_cartesian(g, b, 66)
    mc = g.m + g.nb
    rng = np.random.default_rng(66)
    v = rng.normal(size=(b.B, mc))
    w = rng.normal(size=(b.B, g.n))
    net = ex.Net(g)
    X = torch.as_tensor(x, device="cuda").requires_grad_(True)
    c = autograd.cons(X, net, cartesian=True)
    (gx,) = torch.autograd.grad(c, X, torch.as_tensor(v, device="cuda"), create_graph=True)
    (hw,) = torch.autograd.grad(gx, X, torch.as_tensor(w, device="cuda"))
    gx, hw = gx.detach().cpu().numpy(), hw.cpu().numpy()
    for i in range(b.B):
        r = oracle_mod.evaluate(oracle_mod.OracleNet(g), x[i], v[i], None, None, 1.0, 0.0,
                                cartesian=True)
        J = sp.csr_matrix((r["J"][2], r["J"][1], r["J"][0]), shape=(mc, g.n))
        L = sp.csr_matrix((r["H"][2], r["H"][1], r["H"][0]), shape=(g.n, g.n))
        H = L + L.T - sp.diags(L.diagonal())
        assert_close(c.detach().cpu().numpy()[i], r["gh"], f"cart c [{i}]")
        assert_close(gx[i], J.T @ v[i], f"autograd J' v [{i}]")
        assert_close(hw[i], H @ w[i], f"autograd H w [{i}]")
    net.close()


def test_cartesian_ring_and_caller_workspace(ex):
    """The chunked two-stream schedule over 5 chunks (ring slots reused) with a caller workspace
    of three chunks, and with one chunk's worth (a single ring slot: everything on the caller's
    stream), equals the internal workspace bit for bit."""
    import torch
    g = synth.grid_2000()
    b = synth.contingency_batch(7, g, 190)        # 41-state chunks: 5 chunks, ring of 3
    x, lam = to_cartesian(g, b, 7)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=3)
    ref = run_cart(ex, net, b, x, lam)
    one = 41 * 2 * g.nl * 14 * 8                  # one chunk of branch-end records
    full = 3 * one
    assert ex.exago_eval_cart_workspace_size(net.h, b.B) >= full
    for nbytes in (full, one):
        ws = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
        got = run_cart(ex, net, b, x, lam, workspace=ws)
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{k} ({nbytes} bytes)")
    net.close()


def test_cartesian_30bus_against_golden(ex):
    """The 30-bus cartesian snapshot written by the oracle-only golden script."""
    import json
    import os
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, os.path.join(here, "golden"))
    import make_golden
    g, b, x, lam = make_golden.cartesian_cases()
    stored = json.load(open(os.path.join(here, "golden", "c1_30bus_cartesian.json")))["instances"]
    net = ex.Net(g)
    out = run_cart(ex, net, b, x, lam)
    for i, s in enumerate(stored):
        ref = {"f": s["f"], "grad": np.array(s["grad"]), "gh": np.array(s["gh"]),
               "J": (None, None, np.array(s["J_val"])), "H": (None, None, np.array(s["H_val"]))}
        compare(out, ref, i, "cartesian golden")
    net.close()


def test_cartesian_adjoints_in_chunks(ex):
    """A caller workspace that holds the branch values of 41 states splits the adjoint products of
    190 states into 5 chunks; the results equal one chunk bit for bit."""
    import torch
    g = synth.grid_2000()
    b = synth.contingency_batch(9, g, 190)
    x, lam = to_cartesian(g, b, 9)
    mc = g.m + g.nb
    rng = np.random.default_rng(9)
    U = torch.as_tensor(rng.normal(size=(b.B, g.n)), device="cuda")
    V = torch.as_tensor(rng.normal(size=(b.B, mc)), device="cuda")
    X, LAM = torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")
    M = torch.as_tensor(b.mask, device="cuda")
    net = ex.Net(g)
    ws = torch.empty(41 * g.nl * 4, dtype=torch.float64, device="cuda")
    res = []
    for workspace in (None, ws):
        bt = ex.make_batch(X, LAM, M, obj_factor=0.7, workspace=workspace)
        o = [torch.empty(b.B, k, dtype=torch.float64, device="cuda") for k in (mc, g.n, g.n)]
        ex.exago_eval_cart_jvp(net.h, bt, U, o[0])
        ex.exago_eval_cart_jtv(net.h, bt, V, o[1])
        ex.exago_eval_cart_hvp(net.h, bt, U, o[2])
        torch.cuda.synchronize()
        res.append([t.cpu().numpy() for t in o])
    for a, c in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, c)
    net.close()
