"""GPU: the batched power-flow Newton step (exago_pf_step) against the oracle's step
(oracle/kkt.py, pf_newton_step) from the same points.

Each GPU step is compared with the oracle's step from the same x:
  * the fixed quantities (Va and Vm of the slack bus, Vm of PV buses, Pg, Qg) are copied bit for
    bit;
  * the step d = x_new - x: max |d_gpu - d_ref| <= 1e-9 max |d_ref| + 1e-13 (the two solve
    J_pf d = -g_pf in different orders, so they agree to its conditioning; the floor covers
    steps near convergence);
  * the mismatch max |g_pf(x)| within 1e-11 max(1, |ref|) (the evaluation's tolerance).
The GPU and the oracle also iterate independently from the same start; both converge
quadratically and agree after every step within the same bound.
Inputs: seeded grids with light load (Pd scaled by 0.3), a balanced dispatch, PV set points and a
flat start (the recipe of the oracle's power-flow pins); the 2,000-bus case has no shunts and flat
set points (it then converges from a flat start).
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def case(seed, nb, nl, ng, shunts=True, vspread=0.03):
    g = synth.make_grid(seed, nb, nl, ng, transformer_frac=0.2, shunts=shunts)
    g.Pd *= 0.3
    g.Qd *= 0.3
    rng = np.random.default_rng(seed)
    bt = np.ones(g.nb, np.int32)
    bt[g.gbus] = 2
    bt[g.gbus[0]] = 3
    Pg = np.full(g.ng, g.Pd.sum() / g.ng)
    Vm = np.ones(g.nb)
    if vspread:
        Vm[g.gbus] = rng.uniform(1.0 - vspread / 3, 1.0 + vspread, g.ng)
    x = np.concatenate([np.zeros(g.nb), Vm, Pg, np.zeros(g.ng)])
    return g, bt, x


def gpu_steps(ex, net, pf, X, mask=None, gen_mask=None, pd_scale=None):
    import torch
    t = lambda a, dt=torch.float64: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    x = t(X)
    bt = ex.make_batch(x, None, t(mask, torch.uint8), t(pd_scale), None, 1.0,
                       gen_mask=t(gen_mask, torch.uint8))
    xn = torch.empty_like(x)
    mis = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
    ex.exago_pf_step(pf, bt, xn, mis)
    torch.cuda.synchronize()
    return xn.cpu().numpy(), mis.cpu().numpy()


def compare_step(g, bt, x, x_gpu, x_ref, mis_gpu, mis_ref, what):
    nb = g.nb
    fixed = np.concatenate([np.flatnonzero(bt == 3), nb + np.flatnonzero(bt != 1),
                            np.arange(2 * nb, g.n)])
    np.testing.assert_array_equal(x_gpu[fixed], x[fixed], err_msg=what)
    d_gpu, d_ref = x_gpu - x, x_ref - x
    err = np.abs(d_gpu - d_ref).max()
    assert err <= 1e-9 * np.abs(d_ref).max() + 1e-13, f"{what}: step error {err:.3e}"
    assert abs(mis_gpu - mis_ref) <= 1e-11 * max(1.0, mis_ref), (what, mis_gpu, mis_ref)


@pytest.mark.parametrize("name", ["30bus", "300bus"])
def test_pf_step_against_oracle(ex, oracle_mod, name):
    from oracle import kkt
    g, bt, x0 = case(31, 30, 41, 6) if name == "30bus" else case(32, 300, 389, 60)
    rng = np.random.default_rng(5)
    B = 5
    X = np.repeat(x0[None, :], B, axis=0)
    ns, pq = np.flatnonzero(bt != 3), np.flatnonzero(bt == 1)
    X[1:, ns] += rng.normal(0.0, 0.05, (B - 1, ns.size))
    X[1:, g.nb + pq] += rng.normal(0.0, 0.01, (B - 1, pq.size))
    mask = np.ones((B, g.nl), np.uint8)
    nonbridge = np.flatnonzero(~synth.bridges(g.nb, g.f, g.t))
    mask[3, nonbridge[len(nonbridge) // 2]] = 0      # a branch outage that islands no bus
    gm = np.ones((B, g.ng), np.uint8)
    gm[4, -1] = 0                                    # a generator outage
    ps = np.exp(0.1 * rng.normal(size=(B, g.nb)))
    net = ex.Net(g)
    pf = ex.exago_pf_create(net.h, bt)
    try:
        xg, mg = gpu_steps(ex, net, pf, X, mask, gm, ps)
    finally:
        ex.exago_pf_destroy(pf)
    onet = oracle_mod.OracleNet(g)
    for i in range(B):
        xr, mr = kkt.pf_newton_step(oracle_mod, onet, X[i], bt, gen_mask=gm[i], mask=mask[i],
                                    pd_scale=ps[i])
        compare_step(g, bt, X[i], xg[i], xr, mg[i], mr, f"{name}[{i}]")


@pytest.mark.parametrize("name", ["30bus", "2000bus"])
def test_pf_iterations_converge_with_the_oracle(ex, oracle_mod, name):
    from oracle import kkt
    if name == "30bus":
        g, bt, x0 = case(31, 30, 41, 6)
        B = 2
    else:
        g, bt, x0 = case(33, 2000, 2700, 500, shunts=False, vspread=0.0)
        B = 64
    X = np.repeat(x0[None, :], B, axis=0)
    net = ex.Net(g)
    pf = ex.exago_pf_create(net.h, bt)
    onet = oracle_mod.OracleNet(g)
    xo = x0.copy()
    mis = []
    try:
        for it in range(8):
            Xn, m = gpu_steps(ex, net, pf, X)
            xo_n, mo = kkt.pf_newton_step(oracle_mod, onet, xo, bt)
            compare_step(g, bt, X[0], Xn[0], X[0] + (xo_n - xo), m[0], mo, f"{name} step {it}")
            # every state of the batch is the same start: bitwise the same iterate
            assert np.all(Xn == Xn[0][None, :])
            X, xo = Xn, xo_n
            mis.append(m[0])
            if m[0] < 1e-12:
                break
    finally:
        ex.exago_pf_destroy(pf)
    assert mis[-1] < 1e-10, mis
