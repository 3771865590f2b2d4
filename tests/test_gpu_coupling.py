"""GPU: coupling (ramp) rows between the states of a batch and their transpose product, through
the C ABI, against the oracle (oracle_coupling, oracle_coupling_jtv) on the same seeded inputs.

The rows (one subtraction each) must match bit for bit.  The transpose product sums a state's
children in another order than the oracle's row-by-row scatter, so it is compared within the
evaluator's tolerance, |gpu - oracle| <= 1e-11 max(1, |oracle|).  Structures: chains of periods,
stars of contingencies around a base case (one state with hundreds or thousands of children,
reduced by the block kernel in one or several shared-memory passes), random forests, states with exactly 8 and 9 children (the two sides of the
light/heavy split) and batches of roots only.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def split_parents():
    """State 0 has 8 children, state 9 has 9, the rest are leaves or roots."""
    p = np.full(24, -1, np.int32)
    p[1:9] = 0
    p[10:19] = 9
    p[20] = 19
    return p


CASES = {
    "chain_30bus_x7": (lambda: synth.grid_30bus(), lambda: synth.coupling_parents("chain", 7)),
    "star_30bus_x300": (lambda: synth.grid_30bus(), lambda: synth.coupling_parents("star", 300)),
    # more children than one shared-memory pass of the heavy kernel holds (2,048)
    "star_30bus_x5000": (lambda: synth.grid_30bus(), lambda: synth.coupling_parents("star", 5000)),
    "forest_300bus_x97": (lambda: synth.make_grid(41, 300, 390, 77),
                          lambda: synth.coupling_parents("forest", 97, seed=4, roots=3)),
    "split_8_9": (lambda: synth.make_grid(42, 120, 150, 33), split_parents),
    "roots_only": (lambda: synth.grid_30bus(), lambda: np.full(5, -1, np.int32)),
    "single": (lambda: synth.grid_30bus(), lambda: np.array([-1], np.int32)),
}


def run_case(ex, oracle_mod, g, parent, seed):
    import torch
    B = parent.shape[0]
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, g.n))
    nu = rng.normal(size=(B, g.ng))
    net = ex.Net(g)
    h = ex.exago_coupling_create(net.h, parent)
    try:
        X = torch.as_tensor(x, device="cuda")
        NU = torch.as_tensor(nu, device="cuda")
        r = torch.full((B, g.ng), np.nan, dtype=torch.float64, device="cuda")
        ex.exago_eval_coupling(h, X, r)
        # transpose product stored into a [B][ng] buffer ...
        out = torch.full((B, g.ng), np.nan, dtype=torch.float64, device="cuda")
        ex.exago_eval_coupling_jtv(h, NU, out, ldo=g.ng)
        # ... and added into the Pg block of a [B][n] gradient
        base = rng.normal(size=(B, g.n))
        grad = torch.as_tensor(base.copy(), device="cuda")
        ex.exago_eval_coupling_jtv(h, NU, grad.data_ptr() + 8 * 2 * g.nb, ldo=g.n, accumulate=True)
        torch.cuda.synchronize()
        r, out, grad = r.cpu().numpy(), out.cpu().numpy(), grad.cpu().numpy()
    finally:
        ex.exago_coupling_destroy(h)
        net.close()
    r_ref = oracle_mod.coupling(parent, x, g.nb, g.ng)
    jt_ref = oracle_mod.coupling_jtv(parent, nu, g.n, g.nb)
    pg = slice(2 * g.nb, 2 * g.nb + g.ng)
    np.testing.assert_array_equal(r, r_ref)
    assert_close(out, jt_ref[:, pg], "C^T nu")
    assert_close(grad[:, pg], base[:, pg] + jt_ref[:, pg], "g + C^T nu (Pg block)")
    other = np.ones(g.n, bool)
    other[pg] = False
    np.testing.assert_array_equal(grad[:, other], base[:, other])


@pytest.mark.parametrize("name", sorted(CASES))
def test_coupling_matches_oracle(ex, oracle_mod, name):
    mk_grid, mk_parent = CASES[name]
    run_case(ex, oracle_mod, mk_grid(), mk_parent(), seed=len(name))


def test_coupling_full_size_contingencies(ex, oracle_mod):
    """2,000-bus grid x 512 states: 511 contingencies tied to the base case (eq. (20)), the batch
    of the bench's N-1 workload; every element against the oracle."""
    run_case(ex, oracle_mod, synth.grid_2000(), synth.coupling_parents("star", 512), seed=20)


def test_coupling_full_size_periods(ex, oracle_mod):
    """10,000-bus grid x 64 consecutive periods (eq. (15)); every element against the oracle."""
    run_case(ex, oracle_mod, synth.grid_10k(), synth.coupling_parents("chain", 64), seed=15)


def test_coupling_empty_batch_and_device_check(ex):
    import torch
    g = synth.grid_30bus()
    net = ex.Net(g)
    h = ex.exago_coupling_create(net.h, np.zeros(0, np.int32))
    try:
        z = torch.zeros(0, g.n, dtype=torch.float64, device="cuda")
        assert ex.lib().exago_eval_coupling(h, None, None, None) == 0   # B = 0: nothing to do
        ex.exago_eval_coupling_jtv(h, torch.zeros(0, g.ng, dtype=torch.float64, device="cuda"),
                                   z, ldo=g.ng)
    finally:
        ex.exago_coupling_destroy(h)
    h = ex.exago_coupling_create(net.h, np.array([-1, 0], np.int32))
    try:
        rc = ex.lib().exago_eval_coupling(h, None, None, None)
        assert ex.STATUS[rc] == "EXAGO_EINVAL"
        nu = torch.zeros(2, g.ng, dtype=torch.float64, device="cuda")
        with pytest.raises(ex.ExagoError):
            ex.exago_eval_coupling_jtv(h, nu, torch.zeros(2, g.ng, dtype=torch.float64,
                                                          device="cuda"), ldo=g.ng - 1)
    finally:
        ex.exago_coupling_destroy(h)
        net.close()


def test_coupling_full_size_70k_periods(ex, oracle_mod):
    """70,000-bus grid (17,500 generators) x 512 consecutive periods: 72 MB of rows, larger than
    L2; every element against the oracle."""
    run_case(ex, oracle_mod, synth.grid_sized(9, 70_000), synth.coupling_parents("chain", 512),
             seed=70)


def test_multi_period_stacked_quantities(ex, oracle_mod):
    """The multi-period problem (Sec. IV, eqs. (11)-(15)) over 6 periods of a 300-bus grid with
    per-period load scales: stacked constraints [g | h of every period ; ramp rows] and the
    stacked transpose product J' [lambda ; nu] = per-period exago_eval_jtv plus the coupling
    transpose added into the Pg block, against the oracle's per-period Jacobians (CSR) and its
    coupling rows."""
    import scipy.sparse as sp
    import torch
    from parity_util import to_device
    g = synth.make_grid(71, 300, 389, 77, transformer_frac=0.2, shunts=True)
    T = 6
    b = synth.random_batch(71, g, T, pd_scale=True, sigma=0.5)
    parent = synth.coupling_parents("chain", T)
    nu = np.random.default_rng(72).normal(size=(T, g.ng))
    net = ex.Net(g)
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], None, d["pd_scale"], None, b.sigma)
    gh = torch.empty(T, g.m, dtype=torch.float64, device="cuda")
    ex.exago_eval_cons(net.h, bt, gh)
    r = torch.empty(T, g.ng, dtype=torch.float64, device="cuda")
    cpl = ex.exago_coupling_create(net.h, parent)
    try:
        ex.exago_eval_coupling(cpl, d["x"], r)
        jt = torch.empty(T, g.n, dtype=torch.float64, device="cuda")
        ex.exago_eval_jtv(net.h, bt, d["lam"], jt)
        ex.exago_eval_coupling_jtv(cpl, torch.as_tensor(nu, device="cuda"),
                                   jt.data_ptr() + 8 * 2 * g.nb, ldo=g.n, accumulate=True)
        torch.cuda.synchronize()
    finally:
        ex.exago_coupling_destroy(cpl)
    c_gpu = np.concatenate([gh.cpu().numpy().reshape(-1), r.cpu().numpy().reshape(-1)])
    jt_gpu = jt.cpu().numpy()
    onet = oracle_mod.OracleNet(g)
    c_ref, jt_ref = [], np.zeros((T, g.n))
    for t in range(T):
        o = oracle_mod.evaluate(onet, b.x[t], b.lam[t], None, b.pd_scale[t], 1.0, b.sigma)
        c_ref.append(o["gh"])
        J = sp.csr_matrix((o["J"][2], o["J"][1], o["J"][0]), shape=(g.m, g.n))
        jt_ref[t] = J.T @ b.lam[t]
    c_ref = np.concatenate(c_ref + [oracle_mod.coupling(parent, b.x, g.nb, g.ng).reshape(-1)])
    jt_ref += oracle_mod.coupling_jtv(parent, nu, g.n, g.nb)
    assert_close(c_gpu, c_ref, "stacked constraints")
    assert_close(jt_gpu, jt_ref, "stacked J' [lambda; nu]")
    net.close()


def test_coupling_autograd(ex, oracle_mod):
    """torch.autograd over the coupling rows: backward is C^T (oracle), and differentiating the
    backward again gives C w (the rows are linear)."""
    import torch
    from paper_2203_10587_gb300 import autograd
    g = synth.make_grid(73, 120, 160, 30)
    parent = synth.coupling_parents("forest", 40, seed=6, roots=4)
    rng = np.random.default_rng(73)
    x = torch.as_tensor(rng.normal(size=(40, g.n)), device="cuda").requires_grad_(True)
    v = torch.as_tensor(rng.normal(size=(40, g.ng)), device="cuda")
    net = ex.Net(g)
    cpl = ex.Coupling(net, parent)
    r = autograd.coupling(x, cpl)
    (gx,) = torch.autograd.grad(r, x, v, create_graph=True)
    np.testing.assert_array_equal(r.detach().cpu().numpy(),
                                  oracle_mod.coupling(parent, x.detach().cpu().numpy(), g.nb, g.ng))
    assert_close(gx.detach().cpu().numpy(), oracle_mod.coupling_jtv(parent, v.cpu().numpy(), g.n, g.nb),
                 "autograd C^T v")
    w = torch.as_tensor(rng.normal(size=(40, g.n)), device="cuda")
    vv = v.clone().requires_grad_(True)
    (gx2,) = torch.autograd.grad(autograd.coupling(x, cpl), x, vv, create_graph=True)
    (gv,) = torch.autograd.grad(gx2, vv, w)
    np.testing.assert_array_equal(gv.cpu().numpy(), oracle_mod.coupling(parent, w.cpu().numpy(), g.nb, g.ng))
    cpl.close()
    net.close()


def test_coupling_more_states_than_one_grid_row(ex, oracle_mod):
    """70,000 states (more than one launch's 65,535 grid rows): a chain of 40,000 periods and a
    star of 30,000 contingencies around state 40,000, on the 30-bus grid."""
    parent = np.concatenate([synth.coupling_parents("chain", 40_000),
                             np.full(30_000, 40_000, np.int32)])
    parent[40_000] = -1
    run_case(ex, oracle_mod, synth.grid_30bus(), parent, seed=71)
