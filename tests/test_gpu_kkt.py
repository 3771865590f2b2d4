"""GPU: the batched interior-point KKT step (exago_kkt_solve) against the oracle's sparse direct
solve of the same systems (oracle/kkt.py).

Inputs (every value from the oracle or the seeded generator, none from the CUDA path): J and the
Lagrangian Hessian W of each state from the model oracle, dx_i = 1 + sum_j |W_ij| (W + Dx
strictly diagonally dominant), dc ~ U(0.5, 2), rhs ~ N(0, 1).  Such a K is quasi-definite, so
L D L' without pivoting exists and has exactly m negative pivots.

Tolerance.  The device factors in another order than the oracle's library solve, so the two
agree to the systems' conditioning, not to the last bit.  Two bounds are checked per state:
  * forward: max |sol - ref| <= 1e-9 max |ref|;
  * backward (independent of the conditioning): max |K sol - rhs| <= 1e-13 (max|K| max|sol|
    + max|rhs|) * sqrt(n + m), K applied from its CSR parts.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2203_10587_gb300 import synth
from parity_util import oracle_eval

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-9
BWD_TOL = 1e-13


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def sym_csr(H, n):
    L = sp.csr_matrix((H[2], H[1], H[0]), shape=(n, n))
    return (L + L.T - sp.diags(L.diagonal())).tocsr()


def kkt_inputs(om, g, b, seed):
    """Per-state oracle J, H values and the recipe's dx, dc, rhs."""
    rng = np.random.default_rng(seed)
    B, n, m = b.B, g.n, g.m
    refs = [oracle_eval(om, g, b, i) for i in range(B)]
    jval = np.stack([r["J"][2] for r in refs])
    hval = np.stack([r["H"][2] for r in refs])
    dx = np.stack([1.0 + np.abs(sym_csr(r["H"], n)).sum(axis=1).A1 for r in refs])
    dc = rng.uniform(0.5, 2.0, (B, m))
    rhs = rng.normal(size=(B, n + m))
    return refs, jval, hval, dx, dc, rhs


def run_kkt(ex, net, jval, hval, dx, dc, rhs, workspace=None):
    import torch
    k = ex.exago_kkt_create(net.h)
    try:
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        B = jval.shape[0]
        sol = torch.full((B, rhs.shape[1]), np.nan, dtype=torch.float64, device="cuda")
        inertia = torch.full((B, 2), -1, dtype=torch.int32, device="cuda")
        ex.exago_kkt_solve(k, t(jval), t(hval), t(dx), t(dc), t(rhs), sol, inertia, workspace)
        torch.cuda.synchronize()
        return sol.cpu().numpy(), inertia.cpu().numpy()
    finally:
        ex.exago_kkt_destroy(k)


def check_state(g, ref_eval, dx, dc, rhs, sol, ref=None, what=""):
    from oracle import kkt
    n, m = g.n, g.m
    J = sp.csr_matrix((ref_eval["J"][2], ref_eval["J"][1], ref_eval["J"][0]), shape=(m, n))
    W = sym_csr(ref_eval["H"], n)
    x, y = sol[:n], sol[n:]
    res = np.concatenate([W @ x + dx * x + J.T @ y, J @ x - dc * y]) - rhs
    kmax = max(np.abs(W.data).max() + dx.max(), np.abs(J.data).max() if J.nnz else 0.0, dc.max())
    bound = BWD_TOL * (kmax * np.abs(sol).max() + np.abs(rhs).max()) * np.sqrt(n + m)
    assert np.abs(res).max() <= bound, f"{what}: residual {np.abs(res).max():.3e} > {bound:.3e}"
    if ref is None:
        ref = kkt.kkt_solve(n, m, ref_eval["J"], ref_eval["H"], dx, dc, rhs)
    err = np.abs(sol - ref).max() / np.abs(ref).max()
    assert err <= FWD_TOL, f"{what}: forward error {err:.3e}"


@pytest.mark.parametrize("case", ["30bus", "300bus_outages", "parallel"])
def test_kkt_against_oracle(ex, oracle_mod, case):
    from test_capi_host import parallel_grid
    if case == "30bus":
        g, b = synth.grid_30bus(), None
        b = synth.random_batch(1, g, 3, masks=True, sigma=0.8)
    elif case == "300bus_outages":
        g = synth.make_grid(13, 300, 389, 77, transformer_frac=0.3, shunts=True)
        b = synth.random_batch(13, g, 9, masks=True, sigma=0.7, gen_masks=True)
    else:
        g = parallel_grid()
        b = synth.random_batch(5, g, 4, masks=True, sigma=1.0)
    refs, jval, hval, dx, dc, rhs = kkt_inputs(oracle_mod, g, b, 7)
    net = ex.Net(g)
    sol, inertia = run_kkt(ex, net, jval, hval, dx, dc, rhs)
    for i in range(b.B):
        check_state(g, refs[i], dx[i], dc[i], rhs[i], sol[i], what=f"{case}[{i}]")
        assert tuple(inertia[i]) == (g.m, 0), inertia[i]


def test_kkt_state_alone_equals_in_batch_and_caller_workspace(ex, oracle_mod):
    import torch
    g = synth.make_grid(19, 200, 260, 50, shunts=True)
    b = synth.random_batch(19, g, 37, masks=True, sigma=0.9)
    refs, jval, hval, dx, dc, rhs = kkt_inputs(oracle_mod, g, b, 19)
    net = ex.Net(g)
    full, _ = run_kkt(ex, net, jval, hval, dx, dc, rhs)
    one, _ = run_kkt(ex, net, jval[5:6], hval[5:6], dx[5:6], dc[5:6], rhs[5:6])
    np.testing.assert_array_equal(one[0], full[5])
    k = ex.exago_kkt_create(net.h)
    nbytes = ex.exago_kkt_workspace_size(k, b.B)
    ex.exago_kkt_destroy(k)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    again, _ = run_kkt(ex, net, jval, hval, dx, dc, rhs, workspace=ws)
    np.testing.assert_array_equal(again, full)


def test_kkt_2000_bus_512_states(ex, oracle_mod):
    """The bench's batch: 2,000-bus grid, 512 N-1 states.  Every state is checked against the
    backward bound and its inertia; sampled states against the oracle's solve."""
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 512)
    refs, jval, hval, dx, dc, rhs = kkt_inputs(oracle_mod, g, b, 3)
    net = ex.Net(g)
    sol, inertia = run_kkt(ex, net, jval, hval, dx, dc, rhs)
    assert np.all(inertia[:, 0] == g.m) and np.all(inertia[:, 1] == 0)
    from oracle import kkt
    for i in range(b.B):
        ref = kkt.kkt_solve(g.n, g.m, refs[i]["J"], refs[i]["H"], dx[i], dc[i], rhs[i]) \
            if i in (0, 255, 511) else None
        if ref is not None:
            check_state(g, refs[i], dx[i], dc[i], rhs[i], sol[i], ref=ref, what=f"2000-bus[{i}]")
        else:
            # backward bound only (the forward comparison needs the oracle's solve)
            n, m = g.n, g.m
            J = sp.csr_matrix((jval[i], refs[i]["J"][1], refs[i]["J"][0]), shape=(m, n))
            W = sym_csr((refs[i]["H"][0], refs[i]["H"][1], hval[i]), n)
            x, y = sol[i, :n], sol[i, n:]
            res = np.concatenate([W @ x + dx[i] * x + J.T @ y, J @ x - dc[i] * y]) - rhs[i]
            kmax = max(np.abs(W.data).max() + dx[i].max(), np.abs(J.data).max(), dc[i].max())
            bound = BWD_TOL * (kmax * np.abs(sol[i]).max() + np.abs(rhs[i]).max()) * np.sqrt(n + m)
            assert np.abs(res).max() <= bound, (i, np.abs(res).max(), bound)
