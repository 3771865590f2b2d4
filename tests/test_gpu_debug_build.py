"""GPU: the EXAGO_DEBUG build of the library (device-side index checks that set the status word
instead of trapping; the substitute for compute-sanitizer, which is closed on this machine).

A child process loads the debug build (EXAGO_LIBRARY) and evaluates the same inputs as this
process does with the release build: every schedule (both tilings of the persistent one), an
adjoint product and a KKT step.  The checks are pure comparisons, so the results must be bitwise
the release build's, and the status word must stay clear.  Then the child lowers the bound the checks compare slot indices against
(exago_test_debug_bounds): the checks must fire -- exago_net_check reports EXAGO_EDEVICE -- while
every access the kernels still make stays in bounds (the bound only shrinks, the tables are
untouched); with the bound restored the next evaluation is clean again.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2203_10587_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCHEDULES = (dict(schedule=1, use_graph=2), dict(schedule=2, use_graph=2),
             dict(schedule=3, chunk=2, use_graph=2), dict(schedule=2, tiling=2, use_graph=2))

WORK = r'''
import numpy as np, torch
from paper_2203_10587_gb300 import exago, synth
from parity_util import gpu_eval, to_device

def work(out_path, negative):
    g = synth.make_grid(61, 300, 389, 77, transformer_frac=0.3, shunts=True)
    b = synth.random_batch(61, g, 5, masks=True, pd_scale=True, sigma=0.8)
    net = exago.Net(g)
    res = {}
    for k, cfg in enumerate(SCHEDULES):
        exago.exago_net_set_config(net.h, **cfg)
        for name, v in gpu_eval(net, b).items():
            res[f"s{k}_{name}"] = v
    exago.exago_net_check(net.h)
    d = to_device(b)
    bt = exago.make_batch(d["x"], d["lam"], d["mask"], d["pd_scale"], None, b.sigma)
    v = torch.as_tensor(np.random.default_rng(61).normal(size=(b.B, net.m)), device="cuda")
    o = torch.empty(b.B, net.n, dtype=torch.float64, device="cuda")
    exago.exago_eval_jtv(net.h, bt, v, o)
    torch.cuda.synchronize()
    res["jtv"] = o.cpu().numpy()
    # KKT step on the evaluation's own values
    out = net.outputs(b.B, f=False, grad=False, gh=False)
    net.eval_all(bt, out)
    # dx = 1 + absolute row sums of W, summed on the host in a fixed order
    hp, hc = exago.exago_net_hess_pattern(net.h)
    rows = np.repeat(np.arange(net.n), np.diff(hp))
    a = np.abs(out["hval"].cpu().numpy())
    dxh = np.ones((b.B, net.n))
    for i in range(b.B):
        np.add.at(dxh[i], rows, a[i])
        np.add.at(dxh[i], hc, np.where(rows != hc, a[i], 0.0))
    dx = torch.as_tensor(dxh, device="cuda")
    rng = np.random.default_rng(62)
    dc = torch.as_tensor(rng.uniform(0.5, 2.0, (b.B, net.m)), device="cuda")
    rhs = torch.as_tensor(rng.normal(size=(b.B, net.n + net.m)), device="cuda")
    sol = torch.empty_like(rhs)
    kk = exago.exago_kkt_create(net.h)
    exago.exago_kkt_solve(kk, out["jval"], out["hval"], dx, dc, rhs, sol)
    torch.cuda.synchronize()
    exago.exago_kkt_destroy(kk)
    exago.exago_net_check(net.h)
    res["kkt"] = sol.cpu().numpy()
    if negative:
        exago.exago_net_set_config(net.h, schedule=1, use_graph=2)
        exago.exago_test_debug_bounds(net.h, 2 * g.nl - 7)
        o2 = net.outputs(b.B)
        net.eval_all(bt, o2)
        try:
            exago.exago_net_check(net.h)
            res["fired"] = np.array([0])
        except exago.ExagoError as e:
            res["fired"] = np.array([1 if e.name == "EXAGO_EDEVICE" else 2])
        exago.exago_test_debug_bounds(net.h, -1)
        again = gpu_eval(net, b)
        exago.exago_net_check(net.h)
        res["again_hval"] = again["hval"]
    np.savez(out_path, **res)
'''


def child_script(out_path):
    return (f"import os, sys\nsys.path.insert(0, {ROOT!r})\nsys.path.insert(0, {os.path.join(ROOT, 'tests')!r})\n"
            f"SCHEDULES = {SCHEDULES!r}\n" + WORK + f"\nwork({out_path!r}, True)\n")


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def test_debug_build_equals_release_and_reports_failed_checks(ex, tmp_path):
    from paper_2203_10587_gb300 import build
    lib = build.build(debug=True)
    # the release results, in this process
    ns = {}
    exec(f"SCHEDULES = {SCHEDULES!r}\n" + WORK, ns)
    rel_path = str(tmp_path / "release.npz")
    ns["work"](rel_path, False)
    dbg_path = str(tmp_path / "debug.npz")
    env = dict(os.environ, EXAGO_LIBRARY=lib)
    p = subprocess.run([sys.executable, "-c", child_script(dbg_path)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    rel, dbg = np.load(rel_path), np.load(dbg_path)
    for k in rel.files:
        np.testing.assert_array_equal(dbg[k], rel[k], err_msg=k)
    assert int(dbg["fired"][0]) == 1, "the lowered bound did not raise EXAGO_EDEVICE"
    np.testing.assert_array_equal(dbg["again_hval"], rel["s0_hval"])
