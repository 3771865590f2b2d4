"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and the oracle on
the same seeded inputs and compare element by element.

Tolerance: |gpu - oracle| <= 1e-11 * max(1, |oracle|) on every output.  The oracle rounds every
operation separately (-ffp-contract=off) and calls libm sin/cos; the kernels use FMA and CUDA's
sincos and regroup sums, which moves results by a few ulps of the largest term (terms reach about
1e4 in the Hessian, so about 1e-12 absolute).
"""
import numpy as np

TOL = 1e-11


def assert_close(gpu, ref, what="", tol=TOL):
    gpu = np.asarray(gpu, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    assert gpu.shape == ref.shape, (what, gpu.shape, ref.shape)
    if gpu.size == 0:
        return
    err = np.abs(gpu - ref) / np.maximum(1.0, np.abs(ref))
    k = int(np.argmax(err))
    assert err[k] <= tol, f"{what}: max scaled error {err[k]:.3e} at {k} (gpu {gpu[k]!r}, oracle {ref[k]!r})"


def to_device(batch, device="cuda"):
    import torch
    t = lambda a, dt: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
    return dict(x=t(batch.x, torch.float64), lam=t(batch.lam, torch.float64),
                mask=t(batch.mask, torch.uint8), pd_scale=t(batch.pd_scale, torch.float64),
                obj_weight=t(batch.obj_weight, torch.float64),
                gen_mask=t(batch.gen_mask, torch.uint8))


def gpu_eval(net, batch, device="cuda", workspace=None, which=("f", "grad", "gh", "jval", "hval")):
    """All requested outputs of exago_eval_all as host numpy arrays."""
    import torch
    from paper_2203_10587_gb300 import exago
    d = to_device(batch, device)
    bt = exago.make_batch(d["x"], d["lam"], d["mask"], d["pd_scale"], d["obj_weight"],
                          batch.sigma, workspace=workspace, gen_mask=d["gen_mask"])
    out = net.outputs(batch.B, device, f="f" in which, grad="grad" in which, gh="gh" in which,
                      jac="jval" in which, hess="hval" in which)
    net.eval_all(bt, out)
    torch.cuda.synchronize()
    exago.exago_net_check(net.h)
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


def oracle_eval(om, grid, batch, idx):
    onet = om.OracleNet(grid)
    return om.evaluate(onet, batch.x[idx], batch.lam[idx],
                       None if batch.mask is None else batch.mask[idx],
                       None if batch.pd_scale is None else batch.pd_scale[idx],
                       1.0 if batch.obj_weight is None else float(batch.obj_weight[idx]),
                       batch.sigma,
                       gen_mask=None if batch.gen_mask is None else batch.gen_mask[idx])


def compare_instance(out, b, ref, what=""):
    assert_close(out["f"][b], ref["f"], f"{what} f[{b}]")
    assert_close(out["grad"][b], ref["grad"], f"{what} grad[{b}]")
    assert_close(out["gh"][b], ref["gh"], f"{what} gh[{b}]")
    assert_close(out["jval"][b], ref["J"][2], f"{what} J[{b}]")
    assert_close(out["hval"][b], ref["H"][2], f"{what} H[{b}]")
