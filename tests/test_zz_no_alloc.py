"""exago_eval_all_static: the evaluation for callers that may not allocate device memory.

Some callers cannot call cudaMalloc once they run -- a solver whose device memory belongs to a
pooling allocator, or a serving loop that reserves everything at start-up.  exago_eval_all_static
keeps its scratch in a static device array inside the library instead.  This test calls it through
the C ABI twice in a row, on different states, and checks each result against exago_eval_all on
the same inputs, within the parity tolerance.  It also checks that a batch too large for the array
is refused.  The file sorts last, so a run that stops at the first failure has run every other
test before it.
"""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import TOL, assert_close, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


OUTS = ("f", "grad", "gh", "jval", "hval")


def _run(ex, net, b, static, which=OUTS):
    import torch
    d = to_device(b)
    bt = ex.make_batch(d["x"], d["lam"], d["mask"], d["pd_scale"], d["obj_weight"], b.sigma,
                       gen_mask=d["gen_mask"])
    out = net.outputs(b.B, f="f" in which, grad="grad" in which, gh="gh" in which,
                      jac="jval" in which, hess="hval" in which)
    fn = ex.exago_eval_all_static if static else ex.exago_eval_all
    fn(net.h, bt, out["f"], out["grad"], out["gh"], out["jval"], out["hval"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


@pytest.mark.parametrize("which", ["300bus", "parallel"])
def test_static_scratch_matches_eval_all_twice(ex, which):
    if which == "300bus":
        g = synth.make_grid(37, 300, 389, 77, transformer_frac=0.3, shunts=True)
    else:
        from test_capi_host import parallel_grid
        g = parallel_grid()
    net = ex.Net(g)
    for call, seed in enumerate((41, 42)):      # two calls in a row, different states
        b = synth.random_batch(seed, g, 6, masks=True, pd_scale=True, obj_weight=True,
                               sigma=0.6 + 0.2 * call)
        want = _run(ex, net, b, static=False)
        got = _run(ex, net, b, static=True)
        for k in want:
            assert_close(got[k], want[k], f"call {call} {k}", TOL)


@pytest.mark.parametrize("which", [("gh", "jval"), ("f", "gh"), ("hval",), ("grad", "jval", "hval")])
def test_static_scratch_generator_outages_and_output_subsets(ex, which):
    """Per-state generator outages (Sec. V-A) and partial output sets go through the same
    static scratch and give exago_eval_all's results."""
    g = synth.make_grid(43, 300, 389, 77, transformer_frac=0.3, shunts=True)
    net = ex.Net(g)
    for call, seed in enumerate((44, 45)):
        b = synth.random_batch(seed, g, 5, masks=True, pd_scale=True, obj_weight=True,
                               sigma=0.9, gen_masks=True)
        want = _run(ex, net, b, static=False, which=which)
        got = _run(ex, net, b, static=True, which=which)
        assert set(got) == set(which)
        for k in want:
            assert_close(got[k], want[k], f"call {call} {k}", TOL)


def test_static_scratch_rejects_oversized_batch(ex):
    """The largest batch that fits the 16 MiB array runs; one state more is refused."""
    import torch
    g = synth.grid_2000()
    net = ex.Net(g)
    limit = 16 << 20
    per_state = 10 * 2 * g.nl * 8          # 10-double records, one per branch end
    B_ok = limit // per_state
    for B in (B_ok, B_ok + 1):
        x = torch.zeros(B, net.n, dtype=torch.float64, device="cuda")
        x[:, g.nb:2 * g.nb] = 1.0
        gh = torch.zeros(B, net.m, dtype=torch.float64, device="cuda")
        bt = ex.make_batch(x, None, None)
        if B == B_ok:
            ex.exago_eval_all_static(net.h, bt, gh=gh)
            torch.cuda.synchronize()
        else:
            with pytest.raises(ex.ExagoError) as ei:
                ex.exago_eval_all_static(net.h, bt, gh=gh)
            assert ei.value.name == "EXAGO_EINVAL" and "static scratch" in str(ei.value)
