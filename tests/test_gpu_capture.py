"""GPU: the library's evaluation calls captured into a caller's CUDA graph (torch.cuda.graph) and
replayed with new inputs written into the captured buffers.  Each replay must equal, bit for bit,
a direct call on the same inputs: the polar model on the persistent, pipelined (two streams,
forked and joined by events inside the capture) and multi-kernel schedules, and the cartesian
model's persistent and two-stream chunked schedules.  A call outside the capture comes first, so that the workspace and
the launch-configuration caches exist before capture (nothing may allocate while capturing).
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


def capture_and_replay(ex, call, inputs, new_inputs, outputs):
    """Warm up `call` on a side stream, capture it, copy new_inputs into inputs, replay; returns
    the replayed outputs (host)."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        call(torch.cuda.current_stream())
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call(torch.cuda.current_stream())
    for dst, src in zip(inputs, new_inputs):
        dst.copy_(src)
    g.replay()
    torch.cuda.synchronize()
    return [o.cpu().numpy().copy() for o in outputs]


@pytest.mark.parametrize("schedule", [2, 3, 1])
def test_polar_call_captured_in_a_graph(ex, schedule):
    import torch
    g = synth.make_grid(121, 300, 389, 77, shunts=True)
    b1 = synth.random_batch(121, g, 24, masks=True, sigma=0.8)
    b2 = synth.random_batch(122, g, 24, masks=True, sigma=0.8)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=schedule, chunk=7 if schedule == 3 else 0)
    ex.exago_net_reserve(net.h, b1.B)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    x, lam, mask = t(b1.x, torch.float64), t(b1.lam, torch.float64), t(b1.mask, torch.uint8)
    out = net.outputs(b1.B)
    outs = [out[k] for k in ("f", "grad", "gh", "jval", "hval")]

    def call(stream):
        ex.exago_eval_all(net.h, ex.make_batch(x, lam, mask, obj_factor=0.8, stream=stream), *outs)

    got = capture_and_replay(ex, call, [x, lam, mask],
                             [t(b2.x, torch.float64), t(b2.lam, torch.float64),
                              t(b2.mask, torch.uint8)], outs)
    ref = net.outputs(b2.B)
    ex.exago_eval_all(net.h, ex.make_batch(t(b2.x, torch.float64), t(b2.lam, torch.float64),
                                           t(b2.mask, torch.uint8), obj_factor=0.8),
                      ref["f"], ref["grad"], ref["gh"], ref["jval"], ref["hval"])
    torch.cuda.synchronize()
    for k, v in zip(("f", "grad", "gh", "jval", "hval"), got):
        np.testing.assert_array_equal(v, ref[k].cpu().numpy(), err_msg=k)
    net.close()


@pytest.mark.parametrize("schedule", [2, 3])
def test_cartesian_call_captured_in_a_graph(ex, schedule):
    import torch
    from test_gpu_cartesian import to_cartesian
    g = synth.grid_2000()
    b1 = synth.contingency_batch(3, g, 96)       # chunked: three chunks on two streams
    b2 = synth.contingency_batch(4, g, 96)
    x1, l1 = to_cartesian(g, b1, 5)
    x2, l2 = to_cartesian(g, b2, 6)
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=schedule)
    n, me, mi, nj, nh = ex.exago_net_dims_cart(net.h)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    x, lam, mask = t(x1, torch.float64), t(l1, torch.float64), t(b1.mask, torch.uint8)
    z = lambda *s: torch.empty(*s, dtype=torch.float64, device="cuda")
    outs = [z(b1.B), z(b1.B, n), z(b1.B, me + mi), z(b1.B, nj), z(b1.B, nh)]

    def call(stream):
        ex.exago_eval_cart(net.h, ex.make_batch(x, lam, mask, obj_factor=0.8, stream=stream),
                           *outs)

    got = capture_and_replay(ex, call, [x, lam, mask],
                             [t(x2, torch.float64), t(l2, torch.float64), t(b2.mask, torch.uint8)],
                             outs)
    ref = [z(b1.B), z(b1.B, n), z(b1.B, me + mi), z(b1.B, nj), z(b1.B, nh)]
    ex.exago_eval_cart(net.h, ex.make_batch(t(x2, torch.float64), t(l2, torch.float64),
                                            t(b2.mask, torch.uint8), obj_factor=0.8), *ref)
    torch.cuda.synchronize()
    for k, v, r in zip(("f", "grad", "gh", "jval", "hval"), got, ref):
        np.testing.assert_array_equal(v, r.cpu().numpy(), err_msg=k)
    net.close()
