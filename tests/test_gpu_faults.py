"""GPU: failure paths that fault nothing -- device allocations made to fail on the host (the
library's testing hook), a batch whose workspace exceeds the device, and a serving arena that
cannot be allocated.  Each returns EXAGO_ENOMEM, and the library keeps working afterwards."""
import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import gpu_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    yield exago
    exago.exago_test_fail_allocations(0)


def test_net_create_allocation_failure(ex):
    g = synth.grid_30bus()
    ex.exago_test_fail_allocations(1)
    try:
        with pytest.raises(ex.ExagoError) as ei:
            ex.Net(g)                                 # an upload fails; earlier ones are freed
        assert ei.value.name == "EXAGO_ENOMEM"
    finally:
        ex.exago_test_fail_allocations(0)
    net = ex.Net(g)                                   # and the next create works
    b = synth.random_batch(3, g, 2)
    out = gpu_eval(net, b)
    assert np.all(np.isfinite(out["hval"]))


def test_workspace_allocation_failure_then_recovery(ex):
    import torch
    g = synth.grid_2000()
    net = ex.Net(g)
    b = synth.random_batch(4, g, 8)
    ex.exago_test_fail_allocations(1)
    try:
        with pytest.raises(ex.ExagoError) as ei:
            gpu_eval(net, b)                          # the workspace allocation fails
        assert ei.value.name == "EXAGO_ENOMEM"
    finally:
        ex.exago_test_fail_allocations(0)
    out = gpu_eval(net, b)
    ref = gpu_eval(ex.Net(g), b)
    for k in ref:
        np.testing.assert_array_equal(out[k], ref[k])


def test_batch_larger_than_the_device(ex):
    import torch
    g = synth.grid_30bus()
    net = ex.Net(g)
    ex.exago_net_set_config(net.h, schedule=1)       # workspace grows with the batch
    B = 1 << 30
    need = ex.exago_eval_workspace_size(net.h, B)
    total = torch.cuda.get_device_properties(0).total_memory
    assert need > 4 * total                          # the allocation cannot succeed
    x = torch.zeros(1, net.n, dtype=torch.float64, device="cuda")
    out = net.outputs(1)
    bt = ex.make_batch(x, x.new_zeros(1, net.m))
    bt.B = B                                          # refused before any launch
    with pytest.raises(ex.ExagoError) as ei:
        net.eval_all(bt, out)
    assert ei.value.name == "EXAGO_ENOMEM"
    b = synth.random_batch(5, g, 1)
    assert np.all(np.isfinite(gpu_eval(net, b)["gh"]))


def test_serve_arena_allocation_failure(ex):
    ex.exago_test_fail_allocations(1)
    try:
        with pytest.raises(ex.ExagoError) as ei:
            ex.exago_serve_create(1 << 20, 1, 1)
        assert ei.value.name == "EXAGO_ENOMEM"
    finally:
        ex.exago_test_fail_allocations(0)
    srv = ex.exago_serve_create(1 << 20, 1, 1)
    ex.exago_serve_destroy(srv)


def test_coupling_slack_and_cartesian_allocation_failures(ex):
    """The coupling rows' and the slacks' device tables, and the cartesian schedule's workspace
    growth: each failed allocation returns EXAGO_ENOMEM, and the same call then succeeds."""
    import torch
    g = synth.make_grid(141, 120, 160, 30)
    net = ex.Net(g)
    parent = synth.coupling_parents("chain", 6)
    for make in (lambda: ex.Coupling(net, parent),
                 lambda: ex.Slack(net, [0, 1], [0, 1], [-1, 1], [1.0, 2.0])):
        ex.exago_test_fail_allocations(1)
        try:
            with pytest.raises(ex.ExagoError) as ei:
                make()
            assert ei.value.name == "EXAGO_ENOMEM"
        finally:
            ex.exago_test_fail_allocations(0)
        make().close()
    b = synth.random_batch(141, g, 4)
    x = torch.as_tensor(b.x, device="cuda")
    gh = torch.empty(4, g.m + g.nb, dtype=torch.float64, device="cuda")
    bt = ex.make_batch(x)
    ex.exago_test_fail_allocations(1)        # the net has no workspace yet: growth fails
    try:
        with pytest.raises(ex.ExagoError) as ei:
            ex.exago_eval_cart(net.h, bt, gh=gh)
        assert ei.value.name == "EXAGO_ENOMEM"
    finally:
        ex.exago_test_fail_allocations(0)
    ex.exago_eval_cart(net.h, bt, gh=gh)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(gh.cpu().numpy()))
    net.close()
