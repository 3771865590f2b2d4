"""GPU: calls that share a net's internal workspace from several streams and host threads.

Every call that uses the net's internal workspace is ordered after the workspace's last use on
another stream, and holds the net's lock from the workspace lookup until its kernels are queued,
so that another thread's workspace growth (which frees the old buffer) cannot slip in between.
These tests issue such calls without host synchronisation between them and check that every
result equals the same call made alone, bit for bit.
"""
import threading

import numpy as np
import pytest

from paper_2203_10587_gb300 import synth
from parity_util import compare_instance, oracle_eval, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


class Call:
    """Device inputs and outputs of one polar or cartesian evaluation, kept alive."""

    def __init__(self, ex, net, b, stream, cartesian=False):
        import torch
        self.ex, self.net, self.cart = ex, net, cartesian
        d = to_device(b)
        x, lam = d["x"], d["lam"]
        if cartesian:
            nb = net.nb
            Va, Vm = x[:, :nb], x[:, nb:2 * nb]
            x = x.clone()
            x[:, :nb] = Vm * torch.cos(Va)
            x[:, nb:2 * nb] = Vm * torch.sin(Va)
            lam = torch.cat([lam, torch.ones(b.B, nb, dtype=torch.float64, device="cuda")], 1)
            n, me, mi, nj, nh = ex.exago_net_dims_cart(net.h)
        else:
            n, me, mi, nj, nh = net.n, net.m, 0, net.nnzJ, net.nnzH
        self.keep = (x, lam, d)
        self.bt = ex.make_batch(x, lam, d["mask"], None, None, b.sigma, stream=stream)
        z = lambda *s: torch.full(s, np.nan, dtype=torch.float64, device="cuda")
        self.out = {"f": z(b.B), "grad": z(b.B, n), "gh": z(b.B, me + mi), "jval": z(b.B, nj),
                    "hval": z(b.B, nh)}

    def run(self):
        fn = self.ex.exago_eval_cart if self.cart else self.ex.exago_eval_all
        o = self.out
        fn(self.net.h, self.bt, o["f"], o["grad"], o["gh"], o["jval"], o["hval"])

    def host(self):
        return {k: v.cpu().numpy() for k, v in self.out.items()}


def test_two_streams_internal_workspace_are_ordered(ex, oracle_mod):
    """Back-to-back calls on two streams with the internal workspace (the persistent schedule's
    record ring and ticket counters) give the results of the calls made one at a time."""
    import torch
    g = synth.make_grid(91, 500, 650, 120, shunts=True)
    net = ex.Net(g)
    sA, sB = torch.cuda.Stream(), torch.cuda.Stream()
    batches = [synth.random_batch(91 + k, g, 24, masks=True, sigma=0.8) for k in range(6)]
    calls = [Call(ex, net, b, sA if k % 2 == 0 else sB) for k, b in enumerate(batches)]
    alone = []
    for c in calls:
        c.run()
        torch.cuda.synchronize()
        alone.append(c.host())
    for _ in range(3):
        for c in calls:
            c.out = {k: torch.full_like(v, np.nan) for k, v in c.out.items()}
        torch.cuda.synchronize()
        for c in calls:          # no synchronisation between the calls
            c.run()
        torch.cuda.synchronize()
        ex.exago_net_check(net.h)
        for c, a in zip(calls, alone):
            h = c.host()
            for k in a:
                np.testing.assert_array_equal(h[k], a[k], err_msg=k)
    compare_instance(alone[0], 3, oracle_eval(oracle_mod, g, batches[0], 3), "two streams")


def test_threads_with_workspace_growth(ex):
    """One host thread runs cartesian evaluations while another runs polar evaluations of growing
    batches, each on its own stream, on one net with its internal workspace: the polar calls grow
    (free and reallocate) the workspace the cartesian calls use.  Every result equals the call
    made alone."""
    import torch
    g = synth.make_grid(93, 300, 389, 77, transformer_frac=0.3, shunts=True)
    net = ex.Net(g)
    sA, sB = torch.cuda.Stream(), torch.cuda.Stream()
    cart = [Call(ex, net, synth.random_batch(200 + k, g, 40, masks=True, sigma=0.7), sA, True)
            for k in range(4)]
    polar = [Call(ex, net, synth.random_batch(300 + k, g, B, masks=True, sigma=0.9), sB)
             for k, B in enumerate((1, 3, 9, 27, 81, 243, 729))]
    # results alone, each on a fresh net (so that no call sees a grown workspace)
    alone_c, alone_p = [], []
    for lst, acc in ((cart, alone_c), (polar, alone_p)):
        for c in lst:
            fresh = ex.Net(g)
            h, c.net = c.net, fresh
            c.run()
            torch.cuda.synchronize()
            acc.append(c.host())
            c.net = h
            fresh.close()
    errors = []

    def worker(lst, reps):
        try:
            for _ in range(reps):
                for c in lst:
                    c.run()
        except Exception as e:   # reported by the main thread
            errors.append(e)

    ta = threading.Thread(target=worker, args=(cart, 6))
    tb = threading.Thread(target=worker, args=(polar, 1))
    ta.start(); tb.start(); ta.join(); tb.join()
    torch.cuda.synchronize()
    assert not errors, errors
    ex.exago_net_check(net.h)
    for lst, acc in ((cart, alone_c), (polar, alone_p)):
        for c, a in zip(lst, acc):
            h = c.host()
            for k in a:
                np.testing.assert_array_equal(h[k], a[k], err_msg=k)
