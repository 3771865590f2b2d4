"""GPU: the serving loop (exago_serve_*).  Requests on grids of different sizes run concurrently;
each result must equal the same request evaluated alone; admission is gated by slots and by the
device arena; queue overflow, deadlines and oversized requests return their status codes.
"""
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


class Req:
    """One request's device inputs and outputs (kept alive until it completes)."""

    def __init__(self, ex, net, batch):
        self.batch = batch
        self.d = to_device(batch)
        self.bt = ex.make_batch(self.d["x"], self.d["lam"], self.d["mask"], self.d["pd_scale"],
                                self.d["obj_weight"], batch.sigma, gen_mask=self.d["gen_mask"])
        self.out = net.outputs(batch.B)

    def host(self):
        return {k: v.cpu().numpy() for k, v in self.out.items() if v is not None}


def alone(ex, net, r):
    import torch
    out = net.outputs(r.batch.B, hess=r.out.get("hval") is not None)
    net.eval_all(r.bt, out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


@pytest.mark.parametrize("merge", [1, 32])
def test_mixed_grids_same_alone_and_in_the_mix(ex, oracle_mod, merge):
    """Requests on three grids, with their own branch and generator masks, load scales, weights
    and objective factors, some without the Hessian: merged or not, every result equals the
    request evaluated alone."""
    import torch
    grids = [synth.grid_sized(5, 118), synth.grid_2000(), synth.grid_sized(6, 10_000)]
    nets = [ex.Net(g) for g in grids]
    srv = ex.exago_serve_create(1 << 30, max_slots=6, n_streams=3)
    try:
        ex.exago_serve_set_merge(srv, merge)
        ids = [ex.exago_serve_register(srv, n.h) for n in nets]
        rng = np.random.default_rng(11)
        reqs, tickets = [], []
        for k in range(24):
            gi = int(rng.integers(3))
            B = int(rng.integers(1, 9))
            b = synth.random_batch(100 + k, grids[gi], B, masks=bool(k % 2), pd_scale=bool(k % 3),
                                   obj_weight=bool(k % 4), sigma=float(rng.choice([0.0, 0.8, 1.0])),
                                   gen_masks=k % 3 == 1)
            r = Req(ex, nets[gi], b)
            if k % 5 == 0:
                r.out["hval"] = None           # a different set of outputs: never merged with the rest
            t = ex.exago_serve_submit(srv, ids[gi], r.bt, **r.out)
            reqs.append((gi, r))
            tickets.append(t)
        for t in tickets:
            ex.exago_serve_wait(srv, t)
        torch.cuda.synchronize()
        for (gi, r), t in zip(reqs, tickets):
            got, ref = r.host(), alone(ex, nets[gi], r)
            for key in ref:
                np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
        gi, r = next((gi, r) for gi, r in reqs if r.out["hval"] is not None)
        compare_instance(r.host(), 0, oracle_eval(oracle_mod, grids[gi], r.batch, 0), "served")
        p50, p99, n = ex.exago_serve_stats(srv)
        assert n == len(tickets) and 0 < p50 <= p99
    finally:
        ex.exago_serve_destroy(srv)


def test_memory_gated_admission(ex):
    """An arena that holds one request's workspace at a time still serves every request."""
    import torch
    g = synth.grid_2000()
    net = ex.Net(g)
    ws = ex.exago_eval_workspace_size(net.h, 8)
    srv = ex.exago_serve_create(ws + 4096, max_slots=4, n_streams=2)
    try:
        nid = ex.exago_serve_register(srv, net.h)
        reqs = [Req(ex, net, synth.random_batch(200 + k, g, 8, masks=True)) for k in range(4)]
        tickets = [ex.exago_serve_submit(srv, nid, r.bt, **r.out) for r in reqs]
        for t in tickets:
            ex.exago_serve_wait(srv, t)
        torch.cuda.synchronize()
        for r in reqs:
            got, ref = r.host(), alone(ex, net, r)
            for key in ref:
                np.testing.assert_array_equal(got[key], ref[key])
        # a request that needs more than the whole arena is refused at submission
        big = Req(ex, net, synth.random_batch(300, g, 64))
        with pytest.raises(ex.ExagoError) as ei:
            ex.exago_serve_submit(srv, nid, big.bt, **big.out)
        assert ei.value.name == "EXAGO_ENOMEM"
    finally:
        ex.exago_serve_destroy(srv)


def test_queue_full_and_deadline(ex):
    """The only slot is held by a request whose inputs wait behind a long, bounded GPU sleep on the
    caller's stream: later requests queue, the queue fills (EBUSY) and a short deadline expires."""
    import torch
    g = synth.grid_sized(8, 118)
    net = ex.Net(g)
    srv = ex.exago_serve_create(1 << 28, max_slots=1, n_streams=1)
    try:
        ex.exago_serve_set_merge(srv, 1)       # the late request must queue, not join the first
        i = ex.exago_serve_register(srv, net.h)
        # every input is uploaded before the sleep (a pageable upload would wait for it)
        first = Req(ex, net, synth.random_batch(400, g, 2))
        late = Req(ex, net, synth.random_batch(410, g, 1))
        small = [Req(ex, net, synth.random_batch(420 + k, g, 1)) for k in range(8)]
        torch.cuda.synchronize()
        torch.cuda._sleep(400_000_000)          # about 0.2 s of spinning on the caller's stream
        t_first = ex.exago_serve_submit(srv, i, first.bt, **first.out)
        t_late = ex.exago_serve_submit(srv, i, late.bt, deadline_ms=1.0, **late.out)
        busy, accepted = 0, []
        for r in small:
            try:
                accepted.append((r, ex.exago_serve_submit(srv, i, r.bt, **r.out)))
            except ex.ExagoError as e:
                assert e.name == "EXAGO_EBUSY"
                busy += 1
        assert busy > 0 and len(accepted) >= 3
        assert not ex.exago_serve_poll(srv, t_first)    # still behind the sleep
        with pytest.raises(ex.ExagoError) as ei:
            ex.exago_serve_wait(srv, t_late)
        assert ei.value.name == "EXAGO_ETIMEOUT"
        ex.exago_serve_wait(srv, t_first)
        got, ref = first.host(), alone(ex, net, first)
        for key in ref:
            np.testing.assert_array_equal(got[key], ref[key])
        for r, t in accepted:
            ex.exago_serve_wait(srv, t)
            got, ref = r.host(), alone(ex, net, r)
            np.testing.assert_array_equal(got["hval"], ref["hval"])
        p50, p99, n = ex.exago_serve_stats(srv)
        assert n == 1 + len(accepted) and p99 >= 100.0    # the first waited out the sleep
    finally:
        ex.exago_serve_destroy(srv)


def test_serve_argument_errors(ex):
    with pytest.raises(ex.ExagoError):
        ex.exago_serve_create(0, 1, 1)
    with pytest.raises(ex.ExagoError):
        ex.exago_serve_create(1 << 20, 0, 1)
    srv = ex.exago_serve_create(1 << 20, 1, 1)
    try:
        with pytest.raises(ex.ExagoError):
            ex.exago_serve_set_merge(srv, 0)
        g = synth.grid_30bus()
        net = ex.Net(g)
        r = Req(ex, net, synth.random_batch(1, g, 1))
        with pytest.raises(ex.ExagoError):
            ex.exago_serve_submit(srv, 5, r.bt, **r.out)        # unknown net id
        with pytest.raises(ex.ExagoError):
            ex.exago_serve_wait(srv, 12345)                     # unknown ticket
    finally:
        ex.exago_serve_destroy(srv)


def test_queued_requests_merge_into_one_launch(ex):
    """With the only slot held behind a GPU sleep, requests queue; when it frees, one admission
    takes them all (up to the merge budget), and every result equals its request alone."""
    import torch
    g = synth.grid_sized(9, 118)
    net = ex.Net(g)
    srv = ex.exago_serve_create(1 << 28, max_slots=1, n_streams=1)
    try:
        ex.exago_serve_set_merge(srv, 8)
        i = ex.exago_serve_register(srv, net.h)
        first = Req(ex, net, synth.random_batch(500, g, 1))
        rest = [Req(ex, net, synth.random_batch(510 + k, g, 1 + k % 3, masks=True, sigma=0.5 * k))
                for k in range(3)]
        torch.cuda.synchronize()
        torch.cuda._sleep(200_000_000)
        tickets = [ex.exago_serve_submit(srv, i, first.bt, **first.out)]
        tickets += [ex.exago_serve_submit(srv, i, r.bt, **r.out) for r in rest]
        for t in tickets:
            ex.exago_serve_wait(srv, t)
        for r in [first] + rest:
            got, ref = r.host(), alone(ex, net, r)
            for key in ref:
                np.testing.assert_array_equal(got[key], ref[key])
    finally:
        ex.exago_serve_destroy(srv)


@pytest.mark.parametrize("rate", [0.0, 20000.0])
def test_native_load_generator(ex, rate):
    """exago_serve_drive, closed loop and Poisson arrivals, over clients on two grids: requests
    complete, the server's quantiles come back, and every client's last result equals its
    request evaluated alone."""
    import torch
    grids = [synth.grid_sized(9, 118), synth.grid_sized(10, 300)]
    nets = [ex.Net(g) for g in grids]
    reqs, group = [], []
    for gi, g in enumerate(grids):
        for k in range(6):
            reqs.append(Req(ex, nets[gi], synth.random_batch(700 + 10 * gi + k, g, 1 + k % 2,
                                                            masks=True, sigma=0.8)))
            group.append(gi)
    torch.cuda.synchronize()
    srv = ex.exago_serve_create(1 << 29, max_slots=4, n_streams=2)
    try:
        ids = [ex.exago_serve_register(srv, n.h) for n in nets]
        clients = [(ids[gi], r.bt, r.out) for gi, r in zip(group, reqs)]
        res = ex.exago_serve_drive(srv, clients, group, [0.6, 0.4], rate, 0.3, seed=5)
    finally:
        ex.exago_serve_destroy(srv)
    assert res["completed"] > len(reqs) and res["seconds"] > 0.25
    assert 0.0 < res["p50_ms"] <= res["p99_ms"]
    for gi, r in zip(group, reqs):
        got, ref = r.host(), alone(ex, nets[gi], r)
        for key in ref:
            np.testing.assert_array_equal(got[key], ref[key])
