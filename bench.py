#!/usr/bin/env python
"""Benchmark: batched ACOPF model evaluations per second on one GB300 (or N, one process each).

Workload (the paper's ACTIVSg2000-sized N-1 security case, Sec. V-A, with synthetic data): a
2,000-bus grid (2,700 branches, 500 generators) x 512 contingencies, each taking one non-bridge
branch out of service, with per-contingency states drawn around a base state (sigma 0.02).  One
step evaluates, for all 512 states, the objective, its gradient, g | h, the Jacobian values and
the Lagrangian Hessian values (exago_eval_all).  Inputs rotate over 4 device copies (236 MB) and
each step writes 343 MB of outputs, so neither fits the 126 MB L2 between reuses.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs under torchrun, one rank per GPU; every rank evaluates its own 512 contingencies (weak
scaling, no collective on the data path) and rank 0 prints one JSON line.  --impl reference times
the CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched ACOPF evals/s (f,∇f,g,J,∇²L) + HBM GB/s vs unbatched; p50/p99 latency"
UNIT = "evals/s"
WORKLOAD = "2000-bus x 512 N-1 contingencies: f, grad f, g|h, J values, Lagrangian Hessian values"
B_DEFAULT = 512
N_INPUT_SETS = 4
# FP64 work per unit with every output requested, counted from the kernel source on the fast
# sincos path (an FMA counts 2 flops; doublings run on the integer pipe and count nothing):
# (flops, instructions).  Per 2000-bus state they sum to 515,655 flops / 340,855 instructions.
FP64_PER_BRANCH = (168, 109)   # sincos, flows, 16 derivatives, h and its J row, Hessian fold
FP64_PER_SLOT = (7, 7)         # a branch end's record summed into its bus (all but the first)
FP64_PER_BUS = (16, 9)         # shunt, balances (Euler, from the derivative sums), diagonal terms
FP64_PER_GEN = (12, 9)         # balance, cost Hessian, gradient and objective terms of a generator
FP64_PER_STATE = (255, 255)    # the objective's fixed 256-lane reduction tree
# FP64 peak derived from the unit counts and clocks: 152 SMs x 2 FP64 FMA per SM per clock x
# 2 flops x 2.07 GHz (the probe measured 1.20 TFLOP/s at 1.97 GHz under load).
SMS, FP64_FMA_PER_SM_CLK, SM_MAX_GHZ = 152, 2, 2.07
FP64_PEAK_TFLOPS = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_GHZ / 1e3
FP64_PEAK_GINSTR = SMS * FP64_FMA_PER_SM_CLK * SM_MAX_GHZ
# dram bytes per launch of the dominant kernel from its ncu capture, by kernel name; a kernel
# changed since its capture has no entry
# (the persistent kernel's entry is the per-thread tiling's; "persistent/warp" the warp tiling's)
TRAFFIC_BYTES = {"persistent": 384_794_624,        # 63.7 MB read + 321.1 MB written (ncu, 2000-bus x 512)
                 "persistent/warp": 783_639_296}   # 278.2 MB read + 505.5 MB written (ncu, same workload)
HBM_PEAK_FALLBACK_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=50)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--B", type=int, default=B_DEFAULT)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    p.add_argument("--no-serve", action="store_true", help="skip the serving-mix measurement")
    p.add_argument("--config", default="", help="launch configuration instead of autotuning, "
                   "e.g. schedule=2,block=64,occupancy=16")
    p.add_argument("--serve-seconds", type=float, default=1.5, help="length of each serving phase")
    p.add_argument("--only", default="", choices=["", "kkt", "pflow", "cart"],
                   help="time only the KKT step, the power-flow step (--steps calls after "
                        "--warmup) or the cartesian evaluation, and print its object")
    return p.parse_args()


# ---- multi-rank helpers (one process per GPU; states are independent, so ranks share nothing
# but the timing reduction)

def rank_seed(rank: int, s: int) -> int:
    """Seed of input set s on `rank`: every rank evaluates its own contingency states."""
    return 3 + 1000 * rank + 17 * s


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's elapsed time (all ranks receive it)."""
    if world == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, B: int, elapsed_ms: float) -> float:
    """Whole-job evaluations per second: all ranks' states over the slowest rank's time."""
    return world * steps * B / (elapsed_ms / 1e3)


# ---- clocks during the timed region ------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.lines: list[str] = []
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- CPU oracle ----------------------------------------------------------------------------------

class OracleRunner:
    """The CPU oracle over the batch's states on a pool of host threads (ctypes releases the GIL
    during each evaluation)."""

    def __init__(self, grid, batch, threads: int):
        import concurrent.futures as cf
        from oracle import acopf
        acopf.build()
        self.acopf, self.batch = acopf, batch
        self.onet = acopf.OracleNet(grid)
        self.pool = cf.ThreadPoolExecutor(max_workers=threads)
        self.next = 0
        self.one(0)

    def one(self, i):
        b = i % self.batch.B
        self.acopf.evaluate(self.onet, self.batch.x[b], self.batch.lam[b], self.batch.mask[b], None,
                            1.0, self.batch.sigma)

    def rate(self, n_evals: int):
        """Evaluations per second over the next n_evals states (cycling the batch)."""
        idx = range(self.next, self.next + n_evals)
        self.next += n_evals
        t0 = time.perf_counter()
        list(self.pool.map(self.one, idx))
        dt = time.perf_counter() - t0
        return n_evals / dt, dt

    def close(self):
        self.pool.shutdown()


def oracle_rate(grid, batch, n_evals: int, threads: int):
    """Oracle evaluations per second over n_evals states on `threads` host threads."""
    runner = OracleRunner(grid, batch, threads)
    try:
        return runner.rate(n_evals)
    finally:
        runner.close()


def bench_config(grid, B: int, world: int, n: int, m: int, nnzJ: int, nnzH: int) -> dict:
    """The `config` object of both arms' JSON line (the same keys and values for one workload)."""
    return {"workload": WORKLOAD, "nb": grid.nb, "nl": grid.nl, "ng": grid.ng, "B": B,
            "n": n, "m": m, "nnzJ": nnzJ, "nnzH": nnzH,
            "l2": "inputs rotate over 4 device copies (236 MB) and each step writes 343 MB, "
                  "both larger than L2",
            "parallelism": f"{world} rank(s), each its own 512 contingencies, no collective"}


def oracle_dims(grid, batch):
    """(n, m, nnzJ, nnzH) as the oracle's evaluation of the first state emits them."""
    from oracle import acopf
    r = acopf.evaluate(acopf.OracleNet(grid), batch.x[0], batch.lam[0], batch.mask[0])
    return grid.n, grid.m, int(r["J"][0][-1]), int(r["H"][0][-1])


def run_reference(args, rank: int):
    """--impl reference: the oracle on the host cores; each step is a bounded sample."""
    if rank != 0:
        return
    from paper_2203_10587_gb300 import synth
    grid = synth.grid_2000()
    batch = synth.contingency_batch(3, grid, args.B)
    cores = os.cpu_count() or 1
    per_step = cores
    runner = OracleRunner(grid, batch, cores)
    for _ in range(args.warmup):
        runner.rate(per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        runner.rate(per_step)
    total = time.perf_counter() - t0
    runner.close()
    value = args.steps * per_step / total
    sample = f"{per_step} of the {args.B} contingency states per step (one per host thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded 2000-bus grid and N-1 states; ACTIVSg2000 not available)",
        "config": bench_config(grid, args.B, args.gpus, *oracle_dims(grid, batch)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---- serving mix ---------------------------------------------------------------------------------

SERVE_MIX = ((118, 0.4), (2_000, 0.3), (10_000, 0.2), (70_000, 0.1))
SERVE_CLIENTS = 64
SERVE_SLOTS, SERVE_STREAMS, SERVE_BUDGET = 16, 8, 2 << 30


def quantiles(v):
    v = sorted(v)
    q = lambda p: v[min(len(v) - 1, int(p * (len(v) - 1) + 0.5))] if v else None
    return q(0.50), q(0.99)


class ServeClients:
    """64 simulated IPM clients on grids of 118 / 2,000 / 10,000 / 70,000 buses (40/30/20/10%);
    each owns one device state (B = 1) and its output buffers, and has at most one request out."""

    def __init__(self, exago, synth, torch, np, dev, seed=5):
        import ctypes
        self.exago, self.torch, self.ct = exago, torch, ctypes
        self.grids = [synth.grid_sized(50 + k, nb) for k, (nb, _) in enumerate(SERVE_MIX)]
        self.nets = [exago.Net(g) for g in self.grids]
        share = [p for _, p in SERVE_MIX]
        counts = [int(round(SERVE_CLIENTS * p)) for p in share]
        counts[0] += SERVE_CLIENTS - sum(counts)
        self.by_grid = []
        self.clients = []
        td = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        for gi, cnt in enumerate(counts):
            ids = []
            for _ in range(cnt):
                b = synth.random_batch(seed * 1000 + len(self.clients), self.grids[gi], 1)
                x, lam = td(b.x, torch.float64), td(b.lam, torch.float64)
                bt = exago.make_batch(x, lam, obj_factor=1.0)
                out = self.nets[gi].outputs(1, dev)
                ptrs = [ctypes.c_void_p(out[k].data_ptr()) for k in ("f", "grad", "gh", "jval", "hval")]
                ids.append(len(self.clients))
                self.clients.append((gi, x, lam, bt, out, ptrs))
            self.by_grid.append(ids)
        self.share = share
        torch.cuda.synchronize()

    def one_at_a_time(self, rng, n):
        """The same kind of requests, each launched alone and waited for (no overlap)."""
        seq = [self.pick(rng) for _ in range(n)]
        for c in seq[:8]:
            self.eval_alone(c)
        lat = []
        t0 = time.perf_counter()
        for c in seq:
            t = time.perf_counter()
            self.eval_alone(c)
            lat.append(1e3 * (time.perf_counter() - t))
        dt = time.perf_counter() - t0
        p50, p99 = quantiles(lat)
        return {"evals_per_s": n / dt, "p50_ms": p50, "p99_ms": p99, "requests": n}

    def pick(self, rng):
        gi = int(rng.choice(len(self.share), p=self.share))
        ids = self.by_grid[gi]
        return ids[int(rng.integers(len(ids)))]

    def eval_alone(self, c):
        gi, _, _, bt, out, _ = self.clients[c]
        self.nets[gi].eval_all(bt, out)
        self.torch.cuda.synchronize()

    def run(self, rng, seconds, rate=None):
        """Closed loop (rate None: every client resubmits as soon as its request completes) or
        Poisson arrivals at `rate` requests/s, each taking a free client of a grid drawn from the
        mix, driven by the library's native load generator (exago_serve_drive) on a fresh
        server.  Returns throughput and the server's submit-to-completion latency quantiles."""
        ex = self.exago
        srv = ex.exago_serve_create(SERVE_BUDGET, SERVE_SLOTS, SERVE_STREAMS)
        try:
            nids = [ex.exago_serve_register(srv, n.h) for n in self.nets]
            clients = [(nids[gi], bt, out) for gi, _, _, bt, out, _ in self.clients]
            group = [gi for gi, *_ in self.clients]
            r = ex.exago_serve_drive(srv, clients, group, self.share, rate or 0.0, seconds,
                                     seed=int(rng.integers(1 << 62)))
        finally:
            ex.exago_serve_destroy(srv)
        res = {"evals_per_s": r["completed"] / r["seconds"], "p50_ms": r["p50_ms"],
               "p99_ms": r["p99_ms"], "requests": r["completed"]}
        if rate is not None:
            res.update(offered_per_s=rate, deferred=r["deferred"])
        return res


def time_calls(torch, fn, reps, warm=3):
    """ms per call of fn (CUDA events on the current stream, after warm-up)."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_other_configs(exago, synth, torch, np, dev):
    """The other workloads: a 10,000-bus grid evaluated 1,000 times in sequence (one IPM run),
    10,000 buses x 64 load scenarios with the adjoint products, and a meshed 2,000-bus grid of
    6,000 branches x 512 states under both tilings of the persistent schedule."""
    td = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    g = synth.grid_10k()
    net = exago.Net(g)
    res = {}
    # C2: one state, 1,000 evaluations in sequence
    b1 = synth.random_batch(2, g, 1)
    x1, l1 = td(b1.x, torch.float64), td(b1.lam, torch.float64)
    bt1 = exago.make_batch(x1, l1)
    out1 = net.outputs(1, dev)
    tuned1 = exago.exago_net_autotune(net.h, bt1, out1["f"], out1["grad"], out1["gh"],
                                      out1["jval"], out1["hval"])
    ms = time_calls(torch, lambda: net.eval_all(bt1, out1), 1000)
    res["10k_bus_single_x1000"] = {"evals_per_s": 1e3 / ms, "ms_per_eval": ms,
                                   "launch_config": {k: tuned1[k] for k in
                                                     ("schedule", "block", "occupancy", "tile_group",
                                                      "stage_records", "tiling")}}
    # C4: 64 load scenarios, all outputs, then J^T v and (grad^2 L) u
    b = synth.scenario_batch(4, g, 64)
    x, lam, ps, w = (td(b.x, torch.float64), td(b.lam, torch.float64),
                     td(b.pd_scale, torch.float64), td(b.obj_weight, torch.float64))
    bt = exago.make_batch(x, lam, None, ps, w, b.sigma)
    out = net.outputs(64, dev)
    exago.exago_net_reserve(net.h, 64)
    tuned = exago.exago_net_autotune(net.h, bt, out["f"], out["grad"], out["gh"], out["jval"],
                                     out["hval"])
    ms = time_calls(torch, lambda: net.eval_all(bt, out), 200)
    v = torch.randn(64, net.m, dtype=torch.float64, device=dev)
    u = torch.randn(64, net.n, dtype=torch.float64, device=dev)
    o = torch.empty(64, net.n, dtype=torch.float64, device=dev)
    ms_jtv = time_calls(torch, lambda: exago.exago_eval_jtv(net.h, bt, v, o), 200)
    ms_hvp = time_calls(torch, lambda: exago.exago_eval_hvp(net.h, bt, u, o), 200)
    res["10k_bus_x64_scenarios"] = {"evals_per_s": 64e3 / ms, "ms_per_batch": ms,
                                    "jtv_per_s": 64e3 / ms_jtv, "hvp_per_s": 64e3 / ms_hvp,
                                    "launch_config": {k: tuned[k] for k in
                                                      ("schedule", "block", "occupancy", "tile_group",
                                                       "stage_records", "tiling")}}
    net.close()
    # a meshed grid (2,000 buses, 6,000 branches: mean degree 6, up to 16) x 512 states: the bus
    # degrees within a warp vary more, which the branch-per-warp tiling does not mind
    gd = synth.make_grid(7, 2000, 6000, 500, max_degree=32)
    bd = synth.random_batch(8, gd, 512, masks=True, sigma=0.02)
    netd = exago.Net(gd)
    btd = exago.make_batch(td(bd.x, torch.float64), td(bd.lam, torch.float64), td(bd.mask, torch.uint8))
    outd = netd.outputs(512, dev)
    exago.exago_net_reserve(netd.h, 512)
    tunedd = exago.exago_net_autotune(netd.h, btd, outd["f"], outd["grad"], outd["gh"],
                                      outd["jval"], outd["hval"], reps=5)
    ms_tuned = time_calls(torch, lambda: netd.eval_all(btd, outd), 100)
    timed = {}
    for name, cfg in (("branch_per_thread", dict(schedule=2, block=64, occupancy=16, tile_group=1)),
                      ("branch_per_warp", dict(schedule=2, tiling=2, block=128, occupancy=16,
                                               tile_group=1))):
        exago.exago_net_set_config(netd.h, **cfg)
        timed[name] = time_calls(torch, lambda: netd.eval_all(btd, outd), 100)
    res["2000_bus_6000_branch_x512"] = {
        "evals_per_s": 512e3 / ms_tuned, "ms_per_batch": ms_tuned,
        "ms_per_batch_by_tiling": timed, "mean_degree": 2 * gd.nl / gd.nb,
        "launch_config": {k: tunedd[k] for k in ("schedule", "block", "occupancy", "tile_group",
                                                  "stage_records", "tiling")}}
    netd.close()
    return res


def run_coupling(exago, synth, torch, np, dev, hbm_peak):
    """The coupling (ramp) rows between the states of a batch and their transpose product, on
    three workloads: the 2,000-bus x 512 N-1 batch (511 contingencies tied to the base case), a
    10,000-bus grid over 64 periods and a 70,000-bus grid over 512 periods (chains).  Each launch
    is timed alone with CUDA events after a 256 MB write has flushed L2 ("cold"), and back to back
    ("warm", inputs in L2 as right after the solver wrote them).  Algorithmic bytes: forward -- Pg
    of every state read once, r written, parent indices; transpose -- nu read, out written, the
    parent and child tables."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {}
    for name, grid, kind, B in (("2000bus_x512_contingencies", synth.grid_2000, "star", 512),
                                ("10k_bus_x64_periods", synth.grid_10k, "chain", 64),
                                ("70k_bus_x512_periods", lambda: synth.grid_sized(9, 70_000),
                                 "chain", 512)):
        g = grid()
        net = exago.Net(g)
        parent = synth.coupling_parents(kind, B)
        h = exago.exago_coupling_create(net.h, parent)
        gen = torch.Generator(device=dev)
        gen.manual_seed(11)
        x = torch.randn(B, net.n, dtype=torch.float64, device=dev, generator=gen)
        nu = torch.randn(B, g.ng, dtype=torch.float64, device=dev, generator=gen)
        r = torch.empty(B, g.ng, dtype=torch.float64, device=dev)
        o = torch.empty(B, g.ng, dtype=torch.float64, device=dev)
        fwd = lambda: exago.exago_eval_coupling(h, x, r)
        jtv = lambda: exago.exago_eval_coupling_jtv(h, nu, o, g.ng)
        nchild = int((parent >= 0).sum())
        bytes_fwd = 2 * B * g.ng * 8 + 4 * B
        bytes_jtv = 2 * B * g.ng * 8 + 4 * (3 * B + 1 + nchild)
        out = {"states": B, "ng": g.ng, "structure": kind}
        for what, fn, nbytes in (("rows", fwd, bytes_fwd), ("transpose", jtv, bytes_jtv)):
            warm = time_calls(torch, fn, 500)
            cold = []
            for _ in range(50):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                cold.append(e0.elapsed_time(e1))
            cold_ms = float(np.median(cold))
            out[what] = {"warm_us": warm * 1e3, "cold_us": cold_ms * 1e3,
                         "algorithmic_bytes": nbytes,
                         "cold_gbs": nbytes / (cold_ms * 1e-3) / 1e9,
                         "cold_frac_hbm": nbytes / (cold_ms * 1e-3) / 1e9 / hbm_peak}
        exago.exago_coupling_destroy(h)
        net.close()
        res[name] = out
    return res


def run_slacks(exago, synth, torch, np, dev, hbm_peak):
    """Feasibility slacks (load loss, power imbalance) added to a finished evaluation of the
    2,000-bus x 512 batch: an imbalance pair on every P and Q balance and load loss at the loaded
    buses (about 4.5 slacks per bus), balance terms, objective and gradient in one call; warm
    (inputs in L2, as right after the evaluation).  Algorithmic bytes per state: z read, grad_z
    written, 2 nb balance values read and written, f read and written."""
    g = synth.grid_2000()
    B, nb = 512, g.nb
    load = np.flatnonzero(g.Pd > 0.3)
    bus = np.concatenate([np.tile(np.arange(nb), 4), load, load]).astype(np.int32)
    row = np.concatenate([np.zeros(2 * nb), np.ones(2 * nb), np.zeros(len(load)),
                          np.ones(len(load))]).astype(np.int32)
    sign = np.concatenate([-np.ones(nb), np.ones(nb), -np.ones(nb), np.ones(nb),
                           -np.ones(2 * len(load))]).astype(np.int32)
    cost = np.full(bus.shape[0], 500.0)
    net = exago.Net(g)
    sl = exago.Slack(net, bus, row, sign, cost)
    nz = bus.shape[0]
    z = torch.rand(B, nz, dtype=torch.float64, device=dev) * 0.1
    gh = torch.zeros(B, net.m, dtype=torch.float64, device=dev)
    f = torch.zeros(B, dtype=torch.float64, device=dev)
    gz = torch.empty(B, nz, dtype=torch.float64, device=dev)
    x = torch.zeros(B, net.n, dtype=torch.float64, device=dev)
    bt = exago.make_batch(x)
    ms = time_calls(torch, lambda: exago.exago_eval_slack(sl, bt, z, gh, net.m, f, gz), 500)
    nbytes = B * (16 * nz + 32 * nb + 16)
    # the full evaluation with the slacks, on the N-1 states: exago_eval_all then exago_eval_slack,
    # and the same through exago_eval_all_slack
    b = synth.contingency_batch(3, g, B)
    td = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    bte = exago.make_batch(td(b.x, torch.float64), td(b.lam, torch.float64),
                           td(b.mask, torch.uint8), obj_factor=1.0)
    exago.exago_net_set_config(net.h, schedule=2, block=64, occupancy=16, stage_records=2,
                               tile_group=1)
    out = net.outputs(B, dev)
    ms_eval = time_calls(torch, lambda: net.eval_all(bte, out), 200, warm=5)

    def two_calls():
        net.eval_all(bte, out)
        exago.exago_eval_slack(sl, bte, z, out["gh"], net.m, out["f"], gz)

    ms_two = time_calls(torch, two_calls, 200, warm=5)
    ms_fused = time_calls(torch, lambda: exago.exago_eval_all_slack(
        net.h, bte, sl, z, out["f"], out["grad"], out["gh"], out["jval"], out["hval"], gz),
        200, warm=5)
    sl.close()
    net.close()
    return {"workload": "2000-bus x 512 states, imbalance pairs on every balance plus load loss",
            "slacks_per_state": nz, "us_per_call": ms * 1e3, "algorithmic_bytes": nbytes,
            "gbs": nbytes / (ms * 1e-3) / 1e9, "frac_hbm": nbytes / (ms * 1e-3) / 1e9 / hbm_peak,
            "with_evaluation": {"eval_ms": ms_eval, "eval_then_slack_ms": ms_two,
                                "fused_ms": ms_fused,
                                "fused": "exago_eval_all_slack (the two calls in one)"}}


def run_cartesian(exago, synth, torch, np, dev, hbm_peak, polar_ms):
    """The power-balance-cartesian formulation (exago_eval_cart) on the headline workload, the
    2,000-bus x 512 N-1 batch at the same operating points (e = Vm cos Va, f = Vm sin Va), all
    outputs, CUDA events over back-to-back calls (each call writes 350 MB, more than L2).
    Algorithmic bytes per state: x, lambda (m + nb) and mask read; f, grad, g | h (m + nb),
    J (nnzJ + 2 nb) and H written; the network tables once per call."""
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 512)
    nb = g.nb
    x = b.x.copy()
    x[:, :nb] = b.x[:, nb:2 * nb] * np.cos(b.x[:, :nb])
    x[:, nb:2 * nb] = b.x[:, nb:2 * nb] * np.sin(b.x[:, :nb])
    lam = np.concatenate([b.lam, np.random.default_rng(3).normal(size=(b.B, nb))], axis=1)
    td = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    X, LAM, M = td(x, torch.float64), td(lam, torch.float64), td(b.mask, torch.uint8)
    net = exago.Net(g)
    n, me, mi, nj, nh = exago.exago_net_dims_cart(net.h)
    bt = exago.make_batch(X, LAM, M, obj_factor=b.sigma)
    z = lambda *sh: torch.empty(*sh, dtype=torch.float64, device=dev)
    out = [z(b.B), z(b.B, n), z(b.B, me + mi), z(b.B, nj), z(b.B, nh)]
    ms = time_calls(torch, lambda: exago.exago_eval_cart(net.h, bt, *out), 200, warm=5)
    exago.exago_net_set_config(net.h, schedule=3)       # the chunked two-stream schedule
    ms_chunked = time_calls(torch, lambda: exago.exago_eval_cart(net.h, bt, *out), 200, warm=5)
    exago.exago_net_set_config(net.h)
    v = torch.randn(b.B, me + mi, dtype=torch.float64, device=dev)
    u = torch.randn(b.B, n, dtype=torch.float64, device=dev)
    o = torch.empty(b.B, n, dtype=torch.float64, device=dev)
    ms_jtv = time_calls(torch, lambda: exago.exago_eval_cart_jtv(net.h, bt, v, o), 200)
    ms_hvp = time_calls(torch, lambda: exago.exago_eval_cart_hvp(net.h, bt, u, o), 200)
    per_state = 8 * (n + (me + mi) + 1 + n + (me + mi) + nj + nh) + g.nl
    net_bytes = 8 * (11 * g.nl + 4 * nb + 4 * g.ng) + 4 * (2 * g.nl + 8 * nb + g.ng + 4 * g.nl)
    nbytes = per_state * b.B + net_bytes
    net.close()
    return {"workload": "2000-bus x 512 N-1 states in rectangular voltages, all outputs",
            "evals_per_s": b.B / (ms * 1e-3), "ms_per_batch": ms,
            "vs_polar_same_states": polar_ms / ms,
            "jtv_per_s": b.B / (ms_jtv * 1e-3), "hvp_per_s": b.B / (ms_hvp * 1e-3),
            "algorithmic_bytes": nbytes, "hbm_gbs": nbytes / (ms * 1e-3) / 1e9,
            "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm_peak,
            "schedule": "persistent work list (one launch through the graph cache; records in an "
                        "L2-resident ring of states)",
            "ms_per_batch_chunked": ms_chunked,
            "chunked_schedule": "per chunk of 41 states, branch records on the caller's stream "
                                "while the previous chunk's bus assembly runs on a side stream; "
                                "a ring of 3 chunks of records stays in L2"}


def run_kkt(exago, synth, torch, np, dev, reps=10, warm=2):
    """The interior-point KKT step (exago_kkt_solve) of the 2,000-bus x 512 N-1 batch, with the
    batch's own Jacobian and Lagrangian Hessian (exago_eval_all), dx_i = 1 + sum_j |W_ij|,
    dc ~ U(0.5, 2), rhs ~ N(0, 1): assembly, eliminations, the batched block L D L' and both
    sweeps, CUDA events over back-to-back calls.  FP64-bound: the flops per state are
    exago_kkt_info's count (its 4 x 4 block products dominate)."""
    g = synth.grid_2000()
    b = synth.contingency_batch(3, g, 512)
    B = b.B
    net = exago.Net(g)
    td = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    bt = exago.make_batch(td(b.x, torch.float64), td(b.lam, torch.float64),
                          td(b.mask, torch.uint8), obj_factor=1.0)
    out = net.outputs(B, dev, f=False, grad=False, gh=False)
    net.eval_all(bt, out)
    # dx = 1 + the absolute row sums of W (both triangles from the lower one)
    hp, hc = exago.exago_net_hess_pattern(net.h)
    rows = torch.as_tensor(np.repeat(np.arange(net.n), np.diff(hp)), device=dev)
    cols = torch.as_tensor(hc.astype(np.int64), device=dev)
    a = out["hval"].abs()
    dx = torch.ones(B, net.n, dtype=torch.float64, device=dev)
    dx.index_add_(1, rows, a)
    dx.index_add_(1, cols, a * (rows != cols).to(torch.float64))
    gen = torch.Generator(device=dev)
    gen.manual_seed(3)
    dc = 0.5 + 1.5 * torch.rand(B, net.m, dtype=torch.float64, device=dev, generator=gen)
    rhs = torch.randn(B, net.n + net.m, dtype=torch.float64, device=dev, generator=gen)
    sol = torch.empty_like(rhs)
    inertia = torch.empty(B, 2, dtype=torch.int32, device=dev)
    k = exago.exago_kkt_create(net.h)
    info = exago.exago_kkt_info(k)
    ws = torch.empty(exago.exago_kkt_workspace_size(k, B), dtype=torch.uint8, device=dev)
    fn = lambda: exago.exago_kkt_solve(k, out["jval"], out["hval"], dx, dc, rhs, sol, inertia, ws)
    ms = time_calls(torch, fn, reps, warm=warm)
    ok = bool((inertia[:, 0] == net.m).all().item() and (inertia[:, 1] == 0).all().item())
    exago.exago_kkt_destroy(k)
    net.close()
    flops = info["flops"] * B
    return {"workload": "2000-bus x 512 N-1 states: KKT [[W + Dx, J'], [J, -Dc]] step per state",
            "ms_per_batch": ms, "states_per_s": B / (ms * 1e-3),
            "factor_blocks": info["blocks"], "block_products_per_state": info["pairs"],
            "levels": info["levels"], "flops_per_state": info["flops"],
            "tflops": flops / (ms * 1e-3) / 1e12,
            "frac_fp64_peak": flops / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
            "inertia_all_correct": ok}


def run_pflow(exago, synth, torch, np, dev, reps=20, warm=2):
    """One power-flow Newton step (exago_pf_step: the evaluation of g and J, then the batched
    2 x 2-block LU of J_pf and both sweeps) for 512 states of a 2,000-bus grid (light load, flat
    start), CUDA events over back-to-back calls."""
    g = synth.make_grid(33, 2000, 2700, 500, transformer_frac=0.2)
    g.Pd *= 0.3
    g.Qd *= 0.3
    bt_ = np.ones(g.nb, np.int32)
    bt_[g.gbus] = 2
    bt_[g.gbus[0]] = 3
    x0 = np.concatenate([np.zeros(g.nb), np.ones(g.nb), np.full(g.ng, g.Pd.sum() / g.ng),
                         np.zeros(g.ng)])
    B = 512
    net = exago.Net(g)
    X = torch.as_tensor(np.repeat(x0[None, :], B, axis=0), device=dev)
    pf = exago.exago_pf_create(net.h, bt_)
    ws = torch.empty(exago.exago_pf_workspace_size(pf, B), dtype=torch.uint8, device=dev)
    bt = exago.make_batch(X, workspace=ws)
    Xn = torch.empty_like(X)
    mis = torch.empty(B, dtype=torch.float64, device=dev)
    ms = time_calls(torch, lambda: exago.exago_pf_step(pf, bt, Xn, mis), reps, warm=warm)
    exago.exago_pf_destroy(pf)
    net.close()
    return {"workload": "2000-bus x 512 states: one power-flow Newton step (g, J, factor, solve)",
            "ms_per_batch": ms, "states_per_s": B / (ms * 1e-3)}


def run_serve(exago, synth, torch, np, dev, seconds):
    rng = np.random.default_rng(5)
    sc = ServeClients(exago, synth, torch, np, dev)
    alone = sc.one_at_a_time(rng, 2000)
    sc.run(rng, 0.3)                                   # warm-up
    peak = sc.run(rng, seconds)
    # the fastest arrival rate the native client sustains (arrivals due at once, every one
    # submitted as soon as a client of its grid is free): offered loads stay below it
    client = sc.run(rng, min(seconds, 0.5), rate=1e9)
    ref = min(peak["evals_per_s"], client["evals_per_s"])
    res = {"workload": "Poisson arrivals of B=1 requests from 64 clients on 118 / 2,000 / 10,000 / "
                       "70,000-bus grids (40/30/20/10%), one registered net per grid",
           "server": {"max_slots": SERVE_SLOTS, "streams": SERVE_STREAMS,
                      "arena_mb": SERVE_BUDGET >> 20, "max_merge_states": 32},
           "one_at_a_time": alone, "closed_loop_peak": peak,
           "client_limit_per_s": client["evals_per_s"],
           "loads_relative_to": "min(closed-loop peak, client limit)"}
    for frac in (0.5, 0.9):
        res[f"load_{frac}"] = sc.run(rng, seconds, rate=frac * ref)
    return res


# ---- GPU arm -------------------------------------------------------------------------------------

def run_gpu(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch
    from paper_2203_10587_gb300 import build, exago, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    exago.lib()
    grid = synth.grid_2000()
    net = exago.Net(grid)
    B = args.B
    sets = [synth.contingency_batch(rank_seed(rank, s), grid, B) for s in range(N_INPUT_SETS)]
    td = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    ins = [(td(b.x, torch.float64), td(b.lam, torch.float64), td(b.mask, torch.uint8)) for b in sets]
    stream = torch.cuda.current_stream(dev)
    batches = [exago.make_batch(x, lam, mask, obj_factor=1.0, stream=stream) for x, lam, mask in ins]
    out = net.outputs(B, dev)
    exago.exago_net_reserve(net.h, B)

    def step(k):
        net.eval_all(batches[k % N_INPUT_SETS], out)

    tuned = None
    if args.config:
        cfg = {k: int(v) for k, v in (kv.split("=") for kv in args.config.split(","))}
        exago.exago_net_set_config(net.h, **cfg)
    elif not args.no_autotune:
        tuned = exago.exago_net_autotune(net.h, batches[0], out["f"], out["grad"], out["gh"],
                                         out["jval"], out["hval"], reps=10)
    launch_cfg = exago.exago_net_get_config(net.h, B)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    exago.exago_net_check(net.h)

    # ---- timed region: K steps, barrier + synchronize on both sides
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[0]
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        step(k)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    exago.exago_net_check(net.h)
    elapsed_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    elapsed_ms = max_over_ranks(elapsed_ms, world, dev)
    value = job_value(world, args.steps, B, elapsed_ms)

    # ---- per-kernel timing of the same evaluation (CUDA events on the launching stream)
    prof = exago.exago_eval_profile(net.h, batches[0], out["f"], out["grad"], out["gh"],
                                    out["jval"], out["hval"], reps=min(args.steps, 100))
    phases = {k[len("phase: "):]: v for k, v in prof if k.startswith("phase: ")}
    prof = [(k, v) for k, v in prof if not k.startswith("phase: ")]
    kernels_per_step = len(prof)
    total_prof = sum(ms for _, ms in prof)
    top_name, top_ms = max(prof, key=lambda kv: kv[1])
    # FP64 work of the dominant kernel per launch: the fused persistent kernel does every stage,
    # the multi-kernel schedule's top kernel is the branch kernel
    if top_name == "persistent":
        work = [(FP64_PER_BRANCH, grid.nl), (FP64_PER_SLOT, 2 * grid.nl - grid.nb),
                (FP64_PER_BUS, grid.nb), (FP64_PER_GEN, grid.ng), (FP64_PER_STATE, 1)]
        per_unit = ("per state: %d branches x %d + %d extra branch ends x %d + %d buses x %d + "
                    "%d generators x %d + %d FP64 flops" % (
                        grid.nl, FP64_PER_BRANCH[0], 2 * grid.nl - grid.nb, FP64_PER_SLOT[0],
                        grid.nb, FP64_PER_BUS[0], grid.ng, FP64_PER_GEN[0], FP64_PER_STATE[0]))
    else:
        work = [(FP64_PER_BRANCH, grid.nl)]
        per_unit = "per state: %d branches x %d FP64 flops" % (grid.nl, FP64_PER_BRANCH[0])
    flops_state = sum(w[0] * n for w, n in work)
    instr_state = sum(w[1] * n for w, n in work)
    units = B
    achieved_tf = flops_state * units / (top_ms * 1e-3) / 1e12
    achieved_gi = instr_state * units / (top_ms * 1e-3) / 1e9

    # ---- algorithmic HBM bytes per evaluation (read x, lambda, mask; write every output)
    n, m, nnzJ, nnzH = net.n, net.m, net.nnzJ, net.nnzH
    in_bytes = 8 * (n + m) + grid.nl
    out_bytes = 8 * (1 + n + m + nnzJ + nnzH)
    net_bytes = 112 * grid.nl + 64 * grid.nb + 40 * grid.ng   # network tables, once per launch
    bytes_per_eval = in_bytes + out_bytes
    hbm_gbs = (bytes_per_eval * B + net_bytes) * args.steps / (elapsed_ms / 1e3) / 1e9
    hbm_peak, hbm_src = HBM_PEAK_FALLBACK_GBS, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm_peak, hbm_src = float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        pass

    # ---- the same kernels one instance at a time (unbatched)
    n_single = min(B, 128)
    xs, ls, ms_ = ins[0]
    singles = [exago.make_batch(xs[i:i + 1], ls[i:i + 1], ms_[i:i + 1], stream=stream)
               for i in range(n_single)]
    out1 = net.outputs(1, dev)
    for i in range(min(8, n_single)):
        net.eval_all(singles[i], out1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n_single):
        net.eval_all(singles[i], out1)
    e1.record(stream)
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1) / n_single
    unbatched = {"value": 1e3 / single_ms, "unit": UNIT, "ms_per_eval": single_ms,
                 "hbm_gbs": (bytes_per_eval + net_bytes) / (single_ms * 1e-3) / 1e9,
                 "evals": n_single}

    # ---- end to end through the public API with host buffers.  Three streams pipeline the steps
    # as a client would: inputs of step k+1 go up while step k evaluates and step k-1's outputs
    # come down; events order every buffer reuse.
    pin = lambda tt: tt.cpu().pin_memory()
    hins = [(pin(x), pin(l), pin(mk)) for x, l, mk in ins]
    dins = [(torch.empty_like(x), torch.empty_like(l), torch.empty_like(mk)) for x, l, mk in ins]
    s_in, s_ev, s_out = (torch.cuda.Stream(dev) for _ in range(3))
    dbatches = [exago.make_batch(x, l, mk, stream=s_ev) for x, l, mk in dins]
    outs = [out, net.outputs(B, dev)]
    hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    h2d = sum(tt.numel() * tt.element_size() for tt in hins[0])
    d2h = sum(v.numel() * v.element_size() for v in out.values())
    k_e2e = max(5, min(args.steps, 300))
    ev = lambda: torch.cuda.Event()
    ev_in = [ev() for _ in range(N_INPUT_SETS)]
    ev_eval = [ev() for _ in range(N_INPUT_SETS)]
    ev_out = [ev() for _ in range(2)]
    used = {"eval": [False] * N_INPUT_SETS, "out": [False, False]}

    def e2e_step(k):
        j, o = k % N_INPUT_SETS, k % 2
        with torch.cuda.stream(s_in):
            if used["eval"][j]:
                s_in.wait_event(ev_eval[j])          # step k-4 has read these inputs
            for d, h in zip(dins[j], hins[j]):
                d.copy_(h, non_blocking=True)
            ev_in[j].record(s_in)
        s_ev.wait_event(ev_in[j])
        if used["out"][o]:
            s_ev.wait_event(ev_out[o])               # step k-2's outputs have come down
        net.eval_all(dbatches[j], outs[o])
        ev_eval[j].record(s_ev)
        used["eval"][j] = True
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_eval[j])
            for key, v in outs[o].items():
                hout[key].copy_(v, non_blocking=True)
            ev_out[o].record(s_out)
        used["out"][o] = True

    for k in range(min(3, k_e2e)):
        e2e_step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s_in)
    s_ev.wait_event(t0)
    s_out.wait_event(t0)
    for k in range(k_e2e):
        e2e_step(k)
    s_out.wait_event(ev_eval[(k_e2e - 1) % N_INPUT_SETS])
    t1.record(s_out)
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1)
    e2e_value = job_value(world, k_e2e, B, max_over_ranks(e2e_ms, world, dev))

    if rank != 0:
        return
    serve = None if args.no_serve else run_serve(exago, synth, torch, np, dev, args.serve_seconds)
    others = None if args.no_serve else run_other_configs(exago, synth, torch, np, dev)
    coupling = None if args.no_serve else run_coupling(exago, synth, torch, np, dev, hbm_peak)
    cartesian = None if args.no_serve else run_cartesian(exago, synth, torch, np, dev, hbm_peak,
                                                         top_ms)
    slacks = None if args.no_serve else run_slacks(exago, synth, torch, np, dev, hbm_peak)
    kkt = None if args.no_serve else run_kkt(exago, synth, torch, np, dev)
    pflow = None if args.no_serve else run_pflow(exago, synth, torch, np, dev)
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded 2000-bus grid and N-1 states; ACTIVSg2000 not available)",
        "config": bench_config(grid, B, world, n, m, nnzJ, nnzH),
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": sorted(step_ms)[max(0, int(0.99 * len(step_ms)) - 1)]},
        "hbm_gbs": hbm_gbs,
        "unbatched": unbatched,
        "kernels_ms": {k: v for k, v in prof},
        "kernel_share": {k: v / total_prof for k, v in prof},
        "phases_ms": phases,
        "roofline": {"kernel": top_name, "bound": "alu", "achieved": achieved_tf,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved_tf / FP64_PEAK_TFLOPS,
                     "traffic": TRAFFIC_BYTES.get(
                         top_name + ("/warp" if top_name == "persistent" and
                                     launch_cfg.get("tiling") == exago.TILING_WARP else "")),
                     "per_unit": f"{per_unit} = {flops_state} flops ({instr_state} FP64 instructions)",
                     "units_per_launch": units, "launch_ms": top_ms,
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz",
                     "fp64_instr": {"achieved_g_per_s": achieved_gi, "peak_g_per_s": FP64_PEAK_GINSTR,
                                    "frac": achieved_gi / FP64_PEAK_GINSTR},
                     "hbm": {"achieved_gbs": (bytes_per_eval * B + net_bytes) / (top_ms * 1e-3) / 1e9,
                             "peak_gbs": hbm_peak, "peak_source": hbm_src,
                             "frac": (bytes_per_eval * B + net_bytes) / (top_ms * 1e-3) / 1e9 / hbm_peak,
                             "algorithmic_bytes_per_launch": bytes_per_eval * B + net_bytes}},
        "gpu_launches": kernels_per_step * args.steps,
        "launch_config": {"autotuned": tuned, "used": launch_cfg},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": k_e2e,
                "how": "pinned host inputs up, exago_eval_all, every output down; three streams "
                       "pipeline consecutive steps"},
    }
    if serve is not None:
        res["serve"] = serve
    if others is not None:
        res["other_workloads"] = others
    if coupling is not None:
        res["coupling_rows"] = coupling
    if cartesian is not None:
        res["cartesian"] = cartesian
    if slacks is not None:
        res["feasibility_slacks"] = slacks
    if kkt is not None:
        res["kkt_step"] = kkt
    if pflow is not None:
        res["pflow_step"] = pflow
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        n_evals = 256 * cores
        rate, dt = oracle_rate(grid, sets[0], n_evals, cores)
        res["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{n_evals} evaluations of the first contingency states "
                                         f"({dt:.1f} s wall on {cores} threads)"}
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.only:   # one sub-workload alone (profiling): rank 0 of one process
        import numpy as np
        import torch
        from paper_2203_10587_gb300 import build, exago, synth
        build.build()
        exago.lib()
        dev = torch.device("cuda", local_rank)
        if args.only == "cart":
            res = run_cartesian(exago, synth, torch, np, dev, HBM_PEAK_FALLBACK_GBS, float("nan"))
            print(json.dumps({"cartesian": res}), flush=True)
            return
        fn = run_kkt if args.only == "kkt" else run_pflow
        res = fn(exago, synth, torch, np, dev, reps=max(1, args.steps), warm=args.warmup)
        print(json.dumps({("kkt_step" if args.only == "kkt" else "pflow_step"): res}), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
