"""Host-side checks of the C-ABI library (no GPU): symbols, plans, patterns, validation.

The library is built for sm_103a; these tests only load it and call the host-only planning
entry points, never a kernel.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2203_10587_gb300 import build, exago, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return exago.lib()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "exago.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(exago_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    syms = header_symbols()
    assert len(syms) >= 19
    for s in syms:
        assert hasattr(L, s), f"{s} declared in include/exago.h but not exported"
    assert sorted(exago.EXPORTS) == syms


def plan(grid):
    return exago.Net(grid, plan_only=True)


GRIDS = {
    "30bus": lambda: synth.grid_30bus(),
    "2000bus": lambda: synth.grid_2000(),
    "shunts_tr": lambda: synth.make_grid(5, 50, 70, 20, transformer_frac=0.5, shunts=True),
}


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_patterns_match_oracle(L, oracle_mod, name):
    g = GRIDS[name]()
    net = plan(g)
    b = synth.random_batch(3, g, 1)
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), b.x[0], b.lam[0])
    jr, jc = exago.exago_net_jac_pattern(net.h)
    hr, hc = exago.exago_net_hess_pattern(net.h)
    np.testing.assert_array_equal(jr, r["J"][0])
    np.testing.assert_array_equal(jc, r["J"][1])
    np.testing.assert_array_equal(hr, r["H"][0])
    np.testing.assert_array_equal(hc, r["H"][1])
    assert net.nnzJ == 4 * g.nb + 16 * g.nl + 2 * g.ng
    assert net.nnzH == 3 * g.nb + 4 * g.nl + g.ng


def write_counts(net, g):
    """How many times the kernels' write plan touches each J and H position."""
    A = lambda n: exago.exago_net_plan_array(net.h, n)
    nl, nb = g.nl, g.nb
    cj = np.zeros(net.nnzJ, np.int64)
    ch = np.zeros(net.nnzH, np.int64)
    off = A("br_off").reshape(12, nl)
    shared = A("br_shared")
    # every planned write lands inside its output buffer
    assert np.all(off[:8] >= 0) and np.all(off[:8] < net.nnzJ)
    assert np.all(off[8:] >= 0) and np.all(off[8:] < net.nnzH)
    for name, hi in (("bus_jP", net.nnzJ), ("bus_jQ", net.nnzJ), ("gen_jP", net.nnzJ),
                     ("gen_jQ", net.nnzJ), ("bus_h", net.nnzH), ("gen_h", net.nnzH)):
        a = A(name)
        assert np.all(a >= 0) and np.all(a < hi), name
    assert np.all(A("bus_jP") + A("bus_k") < net.nnzJ)
    sl = A("br_slot")
    assert np.all(sl >= 0) and np.all(sl < 2 * nl)
    assert np.all((shared >= -1) & (shared < max(1, nl)))
    direct = shared < 0
    for c in range(8):
        np.add.at(cj, off[c][direct], 1)
    for c in range(8, 12):
        np.add.at(ch, off[c][direct], 1)
    fix_dst, fix_isH = A("fix_dst"), A("fix_isH")
    np.add.at(cj, fix_dst[fix_isH == 0], 1)
    np.add.at(ch, fix_dst[fix_isH == 1], 1)
    nnzJg = net.nnzJ - 8 * nl
    cj[nnzJg:] += 1                                  # h rows: four entries per row, branch-local
    jP, jQ, k = A("bus_jP"), A("bus_jQ"), A("bus_k")
    for pos in (jP, jP + k, jQ, jQ + k):
        np.add.at(cj, pos, 1)
    np.add.at(cj, A("gen_jP"), 1)
    np.add.at(cj, A("gen_jQ"), 1)
    np.add.at(ch, A("bus_h"), 1)
    np.add.at(ch, A("gen_h"), 1)
    return cj, ch


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_every_output_written_exactly_once(L, name):
    g = GRIDS[name]()
    cj, ch = write_counts(plan(g), g)
    assert np.all(cj == 1) and np.all(ch == 1)


def parallel_grid():
    """Parallel branches (same and opposite direction) and two generators on one bus."""
    from test_oracle import tiny_grid
    return tiny_grid(4, [(0, 1), (1, 0), (1, 2), (2, 3), (1, 2), (3, 0)],
                     [(0.01, 0.1, 0.02, 0.0), (0.02, 0.15, 0.01, 0.98), (0.015, 0.12, 0.0, 0.0),
                      (0.01, 0.2, 0.03, 1.02), (0.03, 0.25, 0.0, 0.0), (0.02, 0.1, 0.01, 0.0)],
                     [(0, 0.01, 20.0), (0, 0.02, 25.0), (2, 0.005, 30.0)],
                     Pd=[0.1, 0.5, 0.4, 0.2], Gs=[0.01, 0.0, 0.02, 0.0], Bs=[0.0, 0.05, 0.0, 0.1])


def test_parallel_branches_plan(L, oracle_mod):
    g = parallel_grid()
    net = plan(g)
    cj, ch = write_counts(net, g)
    assert np.all(cj == 1) and np.all(ch == 1)
    shared = exago.exago_net_plan_array(net.h, "br_shared")
    assert list(shared) == [0, 1, 2, -1, 3, -1]
    b = synth.random_batch(3, g, 1)
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), b.x[0], b.lam[0])
    np.testing.assert_array_equal(exago.exago_net_jac_pattern(net.h)[1], r["J"][1])
    np.testing.assert_array_equal(exago.exago_net_hess_pattern(net.h)[1], r["H"][1])


def test_slots_sorted_by_bus_then_branch(L):
    g = synth.grid_30bus()
    net = plan(g)
    ptr = exago.exago_net_plan_array(net.h, "slot_ptr")
    sl = exago.exago_net_plan_array(net.h, "br_slot").reshape(2, g.nl)
    owner = np.empty(2 * g.nl, np.int64)
    key = np.empty(2 * g.nl, np.int64)
    for side, bus in ((0, g.f), (1, g.t)):
        owner[sl[side]] = bus
        key[sl[side]] = 2 * np.arange(g.nl) + side
    assert np.all(np.diff(owner) >= 0)
    for i in range(g.nb):
        assert np.all(owner[ptr[i]:ptr[i + 1]] == i)
        assert np.all(np.diff(key[ptr[i]:ptr[i + 1]]) > 0)


def test_ineq_bounds(L):
    g = synth.grid_30bus()
    g.rateA[3] = 0.0
    net = plan(g)
    lo, hi = exago.exago_net_ineq_bounds(net.h)
    assert np.all(lo == 0)
    np.testing.assert_array_equal(hi[:g.nl][[0, 1]], g.rateA[[0, 1]] ** 2)
    assert np.isinf(hi[3]) and np.isinf(hi[g.nl + 3])


@pytest.mark.parametrize("case", ["bus_range", "self_loop", "zero_impedance", "neg_tap", "nan",
                                  "gen_range", "nb0", "basemva"])
def test_validation_errors(L, case):
    g = synth.grid_30bus()
    args = list(exago._grid_args(g))
    if case == "bus_range":
        g.t[2] = g.nb
    elif case == "self_loop":
        g.t[2] = g.f[2]
    elif case == "zero_impedance":
        g.r[4] = 0.0
        g.x[4] = 0.0
    elif case == "neg_tap":
        g.tap[1] = -1.0
    elif case == "nan":
        g.x[0] = np.nan
    elif case == "gen_range":
        g.gbus[0] = -1
    args = list(exago._grid_args(g))
    if case == "nb0":
        args[0] = 0
    if case == "basemva":
        args[-1] = 0.0
    with pytest.raises(exago.ExagoError) as ei:
        exago.exago_net_plan(*args)
    assert ei.value.name == "EXAGO_EINVAL"


def test_degenerate_single_bus(L):
    g = synth.Grid(nb=1, Gs=np.array([0.1]), Bs=np.zeros(1), Pd=np.array([0.3]), Qd=np.zeros(1),
                   f=np.zeros(0, np.int32), t=np.zeros(0, np.int32), r=np.zeros(0), x=np.zeros(0),
                   b=np.zeros(0), tap=np.zeros(0), rateA=np.zeros(0), gbus=np.zeros(1, np.int32),
                   c2=np.array([0.01]), c1=np.array([10.0]), c0=np.zeros(1))
    net = plan(g)
    assert (net.n, net.m, net.nnzJ, net.nnzH) == (4, 2, 6, 4)
    cj, ch = write_counts(net, g)
    assert np.all(cj == 1) and np.all(ch == 1)


def test_eval_on_plan_only_net_is_a_state_error(L):
    net = plan(synth.grid_30bus())
    batch = exago.exago_batch(1, 8, None, None, None, None, 1.0, None, None, 0)
    rc = L.exago_eval_all(net.h, ctypes.byref(batch), None, None, None, None, None)
    assert exago.STATUS[rc] == "EXAGO_ESTATE"


def test_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(exago.ExagoError) as ei:
        exago.Net(synth.grid_30bus())
    assert ei.value.name in ("EXAGO_ECUDA", "EXAGO_ENOMEM")
