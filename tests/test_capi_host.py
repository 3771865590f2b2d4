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


def test_binding_structs_and_enums_match_the_header():
    """The ctypes mirrors of the header's structs list the same fields in the same order with
    the same C types, and the binding's enum constants have the header's values."""
    src = open(os.path.join(ROOT, "include", "exago.h")).read()
    ctype = {"int": ctypes.c_int, "long long": ctypes.c_longlong, "double": ctypes.c_double,
             "size_t": ctypes.c_size_t}
    for name, mirror in (("exago_config", exago.exago_config),):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", src).group(1)
        fields = re.findall(r"^\s*([a-z ]+?)\s+(\w+);", body, re.M)
        assert [f for _, f in fields] == [f for f, _ in mirror._fields_], name
        for (ct, f), (mf, mt) in zip(fields, mirror._fields_):
            assert ctypes.sizeof(ctype[ct.strip()]) == ctypes.sizeof(mt), (name, f)
    enums = {f"{a}_{b}": int(v) for a, b, v in
             re.findall(r"\bEXAGO_(SCHED|GRAPH|STAGE|TILING)_(\w+)\s*=\s*(\d+)", src)}
    assert len(enums) == 14
    for k, v in enums.items():
        assert getattr(exago, k) == v, k


def test_binding_struct_layouts_match_the_c_compiler(tmp_path):
    """Every ctypes mirror of a header struct has the size and field offsets that the host C
    compiler gives the header's struct (compiled here with gcc)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    mirrors = {"exago_config": exago.exago_config, "exago_batch": exago.exago_batch,
               "exago_serve_client": exago.exago_serve_client}
    cfield = {"lambda_": "lambda"}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "exago.h"', "int main(void) {"]
    for name, m in mirrors.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in m._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {cfield.get(f, f)}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for name, m in mirrors.items():
        assert int(out[name]) == ctypes.sizeof(m), name
        for f, _ in m._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(m, f).offset, f"{name}.{f}"


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


def write_plan(net, g, slot_parallel=False):
    """Replays the kernels' writes from the plan: returns, for every J and H position, how often
    it is written and which column the writing thread believes it holds.  slot_parallel replays
    the slot-parallel bus tiles, where a group's leading slot writes its neighbour's entries at
    slot_pos."""
    A = lambda n: exago.exago_net_plan_array(net.h, n)
    nl, nb = g.nl, g.nb
    jr, jc = exago.exago_net_jac_pattern(net.h)
    hr, hc = exago.exago_net_hess_pattern(net.h)
    cj = np.zeros(net.nnzJ, np.int64)
    ch = np.zeros(net.nnzH, np.int64)
    colj = np.full(net.nnzJ, -1, np.int64)
    colh = np.full(net.nnzH, -1, np.int64)

    def wj(p, col):
        assert 0 <= p < net.nnzJ
        cj[p] += 1
        colj[p] = col

    def wh(p, col):
        assert 0 <= p < net.nnzH
        ch[p] += 1
        colh[p] = col

    slot_ptr, slot_nbr, slot_ref = A("slot_ptr"), A("slot_nbr"), A("slot_ref")
    # every branch end appears in exactly one slot, at its own bus, naming the other bus; its
    # record lives at that slot (br_slot)
    assert sorted(slot_ref) == list(range(2 * nl))
    br_slot = A("br_slot")
    assert np.all(slot_ref[br_slot] == np.concatenate([2 * np.arange(nl), 2 * np.arange(nl) + 1]))
    for i in range(nb):
        for sl in range(slot_ptr[i], slot_ptr[i + 1]):
            l, end = divmod(int(slot_ref[sl]), 2)
            own, other = (g.f[l], g.t[l]) if end == 0 else (g.t[l], g.f[l])
            assert own == i and slot_nbr[sl] == other
    # branch: two h rows of four entries, columns (Va_lo, Va_hi, Vm_lo, Vm_hi)
    nnzJg = net.nnzJ - 8 * nl
    for l in range(nl):
        lo, hi = sorted((int(g.f[l]), int(g.t[l])))
        for row in (nnzJg + 4 * l, nnzJg + 4 * nl + 4 * l):
            for q, col in enumerate((lo, hi, nb + lo, nb + hi)):
                wj(row + q, col)
    jP, jQ, hA, hM = A("bus_jP"), A("bus_jQ"), A("bus_hA"), A("bus_hM")
    bk, nlow, gptr, gord = A("bus_k"), A("bus_nlow"), A("gen_ptr"), A("gen_ord")
    hpg = hr[2 * nb]
    slot_bus, slot_pos = A("slot_bus"), A("slot_pos")
    for i in range(nb):
        nbrs = slot_nbr[slot_ptr[i]:slot_ptr[i + 1]]
        assert np.all(np.diff(nbrs) >= 0)
        assert np.all(slot_bus[slot_ptr[i]:slot_ptr[i + 1]] == i)
        pos, k = 0, bk[i]
        if slot_parallel:
            lead = [(int(slot_pos[sl]), int(slot_nbr[sl])) for sl in range(slot_ptr[i], slot_ptr[i + 1])
                    if slot_pos[sl] >= 0]
            for sl in range(slot_ptr[i], slot_ptr[i + 1]):   # -1 only for later parallel branches
                assert (slot_pos[sl] < 0) == (sl > slot_ptr[i] and slot_nbr[sl] == slot_nbr[sl - 1])
        else:
            lead = []
            for j in np.unique(nbrs):
                if pos == nlow[i]:
                    pos += 1
                lead.append((pos, int(j)))
                pos += 1
        for pos, j in lead:
            for base, off, col in ((jP[i], 0, j), (jP[i], k, nb + j), (jQ[i], 0, j), (jQ[i], k, nb + j)):
                wj(base + off + pos, col)
            wh(hM[i] + pos, j)
            if j < i:
                wh(hA[i] + pos, j)
                wh(hM[i] + k + pos, nb + j)
        for base, off, col in ((jP[i], 0, i), (jP[i], k, nb + i), (jQ[i], 0, i), (jQ[i], k, nb + i)):
            wj(base + off + nlow[i], col)
        wh(hA[i] + nlow[i], i)
        wh(hM[i] + nlow[i], i)
        wh(hM[i] + k + nlow[i], nb + i)
        for q in range(gptr[i + 1] - gptr[i]):
            kk = gord[gptr[i] + q]
            wj(jP[i] + 2 * k + q, 2 * nb + kk)
            wj(jQ[i] + 2 * k + q, 2 * nb + g.ng + kk)
            wh(hpg + kk, 2 * nb + kk)
    return cj, ch, colj, colh, jc, hc


def check_write_plan(net, g):
    perms = exago.exago_net_plan_array(net.h, "bus_perm").reshape(4, g.nb)
    deg = np.bincount(np.concatenate([g.f, g.t]), minlength=g.nb)
    for t, perm in enumerate(perms):   # per tile size: each aligned tile permuted, by degree
        T = 32 << t
        for g0 in range(0, g.nb, T):
            grp = perm[g0:g0 + T]
            assert sorted(grp) == list(range(g0, min(g0 + T, g.nb)))
            assert np.all(np.diff(deg[grp]) <= 0)
    for sp in (False, True):
        cj, ch, colj, colh, jc, hc = write_plan(net, g, slot_parallel=sp)
        assert np.all(cj == 1) and np.all(ch == 1)
        np.testing.assert_array_equal(colj, jc)
        np.testing.assert_array_equal(colh, hc)


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_every_output_written_exactly_once_in_its_column(L, name):
    g = GRIDS[name]()
    net = plan(g)
    check_write_plan(net, g)


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
    check_write_plan(net, g)
    # parallel branches 0/1 (buses 0-1) and 2/4 (buses 1-2) occupy adjacent slots of each bus
    ref = list(exago.exago_net_plan_array(net.h, "slot_ref"))
    pos = {r: i for i, r in enumerate(ref)}
    assert abs(pos[2 * 0 + 0] - pos[2 * 1 + 1]) == 1          # both ends at bus 0
    assert abs(pos[2 * 2 + 0] - pos[2 * 4 + 0]) == 1          # both from ends at bus 1
    b = synth.random_batch(3, g, 1)
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), b.x[0], b.lam[0])
    np.testing.assert_array_equal(exago.exago_net_jac_pattern(net.h)[1], r["J"][1])
    np.testing.assert_array_equal(exago.exago_net_hess_pattern(net.h)[1], r["H"][1])


def test_slots_sorted_by_bus_other_bus_branch(L):
    g = synth.grid_30bus()
    net = plan(g)
    ptr = exago.exago_net_plan_array(net.h, "slot_ptr")
    ref = exago.exago_net_plan_array(net.h, "slot_ref")
    l, side = ref // 2, ref % 2
    owner = np.where(side == 0, g.f[l], g.t[l]).astype(np.int64)
    other = np.where(side == 0, g.t[l], g.f[l]).astype(np.int64)
    key = other * (4 * g.nl) + ref
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
    check_write_plan(net, g)


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


def test_phase_shift_validation(L):
    """exago_net_create_shift validates the shifts on the host before any device work: a
    non-finite shift is EINVAL (on any machine); without a GPU a valid one fails at the upload."""
    import torch
    g = synth.make_grid(9, 20, 26, 5, shifter_frac=0.3)
    a = exago._grid_args(g)
    bad = g.shift.copy()
    bad[4] = np.nan
    with pytest.raises(exago.ExagoError) as ei:
        exago.exago_net_create_shift(*a[:12], bad, *a[12:])
    assert ei.value.name == "EXAGO_EINVAL" and "phase shift" in str(ei.value)
    if not torch.cuda.is_available():
        with pytest.raises(exago.ExagoError) as ei:
            exago.Net(g)
        assert ei.value.name in ("EXAGO_ECUDA", "EXAGO_ENOMEM")


# ---- coupling (ramp) rows: host side ---------------------------------------------------------

def coupling_parents():
    rng = np.random.default_rng(31)
    B = 40
    forest = np.full(B, -1, np.int32)
    order = rng.permutation(B)
    for j in range(3, B):
        forest[order[j]] = order[rng.integers(0, j)]
    return {"chain": np.arange(-1, 9, dtype=np.int32),
            "star": np.array([-1] + [0] * 20, np.int32),
            "star_last": np.array([5] * 5 + [-1], np.int32),
            "forest": forest,
            "roots": np.full(4, -1, np.int32)}


@pytest.mark.parametrize("kind", sorted(coupling_parents()))
def test_coupling_pattern_matches_oracle(L, oracle_mod, kind):
    """The exported Jacobian of the coupling rows equals the oracle's rows applied to unit vectors
    (the rows are linear, so this recovers the exact Jacobian)."""
    g = synth.make_grid(8, 12, 16, 3)
    net = plan(g)
    parent = coupling_parents()[kind]
    B = parent.shape[0]
    h = exago.exago_coupling_create(net.h, parent)
    try:
        Bc, rows, nnz = exago.exago_coupling_dims(h)
        assert (Bc, rows, nnz) == (B, B * g.ng, 2 * g.ng * int((parent >= 0).sum()))
        rowptr, col, val = exago.exago_coupling_jac_pattern(h)
        dense = np.zeros((rows, B * net.n))
        for r in range(rows):
            cols = col[rowptr[r]:rowptr[r + 1]]
            assert np.all(np.diff(cols) > 0)
            dense[r, cols] = val[rowptr[r]:rowptr[r + 1]]
        ref = np.zeros_like(dense)
        for j in range(B * net.n):
            e = np.zeros(B * net.n)
            e[j] = 1.0
            ref[:, j] = oracle_mod.coupling(parent, e.reshape(B, net.n), g.nb, g.ng).reshape(-1)
        np.testing.assert_array_equal(dense, ref)
    finally:
        exago.exago_coupling_destroy(h)


@pytest.mark.parametrize("bad", [[-2, 0], [0, 0], [-1, 2], [1, 0, 3]])
def test_coupling_rejects_invalid_parents(L, bad):
    net = plan(synth.grid_30bus())
    with pytest.raises(exago.ExagoError) as ei:
        exago.exago_coupling_create(net.h, np.array(bad, np.int32))
    assert ei.value.name == "EXAGO_EINVAL"


def test_coupling_host_only_refuses_evaluation(L):
    net = plan(synth.grid_30bus())
    h = exago.exago_coupling_create(net.h, np.array([-1, 0], np.int32))
    try:
        rc = L.exago_eval_coupling(h, ctypes.c_void_p(8), ctypes.c_void_p(8), None)
        assert exago.STATUS[rc] == "EXAGO_ESTATE"
        rc = L.exago_eval_coupling_jtv(h, ctypes.c_void_p(8), ctypes.c_void_p(8), 6, 0, None)
        assert exago.STATUS[rc] == "EXAGO_ESTATE"
    finally:
        exago.exago_coupling_destroy(h)
    h = exago.exago_coupling_create(net.h, np.zeros(0, np.int32))
    assert exago.exago_coupling_dims(h) == (0, 0, 0)
    exago.exago_coupling_destroy(h)


# ---- power-balance-cartesian formulation: host side ----------------------------------------------

@pytest.mark.parametrize("name", sorted(GRIDS))
def test_cartesian_patterns_match_oracle(L, oracle_mod, name):
    g = GRIDS[name]()
    net = plan(g)
    b = synth.random_batch(4, g, 1)
    lam = np.concatenate([b.lam[0], np.ones(g.nb)])
    r = oracle_mod.evaluate(oracle_mod.OracleNet(g), b.x[0], lam, cartesian=True)
    n, me, mi, nj, nh = exago.exago_net_dims_cart(net.h)
    assert (n, me, mi) == (g.n, 2 * g.nb, 2 * g.nl + g.nb)
    assert nj == 6 * g.nb + 16 * g.nl + 2 * g.ng and nh == net.nnzH
    jr, jc = exago.exago_net_jac_pattern_cart(net.h)
    hr, hc = exago.exago_net_hess_pattern(net.h)
    np.testing.assert_array_equal(jr, r["J"][0])
    np.testing.assert_array_equal(jc, r["J"][1])
    np.testing.assert_array_equal(hr, r["H"][0])
    np.testing.assert_array_equal(hc, r["H"][1])


def test_cartesian_evaluation_needs_a_device_net(L):
    net = plan(synth.grid_30bus())
    rc = L.exago_eval_cart(net.h, None, None, None, None, None, None)
    assert exago.STATUS[rc] == "EXAGO_ESTATE"
    v = ctypes.c_size_t()
    assert exago.STATUS[L.exago_eval_cart_workspace_size(net.h, 4, ctypes.byref(v))] == "EXAGO_ESTATE"


# ---- feasibility slacks: host side ----------------------------------------------------------------

def test_slack_pattern_and_validation(L):
    g = synth.grid_30bus()
    net = plan(g)
    bus = np.array([0, 4, 4, 29], np.int32)
    row = np.array([0, 0, 1, 1], np.int32)
    sign = np.array([-1, 1, -1, 1], np.int32)
    s = exago.Slack(net, bus, row, sign, np.array([1.0, 2.0, 3.0, 4.0]))
    rows, vals = s.pattern()
    np.testing.assert_array_equal(rows, row * g.nb + bus)
    np.testing.assert_array_equal(vals, sign)
    x = np.zeros(1)
    rc = L.exago_eval_slack(s.h, ctypes.byref(exago.exago_batch(1)), x.ctypes.data, None, 0, None,
                            None)
    assert exago.STATUS[rc] == "EXAGO_ESTATE"
    s.close()
    for bad in (dict(bus=[30]), dict(bus=[-1]), dict(row=[2]), dict(sign=[0]), dict(cost=[np.inf])):
        kw = dict(bus=[1], row=[0], sign=[1], cost=[1.0])
        kw.update(bad)
        with pytest.raises(exago.ExagoError) as ei:
            exago.Slack(net, kw["bus"], kw["row"], kw["sign"], kw["cost"])
        assert ei.value.name == "EXAGO_EINVAL"


# ---- KKT step: host symbolic analysis ------------------------------------------------------------

@pytest.mark.parametrize("name", ["30bus", "parallel", "300bus", "2000bus"])
def test_kkt_symbolic_is_minimum_degree_with_its_fill(L, name):
    """exago_kkt_create on a plan-only net runs the symbolic analysis alone.  Replaying the
    elimination on the bus graph here: every eliminated bus had the least current degree (lowest
    index on ties), the number of factor blocks is nb plus the fill-inclusive neighbour counts,
    and each column's level exceeds those of its elimination-tree children."""
    g = {"30bus": synth.grid_30bus, "parallel": parallel_grid, "2000bus": synth.grid_2000,
         "300bus": lambda: synth.make_grid(13, 300, 389, 77)}[name]()
    net = plan(g)
    k = exago.exago_kkt_create(net.h)
    try:
        info = exago.exago_kkt_info(k)
        perm, parent, level = exago.exago_kkt_order(k, g.nb)
    finally:
        exago.exago_kkt_destroy(k)
    assert sorted(perm.tolist()) == list(range(g.nb))
    adj = [set() for _ in range(g.nb)]
    for f, t in zip(g.f.tolist(), g.t.tolist()):
        if f != t:
            adj[f].add(t)
            adj[t].add(f)
    alive = set(range(g.nb))
    blocks = 0
    iperm = np.empty(g.nb, np.int64)
    iperm[perm] = np.arange(g.nb)
    for kk, v in enumerate(perm.tolist()):
        dmin = min(len(adj[u]) for u in alive)
        assert len(adj[v]) == dmin and v == min(u for u in alive if len(adj[u]) == dmin)
        N = adj[v]
        blocks += 1 + len(N)
        want_parent = min(iperm[u] for u in N) if N else -1
        assert parent[kk] == want_parent
        for u in N:
            adj[u] |= N
            adj[u].discard(u)
            adj[u].discard(v)
        alive.discard(v)
        adj[v] = set()
    assert info["blocks"] == blocks
    for kk in range(g.nb):
        if parent[kk] >= 0:
            assert level[parent[kk]] > level[kk]
    assert info["levels"] == level.max() + 1


def test_kkt_solve_needs_a_device_net(L):
    net = plan(synth.grid_30bus())
    k = exago.exago_kkt_create(net.h)
    try:
        rc = L.exago_kkt_solve(k, 1, 8, 8, 8, 8, 8, 8, None, None, 0, None)
        assert exago.STATUS[rc] == "EXAGO_ESTATE"
    finally:
        exago.exago_kkt_destroy(k)
