"""Seeded synthetic power grids and evaluation states.

The paper measures on the ACTIVSg200 / ACTIVSg2000 synthetic grids with 100 / 3095 contingencies
and 5 load/wind scenarios (Sec. IV, Sec. V-A, Sec. VI-A experiments).  Those files are not
available, so grids of the same sizes are generated here.  This module holds no power-flow
arithmetic: it draws graphs, per-unit branch and generator parameters, and states (x, lambda,
contingency masks, load scales).  Both the CPU oracle and the CUDA path consume its output.

Recipe (one numpy PCG64 stream per seed):
  * topology: random recursive spanning tree (bus k attaches to a uniform earlier bus whose degree
    is below ``max_degree``), then extra edges between uniform bus pairs, both below
    ``max_degree``, without self-loops or duplicate pairs;
  * r ~ U(0.001, 0.05), x ~ U(0.01, 0.3), b ~ U(0, 0.1) p.u.; 10% of branches are transformers
    with tap ~ U(0.95, 1.05), the rest carry tap = 0 (read as 1, the MATPOWER convention);
  * rateA ~ U(1, 5) p.u. (limit data only);
  * generators at distinct uniform buses, c2 ~ U(0.001, 0.01), c1 ~ U(10, 40), c0 = 0;
  * Pd ~ U(0, 1), Qd = 0.3 Pd, Gs = Bs = 0 unless ``shunts=True``;
  * state: Va ~ N(0, 0.1), Vm ~ U(0.95, 1.05), Pg ~ U(0, 2), Qg ~ U(-0.5, 0.5); multipliers
    lambda ~ N(0, 1) on every equality and inequality row;
  * N-1 masks knock out one distinct non-bridge branch each (bridges by Tarjan's algorithm);
    per-contingency x and lambda are the base state plus N(0, 0.02^2) noise;
  * load scenarios scale Pd and Qd of each bus by exp(0.1 Z), Z ~ N(0, 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_MVA = 100.0


@dataclass
class Grid:
    """Bus/branch/generator arrays in per-unit, the layout ``exago_net_create`` takes."""

    nb: int
    Gs: np.ndarray
    Bs: np.ndarray
    Pd: np.ndarray
    Qd: np.ndarray
    f: np.ndarray  # int32 from-bus of each branch
    t: np.ndarray  # int32 to-bus
    r: np.ndarray
    x: np.ndarray
    b: np.ndarray
    tap: np.ndarray  # 0 means 1 (no transformer)
    rateA: np.ndarray
    gbus: np.ndarray  # int32 bus of each generator
    c2: np.ndarray
    c1: np.ndarray
    c0: np.ndarray
    baseMVA: float = BASE_MVA
    meta: dict = field(default_factory=dict)
    shift: np.ndarray | None = None  # per-branch phase shift (rad) of phase-shifting transformers

    @property
    def nl(self) -> int:
        return int(self.f.shape[0])

    @property
    def ng(self) -> int:
        return int(self.gbus.shape[0])

    @property
    def n(self) -> int:
        """Number of variables, x = [Va | Vm | Pg | Qg]."""
        return 2 * self.nb + 2 * self.ng

    @property
    def m(self) -> int:
        """Number of constraint rows, [P balance | Q balance | from flow | to flow]."""
        return 2 * self.nb + 2 * self.nl


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_topology(rng: np.random.Generator, nb: int, nl: int, max_degree: int = 8):
    """Random recursive spanning tree plus (nl - nb + 1) extra distinct edges, degree < max_degree."""
    if nl < nb - 1:
        raise ValueError("a connected grid needs nl >= nb - 1")
    deg = np.zeros(nb, dtype=np.int64)
    f = np.empty(nl, dtype=np.int32)
    t = np.empty(nl, dtype=np.int32)
    seen = set()
    # eligible earlier buses (degree below the cap); swap-remove when a bus fills up
    elig = [0]
    pos = {0: 0}
    k = 0
    for bus in range(1, nb):
        j = elig[int(rng.integers(len(elig)))]
        f[k], t[k] = j, bus
        seen.add((min(j, bus), max(j, bus)))
        k += 1
        for u in (j, bus):
            deg[u] += 1
        if deg[j] >= max_degree:  # degree may not exceed max_degree
            p = pos.pop(j)
            last = elig.pop()
            if last != j:
                elig[p] = last
                pos[last] = p
        if deg[bus] < max_degree:
            pos[bus] = len(elig)
            elig.append(bus)
    tries = 0
    while k < nl:
        tries += 1
        if tries > 100 * nl + 1000:
            raise RuntimeError("could not place extra edges under the degree cap")
        a, c = (int(v) for v in rng.integers(nb, size=2))
        if a == c or deg[a] >= max_degree or deg[c] >= max_degree:
            continue
        key = (min(a, c), max(a, c))
        if key in seen:
            continue
        seen.add(key)
        f[k], t[k] = a, c
        deg[a] += 1
        deg[c] += 1
        k += 1
    return f, t


def bridges(nb: int, f: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Boolean mask of bridge branches (Tarjan's lowlink, iterative DFS)."""
    nl = f.shape[0]
    adj = [[] for _ in range(nb)]
    for l in range(nl):
        adj[int(f[l])].append((int(t[l]), l))
        adj[int(t[l])].append((int(f[l]), l))
    disc = [-1] * nb
    low = [0] * nb
    is_bridge = np.zeros(nl, dtype=bool)
    timer = 0
    for root in range(nb):
        if disc[root] >= 0:
            continue
        disc[root] = low[root] = timer
        timer += 1
        stack = [(root, -1, 0)]  # (vertex, edge used to enter, next adjacency index)
        while stack:
            v, pe, i = stack[-1]
            if i < len(adj[v]):
                stack[-1] = (v, pe, i + 1)
                w, e = adj[v][i]
                if e == pe:
                    continue
                if disc[w] < 0:
                    disc[w] = low[w] = timer
                    timer += 1
                    stack.append((w, e, 0))
                else:
                    low[v] = min(low[v], disc[w])
            else:
                stack.pop()
                if stack:
                    u = stack[-1][0]
                    low[u] = min(low[u], low[v])
                    if low[v] > disc[u]:
                        is_bridge[pe] = True
    return is_bridge


def make_grid(seed: int, nb: int, nl: int, ng: int, *, max_degree: int = 8,
              transformer_frac: float = 0.1, shunts: bool = False,
              shifter_frac: float = 0.0) -> Grid:
    """Synthetic grid with the distributions listed in the module docstring.  With
    shifter_frac > 0, that fraction of branches (drawn after everything else, so the rest of the
    grid is the same as without) become phase-shifting transformers: tap ~ U(0.95, 1.05) and
    phase shift ~ U(-0.5, 0.5) rad (about +-29 degrees)."""
    if ng > nb:
        raise ValueError("generators sit at distinct buses, so ng <= nb")
    rng = _rng(seed)
    f, t = random_topology(rng, nb, nl, max_degree)
    r = rng.uniform(0.001, 0.05, nl)
    x = rng.uniform(0.01, 0.3, nl)
    b = rng.uniform(0.0, 0.1, nl)
    tap = np.zeros(nl)
    ntr = int(round(transformer_frac * nl))
    if ntr:
        idx = rng.choice(nl, size=ntr, replace=False)
        tap[idx] = rng.uniform(0.95, 1.05, ntr)
    rateA = rng.uniform(1.0, 5.0, nl)
    gbus = np.sort(rng.choice(nb, size=ng, replace=False)).astype(np.int32)
    c2 = rng.uniform(0.001, 0.01, ng)
    c1 = rng.uniform(10.0, 40.0, ng)
    c0 = np.zeros(ng)
    Pd = rng.uniform(0.0, 1.0, nb)
    Qd = 0.3 * Pd
    if shunts:
        Gs = rng.uniform(0.0, 0.05, nb)
        Bs = rng.uniform(-0.1, 0.1, nb)
    else:
        Gs = np.zeros(nb)
        Bs = np.zeros(nb)
    shift = None
    nps = int(round(shifter_frac * nl))
    if nps:
        shift = np.zeros(nl)
        idx = rng.choice(nl, size=nps, replace=False)
        tap[idx] = rng.uniform(0.95, 1.05, nps)
        shift[idx] = rng.uniform(-0.5, 0.5, nps)
    return Grid(nb=nb, Gs=Gs, Bs=Bs, Pd=Pd, Qd=Qd, f=f, t=t, r=r, x=x, b=b, tap=tap,
                rateA=rateA, gbus=gbus, c2=c2, c1=c1, c0=c0,
                meta={"seed": seed, "max_degree": max_degree}, shift=shift)


def base_state(rng: np.random.Generator, g: Grid):
    """One (x, lambda) draw: x = [Va | Vm | Pg | Qg], lambda = [lamP | lamQ | muF | muT]."""
    Va = rng.normal(0.0, 0.1, g.nb)
    Vm = rng.uniform(0.95, 1.05, g.nb)
    Pg = rng.uniform(0.0, 2.0, g.ng)
    Qg = rng.uniform(-0.5, 0.5, g.ng)
    x = np.concatenate([Va, Vm, Pg, Qg])
    lam = rng.normal(0.0, 1.0, g.m)
    return x, lam


@dataclass
class Batch:
    """B evaluation states on one grid (host arrays, row-major [B][...])."""

    x: np.ndarray  # [B][n] float64
    lam: np.ndarray  # [B][m] float64
    mask: np.ndarray | None = None  # [B][nl] uint8, 1 = in service
    pd_scale: np.ndarray | None = None  # [B][nb] float64
    obj_weight: np.ndarray | None = None  # [B] float64
    sigma: float = 1.0
    gen_mask: np.ndarray | None = None  # [B][ng] uint8, 1 = in service
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.x.shape[0])


def random_batch(seed: int, g: Grid, B: int, *, masks: bool = False, pd_scale: bool = False,
                 obj_weight: bool = False, sigma: float = 1.0, gen_masks: bool = False) -> Batch:
    """B independent states; optional random 0/1 branch masks, load scales, objective weights and
    0/1 generator masks (about 20% of generators out of service)."""
    rng = _rng(seed)
    xs, ls = zip(*(base_state(rng, g) for _ in range(B))) if B else ((), ())
    x = np.array(xs, dtype=np.float64).reshape(B, g.n)
    lam = np.array(ls, dtype=np.float64).reshape(B, g.m)
    mask = (rng.random((B, g.nl)) > 0.2).astype(np.uint8) if masks else None
    ps = np.exp(0.1 * rng.normal(size=(B, g.nb))) if pd_scale else None
    w = rng.uniform(0.1, 1.0, B) if obj_weight else None
    gm = (rng.random((B, g.ng)) > 0.2).astype(np.uint8) if gen_masks else None
    return Batch(x=x, lam=lam, mask=mask, pd_scale=ps, obj_weight=w, sigma=sigma, gen_mask=gm)


def contingency_batch(seed: int, g: Grid, B: int, sigma_state: float = 0.02) -> Batch:
    """N-1 security batch: B distinct non-bridge outages around one base state."""
    rng = _rng(seed)
    x0, l0 = base_state(rng, g)
    cand = np.flatnonzero(~bridges(g.nb, g.f, g.t))
    if B > cand.shape[0]:
        raise ValueError(f"only {cand.shape[0]} non-bridge branches for {B} contingencies")
    out = np.sort(rng.choice(cand, size=B, replace=False))
    mask = np.ones((B, g.nl), dtype=np.uint8)
    mask[np.arange(B), out] = 0
    x = x0[None, :] + rng.normal(0.0, sigma_state, (B, g.n))
    lam = l0[None, :] + rng.normal(0.0, sigma_state, (B, g.m))
    return Batch(x=x, lam=lam, mask=mask, meta={"outage": out})


def scenario_batch(seed: int, g: Grid, S: int, sigma_load: float = 0.1) -> Batch:
    """Stochastic load batch: S scenarios scaling each bus load by exp(sigma_load Z)."""
    rng = _rng(seed)
    x0, l0 = base_state(rng, g)
    ps = np.exp(sigma_load * rng.normal(size=(S, g.nb)))
    w = np.full(S, 1.0 / S)
    x = np.repeat(x0[None, :], S, axis=0)
    lam = np.repeat(l0[None, :], S, axis=0)
    return Batch(x=x, lam=lam, pd_scale=ps, obj_weight=w)


# ---- the paper-sized workloads ---------------------------------------------------------------

def grid_30bus() -> Grid:
    """30 buses, 41 branches (spanning tree + 12 extra edges), 6 generators, seed 1."""
    return make_grid(1, 30, 41, 6)


def grid_10k() -> Grid:
    """10,000 buses, 13,000 branches, 2,500 generators, seed 2 (ACTIVSg10k-sized)."""
    return make_grid(2, 10_000, 13_000, 2_500)


def grid_2000() -> Grid:
    """2,000 buses, 2,700 branches, 500 generators, seed 3 (ACTIVSg2000-sized)."""
    return make_grid(3, 2_000, 2_700, 500)


def grid_sized(seed: int, nb: int) -> Grid:
    """Serving-mix grid: nl = round(1.3 nb), ng = round(nb / 4)."""
    return make_grid(seed, nb, int(round(1.3 * nb)), int(round(nb / 4)))


def coupling_parents(kind: str, B: int, seed: int = 0, roots: int = 1):
    """Parent index of each state of a coupled batch (-1: none), as the multi-stage problems tie
    their subproblems together: "chain" -- consecutive periods (state t tied to t - 1); "star" --
    contingencies or scenarios tied to state 0, the base case; "forest" -- a random forest with
    `roots` roots (e.g. contingencies of several multi-period cases)."""
    if kind == "chain":
        return np.arange(-1, B - 1, dtype=np.int32)
    if kind == "star":
        p = np.zeros(B, np.int32)
        if B:
            p[0] = -1
        return p
    if kind == "forest":
        rng = _rng(seed)
        order = rng.permutation(B)
        p = np.full(B, -1, np.int32)
        for j in range(min(roots, B), B):
            p[order[j]] = order[rng.integers(0, j)]
        return p
    raise ValueError(kind)


def generator_contingency_batch(seed: int, g: Grid, B: int, sigma_state: float = 0.02) -> Batch:
    """Security batch of generator outages (Sec. V-A: a contingency may be a generator outage, or
    a generator and a line together): state c takes generator c mod ng out of service, and every
    third state also one non-bridge branch; states around one base state as contingency_batch."""
    rng = _rng(seed)
    x0, l0 = base_state(rng, g)
    cand = np.flatnonzero(~bridges(g.nb, g.f, g.t))
    gm = np.ones((B, g.ng), dtype=np.uint8)
    gm[np.arange(B), np.arange(B) % g.ng] = 0
    mask = np.ones((B, g.nl), dtype=np.uint8)
    both = np.arange(0, B, 3)
    mask[both, rng.choice(cand, size=both.shape[0])] = 0
    x = x0[None, :] + rng.normal(0.0, sigma_state, (B, g.n))
    lam = l0[None, :] + rng.normal(0.0, sigma_state, (B, g.m))
    return Batch(x=x, lam=lam, mask=mask, gen_mask=gm)


# Angle differences of the wide-angle batches: both sides of the switch between the kernels'
# polynomial and the library sine and cosine (the double nearest pi/4 and its neighbours), the
# quarter and half turns, and angles beyond a half turn.
_PI4 = float.fromhex("0x1.921fb54442d18p-1")      # the double nearest pi/4
WIDE_ANGLES = np.array([
    np.nextafter(_PI4, 0.0), _PI4, np.nextafter(_PI4, 4.0),
    -np.nextafter(_PI4, 0.0), -_PI4, -np.nextafter(_PI4, 4.0),
    np.pi / 2, -np.pi / 2, np.pi, -np.pi, 3.5, -3.5, 2 * np.pi + 0.3, -7.0, 20.0, -45.25,
    0.78, 0.79, -0.78, -0.79])


def branch_matching(g: Grid) -> np.ndarray:
    """Branches with pairwise distinct end buses (a greedy matching in branch order), so that each
    one's angle difference can be set exactly by the angles of its own two buses."""
    used = np.zeros(g.nb, dtype=bool)
    pick = []
    for l in range(g.nl):
        a, c = int(g.f[l]), int(g.t[l])
        if a != c and not used[a] and not used[c]:
            used[a] = used[c] = True
            pick.append(l)
    return np.array(pick, dtype=np.int64)


def wide_angle_batch(seed: int, g: Grid, B: int, *, masks: bool = False,
                     sigma: float = 1.0) -> Batch:
    """States whose branch angle differences Va_f - Va_t reach far beyond the normal operating
    range.  State 0 and every other even state put each matched branch (branch_matching) on one of
    WIDE_ANGLES exactly, cycling through the list with a per-state offset: Va_t = 0 and
    Va_f = angle, so the subtraction is exact.  Odd states draw every angle from U(-pi, pi)."""
    rng = _rng(seed)
    b = random_batch(seed, g, B, masks=masks, sigma=sigma)
    match = branch_matching(g)
    for s in range(B):
        if s % 2 == 1:
            b.x[s, :g.nb] = rng.uniform(-np.pi, np.pi, g.nb)
            continue
        for j, l in enumerate(match):
            a = WIDE_ANGLES[(j + s // 2) % WIDE_ANGLES.shape[0]]
            b.x[s, g.t[l]] = 0.0
            b.x[s, g.f[l]] = a
    b.meta["matched"] = match
    return b
