"""Python access to the plain C FP64 oracle (acopf_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline
are the only callers.  Nothing here touches the CUDA library.

The oracle evaluates the polar pi-model AC-OPF of ExaGO (arXiv 2203.10587, Sec. III, eqs. (7)-(10))
for one state at a time; ``evaluate_batch`` loops over instances.  ``coupling`` and
``coupling_jtv`` evaluate the linear coupling (ramp) rows between the states of a batch (eqs. (5)-(6),
(15), (20), (31)) and their transpose product.  ``evaluate(..., cartesian=True)`` evaluates the
power-balance-cartesian formulation that Sec. III names beside the polar one.  J and the lower-triangle
Lagrangian Hessian come back as CSR (int64 row pointers, int32 ascending columns, float64 values).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acopf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        compile_source(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


class _Net(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("nl", ctypes.c_int), ("ng", ctypes.c_int),
                ("Gs", ctypes.c_void_p), ("Bs", ctypes.c_void_p), ("Pd", ctypes.c_void_p),
                ("Qd", ctypes.c_void_p), ("f", ctypes.c_void_p), ("t", ctypes.c_void_p),
                ("r", ctypes.c_void_p), ("x", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("tap", ctypes.c_void_p), ("gbus", ctypes.c_void_p), ("c2", ctypes.c_void_p),
                ("c1", ctypes.c_void_p), ("c0", ctypes.c_void_p), ("baseMVA", ctypes.c_double),
                ("shift", ctypes.c_void_p)]


class _Coo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cap", ctypes.c_int64), ("row", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


def bind_library(path: str):
    """Load one compiled oracle library (the default one, or a test's mutated copy)."""
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.oracle_eval.argtypes = [ctypes.POINTER(_Net), vp, vp, vp, vp, vp, ctypes.c_double,
                                ctypes.c_double, vp, vp, vp, ctypes.POINTER(_Coo),
                                ctypes.POINTER(_Coo)]
    lib.oracle_eval.restype = ctypes.c_int
    lib.oracle_coo_to_csr.argtypes = [ctypes.POINTER(_Coo), ctypes.c_int, vp, vp, vp]
    lib.oracle_coo_to_csr.restype = ctypes.c_int64
    lib.oracle_coo_capacity.argtypes = [ctypes.POINTER(_Net), vp, vp]
    lib.oracle_eval_cart.argtypes = lib.oracle_eval.argtypes
    lib.oracle_eval_cart.restype = ctypes.c_int
    lib.oracle_coo_capacity_cart.argtypes = [ctypes.POINTER(_Net), vp, vp]
    lib.oracle_pi_model.argtypes = [ctypes.c_double] * 4 + [vp]
    lib.oracle_pi_model.restype = ctypes.c_int
    lib.oracle_pi_model_shift.argtypes = [ctypes.c_double] * 5 + [vp]
    lib.oracle_pi_model_shift.restype = ctypes.c_int
    lib.oracle_slack.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp,
                                 ctypes.c_double, vp, vp, vp]
    lib.oracle_slack.restype = ctypes.c_int
    for fn in (lib.oracle_coupling, lib.oracle_coupling_jtv):
        fn.argtypes = [ctypes.c_int] * 4 + [vp, vp, vp]
        fn.restype = ctypes.c_int
    return lib


def compile_source(src: str, out: str) -> str:
    """Compile a C oracle source file with the oracle's flags (used for the default build and for
    the mutation tests' deliberately broken copies)."""
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", src, "-o", out, "-lm"])
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind_library(_LIB)
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


class OracleNet:
    """Holds contiguous copies of a grid's arrays and the C struct pointing at them."""

    def __init__(self, grid):
        self.nb, self.nl, self.ng = int(grid.nb), int(grid.nl), int(grid.ng)
        d = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        i = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        self._keep = dict(Gs=d(grid.Gs), Bs=d(grid.Bs), Pd=d(grid.Pd), Qd=d(grid.Qd),
                          f=i(grid.f), t=i(grid.t), r=d(grid.r), x=d(grid.x), b=d(grid.b),
                          tap=d(grid.tap), gbus=i(grid.gbus), c2=d(grid.c2), c1=d(grid.c1),
                          c0=d(grid.c0))
        shift = getattr(grid, "shift", None)
        self._keep["shift"] = None if shift is None else d(shift)
        k = self._keep
        self.c = _Net(self.nb, self.nl, self.ng, _p(k["Gs"]), _p(k["Bs"]), _p(k["Pd"]),
                      _p(k["Qd"]), _p(k["f"]), _p(k["t"]), _p(k["r"]), _p(k["x"]), _p(k["b"]),
                      _p(k["tap"]), _p(k["gbus"]), _p(k["c2"]), _p(k["c1"]), _p(k["c0"]),
                      float(grid.baseMVA), _p(k["shift"]))
        self.n = 2 * self.nb + 2 * self.ng
        self.m = 2 * self.nb + 2 * self.nl


def pi_model(r: float, x: float, b: float, tap: float, lib=None, shift: float | None = None) -> np.ndarray:
    """[Gff, Bff, Gft, Bft, Gtf, Btf, Gtt, Btt] of one branch (phase shift in rad, or None)."""
    Y = np.zeros(8)
    L = lib or _load()
    rc = (L.oracle_pi_model(r, x, b, tap, _p(Y)) if shift is None
          else L.oracle_pi_model_shift(r, x, b, tap, shift, _p(Y)))
    if rc != 0:
        raise ValueError("zero series impedance")
    return Y


def _csr(lib, coo: _Coo, nrows: int):
    n = coo.n
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    col = np.zeros(max(n, 1), dtype=np.int32)
    val = np.zeros(max(n, 1), dtype=np.float64)
    nnz = lib.oracle_coo_to_csr(ctypes.byref(coo), nrows, _p(rowptr), _p(col), _p(val))
    if nnz < 0:
        raise RuntimeError("oracle_coo_to_csr failed")
    return rowptr, col[:nnz].copy(), val[:nnz].copy()


def evaluate(net: OracleNet, x, lam, mask=None, pd_scale=None, obj_weight: float = 1.0,
             sigma: float = 1.0, want_jac: bool = True, want_hess: bool = True,
             lib=None, cartesian: bool = False, gen_mask=None) -> dict:
    """One evaluation.  Returns f, grad[n], gh[m], and J / H as (rowptr, col, val) CSR.
    cartesian=True evaluates the power-balance-cartesian formulation (oracle_eval_cart): x holds
    [e | f | Pg | Qg] and lam, gh have m + nb entries (the voltage rows last).  gen_mask [ng]
    (1 in service, 0 out) takes generators out of service; None = all in service."""
    lib = lib or _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    m = net.m + net.nb if cartesian else net.m
    if x.shape != (net.n,) or lam.shape != (m,):
        raise ValueError("x / lam shape")
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    gen_mask = None if gen_mask is None else np.ascontiguousarray(gen_mask, dtype=np.uint8)
    pd_scale = None if pd_scale is None else np.ascontiguousarray(pd_scale, dtype=np.float64)
    capJ = ctypes.c_int64()
    capH = ctypes.c_int64()
    (lib.oracle_coo_capacity_cart if cartesian else lib.oracle_coo_capacity)(
        ctypes.byref(net.c), ctypes.addressof(capJ), ctypes.addressof(capH))
    keep = []

    def coo(cap):
        r = np.zeros(cap, dtype=np.int32)
        c = np.zeros(cap, dtype=np.int32)
        v = np.zeros(cap, dtype=np.float64)
        keep.extend([r, c, v])
        return _Coo(0, cap, _p(r), _p(c), _p(v))

    J = coo(capJ.value) if want_jac else None
    H = coo(capH.value) if want_hess else None
    fval = np.zeros(1)
    grad = np.zeros(net.n)
    gh = np.zeros(m)
    rc = (lib.oracle_eval_cart if cartesian else lib.oracle_eval)(
        ctypes.byref(net.c), _p(x), _p(lam), _p(mask), _p(gen_mask), _p(pd_scale),
        float(obj_weight), float(sigma), _p(fval), _p(grad), _p(gh),
        ctypes.byref(J) if J is not None else None, ctypes.byref(H) if H is not None else None)
    if rc != 0:
        raise ValueError(f"oracle_eval failed ({rc})")
    out = {"f": float(fval[0]), "grad": grad, "gh": gh}
    if J is not None:
        out["J"] = _csr(lib, J, m)
    if H is not None:
        out["H"] = _csr(lib, H, net.n)
    return out


def evaluate_batch(net: OracleNet, batch, **kw) -> list[dict]:
    """Loop of single evaluations over the B instances of a synth.Batch."""
    res = []
    for b in range(batch.B):
        res.append(evaluate(net, batch.x[b], batch.lam[b],
                            None if batch.mask is None else batch.mask[b],
                            None if batch.pd_scale is None else batch.pd_scale[b],
                            1.0 if batch.obj_weight is None else float(batch.obj_weight[b]),
                            batch.sigma,
                            gen_mask=None if batch.gen_mask is None else batch.gen_mask[b], **kw))
    return res


def coupling(parent, x, nb: int, ng: int, lib=None) -> np.ndarray:
    """Coupling (ramp) rows r[B][ng] = Pg(x_b) - Pg(x_parent(b)) of the stacked states x [B][n]
    (zero rows for parent -1); see oracle_coupling."""
    lib = lib or _load()
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    B, n = x.shape
    if parent.shape != (B,):
        raise ValueError("parent shape")
    r = np.zeros((B, ng))
    if lib.oracle_coupling(B, n, nb, ng, _p(parent), _p(x), _p(r)) != 0:
        raise ValueError("invalid parent index")
    return r


def coupling_jtv(parent, nu, n: int, nb: int, lib=None) -> np.ndarray:
    """C^T nu in the stacked variable layout [B][n] for multipliers nu [B][ng] of the coupling
    rows; see oracle_coupling_jtv."""
    lib = lib or _load()
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    B, ng = nu.shape
    if parent.shape != (B,):
        raise ValueError("parent shape")
    out = np.zeros((B, n))
    if lib.oracle_coupling_jtv(B, n, nb, ng, _p(parent), _p(nu), _p(out)) != 0:
        raise ValueError("invalid parent index")
    return out


def slack(nb: int, bus, row, sign, cost, z, w: float = 1.0, gh=None, f: float | None = None,
          lib=None):
    """Feasibility slacks (load loss, power imbalance) of one state: returns (gh + the slacks'
    balance terms, f + their cost, grad_z); see oracle_slack.  gh, f default to zero."""
    lib = lib or _load()
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    bus, row, sign = i32(bus), i32(row), i32(sign)
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    nz = bus.shape[0]
    gh = np.zeros(2 * nb) if gh is None else np.array(gh, dtype=np.float64)
    fv = np.array([0.0 if f is None else float(f)])
    grad = np.zeros(nz)
    if lib.oracle_slack(nb, nz, _p(bus), _p(row), _p(sign), _p(cost), _p(z), float(w), _p(gh),
                        _p(fv), _p(grad)) != 0:
        raise ValueError("invalid slack bus, row or sign")
    return gh, float(fv[0]), grad


def csr_to_dense(csr, shape) -> np.ndarray:
    rowptr, col, val = csr
    A = np.zeros(shape)
    for r in range(shape[0]):
        for p in range(rowptr[r], rowptr[r + 1]):
            A[r, col[p]] += val[p]
    return A
