"""Thin ctypes binding of the C ABI in include/exago.h (argument marshalling only).

Function names match the C entry points.  Device buffers are torch CUDA tensors (float64 /
uint8, contiguous); their data pointers are passed through unchanged and every computation
happens in the library's CUDA kernels.  There is no fallback: if the compiled library
(paper_2203_10587_gb300/_build/libexago_gb300.so) is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# EXAGO_LIBRARY selects another build of the library (the EXAGO_DEBUG build in its tests)
LIBPATH = os.environ.get("EXAGO_LIBRARY") or os.path.join(HERE, "_build", "libexago_gb300.so")

_lock = threading.Lock()
_lib = None

STATUS = {0: "EXAGO_OK", 1: "EXAGO_EINVAL", 2: "EXAGO_ENOMEM", 3: "EXAGO_ECUDA",
          4: "EXAGO_ETIMEOUT", 5: "EXAGO_EBUSY", 6: "EXAGO_ESTATE", 7: "EXAGO_EDEVICE"}

# every symbol include/exago.h declares (checked by tests/test_capi_host.py)
EXPORTS = [
    "exago_last_error", "exago_status_name", "exago_net_create", "exago_net_create_shift",
    "exago_net_plan",
    "exago_net_destroy", "exago_net_dims", "exago_net_jac_pattern", "exago_net_hess_pattern",
    "exago_net_ineq_bounds", "exago_net_plan_array", "exago_eval_workspace_size",
    "exago_net_reserve", "exago_eval_obj", "exago_eval_grad", "exago_eval_cons",
    "exago_eval_jac", "exago_eval_hess", "exago_eval_all", "exago_eval_jvp", "exago_eval_jtv",
    "exago_eval_hvp", "exago_eval_all_static",
    "exago_eval_profile", "exago_net_set_config", "exago_net_get_config", "exago_net_autotune",
    "exago_net_check", "exago_serve_create", "exago_serve_register", "exago_serve_submit",
    "exago_serve_set_merge", "exago_serve_poll", "exago_serve_wait", "exago_serve_stats",
    "exago_serve_destroy", "exago_test_fail_allocations", "exago_coupling_create",
    "exago_coupling_destroy", "exago_coupling_dims", "exago_coupling_jac_pattern",
    "exago_eval_coupling", "exago_eval_coupling_jtv", "exago_net_dims_cart",
    "exago_net_jac_pattern_cart", "exago_eval_cart_workspace_size", "exago_eval_cart",
    "exago_eval_cart_jvp", "exago_eval_cart_jtv", "exago_eval_cart_hvp", "exago_slack_create",
    "exago_slack_destroy", "exago_slack_pattern", "exago_eval_slack", "exago_eval_slack_jtv",
    "exago_eval_all_slack",
    "exago_kkt_create", "exago_kkt_destroy", "exago_kkt_info", "exago_kkt_order",
    "exago_kkt_workspace_size", "exago_pf_create", "exago_pf_destroy", "exago_pf_workspace_size",
    "exago_pf_step", "exago_test_debug_bounds", "exago_serve_drive", "exago_serve_register_cart",
    "exago_test_work_list",
    "exago_kkt_solve",
]

SCHED_AUTO, SCHED_KERNELS, SCHED_PERSISTENT, SCHED_PIPELINED = 0, 1, 2, 3
GRAPH_DEFAULT, GRAPH_ON, GRAPH_OFF = 0, 1, 2
STAGE_DEFAULT, STAGE_ON, STAGE_OFF, STAGE_BULK = 0, 1, 2, 3
TILING_DEFAULT, TILING_THREAD, TILING_WARP = 0, 1, 2


class ExagoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class exago_config(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int), ("block", ctypes.c_int),
                ("occupancy", ctypes.c_int), ("stage_records", ctypes.c_int), ("lag", ctypes.c_int),
                ("ring", ctypes.c_int), ("chunk", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("spin_limit", ctypes.c_longlong), ("test_force_timeout", ctypes.c_int),
                ("tile_group", ctypes.c_int), ("tiling", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class exago_batch(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("x", ctypes.c_void_p), ("lambda_", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("pd_scale", ctypes.c_void_p),
                ("obj_weight", ctypes.c_void_p), ("obj_factor", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("gen_mask", ctypes.c_void_p)]


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIBPATH):
                raise RuntimeError(f"{LIBPATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIBPATH)
            vp, i32, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
            net_args = [i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp,
                        vp, ctypes.c_double, ctypes.POINTER(vp)]
            sig = {
                "exago_last_error": ([], ctypes.c_char_p),
                "exago_status_name": ([i32], ctypes.c_char_p),
                "exago_net_create": (net_args, i32),
                "exago_net_create_shift": (net_args[:12] + [vp] + net_args[12:], i32),
                "exago_net_plan": (net_args, i32),
                "exago_net_destroy": ([vp], i32),
                "exago_net_dims": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32), i64p, i64p], i32),
                "exago_net_jac_pattern": ([vp, vp, vp], i32),
                "exago_net_hess_pattern": ([vp, vp, vp], i32),
                "exago_net_ineq_bounds": ([vp, vp, vp], i32),
                "exago_net_plan_array": ([vp, ctypes.c_char_p, vp, ctypes.c_size_t,
                                          ctypes.POINTER(ctypes.c_size_t)], i32),
                "exago_eval_workspace_size": ([vp, i32, ctypes.POINTER(ctypes.c_size_t)], i32),
                "exago_net_reserve": ([vp, i32], i32),
                "exago_eval_obj": ([vp, ctypes.POINTER(exago_batch), vp], i32),
                "exago_eval_grad": ([vp, ctypes.POINTER(exago_batch), vp], i32),
                "exago_eval_cons": ([vp, ctypes.POINTER(exago_batch), vp], i32),
                "exago_eval_jac": ([vp, ctypes.POINTER(exago_batch), vp], i32),
                "exago_eval_hess": ([vp, ctypes.POINTER(exago_batch), vp], i32),
                "exago_eval_all": ([vp, ctypes.POINTER(exago_batch), vp, vp, vp, vp, vp], i32),
                "exago_eval_jvp": ([vp, ctypes.POINTER(exago_batch), vp, vp], i32),
                "exago_eval_jtv": ([vp, ctypes.POINTER(exago_batch), vp, vp], i32),
                "exago_eval_hvp": ([vp, ctypes.POINTER(exago_batch), vp, vp], i32),
                "exago_eval_all_static": ([vp, ctypes.POINTER(exago_batch), vp, vp, vp, vp, vp],
                                          i32),
                "exago_eval_profile": ([vp, ctypes.POINTER(exago_batch), vp, vp, vp, vp, vp, i32,
                                        ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.POINTER(ctypes.c_double)], i32),
                "exago_net_set_config": ([vp, ctypes.POINTER(exago_config)], i32),
                "exago_net_get_config": ([vp, i32, ctypes.POINTER(exago_config)], i32),
                "exago_net_autotune": ([vp, ctypes.POINTER(exago_batch), vp, vp, vp, vp, vp, i32,
                                        ctypes.POINTER(exago_config)], i32),
                "exago_net_check": ([vp, vp], i32),
                "exago_serve_create": ([ctypes.c_size_t, i32, i32, ctypes.POINTER(vp)], i32),
                "exago_serve_register": ([vp, vp, ctypes.POINTER(i32)], i32),
                "exago_serve_register_cart": ([vp, vp, ctypes.POINTER(i32)], i32),
                "exago_test_work_list": ([i32, i32, i32, i32, vp, vp, vp], i32),
                "exago_serve_submit": ([vp, i32, ctypes.POINTER(exago_batch), vp, vp, vp, vp, vp,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)], i32),
                "exago_serve_set_merge": ([vp, i32], i32),
                "exago_test_fail_allocations": ([i32], None),
                "exago_serve_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(i32)], i32),
                "exago_serve_wait": ([vp, ctypes.c_uint64, ctypes.c_double], i32),
                "exago_serve_stats": ([vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_uint64)], i32),
                "exago_serve_destroy": ([vp], i32),
                "exago_net_dims_cart": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32), i64p, i64p], i32),
                "exago_net_jac_pattern_cart": ([vp, vp, vp], i32),
                "exago_eval_cart_workspace_size": ([vp, i32, ctypes.POINTER(ctypes.c_size_t)], i32),
                "exago_eval_cart": ([vp, ctypes.POINTER(exago_batch), vp, vp, vp, vp, vp], i32),
                "exago_eval_cart_jvp": ([vp, ctypes.POINTER(exago_batch), vp, vp], i32),
                "exago_eval_cart_jtv": ([vp, ctypes.POINTER(exago_batch), vp, vp], i32),
                "exago_eval_cart_hvp": ([vp, ctypes.POINTER(exago_batch), vp, vp], i32),
                "exago_slack_create": ([vp, i32, vp, vp, vp, vp, ctypes.POINTER(vp)], i32),
                "exago_slack_destroy": ([vp], i32),
                "exago_slack_pattern": ([vp, vp, vp], i32),
                "exago_eval_slack": ([vp, ctypes.POINTER(exago_batch), vp, vp, ctypes.c_int64, vp,
                                      vp], i32),
                "exago_eval_slack_jtv": ([vp, ctypes.POINTER(exago_batch), vp, ctypes.c_int64, vp],
                                         i32),
                "exago_eval_all_slack": ([vp, ctypes.POINTER(exago_batch), vp, vp, vp, vp, vp, vp,
                                          vp, vp], i32),
                "exago_coupling_create": ([vp, i32, vp, ctypes.POINTER(vp)], i32),
                "exago_coupling_destroy": ([vp], i32),
                "exago_coupling_dims": ([vp, ctypes.POINTER(i32), i64p, i64p], i32),
                "exago_coupling_jac_pattern": ([vp, vp, vp, vp], i32),
                "exago_eval_coupling": ([vp, vp, vp, vp], i32),
                "exago_eval_coupling_jtv": ([vp, vp, vp, ctypes.c_int64, i32, vp], i32),
                "exago_kkt_create": ([vp, ctypes.POINTER(vp)], i32),
                "exago_kkt_destroy": ([vp], i32),
                "exago_kkt_info": ([vp, i64p, i64p, ctypes.POINTER(i32),
                                    ctypes.POINTER(ctypes.c_double)], i32),
                "exago_kkt_order": ([vp, vp, vp, vp], i32),
                "exago_kkt_workspace_size": ([vp, i32, ctypes.POINTER(ctypes.c_size_t)], i32),
                "exago_kkt_solve": ([vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp],
                                    i32),
                "exago_pf_create": ([vp, vp, ctypes.POINTER(vp)], i32),
                "exago_pf_destroy": ([vp], i32),
                "exago_pf_workspace_size": ([vp, i32, ctypes.POINTER(ctypes.c_size_t)], i32),
                "exago_pf_step": ([vp, ctypes.POINTER(exago_batch), vp, vp], i32),
                "exago_test_debug_bounds": ([vp, i32], i32),
                "exago_serve_drive": ([vp, vp, vp, i32, vp, i32, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, vp], i32),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise ExagoError(rc, lib().exago_last_error().decode())


def _np(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return None if a is None else a.ctypes.data


def _dp(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return t.data_ptr()


def _net_call(fn, nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus, c2, c1, c0,
              baseMVA):
    d = lambda a: _np(a, np.float64)
    i = lambda a: _np(a, np.int32)
    keep = [d(Gs), d(Bs), d(Pd), d(Qd), i(f), i(t), d(r), d(x), d(b), d(tap), d(rateA), i(gbus),
            d(c2), d(c1), d(c0)]
    h = ctypes.c_void_p()
    _check(fn(int(nb), *map(_hp, keep[:4]), int(nl), *map(_hp, keep[4:11]), int(ng),
              *map(_hp, keep[11:]), float(baseMVA), ctypes.byref(h)))
    return h


def exago_net_create(nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus, c2, c1, c0,
                     baseMVA):
    """Host numpy arrays in; returns the opaque net handle (on the current CUDA device)."""
    return _net_call(lib().exago_net_create, nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA,
                     ng, gbus, c2, c1, c0, baseMVA)


def exago_net_create_shift(nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, shift, rateA, ng, gbus,
                           c2, c1, c0, baseMVA):
    """exago_net_create with a per-branch phase shift (rad) of phase-shifting transformers."""
    d = lambda a: _np(a, np.float64)
    i = lambda a: _np(a, np.int32)
    keep = [d(Gs), d(Bs), d(Pd), d(Qd), i(f), i(t), d(r), d(x), d(b), d(tap),
            None if shift is None else d(shift), d(rateA), i(gbus), d(c2), d(c1), d(c0)]
    h = ctypes.c_void_p()
    _check(lib().exago_net_create_shift(int(nb), *map(_hp, keep[:4]), int(nl),
                                        *map(_hp, keep[4:12]), int(ng), *map(_hp, keep[12:]),
                                        float(baseMVA), ctypes.byref(h)))
    return h


def exago_net_plan(nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng, gbus, c2, c1, c0,
                   baseMVA):
    """Host-only plan (no GPU needed)."""
    return _net_call(lib().exago_net_plan, nb, Gs, Bs, Pd, Qd, nl, f, t, r, x, b, tap, rateA, ng,
                     gbus, c2, c1, c0, baseMVA)


def exago_net_destroy(h):
    _check(lib().exago_net_destroy(h))


def exago_net_dims(h):
    n, me, mi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nj, nh = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().exago_net_dims(h, ctypes.byref(n), ctypes.byref(me), ctypes.byref(mi),
                                ctypes.byref(nj), ctypes.byref(nh)))
    return n.value, me.value, mi.value, nj.value, nh.value


def exago_net_jac_pattern(h):
    n, me, mi, nj, _ = exago_net_dims(h)
    rowptr = np.zeros(me + mi + 1, np.int64)
    col = np.zeros(max(nj, 1), np.int32)
    _check(lib().exago_net_jac_pattern(h, _hp(rowptr), _hp(col)))
    return rowptr, col[:nj]


def exago_net_hess_pattern(h):
    n, _, _, _, nh = exago_net_dims(h)
    rowptr = np.zeros(n + 1, np.int64)
    col = np.zeros(max(nh, 1), np.int32)
    _check(lib().exago_net_hess_pattern(h, _hp(rowptr), _hp(col)))
    return rowptr, col[:nh]


def exago_net_ineq_bounds(h):
    _, _, mi, _, _ = exago_net_dims(h)
    lo = np.zeros(max(mi, 1))
    hi = np.zeros(max(mi, 1))
    _check(lib().exago_net_ineq_bounds(h, _hp(lo), _hp(hi)))
    return lo[:mi], hi[:mi]


def exago_net_plan_array(h, name: str):
    need = ctypes.c_size_t()
    _check(lib().exago_net_plan_array(h, name.encode(), None, 0, ctypes.byref(need)))
    dt = np.int32
    out = np.zeros(need.value // np.dtype(dt).itemsize, dt)
    _check(lib().exago_net_plan_array(h, name.encode(), _hp(out) if out.size else None,
                                      need.value, ctypes.byref(need)))
    return out


def exago_eval_workspace_size(h, B: int) -> int:
    v = ctypes.c_size_t()
    _check(lib().exago_eval_workspace_size(h, int(B), ctypes.byref(v)))
    return v.value


def exago_net_reserve(h, B: int):
    _check(lib().exago_net_reserve(h, int(B)))


def make_batch(x, lam=None, mask=None, pd_scale=None, obj_weight=None, obj_factor=1.0,
               stream=None, workspace=None, gen_mask=None) -> exago_batch:
    """exago_batch over torch CUDA tensors x [B][n] (float64), lam [B][m], mask [B][nl] (uint8),
    pd_scale [B][nb], obj_weight [B], gen_mask [B][ng] (uint8); stream is a torch.cuda.Stream or
    None (current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    ws_ptr, ws_bytes = (None, 0)
    if workspace is not None:
        ws_ptr, ws_bytes = _dp(workspace), workspace.numel() * workspace.element_size()
    bt = exago_batch(int(x.shape[0]), _dp(x, torch.float64), _dp(lam, torch.float64),
                     _dp(mask, torch.uint8), _dp(pd_scale, torch.float64),
                     _dp(obj_weight, torch.float64), float(obj_factor),
                     ctypes.c_void_p(stream.cuda_stream), ws_ptr, ws_bytes,
                     _dp(gen_mask, torch.uint8))
    # the struct holds raw device pointers: keep the tensors alive as long as the batch
    bt._tensors = (x, lam, mask, pd_scale, obj_weight, workspace, gen_mask)
    return bt


def _out(t):
    import torch
    return _dp(t, torch.float64)


def exago_eval_obj(h, batch: exago_batch, f):
    _check(lib().exago_eval_obj(h, ctypes.byref(batch), _out(f)))


def exago_eval_grad(h, batch: exago_batch, grad):
    _check(lib().exago_eval_grad(h, ctypes.byref(batch), _out(grad)))


def exago_eval_cons(h, batch: exago_batch, gh):
    _check(lib().exago_eval_cons(h, ctypes.byref(batch), _out(gh)))


def exago_eval_jac(h, batch: exago_batch, jval):
    _check(lib().exago_eval_jac(h, ctypes.byref(batch), _out(jval)))


def exago_eval_hess(h, batch: exago_batch, hval):
    _check(lib().exago_eval_hess(h, ctypes.byref(batch), _out(hval)))


def exago_eval_all(h, batch: exago_batch, f=None, grad=None, gh=None, jval=None, hval=None):
    _check(lib().exago_eval_all(h, ctypes.byref(batch), _out(f), _out(grad), _out(gh), _out(jval),
                                _out(hval)))


def exago_eval_jvp(h, batch: exago_batch, u, out):
    """out [B][m] = J u."""
    import torch
    _check(lib().exago_eval_jvp(h, ctypes.byref(batch), _dp(u, torch.float64), _out(out)))


def exago_eval_jtv(h, batch: exago_batch, v, out):
    """out [B][n] = J^T v."""
    import torch
    _check(lib().exago_eval_jtv(h, ctypes.byref(batch), _dp(v, torch.float64), _out(out)))


def exago_eval_hvp(h, batch: exago_batch, u, out):
    """out [B][n] = (Lagrangian Hessian at the batch's lambda and obj_factor) u."""
    import torch
    _check(lib().exago_eval_hvp(h, ctypes.byref(batch), _dp(u, torch.float64), _out(out)))


def exago_eval_all_static(h, batch: exago_batch, f=None, grad=None, gh=None, jval=None,
                          hval=None):
    """exago_eval_all with its scratch in the library's static device array (no allocation)."""
    _check(lib().exago_eval_all_static(h, ctypes.byref(batch), _out(f), _out(grad), _out(gh),
                                       _out(jval), _out(hval)))


def exago_eval_profile(h, batch: exago_batch, f=None, grad=None, gh=None, jval=None, hval=None,
                       reps: int = 10):
    """Mean per-kernel milliseconds of one exago_eval_all: list of (name, ms)."""
    nk = ctypes.c_int()
    names = (ctypes.c_char_p * 16)()
    ms = (ctypes.c_double * 16)()
    _check(lib().exago_eval_profile(h, ctypes.byref(batch), _out(f), _out(grad), _out(gh),
                                    _out(jval), _out(hval), int(reps), ctypes.byref(nk), names, ms))
    return [(names[k].decode(), ms[k]) for k in range(nk.value)]


def exago_net_set_config(h, schedule=0, block=0, occupancy=0, stage_records=0, lag=0, ring=0,
                         chunk=0, use_graph=0, spin_limit=0, test_force_timeout=0, tile_group=0,
                         tiling=0):
    c = exago_config(schedule, block, occupancy, stage_records, lag, ring, chunk, use_graph,
                     spin_limit, test_force_timeout, tile_group, tiling)
    _check(lib().exago_net_set_config(h, ctypes.byref(c)))


def exago_net_get_config(h, B: int) -> dict:
    c = exago_config()
    _check(lib().exago_net_get_config(h, int(B), ctypes.byref(c)))
    return c.as_dict()


def exago_net_autotune(h, batch: exago_batch, f=None, grad=None, gh=None, jval=None, hval=None,
                       reps: int = 5) -> dict:
    c = exago_config()
    _check(lib().exago_net_autotune(h, ctypes.byref(batch), _out(f), _out(grad), _out(gh),
                                    _out(jval), _out(hval), int(reps), ctypes.byref(c)))
    return c.as_dict()


def exago_net_check(h, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().exago_net_check(h, ctypes.c_void_p(stream.cuda_stream)))


def exago_serve_create(device_mem_budget: int, max_slots: int, n_streams: int):
    h = ctypes.c_void_p()
    _check(lib().exago_serve_create(int(device_mem_budget), int(max_slots), int(n_streams),
                                    ctypes.byref(h)))
    return h


def exago_serve_register(s, net_h) -> int:
    i = ctypes.c_int()
    _check(lib().exago_serve_register(s, net_h, ctypes.byref(i)))
    return i.value


def exago_test_work_list(B: int, Tbr: int, Tbu: int, lag: int):
    """The persistent schedule's work list decoded on the host: (kind, state, tile) per ticket."""
    import numpy as np
    n = B * (Tbr + Tbu)
    k, st, tl = (np.zeros(max(n, 1), dtype=np.int32) for _ in range(3))
    _check(lib().exago_test_work_list(int(B), int(Tbr), int(Tbu), int(lag), _hp(k), _hp(st),
                                      _hp(tl)))
    return k[:n], st[:n], tl[:n]


def exago_serve_register_cart(s, net_h) -> int:
    i = ctypes.c_int()
    _check(lib().exago_serve_register_cart(s, net_h, ctypes.byref(i)))
    return i.value


def exago_serve_submit(s, net_id: int, batch: exago_batch, f=None, grad=None, gh=None, jval=None,
                       hval=None, deadline_ms: float = 0.0) -> int:
    t = ctypes.c_uint64()
    _check(lib().exago_serve_submit(s, int(net_id), ctypes.byref(batch), _out(f), _out(grad),
                                    _out(gh), _out(jval), _out(hval), float(deadline_ms),
                                    ctypes.byref(t)))
    return t.value


def exago_test_debug_bounds(h, slots: int):
    _check(lib().exago_test_debug_bounds(h, int(slots)))


class exago_serve_client(ctypes.Structure):
    _fields_ = [("net_id", ctypes.c_int), ("batch", ctypes.POINTER(exago_batch)),
                ("f", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("gh", ctypes.c_void_p),
                ("jval", ctypes.c_void_p), ("hval", ctypes.c_void_p)]


def exago_serve_drive(s, clients, group, weight, rate: float, seconds: float, seed: int = 0) -> dict:
    """Native load generator (exago_serve_drive).  clients: list of (net_id, exago_batch, outputs
    dict of CUDA tensors or None); group: list of group ids; weight: per-group arrival share.
    rate <= 0: closed loop.  Returns completed, seconds, p50_ms, p99_ms, deferred."""
    n = len(clients)
    arr = (exago_serve_client * n)()
    keep = []
    for i, (nid, bt, out) in enumerate(clients):
        keep.append(bt)
        arr[i].net_id = int(nid)
        arr[i].batch = ctypes.pointer(bt)
        for k in ("f", "grad", "gh", "jval", "hval"):
            t = out.get(k)
            setattr(arr[i], k, None if t is None else t.data_ptr())
    g = np.ascontiguousarray(group, dtype=np.int32)
    w = np.ascontiguousarray(weight, dtype=np.float64)
    res = np.zeros(5)
    _check(lib().exago_serve_drive(s, arr, _hp(g), n, _hp(w), int(w.shape[0]), float(rate),
                                   float(seconds), int(seed), _hp(res)))
    return {"completed": int(res[0]), "seconds": float(res[1]), "p50_ms": float(res[2]),
            "p99_ms": float(res[3]), "deferred": int(res[4])}


def exago_test_fail_allocations(n: int):
    lib().exago_test_fail_allocations(int(n))


def exago_serve_set_merge(s, max_states: int):
    _check(lib().exago_serve_set_merge(s, int(max_states)))


def exago_serve_poll(s, ticket: int) -> bool:
    d = ctypes.c_int()
    _check(lib().exago_serve_poll(s, ctypes.c_uint64(ticket), ctypes.byref(d)))
    return bool(d.value)


def exago_serve_wait(s, ticket: int, timeout_ms: float = 0.0):
    _check(lib().exago_serve_wait(s, ctypes.c_uint64(ticket), float(timeout_ms)))


def exago_serve_stats(s):
    p50, p99, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
    _check(lib().exago_serve_stats(s, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n)))
    return p50.value, p99.value, n.value


def exago_serve_destroy(s):
    _check(lib().exago_serve_destroy(s))


def exago_net_dims_cart(h):
    """(n, m_eq, m_ineq, nnzJ, nnzH) of the power-balance-cartesian formulation."""
    n, me, mi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nj, nh = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().exago_net_dims_cart(h, ctypes.byref(n), ctypes.byref(me), ctypes.byref(mi),
                                     ctypes.byref(nj), ctypes.byref(nh)))
    return n.value, me.value, mi.value, nj.value, nh.value


def exago_net_jac_pattern_cart(h):
    n, me, mi, nj, _ = exago_net_dims_cart(h)
    rowptr = np.zeros(me + mi + 1, np.int64)
    col = np.zeros(max(nj, 1), np.int32)
    _check(lib().exago_net_jac_pattern_cart(h, _hp(rowptr), _hp(col)))
    return rowptr, col[:nj]


def exago_eval_cart_workspace_size(h, B: int) -> int:
    v = ctypes.c_size_t()
    _check(lib().exago_eval_cart_workspace_size(h, int(B), ctypes.byref(v)))
    return v.value


def exago_eval_cart(h, batch: exago_batch, f=None, grad=None, gh=None, jval=None, hval=None):
    """The power-balance-cartesian evaluation: x = [e | f | Pg | Qg], lambda and gh of m + nb."""
    _check(lib().exago_eval_cart(h, ctypes.byref(batch), _out(f), _out(grad), _out(gh),
                                 _out(jval), _out(hval)))


def exago_eval_cart_jvp(h, batch: exago_batch, u, out):
    """out [B][m + nb] = J u of the cartesian constraint map."""
    import torch
    _check(lib().exago_eval_cart_jvp(h, ctypes.byref(batch), _dp(u, torch.float64), _out(out)))


def exago_eval_cart_jtv(h, batch: exago_batch, v, out):
    """out [B][n] = J^T v of the cartesian constraint map (v [B][m + nb])."""
    import torch
    _check(lib().exago_eval_cart_jtv(h, ctypes.byref(batch), _dp(v, torch.float64), _out(out)))


def exago_eval_cart_hvp(h, batch: exago_batch, u, out):
    """out [B][n] = (cartesian Lagrangian Hessian at the batch's lambda and obj_factor) u."""
    import torch
    _check(lib().exago_eval_cart_hvp(h, ctypes.byref(batch), _dp(u, torch.float64), _out(out)))


class Slack:
    """Owns a set of feasibility slacks (load loss, power imbalance) of a net: host arrays bus,
    row (0 = P balance, 1 = Q balance), sign (+1 / -1) and cost, all [nz]."""

    def __init__(self, net: Net, bus, row, sign, cost):
        i = lambda a: _np(a, np.int32)
        keep = [i(bus), i(row), i(sign), _np(cost, np.float64)]
        self.nz = int(keep[0].shape[0])
        h = ctypes.c_void_p()
        _check(lib().exago_slack_create(net.h, self.nz, *map(_hp, keep), ctypes.byref(h)))
        self.h = h
        self.nb = net.nb

    def pattern(self):
        rows = np.zeros(max(self.nz, 1), np.int64)
        vals = np.zeros(max(self.nz, 1), np.float64)
        _check(lib().exago_slack_pattern(self.h, _hp(rows), _hp(vals)))
        return rows[:self.nz], vals[:self.nz]

    def close(self):
        if self.h is not None and self.h.value:
            lib().exago_slack_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exago_eval_slack(slack: Slack, batch: exago_batch, z, gh=None, ldgh: int = 0, f=None,
                     grad_z=None):
    """Adds the slacks' balance terms to gh [B][ldgh] and their cost to f [B]; writes grad_z."""
    import torch
    _check(lib().exago_eval_slack(slack.h, ctypes.byref(batch), _dp(z, torch.float64), _out(gh),
                                  int(ldgh), _out(f), _out(grad_z)))


def exago_eval_all_slack(net_h, batch: exago_batch, slack: Slack, z, f=None, grad=None, gh=None,
                         jval=None, hval=None, grad_z=None):
    """exago_eval_all and exago_eval_slack in one call (one launch when the fused variant
    applies)."""
    import torch
    _check(lib().exago_eval_all_slack(net_h, ctypes.byref(batch), slack.h, _dp(z, torch.float64),
                                      _out(f), _out(grad), _out(gh), _out(jval), _out(hval),
                                      _out(grad_z)))


def exago_eval_slack_jtv(slack: Slack, batch: exago_batch, v, ldv: int, out):
    """out [B][nz] = sign_k v[b][row_k] (the slack columns of J^T v)."""
    import torch
    _check(lib().exago_eval_slack_jtv(slack.h, ctypes.byref(batch), _dp(v, torch.float64),
                                      int(ldv), _out(out)))


def exago_coupling_create(net_h, parent):
    """Coupling rows of a batch whose state b is tied to state parent[b] (-1: none); host array."""
    parent = _np(parent, np.int32)
    h = ctypes.c_void_p()
    _check(lib().exago_coupling_create(net_h, int(parent.shape[0]), _hp(parent), ctypes.byref(h)))
    return h


def exago_coupling_destroy(h):
    _check(lib().exago_coupling_destroy(h))


def exago_coupling_dims(h):
    B, rows, nnz = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().exago_coupling_dims(h, ctypes.byref(B), ctypes.byref(rows), ctypes.byref(nnz)))
    return B.value, rows.value, nnz.value


def exago_coupling_jac_pattern(h):
    """(rowptr, col, val) of the coupling rows' Jacobian over the stacked variables of all states."""
    _, rows, nnz = exago_coupling_dims(h)
    rowptr = np.zeros(rows + 1, np.int64)
    col = np.zeros(max(nnz, 1), np.int64)
    val = np.zeros(max(nnz, 1), np.float64)
    _check(lib().exago_coupling_jac_pattern(h, _hp(rowptr), _hp(col), _hp(val)))
    return rowptr, col[:nnz], val[:nnz]


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def exago_eval_coupling(h, x, r, stream=None):
    """r [B][ng] = Pg(x_b) - Pg(x_parent(b)) for x [B][n] (CUDA float64 tensors)."""
    import torch
    _check(lib().exago_eval_coupling(h, _dp(x, torch.float64), _out(r), _stream_ptr(stream)))


def exago_eval_coupling_jtv(h, nu, out, ldo: int, accumulate: bool = False, stream=None):
    """out[b * ldo + k] (+)= (C^T nu) at (state b, Pg_k); out is a CUDA float64 tensor or a raw
    device address (an int), e.g. grad.data_ptr() + 16 * nb to add into a [B][n] gradient."""
    import torch
    optr = out if isinstance(out, int) else _out(out)
    _check(lib().exago_eval_coupling_jtv(h, _dp(nu, torch.float64), optr, int(ldo),
                                         1 if accumulate else 0, _stream_ptr(stream)))


# ---- interior-point KKT step ------------------------------------------------------------------

def exago_kkt_create(net_h):
    h = ctypes.c_void_p()
    _check(lib().exago_kkt_create(net_h, ctypes.byref(h)))
    return h


def exago_kkt_destroy(h):
    _check(lib().exago_kkt_destroy(h))


def exago_kkt_info(h) -> dict:
    blocks, pairs = ctypes.c_int64(), ctypes.c_int64()
    levels, flops = ctypes.c_int(), ctypes.c_double()
    _check(lib().exago_kkt_info(h, ctypes.byref(blocks), ctypes.byref(pairs), ctypes.byref(levels),
                                ctypes.byref(flops)))
    return {"blocks": blocks.value, "pairs": pairs.value, "levels": levels.value,
            "flops": flops.value}


def exago_kkt_order(h, nb: int):
    """(perm, parent, level) of the KKT factorisation's elimination order (numpy int32 [nb])."""
    perm, parent, level = (np.zeros(nb, np.int32) for _ in range(3))
    _check(lib().exago_kkt_order(h, _hp(perm), _hp(parent), _hp(level)))
    return perm, parent, level


def exago_kkt_workspace_size(h, B: int) -> int:
    v = ctypes.c_size_t()
    _check(lib().exago_kkt_workspace_size(h, int(B), ctypes.byref(v)))
    return v.value


def exago_kkt_solve(h, jval, hval, dx, dc, rhs, sol, inertia=None, workspace=None, stream=None):
    """sol [B][n + m] = K^{-1} rhs per state (CUDA float64 tensors, row-major per state);
    inertia: CUDA int32 [B][2] or None."""
    import torch
    B = int(jval.shape[0])
    ws, wb = (None, 0) if workspace is None else (_dp(workspace), workspace.numel() * workspace.element_size())
    _check(lib().exago_kkt_solve(h, B, _dp(jval, torch.float64), _dp(hval, torch.float64),
                                 _dp(dx, torch.float64), _dp(dc, torch.float64),
                                 _dp(rhs, torch.float64), _out(sol),
                                 None if inertia is None else _dp(inertia, torch.int32), ws, wb,
                                 _stream_ptr(stream)))


# ---- power-flow Newton step ---------------------------------------------------------------------

def exago_pf_create(net_h, bus_type):
    bt = _np(bus_type, np.int32)
    h = ctypes.c_void_p()
    _check(lib().exago_pf_create(net_h, _hp(bt), ctypes.byref(h)))
    return h


def exago_pf_destroy(h):
    _check(lib().exago_pf_destroy(h))


def exago_pf_workspace_size(h, B: int) -> int:
    v = ctypes.c_size_t()
    _check(lib().exago_pf_workspace_size(h, int(B), ctypes.byref(v)))
    return v.value


def exago_pf_step(h, batch: exago_batch, x_new, mismatch=None):
    """x_new [B][n] = x + d (one Newton step per state); mismatch [B] = max |g_pf(x)|."""
    _check(lib().exago_pf_step(h, ctypes.byref(batch), _out(x_new),
                               None if mismatch is None else _out(mismatch)))


# ---- convenience ------------------------------------------------------------------------------

def _grid_args(grid):
    return (grid.nb, grid.Gs, grid.Bs, grid.Pd, grid.Qd, grid.nl, grid.f, grid.t, grid.r, grid.x,
            grid.b, grid.tap, grid.rateA, grid.ng, grid.gbus, grid.c2, grid.c1, grid.c0,
            grid.baseMVA)


class Net:
    """Owns a net handle built from a synth.Grid-like object (nb, Gs, ..., baseMVA)."""

    def __init__(self, grid, plan_only: bool = False):
        shift = getattr(grid, "shift", None)
        if shift is not None and not plan_only:   # phase-shifting transformers
            a = _grid_args(grid)
            self.h = exago_net_create_shift(*a[:12], shift, *a[12:])
        else:
            self.h = (exago_net_plan if plan_only else exago_net_create)(*_grid_args(grid))
        self.n, self.m_eq, self.m_ineq, self.nnzJ, self.nnzH = exago_net_dims(self.h)
        self.m = self.m_eq + self.m_ineq
        self.nb, self.nl, self.ng = grid.nb, grid.nl, grid.ng

    def close(self):
        if self.h is not None and self.h.value:
            exago_net_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, B: int, device="cuda", f=True, grad=True, gh=True, jac=True, hess=True):
        import torch
        z = lambda *s: torch.empty(*s, dtype=torch.float64, device=device)
        return {"f": z(B) if f else None, "grad": z(B, self.n) if grad else None,
                "gh": z(B, self.m) if gh else None, "jval": z(B, self.nnzJ) if jac else None,
                "hval": z(B, self.nnzH) if hess else None}

    def eval_all(self, batch: exago_batch, out: dict):
        exago_eval_all(self.h, batch, out.get("f"), out.get("grad"), out.get("gh"),
                       out.get("jval"), out.get("hval"))
        return out


class Coupling:
    """Owns the coupling rows of a batch of B states of a net, state b tied to parent[b] (-1:
    none): r = Pg(x_b) - Pg(x_parent(b)) and its transpose product (exago_coupling_*)."""

    def __init__(self, net: Net, parent):
        self.h = exago_coupling_create(net.h, parent)
        self.B, self.rows, self.nnz = exago_coupling_dims(self.h)
        self.nb, self.ng, self.n = net.nb, net.ng, net.n

    def close(self):
        if self.h is not None and self.h.value:
            exago_coupling_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
