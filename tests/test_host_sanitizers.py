"""CPU: the library's host code and the plain C oracle under the address and undefined-behaviour
sanitizers (compute-sanitizer is closed on this machine, so device-side checks are the EXAGO_DEBUG
build's; the host side is checked here).

tests/sanitize/host_driver.cpp runs the plan's validation and construction (plan.cpp) and the
block factorisation's symbolic analysis (blockfact_sym.cpp) on grid files: valid grids (the 30-bus
grid, parallel branches with shared generator buses, a 300-bus grid with shunts, transformers and
phase shifters, a bus with no branch, a single bus) and invalid ones that must be rejected (a bus
index out of range, a self loop, zero impedance, a non-finite value, a negative tap, a generator
at a missing bus, a non-finite phase shift).  tests/sanitize/oracle_driver.c runs every oracle entry
point on the valid grids.  Both are built with -fsanitize=address,undefined
-fno-sanitize-recover=all, so any report aborts the driver.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2203_10587_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_10587_gb300", "csrc")
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g"]


def cuda_include():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return os.path.join(c, "include")
    pytest.skip("CUDA headers not found")


def write_grid(path, g, expect=0, seed=0):
    b = synth.random_batch(seed, g, 1, masks=True) if expect == 0 else None
    shift = getattr(g, "shift", None)
    with open(path, "w") as fp:
        w = lambda a, fmt="%.17g": fp.write(" ".join(fmt % v for v in np.asarray(a).ravel()) + "\n")
        fp.write(f"{expect} {g.nb} {g.nl} {g.ng} {g.baseMVA!r} {0 if shift is None else 1}\n")
        for a in (g.Gs, g.Bs, g.Pd, g.Qd):
            w(a)
        w(g.f, "%d"), w(g.t, "%d")
        for a in (g.r, g.x, g.b, g.tap, g.rateA):
            w(a)
        w(g.gbus, "%d")
        for a in (g.c2, g.c1, g.c0):
            w(a)
        if shift is not None:
            w(shift)
        if b is None:
            w(np.zeros(g.n)), w(np.zeros(g.m)), w(np.ones(g.nl), "%d")
        else:
            w(b.x[0]), w(b.lam[0]), w(b.mask[0], "%d")


def grids():
    from test_capi_host import parallel_grid
    valid = {
        "30bus": synth.grid_30bus(),
        "parallel": parallel_grid(),
        "300bus_shifters": synth.make_grid(7, 300, 389, 77, transformer_frac=0.2, shunts=True,
                                           shifter_frac=0.2),
    }
    g = synth.make_grid(8, 20, 26, 5, shunts=True)
    valid["isolated_bus"] = synth.Grid(**{**g.__dict__, "nb": g.nb + 1,
                                          "Gs": np.append(g.Gs, 0.1), "Bs": np.append(g.Bs, 0.0),
                                          "Pd": np.append(g.Pd, 0.2), "Qd": np.append(g.Qd, 0.0)})
    valid["single_bus"] = synth.Grid(nb=1, Gs=np.array([0.1]), Bs=np.array([0.2]),
                                     Pd=np.array([0.3]), Qd=np.array([0.1]),
                                     f=np.zeros(0, np.int32), t=np.zeros(0, np.int32),
                                     r=np.zeros(0), x=np.zeros(0), b=np.zeros(0), tap=np.zeros(0),
                                     rateA=np.zeros(0), gbus=np.zeros(1, np.int32),
                                     c2=np.array([0.01]), c1=np.array([10.0]), c0=np.array([0.0]))
    base = synth.make_grid(9, 12, 16, 3)

    def bad(**kw):
        d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.__dict__.items()}
        for k, v in kw.items():
            d[k] = v(d[k]) if callable(v) else v
        return synth.Grid(**d)

    def setv(i, v):
        def f(a):
            a = a.copy()
            a[i] = v
            return a
        return f

    invalid = {
        "bus_out_of_range": bad(t=setv(3, 99)),
        "self_loop": bad(t=lambda t: np.where(np.arange(t.size) == 2, base.f[2], t).astype(np.int32)),
        "zero_impedance": bad(r=setv(1, 0.0), x=setv(1, 0.0)),
        "nan_load": bad(Pd=setv(0, np.nan)),
        "negative_tap": bad(tap=setv(0, -1.0)),
        "gen_bus_missing": bad(gbus=setv(0, 57)),
        "nan_shift": bad(shift=np.where(np.arange(base.nl) == 4, np.nan, 0.1)),
    }
    return valid, invalid


def build_and_run(tmp_path, name, cmd_build, files):
    exe = str(tmp_path / name)
    subprocess.check_call(cmd_build + ["-o", exe])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    p = subprocess.run([exe] + files, capture_output=True, text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    assert "AddressSanitizer" not in p.stderr and "runtime error" not in p.stderr, p.stderr[-4000:]
    return p.stdout


@pytest.fixture(scope="module")
def grid_files(tmp_path_factory):
    if shutil.which("g++") is None or shutil.which("gcc") is None:
        pytest.skip("no host compiler")
    d = tmp_path_factory.mktemp("grids")
    valid, invalid = grids()
    files = []
    for i, (k, g) in enumerate(valid.items()):
        p = str(d / f"valid_{k}.txt")
        write_grid(p, g, 0, seed=i)
        files.append(p)
    for k, g in invalid.items():
        p = str(d / f"invalid_{k}.txt")
        write_grid(p, g, 1)
        files.append(p)
    return files


def test_host_library_under_asan_ubsan(tmp_path, grid_files):
    out = build_and_run(tmp_path, "host_driver",
                        ["g++", "-std=c++17", "-O1", *SAN, "-I", cuda_include(),
                         os.path.join(ROOT, "tests", "sanitize", "host_driver.cpp"),
                         os.path.join(CSRC, "plan.cpp"), os.path.join(CSRC, "blockfact_sym.cpp")],
                        grid_files)
    assert out.count("levels") == 5, out


def test_oracle_under_asan_ubsan(tmp_path, grid_files):
    out = build_and_run(tmp_path, "oracle_driver",
                        ["gcc", "-std=c99", "-O1", "-ffp-contract=off", *SAN,
                         os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c"),
                         os.path.join(ROOT, "oracle", "acopf_oracle.c"), "-lm"],
                        grid_files)
    assert out.count(": ok") == 5, out
