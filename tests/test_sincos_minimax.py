"""CPU: the branch kernel's sine and cosine polynomials (|theta| <= pi/4).

The literals in the kernel source must be the minimax coefficients that
paper_2203_10587_gb300/sincos_minimax.py derives (Remez exchange), and the kernel's evaluation
order -- Horner's rule with single-rounding fused multiply-adds -- must stay within 0.75 ulp
(sin) and 1.25 ulp (cos) of the exact values, checked against 40-digit mpmath on the interval's
end points and 1,500 seeded points inside it.
"""
import math
import os
import random
import re

import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2203_10587_gb300", "csrc", "eval_items.cuh")


def kernel_literals():
    text = open(SRC).read()
    block = text[text.index("SINCOS_COEFFS_BEGIN"):text.index("SINCOS_COEFFS_END")]
    vals = dict(re.findall(r"\b([pq][0-5]) = (-?0x[0-9a-f.]+p-?\d+)", block))
    p = [float.fromhex(vals[f"p{j}"]) for j in range(6)]
    q = [float.fromhex(vals[f"q{j}"]) for j in range(6)]
    return p, q


def test_kernel_literals_are_the_derived_minimax_coefficients():
    from paper_2203_10587_gb300 import sincos_minimax as sm
    p, q = sm.coefficients()
    kp, kq = kernel_literals()
    assert kp == p and kq == q


def test_kernel_evaluation_error_bound():
    from paper_2203_10587_gb300 import sincos_minimax as sm
    p, q = kernel_literals()
    rng = random.Random(7)
    x_max = float(mp.pi / 4)
    xs = [rng.uniform(-x_max, x_max) for _ in range(1500)] + [x_max, -x_max, 0.5, 1e-8, 2.0 ** -30]
    worst_s = worst_c = 0.0
    for x in xs:
        s, c = sm.kernel_sincos(x, p, q)
        mp.mp.dps = 40
        S, C = mp.sin(x), mp.cos(x)
        worst_s = max(worst_s, float(abs(mp.mpf(s) - S)) / math.ulp(float(S)))
        worst_c = max(worst_c, float(abs(mp.mpf(c) - C)) / math.ulp(float(C)))
    assert worst_s <= 0.75, worst_s
    assert worst_c <= 1.25, worst_c
    assert sm.kernel_sincos(0.0, p, q) == (0.0, 1.0)


def test_switch_point_is_the_double_nearest_pi_over_4():
    """The kernel switches to the library sincos where |theta| exceeds, by bit pattern, the double
    nearest pi/4; the polynomial's bound above holds up to and including that double."""
    import struct
    text = open(SRC).read()
    lit = re.search(r"setp\.le\.u64 p, %1, (0x[0-9A-Fa-f]+);", text).group(1)
    mp.mp.dps = 40
    pi4 = float(mp.pi / 4)
    assert int(lit, 16) == struct.unpack("<Q", struct.pack("<d", pi4))[0]
    # the double nearest pi/4 lies below pi/4, so every double the polynomial takes is inside
    # [-pi/4, pi/4]
    assert mp.mpf(pi4) < mp.pi / 4 < mp.mpf(math.nextafter(pi4, 1.0))


def test_wide_angle_inputs_cross_the_switch_point():
    """The wide-angle GPU parity batches put branches exactly on the switch point, one ulp either
    side (both signs), on the quarter and half turns and beyond, and draw whole grids from
    U(-pi, pi)."""
    import numpy as np
    from paper_2203_10587_gb300 import synth
    g = synth.make_grid(13, 300, 389, 77, transformer_frac=0.3, shunts=True)
    b = synth.wide_angle_batch(5, g, 6, masks=True)
    m = b.meta["matched"]
    th = b.x[0, g.f[m]] - b.x[0, g.t[m]]
    pi4 = float.fromhex("0x1.921fb54442d18p-1")
    for a in (pi4, math.nextafter(pi4, 0.0), math.nextafter(pi4, 4.0), -pi4,
              -math.nextafter(pi4, 4.0), math.pi, -math.pi, math.pi / 2, 20.0, -45.25):
        assert np.any(th == a), a
    allth = b.x[:, g.f] - b.x[:, g.t]
    assert np.mean(np.abs(allth[1::2]) > math.pi / 4) > 0.4
