"""Coefficients of the branch kernel's sine and cosine for |theta| <= pi/4.

Minimax polynomials by the Remez exchange algorithm (Remez 1934; see e.g. Muller, "Elementary
Functions", ch. 3), computed here in 60-digit arithmetic with mpmath:
  sin x = x + x^3 p(x^2),  p of degree 5, minimising the relative error of sin;
  cos x = 1 + x^2 q(x^2),  q of degree 5, minimising the relative error of cos.
The kernel evaluates both by Horner's rule with fused multiply-adds (14 FP64 instructions for
the pair, z = x^2 shared).  `python -m paper_2203_10587_gb300.sincos_minimax` prints the
coefficients as C hex-float literals; tests/test_sincos_minimax.py checks that the literals in
the kernel source are these and bounds the error of the kernel's evaluation order.
Build-time tool only: nothing in the evaluation path imports it.
"""
import mpmath as mp

X_MAX = mp.pi / 4
DEG = 5          # degree of p and q in z = x^2


def _remez(f, w, a, b, n, iters=40, grid=3000):
    """Minimax polynomial c[0] + c[1] z + ... + c[n] z^n of the weighted error w (f - poly)."""
    N = n + 2
    zs = [(a + b) / 2 - (b - a) / 2 * mp.cos(mp.pi * k / (N - 1)) for k in range(N)]
    c = None
    for _ in range(iters):
        A = mp.matrix(N, N)
        rhs = mp.matrix(N, 1)
        for k, z in enumerate(zs):
            for j in range(n + 1):
                A[k, j] = z ** j
            A[k, n + 1] = (-1) ** k / w(z)
            rhs[k] = f(z)
        sol = mp.lu_solve(A, rhs)
        c = [sol[j] for j in range(n + 1)]

        def err(z):
            return w(z) * (f(z) - mp.polyval(c[::-1], z))
        pts = [a + (b - a) * mp.mpf(i) / grid for i in range(grid + 1)]
        vals = [err(z) for z in pts]
        ext = [pts[0]] + [pts[i] for i in range(1, grid)
                          if (vals[i] - vals[i - 1]) * (vals[i + 1] - vals[i]) <= 0] + [pts[-1]]
        alt = []
        for z in ext:                      # one extremum per sign run, the largest
            e = err(z)
            if alt and mp.sign(e) == mp.sign(err(alt[-1])):
                if abs(e) > abs(err(alt[-1])):
                    alt[-1] = z
            else:
                alt.append(z)
        while len(alt) > N:
            alt.pop(0 if abs(err(alt[0])) < abs(err(alt[-1])) else -1)
        if len(alt) < N:
            break
        zs = alt
    return c


def coefficients():
    """(p, q) as lists of Python floats (degree 0 first), rounded to double."""
    mp.mp.dps = 60
    tiny, z1 = mp.mpf("1e-40"), X_MAX ** 2
    fs = lambda z: (mp.sin(mp.sqrt(z)) / mp.sqrt(z) - 1) / z if z > tiny else mp.mpf(-1) / 6
    fc = lambda z: (mp.cos(mp.sqrt(z)) - 1) / z if z > tiny else mp.mpf(-1) / 2
    # sin: the error of x + x^3 p relative to sin x is about z (fs - p); cos: z (fc - q) / cos x
    p = _remez(fs, lambda z: z, tiny, z1, DEG)
    q = _remez(fc, lambda z: z / mp.cos(mp.sqrt(z)), tiny, z1, DEG)
    return [float(v) for v in p], [float(v) for v in q]


def _fma(a, b, c):
    """a * b + c rounded once to double."""
    mp.mp.dps = 80
    return float(mp.mpf(a) * mp.mpf(b) + mp.mpf(c))


def kernel_sincos(x, p, q):
    """The kernel's evaluation order, in double with single-rounding fma."""
    z = x * x
    u = p[DEG]
    for j in range(DEG - 1, -1, -1):
        u = _fma(u, z, p[j])
    s = _fma(x * z, u, x)
    v = q[DEG]
    for j in range(DEG - 1, -1, -1):
        v = _fma(v, z, q[j])
    c = _fma(v, z, 1.0)
    return s, c


if __name__ == "__main__":
    p, q = coefficients()
    print("p:", ", ".join(v.hex() for v in p))
    print("q:", ", ".join(v.hex() for v in q))
