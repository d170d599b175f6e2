"""Derive the float polynomials used for sin(u)/u on the wrapped interval [-pi, pi].

sin(u)/u = f(v) with v = u^2 is entire in v, so a low-degree polynomial in v is accurate on
v in [0, V], V = (pi + 0.01)^2 (the margin covers the rounding of the float wrap).  The
coefficients are the discrete minimax (Remez exchange) fit of degree 5 to f on a dense grid,
printed as float literals for k_data.cu.  Degree 5 leaves a truncation error of 6.4e-8 and,
evaluated by float Horner, 2.3e-7 (degree 6: 7.7e-10 and 8.9e-8), at the level of float
rounding of the sinc weights, for one multiply-add less per term.

The second fit is the same function of the angle in turns, x = u / (2 pi) in [-1/2, 1/2]
(v = x^2 in [0, 1/4], no margin: the fixed-point wrap is exact), for the FP32 literal
curvature path, whose angles are fixed-point turns.  Run:  python sinc_poly.py
"""
import numpy as np


def f(v):
    u = np.sqrt(v)
    out = np.ones_like(v)
    nz = u > 0
    out[nz] = np.sin(u[nz]) / u[nz]
    return out


def f_turns(v):
    return f((2.0 * np.pi) ** 2 * v)


def remez(deg, V, n=20001, iters=40, func=f):
    x = np.linspace(0.0, V, n)
    y = func(x)
    # start from Chebyshev extrema
    k = np.arange(deg + 2)
    ref = np.sort(0.5 * V * (1 - np.cos(np.pi * k / (deg + 1))))
    idx = np.searchsorted(x, ref).clip(0, n - 1)
    for _ in range(iters):
        xr = x[idx]
        A = np.vander(xr, deg + 1, increasing=True)
        A = np.hstack([A, ((-1.0) ** np.arange(deg + 2))[:, None]])
        sol = np.linalg.solve(A, y[idx])
        c = sol[:-1]
        err = np.polynomial.polynomial.polyval(x, c) - y
        # new reference: alternating extrema of the error
        s = np.sign(err)
        bounds = np.flatnonzero(np.diff(s) != 0) + 1
        segs = np.split(np.arange(n), bounds)
        ext = [sg[np.argmax(np.abs(err[sg]))] for sg in segs if len(sg)]
        while len(ext) > deg + 2:
            a = np.abs(err[ext])
            i = int(np.argmin(a))
            ext.pop(i)
        if len(ext) < deg + 2:
            break
        idx = np.array(ext)
    return c, np.max(np.abs(err))


def report(name, V, func):
    c, e = remez(5, V, func=func)
    c32 = c.astype(np.float32)
    x = np.linspace(0, V, 200001)
    p = np.zeros_like(x, dtype=np.float32)
    xs = x.astype(np.float32)
    for ck in c32[::-1]:  # Horner in float with fused multiply-add rounding emulated by float64 then rounding
        p = (p.astype(np.float64) * xs + ck).astype(np.float32)
    print(name)
    print("  max |poly - sinc| (float64 coefficients):", e)
    print("  max |poly - sinc| (float32 Horner):", np.max(np.abs(p.astype(np.float64) - func(x))))
    for k, ck in enumerate(c32):
        print(f"  c{k} = {float(ck)!r}f")


if __name__ == "__main__":
    report("v = u^2, u in radians", (np.pi + 0.01) ** 2, f)
    report("v = x^2, x in turns", 0.25, f_turns)
