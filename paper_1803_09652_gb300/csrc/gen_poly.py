"""Writes poly_coeffs.h: FP32 polynomials for the far-field HCT integral.

For spheres that do not overlap (r >= a + s) the descreening integral is
    H(r) = (1/(2r)) [x/(1 - x^2) - artanh x],   x = s/r,
whose Taylor series about x = 0 is (1/(2r)) sum_{k>=1} 2k/(2k+1) x^(2k+1).
Writing y = x^2:
    H     =  1/2 * x^3 / r   * g(y),  g(y) = sum_{k>=1} 2k/(2k+1)        y^(k-1)
    dH/dr = -1/2 * x^3 / r^2 * h(y),  h(y) = sum_{k>=1} 4k(k+1)/(2k+1)   y^(k-1)
Both are fitted on [0, Y_MAX] by interpolation at Chebyshev nodes (a
near-minimax fit), reference values from the series summed in FP64 to
convergence, and emitted as monomial coefficients for Horner evaluation.
A second, lower-degree pair (suffix "f") covers only the far field
y <= Y_FAR, where fewer terms reach the same FP32 accuracy.
Run:  python gen_poly.py  (rewrites poly_coeffs.h beside this file).
"""
import os

import numpy as np

Y_MAX = 0.36     # x <= 0.6: every non-overlapping pair of the radius sets used here
Y_FAR = 0.10     # x <= 0.316: pairs more than ~3 screened radii apart


def series(y, coef):
    out = np.zeros_like(y)
    p = np.ones_like(y)
    for k in range(1, 400):
        out += coef(k) * p
        p = p * y
        if np.all(p < 1e-30):
            break
    return out


def g_exact(y):
    return series(y, lambda k: 2.0 * k / (2.0 * k + 1.0))


def h_exact(y):
    return series(y, lambda k: 4.0 * k * (k + 1.0) / (2.0 * k + 1.0))


def fit(f, deg):
    k = np.arange(deg + 1)
    t = np.cos((2 * k + 1) * np.pi / (2 * (deg + 1)))
    y = 0.5 * Y_MAX * (t + 1.0)
    V = np.vander(y, deg + 1, increasing=True)
    # weight rows by 1/f: relative error
    c = np.linalg.solve(V, f(y))
    return c


def horner32(c, y):
    y = y.astype(np.float32)
    acc = np.float32(c[-1])
    for v in c[-2::-1]:
        acc = np.float32(acc * y + np.float32(v))
    return acc


def best_fits(y_max):
    global Y_MAX
    keep = Y_MAX
    Y_MAX = y_max
    ys = np.linspace(0.0, y_max, 20001)
    best = {}
    for name, f in (("g", g_exact), ("h", h_exact)):
        for deg in range(2, 16):
            c = fit(f, deg)
            c32 = c.astype(np.float32)
            err = np.max(np.abs(horner32(c32, ys).astype(np.float64) / f(ys) - 1.0))
            if err < 1.5e-7:
                best[name] = (deg, c32, err)
                break
    Y_MAX = keep
    return best


def emit(fh, name, deg, c, err, y_max):
    fh.write(f"/* {name}(y) on [0, {y_max}], degree {deg}, max relative error in FP32 Horner {err:.2e} */\n")
    expr = f"{float(c[-1]):.9e}f"
    for v in c[-2::-1]:
        expr = f"fmaf({expr}, y, {float(v):.9e}f)"
    fh.write(f"__device__ __forceinline__ float gb_poly_{name}(float y) {{\n    return {expr};\n}}\n")
    # the same polynomial on two values at once (packed FP32x2 FMA)
    expr = f"make_float2({float(c[-1]):.9e}f, {float(c[-1]):.9e}f)"
    for v in c[-2::-1]:
        expr = f"__ffma2_rn({expr}, y, make_float2({float(v):.9e}f, {float(v):.9e}f))"
    fh.write(f"__device__ __forceinline__ float2 gb_poly_{name}2(float2 y) {{\n    return {expr};\n}}\n")


def main():
    full = best_fits(Y_MAX)
    far = best_fits(Y_FAR)
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "poly_coeffs.h"), "w") as fh:
        fh.write("/* Generated by gen_poly.py: far-field HCT polynomials, see that script. */\n")
        fh.write("#pragma once\n")
        fh.write(f"#define GB_POLY_YMAX {Y_MAX:.8f}f\n")
        fh.write(f"#define GB_POLY_YFAR {Y_FAR:.8f}f\n")
        for name, (deg, c, err) in full.items():
            emit(fh, name, deg, c, err, Y_MAX)
        for name, (deg, c, err) in far.items():
            emit(fh, name + "f", deg, c, err, Y_FAR)
    for name, (deg, c, err) in full.items():
        print(name, deg, err)
    for name, (deg, c, err) in far.items():
        print(name + "f", deg, err)


if __name__ == "__main__":
    main()
