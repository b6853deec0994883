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

With a Born-radius cutoff the integral of disjoint spheres is restricted to
shells t in [L, U'] (L = r - s, U' = min(r + s, rc)).  With z = (U' - L)/U'
it takes the form 1/(4r) [(s/L) z^2 - J(z)], where
    J(z) = int_0^z t^2/(1 - t) dt = -ln(1 - z) - z - z^2/2 = z^3 q(z),
    q(z) = sum_{k>=0} z^k / (k + 3),
a series of positive terms; q is fitted the same way on [0, Z_J] and, in
the shifted variable z - (Z_J + Z_J2)/2, on [Z_J, Z_J2].
Run:  python gen_poly.py  (rewrites poly_coeffs.h beside this file).
"""
import os

import numpy as np

Y_MAX = 0.36     # x <= 0.6: every non-overlapping pair of the radius sets used here
Y_FAR = 0.10     # x <= 0.316: pairs more than ~3 screened radii apart
Z_J = 0.50       # z <= 1/2: restricted shells no wider than their inner radius
Z_J2 = 0.75      # z <= 3/4: every pair of disjoint spheres of the radius sets used here


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


def q_exact(z):
    return series(z, lambda k: 1.0 / (k + 2.0))


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


def emit(fh, name, deg, c, err, y_max, y_min=0.0):
    fh.write(f"/* {name}(y) on [{y_min:g}, {y_max:g}], degree {deg}, max relative error in FP32 Horner {err:.2e} */\n")
    expr = f"{float(c[-1]):.9e}f"
    for v in c[-2::-1]:
        expr = f"fmaf({expr}, y, {float(v):.9e}f)"
    fh.write(f"__device__ __forceinline__ float gb_poly_{name}(float y) {{\n    return {expr};\n}}\n")
    # the same polynomial on two values at once (packed FP32x2 FMA)
    expr = f"make_float2({float(c[-1]):.9e}f, {float(c[-1]):.9e}f)"
    for v in c[-2::-1]:
        expr = f"__ffma2_rn({expr}, y, make_float2({float(v):.9e}f, {float(v):.9e}f))"
    fh.write(f"__device__ __forceinline__ float2 gb_poly_{name}2(float2 y) {{\n    return {expr};\n}}\n")


def q_fit():
    zs = np.linspace(0.0, Z_J, 20001)
    for deg in range(2, 20):
        k = np.arange(deg + 1)
        t = np.cos((2 * k + 1) * np.pi / (2 * (deg + 1)))
        z = 0.5 * Z_J * (t + 1.0)
        c = np.linalg.solve(np.vander(z, deg + 1, increasing=True), q_exact(z)).astype(np.float32)
        err = np.max(np.abs(horner32(c, zs).astype(np.float64) / q_exact(zs) - 1.0))
        if err < 1.5e-7:
            return deg, c, err
    raise RuntimeError("no fit")


def q2_fit():
    z0 = 0.5 * (Z_J + Z_J2)
    zs = np.linspace(Z_J, Z_J2, 20001)
    for deg in range(2, 20):
        k = np.arange(deg + 1)
        t = np.cos((2 * k + 1) * np.pi / (2 * (deg + 1)))
        z = z0 + 0.5 * (Z_J2 - Z_J) * t
        c = np.linalg.solve(np.vander(z - z0, deg + 1, increasing=True), q_exact(z)).astype(np.float32)
        err = np.max(np.abs(horner32(c, (zs - z0).astype(np.float32)).astype(np.float64) / q_exact(zs) - 1.0))
        if err < 1.5e-7:
            return deg, c, err, z0
    raise RuntimeError("no fit")


def main(out=None):
    full = best_fits(Y_MAX)
    far = best_fits(Y_FAR)
    qdeg, qc, qerr = q_fit()
    q2deg, q2c, q2err, z0 = q2_fit()
    here = os.path.dirname(os.path.abspath(__file__))
    with open(out or os.path.join(here, "poly_coeffs.h"), "w") as fh:
        fh.write("/* Generated by gen_poly.py: far-field HCT polynomials, see that script. */\n")
        fh.write("#pragma once\n")
        fh.write(f"#define GB_POLY_YMAX {Y_MAX:.8f}f\n")
        fh.write(f"#define GB_POLY_YFAR {Y_FAR:.8f}f\n")
        for name, (deg, c, err) in full.items():
            emit(fh, name, deg, c, err, Y_MAX)
        for name, (deg, c, err) in far.items():
            emit(fh, name + "f", deg, c, err, Y_FAR)
        fh.write(f"#define GB_POLY_ZJ {Z_J:.8f}f\n")
        emit(fh, "q", qdeg, qc, qerr, Z_J)
        fh.write(f"#define GB_POLY_ZJ2 {Z_J2:.8f}f\n#define GB_POLY_ZMID {z0:.8f}f\n")
        fh.write(f"/* q(z) on [{Z_J}, {Z_J2}] as a polynomial in y = z - {z0}: */\n")
        emit(fh, "q_hi", q2deg, q2c, q2err, Z_J2 - z0, Z_J - z0)
    print("q", qdeg, qerr)
    print("q_hi", q2deg, q2err)
    for name, (deg, c, err) in full.items():
        print(name, deg, err)
    for name, (deg, c, err) in far.items():
        print(name + "f", deg, err)


if __name__ == "__main__":
    main()
