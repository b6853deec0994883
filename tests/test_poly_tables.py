"""The FP32 polynomial tables of the pair kernels (poly_coeffs.h, written by
csrc/gen_poly.py): the committed header is what the generator writes, each
polynomial reproduces its closed form in FP32 Horner evaluation over its
range, and the restricted-integral form the cutoff kernels build on q(z)
equals the oracle's shell integral (an independent derivation)."""
import importlib.util
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1803_09652_gb300", "csrc")


@pytest.fixture(scope="module")
def gen():
    spec = importlib.util.spec_from_file_location("gen_poly", os.path.join(CSRC, "gen_poly.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def coeffs(name):
    """Coefficients (lowest degree first) of gb_poly_<name> in the header."""
    text = open(os.path.join(CSRC, "poly_coeffs.h")).read()
    body = re.search(r"float gb_poly_%s\(float y\) \{\s*return (.*?);\s*\}" % name, text, re.S).group(1)
    vals = [float(v) for v in re.findall(r"(-?\d\.\d+e[+-]\d+)f", body)]
    return np.array(vals[::-1], dtype=np.float32)       # Horner lists the top coefficient first


def horner32(c, y):
    y = np.asarray(y, dtype=np.float32)
    acc = np.full_like(y, c[-1])
    for v in c[-2::-1]:
        acc = (acc * y + np.float32(v)).astype(np.float32)
    return acc


def test_header_is_what_the_generator_writes(gen, tmp_path):
    out = tmp_path / "poly_coeffs.h"
    gen.main(str(out))
    assert out.read_text() == open(os.path.join(CSRC, "poly_coeffs.h")).read()


@pytest.mark.parametrize("name,ymax", [("g", 0.36), ("gf", 0.10)])
def test_g_reproduces_the_far_field_integral(name, ymax):
    """H = 1/(2r) [x/(1-x^2) - artanh x] = 1/2 x^3/r g(x^2) for disjoint spheres."""
    c = coeffs(name)
    x = np.linspace(1e-2, math.sqrt(ymax), 4001)
    exact = (x / (1 - x * x) - np.arctanh(x)) / x ** 3
    assert np.max(np.abs(horner32(c, x * x) / exact - 1)) < 2e-7


@pytest.mark.parametrize("name,ymax", [("h", 0.36), ("hf", 0.10)])
def test_h_reproduces_the_far_field_derivative(name, ymax):
    """-dH/dr = 1/2 x^3/r^2 h(x^2): finite differences of the closed form in r."""
    c = coeffs(name)
    s = 1.0
    for x in np.linspace(0.05, math.sqrt(ymax) * 0.999, 40):
        r = s / x
        Hf = lambda rr: (s / rr / (1 - (s / rr) ** 2) - np.arctanh(s / rr)) / (2 * rr)
        d = 1e-5 * r
        dH = (Hf(r + d) - Hf(r - d)) / (2 * d)
        assert -dH == pytest.approx(0.5 * x ** 3 / r ** 2 * float(horner32(c, np.float32(x * x))), rel=3e-7)


def test_q_reproduces_the_restricted_shell_integral():
    """z^3 q(z) = -ln(1 - z) - z - z^2/2 on [0, 1/2] (q) and [1/2, 3/4] (q_hi in z - 5/8)."""
    z = np.linspace(1e-3, 0.5, 4001)
    J = -np.log1p(-z) - z - z * z / 2
    assert np.max(np.abs(z ** 3 * horner32(coeffs("q"), z) / J - 1)) < 2e-7
    z = np.linspace(0.5, 0.75, 4001)
    J = -np.log1p(-z) - z - z * z / 2
    assert np.max(np.abs(z ** 3 * horner32(coeffs("q_hi"), (z - 0.625).astype(np.float32)) / J - 1)) < 2e-7


def test_z_form_equals_the_oracle_shell_integral(orc):
    """H = 1/(4r) [(s/L) z^2 - J(z)], z = (U' - L)/U', with its r-derivative,
    against the oracle's antiderivative form for disjoint spheres."""
    rng = np.random.default_rng(11)
    for _ in range(3000):
        s = rng.uniform(0.5, 1.6)
        a = rng.uniform(0.9, 2.0)
        rc = rng.uniform(2.5, 25.0)
        r = rng.uniform(a + s, rc + s + 1.0)
        L = r - s
        wc = (rc - r) + s
        cut = wc < 2 * s
        w = max(0.0, wc if cut else 2 * s)
        U = L + w
        z = w / U
        J = -math.log1p(-z) - z - z * z / 2
        B = s / L * z * z - J
        H = B / (4 * r)
        zp = -1 / U if cut else -z / U
        dB = -s / L ** 2 * z * z + zp * z * (2 * s - w) / L
        dH = (dB - B / r) / (4 * r)
        Ho, dHo = orc.hct_pair_cut(r, a, s, rc), orc.hct_pair_dr_cut(r, a, s, rc)
        assert H == pytest.approx(Ho, rel=1e-7, abs=1e-13)
        assert dH == pytest.approx(dHo, rel=1e-7, abs=1e-13)
