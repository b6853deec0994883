"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

GB model (Sec. III.D, OBC "igb=2"): the HCT pair integral against direct 2-D
quadrature of its defining volume integral, against the exact large-distance
series, isolated-ion Born energy, distant-ion limit, GB function limits,
central finite differences of forces and charge derivatives, Euler's relation
for a quadratic form, zero net force/torque and rigid-motion invariance.
"""
import decimal
import math

import numpy as np
import pytest
from scipy import integrate

import synth

KE = 332.0522173
TAU = 1.0 - 1.0 / 78.5


# --- HCT descreening integral ------------------------------------------------

def hct_by_quadrature(r, a, s):
    """(1/4pi) * integral over the ball (centre x_j, radius s) of |y - x_i|^-4,
    restricted to |y - x_i| > a, with |x_i - x_j| = r.  Spherical coordinates
    about x_j, polar axis towards x_i; the azimuth gives 2 pi."""
    def inner(u):
        # |y - x_i|^2 = u^2 + r^2 - 2 u r c ; keep points with |y - x_i| > a
        if u == 0.0:
            return 2.0 / r ** 4 if r > a else 0.0
        c0 = (u * u + r * r - a * a) / (2.0 * u * r)
        hi = min(1.0, c0)
        if hi <= -1.0:
            return 0.0
        val, _ = integrate.quad(lambda c: (u * u + r * r - 2 * u * r * c) ** -2, -1.0, hi,
                                epsabs=0, epsrel=1e-12, limit=200)
        return val

    pts = [p for p in (abs(r - a), r + a, r) if 0 < p < s]
    val, _ = integrate.quad(lambda u: 0.5 * u * u * inner(u), 0.0, s, points=pts or None,
                            epsabs=0, epsrel=1e-11, limit=400)
    return val


@pytest.mark.parametrize("r,a,s,regime", [
    (4.0, 1.5, 1.2, "disjoint"),
    (2.0, 1.5, 1.2, "partial overlap, L = a"),
    (1.0, 1.1, 1.5, "centre of i inside j, not engulfed"),
    (0.3, 0.8, 1.5, "i engulfed by j"),
    (0.5, 0.6, 1.6, "i engulfed, larger j"),
    (2.6, 1.11, 1.528, "closest non-bonded distances"),
    (12.0, 1.71, 1.2, "far"),
])
def test_hct_pair_matches_quadrature(orc, r, a, s, regime):
    ref = hct_by_quadrature(r, a, s)
    got = orc.hct_pair(r, a, s)
    assert abs(got - ref) <= 1e-9 * max(abs(ref), 1e-12), (regime, got, ref)


def test_hct_pair_zero_when_j_inside_i(orc):
    assert orc.hct_pair(0.2, 1.5, 1.0) == 0.0
    assert hct_by_quadrature(0.2, 1.5, 1.0) == pytest.approx(0.0, abs=1e-14)


def _series_decimal(r, s, terms=400):
    """(1/(2r)) * sum_{k>=1} 2k/(2k+1) x^(2k+1), x = s/r, in 50-digit decimal:
    the expansion of the disjoint-sphere integral about x = 0."""
    decimal.getcontext().prec = 50
    D = decimal.Decimal
    x = D(s) / D(r)
    acc = D(0)
    xp = x ** 3
    for k in range(1, terms):
        acc += D(2 * k) / D(2 * k + 1) * xp
        xp *= x * x
        if xp < D(10) ** -45:
            break
    return acc / (2 * D(r))


@pytest.mark.parametrize("r", [5.0, 8.0, 20.0, 55.0, 150.0, 1000.0])
def test_hct_pair_far_field_series(orc, r):
    s, a = 1.528, 1.11
    ref = float(_series_decimal(r, s))
    got = orc.hct_pair(r, a, s)
    # the closed form's terms are O(1/(r - s)); FP64 keeps them to a few ulp
    assert abs(got - ref) <= 64 * 2.2e-16 / (r - s), (r, got, ref)
    # leading term s^3 / (3 r^4)
    assert ref == pytest.approx(s ** 3 / (3 * r ** 4), rel=2 * (s / r) ** 2)


@pytest.mark.parametrize("r,a,s", [(4.0, 1.5, 1.2), (2.0, 1.5, 1.2), (1.0, 1.1, 1.5),
                                   (0.3, 0.8, 1.5), (0.9, 1.3, 1.6), (30.0, 1.1, 1.5)])
def test_hct_pair_derivative_fd(orc, r, a, s):
    h = 1e-6
    fd = (orc.hct_pair(r + h, a, s) - orc.hct_pair(r - h, a, s)) / (2 * h)
    assert orc.hct_pair_dr(r, a, s) == pytest.approx(fd, rel=1e-6, abs=1e-12)


# --- Born radii and energies: closed forms -----------------------------------

@pytest.mark.parametrize("rho,q", [(1.5, 1.0), (2.0, -0.7), (1.2, 0.3)])
def test_isolated_ion_born_energy(orc, rho, q):
    o = orc.energy_forces(np.zeros((1, 3)), [q], [rho], [0.8])
    a = rho - 0.09
    assert o["R"][0] == pytest.approx(a, rel=1e-15)
    assert o["E"][0] == pytest.approx(-0.5 * KE * TAU * q * q / a, rel=1e-14)
    assert o["E"][1] == 0.0
    assert np.all(o["F"] == 0.0)


def test_two_distant_ions(orc):
    r = 2.0e4
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    q, rho = np.array([0.8, -0.6]), np.array([1.5, 1.8])
    o = orc.energy_forces(x, q, rho, [0.8, 0.8])
    a = rho - 0.09
    e_self = -0.5 * TAU * KE * (q[0] ** 2 / a[0] + q[1] ** 2 / a[1])
    e_pair = -TAU * KE * q[0] * q[1] / r
    assert o["E"][0] == pytest.approx(e_self + e_pair, rel=1e-12)
    assert o["E"][1] == pytest.approx(KE * q[0] * q[1] / r, rel=1e-14)


def test_gb_function_limits(orc):
    R = np.array([1.7, 2.3])
    q = np.array([0.5, 0.4])
    # r -> 0: f -> sqrt(R1 R2)
    x = np.array([[0, 0, 0], [1e-7, 0, 0]], dtype=float)
    E = orc.energy_fixed_radii(x, q, R)
    expect = -0.5 * TAU * KE * (q[0] ** 2 / R[0] + q[1] ** 2 / R[1] + 2 * q[0] * q[1] / math.sqrt(R[0] * R[1]))
    assert E[0] == pytest.approx(expect, rel=1e-9)
    # r >> R: f -> r
    x = np.array([[0, 0, 0], [500.0, 0, 0]])
    E = orc.energy_fixed_radii(x, q, R)
    expect = -0.5 * TAU * KE * (q[0] ** 2 / R[0] + q[1] ** 2 / R[1] + 2 * q[0] * q[1] / 500.0)
    assert E[0] == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("R1,R2", [(1.7, 2.3), (1.2, 1.2), (3.0, 1.4)])
def test_gb_function_small_distance_expansion(orc, R1, R2):
    """Between the two limits: expanding exp(-D) = 1 - D + D^2/2 - ... with
    D = r^2 / (4 R1 R2) gives, by hand,
        f^2 - R1 R2 = r^2 (1 - 1/4) + r^4 / (32 R1 R2) + O(r^6),
    so the slope 3/4 at small r fixes the 4 in D, which both limits leave
    free.  f is read back from the pair term of the oracle's GB energy."""
    R = np.array([R1, R2])
    q = np.array([0.5, 0.4])
    e_self = -0.5 * TAU * KE * (q[0] ** 2 / R[0] + q[1] ** 2 / R[1])
    RR = R1 * R2
    for r in (0.02, 0.05, 0.1):
        x = np.array([[0, 0, 0], [r, 0, 0]], dtype=float)
        E = orc.energy_fixed_radii(x, q, R)
        f = -TAU * KE * q[0] * q[1] / (E[0] - e_self)
        slope = (f * f - RR) / (r * r)
        assert slope == pytest.approx(0.75 + r * r / (32.0 * RR), abs=r ** 4 / RR ** 2 * 0.01 + 1e-9)


def test_obc_zero_descreening_and_hct_limit(orc):
    """psi -> 0 gives R = rho - offset; with alpha=1, beta=gamma=0 and small psi
    the OBC radius reduces to the HCT radius 1/R = 1/a - I a / rho."""
    x = np.array([[0, 0, 0], [60.0, 0, 0], [0, 70.0, 0]])
    rho, scr = np.array([1.5, 1.7, 2.0]), np.array([0.8, 0.8, 0.8])
    p = orc.default_params(alpha=1.0, beta=0.0, gamma=0.0)
    o = orc.born_radii(x, rho, scr, p)
    a = rho - 0.09
    hct = 1.0 / (1.0 / a - o["I"] * a / rho)
    assert np.allclose(o["R"], hct, rtol=1e-14)
    assert np.all(np.abs(o["R"] - a) < 1e-6)


def test_obc_tanh_saturation(orc):
    """Deeply buried atom: psi large, tanh -> 1, R -> a rho / (rho - a) = a rho / offset."""
    b = synth.config_plain()
    x, q, rho, scr, _ = orc.batch_arrays(b)
    o = orc.born_radii(x, rho, scr)
    a = rho - 0.09
    rmax = a * rho / 0.09
    assert np.all(o["R"] > a - 1e-12) and np.all(o["R"] < rmax + 1e-9)
    k = int(np.argmax(o["psi"]))
    phi = 1.0 * o["psi"][k] - 0.8 * o["psi"][k] ** 2 + 4.85 * o["psi"][k] ** 3
    if phi > 8:  # tanh saturated to ~1e-7
        assert o["R"][k] == pytest.approx(rmax[k], rel=1e-5)


# --- forces and charge derivatives -------------------------------------------

@pytest.fixture(scope="module")
def plain(orc):
    b = synth.config_plain()
    x, q, rho, scr, _ = orc.batch_arrays(b)
    return x, q, rho, scr, orc.energy_forces(x, q, rho, scr)


def test_forces_central_differences(orc, plain):
    x, q, rho, scr, o = plain
    rng = np.random.default_rng(11)
    h = 1e-4
    for _ in range(24):
        i, k = int(rng.integers(x.shape[0])), int(rng.integers(3))
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        fd = -(orc.energy(xp, q, rho, scr) - orc.energy(xm, q, rho, scr)) / (2 * h)
        assert abs(fd - o["F"][i, k]) < 2e-6 * max(1.0, abs(fd)), (i, k, fd, o["F"][i, k])


def test_net_force_and_torque_vanish(plain):
    x, q, rho, scr, o = plain
    F = o["F"]
    scale = np.abs(F).sum()
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * scale
    assert np.abs(np.cross(x, F).sum(axis=0)).max() < 1e-11 * scale * np.abs(x).max()


def test_rigid_motion_invariance(orc, plain):
    x, q, rho, scr, o = plain
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    y = x @ Q.T + rng.normal(size=3) * 7.0
    o2 = orc.energy_forces(y, q, rho, scr)
    assert o2["E"].sum() == pytest.approx(o["E"].sum(), rel=1e-12)
    assert np.allclose(o2["F"], o["F"] @ Q.T, atol=1e-9 * np.abs(o["F"]).max())


def test_charge_derivative_fd_and_euler(orc, plain):
    x, q, rho, scr, o = plain
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(16):
        i = int(rng.integers(q.size))
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (orc.energy(x, qp, rho, scr) - orc.energy(x, qm, rho, scr)) / (2 * h)
        assert fd == pytest.approx(o["phi"][i], rel=1e-7, abs=1e-6)
    # E is homogeneous of degree 2 in q at fixed Born radii: sum q dE/dq = 2E
    assert (q * o["phi"]).sum() == pytest.approx(2 * o["E"].sum(), rel=1e-12)


def test_restraint_forces_fd(orc, plain):
    x = plain[0]
    E, F = orc.restraints(x)
    rng = np.random.default_rng(8)
    h = 1e-5
    for _ in range(12):
        i, k = int(rng.integers(x.shape[0])), int(rng.integers(3))
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        fd = -(orc.restraints(xp)[0].sum() - orc.restraints(xm)[0].sum()) / (2 * h)
        assert fd == pytest.approx(F[i, k], abs=1e-5)


def test_born_radii_subset_matches_full(orc):
    b = synth.random_batch([300], seed=2, sites=False)
    x, q, rho, scr, _ = orc.batch_arrays(b)
    full = orc.born_radii(x, rho, scr)["R"]
    idx = np.array([0, 5, 77, 299])
    assert np.array_equal(orc.born_radii_subset(x, rho, scr, idx), full[idx])
