"""Pins of the oracle's Langevin (BAOAB) driver.

The paper runs Langevin dynamics with a 2 fs step (Sec. III.D); the splitting
is BAOAB.  Pins: without friction the scheme is velocity Verlet and conserves
the total energy (kinetic energy in kcal/mol from CODATA constants, not from
the oracle's conversion factor); with friction a free particle samples the
Maxwell distribution <v_x^2> = kT/m; a harmonic pair at a large step keeps
the exact configurational variance, which pins the order of the splitting
(B A O A B) and not only its pieces.
"""
import math

import numpy as np

import synth

AMU_KG = 1.66053906660e-27
NA = 6.02214076e23
# 1 amu * A^2 / ps^2 in kcal/mol
AMU_A2_PS2_KCAL = AMU_KG * 1e-20 / 1e-24 * NA / 4184.0


def test_verlet_limit_conserves_energy(orc):
    """friction 0: the energy error after a fixed 20 fs is second order in dt."""
    b = synth.random_batch([40], seed=4, sites=False)
    drift = []
    for dt in (0.0005, 0.00025, 0.000125):
        x, q, rho, scr, off = orc.batch_arrays(b)
        p = orc.default_params(friction=0.0, dt=dt)
        v = np.zeros_like(x)
        F, E = orc.forces_all(off, x, q, rho, scr, p)
        e0 = E.sum()
        for step in range(int(round(0.02 / dt))):
            E = orc.md_step(off, x, v, q, rho, scr, F, 1, step, p)
        ke = 0.5 * p.mass * (v ** 2).sum() * AMU_A2_PS2_KCAL
        assert ke > 10.0        # the chain really moved
        drift.append(abs(E.sum() + ke - e0))
    assert drift[0] < 1e-3 * ke
    assert 3.5 < drift[0] / drift[1] < 4.5 and 3.5 < drift[1] / drift[2] < 4.5


def test_free_particle_maxwell(orc):
    p = orc.default_params(friction=50.0)
    off = np.array([0, 1], np.int64)
    x = np.zeros((1, 3))
    v = np.zeros((1, 3))
    q, rho, scr = np.zeros(1), np.array([1.5]), np.array([0.8])
    F = np.zeros((1, 3))
    vs = []
    for step in range(20000):
        orc.md_step(off, x, v, q, rho, scr, F, 7, step, p)
        if step > 100:
            vs.append(v[0].copy())
    vs = np.array(vs)
    expect = p.kT / (p.mass * AMU_A2_PS2_KCAL)
    # friction*dt = 0.1: velocities decorrelate in ~10 steps
    assert abs(vs.var() / expect - 1) < 0.05


def test_harmonic_configurations_exact_at_a_large_step(orc):
    """BAOAB samples the configurations of a harmonic system exactly at any
    stable time step (Leimkuhler and Matthews, 2013): with ω dt = 1.2 the
    position variance is still kT/κ, where orderings that put the O step
    elsewhere (ABOBA, or velocity Verlet followed by O) give
    kT/κ / (1 - (ω dt/2)^2), 56 % more.

    System: two uncharged atoms of mass m joined by the chain bond with
    r0 = 0, E = k r^2 = k |x1 - x0|^2.  The relative coordinate u = x1 - x0 is a
    3-D harmonic oscillator of reduced mass m/2 and spring κ = 2k, and its O
    step draws z1 - z0, the noise of mass m/2; so <u_x^2> = kT/(2k), ω^2 =
    4k/m.  Uncharged atoms have no GB or Coulomb forces, and the spheres of
    the two atoms (a = 1.41, s = 1.2 A) give no descreening NaN at any r > 0.
    """
    p0 = orc.default_params()
    k = 0.05                                      # kcal/mol/A^2
    m = p0.mass
    omega = math.sqrt(4.0 * k * 418.4 / m)        # 1/ps (418.4: kcal/mol/A/amu -> A/ps^2)
    dt = 1.2 / omega
    p = orc.default_params(bond_k=k, bond_r0=0.0, rep_k=0.0, dt=dt, friction=omega)
    off = np.array([0, 2], np.int64)
    x = np.array([[0.0, 0.0, 0.0], [2.0, 1.0, -1.0]])
    v = np.zeros((2, 3))
    q, rho, scr = np.zeros(2), np.full(2, 1.5), np.full(2, 0.8)
    F, _ = orc.forces_all(off, x, q, rho, scr, p)
    us = []
    for step in range(40000):
        orc.md_step(off, x, v, q, rho, scr, F, 11, step, p)
        if step >= 200:
            us.append(x[1] - x[0])
    us = np.array(us)
    expect = p.kT / (2.0 * k)
    ratio = (us ** 2).mean() / expect
    # about 4e4 nearly independent samples per component: ~1 % standard error
    assert abs(ratio - 1.0) < 0.04, ratio
    assert np.abs(us.mean(axis=0)).max() < 0.1 * math.sqrt(expect)
