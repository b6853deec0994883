"""Oracle GB with Debye-Hueckel salt screening of the solvent term (inverse
Debye length kappa): pinned by the screened-Coulomb law between distant ions,
by continuity at kappa -> 0, and by finite differences of the energy for the
forces and the charge derivative at kappa != 0."""
import math

import numpy as np
import pytest

import synth

KE = 332.0522173


def _p(orc, kappa):
    return orc.default_params(kappa=kappa)


@pytest.mark.parametrize("kappa", [0.05, 0.125, 0.3])
@pytest.mark.parametrize("r", [25.0, 60.0])
def test_distant_ions_interact_by_screened_coulomb(orc, kappa, r):
    """Two ions far apart at fixed Born radii: E(r) - E(infinity) =
    k_e q1 q2 exp(-kappa r) / (eps_out r) -- the vacuum Coulomb term cancels
    against the GB cross term and the solvent part is screened (Debye-Hueckel)."""
    q, R = np.array([0.8, -0.6]), np.array([1.41, 1.71])
    p = _p(orc, kappa)
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    far = np.array([[0.0, 0.0, 0.0], [1.0e7, 0.0, 0.0]])
    dE = orc.energy_fixed_radii(x, q, R, p).sum() - orc.energy_fixed_radii(far, q, R, p).sum()
    expect = KE * q[0] * q[1] * math.exp(-kappa * r) / (78.5 * r)
    assert dE == pytest.approx(expect, rel=1e-9, abs=1e-12)


def test_isolated_ion_salt_lowers_the_born_energy(orc):
    """A lone ion's energy decreases monotonically with salt and tends to the
    kappa = 0 value as kappa -> 0."""
    x = np.zeros((1, 3))
    q, rho = np.array([0.7]), np.array([1.7])
    E = [orc.energy_forces(x, q, rho, [0.8], _p(orc, k))["E"][0] for k in (0.0, 1e-9, 0.05, 0.2, 1.0)]
    assert E[1] == pytest.approx(E[0], rel=1e-8)
    assert E[0] > E[2] > E[3] > E[4]


@pytest.fixture(scope="module")
def small():
    rep = synth.make_replica(40, 71, [])
    x, q = rep.xyz.astype(np.float64), rep.q.astype(np.float64)
    return x, q, rep.rho.astype(np.float64), rep.screen.astype(np.float64)


@pytest.mark.parametrize("kappa", [0.1, 0.4])
def test_forces_and_charge_derivative_fd_with_salt(orc, small, kappa):
    x, q, rho, scr = small
    p = _p(orc, kappa)
    o = orc.energy_forces(x, q, rho, scr, p)
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(6):
        i, k = int(rng.integers(len(q))), int(rng.integers(3))
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        fd = -(orc.energy(xp, q, rho, scr, p) - orc.energy(xm, q, rho, scr, p)) / (2 * h)
        assert o["F"][i, k] == pytest.approx(fd, abs=2e-6 * max(1.0, abs(fd)))
    for _ in range(6):
        i = int(rng.integers(len(q)))
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (orc.energy(x, qp, rho, scr, p) - orc.energy(x, qm, rho, scr, p)) / (2 * h)
        assert o["phi"][i] == pytest.approx(fd, abs=2e-6 * max(1.0, abs(fd)))
    # degree-2 homogeneity in q at fixed radii survives the screening
    assert (q * o["phi"]).sum() == pytest.approx(2 * o["E"].sum(), rel=1e-10)
