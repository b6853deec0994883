"""Sec. II.D relations (Eq. 16, 17, 18) and the Hill form of Eq. 3, checked
on an exactly enumerable system: one redox site and one pH site at frozen
coordinates, with joint-state free energies built from the oracle's GB +
Coulomb energy and the state terms of Eq. 8 and 9,
    G(s) = E_elec(q(s)) - G_ref(s) + F (E - E0_ref) n_e(s) + kT ln10 (pH - pKa_ref) n_H(s).
Midpoints are found by bisection on the exact populations; the relations are
thermodynamic identities for a single redox site, so they must hold to
rounding.  The same enumeration is the expected value of the GPU statistical
test."""
import math

import numpy as np
import pytest

import synth
from thermo_enum import F, KT, LN10, f_protonated, f_reduced, joint_energies


def bisect(fun, lo, hi, tol=1e-12):
    flo = fun(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        fm = fun(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def midpoint_E(J, pH):
    return bisect(lambda E: f_reduced(J, E, pH) - 0.5, -3.0, 3.0)


def midpoint_pH(J, E):
    return bisect(lambda pH: f_protonated(J, E, pH) - 0.5, -20.0, 30.0)


@pytest.fixture(scope="module")
def system(orc):
    """Redox site (8 atoms) next to a pH site (6 atoms), close enough to couple;
    reference energies near each site's own charging energy."""
    rep = synth.make_replica(60, 52, [(1, 8, 2), (0, 6, 2)])
    b = synth.Batch([rep], pH=np.array([4.6]), E=np.array([synth.E0_REF_V]))
    G_ref = orc.site_reference_energies(b) + np.array([0.0, 0.4, 0.0, -0.3])
    return joint_energies(orc, rep, G_ref)


@pytest.fixture(scope="module")
def limits(system):
    J = system
    E0_prot = midpoint_E(J, -15.0)          # pH site fully protonated
    E0_deprot = midpoint_E(J, 25.0)         # fully deprotonated
    pKa_red = midpoint_pH(J, -2.0)          # redox site fully reduced
    pKa_oxi = midpoint_pH(J, 2.0)           # fully oxidized
    return E0_prot, E0_deprot, pKa_red, pKa_oxi


def test_sites_are_coupled(limits):
    E0_prot, E0_deprot, pKa_red, pKa_oxi = limits
    assert abs(pKa_red - pKa_oxi) > 0.05        # the relations below are not trivial here


def test_eq16_redox_and_pka_shifts(limits):
    """v F (E0_prot - E0_deprot) = kT ln10 (pKa_red - pKa_oxi), v = 1."""
    E0_prot, E0_deprot, pKa_red, pKa_oxi = limits
    assert F * (E0_prot - E0_deprot) == pytest.approx(KT * LN10 * (pKa_red - pKa_oxi), abs=1e-8)


@pytest.mark.parametrize("pH", [2.0, 4.0, 4.6, 5.5, 8.0])
def test_eq17_ph_dependent_midpoint(system, limits, pH):
    E0_prot, E0_deprot, pKa_red, pKa_oxi = limits
    pred = E0_prot + KT / F * math.log((10 ** -pKa_red + 10 ** -pH) / (10 ** -pKa_oxi + 10 ** -pH))
    assert midpoint_E(system, pH) == pytest.approx(pred, abs=1e-9)


@pytest.mark.parametrize("dE", [-0.2, -0.05, 0.0, 0.03, 0.2])
def test_eq18_potential_dependent_pka(system, limits, dE):
    E0_prot, E0_deprot, pKa_red, pKa_oxi = limits
    E = 0.5 * (E0_prot + E0_deprot) + dE
    num = math.exp(-F * E0_prot / KT) + math.exp(-F * E / KT)
    den = math.exp(-F * E0_deprot / KT) + math.exp(-F * E / KT)
    assert midpoint_pH(system, E) == pytest.approx(pKa_red + math.log10(num / den), abs=1e-9)


def test_eq3_hill_coefficient_one_for_isolated_site(orc):
    """A lone redox site follows Eq. 3 with n = 1 and E0 = E0_ref when
    G_ref equals its own charging energy (Eq. 4)."""
    rep = synth.make_replica(40, 53, [(1, 8, 2)])
    b = synth.Batch([rep], pH=np.array([7.0]), E=np.array([synth.E0_REF_V]))
    J = joint_energies(orc, rep, orc.site_reference_energies(b))
    for dE in (-0.08, -0.01, 0.0, 0.04, 0.1):
        E = synth.E0_REF_V + dE
        assert f_reduced(J, E, 7.0) == pytest.approx(1.0 / (1.0 + math.exp(F * dE / KT)), abs=1e-12)
