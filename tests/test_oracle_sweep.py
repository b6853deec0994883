"""Oracle per-residue sweep (Sec. III.A.2): every site of the kind gets one
attempt per halt, the sites visited in a uniformly random order.  Pinned by
the visiting rule itself (each site once; all orders equally likely), by
Nernst / Henderson-Hasselbalch populations of independent sites, and by exact
enumeration of coupled sites (a sequence of Metropolis moves that each obey
detailed balance leaves the Boltzmann distribution invariant)."""
import math

import numpy as np
import pytest

import synth
from thermo_enum import KT, F, joint_energies, populations


def _system(seed, specs, n, pH=4.6, E=None):
    rep = synth.make_replica(n, seed, specs)
    return rep, synth.Batch([rep], pH=np.array([pH]), E=np.array([synth.E0_REF_V if E is None else E]))


def _sweeps(orc, b, G_ref, n_sweeps, kinds=(0, 1), seed=7, R=None):
    x, q, rho, scr, off = orc.batch_arrays(b)
    if R is None:   # per replica: replicas are separate molecules
        R = np.concatenate([orc.born_radii(x[a:c], rho[a:c], scr[a:c])["R"] for a, c in zip(off[:-1], off[1:])])
    t = b.site_tables(G_ref)
    states = b.initial_states()
    q = q.copy()
    hist = []
    outs = []
    for step in range(n_sweeps):
        for kind in kinds:
            outs.append(orc.mc_sweep(off, x, q, R, t, states, b.pH, b.E, KT, seed, step, kind))
        hist.append(states.copy())
    return np.array(hist), outs, t


def test_each_site_of_the_kind_visited_once(orc):
    rep, b = _system(61, [(0, 6, 2), (1, 8, 2), (0, 5, 3), (0, 7, 2), (1, 6, 2)], n=80)
    G = orc.site_reference_energies(b)
    _, outs, t = _sweeps(orc, b, G, 20, kinds=(0,))
    kinds = t["site_kind"]
    for o in outs:
        vis = o["visit"][kinds == 0]
        assert sorted(vis.tolist()) == list(range((kinds == 0).sum()))
        assert np.all(o["visit"][kinds == 1] == -1) and np.all(o["acc"][kinds == 1] == 2)
        assert np.all(o["acc"][kinds == 0] <= 1)


def test_visiting_order_is_uniform(orc):
    """Three pH sites: the 6 visiting orders over 3000 sweeps, each close to 1/6."""
    rep, b = _system(62, [(0, 5, 2), (0, 5, 2), (0, 5, 2)], n=40)
    G = orc.site_reference_energies(b)
    _, outs, t = _sweeps(orc, b, G, 3000, kinds=(0,))
    counts = {}
    for o in outs:
        order = tuple(np.argsort(o["visit"]).tolist())
        counts[order] = counts.get(order, 0) + 1
    assert len(counts) == 6
    n = len(outs)
    for c in counts.values():
        assert abs(c / n - 1 / 6) < 4 * math.sqrt((1 / 6) * (5 / 6) / n)


@pytest.mark.parametrize("dE_mV,dpH", [(-30.0, 0.5), (20.0, -0.4)])
def test_lone_sites_follow_nernst_and_hh(orc, dE_mV, dpH):
    """Two replicas, one with a lone redox site and one with a lone pH site,
    reference energies equal to their own charging energies: sweep
    populations follow Eq. 3 with n = 1 and Henderson-Hasselbalch."""
    r0 = synth.make_replica(40, 63, [(1, 8, 2)])
    r1 = synth.make_replica(40, 64, [(0, 6, 2)])
    pka = r1.sites[0].pKa_ref
    E = synth.E0_REF_V + dE_mV * 1e-3
    b = synth.Batch([r0, r1], pH=np.array([7.0, pka + dpH]), E=np.array([E, 0.0]))
    G = orc.site_reference_energies(b)
    hist, _, _ = _sweeps(orc, b, G, 6000)
    f_red = float((hist[:, 0] == 0).mean())
    f_prot = float((hist[:, 1] >= 1).mean())
    e_red = 1 / (1 + math.exp(F * dE_mV * 1e-3 / KT))
    e_prot = 1 / (1 + 10 ** dpH)
    assert abs(f_red - e_red) < 4 * math.sqrt(e_red * (1 - e_red) / 6000) + 1e-3
    assert abs(f_prot - e_prot) < 4 * math.sqrt(e_prot * (1 - e_prot) / 6000) + 1e-3


def test_coupled_sites_match_enumeration(orc):
    """Redox site next to two pH sites (2 and 3 states): joint populations of
    a chain of sweeps against exact enumeration."""
    rep, b = _system(66, [(1, 6, 2), (0, 5, 2), (0, 5, 3)], n=30, pH=4.6, E=synth.E0_REF_V + 0.01)
    G = orc.site_reference_energies(b) + np.array([0.0, 0.3, 0.0, -0.4, 0.0, 0.5, -0.2])
    J = joint_energies(orc, rep, G)
    exact = populations(J, b.E[0], b.pH[0])
    hist, _, _ = _sweeps(orc, b, G, 12000, seed=11)
    for combo, pe in exact.items():
        pm = float(np.all(hist == np.array(combo), axis=1).mean())
        assert abs(pm - pe) < 0.02, (combo, pm, pe)
