"""Exact enumeration of joint site states at frozen coordinates (test
infrastructure): free energies from the oracle's GB + Coulomb energy at fixed
Born radii plus the state terms of Eq. 8 and 9,
    G(s) = E_elec(q(s)) - G_ref(s) + F (E - E0_ref) n_e(s) + kT ln10 (pH - pKa_ref) n_H(s),
and their Boltzmann populations."""
import itertools
import math

import numpy as np

import synth

KB = 0.0019872043
T = 300.0
KT = KB * T
F = 23.0605478
LN10 = math.log(10.0)


def joint_energies(orc, rep, G_ref, p=None):
    """Per joint state (tuple of site states): (E_elec - sum G_ref, n_e, n_H, pKa, E0)."""
    b = synth.Batch([rep], pH=np.array([7.0]), E=np.array([0.0]))
    x, q0, rho, scr, off = orc.batch_arrays(b)
    R = orc.born_radii(x, rho, scr, p)["R"]
    t = b.site_tables()
    out = {}
    for combo in itertools.product(*[range(s.n_states) for s in rep.sites]):
        qq = q0.copy()
        g, terms = 0.0, []
        for s_idx, (s, k) in enumerate(zip(rep.sites, combo)):
            qq[s.atoms] = s.q_state[k].astype(np.float64)
            g -= G_ref[t["site_state_off"][s_idx] + k]
            terms.append((s.kind, int(s.n_e[k]), int(s.n_H[k]), s.pKa_ref, s.E0_ref))
        g += orc.energy_fixed_radii(x, qq, R, p).sum()
        out[combo] = (g, terms)
    return out


def populations(J, E, pH):
    """Exact joint-state probabilities at (E, pH)."""
    G = {}
    for c, (g, terms) in J.items():
        v = g
        for kind, ne, nh, pka, e0 in terms:
            v += F * (E - e0) * ne if kind == 1 else KT * LN10 * (pH - pka) * nh
        G[c] = v
    gmin = min(G.values())
    w = {c: math.exp(-(v - gmin) / KT) for c, v in G.items()}
    z = sum(w.values())
    return {c: v / z for c, v in w.items()}


def f_reduced(J, E, pH, site=0):
    return sum(p for c, p in populations(J, E, pH).items() if c[site] == 0)


def f_protonated(J, E, pH, site=1):
    return sum(p for c, p in populations(J, E, pH).items() if c[site] >= 1)


