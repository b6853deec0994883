"""Pins of the oracle's Monte Carlo, exchange and random-number pieces.

- Philox4x64-10 against numpy's independent implementation (numpy generates
  its first block from counter + 1).
- Redox MC (Eq. 8) against the Nernst fraction, Eq. 3 with n = v = 1; protonation
  MC (Eq. 9) against Henderson-Hasselbalch; coupled sites against exact
  enumeration of the joint Boltzmann weights.
- The state-change energy against the site-row expansion of the quadratic form.
- E-REMD exchange (Eq. 14-15): the worked example printed after Eq. 15, the
  neighbour schedule of Sec. III.B and detailed balance on a two-replica toy.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

KB = 0.0019872043
KT = KB * 300.0
F = 23.0605478
LN10 = math.log(10.0)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Philox --------------------------------------------------------------------

@pytest.mark.parametrize("counter,key", [
    ((1, 0, 0, 0), (5, 0)),
    ((7, 123456789, 2, 0), (0xDEADBEEF, 0)),
    ((2 ** 64 - 1, 3, 4, 5), (1, 2)),
    ((0, 0, 0, 1), (2 ** 63 + 11, 0)),
])
def test_philox_matches_numpy(orc, counter, key):
    c = np.array(counter, dtype=object)
    # numpy increments the 256-bit counter before its first block
    prev = [int(v) for v in counter]
    for k in range(4):
        if prev[k] > 0:
            prev[k] -= 1
            break
        prev[k] = 2 ** 64 - 1
    bg = np.random.Philox(counter=np.array(prev, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    assert list(bg.random_raw(4)) == list(orc.philox4x64(counter, key))


def test_normals_moments(orc):
    z = np.array([orc.normals(9, 0, s, a) for s in range(50) for a in range(100)]).ravel()
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)


# --- Monte Carlo ---------------------------------------------------------------

def _tiny_system(seed, specs, n=40):
    rep = synth.make_replica(n, seed, specs)
    b = synth.Batch([rep], pH=np.array([4.85]), E=np.array([synth.E0_REF_V]))
    return b


def _run_chain(orc, b, G_ref, pH, E, n_att, kinds=(0, 1), seed=17):
    x, q, rho, scr, off = orc.batch_arrays(b)
    R = orc.born_radii(x, rho, scr)["R"]
    t = b.site_tables(G_ref)
    states = b.initial_states()
    q = q.copy()
    counts = []
    for step in range(n_att):
        for kind in kinds:
            orc.mc_step(off, x, q, R, t, states, [pH], [E], KT, seed, step, kind)
        counts.append(states.copy())
    return np.array(counts), t


def test_site_row_expansion_equals_two_evaluations(orc):
    """E is quadratic in q at fixed R, so for a change dq on site atoms
    dE = sum_k dq_k phi_k + 1/2 sum_kl dq_k dq_l A_kl with
    A_kl = k_e[(1/eps_in)/r_kl (k != l) - tau/f_kl], A_kk = -k_e tau / R_k."""
    b = synth.config_plain()
    x, q, rho, scr, off = orc.batch_arrays(b)
    o = orc.energy_forces(x, q, rho, scr)
    R, phi = o["R"], o["phi"]
    t = b.site_tables()
    tau = 1.0 - 1.0 / 78.5
    for s in range(t["n_sites"]):
        idx = t["site_atom_idx"][t["site_atom_off"][s]:t["site_atom_off"][s + 1]]
        na = idx.size
        qo = t["site_q_off"][s] + na
        dq = t["q_state"][qo:qo + na].astype(np.float64) - q[idx]
        xs = x[idx]
        r = np.linalg.norm(xs[:, None] - xs[None], axis=2)
        RR = np.outer(R[idx], R[idx])
        f = np.sqrt(r ** 2 + RR * np.exp(-r ** 2 / (4 * RR)))
        with np.errstate(divide="ignore"):
            A = 332.0522173 * (np.where(r > 0, 1.0 / np.where(r > 0, r, 1), 0.0) - tau / f)
        np.fill_diagonal(A, -332.0522173 * tau / R[idx])
        dE_rows = dq @ phi[idx] + 0.5 * dq @ A @ dq
        q2 = q.copy()
        q2[idx] += dq
        dE_two = orc.energy_fixed_radii(x, q2, R).sum() - orc.energy_fixed_radii(x, q, R).sum()
        assert dE_rows == pytest.approx(dE_two, abs=1e-9 * max(1.0, abs(dE_two)))


@pytest.mark.parametrize("dE_mV", [-60.0, 0.0, 25.0])
def test_redox_fraction_follows_nernst(orc, dE_mV):
    """One 2-state redox site with G_ref(1) - G_ref(0) = dE_elec(0->1):
    P(reduced) = 1 / (1 + exp(F (E - E0) / kT))   (Eq. 3, n = v = 1)."""
    b = _tiny_system(21, [(1, 8, 2)])
    G = orc.site_reference_energies(b)
    E = synth.E0_REF_V + dE_mV * 1e-3
    st, _ = _run_chain(orc, b, G, 4.85, E, 6000, kinds=(1,))
    f_red = float((st[:, 0] == 0).mean())
    expect = 1.0 / (1.0 + math.exp(F * (E - synth.E0_REF_V) / KT))
    # two-state Metropolis chain: lag-1 anticorrelated, variance below binomial
    assert abs(f_red - expect) < 4 * math.sqrt(expect * (1 - expect) / 6000) + 1e-3


@pytest.mark.parametrize("dpH", [-1.0, 0.0, 0.6])
def test_protonation_fraction_follows_henderson_hasselbalch(orc, dpH):
    b = _tiny_system(22, [(0, 10, 2)])
    G = orc.site_reference_energies(b)
    pka = b.replicas[0].sites[0].pKa_ref
    st, _ = _run_chain(orc, b, G, pka + dpH, synth.E0_REF_V, 6000, kinds=(0,))
    f_prot = float((st[:, 0] == 1).mean())
    expect = 1.0 / (1.0 + 10 ** dpH)
    assert abs(f_prot - expect) < 4 * math.sqrt(expect * (1 - expect) / 6000) + 1e-3


def test_single_attempt_acceptance_probability(orc):
    """From state 0 the move 0 -> 1 is accepted with probability min(1, e^-dG/kT)."""
    b = _tiny_system(23, [(1, 8, 2)])
    x, q, rho, scr, off = orc.batch_arrays(b)
    R = orc.born_radii(x, rho, scr)["R"]
    t = b.site_tables(orc.site_reference_energies(b))
    E = synth.E0_REF_V + 0.02
    acc, dGs = [], []
    for step in range(4000):
        states = b.initial_states()
        o = orc.mc_step(off, x, q.copy(), R, t, states, [4.85], [E], KT, 3, step, 1)
        acc.append(o["acc"][0])
        dGs.append(o["dG"][0])
    dG = float(np.mean(dGs))
    assert np.allclose(dGs, dG)
    # oxidation: one electron leaves, dG = -F (E - E0)
    assert dG == pytest.approx(-F * 0.02, abs=1e-9)
    p = min(1.0, math.exp(-dG / KT))
    assert abs(np.mean(acc) - p) < 4 * math.sqrt(max(p * (1 - p), 1e-4) / 4000)


def test_coupled_sites_match_enumeration(orc):
    """Three interacting sites (redox 2 states, pH 2 and 3 states) at frozen
    coordinates: MC marginals against exact enumeration of exp(-G(s)/kT) with
    G(s) = E_elec(q(s)) - sum G_ref + F(E - E0) n_e + kT ln10 (pH - pKa) n_H."""
    b = _tiny_system(31, [(1, 6, 2), (0, 5, 2), (0, 5, 3)], n=24)
    x, q0, rho, scr, off = orc.batch_arrays(b)
    R = orc.born_radii(x, rho, scr)["R"]
    t = b.site_tables()
    # reference energies near each site's own charging energy, shifted by a
    # fraction of kT, so that several joint states carry weight
    G_ref = orc.site_reference_energies(b) + np.array([0, 0.3, 0, -0.4, 0, 0.5, -0.2])
    pH, E = 4.6, synth.E0_REF_V + 0.01
    sites = b.replicas[0].sites
    import itertools
    weights = {}
    for combo in itertools.product(*[range(s.n_states) for s in sites]):
        qq = q0.copy()
        G = 0.0
        for s_idx, (s, k) in enumerate(zip(sites, combo)):
            qq[s.atoms] = s.q_state[k].astype(np.float64)
            G -= G_ref[t["site_state_off"][s_idx] + k]
            G += F * (E - s.E0_ref) * s.n_e[k] if s.kind == 1 else 0.0
            G += KT * LN10 * (pH - s.pKa_ref) * s.n_H[k] if s.kind == 0 else 0.0
        G += orc.energy_fixed_radii(x, qq, R).sum()
        weights[combo] = G
    Gmin = min(weights.values())
    Z = sum(math.exp(-(g - Gmin) / KT) for g in weights.values())
    exact = {c: math.exp(-(g - Gmin) / KT) / Z for c, g in weights.items()}
    st, _ = _run_chain(orc, b, G_ref, pH, E, 30000, seed=99)
    for s_idx, s in enumerate(sites):
        for k in range(s.n_states):
            pe = sum(p for c, p in exact.items() if c[s_idx] == k)
            pm = float((st[:, s_idx] == k).mean())
            # effective sample size well below 30000 (correlated chain): loose bound
            assert abs(pm - pe) < 0.02, (s_idx, k, pm, pe)


# --- exchange --------------------------------------------------------------------

def test_worked_example_after_eq15(orc):
    g = json.load(open(os.path.join(GOLDEN, "eremd_worked_example.json")))
    kT = KB * g["T_K"]
    # oracle Delta for replica i (N = dN) at E, replica j (N = 0) at E + dE
    rep = np.array([0, 1], np.int32)
    delta, acc = orc.exchange([0.0, g["dE_V"]], rep, [g["dN"], 0], 0, 0, 1, kT, wrap=False)
    assert round(math.exp(-delta[0]), g["acceptance_digits"]) == g["acceptance_printed"]
    # acceptance frequency over independent attempts
    hits = 0
    n = 20000
    for att in range(0, 2 * n, 2):
        rep = np.array([0, 1], np.int32)
        d, a = orc.exchange([0.0, g["dE_V"]], rep, [g["dN"], 0], 0, att, 5, kT, wrap=False)
        hits += int(a[0])
    p = math.exp(-delta[0])
    assert abs(hits / n - p) < 4 * math.sqrt(p * (1 - p) / n)
    # 1 pH unit in volts: kT ln10 / F
    assert round(kT * LN10 / F * 1000, g["mV_per_pH_digits"]) == g["mV_per_pH_printed"]


def test_neighbour_schedule_sec_iii_b(orc):
    """4 replicas: first attempt pairs (1,2),(3,4), the next (2,3),(1,4)."""
    rep = np.arange(4, dtype=np.int32)
    vals = np.array([0.0, 0.1, 0.2, 0.3])
    same = np.zeros(4, np.int32)   # equal electron counts: Delta = 0, always accepted
    d, a = orc.exchange(vals, rep, same, 0, 0, 1, KT)
    assert list(rep) == [1, 0, 3, 2] and list(a) == [1, 0, 1, 0]
    d, a = orc.exchange(vals, rep, same, 0, 1, 1, KT)
    # slots (1,2) swap and the wrap pair (3,0) swaps
    assert list(rep) == [2, 3, 0, 1] and list(a) == [0, 1, 0, 1]
    rep = np.arange(4, dtype=np.int32)
    orc.exchange(vals, rep, same, 0, 1, 1, KT, wrap=False)
    assert list(rep) == [0, 2, 1, 3]


def test_exchange_detailed_balance_two_replicas(orc):
    """Fixed N = (1, 0) on a two-slot ladder: the fraction of attempts that end
    with replica 0 at the low potential is 1/(1 + e^-Delta0), where Delta0 is the
    exponent for moving replica 0 from the low to the high slot."""
    vals = np.array([synth.E0_REF_V, synth.E0_REF_V + 0.02])
    ncount = np.array([1, 0], np.int32)
    rep = np.array([0, 1], np.int32)
    n = 40000
    at_low = 0
    for att in range(n):
        orc.exchange(vals, rep, ncount, 0, 2 * att, 13, KT, wrap=False)
        at_low += int(rep[0] == 0)
    d0 = F / KT * (vals[1] - vals[0]) * (1 - 0)
    expect = 1.0 / (1.0 + math.exp(-d0))
    assert abs(at_low / n - expect) < 5 * math.sqrt(expect * (1 - expect) / n) * 2


def test_ph_exchange_uses_ln10(orc):
    rep = np.array([0, 1], np.int32)
    d, _ = orc.exchange([4.0, 4.5], rep, [2, 1], 1, 0, 1, KT, wrap=False)
    assert d[0] == pytest.approx(LN10 * 0.5 * 1)


def test_two_dimensional_grid_lines(orc):
    """E exchanges run along rows of a (pH x E) grid, pH exchanges along columns."""
    n_pH, n_E = 3, 4
    grid = np.arange(n_pH * n_E, dtype=np.int32)       # replica at (p, e) = p*n_E + e
    same = np.zeros(n_pH * n_E, np.int32)
    orc.exchange(np.zeros(n_E), grid, same, 0, 0, 1, KT, wrap=False,
                 n_ladders=n_pH, ladder_len=n_E, ladder_stride=n_E, slot_stride=1)
    assert grid.reshape(n_pH, n_E).tolist() == [[1, 0, 3, 2], [5, 4, 7, 6], [9, 8, 11, 10]]
    orc.exchange(np.zeros(n_pH), grid, same, 1, 0, 1, KT, wrap=False,
                 n_ladders=n_E, ladder_len=n_pH, ladder_stride=1, slot_stride=n_E)
    assert grid.reshape(n_pH, n_E).tolist() == [[5, 4, 7, 6], [1, 0, 3, 2], [9, 8, 11, 10]]
