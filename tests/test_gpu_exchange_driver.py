"""The MD driver's own replica exchange (k_grid_exchange inside gb_md_segment)
against the oracle's exchange, attempt by attempt.

Sec. II.C, Eq. 14-15 (E ladder) and Sec. III.B (neighbour schedule), with the
pH analogue along the other dimension of a 2-D grid.  The driver counts the
bound electrons and protons of every replica on the device from its site
states, pairs the grid's slots, draws from Philox and swaps labels, all inside
a captured graph.  Here coordinates are frozen (dt = 0) and no Monte Carlo
runs (mc_every = 0), so the states are fixed and set by hand, with several
sites per replica in changed states.  Each run(1) is one MD step and one
exchange attempt.  After every attempt the grid and the per-replica E and pH
must equal the oracle's result for the same grid, counts, attempt and seed.
The decisions must be identical: both sides take Delta in FP64 from the same
integers and ladder values, so only a u within rounding of exp(-Delta) could
differ, and such a case is reported, not counted.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import KT, device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _counts(t, state, M):
    """Bound electrons (redox sites) and protons (pH sites) per replica."""
    N_e, N_H = np.zeros(M, np.int32), np.zeros(M, np.int32)
    for r in range(M):
        for s in range(t["site_off"][r], t["site_off"][r + 1]):
            k = t["site_state_off"][s] + state[s]
            if t["site_kind"][s] == 1:
                N_e[r] += t["n_e"][k]
            else:
                N_H[r] += t["n_H"][k]
    return N_e, N_H


def _u(seed, first_slot, attempt):
    w = oracle.philox4x64([first_slot, attempt, 3, 0], [seed, 0])
    return float(int(w[0]) >> 11) * 2.0 ** -53


@pytest.mark.parametrize("n_pH,n_E,ex_dim,wrap", [
    (1, 8, 0, True),            # E-REMD ladder (Sec. III.B schedule with its wrap pair)
    (1, 8, 0, False),
    (1, 7, 0, True),            # odd ladder: one slot sits out each attempt
    (2, 4, 2, True),            # 2-D grid, exchanges alternating along E and pH
    (3, 2, 2, False),
    (4, 2, 1, True),            # pH ladders only
])
def test_driver_exchange_matches_oracle(pkg, n_pH, n_E, ex_dim, wrap):
    import torch
    device()
    M = n_pH * n_E
    seed = 17 + M
    rng = np.random.default_rng(seed)
    specs = [(1, 6, 2)] * 3 + [(0, 5, 3)] * 3 + [(0, 4, 2)]
    reps = [synth.make_replica(90 + 6 * r, 300 + r, specs) for r in range(M)]
    E_lad = synth.e_ladder(n_E, half_width=0.04)
    pH_lad = np.linspace(4.3, 5.3, n_pH)
    pH = np.array([pH_lad[r // n_E] for r in range(M)])
    E = np.array([E_lad[r % n_E] for r in range(M)])
    b = synth.Batch(reps, pH=pH, E=E)
    t = b.site_tables(np.zeros(sum(s.n_states for r in reps for s in r.sites)))
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         sites=t, pH=pH, E=E, E_ladder=E_lad, pH_ladder=pH_lad, dt=0.0, mc_every=0,
                         ex_every=1, ex_dim=ex_dim, wrap=wrap, seed=seed)
    # several sites per replica away from state 0
    state = np.array([rng.integers(t["site_nstates"][s]) for s in range(t["n_sites"])], np.int32)
    sim.state.copy_(torch.as_tensor(state))
    N_e, N_H = _counts(t, state, M)
    assert len(set(N_e.tolist())) > 2 and len(set(N_H.tolist())) > 2
    grid = np.arange(M, dtype=np.int32)
    E_rep, pH_rep = E.copy(), pH.copy()
    n_acc, n_near = 0, 0
    for attempt in range(48):
        sim.run(1)
        assert sim.st.attempt == attempt + 1
        dimE = ex_dim == 0 or (ex_dim == 2 and ((attempt >> 1) & 1) == 0)
        if dimE:
            delta, acc = oracle.exchange(E_lad, grid, N_e, 0, attempt, seed, KT, wrap=wrap,
                                         n_ladders=n_pH, ladder_len=n_E, ladder_stride=n_E, slot_stride=1)
        else:
            delta, acc = oracle.exchange(pH_lad, grid, N_H, 1, attempt, seed, KT, wrap=wrap,
                                         n_ladders=n_E, ladder_len=n_pH, ladder_stride=1, slot_stride=n_E)
        for k in range(M):                  # every slot's replica carries its slot's values
            E_rep[grid[k]] = E_lad[k % n_E]
            pH_rep[grid[k]] = pH_lad[k // n_E]
        got = sim.grid.cpu().numpy()
        if not np.array_equal(got, grid):
            # only a u within rounding of exp(-Delta) may decide differently
            tried = np.flatnonzero(np.isfinite(delta))
            near = [a for a in tried if abs(delta[a] + np.log(_u(seed, a, attempt))) < 1e-9]
            assert near, (attempt, got, grid)
            n_near += 1
            grid = got.copy()
            continue
        assert np.array_equal(sim.E.cpu().numpy(), E_rep), attempt
        assert np.array_equal(sim.pH.cpu().numpy(), pH_rep), attempt
        n_acc += int(acc.sum())
    sim.sync()
    assert n_near == 0 or n_near < 2
    assert n_acc >= 10                     # the test exercised accepted swaps
