"""Run metrics of the MD driver: the per-pair exchange counters of
gb_md_state against a host tally of the grid before and after every
exchange, and the JSON-lines record of Simulation.metrics."""
import json

import numpy as np
import pytest

import oracle
import synth
from gpu_common import device, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _pairs(attempt, n_pH, n_E, ex_dim, wrap):
    """(dimension, first grid index, second grid index) of every pair the
    exchange of this attempt number tries (Sec. III.B schedule)."""
    dimE = ex_dim == 0 or (ex_dim == 2 and ((attempt >> 1) & 1) == 0)
    n_lad, length = (n_pH, n_E) if dimE else (n_E, n_pH)
    lad_stride, slot_stride = (n_E, 1) if dimE else (1, n_E)
    out = []
    for l in range(n_lad):
        for a in range(length):
            if (a & 1) != (attempt & 1):
                continue
            b = a + 1
            if b == length:
                if not (wrap and (attempt & 1) and length % 2 == 0):
                    continue
                b = 0
            out.append((0 if dimE else 1, l * lad_stride + a * slot_stride, l * lad_stride + b * slot_stride))
    return out


@pytest.mark.parametrize("n_pH,n_E,ex_dim", [(1, 4, 0), (2, 3, 2), (2, 2, 1)])
def test_exchange_counters_match_the_grid_history(pkg, n_pH, n_E, ex_dim):
    import torch
    device()
    M = n_pH * n_E
    b = synth.random_batch([64 + 8 * r for r in range(M)], seed=51 + M)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    E_lad = synth.e_ladder(n_E, half_width=0.05)
    pH_lad = np.linspace(4.5, 5.2, n_pH)
    pH = np.array([pH_lad[r // n_E] for r in range(M)])
    E = np.array([E_lad[r % n_E] for r in range(M)])
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         sites=t, pH=pH, E=E, E_ladder=E_lad, pH_ladder=pH_lad, mc_every=1, ex_every=1,
                         ex_dim=ex_dim, seed=5)
    want = np.zeros((2, 2, M), np.int64)
    for attempt in range(24):
        before = sim.grid.cpu().numpy().copy()
        sim.run(1)
        after = sim.grid.cpu().numpy()
        for d, ga, gb in _pairs(attempt, n_pH, n_E, ex_dim, True):
            want[d, 0, ga] += 1
            swapped = after[ga] == before[gb] and after[gb] == before[ga]
            assert swapped or (after[ga] == before[ga] and after[gb] == before[gb])
            want[d, 1, ga] += int(swapped)
    sim.sync()
    got = sim.ex_count.cpu().numpy()
    assert np.array_equal(got, want), (got, want)
    assert want[:, 1].sum() > 0          # some exchanges were accepted
    st = sim.exchange_stats()
    assert np.array_equal(st["E"]["attempts"], want[0, 0].reshape(n_pH, n_E))
    r = st["pH"]["ratio"]
    att = want[1, 0].reshape(n_pH, n_E)
    assert np.all(np.isnan(r[att == 0]))
    assert np.allclose(r[att > 0], want[1, 1].reshape(n_pH, n_E)[att > 0] / att[att > 0])


def test_metrics_record_is_json_lines(pkg, tmp_path):
    import torch
    device()
    b = synth.random_batch([90, 70, 110], seed=55)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    lad = synth.e_ladder(3)
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         sites=t, pH=b.pH, E=lad, E_ladder=lad, mc_every=5, ex_every=10, seed=2)
    p = str(tmp_path / "run.jsonl")
    for _ in range(3):
        sim.run(10)
        sim.log_metrics(p)
    sim.sync()
    lines = [json.loads(x) for x in open(p).read().splitlines()]
    assert [x["step"] for x in lines] == [10, 20, 30]
    assert [x["attempt"] for x in lines] == [1, 2, 3]
    last = lines[-1]
    assert sorted(last["grid"]) == [0, 1, 2]
    assert len(last["energies"]) == 3 and all(len(e) == 3 for e in last["energies"])
    off = t["site_off"]
    assert [len(s) for s in last["states"]] == [off[r + 1] - off[r] for r in range(3)]
    assert np.array_equal(np.array(last["states"][0]), sim.state[off[0]:off[1]].cpu().numpy())
    assert sum(sum(row) for row in last["ex_attempts"]) == int(sim.ex_count[:, 0].sum())
    assert all(np.isfinite(e) for row in last["energies"] for e in row)


@pytest.mark.parametrize("n_pH,n_E,ex_every", [(2, 2, 2), (1, 3, 0)])
def test_occupancy_counts_match_a_host_tally(pkg, n_pH, n_E, ex_every):
    """gb_md_state.occ_count against the states and the grid read after
    every step: one count per site and halt, at the state's column and the
    row of the grid slot its replica holds (the replica itself without
    exchanges); Simulation.occupancy gives the fractions."""
    import torch
    device()
    M = n_pH * n_E
    rep = synth.make_replica(160, 71, [(1, 10, 2), (0, 8, 3), (0, 6, 2)])
    E_lad = synth.e_ladder(n_E, half_width=0.03)
    pH_lad = np.linspace(4.6, 5.0, n_pH)
    b = synth.Batch([rep] * M, pH=np.repeat(pH_lad, n_E), E=np.tile(E_lad, n_pH))
    one = synth.Batch([rep], pH=b.pH[:1], E=b.E[:1])
    t = b.site_tables(np.tile(oracle.site_reference_energies(one, oracle_params()), M))
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         sites=t, pH=b.pH, E=b.E, E_ladder=E_lad, pH_ladder=pH_lad, mc_every=1,
                         ex_every=ex_every or 100, seed=9, occupancy=True)
    if not ex_every:
        sim.st.ex_every = 0
    S = 2 + 3 + 2
    want = np.zeros((M, S), np.int64)
    cols = np.array([0, 2, 5])                    # first column of each site of a replica
    for _ in range(30):
        sim.run(1)
        st = sim.state.cpu().numpy().reshape(M, 3)
        grid = sim.grid.cpu().numpy()
        slot = np.argsort(grid) if ex_every else np.arange(M)   # replica -> slot
        for r in range(M):
            want[slot[r], cols + st[r]] += 1
    sim.sync()
    assert np.array_equal(sim.occ.cpu().numpy(), want)
    frac = sim.occupancy()
    assert np.allclose(frac, want / 30.0)
    assert np.allclose(frac[:, 0] + frac[:, 1], 1.0)           # the redox site is in one of its states
