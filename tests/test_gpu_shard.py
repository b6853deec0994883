"""An ensemble split over two processes (ShardedSimulation, gloo group) on the
library's kernels, against the single-batch Simulation of the whole ensemble:
coordinates, velocities, site states, E and pH of every replica identical bit
for bit after 20 exchange periods (MD, Monte Carlo every 5 steps, exchanges
every 10, on a 2 x 3 (pH x E) grid of uneven replicas).

Both ranks run on the one GPU of this run.  They never wait on each other on
the device: the only exchange between them is the all-gather of the counts on
the host (gloo), between their kernel launches."""
import json
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from gpu_common import device, oracle_params

pytestmark = pytest.mark.gpu

N_PH, N_E = 2, 3
SIZES = [180, 120, 260, 90, 150, 210]


def _ensemble():
    b = synth.random_batch(SIZES, seed=71)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    E_lad = synth.e_ladder(N_E, half_width=0.03)
    pH_lad = np.array([4.6, 5.0])
    return b, t, E_lad, pH_lad


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    import paper_1803_09652_gb300 as pkg
    from paper_1803_09652_gb300.shard import ShardedSimulation
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, t, E_lad, pH_lad = _ensemble()
    sim = ShardedSimulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                            t, E_lad, pH_lad, rank=rank, world=world, seed=8, mc_every=5, ex_every=10)
    sim.run(200)
    sim.sim.sync()
    s = sim.sim
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), xyzq=s.xyzq.cpu().numpy(), vel=s.vel.cpu().numpy(),
             state=s.state.cpu().numpy(), E=s.E.cpu().numpy(), pH=s.pH.cpu().numpy(),
             grid=sim.ladder.grid.cpu().numpy(), replicas=np.array(sim.replicas))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_ensemble_equals_the_single_batch(tmp_path):
    device()                                   # skips without a GPU
    import __graft_entry__
    __graft_entry__.build()
    import torch
    import torch.multiprocessing as mp
    import paper_1803_09652_gb300 as pkg
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    b, t, E_lad, pH_lad = _ensemble()
    pH = np.repeat(pH_lad, N_E)
    E = np.tile(E_lad, N_PH)
    ref = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         sites=t, pH=pH, E=E, E_ladder=E_lad, pH_ladder=pH_lad, seed=8, mc_every=5, ex_every=10)
    ref.run(200)
    ref.sync()
    assert int(ref.st.attempt) == 20
    off = b.atom_off
    so = t["site_off"]
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    assert [tuple(p["replicas"]) for p in parts] == [(0, 3), (3, 6)]
    for p in parts:
        r0, r1 = p["replicas"]
        a0, a1 = off[r0], off[r1]
        assert np.array_equal(p["grid"], ref.grid.cpu().numpy())
        assert np.array_equal(p["xyzq"], ref.xyzq[a0:a1].cpu().numpy())
        assert np.array_equal(p["vel"], ref.vel[a0:a1].cpu().numpy())
        assert np.array_equal(p["state"], ref.state[so[r0]:so[r1]].cpu().numpy())
        assert np.array_equal(p["E"], ref.E[r0:r1].cpu().numpy())
        assert np.array_equal(p["pH"], ref.pH[r0:r1].cpu().numpy())
    # the exchanges moved replicas across the rank boundary
    assert not np.array_equal(ref.grid.cpu().numpy(), np.arange(N_PH * N_E))
