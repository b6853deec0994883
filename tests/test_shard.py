"""Host logic of replica ensembles split over processes (paper_1803_09652_gb300.shard),
on CPU: block bounds, site-table slicing, the exchange schedule, and a
world-size-2 gloo run in which two ranks, each holding half of the grid,
reproduce attempt by attempt the oracle's exchange over the whole grid.

In these CPU tests the oracle's exchange stands in for the library's
eremd_exchange kernel (the decision maker is injected); what is under test is
the sharding around it: who owns which replica, the gather of the counts in
replica order, the attempt counter, the E / pH alternation and strides, and
the new E and pH each rank reads back.  The GPU test (test_gpu_shard.py) runs
the library's kernels."""
import json
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_1803_09652_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KT = oracle.KB * 300.0


def test_shard_bounds_cover_every_replica_once():
    for M in (0, 1, 7, 8, 48, 64):
        for world in (1, 2, 3, 8):
            b = shard.shard_bounds(M, world)
            assert b[0] == 0 and b[-1] == M and len(b) == world + 1
            sizes = np.diff(b)
            assert sizes.min() >= 0 and sizes.max() - sizes.min() <= 1
            assert list(sizes) == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard.shard_bounds(4, 0)


def _site_view(t, s):
    """Everything the tables say about site s (of its own batch)."""
    a0, a1 = t["site_atom_off"][s], t["site_atom_off"][s + 1]
    k0, k1 = t["site_state_off"][s], t["site_state_off"][s + 1]
    q0, q1 = t["site_q_off"][s], t["site_q_off"][s + 1]
    return (int(t["site_kind"][s]), int(t["site_nstates"][s]), tuple(t["site_atom_idx"][a0:a1]),
            tuple(t["n_H"][k0:k1]), tuple(t["n_e"][k0:k1]), tuple(t["G_ref"][k0:k1]),
            tuple(t["q_state"][q0:q1]), float(t["pKa_ref"][s]), float(t["E0_ref"][s]))


def test_slice_sites_keeps_every_replicas_sites():
    b = synth.config_uneven(n_rep=7, seed=5, n_min=400, n_max=900)
    t = b.site_tables(np.arange(b.site_tables()["site_state_off"][-1], dtype=np.float64))
    for r0, r1 in ((0, 7), (0, 3), (3, 7), (2, 5), (6, 7), (4, 4)):
        u = shard.slice_sites(t, r0, r1)
        assert u["n_sites"] == t["site_off"][r1] - t["site_off"][r0]
        assert len(u["site_off"]) == r1 - r0 + 1 and u["site_off"][0] == 0
        for r in range(r0, r1):
            sites_t = range(t["site_off"][r], t["site_off"][r + 1])
            sites_u = range(u["site_off"][r - r0], u["site_off"][r - r0 + 1])
            assert [_site_view(t, s) for s in sites_t] == [_site_view(u, s) for s in sites_u]


def test_exchange_dim_alternates_by_pairs():
    assert [shard.exchange_dim(k, 2) for k in range(8)] == [0, 0, 1, 1, 0, 0, 1, 1]
    assert all(shard.exchange_dim(k, 0) == 0 and shard.exchange_dim(k, 1) == 1 for k in range(8))


def _oracle_exchange_fn(values, rep_at_slot, n_count, dim, attempt, seed, kT, wrap, n_ladders, ladder_len,
                        ladder_stride, slot_stride, value_of_rep):
    """The oracle's exchange in the place of the library kernel (CPU tensors,
    updated in place), with the kernel's value_of_rep output."""
    g = rep_at_slot.numpy()
    oracle.exchange(values.numpy(), g, n_count.numpy().astype(np.int32), dim, attempt, seed, kT, wrap=wrap,
                    n_ladders=n_ladders, ladder_len=ladder_len, ladder_stride=ladder_stride,
                    slot_stride=slot_stride)
    for l in range(n_ladders):
        for k in range(ladder_len):
            value_of_rep[int(g[l * ladder_stride + k * slot_stride])] = float(values[k])


def _counts(M, attempt):
    """Bound electrons and protons of every replica at this attempt (a fixed
    pseudo-random table, as site states would give)."""
    rng = np.random.default_rng(1000 + attempt)
    return rng.integers(0, 5, M).astype(np.int32), rng.integers(0, 9, M).astype(np.int32)


def _rank_main(rank, world, port, out_dir, n_pH, n_E, ex_dim, wrap, attempts):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lad = shard.ShardedLadder(n_pH, n_E, synth.e_ladder(n_E, half_width=0.04), np.linspace(4.2, 5.4, n_pH),
                              rank=rank, world=world, kT=KT, seed=21, ex_dim=ex_dim, wrap=wrap,
                              exchange_fn=_oracle_exchange_fn)
    r0, r1 = lad.local_range()
    hist = []
    for k in range(attempts):
        n_e, n_H = _counts(n_pH * n_E, k)
        E, pH = lad.exchange(torch.as_tensor(n_e[r0:r1]), torch.as_tensor(n_H[r0:r1]))
        hist.append({"grid": lad.grid.tolist(), "E": E.tolist(), "pH": pH.tolist()})
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"range": [r0, r1], "hist": hist}, f)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_pH,n_E,ex_dim,wrap", [(1, 8, 0, True), (2, 4, 2, True), (3, 3, 2, False)])
def test_two_ranks_reproduce_the_oracle_exchange_on_the_whole_grid(tmp_path, n_pH, n_E, ex_dim, wrap):
    import torch.multiprocessing as mp
    attempts = 36
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path), n_pH, n_E, ex_dim, wrap, attempts),
                       nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert res[0]["range"] == [0, (n_pH * n_E + 1) // 2] and res[1]["range"][1] == n_pH * n_E
    # the whole grid, one process, the oracle's exchange attempt after attempt
    M = n_pH * n_E
    E_lad, pH_lad = synth.e_ladder(n_E, half_width=0.04), np.linspace(4.2, 5.4, n_pH)
    grid = np.arange(M, dtype=np.int32)
    swaps = 0
    for k in range(attempts):
        n_e, n_H = _counts(M, k)
        dim = shard.exchange_dim(k, ex_dim)
        before = grid.copy()
        if dim == 0:
            oracle.exchange(E_lad, grid, n_e, 0, k, 21, KT, wrap=wrap, n_ladders=n_pH, ladder_len=n_E,
                            ladder_stride=n_E, slot_stride=1)
        else:
            oracle.exchange(pH_lad, grid, n_H, 1, k, 21, KT, wrap=wrap, n_ladders=n_E, ladder_len=n_pH,
                            ladder_stride=1, slot_stride=n_E)
        swaps += int(np.count_nonzero(grid != before))
        E_rep = np.empty(M)
        pH_rep = np.empty(M)
        E_rep[grid] = np.tile(E_lad, n_pH)
        pH_rep[grid] = np.repeat(pH_lad, n_E)
        for r in res:
            h = r["hist"][k]
            r0, r1 = r["range"]
            assert h["grid"] == grid.tolist(), (k, r["range"])
            assert h["E"] == E_rep[r0:r1].tolist() and h["pH"] == pH_rep[r0:r1].tolist(), k
    assert swaps >= 10            # accepted exchanges happened, across the rank boundary too


def test_negative_counts_are_refused():
    import torch
    lad = shard.ShardedLadder(1, 4, synth.e_ladder(4), [7.0], rank=0, world=1, kT=KT,
                              exchange_fn=_oracle_exchange_fn, gather_fn=lambda x: x)
    with pytest.raises(RuntimeError, match="outside its table"):
        lad.exchange(torch.tensor([1, -1, 0, 2], dtype=torch.int32), torch.zeros(4, dtype=torch.int32))
    with pytest.raises(ValueError):
        lad.exchange(torch.zeros(3, dtype=torch.int32), torch.zeros(3, dtype=torch.int32))
