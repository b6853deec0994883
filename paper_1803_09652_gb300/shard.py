"""Replica ensembles split over processes, one GPU each: the replica exchange
of Sec. II.C (Eq. 14-15) and Sec. III.B across ranks.

Replicas are independent between exchanges (each runs its own MD and Monte
Carlo), so an ensemble of M replicas shards by replica.  Rank k owns the
contiguous block [bounds[k], bounds[k+1]) of the ensemble's replicas and runs
them as one batch of its own (gb_md_segment), with rep_base = bounds[k] so
that every replica draws the random numbers it would draw in a single batch.

An exchange needs, from every replica, one integer: its bound electrons
(along the E ladder) or protons (along pH).  The ranks all-gather these int32
counts, one collective of M integers per exchange.  Every rank then holds the
same global grid, counts, attempt number and seed, and runs the same exchange
kernel (eremd_exchange) on them, so all ranks take the same decisions with no
further message; each rank then reads the new E and pH of its own replicas.

Host logic and collectives only: the counts, the decisions and the label
updates run in the library's kernels (gb_count_bound, eremd_exchange).
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

import numpy as np


def shard_bounds(M: int, world: int) -> list:
    """Replica block boundaries: rank k owns [b[k], b[k+1]), sizes differing
    by at most one, larger blocks first."""
    if world < 1 or M < 0:
        raise ValueError("need world >= 1 and M >= 0")
    q, r = divmod(M, world)
    b = [0]
    for k in range(world):
        b.append(b[-1] + q + (1 if k < r else 0))
    return b


def slice_sites(t: dict, r0: int, r1: int) -> dict:
    """The site tables of replicas [r0, r1) of a batch, rebased to a batch of
    their own (same layout as synth.Batch.site_tables; atom indices are
    replica-local and stay as they are)."""
    so = np.asarray(t["site_off"])
    s0, s1 = int(so[r0]), int(so[r1])
    aoff = np.asarray(t["site_atom_off"])
    soff = np.asarray(t["site_state_off"])
    qoff = np.asarray(t["site_q_off"])
    i32 = lambda v: np.ascontiguousarray(v, dtype=np.int32)
    return dict(
        n_sites=s1 - s0,
        site_off=i32(so[r0:r1 + 1] - s0),
        site_kind=i32(t["site_kind"][s0:s1]),
        site_nstates=i32(t["site_nstates"][s0:s1]),
        site_atom_off=i32(aoff[s0:s1 + 1] - aoff[s0]),
        site_atom_idx=i32(t["site_atom_idx"][aoff[s0]:aoff[s1]]),
        site_state_off=i32(soff[s0:s1 + 1] - soff[s0]),
        site_q_off=i32(qoff[s0:s1 + 1] - qoff[s0]),
        q_state=np.ascontiguousarray(t["q_state"][qoff[s0]:qoff[s1]], dtype=np.float32),
        n_H=i32(t["n_H"][soff[s0]:soff[s1]]),
        n_e=i32(t["n_e"][soff[s0]:soff[s1]]),
        G_ref=np.ascontiguousarray(t["G_ref"][soff[s0]:soff[s1]], dtype=np.float64),
        pKa_ref=np.ascontiguousarray(t["pKa_ref"][s0:s1], dtype=np.float64),
        E0_ref=np.ascontiguousarray(t["E0_ref"][s0:s1], dtype=np.float64),
    )


def exchange_dim(attempt: int, ex_dim: int) -> int:
    """0 (E ladder) or 1 (pH ladder) for this attempt: ex_dim 0 and 1 fix the
    dimension, 2 alternates by pairs of attempts (E when floor(k/2) is even),
    the schedule of the MD driver's own exchange."""
    if ex_dim in (0, 1):
        return ex_dim
    return 0 if ((attempt >> 1) & 1) == 0 else 1


class ShardedLadder:
    """The exchange grid of an ensemble split over the ranks of a
    torch.distributed process group.

    n_pH x n_E grid, replica p * n_E + e starting at (pH row p, E column e),
    as in the single-batch driver.  Every rank keeps the whole grid (slot ->
    replica), the per-replica E and pH and the attempt counter, identical on
    all ranks.  exchange(n_e_local, n_H_local) gathers the counts, runs one
    exchange attempt on the whole grid and returns the new E and pH of this
    rank's replicas.

    exchange_fn: the decision kernel, called as
      exchange_fn(values, rep_at_slot, n_count, dim, attempt, seed, kT, wrap,
                  n_ladders, ladder_len, ladder_stride, slot_stride, value_of_rep)
    on tensors of `device`; the default is the library's eremd_exchange.
    gather_fn: all-gather of equal-length int32 tensors (default
    torch.distributed.all_gather on the group; tensors on the CPU for gloo,
    on `device` for NCCL)."""

    def __init__(self, n_pH: int, n_E: int, E_ladder: Sequence[float], pH_ladder: Sequence[float], *,
                 rank: int, world: int, kT: float, seed: int = 0, ex_dim: Optional[int] = None,
                 wrap: bool = True, device=None, group=None,
                 exchange_fn: Optional[Callable] = None, gather_fn: Optional[Callable] = None):
        import torch
        self.n_pH, self.n_E = int(n_pH), int(n_E)
        self.M = self.n_pH * self.n_E
        if len(E_ladder) != self.n_E or len(pH_ladder) != self.n_pH:
            raise ValueError("ladder lengths do not match the grid")
        self.rank, self.world = int(rank), int(world)
        self.bounds = shard_bounds(self.M, self.world)
        self.kT, self.seed, self.wrap = float(kT), int(seed), bool(wrap)
        self.ex_dim = (2 if self.n_pH > 1 else 0) if ex_dim is None else int(ex_dim)
        self.device = torch.device("cpu") if device is None else torch.device(device)
        self.group = group
        f64 = dict(dtype=torch.float64, device=self.device)
        self.E_ladder = torch.as_tensor(np.asarray(E_ladder, np.float64), **f64)
        self.pH_ladder = torch.as_tensor(np.asarray(pH_ladder, np.float64), **f64)
        self.grid = torch.arange(self.M, dtype=torch.int32, device=self.device)
        self.E_rep = self.E_ladder.repeat(self.n_pH).clone()
        self.pH_rep = self.pH_ladder.repeat_interleave(self.n_E).clone()
        self.attempt = 0
        self._exchange = exchange_fn or _library_exchange
        self._gather = gather_fn or self._dist_gather

    def local_range(self):
        return self.bounds[self.rank], self.bounds[self.rank + 1]

    def _dist_gather(self, local):
        import torch
        import torch.distributed as dist
        comm = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(self.group) == "nccl" \
            else torch.device("cpu")
        width = max(b - a for a, b in zip(self.bounds[:-1], self.bounds[1:]))
        buf = torch.full((width,), -2, dtype=torch.int32, device=comm)
        buf[:local.numel()] = local.to(comm)
        parts = [torch.empty_like(buf) for _ in range(self.world)]
        dist.all_gather(parts, buf, group=self.group)
        return torch.cat([p[:b - a] for p, a, b in zip(parts, self.bounds[:-1], self.bounds[1:])])

    def gather_counts(self, local):
        """The counts of every replica, in replica order (int32 [M])."""
        import torch
        r0, r1 = self.local_range()
        local = torch.as_tensor(local).to(torch.int32).reshape(-1)
        if local.numel() != r1 - r0:
            raise ValueError(f"rank {self.rank} holds {r1 - r0} replicas, got {local.numel()} counts")
        full = self._gather(local).to(self.device)
        if bool((full < 0).any()):
            raise RuntimeError("a replica reports a site in a state outside its table (count < 0)")
        return full

    def exchange(self, n_e_local, n_H_local):
        """One exchange attempt over the whole grid; returns (E, pH) of this
        rank's replicas (float64 tensors on `device`)."""
        dim = exchange_dim(self.attempt, self.ex_dim)
        counts = self.gather_counts(n_e_local if dim == 0 else n_H_local)
        if dim == 0:
            self._exchange(self.E_ladder, self.grid, counts, 0, self.attempt, self.seed, self.kT, self.wrap,
                           self.n_pH, self.n_E, self.n_E, 1, self.E_rep)
        else:
            self._exchange(self.pH_ladder, self.grid, counts, 1, self.attempt, self.seed, self.kT, self.wrap,
                           self.n_E, self.n_pH, 1, self.n_E, self.pH_rep)
        self.attempt += 1
        r0, r1 = self.local_range()
        return self.E_rep[r0:r1], self.pH_rep[r0:r1]


def _library_exchange(values, rep_at_slot, n_count, dim, attempt, seed, kT, wrap, n_ladders, ladder_len,
                      ladder_stride, slot_stride, value_of_rep):
    from . import eremd_exchange
    eremd_exchange(values, rep_at_slot, n_count, dim, attempt, seed, kT, wrap=wrap, n_ladders=n_ladders,
                   ladder_len=ladder_len, ladder_stride=ladder_stride, slot_stride=slot_stride,
                   value_of_rep=value_of_rep)


class ShardedSimulation:
    """One rank's part of a C(pH,E)-REMD ensemble split over processes.

    Every rank passes the same global description: atom_off [M+1], xyzq
    [N, 4], rad_screen [N, 2], the site tables (synth layout), and the ladders
    of the n_pH x n_E grid (M = n_pH n_E, replica p * n_E + e starting at pH
    row p, E column e).  The rank runs its block of replicas as a Simulation
    with rep_base at the block's first replica, exchanges switched off inside
    the batch, and after every ex_every MD steps takes part in one exchange
    over the whole grid (ShardedLadder).  The result equals, replica by
    replica and bit for bit, the single-batch Simulation of the whole ensemble
    with the same arguments."""

    def __init__(self, atom_off, xyzq, rad_screen, params, sites: dict, E_ladder, pH_ladder, *, rank: int,
                 world: int, seed: int = 0, mc_every: int = 10, ex_every: int = 100, ex_dim=None,
                 wrap: bool = True, mc_mode: int = 0, temperature: float = 300.0, device: int = 0, group=None,
                 **md_kw):
        from . import KB, Simulation
        E_ladder = np.asarray(E_ladder, np.float64)
        pH_ladder = np.asarray(pH_ladder, np.float64)
        n_E, n_pH = len(E_ladder), len(pH_ladder)
        atom_off = np.asarray(atom_off, np.int64)
        M = len(atom_off) - 1
        if n_E * n_pH != M:
            raise ValueError("the grid must hold every replica once")
        if ex_every <= 0 or (mc_every > 0 and ex_every % mc_every):
            raise ValueError("ex_every must be a positive multiple of mc_every")
        self.ladder = ShardedLadder(n_pH, n_E, E_ladder, pH_ladder, rank=rank, world=world,
                                    kT=KB * temperature, seed=seed, ex_dim=ex_dim, wrap=wrap,
                                    device=f"cuda:{device}", group=group)
        r0, r1 = self.ladder.local_range()
        a0, a1 = int(atom_off[r0]), int(atom_off[r1])
        E_rep = np.tile(E_ladder, n_pH)[r0:r1]
        pH_rep = np.repeat(pH_ladder, n_E)[r0:r1]
        self.sim = Simulation(atom_off[r0:r1 + 1] - a0, np.asarray(xyzq)[a0:a1], np.asarray(rad_screen)[a0:a1],
                              params, sites=slice_sites(sites, r0, r1), pH=pH_rep, E=E_rep,
                              E_ladder=E_rep[:1], pH_ladder=pH_rep[:1], seed=seed, mc_every=mc_every,
                              ex_every=0, wrap=wrap, mc_mode=mc_mode, temperature=temperature,
                              device=device, rep_base=r0, **md_kw)
        self.ex_every = int(ex_every)
        self.replicas = (r0, r1)

    @property
    def step(self) -> int:
        return self.sim.step

    def run(self, nsteps: int) -> "ShardedSimulation":
        """nsteps MD steps (a multiple of ex_every), each block of ex_every
        steps followed by one exchange over the whole grid."""
        from . import count_bound
        if nsteps % self.ex_every or self.sim.step % self.ex_every:
            raise ValueError("run in whole exchange periods")
        for _ in range(nsteps // self.ex_every):
            self.sim.run(self.ex_every)
            n_e = count_bound(self.sim.sites, self.sim.state, 1)
            n_H = count_bound(self.sim.sites, self.sim.state, 0)
            E, pH = self.ladder.exchange(n_e, n_H)
            self.sim.E.copy_(E)
            self.sim.pH.copy_(pH)
        return self
