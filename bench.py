"""Benchmark of the GB / C(pH,E)MD / E-REMD hot path on one GB300.

Default workload: the 2-D C(pH,E) grid, 6 pH x 8 E = 48 replicas of
25,000-atom compact chains with 40 titratable sites each (8 redox, 32 pH with
2-4 states), exchanges alternating along E and pH; Langevin 2 fs with GB +
Coulomb + chain bonds + soft repulsion, MC attempt (protonation then redox)
every 10 steps, neighbour exchange every 100 steps.  One bench "step" = one
exchange period: 100 MD steps of every replica, 10 MC rounds, 1 exchange, run
through gb_md_segment (captured CUDA graphs).  --workload picks one of the
other configurations (8 x 2048 E-REMD batch, 16 x 4096, uneven 64, a
100,000-atom chain with cutoffs).

Headline metric: GB pair-interactions/s = sum_r N_r (N_r - 1)/2 per MD step
x MD steps / device seconds (each MD step evaluates all pairs in three passes).
Also reported: replica MD-steps/s, the plain form (one context and one launch
sequence per replica, no graph), the dominant pass's FP32 roofline, an
end-to-end number through gb_md_segment_host with the state in pinned host
memory, and the FP64 oracle on host cores.

--impl reference times the FP64 CPU oracle (the reference arm)
on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

MD_PER_STEP = 100          # MD steps per bench step (one exchange period)
MC_EVERY, EX_EVERY = 10, 100
FP32_LANES = 128           # FP32 lanes per SM
# Algorithmic FP32 flops per unordered pair and pass (FMA = 2, add / mul = 1;
# MUFU ops counted apart), counted on the far-field arithmetic every disjoint
# pair needs (short polynomials); pairs in near blocks cost more, so these
# figures are a lower bound of the FP32 work done.
FLOPS_PER_PAIR = {"born": 34.0, "energy": 43.0, "chain": 51.0}
MUFU_PER_PAIR = {"born": 1, "energy": 3, "chain": 1}
PASS_NAMES = ["born", "energy", "chain"]


WORKLOADS = ("grid_48x25000", "eremd_8x2048", "diff_16x4096", "uneven_64", "cutoff_1x100000")
DEFAULT_WORKLOAD = "grid_48x25000"
# GB with cutoffs: Born-radius cutoff and pair cutoff (A) of the cutoff workload
CUTOFFS = {"cutoff_1x100000": dict(rgbmax=12.0, cut=12.0)}


def workload(name=DEFAULT_WORKLOAD):
    """The batch of a named configuration (the headline is the 2-D grid, the
    largest single-GPU configuration; the others are benched on request)."""
    import synth
    if name == "eremd_8x2048":
        return synth.config_eremd(8, 2048, seed=0)
    if name == "diff_16x4096":
        return synth.config_diff(16, 4096)
    if name == "uneven_64":
        return synth.config_uneven()
    if name == "grid_48x25000":
        return synth.config_grid()
    if name == "cutoff_1x100000":
        return synth.config_cutoff(100000)
    raise ValueError(name)


def est_md_step_s(b):
    """Rough seconds per MD step of the batched form (about 2.5e11 pair
    interactions/s), used only to size the untimed and auxiliary regions."""
    return max(b.pairs_per_eval(), 1) / 2.5e11


def bench_config(name, b, pairs_md):
    """The workload as both arms report it (identical dicts)."""
    return {"workload": name, "replicas": b.n_rep, "atoms_total": b.n_atoms,
            "md_steps_per_step": MD_PER_STEP, "mc_every": MC_EVERY, "exchange_every": EX_EVERY,
            "pairs_per_md_step": pairs_md, "cutoffs_A": CUTOFFS.get(name),
            "pairs_counted": "within the pair cutoff at the start" if name in CUTOFFS else "all pairs",
            "l2": "flushed between GPU steps (256 MB write)", "parallelism": "replicas"}


def pairs_per_md_step(b, name):
    """Pair terms of one force evaluation: all pairs, or with a pair cutoff
    the pairs within it at the starting coordinates."""
    import synth
    cut = CUTOFFS.get(name, {}).get("cut", 0.0)
    return synth.pairs_within(b, cut) if cut > 0 else b.pairs_per_eval()


# ----------------------------------------------------------------------------------
# clocks during the timed region
class ClockSampler:
    def __init__(self, gpu_index=0):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for s in self.samples for n, v in zip(names, s[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ----------------------------------------------------------------------------------
def _oracle_md_worker(job):
    """One host process: the FP64 oracle's BAOAB MD step (force evaluation of
    GB + Coulomb + restraints, then the update) of replica 0 of the workload,
    n_steps times.  First, untimed: the forces at the starting coordinates and
    `warm` MD steps (the process's warm-up).  Returns (MD steps, timed
    seconds, pair interactions per MD step)."""
    name, n_steps, warm, seed = job
    import oracle
    import synth
    oracle.build()
    b = workload(name)
    sb = synth.Batch([b.replicas[0]], pH=b.pH[:1], E=b.E[:1])
    x, q, rho, scr, off = oracle.batch_arrays(sb)
    v = np.zeros_like(x)
    p = oracle.default_params(rep_k=100.0, rep_sigma=2.5, **CUTOFFS.get(name, {}))
    F, _ = oracle.forces_all(off, x, q, rho, scr, p)
    for k in range(warm):
        oracle.md_step(off, x, v, q, rho, scr, F, seed, k + 1, p)
    t0 = time.perf_counter()
    for k in range(warm, warm + n_steps):
        oracle.md_step(off, x, v, q, rho, scr, F, seed, k + 1, p)
    pairs = pairs_per_md_step(sb, name)
    return n_steps, time.perf_counter() - t0, pairs


def oracle_throughput(name, n_steps, procs, warmup=0):
    """The oracle as it stands on host cores: n_steps MD steps of one replica
    of the workload (replicas are independent between exchanges), spread over
    `procs` spawned processes, one per core.  Each process first computes its
    starting forces (one force evaluation, untimed); when there are fewer
    processes than `warmup` steps, each also runs untimed MD steps until the
    processes' warm-up covers them.  The job's time is the slowest process's
    timed region (as the slowest rank's time on GPUs).  Returns
    (pair-interactions/s, MD steps, seconds, processes)."""
    import oracle
    oracle.build()
    procs = max(1, min(procs, n_steps))
    warm = -(-max(0, warmup - procs) // procs)
    jobs = [(name, n_steps // procs + (1 if k < n_steps % procs else 0), warm, 1 + k) for k in range(procs)]
    if procs == 1:
        res = [_oracle_md_worker(jobs[0])]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_md_worker, jobs)
    secs = max(r[1] for r in res)
    steps = sum(r[0] for r in res)
    return res[0][2] * steps / secs, steps, secs, procs


def synth_one(b):
    """The batch of replica 0 alone."""
    import synth
    return synth.Batch([b.replicas[0]], pH=b.pH[:1], E=b.E[:1])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def reference_arm(args):
    """The FP64 oracle on the host cores, on a bounded sample of the same
    workload: each bench step is one whole MD step of one replica of the
    workload (a 25,000-atom replica by default), the K steps spread over
    spawned processes (one per step up to twice the core count, else one per
    core) and timed in each process after its warm-up (the
    untimed force evaluation at the starting coordinates, one per process,
    which also covers the W warm-up steps when there are at least W
    processes)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload
    b = workload(name)
    pairs_md = pairs_per_md_step(b, name)
    # one process per timed step while that keeps every core busy (K steps on
    # C cores in ceil(K / C) rounds would leave cores idle in the last one)
    cores = host_cores()
    procs = args.steps if args.steps <= 2 * cores else cores
    rate, steps, secs, procs = oracle_throughput(name, args.steps, procs, args.warmup)
    rep_n = b.replicas[0].n
    sample = (f"{steps} BAOAB MD steps (GB + Coulomb + restraint forces) of one {rep_n}-atom replica "
              f"of the workload, spread over {procs} spawned processes on {cores} cores; time = the "
              f"slowest process's timed steps")
    line = {
        "impl": "reference", "metric": "GB pair-interactions/s", "value": rate,
        "unit": "pair-interactions/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * secs / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(name, b, pairs_md),
        "sample": sample,
        "cpu_baseline": {"value": rate, "unit": "pair-interactions/s", "cores": min(procs, cores),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(name):
    """The oracle on a bounded sample of the workload: MD steps of one
    replica in one process per host core (each after its untimed starting
    force evaluation), about ten seconds of them per process (at least one
    step; the oracle does about 6.5e6 pair interactions per second on a
    core)."""
    cores = host_cores()
    b = workload(name)
    per = max(1, int(round(10.0 * 6.5e6 / max(pairs_per_md_step(synth_one(b), name), 1))))
    rate, steps, secs, procs = oracle_throughput(name, cores * per, cores)
    return {"value": rate, "unit": "pair-interactions/s", "cores": procs, "kind": "oracle",
            "sample": f"{steps} BAOAB MD steps (GB + Coulomb + restraint forces) of one "
                      f"{b.replicas[0].n}-atom replica of the workload, {per} per process on {procs} "
                      f"cores, {secs:.1f} s"}


# ----------------------------------------------------------------------------------
class Setup:
    """Device state of the workload and the gb_md_state that points at it."""

    def __init__(self, pkg, batch, dev, seed, params, G=None):
        import torch
        self.pkg, self.b, self.dev = pkg, batch, dev
        self.ctx = pkg.Context(batch.atom_off, params)
        N, M = batch.n_atoms, batch.n_rep
        self.xyzq = torch.as_tensor(batch.xyzq(), device=dev)
        self.rad = torch.as_tensor(batch.rad_screen(), device=dev)
        self.vel = torch.zeros((N, 4), dtype=torch.float32, device=dev)
        self.force = torch.zeros((N, 4), dtype=torch.float32, device=dev)
        self.R = torch.zeros(N, dtype=torch.float32, device=dev)
        if G is None:
            G = site_reference_energies_gpu(pkg, batch, dev, params)
        self.tables = batch.site_tables(G)
        self.sites = pkg.SiteTables(self.tables, M, dev)
        self.state = torch.zeros(self.tables["n_sites"], dtype=torch.int32, device=dev)
        self.pH = torch.as_tensor(batch.pH.copy(), device=dev)
        self.E = torch.as_tensor(batch.E.copy(), device=dev)
        E_lad = batch.E_ladder if batch.E_ladder is not None else batch.E[:1]
        pH_lad = batch.pH_ladder if batch.pH_ladder is not None else batch.pH[:1]
        self.E_ladder = torch.as_tensor(np.asarray(E_lad, np.float64), device=dev)
        self.pH_ladder = torch.as_tensor(np.asarray(pH_lad, np.float64), device=dev)
        self.grid = torch.arange(M, dtype=torch.int32, device=dev)   # replica p * n_E + e at (p, e)
        # exchanges need a full ladder (or grid) of replicas; otherwise none
        n_E, n_pH = len(E_lad), len(pH_lad)
        ladder_ok = n_E * n_pH == M and M > 1
        st = pkg.MDState()
        st.xyzq, st.vel, st.force = self.xyzq.data_ptr(), self.vel.data_ptr(), self.force.data_ptr()
        st.rad_screen, st.R = self.rad.data_ptr(), self.R.data_ptr()
        st.state, st.pH, st.E = self.state.data_ptr(), self.pH.data_ptr(), self.E.data_ptr()
        st.grid, st.E_ladder, st.pH_ladder = (self.grid.data_ptr(), self.E_ladder.data_ptr(),
                                              self.pH_ladder.data_ptr())
        st.n_E, st.n_pH = (n_E, n_pH) if ladder_ok else (M, 1)
        st.dt, st.friction, st.mass, st.kT = 0.002, 10.0, 12.0, pkg.KB * 300.0
        st.bond_k, st.bond_r0 = 300.0, 1.5
        st.seed, st.step, st.attempt = seed, 0, 0
        st.mc_every, st.ex_every, st.wrap = MC_EVERY, EX_EVERY if ladder_ok else 0, 1
        st.ex_dim = 2 if n_pH > 1 else 0          # alternate E and pH lines on a 2-D grid
        self.st = st
        self.ctx.md_init(st)


def site_reference_energies_gpu(pkg, batch, dev, params):
    """G_ref(s) = E_elec(q(s)) - E_elec(q(0)) at the starting conformation, from
    gb_energy_forces (GB + Coulomb, repulsion excluded) on the device."""
    import torch
    t = batch.site_tables()
    G = np.zeros(t["site_state_off"][-1])
    p0 = pkg.default_params(alpha=params.alpha, beta=params.beta, gamma=params.gamma,
                            offset=params.offset, eps_in=params.eps_in, eps_out=params.eps_out)
    cache = {}
    for r, rep in enumerate(batch.replicas):
        key = id(rep)
        if key in cache:
            lo = t["site_off"][r]
            G[t["site_state_off"][lo]:t["site_state_off"][t["site_off"][r + 1]]] = cache[key]
            continue
        ctx = pkg.Context([0, rep.n], p0)
        base = np.zeros((rep.n, 4), np.float32)
        base[:, :3], base[:, 3] = rep.xyz, rep.q
        rad = torch.as_tensor(np.stack([rep.rho, rep.screen], 1).astype(np.float32), device=dev)

        def elec(qv):
            x = base.copy()
            x[:, 3] = qv
            E = ctx.energy_forces(torch.as_tensor(x, device=dev), rad, want=("E",))["E"]
            return float(E[0, 0] + E[0, 1])

        e0 = elec(rep.q)
        vals = []
        for s in rep.sites:
            for k in range(s.n_states):
                qq = rep.q.copy()
                qq[s.atoms] = s.q_state[k]
                vals.append(elec(qq) - e0)
        lo = t["site_off"][r]
        G[t["site_state_off"][lo]:t["site_state_off"][t["site_off"][r + 1]]] = vals
        cache[key] = vals
        ctx.close()
    return G


def launches_per_segment(md_steps, persistent=True, cutoff=False):
    """Kernels of this library enqueued by one gb_md_segment call of md_steps."""
    n_mc = md_steps // MC_EVERY
    mc = 4 * n_mc                                  # (slice rows + decision) x (protonation, redox)
    ex = 2 * (md_steps // EX_EVERY)                # exchange + attempt counter
    if persistent:
        md = n_mc                                  # one persistent launch per run between MC points
    else:
        # per step: 3 pair passes, 2 transforms, one close-and-open launch
        # (with a cutoff also the list reset and the block-list build);
        # plus the opening half step of the segment
        md = (8 if cutoff else 6) * md_steps + 1
    return 1 + md + mc + ex + 1                    # + set counters, + advance step counter


# ---- one process per GPU: replicas only (each rank runs its own batch) --------
def dist_init(backend):
    """Rank layout from the launcher's environment; a process group only for
    N > 1 (its barrier and max-over-ranks timing; no data-path collective)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(seconds, world, device):
    """The slowest rank's time: the whole job ends when it does."""
    if world == 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processed the same units (weak scaling)."""
    return units_per_rank * world / seconds


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=WORKLOADS,
                    help="configuration to run (default: the 2-D grid of 48 x 25,000-atom replicas)")
    ap.add_argument("--max-replicas", type=int, default=0,
                    help="keep only the first M replicas of the workload (small cases for profiler captures)")
    ap.add_argument("--persistent", action="store_true",
                    help="one persistent launch per run of MD steps instead of six launches per step")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch
    world, rank, local = dist_init("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_1803_09652_gb300 as pkg
    pkg.load()

    params = pkg.default_params(rep_k=100.0, rep_sigma=2.5, **CUTOFFS.get(args.workload, {}))
    b = workload(args.workload)
    if 0 < args.max_replicas < b.n_rep:
        import synth
        M = args.max_replicas
        b = synth.Batch(b.replicas[:M], pH=b.pH[:M], E=b.E[:M], name=b.name)
    S = Setup(pkg, b, dev, seed=1234 + rank, params=params)
    if not args.no_autotune:
        S.ctx.autotune(S.xyzq, S.rad)
        # register caps re-tuned on MD segments of this batch (state restored); trial
        # segments of about 50 ms at ~1.5e11 pair interactions/s
        est_step_s = 3.0 * max(b.pairs_per_eval(), 1) / 1.5e11
        S.ctx.autotune_md(S.st, S.sites, trial_steps=int(min(MD_PER_STEP, max(2, 0.05 / est_step_s))))
    persistent = args.persistent
    S.ctx.set_persistent(persistent)
    stream = torch.cuda.current_stream()
    pairs_md = pairs_per_md_step(b, args.workload)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    for _ in range(args.warmup):
        S.ctx.md_segment(S.st, S.sites, MD_PER_STEP)
    torch.cuda.synchronize()
    S.ctx.sync_status()

    # ---- timed region: K bench steps, L2 flushed between steps ------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        S.ctx.md_segment(S.st, S.sites, MD_PER_STEP)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    S.ctx.sync_status()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    dev_s = sum(step_ms) / 1000.0
    dev_s = max_over_ranks(dev_s, world, dev)
    value = job_rate(pairs_md * MD_PER_STEP * args.steps, world, dev_s)
    rep_steps = job_rate(b.n_rep * MD_PER_STEP * args.steps, world, dev_s)

    # ---- kernel timing: the same bench steps with CUDA events around every pair
    # pass (or persistent launch) inside the captured graph, on the graph's
    # stream.  Kept apart from the headline region, whose graph has no events
    # between kernels (they would break the programmatic launch edges).  About
    # two seconds of bench steps (at least one: 100 MD steps, 100 samples of
    # each pass).
    S.ctx.set_profiling(True)
    pass_ms = []
    n_prof = int(max(1, min(20, 2.0 / (est_md_step_s(b) * MD_PER_STEP))))
    for k in range(n_prof):
        flush.zero_()
        S.ctx.md_segment(S.st, S.sites, MD_PER_STEP)
        torch.cuda.synchronize()
        pass_ms.append(S.ctx.persist_times() if persistent else S.ctx.pass_times())
    S.ctx.set_profiling(False)
    S.ctx.sync_status()
    pm = np.mean(np.array(pass_ms), axis=0)

    # ---- roofline of the dominant kernel (FP32 ALU bound) ------------------------
    sm_max = (clk.get("sm_max_mhz") or 2070.0)
    peak = sm_count * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    sm_load = clk.get("sm_mhz") or sm_max
    peak_load = sm_count * FP32_LANES * 2 * sm_load * 1e6 / 1e12
    all_flops = pairs_md * sum(FLOPS_PER_PAIR.values())
    if persistent:
        # one launch runs pm[2] MD steps: three pair passes per step
        name = "k_md_persist"
        achieved = all_flops * pm[2] / (pm[1] * 1e-3) / 1e12
        timing = {"ms_per_md_step_in_kernel": float(pm[0]), "ms_per_launch": float(pm[1]),
                  "md_steps_per_launch": float(pm[2])}
    else:
        dom = int(np.argmax(pm))
        name = "k_pairs<%s>" % PASS_NAMES[dom]
        achieved = pairs_md * FLOPS_PER_PAIR[PASS_NAMES[dom]] / (pm[dom] * 1e-3) / 1e12
        timing = {"region": "a separate profiled region after the timed one: the same bench steps with CUDA "
                            "events around each pair pass on the graph's stream (the timed graph carries no "
                            "events; the events there break the programmatic launch overlap)",
                  "pass_ms": dict(zip(PASS_NAMES, [float(v) for v in pm])),
                  "pass_pairs_per_s": {k: pairs_md / (float(v) * 1e-3) for k, v in zip(PASS_NAMES, pm)},
                  "pass_tflops": {k: pairs_md * FLOPS_PER_PAIR[k] / (float(v) * 1e-3) / 1e12
                                  for k, v in zip(PASS_NAMES, pm)}}
    step_fp32 = all_flops * MD_PER_STEP * args.steps / dev_s / 1e12
    traffic = read_traffic(name, b.n_atoms) if args.workload == DEFAULT_WORKLOAD else None

    # ---- plain form: one context per replica, direct launches, no graph ---------
    plain = None
    if not args.no_plain and rank == 0:
        plain = plain_form(pkg, S, dev, params, pairs_md=pairs_md)

    # ---- end to end through gb_md_segment_host (state in pinned host memory) ----
    n_e2e = int(max(2, min(5, 10.0 / (est_md_step_s(b) * MD_PER_STEP))))
    e2e = end_to_end(pkg, S, n_bench=n_e2e, pairs_md=pairs_md)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(args.workload)

    if rank == 0:
        line = {
            "metric": "GB pair-interactions/s", "value": value, "unit": "pair-interactions/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * dev_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pairs, int64 fixed-point sums, f64 totals",
            "data": "synthetic",
            "config": bench_config(args.workload, b, pairs_md),
            "tuning": {"tiles": list(S.ctx.tiles()), "reg_caps": list(S.ctx.reg_caps()),
                       "sm_count": sm_count},
            "replica_md_steps_per_s": rep_steps,
            "kernel_timing": timing,
            "fp32_flops_per_pair": FLOPS_PER_PAIR,
            "mufu_per_pair": MUFU_PER_PAIR,
            "fp32_tflops_whole_step": step_fp32,
            "fp32_peak_frac_whole_step": step_fp32 / peak,
            "roofline": {"bound": "alu", "kernel": name, "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "frac_at_load_clock": achieved / peak_load, "traffic": traffic,
                         "peak_source": f"{sm_count} SMs (device properties) x {FP32_LANES} FP32 lanes x 2 x "
                                        f"{sm_max:.0f} MHz"},
            "plain": plain,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": launches_per_segment(MD_PER_STEP, persistent, args.workload in CUTOFFS) * args.steps,
            "md_kernel": "persistent (one launch per run between MC points)" if persistent else
                         ("eight launches per MD step (block neighbour list)" if args.workload in CUTOFFS
                          else "six launches per MD step"),
            "clocks": clk,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


PAIR_SOURCES = ("pairs_impl.cuh", "pairs.cu", "poly_coeffs.h", "common.cuh")


def pair_source_hash():
    """First 16 hex digits of the sha256 of the pair-kernel sources."""
    import hashlib
    h = hashlib.sha256()
    for f in PAIR_SOURCES:
        with open(os.path.join(ROOT, "paper_1803_09652_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(name, atoms_total):
    """DRAM bytes per launch of `name` from the committed ncu summary, scaled
    from the captured replica to the launch's atoms; None when there is none
    or the pair-kernel sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    table, src, atoms = {}, None, None
    for line in open(path):
        parts = line.split()
        if len(parts) < 2 or parts[0].startswith("#"):
            continue
        if parts[0] == "sources":
            src = parts[1]
            continue
        try:
            if parts[0] == "atoms":
                atoms = int(parts[1])
            else:
                table[parts[0]] = float(parts[1])
        except ValueError:
            pass
    if src != pair_source_hash() or name not in table or not atoms:
        return None
    return table[name] * atoms_total / atoms


def plain_form(pkg, S_batch, dev, params, pairs_md):
    """Each replica in its own context, MD + MC one step at a time with direct
    launches (no graph, no batching); same arithmetic and the batch's site
    reference energies.  Exchanges are O(M) and left out of this form.
    Timed over whole MC periods, about half a second per timed block (at
    least one period), median of five blocks."""
    import synth
    import torch
    b = S_batch.b
    t = S_batch.tables
    setups = []
    for r, rep in enumerate(b.replicas):
        sb = synth.Batch([rep], pH=b.pH[r:r + 1], E=b.E[r:r + 1], E_ladder=b.E[r:r + 1])
        lo, hi = t["site_state_off"][t["site_off"][r]], t["site_state_off"][t["site_off"][r + 1]]
        S = Setup(pkg, sb, dev, seed=99 + r, params=params, G=t["G_ref"][lo:hi])
        S.st.ex_every = 0
        S.ctx.set_persistent(False)
        setups.append(S)
    md = MC_EVERY * int(max(1, min(MD_PER_STEP // MC_EVERY, 0.5 / (est_md_step_s(b) * MC_EVERY))))
    for S in setups:
        S.ctx.md_segment(S.st, S.sites, MC_EVERY)
    torch.cuda.synchronize()
    n_bench = 5
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_bench)]
    for k in range(n_bench):
        ev[k][0].record()
        for _ in range(md):
            for S in setups:
                S.ctx.md_segment(S.st, S.sites, 1)
        ev[k][1].record()
    torch.cuda.synchronize()
    for S in setups:
        S.ctx.sync_status()
    ms = statistics.median(a.elapsed_time(c) for a, c in ev)      # per block of md MD steps
    s = ms / 1000.0
    return {"value": pairs_md * md / s, "unit": "pair-interactions/s", "ms_per_step": ms * MD_PER_STEP / md,
            "replica_md_steps_per_s": b.n_rep * md / s, "md_steps_per_block": md, "blocks": n_bench,
            "statistic": "median", "form": "one context per replica, direct launches per MD step, no graph"}


def end_to_end(pkg, S, n_bench, pairs_md):
    """Same metric through the public C ABI with the dynamic state in pinned
    host memory: every bench step is one gb_md_segment_host call, which copies
    the state (coordinates and charges, velocities, forces, site states, pH,
    E, exchange grid) from the host arrays to the device, runs the 100 MD
    steps and copies the new state back before it returns."""
    import torch
    keys = ("xyzq", "vel", "force", "state", "pH", "E", "grid")
    torch.cuda.synchronize()
    host = {k: getattr(S, k).detach().cpu().pin_memory() for k in keys}
    nbytes = sum(t.numel() * t.element_size() for t in host.values())
    S.ctx.md_segment_host(S.st, S.sites, MD_PER_STEP, host)        # untimed: the first call
    t0 = time.perf_counter()
    for _ in range(n_bench):
        S.ctx.md_segment_host(S.st, S.sites, MD_PER_STEP, host)
    s = time.perf_counter() - t0
    return {"value": pairs_md * MD_PER_STEP * n_bench / s, "unit": "pair-interactions/s",
            "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(nbytes), "steps": n_bench,
            "call": "gb_md_segment_host (host wall clock; the call returns with the state on the host)"}


if __name__ == "__main__":
    main()
