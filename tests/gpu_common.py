"""Shared helpers of the GPU parity tests (oracle parameters rounded to the
FP32 values the library receives, tolerances, device set-up)."""
import numpy as np

import oracle

KT = oracle.KB * 300.0

# Tolerances (spec values): energy relative 1e-6, forces 1e-3
# kcal/mol/A max-abs, state-change energy 1e-3 kcal/mol.
E_REL = 1e-6
F_ABS = 1e-3
DG_ABS = 1e-3
# Born radii are FP32 results of FP32 pair sums: a few ulp of R.
R_REL = 2e-6
# dE/dq: FP32 pair terms of magnitude up to ~k_e/r summed in fixed point
PHI_ABS = 2e-3


def f32(v):
    return float(np.float32(v))


def oracle_params(**kw):
    """Oracle parameters equal to the float32 values the CUDA library stores."""
    d = dict(alpha=f32(1.0), beta=f32(0.8), gamma=f32(4.85), offset=f32(0.09), eps_in=1.0,
             eps_out=78.5)
    d.update(kw)
    return oracle.default_params(**d)


def device():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(batch, dev):
    import torch
    return (torch.as_tensor(batch.xyzq(), device=dev), torch.as_tensor(batch.rad_screen(), device=dev))


def energy_rel_err(E_gpu, E_ref):
    """Per replica |dE| / |E| of E_GB + E_Coul (E_gpu: [M,3] GB, Coul, rep)."""
    tot_g = E_gpu[:, 0] + E_gpu[:, 1]
    tot_r = E_ref[:, 0] + E_ref[:, 1]
    return np.abs(tot_g - tot_r) / np.maximum(np.abs(tot_r), 1e-30)


# Pair cutoff.  The library decides whether a pair lies within `cut` from its
# FP32 squared distance; the oracle from the exact distance.  Rounding of the
# FP32 differences and of r^2 moves r by a few float ulps (one ulp of r is
# about 1.2e-7 r), so the two decisions can differ only for pairs with
# |r - cut| <= CUT_BAND * cut (about 8 ulps).  Each such pair moves the
# energy by up to kcal/mol.  The parity tests therefore list the pairs in
# that band, and take a cutoff (within a few 1e-4 A of the one they ask for)
# whose band is empty: on their inputs both sides count the same pairs.
CUT_BAND = 1e-6


def pairs_near_cut(xyz_list, cut, band=None):
    """Number of pairs, over the given coordinate sets (each (n, 3), any
    float type, taken as exact doubles), whose distance lies within `band`
    of `cut` (default CUT_BAND * cut)."""
    band = CUT_BAND * cut if band is None else band
    count = 0
    for x in xyz_list:
        x = np.asarray(x, dtype=np.float64)
        n = len(x)
        for a in range(0, n, 1024):
            d = np.sqrt(((x[a:a + 1024, None, :] - x[None, :, :]) ** 2).sum(-1))
            i, j = np.nonzero(np.abs(d - cut) <= band)
            count += int(np.count_nonzero(j > i + a))
    return count


def batch_xyz(b):
    """Coordinates of every replica of a synth.Batch, one array each."""
    x = b.xyzq()[:, :3]
    return [x[b.atom_off[r]:b.atom_off[r + 1]] for r in range(b.n_rep)]


def clear_cut(xyz_list, near, band=None, tries=200):
    """The float32 value closest to `near` on a 1e-4 A grid (near, near +
    1e-4, near - 1e-4, ...) with no pair of the coordinate sets within the
    band of it."""
    for k in range(tries):
        step = (k + 1) // 2 * (1 if k % 2 else -1)
        c = f32(near + 1e-4 * step)
        if pairs_near_cut(xyz_list, c, band) == 0:
            return c
    raise AssertionError(f"no cutoff near {near} leaves the band empty")


def oracle_energy_forces_job(args):
    """Full FP64 oracle evaluation of one molecule: dict(E, F, phi, R).  A
    module-level function, so that spawned worker processes can run it."""
    x, q, rho, scr, kw = args
    o = oracle.energy_forces(x, q, rho, scr, oracle_params(**kw))
    return {k: o[k] for k in ("E", "F", "phi", "R")}


def oracle_pool(n_jobs):
    """A pool of spawned worker processes for oracle evaluations (spawned, not
    forked: a child forked from a process that holds a CUDA context can
    hang), sized to the host's cores."""
    import multiprocessing as mp
    import os
    n = max(2, min(n_jobs, (os.cpu_count() or 2) - 1))
    return mp.get_context("spawn").Pool(n)


def oracle_mc_job(args):
    """The oracle's Monte Carlo attempt of replica r alone (a module-level
    function for spawned worker processes).  The oracle draws its random
    numbers by replica index, so replica r runs behind r empty replicas.
    args: (r, x, q, R (float64, the replica's), site table of the replica
    alone (synth layout), states, pH, E, kT, seed, step, kind).  Returns
    dict(dG, acc, thresh, site, new_state) of replica r."""
    r, x, q, R, t, st, pH, E, kT, seed, step, kind = args
    n = len(q)
    off = np.array([0] * (r + 1) + [n], dtype=np.int64)
    tt = dict(t)
    tt["site_off"] = np.concatenate([np.zeros(r, np.int32), np.asarray(t["site_off"], np.int32)])
    pHv = np.full(r + 1, float(pH))
    Ev = np.full(r + 1, float(E))
    o = oracle.mc_step(off, np.ascontiguousarray(x), np.ascontiguousarray(q).copy(), np.ascontiguousarray(R), tt,
                       np.ascontiguousarray(st, np.int32).copy(), pHv, Ev, kT, seed, step, kind, oracle_params())
    return {k: v[r] for k, v in o.items()}
