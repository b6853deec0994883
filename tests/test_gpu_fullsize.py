"""GPU parity at the full workload sizes, in the same launch configuration the
benchmark uses (one context over the whole batch, default tiles).

* 8 x 2048 E-REMD batch and 16 x 4096 differentiation batch: every replica
  holds the same molecule, so one FP64 oracle evaluation checks all of them
  element by element; the 16 x 4096 case also checks the gradient against
  central finite differences of the oracle (h = 1e-4 A, 1e-5 e) and the
  autograd wrapper.
* uneven batch (64 replicas, 500..20000 atoms): every replica element by
  element, up to the largest (18134 atoms), plus properties that hold at any
  size.
* Monte Carlo attempts (both kinds) on every uneven replica and on three
  25,000-atom grid replicas against the oracle's two-evaluation energy change.
* 48 x 25000 grid batch: one 25,000-atom replica element by element (energy,
  forces, Born radii, dE/dq), identical results on identical replicas, and the
  same properties.  At these sizes the FP32 far-field terms, the int64
  fixed-point sums and the energy's cancellation are at their largest.

The oracle needs about a minute for a 25,000-atom molecule on one core, so
the large replicas are evaluated in spawned worker processes, one molecule
each, started by the first test of this module and collected where needed.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import (DG_ABS, E_REL, F_ABS, KT, PHI_ABS, R_REL, device, energy_rel_err, oracle_energy_forces_job,
                        oracle_mc_job, oracle_params, oracle_pool, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


@pytest.fixture(scope="module")
def uneven():
    return synth.config_uneven()


@pytest.fixture(scope="module", autouse=True)
def big_refs(uneven):
    """Oracle evaluations of the 25,000-atom grid replica and of every uneven
    replica, running in worker processes while the module's tests use the
    GPU.  Largest first, so that the pool's tail is short."""
    if not _has_gpu():
        yield {}
        return
    grid = synth.config_grid()
    jobs = []
    x, q, rho, scr, off = oracle.batch_arrays(grid)
    jobs.append(("grid", (x[:25000], q[:25000], rho[:25000], scr[:25000], {})))
    x, q, rho, scr, off = oracle.batch_arrays(uneven)
    for r in np.argsort(-np.diff(off)):
        a, c = off[r], off[r + 1]
        jobs.append((int(r), (x[a:c], q[a:c], rho[a:c], scr[a:c], {})))
    pool = oracle_pool(len(jobs))
    res = {k: pool.apply_async(oracle_energy_forces_job, (args,)) for k, args in jobs}
    yield res
    pool.terminate()
    pool.join()


def _has_gpu():
    import torch
    return torch.cuda.is_available()


def _gpu(pkg, batch):
    import torch
    dev = device()
    xyzq, rad = to_dev(batch, dev)
    ctx = pkg.Context(batch.atom_off)
    out = ctx.energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    ctx.sync_status()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    ctx.close()
    return res


def _check_replica(out, a, b, r, ref):
    e = energy_rel_err(out["E"][r:r + 1], ref["E"][None, :])
    assert e.max() <= E_REL, (r, e)
    assert np.abs(out["F"][a:b] - ref["F"]).max() <= F_ABS, r
    assert np.max(np.abs(out["R"][a:b] - ref["R"]) / ref["R"]) <= R_REL, r
    assert np.abs(out["dEdq"][a:b] - ref["phi"]).max() <= PHI_ABS, r


def _properties(out, batch):
    """Sum_i q_i phi_i = 2 E (degree-2 homogeneity at fixed radii) and zero net
    force, per replica, within FP32 resolution of the summed magnitudes."""
    q = batch.xyzq()[:, 3].astype(np.float64)
    off = batch.atom_off
    for r in range(batch.n_rep):
        a, b = off[r], off[r + 1]
        if b - a < 2:
            continue
        qp = q[a:b] * out["dEdq"][a:b]
        E = out["E"][r, 0] + out["E"][r, 1]
        assert abs(qp.sum() - 2 * E) <= 2e-6 * np.abs(qp).sum(), r
        F = out["F"][a:b].astype(np.float64)
        assert np.abs(F.sum(0)).max() <= 1e-6 * np.abs(F).sum() + 1e-3, r


def test_eremd_8x2048_every_replica(pkg):
    b = synth.config_eremd(8, 2048)
    out = _gpu(pkg, b)
    x, q, rho, scr, off = oracle.batch_arrays(b)
    ref = oracle.energy_forces(x[:2048], q[:2048], rho[:2048], scr[:2048], oracle_params())
    for r in range(8):
        _check_replica(out, off[r], off[r + 1], r, ref)


def test_diff_16x4096_gradient(pkg):
    import torch
    b = synth.config_diff(16, 4096)
    out = _gpu(pkg, b)
    x, q, rho, scr, off = oracle.batch_arrays(b)
    n = 4096
    p = oracle_params()
    ref = oracle.energy_forces(x[:n], q[:n], rho[:n], scr[:n], p)
    for r in range(16):
        _check_replica(out, off[r], off[r + 1], r, ref)
    # central finite differences of the FP64 oracle on random coordinates and charges
    rng = np.random.default_rng(2)
    h, hq = 1e-4, 1e-5
    for _ in range(12):
        i, k = int(rng.integers(n)), int(rng.integers(3))
        xp, xm = x[:n].copy(), x[:n].copy()
        xp[i, k] += h
        xm[i, k] -= h
        fd = -(oracle.energy(xp, q[:n], rho[:n], scr[:n], p) - oracle.energy(xm, q[:n], rho[:n], scr[:n], p)) / (2 * h)
        assert abs(out["F"][i, k] - fd) <= F_ABS, (i, k, out["F"][i, k], fd)
    for _ in range(12):
        i = int(rng.integers(n))
        qp, qm = q[:n].copy(), q[:n].copy()
        qp[i] += hq
        qm[i] -= hq
        fd = (oracle.energy(x[:n], qp, rho[:n], scr[:n], p) - oracle.energy(x[:n], qm, rho[:n], scr[:n], p)) / (2 * hq)
        assert abs(out["dEdq"][i] - fd) <= PHI_ABS, (i, out["dEdq"][i], fd)
    # autograd wrapper: d(sum w_r E_r)/d(xyzq) = (-w F, w phi)
    dev = device()
    xyzq, rad = to_dev(b, dev)
    xyzq.requires_grad_(True)
    ctx = pkg.Context(b.atom_off)
    E = pkg.GBEnergy.apply(ctx, xyzq, rad)
    w = torch.linspace(0.5, 2.0, b.n_rep, dtype=torch.float64, device=dev)
    (E * w).sum().backward()
    g = xyzq.grad.cpu().numpy()
    wa = np.repeat(w.cpu().numpy(), 4096)
    assert np.allclose(g[:, :3], -out["F"] * wa[:, None], atol=1e-3)
    assert np.allclose(g[:, 3], out["dEdq"] * wa, atol=1e-3)
    assert np.allclose(E.detach().cpu().numpy(), out["E"][:, 0] + out["E"][:, 1], rtol=1e-12)


def test_uneven_64_replicas(pkg, uneven, big_refs):
    """Every replica element by element: 64 molecules of 500 to 18134 atoms."""
    b = uneven
    out = _gpu(pkg, b)
    off = b.atom_off
    for r in range(b.n_rep):
        ref = big_refs[r].get(timeout=1800)
        _check_replica(out, off[r], off[r + 1], r, ref)
    _properties(out, b)


def test_grid_48x25000(pkg, big_refs):
    b = synth.config_grid()
    out = _gpu(pkg, b)
    off = b.atom_off
    n = 25000
    ref = big_refs["grid"].get(timeout=1800)
    for r in (0, 17, 47):
        _check_replica(out, off[r], off[r + 1], r, ref)
    # identical molecules give bitwise identical results in every replica
    for r in range(1, b.n_rep):
        a, c = off[r], off[r + 1]
        assert np.array_equal(out["F_fixed"][:, a:c], out["F_fixed"][:, :n]), r
        assert np.array_equal(out["R"][a:c], out["R"][:n]), r
        assert np.array_equal(out["E"][r], out["E"][0]), r
    one = synth.Batch(b.replicas[:1], pH=b.pH[:1], E=b.E[:1])
    _properties(out, one)


def test_mc_decisions_eremd_8x2048(pkg):
    """Protonation and redox attempts on the full E-REMD batch (different E per
    replica) against the oracle's two-evaluation energy change."""
    import torch
    b = synth.config_eremd(8, 2048)
    dev = device()
    p = oracle_params()
    G = oracle.site_reference_energies(synth.Batch(b.replicas[:1], pH=b.pH[:1], E=b.E[:1]), p)
    t = b.site_tables(np.tile(G, 8))
    xyzq, rad = to_dev(b, dev)
    ctx = pkg.Context(b.atom_off)
    R = ctx.born_radii(xyzq, rad)
    sites = pkg.SiteTables(t, b.n_rep, dev)
    state = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
    pH, E = torch.as_tensor(b.pH, device=dev), torch.as_tensor(b.E, device=dev)
    x, q, rho, scr, off = oracle.batch_arrays(b)
    q = q.copy()
    st = b.initial_states()
    Rn = R.double().cpu().numpy()
    for step in (10, 20):
        for kind in (0, 1):
            dG, acc = ctx.mc_step(sites, xyzq, R, pH, E, KT, 3, step, kind, state)
            o = oracle.mc_step(off, x, q, Rn, t, st, b.pH, b.E, KT, 3, step, kind, p)
            dG, acc = dG.cpu().numpy(), acc.cpu().numpy()
            assert np.all(np.abs(dG - o["dG"]) <= DG_ABS), (step, kind)
            near = np.abs(o["dG"] - o["thresh"]) <= DG_ABS
            assert np.array_equal(acc[~near], o["acc"][~near])
            if near.any():
                state.copy_(torch.as_tensor(st, device=dev))
                xyzq[:, 3] = torch.as_tensor(q, dtype=torch.float32, device=dev)


def test_single_replica_50000_atoms(pkg):
    """Largest replica tested: one 50,000-atom chain (1.25e9 pairs, 782
    tiles).  Sampled Born radii against the oracle one atom at a time, the
    charge-derivative identity and the net force."""
    rep = synth.make_replica(50000, 7, [(1, 20, 2), (0, 12, 2)])
    b = synth.Batch([rep], pH=np.array([4.85]), E=np.array([synth.E0_REF_V]))
    out = _gpu(pkg, b)
    x, q, rho, scr, off = oracle.batch_arrays(b)
    idx = np.random.default_rng(8).choice(50000, size=8, replace=False)
    R = oracle.born_radii_subset(x, rho, scr, idx, oracle_params())
    assert np.max(np.abs(out["R"][idx] - R) / R) <= R_REL
    assert np.all(np.isfinite(out["F"])) and np.all(out["R"] > 0)
    _properties(out, b)


def _mc_full(pkg, b, reps, kinds=(0, 1), seed=3, step=10):
    """GPU single-site attempts on the whole batch, one per kind, each from
    the initial states (all 0, G_ref = 0), and the oracle's attempt for each
    listed replica and kind (its two-evaluation energy change), one spawned
    worker per replica and kind.  Returns {kind: (dG, acc, {r: oracle})}."""
    import torch
    from paper_1803_09652_gb300.shard import slice_sites
    dev = device()
    t = b.site_tables()                     # G_ref = 0: an input like any other
    xyzq, rad = to_dev(b, dev)
    ctx = pkg.Context(b.atom_off)
    R = ctx.born_radii(xyzq, rad)
    sites = pkg.SiteTables(t, b.n_rep, dev)
    pH, E = torch.as_tensor(b.pH, device=dev), torch.as_tensor(b.E, device=dev)
    gpu = {}
    for kind in kinds:
        state = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
        x4 = xyzq.clone()
        dG, acc = ctx.mc_step(sites, x4, R, pH, E, KT, seed, step, kind, state)
        torch.cuda.synchronize()
        gpu[kind] = (dG.cpu().numpy(), acc.cpu().numpy())
    ctx.sync_status()
    Rn = R.double().cpu().numpy()
    x, q, rho, scr, off = oracle.batch_arrays(b)
    jobs, keys = [], []
    for kind in kinds:
        for r in reps:
            a, c = off[r], off[r + 1]
            tr = slice_sites(t, r, r + 1)
            jobs.append((r, x[a:c], q[a:c], Rn[a:c], tr, np.zeros(tr["n_sites"], np.int32), b.pH[r], b.E[r], KT,
                         seed, step, kind))
            keys.append((kind, r))
    # largest replicas first, so that the pool's tail is short
    order = np.argsort([-(off[r + 1] - off[r]) for _, r in keys])
    pool = oracle_pool(len(jobs))
    try:
        outs = pool.map(oracle_mc_job, [jobs[i] for i in order])
    finally:
        pool.terminate()
        pool.join()
    ctx.close()
    res = {kind: (gpu[kind][0], gpu[kind][1], {}) for kind in kinds}
    for i, o in zip(order, outs):
        kind, r = keys[i]
        res[kind][2][r] = o
    return res


def test_mc_energy_change_every_uneven_replica(pkg, uneven):
    """Protonation (multi-state sites, 2-5 states) and redox attempts on every
    replica of the uneven batch, 500 to 18,134 atoms, against the oracle's
    two full energy evaluations at the same radii."""
    b = uneven
    for kind, (dG, acc, ref) in _mc_full(pkg, b, list(range(b.n_rep))).items():
        n_near = 0
        for r, o in ref.items():
            assert abs(dG[r] - o["dG"]) <= DG_ABS, (kind, r, dG[r], o["dG"])
            if acc[r] != o["acc"]:
                assert abs(o["dG"] - o["thresh"]) <= DG_ABS, (kind, r)
                n_near += 1
        assert n_near <= 1


def test_mc_energy_change_grid_replicas(pkg):
    """Redox and protonation attempts on three 25,000-atom replicas of the
    2-D grid (each at its own pH and E) against the oracle."""
    b = synth.config_grid()
    for kind, (dG, acc, ref) in _mc_full(pkg, b, [0, 17, 47]).items():
        for r, o in ref.items():
            assert abs(dG[r] - o["dG"]) <= DG_ABS, (kind, r, dG[r], o["dG"])
            assert acc[r] == o["acc"] or abs(o["dG"] - o["thresh"]) <= DG_ABS, (kind, r)
