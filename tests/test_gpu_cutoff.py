"""GPU GB with cutoffs (gb_params.rgbmax, gb_params.cut) against the FP64
oracle with the same cutoffs: Born radii, energies, forces and dE/dq element
by element on ragged batches (cutoffs from below a contact distance to past
the molecule; batches with empty replicas), the Monte Carlo energy change and
the per-residue sweep, one MD step, the allocation-free entry point, cutoffs
past the molecule bitwise equal to none, and the block neighbour list (a cut
evaluation of a 100000-atom chain runs in a fraction of the time of the full
one, with sampled radii and the zero net force still right).

The oracle counts a pair iff its exact distance is within the pair cutoff;
the library decides from its FP32 r^2.  Each test that compares against the
oracle with a pair cutoff takes the cutoff nearest the one it names that has
no pair within the FP32 band of it (gpu_common.CUT_BAND), and asserts so."""
import ctypes as C
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_common import (DG_ABS, E_REL, F_ABS, KT, PHI_ABS, R_REL, batch_xyz, clear_cut, device,
                        energy_rel_err, f32, oracle_params, pairs_near_cut, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _run(pkg, b, **kw):
    import torch
    xyzq, rad = to_dev(b, device())
    ctx = pkg.Context(b.atom_off, pkg.default_params(**kw))
    out = ctx.energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    ctx.sync_status()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    ctx.close()
    return res


# Born radii with cutoffs: the descreening sum psi to 5e-7 relative (FP32
# closed-form terms of overlapping pairs cancel to about a tenth of their size,
# and with a small rgbmax every such pair takes the restricted form), carried
# into R through its condition number kappa = dln R / dln psi (about 4.6 for
# the most buried atoms here), plus the FP32 rounding of R.
PSI_REL = 5e-7


def born_bar(b, p):
    """Per-atom bar on |dR| / R for batch b under oracle parameters p."""
    x, q, rho, scr, off = oracle.batch_arrays(b)
    kappa = np.zeros(b.n_atoms)
    for r in range(b.n_rep):
        a0, a1 = off[r], off[r + 1]
        o = oracle.born_radii(x[a0:a1], rho[a0:a1], scr[a0:a1], p)
        kappa[a0:a1] = np.abs(o["dRdpsi"] * o["psi"] / o["R"])
    return np.maximum(R_REL, PSI_REL * kappa + 1.2e-7)


def _check(out, ref, bar):
    assert energy_rel_err(out["E"], ref["E"]).max() <= E_REL
    assert np.abs(out["F"] - ref["F"]).max() <= F_ABS
    assert np.all(np.abs(out["R"] - ref["R"]) / ref["R"] <= bar)
    assert np.abs(out["dEdq"] - ref["phi"]).max() <= PHI_ABS


@pytest.mark.parametrize("rgbmax,cut,kappa", [
    (12.0, 10.0, 0.0),
    (6.0, 8.0, 0.0),
    (3.0, 3.5, 0.0),        # cutoffs inside contact distances: near pairs straddle
    (0.0, 9.0, 0.0),        # pair cutoff only
    (9.0, 0.0, 0.0),        # Born-radius cutoff only
    (15.0, 12.0, 0.1),      # with salt screening
])
def test_cutoff_energy_forces_match_oracle(pkg, rgbmax, cut, kappa):
    b = synth.random_batch([2100, 300, 64, 33, 1], seed=41)
    if cut:
        cut = clear_cut(batch_xyz(b), cut)
        assert pairs_near_cut(batch_xyz(b), cut) == 0
    out = _run(pkg, b, rgbmax=rgbmax, cut=cut, kappa=kappa)
    p = oracle_params(rgbmax=f32(rgbmax), cut=f32(cut), kappa=f32(kappa))
    ref = oracle.batch_energy_forces(b, p, with_phi=True)
    _check(out, ref, born_bar(b, p))


def test_cutoff_batch_with_empty_replicas(pkg):
    """Empty replicas before, between and after the others: the list builder's
    replica search and the lists' runs stay inside each replica."""
    b = synth.random_batch([0, 700, 0, 33, 1, 1200, 0], seed=47)
    cut = clear_cut(batch_xyz(b), 9.0)
    assert pairs_near_cut(batch_xyz(b), cut) == 0
    out = _run(pkg, b, rgbmax=8.0, cut=cut)
    p = oracle_params(rgbmax=8.0, cut=cut)
    ref = oracle.batch_energy_forces(b, p, with_phi=True)
    _check(out, ref, born_bar(b, p))


def test_cutoff_sweep_matches_oracle(pkg):
    """Per-residue sweeps (every site of a kind in random order) with the pair
    cutoff in the site rows and the site-site block."""
    import torch
    dev = device()
    reps = [synth.make_replica(n, 90 + k, specs) for k, (n, specs) in enumerate([
        (400, [(1, 8, 2), (0, 6, 4), (0, 9, 3), (0, 5, 2), (1, 12, 2)]),
        (150, [(0, 12, 3), (1, 6, 2)]),
    ])]
    b = synth.Batch(reps, pH=np.array([4.4, 4.9]), E=synth.E0_REF_V + np.array([0.0, 0.03]))
    rgbmax, cut = 10.0, clear_cut(batch_xyz(b), 7.0)
    assert pairs_near_cut(batch_xyz(b), cut) == 0
    p = oracle_params(rgbmax=f32(rgbmax), cut=f32(cut))
    G = np.concatenate([oracle.site_reference_energies(synth.Batch([r], pH=b.pH[k:k + 1], E=b.E[k:k + 1]), p)
                        for k, r in enumerate(b.replicas)])
    t = b.site_tables(G)
    xyzq, rad = to_dev(b, dev)
    ctx = pkg.Context(b.atom_off, pkg.default_params(rgbmax=rgbmax, cut=cut))
    R = ctx.born_radii(xyzq, rad)
    sites = pkg.SiteTables(t, b.n_rep, dev)
    state = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
    pH, E = torch.as_tensor(b.pH, device=dev), torch.as_tensor(b.E, device=dev)
    x, q, rho, scr, off = oracle.batch_arrays(b)
    q = q.copy()
    st = b.initial_states()
    Rn = R.double().cpu().numpy()
    for step in range(10):
        for kind in (0, 1):
            dG, acc = ctx.mc_sweep(sites, xyzq, R, pH, E, KT, 13, step, kind, state)
            o = oracle.mc_sweep(off, x, q, Rn, t, st, b.pH, b.E, KT, 13, step, kind, p)
            dG, acc = dG.cpu().numpy(), acc.cpu().numpy()
            vis = o["visit"] >= 0
            assert np.all(np.abs(dG[vis] - o["dG"][vis]) <= DG_ABS), (step, kind)
            diff = np.flatnonzero(acc[vis] != o["acc"][vis])
            for s_ in np.flatnonzero(vis)[diff]:
                assert abs(o["dG"][s_] - o["thresh"][s_]) <= DG_ABS
            if diff.size:
                state.copy_(torch.as_tensor(st, device=dev))
                xyzq[:, 3] = torch.as_tensor(q, dtype=torch.float32, device=dev)
            assert np.array_equal(state.cpu().numpy(), st)
    ctx.sync_status()


def test_cutoffs_past_the_molecule_are_the_uncut_path(pkg):
    """No block straddles and none is skipped: the same arithmetic as without
    cutoffs, bit for bit."""
    b = synth.random_batch([900, 130], seed=42)
    a = _run(pkg, b, rgbmax=1.0e4, cut=1.0e4)
    d = _run(pkg, b)
    for k in ("F_fixed", "R", "E", "dEdq"):
        assert np.array_equal(a[k], d[k]), k
    c = _run(pkg, b, rgbmax=8.0, cut=8.0)
    assert not np.array_equal(a["E"], c["E"])          # the cutoffs are live


def test_cutoff_mc_energy_change_matches_oracle(pkg):
    import torch
    dev = device()
    b = synth.config_plain()
    rgbmax, cut = 10.0, clear_cut(batch_xyz(b), 8.0)
    assert pairs_near_cut(batch_xyz(b), cut) == 0
    p = oracle_params(rgbmax=f32(rgbmax), cut=f32(cut))
    G = oracle.site_reference_energies(b, p)
    t = b.site_tables(G)
    xyzq, rad = to_dev(b, dev)
    ctx = pkg.Context(b.atom_off, pkg.default_params(rgbmax=rgbmax, cut=cut))
    R = ctx.born_radii(xyzq, rad)
    x, q, rho, scr, off = oracle.batch_arrays(b)
    R_ref = oracle.born_radii(x, rho, scr, p)["R"]
    assert np.all(np.abs(R.cpu().numpy() - R_ref) / R_ref <= born_bar(b, p))
    sites = pkg.SiteTables(t, 1, dev)
    state = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
    pH, E = torch.as_tensor(b.pH, device=dev), torch.as_tensor(b.E, device=dev)
    q = q.copy()
    st = b.initial_states()
    Rn = R.double().cpu().numpy()
    for step in range(12):
        for kind in (0, 1):
            dG, acc = ctx.mc_step(sites, xyzq, R, pH, E, KT, 9, step, kind, state)
            o = oracle.mc_step(off, x, q, Rn, t, st, b.pH, b.E, KT, 9, step, kind, p)
            assert abs(dG.cpu().numpy()[0] - o["dG"][0]) <= DG_ABS
            if acc.cpu().numpy()[0] != o["acc"][0]:
                assert abs(o["dG"][0] - o["thresh"][0]) <= DG_ABS
                state.copy_(torch.as_tensor(st, device=dev))
                xyzq[:, 3] = torch.as_tensor(q, dtype=torch.float32, device=dev)
    ctx.sync_status()


def test_cutoff_md_step_matches_oracle(pkg):
    import torch
    dev = device()
    b = synth.random_batch([400, 120, 33], seed=43, sites=False)
    x, q, rho, scr, off = oracle.batch_arrays(b)
    # the forces are compared at the start (same coordinates on both sides)
    # and after the step, where the two sides' coordinates differ by up to
    # 1e-5 A per atom: the cutoff must leave both bands empty
    cut, near = None, 8.0
    for _ in range(40):
        c = clear_cut(batch_xyz(b), near)
        pc = oracle_params(rep_k=100.0, rep_sigma=2.5, rgbmax=9.0, cut=c)
        Fc, _ = oracle.forces_all(off, x, q, rho, scr, pc)
        xc, vc = x.copy(), np.zeros_like(x)
        oracle.md_step(off, xc, vc, q, rho, scr, Fc, 5, 1, pc)
        moved = [xc[off[r]:off[r + 1]] for r in range(b.n_rep)]
        if pairs_near_cut(moved, c, band=1e-6 * c + 2e-5) == 0:
            cut = c
            break
        near = c + 2e-4
    assert cut is not None
    params = pkg.default_params(rep_k=100.0, rep_sigma=2.5, rgbmax=9.0, cut=cut)
    p = oracle_params(rep_k=100.0, rep_sigma=2.5, rgbmax=9.0, cut=cut)
    ctx = pkg.Context(b.atom_off, params)
    N, M = b.n_atoms, b.n_rep
    S = dict(xyzq=torch.as_tensor(b.xyzq(), device=dev), rad=torch.as_tensor(b.rad_screen(), device=dev),
             vel=torch.zeros((N, 4), dtype=torch.float32, device=dev),
             force=torch.zeros((N, 4), dtype=torch.float32, device=dev),
             R=torch.zeros(N, dtype=torch.float32, device=dev),
             pH=torch.as_tensor(b.pH.copy(), device=dev), E=torch.as_tensor(b.E.copy(), device=dev))
    st = pkg.MDState()
    for k in ("xyzq", "vel", "force", "R", "pH", "E"):
        setattr(st, k, S[k].data_ptr())
    st.rad_screen = S["rad"].data_ptr()
    st.n_E, st.n_pH = M, 1
    st.dt, st.friction, st.mass, st.kT = 0.002, 10.0, 12.0, KT
    st.bond_k, st.bond_r0 = 300.0, 1.5
    st.seed, st.step, st.attempt = 5, 0, 0
    st.mc_every, st.ex_every, st.ex_dim, st.wrap = 0, 0, 0, 1
    ctx.md_init(st)
    torch.cuda.synchronize()
    F0, _ = oracle.forces_all(off, x, q, rho, scr, p)
    assert np.abs(S["force"][:, :3].cpu().numpy() - F0).max() <= F_ABS
    ctx.md_segment(st, None, 1)
    torch.cuda.synchronize()
    ctx.sync_status()
    v = np.zeros_like(x)
    oracle.md_step(off, x, v, q, rho, scr, F0, 5, 1, p)
    assert np.abs(S["xyzq"][:, :3].cpu().numpy() - x).max() <= 1e-5
    assert np.abs(S["vel"][:, :3].cpu().numpy() - v).max() <= 1e-4
    assert np.abs(S["force"][:, :3].cpu().numpy() - F0).max() <= F_ABS


def test_cutoff_static_entry_matches_oracle(pkg):
    import torch
    dev = device()
    lib = pkg.load()
    f = lib.gb_energy_forces_static
    P = C.c_void_p
    f.argtypes = [C.c_int32, C.POINTER(pkg.Params), P, P, P, P, P, P, P, P]
    f.restype = C.c_int
    b = synth.random_batch([1500], seed=44)
    n = b.n_atoms
    cut = clear_cut(batch_xyz(b), 9.0)
    assert pairs_near_cut(batch_xyz(b), cut) == 0
    xyzq, rad = to_dev(b, dev)
    params = pkg.default_params(rgbmax=8.0, cut=cut)
    out = dict(R=torch.empty(n, dtype=torch.float32, device=dev),
               F=torch.empty((n, 3), dtype=torch.float32, device=dev),
               F_fixed=torch.zeros((3, n), dtype=torch.int64, device=dev),
               E=torch.empty((1, 3), dtype=torch.float64, device=dev),
               dEdq=torch.empty(n, dtype=torch.float64, device=dev))
    rc = f(n, C.byref(params), xyzq.data_ptr(), rad.data_ptr(), out["R"].data_ptr(),
           out["F_fixed"].data_ptr(), out["F"].data_ptr(), out["E"].data_ptr(), out["dEdq"].data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    p = oracle_params(rgbmax=8.0, cut=cut)
    ref = oracle.batch_energy_forces(b, p, with_phi=True)
    _check(o, ref, born_bar(b, p))


def test_invalid_cutoffs_are_rejected(pkg):
    device()                                   # skips without a GPU
    b = synth.random_batch([64], seed=45)
    for kw in (dict(rgbmax=-1.0), dict(cut=-2.0), dict(cut=float("nan")), dict(rgbmax=float("inf"))):
        with pytest.raises(RuntimeError):
            pkg.Context(b.atom_off, pkg.default_params(**kw))


def test_cutoff_skips_out_of_range_blocks_on_a_large_chain(pkg):
    """100000 atoms, 12 A cutoffs: about 5 % of the 64 x 32 blocks are in
    range, so the evaluation takes well under half the time of the full one."""
    import torch
    dev = device()
    rep = synth.make_replica(100000, 46, [])
    b = synth.Batch([rep], pH=np.array([7.0]), E=np.array([synth.E0_REF_V]))
    xyzq, rad = to_dev(b, dev)
    times, outs = {}, {}
    for name, kw in (("full", {}), ("cut", dict(rgbmax=12.0, cut=12.0))):
        ctx = pkg.Context(b.atom_off, pkg.default_params(**kw))
        for _ in range(2):
            o = ctx.energy_forces(xyzq, rad)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            o = ctx.energy_forces(xyzq, rad)
        torch.cuda.synchronize()
        times[name] = (time.perf_counter() - t0) / 5
        ctx.sync_status()
        outs[name] = {k: v.cpu().numpy() for k, v in o.items()}
        ctx.close()
    print(f"100000 atoms: full {times['full'] * 1e3:.2f} ms, cutoffs 12 A {times['cut'] * 1e3:.2f} ms")
    assert times["cut"] < 0.5 * times["full"]
    # sampled Born radii against the oracle, one atom at a time
    x, q, rho, scr, off = oracle.batch_arrays(b)
    idx = np.random.default_rng(7).choice(b.n_atoms, 48, replace=False)
    R_ref = oracle.born_radii_subset(x, rho, scr, idx, oracle_params(rgbmax=12.0))
    R = outs["cut"]["R"][idx]
    # the conditioned bar with kappa <= 5 (its largest value at this density is 4.6)
    assert np.max(np.abs(R - R_ref) / R_ref) <= max(R_REL, PSI_REL * 5.0 + 1.2e-7)
    # properties that hold at any size with a truncated pair sum too: zero net
    # force (every pair enters with both signs) and sum_i q_i phi_i = 2 E
    # (degree-2 homogeneity in the charges at fixed radii)
    o = outs["cut"]
    F = o["F"].astype(np.float64)
    assert np.abs(F.sum(0)).max() <= 1e-6 * np.abs(F).sum() + 1e-3
    qp = b.xyzq()[:, 3].astype(np.float64) * o["dEdq"]
    assert abs(qp.sum() - 2 * (o["E"][0, 0] + o["E"][0, 1])) <= 2e-6 * np.abs(qp).sum()


def test_autotune_md_with_cutoffs_keeps_the_state_and_valid_caps(pkg):
    """On a context with cutoffs the MD-level autotuner tries only the caps the
    cutoff kernels have (1, 3) and puts the MD state back."""
    device()                                   # skips without a GPU
    import torch
    b = synth.config_eremd(2, 600)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(),
                         pkg.default_params(rep_k=100.0, rep_sigma=2.5, rgbmax=9.0, cut=9.0), sites=t,
                         pH=b.pH, E=b.E, E_ladder=synth.e_ladder(2), pH_ladder=[b.pH[0]], seed=4,
                         mc_every=5, ex_every=10)
    before = {k: getattr(sim, k).clone() for k in ("xyzq", "vel", "force", "state", "E", "grid")}
    caps = sim.ctx.autotune_md(sim.st, sim.sites, trial_steps=10)
    sim.sync()
    assert all(c in (1, 3) for c in caps)
    assert sim.step == 0
    for k, v in before.items():
        assert torch.equal(getattr(sim, k), v), k
    sim.run(20)
    sim.sync()
    assert torch.isfinite(sim.xyzq).all()
