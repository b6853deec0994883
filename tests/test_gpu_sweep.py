"""GPU per-residue sweep (redox_ph_mc_sweep, Sec. III.A.2) against the
oracle's sweep on the same inputs and Born radii: per-site dG within 1e-3
kcal/mol, identical visits and decisions except where |dG - threshold| is
inside that tolerance (then both chains follow the oracle), identical states
and charges after every sweep; the sweep inside the MD driver; the limits."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import DG_ABS, KT, device, oracle_params, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _sweep_case(pkg, b, n_sweeps, seed=31):
    import torch
    dev = device()
    p = oracle_params()
    t = b.site_tables(oracle.site_reference_energies(b, p) if b.n_rep == 1 else
                      np.concatenate([oracle.site_reference_energies(
                          synth.Batch([r], pH=b.pH[k:k + 1], E=b.E[k:k + 1]), p)
                          for k, r in enumerate(b.replicas)]))
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
    near = accepted = 0
    for step in range(n_sweeps):
        for kind in (0, 1):
            dG, acc = ctx.mc_sweep(sites, xyzq, R, pH, E, KT, seed, step, kind, state)
            o = oracle.mc_sweep(off, x, q, Rn, t, st, b.pH, b.E, KT, seed, step, kind, p)
            dG, acc = dG.cpu().numpy(), acc.cpu().numpy()
            vis = o["visit"] >= 0
            assert np.array_equal(acc == 2, ~vis), (step, kind)
            assert np.all(np.abs(dG[vis] - o["dG"][vis]) <= DG_ABS), (step, kind)
            diff = np.flatnonzero(acc[vis] != o["acc"][vis])
            for s in np.flatnonzero(vis)[diff]:
                assert abs(o["dG"][s] - o["thresh"][s]) <= DG_ABS, (step, kind, s)
                near += 1
            accepted += int(o["acc"][vis].sum())
            if diff.size:   # follow the oracle so both chains stay in step
                state.copy_(torch.as_tensor(st, device=dev))
                xyzq[:, 3] = torch.as_tensor(q, dtype=torch.float32, device=dev)
            assert np.array_equal(state.cpu().numpy(), st), (step, kind)
            assert np.array_equal(xyzq[:, 3].cpu().numpy().astype(np.float64), q), (step, kind)
    ctx.sync_status()
    return accepted, near


def test_sweep_matches_oracle_multisite(pkg):
    reps = [synth.make_replica(n, 70 + k, specs) for k, (n, specs) in enumerate([
        (90, [(1, 8, 2), (0, 6, 4), (0, 9, 3), (0, 5, 2)]),
        (45, [(0, 12, 5)]),
        (60, []),
        (150, [(1, 30, 2), (1, 20, 2), (0, 10, 2), (0, 7, 3), (1, 6, 2)]),
    ])]
    b = synth.Batch(reps, pH=np.array([4.0, 4.85, 5.0, 4.4]),
                    E=synth.E0_REF_V + np.array([0.0, 0.02, -0.01, 0.05]))
    accepted, near = _sweep_case(pkg, b, 20)
    assert accepted > 20


def test_sweep_many_sites_large_replica(pkg):
    """32 pH sites and 8 redox sites in a 1200-atom chain (the grid workload's
    site mix): sweeps through the slice-partial rows of five slices."""
    rng = np.random.default_rng(5)
    specs = [(1, int(rng.integers(8, 31)), 2) for _ in range(8)]
    specs += [(0, int(rng.integers(8, 31)), int(rng.integers(2, 5))) for _ in range(32)]
    rep = synth.make_replica(1200, 81, specs)
    b = synth.Batch([rep], pH=np.array([4.6]), E=np.array([synth.E0_REF_V + 0.01]))
    accepted, near = _sweep_case(pkg, b, 2)
    assert accepted > 5


def test_sweep_in_md_driver_keeps_charges_consistent(pkg):
    import torch
    dev = device()
    b = synth.config_eremd(4, 300)
    p = oracle_params()
    G = oracle.site_reference_energies(synth.Batch(b.replicas[:1], pH=b.pH[:1], E=b.E[:1]), p)
    t = b.site_tables(np.tile(G, 4))
    ctx = pkg.Context(b.atom_off, pkg.default_params(rep_k=100.0, rep_sigma=2.5))
    sites = pkg.SiteTables(t, 4, dev)
    N = b.n_atoms
    S = dict(xyzq=torch.as_tensor(b.xyzq(), device=dev), rad=torch.as_tensor(b.rad_screen(), device=dev),
             vel=torch.zeros((N, 4), dtype=torch.float32, device=dev),
             force=torch.zeros((N, 4), dtype=torch.float32, device=dev),
             R=torch.zeros(N, dtype=torch.float32, device=dev),
             pH=torch.as_tensor(b.pH.copy(), device=dev), E=torch.as_tensor(b.E.copy(), device=dev),
             grid=torch.arange(4, dtype=torch.int32, device=dev),
             E_ladder=torch.as_tensor(synth.e_ladder(4), device=dev),
             pH_ladder=torch.as_tensor(np.array([b.pH[0]]), device=dev),
             state=torch.zeros(t["n_sites"], dtype=torch.int32, device=dev))
    st = pkg.MDState()
    for k in ("xyzq", "vel", "force", "R", "pH", "E", "grid", "E_ladder", "pH_ladder", "state"):
        setattr(st, k, S[k].data_ptr())
    st.rad_screen = S["rad"].data_ptr()
    st.n_E, st.n_pH = 4, 1
    st.dt, st.friction, st.mass, st.kT = 0.002, 10.0, 12.0, KT
    st.bond_k, st.bond_r0 = 300.0, 1.5
    st.seed, st.step, st.attempt = 5, 0, 0
    st.mc_every, st.ex_every, st.ex_dim, st.wrap, st.mc_mode = 5, 20, 0, 1, 1
    ctx.md_init(st)
    ctx.md_segment(st, sites, 200)
    torch.cuda.synchronize()
    ctx.sync_status()
    x = S["xyzq"].cpu().numpy()
    st_h = S["state"].cpu().numpy()
    assert np.all(np.isfinite(x)) and st_h.any()          # some site left state 0
    for s in range(t["n_sites"]):
        r = np.searchsorted(t["site_off"], s, side="right") - 1
        a0, a1 = t["site_atom_off"][s], t["site_atom_off"][s + 1]
        idx = t["site_atom_idx"][a0:a1] + b.atom_off[r]
        qo = t["site_q_off"][s] + st_h[s] * (a1 - a0)
        assert np.array_equal(x[idx, 3], t["q_state"][qo:qo + a1 - a0])


def test_sweep_over_the_limits_reports_an_error(pkg):
    """A replica with more than 1024 pH-site atoms is skipped and the error
    is reported through gb_sync_status."""
    import torch
    dev = device()
    rep = synth.make_replica(3000, 91, [(0, 30, 2)] * 40)     # 1200 pH-site atoms
    b = synth.Batch([rep], pH=np.array([4.6]), E=np.array([synth.E0_REF_V]))
    t = b.site_tables()
    xyzq, rad = to_dev(b, dev)
    ctx = pkg.Context(b.atom_off)
    R = ctx.born_radii(xyzq, rad)
    sites = pkg.SiteTables(t, 1, dev)
    state = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
    pH, E = torch.as_tensor(b.pH, device=dev), torch.as_tensor(b.E, device=dev)
    q0 = xyzq[:, 3].clone()
    dG, acc = ctx.mc_sweep(sites, xyzq, R, pH, E, KT, 1, 0, 0, state)
    torch.cuda.synchronize()
    with pytest.raises(RuntimeError):
        ctx.sync_status()
    assert torch.equal(xyzq[:, 3], q0) and not state.any()
    assert np.all(acc.cpu().numpy() == 2)
