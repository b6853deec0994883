"""GPU MD driver: one BAOAB step against the oracle on identical inputs (MD is
chaotic, so parity is per step), graph replay against direct launches, and
E-REMD bookkeeping over a longer segment."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import F_ABS, KT, device, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _setup(pkg, b, seed, mc_every=0, ex_every=0, with_sites=False, persistent=False):
    import torch
    dev = device()
    params = pkg.default_params(rep_k=100.0, rep_sigma=2.5)
    ctx = pkg.Context(b.atom_off, params)
    ctx.set_persistent(persistent)
    N, M = b.n_atoms, b.n_rep
    S = dict(xyzq=torch.as_tensor(b.xyzq(), device=dev),
             rad=torch.as_tensor(b.rad_screen(), device=dev),
             vel=torch.zeros((N, 4), dtype=torch.float32, device=dev),
             force=torch.zeros((N, 4), dtype=torch.float32, device=dev),
             R=torch.zeros(N, dtype=torch.float32, device=dev),
             pH=torch.as_tensor(b.pH.copy(), device=dev), E=torch.as_tensor(b.E.copy(), device=dev),
             grid=torch.arange(M, dtype=torch.int32, device=dev),
             E_ladder=torch.as_tensor(synth.e_ladder(M), device=dev),
             pH_ladder=torch.as_tensor(np.array([b.pH[0]]), device=dev))
    sites = None
    if with_sites:
        t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
        sites = pkg.SiteTables(t, M, dev)
        S["state"] = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
    st = pkg.MDState()
    for k in ("xyzq", "vel", "force", "R", "pH", "E", "grid", "E_ladder", "pH_ladder"):
        setattr(st, k, S[k].data_ptr())
    st.rad_screen = S["rad"].data_ptr()
    st.state = S["state"].data_ptr() if with_sites else None
    st.n_E, st.n_pH = M, 1
    st.dt, st.friction, st.mass, st.kT = 0.002, 10.0, 12.0, KT
    st.bond_k, st.bond_r0 = 300.0, 1.5
    st.seed, st.step, st.attempt = seed, 0, 0
    st.mc_every, st.ex_every, st.ex_dim, st.wrap = mc_every, ex_every, 0, 1
    ctx.md_init(st)
    return ctx, st, S, sites


@pytest.mark.parametrize("persistent", [False, True])
def test_one_baoab_step_matches_oracle(pkg, persistent):
    import torch
    b = synth.random_batch([120, 64, 33], seed=3, sites=False)
    ctx, st, S, _ = _setup(pkg, b, seed=5, persistent=persistent)
    torch.cuda.synchronize()
    x, q, rho, scr, off = oracle.batch_arrays(b)
    p = oracle_params(rep_k=100.0, rep_sigma=2.5)
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
    assert st.step == 1


@pytest.mark.parametrize("persistent", [False, True])
def test_graph_replay_equals_direct_launches(pkg, persistent):
    import torch
    b = synth.config_eremd(4, 300)
    ctx1, st1, S1, sites1 = _setup(pkg, b, seed=8, mc_every=10, ex_every=50, with_sites=True,
                                   persistent=persistent)
    ctx2, st2, S2, sites2 = _setup(pkg, b, seed=8, mc_every=10, ex_every=50, with_sites=True,
                                   persistent=persistent)
    ctx1.md_segment(st1, sites1, 100)           # two captured blocks of 50
    for _ in range(100):
        ctx2.md_segment(st2, sites2, 1)         # direct launches
    torch.cuda.synchronize()
    ctx1.sync_status()
    ctx2.sync_status()
    for k in ("xyzq", "vel", "force", "state", "E", "grid"):
        assert torch.equal(S1[k], S2[k]), k
    assert st1.step == st2.step == 100 and st1.attempt == st2.attempt == 2


@pytest.mark.parametrize("persistent", [False, True])
def test_eremd_segment_bookkeeping(pkg, persistent):
    import torch
    b = synth.config_eremd(8, 256)
    ctx, st, S, sites = _setup(pkg, b, seed=11, mc_every=10, ex_every=20, with_sites=True,
                               persistent=persistent)
    ctx.md_segment(st, sites, 400)
    torch.cuda.synchronize()
    ctx.sync_status()
    grid = S["grid"].cpu().numpy()
    assert sorted(grid.tolist()) == list(range(8))
    E = S["E"].cpu().numpy()
    lad = synth.e_ladder(8)
    assert np.allclose(E[grid], lad)
    x = S["xyzq"].cpu().numpy()
    assert np.all(np.isfinite(x))
    # charges always equal the site-state charges
    t = sites.t
    st_h = S["state"].cpu().numpy()
    tables = b.site_tables()
    for s in range(tables["n_sites"]):
        r = np.searchsorted(tables["site_off"], s, side="right") - 1
        a0, a1 = tables["site_atom_off"][s], tables["site_atom_off"][s + 1]
        idx = tables["site_atom_idx"][a0:a1] + b.atom_off[r]
        na = a1 - a0
        qo = tables["site_q_off"][s] + st_h[s] * na
        assert np.array_equal(x[idx, 3], tables["q_state"][qo:qo + na])
    assert st.attempt == 20


def test_persistent_driver_tracks_three_pass_driver(pkg):
    """Same trajectory start, both drivers: positions agree to FP32 rounding
    after 20 steps (they differ only in where the bond forces are rounded)."""
    import torch
    b = synth.random_batch([300, 257, 64, 1], seed=13, sites=False)
    c1, st1, S1, _ = _setup(pkg, b, seed=4, persistent=False)
    c2, st2, S2, _ = _setup(pkg, b, seed=4, persistent=True)
    c1.md_segment(st1, None, 20)
    c2.md_segment(st2, None, 20)
    torch.cuda.synchronize()
    c1.sync_status()
    c2.sync_status()
    d = (S1["xyzq"] - S2["xyzq"]).abs().max().item()
    assert d < 1e-3, d


def test_persistent_wait_that_runs_out_reports_a_timeout(pkg):
    """A dependency wait of the persistent kernel limited to one poll runs out
    (the phases of a 2048-atom replica take microseconds): the launch ends,
    gb_sync_status reports GB_ERR_TIMEOUT, and after the default limit is
    restored the same context runs the same segment to the same result as the
    multi-launch path."""
    device()                                   # skips without a GPU
    import torch
    b = synth.random_batch([2048, 1500], seed=21, sites=False)
    ctx, st, S, _ = _setup(pkg, b, seed=8, persistent=True)
    x0 = S["xyzq"].clone()
    ctx.set_wait_limit(1)
    ctx.md_segment(st, None, 4)
    torch.cuda.synchronize()
    with pytest.raises(RuntimeError, match="TIMEOUT"):
        ctx.sync_status()
    ctx.set_wait_limit(0)
    S["xyzq"].copy_(x0)
    S["vel"].zero_()
    st.step, st.attempt = 0, 0
    ctx.md_init(st)
    ctx.md_segment(st, None, 4)
    torch.cuda.synchronize()
    ctx.sync_status()
    ref, st2, S2, _ = _setup(pkg, b, seed=8, persistent=False)
    ref.md_segment(st2, None, 4)
    torch.cuda.synchronize()
    ref.sync_status()
    assert torch.equal(S["xyzq"], S2["xyzq"]) and torch.equal(S["vel"], S2["vel"])


def test_non_finite_coordinates_are_reported(pkg):
    """A NaN coordinate gives a non-finite Born radius: the evaluation records
    GB_ERR_NONFINITE, and the context evaluates valid input afterwards."""
    import torch
    dev = device()
    b = synth.random_batch([300, 64], seed=22, sites=False)
    ctx = pkg.Context(b.atom_off)
    xyzq = torch.as_tensor(b.xyzq(), device=dev)
    rad = torch.as_tensor(b.rad_screen(), device=dev)
    bad = xyzq.clone()
    bad[17, 0] = float("nan")
    ctx.energy_forces(bad, rad)
    torch.cuda.synchronize()
    with pytest.raises(RuntimeError, match="NONFINITE"):
        ctx.sync_status()
    out = ctx.energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert torch.isfinite(out["F"]).all() and torch.isfinite(out["E"]).all()


def test_simulation_driver_equals_the_state_struct_path(pkg):
    """pkg.Simulation (the Python driver) runs the same MD, MC and exchanges as
    a gb_md_state filled by hand: identical coordinates, site states and
    exchange grid after 60 steps."""
    device()                                   # skips without a GPU
    import torch
    b = synth.config_eremd(4, 300)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         sites=t, pH=b.pH, E=b.E, E_ladder=synth.e_ladder(4), pH_ladder=[b.pH[0]], seed=5,
                         mc_every=5, ex_every=20)
    sim.run(60)
    sim.sync()
    ctx, st, S, sites = _setup(pkg, b, seed=5, mc_every=5, ex_every=20, with_sites=True)
    ctx.md_segment(st, sites, 60)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert sim.step == 60 and st.step == 60
    assert torch.equal(sim.xyzq, S["xyzq"]) and torch.equal(sim.vel, S["vel"])
    assert torch.equal(sim.state, S["state"]) and torch.equal(sim.grid, S["grid"])
    E = sim.energies().cpu().numpy()
    assert E.shape == (4, 3) and np.all(np.isfinite(E))


def test_autotune_md_restores_the_state(pkg):
    """gb_autotune_md times MD segments from a saved state: the state buffers
    and counters come back unchanged, the chosen caps stay on the context, and
    the run that follows equals one on a context given those caps by hand."""
    device()                                   # skips without a GPU
    import torch
    b = synth.config_eremd(4, 300)
    ctx, st, S, sites = _setup(pkg, b, seed=3, mc_every=5, ex_every=20, with_sites=True)
    keys = ("xyzq", "vel", "force", "R", "state", "E", "grid")
    before = {k: S[k].clone() for k in keys}
    caps = ctx.autotune_md(st, sites, trial_steps=20)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert st.step == 0 and st.attempt == 0
    for k in keys:
        assert torch.equal(S[k], before[k]), k
    assert len(caps) == 3 and all(c in (1, 3, 4) for c in caps)
    ctx.md_segment(st, sites, 40)
    ref, st2, S2, sites2 = _setup(pkg, b, seed=3, mc_every=5, ex_every=20, with_sites=True)
    for p, c in enumerate(caps):
        ref.set_reg_cap(c, p)
    ref.md_segment(st2, sites2, 40)
    torch.cuda.synchronize()
    ctx.sync_status()
    ref.sync_status()
    assert torch.equal(S["xyzq"], S2["xyzq"]) and torch.equal(S["state"], S2["state"])


@pytest.mark.parametrize("cutoffs", [{}, dict(rgbmax=12.0, cut=12.0)])
def test_langevin_driver_holds_the_temperature(pkg, cutoffs):
    """2000 BAOAB steps of 8 x 2048 atoms from rest with MC and exchanges: the
    kinetic temperature sum m v^2 / (3 N k_B) over the second half is 300 K
    within 3 % (the thermostat's target; 3N degrees of freedom, no
    constraints; BAOAB's full-step velocities read a little low at 2 fs), and
    nothing diverges."""
    device()                                   # skips without a GPU
    import torch
    b = synth.config_eremd(8, 2048)
    t = b.site_tables(oracle.site_reference_energies(synth.Batch(b.replicas[:1], pH=b.pH[:1], E=b.E[:1]),
                                                     oracle_params()).tolist() * 8)
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(),
                         pkg.default_params(rep_k=100.0, rep_sigma=2.5, **cutoffs), sites=t, pH=b.pH, E=b.E,
                         E_ladder=synth.e_ladder(8), pH_ladder=[b.pH[0]], seed=11)
    sim.run(1000)
    temps = []
    for _ in range(10):
        sim.run(100)
        v = sim.vel[:, :3].double()
        ke = 0.5 * 12.0 * (v * v).sum().item() / 418.4          # kcal/mol (amu A^2/ps^2 -> kcal/mol)
        temps.append(2.0 * ke / (3.0 * b.n_atoms * pkg.KB))
    sim.sync()
    assert torch.isfinite(sim.xyzq).all()
    assert abs(np.mean(temps) / 300.0 - 1.0) < 0.03, temps


def test_simulation_in_sweep_mode_keeps_charges_consistent(pkg):
    """Simulation with mc_mode 1 (every residue once per halt): after a run the
    charges of every site are those of its state."""
    device()                                   # skips without a GPU
    b = synth.config_eremd(4, 300)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         sites=t, pH=b.pH, E=b.E, E_ladder=synth.e_ladder(4), pH_ladder=[b.pH[0]], seed=6,
                         mc_every=5, ex_every=20, mc_mode=1)
    sim.run(100)
    sim.sync()
    x = sim.xyzq.cpu().numpy()
    st = sim.state.cpu().numpy()
    assert st.any()
    for s in range(t["n_sites"]):
        r = np.searchsorted(t["site_off"], s, side="right") - 1
        a0, a1 = t["site_atom_off"][s], t["site_atom_off"][s + 1]
        idx = t["site_atom_idx"][a0:a1] + b.atom_off[r]
        qo = t["site_q_off"][s] + st[s] * (a1 - a0)
        assert np.array_equal(x[idx, 3], t["q_state"][qo:qo + a1 - a0])


def test_host_buffer_segment_equals_the_device_segment(pkg):
    """gb_md_segment_host with the dynamic state in pinned host memory: the
    host arrays after each call equal, bit for bit, the device state of a
    twin run through gb_md_segment (MC every 5 steps, exchanges every 10)."""
    import torch
    b = synth.random_batch([300, 180, 64, 140], seed=12)
    ctx, st, S, sites = _setup(pkg, b, seed=9, mc_every=5, ex_every=10, with_sites=True)
    ctx2, st2, S2, sites2 = _setup(pkg, b, seed=9, mc_every=5, ex_every=10, with_sites=True)
    torch.cuda.synchronize()
    keys = ("xyzq", "vel", "force", "state", "pH", "E", "grid")
    host = {k: S2[k].cpu().pin_memory() for k in keys}
    for k in keys:                              # the device copies of the host run start as garbage
        S2[k].fill_(7)
    for _ in range(3):
        ctx.md_segment(st, sites, 20)
        ctx2.md_segment_host(st2, sites2, 20, host)
        torch.cuda.synchronize()
        for k in keys:
            assert torch.equal(host[k], S[k].cpu()), k
    ctx.sync_status()
    assert st2.step == st.step == 60 and st2.attempt == st.attempt == 6
