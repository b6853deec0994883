"""Device-side error reporting on bad input, and no write outside the caller's
buffers.

Every fault here is made on the host side of the data: a site table entry,
a state or a coordinate is set to a wrong value before the call.  The kernels
check these values before they use them as indices (a corrupt table never
reaches memory), so no case can fault the GPU: each must come back as an
error code from gb_sync_status with the affected attempt skipped and every
other replica's result unchanged."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_common import F_ABS, KT, R_REL, device, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _mc_setup(pkg, b, dev):
    import torch
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    ctx = pkg.Context(b.atom_off)
    xyzq = torch.as_tensor(b.xyzq(), device=dev)
    rad = torch.as_tensor(b.rad_screen(), device=dev)
    R = ctx.born_radii(xyzq, rad)
    sites = pkg.SiteTables(t, b.n_rep, dev)
    state = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
    pH = torch.as_tensor(b.pH, device=dev)
    E = torch.as_tensor(b.E, device=dev)
    return t, ctx, xyzq, R, sites, state, pH, E


def _rep_sites(t, r):
    return np.arange(t["site_off"][r], t["site_off"][r + 1])


def _rep_atoms(b, r):
    return np.arange(b.atom_off[r], b.atom_off[r + 1])


def test_site_atom_index_out_of_range_skips_only_that_replica(pkg):
    """The first atom of every site of replica 0 points one past the
    replica's end (the next replica's first atom: a silent wrong answer
    without the check).  Single-site attempts and sweeps of replica 0 are
    skipped (NaN dG / "not visited", no state or charge change) and
    GB_ERR_INVALID_ARG is recorded; replicas 1 and 2 give bit-identical
    results to an uncorrupted run."""
    import torch
    dev = device()
    b = synth.random_batch([300, 64, 129], seed=31)
    t, ctx, xyzq, R, sites, state, pH, E = _mc_setup(pkg, b, dev)
    _, ctx_ok, xyzq_ok, _, sites_ok, state_ok, _, _ = _mc_setup(pkg, b, dev)
    n0 = int(b.atom_off[1])
    for s in _rep_sites(t, 0):
        sites.t["site_atom_idx"][int(t["site_atom_off"][s])] = n0
    rest = np.concatenate([_rep_sites(t, 1), _rep_sites(t, 2)])
    for step in range(12):
        for kind in (0, 1):
            dG, acc = ctx.mc_step(sites, xyzq, R, pH, E, KT, 5, step, kind, state)
            dG_ok, acc_ok = ctx_ok.mc_step(sites_ok, xyzq_ok, R, pH, E, KT, 5, step, kind, state_ok)
            torch.cuda.synchronize()
            with pytest.raises(RuntimeError, match="INVALID_ARG"):
                ctx.sync_status()
            ctx_ok.sync_status()
            assert torch.isnan(dG[0]) and int(acc[0]) == 0
            assert torch.equal(dG[1:], dG_ok[1:]) and torch.equal(acc[1:], acc_ok[1:])
            assert torch.equal(state[_rep_sites(t, 0)], torch.zeros(len(_rep_sites(t, 0)), dtype=torch.int32,
                                                                     device=dev))
            assert torch.equal(state[rest], state_ok[rest])
    q0 = torch.as_tensor(b.xyzq(), device=dev)[:, 3]
    assert torch.equal(xyzq[_rep_atoms(b, 0), 3], q0[_rep_atoms(b, 0)])
    assert torch.equal(xyzq[n0:], xyzq_ok[n0:])
    for step in range(4):
        for kind in (0, 1):
            dG, acc = ctx.mc_sweep(sites, xyzq, R, pH, E, KT, 6, step, kind, state)
            dG_ok, acc_ok = ctx_ok.mc_sweep(sites_ok, xyzq_ok, R, pH, E, KT, 6, step, kind, state_ok)
            torch.cuda.synchronize()
            with pytest.raises(RuntimeError, match="INVALID_ARG"):
                ctx.sync_status()
            ctx_ok.sync_status()
            s0 = _rep_sites(t, 0)
            assert (acc[s0] == 2).all() and (dG[s0] == 0).all()
            assert torch.equal(dG[rest], dG_ok[rest]) and torch.equal(acc[rest], acc_ok[rest])
            assert torch.equal(state[rest], state_ok[rest])
    assert torch.equal(xyzq[_rep_atoms(b, 0), 3], q0[_rep_atoms(b, 0)])
    assert torch.equal(xyzq[n0:], xyzq_ok[n0:])


def test_negative_site_atom_index_is_rejected(pkg):
    """A negative atom index (the previous replica's last atom) in a site of
    the middle replica: its attempts are skipped with GB_ERR_INVALID_ARG."""
    import torch
    dev = device()
    b = synth.random_batch([200, 96, 150], seed=32)
    t, ctx, xyzq, R, sites, state, pH, E = _mc_setup(pkg, b, dev)
    for s in _rep_sites(t, 1):
        a0, a1 = int(t["site_atom_off"][s]), int(t["site_atom_off"][s + 1])
        sites.t["site_atom_idx"][a1 - 1] = -1
    q_before = xyzq[:, 3].clone()
    for step in range(6):
        for kind in (0, 1):
            dG, acc = ctx.mc_step(sites, xyzq, R, pH, E, KT, 8, step, kind, state)
            torch.cuda.synchronize()
            with pytest.raises(RuntimeError, match="INVALID_ARG"):
                ctx.sync_status()
            assert torch.isnan(dG[1]) and int(acc[1]) == 0
    a1 = _rep_atoms(b, 1)
    assert torch.equal(xyzq[a1, 3], q_before[a1])
    assert (state[_rep_sites(t, 1)] == 0).all()


def test_state_out_of_range_is_rejected(pkg):
    """States outside [0, nstates) in replica 0 (7 on its two-state redox
    site, -1 on its three-state protonation site): gb_count_bound gives -1
    for that replica and the right counts for the others; MC attempts on it
    are skipped with GB_ERR_INVALID_ARG and the corrupt states stay as they
    were; replica 1 proceeds as in an uncorrupted run."""
    import torch
    dev = device()
    b = synth.random_batch([150, 90], seed=33)
    t, ctx, xyzq, R, sites, state, pH, E = _mc_setup(pkg, b, dev)
    _, ctx_ok, xyzq_ok, _, sites_ok, state_ok, _, _ = _mc_setup(pkg, b, dev)
    s0 = _rep_sites(t, 0)
    kinds = np.asarray(t["site_kind"])
    s_redox = int(s0[kinds[s0] == 1][0])
    s_prot = int(s0[kinds[s0] == 0][0])
    state[s_redox] = 7
    state[s_prot] = -1
    st_ok = np.zeros(t["n_sites"], np.int64)
    for kind, table in ((1, "n_e"), (0, "n_H")):
        cnt = pkg.count_bound(sites, state, kind)
        torch.cuda.synchronize()
        assert int(cnt[0]) == -1
        so = np.asarray(t["site_state_off"])
        tab = np.asarray(t[table])
        want = sum(int(tab[so[s] + st_ok[s]]) for s in _rep_sites(t, 1) if kinds[s] == kind)
        assert int(cnt[1]) == want
    for step in range(8):
        for kind in (0, 1):
            dG, acc = ctx.mc_step(sites, xyzq, R, pH, E, KT, 12, step, kind, state)
            dG_ok, acc_ok = ctx_ok.mc_step(sites_ok, xyzq_ok, R, pH, E, KT, 12, step, kind, state_ok)
            torch.cuda.synchronize()
            with pytest.raises(RuntimeError, match="INVALID_ARG"):
                ctx.sync_status()
            ctx_ok.sync_status()
            assert torch.isnan(dG[0]) and int(acc[0]) == 0
            assert torch.equal(dG[1:], dG_ok[1:]) and torch.equal(acc[1:], acc_ok[1:])
    assert int(state[s_redox]) == 7 and int(state[s_prot]) == -1
    s1 = _rep_sites(t, 1)
    assert torch.equal(state[s1], state_ok[s1])
    a0 = _rep_atoms(b, 0)
    assert torch.equal(xyzq[a0, 3], torch.as_tensor(b.xyzq(), device=dev)[a0, 3])


def test_exchange_with_a_corrupt_state_is_skipped(pkg):
    """E-REMD inside the MD driver with replica 0's redox state out of range:
    every exchange that would count its electrons is skipped, so replica 0
    keeps slot 0 and its ladder value, and gb_sync_status reports
    GB_ERR_INVALID_ARG."""
    import torch
    device()
    b = synth.random_batch([120, 120, 120, 120], seed=34)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    lad = synth.e_ladder(b.n_rep)
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         sites=t, pH=b.pH, E=lad, E_ladder=lad, mc_every=0, ex_every=1, seed=4)
    kinds = np.asarray(t["site_kind"])
    s0 = _rep_sites(t, 0)
    sim.state[int(s0[kinds[s0] == 1][0])] = 7
    sim.run(6)
    torch.cuda.synchronize()
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        sim.sync()
    assert int(sim.grid[0]) == 0
    assert float(sim.E[0]) == float(lad[0])
    g = sim.grid.cpu().numpy()
    assert sorted(g.tolist()) == list(range(b.n_rep))


@pytest.mark.parametrize("cut", [0.0, 12.0])
@pytest.mark.parametrize("j", [5, 250])
def test_coincident_atoms_are_reported(pkg, cut, j):
    """Atom j moved onto atom 4 of the same replica (same tile for j = 5, a
    block off the diagonal for j = 250), without and with the cutoffs: the
    Born pass records GB_ERR_NONFINITE, and the same context then evaluates
    valid input to the same result as a fresh one."""
    import torch
    dev = device()
    b = synth.random_batch([300, 64], seed=35, sites=False)
    params = pkg.default_params(rgbmax=cut, cut=cut)
    ctx = pkg.Context(b.atom_off, params)
    xyzq = torch.as_tensor(b.xyzq(), device=dev)
    rad = torch.as_tensor(b.rad_screen(), device=dev)
    bad = xyzq.clone()
    bad[j, :3] = bad[4, :3]
    ctx.energy_forces(bad, rad)
    torch.cuda.synchronize()
    with pytest.raises(RuntimeError, match="NONFINITE"):
        ctx.sync_status()
    out = ctx.energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    ctx.sync_status()
    ref = pkg.Context(b.atom_off, params).energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    for k in ("R", "F_fixed", "E", "dEdq"):
        assert torch.equal(out[k], ref[k]), k


def test_close_but_distinct_atoms_are_not_reported(pkg):
    """Two atoms 0.01 A apart are far above the coincidence bound: no error."""
    import torch
    dev = device()
    b = synth.random_batch([300], seed=36, sites=False)
    ctx = pkg.Context(b.atom_off)
    xyzq = torch.as_tensor(b.xyzq(), device=dev)
    rad = torch.as_tensor(b.rad_screen(), device=dev)
    xyzq[9, :3] = xyzq[8, :3] + torch.tensor([0.01, 0.0, 0.0], device=dev)
    out = ctx.energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert torch.isfinite(out["R"]).all() and torch.isfinite(out["E"]).all()


# --- canaries: nothing is written outside the caller's buffers ----------------------

GUARD = 4096            # bytes of guard on each side (keeps 256-byte alignment)
CANARY = 0xA5


def _guarded(n, dtype, dev, fill=None):
    """A view of n elements of dtype inside a byte buffer whose guard bytes
    on both sides hold CANARY; returns (whole, view)."""
    import torch
    item = torch.empty(0, dtype=dtype).element_size()
    whole = torch.full((2 * GUARD + n * item,), CANARY, dtype=torch.uint8, device=dev)
    view = whole[GUARD:GUARD + n * item].view(dtype)
    if fill is not None:
        view.copy_(fill.reshape(-1).to(dtype))
    return whole, view


def _guards_intact(whole):
    import torch
    torch.cuda.synchronize()
    return bool((whole[:GUARD] == CANARY).all()) and bool((whole[-GUARD:] == CANARY).all())


@pytest.mark.parametrize("cut", [0.0, 12.0])
def test_energy_outputs_stay_inside_their_buffers(pkg, cut):
    """R, F_fixed, F, E and dEdq of gb_energy_forces (and gb_born_radii's R)
    written into guarded views: every guard byte is unchanged, and the
    results equal those of plain buffers."""
    import torch
    dev = device()
    b = synth.random_batch([300, 64, 129], seed=37, sites=False)
    ctx = pkg.Context(b.atom_off, pkg.default_params(rgbmax=cut, cut=cut))
    N, M = b.n_atoms, b.n_rep
    xyzq_w, xyzq = _guarded(4 * N, torch.float32, dev, torch.as_tensor(b.xyzq(), device=dev))
    rad_w, rad = _guarded(2 * N, torch.float32, dev, torch.as_tensor(b.rad_screen(), device=dev))
    bufs = dict(R=_guarded(N, torch.float32, dev), F_fixed=_guarded(3 * N, torch.int64, dev),
                F=_guarded(3 * N, torch.float32, dev), E=_guarded(3 * M, torch.float64, dev),
                dEdq=_guarded(N, torch.float64, dev))
    p = {k: v[1].data_ptr() for k, v in bufs.items()}
    rc = ctx.lib.gb_energy_forces(ctx.h, xyzq.data_ptr(), rad.data_ptr(), p["R"], p["F_fixed"], p["F"],
                                  p["E"], p["dEdq"], None)
    assert rc == 0
    ctx.sync_status()
    for k, (w, _) in bufs.items():
        assert _guards_intact(w), k
    assert _guards_intact(xyzq_w) and _guards_intact(rad_w)
    ref = ctx.energy_forces(xyzq.view(N, 4), rad.view(N, 2))
    torch.cuda.synchronize()
    assert torch.equal(bufs["R"][1], ref["R"]) and torch.equal(bufs["E"][1].view(M, 3), ref["E"])
    assert torch.equal(bufs["F_fixed"][1].view(3, N), ref["F_fixed"])
    assert torch.equal(bufs["dEdq"][1], ref["dEdq"])
    Rw, Rv = _guarded(N, torch.float32, dev)
    assert ctx.lib.gb_born_radii(ctx.h, xyzq.data_ptr(), rad.data_ptr(), Rv.data_ptr(), None) == 0
    assert _guards_intact(Rw) and torch.equal(Rv, ref["R"])


def test_mc_exchange_and_count_outputs_stay_inside_their_buffers(pkg):
    """Single-site attempts, sweeps, gb_count_bound and eremd_exchange with
    every written array (charges, states, dG, acc, counts, ladder slots,
    values, exchange outputs) a guarded view: all guard bytes unchanged, and
    states and charges equal to a run on plain buffers."""
    import torch
    dev = device()
    b = synth.random_batch([300, 64, 129, 45], seed=38)
    t, ctx, xyzq_p, R, sites, state_p, pH, E = _mc_setup(pkg, b, dev)
    N, M, S = b.n_atoms, b.n_rep, int(t["n_sites"])
    xyzq_w, xyzq = _guarded(4 * N, torch.float32, dev, xyzq_p)
    state_w, state = _guarded(S, torch.int32, dev, state_p)
    xyzq = xyzq.view(N, 4)
    walls = [xyzq_w, state_w]
    for step in range(6):
        for kind in (0, 1):
            dw, dG = _guarded(M, torch.float64, dev)
            aw, acc = _guarded(M, torch.uint8, dev)
            ctx.mc_step(sites, xyzq, R, pH, E, KT, 3, step, kind, state, dG_out=dG, acc_out=acc)
            ctx.mc_step(sites, xyzq_p, R, pH, E, KT, 3, step, kind, state_p)
            dw2, dG2 = _guarded(S, torch.float64, dev)
            aw2, acc2 = _guarded(S, torch.uint8, dev)
            ctx.mc_sweep(sites, xyzq, R, pH, E, KT, 4, step, kind, state, dG_out=dG2, acc_out=acc2)
            ctx.mc_sweep(sites, xyzq_p, R, pH, E, KT, 4, step, kind, state_p)
            cw, cnt = _guarded(M, torch.int32, dev)
            pkg.count_bound(sites, state, kind, out=cnt)
            walls += [dw, aw, dw2, aw2, cw]
    ctx.sync_status()
    assert all(_guards_intact(w) for w in walls)
    assert torch.equal(state, state_p) and torch.equal(xyzq, xyzq_p)
    lad = torch.as_tensor(synth.e_ladder(M), device=dev)
    counts = pkg.count_bound(sites, state, 1)
    rw, rep = _guarded(M, torch.int32, dev, torch.arange(M, device=dev))
    vw, vor = _guarded(M, torch.float64, dev, torch.zeros(M, device=dev))
    for attempt in range(5):
        dw, d = _guarded(M, torch.float64, dev)
        aw, a = _guarded(M, torch.uint8, dev)
        pkg.eremd_exchange(lad, rep, counts, 0, attempt, 9, KT, wrap=True, value_of_rep=vor,
                           delta_out=d, acc_out=a)
        assert _guards_intact(dw) and _guards_intact(aw)
    assert _guards_intact(rw) and _guards_intact(vw)
    assert sorted(rep.cpu().tolist()) == list(range(M))


def test_static_entry_outputs_stay_inside_their_buffers(pkg):
    """gb_energy_forces_static with guarded outputs: guards unchanged and
    results equal to those of a context."""
    import torch
    dev = device()
    b = synth.random_batch([777], seed=39, sites=False)
    n = b.n_atoms
    params = pkg.default_params()
    xyzq = torch.as_tensor(b.xyzq(), device=dev)
    rad = torch.as_tensor(b.rad_screen(), device=dev)
    bufs = dict(R=_guarded(n, torch.float32, dev), F_fixed=_guarded(3 * n, torch.int64, dev),
                F=_guarded(3 * n, torch.float32, dev), E=_guarded(3, torch.float64, dev),
                dEdq=_guarded(n, torch.float64, dev))
    p = {k: v[1].data_ptr() for k, v in bufs.items()}
    lib = pkg.load()
    f = lib.gb_energy_forces_static
    f.argtypes = [C.c_int32, C.POINTER(pkg.Params)] + [C.c_void_p] * 8
    f.restype = C.c_int
    rc = f(n, C.byref(params), xyzq.data_ptr(), rad.data_ptr(), p["R"], p["F_fixed"], p["F"], p["E"],
           p["dEdq"], None)
    assert rc == 0
    for k, (w, _) in bufs.items():
        assert _guards_intact(w), k
    ref = pkg.Context(b.atom_off, params).energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    # the static path proves no block far, so its terms may take the other
    # polynomial branch: equal within the parity bounds, not bit for bit
    R = bufs["R"][1].double().cpu().numpy()
    R_ref = ref["R"].double().cpu().numpy()
    assert np.max(np.abs(R - R_ref) / R_ref) <= R_REL
    F = bufs["F"][1].view(n, 3).cpu().numpy()
    assert np.abs(F - ref["F"].cpu().numpy()).max() <= F_ABS
