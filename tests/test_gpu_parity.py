"""GPU parity of the C-ABI hot path against the FP64 oracle (small and ragged
cases, element by element).  Tolerances are the spec bars: energy
relative 1e-6, forces 1e-3 kcal/mol/A max-abs, dG 1e-3 kcal/mol, decisions
identical except where |dG - threshold| is inside the dG tolerance."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import (DG_ABS, E_REL, F_ABS, KT, PHI_ABS, R_REL, device, energy_rel_err,
                        oracle_params, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _run(pkg, batch, **tiles):
    import torch
    dev = device()
    xyzq, rad = to_dev(batch, dev)
    ctx = pkg.Context(batch.atom_off)
    if tiles:
        ctx.set_tiles(tiles.get("wpb", 8), tiles.get("tpt", 4))
    out = ctx.energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    ctx.sync_status()
    return {k: v.cpu().numpy() for k, v in out.items()}, ctx


def _compare(batch, out, ref):
    e = energy_rel_err(out["E"], ref["E"])
    assert e.max() <= E_REL, f"energy relative error {e.max():.3e}"
    fe = np.abs(out["F"] - ref["F"]).max() if ref["F"].size else 0.0
    assert fe <= F_ABS, f"force max-abs error {fe:.3e}"
    rr = np.abs(out["R"] - ref["R"]) / ref["R"] if ref["R"].size else np.zeros(1)
    assert rr.max() <= R_REL, f"Born radius relative error {rr.max():.3e}"
    pe = np.abs(out["dEdq"] - ref["phi"]).max() if ref["phi"].size else 0.0
    assert pe <= PHI_ABS, f"dE/dq max-abs error {pe:.3e}"


def test_plain_256_atoms(pkg):
    b = synth.config_plain()
    out, _ = _run(pkg, b)
    ref = oracle.batch_energy_forces(b, oracle_params(), with_phi=True)
    _compare(b, out, ref)
    # fixed-point forces are the float forces' source
    assert np.allclose(out["F_fixed"].T / 2.0 ** 32, out["F"], atol=1e-6)


@pytest.mark.parametrize("sizes", [[1, 2, 31, 32, 33], [0, 5, 64, 0, 97, 130], [300, 1, 257]])
def test_ragged_uneven_batch(pkg, sizes):
    b = synth.random_batch(sizes, seed=len(sizes))
    out, _ = _run(pkg, b)
    ref = oracle.batch_energy_forces(b, oracle_params(), with_phi=True)
    _compare(b, out, ref)


def test_isolated_ion_and_empty_replica(pkg):
    b = synth.random_batch([1, 0, 1], seed=9, sites=False)
    out, _ = _run(pkg, b)
    rho = b.rad_screen()[:, 0].astype(np.float64)
    q = b.xyzq()[:, 3].astype(np.float64)
    a = rho - np.float32(0.09)
    tau = 1 - 1 / 78.5
    expect = -0.5 * oracle.KE * tau * q ** 2 / a
    assert np.allclose(out["R"], a, rtol=1e-7)
    assert np.allclose(out["E"][[0, 2], 0], expect, rtol=1e-7)
    assert out["E"][1].tolist() == [0.0, 0.0, 0.0]
    assert np.all(out["F"] == 0)


def test_batched_equals_single_bitwise(pkg):
    b = synth.random_batch([200, 77, 130], seed=5)
    out, _ = _run(pkg, b)
    for k, rep in enumerate(b.replicas):
        single = synth.Batch([rep], pH=b.pH[:1], E=b.E[:1])
        o1, _ = _run(pkg, single)
        a, c = b.atom_off[k], b.atom_off[k + 1]
        assert np.array_equal(o1["F_fixed"], out["F_fixed"][:, a:c])
        assert np.array_equal(o1["R"], out["R"][a:c])


def test_repeat_and_tile_shapes_bitwise(pkg):
    b = synth.random_batch([500, 260], seed=6)
    ref, _ = _run(pkg, b)
    for wpb, tpt in [(8, 1), (4, 3), (2, 17), (8, 64)]:
        o, _ = _run(pkg, b, wpb=wpb, tpt=tpt)
        assert np.array_equal(o["F_fixed"], ref["F_fixed"]), (wpb, tpt)
        assert np.array_equal(o["R"], ref["R"])
        assert np.array_equal(o["E"], ref["E"])


def test_register_caps_and_autotune_bitwise(pkg):
    """Register caps change only scheduling: results stay bitwise identical,
    per pass and for the autotuner's choice."""
    import torch
    b = synth.random_batch([500, 260, 33], seed=7)
    ref, _ = _run(pkg, b)
    xyzq, rad = to_dev(b, device())
    for caps in [(1, 1, 1), (4, 4, 4), (1, 3, 4), (4, 1, 3)]:
        ctx = pkg.Context(b.atom_off)
        for p, c in enumerate(caps):
            ctx.set_reg_cap(c, p)
        assert ctx.reg_caps() == caps
        o = {k: v.cpu().numpy() for k, v in ctx.energy_forces(xyzq, rad).items()}
        ctx.sync_status()
        for k in ("F_fixed", "R", "E", "dEdq"):
            assert np.array_equal(o[k], ref[k]), (caps, k)
    ctx = pkg.Context(b.atom_off)
    ctx.autotune(xyzq, rad)
    assert all(c in (1, 3, 4) for c in ctx.reg_caps())
    o = {k: v.cpu().numpy() for k, v in ctx.energy_forces(xyzq, rad).items()}
    torch.cuda.synchronize()
    ctx.sync_status()
    for k in ("F_fixed", "R", "E", "dEdq"):
        assert np.array_equal(o[k], ref[k]), k
    with pytest.raises(Exception):
        ctx.set_reg_cap(2, 0)


def test_charge_derivative_sums_to_twice_energy(pkg):
    b = synth.random_batch([400], seed=12)
    out, _ = _run(pkg, b)
    q = b.xyzq()[:, 3].astype(np.float64)
    E = out["E"][0, 0] + out["E"][0, 1]
    # both sides are sums of the same FP32 pair terms rounded differently:
    # bound by FP32 resolution on the sum of magnitudes, not on the cancelled total
    scale = np.abs(q * out["dEdq"]).sum()
    assert abs((q * out["dEdq"]).sum() - 2 * E) <= 2e-6 * scale


def test_net_force_vanishes(pkg):
    b = synth.config_plain()
    out, _ = _run(pkg, b)
    assert np.abs(out["F"].sum(0)).max() < 1e-3


# --- Monte Carlo ------------------------------------------------------------------

def _mc_case(pkg, batch, kinds, n_steps, seed=21):
    import torch
    dev = device()
    p = oracle_params()
    G = oracle.site_reference_energies(batch, p)
    t = batch.site_tables(G)
    xyzq, rad = to_dev(batch, dev)
    ctx = pkg.Context(batch.atom_off)
    R = ctx.born_radii(xyzq, rad)
    sites = pkg.SiteTables(t, batch.n_rep, dev)
    state = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
    pH = torch.as_tensor(batch.pH, device=dev)
    E = torch.as_tensor(batch.E, device=dev)
    x, q, rho, scr, off = oracle.batch_arrays(batch)
    q = q.copy()
    st = batch.initial_states()
    Rn = R.double().cpu().numpy()
    mism, near = 0, 0
    for step in range(n_steps):
        for kind in kinds:
            dG, acc = ctx.mc_step(sites, xyzq, R, pH, E, KT, seed, step, kind, state)
            o = oracle.mc_step(off, x, q, Rn, t, st, batch.pH, batch.E, KT, seed, step, kind, p)
            dG, acc = dG.cpu().numpy(), acc.cpu().numpy()
            has = o["site"] >= 0
            assert np.all(np.abs(dG[has] - o["dG"][has]) <= DG_ABS), (step, kind, dG, o["dG"])
            resync = False
            for r in np.flatnonzero(has):
                if acc[r] != o["acc"][r]:
                    if abs(o["dG"][r] - o["thresh"][r]) <= DG_ABS:
                        near += 1          # reported, not a mismatch
                        resync = True
                    else:
                        mism += 1
            if resync:  # follow the oracle so both chains stay in step
                state.copy_(torch.as_tensor(st, device=dev))
                xyzq[:, 3] = torch.as_tensor(q, dtype=torch.float32, device=dev)
            assert np.array_equal(state.cpu().numpy(), st), (step, kind)
            assert np.array_equal(xyzq[:, 3].cpu().numpy().astype(np.float64), q)
    assert mism == 0
    return state.cpu().numpy()


def test_mc_plain_decisions_match_oracle(pkg):
    b = synth.config_plain()
    _mc_case(pkg, b, (0, 1), 40)


def test_mc_uneven_multistate_sites(pkg):
    reps = [synth.make_replica(n, 40 + k, specs) for k, (n, specs) in enumerate([
        (90, [(1, 8, 2), (0, 6, 4), (0, 9, 3)]),
        (45, [(0, 12, 5)]),
        (60, []),
        (150, [(1, 30, 2), (1, 20, 2), (0, 10, 2)]),
    ])]
    b = synth.Batch(reps, pH=np.array([4.0, 4.85, 5.0, 4.4]),
                    E=synth.E0_REF_V + np.array([0.0, 0.02, -0.01, 0.05]))
    _mc_case(pkg, b, (0, 1), 25)


# --- exchange ----------------------------------------------------------------------

@pytest.mark.parametrize("M,wrap", [(8, 1), (7, 1), (6, 0), (2, 1)])
def test_exchange_matches_oracle(pkg, M, wrap):
    import torch
    dev = device()
    rng = np.random.default_rng(M)
    ladder = synth.e_ladder(M)
    counts = rng.integers(0, 3, size=M).astype(np.int32)
    rep_o = rng.permutation(M).astype(np.int32)
    rep_g = torch.as_tensor(rep_o.copy(), device=dev)
    vals = torch.as_tensor(ladder, device=dev)
    cnt = torch.as_tensor(counts, device=dev)
    vor = torch.zeros(M, dtype=torch.float64, device=dev)
    for attempt in range(30):
        d_o, a_o = oracle.exchange(ladder, rep_o, counts, 0, attempt, 77, KT, wrap=bool(wrap))
        d_g, a_g = pkg.eremd_exchange(vals, rep_g, cnt, 0, attempt, 77, KT, wrap=wrap, value_of_rep=vor)
        d_g, a_g = d_g.cpu().numpy(), a_g.cpu().numpy()
        paired = ~np.isnan(d_o)
        assert np.array_equal(paired, ~np.isnan(d_g))
        assert np.allclose(d_g[paired], d_o[paired], rtol=1e-12, atol=1e-12)
        assert np.array_equal(a_g, a_o)
        assert np.array_equal(rep_g.cpu().numpy(), rep_o)
    # value_of_rep agrees with the final permutation for every paired slot
    v = vor.cpu().numpy()
    for k, r in enumerate(rep_o):
        if v[r] != 0.0:
            assert v[r] == ladder[k]


def test_exchange_grid_lines(pkg):
    import torch
    dev = device()
    n_pH, n_E = 3, 4
    grid_o = np.arange(n_pH * n_E, dtype=np.int32)
    grid_g = torch.as_tensor(grid_o.copy(), device=dev)
    counts = np.arange(n_pH * n_E, dtype=np.int32) % 3
    cnt = torch.as_tensor(counts, device=dev)
    for attempt in range(8):
        lad = synth.e_ladder(n_E)
        oracle.exchange(lad, grid_o, counts, 0, attempt, 5, KT, wrap=False, n_ladders=n_pH,
                        ladder_len=n_E, ladder_stride=n_E, slot_stride=1)
        pkg.eremd_exchange(torch.as_tensor(lad, device=dev), grid_g, cnt, 0, attempt, 5, KT, wrap=0,
                           n_ladders=n_pH, ladder_len=n_E, ladder_stride=n_E, slot_stride=1)
        lp = 3.5 + 0.5 * np.arange(n_pH)
        oracle.exchange(lp, grid_o, counts, 1, attempt, 6, KT, wrap=False, n_ladders=n_E,
                        ladder_len=n_pH, ladder_stride=1, slot_stride=n_E)
        pkg.eremd_exchange(torch.as_tensor(lp, device=dev), grid_g, cnt, 1, attempt, 6, KT, wrap=0,
                           n_ladders=n_E, ladder_len=n_pH, ladder_stride=1, slot_stride=n_E)
        assert np.array_equal(grid_g.cpu().numpy(), grid_o)


def test_batch_of_empty_replicas(pkg):
    """Every replica empty (N = 0): energies are zero, the per-atom outputs
    empty, and an MD segment with Monte Carlo and exchanges runs to the
    end with nothing to move."""
    import torch
    dev = device()
    b = synth.random_batch([0, 0, 0], seed=10, sites=False)
    assert b.n_atoms == 0
    ctx = pkg.Context(b.atom_off)
    xyzq, rad = to_dev(b, dev)
    out = ctx.energy_forces(xyzq, rad)
    R = ctx.born_radii(xyzq, rad)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert out["E"].shape == (3, 3) and bool((out["E"] == 0).all())
    assert out["F"].numel() == 0 and R.numel() == 0
    sim = pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                         pH=b.pH, E=b.E)
    sim.run(25)
    sim.sync()
    assert sim.step == 25
