"""GPU GB with Debye-Hueckel salt screening (gb_params.kappa) against the FP64
oracle: energies, forces, Born radii and dE/dq element by element on ragged
batches, the Monte Carlo energy change, and kappa = 0 bitwise equal to the
default (unscreened) parameters."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import DG_ABS, E_REL, F_ABS, KT, PHI_ABS, R_REL, device, energy_rel_err, oracle_params, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _run(pkg, b, kappa):
    import torch
    xyzq, rad = to_dev(b, device())
    ctx = pkg.Context(b.atom_off, pkg.default_params(kappa=kappa))
    out = ctx.energy_forces(xyzq, rad)
    torch.cuda.synchronize()
    ctx.sync_status()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("kappa", [0.05, 0.125, 0.5])
def test_salt_energy_forces_match_oracle(pkg, kappa):
    b = synth.random_batch([300, 64, 33, 1], seed=17)
    out = _run(pkg, b, kappa)
    p = oracle_params(kappa=float(np.float32(kappa)))
    ref = oracle.batch_energy_forces(b, p, with_phi=True)
    assert energy_rel_err(out["E"], ref["E"]).max() <= E_REL
    assert np.abs(out["F"] - ref["F"]).max() <= F_ABS
    assert np.max(np.abs(out["R"] - ref["R"]) / ref["R"]) <= R_REL
    assert np.abs(out["dEdq"] - ref["phi"]).max() <= PHI_ABS


def test_kappa_zero_is_the_unscreened_path(pkg):
    b = synth.random_batch([200, 77], seed=18)
    import torch
    a = _run(pkg, b, 0.0)
    xyzq, rad = to_dev(b, device())
    ctx = pkg.Context(b.atom_off)                       # parameters without the salt field set
    d = {k: v.cpu().numpy() for k, v in ctx.energy_forces(xyzq, rad).items()}
    torch.cuda.synchronize()
    for k in ("F_fixed", "R", "E", "dEdq"):
        assert np.array_equal(a[k], d[k])
    s = _run(pkg, b, 0.2)
    assert not np.array_equal(a["E"], s["E"])           # the screening is live


def test_salt_mc_energy_change_matches_oracle(pkg):
    import torch
    dev = device()
    kappa = 0.1
    p = oracle_params(kappa=float(np.float32(kappa)))
    b = synth.config_plain()
    G = oracle.site_reference_energies(b, p)
    t = b.site_tables(G)
    xyzq, rad = to_dev(b, dev)
    ctx = pkg.Context(b.atom_off, pkg.default_params(kappa=kappa))
    R = ctx.born_radii(xyzq, rad)
    sites = pkg.SiteTables(t, 1, dev)
    state = torch.zeros(t["n_sites"], dtype=torch.int32, device=dev)
    pH, E = torch.as_tensor(b.pH, device=dev), torch.as_tensor(b.E, device=dev)
    x, q, rho, scr, off = oracle.batch_arrays(b)
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
