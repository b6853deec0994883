"""Statistical validation of the batched C(pH,E)-REMD path on the GPU:
coupled redox and pH sites at frozen coordinates (dt = 0), twelve replicas
on an E ladder, a protonation and a redox attempt every step (Eq. 8, 9) and a
neighbour exchange every second step (Eq. 14, 15).  The populations each E
slot visits are compared with exact enumeration of the joint states (the
oracle's energies and the Eq. 8 / 9 state terms), and the Hill fit of Eq. 3
to the sampled reduced fractions with the fit to the exact curve."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_common import device, oracle_params
from thermo_enum import F, KT, f_protonated, f_reduced, joint_energies

pytestmark = pytest.mark.gpu

M = 12
PH = 4.6


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _hill_fit(E, f):
    """Least-squares E0, n of f = 1 / (1 + exp(n F (E - E0) / kT)) via the
    logit, on points away from 0 and 1."""
    f = np.asarray(f)
    keep = (f > 0.03) & (f < 0.97)
    y = np.log(1.0 / f[keep] - 1.0)           # = n F (E - E0) / kT
    A = np.stack([np.asarray(E)[keep], np.ones(keep.sum())], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, y, rcond=None)
    n = a * KT / F
    return -b / a, n


def test_eremd_frozen_sites_match_enumeration(pkg):
    import torch
    dev = device()
    p = oracle_params()
    rep = synth.make_replica(60, 52, [(1, 8, 2), (0, 6, 2)])
    one = synth.Batch([rep], pH=np.array([PH]), E=np.array([synth.E0_REF_V]))
    G1 = oracle.site_reference_energies(one, p) + np.array([0.0, 0.4, 0.0, -0.3])
    J = joint_energies(oracle, rep, G1, p)

    ladder = synth.E0_REF_V + np.linspace(-0.12, 0.12, M)
    b = synth.Batch([rep] * M, pH=np.full(M, PH), E=ladder.copy(), E_ladder=ladder)
    params = pkg.default_params()
    ctx = pkg.Context(b.atom_off, params)
    t = b.site_tables(np.tile(G1, M))
    sites = pkg.SiteTables(t, M, dev)
    N = b.n_atoms
    S = dict(xyzq=torch.as_tensor(b.xyzq(), device=dev), rad=torch.as_tensor(b.rad_screen(), device=dev),
             vel=torch.zeros((N, 4), dtype=torch.float32, device=dev),
             force=torch.zeros((N, 4), dtype=torch.float32, device=dev),
             R=torch.zeros(N, dtype=torch.float32, device=dev),
             pH=torch.full((M,), PH, dtype=torch.float64, device=dev),
             E=torch.as_tensor(ladder.copy(), device=dev),
             grid=torch.arange(M, dtype=torch.int32, device=dev),
             E_ladder=torch.as_tensor(ladder, device=dev),
             pH_ladder=torch.tensor([PH], dtype=torch.float64, device=dev),
             state=torch.zeros(t["n_sites"], dtype=torch.int32, device=dev))
    st = pkg.MDState()
    for k in ("xyzq", "vel", "force", "R", "pH", "E", "grid", "E_ladder", "pH_ladder", "state"):
        setattr(st, k, S[k].data_ptr())
    st.rad_screen = S["rad"].data_ptr()
    st.n_E, st.n_pH = M, 1
    st.dt, st.friction, st.mass, st.kT = 0.0, 10.0, 12.0, KT      # frozen coordinates
    st.bond_k, st.bond_r0 = 0.0, 1.5
    st.seed, st.step, st.attempt = 2024, 0, 0
    st.mc_every, st.ex_every, st.ex_dim, st.wrap = 1, 2, 0, 0
    ctx.md_init(st)
    x0 = S["xyzq"].clone()

    n_chunks, burn = 6000, 200
    red = np.zeros(M)
    prot = np.zeros(M)
    swaps = 0
    prev = np.arange(M)
    for c in range(n_chunks):
        ctx.md_segment(st, sites, 2)
        grid = S["grid"].cpu().numpy()            # replica at each E slot
        state = S["state"].cpu().numpy().reshape(M, 2)
        swaps += int((grid != prev).sum())
        prev = grid
        if c >= burn:
            red += state[grid, 0] == 0
            prot += state[grid, 1] >= 1
    ctx.sync_status()
    n = n_chunks - burn
    f_red, f_prot = red / n, prot / n
    assert torch.equal(S["xyzq"][:, :3], x0[:, :3])              # coordinates stayed frozen
    assert swaps > 0.2 * n_chunks * M / 2                           # exchanges happen

    exp_red = np.array([f_reduced(J, E, PH) for E in ladder])
    exp_prot = np.array([f_protonated(J, E, PH) for E in ladder])
    # correlated samples (a few attempts per decorrelation): ~4.5 standard
    # errors of an effective sample of n / 4
    tol = 4.5 * np.sqrt(np.maximum(exp_red * (1 - exp_red), 0.02) / (n / 4))
    assert np.all(np.abs(f_red - exp_red) <= tol), (f_red, exp_red)
    tol_p = 4.5 * np.sqrt(np.maximum(exp_prot * (1 - exp_prot), 0.02) / (n / 4))
    assert np.all(np.abs(f_prot - exp_prot) <= tol_p), (f_prot, exp_prot)
    # Eq. 3 fits: midpoint within 4 mV, Hill coefficient within 0.12
    E0_s, n_s = _hill_fit(ladder, f_red)
    E0_x, n_x = _hill_fit(ladder, exp_red)
    print(f"max |f_red - exact| {np.abs(f_red - exp_red).max():.4f}, "
          f"max |f_prot - exact| {np.abs(f_prot - exp_prot).max():.4f}, "
          f"Eq. 3 fit E0 {E0_s * 1e3:.2f} mV (exact {E0_x * 1e3:.2f}), n {n_s:.3f} (exact {n_x:.3f})")
    assert abs(E0_s - E0_x) < 4e-3, (E0_s, E0_x)
    assert abs(n_s - n_x) < 0.12, (n_s, n_x)
