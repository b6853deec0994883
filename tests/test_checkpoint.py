"""Checkpoint / resume of the MD driver: the file format on the CPU, and on
the GPU a resumed run that must equal the uninterrupted one bit for bit
(counter-based random numbers, forces recomputed by the kernels a step ends
with)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import device, oracle_params


def test_checkpoint_file_round_trip(tmp_path):
    import paper_1803_09652_gb300 as pkg
    rng = np.random.default_rng(0)
    ck = {"xyzq": rng.normal(size=(37, 4)).astype(np.float32),
          "vel": rng.normal(size=(37, 4)).astype(np.float32),
          "state": rng.integers(0, 3, size=5).astype(np.int32),
          "grid": rng.permutation(4).astype(np.int32),
          "pH": rng.normal(size=4), "E": rng.normal(size=4),
          "step": 123456789012, "attempt": 77, "seed": 2 ** 63 + 5}
    p = str(tmp_path / "ck.npz")
    pkg.save_checkpoint(p, ck)
    back = pkg.load_checkpoint(p)
    assert set(back) == set(ck)
    for k, v in ck.items():
        if isinstance(v, int):
            assert back[k] == v and isinstance(back[k], int), k
        else:
            assert back[k].dtype == v.dtype and np.array_equal(back[k], v), k


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as p
    return p


def _sim(pkg, b, t, lad, mc_mode):
    return pkg.Simulation(b.atom_off, b.xyzq(), b.rad_screen(), pkg.default_params(rep_k=100.0, rep_sigma=2.5),
                          sites=t, pH=b.pH, E=lad, E_ladder=lad, mc_every=5, ex_every=10, seed=11,
                          mc_mode=mc_mode)


@pytest.mark.gpu
@pytest.mark.parametrize("mc_mode", [0, 1])
def test_resumed_run_equals_the_uninterrupted_one(pkg, tmp_path, mc_mode):
    """40 steps in one simulation against 20 steps, a checkpoint written to a
    file, a fresh simulation restored from it and 20 more steps: coordinates,
    charges, velocities, site states, exchange grid, E and the exchange
    counters identical."""
    import torch
    device()
    b = synth.random_batch([300, 150, 220, 96], seed=41)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    lad = synth.e_ladder(b.n_rep)
    a = _sim(pkg, b, t, lad, mc_mode).run(40)
    a.sync()
    first = _sim(pkg, b, t, lad, mc_mode).run(20)
    first.sync()
    p = str(tmp_path / "md.npz")
    pkg.save_checkpoint(p, first.checkpoint())
    del first
    c = _sim(pkg, b, t, lad, mc_mode).restore(pkg.load_checkpoint(p)).run(20)
    c.sync()
    assert c.step == a.step == 40
    for k in ("xyzq", "vel", "state", "grid", "E", "pH", "ex_count"):
        assert torch.equal(getattr(a, k), getattr(c, k)), k
    assert int(c.st.attempt) == int(a.st.attempt) == 4
    # the run moved: exchanges and MC did something
    assert not torch.equal(a.xyzq, torch.as_tensor(b.xyzq(), device=a.xyzq.device))


@pytest.mark.gpu
def test_restore_rejects_a_checkpoint_of_another_layout(pkg):
    device()
    b = synth.random_batch([120, 80], seed=42)
    t = b.site_tables(oracle.site_reference_energies(b, oracle_params()))
    lad = synth.e_ladder(b.n_rep)
    ck = _sim(pkg, b, t, lad, 0).checkpoint()
    b2 = synth.random_batch([120, 81], seed=42)
    t2 = b2.site_tables(oracle.site_reference_energies(b2, oracle_params()))
    with pytest.raises(ValueError, match="xyzq"):
        _sim(pkg, b2, t2, lad, 0).restore(ck)


def test_exchange_ratios_of_the_counters():
    """The host view of the exchange counters: per direction, attempts and
    acceptances in [n_pH, n_E] by first slot, ratios NaN where nothing was
    attempted."""
    import paper_1803_09652_gb300 as pkg
    n_pH, n_E = 2, 3
    c = np.zeros((2, 2, n_pH * n_E), np.int64)
    c[0, 0, [0, 1, 3]] = [10, 4, 8]          # E pairs: (0,0)-(0,1), (0,1)-(0,2), (1,0)-(1,1)
    c[0, 1, [0, 1, 3]] = [5, 4, 0]
    c[1, 0, 2] = 6                            # pH pair: (0,2)-(1,2)
    c[1, 1, 2] = 3
    st = pkg.exchange_ratios(c, n_pH, n_E)
    assert st["E"]["attempts"].shape == (n_pH, n_E)
    assert st["E"]["ratio"][0, 0] == 0.5 and st["E"]["ratio"][0, 1] == 1.0 and st["E"]["ratio"][1, 0] == 0.0
    assert np.isnan(st["E"]["ratio"][0, 2]) and np.isnan(st["E"]["ratio"][1, 2])
    assert st["pH"]["ratio"][0, 2] == 0.5 and np.isnan(st["pH"]["ratio"]).sum() == 5
    assert st["pH"]["accepted"].sum() == 3 and st["E"]["attempts"].sum() == 22
