"""Host logic of bench.py that shapes its JSON line: the pair count of a
workload with a pair cutoff (k-d tree count against brute force), the
launches counted per MD segment, the workload table, and the DRAM traffic
table (scaled by atoms, void once a pair-kernel source changes)."""
import numpy as np
import pytest

import bench
import synth


def test_pairs_within_matches_brute_force():
    b = synth.random_batch([300, 0, 77, 1], seed=61, sites=False)
    for cut in (3.0, 8.0, 1e4):
        brute = 0
        for rep in b.replicas:
            x = rep.xyz.astype(np.float64)
            d = np.linalg.norm(x[:, None] - x[None], axis=2)
            brute += int(np.sum(d[np.triu_indices(len(x), 1)] < cut))
        assert synth.pairs_within(b, cut) == brute
    assert synth.pairs_within(b, 1e4) == b.pairs_per_eval()


def test_pairs_per_md_step_counts_within_the_cutoff_only_with_a_cutoff():
    b = synth.random_batch([200, 90], seed=62, sites=False)
    assert bench.pairs_per_md_step(b, "eremd_8x2048") == b.pairs_per_eval()
    cut = bench.CUTOFFS["cutoff_1x100000"]["cut"]
    assert bench.pairs_per_md_step(b, "cutoff_1x100000") == synth.pairs_within(b, cut)


@pytest.mark.parametrize("cutoff,per_step", [(False, 6), (True, 8)])
def test_launches_per_segment(cutoff, per_step):
    n = 100
    mc = 4 * (n // bench.MC_EVERY)
    ex = 2 * (n // bench.EX_EVERY)
    assert bench.launches_per_segment(n, False, cutoff) == 1 + per_step * n + 1 + mc + ex + 1
    assert bench.launches_per_segment(n, True) == 1 + n // bench.MC_EVERY + mc + ex + 1


def test_every_workload_is_known():
    assert set(bench.CUTOFFS) <= set(bench.WORKLOADS)
    with pytest.raises(ValueError):
        bench.workload("no_such_workload")


def test_default_workload_is_the_largest_single_gpu_configuration():
    assert bench.DEFAULT_WORKLOAD == "grid_48x25000"
    b = synth.config_grid()
    c = bench.bench_config(bench.DEFAULT_WORKLOAD, b, b.pairs_per_eval())
    assert c["replicas"] == 48 and c["atoms_total"] == 48 * 25000
    assert c["pairs_per_md_step"] == 48 * 25000 * 24999 // 2
    assert c["md_steps_per_step"] == 100 and c["mc_every"] == 10 and c["exchange_every"] == 100


REPO_ROOT = bench.ROOT


def _traffic_tree(tmp_path, src_hash):
    """A copy of the pair-kernel sources and a traffic table under tmp_path."""
    import os
    import shutil
    csrc = tmp_path / "paper_1803_09652_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.PAIR_SOURCES:
        shutil.copy(os.path.join(REPO_ROOT, "paper_1803_09652_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        "# DRAM bytes per launch\n"
        f"sources {src_hash}\n"
        "atoms 1000\n"
        "k_pairs<born> 4000\n"
        "k_pairs<energy> 7000\n")


def test_traffic_is_scaled_by_atoms_and_only_for_the_captured_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _traffic_tree(tmp_path, "0" * 16)
    h = bench.pair_source_hash()
    assert bench.read_traffic("k_pairs<energy>", 1000) is None        # sources changed since the capture
    _traffic_tree(tmp_path / "x", h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "x"))
    assert bench.pair_source_hash() == h
    assert bench.read_traffic("k_pairs<energy>", 1000) == 7000.0
    assert bench.read_traffic("k_pairs<energy>", 3000) == 21000.0     # scaled by atoms
    assert bench.read_traffic("k_pairs<chain>", 1000) is None         # not in the table
    # any edit of a pair-kernel source invalidates the table
    p = tmp_path / "x" / "paper_1803_09652_gb300" / "csrc" / bench.PAIR_SOURCES[0]
    p.write_text(p.read_text() + "\n")
    assert bench.read_traffic("k_pairs<energy>", 1000) is None
