"""Host arithmetic of the benchmark: the per-segment byte model, the two-level roofline, the
weak-scaling aggregate and the staleness check of profiled DRAM traffic (no GPU)."""
import os
import shutil

import pytest

import bench


def test_forward_bytes_per_segment_and_ray():
    # SH degree 3 (K = 16) in FP16: payload 98 B, plus a 4-byte child word, per occupied segment;
    # 2 B density + 4 B child word per empty one; 12 B of colour per ray
    st = {"segments": 10, "occupied": 3}
    assert bench.alg_bytes_of(st, 2, 2, 16) == 3 * (98 + 4) + 7 * (2 + 4) + 2 * 12
    # FP32, SH degree 1 (K = 4): payload 52 B
    assert bench.alg_bytes_of(st, 1, 4, 4) == 3 * (52 + 4) + 7 * (4 + 4) + 12


def test_backward_bytes_add_the_gradient_update():
    st = {"segments": 10, "occupied": 3}
    assert bench.grad_bytes_per_occupied(16) == 196          # dL/dsigma + 48 SH gradients, FP32
    fwd = bench.alg_bytes_of(st, 2, 2, 16)
    # the backward re-reads what the forward reads, updates 196 B per occupied segment and reads
    # dL/dC and C (24 B) instead of writing C (12 B) per ray
    assert bench.alg_bytes_bwd(st, 2, 2, 16) == fwd - 2 * 12 + 3 * 196 + 2 * 24


def test_two_level_takes_the_larger_term():
    # 1 GB compulsory at 1000 GB/s = 1 ms; 10 GB of samples at 20,000 GB/s = 0.5 ms: HBM-bound
    r = bench.two_level(1e9, 1e10, 4e-3, 1000.0, 20000.0)
    assert r["bound"] == "hbm"
    assert r["t_roof_ms"] == pytest.approx(1.0)
    assert r["frac"] == pytest.approx(0.25)
    # more samples: the L2 term (2 ms) decides
    r = bench.two_level(1e9, 4e10, 4e-3, 1000.0, 20000.0)
    assert r["bound"] == "l2"
    assert r["t_l2_ms"] == pytest.approx(2.0)
    assert r["frac"] == pytest.approx(0.5)


def test_weak_scaling_value_counts_every_rank():
    # 64 M rays per rank and step, 10 steps, 4 ranks, 100 ms for the slowest rank
    assert bench.weak_scaling_value(64_000_000, 10, 4, 100.0) == pytest.approx(25600.0)


def test_csrc_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2307_15333_gb300", "csrc")
    root = tmp_path / "repo"
    csrc = root / "paper_2307_15333_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.MARCH_SOURCES:
        shutil.copy(os.path.join(src, f), csrc / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.csrc_hash()
    p = csrc / "march.cuh"
    p.write_text("// a comment\n" + p.read_text().replace("\n", "\n\n") + "\n/* another */\n")
    assert bench.csrc_hash() == h0
    p.write_text(p.read_text() + "\nstatic int changed_code = 1;\n")
    assert bench.csrc_hash() != h0


def test_profiled_traffic_only_for_the_profiled_sources(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2307_15333_gb300", "csrc")
    root = tmp_path / "repo"
    csrc = root / "paper_2307_15333_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.MARCH_SOURCES:
        shutil.copy(os.path.join(src, f), csrc / f)
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    prof = root / "profiles" / "k.md"
    prof.write_text(f"dram_bytes_per_launch: 12345\ncsrc_sha: {bench.csrc_hash()}\n")
    assert bench.profiled_traffic("k") == 12345.0
    prof.write_text("dram_bytes_per_launch: 12345\ncsrc_sha: 0123456789abcdef\n")
    assert bench.profiled_traffic("k") is None
    assert bench.profiled_traffic("missing") is None
