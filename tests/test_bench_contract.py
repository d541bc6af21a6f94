"""Host arithmetic of the bench line (no GPU): the algorithmic bytes per apply, the
ALU roofline fields, and the traffic record that is used only while the kernel
source still has the hash of the ncu capture."""
import hashlib
import json
import os

import pytest

import bench


def test_algorithmic_bytes_of_the_32cubed_k3_apply():
    # x and y (8 + 8 bytes per DoF) and nu at the n^3 cell and 6 n^2 face points per cell
    n_dofs, cells, n = 32 ** 3 * 3 * 4 ** 3, 32 ** 3, 4
    assert bench.algorithmic_bytes(n_dofs, cells, n) == 16 * n_dofs + 8 * cells * (64 + 96)
    assert bench.algorithmic_bytes(n_dofs, cells, n) == 142606336


def test_roofline_fields(monkeypatch):
    monkeypatch.setattr(bench, "traffic_record", lambda key: 123)
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6000.0})
    n, ms = 6291456, 0.8
    alg = bench.algorithmic_bytes(n, 32 ** 3, 4)
    pk = {"f64": 1.0, "f32": 72.0, "f64ff": 6.0}
    r = bench.roofline(ms, n, alg, "f64ff", pk, "k")
    achieved = bench.FLOP_PER_DOF * n / (ms * 1e-3) / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] == 123
    assert r["achieved"] == pytest.approx(achieved) and r["peak"] == 6.0
    assert r["frac"] == pytest.approx(achieved / 6.0)
    assert r["hbm_frac"] == pytest.approx(alg / (ms * 1e-3) / 1e9 / 6000.0)
    assert r["algorithmic_bytes_per_launch"] == alg
    assert r["algorithmic_flops_per_launch"] == pytest.approx(bench.FLOP_PER_DOF * n)


def test_traffic_record_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "paper_2506_14424_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cuh").write_bytes(b"kernel source v1")
    (tmp_path / "profiles").mkdir()
    sha = hashlib.sha256(b"kernel source v1").hexdigest()[:16]
    rec = {"k": {"source": "k.cuh", "source_sha": sha, "dram_bytes_per_launch": 4242}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("k") == 4242
    assert bench.traffic_record("other") is None
    (src / "k.cuh").write_bytes(b"kernel source v2")  # the kernel changed since the capture
    assert bench.traffic_record("k") is None


def test_committed_traffic_records_name_existing_sources():
    p = os.path.join(bench.ROOT, "profiles", "traffic.json")
    recs = json.load(open(p))
    for key, rec in recs.items():
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2506_14424_gb300", "csrc", rec["source"])), key
        assert rec["dram_bytes_per_launch"] > 0 and len(rec["source_sha"]) == 16
