"""Host logic of bench.py that needs no GPU: the committed ncu evidence
(pipe fractions of the batched kernels, DRAM traffic of the pass kernel)
is used only while the kernel sources it was taken on are unchanged, and
is reported as a well-formed roofline object."""
import hashlib
import json
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _copy_tree(tmp_path, json_name, sources):
    """A repository stand-in holding one profile JSON and its sources."""
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", json_name), tmp_path / "profiles" / json_name)
    for src in sources:
        dst = tmp_path / src
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, src), dst)


@pytest.mark.parametrize("name", ["batched_kernel_pipes.json", "batched_k_kernel_pipes.json"])
def test_pipe_fractions_follow_the_sources(tmp_path, monkeypatch, name):
    with open(os.path.join(ROOT, "profiles", name)) as f:
        d = json.load(f)
    srcs = list(d["kernel_sources"])
    assert srcs and all(len(h) == 64 for h in d["kernel_sources"].values())
    _copy_tree(tmp_path, name, srcs)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the copied sources carry the recorded hashes or not; either way the
    # loader must agree with a direct check
    fresh = all(hashlib.sha256((tmp_path / s).read_bytes()).hexdigest() == h
                for s, h in d["kernel_sources"].items())
    r = bench.batched_roofline(name)
    if fresh:
        assert r is not None
        assert r["bound"] == "alu" and r["pipe"] == "FP64" and r["peak"] == 1.0
        assert 0.0 < r["frac"] <= 1.0 and r["frac"] == r["achieved"]
        assert 0.0 < r["sm_active_frac_of_elapsed"] <= 1.0
        assert name in r["source"]
    else:
        assert r is None
    # any change to a source makes the evidence stale
    with open(tmp_path / srcs[0], "ab") as f:
        f.write(b"\n// edited\n")
    assert bench.batched_pipes(name) is None
    assert bench.batched_roofline(name) is None


def test_missing_pipe_file_gives_no_roofline(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.batched_roofline("batched_kernel_pipes.json") is None


def test_pass_traffic_scales_with_the_entries_and_follows_the_source(tmp_path, monkeypatch):
    src = os.path.join("paper_2306_08152_gb300", "csrc", "qf_pass.cu")
    _copy_tree(tmp_path, "pass_kernel_traffic.json", [src])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    with open(tmp_path / "profiles" / "pass_kernel_traffic.json") as f:
        d = json.load(f)
    fresh = d.get("kernel_sha256") == hashlib.sha256((tmp_path / src).read_bytes()).hexdigest()
    for key, entry in d.get("per_launch", {}).items():
        t1 = bench.kernel_traffic(key, 1, 12)
        t2 = bench.kernel_traffic(key, 2, 12)
        if fresh:
            assert t1 is not None and t2 == pytest.approx(2 * t1)
            assert t1 == pytest.approx(entry["dram_bytes"] * 4**12 / entry["entries"])
        else:
            assert t1 is None
    with open(tmp_path / src, "ab") as f:
        f.write(b"\n// edited\n")
    for key in d.get("per_launch", {}):
        assert bench.kernel_traffic(key, 4, 12) is None
