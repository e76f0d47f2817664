"""Host logic of bench.py that needs no GPU: the per-kernel source hash that
ties ncu traffic figures to the kernel they were taken on, and the guard that
keeps an optional leg from breaking the headline line."""
import json
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources and headers that the hash reads."""
    for sub in (os.path.join("paper_1712_03554_gb300", "csrc"), "include", "profiles"):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_hash_follows_included_headers(tree):
    h0 = {c: bench.kernel_sources_hash(c) for c in ("gprog", "segment", "cofactor")}
    warp = tree / "paper_1712_03554_gb300" / "csrc" / "sf_warp.cuh"
    warp.write_text(warp.read_text() + "\n// touched\n")
    h1 = {c: bench.kernel_sources_hash(c) for c in h0}
    # sf_gprog.cu and sf_campaign.cu include sf_warp.cuh; sf_frame.cu does not
    assert h1["gprog"] != h0["gprog"] and h1["segment"] != h0["segment"]
    assert h1["cofactor"] == h0["cofactor"]


def test_hash_ignores_unrelated_sources(tree):
    h0 = bench.kernel_sources_hash("gprog")
    (tree / "paper_1712_03554_gb300" / "csrc" / "sf_new_kernel.cu").write_text("// another file\n")
    api = tree / "paper_1712_03554_gb300" / "csrc" / "sf_api.cu"
    api.write_text(api.read_text() + "\n// host code only\n")
    assert bench.kernel_sources_hash("gprog") == h0


def test_traffic_is_null_once_the_kernel_changed(tree):
    t = json.loads((tree / "profiles" / "traffic.json").read_text())
    t["sources"] = {cls: bench.kernel_sources_hash(cls) for cls in t["bytes_per_launch"]}
    (tree / "profiles" / "traffic.json").write_text(json.dumps(t))
    for cls, v in t["bytes_per_launch"].items():
        assert bench.ncu_traffic(cls) == float(v), cls
    frame = tree / "paper_1712_03554_gb300" / "csrc" / "sf_frame.cu"
    frame.write_text(frame.read_text() + "\n// changed\n")
    assert bench.ncu_traffic("cofactor") is None
    assert bench.ncu_traffic("gprog") == float(t["bytes_per_launch"]["gprog"])


def test_multiframe_leg_reports_errors_instead_of_raising():
    class NoDevice:
        class Frame:
            def __init__(self, *a, **k):
                raise RuntimeError("no device")

    out = bench.multiframe_leg(NoDevice, nb=2, reps=1)
    assert set(out) == {"error"} and "no device" in out["error"]
