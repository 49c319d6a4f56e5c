"""The DRAM traffic that bench.py reports beside its roofline comes from a
committed ncu summary, stamped with a hash of the step kernels' sources: it is
used only while those sources are unchanged, and reported as unknown (None)
otherwise, so a number taken on older kernels is never shown as current."""
import json
import os

import bench


def _write(root, stamp, kernels):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", "step_kernel_traffic.json"), "w") as f:
        json.dump({"src_hash": stamp, "kernels": kernels}, f)


def test_traffic_is_used_only_on_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    root = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc123")
    entry = {"dram_bytes_per_launch": 585e6, "dram_read": 328e6, "dram_write": 257e6}
    _write(root, "abc123", {"channel/f32": entry})
    assert bench.ncu_traffic("channel", "f32") == 585e6
    assert bench.ncu_traffic("channel", "f16s") is None  # no capture of that kernel
    _write(root, "0ld5tamp", {"channel/f32": entry})  # the sources changed since
    assert bench.ncu_traffic("channel", "f32") is None


def test_missing_or_unreadable_record_gives_no_traffic(tmp_path, monkeypatch):
    root = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.ncu_traffic("channel", "f32") is None
    os.makedirs(os.path.join(root, "profiles"))
    with open(os.path.join(root, "profiles", "step_kernel_traffic.json"), "w") as f:
        f.write("{not json")
    assert bench.ncu_traffic("channel", "f32") is None


def test_source_hash_covers_the_step_kernel_sources(tmp_path, monkeypatch):
    """The stamp changes with any byte of a step-kernel source and ignores
    sources outside the step kernels (here the reverse-step unit)."""
    csrc = tmp_path / "paper_1112_0850_gb300" / "csrc"
    inc = tmp_path / "include"
    csrc.mkdir(parents=True)
    inc.mkdir()
    for n in ("lbm_device.cuh", "lbm_launch.h", "lbm_kernels.cuh", "lbm_capi.cu", "lbm_setup.cu",
              "lbm_ops_f32.cu", "lbm_adjoint.cu"):
        (csrc / n).write_text("// " + n + "\n")
    (inc / "lbm_capi.h").write_text("/* header */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (csrc / "lbm_adjoint.cu").write_text("// changed\n")
    assert bench.kernel_source_hash() == h0
    (csrc / "lbm_kernels.cuh").write_text("// lbm_kernels.cuh \n")
    h1 = bench.kernel_source_hash()
    assert h1 != h0
    (csrc / "lbm_ops_f32.cu").write_text("// changed\n")
    assert bench.kernel_source_hash() != h1
