"""Host logic of the benchmark that decides which committed ncu figures a bench line may use:
a kernel's source hash follows the file that defines it and the kernel sources it includes
(and nothing else), and a DRAM-traffic figure is used only while that hash matches and for the
tile shape it was captured with; the single-view forms keep the fastest of their tile shapes."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2509_17513_b300", "csrc")


def test_include_closure_of_the_multi_level_blend():
    files = {os.path.basename(f) for f in bench._include_closure(os.path.join(CSRC, "gc_levels.cu"))}
    assert "gc_levels.cu" in files and "gc_tile.cuh" in files and "gc_internal.cuh" in files
    # files the blend does not include, and the public header's declarations, stay out
    assert "gc_state.cuh" not in files and "gc_kde.cu" not in files and "gc4d.h" not in files


def test_include_closure_follows_nested_includes(tmp_path):
    (tmp_path / "a.cu").write_text('#include "b.cuh"\n')
    (tmp_path / "b.cuh").write_text('  #  include "c.cuh"\n#include <cuda_runtime.h>\n')
    (tmp_path / "c.cuh").write_text('#include "b.cuh"\n')  # a cycle ends
    (tmp_path / "d.cuh").write_text("")
    got = [os.path.basename(f) for f in bench._include_closure(str(tmp_path / "a.cu"))]
    assert got == ["a.cu", "b.cuh", "c.cuh"]


def test_kernel_hash_ignores_unrelated_sources_and_follows_its_own(monkeypatch, tmp_path):
    src = tmp_path / "paper_2509_17513_b300" / "csrc"
    src.mkdir(parents=True)
    (src / "gc_levels.cu").write_text('#include "gc_tile.cuh"\nkernel\n')
    (src / "gc_tile.cuh").write_text("tile v1\n")
    (src / "gc_kde.cu").write_text("kde v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash("k_blend_levels_fwd")
    (src / "gc_kde.cu").write_text("kde v2\n")
    assert bench.kernel_source_hash("k_blend_levels_fwd") == h0
    (src / "gc_tile.cuh").write_text("tile v2\n")
    assert bench.kernel_source_hash("k_blend_levels_fwd") != h0
    # a kernel not listed depends on every source
    a = bench.kernel_source_hash("k_unlisted")
    (src / "gc_kde.cu").write_text("kde v3\n")
    assert bench.kernel_source_hash("k_unlisted") != a


def test_traffic_needs_matching_sources_and_tile(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k=None: "abc")
    entry = {"dram_bytes_per_unit": 1000, "unit": "frame", "source_hash": "abc", "tile": "8x32"}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"kernels": {"k_blend_levels_fwd": entry}}))
    assert bench.load_traffic("k_blend_levels_fwd", 3, "8x32") == 3000
    assert bench.load_traffic("k_blend_levels_fwd", 3, "16x16") is None
    assert bench.load_traffic("k_blend_levels_bwd", 3, "8x32") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k=None: "changed")
    assert bench.load_traffic("k_blend_levels_fwd", 3, "8x32") is None


def test_committed_traffic_entries_are_well_formed():
    """Every committed figure names its unit, a 16-hex-digit source hash and (for the blends)
    the tile shape; whether it is current is decided at bench time (null when stale)."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for k, e in d["kernels"].items():
        assert isinstance(e["dram_bytes_per_unit"], int) and e["dram_bytes_per_unit"] > 0, k
        assert len(e["source_hash"]) == 16 and int(e["source_hash"], 16) >= 0, k
        assert e["unit"], k
    for k in ("k_blend_levels_fwd", "k_blend_levels_bwd"):
        assert d["kernels"][k]["tile"] == "%dx%d" % bench.HEADLINE_TILE


def test_pick_tile_keeps_the_fastest_shape(monkeypatch):
    """The single-view forms' tile sweep: each shape gets its own step (built after the shape is
    set), and the fastest shape is the one left set, with grow-as-needed key capacity."""
    import time

    import torch
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)

    class FakeRenderer:
        def __init__(self):
            self.opts = {}

        def set_options(self, **kw):
            self.opts.update(kw)

    r = FakeRenderer()
    cost = {(16, 16): 0.004, (8, 32): 0.001, (32, 8): 0.003}
    built = []

    def make_step():
        tile = r.opts["tile"]
        built.append(tile)
        return lambda: time.sleep(cost[tile])

    best, ms = bench.pick_tile(r, make_step, reps=2)
    assert best == (8, 32)
    assert built == [(16, 16), (8, 32), (32, 8)]
    assert r.opts == {"key_capacity": 0, "tile": (8, 32)}
    assert set(ms) == {"16x16", "8x32", "32x8"} and ms["8x32"] < ms["32x8"] < ms["16x16"]
