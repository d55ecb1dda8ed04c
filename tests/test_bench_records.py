"""Host logic of bench.py's DRAM-traffic records (no GPU).

A record under profiles/ gives a kernel's DRAM bytes per launch from one ncu
capture, with the SHA-256 of the kernel's source files at capture time; bench.py
reports the bytes only while those files are unchanged, and null once any of
them differs, so a number is never carried over to a kernel that changed."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path, sources, recorded_bytes, hash_of=None):
    csrc = tmp_path / "paper_1901_10559_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in sources.items():
        (csrc / name).write_text(text)
    h = hashlib.sha256()
    for name, text in (hash_of or sources).items():
        h.update(text.encode())
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_k_w.txt").write_text(
        "# a comment line: with a colon\n"
        f"dram_bytes_per_launch: {recorded_bytes}\n"
        f"source_sha256: {h.hexdigest()}\n")


def test_record_read_while_sources_match(tmp_path, monkeypatch):
    _tree(tmp_path, {"a.cu": "kernel A\n", "b.cuh": "helper B\n"}, 12345)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k", "w", ["a.cu", "b.cuh"]) == 12345.0


def test_record_null_after_a_source_changes(tmp_path, monkeypatch):
    _tree(tmp_path, {"a.cu": "kernel A, edited\n", "b.cuh": "helper B\n"}, 12345,
          hash_of={"a.cu": "kernel A\n", "b.cuh": "helper B\n"})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k", "w", ["a.cu", "b.cuh"]) is None


def test_record_hash_follows_the_file_order(tmp_path, monkeypatch):
    _tree(tmp_path, {"a.cu": "kernel A\n", "b.cuh": "helper B\n"}, 7)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k", "w", ["b.cuh", "a.cu"]) is None


def test_missing_record_is_null(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("nothing", "w", ["a.cu"]) is None
