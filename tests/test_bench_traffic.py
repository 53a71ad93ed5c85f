"""Host-side logic of the bench's roofline line (CPU): the DRAM traffic of the dominant kernel
comes from the committed ncu summary only while the captured kernel is the one timed and its
source is unchanged since the capture."""
import hashlib
import os

import bench

TABLE = """| class | kernel | entries | read MB | write MB | traffic bytes | source | sha256[:16] |
|---|---|---:|---:|---:|---:|---|---|
| xprox | `tc::k_tc_xprox_pers` | 5000000 | 83.50 | 10.59 | 94089728 | src/k.cu | {h} |
"""


def _tree(tmp_path, source=b"kernel source\n"):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "src").mkdir()
    (tmp_path / "src" / "k.cu").write_bytes(source)
    h = hashlib.sha256(source).hexdigest()[:16]
    (tmp_path / "profiles" / "dram_traffic_500x10000.md").write_text(TABLE.format(h=h))


def test_traffic_scales_the_captured_bytes_per_entry(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.profiled_traffic("xprox", 2_500_000, "k_tc_xprox_pers")
    assert got == 94089728 / 5000000 * 2_500_000
    assert bench.profiled_traffic("xprox", 2_500_000) == got          # no name given: the class's row


def test_traffic_is_null_for_another_kernel_of_the_class(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("xprox", 2_500_000, "k_tc_xprox") is None
    assert bench.profiled_traffic("roots", 2_500_000) is None          # no row for the class


def test_traffic_is_null_once_the_source_changed(tmp_path, monkeypatch):
    _tree(tmp_path)
    (tmp_path / "src" / "k.cu").write_bytes(b"kernel source, changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("xprox", 2_500_000, "k_tc_xprox_pers") is None
