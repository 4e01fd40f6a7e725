"""Host-side logic of bench.py that needs no GPU: when a bench line may take
the DRAM traffic of its dominant kernel from a committed ncu summary.

The summary records the SHA-1 of the kernel sources it was captured on and
the number of time steps one captured launch made; the traffic is reported
per time step, and only while both still hold."""
import os

import pytest

import bench

CSRC = ("teuk_dev.cuh", "teuk_split.cuh")


def _tree(tmp_path, kernel_text=("// a\n", "// b\n")):
    d = tmp_path / "paper_0909_4039_gb300" / "csrc"
    d.mkdir(parents=True)
    for name, text in zip(CSRC, kernel_text):
        (d / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    return tmp_path


def _summary(root, name, sha, steps=3, traffic=300, rows="28"):
    lines = ["# a summary", ""]
    if rows is not None:
        lines.append(f"tile_rows: {rows}")
    lines += [f"steps_per_launch: {steps}", f"traffic_bytes_per_launch: {traffic}", f"source_sha1: {sha}", ""]
    (root / "profiles" / name).write_text("\n".join(lines))


@pytest.fixture
def root(tmp_path, monkeypatch):
    r = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(r))
    return r


def test_traffic_per_step_while_sources_and_steps_match(root):
    sha = bench.kernel_source_sha1()
    _summary(root, "k_split_step3_16384x128_fp32.md", sha, steps=3, traffic=300)
    assert bench._profiled_traffic("k_split_step3", "16384x128", 3) == (100, [28])
    _summary(root, "k_split_batch_batch64_fp32.md", sha, steps=2, traffic=1001, rows="44, 76, 156")
    assert bench._profiled_traffic("k_split_batch", "batch64", 2) == (500, [44, 76, 156])


def test_no_traffic_for_other_steps_per_launch(root):
    _summary(root, "k_split_step3_16384x128_fp32.md", bench.kernel_source_sha1(), steps=3)
    assert bench._profiled_traffic("k_split_step3", "16384x128", 2) == (None, None)


def test_no_traffic_once_a_kernel_source_changes(root):
    _summary(root, "k_split_step3_16384x128_fp32.md", bench.kernel_source_sha1(), steps=3)
    f = root / "paper_0909_4039_gb300" / "csrc" / "teuk_split.cuh"
    f.write_text(f.read_text() + "// changed\n")
    assert bench._profiled_traffic("k_split_step3", "16384x128", 3) == (None, None)


def test_no_traffic_without_a_summary_or_its_fields(root):
    assert bench._profiled_traffic("k_split_step3", "16384x128", 3) == (None, None)
    (root / "profiles" / "k_split_step3_16384x128_fp32.md").write_text("# no fields\n")
    assert bench._profiled_traffic("k_split_step3", "16384x128", 3) == (None, None)


def test_sha_covers_both_kernel_sources_in_order(root):
    import hashlib
    h = hashlib.sha1()
    for name in CSRC:
        h.update(open(os.path.join(root, "paper_0909_4039_gb300", "csrc", name), "rb").read())
    assert bench.kernel_source_sha1() == h.hexdigest()
