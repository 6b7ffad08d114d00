"""Host-side logic of bench.py that needs no GPU: the per-launch DRAM traffic lookup
(keyed by the hash of the kernel source, so counters taken on other code are never
reported) and the whole-job throughput arithmetic."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path, source_text, lines):
    csrc = tmp_path / "paper_1912_04582_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "tucker_kernels.cu").write_text(source_text)
    (csrc / "full_kernels.cu").write_text("full " + source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text("\n".join(lines) + "\n")
    return tmp_path


def _h(text):
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def test_traffic_is_read_for_the_current_source_only(tmp_path, monkeypatch):
    src = "// kernels, version A\n"
    root = _tree(tmp_path, src, [
        "# comment line tucker_eig 0000000000000000 1",
        f"tucker_eig {_h(src)} 54138965",
        "tucker_asm 0123456789abcdef 601009152",  # taken on other code
        f"full {_h('full ' + src)} 4362103000",
    ])
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic("tucker_eig") == 54138965.0
    assert bench._traffic("tucker_asm") is None
    assert bench._traffic("tucker_gram_mode1") is None
    assert bench._traffic("full") == 4362103000.0
    # any change to the kernel source invalidates its counters
    (root / "paper_1912_04582_gb300" / "csrc" / "tucker_kernels.cu").write_text(src + " ")
    assert bench._traffic("tucker_eig") is None


def test_traffic_without_the_file_is_null(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("tucker_eig") is None


@pytest.mark.parametrize("world,steps,ms", [(1, 20, 61.5), (2, 20, 70.0), (8, 5, 12.0)])
def test_job_value_counts_every_rank(world, steps, ms):
    upd = 4096 * 32 ** 3
    v = bench.job_value(world, upd, steps, ms)
    assert v == pytest.approx(world * upd * steps / (ms / 1e3), rel=1e-12)
