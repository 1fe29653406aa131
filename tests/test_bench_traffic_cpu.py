"""The S'v roofline's `traffic` in the bench line comes from a committed ncu summary of the product in use
(two passes or the grid product) and is reported only while the SR source is the one that was captured
(its SHA-1 recorded beside the figure); otherwise null."""
import importlib.util
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("mode,reads", [(0, 2), (2, 1)])
def test_committed_capture_matches_the_sr_source(mode, reads):
    per_row, source = load_bench().sr_traffic_per_row(mode=mode)
    assert per_row is not None, source
    # one S'v product reads each BF16-pair row of O twice (two passes) or once (grid product):
    # reads x 198,276 x 4 bytes, plus partial sums
    assert reads * 198276 * 4 <= per_row <= 1.01 * reads * 198276 * 4
    assert "ncu" in source


def test_changed_source_gives_null_traffic(tmp_path):
    src = tmp_path / "k_sr.cu"
    shutil.copy(os.path.join(ROOT, "paper_2502_20723_gb300", "csrc", "k_sr.cu"), src)
    with open(src, "a") as f:
        f.write("\n// changed\n")
    per_row, source = load_bench().sr_traffic_per_row(src=str(src))
    assert per_row is None and "changed" in source
