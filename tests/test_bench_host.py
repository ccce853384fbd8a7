"""Host logic of ``bench.py`` on CPU: the compulsory-byte counts behind the
roofline, the guard that drops the committed ncu traffic figure once the
kernel it was taken on changes, and the row-parallel oracle timing."""
import json
import os
import shutil

import pytest

import bench


def test_algorithmic_bytes_of_the_27_point_workload():
    # the 27-point product on 100^3: 224 MB symbolic + 2,094 MB numeric with
    # 4-byte C row pointers (scope table of the hot path); int64 row pointers
    # add 4 (m + 1) bytes to each phase
    m = 1_000_000
    sym, num = bench.algorithmic_bytes(m, m, 26_463_592, 26_463_592, 120_553_784)
    assert sym == pytest.approx(224e6 + 4 * (m + 1), rel=0.01)
    assert num == pytest.approx(2094e6 + 4 * (m + 1), rel=0.01)


def _copy_record(tmp_path):
    root = os.path.dirname(os.path.abspath(bench.__file__))
    rec = json.load(open(os.path.join(root, "profiles", "ncu_traffic.json")))
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(root, "profiles", "ncu_traffic.json"), tmp_path / "profiles")
    src = tmp_path / "paper_2103_11991_gb300" / "csrc"
    src.mkdir(parents=True)
    import hashlib
    h = hashlib.sha256()
    for name in rec["sources"]:
        shutil.copy(os.path.join(root, "paper_2103_11991_gb300", "csrc", name), src / name)
        h.update((src / name).read_bytes())
    # the copy's record matches the copied sources, whether or not the
    # committed record is current
    rec["source_sha256"] = h.hexdigest()
    with open(tmp_path / "profiles" / "ncu_traffic.json", "w") as f:
        json.dump(rec, f)
    return rec, src


def test_ncu_traffic_is_dropped_when_the_kernel_changes(tmp_path, monkeypatch):
    rec, src = _copy_record(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    traffic, kernel = bench._ncu_traffic()
    assert kernel == rec["kernel"]
    assert traffic == float(rec["dram_bytes_per_step"])
    with open(src / rec["sources"][-1], "a") as f:
        f.write("\n// changed\n")
    traffic, kernel = bench._ncu_traffic()
    assert traffic is None and kernel == rec["kernel"]


def test_parallel_oracle_timing_counts_the_work_it_ran():
    import oracle
    from paper_2103_11991_gb300 import inputs as I
    A = I.stencil_3d(24, 24, 24, 27, 26.0, -1.0)  # 13,824 rows = 256 blocks of 54
    flops = oracle.row_flops(A, A)
    rate, rows, secs = bench.cpu_oracle_parallel_rate(A, A, flops, 0.3, 4)
    block = A.m // 256
    assert secs >= 0.3 and rows > 0 and rows % (4 * block) == 0
    # blocks are taken in order, wrapping around: the multiply-adds of the
    # first rows / block of them
    per_block = flops.reshape(256, block).sum(axis=1)
    nb = rows // block
    done = per_block.sum() * (nb // 256) + per_block[:nb % 256].sum()
    assert rate * 1e9 * secs / 2.0 == pytest.approx(float(done), rel=1e-9)
