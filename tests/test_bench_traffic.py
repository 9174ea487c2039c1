"""bench.py reports an ncu traffic figure only for the kernel sources it was taken
on: a change to the code of the tile kernel, its header or its planner makes
recorded_traffic() return None, while an edit to comments or whitespace does not."""
import json
import os
import shutil

import bench

SRC = os.path.join(bench.ROOT, "paper_1908_07187_gb300", "csrc")


def _fake_root(tmp_path):
    csrc = tmp_path / "paper_1908_07187_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES["tile"]:
        shutil.copy(os.path.join(SRC, f), csrc / f)
    (tmp_path / "profiles").mkdir()
    return tmp_path, csrc


def _record(root, sha, nbytes=1.5e10):
    rec = {"tile_n30": {"src_sha": sha, "dram_bytes_per_launch": nbytes}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))


def test_code_only_drops_comments_and_whitespace():
    a = 'int x = 1; // one\n/* block */ float y;  \n  const char *s = "a // not a comment";\n'
    b = 'int x = 1;\nfloat y; const char *s = "a // not a comment";'
    assert bench.code_only(a) == bench.code_only(b)
    assert "not a comment" in bench.code_only(a)


def test_traffic_is_kept_for_the_same_code_and_dropped_after_a_code_change(tmp_path, monkeypatch):
    root, csrc = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    _record(root, bench.kernel_source_sha("tile"))
    assert bench.recorded_traffic("tile", 30) == 1.5e10
    assert bench.recorded_traffic("tile", 26) is None        # no record for that size

    plan = csrc / "qk_plan.cu"
    plan.write_text(plan.read_text() + "\n// a comment only\n")
    assert bench.recorded_traffic("tile", 30) == 1.5e10      # comments do not count

    kern = csrc / "kernels_tile.cu"
    kern.write_text(kern.read_text() + "\nstatic int extra_code = 1;\n")
    assert bench.recorded_traffic("tile", 30) is None        # a code change does

