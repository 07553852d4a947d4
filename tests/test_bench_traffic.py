"""bench.py reports roofline.traffic from an ncu summary only for the
history-sum source revision the counters were taken on: the revision hash
ignores comment edits, changes with any code edit, and a summary for
another revision is not used."""

import os
import shutil

import bench


def _copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2111_05205_gb300", "csrc")
    dst = tmp_path / "paper_2111_05205_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("march.cu", "tdbem_internal.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    return dst


def test_revision_ignores_comments_and_follows_code(tmp_path, monkeypatch):
    dst = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r0 = bench._kernel_rev()
    assert len(r0) == 12
    m = (dst / "march.cu").read_text()
    (dst / "march.cu").write_text(m.replace("namespace tdbem {", "namespace tdbem {  // a remark", 1))
    assert bench._kernel_rev() == r0
    (dst / "march.cu").write_text("static int edited_line = 0;\n" + m)
    assert bench._kernel_rev() != r0


def test_traffic_only_for_its_revision(tmp_path, monkeypatch):
    _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    st = {"near_bytes_per_step": 1000}
    assert bench._traffic(st) is None  # no summary
    summary = tmp_path / "profiles" / "near_sum_traffic.txt"
    summary.write_text("# comment\nkernel_rev: %s\nbytes_per_algorithmic_byte: 1.25\n" % bench._kernel_rev())
    assert bench._traffic(st) == 1250.0
    summary.write_text("kernel_rev: 000000000000\nbytes_per_algorithmic_byte: 1.25\n")
    assert bench._traffic(st) is None
