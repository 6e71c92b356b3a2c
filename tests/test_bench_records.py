"""The benchmark's DRAM-traffic records (profiles/traffic_paw96.md): a record counts only while
the hash of the kernel's source files matches, so a changed kernel reports no traffic."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _with_records(tmp_path, monkeypatch, lines, files):
    (tmp_path / "profiles").mkdir()
    for name, text in files.items():
        p = tmp_path / name
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_bytes(text)
    (tmp_path / "profiles" / "traffic_paw96.md").write_text("# records\n\n" + "\n".join(lines) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))


def test_committed_records_name_existing_sources():
    """Every record in the repository names files that exist and carries a hash and a byte
    count; the plane pass has one."""
    path = os.path.join(ROOT, "profiles", "traffic_paw96.md")
    tags = []
    for line in open(path):
        if line.startswith("traffic:"):
            f = dict(kv.split("=", 1) for kv in line.split()[1:])
            assert all(os.path.exists(os.path.join(ROOT, n)) for n in f["files"].split(","))
            assert len(f["sha1"]) == 40 and float(f["bytes_per_launch"]) > 0
            tags.append(f["tag"])
    assert "k_plane" in tags


def test_record_follows_the_hash_of_its_files(tmp_path, monkeypatch):
    a, b = b"kernel A source\n", b"shared header\n"
    sha = hashlib.sha1(a + b).hexdigest()
    files = {"src/a.cu": a, "src/b.cuh": b}
    line = "traffic: tag=k_x files=src/a.cu,src/b.cuh sha1=%s bytes_per_launch=1.5e+09" % sha
    _with_records(tmp_path, monkeypatch, [line], files)
    assert bench._traffic("k_x") == 1.5e9
    assert bench._traffic("k_other") is None
    # a changed source invalidates the record
    (tmp_path / "src" / "b.cuh").write_bytes(b"shared header, edited\n")
    assert bench._traffic("k_x") is None


def test_records_without_a_file_list_or_with_a_missing_file_are_ignored(tmp_path, monkeypatch):
    a = b"kernel source\n"
    sha = hashlib.sha1(a).hexdigest()
    lines = ["traffic: tag=k_old file=src/a.cu sha1=%s bytes_per_launch=2e9" % sha,
             "traffic: tag=k_gone files=src/missing.cu sha1=%s bytes_per_launch=2e9" % sha]
    _with_records(tmp_path, monkeypatch, lines, {"src/a.cu": a})
    assert bench._traffic("k_old") is None
    assert bench._traffic("k_gone") is None
