"""Host logic of bench.py: the DRAM traffic it reports comes from an ncu
summary in profiles/ only while the kernel sources still hash to the value
recorded with it; any change to a source makes it null."""
import hashlib
import os

import bench


def write_tree(root, sources, text):
    os.makedirs(os.path.join(root, "profiles"))
    os.makedirs(os.path.join(root, "paper_2403_02816_gb300", "csrc"))
    for name, body in sources.items():
        with open(os.path.join(root, "paper_2403_02816_gb300", "csrc", name), "wb") as f:
            f.write(body)
    with open(os.path.join(root, "profiles", "k.md"), "w") as f:
        f.write(text)


def sha16(bodies):
    h = hashlib.sha256()
    for b in bodies:
        h.update(b)
    return h.hexdigest()[:16]


def test_traffic_is_reported_while_the_sources_match(tmp_path, monkeypatch):
    src = {"a.cu": b"kernel a", "b.cuh": b"header b"}
    text = "summary\ntraffic_bytes_per_launch: 12345\nsource_sha256_16: %s (a.cu, b.cuh)\n" % sha16(
        [src["a.cu"], src["b.cuh"]])
    write_tree(str(tmp_path), src, text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k.md", ["a.cu", "b.cuh"]) == 12345.0
    # the order of the sources is part of the hash
    assert bench.profiled_traffic("k.md", ["b.cuh", "a.cu"]) is None


def test_traffic_is_null_once_a_source_changes(tmp_path, monkeypatch):
    src = {"a.cu": b"kernel a", "b.cuh": b"header b"}
    text = "traffic_bytes_per_launch: 999\nsource_sha256_16: %s\n" % sha16([src["a.cu"], src["b.cuh"]])
    write_tree(str(tmp_path), src, text)
    with open(os.path.join(str(tmp_path), "paper_2403_02816_gb300", "csrc", "a.cu"), "ab") as f:
        f.write(b" changed")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k.md", ["a.cu", "b.cuh"]) is None
    assert bench.profiled_traffic("missing.md", ["a.cu"]) is None

