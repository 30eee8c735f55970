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



def test_timed_steps_reports_each_call(monkeypatch):
    """timed_steps on a fake clock: the mean over the timed calls per time
    step, and every call's own figure in `each` (an outlier stays visible)."""
    import torch

    clock = {"t": 0.0}

    class FakeEvent:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = clock["t"]

        def elapsed_time(self, other):
            return other.t - self.t

    class FakeFlush:
        def fill_(self, v):
            clock["t"] += 100.0  # outside the events

    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    calls = []

    def step(k):
        calls.append(k)
        # 2 ms per time step, the third timed call 10x slower
        clock["t"] += (20.0 if len(calls) == 3 + 3 else 2.0) * k

    each = []
    ms = bench.timed_steps(step, 4, 5, 3, FakeFlush(), None, each)
    assert calls == [1, 1, 1, 5, 5, 5, 5]
    assert each == [2.0, 2.0, 20.0, 2.0]
    assert abs(ms - (2.0 + 2.0 + 20.0 + 2.0) / 4) < 1e-12
    assert bench.timed_steps(step, 1, 5, 3, FakeFlush(), None) == 2.0
