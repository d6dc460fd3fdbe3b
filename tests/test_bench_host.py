"""Host logic of bench.py (no GPU): the roofline's `traffic` is reported only for
the kernel, shape, size and chunk count it was measured on, and only while the
kernel sources hash to what they were when it was measured."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def _hash(bench, files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(bench.ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def test_traffic_needs_the_measured_configuration(monkeypatch):
    bench = _bench()
    srcs = bench.MEASURED_TRAFFIC["sources"]
    fake = dict(kernel=("k_pair2x", 0, 1 << 18), bytes={(128, 4, 13): 111, (128, 4, 19): 222, (128, 8, 7): 333},
                sources=srcs, sha256=_hash(bench, srcs))
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", fake)
    assert bench.measured_traffic("k_pair2x", 0, 128, 4, 1 << 18, 19) == 222
    assert bench.measured_traffic("k_pair2x", 0, 128, 4, 1 << 18, 13) == 111
    assert bench.measured_traffic("k_pair2x", 0, 128, 8, 1 << 18, 7) == 333
    assert bench.measured_traffic("k_pair2x", 0, 128, 4, 1 << 18, 26) is None     # chunk count not measured
    assert bench.measured_traffic("k_pair2x", 0, 128, 8, 1 << 18, 19) is None     # another shape
    assert bench.measured_traffic("k_pair2x", 1, 128, 4, 1 << 18, 19) is None     # the other pair kind
    assert bench.measured_traffic("k_pair2x", 0, 128, 4, 1 << 16, 19) is None     # another size


def test_traffic_is_dropped_when_the_sources_change(monkeypatch):
    bench = _bench()
    srcs = bench.MEASURED_TRAFFIC["sources"]
    fake = dict(kernel=("k_pair2x", 0, 1 << 18), bytes={(128, 4, 19): 222}, sources=srcs, sha256="0" * 64)
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", fake)
    assert bench.measured_traffic("k_pair2x", 0, 128, 4, 1 << 18, 19) is None


def test_recorded_traffic_covers_the_chunk_counts_the_autotuner_can_pick():
    """The autotuner tries 1, 1.5, 2 and 2.5 times the planned chunk count of the
    fastest shape: 13 for the 128 x 4 step-1 shape at N = 2^18 (capped at 32), 7 for
    128 x 8."""
    bench = _bench()
    got = set(bench.MEASURED_TRAFFIC["bytes"])
    assert got >= {(128, 4, c) for c in (13, 19, 26, 32)}
    assert got >= {(128, 8, c) for c in (7, 10, 14, 17)}
