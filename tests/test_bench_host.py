"""Host logic of bench.py that the roofline line rests on (no GPU): the
algorithmic byte counts of a sparse product and of a whole solve, and the
gate that reports measured DRAM traffic only for a captured numbering, shape
and source state."""
import dataclasses
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@dataclasses.dataclass
class Shape:
    m: int
    n: int
    nnz: int


def test_spmv_bytes_by_hand():
    P = Shape(m=3, n=5, nnz=8)
    # FP32 values, 32-bit columns: A = 8*(4+4) + 4*4 + 3*4 + 5*4, A^T = 8*8 + 6*4 + 5*4 + 3*4
    a = 8 * 8 + 16 + 12 + 20
    at = 8 * 8 + 24 + 20 + 12
    assert bench.spmv_bytes(P, "f32") == pytest.approx(0.5 * (a + at))
    # 16-bit offsets on A only: 2.5 bytes of column storage per entry
    a16 = 8 * (4 + 2.5) + 16 + 12 + 20
    assert bench.spmv_bytes(P, "f32", True, False) == pytest.approx(0.5 * (a16 + at))
    # BF16 values, FP32 basis; FP64 values with an FP64 basis
    assert bench.spmv_bytes(P, "bf16") == pytest.approx(0.5 * (a + at) - 8 * 2)
    a64 = 8 * 12 + 16 + 24 + 40
    at64 = 8 * 12 + 24 + 40 + 24
    assert bench.spmv_bytes(P, "f64") == pytest.approx(0.5 * (a64 + at64))


def test_solve_bytes_by_hand():
    P = Shape(m=3, n=5, nnz=8)
    K = 2
    sb = 4
    elim = sum((5 * k + 3 * (k + 1)) * sb + 4 * 8 * sb for k in range(K))
    expect = K * 2 * bench.spmv_bytes(P, "f32") + elim + 5 * K * sb + 5 * 8
    assert bench.solve_bytes(P, "f32", K) == pytest.approx(expect)


def _current_digests():
    import hashlib

    out = {}
    for rel in bench.SPMV_TRAFFIC["sources"]:
        with open(os.path.join(bench.ROOT, rel), "rb") as f:
            out[rel] = hashlib.sha256(f.read()).hexdigest()
    return out


def test_traffic_gate(monkeypatch):
    # the gate's lookups, with the recorded digests set to the sources as
    # they are (whether the capture is current is the gate's own business)
    monkeypatch.setitem(bench.SPMV_TRAFFIC, "sources", _current_digests())
    tab = bench.SPMV_TRAFFIC
    ok = bench.spmv_traffic("ct512", "f32", "tiles", "16x2/16-bit", "16x2/16-bit")
    assert ok == pytest.approx(0.5 * (tab["bytes"]["tiles"]["16x2/16-bit"][0] +
                                      tab["bytes"]["tiles"]["16x2/16-bit"][1]))
    # the average of A's traffic in its shape and A^T's in its own
    mixed = bench.spmv_traffic("ct512", "f32", "natural", "16x2/16-bit", "16x2")
    assert mixed == pytest.approx(0.5 * (tab["bytes"]["natural"]["16x2/16-bit"][0] +
                                         tab["bytes"]["natural"]["16x2"][1]))
    assert bench.spmv_traffic("ct256", "f32", "tiles", "16x2", "16x2") is None
    assert bench.spmv_traffic("ct512", "bf16", "tiles", "16x2", "16x2") is None
    assert bench.spmv_traffic("ct512", "f32", "other", "16x2", "16x2") is None
    assert bench.spmv_traffic("ct512", "f32", "tiles", "no-such-shape", "16x2") is None


def test_traffic_gate_closes_when_a_source_changes(monkeypatch):
    src = _current_digests()
    monkeypatch.setitem(bench.SPMV_TRAFFIC, "sources", dict(src))
    assert bench.spmv_traffic("ct512", "f32", "tiles", "16x2", "16x2") is not None
    first = next(iter(src))
    src[first] = "0" * 64
    monkeypatch.setitem(bench.SPMV_TRAFFIC, "sources", src)
    assert bench.spmv_traffic("ct512", "f32", "tiles", "16x2", "16x2") is None


def test_every_numbering_has_a_note_and_a_table():
    for order in ("tiles", "natural"):
        assert order in bench.ORDER_NOTE
        assert set(bench.SPMV_TRAFFIC["bytes"][order]) >= {"16x2", "16x2/16-bit"}


def test_cpu_baseline_from_concurrent_oracle_runs():
    """cpu_baseline takes the FP64 run of the benchmark's noise level as the
    one-thread figure and the span of all concurrent runs as the multi-core
    one (runs are supplied by a stand-in for the process pool's result)."""

    class Done:
        def __init__(self, runs):
            self.runs = runs

        def get(self):
            return self.runs

    runs = [
        {"value_type": vt, "eta": eta, "k_done": 300, "seconds": sec,
         "wall_start": 100.0 + i, "wall_end": 100.0 + i + sec}
        for i, (vt, eta, sec) in enumerate([("f64", 0.005, 200.0), ("f32", 0.005, 190.0),
                                            ("f64", 0.02, 210.0)])]

    @dataclasses.dataclass
    class P:
        eta: float = 0.005

    cb = bench.cpu_baseline(P(), 300, 15.0, oracle_runs=Done(runs))
    assert cb["cores"] == 1 and cb["value"] == pytest.approx(300 / 200.0)
    mc = cb["multi_core"]
    # earliest start 100, latest end 102 + 210 = 312
    assert mc["cores"] == 3 and mc["value"] == pytest.approx(900 / 212.0)
