"""bench.py's host-side arithmetic (no GPU): the TEPS mean, the per-level
algorithmic-bytes model and the traffic record of the committed capture."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_harmonic_gteps_hand_values():
    # two searches of 1e9 edges in 1 s and 0.5 s: rates 1 and 2 GTEPS, harmonic
    # mean 2 / (1 + 0.5) = 4/3
    assert bench.harmonic_gteps([10 ** 9, 10 ** 9], [1000.0, 500.0]) == pytest.approx(4 / 3)
    assert bench.harmonic_gteps([5 * 10 ** 8], [250.0]) == pytest.approx(2.0)


def test_level_bytes_model_hand_values():
    nb = 64  # two bitmap words
    bu = {"dir": 1, "n_u": 10, "examined": 7, "n_next": 3, "n_f": 0, "m_f": 0}
    # 4*2 visited words + 8*10 row bounds + 8*7 probes + 8*3 outputs + 8*2 writes
    assert bench.level_bytes(bu, nb) == 8 + 80 + 56 + 24 + 16
    td = {"dir": 0, "n_f": 5, "m_f": 40, "n_next": 6, "n_u": 0, "examined": 0}
    # 20 per frontier vertex + 8 per edge + 16 per new vertex
    assert bench.level_bytes(td, nb) == 100 + 320 + 96


def test_committed_traffic_record_parses():
    # a number while bfs.cu is the captured source, else None with the reason
    traffic, src = bench.measured_traffic("bu_pull")
    assert (traffic is not None and traffic > 0) or src == "kernel source changed since the capture"
    assert bench.measured_traffic("no_such_kernel")[0] is None
