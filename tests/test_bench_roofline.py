"""CPU checks of the benchmark's roofline bookkeeping: the ncu traffic summary of the odd-even
half apply parses into per-layout, per-precision bytes that sit just above the algorithmic bytes
of one S apply (9 n^2 V block entries + 2.5 V n vector entries), and the layout the autotuner
chose is read back from its report, so that a line's `traffic` belongs to the kernel it timed."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_profiled_traffic_per_layout():
    traffic, src = bench.profiled_traffic("tm16")
    assert src == os.path.join("profiles", "k_eo_half_tm16.md")
    V, n = 16 ** 4, 48
    alg = {"fp32": 9 * n * n * V * 8 + 2.5 * V * n * 8, "bf16": 9 * n * n * V * 4 + 2.5 * V * n * 8}
    layouts = {k[0] for k in traffic}
    assert {1, 2, 3, 6} <= layouts
    for (layout, prec), b in traffic.items():
        assert prec in alg, (layout, prec)
        assert 1.0 <= b / alg[prec] <= 1.02, (layout, prec, b / alg[prec])


def test_profiled_traffic_missing_workload():
    assert bench.profiled_traffic("no-such-workload") == ({}, None)


class _FakeLib:
    def __init__(self, report):
        self.report = report

    def autotune_report(self):
        return self.report


def test_eo_choice_reads_the_autotuner_report():
    rep = ("apply/p2/n48/v16@sm103x152 -> 1 0 0 46.7 | 0,0,0:50 1,0,0:46.7\n"
           "eo/p1/n48/v16@sm103x152 -> 2 0 0 797.3 | 0,0,0:1050 2,0,0:797.3\n"
           "eo/p2/n48/v16@sm103x152 -> 1 0 0 413.3 | 0,0,0:473 1,0,0:413.3\n")
    cg = _FakeLib(rep)
    assert bench.eo_choice(cg, 1, 48) == 2
    assert bench.eo_choice(cg, 2, 48) == 1
    assert bench.eo_choice(cg, 2, 32) is None
    assert bench.eo_layout(cg, 2, 48) == bench.EO_LAYOUTS[1]
    assert bench.eo_layout(cg, 2, 32) == "k_eo_half"
