"""Pins of the paper's flop convention (Table 1, Sec. 3; the Appendix counts 19
flops per gravity interaction): for every kernel the printed GFLOPS divided by
the printed giga-interactions per second gives the printed flops per
interaction, and the benchmark converts interactions to the paper's GFLOPS with
the gravity row's count."""
import csv
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    with open(os.path.join(HERE, "golden", "table1_kernels.csv")) as fh:
        lines = [ln for ln in fh if not ln.startswith("#")]
    return list(csv.DictReader(lines))


def test_table1_flops_per_interaction_consistent():
    rows = _rows()
    assert len(rows) == 5
    for r in rows:
        ratio = float(r["gflops"]) / float(r["giga_interactions_per_s"])
        assert abs(ratio / float(r["flops_per_interaction"]) - 1.0) < 0.01, r


def test_bench_uses_the_gravity_flop_count():
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    import bench
    grav = [r for r in _rows() if r["kernel"] == "gravity_accel"][0]
    assert bench.PAPER_FLOPS_PER_PAIR == int(grav["flops_per_interaction"])
    assert bench.paper_gflops(4.97) == float(grav["flops_per_interaction"]) * 4.97
