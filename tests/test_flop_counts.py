"""The fixed-work benchmark's flop accounting against the paper's Table I
(tests/golden/table1_flop_counts.txt, typed from Table I and Sec. IV-B)."""
import os

import bench_suite

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_flop_counts.txt")


def table1():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_constants_match_table1():
    t = table1()
    assert bench_suite.FLOP_DHAT == t["DHAT"]
    assert bench_suite.FLOP_AXPY == t["AXPY"]
    assert bench_suite.FLOP_DOT == t["DOT"]
    assert bench_suite.FLOP_NORM == t["NORM2"]


def test_table1_is_self_consistent():
    t = table1()
    # D^ = 1 - kappa^2 H~ H~: two MULTs and one 24-real complex update
    assert t["DHAT"] == 2 * t["MULT"] + 48
    # Sec. IV-B: 180 single-precision complex numbers (8 bytes) per 2232 flop
    assert abs(t["MULT_COMPLEX_PER_SITE"] * 8 / t["MULT"] - t["BYTE_PER_FLOP_NO_REUSE"]) < 5e-4


def test_inner_iteration_count():
    # two D^, six vector updates, three dots and three norms per iteration
    t = table1()
    n = 2 * t["DHAT"] + 6 * t["AXPY"] + 3 * t["DOT"] + 3 * t["NORM2"]
    assert bench_suite.FLOP_INNER_ITER == n == 10032
