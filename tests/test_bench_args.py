"""Host logic of the benchmark's arguments (CPU only)."""
import sys

import bench


def _parse(argv):
    old = sys.argv
    sys.argv = ["bench.py"] + argv
    try:
        return bench.parse_args()
    finally:
        sys.argv = old


def test_defaults_run_the_accuracy_ladder_at_the_tight_reference():
    a = _parse([])
    assert a.gpus == 1 and not a.no_accuracy
    assert a.ref_tol == bench.REF_TOL


def test_large_workload_skips_the_ladder_unless_asked():
    a = _parse(["--workload", "large"])
    assert a.no_accuracy and a.ref_tol == 1e-10
    b = _parse(["--workload", "large", "--accuracy", "--ref-tol", "1e-12"])
    assert not b.no_accuracy and b.ref_tol == 1e-12
