"""The stored expected values under tests/golden/ are well formed and self-consistent (CPU only).

* point_source_residuals_lattice.txt (written by make_point_source_residuals.py from the oracle):
  for each wavenumber 32 per-body norms whose root sum of squares is the stored total, a total at
  the discretisation level at k = 0, and growth with k (the quadrature error of the rows next to
  another body's surface).
* table1_rms.txt (the paper's Table I): three rows, K = 5, 10, 20, errors falling with K.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def test_point_source_residuals_are_consistent():
    rows = _rows("point_source_residuals_lattice.txt")
    by_k = {}
    for k, b, v in rows:
        by_k.setdefault(float(k), {})[int(b)] = float(v)
    assert sorted(by_k) == [0.0, 6.0, 24.0]
    totals = []
    for k, d in sorted(by_k.items()):
        assert sorted(d) == list(range(-1, 32)), k
        bodies = np.array([d[b] for b in range(32)])
        assert np.all(bodies > 0)
        assert abs(np.sqrt(np.sum(bodies ** 2)) - d[-1]) <= 1e-9 * d[-1], k
        totals.append(d[-1])
    assert totals[0] < 2e-4 and totals[0] < totals[1] < totals[2]


def test_table1_fixture():
    rows = _rows("table1_rms.txt")
    assert [int(r[0]) for r in rows] == [5, 10, 20]
    rms = np.array([[float(r[2]), float(r[3])] for r in rows])
    assert np.all(np.diff(rms, axis=0) < 0)
