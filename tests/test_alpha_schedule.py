"""The annealing schedule of Sec. VII (Fig. 5): geometric from 1 to 100 over 100 iterations."""
import os

import numpy as np

from paper_2401_11882_gb300.batched import geometric_alpha

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig5_alpha_schedule.txt")


def test_printed_alpha_values():
    sched = geometric_alpha(1.0, 100.0, 100)
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for i, val, tol in rows:
        assert abs(sched[int(i)] - float(val)) <= float(tol)
    assert sched[0] == 1.0 and abs(sched[-1] - 100.0) < 1e-4
    assert np.all(np.diff(sched) > 0)
