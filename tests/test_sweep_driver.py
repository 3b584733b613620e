"""Host logic of run_until_slip (the onset-of-slip driver of Sec. 5's
stress-rotation study) against a stand-in solver, no GPU: it stops at the
first step whose state holds a slipping pair and reports the elapsed time and
the injected volume."""
import numpy as np

import paper_2410_17133_gb300 as gm


class FakeSolver:
    def __init__(self, slip_at):
        self.n = 0
        self.slip_at = slip_at
        self.dts = []

    def step(self, dt, **kw):
        self.n += 1
        self.dts.append(dt)

    def get_state(self):
        flags = np.full(5, gm.STICK, np.int8)
        if self.slip_at is not None and self.n >= self.slip_at:
            flags[2] = gm.SLIP
        return {"flags": flags}


def test_stops_at_first_slip():
    s = FakeSolver(slip_at=3)
    n, t, vol, st = gm.run_until_slip(s, [1.0, 2.0, 4.0, 8.0, 16.0], Q=0.5)
    assert (n, t, vol) == (3, 7.0, 3.5)
    assert s.dts == [1.0, 2.0, 4.0]
    assert (st["flags"] == gm.SLIP).sum() == 1


def test_runs_all_steps_without_slip():
    s = FakeSolver(slip_at=None)
    n, t, vol, st = gm.run_until_slip(s, [1.0, 1.0], Q=2.0)
    assert (n, t, vol) == (2, 2.0, 4.0)
    assert not np.any(st["flags"] == gm.SLIP)
