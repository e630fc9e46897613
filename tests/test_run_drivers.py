"""Host logic of the long-run drivers (no GPU): the chunked advance reaches the target time with
few steps at dt = 0 after the stop, and only advancing steps are counted. A fake solver stands in
for the device: dt grows slowly and is capped at the stop time, as the device's dt is."""
import numpy as np

from paper_2501_15923_gb300.precision import advance, advancing_steps


class FakeSolver:
    def __init__(self, dt0=0.01, growth=1.00005):
        self.t, self.dt0, self.growth, self.stop, self.k = 0.0, dt0, growth, 0.0, 0
        self.ring = [(0.0,)]
        self.launched = 0

    def set_stop_time(self, t):
        self.stop = t

    def _dt(self):
        dt = self.dt0 * self.growth ** self.k
        return max(min(dt, self.stop - self.t), 0.0) if self.stop > 0 else dt

    def time(self):
        return self.t, self._dt()

    def step(self, n):
        for _ in range(n):
            dt = self._dt()
            self.t += dt
            self.k += 1
            self.launched += 1
            self.ring.append((self.t,))

    def sample(self, traj, cap):
        rec = np.array(self.ring[:cap], dtype=float).reshape(-1, 1, 1)
        self.ring = self.ring[cap:]
        return rec, rec.shape[0]


def test_advance_stops_on_time_with_few_idle_steps():
    s = FakeSolver()
    recs = []
    for target in (3.0, 7.5, 12.25):
        s.set_stop_time(target)
        advance(s, target, chunk=500, ring=1 << 16, recs=recs)
        assert abs(s.t - target) <= 1e-12 * target
    series = np.concatenate(recs)
    n_adv = advancing_steps(series)
    assert s.launched - n_adv <= 3            # at most one dt = 0 step per target
    assert n_adv == int((np.diff(series[:, 0, 0]) > 0).sum())


def test_advancing_steps_ignores_repeated_times():
    t = np.array([0.0, 1.0, 2.0, 2.0, 2.0, 3.0]).reshape(-1, 1, 1)
    assert advancing_steps(t) == 3
