"""The schedule table's host logic (keys, JSON round trip, apply rules) with a
stand-in solver; the timing itself is covered by the GPU tests."""
import json

from paper_1805_03155_gb300 import tune


class FakeCfg:
    def __init__(self, dims, n, precision):
        self.dims = dims
        self.n = list(n) + [1] * (3 - len(n))
        self.precision = precision


class FakeSolver:
    def __init__(self, dims, n, precision, candidates):
        self.cfg = FakeCfg(dims, n, precision)
        self.cand = candidates
        self.sched = [0, 0, 0]

    def spstd_schedule_candidates(self, ax):
        return self.cand[ax]

    def spstd_set_schedule(self, ax, v):
        assert v in self.cand[ax]
        self.sched[ax] = v

    def spstd_get_schedule(self, ax):
        return self.sched[ax]

    def spstd_tune(self, reps):
        self.sched = [self.cand[a][-1] for a in range(self.cfg.dims)] + [0] * (3 - self.cfg.dims)
        return [[0.1 * (a + 1) + 0.01 * v for v in range(5)] for a in range(3)]


def test_keys():
    assert tune.shape_key(3, (256, 256, 256), 32) == "3d:256x256x256:fp32"
    assert tune.shape_key(1, (4096, 1, 1), 64) == "1d:4096:fp64"
    assert tune.solver_key(FakeSolver(2, (128, 64), 32, [[0], [0]])) == "2d:128x64:fp32"


def test_round_trip_and_apply(tmp_path):
    t = tune.ScheduleTable()
    s = FakeSolver(2, (128, 64), 32, [[0, 1, 2, 3], [0, 2]])
    assert t.tune(s) == [3, 2]
    path = str(tmp_path / "sched.json")
    t.save(path)
    doc = json.load(open(path))
    assert doc["version"] == tune.VERSION and doc["entries"]["2d:128x64:fp32"]["schedule"] == [3, 2]
    t2 = tune.ScheduleTable.load(path)
    s2 = FakeSolver(2, (128, 64), 32, [[0, 1, 2, 3], [0, 2]])
    assert t2.apply(s2) and s2.sched[:2] == [3, 2]
    # a build without that schedule, or an unknown shape, leaves the solver alone
    s3 = FakeSolver(2, (128, 64), 32, [[0, 1], [0, 2]])
    assert not t2.apply(s3) and s3.sched == [0, 0, 0]
    assert not t2.apply(FakeSolver(2, (64, 64), 32, [[0], [0]]))
    assert tune.ScheduleTable.load(str(tmp_path / "absent.json")).entries == {}
