"""The autotuner picks the fastest shape, skips refused shapes and caches."""
from paper_2310_02043_gb300 import autotune


class FakeTracer:
    def __init__(self, refuse=()):
        self.shape = None
        self.refuse = set(refuse)

    def set_launch(self, *shape):
        if tuple(shape) in self.refuse:
            raise RuntimeError("does not fit")
        self.shape = tuple(shape)


def test_picks_fastest_skips_refused_and_caches(tmp_path):
    cost = {c: 10.0 + i for i, c in enumerate(autotune.CANDIDATES)}
    fast = autotune.CANDIDATES[3]
    cost[fast] = 1.0
    tr = FakeTracer(refuse=[autotune.CANDIDATES[0]])
    timer = lambda run: cost[tr.shape]
    path = str(tmp_path / "tune.json")
    best, res = autotune.tune(tr, lambda: None, "k", cache_path=path, timer=timer)
    assert best == fast and tr.shape == fast
    assert autotune.CANDIDATES[0] not in res
    tr2 = FakeTracer()
    best2, res2 = autotune.tune(tr2, lambda: None, "k", cache_path=path, timer=lambda run: 1 / 0)
    assert best2 == fast and tr2.shape == fast and res2 == res
