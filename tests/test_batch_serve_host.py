"""Host logic of the batch runner, the autotuner and the serving loop (no GPU)."""
import json

import pytest

from paper_2005_06170_gb300 import autotune
from paper_2005_06170_gb300.batch import deal
from paper_2005_06170_gb300.serve import AdmissionPolicy, Request, percentiles


def test_deal_balances_lanes_largest_first():
    costs = [10, 1, 7, 3, 3, 2]
    lanes = deal(costs, 2)
    load = [sum(c for c, l in zip(costs, lanes) if l == k) for k in range(2)]
    assert sorted(load) == [13, 13]
    assert lanes[0] == 0  # the largest goes first, to lane 0
    assert deal([], 3) == []
    assert deal([5], 4) == [0]


def _req(fp, rid):
    r = Request(pos=None, vel=None, params=None)
    r.footprint, r.rid = fp, rid
    return r


def test_admission_first_fit_within_budget_and_lanes():
    pol = AdmissionPolicy(budget_bytes=100)
    q = [_req(60, 0), _req(50, 1), _req(30, 2), _req(10, 3)]
    got = pol.admit(q, free_lanes=4, in_use=0)
    assert [r.rid for r in got] == [0, 2, 3]  # 60 + 30 + 10; the 50 waits
    assert q[1].overtaken == 1
    got = pol.admit(q, free_lanes=1, in_use=0)
    assert [r.rid for r in got] == [0]


def test_admission_bounds_overtaking():
    pol = AdmissionPolicy(budget_bytes=100, max_overtake=2)
    big = _req(90, 0)
    q = [big, _req(20, 1)]
    for _ in range(2):
        assert [r.rid for r in pol.admit(q, free_lanes=2, in_use=30)] == [1]
    # overtaken twice: now nothing behind it may start until it fits
    assert pol.admit(q, free_lanes=2, in_use=30) == []
    assert [r.rid for r in pol.admit(q, free_lanes=2, in_use=0)] == [0]


def test_admission_strict_lane_kinds():
    """Separate lanes for large requests: a large request starts only on a free large
    lane and a small one only on a free small lane; waiting for its kind of lane is not
    an overtake."""
    pol = AdmissionPolicy(budget_bytes=1000, max_overtake=1)
    large = lambda r: r.footprint > 100  # noqa: E731
    q = [_req(500, 0), _req(10, 1), _req(20, 2), _req(400, 3), _req(30, 4)]
    got = pol.admit(q, free_lanes=3, in_use=0, free_large=1, is_large=large)
    assert [r.rid for r in got] == [0, 1, 2]  # one large lane, two small ones
    assert q[3].overtaken == 0
    rest = [q[3], q[4]]
    got = pol.admit(rest, free_lanes=2, in_use=500, free_large=0, is_large=large)
    assert [r.rid for r in got] == [4]  # the large lane is busy: the large request waits
    assert q[3].overtaken == 0
    for _ in range(3):  # lane-bound waits never make it block the small requests
        assert [r.rid for r in pol.admit(rest, free_lanes=2, in_use=500, free_large=0, is_large=large)] == [4]
    got = pol.admit(rest, free_lanes=1, in_use=500, free_large=1, is_large=large)
    assert [r.rid for r in got] == [3]


def test_admission_respects_memory_in_use():
    pol = AdmissionPolicy(budget_bytes=100)
    q = [_req(40, 0)]
    assert pol.admit(q, free_lanes=3, in_use=70) == []
    assert len(pol.admit(q, free_lanes=3, in_use=60)) == 1


def test_percentiles():
    lat = list(range(1, 101))
    p = percentiles(lat)
    assert p["p50"] == 50 and p["p99"] == 99
    assert percentiles([])["p50"] is None


def test_autotune_candidates_and_classes():
    assert autotune.density_class(256 ** 3, 256) == 0
    assert autotune.density_class(32 ** 3, 256) == -9
    assert autotune.density_class(1, 1024) == -10
    c = autotune.candidates(256, 0)
    assert (0, -1) in c and (1, 0) in c and (3, -1) in c
    assert (7, -1) in c and (7, 0) not in c  # home tiles keep no particle list
    assert all(t in autotune.F32_TILES for t, _ in c)
    c40 = autotune.candidates(40, 0)
    assert {t for t, _ in c40} == {3}  # only 8x8x8 divides 40
    c64 = autotune.candidates(64, 1)
    assert {t for t, _ in c64} == {4, 5, 6} and all(cap == -1 for _, cap in c64)


class _Cat:
    def __init__(self, n):
        self.n = n


class _P:
    def __init__(self, ng, precision=0):
        self.ng, self.precision = ng, precision


def test_autotune_picks_fastest_and_caches(tmp_path):
    calls = []

    def timer(ctx, cat, p, tile, cap):
        calls.append((tile, cap))
        return {(1, 0): 1.0}.get((tile, cap), 5.0)

    path = str(tmp_path / "tune.json")
    t = autotune.Autotuner(path=path, timer=timer)
    assert t.choose(None, _Cat(256 ** 3), _P(256), "GB300") == (1, 0)
    n_first = len(calls)
    assert t.choose(None, _Cat(250 ** 3), _P(256), "GB300") == (1, 0)  # same class: cached
    assert len(calls) == n_first
    saved = json.load(open(path))
    assert list(saved) == [autotune.Autotuner.key("GB300", 256, 0, 256 ** 3)]
    t2 = autotune.Autotuner(path=path, timer=lambda *a: pytest.fail("should come from the cache"))
    assert t2.choose(None, _Cat(256 ** 3), _P(256), "GB300") == (1, 0)


def test_requests_compare_by_identity():
    a, b = _req(10, 0), _req(10, 0)
    assert a != b and a == a
    q = [a, b]
    assert q.index(b) == 1


def test_autotuner_restricted_tiles(tmp_path):
    """A restricted choice times only the allowed tiles and is cached under its own key."""
    calls = []

    def timer(ctx, cat, p, tile, cap):
        calls.append((tile, cap))
        return {0: 3.0, 2: 1.0, 7: 2.0}.get(tile, 5.0)

    class P:
        ng, precision = 64, 0

    class C:
        n = 64 ** 3

    t = autotune.Autotuner(path=str(tmp_path / "t.json"), timer=timer)
    assert t.choose(None, C, P, "g") == (2, -1)
    free = len(calls)
    assert t.choose(None, C, P, "g", tiles=(0, 7))[0] == 7
    assert all(tile in (0, 7) for tile, _ in calls[free:])
    assert t.choose(None, C, P, "g", tiles=(0, 7))[0] == 7  # cached
    assert len(calls) == free + len([c for c in autotune.candidates(64, 0) if c[0] in (0, 7)])
