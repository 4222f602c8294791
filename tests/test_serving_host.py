"""Host logic of the serving loop's HBM admission (no GPU): reservation, LRU eviction of idle
operators, and the rule that a batch never evicts the operator it is about to reuse."""
import collections
import threading

import numpy as np
import pytest

from paper_1909_08734_gb300 import CpmError, serving


class _FakePc:
    destroyed = []

    def __init__(self, name):
        self.name = name

    def __del__(self):
        _FakePc.destroyed.append(self.name)


def _server(budget, ops, n_active=1000):
    s = serving.Server.__new__(serving.Server)
    s.budget = budget
    s._lock = threading.RLock()
    s._busy = set()
    s._ops = collections.OrderedDict()
    s.used = 0
    s.reserved = 0
    s.counters = collections.Counter()
    s.method, s.precision, s.restart = "oras", "fp32", 50
    cp = np.zeros((n_active, 3))
    s.band = lambda surface, h: (None, None, cp)
    for key, resident in ops:
        s._ops[key] = serving._Operator(_FakePc(key[2]), resident)
        s.used += resident
    return s


def test_reuse_evicts_other_idle_operators_not_its_own():
    _FakePc.destroyed.clear()
    a, b = ("sphere", 0.05, 1.0), ("sphere", 0.05, 2.0)
    vec = 2 * 8 * 4 * 1000                       # 4 right-hand sides: solution and rhs vectors
    s = _server(budget=1000 + 1000 + vec - 1, ops=[(a, 1000), (b, 1000)])   # a is least recent
    got = s._reserve(a, 4)
    assert got is not None and got[1] is None     # reuse: no plan, vectors only
    assert a in s._ops and b not in s._ops        # b (idle) made room; a was kept
    assert s.counters["evictions"] == 1
    assert s.used == 1000 and s.reserved == vec and a in s._busy
    assert list(s._ops) == [a]
    s._release(a, vec)
    assert s.reserved == 0 and not s._busy


def test_busy_operators_are_not_evicted_and_reservation_waits():
    a, b = ("sphere", 0.05, 1.0), ("sphere", 0.05, 2.0)
    vec = 2 * 8 * 1 * 1000
    s = _server(budget=2000 + vec - 1, ops=[(a, 1000), (b, 1000)])
    s._busy.add(b)                                # b runs a batch
    assert s._reserve(a, 1) is None               # a stays, b is busy: nothing fits now
    assert a in s._ops and b in s._ops and s.reserved == 0 and a not in s._busy


def test_new_operator_evicts_lru_and_never_fitting_raises(monkeypatch):
    a, b, c = ("sphere", 0.05, 1.0), ("sphere", 0.05, 2.0), ("sphere", 0.05, 3.0)
    plan = {"setup_peak_bytes": 1500, "resident_bytes": 900}
    monkeypatch.setattr(serving, "oras_plan", lambda *args: plan)
    vec = 2 * 8 * 1 * 1000
    s = _server(budget=2000 + 1500 + vec - 1, ops=[(a, 1000), (b, 1000)])
    need, got_plan = s._reserve(c, 1)
    assert got_plan is plan and need == 1500 + vec
    assert list(s._ops) == [b]                    # a (least recent) went
    plan["setup_peak_bytes"] = 10 ** 9
    with pytest.raises(CpmError):
        s._reserve(("torus", 0.05, 1.0), 1)
