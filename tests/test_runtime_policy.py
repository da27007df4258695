"""Admission choice of the continuous-batching server (host logic, no GPU): arrival, HBM
budget and the FIFO / shortest-job-first policies."""
import pytest

from paper_2208_06970_b300.runtime import pick_next


def _reqs():
    return [dict(arrival=0.0, bytes=8, work=800), dict(arrival=0.1, bytes=2, work=100),
            dict(arrival=0.2, bytes=4, work=50), dict(arrival=5.0, bytes=1, work=1)]


def test_only_arrived_requests_are_admitted():
    r = _reqs()
    assert pick_next([0, 1, 2, 3], r, -1.0, 0, 100, 0) is None
    assert pick_next([3], r, 4.9, 0, 100, 1, "sjf") is None
    assert pick_next([3], r, 5.0, 0, 100, 1, "sjf") == 3


def test_fifo_takes_the_earliest_and_waits_for_it():
    r = _reqs()
    assert pick_next([0, 1, 2, 3], r, 1.0, 0, 100, 1) == 0
    # the head does not fit the budget left: FIFO waits (no overtaking)
    assert pick_next([0, 1, 2, 3], r, 1.0, 95, 100, 1) is None


def test_sjf_takes_the_least_work_that_fits():
    r = _reqs()
    assert pick_next([0, 1, 2, 3], r, 1.0, 0, 100, 1, "sjf") == 2
    # 2 does not fit (4 bytes over 97 used of 100): the next smallest that fits
    assert pick_next([0, 1, 2, 3], r, 1.0, 97, 100, 1, "sjf") == 1
    # ties on work go to the earlier arrival
    r[1]["work"] = 50
    assert pick_next([0, 1, 2], r, 1.0, 0, 100, 1, "sjf") == 1


def test_an_idle_server_admits_an_oversized_request():
    r = _reqs()
    assert pick_next([0], r, 1.0, 0, 4, 0) == 0
    assert pick_next([0], r, 1.0, 0, 4, 0, "sjf") == 0
    assert pick_next([0], r, 1.0, 0, 4, 1) is None


def test_unknown_policy():
    with pytest.raises(ValueError):
        pick_next([0], _reqs(), 1.0, 0, 100, 0, "lifo")
