"""Admission choice of the continuous-batching server (host logic, no GPU): arrival, HBM
budget and the FIFO / shortest-job-first policies."""
import pytest
import torch

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


def test_crop_pool_cuts_each_request_inside_the_masters():
    """The served stream's inputs are sub-volumes of resident masters: every request gets its
    own dims and number of variables, at a seeded offset that keeps the cut inside the masters,
    and the same request always gets the same data."""
    import workloads
    pool = workloads.CropPool(side=24, n_aux=16, seed=7, device="cpu")
    reqs = workloads.request_stream(n_requests=30, rate=50.0, seed=5, lo=4, hi=24)
    for r in reqs:
        f, aux = pool.request_data(r)
        nx, ny, nz = r["dims"]
        assert f.shape == (nz, ny, nx) and f.is_contiguous()
        assert len(aux) == r["n_aux"] and all(a.shape == f.shape for a in aux)
        f2, _ = pool.request_data(r)
        assert torch.equal(f, f2)
        # the cut is a window of the master: find it by its first voxel's row
        assert any(torch.equal(f, pool.field[z:z + nz, y:y + ny, x:x + nx])
                   for z in range(24 - nz + 1) for y in range(24 - ny + 1) for x in range(24 - nx + 1)
                   if pool.field[z, y, x] == f[0, 0, 0])


def test_fill_slots_take_only_small_requests_and_may_overtake():
    r = _reqs()  # work 800, 100, 50, 1
    # a fill slot (max_work 100) skips the large head and takes the earliest small request
    assert pick_next([0, 1, 2, 3], r, 1.0, 0, 100, 1, "fifo", max_work=100) == 1
    assert pick_next([0, 2, 3], r, 1.0, 0, 100, 1, "fifo", max_work=100) == 2
    # nothing small has arrived yet
    assert pick_next([0, 3], r, 1.0, 0, 100, 1, "fifo", max_work=100) is None
    # the main slot keeps arrival order
    assert pick_next([0, 1, 2, 3], r, 1.0, 0, 100, 1, "fifo") == 0
