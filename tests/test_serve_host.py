"""Host-side logic of the relight serving loop (CPU): the arrival trace and the scheduler's
arguments, checked without a device."""
import numpy as np
import pytest

from paper_2607_22780_b300 import serve


def test_poisson_trace_is_seeded_sorted_and_drawn_from_the_workload():
    dist = {"a": 3.0, "b": 30.0}
    t1 = serve.make_trace(400, 200.0, dist, seed=3)
    t2 = serve.make_trace(400, 200.0, dist, seed=3)
    assert [r.arrival for r in t1] == [r.arrival for r in t2]
    arr = np.array([r.arrival for r in t1])
    assert np.all(np.diff(arr) >= 0)
    # mean gap of a Poisson process at 200/s: 5 ms (400 samples: within 20 %)
    assert 0.004 < np.diff(arr).mean() < 0.006
    assert {r.scene for r in t1} == {"a", "b"}
    assert {r.camera.width for r in t1} <= {256, 512, 1024}
    assert {r.rays for r in t1} <= {8, 16, 32, 64}
    for r in t1:
        assert sum(r.alloc) == r.rays and r.alloc == (r.rays // 2, r.rays // 4, r.rays // 4)


def test_scheduler_rejects_an_unknown_slice_order():
    with pytest.raises(ValueError):
        serve.RelightServer({}, order="lifo")
