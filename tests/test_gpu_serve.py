"""Relight serving loop: every request's image is the same alone and in the mix; HBM
admission bounds the admitted set; cancelled requests are dropped without disturbing
the others."""
import pytest
import torch

from paper_2607_22780_b300 import api, serve, workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]


def _scenes():
    return {"a": api.Scene.from_workload(wl.scene_objects(20000, seed=3)),
            "b": api.Scene.from_workload(wl.scene_objects(8000, seed=4))}


def _trace(n=6, seed=5):
    return serve.make_trace(n, 0.0, {"a": 3.0, "b": 3.0}, seed=seed, res_choices=(24, 40), rpp_choices=(4, 8, 16),
                            env_size=(64, 32))


def _alone(st):
    a = st.req.alloc
    return api.shade_pixels(st.scene, st.gb, st.env, a[0], a[1], a[2], st.req.seed, brdf=1)


@pytest.mark.parametrize("order", ["fifo", "srpt"])
def test_batched_equals_alone_with_sliced_mixed_launches(order):
    # either slice order (oldest request first, or fewest rays left first) only schedules:
    # every request's image is its run-alone image
    srv = serve.RelightServer(_scenes(), ray_budget=3000, max_batch=4, order=order)
    trace = _trace()
    out = srv.run_batched(trace, realtime=False)
    assert out["requests"] == len(trace)
    assert out["launches"] > len(trace)          # requests were split and mixed
    for st in out["outputs"].values():
        col, vis, ind = _alone(st)
        assert torch.equal(col, st.color) and torch.equal(vis, st.vis) and torch.equal(ind, st.ind)


def test_serial_comparator_matches_batched():
    srv = serve.RelightServer(_scenes(), ray_budget=5000)
    trace = _trace(4, seed=9)
    b = srv.run_batched(trace, realtime=False)["outputs"]
    s = srv.run_serial(trace, realtime=False)["outputs"]
    for rid in b:
        assert torch.equal(b[rid].color, s[rid].color)


def test_hbm_budget_admits_one_at_a_time():
    srv = serve.RelightServer(_scenes(), hbm_budget=1, ray_budget=2000)
    out = srv.run_batched(_trace(4, seed=11), realtime=False)
    assert srv.peak_active == 1 and out["requests"] == 4


def test_cancelled_request_is_dropped():
    srv = serve.RelightServer(_scenes(), ray_budget=2000)
    trace = _trace(5, seed=13)
    srv.cancel(trace[2].rid)
    out = srv.run_batched(trace, realtime=False)
    assert trace[2].rid not in out["outputs"] and out["requests"] == 4
    for st in out["outputs"].values():
        assert torch.equal(_alone(st)[0], st.color)


def test_cancel_between_slices_leaves_the_others_intact():
    """A request cancelled after its first slice was launched, while that launch may still
    be writing its outputs: its memory must not be handed to the requests admitted after
    it, so every other request still equals its run-alone image."""
    # about two requests fit the budget at a time, so most are admitted after the cancellation
    srv = serve.RelightServer(_scenes(), hbm_budget=300_000, ray_budget=1500, max_batch=2, inflight=2)
    trace = _trace(7, seed=17)
    victim = trace[1].rid
    seen = []

    def on_launch(i, slices):
        seen.extend(rid for rid, _, _ in slices)
        if victim in seen:
            srv.cancel(victim)

    out = srv.run_batched(trace, realtime=False, on_launch=on_launch)
    assert victim in seen and victim not in out["outputs"]
    assert out["requests"] == len(trace) - 1
    for st in out["outputs"].values():
        col, vis, ind = _alone(st)
        assert torch.equal(col, st.color) and torch.equal(vis, st.vis) and torch.equal(ind, st.ind)
