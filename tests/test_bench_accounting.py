"""Byte accounting of the benchmark's roofline (CPU): the survey's per-unit figures, the
kernels' layout figures and the BVH-independent floor, on hand-counted traversals."""
import pytest

import bench


def test_survey_layout_and_floor_bytes_per_unit():
    alloc = (16, 8, 8)   # 32 rays per pixel, 8 of them environment samples
    io = (48 + 28) / 32 + 4 * 8 / 32   # G-buffer in and pixel out per ray, env-table reads
    assert io == pytest.approx(3.375)
    one = {"node": (1, 0, 0), "test": (0, 1, 0), "hit": (0, 0, 1)}
    assert bench.alg_bytes(one["node"], 1, alloc) == pytest.approx(64 + io)
    assert bench.alg_bytes(one["test"], 1, alloc) == pytest.approx(48 + io)
    assert bench.alg_bytes(one["hit"], 1, alloc) == pytest.approx(192 + io)
    assert bench.layout_bytes(one["node"], 1) == pytest.approx(112 + 44)
    assert bench.layout_bytes(one["test"], 1) == pytest.approx(64 + 44)
    # the floor counts a record and the colour of each composited hit, no nodes, no misses
    assert bench.floor_bytes(one["node"], 1, alloc) == pytest.approx(io)
    assert bench.floor_bytes(one["test"], 1, alloc) == pytest.approx(io)
    assert bench.floor_bytes(one["hit"], 1, alloc) == pytest.approx(48 + 192 + io)


def test_floor_is_below_the_survey_count_and_reported_beside_it():
    alloc, R = (16, 8, 8), 1000
    cnt = (26.6 * R, 14.5 * R, 5.4 * R)   # every composited hit was tested: tests >= hits
    a, f = bench.alg_bytes(cnt, R, alloc), bench.floor_bytes(cnt, R, alloc)
    assert f < a
    r = bench.roofline("k", a, bench.layout_bytes(cnt, R), 2.0, 6000.0, "measured", floor=f, rays=R)
    assert r["frac"] == pytest.approx(a / 2e-3 / 1e9 / 6000.0)
    assert r["floor"]["bytes_per_ray"] == pytest.approx(f / R)
    assert r["floor"]["survey_over_floor"] == pytest.approx(a / f)
    assert r["floor"]["ms_at_peak"] == pytest.approx(f / 6000e9 * 1e3)
    assert "floor" not in bench.roofline("k", a, a, 2.0, 6000.0, "measured")


def test_clock_sampler_decodes_nvml_samples():
    """The sampler's host logic on a fake NVML reader: reasons decoded from the clock-event
    bits, the clock the median of the samples, the reader closed at the end."""
    import time
    import types

    seq = iter([(1980.0, 0x0), (2032.0, 0x4), (2032.0, 0x4 | 0x40)] + [(2032.0, 0x0)] * 1000)
    cur = {}

    def sm():
        cur["s"] = next(seq)
        return cur["s"][0]

    closed = []
    fake = types.SimpleNamespace(sm_mhz=sm, max_sm_mhz=lambda: 2032.0, power_w=lambda: 900.0,
                                 reasons=lambda: cur["s"][1], close=lambda: closed.append(1))
    c = bench.ClockSampler(0, reader=fake)
    c.start()
    time.sleep(0.08)
    r = c.stop()
    assert r["samples"] >= 3 and r["source"].startswith("nvml") and closed == [1]
    assert r["sm_mhz"] == 2032.0 and r["sm_max_mhz"] == 2032.0 and r["power_w_median"] == 900.0
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
