"""Benchmark of the 2DGRT secondary-ray hot path on synthetic workloads.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl grt|reference]
                    [--mode shade|train|serve|large|relight] [--no-cpu-baseline]

Default workload (mode "shade"): 300,000 SH surfels on 3 spheres, 2 tori, a box and a
ground plane; an 800x800 G-buffer; 32 secondary rays per pixel by MIS (16 cosine / 8 GGX /
8 environment) under a 512x256 log-normal HDR map with a sun; metallic GGX BRDF.  One
step = in-place LBVH rebuild + traced primary G-buffer + fused sample/trace/shade of every
pixel.  The metric is secondary rays per second (valid pixels x 32 / step time).

Mode "train": 400x400, 16 rays/pixel (8/4/4) on the same scene, forward + adjoint of an
L2 loss against a seeded target (shade_pixels + shade_backward).
Mode "large": 2M surfels (ground plane, 50 primitives, background shell), 1920x1080,
16 rays/pixel (8/4/4), forward and forward + backward with recomputed hit lists.
Mode "serve": the relight request loop (see paper_2607_22780_b300.serve).
Mode "relight": split-sum relighting of the default frame (Eq. 14-15), Gaussian backend and
mesh backend (the same objects as 310,670 triangles).
Mode "c1": the plain forward (8k RGB surfels, 64x64, 4 cosine rays, constant white map).
Mode "cpu": the FP64 oracle timed on the host cores for C1 (whole frame), C2 and C4
(4,096-ray samples) and the C3 backward at 32x32.

Under torchrun every rank renders its own frame (weak scaling, no data-path collective);
ranks meet only at the barriers around the timed region and in the final max/sum.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SEED = 2607
N_SURFELS = 300_000
W_IMG = H_IMG = 800
ALLOC = (16, 8, 8)
ENV_W, ENV_H = 512, 256
TRAIN_IMG = 400
TRAIN_ALLOC = (8, 4, 4)
# Algorithmic bytes per ray of the trace (the survey's count, which the roofline fraction
# uses): 64 per internal node visited, 48 per surfel record tested, 192 per composited SH
# hit, plus the shading call's ray I/O (48 B of G-buffer in and 28 B out per pixel over the
# N_r rays of the pixel, ~4 B of environment-table reads per environment sample).
ALG_NODE_BYTES = 64
ALG_REC_BYTES = 48
# Bytes the kernels' own layouts move (second field of each roofline): a 4-wide node visit
# loads 6 child-plane float4 + 1 child-ref float4, a record is 64 B, a ray reads its
# direction (16) and origin (12) and writes (c_rt, T) (16).
REC_BYTES = 64      # packed surfel record read per surfel test
NODE_BYTES = 112    # 4-wide node visit: 6 child-plane float4 + 1 child-ref float4
SH_BYTES = 192      # 48 SH coefficients read per composited hit
HIT_REC_BYTES = 12  # recorded hit (surfel id, tau, alpha), written by the saving trace, read by the replay
SURFEL_BYTES = 232  # mu 12 + quat 16 + scale 8 + opacity 4 + SH 192, read per replayed hit
GRAD_RMW_BYTES = 464  # the same 232 B of gradients read and written (atomics) per replayed hit
REPLAY_RAY_BYTES = 64  # per traced ray in the replay: hit count 4, direction 16, origin 12, (c_rt, T) 16, adjoint 16
RAY_IO_BYTES = 44   # direction 16 + origin 12 read, (c_rt, T) 16 written
COLLAPSE_LAUNCHES = 2  # the collapse's cost pass (bottom-up) and the 4-wide collapse (a thread per binary node)
# dram__bytes_read.sum + dram__bytes_write.sum of one k_trace_rays_ww launch of the default
# workload (k = 16, 800x800) from one ncu capture of the current kernel; None until taken
TRACE_DRAM_BYTES = 1_187_873_280  # 847.4 MB read + 340.5 MB written
# L2 traffic of the same kernel (lts__t_bytes.sum) per ray and the L2 throughput fraction,
# from one ncu capture of the 256x256 case of the same step (1,031,680 rays: 4.23 GB in one
# launch); None until taken for the current kernel
TRACE_L2 = {"lts_bytes_per_ray": 4_228_348_672 / 1_031_680, "lts_throughput_pct_of_peak": 16.22,
            "lts_sector_hit_pct": 93.51, "case": "256x256, 300k surfels, 32 rays/pixel (one ncu capture)"}
LARGE_N = 2_000_000          # unbounded scene: ground plane, 50 primitives, r = 50 shell
LARGE_W, LARGE_H = 1920, 1080
LARGE_ALLOC = (8, 4, 4)
LARGE_DISTANCE = 12.0


def alg_bytes(cnt, R, alloc, extra_per_hit=0.0, extra_per_ray=0.0):
    """Algorithmic bytes of one trace launch over R rays from its traversal counters
    (nodes, tests, composited), by the survey's count."""
    nr = float(sum(alloc))
    io = (48.0 + 28.0) / nr + 4.0 * alloc[2] / nr
    return (ALG_NODE_BYTES * cnt[0] + ALG_REC_BYTES * cnt[1] + (SH_BYTES + extra_per_hit) * cnt[2] +
            (io + extra_per_ray) * R)


def floor_bytes(cnt, R, alloc):
    """The survey's BVH-independent floor of the same launch: a 48-byte record and the
    colour of every composited hit plus the ray I/O, with no node or missed-record bytes.
    The composited counts are the counting pass's, which equal the oracle's on every
    unflagged ray (the hit lists are bit-exact)."""
    nr = float(sum(alloc))
    io = (48.0 + 28.0) / nr + 4.0 * alloc[2] / nr
    return (ALG_REC_BYTES + SH_BYTES) * cnt[2] + io * R


def layout_bytes(cnt, R, extra_per_hit=0.0, extra_per_ray=0.0):
    """Bytes the kernel's own node and record layout loads for the same traversal."""
    return (NODE_BYTES * cnt[0] + REC_BYTES * cnt[1] + (SH_BYTES + extra_per_hit) * cnt[2] +
            (RAY_IO_BYTES + extra_per_ray) * R)


def roofline(kernel, nbytes, lbytes, t_ms, peak, peak_kind, floor=None, rays=None, **extra):
    ach = nbytes / (t_ms * 1e-3) / 1e9
    lach = lbytes / (t_ms * 1e-3) / 1e9
    out = {"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "frac_of_8tbs": ach / 8000.0, "peak_kind": peak_kind, "alg_bytes_per_launch": nbytes, "kernel_ms": t_ms,
           "bytes": "survey count: 64 per node visit + 48 per record test + 192 per SH hit + ray I/O",
           "layout": {"bytes_per_launch": lbytes, "achieved": lach, "frac": lach / peak,
                      "bytes": "kernel layout: 112 per 4-wide node visit + 64 per record + 192 per SH hit + 44 per ray"}}
    if floor is not None:
        out["floor"] = {"bytes_per_launch": floor, "bytes_per_ray": floor / rays, "survey_over_floor": nbytes / floor,
                        "ms_at_peak": floor / (peak * 1e9) * 1e3,
                        "bytes": "BVH-independent floor: (48 + 192) per composited hit + ray I/O"}
    out.update(extra)
    return out


def l2_summary(R, t_ms):
    """L2 traffic of the trace launch: the captured bytes per ray scaled to this launch's
    rays, over its event-timed duration."""
    if TRACE_L2 is None:
        return None
    b = TRACE_L2["lts_bytes_per_ray"] * R
    return dict(TRACE_L2, bytes_per_launch=b, achieved_GBps=b / (t_ms * 1e-3) / 1e9)


def reduce_ranks(ms: float, rays: float, device) -> tuple:
    """Weak scaling across ranks: (max step time over ranks, rays summed over ranks)."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms, float(rays)], device=device, dtype=torch.float64)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = tt.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class _Nvml:
    """Read-only NVML queries (SM clock, its maximum, power, clock-event reasons) through the
    driver's libnvidia-ml by ctypes, on the device whose UUID torch reports for `dev`."""

    def __init__(self, dev: int):
        import ctypes
        import torch
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        self._ok(self.lib.nvmlInit_v2())
        uuid = ("GPU-" + str(torch.cuda.get_device_properties(dev).uuid)).encode()
        self.h = ctypes.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(uuid), ctypes.byref(self.h)))
        self.reasons_fn = (getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
                           or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons)

    @staticmethod
    def _ok(rc):
        if rc != 0:
            raise RuntimeError(f"NVML error {rc}")

    def _uint(self, fn, *args):
        v = self.c.c_uint()
        self._ok(fn(self.h, *args, self.c.byref(v)))
        return v.value

    def sm_mhz(self):
        return float(self._uint(self.lib.nvmlDeviceGetClockInfo, 1))   # NVML_CLOCK_SM

    def max_sm_mhz(self):
        return float(self._uint(self.lib.nvmlDeviceGetMaxClockInfo, 1))

    def power_w(self):
        return self._uint(self.lib.nvmlDeviceGetPowerUsage) / 1000.0   # milliwatts

    def reasons(self):
        v = self.c.c_ulonglong()
        self._ok(self.reasons_fn(self.h, self.c.byref(v)))
        return int(v.value)

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """SM clock, power and throttle reasons sampled during the timed region.

    NVML is read from a thread every 10 ms, so a region of a few hundred milliseconds still
    gets tens of samples; start() returns once the first sample is in.  Without NVML it falls
    back to `nvidia-smi -lms 100`, which starts slowly and samples a short region once or
    twice."""

    # clock-event reason bits of NVML
    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int, reader=None):
        self.dev = dev
        self.reader = reader
        self.proc = None
        self.thread = None
        self.samples = []
        self.path = os.path.join("/tmp", f"grt_clocks_{os.getpid()}.csv")

    def _poll(self, nv, mx):
        while not self.done.is_set():
            try:
                self.samples.append((nv.sm_mhz(), mx, nv.power_w(), nv.reasons()))
            except Exception:
                pass
            self.first.set()
            self.done.wait(0.01)

    def start(self):
        import threading
        try:
            nv = self.reader if self.reader is not None else _Nvml(self.dev)
            self.reader = nv
            mx = nv.max_sm_mhz()
            nv.sm_mhz(), nv.reasons(), nv.power_w()   # a failing query falls back to nvidia-smi here
            self.done, self.first = threading.Event(), threading.Event()
            self.thread = threading.Thread(target=self._poll, args=(nv, mx), daemon=True)
            self.thread.start()
            self.first.wait(2.0)
            return
        except Exception:
            self.thread = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.done.set()
            self.thread.join(timeout=5)
            try:
                self.reader.close()
            except Exception:
                pass
            sm = [x[0] for x in self.samples]
            mx = [x[1] for x in self.samples]
            reasons = {nm for nm, bit in self.REASONS for x in self.samples if x[3] & bit}
            return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                    "reasons": sorted(reasons), "samples": len(sm), "source": "nvml, 10 ms",
                    "power_w_median": float(np.median([x[2] for x in self.samples])) if sm else None}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for (nm, _), v in zip(self.REASONS, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 100 ms"}


# ----------------------------------------------------------------------------- workload

def make_inputs(rank: int):
    from paper_2607_22780_b300 import workloads as wl
    sc = wl.scene_objects(N_SURFELS, seed=SEED)
    cam = wl.camera_orbit(SEED + rank, W_IMG, H_IMG, 3.0)
    env = wl.envmap_hdr(SEED + rank, ENV_W, ENV_H)
    return sc, cam, env


def oracle_view_gbuffer(sc, cam, size=80):
    """The oracle's own G-buffer of a size x size view from the benchmark camera (the
    oracle's timed samples shade pixels of this view: no input comes from the GPU)."""
    import oracle
    from paper_2607_22780_b300 import workloads as wl
    small = wl.Camera(cam.eye, cam.target, cam.up, cam.tan_half_fovy, size, size)
    return oracle.gbuffer_f32(oracle.gbuffer(sc, small))


def cpu_oracle_sample(sc, env, gb32, budget_s=12.0):
    """Time the FP64 oracle on a bounded pixel sample of the same scene, map and camera."""
    import oracle
    valid = np.nonzero(gb32["valid"])[0]
    rng = np.random.default_rng(0)
    Nr = sum(ALLOC)

    def timed(n):
        pix = rng.choice(valid, size=min(n, len(valid)), replace=False).astype(np.int32)
        t0 = time.perf_counter()
        oracle.shade_pixels(sc, gb32, env, *ALLOC, seed=SEED, pixels=pix)
        return len(pix), time.perf_counter() - t0

    _, t_a = timed(4)
    _, t_b = timed(20)
    per_px = max((t_b - t_a) / 16, 1e-6)  # the difference removes the per-call setup
    n, dt = timed(int(max(4, budget_s / per_px)))
    return {"value": n * Nr / dt, "unit": "rays/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} random valid pixels x {Nr} MIS rays of an 80x80 view from the benchmark camera, "
                      f"300k surfels, FP64 brute force (every ray against every surfel), {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sc, cam, env = make_inputs(0)
    t0 = time.perf_counter()
    gb = oracle_view_gbuffer(sc, cam)
    t_gb = time.perf_counter() - t0
    steps, walls = [], []
    cb = None
    for s in range(args.warmup + args.steps):
        ts = time.perf_counter()
        cb = cpu_oracle_sample(sc, env, gb, budget_s=max(2.0, 60.0 / (args.steps + args.warmup)))
        if s >= args.warmup:
            steps.append(cb["value"])
            walls.append((time.perf_counter() - ts) * 1e3)
    value = float(np.median(steps))
    cb["value"] = value
    # a step is one bounded sample of the workload (see config.sample), not the whole frame
    out = {"impl": "reference", "metric": "secondary_rays_per_s", "value": value, "unit": "rays/s",
           "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.median(walls)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"mis_shade_300k_{W_IMG}x{H_IMG}_32spp", "surfels": N_SURFELS, "image": [W_IMG, H_IMG],
                      "rays_per_pixel": sum(ALLOC), "alloc_cos_ggx_env": list(ALLOC), "env": [ENV_W, ENV_H],
                      "k": 16, "sample": "each step shades a bounded random sample of valid pixels of an 80x80 "
                                         "view from the same camera (same scene, map and seeds)"},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "note": f"G-buffer of the sampled view took {t_gb:.1f} s"}
    print(json.dumps(out), flush=True)


def run_grt(args):
    import torch
    import torch.distributed as dist

    from paper_2607_22780_b300 import api, build as gbuild

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(gbuild.OUT):
        raise RuntimeError("libgrt.so is missing: run __graft_entry__.build() first")

    sc, cam, env = make_inputs(rank)
    # ---- device-resident inputs
    S = api.Scene.from_workload(sc, device=dev, params=api.trace_params(k=args.k))
    E = api.Environment(torch.from_numpy(env).to(dev))
    G = api.GBuffer.empty(W_IMG, H_IMG, cam.eye, device=dev)
    P = W_IMG * H_IMG
    outs = (torch.empty((P, 3), device=dev), torch.empty((P,), device=dev), torch.empty((P, 3), device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 126 MB L2
    stream = torch.cuda.current_stream()

    def step():
        S.rebuild()
        api.gbuffer_primary(S, cam, out=G)
        api.shade_pixels(S, G, E, *ALLOC, seed=SEED, outputs=outs)

    step()
    torch.cuda.synchronize()
    n_valid = int(G.valid.sum().item())
    R = n_valid * sum(ALLOC)
    # kernel launches per step: prep + Morton, 4 x (histogram, scan, scatter), hierarchy + records + refit, one per
    # treelet-restructuring pass, collapse (cost pass + collapse), G-buffer, then sample + bucket scan (tile
    # sums, their scan, tile scans) + ray scatter + trace + accumulate
    launches_per_step = 2 + 12 + 3 + int(S.params.build_passes) + COLLAPSE_LAUNCHES + 1 + 7

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: per-step events, L2 flushed between steps (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases = []
    api.phase_timing(True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        S.rebuild()
        api.gbuffer_primary(S, cam, out=G)
        kev[i][0].record(stream)
        api.shade_pixels(S, G, E, *ALLOC, seed=SEED, outputs=outs)
        kev[i][1].record(stream)
        ev[i][1].record(stream)
        phases.append(api.phase_timing(read=True))
    torch.cuda.synchronize()
    api.phase_timing(False)
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    shade_ms = [a.elapsed_time(b) for a, b in kev]
    ms = float(np.mean(step_ms))
    t_max = ms
    rays_total = R
    if world > 1:
        t_max, rays_total = reduce_ranks(ms, R, dev)
    value = rays_total / (t_max * 1e-3)

    # ---- algorithmic bytes of the dominant kernel (the persistent trace kernel), from the
    # traversal counters of the same rays (counting pass outside the timed region)
    cnt = api.shade_count(S, G, E, *ALLOC, seed=SEED).cpu().numpy().astype(np.float64)
    ph = np.array(phases)
    trace_s = float(np.mean(ph[:, 1])) * 1e-3
    shade_s = float(np.mean(shade_ms)) * 1e-3
    peak, peak_kind = measured_peaks()

    # ---- end to end through the public API with host buffers
    # Every step uploads its scene and map from pinned host memory and downloads its image.
    # Two slots of device inputs and outputs alternate so that, on a copy stream, step i+1's
    # upload and step i's download overlap step i's compute (a serving pipeline); the timed
    # region holds all K uploads and downloads.
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        host = {k: pin(v) for k, v in sc.arrays().items()}
        henv = pin(env)
        copy_s = torch.cuda.Stream(device=dev)

        def make_slot():
            d_in = {k: v.to(dev) for k, v in host.items()}
            d_env = henv.to(dev)
            # contiguous pinned destinations: a strided host destination makes torch stage
            # the copy through pageable memory
            return dict(inp=d_in, env=d_env, S=api.Scene(**d_in), E=api.Environment(d_env),
                        G=api.GBuffer.empty(W_IMG, H_IMG, cam.eye, device=dev),
                        out=(torch.empty((P, 3), device=dev), torch.empty((P,), device=dev),
                             torch.empty((P, 3), device=dev)),
                        hout=[torch.empty(sh, dtype=torch.float32).pin_memory() for sh in ((P, 3), (P,), (P, 3))],
                        up=torch.cuda.Event(), done=torch.cuda.Event())

        slots = [make_slot(), make_slot()]
        h2d = sum(v.numel() * 4 for v in host.values()) + henv.numel() * 4
        d2h = sum(h.numel() * 4 for h in slots[0]["hout"])
        torch.cuda.synchronize()

        def upload(sl):
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(sl["done"])  # the slot's previous step has finished with it
                for k in host:
                    sl["inp"][k].copy_(host[k], non_blocking=True)
                sl["env"].copy_(henv, non_blocking=True)
                sl["up"].record(copy_s)

        def run_steps(n):
            for sl in slots:
                sl["done"].record(stream)
            upload(slots[0])
            for i in range(n):
                c = slots[i % 2]
                stream.wait_event(c["up"])
                c["S"].rebuild()
                c["E"].update(c["env"])
                api.gbuffer_primary(c["S"], cam, out=c["G"])
                api.shade_pixels(c["S"], c["G"], c["E"], *ALLOC, seed=SEED, outputs=c["out"])
                c["done"].record(stream)
                if i + 1 < n:
                    upload(slots[(i + 1) % 2])
                with torch.cuda.stream(copy_s):
                    copy_s.wait_event(c["done"])
                    for h, d in zip(c["hout"], c["out"]):
                        h.copy_(d, non_blocking=True)
            stream.wait_stream(copy_s)

        run_steps(3)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_steps(args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = a.elapsed_time(b) / args.steps
        e2e = {"value": R / (e_ms * 1e-3), "unit": "rays/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e_ms,
               "pipeline": "two slots: step i+1's upload and step i's download overlap step i's compute"}

    # ---- fwd+bwd (training form) on the 400x400 / 16-ray configuration
    fb = None
    if not args.no_train:
        fb = time_train(api, S, cam, E, dev, args)
    large = None
    if rank == 0 and world == 1 and not args.no_large:
        large = time_large(api, dev, args)
    den = time_denoise(api, G, outs[0], args) if rank == 0 else None
    c1 = time_c1(api, dev, args) if rank == 0 and not args.no_c1 else None
    rel = time_relight(api, S, G, E, R, args) if rank == 0 and not args.no_relight else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(sc, env, oracle_view_gbuffer(sc, cam))

    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        serving = serve_summary(args)

    if rank == 0:
        out = {"metric": "secondary_rays_per_s", "value": value, "unit": "rays/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"mis_shade_300k_{W_IMG}x{H_IMG}_32spp", "surfels": N_SURFELS,
                          "image": [W_IMG, H_IMG], "rays_per_pixel": sum(ALLOC), "alloc_cos_ggx_env": list(ALLOC),
                          "env": [ENV_W, ENV_H], "valid_pixels": n_valid, "rays_per_step": R,
                          "step": "rebuild LBVH + primary G-buffer + MIS shade", "k": args.k,
                          "l2": "flushed between steps (256 MB write outside the timed events)",
                          "parallelism": f"replicas x{world}"},
               "gpu_launches": launches_per_step * args.steps,
               "roofline": roofline(
                   "k_trace_rays_ww", alg_bytes(cnt, R, ALLOC), layout_bytes(cnt, R), trace_s * 1e3, peak, peak_kind,
                   floor=floor_bytes(cnt, R, ALLOC), rays=R,
                   traffic=TRACE_DRAM_BYTES if (args.k == 16 and W_IMG == 800) else None,
                   l2=l2_summary(R, trace_s * 1e3) if args.k == 16 else None,
                   phase_ms={"sample": float(np.mean(ph[:, 0])), "trace": float(np.mean(ph[:, 1])),
                             "accumulate": float(np.mean(ph[:, 2])), "shade_call": shade_s * 1e3},
                   per_ray={"nodes": cnt[0] / R, "tests": cnt[1] / R, "composited": cnt[2] / R}),
               "clocks": clk, "e2e": e2e, "fwd_bwd": fb, "large": large, "c1": c1, "denoise": den, "relight": rel, "cpu_baseline": cpu, "serving": serving,
               "wall_s_timed": t_wall}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def serve_summary(args):
    """Relight serving on the three resident scenes (300k, 1M, 2M surfels): a Poisson trace at
    200 requests/s and one at 80% of the batched arm's capacity, each served with continuous
    batching and one request at a time; p50/p99 latency and rays/s.  The default line runs a
    shortened trace (30 warm-up + 100 measured requests each); --mode serve runs the full one
    (100 + 2,000)."""
    from paper_2607_22780_b300 import serve
    return serve.serve_benchmark(n_warm=30, n_meas=100, n_warm80=10, n_meas80=60)


def run_train_only(args):
    """Forward + adjoint of the training configuration only (profiling entry)."""
    import torch
    from paper_2607_22780_b300 import api
    torch.cuda.set_device(0)
    sc, cam, env = make_inputs(0)
    S = api.Scene.from_workload(sc, params=api.trace_params(k=args.k))
    E = api.Environment(torch.from_numpy(env).cuda())
    print(json.dumps(time_train(api, S, cam, E, torch.device("cuda"), args)), flush=True)


def run_relight_only(args):
    """Relighting of the shading frame only, Gaussian and mesh backends (profiling entry)."""
    import torch
    from paper_2607_22780_b300 import api
    torch.cuda.set_device(0)
    sc, cam, env = make_inputs(0)
    S = api.Scene.from_workload(sc, params=api.trace_params(k=args.k))
    E = api.Environment(torch.from_numpy(env).cuda())
    G = api.gbuffer_primary(S, cam)
    R = int(G.valid.sum().item()) * sum(ALLOC)
    print(json.dumps(time_relight(api, S, G, E, R, args)), flush=True)


def time_train(api, S, cam, E, dev, args):
    import torch
    from paper_2607_22780_b300 import workloads as wl
    img = args.image or TRAIN_IMG if args.mode == "train" else TRAIN_IMG
    c = wl.Camera(cam.eye, cam.target, cam.up, cam.tan_half_fovy, img, img)
    G = api.gbuffer_primary(S, c)
    tgt = torch.from_numpy(wl.target_image(SEED, img, img).reshape(-1, 3)).to(dev)
    grads = api.SurfelGrads.zeros(S)

    valid = G.valid.unsqueeze(1).float()

    def zero():
        for t_ in (grads.mu, grads.quat, grads.scale, grads.opacity, grads.color):
            t_.zero_()

    def step_stored():
        # forward keeps each ray's first 64 hits, the backward replays them
        col, vis, ind, saved = api.shade_pixels_save(S, G, E, *TRAIN_ALLOC, seed=SEED, max_hits=64)
        dl = (col - tgt) * valid
        zero()
        api.shade_backward(S, G, E, *TRAIN_ALLOC, SEED, dl.contiguous(), grads=grads, saved=saved)

    def step_recompute():
        # no per-ray state between the passes: the backward samples and traces again
        col, vis, ind = api.shade_pixels(S, G, E, *TRAIN_ALLOC, seed=SEED)
        dl = (col - tgt) * valid
        zero()
        api.shade_backward(S, G, E, *TRAIN_ALLOC, SEED, dl.contiguous(), grads=grads)

    def fwd():
        api.shade_pixels(S, G, E, *TRAIN_ALLOC, seed=SEED)

    mg = api.MaterialGrads(torch.zeros((E.H, E.W, 3), device=dev), torch.zeros((img * img, 3), device=dev),
                           torch.zeros(img * img, device=dev), torch.zeros(img * img, device=dev))

    def step_material():
        # forward with the mean incident radiance of Eq. 16, then the adjoint into the map
        # and the per-pixel materials (L1-style upstream gradients)
        col, vis, ind, light = api.shade_pixels(S, G, E, *TRAIN_ALLOC, seed=SEED, light=True)
        dl = (torch.sign(col - tgt) * valid).contiguous()
        dlight = (torch.sign(light - light.mean(1, keepdim=True)) * valid).contiguous()
        for t_ in (mg.env, mg.albedo, mg.rough, mg.metal):
            t_.zero_()
        api.shade_backward_material(S, G, E, *TRAIN_ALLOC, SEED, dl, dlight, grads=mg)

    n = max(1, args.steps)
    ms = {}
    for name, fn in (("fwd_bwd", step_stored), ("fwd_bwd_recompute", step_recompute), ("fwd", fwd),
                     ("fwd_bwd_material", step_material)):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        ms[name] = a.elapsed_time(b) / n
    nv = int(G.valid.sum().item())
    R = nv * sum(TRAIN_ALLOC)
    # rooflines of the stored form's two dominant kernels, event-timed inside the library on
    # the call's stream: the saving trace (forward walk + hit record) and the replay
    cnt = [int(x) for x in api.shade_count(S, G, E, *TRAIN_ALLOC, seed=SEED).cpu()]
    api.phase_timing(True)
    api.adjoint_timing(True)
    tr, rp = [], []
    for _ in range(3):
        step_stored()
        tr.append(api.phase_timing(read=True)[1])
        rp.append(api.adjoint_timing(read=True)[1])
    api.phase_timing(False)
    api.adjoint_timing(False)
    peak, peak_kind = measured_peaks()
    replay_bytes = (HIT_REC_BYTES + SURFEL_BYTES + GRAD_RMW_BYTES) * cnt[2] + REPLAY_RAY_BYTES * R

    tr_ms, rp_ms = float(np.median(tr)), float(np.median(rp))
    replay = roofline("k_adjoint_replay", replay_bytes, replay_bytes, rp_ms, peak, peak_kind)
    replay["bytes"] = replay["layout"]["bytes"] = "(12 + 232 + 464) per composited hit + 64 per ray"
    save = roofline("k_trace_rays_save", alg_bytes(cnt, R, TRAIN_ALLOC, HIT_REC_BYTES, 4),
                    layout_bytes(cnt, R, HIT_REC_BYTES, 4), tr_ms, peak, peak_kind)
    return {"workload": f"train_300k_{img}x{img}_16spp", "rays": R, "fwd_ms": ms["fwd"], "fwd_bwd_ms": ms["fwd_bwd"],
            "fwd_bwd_recompute_ms": ms["fwd_bwd_recompute"], "stored_hits": 64,
            "fwd_bwd_material_ms": ms["fwd_bwd_material"],
            "fwd_rays_per_s": R / (ms["fwd"] * 1e-3), "fwd_bwd_rays_per_s": R / (ms["fwd_bwd"] * 1e-3),
            "fwd_bwd_recompute_rays_per_s": R / (ms["fwd_bwd_recompute"] * 1e-3),
            "per_ray": {"nodes": cnt[0] / R, "tests": cnt[1] / R, "composited": cnt[2] / R},
            "roofline_save_trace": save, "roofline_replay": replay}


def time_relight(api, S, G, E, R, args):
    """Split-sum relighting (Eq. 15) of the benchmark frame under its map: prefiltering of
    the map, then the MIS estimate with Trace_attr (Eq. 14) for every secondary ray."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        E.prefilter()
    a.record()
    E.prefilter()
    b.record()
    torch.cuda.synchronize()
    pre_ms = a.elapsed_time(b)
    outs = api.shade_relight(S, G, E, *ALLOC, seed=SEED)
    for _ in range(3):
        api.shade_relight(S, G, E, *ALLOC, seed=SEED, outputs=outs)
    torch.cuda.synchronize()
    n = 5
    a.record()
    for _ in range(n):
        api.shade_relight(S, G, E, *ALLOC, seed=SEED, outputs=outs)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    api.phase_timing(True)
    tr = []
    for _ in range(3):
        api.shade_relight(S, G, E, *ALLOC, seed=SEED, outputs=outs)
        tr.append(api.phase_timing(read=True)[1])
    api.phase_timing(False)
    mesh = time_relight_mesh(api, G, E, R)
    return {"workload": "relight_300k_800x800_32spp", "prefilter_ms": pre_ms, "ms": ms, "trace_ms": float(np.median(tr)),
            "rays": R, "rays_per_s": R / (ms * 1e-3), "mesh": mesh}


def time_relight_mesh(api, G, E, R):
    """The same relighting with the mesh backend of Eq. 14: the analytic objects of the
    benchmark scene as 310,670 triangles (per-vertex materials), closest hit per ray."""
    import torch
    from paper_2607_22780_b300 import workloads as wl
    m = wl.mesh_objects(SEED, res=96)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    M = api.MeshScene.from_workload(m)
    torch.cuda.synchronize()
    a.record()
    M2 = api.MeshScene.from_workload(m)
    b.record()
    torch.cuda.synchronize()
    build_ms = a.elapsed_time(b)
    M2.close()
    outs = api.shade_relight_mesh(M, G, E, *ALLOC, seed=SEED)
    for _ in range(3):
        api.shade_relight_mesh(M, G, E, *ALLOC, seed=SEED, outputs=outs)
    torch.cuda.synchronize()
    n = 5
    a.record()
    for _ in range(n):
        api.shade_relight_mesh(M, G, E, *ALLOC, seed=SEED, outputs=outs)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    api.phase_timing(True)
    tr = []
    for _ in range(3):
        api.shade_relight_mesh(M, G, E, *ALLOC, seed=SEED, outputs=outs)
        tr.append(api.phase_timing(read=True)[1])
    api.phase_timing(False)
    st = M.status()
    M.close()
    return {"triangles": int(len(m.tri)), "build_ms_incl_upload": build_ms, "ms": ms, "trace_ms": float(np.median(tr)),
            "rays_per_s": R / (ms * 1e-3), "status": st}


def time_c1(api, dev, args):
    """Plain forward of the sphere + plane scene: 8,000 RGB surfels, 64x64 G-buffer from the
    camera at distance 3 (60 degree fov), 4 cosine rays per pixel, Lambert, constant white
    map.  The frame is tiny and launch-bound: reported per frame (shading alone, G-buffer +
    shading, and with the LBVH rebuild) as well as in rays/s."""
    import torch
    from paper_2607_22780_b300 import workloads as wl
    sc = wl.scene_sphere_plane(8000, seed=SEED)
    cam = wl.camera_c1(64, 64)
    S = api.Scene.from_workload(sc, device=dev)
    E = api.Environment(torch.from_numpy(wl.envmap_constant(1.0)).to(dev))
    G = api.gbuffer_primary(S, cam)
    outs = (torch.empty((64 * 64, 3), device=dev), torch.empty((64 * 64,), device=dev),
            torch.empty((64 * 64, 3), device=dev))

    def shade():
        api.shade_pixels(S, G, E, 4, 0, 0, seed=SEED, brdf=0, outputs=outs)

    def frame():
        api.gbuffer_primary(S, cam, out=G)
        shade()

    def step():
        S.rebuild()
        frame()

    res = {}
    n = 200
    for name, fn in (("shade", shade), ("gbuffer_shade", frame), ("rebuild_gbuffer_shade", step)):
        for _ in range(10):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        res[name + "_us"] = a.elapsed_time(b) / n * 1e3
    # the same frame replayed from a CUDA graph: the device time without the host-side
    # launch overhead of the per-frame calls
    try:
        gstream = torch.cuda.Stream(device=dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gstream):
            frame()
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=gstream):
                frame()
        for _ in range(10):
            graph.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            graph.replay()
        b.record()
        torch.cuda.synchronize()
        res["gbuffer_shade_graph_us"] = a.elapsed_time(b) / n * 1e3
    except Exception as e:  # capture not possible here: reported, not fatal
        res["graph_error"] = repr(e)[:200]
    R = int(G.valid.sum().item()) * 4
    if "gbuffer_shade_graph_us" in res:
        res["rays_per_s_gbuffer_shade_graph"] = R / (res["gbuffer_shade_graph_us"] * 1e-6)
    return {"workload": "plain_8k_64x64_4cos", "surfels": 8000, "rays": R,
            "rays_per_s_shade": R / (res["shade_us"] * 1e-6),
            "rays_per_s_gbuffer_shade": R / (res["gbuffer_shade_us"] * 1e-6), **res, "frames_timed": n,
            "l2": "scene (1 MB) L2-resident; launch-bound"}


def run_cpu_baselines(args):
    """The FP64 oracle timed on this host's cores for every configuration the survey lists:
    the C1 frame whole, 4,096-ray samples of C2 and C4, the C3 backward at 32x32."""
    import platform
    import oracle
    from paper_2607_22780_b300 import workloads as wl
    cpu = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                cpu = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    out = {"metric": "oracle_rays_per_s", "cores": os.cpu_count(), "cpu": cpu, "host": platform.node()}

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    # C1: whole 64x64 frame, 4 cosine rays, constant white map, Lambert
    sc1 = wl.scene_sphere_plane(8000, seed=SEED)
    gb1 = oracle.gbuffer_f32(oracle.gbuffer(sc1, wl.camera_c1(64, 64)))
    dt = timed(lambda: oracle.shade_pixels(sc1, gb1, wl.envmap_constant(1.0), 4, 0, 0, seed=SEED, brdf=0))
    r1 = int(gb1["valid"].sum()) * 4
    out["c1"] = {"rays": r1, "s": dt, "rays_per_s": r1 / dt, "sample": "whole frame"}
    # C2: 128 valid pixels x 32 MIS rays = 4,096 rays of the 300k-surfel frame (80x80 view)
    sc2, cam2, env2 = make_inputs(0)
    gb2 = oracle_view_gbuffer(sc2, cam2)
    pix = np.random.default_rng(0).choice(np.nonzero(gb2["valid"])[0], 128, replace=False).astype(np.int32)
    dt = timed(lambda: oracle.shade_pixels(sc2, gb2, env2, *ALLOC, seed=SEED, pixels=pix))
    out["c2"] = {"rays": 4096, "s": dt, "rays_per_s": 4096 / dt,
                 "sample": "128 valid pixels x 32 rays of an 80x80 view from the benchmark camera",
                 "full_frame_s_extrapolated": dt / 4096 * 10_071_424}
    # C3: backward of the L2 loss at 32x32 (central crop of the 400x400 frame), 16 rays
    from paper_2607_22780_b300 import workloads as wl2
    c3 = wl2.Camera(cam2.eye, cam2.target, cam2.up, cam2.tan_half_fovy, 32, 32)
    gb3 = oracle.gbuffer_f32(oracle.gbuffer(sc2, c3))
    tgt = wl.target_image(SEED, 32, 32).reshape(-1, 3)
    fw = oracle.shade_pixels(sc2, gb3, env2, *TRAIN_ALLOC, seed=SEED)
    dl = (fw["color"] - tgt) * gb3["valid"][:, None]
    dt = timed(lambda: oracle.backward_pixels(sc2, gb3, env2, *TRAIN_ALLOC, SEED, dl))
    r3 = int(gb3["valid"].sum()) * sum(TRAIN_ALLOC)
    out["c3_backward"] = {"rays": r3, "s": dt, "rays_per_s": r3 / dt, "sample": "32x32 view, whole"}
    # C4: 256 valid pixels x 16 rays = 4,096 rays of the 2M-surfel scene (48x27 view)
    sc4 = wl.scene_large(LARGE_N, seed=SEED)
    gb4 = oracle.gbuffer_f32(oracle.gbuffer(sc4, wl.camera_orbit(SEED, 48, 27, LARGE_DISTANCE)))
    env4 = wl.envmap_hdr(SEED + 1, ENV_W, ENV_H)
    pix4 = np.random.default_rng(1).choice(np.nonzero(gb4["valid"])[0], 256, replace=False).astype(np.int32)
    dt = timed(lambda: oracle.shade_pixels(sc4, gb4, env4, *LARGE_ALLOC, seed=SEED, pixels=pix4))
    out["c4"] = {"rays": 4096, "s": dt, "rays_per_s": 4096 / dt,
                 "sample": "256 valid pixels x 16 rays of a 48x27 view from the benchmark camera"}
    print(json.dumps(out), flush=True)


def time_denoise(api, G, color, args):
    """Cross-bilateral denoiser (default window 7x7) over the shaded frame, guided by the
    G-buffer depth and normals."""
    import torch
    out = torch.empty_like(color)

    def run():
        api.denoise(color, G.depth, G.normal, G.valid, G.W, G.H, out=out)

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 20
    a.record()
    for _ in range(n):
        run()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    P = G.W * G.H
    return {"workload": f"denoise_{G.W}x{G.H}", "params": dict(api.DENOISE_DEFAULTS), "ms": ms,
            "pixels_per_s": P / (ms * 1e-3), "bytes_per_launch": P * 44,
            "achieved_GBps": P * 44 / (ms * 1e-3) / 1e9}


def time_large(api, dev, args):
    """2M-surfel unbounded scene, 1920x1080, 16 rays/pixel (8/4/4), k = 16: the forward
    (shade_pixels) and forward + backward (shade_pixels, L2 upstream gradient against the
    seeded target, shade_backward with recomputed hit lists) per frame.  The scene's
    records, tree and SH coefficients (~0.7 GB) exceed L2, so no flush is needed."""
    import torch
    from paper_2607_22780_b300 import workloads as wl
    W, H = (args.image, args.image * 9 // 16) if args.mode == "large" and args.image else (LARGE_W, LARGE_H)
    sc = wl.scene_large(LARGE_N, seed=SEED)
    cam = wl.camera_orbit(SEED, W, H, LARGE_DISTANCE)
    S = api.Scene.from_workload(sc, device=dev, params=api.trace_params(k=16))
    E = api.Environment(torch.from_numpy(wl.envmap_hdr(SEED + 1, ENV_W, ENV_H)).to(dev))
    G = api.gbuffer_primary(S, cam)
    tgt = torch.from_numpy(wl.target_image(SEED, H, W).reshape(-1, 3)).to(dev)
    valid = G.valid.unsqueeze(1).float()
    grads = api.SurfelGrads.zeros(S)
    P = W * H
    outs = (torch.empty((P, 3), device=dev), torch.empty((P,), device=dev), torch.empty((P, 3), device=dev))

    def fwd():
        api.shade_pixels(S, G, E, *LARGE_ALLOC, seed=SEED, outputs=outs)

    def fwd_bwd():
        fwd()
        dl = (outs[0] - tgt) * valid
        for t_ in (grads.mu, grads.quat, grads.scale, grads.opacity, grads.color):
            t_.zero_()
        api.shade_backward(S, G, E, *LARGE_ALLOC, SEED, dl.contiguous(), grads=grads)

    res = {}
    n = max(1, min(args.steps, 10))
    for name, fn in (("fwd", fwd), ("fwd_bwd", fwd_bwd)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(b) / n
    R = int(G.valid.sum().item()) * sum(LARGE_ALLOC)
    # roofline of the forward trace kernel: logical bytes from the traversal counters over
    # its event time inside the shading call
    api.phase_timing(True)
    tr = []
    for _ in range(3):
        fwd()
        tr.append(api.phase_timing(read=True)[1])
    api.phase_timing(False)
    cnt = api.shade_count(S, G, E, *LARGE_ALLOC, seed=SEED).cpu().numpy().astype(np.float64)
    trace_ms = float(np.median(tr))
    peak, peak_kind = measured_peaks()
    assert S.status() == 0
    return {"workload": f"large_2m_{W}x{H}_16spp", "surfels": LARGE_N, "rays": R, "k": 16,
            "fwd_ms": res["fwd"], "fwd_bwd_ms": res["fwd_bwd"],
            "fwd_rays_per_s": R / (res["fwd"] * 1e-3), "fwd_bwd_rays_per_s": R / (res["fwd_bwd"] * 1e-3),
            "trace_kernel_ms": trace_ms, "per_ray": {"nodes": cnt[0] / R, "tests": cnt[1] / R, "composited": cnt[2] / R},
            "roofline_trace": roofline("k_trace_rays_ww", alg_bytes(cnt, R, LARGE_ALLOC), layout_bytes(cnt, R),
                                       trace_ms, peak, peak_kind, floor=floor_bytes(cnt, R, LARGE_ALLOC), rays=R),
            "steps": n, "l2": "inputs larger than L2"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="grt", choices=["grt", "reference"])
    ap.add_argument("--mode", default="shade", choices=["shade", "serve", "train", "large", "relight", "c1", "cpu"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 2M-surfel 1080p forward/backward line")
    ap.add_argument("--no-relight", action="store_true", help="skip the relighting lines")
    ap.add_argument("--no-c1", action="store_true", help="skip the plain-forward 64x64 line")
    ap.add_argument("--k", type=int, default=16, help="k-buffer size (results do not depend on it)")
    ap.add_argument("--serve-requests", type=int, default=2000, help="measured requests of --mode serve")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--image", type=int, default=0,
                    help="square image size override (small profiling case); default 800")
    args = ap.parse_args()
    if args.image:
        global W_IMG, H_IMG
        W_IMG = H_IMG = args.image
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "serve":
        from paper_2607_22780_b300 import serve
        serve.bench_main(args)
    elif args.mode == "train":
        run_train_only(args)
    elif args.mode == "relight":
        run_relight_only(args)
    elif args.mode == "cpu":
        run_cpu_baselines(args)
    elif args.mode == "c1":
        import torch
        from paper_2607_22780_b300 import api
        torch.cuda.set_device(0)
        print(json.dumps(time_c1(api, torch.device("cuda"), args)), flush=True)
    elif args.mode == "large":
        import torch
        from paper_2607_22780_b300 import api
        torch.cuda.set_device(0)
        print(json.dumps(time_large(api, torch.device("cuda"), args)), flush=True)
    else:
        run_grt(args)


if __name__ == "__main__":
    main()
