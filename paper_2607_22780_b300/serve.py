"""Relight serving: resident scenes, continuous batching of shading requests.

Each request names a resident scene and carries a camera, an HDR environment map, a
resolution and a sample count (N_r/2 cosine, N_r/4 GGX, N_r/4 environment samples).
Serving a request = upload its map, build its proposal tables and traced G-buffer, then
shade every pixel with the MIS estimator against the scene's 2D Gaussian surfels.

Continuous batching (iteration-level scheduling): the loop runs "iterations"; each takes
pixel slices from the admitted requests in arrival order until a ray budget is filled and
shades them all in ONE grt_shade_batch launch.  Requests that arrive while launches are on
the GPU are admitted at the next iteration as long as their device memory fits the HBM
budget; their map upload, tables and G-buffer run on a separate stream and overlap the
shading of the others.  Launches alternate over two compute streams, so that one launch
starts while the previous one drains its last rays.  A request completes when every launch
holding one of its slices has ended (CUDA events on the GPU timeline); latency = completion -
arrival.

The comparator serves the same arrival trace one request at a time (each request's
G-buffer and a whole-image grt_shade_pixels launch, back to back).  Results are
bit-identical either way: a pixel's value depends only on its own samples.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Dict, List, Optional

import numpy as np
import torch

from . import api
from . import workloads as wl


@dataclasses.dataclass
class RelightRequest:
    rid: int
    arrival: float          # seconds after the start of the trace
    scene: str
    camera: wl.Camera
    env: object             # [H, W, 3] float32 HDR map (numpy array, or a pinned torch tensor)
    res: int
    rays: int               # N_r
    seed: int

    @property
    def alloc(self):
        return (self.rays // 2, self.rays // 4, self.rays - self.rays // 2 - self.rays // 4)


def env_pool(n: int, seed: int, env_size=(512, 256)) -> List[torch.Tensor]:
    """n distinct seeded log-normal HDR maps (the C2 recipe) for long request traces, in
    pinned host memory (pinned once, uploaded per request)."""
    return [torch.from_numpy(wl.envmap_hdr(seed + i, env_size[0], env_size[1])).pin_memory() for i in range(n)]


def make_trace(n: int, rate: float, scenes: Dict[str, float], seed: int, res_choices=(256, 512, 1024),
               rpp_choices=(8, 16, 32, 64), env_size=(512, 256), start: float = 0.0,
               envs: Optional[List[np.ndarray]] = None) -> List[RelightRequest]:
    """Poisson arrivals at `rate` per second; scenes maps name -> camera distance.  Each
    request draws its own map, or with `envs` takes one of those maps (request i uses
    envs[i % len(envs)]; it is still uploaded and prepared per request)."""
    rng = np.random.default_rng(seed)
    t = start
    names = sorted(scenes)
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        name = names[int(rng.integers(len(names)))]
        res = int(rng.choice(res_choices))
        rpp = int(rng.choice(rpp_choices))
        s = int(rng.integers(1 << 31))
        cam = wl.camera_orbit(s, res, res, scenes[name])
        env = envs[i % len(envs)] if envs else wl.envmap_hdr(s, env_size[0], env_size[1])
        out.append(RelightRequest(i, t, name, cam, env, res, rpp, s))
    return out


class _State:
    """Device-side state of an admitted request."""

    def __init__(self, req: RelightRequest, scene: api.Scene, dev, stream):
        self.req = req
        self.scene = scene
        P = req.res * req.res
        self.P = P
        with torch.cuda.stream(stream):
            if torch.is_tensor(req.env) and req.env.is_pinned():
                henv = req.env  # a pinned map of a pool, shared by several requests
            else:
                henv = torch.from_numpy(np.ascontiguousarray(req.env)).pin_memory()
            self.env_rgb = torch.empty(henv.shape, dtype=torch.float32, device=dev)
            self.env_rgb.copy_(henv, non_blocking=True)
            self.env = api.Environment(self.env_rgb, stream=stream)
            self.gb = api.gbuffer_primary(scene, req.camera, stream=stream)
            self.n_valid = self.gb.valid.sum()   # device scalar: the request's traced pixels
            self.color = torch.empty((P, 3), device=dev)
            self.vis = torch.empty((P,), device=dev)
            self.ind = torch.empty((P, 3), device=dev)
        self.ready = torch.cuda.Event()
        self.ready.record(stream)
        self._henv = henv
        self.next = 0
        self.done_ms: Optional[float] = None
        self.start_ms: Optional[float] = None
        self.evs: Dict[int, torch.cuda.Event] = {}   # compute stream -> end of its last launch with a slice
        self._streams = set()

    def tensors(self):
        """Every device tensor of the request (allocated on the prep stream)."""
        ts = [self.env_rgb, self.color, self.vis, self.ind, self.env.tables]
        ts += [t for t in (self.gb.pos, self.gb.normal, self.gb.albedo, self.gb.rough, self.gb.metal, self.gb.valid,
                           self.gb.alpha, self.gb.depth) if t is not None]
        return ts

    def release(self):
        """Drop the request's device buffers (statistics keep only the valid-pixel count)."""
        self.env_rgb = self.color = self.vis = self.ind = self.env = self.gb = None

    def use_on(self, stream):
        """Mark the request's tensors as used by `stream`: the caching allocator then keeps
        their blocks until the work queued there when they are freed has finished, so a
        request dropped while a launch still writes its outputs cannot hand those blocks to
        another request."""
        if stream.cuda_stream not in self._streams:
            for t in self.tensors():
                t.record_stream(stream)
            self._streams.add(stream.cuda_stream)

    def launches_done(self) -> bool:
        return all(e.query() for e in self.evs.values())

    def wait_launches(self):
        for e in self.evs.values():
            e.synchronize()

    @staticmethod
    def bytes_needed(req: RelightRequest) -> int:
        P = req.res * req.res
        H, W = req.env.shape[:2]
        return P * (56 + 28) + W * H * (12 + 16 + 4) + H * 4 + 4096


class RelightServer:
    """Resident scenes + continuous batching of relight requests on one GPU."""

    def __init__(self, scenes: Dict[str, api.Scene], device="cuda", hbm_budget: int = 8 << 30,
                 ray_budget: int = 8 << 20, max_batch: int = 16, inflight: int = 2, streams: int = 2,
                 order: str = "fifo", whole_when_alone: bool = True):
        if order not in ("fifo", "srpt"):
            raise ValueError(f"order must be 'fifo' or 'srpt', got {order!r}")
        self.order = order    # slices oldest request first, or least remaining work first
        self.whole_when_alone = bool(whole_when_alone)
        self.scenes = scenes
        self.device = torch.device(device)
        self.hbm_budget = int(hbm_budget)
        self.ray_budget = int(ray_budget)
        self.max_batch = int(max_batch)
        self.inflight = int(inflight)
        self.streams = max(1, int(streams))
        self.cancelled = set()
        self.peak_active = 0
        self.peak_mem = 0
        self.skip = 0   # statistics leave out requests with rid < skip (warm-up)

    def cancel(self, rid: int):
        """Drop a request: pending requests are skipped, admitted ones stop getting slices."""
        self.cancelled.add(rid)

    # ------------------------------------------------------------------ batched
    def run_batched(self, trace: List[RelightRequest], realtime: bool = True, on_launch=None,
                    keep_outputs: bool = True) -> dict:
        """Serve `trace` with continuous batching.  `on_launch(i, slices)`, if given, is
        called after launch i with its (request id, first pixel, pixels) slices.  With
        keep_outputs False a finished request's device buffers are released (long traces).

        Launches alternate over `streams` compute streams, so that one launch's kernels start
        while the previous one's persistent walk drains its last rays; a request is complete
        when every launch holding one of its slices has ended.  At most `inflight` launches
        wait on the GPU: a deeper queue delays a new request's first slice behind it.

        Slices go to the oldest request first (order "fifo"), or to the request with the
        fewest rays left ("srpt"), which lowers the median latency and raises the tail.  A
        request alone in the server with no arrival waiting runs its remaining rays as one
        launch (whole_when_alone), as the one-at-a-time arm does.  The
        rays/s statistic counts from the end of the warm-up requests, so it holds for "fifo",
        under which they finish first."""
        dev = self.device
        compute = [torch.cuda.Stream(dev) for _ in range(self.streams)]
        prep = torch.cuda.Stream(dev)
        ref = torch.cuda.Event(enable_timing=True)
        pending = collections.deque(sorted(trace, key=lambda r: r.arrival))
        active: List[_State] = []
        finished: List[_State] = []
        completing: List[_State] = []  # every slice launched, some launch still running
        inflight = collections.deque()  # launch end events, oldest first
        retiring: List[_State] = []     # cancelled after a launch: memory counted until it ends
        mem = 0
        launches = 0
        torch.cuda.synchronize(dev)
        ref.record(compute[0])
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        while pending or active or inflight or retiring or completing:
            now = (time.perf_counter() - t0) if realtime else math.inf
            # admit arrivals while their memory fits the budget
            while pending and pending[0].arrival <= now:
                req = pending[0]
                if req.rid in self.cancelled:
                    pending.popleft()
                    continue
                need = _State.bytes_needed(req)
                if active and mem + need > self.hbm_budget:
                    break
                pending.popleft()
                st = _State(req, self.scenes[req.scene], dev, prep)
                st.bytes = need
                mem += need
                active.append(st)
            self.peak_active = max(self.peak_active, len(active))
            # requests whose launches have all ended
            while inflight and inflight[0].query():
                inflight.popleft()
            for st in [s for s in completing if s.launches_done()]:
                completing.remove(st)
                st.done_ms = max(ref.elapsed_time(e) for e in st.evs.values())
                mem -= st.bytes
                if not keep_outputs:
                    st.release()
                finished.append(st)
            for st in [s for s in active if s.req.rid in self.cancelled]:
                active.remove(st)
                retiring.append(st)
            for st in [s for s in retiring if s.launches_done()]:
                retiring.remove(st)
                mem -= st.bytes
            self.peak_mem = max(self.peak_mem, mem)
            # at most `inflight` launches queued on the GPU before building the next one
            if len(inflight) >= self.inflight:
                inflight[0].synchronize()
                continue
            # next iteration: slices up to the ray budget, oldest request first or (srpt) the
            # request with the fewest rays left first
            batch, budget = [], self.ray_budget
            live = [st for st in active if st.next < st.P]
            if self.whole_when_alone and len(live) == 1 and not (pending and pending[0].arrival <= now):
                # a request alone in the server runs its remaining rays as one launch, as the
                # one-at-a-time arm does: slicing only pays when requests share the GPU
                budget = max(budget, (live[0].P - live[0].next) * live[0].req.rays)
            cand = active if self.order == "fifo" else sorted(active, key=lambda q: (q.P - q.next) * q.req.rays)
            for st in cand:
                if len(batch) >= self.max_batch or budget <= 0:
                    break
                left = st.P - st.next
                if left <= 0:
                    continue
                npx = min(left, max(32, budget // st.req.rays))
                batch.append((st, st.next, npx))
                st.next += npx
                budget -= npx * st.req.rays
            if batch:
                si = launches % len(compute)
                cs = compute[si]
                reqs = []
                for st, off, npx in batch:
                    cs.wait_event(st.ready)
                    st.use_on(cs)
                    a = st.req.alloc
                    reqs.append(api.ShadeRequest(st.scene, st.gb, st.env, a[0], a[1], a[2], st.req.seed, brdf=1,
                                                 pixel_offset=off, count=npx, color=st.color[off:off + npx],
                                                 vis=st.vis[off:off + npx], ind=st.ind[off:off + npx]))
                api.shade_batch(reqs, stream=cs)
                launches += 1
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(cs)
                for st, _, _ in batch:
                    st.evs[si] = ev
                for st in [st for st, _, _ in batch if st.next >= st.P]:
                    active.remove(st)
                    completing.append(st)
                inflight.append(ev)
                if on_launch is not None:
                    on_launch(launches - 1, [(st.req.rid, off, npx) for st, off, npx in batch])
                continue
            if inflight:
                inflight[0].synchronize()
            elif retiring:
                retiring[0].wait_launches()
            elif completing:
                completing[0].wait_launches()
            elif active and not any(st.next < st.P for st in active):
                raise RuntimeError("scheduler stalled: admitted requests without work or launch")
            elif pending:
                wait = pending[0].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.05))
        torch.cuda.synchronize(dev)
        return self._stats(finished, launches, "batched", self.skip)

    # ------------------------------------------------------------------ one at a time
    def run_serial(self, trace: List[RelightRequest], realtime: bool = True, keep_outputs: bool = True) -> dict:
        dev = self.device
        s = torch.cuda.Stream(dev)
        ref = torch.cuda.Event(enable_timing=True)
        finished = []
        torch.cuda.synchronize(dev)
        ref.record(s)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for req in sorted(trace, key=lambda r: r.arrival):
            if req.rid in self.cancelled:
                continue
            if realtime:
                wait = req.arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            st = _State(req, self.scenes[req.scene], dev, s)
            a = req.alloc
            with torch.cuda.stream(s):
                api.shade_pixels(st.scene, st.gb, st.env, a[0], a[1], a[2], req.seed, brdf=1,
                                 outputs=(st.color, st.vis, st.ind), stream=s)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
            ev.synchronize()
            st.done_ms = ref.elapsed_time(ev)
            if not keep_outputs:
                st.release()
            finished.append(st)
        return self._stats(finished, len(finished), "serial", self.skip)

    # ------------------------------------------------------------------ stats
    @staticmethod
    def _stats(states: List[_State], launches: int, mode: str, skip: int = 0) -> dict:
        warm = [st for st in states if st.req.rid < skip]
        states = [st for st in states if st.req.rid >= skip]
        if not states:
            return {"mode": mode, "requests": 0}
        lat = np.array([st.done_ms - 1e3 * st.req.arrival for st in states])
        rays = sum(int(st.n_valid.item()) * st.req.rays for st in states)
        # the measured requests are served from the first measured arrival, or from the end
        # of the warm-up requests if those finish later (a queue built up by the warm-up)
        first = min(st.req.arrival for st in states) * 1e3
        if warm:
            first = max(first, max(st.done_ms for st in warm))
        last = max(st.done_ms for st in states)
        span_s = max(last - first, 1e-6) * 1e-3
        return {"mode": mode, "requests": len(states), "launches": launches, "rays": rays,
                "rays_per_s": rays / span_s, "span_s": span_s,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
                "outputs": {st.req.rid: st for st in states}}


def default_scenes(device="cuda", sizes=(300_000, 1_000_000, 2_000_000)) -> Dict[str, api.Scene]:
    """The three resident scenes of the serving workload (object scene + two large scenes)."""
    out = {}
    for n in sizes:
        sc = wl.scene_objects(n, seed=2607) if n <= 300_000 else wl.scene_large(n, seed=2607 + n)
        out[f"s{n // 1000}k"] = api.Scene.from_workload(sc, device=device)
    return out


def scene_distances(scenes: Dict[str, api.Scene]) -> Dict[str, float]:
    return {k: (3.0 if v.n <= 300_000 else 30.0) for k, v in scenes.items()}


def poisson_run(srv: RelightServer, scenes_dist: Dict[str, float], rate: float, n_warm: int, n_meas: int,
                seed: int, envs) -> dict:
    """One arrival trace served both ways: n_warm warm-up requests then n_meas measured ones,
    Poisson at `rate` per second; p50/p99 latency and rays/s of the measured requests."""
    trace = make_trace(n_warm + n_meas, rate, scenes_dist, seed=seed, envs=envs)
    srv.skip = n_warm
    keep = ("requests", "launches", "rays", "rays_per_s", "span_s", "p50_ms", "p99_ms", "mean_ms", "max_ms")
    b = srv.run_batched(trace, keep_outputs=False)
    o = srv.run_serial(trace, keep_outputs=False)
    srv.skip = 0
    return {"rate_per_s": rate, "warmup_requests": n_warm, "batched": {k: b[k] for k in keep},
            "one_at_a_time": {k: o[k] for k in keep}}


def serve_benchmark(n_warm=100, n_meas=2000, n_warm80=None, n_meas80=None, rate=200.0, seed=7) -> dict:
    """The relight-serving workload: three resident scenes (300k, 1M, 2M surfels), random
    cameras, 512x256 HDR maps, resolutions {256^2, 512^2, 1024^2}, {8, 16, 32, 64} rays per
    pixel.  A Poisson trace at `rate` requests/s (far above capacity: the queue grows and both
    arms run saturated), then one at 80% of the batched arm's measured capacity."""
    scenes = default_scenes()
    dist = scene_distances(scenes)
    envs = env_pool(32, seed=1000)
    srv = RelightServer(scenes)
    # warm the kernels and the allocator on a short trace
    srv.run_batched(make_trace(6, 0.0, dist, seed=1, envs=envs), realtime=False)
    sat = poisson_run(srv, dist, rate, n_warm, n_meas, seed, envs)
    per_req = sat["batched"]["rays"] / max(1, sat["batched"]["requests"])
    cap = sat["batched"]["rays_per_s"] / per_req          # requests/s the batched arm sustained
    n_w80 = n_warm if n_warm80 is None else n_warm80
    n_m80 = n_meas if n_meas80 is None else n_meas80
    low = poisson_run(srv, dist, 0.8 * cap, n_w80, n_m80, seed + 1, envs)
    return {"workload": "relight_3scenes_300k_1M_2M_poisson", "scenes": {k: v.n for k, v in scenes.items()},
            "saturated": sat, "load80_batched_capacity": low, "batched_capacity_req_per_s": cap,
            "env_maps": "pool of 32 seeded 512x256 maps, uploaded and prepared per request"}


def bench_main(args):
    """bench.py --mode serve: the full trace (100 warm-up + 2,000 measured requests at 200/s,
    then 80% of the batched capacity), batched vs one at a time."""
    import json
    torch.cuda.set_device(0)
    out = {"metric": "relight_serving", "unit": "ms", "higher_is_better": False, "n_gpus": 1}
    out.update(serve_benchmark(n_warm=100, n_meas=args.serve_requests))
    print(json.dumps(out), flush=True)
