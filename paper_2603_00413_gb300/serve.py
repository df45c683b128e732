"""Serving loop with continuous batching for render and gradient requests.

Meshes, their BVHs, vertex normals and environment maps stay resident on the
device.  Requests (a mesh, a camera, a resolution, a depth, and for gradient
requests a target image) arrive over time; the scheduler, one host thread
that never blocks on the GPU:

* admits pending requests in arrival order as batch slots and device memory
  free up (each request is charged an estimate of its segment arena, image,
  gradient and backward scratch against a memory budget);
* groups the admitted requests of one kind (render or gradient) into a
  batch, launched with dt_render_batch on one of several CUDA streams, so
  batches that arrive while others run overlap on the device;
* advances gradient batches in two phases (forward, then loss seed and
  backward, sized from the forward's statistics), polling CUDA events;
* retries a batch whose arena overflowed with a larger one, and learns the
  segments per pixel of each mesh and depth to size later arenas;
* copies results back to pinned host memory and records arrival, start and
  finish times for latency percentiles;
* keeps one segment arena and one backward scratch per stream, grown when a
  batch needs more and reused by the next batch on that stream, so that a
  steady stream of requests allocates no device memory (an allocation that
  misses the caching allocator can stall every stream).

One request per launch is the same loop with max_batch=1 and one stream.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import (DT_ERR_QUEUE_OVERFLOW, DT_OK, BatchItem, Params, Workspace, _aligned_empty, batch_backward_workspace_size,
               build_bvh, l2_loss_grad, read_stats, render_batch, render_batch_backward, render_workspace_size,
               vertex_normals)


@dataclasses.dataclass
class ResidentScene:
    """One mesh kept on the device with everything a render needs."""
    V: torch.Tensor
    F: torch.Tensor
    N: torch.Tensor
    bvh: object
    ior: torch.Tensor
    sigma: torch.Tensor
    env: torch.Tensor

    @classmethod
    def from_arrays(cls, V, F, ior, sigma, env, device):
        Vt = torch.from_numpy(np.asarray(V, np.float32)).to(device)
        Ft = torch.from_numpy(np.asarray(F, np.int32)).to(device)
        return cls(Vt, Ft, vertex_normals(Vt, Ft), build_bvh(Vt, Ft),
                   torch.tensor([float(ior)], dtype=torch.float32, device=device),
                   torch.from_numpy(np.asarray(sigma, np.float32).reshape(3)).to(device),
                   torch.from_numpy(np.asarray(env, np.float32)).to(device))


@dataclasses.dataclass
class Request:
    rid: int
    scene: int
    cam: np.ndarray          # float32 [10]: eye, at, up, fov_y_deg
    width: int
    height: int
    depth: int
    kind: str                # "render" or "grad"
    arrival: float           # seconds on the serving clock
    target: np.ndarray = None  # float32 [H, W, 3] for gradient requests
    start: float = None
    finish: float = None
    image: np.ndarray = None
    grad_V: np.ndarray = None
    grad_ior: float = None
    grad_sigma: np.ndarray = None
    loss: float = None
    segments: int = 0

    @property
    def pixels(self):
        return self.width * self.height


class _Batch:
    def __init__(self, reqs, stream):
        self.reqs, self.stream = reqs, stream
        self.phase = "fwd"
        self.event = None
        self.items = self.outs = self.ws = self.tape = None
        self.host = None
        self.mem = 0


class Server:
    """Continuous-batching server over resident scenes (see module doc)."""

    def __init__(self, scenes, memory_budget: int, max_batch: int = 32, streams: int = 2, device=None):
        self.scenes = scenes
        self.device = device or scenes[0].V.device
        self.budget = int(memory_budget)
        self.max_batch = int(max_batch)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.free_streams = collections.deque(self.streams)
        self.pending = collections.deque()
        self.inflight = []
        self.done = []
        self.mem_used = 0
        self.seg_per_pixel = {}  # (scene, depth) -> largest observed segments per pixel
        self.arenas = {}  # stream -> Workspace reused by the stream's next batch
        self.scratch = {}  # stream -> (owner, aligned view) of the backward scratch
        self.t0 = None
        self.launches = 0

    # ---- memory model --------------------------------------------------------
    def _seg_estimate(self, r: Request) -> int:
        spp = self.seg_per_pixel.get((r.scene, r.depth))
        per_px = 1.25 * spp if spp else float(min(2 * r.depth + 3, 24))
        return int(r.pixels * per_px) + 1024

    def _mem_estimate(self, r: Request) -> int:
        seg = self._seg_estimate(r)
        mem = render_workspace_size(seg) + r.pixels * 12
        if r.kind == "grad":
            nv = self.scenes[r.scene].V.shape[0]
            mem += r.pixels * 12 * 2 + nv * 24 + 2 * 48 * max(r.pixels, seg // 4)
        return mem

    def _arena(self, stream, seg: int):
        """The stream's segment arena, grown (by at least a quarter) when it
        holds fewer than seg segments."""
        ws = self.arenas.get(stream)
        if ws is None or ws.capacity < seg:
            cap = seg if ws is None else max(seg, ws.capacity + ws.capacity // 4)
            ws = Workspace(min(cap, 2 ** 31 - 1), self.device)
            self.arenas[stream] = ws
        return ws

    def _scratch(self, stream, nbytes: int):
        cur = self.scratch.get(stream)
        if cur is None or cur[1].numel() < nbytes:
            n = nbytes if cur is None else max(nbytes, cur[1].numel() + cur[1].numel() // 4)
            cur = _aligned_empty(n, self.device)
            self.scratch[stream] = cur
        return cur[1]

    # ---- scheduling ---------------------------------------------------------------
    def now(self):
        return time.perf_counter() - self.t0

    def _admit(self):
        while self.pending and self.free_streams:
            head = self.pending[0]
            kind = head.kind
            batch, mem = [], 0
            for r in list(self.pending):
                if len(batch) >= self.max_batch:
                    break
                if r.kind != kind:
                    continue
                m = self._mem_estimate(r)
                if self.mem_used + mem + m > self.budget and batch:
                    break
                if self.mem_used + mem + m > self.budget and self.inflight:
                    break  # wait for memory to free up
                batch.append(r)
                mem += m
            if not batch:
                return
            for r in batch:
                self.pending.remove(r)
            self._launch(batch, mem)

    def _launch(self, reqs, mem):
        stream = self.free_streams.popleft()
        b = _Batch(reqs, stream)
        b.mem = mem
        self.mem_used += mem
        t = self.now()
        for r in reqs:
            r.start = t
        with torch.cuda.stream(stream):
            dev = self.device
            b.items = []
            for r in reqs:
                sc = self.scenes[r.scene]
                cams = torch.from_numpy(r.cam.reshape(1, 10)).pin_memory().to(dev, non_blocking=True)
                b.items.append(BatchItem(sc.V, sc.F, sc.bvh, sc.N, sc.ior, sc.sigma, sc.env, cams, r.width, r.height,
                                         Params(r.depth)))
            b.outs = [torch.empty(1, r.height, r.width, 3, device=dev) for r in reqs]
            b.ws = self._arena(stream, sum(self._seg_estimate(r) for r in reqs))
            self._forward(b)
        self.inflight.append(b)

    def _forward(self, b):
        render_batch(b.items, ws=b.ws, outs=b.outs, stream=b.stream, check=False)
        self.launches += 1
        b.phase = "fwd"
        b.event = torch.cuda.Event()
        b.event.record(b.stream)

    def _after_forward(self, b):
        st = read_stats(b.ws, stream=b.stream)  # the batch has finished: no wait
        if st["status"] == DT_ERR_QUEUE_OVERFLOW:
            with torch.cuda.stream(b.stream):
                b.ws = self._arena(b.stream, min(max(2 * b.ws.capacity, int(1.3 * st["seg_needed"])), 2 ** 31 - 1))
                self._forward(b)
            return
        if st["status"] != DT_OK:
            raise RuntimeError(f"device-side error {st['status']} in a served batch")
        b.tape_stats = st
        # learn segments per pixel per (scene, depth): a batch gives its
        # average, an underestimate for some members only costs a retry
        per_batch = st["segments"] / max(1, sum(r.pixels for r in b.reqs))
        for r in b.reqs:
            key = (r.scene, r.depth)
            self.seg_per_pixel[key] = max(self.seg_per_pixel.get(key, 0.0), per_batch)
        with torch.cuda.stream(b.stream):
            if b.reqs[0].kind == "grad":
                dev = self.device
                grads, losses = [], []
                for r, img in zip(b.reqs, b.outs):
                    tgt = torch.from_numpy(r.target.reshape(1, r.height, r.width, 3)).pin_memory().to(
                        dev, non_blocking=True)
                    g, loss = l2_loss_grad(img, tgt)
                    grads.append(g)
                    losses.append(loss)
                from . import BatchTape
                tape = BatchTape(b.ws, b.items, st)
                nb = batch_backward_workspace_size(b.items, max(1, st["max_level"]))
                bws = self._scratch(b.stream, nb)
                b.gouts = render_batch_backward(tape, grads, bws=bws, stream=b.stream)
                b.losses = losses
                self.launches += 1
            self._copy_back(b)
        b.phase = "copy"
        b.event = torch.cuda.Event()
        b.event.record(b.stream)

    def _copy_back(self, b):
        def pinned(t):
            h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
            h.copy_(t, non_blocking=True)
            return h
        b.host = [pinned(o) for o in b.outs]
        if b.reqs[0].kind == "grad":
            b.host_grads = [(pinned(dV), pinned(di), pinned(ds), pinned(l)) for (dV, di, ds), l in zip(b.gouts, b.losses)]

    def _finish(self, b):
        t = self.now()
        seg = b.tape_stats["segments"]
        tot_px = max(1, sum(r.pixels for r in b.reqs))
        for k, r in enumerate(b.reqs):
            r.finish = t
            r.image = b.host[k][0].numpy()
            r.segments = int(round(seg * r.pixels / tot_px))
            if r.kind == "grad":
                dV, di, ds, l = b.host_grads[k]
                r.grad_V, r.grad_ior, r.grad_sigma, r.loss = dV.numpy(), float(di[0]), ds.numpy(), float(l[0])
            self.done.append(r)
        self.mem_used -= b.mem
        self.free_streams.append(b.stream)

    def _poll(self):
        progressed = False
        for b in list(self.inflight):
            if not b.event.query():
                continue
            progressed = True
            if b.phase == "fwd":
                self._after_forward(b)
            else:
                self.inflight.remove(b)
                self._finish(b)
        return progressed

    def run(self, requests, timeout: float = 600.0):
        """Serve `requests` (sorted by arrival time, seconds from start) in
        open loop: each becomes pending at its arrival time.  Returns the
        finished requests.  A server can run several streams of requests one
        after another; its arenas and learned sizes carry over."""
        self.t0 = time.perf_counter()
        self.done, self.launches = [], 0
        todo = collections.deque(sorted(requests, key=lambda r: r.arrival))
        total = len(todo)
        while len(self.done) < total:
            now = self.now()
            if now > timeout:
                raise TimeoutError(f"served {len(self.done)} of {total} requests in {timeout} s")
            while todo and todo[0].arrival <= now:
                self.pending.append(todo.popleft())
            progressed = self._poll()
            self._admit()
            if not progressed and not (todo and todo[0].arrival <= self.now()):
                time.sleep(0.0002)
        torch.cuda.synchronize(self.device)
        return self.done


def latency_summary(done, wall: float) -> dict:
    lat = np.array([r.finish - r.arrival for r in done])
    seg = sum(r.segments for r in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "segments_per_s": seg / wall, "requests_per_s": len(done) / wall}


def poisson_requests(rng: np.random.Generator, n: int, rate: float, n_scenes: int, sides=(64, 1024),
                     depths=(4, 16), grad_frac: float = 0.5, view_fn=None, target_fn=None):
    """n requests arriving as a Poisson process of the given rate: random
    scene, random view (view_fn(rng, side) -> cam [10]), square side
    log-uniform in `sides`, depth uniform in `depths`, a gradient request
    with probability grad_frac (target_fn(req) -> target image)."""
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        side = int(round(np.exp(rng.uniform(np.log(sides[0]), np.log(sides[1])))))
        kind = "grad" if rng.uniform() < grad_frac else "render"
        r = Request(rid=i, scene=int(rng.integers(0, n_scenes)), cam=view_fn(rng, side), width=side, height=side,
                    depth=int(rng.integers(depths[0], depths[1] + 1)), kind=kind, arrival=t)
        if kind == "grad":
            r.target = target_fn(r)
        out.append(r)
    return out
