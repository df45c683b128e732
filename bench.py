"""Throughput of the recursive differentiable transparent-mesh tracer on GB300.

Default workload (one GPU): forward+backward of the genus-2 two-tori mesh
(about 52.5k triangles), 100 views on a Fibonacci sphere at 512x512, depth 8,
IoR ~ U[1.3,1.7] and per-channel absorption ~ U[0,2] from seed 1, L2 loss
against a render of the vertices perturbed by N(0, 0.005).  One step =
vertex normals + LBVH refit + forward render of all views + loss seed +
backward (all in libdifftrans kernels).  The metric is traced ray segments
(closest-hit queries) per second over forward+backward.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-segments/s fwd and fwd+bwd vs plain kernel; p50/p99 request latency"
UNIT = "segments/s"

# Algorithmic bytes each kernel must move per unit of work: the tape and ray
# records it reads and writes once, the scene data of the hit, and the BVH
# nodes / triangles the traversal visits.
RAY_RECORD = 48          # origin+sample, direction+node, throughput+source tri
HIT_RECORD = 16          # t, b1, b2, tri
LINK_RECORD = 8          # child index + flags
NODE_BYTES = 64          # one internal node: two child boxes + child ids
TRI_BYTES = 48           # v0, e1, e2 of a leaf triangle
ORDER_ENTRY = 4          # a level's traversal-order entry / a child's order bucket
HIT_SCENE = 84           # 3 indices + 3 positions + 3 vertex normals
ENV_MISS = 4 * 12 + 12   # 4 texels + pixel accumulation
ADJ_OUT = 36             # (L, obar, dbar) handed to the parent
ADJ_ATOMICS = 18 * 4     # dV and dN of three vertices


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--views", type=int, default=100)
    ap.add_argument("--res", type=int, default=512)
    ap.add_argument("--depth", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--cpu-sample", type=int, default=12, help="pixels in the CPU oracle sample")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-scene batching comparison")
    ap.add_argument("--batch-scenes", type=int, default=64)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving comparison")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests per arrival rate, at most")
    ap.add_argument("--serve-seconds", type=float, default=15.0,
                    help="arrival window per rate, at most (a low rate sends rate x seconds requests)")
    ap.add_argument("--serve-rates", type=str, default="10,30,100,300,1000,2000")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large optimisation step (about 1.1M-triangle noisy sphere, 800x800, 8 jittered "
                         "spp, depth 16, per-bounce checkpointing, BVH rebuild every step)")
    ap.add_argument("--no-c0", action="store_true", help="skip the forward-only icosphere leg")
    ap.add_argument("--c0-frames", type=int, default=1000)
    ap.add_argument("--large-grid", type=int, default=240)
    ap.add_argument("--large-res", type=int, default=800)
    ap.add_argument("--large-steps", type=int, default=5)
    ap.add_argument("--no-medium", action="store_true", help="skip the spatially varying absorption leg")
    ap.add_argument("--medium-grid", type=int, default=64, help="nodes per axis of the absorption grid")
    ap.add_argument("--medium-views", type=int, default=100)
    ap.add_argument("--medium-steps", type=int, default=5)
    ap.add_argument("--medium-modes", type=str,
                    default="medium,medium_moments,hash_texture,hash_texture_moments,sigma_only,sigma_only_env_grad",
                    help="comma-separated modes of the absorption leg")
    ap.add_argument("--hash-levels", type=int, default=8, help="levels of the hash-texture absorption mode")
    ap.add_argument("--hash-log2-table", type=int, default=19, help="log2 of the entries per hash-texture level")
    ap.add_argument("--hash-res", type=str, default="16,128", help="nodes per axis of the coarsest,finest level")
    return ap.parse_args()


# the source files that define each measured kernel
KERNEL_FILES = {
    "k_trace": ["dt_trace.cu", "dt_shade.cuh", "dt_internal.cuh"],
    "k_shade": ["dt_trace.cu", "dt_shade.cuh", "dt_internal.cuh"],
    "k_adjoint": ["dt_adjoint.cu", "dt_shade.cuh", "dt_internal.cuh"],
}


def kernel_sources_hash(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_00413_gb300", "csrc")
    for f in KERNEL_FILES.get(kernel, sorted(os.listdir(csrc))):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, units_per_launch: float):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (bytes per unit there, scaled to this launch's units), if it was taken on
    the current sources of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("kernel_sources") != kernel_sources_hash(kernel):
        return None
    return e.get("dram_bytes_per_unit") * units_per_launch


def ncu_issue(kernel: str):
    """(warp instructions per unit, threads active per instruction) of
    `kernel` from the committed ncu summary, if it was taken on the current
    sources of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        e = json.load(open(path)).get(kernel)
    except Exception:
        return None
    if not e or e.get("kernel_sources") != kernel_sources_hash(kernel) or "inst_per_unit" not in e:
        return None
    return float(e["inst_per_unit"]), float(e["threads_per_inst"])


def issue_roofline(inst_per_unit: float, threads_per_inst: float, units_per_launch: float, ms_per_launch: float,
                   n_sm: int, sm_mhz: float) -> dict:
    """The instruction-issue rate of a launch against the chip's issue peak:
    one warp instruction per cycle per scheduler, four schedulers per SM."""
    achieved = inst_per_unit * units_per_launch / (ms_per_launch / 1000.0) / 1e9
    peak = n_sm * 4 * sm_mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G warp-instructions/s", "frac": achieved / peak,
            "instructions_per_segment": inst_per_unit, "threads_per_instruction": threads_per_inst,
            "peak_source": f"{n_sm} SMs x 4 schedulers x {sm_mhz:.0f} MHz (median SM clock of the timed steps)"}


def genus2_workload(n_views, res, depth, seed=1):
    from paper_2603_00413_gb300 import scenes as S
    sc, Vt = S.genus2_scene(n_views=n_views, width=res, height=res, max_depth=depth, seed=seed)
    return sc, Vt


class ClockSampler:
    """nvidia-smi samples during the timed region (every 200 ms)."""

    def __init__(self, gpu_index=0):
        self.rows, self.proc, self.gpu = [], None, gpu_index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
def oracle_sample(sc, Vt, n_pix, seed=12345):
    """A bounded, seeded sample of the workload for the FP64 oracle: n_pix
    random pixels of the 100 views, traced forward and differentiated
    (forward mode over every parameter that can influence them)."""
    import oracle as O
    rng = np.random.default_rng(seed)
    views = rng.integers(0, len(sc.cams), size=n_pix)
    cam0 = sc.cams[0]
    pix = rng.integers(0, cam0.width * cam0.height, size=n_pix)
    o = np.zeros((n_pix, 3))
    d = np.zeros((n_pix, 3))
    for i, (v, p) in enumerate(zip(views, pix)):
        oo, dd = O.camera_rays(sc.cams[v])
        o[i], d[i] = oo[p], dd[p]
    g = rng.normal(size=(n_pix, 3))
    t0 = time.perf_counter()
    dV, dior, dsig, nseg = O.rays_grad(sc.V, sc.F, sc.ior, sc.sigma, sc.env, o, d, sc.max_depth, g)
    dt = time.perf_counter() - t0
    return nseg, dt


def workload_config(sc, views_per_rank, res, depth, world):
    """The config object both arms print for the genus-2 workload."""
    return {"workload": f"genus-2 two-tori mesh ({sc.F.shape[0]} triangles), {views_per_rank * world} views "
                        f"{res}x{res}, depth {depth}, 1 spp, IoR {sc.ior:.4f}, fwd+bwd of an L2 image loss",
            "views": views_per_rank * world, "width": res, "height": res, "max_depth": depth,
            "triangles": int(sc.F.shape[0])}


def cpu_model():
    """The host CPU's model string (x86 'model name', Arm implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return None
    for key in ("model name", "Model", "Hardware"):
        for line in info:
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    arm = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1", "0xd49": "Arm Neoverse N2"}
    parts = sorted({line.split(":", 1)[1].strip() for line in info if line.startswith("CPU part")})
    return ", ".join(arm.get(p, "CPU part " + p) for p in parts) if parts else None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    O.build()
    sc, Vt = genus2_workload(args.views, args.res, args.depth)
    n_pix = max(1, args.cpu_sample // 3)
    for w in range(args.warmup):
        oracle_sample(sc, Vt, n_pix, seed=1000 + w)
    segs, secs = 0, 0.0
    for k in range(args.steps):
        n, t = oracle_sample(sc, Vt, n_pix, seed=2000 + k)
        segs += n
        secs += t
    value = segs / secs
    sample = (f"{n_pix} seeded pixels per step of the 100-view 512^2 genus-2 workload (depth {args.depth}); "
              f"forward + gradient by forward mode over the parameters those paths touch")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": workload_config(sc, args.views, args.res, args.depth, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "cpu": cpu_model(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
# kernels launched per profiled scope (a scope may hold more than one kernel)
KERNELS_PER_SCOPE = {"k_vertex_normals": 2, "k_refit": 3, "k_camera": 1, "k_trace": 1,
                     "k_shade": 1, "k_order": 2, "order_clear": 0,
                     "k_l2_loss_grad": 1, "k_adjoint": 1, "k_face_normals_backward": 1, "lbvh_build": 21,
                     "k_write_table": 1, "k_zero_grads": 1}


def sah_levels(nf: int) -> int:
    """Large-task levels the binned-SAH builder launches for nf triangles:
    tasks above 128 triangles are split level by level, with 24 levels of
    free splits plus the median levels below them, at most 64."""
    if nf <= 128:
        return 0
    lg = 0
    while (128 << lg) < nf:
        lg += 1
    return min(24 + lg + 2, 64)


def scope_kernels(scope: str, nf: int) -> int:
    """Kernels launched per entry of a profiled scope; the SAH build's scopes
    nest (sah_build holds sah_large_levels and sah_small), so each counts only
    its own launches."""
    if scope == "sah_build":
        return 10  # header, bounds x2, primitives, root, 4-wide topology x4, validation
    if scope == "sah_large_levels":
        return 4 * sah_levels(nf)
    if scope == "sah_small":
        return 1
    return KERNELS_PER_SCOPE.get(scope, 1)


def serve_leg(args, dev):
    """Poisson streams of render and gradient requests (50/50) over 32
    resident meshes (random blobs, faces log-uniform in [5k, 500k]); square
    images with side log-uniform in [64, 1024], depth uniform in 4..16, a
    random view each.  The continuous-batching server against the same loop
    serving one request per launch, at each arrival rate: min(2000, rate x
    15 s) requests, the same stream for both servers."""
    import torch
    from paper_2603_00413_gb300 import serve
    from paper_2603_00413_gb300 import scenes as S
    t0 = time.time()
    scs = S.serve_scenes(32, 4)
    gen_s = time.time() - t0
    res = [serve.ResidentScene.from_arrays(sc.V, sc.F, sc.ior, sc.sigma, sc.env, dev) for sc in scs]
    budget = int(0.5 * torch.cuda.mem_get_info(dev)[0])
    rates = [float(x) for x in args.serve_rates.split(",")]
    out = {"workload": f"{len(res)} resident meshes ({min(r.F.shape[0] for r in res)}-"
                       f"{max(r.F.shape[0] for r in res)} faces), Poisson arrivals, min({args.serve_requests}, "
                       f"rate x {args.serve_seconds:g} s) requests per rate, 50% render / 50% gradient, side "
                       f"64-1024, depth 4-16", "mesh_gen_s": round(gen_s, 1), "rates": {}}

    def view(rng, side):
        return S.random_view(rng, 3.0, side, side).as_array()

    targets = {}

    def target(r):  # one fixed random target image per size
        if r.width not in targets:
            targets[r.width] = np.random.default_rng(r.width).uniform(0, 2, size=(r.height, r.width, 3)).astype(
                np.float32)
        return targets[r.width]

    servers = {"batched": serve.Server(res, budget, max_batch=32, streams=2),
               "one_per_launch": serve.Server(res, budget, max_batch=1, streams=1)}
    # one untimed burst per server first: its arenas, the allocator's cache
    # and the learned segments per pixel start warm, as in a running service
    for srv in servers.values():
        srv.run(serve.poisson_requests(np.random.default_rng(99), 200, 2000.0, len(res), sides=(64, 1024),
                                       depths=(4, 16), grad_frac=0.5, view_fn=view, target_fn=target), timeout=600)
    for rate in rates:
        n = int(min(args.serve_requests, max(20, round(rate * args.serve_seconds))))
        row = {"requests": n}
        for name, srv in servers.items():
            rng = np.random.default_rng(int(rate))
            reqs = serve.poisson_requests(rng, n, rate, len(res), sides=(64, 1024), depths=(4, 16),
                                          grad_frac=0.5, view_fn=view, target_fn=target)
            done = srv.run(reqs, timeout=600)
            wall = max(r.finish for r in done)
            summ = serve.latency_summary(done, wall)
            row[name] = {k: (round(v, 2) if isinstance(v, float) else v) for k, v in summ.items()}
            row[name]["launches"] = srv.launches
        out["rates"][str(int(rate))] = row
    return out


def c0_leg(args, dt, dev):
    """The plain forward-only icosphere: subdivision 3 (1280 triangles),
    IoR 1.5, no absorption, camera at distance 3, 64x64 at pixel centres,
    depth 4, 64x32 SH environment.  A frame is one forward render (camera
    rays and five trace/shade levels), launch-latency bound at ~23k
    segments; 1000 frames are timed back to back as eager launches and as
    replays of a captured CUDA graph of one frame."""
    import torch
    from paper_2603_00413_gb300 import scenes as S
    sc = S.glass_icosphere_scene()
    cam = sc.cams[0]
    V = torch.from_numpy(sc.V).to(dev)
    F = torch.from_numpy(sc.F).to(dev)
    ior = torch.tensor([sc.ior], device=dev)
    sigma = torch.from_numpy(np.asarray(sc.sigma, np.float32)).to(dev)
    env = torch.from_numpy(sc.env).to(dev)
    cams = torch.from_numpy(cam.as_array()[None]).to(dev)
    params = dt.Params(sc.max_depth)
    bvh = dt.build_bvh(V, F)
    N = dt.vertex_normals(V, F)
    img, tape = dt.render(V, F, bvh, N, ior, sigma, env, cams, cam.width, cam.height, params)
    stats = tape.stats
    seg = stats["segments"]
    stream = torch.cuda.current_stream()

    def frame():
        dt.render(V, F, bvh, N, ior, sigma, env, cams, cam.width, cam.height, params, ws=tape.ws, out=img,
                  check=False)

    def timed(fn, k):
        for _ in range(10):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    k = args.c0_frames
    ms_eager = timed(frame, k)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        frame()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            frame()
    ms_graph = timed(graph.replay, k)
    chk = dt.read_stats(tape.ws)
    assert chk["status"] == dt.DT_OK and chk["segments"] == seg, chk
    return {"workload": f"glass icosphere ({sc.F.shape[0]} triangles), 64x64, 1 spp at pixel centres, depth "
                        f"{sc.max_depth}, IoR {sc.ior}, forward only, {k} frames back to back",
            "segments_per_frame": int(seg), "eager_ms_per_frame": round(ms_eager, 4),
            "eager_segments_per_s": seg / (ms_eager / 1e3), "graph_ms_per_frame": round(ms_graph, 4),
            "graph_segments_per_s": seg / (ms_graph / 1e3)}


def large_leg(args, dt, dev):
    """The large optimisation step: sphere SDF (r = 1) plus 3 octaves of value
    noise (amplitude 0.1) meshed by marching tetrahedra on a 240^3 grid over
    [-1.3, 1.3]^3 (about 1.1M triangles), one 800x800 view with 8 jittered
    samples per pixel (5.12M camera rays), depth 16, IoR 1.52, sigma (0.3,
    0.1, 0.05), a 2048x1024 environment; L2 loss against a render of the
    vertices perturbed by N(0, 0.001).  One step = BVH rebuild (the tuned
    builder: binned SAH by default) + vertex normals + checkpointed forward
    + loss seed + backward (hits recovered from the children's source
    triangles).  The same step with the full tape is timed beside it, and
    the mesh update that closes the loop (L_edge gradient + large-steps
    AdamUniform, App. A) after them."""
    import torch
    from paper_2603_00413_gb300 import scenes as S
    t0 = time.time()
    Vn, Fn = S.noisy_sphere_mesh(args.large_grid, seed=3, amplitude=0.1, octaves=3)
    env_np = S.sh_env_map(2048, 1024, 3)
    gen_s = time.time() - t0
    rng = np.random.default_rng(4)
    res, D, spp = args.large_res, 16, 8
    cam = S.camera((0.45, 0.35, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, res, res)
    V = torch.from_numpy(Vn).to(dev)
    F = torch.from_numpy(Fn).to(dev)
    Vt = torch.from_numpy((Vn + rng.normal(scale=0.001, size=Vn.shape)).astype(np.float32)).to(dev)
    ior = torch.tensor([1.52], device=dev)
    sigma = torch.tensor([0.3, 0.1, 0.05], device=dev)
    env = torch.from_numpy(env_np).to(dev)
    cams = torch.from_numpy(cam.as_array()[None]).to(dev)
    stream = torch.cuda.current_stream()
    out = {"workload": f"noisy sphere ({Fn.shape[0]} triangles, marching tetrahedra {args.large_grid}^3), 1 view "
                       f"{res}x{res}, {spp} jittered spp, depth {D}, IoR 1.52, sigma (0.3, 0.1, 0.05), env 2048x1024",
           "triangles": int(Fn.shape[0]), "camera_rays": res * res * spp, "mesh_gen_s": round(gen_s, 1)}
    bvh = dt.build_bvh(V, F)
    N = dt.vertex_normals(V, F)
    for mode in ("checkpoint", "full"):
        params = dt.Params(D, spp=spp, jitter=1, seed=11, checkpoint=(mode == "checkpoint"))
        bvh_t = dt.build_bvh(Vt, F)
        target, _ = dt.render(Vt, F, bvh_t, dt.vertex_normals(Vt, F), ior, sigma, env, cams, res, res, params)
        del bvh_t
        img, tape = dt.render(V, F, bvh, N, ior, sigma, env, cams, res, res, params)
        stats = tape.stats
        ws = tape.ws
        _, bws = dt._aligned_empty(dt.backward_workspace_size(stats["max_level"], V.shape[0]), dev)
        grad = torch.empty_like(img)
        loss = torch.empty(1, device=dev)

        def step():
            bvh.build(V, F)
            dt.vertex_normals(V, F, out=N)
            o, tp = dt.render(V, F, bvh, N, ior, sigma, env, cams, res, res, params, ws=ws, out=img, check=False)
            tp.stats = stats
            dt.l2_loss_grad(o, target, grad=grad, loss=loss)
            return dt.render_backward(tp, grad, bws=bws)

        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        dt.profile_read()
        dt.profile_enable(True)
        ev = []
        for _ in range(args.large_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        dt.profile_enable(False)
        prof = dt.profile_read()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.large_steps
        chk = dt.read_stats(ws)
        assert chk["status"] == dt.DT_OK and chk["segments"] == stats["segments"], chk
        seg = stats["segments"]
        tot = sum(v[1] for v in prof.values())
        top = sorted(prof.items(), key=lambda kv: -kv[1][1])[:5]
        out[mode] = {"ms_per_step": round(ms, 3), "segments_per_step": int(seg), "segments_per_s": seg / (ms / 1e3),
                     "tape_bytes": int(ws.bytes), "level_capacity": int(ws.level_capacity),
                     "rebuild_ms": round((prof.get("lbvh_build", (1, 0.0))[1] + prof.get("sah_build", (1, 0.0))[1])
                                         / args.large_steps, 3),
                     "top_kernel_share": {k: round(v[1] / tot, 4) for k, v in top},
                     "gpu_launches_per_step": int(sum(v[0] * scope_kernels(k, Fn.shape[0]) for k, v in prof.items())
                                                  / args.large_steps),
                     "loss": float(loss.item())}
        del ws, bws, tape, img, target, grad
        torch.cuda.empty_cache()
    # the step after the gradient (App. A): L_edge's gradient added to a
    # vertex gradient and the large-steps AdamUniform update, on a copy of
    # the mesh; with the checkpointed step it closes the optimisation loop
    Vc = V.clone()
    topo = dt.Topology(F, V.shape[0])
    opt = dt.LargeStepsOptimizer(Vc, F, lam=10.0, lr=1e-3, topo=topo)
    gV = torch.randn(V.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(9)) * 1e-3

    def update():
        _, dVe = dt.edge_loss_grad(Vc, F, topo)
        opt.step(gV + 1e-3 * dVe)

    for _ in range(2):
        update()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.large_steps):
        update()
    e1.record(stream)
    torch.cuda.synchronize()
    upd = e0.elapsed_time(e1) / args.large_steps
    out["mesh_update"] = {"ms": upd, "vertices": int(V.shape[0]), "edges": int(topo.info()[0]),
                          "cg_iterations_max": opt.iters,
                          "optimisation_step_ms": out["checkpoint"]["ms_per_step"] + upd}
    return out


def medium_leg(args, dt, dev):
    """The bench workload (genus-2 mesh, n views 512x512, depth 8, the same
    IoR and sigma) with a spatially varying absorption rate on top of sigma
    (Eq. 11): a grid^3 lattice of smooth random rates over [-1.25, 1.25]^3,
    trilinear, sampled every half cell along interior segments.  One step =
    normals + refit + forward + backward seeded by a fixed random image
    gradient, with the node-value gradient; the same step without the grid
    is timed beside it, and once more with the environment-texel gradient.
    The hash_texture mode replaces the grid by a multi-resolution hash
    texture (levels from n_min to n_max nodes per axis, 2^k entries per
    level, random rates averaging 1) sampled with the same step."""
    import torch
    from paper_2603_00413_gb300 import scenes as S
    sc, _ = genus2_workload(args.medium_views, args.res, args.depth)
    V = torch.from_numpy(sc.V).to(dev)
    F = torch.from_numpy(sc.F).to(dev)
    ior = torch.tensor([sc.ior], device=dev)
    sigma = torch.from_numpy(sc.sigma).to(dev)
    env = torch.from_numpy(sc.env).to(dev)
    cams = torch.from_numpy(np.stack([c.as_array() for c in sc.cams])).to(dev)
    g = args.medium_grid
    lo, hi = (-1.25, -1.25, -1.25), (1.25, 1.25, 1.25)
    med = S.random_absorption_grid((g, g, g), lo, hi, seed=6, scale=1.0)
    medium = dt.Medium(torch.from_numpy(med["mu"]).to(dev), lo, hi, med["step"])
    n_min, n_max = (int(x) for x in args.hash_res.split(","))
    tex = S.random_hash_texture(args.hash_levels, args.hash_log2_table, n_min, n_max, lo, hi, seed=8, scale=1.0,
                                step=med["step"])
    texture = dt.HashTexture(torch.from_numpy(tex["table"]).to(dev), tex["res"], lo, hi, tex["step"])
    bvh = dt.build_bvh(V, F)
    N = dt.vertex_normals(V, F)
    res = args.res
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    out = {"workload": f"genus-2 two-tori mesh ({sc.F.shape[0]} triangles), {args.medium_views} views {res}x{res}, "
                       f"depth {args.depth}, IoR {sc.ior:.4f}, sigma {tuple(round(float(x), 4) for x in sc.sigma)} "
                       f"plus a {g}^3 grid of smooth random absorption rates over [-1.25, 1.25]^3 sampled every "
                       f"{med['step']:.4f} (half a cell) along interior segments; fwd+bwd with a fixed image gradient",
           "grid_nodes": g ** 3, "step": med["step"],
           "hash_texture_config": {"levels": args.hash_levels, "entries_per_level": 1 << args.hash_log2_table,
                                   "res": tex["res"], "table_bytes": int(texture.mu.numel() * 4)}}
    # *_moments: the same step on a tape that keeps the medium's moments
    # (tape_mode 2: a medium pass marches each interior segment once, in the
    # forward, and the backward reads no medium value)
    for mode in args.medium_modes.split(","):
        m = {"medium": medium, "hash_texture": texture}.get(mode.replace("_moments", ""))
        want_env = mode == "sigma_only_env_grad"
        params = dt.Params(args.depth, moments=mode.endswith("_moments"))
        img, tape = dt.render(V, F, bvh, N, ior, sigma, env, cams, res, res, params, medium=m)
        # the timed steps run in a workspace sized to the segments the render needs
        ws = dt.Workspace(int(tape.stats["segments"] * 1.02) + 4096, dev, moments=params.moments)
        del tape
        torch.cuda.empty_cache()
        img, tape = dt.render(V, F, bvh, N, ior, sigma, env, cams, res, res, params, ws=ws, out=img, medium=m)
        stats = tape.stats
        _, bws = dt._aligned_empty(dt.backward_workspace_size(stats["max_level"], V.shape[0]), dev)
        grad = torch.randn(img.shape, device=dev, generator=gen)

        def step():
            dt.vertex_normals(V, F, out=N)
            bvh.refit(V, F)
            _, tp = dt.render(V, F, bvh, N, ior, sigma, env, cams, res, res, params, ws=tape.ws, out=img,
                              check=False, medium=m)
            tp.stats = stats
            return dt.render_backward(tp, grad, bws=bws, env_grad=want_env)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        dt.profile_read()
        dt.profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.medium_steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        dt.profile_enable(False)
        prof = dt.profile_read()
        ms = e0.elapsed_time(e1) / args.medium_steps
        chk = dt.read_stats(tape.ws)
        assert chk["status"] == dt.DT_OK and chk["segments"] == stats["segments"], chk
        tot = sum(v[1] for v in prof.values())
        top = sorted(prof.items(), key=lambda kv: -kv[1][1])[:4]
        out[mode] = {"ms_per_step": round(ms, 3), "segments_per_step": int(stats["segments"]),
                     "segments_per_s": stats["segments"] / (ms / 1e3),
                     "grid_samples_per_step": int(stats["medium_samples"]),
                     "top_kernels_ms": {k: round(v[1] / args.medium_steps, 3) for k, v in top}}
        del tot
        del tape, ws, bws, img, grad
        torch.cuda.empty_cache()
    return out


def batch_leg(args, dt, dev, steps):
    """64 scenes of uneven size (2k-200k faces, 128^2-800^2 images, depth
    4-12), fwd+bwd with a fixed image gradient: the plain loop (each scene
    rendered and differentiated by its own calls), one batched render +
    backward, and the batched step replayed from a captured CUDA graph."""
    import torch
    from paper_2603_00413_gb300 import scenes as S
    scs = S.batch_scenes(args.batch_scenes, 2)
    items = []
    for sc in scs:
        V = torch.from_numpy(sc.V).to(dev)
        F = torch.from_numpy(sc.F).to(dev)
        c = sc.cams[0]
        items.append(dt.BatchItem(V, F, dt.build_bvh(V, F), dt.vertex_normals(V, F),
                                  torch.tensor([sc.ior], device=dev), torch.from_numpy(sc.sigma).to(dev),
                                  torch.from_numpy(sc.env).to(dev), torch.from_numpy(c.as_array()[None]).to(dev),
                                  c.width, c.height, dt.Params(sc.max_depth)))
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    grads = [torch.randn(1, it.height, it.width, 3, device=dev, generator=gen) for it in items]
    stream = torch.cuda.current_stream()
    # batched
    imgs, tape = dt.render_batch(items)
    st = tape.stats
    seg = st["segments"]
    _, bws = dt._aligned_empty(dt.batch_backward_workspace_size(items, st["max_level"]), dev)
    gouts = [(torch.empty_like(it.V), torch.empty(1, device=dev), torch.empty(3, device=dev)) for it in items]

    def batched():
        _, t = dt.render_batch(items, ws=tape.ws, outs=imgs, check=False)
        t.stats = st
        dt.render_batch_backward(t, grads, bws=bws, outs=gouts)

    # plain: each scene on its own, with its own workspace sized by a first render
    plain_ws = []
    for it in items:
        _, t = dt.render(it.V, it.F, it.bvh, it.N, it.ior, it.sigma, it.env, it.cams, it.width, it.height, it.params)
        _, b = dt._aligned_empty(dt.backward_workspace_size(t.stats["max_level"], it.V.shape[0]), dev)
        plain_ws.append((t, b))
    plain_seg = sum(t.stats["segments"] for t, _ in plain_ws)

    def plain():
        for it, (t, b), img, g in zip(items, plain_ws, imgs, grads):
            _, tp = dt.render(it.V, it.F, it.bvh, it.N, it.ior, it.sigma, it.env, it.cams, it.width, it.height,
                              it.params, ws=t.ws, out=img, check=False)
            tp.stats = t.stats
            dt.render_backward(tp, g, bws=b)

    def timed(fn, k):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    from paper_2603_00413_gb300 import autotune
    import tempfile
    tuned = autotune.tune(batched, key=f"batch{len(items)}-seed2", reps=1, retune=True,
                          cache_path=os.path.join(tempfile.gettempdir(), "difftrans_bench_tuning.json"))
    ms_batched = timed(batched, steps)
    ms_plain = timed(plain, steps)
    # the batched step captured once in a CUDA graph and replayed
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        batched()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            batched()
    ms_graph = timed(graph.replay, steps)
    chk = dt.read_stats(tape.ws)
    assert chk["status"] == dt.DT_OK and chk["segments"] == seg, chk
    depth_max = max(it.params.max_depth for it in items)
    return {
        "workload": f"{len(items)} random-blob scenes, {sum(it.F.shape[0] for it in items)} faces in all "
                    f"({min(it.F.shape[0] for it in items)}-{max(it.F.shape[0] for it in items)}), "
                    f"{sum(it.width * it.height for it in items)} pixels ({min(it.width for it in items)}^2-"
                    f"{max(it.width for it in items)}^2), depth {min(it.params.max_depth for it in items)}-"
                    f"{depth_max}, fwd+bwd with a fixed image gradient",
        "segments_per_step": int(seg),
        "plain_segments_per_s": plain_seg / (ms_plain / 1e3), "plain_ms": ms_plain,
        "batched_segments_per_s": seg / (ms_batched / 1e3), "batched_ms": ms_batched,
        "graph_segments_per_s": seg / (ms_graph / 1e3), "graph_ms": ms_graph,
        "tuning": tuned["tuning"], "tuning_trials": len(tuned["trials"]),
        "launches_per_step_plain": int(sum(3 * (it.params.max_depth + 1) + 8 for it in items)),
        "launches_per_step_batched": int(3 * (depth_max + 1) + 4 + 2 * (1 + (len(items) + 23) // 24)),
    }


def summary_digest(out: dict) -> dict:
    """The headline numbers of every workload of one bench line, rounded."""
    def r(x, n=3):
        return None if x is None else round(float(x), n)

    g = {"fwd_bwd_gseg_s": r(out["value"] / 1e9), "fwd_gseg_s": r(out["fwd_segments_per_s"] / 1e9),
         "ms_per_step": r(out["ms_per_step"], 2),
         "e2e_gseg_s": r(out["e2e"]["value"] / 1e9) if out.get("e2e") else None,
         "k_trace_ms_per_launch": r(out["roofline"]["ms_per_launch"]), "k_trace_hbm_frac": r(out["roofline"]["frac"]),
         "k_trace_l2_frac": r((out["roofline"].get("l2") or {}).get("frac")),
         "k_trace_issue_frac": r((out["roofline"].get("issue") or {}).get("frac"))}
    lg = out.get("large")
    if lg:
        g["large"] = {"ckpt_ms": r(lg["checkpoint"]["ms_per_step"], 2), "full_ms": r(lg["full"]["ms_per_step"], 2),
                      "gseg_s": r(lg["checkpoint"]["segments_per_s"] / 1e9), "rebuild_ms": lg["checkpoint"]["rebuild_ms"],
                      "mesh_update_ms": r(lg["mesh_update"]["ms"], 2),
                      "opt_step_ms": r(lg["mesh_update"]["optimisation_step_ms"], 2)}
    b = out.get("batch")
    if b:
        g["batch"] = {"one_launch_ms": r(b["batched_ms"], 2), "graph_ms": r(b["graph_ms"], 2),
                      "one_scene_per_launch_ms": r(b["plain_ms"], 2), "gseg_s": r(b["graph_segments_per_s"] / 1e9)}
    c = out.get("c0")
    if c:
        g["c0"] = {"eager_ms_per_frame": c["eager_ms_per_frame"], "graph_ms_per_frame": c["graph_ms_per_frame"]}
    m = out.get("medium")
    if m:
        g["medium_ms"] = {k: m[k]["ms_per_step"] for k in ("sigma_only", "sigma_only_env_grad", "medium",
                                                           "medium_moments", "hash_texture", "hash_texture_moments")
                          if isinstance(m.get(k), dict)}
    pl = out.get("paper_loss")
    if pl:
        g["paper_loss_ms"] = r(pl["ms"])
    sv = out.get("serve")
    if sv and sv.get("rates"):
        g["serve"] = {"[p50, p99] ms, req/s: batched | one per launch": None}
        for rate, e in sv["rates"].items():
            bb, oo = e["batched"], e["one_per_launch"]
            g["serve"][rate] = [bb["p50_ms"], bb["p99_ms"], bb["requests_per_s"], "|", oo["p50_ms"], oo["p99_ms"],
                                oo["requests_per_s"]]
    return g


def rank_cameras(n_views: int, world: int, rank: int, res: int):
    """The views of one rank: every world-th view of a Fibonacci set of
    n_views * world, so ranks hold disjoint sets of the same size (weak
    scaling) and their union is the whole set."""
    from paper_2603_00413_gb300 import scenes as S
    allc = S.fibonacci_views(n_views * world, 3.0, res, res)
    return allc[rank::world]


def reduce_over_ranks(times, units, device):
    """(max over ranks of each time, sum over ranks of units): the whole-job
    time is the slowest rank's, the work is everyone's."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return [float(x) for x in times], float(units)
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    tdist.all_reduce(u, op=tdist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], float(u.item())


def run_ours(args):
    import torch
    import torch.distributed as tdist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2603_00413_gb300 import build as B
    B.build()
    import paper_2603_00413_gb300 as dt

    sc, Vt_np = genus2_workload(args.views, args.res, args.depth)
    # disjoint view sets per rank (weak scaling)
    if world > 1:
        sc.cams = rank_cameras(args.views, world, rank, args.res)
    res, D = args.res, args.depth
    nvw = len(sc.cams)
    V = torch.from_numpy(sc.V).to(dev)
    F = torch.from_numpy(sc.F).to(dev)
    ior = torch.tensor([sc.ior], dtype=torch.float32, device=dev)
    sigma = torch.from_numpy(sc.sigma).to(dev)
    env = torch.from_numpy(sc.env).to(dev)
    cams = torch.from_numpy(np.stack([c.as_array() for c in sc.cams])).to(dev)
    params = dt.Params(D)
    stream = torch.cuda.current_stream()

    # target images: render of the perturbed vertices
    Vtt = torch.from_numpy(Vt_np).to(dev)
    bvh_t = dt.build_bvh(Vtt, F)
    target, tape_t = dt.render(Vtt, F, bvh_t, dt.vertex_normals(Vtt, F), ior, sigma, env, cams, res, res, params)
    del tape_t, bvh_t
    # workspaces sized by a first render, kept for every step
    bvh = dt.build_bvh(V, F)
    N = dt.vertex_normals(V, F)
    img, tape = dt.render(V, F, bvh, N, ior, sigma, env, cams, res, res, params)
    stats = tape.stats
    ws = tape.ws
    bws_bytes = dt.backward_workspace_size(stats["max_level"], V.shape[0])
    _, bws = dt._aligned_empty(bws_bytes, dev)
    grad = torch.empty_like(img)
    loss = torch.empty(1, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def step(fwd_only=False, target_ready=None):
        dt.vertex_normals(V, F, out=N)
        bvh.refit(V, F)
        out, tp = dt.render(V, F, bvh, N, ior, sigma, env, cams, res, res, params, ws=ws, out=img, check=False)
        if fwd_only:
            return None
        tp.stats = stats
        if target_ready is not None:  # the target arrives on another stream
            stream.wait_event(target_ready)
        dt.l2_loss_grad(out, target, grad=grad, loss=loss)
        return dt.render_backward(tp, grad, bws=bws)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    chk = dt.read_stats(ws)
    assert chk["status"] == dt.DT_OK and chk["segments"] == stats["segments"], chk

    # ---- timed fwd+bwd ----------------------------------------------------
    def timed(fwd_only, k_steps, profile=False):
        times = []
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()
        if profile:
            dt.profile_read()
            dt.profile_enable(True)
        for _ in range(k_steps):
            flush.fill_(1.0)  # evict L2 between steps (outside the events)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(fwd_only)
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize()
        prof = None
        if profile:
            dt.profile_enable(False)
            prof = dt.profile_read()
        ms = [a.elapsed_time(b) for a, b in times]
        if world > 1:
            tdist.barrier()
        return ms, prof

    with ClockSampler(dev.index or 0) as clk:
        ms, prof = timed(False, args.steps, profile=True)
    ms_fwd, _ = timed(True, args.steps)
    seg = stats["segments"]
    (total_ms, fwd_ms), seg_all = reduce_over_ranks([sum(ms), sum(ms_fwd)], seg, dev)
    value = seg_all * args.steps / (total_ms / 1000.0)
    fwd_value = seg_all * args.steps / (fwd_ms / 1000.0)
    chk = dt.read_stats(ws)
    assert chk["status"] == dt.DT_OK and chk["segments"] == seg, chk

    # ---- roofline of the dominant kernel ---------------------------------
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    kt = {k: v for k, v in prof.items()}
    dom = max(kt, key=lambda k: kt[k][1])
    hits, misses = stats["hits"], stats["misses"]
    spawners = hits - stats["discarded"] - stats["backfacing"]
    children = seg - nvw * res * res
    bvh_bytes = (sc.F.shape[0] - 1) * NODE_BYTES + sc.F.shape[0] * TRI_BYTES
    # bytes that must cross HBM per step (the BVH, the scene and the
    # environment stay in L2; the tape, the image and its gradient do not)
    # (levels after the camera rays, when traced in bucket order: + the
    # order entry the traversal reads, + the bucket the shading pass writes)
    ordered = children if dt.get_tuning()["trace_order"] else 0
    hbm_step = {
        "k_trace": seg * (RAY_RECORD + HIT_RECORD) + ordered * ORDER_ENTRY + (D + 1) * bvh_bytes,
        "k_shade": seg * (RAY_RECORD + HIT_RECORD + LINK_RECORD) + children * RAY_RECORD + ordered * ORDER_ENTRY
        + misses * 2 * 12,
        "k_adjoint": seg * (RAY_RECORD + HIT_RECORD + LINK_RECORD + 12) + (seg - nvw * res * res) * 48
        + spawners * 2 * 48,
    }
    # bytes the kernel moves through L2 (on-chip reuse included)
    l2_step = {
        "k_trace": seg * (RAY_RECORD + HIT_RECORD) + ordered * ORDER_ENTRY + stats["nodes_visited"] * NODE_BYTES
        + stats["tris_tested"] * TRI_BYTES,
        "k_shade": hbm_step["k_shade"] + hits * HIT_SCENE + misses * ENV_MISS,
        "k_adjoint": hbm_step["k_adjoint"] + spawners * (HIT_SCENE + ADJ_ATOMICS) + misses * 48,
    }
    launches, dom_ms = kt[dom]
    per_launch_ms = dom_ms / launches
    hbm_per_launch = hbm_step.get(dom, 0) * args.steps / launches
    l2_per_launch = l2_step.get(dom, 0) * args.steps / launches
    achieved = hbm_per_launch / (per_launch_ms / 1000.0) / 1e9
    # best of five 200-pass reads of a 32 MB buffer (a single short read can
    # land on a clock ramp)
    l2_peak = max(dt.measure_l2_read_bandwidth(iters=200) for _ in range(5))
    l2_achieved = l2_per_launch / (per_launch_ms / 1000.0) / 1e9
    traffic = ncu_traffic(dom, seg * args.steps / launches)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "kernel": dom,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_launch": hbm_per_launch, "ms_per_launch": per_launch_ms,
                "l2": {"achieved": l2_achieved, "peak": l2_peak, "unit": "GB/s", "frac": l2_achieved / l2_peak,
                       "bytes_per_launch": l2_per_launch,
                       "peak_source": "measured in this run (dt_measure_l2_read_bandwidth, 32 MB x 200 passes, L1 bypassed, best of 5)"}}
    # the traversal is bound by instruction issue (ncu: ~72 % issue-active at
    # 4 % of HBM): its issue rate from the committed instruction count
    iss = ncu_issue(dom)
    if iss is not None:
        sm_mhz = clk.summary().get("sm_mhz") or 2070.0
        roofline["issue"] = issue_roofline(iss[0], iss[1], seg * args.steps / launches, per_launch_ms,
                                           torch.cuda.get_device_properties(dev).multi_processor_count, sm_mhz)
    gpu_launches = int(sum(v[0] * KERNELS_PER_SCOPE.get(k, 1) for k, v in kt.items()))
    kernel_share = {k: round(v[1] / sum(x[1] for x in kt.values()), 4) for k, v in kt.items()}

    # ---- the paper's losses (Eqs. 14-15) as the seed, on the same image ----
    pgrad = torch.empty_like(img)
    ploss = torch.empty(3, device=dev)
    for _ in range(3):
        dt.paper_loss_grad(img, target, 1.0, 1.0, grad=pgrad, loss=ploss)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        dt.paper_loss_grad(img, target, 1.0, 1.0, grad=pgrad, loss=ploss)
    e1.record(stream)
    torch.cuda.synchronize()
    paper_loss = {"ms": e0.elapsed_time(e1) / 10, "pixels": img.numel() // 3,
                  "l2_seed_ms": kt.get("k_l2_loss_grad", (1, 0.0))[1] / max(1, kt.get("k_l2_loss_grad", (1, 0.0))[0])}
    del pgrad, ploss

    # ---- end to end through the public API with host buffers -------------
    e2e = None
    if not args.no_e2e:
        hV = torch.from_numpy(sc.V).pin_memory()
        hior = torch.tensor([sc.ior], dtype=torch.float32).pin_memory()
        hsig = torch.from_numpy(sc.sigma).pin_memory()
        htarget = target.cpu().pin_memory()
        outV = torch.empty_like(hV).pin_memory()
        outs = torch.empty(5, dtype=torch.float32).pin_memory()
        h2d = hV.numel() * 4 + 4 + 12 + htarget.numel() * 4
        d2h = outV.numel() * 4 + 5 * 4

        copy_stream = torch.cuda.Stream(device=dev)

        def e2e_step():
            # the inputs the forward needs first on the compute stream; the
            # target images (the bulk of the bytes) on a copy stream, overlapped
            # with the forward and waited for before the loss
            V.copy_(hV, non_blocking=True)
            ior.copy_(hior, non_blocking=True)
            sigma.copy_(hsig, non_blocking=True)
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                target.copy_(htarget, non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(copy_stream)
            dV, dior, dsig = step(target_ready=ready)
            outV.copy_(dV, non_blocking=True)
            outs[0:1].copy_(dior, non_blocking=True)
            outs[1:4].copy_(dsig, non_blocking=True)
            outs[4:5].copy_(loss, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        tt = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            tt.append(time.perf_counter() - t0)
        (e2e_s,), _ = reduce_over_ranks([sum(tt)], seg, dev)
        e2e = {"value": seg_all * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle as O
        O.build()
        nseg, secs = oracle_sample(sc, Vt_np, args.cpu_sample)
        cpu = {"value": nseg / secs, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "cpu": cpu_model(),
               "sample": f"{args.cpu_sample} seeded pixels of the same workload ({nseg} segments), forward + "
                         f"gradient by forward mode over the parameters those paths touch, {secs:.1f} s"}

    # the serving leg first among the other workloads, right after the main
    # step's buffers are released: its latencies should not inherit the
    # allocator state of the large legs
    serving = None
    if rank == 0 and world == 1:
        del ws, bws, tape
        torch.cuda.empty_cache()
        if not args.no_serve:
            with ClockSampler(dev.index or 0) as clk_s:
                serving = serve_leg(args, dev)
            serving["clocks"] = clk_s.summary()
            torch.cuda.empty_cache()

    c0 = None
    if rank == 0 and world == 1 and not args.no_c0:
        with ClockSampler(dev.index or 0) as clk_c0:
            c0 = c0_leg(args, dt, dev)
        c0["clocks"] = clk_c0.summary()

    large = None
    if rank == 0 and world == 1 and not args.no_large:
        with ClockSampler(dev.index or 0) as clk_large:
            large = large_leg(args, dt, dev)
        large["clocks"] = clk_large.summary()

    medium = None
    if rank == 0 and world == 1 and not args.no_medium:
        with ClockSampler(dev.index or 0) as clk_med:
            medium = medium_leg(args, dt, dev)
        medium["clocks"] = clk_med.summary()

    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        torch.cuda.empty_cache()
        with ClockSampler(dev.index or 0) as clk_b:
            batch = batch_leg(args, dt, dev, max(3, args.steps // 4))
        batch["clocks"] = clk_b.summary()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**workload_config(sc, nvw, res, D, world),
                       "segments_per_step": int(seg_all), "l2": "flushed by a 512 MB write before every timed step",
                       "bvh": "binned SAH" if dt.get_tuning()["bvh_builder"] == 1 else "LBVH",
                       "parallelism": f"replicas over disjoint views x{world}"},
            "fwd_segments_per_s": fwd_value,
            "ms_per_step_fwd": fwd_ms / args.steps,
            "ms_per_step_p50": float(np.percentile(ms, 50)), "ms_per_step_p90": float(np.percentile(ms, 90)),
            "roofline": roofline,
            "kernel_share": kernel_share,
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "levels": stats["level_count"],
            "nodes_per_segment": round(stats["nodes_visited"] / seg, 3),
            "tris_per_segment": round(stats["tris_tested"] / seg, 3),
            "paper_loss": paper_loss,
            "medium": medium,
            # the other workloads last, so that the end of the line (which
            # log tails keep) holds them
            "large": large,
            "batch": batch,
            "c0": c0,
            "serve": serving,
        }
        # a compact digest of every workload last, so that a log tail that
        # keeps only the end of the line still shows each of them
        out["summary"] = summary_digest(out)
        print(json.dumps(out))
    if world > 1:
        tdist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
