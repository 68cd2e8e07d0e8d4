"""Throughput benchmark of the GB300 LSE library.

One step = one pass of the whole hot path over the benchmark scene: the
region-based evolution (Eq. 17, prologue + `iters` fused iterations + output)
and the edge-based one (Eq. 14: edge-indicator precompute + prologue +
`iters` iterations + output), each through the C ABI.  The scene is the
8192 x 8192 single-band rectangle scene (about 2000 roofs, 200 road strips,
noise 0.05), dt = 15, sigma = 1, TS = 9, 300 iterations per term, FP32.
Every plane is 268 MB, larger than L2, so no flush is needed between steps.

Reported (one JSON line on rank 0):
  value        Mpixel-iterations/s over all ranks, inputs resident in HBM;
  e2e          the same with the step's inputs and results in pinned host
               memory, copied by the library inside the timing (region and
               edge term on two streams, the edge evolution ordered after the
               region's, so copies overlap kernels);
  roofline     the region evolution's kernel (one persistent launch for all
               iterations on the tile form): algorithmic bytes per launch
               (12 B/px per iteration: read I, read phi, write v) / its mean
               duration from CUDA events on the library's stream, against
               measured HBM; `gpu_launches` is the library's own count
               (lse_kernel_launches) over the timed steps;
  cpu_baseline the FP64 oracle on the host cores, on crops of the same scene;
  storage_variants  the same workload with BF16 and F16 storage of the data
               term and the LSF (FP32 arithmetic, 6 B/px per region step), and
               each storage type's error against the FP64 oracle on a
               2048 x 2048 crop (mask disagreement, max |v - v_oracle|);
  multiband    the 4-band 2048x2048 scene: vector region term and edge term,
               500 iterations each, CUDA events of lse_evolve
  sizes        per-iteration time of one lse_evolve call on square crops
               (sides 256-4096), region and edge term, FP32
  strips       the row-strip driver with one rank (lse_strip_* per
               iteration) against one lse_evolve call, 4096x4096 region term
  batch        256 uneven images (sides 128-1024, caps 100-600, early stop)
               through lse_evolve_batch with and without a CUDA graph, and
               one lse_evolve call per image in sequence, on a context whose
               tile heights lse_autotune chose on a separate sample;
  serve        Poisson-arriving requests (sides 256-4096, BF16 storage where
               it applies) through lse_server (continuous batching in a
               40 GiB budget) against one lse_evolve call per request, at
               50 and 2000 requests/s offered: p50 / p99 latency and
               requests/s.
`--impl reference` times the FP64 oracle alone (the reference arm).
Under torchrun each rank runs its own replica (no collective on the data
path): weak scaling.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LSE Mpixel-iters/s"
UNIT = "Mpixel-iters/s"
BYTES_PER_PX_ITER = 12            # FP32 single band: I 4 + phi 4 + v 4
WORKLOAD = ("8192x8192 single-band rectangle scene (2000 roofs, 200 road strips, "
            "noise 0.05); region term (Eq. 17) + edge term (Eq. 14, with g "
            "precompute) per step; dt=15 sigma=1 TS=9; 300 iterations each; FP32")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the 16-bit storage variants")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the storage types' error against the FP64 oracle")
    ap.add_argument("--no-sizes", action="store_true",
                    help="skip the per-iteration time of single calls by image side")
    ap.add_argument("--no-strips", action="store_true",
                    help="skip the one-rank row-strip path against lse_evolve")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched uneven-image measurement")
    ap.add_argument("--batch-images", type=int, default=256)
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the continuous-batching serving measurement")
    ap.add_argument("--serve-requests", type=int, default=240)
    ap.add_argument("--serve-rates", default="50,2000",
                    help="offered request rates (per second), comma-separated")
    ap.add_argument("--no-multiband", action="store_true",
                    help="skip the 4-band 2048x2048 measurement")
    ap.add_argument("--multiband-iters", type=int, default=500)
    ap.add_argument("--only-multiband", action="store_true",
                    help="run and print only the 4-band measurement (profiling)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """MAX of a scalar over ranks (identity on one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def scene_inputs(size: int):
    from paper_1409_7474_gb300 import scenes
    sc = scenes.large_scene(size, size, n_roofs=max(1, 2000 * size * size // 8192 ** 2),
                            n_roads=max(1, 200 * size // 8192))
    img = sc["image"]
    phi_r = scenes.circle_phi(size, size, radius=size / 4)
    boxes = [(y0 - 6, x0 - 6, y1 + 6, x1 + 6) for (y0, x0, y1, x1) in sc["roof_boxes"][:200]]
    phi_e = scenes.box_phi(size, size, boxes)
    return img, phi_r, phi_e


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except ValueError:
                pass
        os.remove(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ oracle legs
def _oracle_crop_job(args):
    import oracle
    img, phi_r, phi_e, iters = args
    oracle.evolve(img, phi_r, "region", iterations=iters)
    g = oracle.edge_indicator(img, 1.0, 9, 255.0)
    oracle.evolve(img, phi_e, "edge", g=g, iterations=iters)
    return img.shape[-1] * img.shape[-2] * iters * 2


def oracle_throughput(img, phi_r, phi_e, seconds: float, crop: int = 256):
    """Runs the FP64 oracle (unchanged) on crops of the scene in one thread per
    host core (ctypes releases the GIL) for about `seconds`; Mpixel-iters/s."""
    import oracle
    oracle.build()
    oracle.set_threads(1)     # one thread per crop: the crops run side by side
    cores = os.cpu_count() or 1
    H, W = img.shape[-2:]
    r = np.random.default_rng(0)
    crops = []
    for k in range(cores):
        y = int(r.integers(0, H - crop + 1))
        x = int(r.integers(0, W - crop + 1))
        crops.append((np.ascontiguousarray(img[:, y:y + crop, x:x + crop]),
                      np.ascontiguousarray(phi_r[y:y + crop, x:x + crop]),
                      np.ascontiguousarray(phi_e[y:y + crop, x:x + crop])))
    t = time.perf_counter()
    _oracle_crop_job(crops[0] + (2,))
    per_iter = (time.perf_counter() - t) / 2
    iters = max(2, int(seconds / max(per_iter, 1e-6)))
    t = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as ex:
        work = sum(ex.map(_oracle_crop_job, [c + (iters,) for c in crops]))
    wall = time.perf_counter() - t
    return {"value": work / wall / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} crops of {crop}x{crop} px of the benchmark scene, "
                      f"region + edge term, {iters} iterations each, FP64, one thread "
                      f"per crop"}


def precision_report(torch, lse, dev, img, phi_r, phi_e, crop: int = 2048, iters: int = 300,
                     y0: int = 2048, x0: int = 2048):
    """The error of each storage type against the FP64 oracle on a crop of
    the benchmark scene (the crop is its own problem: both sides run it),
    outside any timed region: the fraction of mask pixels that differ, those
    more than 1 px from the oracle's contour, and max |v - v_oracle| over the
    pixels where the masks agree.  Region term and edge term (g from each
    side's own edge indicator), `iters` iterations."""
    import oracle
    from scipy import ndimage
    sl = (slice(y0, y0 + crop), slice(x0, x0 + crop))
    im = np.ascontiguousarray(img[:, sl[0], sl[1]])
    pr = np.ascontiguousarray(phi_r[sl])
    pe = np.ascontiguousarray(phi_e[sl])
    oracle.build()
    oracle.set_threads(0)
    t = time.perf_counter()
    g_ref = oracle.edge_indicator(im, 1.0, 9, 255.0)
    ref = {"region": oracle.evolve(im, pr, "region", iterations=iters),
           "edge": oracle.evolve(im, pe, "edge", g=g_ref, iterations=iters)}
    oracle_s = time.perf_counter() - t
    cross = ndimage.generate_binary_structure(2, 1)
    out = {"crop": f"{crop}x{crop} at ({y0}, {x0}) of the benchmark scene, {iters} iterations",
           "oracle_seconds": round(oracle_s, 1)}
    with lse.Context(dev.index, max_pixels=crop * crop, max_bands=1) as c:
        x = torch.from_numpy(im).to(dev)
        g = c.precompute_edge(x, 1.0, 9, 255.0)
        for term, phi in (("region", pr), ("edge", pe)):
            v_ref, m_ref, _ = ref[term]
            r = ref_mask = m_ref.astype(bool)
            ring = (ndimage.binary_dilation(r, cross) & ~r) | (r & ~ndimage.binary_erosion(
                r, cross, border_value=1))
            near = ndimage.binary_dilation(ring, np.ones((3, 3), bool))
            out[term] = {}
            for sto in ("f32", "bf16", "f16"):
                v, m, st = c.evolve(x if term == "region" else None,
                                    torch.from_numpy(phi).to(dev), term,
                                    g=g if term == "edge" else None, iterations=iters,
                                    storage=sto)
                v = v.cpu().numpy()
                m = m.cpu().numpy().astype(bool)
                bad = m != ref_mask
                same = ~bad
                out[term][sto] = {
                    "mask_disagree_frac": float(bad.mean()),
                    "mask_disagree_far_px": int((bad & ~near).sum()),
                    "v_max_abs_err_where_masks_agree":
                        float(np.abs(v - v_ref)[same].max()) if same.any() else None,
                    "status": st["status"]}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    img, phi_r, phi_e = scene_inputs(args.size)
    cores = os.cpu_count() or 1
    # the whole run stays near two minutes: each step is a bounded sample
    per_step_seconds = min(20.0, max(2.0, 120.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_throughput(img, phi_r, phi_e, seconds=min(per_step_seconds, 3.0))
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_throughput(img, phi_r, phi_e, seconds=per_step_seconds))
    wall = time.perf_counter() - t0
    value = statistics.mean(v["value"] for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall * 1e3 / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "size": args.size},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def serve_measurement(torch, lse, dev, n_req: int, rates, seed: int = 9,
                      ticks: int = 16, budget: int = 40 << 30):
    """Requests arriving as a Poisson process of uneven images (sides
    log-uniform 256-4096, 1 or 4 bands, region or edge term, caps 100-600,
    early stop at 1e-4 of the pixels; BF16 storage for the single-band and
    edge requests, FP32 for the 4-band region ones, which 16-bit storage does
    not serve), replayed in real time at each offered rate (requests per
    second): through lse_server (continuous batching of the small
    single-band and edge requests, `ticks` iterations per advance, a
    `budget`-byte memory budget; large images alone, one per advance; the
    queued small vector images together as one batch of group launches),
    and one lse_evolve call per request in arrival order with the same
    storage.  Latency = completion - arrival; throughput = requests over
    the makespan; percentiles over all requests of one trial."""
    import time
    from paper_1409_7474_gb300 import scenes
    distinct = max(min(n_req // 2, 48), 1)
    probs = scenes.batch_problems(distinct, seed=seed, min_side=256, max_side=4096)
    ctx = lse.Context(dev.index, max_pixels=4096 * 4096, max_bands=4)
    sample = scenes.batch_problems(max(distinct // 2, 1), seed=seed + 1000, min_side=256,
                                   max_side=4096)
    for q in sample:
        if q["term"] == "edge" or q["image"].shape[0] == 1:
            q["storage"] = "bf16"
    tune = tune_context(torch, lse, ctx, dev, sample)
    base = []
    for q in probs:
        img = torch.from_numpy(q["image"]).to(dev)
        half = q["term"] == "edge" or q["image"].shape[0] == 1
        it = {"phi0": torch.from_numpy(q["phi0"]).to(dev), "term": q["term"],
              "iterations": q["iterations"], "early_stop_frac": q["early_stop_frac"],
              "storage": "bf16" if half else "f32"}
        if q["term"] == "region":
            it["image"] = img
        else:
            it["g"] = ctx.precompute_edge(img, 1.0, 9, 255.0)
        base.append(it)
    items = []
    for k in range(n_req):
        it = dict(base[k % distinct])
        H, W = it["phi0"].shape
        it["phi_out"] = torch.empty((H, W), dtype=torch.float32, device=dev)
        it["mask_out"] = torch.empty((H, W), dtype=torch.uint8, device=dev)
        items.append(it)
    px_it_cap = sum(int(it["phi0"].numel()) * it["iterations"] for it in items)
    torch.cuda.synchronize()

    def wait_until(t0, t):
        while time.perf_counter() - t0 < t:
            pass

    def alone(it, **kw):
        ctx.evolve(it.get("image"), it["phi0"], it["term"], g=it.get("g"),
                   storage=it["storage"], **kw)

    # warm-up of both paths (modules, scratch)
    sv = lse.Server(ctx, budget)
    warm = [sv.submit(dict(it, iterations=2)) for it in base[:4]]
    while warm:
        sv.advance(2)
        warm = [rid for rid in warm if sv.poll(rid) is None]
    for it in base[:4]:
        alone(it, iterations=2)
    torch.cuda.synchronize()
    sv.destroy()

    def summary(lat, span):
        return {"p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "requests_per_s": n_req / span, "makespan_s": float(span)}

    out = {"workload": f"{n_req} requests, Poisson arrivals; sides log-uniform 256-4096, "
                       "1 or 4 bands, region or edge term, caps U{100..600}, early stop "
                       "1e-4; BF16 storage (1 band or edge), FP32 (4-band region); "
                       f"budget {budget >> 30} GiB; {ticks} iterations per advance",
           "pixel_iterations_at_caps": px_it_cap, "autotune": tune, "rates": {}}
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0, size=n_req)
    for rate in rates:
        arrivals = np.cumsum(gaps / rate)
        # continuous batching
        sv = lse.Server(ctx, budget)
        done = np.zeros(n_req)
        t0 = time.perf_counter()
        k, live = 0, {}
        while len(live) or k < n_req:
            now = time.perf_counter() - t0
            while k < n_req and arrivals[k] <= now:
                live[sv.submit(items[k])] = k
                k += 1
            if not live:
                wait_until(t0, arrivals[k])
                continue
            sv.advance(ticks)
            for rid in list(live):
                if sv.poll(rid) is not None:
                    done[live.pop(rid)] = time.perf_counter() - t0
        lat_s = done - arrivals
        span_s = done.max() - arrivals[0]
        sv.destroy()
        # one request at a time
        done_q = np.zeros(n_req)
        t0 = time.perf_counter()
        for k, it in enumerate(items):
            wait_until(t0, arrivals[k])
            alone(it, iterations=it["iterations"], early_stop_frac=it["early_stop_frac"],
                  phi_out=it["phi_out"], mask_out=it["mask_out"])
            done_q[k] = time.perf_counter() - t0
        lat_q = done_q - arrivals
        span_q = done_q.max() - arrivals[0]
        out["rates"][f"{rate:g}/s"] = {"server": summary(lat_s, span_s),
                                       "sequential": summary(lat_q, span_q)}
    ctx.destroy()
    return out


def tune_context(torch, lse, ctx, dev, probs, iterations: int = 16):
    """lse_autotune on a separate sample of the workload's generator: the
    tile height per shape class that the timed runs then use."""
    import time
    items = []
    for q in probs:
        img = torch.from_numpy(q["image"]).to(dev)
        it = {"phi0": torch.from_numpy(q["phi0"]).to(dev), "term": q["term"],
              "iterations": q["iterations"], "storage": q.get("storage", "f32")}
        if q["term"] == "region":
            it["image"] = img
        else:
            it["g"] = ctx.precompute_edge(img, 1.0, 9, 255.0)
        items.append(it)
    t0 = time.perf_counter()
    rows = ctx.autotune(items, iterations=iterations)
    return {"sample_images": len(items), "iterations": iterations,
            "seconds": round(time.perf_counter() - t0, 3),
            "rows_32": rows.count(32), "rows_64": rows.count(64)}


def batch_measurement(torch, lse, dev, n_images: int, seed: int = 3):
    """The uneven-image work list (sides 128-1024, 1 or 4 bands, region or
    edge term, caps 100-600, early stop at 1e-4 of the pixels) run three
    ways on one context: one lse_evolve call per image in sequence, and
    lse_evolve_batch with and without CUDA-graph capture.  Each is timed with
    CUDA events around the whole call (staging, prologues, iterations,
    outputs); g of the edge images is computed beforehand for all three."""
    from paper_1409_7474_gb300 import scenes
    probs = scenes.batch_problems(n_images, seed=seed)
    ctx = lse.Context(dev.index, max_pixels=1024 * 1024, max_bands=4)
    # tuned on an equally large sample of the generator (another seed): the
    # tuner judges each class in a mix as full as the timed one
    tune = tune_context(torch, lse, ctx, dev, scenes.batch_problems(n_images, seed=seed + 1000))
    items = []
    for q in probs:
        img = torch.from_numpy(q["image"]).to(dev)
        it = {"phi0": torch.from_numpy(q["phi0"]).to(dev), "term": q["term"],
              "iterations": q["iterations"], "early_stop_frac": q["early_stop_frac"]}
        H, W = q["phi0"].shape
        it["phi_out"] = torch.empty((H, W), dtype=torch.float32, device=dev)
        it["mask_out"] = torch.empty((H, W), dtype=torch.uint8, device=dev)
        if q["term"] == "region":
            it["image"] = img
        else:
            it["g"] = ctx.precompute_edge(img, 1.0, 9, 255.0)
        items.append(it)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        out = fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1), out

    def sequential():
        runs = []
        for it in items:
            ctx.evolve(it.get("image"), it["phi0"], it["term"], g=it.get("g"),
                       iterations=it["iterations"], early_stop_frac=it["early_stop_frac"],
                       phi_out=it["phi_out"], mask_out=it["mask_out"], sync=False)
            runs.append(None)
        return runs

    ctx.evolve_batch(items, use_graph=False)      # warm-up: scratch, modules
    ms_graph, res = timed(lambda: ctx.evolve_batch(items, use_graph=True))
    ms_direct, _ = timed(lambda: ctx.evolve_batch(items, use_graph=False))
    sequential()
    ms_seq, _ = timed(sequential)
    px_it = sum(int(it["phi0"].numel()) * r[2]["iterations_run"] for it, r in zip(items, res))
    ctx.destroy()
    out = {"workload": f"{n_images} uneven images: sides log-uniform 128-1024, 1 or 4 bands, "
                       "region or edge term, caps U{100..600}, early stop 1e-4",
           "pixel_iterations": px_it, "unit": "Mpixel-iters/s", "autotune": tune}
    for name, ms in (("batch_graph", ms_graph), ("batch_direct", ms_direct),
                     ("sequential", ms_seq)):
        out[name] = {"ms": ms, "value": px_it / (ms / 1e3) / 1e6,
                     "images_per_s": n_images / (ms / 1e3)}
    return out


def step_form() -> str:
    """The region step kernel that runs: the tile form unless LSE_STEP_KERNEL
    narrows the library's choice."""
    return {"stream": "tma", "generic": "generic"}.get(os.environ.get("LSE_STEP_KERNEL", ""),
                                                        "tile")


def multiband_measurement(torch, lse, dev, iters: int, steps: int, peak: float):
    """The 4-band 2048x2048 scene (B, G, R, NIR, uint16 normalised to FP32):
    the vector region term (Eq. 17) and, separately, the edge term on its
    precomputed g, `iters` iterations each through lse_evolve, timed with the
    library's CUDA events.  Bytes per pixel-iteration of the region term as
    the method needs them: the 4 bands, phi in and phi out (24)."""
    from paper_1409_7474_gb300 import scenes
    H = W = 2048
    sc = scenes.multiband_scene(H, W, 4, seed=7)
    x = (torch.from_numpy(sc["image"].astype(np.int32)).to(dev).float() / 65535.0).contiguous()
    phi_r = torch.from_numpy(scenes.circle_phi(H, W, radius=512)).to(dev)
    y0, x0, y1, x1 = sc["runway_box"]
    phi_e = torch.from_numpy(scenes.box_phi(H, W, [(y0 - 20, x0 - 20, y1 + 20, x1 + 20)])).to(dev)
    out = {}
    with lse.Context(dev.index, max_pixels=H * W, max_bands=4) as c:
        g = c.precompute_edge(x, 1.0, 9, 255.0)
        for name, img, phi, term in (("region", x, phi_r, "region"), ("edge", None, phi_e, "edge")):
            kw = dict(g=g) if term == "edge" else {}
            c.evolve(img, phi, term, iterations=iters, **kw)          # warm-up
            ms = []
            for _ in range(max(1, steps)):
                _, _, st = c.evolve(img, phi, term, iterations=iters, **kw)
                ms.append(st["elapsed_ms"])
            best = statistics.median(ms)
            out[name] = {"us_per_iter": best / iters * 1e3,
                         "value": H * W * iters / (best / 1e3) / 1e6,
                         "status": st["status"], "iterations_run": st["iterations_run"]}
        torch.cuda.synchronize()
    alg = 24 * H * W
    out["region"]["bytes_per_iter"] = alg
    out["region"]["frac"] = alg / (out["region"]["us_per_iter"] / 1e6) / 1e9 / peak
    out["workload"] = (f"2048x2048 4-band uint16 scene normalised to FP32; vector region term "
                       f"and edge term, {iters} iterations each, dt=15 sigma=1 TS=9")
    out["unit"] = UNIT
    return out


def sizes_measurement(torch, lse, dev, iters: int = 200):
    """Per-iteration time of one lse_evolve on square crops of the benchmark
    scene (sides 256-4096), region and edge term, FP32, `iters` iterations,
    the library's CUDA events (best of 3): what one call costs when the image
    is too small to fill the GPU."""
    from paper_1409_7474_gb300 import scenes
    out = {"workload": f"square crops of the benchmark scene, {iters} iterations, "
                       "FP32, dt=15 sigma=1 TS=9; one lse_evolve call each",
           "unit": "us per iteration", "sides": {}}
    big = 4096
    img = scenes.large_scene(big, big, n_roofs=500, n_roads=50)["image"]
    with lse.Context(dev.index, max_pixels=big * big, max_bands=1) as c:
        for side in (256, 512, 1024, 2048, 4096):
            x = torch.from_numpy(np.ascontiguousarray(img[:, :side, :side])).to(dev)
            pr = torch.from_numpy(scenes.circle_phi(side, side, radius=side / 4)).to(dev)
            pe = torch.from_numpy(scenes.box_phi(side, side, [(4, 4, side - 4, side - 4)])).to(dev)
            g = c.precompute_edge(x, 1.0, 9, 255.0)
            row = {}
            for term, phi in (("region", pr), ("edge", pe)):
                kw = {"g": g} if term == "edge" else {}
                src = x if term == "region" else None
                c.evolve(src, phi, term, iterations=iters, **kw)         # warm-up
                ms = min(c.evolve(src, phi, term, iterations=iters, **kw)[2]["elapsed_ms"]
                         for _ in range(3))
                row[term] = ms / iters * 1e3
            row["region_mpx_it_s"] = side * side / row["region"]
            out["sides"][str(side)] = row
        torch.cuda.synchronize()
    return out


def strips_measurement(torch, lse, dev, size: int = 4096, iters: int = 50):
    """The row-strip path on one GPU: the strip driver with one rank
    (`strips.LocalComm`, the library's lse_strip_* calls: exact partial sums,
    one strip step and a host synchronisation per iteration) against one
    lse_evolve call on the same image, region term, FP32.  What a rank of
    a split evolution pays for stepping one launch at a time with
    host-visible statistics; no collective runs (one GPU)."""
    import time
    from paper_1409_7474_gb300 import scenes, strips
    img = scenes.large_scene(size, size, n_roofs=500, n_roads=50)["image"]
    phi0 = scenes.circle_phi(size, size, radius=size / 4)
    x = torch.from_numpy(img).to(dev)
    p0 = torch.from_numpy(phi0).to(dev)
    out = {"workload": f"{size}x{size} crop of the benchmark scene's generator, region "
                       f"term, {iters} iterations, FP32; one rank",
           "unit": "us per iteration"}
    with lse.Context(dev.index, max_pixels=size * size, max_bands=1) as c:
        part = strips.partition(size, size, 9, 0, 1)
        comp = strips.LibraryCompute(c, part, x, term="region")
        runs = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            strips.evolve(strips.LocalComm(), comp, part, p0, term="region",
                          iterations=iters)
            torch.cuda.synchronize()
            runs.append((time.perf_counter() - t0) / iters * 1e6)
        out["strip_driver"] = min(runs)
        ms = min(c.evolve(x, p0, "region", iterations=iters)[2]["elapsed_ms"] for _ in range(3))
        out["lse_evolve"] = ms / iters * 1e3
    return out


def kernel_profile(size: int, name: str, iterations: int):
    """DRAM traffic per launch of the region kernel `name` from a committed ncu
    summary (profiles/<name>_region_traffic.json), if it was taken on the
    current kernel source; scaled to `size` x `size` pixels and `iterations`
    steps per launch (traffic grows with both)."""
    path = os.path.join(ROOT, "profiles", f"{name}_region_traffic.json")
    try:
        prof = json.load(open(path))
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for rel in prof.get("hashed_sources", []):
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    digest = h.hexdigest()[:16]
    if prof.get("kernel_sha256_16") != digest:
        return None
    per_px_step = prof["dram_bytes_per_launch"] / prof["pixels"] / prof.get("iterations", 1)
    return per_px_step * size * size * iterations


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_1409_7474_gb300.lse as lse

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    if args.only_multiband:
        if rank == 0:
            mb = multiband_measurement(torch, lse, dev, args.multiband_iters, args.steps, peak)
            print(json.dumps({"impl": "gb300", "multiband": mb}))
        return 0

    size, iters = args.size, args.iters
    img, phi_r, phi_e = scene_inputs(size)
    npx = size * size
    px_iters_per_step = npx * iters * 2

    ctx_r = lse.Context(local, max_pixels=npx, max_bands=1)
    ctx_e = lse.Context(local, max_pixels=npx, max_bands=1)
    x = torch.from_numpy(img).to(dev)
    pr = torch.from_numpy(phi_r).to(dev)
    pe = torch.from_numpy(phi_e).to(dev)
    out_r = torch.empty((size, size), dtype=torch.float32, device=dev)
    mask_r = torch.empty((size, size), dtype=torch.uint8, device=dev)
    out_e = torch.empty_like(out_r)
    mask_e = torch.empty_like(mask_r)
    g = torch.empty_like(out_r)
    stream = torch.cuda.current_stream(dev)
    common = dict(dt=15.0, sigma=1.0, ts=9, iterations=iters, sync=False)

    def step():
        ctx_r.evolve(x, pr, "region", phi_out=out_r, mask_out=mask_r, **common)
        ctx_e.precompute_edge(x, 1.0, 9, 255.0, out=g)
        ctx_e.evolve(None, pe, "edge", g=g, phi_out=out_e, mask_out=mask_e, **common)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms_r, step_ms_e = [], []
    launches0 = ctx_r.kernel_launches() + ctx_e.kernel_launches()
    region_launches0 = ctx_r.kernel_launches()
    with ClockSampler(local) as clocks:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(args.steps):
            step()
            torch.cuda.synchronize()      # makes the library's loop events readable
            step_ms_r.append(ctx_r.stats()["elapsed_ms"])
            step_ms_e.append(ctx_e.stats()["elapsed_ms"])
        t1.record(stream)
        torch.cuda.synchronize()
    launches = ctx_r.kernel_launches() + ctx_e.kernel_launches() - launches0
    region_per_call = (ctx_r.kernel_launches() - region_launches0) // args.steps
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    st_r, st_e = ctx_r.stats(), ctx_e.stats()
    value = world * px_iters_per_step * args.steps / (ms / 1e3) / 1e6

    # The region evolution's step kernel.  On the tile form every iteration
    # runs in one persistent launch (prologue + 1 + output = 3 kernels per
    # call); otherwise one launch per iteration.  The library's CUDA events
    # bracket the iteration loop on its stream, so their time is the
    # launch's (or the launches') own.
    loop_ms = statistics.mean(step_ms_r)
    step_kernel_ms = loop_ms / iters
    alg_step = BYTES_PER_PX_ITER * npx
    edge_kernel_ms = statistics.mean(step_ms_e) / iters
    persistent = region_per_call == 3
    form = step_form()
    if persistent:
        kname, per_launch = "evolve_tile", iters
    else:
        kname, per_launch = f"step_{form}", 1
    roofline = {"bound": "hbm", "achieved": alg_step / (step_kernel_ms / 1e3) / 1e9,
                "peak": peak, "unit": "GB/s",
                "frac": alg_step / (step_kernel_ms / 1e3) / 1e9 / peak,
                "traffic": kernel_profile(size, kname, per_launch),
                "kernel": f"{kname}_kernel<region, r=4>", "peak_source": peak_src,
                "iterations_per_launch": per_launch,
                "bytes_per_launch": alg_step * per_launch,
                "mean_launch_ms": step_kernel_ms * per_launch,
                "bytes_per_step": alg_step, "step_ms": step_kernel_ms,
                "edge_kernel_frac": alg_step / (edge_kernel_ms / 1e3) / 1e9 / peak}

    # e2e: the step's inputs (image, both initial LSFs) and results (v and
    # mask of both terms) are pinned host buffers passed to the C ABI, which
    # copies them in and out inside the timed region.  The edge indicator g
    # is an intermediate between two calls and stays on the device.  Three
    # streams, one context each: the region evolution, the edge precompute
    # and the edge evolution.  The library runs its persistent evolutions
    # one at a time, each after the previous one's output kernel, and issues
    # a call's host copies before its kernels, so one term's copies overlap
    # the other term's evolution.  The edge precompute runs one step ahead
    # into a second g buffer (its kernels fill a gap between evolutions
    # instead of holding back the edge evolution's copies); every timed step
    # still runs one precompute.
    e2e = None
    if not args.no_e2e:
        hx = torch.from_numpy(img).pin_memory()
        hpr = torch.from_numpy(phi_r).pin_memory()
        hpe = torch.from_numpy(phi_e).pin_memory()
        ho_r = torch.empty((size, size), dtype=torch.float32).pin_memory()
        hm_r = torch.empty((size, size), dtype=torch.uint8).pin_memory()
        ho_e = torch.empty_like(ho_r).pin_memory()
        hm_e = torch.empty_like(hm_r).pin_memory()
        dgs = [torch.empty((size, size), dtype=torch.float32, device=dev) for _ in range(2)]
        ctx_g = lse.Context(local, max_pixels=npx, max_bands=1)
        s_r = torch.cuda.Stream(dev)
        s_g = torch.cuda.Stream(dev)
        s_e = torch.cuda.Stream(dev)
        g_ready = [None, None]      # precompute of each g buffer done
        g_used = [None, None]       # the edge evolution that last read it
        n_host = [0]

        def precompute(k):
            if g_used[k % 2] is not None:
                s_g.wait_event(g_used[k % 2])
            ctx_g.precompute_edge(hx, 1.0, 9, 255.0, out=dgs[k % 2], stream=s_g)
            ev = torch.cuda.Event()
            ev.record(s_g)
            g_ready[k % 2] = ev

        def step_host():
            k = n_host[0]
            n_host[0] += 1
            ctx_r.evolve(hx, hpr, "region", phi_out=ho_r, mask_out=hm_r, stream=s_r, **common)
            precompute(k + 1)
            s_e.wait_event(g_ready[k % 2])
            ctx_e.evolve(None, hpe, "edge", g=dgs[k % 2], phi_out=ho_e, mask_out=hm_e,
                         stream=s_e, **common)
            done = torch.cuda.Event()
            done.record(s_e)
            g_used[k % 2] = done

        precompute(0)
        step_host()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sx in (s_r, s_g, s_e):
            sx.wait_event(e0)
        for _ in range(args.steps):
            step_host()
        for sx in (s_r, s_g, s_e):
            ev = torch.cuda.Event()
            ev.record(sx)
            stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), world, dev)
        for c in (ctx_r, ctx_e):
            assert c.stats()["status"] == "LSE_OK", c.stats()["status"]
        ctx_g.destroy()
        plane = npx * 4
        e2e = {"value": world * px_iters_per_step * args.steps / (ems / 1e3) / 1e6,
               "unit": UNIT,
               # image and phi0 (region), image (edge precompute), phi0 (edge)
               "h2d_bytes_per_step": 4 * plane,
               # v + mask (region), v + mask (edge)
               "d2h_bytes_per_step": 2 * plane + 2 * npx,
               "streams": "region evolution, edge precompute and edge evolution on three "
                          "streams (the library runs the persistent evolutions one at a "
                          "time, each after the previous one's output kernel, and issues a "
                          "call's host copies before its kernels); the edge precompute runs "
                          "one step ahead into a second g buffer; host buffers for inputs "
                          "and results"}

    # the same workload with 16-bit storage of the data term and the LSF
    # (FP32 arithmetic): 6 bytes per pixel-iteration of the region step
    variants = None
    if not args.no_variants:
        variants = {}
        for sto in ("bf16", "f16"):
            vcommon = dict(common, storage=sto)

            def vstep():
                ctx_r.evolve(x, pr, "region", phi_out=out_r, mask_out=mask_r, **vcommon)
                ctx_e.precompute_edge(x, 1.0, 9, 255.0, out=g)
                ctx_e.evolve(None, pe, "edge", g=g, phi_out=out_e, mask_out=mask_e, **vcommon)

            vstep()
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            v_ms_r, v_ms_e = [], []
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            for _ in range(args.steps):
                vstep()
                torch.cuda.synchronize()
                v_ms_r.append(ctx_r.stats()["elapsed_ms"])
                v_ms_e.append(ctx_e.stats()["elapsed_ms"])
            q1.record(stream)
            torch.cuda.synchronize()
            vms = max_over_ranks(q0.elapsed_time(q1), world, dev)
            kms = statistics.mean(v_ms_r) / iters
            vbytes = 6 * npx
            variants[sto] = {
                "value": world * px_iters_per_step * args.steps / (vms / 1e3) / 1e6,
                "ms_per_step": vms / args.steps,
                "region_step_ms": kms,
                "bytes_per_launch": vbytes,
                "frac": vbytes / (kms / 1e3) / 1e9 / peak,
                "edge_step_frac": vbytes / (statistics.mean(v_ms_e) / iters / 1e3) / 1e9 / peak,
                "status": [ctx_r.stats()["status"], ctx_e.stats()["status"]]}

    if variants is not None and not args.no_precision and rank == 0 and world == 1:
        variants["error_vs_oracle"] = precision_report(torch, lse, dev, img, phi_r, phi_e)

    multiband = None
    if not args.no_multiband and world == 1:
        multiband = multiband_measurement(torch, lse, dev, args.multiband_iters, args.steps,
                                          peak)

    sizes = None
    if not args.no_sizes and rank == 0 and world == 1:
        sizes = sizes_measurement(torch, lse, dev)
    strip_leg = None
    if not args.no_strips and rank == 0 and world == 1:
        strip_leg = strips_measurement(torch, lse, dev)
    batch = None
    if not args.no_batch:
        batch = batch_measurement(torch, lse, dev, args.batch_images)
    serve = None
    if not args.no_serve and world == 1:
        serve = serve_measurement(torch, lse, dev, args.serve_requests,
                                  [float(r) for r in args.serve_rates.split(",") if r])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_throughput(img, phi_r, phi_e, seconds=args.cpu_seconds)

    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "size": size, "iterations": iters,
                           "l2": "inputs larger than L2 (268 MB per plane), no flush",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks.summary(), "gpu_launches": launches,
                "storage_variants": variants, "multiband": multiband, "sizes": sizes,
                "strips": strip_leg,
                "batch": batch,
                "serve": serve,
                "impl": "gb300",
                "stats": {"region": {k: st_r[k] for k in ("iterations_run", "status",
                                                          "last_flips", "area_plus")},
                          "edge": {k: st_e[k] for k in ("iterations_run", "status",
                                                        "last_flips", "area_plus")}}}
        print(json.dumps(line))
    ctx_r.destroy()
    ctx_e.destroy()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
