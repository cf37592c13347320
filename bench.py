#!/usr/bin/env python
"""Benchmark of the RTSDF SDF update on one GB300.

Workload (one step = one animated frame of the whole SDF update):
  coarse 256^3 / fine 512^3 fp32, 500 displaced UV spheres (1,000,000
  triangles), every object translated by a random vector of length <= 0.5
  coarse voxel per frame; per frame: move objects, BVH rebuild (binned SAH), voxelize,
  jump flood (8 passes), mask + reset in changed regions, trace 64 Philox
  rays per masked fine texel with the Eq. 1 update.

Metric: SDF update ms/frame (lower is better), with traced rays/s and the
jump-flood HBM GB/s reported beside it.  Inputs are synthetic (procedural
scene, seeded), resident in HBM before the timed region; the fine grids
(3 x 512 MB) exceed the 129 MB L2, so no explicit flush is needed.

--impl reference times the CPU oracle (oracle/) on the host cores on a
bounded sample of the same frame, extrapolated to ms/frame.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SDF update ms/frame at 256^3->512^3 (animated ~1M tris, 64 rays/texel); traced rays/s; JFA HBM GB/s"
UNIT = "ms/frame"
NC, D_VOX, BETA, RAYS, SEED = 256, 2.0, 0.5, 64, 2
N_OBJ = 500

# Algorithmic fp32 work of the tracer as the scope table counts it: 24 flop
# per internal node visited (two slab tests, 6 fma each, counted as 2 flops)
# and 30 per ray-triangle test.
FLOP_PER_VISIT = 24
FLOP_PER_TEST = 30

# Warp instructions per traced ray of k_trace on the benchmark workload, from
# an ncu capture of smsp__inst_executed.sum on one full-size launch (1 pass),
# keyed like TRAFFIC below; the tracer's issue-roof fraction is computed from
# it (null once the sources change).
INST_PER_RAY = {
    # ncu --metrics smsp__inst_executed.sum,gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
    # -k regex:k_trace -c 1 on "bench.py --steps 2 --warmup 1 --no-cpu-baseline --no-batch --no-variant
    # --no-configs" (1 pass; the first frame's launch, 374.85 ms): 372,760,948,333 warp instructions over
    # 2,557,074 masked voxels x 8 texels x 64 rays = 1,309,221,888 rays
    "4585f2179a4ae7de": 284.72,
}

# DRAM bytes per launch of the tracer, from an ncu capture (profiles/), keyed
# by the sha256 of the sources it was measured on (the kernel and the BVH
# builders, whose tree it walks); reported as null once any of them changes.
TRAFFIC = {
    # the same capture as INST_PER_RAY above (first k_trace<0, 1> launch, SAH tree): 10.76 GB read +
    # 174.75 MB written
    "4585f2179a4ae7de": 10.76e9 + 174.75e6,
}
TRAFFIC_SOURCES = ("trace.cu", "trace_dev.cuh", "bvh.cu", "bvh_sah.cu")


def _src_hash(*names):
    h = hashlib.sha256()
    for name in names:
        p = os.path.join(ROOT, "paper_2210_04449_gb300", "csrc", name)
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def reduce_max(x, world, device=None):
    """Largest value of x over the ranks (every rank gets it): replicas are
    timed by the slowest one.  Any torch.distributed backend: pass a CUDA
    device for NCCL, None for gloo."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_frame(ms_frame_slowest, world):
    """Whole-job ms per frame of `world` replicas that each run one frame per
    step: world frames every ms_frame_slowest."""
    return ms_frame_slowest / max(int(world), 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rtsdf", choices=["rtsdf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form comparison")
    ap.add_argument("--no-variant", action="store_true", help="skip the nearest-face sign variant comparison")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the room (128^3 -> 256^3, 8 frames) and differentiable-shadow (512^3) lines")
    ap.add_argument("--bvh", default="rebuild", choices=["rebuild", "refit"],
                    help="per-frame BVH maintenance: full rebuild (default) or refit of the first frame's tree")
    ap.add_argument("--builder", default="sah", choices=["sah", "lbvh", "two_level"],
                    help="BVH topology: binned SAH (default), Morton radix tree, or two-level (per-object SAH subtrees under a top tree that a refit rebuilds)")
    ap.add_argument("--objects", type=int, default=N_OBJ, help="sphere count (500 = the 1M-triangle workload)")
    ap.add_argument("--coarse-n", type=int, default=NC, help="coarse grid size (256 = the benchmark workload; "
                                                              "smaller only for profiling captures)")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world):
    import numpy as np
    import torch

    from paper_2210_04449_gb300 import RTSDF
    from synth import scenes as S

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    mesh = S.animated_scene(SEED, n_objects=args.objects)
    n_frames = args.warmup + args.steps
    nc = args.coarse_n
    trans = np.stack([S.object_translations(SEED, t, mesh.n_objects, 0.5 / nc) for t in range(n_frames + 1)])
    trans_dev = torch.tensor(trans, device=dev)
    stream = torch.cuda.current_stream(dev)

    rt = RTSDF(nc, beta_vox=BETA, seed=SEED)
    rt.set_bvh_builder(args.builder)
    rt.upload_mesh(mesh.verts, mesh.tris)
    rt.set_objects(mesh.vert_object, mesh.n_objects)
    rt.build_bvh()

    def frame(t, tr):
        if t > 0:
            rt.move_objects(tr)
            rt.build_bvh(refit=args.bvh == "refit")
        rt.voxelize()
        rt.jfa()
        rt.trace(D_VOX, RAYS, t)

    frame(0, None)
    # launch parameters from the autotuner (untimed; the accumulated SDF is
    # saved and restored by it)
    tuning = rt.autotune(D_VOX, RAYS, 1, use_cache=True)
    for t in range(1, args.warmup + 1):
        frame(t, trans_dev[t])
    rt.sync()
    rt.set_profiling(True)
    rt.stats()                          # reset the per-stage sums
    launches0 = rt.stats()["launches"]

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(dev.index)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for t in range(args.warmup + 1, args.warmup + 1 + args.steps):
        frame(t, trans_dev[t])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    st = rt.stats()
    launches = st["launches"] - launches0
    rt.sync()
    n_masked_tex = st["n_masked_texels"]
    ms_total = reduce_max(ms_total, world, dev)
    ms_frame = ms_total / args.steps
    stage = {k: (v / args.steps if st["stage_calls"][k] else None) for k, v in st["stage_ms"].items()}

    # one counted frame (not timed): tracer work per ray
    rt.set_profiling(False)
    rt.set_counting(True)
    tnext = args.warmup + 1 + args.steps
    frame(tnext, trans_dev[min(tnext, n_frames)])
    cnt = rt.stats()
    rt.set_counting(False)

    # end-to-end through the public API with host buffers: per frame the
    # translations go host (pinned) -> device, and the frame's result
    # (masked-texel count and device status) comes back to the host
    trans_host = torch.tensor(trans, dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        t = tnext + 1 + i
        frame(t, trans_host[(t % n_frames) or 1])
        rt.masked_count()
        rt.sync()
    e2e_ms = reduce_max((time.perf_counter() - t0) * 1e3 / e2e_steps, world, dev)

    # Sec. 2.3 on the frame's fine SDF: 1920x1080 floor points, one light,
    # k = 8, 64 steps (forward) and the adjoint at 1024x1024
    shadow = time_shadow(rt, dev)

    rays_frame = n_masked_tex * RAYS
    trace_ms = stage["trace"]
    jfa_ms = stage["jfa"]
    passes = math.ceil(math.log2(nc))
    jfa_bytes = passes * nc ** 3 * 8 + nc ** 3 * 4
    jfa_gbs = jfa_bytes / (jfa_ms * 1e-3) / 1e9 if jfa_ms else None

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = sms * 128 * 2 * sm_mhz * 1e6 / 1e12

    visits_per_ray = cnt["node_visits"] / max(cnt["rays"], 1)
    tests_per_ray = cnt["tri_tests"] / max(cnt["rays"], 1)
    # node entries include the leaves; a leaf entry is one triangle test
    flop_per_ray = (visits_per_ray - tests_per_ray) * FLOP_PER_VISIT + tests_per_ray * FLOP_PER_TEST
    trace_tflops = rays_frame * flop_per_ray / (trace_ms * 1e-3) / 1e12 if trace_ms else None
    th = _src_hash(*TRAFFIC_SOURCES)
    traffic = TRAFFIC.get(th)
    # the roof that binds the tracer: instruction issue, 4 schedulers per SM
    issue_peak = sms * 4 * sm_mhz * 1e6 / 1e9          # G warp instructions / s
    ipr = INST_PER_RAY.get(th) if nc == NC and args.objects == N_OBJ else None
    issue = None
    if ipr and trace_ms:
        ach = ipr * rays_frame / (trace_ms * 1e-3) / 1e9
        issue = {"bound": "issue", "achieved": round(ach, 1), "peak": round(issue_peak, 1),
                 "unit": "G warp-instructions/s", "frac": round(ach / issue_peak, 4),
                 "inst_per_ray": ipr,
                 "source": "ncu smsp__inst_executed.sum of one full-size k_trace launch / its rays, "
                           f"x rays / trace ms; peak {sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz"}

    # mask + fill + reset: the scope table's bytes are the fine write and the
    # coarse seed read (the reset test and the accumulator reads of masked
    # texels come on top)
    mask_ms = stage["mask"]
    mask_bytes = (2 * nc) ** 3 * 4 + nc ** 3 * 4
    mask_gbs = mask_bytes / (mask_ms * 1e-3) / 1e9 if mask_ms else None
    mask_line = {"ms": round(mask_ms, 4) if mask_ms else None, "algorithmic_bytes": mask_bytes,
                 "gbs": round(mask_gbs, 1) if mask_gbs else None, "peak_gbs": hbm_peak,
                 "frac": round(mask_gbs / hbm_peak, 4) if mask_gbs else None, "peak_source": hbm_src}

    line = {
        "metric": METRIC,
        "value": round(job_ms_per_frame(ms_frame, world), 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_frame, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded procedural scene: 500 displaced UV spheres, random rigid motion)",
        "config": dict(workload_config(nc, mesh.n_objects, mesh.nt),
                       bvh=f"per-frame {args.bvh} ({args.builder})",
                       parallelism="replicas" if world > 1 else "single GPU",
                       l2=f"inputs larger than L2 (fine grids 3 x {(2 * nc) ** 3 * 4 >> 20} MB)"),
        "gpu_launches": int(launches),
        "rays_per_s": round(rays_frame / (trace_ms * 1e-3)) if trace_ms else None,
        "masked_texels": int(n_masked_tex),
        "stage_ms": {k: (round(v, 4) if v is not None else None) for k, v in stage.items()},
        "jfa": {"ms": round(jfa_ms, 4) if jfa_ms else None, "passes": passes,
                "algorithmic_bytes": jfa_bytes, "gbs": round(jfa_gbs, 1) if jfa_gbs else None,
                "peak_gbs": hbm_peak, "frac": round(jfa_gbs / hbm_peak, 4) if jfa_gbs else None,
                "peak_source": hbm_src},
        "mask": mask_line,
        "tracer": {"node_visits_per_ray": round(visits_per_ray, 2), "tri_tests_per_ray": round(tests_per_ray, 2),
                   "flop_per_ray": round(flop_per_ray, 1),
                   # SIMT use of the traversal loop: lanes entering an internal
                   # node per node step, lanes testing a triangle per leaf round
                   "node_lanes_per_step": round(32 * (cnt["node_visits"] - cnt["tri_tests"])
                                                / max(cnt["lane_slots"], 1), 2),
                   "leaf_lanes_per_round": round(32 * cnt["tri_tests"] / max(cnt["leaf_slots"], 1), 2),
                   "leaf_rounds_per_node_step": round(cnt["leaf_slots"] / max(cnt["lane_slots"], 1), 3)},
        "roofline": {"kernel": "k_trace", "bound": "alu",
                     "achieved": round(trace_tflops, 3) if trace_tflops else None,
                     "peak": round(fp32_peak_tflops, 2), "unit": "TFLOP/s",
                     "frac": round(trace_tflops / fp32_peak_tflops, 4) if trace_tflops else None,
                     "traffic": traffic,
                     "count": f"{FLOP_PER_VISIT} flop per internal node visit, {FLOP_PER_TEST} per triangle test",
                     "peak_source": f"derived: {sms} SMs x 128 fp32 lanes x 2 x {sm_mhz:.0f} MHz (sampled)",
                     "issue": issue},
        "clocks": clk,
        "e2e": {"value": round(job_ms_per_frame(e2e_ms, world), 3), "unit": UNIT, "h2d_bytes_per_step": N_OBJ * 3 * 4,
                "d2h_bytes_per_step": 8 + 4},
        "shadow": shadow,
        "tuning": tuning,
    }
    rt.close()
    return line, n_masked_tex


def time_shadow(rt, dev, reps=5):
    """Shadow forward (1920x1080), adjoint (1024x1024), jittered forward +
    TAA resolve (1920x1080), the resolve alone, and the thin-surface
    fallback (exact occlusion toward the light, 1920x1080), on the
    context's fine SDF and BVH; CUDA events over `reps` launches each."""
    import torch

    from synth import scenes as S
    out = {}
    L = (0.4, 1.0, 0.3)
    for name, (w, h) in (("forward", (1920, 1080)), ("backward", (1024, 1024)),
                         ("jittered_taa", (1920, 1080)), ("taa", (1920, 1080)), ("fallback", (1920, 1080))):
        pos, nrm = S.floor_gbuffer(w, h, y=0.02)
        pos_t, nrm_t = torch.tensor(pos, device=dev), torch.tensor(nrm, device=dev)
        vis = torch.empty((h, w), device=dev)
        hist = torch.zeros((h, w), device=dev)
        frame = [0]
        if name == "backward":
            dvis = torch.full((h, w), 1.0 / (w * h), device=dev)
            dsdf = torch.zeros(rt.fine_n ** 3, device=dev)
            dl = torch.zeros(3, device=dev)

        def once():
            if name == "forward":
                rt.shadow(pos_t, nrm_t, L, k=8.0, steps=64, out=vis)
            elif name == "backward":
                rt.shadow_backward(pos_t, nrm_t, L, dvis, dsdf, dl, k=8.0, steps=64)
            elif name == "jittered_taa":
                # one displayed frame: origin jittered by up to 2 texels, then the resolve
                rt.shadow(pos_t, nrm_t, L, k=8.0, steps=64, out=vis, jitter_vox=2.0, frame=frame[0])
                rt.taa_resolve(vis, hist, 1.0 if frame[0] == 0 else 0.1)
                frame[0] += 1
            elif name == "taa":
                rt.taa_resolve(vis, hist, 0.1)
            else:
                rt.shadow_fallback(pos_t, nrm_t, L, vis.view(-1))
        if name == "fallback":
            rt.shadow(pos_t, nrm_t, L, k=8.0, steps=64, out=vis)
        once()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            once()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": round(ms, 4), "points": w * h, "points_per_s": round(w * h / (ms * 1e-3))}
    rt.sync()
    return out


def run_sign_variant(dev, frames=8, rays=RAYS, nc=128):
    """The nearest-face sign variant (rays capped at the texel's running
    minimum) against Sec. 2.2's vote on the static room scene (128^3 ->
    256^3, ~100k triangles): trace ms of the first frame and of the later
    frames, work per ray from a counted last frame, and how the two compare
    (the distances must be identical, the signs may differ)."""
    import numpy as np

    from paper_2210_04449_gb300 import RTSDF
    from synth import scenes as S
    mesh = S.room_scene(1)
    out, grids = {}, {}
    for mode in ("vote", "nearest"):
        rt = RTSDF(nc, beta_vox=BETA, seed=SEED)
        rt.set_sign_mode(mode)
        rt.upload_mesh(mesh.verts, mesh.tris)
        rt.build_bvh()
        rt.set_profiling(True)
        per = []
        for f in range(frames):
            last = f == frames - 1
            rt.set_counting(last)
            rt.stats()
            rt.update(D_VOX, rays, f)
            rt.sync()
            st = rt.stats()
            if not last:
                per.append(st["stage_ms"]["trace"])
            else:
                cnt = st
        rt.set_counting(False)
        g = rt.grids()
        grids[mode] = (g["accum"].cpu().numpy(), g["fine"].cpu().numpy())
        out[mode] = {"first_frame_trace_ms": round(per[0], 3),
                     "later_frames_trace_ms": round(float(np.mean(per[2:])), 3),
                     "node_visits_per_ray": round(cnt["node_visits"] / max(cnt["rays"], 1), 2),
                     "tri_tests_per_ray": round(cnt["tri_tests"] / max(cnt["rays"], 1), 2)}
        rt.close()
    uv, fv = grids["vote"]
    un, fn = grids["nearest"]
    hit = np.isfinite(uv)
    out["workload"] = (f"static room {nc}^3->{2 * nc}^3, {mesh.nt:,} tris, {rays} rays/texel, {frames} frames "
                       f"(later = frames 2..{frames - 2}; the last frame is counted, untimed)")
    out["distances_identical"] = bool(np.array_equal(uv, un))
    out["sign_agreement"] = round(float(np.mean(np.sign(fv[hit]) == np.sign(fn[hit]))), 5) if hit.any() else None
    out["later_frames_speedup"] = round(out["vote"]["later_frames_trace_ms"]
                                        / max(out["nearest"]["later_frames_trace_ms"], 1e-9), 2)
    return out


def _events_ms(fn, reps, dev):
    """Mean ms of fn() over reps calls, CUDA events on the current stream."""
    import torch
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / reps


def run_config2(dev, frames=8, warm=3, rays=RAYS, nc=128):
    """The procedural room (~100k triangles) at 128^3 -> 256^3, 64 rays per
    texel, 8 frames of the plain pipeline (voxelize, JFA, mask, trace with
    Eq. 1); ms/frame over the frames after the first `warm`, then the soft
    shadow pass at 1920x1080 (k = 8, 64 steps) on the frame's fine SDF."""
    import numpy as np
    import torch

    from paper_2210_04449_gb300 import RTSDF
    from synth import scenes as S
    mesh = S.room_scene(1)
    rt = RTSDF(nc, beta_vox=BETA, seed=1)
    rt.upload_mesh(mesh.verts, mesh.tris)
    rt.build_bvh()
    rt.set_profiling(True)
    per, trace = [], []
    for f in range(frames):
        rt.stats()
        ms = _events_ms(lambda: rt.update(D_VOX, rays, f), 1, dev)
        st = rt.stats()
        if f >= warm:
            per.append(ms)
            trace.append(st["stage_ms"]["trace"])
    m_tex = rt.masked_count() * 8
    pos, nrm = S.floor_gbuffer(1920, 1080, y=0.02)
    pt, nt = torch.tensor(pos, device=dev), torch.tensor(nrm, device=dev)
    vis = torch.empty((1080, 1920), device=dev)
    L = (0.4, 1.0, 0.3)
    rt.shadow(pt, nt, L, k=8.0, steps=64, out=vis)
    sh = _events_ms(lambda: rt.shadow(pt, nt, L, k=8.0, steps=64, out=vis), 5, dev)
    rt.sync()
    rt.close()
    tr = float(np.mean(trace))
    return {"workload": f"static room {nc}^3->{2 * nc}^3, {mesh.nt:,} tris, {rays} rays/texel, {frames} frames "
                        f"(frames {warm}..{frames - 1} timed), shadow 1920x1080 k=8 64 steps",
            "ms_per_frame": round(float(np.median(per)), 3), "trace_ms": round(tr, 3),
            "masked_texels": int(m_tex), "rays_per_s": round(m_tex * rays / (tr * 1e-3)),
            "shadow_1080p_ms": round(sh, 4)}


def run_config5(dev, reps=5, warm=3, rays=RAYS, nc=256, frames=2):
    """The differentiable shadow: the room's geometry traced at 256^3 ->
    512^3 (64 rays, 2 frames), 1024x1024 floor points, 64 steps, k = 8;
    loss = mean (vis - target)^2 against the target rendered with the light
    rotated 5 degrees about the horizontal axis perpendicular to it.  One
    step = forward march, loss and its gradient dLoss/dvis, zeroing of
    dLoss/dsdf, and the adjoint (dLoss/dsdf, dLoss/dlight)."""
    import numpy as np
    import torch

    from paper_2210_04449_gb300 import RTSDF
    from synth import scenes as S
    mesh = S.room_scene(1)
    rt = RTSDF(nc, beta_vox=BETA, seed=1)
    rt.upload_mesh(mesh.verts, mesh.tris)
    rt.build_bvh()
    for f in range(frames):
        rt.update(D_VOX, rays, f)
    L0 = np.array([0.4, 1.0, 0.3]) / np.linalg.norm([0.4, 1.0, 0.3])
    ax = np.array([L0[2], 0.0, -L0[0]]) / np.hypot(L0[2], L0[0])
    a = math.radians(5.0)
    L1 = L0 * math.cos(a) + np.cross(ax, L0) * math.sin(a) + ax * np.dot(ax, L0) * (1 - math.cos(a))
    pos, nrm = S.floor_gbuffer(1024, 1024, y=0.02)
    pt, nt = torch.tensor(pos, device=dev), torch.tensor(nrm, device=dev)
    target = rt.shadow(pt, nt, L1, k=8.0, steps=64)
    vis = torch.empty_like(target)
    dsdf = torch.zeros((2 * nc) ** 3, device=dev)
    dl = torch.zeros(3, device=dev)
    loss = torch.zeros((), device=dev)
    inv = 1.0 / target.numel()

    def fwd():
        rt.shadow(pt, nt, L0, k=8.0, steps=64, out=vis)

    def bwd():
        dsdf.zero_()
        dl.zero_()
        rt.shadow_backward(pt, nt, L0, dvis, dsdf, dl, k=8.0, steps=64)

    def step():
        fwd()
        diff = vis - target
        loss.copy_((diff * diff).sum() * inv)
        dvis.copy_(diff * (2.0 * inv))
        bwd()
    dvis = torch.empty_like(target)
    for _ in range(warm):
        step()
    ms = _events_ms(step, reps, dev)
    f_ms = _events_ms(fwd, reps, dev)
    b_ms = _events_ms(bwd, reps, dev)
    out = {"workload": f"room {nc}^3->{2 * nc}^3 ({mesh.nt:,} tris, {rays} rays, {frames} frames), 1024x1024 "
                       "floor points, k=8, 64 steps, MSE vs the light rotated 5 deg",
           "ms_per_step": round(ms, 4), "forward_ms": round(f_ms, 4), "backward_ms": round(b_ms, 4),
           "loss": float(loss.item()), "dlight": [round(float(x), 6) for x in dl.cpu()]}
    rt.sync()
    rt.close()
    return out


def run_batched(dev, frames=8, rays=32, d_vox=2.0):
    """The batched form against plain per-scene frames on 64 uneven scenes
    (coarse 32..128, 1k-200k triangles), 8 frames each after a first
    untimed one: ms/frame for all scenes, and whether the two give the same
    grids element by element (accumulator, counts, fine SDF)."""
    import numpy as np
    import torch

    from paper_2210_04449_gb300 import RTSDF, RTSDFBatch
    from synth import scenes as S
    meshes = S.batch_scenes(3, 64)
    cfgs = [dict(coarse_n=m.meta["coarse_n"], beta_vox=BETA, seed=100 + i) for i, m in enumerate(meshes)]
    # plain: one context per scene, frames run scene after scene
    ctxs = []
    for c, m in zip(cfgs, meshes):
        rt = RTSDF(**c)
        rt.upload_mesh(m.verts, m.tris)
        rt.build_bvh()
        ctxs.append(rt)
    stream = torch.cuda.current_stream(dev)

    def plain_frame(f):
        for rt in ctxs:
            rt.update(d_vox, rays, f)
    plain_frame(0)
    for rt in ctxs:
        rt.set_profiling(True)
        rt.stats()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for f in range(1, frames + 1):
        plain_frame(f)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = e0.elapsed_time(e1) / frames
    plain_stage = {}
    for rt in ctxs:
        for k, v in rt.stats()["stage_ms"].items():
            plain_stage[k] = plain_stage.get(k, 0.0) + v / frames
    # bit patterns (int32 views) of each scene's grids, kept on the device
    ref = [{k: rt.grids()[k].view(torch.int32).clone() for k in ("accum", "counts", "fine")} for rt in ctxs]
    for rt in ctxs:
        rt.close()
    del ctxs
    torch.cuda.empty_cache()
    # batched
    b = RTSDFBatch(cfgs)
    for sc, m in zip(b.scenes, meshes):
        sc.upload_mesh(m.verts, m.tris)
        sc.build_bvh()
    b.frame(d_vox, rays, 0)
    b.sync()
    tuned = b.autotune(d_vox, rays, 1, use_cache=True)
    t0 = time.perf_counter()
    ms = []
    for f in range(1, frames + 1):
        b.frame(d_vox, rays, f)
        b.sync()
        ms.append(b.stats()["last_frame_ms"])
    wall = (time.perf_counter() - t0) * 1e3 / frames
    info = b.stats()
    identical = all(torch.equal(sc.grids()[k].view(torch.int32), r[k]) for sc, r in zip(b.scenes, ref) for k in r)
    b.close()
    del ref
    tris = sum(m.nt for m in meshes)
    return {"workload": f"64 scenes, coarse 32..128, {tris:,} tris total, {rays} rays/texel",
            "plain_ms_per_frame": round(plain_ms, 3), "batched_ms_per_frame": round(float(np.mean(ms)), 3),
            "batched_wall_ms_per_frame": round(wall, 3), "speedup": round(plain_ms / float(np.mean(ms)), 3),
            "frames": frames, "identical": bool(identical), "compared": "accum, counts, fine: every element",
            "graph": bool(info["graph"]),
            "grid": info["grid"], "tuning": tuned, "launches_per_frame": 1, "stage_ms": info["stage_ms"],
            "plain_stage_ms": {k: round(v, 3) for k, v in plain_stage.items() if v > 0}}


# ----------------------------------------------------------------- CPU oracle
def workload_config(nc, n_objects, n_tris):
    """The benchmark workload, named by what it is (both arms report it)."""
    return {"workload": f"animated {nc}^3->{2 * nc}^3, {n_objects} spheres / {n_tris:,} tris, "
                        f"{RAYS} rays/texel, d={D_VOX:g} voxels, beta={BETA:g}, reset in changed regions, "
                        "per frame: move, BVH, voxelize, JFA, mask, trace",
            "coarse_n": nc, "fine_n": 2 * nc, "triangles": int(n_tris), "rays_per_texel": RAYS}


def oracle_frame_sample(n_texels, seed=SEED, objects=N_OBJ, masked_texels=None, brute_texels=16):
    """Time the oracle (as it stands) on one frame of the same workload:
    voxelize + jump flood + mask in full, then the closest hits of all 64
    rays of n_texels sampled masked texels through the oracle's hierarchy
    path (bit-identical to its brute force over all triangles, and the
    faster of its two), extrapolated to the frame's masked texels; returns
    (ms/frame, details).  The details also time the brute-force path on
    `brute_texels` of the same texels."""
    import numpy as np

    import oracle
    from synth import scenes as S
    mesh = S.animated_scene(seed, n_objects=objects)
    B = np.zeros(3, np.float32)
    t0 = time.perf_counter()
    occ = oracle.voxelize(mesh.verts, mesh.tris, B, 1.0, NC)
    t1 = time.perf_counter()
    seeds, _ = oracle.jfa(occ, NC)
    t2 = time.perf_counter()
    d2 = oracle.seed_d2(seeds, NC)
    T = oracle.mask_threshold(D_VOX, BETA)
    masked = np.nonzero((d2 >= 0) & (d2 <= T))[0]
    t3 = time.perf_counter()
    rng = np.random.default_rng(0)
    pick = rng.choice(masked, size=min(n_texels, masked.size), replace=False)
    nf = 2 * NC
    x, y, z = pick % NC, (pick // NC) % NC, pick // (NC * NC)
    tex = (2 * x) + nf * ((2 * y) + nf * (2 * z))
    t4 = time.perf_counter()
    oracle.trace(mesh.verts, mesh.tris, B, 1.0, nf, seed, 1, RAYS, tex, accel="bvh")
    t5 = time.perf_counter()
    # the brute-force path (every ray against every triangle) on a few of
    # the same texels, for reference
    nb = min(brute_texels, pick.size)
    oracle.trace(mesh.verts, mesh.tris, B, 1.0, nf, seed, 1, RAYS, tex[:nb])
    t6 = time.perf_counter()
    m_tex = masked.size * 8 if masked_texels is None else masked_texels
    per_texel = (t5 - t4) / max(pick.size, 1)
    per_texel_brute = (t6 - t5) / max(nb, 1)
    coarse_s = (t1 - t0) + (t2 - t1) + (t3 - t2)
    total = coarse_s + per_texel * m_tex
    return total * 1e3, {"voxelize_s": round(t1 - t0, 3), "jfa_s": round(t2 - t1, 3), "mask_s": round(t3 - t2, 3),
                         "trace_s_per_texel": round(per_texel, 7), "texels_sampled": int(pick.size),
                         "masked_texels": int(m_tex), "sample_cpu_s": round(t6 - t0, 2),
                         "triangles": int(mesh.nt),
                         "brute_force_trace_s_per_texel": round(per_texel_brute, 5), "brute_force_texels": int(nb),
                         "brute_force_ms_per_frame": round((coarse_s + per_texel_brute * m_tex) * 1e3, 1)}


def oracle_threads():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else os.cpu_count()


def run_reference(args, rank, world):
    if rank != 0:
        return None
    # about 2.5 minutes for the whole run: per step ~5 s of voxelize + JFA +
    # mask plus ~0.1 ms of hierarchy tracing per sampled texel (16 Grace cores)
    per_step_s = min(30.0, 150.0 / (args.steps + args.warmup))
    n_tex = int(min(200_000, max(1000, (per_step_s - 5.0) / 1e-4)))
    vals, info = [], None
    for i in range(args.warmup + args.steps):
        ms, info = oracle_frame_sample(n_tex)
        if i >= args.warmup:
            vals.append(ms)
    v = sum(vals) / len(vals)
    return {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": dict(workload_config(NC, N_OBJ, info["triangles"]), parallelism="host cores"),
            "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                             "sample": f"per step: one frame's voxelize + JFA + mask in full, closest hits of "
                                       f"{info['texels_sampled']} masked texels x {RAYS} rays through the oracle's "
                                       f"hierarchy path, extrapolated to all {info['masked_texels']} masked texels",
                             "detail": info},
            "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line, m_tex = run_gpu(args, rank, world)
    if not args.no_batch:
        import torch
        line["batched"] = run_batched(torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
    if not args.no_variant:
        import torch
        line["sign_variant"] = run_sign_variant(torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
    if not args.no_configs:
        import torch
        d = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        line["config2"] = run_config2(d)
        line["config5"] = run_config5(d)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            # ~10-15 s of host work: the full coarse stages and 50,000 traced texels
            ms, info = oracle_frame_sample(50_000, masked_texels=m_tex)
            line["cpu_baseline"] = {
                "value": round(ms, 1), "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                "sample": f"one frame: voxelize + JFA + mask in full, closest hits of "
                          f"{info['texels_sampled']} masked texels x {RAYS} rays over the 1M triangles through "
                          f"the oracle's hierarchy path (bit-identical to its brute force), extrapolated to the "
                          f"frame's {info['masked_texels']} masked texels",
                "detail": info}
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
