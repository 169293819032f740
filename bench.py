#!/usr/bin/env python
"""Benchmark of the full-size frame: 32^3 -> 256^3 coarse-to-fine localization
(Sec. 3.2) plus a 512x512 mesh-free render (Eq. 3), with the 257-1024-512-
256-128-1 occupancy MLP and the 513-1024-512-256-128-3 colour MLP over
256x128x128 feature maps.  One step = one frame.

Prints ONE JSON line (rank 0).  `value` is frames/s over all ranks (each rank
renders its own frames: independent replicas, no collective), measured with
CUDA events around each step on the library's stream, L2 flushed between
steps.  `e2e` repeats the measurement through the public API with the
frame's feature maps copied in from pinned host memory and depth/colour/mask
copied out every step.  `roofline` reports the dominant kernel class
(hidden MLP layers) from the library's own per-launch CUDA-event timing over
the same timed steps.

--impl reference times the FP64 CPU oracle (the plain statement of the
method) on the host cores instead: one full frame of the same workload per
step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s & query pts/s at 256³ + 512² render, vs plain FP32 at IoU≥0.995"
UNIT = "frames/s"
L2_FLUSH_BYTES = 512 << 20
COUNTS_FILE = os.path.join(ROOT, "tests", "golden", "full_frame_counts.txt")
PROFILES = os.path.join(ROOT, "profiles")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp32", "bf16", "mixed"), default="mixed")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison")
    ap.add_argument("--no-stream", action="store_true",
                    help="skip the batched video-stream workload")
    ap.add_argument("--batch", type=int, default=8, help="frames per lockstep batch (stream)")
    ap.add_argument("--stream-slots", type=int, nargs="+", default=[8, 16],
                    help="frame slots of the work-queue stream (each count is timed)")
    ap.add_argument("--stream-subjects", type=int, default=8)
    ap.add_argument("--stream-frames", type=int, default=64)
    ap.add_argument("--no-culled", action="store_true",
                    help="skip the paper's view-culled final level render")
    ap.add_argument("--no-512", action="store_true",
                    help="skip the 512^3 precision form (timing and accuracy vs the oracle)")
    ap.add_argument("--no-fitted", action="store_true",
                    help="skip the frame with the fitted f_O")
    ap.add_argument("--no-cbn", action="store_true",
                    help="skip the CBN + SoftZ occupancy network (the paper's final f_O)")
    ap.add_argument("--no-octree", action="store_true",
                    help="skip the Fig. 3 comparison with the two octree baselines")
    ap.add_argument("--form", choices=("graph", "host"), default="graph")
    ap.add_argument("--schedule", choices=("chained", "per_layer"), default="per_layer",
                    help="tensor-core hidden layers: one launch per batch, or one per layer")
    ap.add_argument("--query-points", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--surrogate", choices=("on", "off"), default="on",
                    help="also time the form with the learned f_S at the coarse levels "
                         "(distilled before any timed region)")
    ap.add_argument("--sur-figures", type=int, default=64)
    ap.add_argument("--sur-tuples", type=int, default=10_000_000)
    ap.add_argument("--sur-steps", type=int, default=6000)
    return ap.parse_args()


def read_kv(path):
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if "=" in line:
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks ---

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, enabled=True):
        self.proc = None
        self.path = None
        self.dev = device_index
        if not enabled:
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={device_index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]),
                             "power": float(parts[3]) if parts[3] not in ("[N/A]", "") else 0.0,
                             "reasons": {"hw_slowdown": parts[5], "hw_thermal_slowdown": parts[6],
                                         "sw_thermal_slowdown": parts[7], "sw_power_cap": parts[8]}})
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = sorted({k for r in rows for k, v in r["reasons"].items() if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["max"] for r in rows),
                "power_w_max": max(r["power"] for r in rows),
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------- roofline ---

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def fp32_simt_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flop (FFMA) per clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def source_digest(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key, digest):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source (matching digest)."""
    if not os.path.isdir(PROFILES):
        return None
    pat = re.compile(r"^traffic\[(\S+)\]\s*=\s*([0-9.eE+]+)\s+bytes/launch\s+source=(\w+)")
    for f in sorted(os.listdir(PROFILES)):
        if not f.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(PROFILES, f)):
            m = pat.match(line.strip())
            if m and m.group(1) == kernel_key and m.group(3) == digest:
                return float(m.group(2))
    return None


# ----------------------------------------------------------------- oracle ---

def oracle_frame(w, keep=False, levels=None):
    """One full frame of the FP64 oracle; returns (seconds, counts[, levels])."""
    import numpy as np
    from oracle import field, localize, render
    t0 = time.perf_counter()
    lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                               w.n0, w.num_levels if levels is None else levels)
    rgb, depth, hit = render.render(lv[-1].values, w.render, w.col_net, w.occ_map, w.col_map,
                                    w.calib)
    dt = time.perf_counter() - t0
    counts = {"evals": int(sum(l.n_eval for l in lv)), "hits": int(np.count_nonzero(hit))}
    return (dt, counts, (lv, rgb, hit)) if keep else (dt, counts)


def oracle_tiny_times():
    """The tiny workload (16^3 -> 64^3 + 64^2 render) through the FP64 oracle,
    all cores and one thread (a child process whose BLAS is limited to one
    thread before numpy loads): (all-core s, single-thread s, cores)."""
    from paper_2007_13988_gb300 import synth
    t_all, _ = oracle_frame(synth.tiny(0))
    code = ("import sys, time; sys.path.insert(0, %r)\n"
            "from paper_2007_13988_gb300 import synth\n"
            "import bench\n"
            "t, _ = bench.oracle_frame(synth.tiny(0)); print(t)") % ROOT
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
              "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    t_one = None
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600)
        if r.returncode == 0:
            t_one = float(r.stdout.strip().splitlines()[-1])
    except Exception:
        t_one = None
    return t_all, t_one, cpu_threads()


def run_reference(args, rank, world):
    """FP64 oracle on the host cores: each step is one full frame of the
    workload (32^3 -> 256^3 localization and the 512^2 render with colour,
    all in the oracle); warm-up steps are full frames too."""
    if rank != 0:
        return
    from paper_2007_13988_gb300 import synth
    w = synth.full(0)
    for _ in range(args.warmup):
        oracle_frame(w)
    times, counts = [], None
    for _ in range(args.steps):
        t, counts = oracle_frame(w)
        times.append(t)
    value = len(times) / sum(times)
    cores = cpu_threads()
    sample = (f"one full frame of the FP64 oracle (numpy) per step: {counts['evals']} f_O + "
              f"{counts['hits']} f_T evaluations, localization bookkeeping and ray scan")
    t_all, t_one, _ = oracle_tiny_times()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, counts["evals"], counts["hits"], "fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample,
                             "tiny_workload_frame_s": {"all_cores": t_all, "one_thread": t_one,
                                                       "workload": "16^3 -> 64^3 + 64^2 render, "
                                                                   "33-128-64-1 MLP"}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(w, evals, hits, precision="mixed"):
    return {"workload": "one 512x512 frame: 32^3->256^3 hierarchical localization + 512^2 "
                        "mesh-free render; f_O 257-1024-512-256-128-1 (skips at 2-4), "
                        "f_T 513-1024-512-256-128-3; 256x128x128 FP32 feature maps",
            "levels": f"{w.n0}->{w.n0 << (w.num_levels - 1)}", "render": w.render,
            "precision": precision, "evals_per_frame": evals, "hits_per_frame": hits,
            "l2": "flushed between timed steps (512 MB write, outside the step events)",
            "parallelism": "replicas (independent frames per GPU)"}


# -------------------------------------------------------------------- ours ---

PREC = {"fp32": 0, "bf16": 1, "mixed": 2, "fp8_mixed": 3, "fp8": 4}
PREC_NAME = {v: k for k, v in PREC.items()}
DTYPE = {"fp32": "f32", "bf16": "bf16", "mixed": "bf16+f32", "fp8_mixed": "e4m3+bf16+f32",
         "fp8": "e4m3+bf16"}


class Frame:
    """One workload on one device: context, resident inputs and outputs."""

    def __init__(self, dev, stream, schedule="per_layer"):
        import torch
        from paper_2007_13988_gb300 import pifu, synth
        self.pifu = pifu
        self.w = w = synth.full(0)
        self.ctx = pifu.pifu_create(pifu.blob_from_nets(w.occ_net, w.col_net))
        self.schedule = (pifu.PIFU_SCHED_CHAINED if schedule == "chained"
                         else pifu.PIFU_SCHED_PER_LAYER)
        pifu.pifu_set_schedule(self.ctx, self.schedule)
        self.stream = stream
        self.dev = dev
        R = w.render
        with torch.cuda.stream(stream):
            self.occ = torch.from_numpy(w.occ_map).to(dev)
            self.col = torch.from_numpy(w.col_map).to(dev)
            self.depth = torch.empty((R, R), dtype=torch.float32, device=dev)
            self.rgb = torch.empty((R, R, 3), dtype=torch.float32, device=dev)
            self.mask = torch.empty((R, R), dtype=torch.uint8, device=dev)
            self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        stream.synchronize()
        # scales of the FP8 form from the frame's own dense coarsest grid
        pifu.pifu_calibrate_fp8(self.ctx, self.occ, w.calib, w.n0, stream=stream)

    def run(self, prec, form="graph", margin=0.02, sur_margin=None, levels=None, final_level=0,
            wait=True):
        """One frame.  Graph form: pifu_frame, or with wait=False
        pifu_frame_async (the host does not wait; pifu_frame_wait later)."""
        w, p = self.w, self.pifu
        L = w.num_levels if levels is None else levels
        sur = {} if sur_margin is None else {"use_surrogate": True, "surrogate_margin": sur_margin}
        if form == "graph" and prec != 0:
            # one CUDA graph per frame (captured on the first call)
            call = p.pifu_frame if wait else p.pifu_frame_async
            return call(self.ctx, self.occ, self.col, w.calib, w.n0, L,
                        w.render, w.render, self.depth, self.rgb, self.mask,
                        precision=prec, margin=margin, stream=self.stream,
                        final_level=final_level, **sur)
        vol = p.pifu_localize(self.ctx, self.occ, w.calib, w.n0, L, precision=prec,
                              margin=margin, stream=self.stream, **sur)
        p.pifu_render(self.ctx, w.render, w.render, self.occ, self.col, w.calib, self.depth,
                      self.rgb, self.mask, precision=1 if prec != 0 else 0, stream=self.stream,
                      final_level=final_level)
        return p.pifu_sync_stats(self.ctx) if final_level else vol

    def close(self):
        self.pifu.pifu_destroy(self.ctx)


def time_form(fr, prec, steps, warmup, world, clocks=None, form="graph", sur_margin=None,
              levels=None, final_level=0, asynchronous=True):
    """Device-timed frames of one precision form; returns a dict."""
    import torch
    vol = None
    for _ in range(max(1, warmup)):
        vol = fr.run(prec, form, sur_margin=sur_margin, levels=levels, final_level=final_level)
    fr.stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    fr.pifu.pifu_profile(fr.ctx, True)
    # graph form: the frames go out through pifu_frame_async, so the host
    # never waits between steps and each step's events bracket its device
    # work only (with pifu_frame the host's wait and relaunch would sit
    # between the events); pifu_frame_wait reports their errors at the end
    graph = form == "graph" and prec != 0 and asynchronous
    for i in range(steps):
        with torch.cuda.stream(fr.stream):
            fr.flush.zero_()
        ev[i][0].record(fr.stream)
        vol = fr.run(prec, form, sur_margin=sur_margin, levels=levels, final_level=final_level,
                     wait=not graph)
        ev[i][1].record(fr.stream)
    if graph:
        vol = fr.pifu.pifu_frame_wait(fr.ctx, fr.stream)
    torch.cuda.synchronize()
    prof = fr.pifu.pifu_profile_read(fr.ctx)
    fr.pifu.pifu_profile(fr.ctx, False)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks is not None else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1000.0
    if world > 1:
        t = torch.tensor([total_s], device=fr.dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    L = vol.num_levels
    return {"value": world * steps / total_s, "ms_per_step": 1000.0 * total_s / steps,
            "step_ms": step_ms, "prof": prof, "clocks": clk, "vol": vol,
            "evals": int(vol.n_eval),
            "rechecked": int(sum(vol.rechecked_per_level[i] for i in range(L))),
            "fallback": int(sum(vol.fallback_per_level[i] for i in range(L))),
            "coarse_evals": int(sum(vol.evals_per_level[i] for i in range(L - 1))),
            "evals_per_level": [int(vol.evals_per_level[i]) for i in range(L)],
            "rounds": [int(vol.conflict_rounds[i]) for i in range(L)],
            "hits": int(fr.mask.sum().item())}


def octree_tradeoff(fr, prec, reps=3):
    """Fig. 3: for the method and the two octree baselines, the acceleration
    factor (brute-force evaluations / evaluations), the IoU of the binarized
    finest grid against the brute-force dense grid in the same arithmetic,
    and the localization time (host-driven form, device-timed)."""
    import numpy as np
    import torch
    p, w = fr.pifu, fr.w
    N = w.n0 << (w.num_levels - 1)

    def timed(n0, L, **kw):
        run = lambda: p.pifu_localize(fr.ctx, fr.occ, w.calib, n0, L, precision=prec,
                                      stream=fr.stream, **kw)
        vol = run()
        ms = []
        for _ in range(reps):
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            with torch.cuda.stream(fr.stream):
                fr.flush.zero_()
            e[0].record(fr.stream)
            vol = run()
            e[1].record(fr.stream)
            fr.stream.synchronize()
            ms.append(e[0].elapsed_time(e[1]))
        occ, _, _ = p.volume_tensors(vol)
        b = p.unpack_bits(occ.cpu().numpy(), vol.n, vol.row_words)
        return int(vol.n_eval), float(np.median(ms)), b

    from scipy import ndimage
    cell = (N // w.n0) ** 3

    def main_body(b):
        # 26-connected components of at least one coarsest cell's volume
        lab, _ = ndimage.label(b, structure=np.ones((3, 3, 3)))
        sz = np.bincount(lab.ravel())
        sz[0] = 0
        return sz[lab] >= cell

    def iou(a, b):
        return float(np.count_nonzero(a & b)) / max(1, int(np.count_nonzero(a | b)))

    n_b, ms_b, bb = timed(N, 1)
    body_bb = main_body(bb)

    def entry(n0, L, **kw):
        n, ms, b = timed(n0, L, **kw)
        return {"acceleration": (N + 1) ** 3 / n, "iou_vs_brute_force": iou(b, bb),
                "main_body_iou_vs_brute_force": iou(main_body(b), body_bb), "evals": n,
                "localize_ms": ms, "time_speedup_vs_brute_force": ms_b / ms}

    out = {"workload": f"{w.n0}^3 -> {N}^3 localization of the full-size frame, "
                       f"{DTYPE[PREC_NAME[prec]]} arithmetic, host-driven form",
           "brute_force": {"evals": n_b, "localize_ms": ms_b},
           "method": entry(w.n0, w.num_levels),
           "binarized_octree": entry(w.n0, w.num_levels, subdivision=p.PIFU_SUBDIV_BINARIZED)}
    out["threshold_octree"] = {
        str(t): entry(w.n0, w.num_levels, subdivision=p.PIFU_SUBDIV_THRESHOLD, threshold=t)
        for t in (0.01, 0.02, 0.03, 0.05, 0.08, 0.12, 0.2, 0.3, 0.4)}
    out["notes"] = ("thresholds 0.05 .. 0.4 are Fig. 3's, 0.01 .. 0.03 extend the curve to the "
                    "method's evaluation count; main body: 26-connected inside components of at "
                    f"least one coarsest cell ({cell} voxels)")
    return out


def cbn_form(fr, args, world):
    """The paper's final f_O (CBN + SoftZ, Appendix, Eq. 7 and Eq. 8) on the
    same frame and maps: the MIXED frame as one CUDA graph (the headline's
    form), the host-driven MIXED form for per-kernel times, and the plain
    FP32 form, device-timed like the headline, with the CBN kernel's own
    roofline."""
    from paper_2007_13988_gb300 import synth
    p = fr.pifu
    wc = synth.full_cbn(0)
    ctx = p.pifu_create(p.blob_from_nets(wc.occ_net, wc.col_net))
    p.pifu_set_schedule(ctx, fr.schedule)
    saved = fr.ctx, fr.w
    fr.ctx, fr.w = ctx, wc
    try:
        side = max(3, min(args.steps, 10))
        graph = time_form(fr, PREC["mixed"], args.steps, args.warmup, world, form="graph")
        graph["snap"] = snapshot(fr, graph["vol"])
        mixed = time_form(fr, PREC["mixed"], side, 2, world, form="host")
        plain = time_form(fr, 0, side, 2, world, form="host")
    finally:
        fr.ctx, fr.w = saved
        p.pifu_destroy(ctx)
    return wc, graph, mixed, plain


def fitted_form(fr, args, world):
    """The same frame with the fitted f_O (2000 Adam steps of BCE on 65,536
    points against the capsules' occupancy, fitted once by the oracle's
    trainer and stored): the MIXED frame as one CUDA graph, the host-driven
    MIXED form, and the plain FP32 form, device-timed like the headline."""
    from paper_2007_13988_gb300 import synth
    p = fr.pifu
    wf = synth.full_fitted()
    ctx = p.pifu_create(p.blob_from_nets(wf.occ_net, wf.col_net))
    p.pifu_set_schedule(ctx, fr.schedule)
    saved = fr.ctx, fr.w
    fr.ctx, fr.w = ctx, wf
    try:
        side = max(3, min(args.steps, 10))
        graph = time_form(fr, PREC["mixed"], args.steps, args.warmup, world, form="graph")
        graph["snap"] = snapshot(fr, graph["vol"])
        mixed = time_form(fr, PREC["mixed"], side, 2, world, form="host")
        plain = time_form(fr, 0, side, 2, world, form="host")
    finally:
        fr.ctx, fr.w = saved
        p.pifu_destroy(ctx)
    return wf, graph, mixed, plain


def snapshot(fr, vol):
    """Host copies of a frame's result: binarized fine grid, node values
    (tentative 0/1 where not evaluated), colour and hit mask."""
    import numpy as np
    p = fr.pifu
    occ_b, ev_b, val = p.volume_tensors(vol)
    b = p.unpack_bits(occ_b.cpu().numpy(), vol.n, vol.row_words)
    e = p.unpack_bits(ev_b.cpu().numpy(), vol.n, vol.row_words)
    v = val.cpu().numpy().astype(np.float64).reshape((vol.n + 1,) * 3)
    return {"b": b, "vals": np.where(e, v, b.astype(np.float64)), "rgb": fr.rgb.cpu().numpy(),
            "mask": fr.mask.cpu().numpy().astype(bool)}


def accuracy(snap, lv, o_rgb, o_hit, fp32_rgb=None):
    """IoU / Chamfer of the fine grid and colour PSNR against the oracle's
    frame (and PSNR against the plain FP32 render, if given)."""
    import numpy as np
    from oracle import metrics
    both = snap["mask"] & o_hit
    d = snap["rgb"].astype(np.float64)[both] - o_rgb[both]
    mse = float(np.mean(d * d)) if d.size else 0.0
    out = {"iou_vs_oracle": metrics.iou(snap["b"], lv[-1].binary),
           "chamfer_vox_vs_oracle": metrics.chamfer_voxels(snap["vals"], lv[-1].values),
           "colour_psnr_vs_oracle_db": float("inf") if mse == 0 else 10 * np.log10(1.0 / mse),
           "mask_disagreement_px": int(np.count_nonzero(snap["mask"] != o_hit))}
    if fp32_rgb is not None:
        d = snap["rgb"].astype(np.float64) - fp32_rgb.astype(np.float64)
        mse = float(np.mean(d * d))
        out["colour_psnr_vs_fp32_db"] = float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)
    return out


def train_surrogate(fr, args):
    """Distil f_S from f_O on the GPU (the library's own training kernels),
    before any timed region; returns (margin, report)."""
    import torch
    from paper_2007_13988_gb300 import distill
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per = max(1, args.sur_tuples // args.sur_figures)
    x, y = distill.build_samples(fr.ctx, n_figures=args.sur_figures, per_figure=per, seed0=1000)
    first, last = distill.train(fr.ctx, x, y, steps=args.sur_steps, batch=4096, lr=3e-3)
    n = int(x.shape[0])
    del x, y
    torch.cuda.empty_cache()
    # the largest held-out disagreement: a confident wrong decision at a
    # coarse level costs extra conflict rounds at the next one
    margin, disagree = distill.calibrate_margin(fr.ctx, seeds=[2000, 2001, 2002, 2003],
                                                per_figure=200000, quantile=1.0)
    torch.cuda.synchronize()
    return margin, {"net": "257-128-64-1 (leaky-ReLU, sigmoid); BF16 tensor cores in the frame",
                    "tuples": n, "figures": args.sur_figures, "steps": args.sur_steps,
                    "batch": 4096, "lr": 3e-3, "loss_first": first, "loss_last": last,
                    "margin": margin, "margin_quantile": 1.0,
                    "held_out_sign_disagreement": disagree,
                    "train_s": time.perf_counter() - t0,
                    "levels": "all but the finest (the finest level always runs f_O)"}


def run_stream(fr, args, world, sur_margin):
    """The video-stream workload: subjects x frames animated figures with BF16
    maps, all frames through the device work queue in one graph launch
    (pifu_stream), and in lockstep batches of args.batch frames (one CUDA
    graph each) beside it.  Returns a dict for the JSON line (rank-local
    timings)."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_2007_13988_gb300 import synth
    pifu, w, dev, s = fr.pifu, fr.w, fr.dev, fr.stream
    subj = synth.stream(n_figures=args.stream_subjects, frames=args.stream_frames, seed=100)
    H = W = 128
    C = 256
    t0 = time.perf_counter()
    occ, col = [], []
    with torch.cuda.stream(s):
        for sj in subj:
            g_o, g_t = sj.texture(H, W, C)
            base_o = torch.from_numpy(g_o).to(dev).to(torch.bfloat16)
            base_t = torch.from_numpy(g_t).to(dev).to(torch.bfloat16)
            with ThreadPoolExecutor(8) as ex:
                geo = list(ex.map(lambda t: sj.geometry(t, H, W), range(args.stream_frames)))
            fo, ft = [], []
            for g, cc in geo:
                m_o = base_o.clone()
                m_o[:, :, :3] = torch.from_numpy(g).to(dev).to(torch.bfloat16)
                m_t = base_t.clone()
                m_t[:, :, :3] = torch.from_numpy(cc).to(dev).to(torch.bfloat16)
                fo.append(m_o)
                ft.append(m_t)
            occ.append(fo)
            col.append(ft)
    s.synchronize()
    gen_s = time.perf_counter() - t0
    B = args.batch
    n_subj, n_frames = len(subj), args.stream_frames
    # frame order: frame t of every subject, then t + 1 ...
    order = [(i, t) for t in range(n_frames) for i in range(n_subj)]
    batches = [order[k:k + B] for k in range(0, len(order), B) if len(order[k:k + B]) == B]
    R = w.render
    depth = torch.empty((B, R, R), dtype=torch.float32, device=dev)
    rgb = torch.empty((B, R, R, 3), dtype=torch.float32, device=dev)
    mask = torch.empty((B, R, R), dtype=torch.uint8, device=dev)
    calibs = [w.calib] * B
    # FP8 scales from the stream's own first frame; tiles for a level-0 batch
    pifu.pifu_calibrate_fp8(fr.ctx, occ[0][0], w.calib, w.n0, stream=s)
    tuned = pifu.pifu_autotune(fr.ctx, B * (w.n0 + 1) ** 3, stream=s)

    def run(prec, sur):
        kw = {"use_surrogate": True, "surrogate_margin": sur} if sur is not None else {}
        lat, vols = [], None
        for rep in range(2):   # first pass: capture + warm-up
            lat = []
            for bt in batches:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(s):
                    fr.flush.zero_()
                e0.record(s)
                vols = pifu.pifu_frames(fr.ctx, [occ[i][t] for i, t in bt],
                                        [col[i][t] for i, t in bt], calibs, w.n0, w.num_levels,
                                        R, R, depth, rgb, mask, precision=prec, stream=s, **kw)
                e1.record(s)
                e1.synchronize()
                lat.append(e0.elapsed_time(e1))
        total_s = sum(lat) / 1000.0
        n = len(batches) * B
        return {"value": world * n / total_s, "unit": UNIT, "frames": n,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "batch_ms_min": min(lat), "batch_ms_max": max(lat),
                "rounds_last_batch": [int(vols[0].conflict_rounds[l]) for l in range(w.num_levels)],
                "evals_per_frame_mean": float(np.mean([v.n_eval for v in vols]))}

    def run_single(prec):
        # the same frames one graph launch each (pifu_frame), for comparison
        lat = []
        for rep in range(2):
            lat = []
            for i, t in order[:len(batches) * B]:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                pifu.pifu_frame(fr.ctx, occ[i][t], col[i][t], w.calib, w.n0, w.num_levels, R, R,
                                depth[0], rgb[0], mask[0], precision=prec, stream=s)
                e1.record(s)
                e1.synchronize()
                lat.append(e0.elapsed_time(e1))
        return {"value": world * len(lat) / (sum(lat) / 1000.0), "unit": UNIT,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}

    # the work-queue form: every frame of the stream in one pifu_stream call
    F = len(order)
    q_depth = torch.empty((F, R, R), dtype=torch.float32, device=dev)
    q_rgb = torch.empty((F, R, R, 3), dtype=torch.float32, device=dev)
    q_mask = torch.empty((F, R, R), dtype=torch.uint8, device=dev)
    q_occ = [occ[i][t] for i, t in order]
    q_col = [col[i][t] for i, t in order]

    def run_queue(prec, sur, slots):
        kw = {"use_surrogate": True, "surrogate_margin": sur} if sur is not None else {}
        ms, vols, times = 0.0, None, None
        for rep in range(2):   # first pass: capture + warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s):
                fr.flush.zero_()
            e0.record(s)
            vols, times = pifu.pifu_stream(fr.ctx, q_occ, q_col, [w.calib] * F, slots, w.n0,
                                           w.num_levels, R, R, q_depth, q_rgb, q_mask,
                                           precision=prec, stream=s, **kw)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
        lat = [tm.done_ms - tm.admit_ms for tm in times]
        steps = [w.num_levels + 1 + sum(int(v.conflict_rounds[l]) for l in range(w.num_levels))
                 for v in vols]
        return {"value": world * F / (ms / 1000.0), "unit": UNIT, "frames": F, "slots": slots,
                "ms_total": ms, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)),
                "stream_rounds": int(times[0].stream_rounds),
                "rounds_per_frame_mean": float(np.mean(steps)),
                "rounds_per_frame_max": int(max(steps)),
                "evals_per_frame_mean": float(np.mean([v.n_eval for v in vols])),
                "rechecked_total": int(vols[0].rechecked_per_level[0]),
                "fallback_total": int(vols[0].fallback_per_level[0])}

    out = {"workload": f"{n_subj} subjects x {n_frames} frames (scales "
                       f"{min(x.scale for x in subj):.2f}-{max(x.scale for x in subj):.2f}, joints "
                       f"animated per frame), 256x128x128 BF16 maps per frame, 32^3->256^3 + "
                       f"512^2 render per frame",
           "form": "pifu_stream: every frame of the stream in one graph launch, frames "
                   "fed to slots by a device work queue (value); pifu_frames lockstep "
                   "batches beside it",
           "latency": "work queue: per frame, from its admission to a slot to the end of its "
                      "render (device clock); lockstep: per frame = its batch's device time",
           "map_generation_s": gen_s, "autotuned_tiles": [bn for bn, _ in tuned],
           "count_readings": {"subjects_x_frames": n_subj * n_frames,
                              "frames_total_alternative": n_frames}}
    prec8 = PREC["fp8_mixed"]
    queue = {}
    if sur_margin is not None:
        queue["fp8_mixed_surrogate"] = {sl: run_queue(prec8, sur_margin, sl)
                                        for sl in args.stream_slots}
    queue["fp8_mixed"] = {sl: run_queue(prec8, None, sl) for sl in args.stream_slots}
    queue["mixed"] = {sl: run_queue(PREC["mixed"], None, sl) for sl in args.stream_slots}
    head_q = queue.get("fp8_mixed_surrogate", queue["fp8_mixed"])
    best = max(head_q, key=lambda sl: head_q[sl]["value"])
    out["work_queue"] = {k: {str(sl): r for sl, r in v.items()} for k, v in queue.items()}
    out["value"] = head_q[best]["value"]
    out["value_form"] = ("work queue, " + ("FP8_MIXED + surrogate" if sur_margin is not None
                                           else "FP8_MIXED") + f", {best} slots")
    out["p50_ms"] = head_q[best]["p50_ms"]
    out["p99_ms"] = head_q[best]["p99_ms"]
    lock = {"batch": B, "form": "pifu_frames: lockstep batches, one CUDA graph"}
    if sur_margin is not None:
        lock["fp8_mixed_surrogate"] = run(prec8, sur_margin)
    lock["fp8_mixed"] = run(prec8, None)
    lock["mixed"] = run(PREC["mixed"], None)
    out["lockstep"] = lock
    out["single_frame_graphs_mixed"] = run_single(PREC["mixed"])
    out["unit"] = UNIT
    return out, (occ, col, subj)


def stream_accuracy(fr, args, stream_inputs, sur_margin):
    """Two stream frames (the smallest subject's first frame and the largest
    subject's middle frame) through the work-queue form in the stream's
    precision (FP8_MIXED, with the surrogate when it was trained), against the
    FP64 oracle's localization and render on the same BF16-rounded maps: the
    checks and bars of the stream's GPU test (occupancy IoU >= 0.995, colour
    PSNR >= 40 dB on the pixels both hit)."""
    import numpy as np
    import torch
    from oracle import field, localize, metrics, render
    pifu, w = fr.pifu, fr.w
    occ, col, subj = stream_inputs
    small = min(range(len(subj)), key=lambda i: subj[i].scale)
    big = max(range(len(subj)), key=lambda i: subj[i].scale)
    pick = ((small, 0), (big, args.stream_frames // 2))
    R = w.render
    n = w.n0 << (w.num_levels - 1)
    rw = (n + 1 + 31) // 32
    F = len(pick)
    dev = occ[0][0].device
    depth = torch.empty((F, R, R), dtype=torch.float32, device=dev)
    rgb = torch.empty((F, R, R, 3), dtype=torch.float32, device=dev)
    mask = torch.empty((F, R, R), dtype=torch.uint8, device=dev)
    bits = torch.zeros((F, (n + 1) * (n + 1) * rw), dtype=torch.int32, device=dev)
    kw = {"use_surrogate": True, "surrogate_margin": sur_margin} if sur_margin is not None else {}
    pifu.pifu_stream(fr.ctx, [occ[i][t] for i, t in pick], [col[i][t] for i, t in pick],
                     [w.calib] * F, 2, w.n0, w.num_levels, R, R, depth, rgb, mask, bits,
                     precision=PREC["fp8_mixed"], stream=fr.stream, **kw)
    fr.stream.synchronize()
    samples = []
    for k, (i, t) in enumerate(pick):
        m_r = occ[i][t].float().cpu().numpy().astype(np.float64)
        c_r = col[i][t].float().cpu().numpy().astype(np.float64)
        lvs = localize.hierarchical(lambda P: field.occupancy(w.occ_net, m_r, w.calib, P), w.n0,
                                    w.num_levels)
        o_rgb, _, o_hit = render.render(lvs[-1].values, R, w.col_net, m_r, c_r, w.calib)
        b = pifu.unpack_bits(bits[k].cpu().numpy(), n, rw)
        msk = mask[k].cpu().numpy().astype(bool)
        both = msk & o_hit
        d = rgb[k].cpu().numpy().astype(np.float64)[both] - o_rgb[both]
        mse = float(np.mean(d * d)) if d.size else 0.0
        iou = metrics.iou(b, lvs[-1].binary)
        psnr = float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)
        samples.append({"subject": i, "frame": t, "scale": subj[i].scale,
                        "form": "work queue, FP8_MIXED" + (" + surrogate" if kw else ""),
                        "iou_vs_oracle": iou, "colour_psnr_vs_oracle_db": psnr,
                        "meets_bar": bool(iou >= 0.995 and psnr >= 40.0),
                        "inside_fraction": float(np.mean(lvs[-1].binary)),
                        "evaluated_fraction_finest": lvs[-1].n_eval / lvs[-1].binary.size})
    return samples


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2007_13988_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    fr = Frame(dev, stream, args.schedule)
    pifu = fr.pifu
    w = fr.w
    R = w.render
    prec = PREC[args.precision]

    # ---- the learned surrogate, distilled before any timed region ----------
    sur_margin, sur_report = None, None
    if args.surrogate == "on" and prec != 0:
        sur_margin, sur_report = train_surrogate(fr, args)

    # ---- headline form: device-resident timed region -----------------------
    form = args.form if prec != 0 else "host"
    head = time_form(fr, prec, args.steps, args.warmup, world,
                     ClockSampler(local_rank, enabled=not args.no_clocks), form=form)
    head_snap = snapshot(fr, head["vol"])
    # ---- per-kernel timing: a graph has no per-launch events, so the kernel
    # classes of the same frame are timed on its host-driven form ------------
    prof_run = head
    sync_call = None
    if form == "graph":
        prof_run = time_form(fr, prec, max(3, min(args.steps, 10)), 1, world, form="host")
        # the same graph through pifu_frame, which waits for each frame
        sync_call = time_form(fr, prec, args.steps, 2, world, form="graph", asynchronous=False)
    # ---- the same form with the learned surrogate at the coarse levels -------
    sur = None
    if sur_margin is not None:
        sur = time_form(fr, prec, args.steps, args.warmup, world, form=form,
                        sur_margin=sur_margin)
        sur_snap = snapshot(fr, sur["vol"])
    # ---- the other tensor-core precision forms of the same frame ------------
    side_steps = max(3, min(args.steps, 10))
    others = {}
    if prec != 0:
        for name in ("mixed", "fp8_mixed"):
            if PREC[name] != prec:
                r = time_form(fr, PREC[name], side_steps, 2, world, form=form)
                others[name] = (r, snapshot(fr, r["vol"]))
    # ---- the headline form with the FP32 SIMT re-check (the default re-check
    # is the split-TF32 pass on the tensor cores) ----------------------------
    simt_rc = None
    if prec in (2, 3):
        pp = fr.pifu
        pp.pifu_set_recheck(fr.ctx, pp.PIFU_RECHECK_SIMT)
        try:
            r = time_form(fr, prec, side_steps, 2, world, form=form)
            rh = time_form(fr, prec, side_steps, 1, world, form="host") if form == "graph" else r
        finally:
            pp.pifu_set_recheck(fr.ctx, pp.PIFU_RECHECK_TENSOR)
        simt_rc = (r, rh)
    # ---- the plain FP32 form on the same GPU, for the speedup ---------------
    plain = None
    if prec != 0 and not args.no_plain:
        plain = time_form(fr, 0, side_steps, 2, world)
        plain_rgb = fr.rgb.cpu().numpy()
    # ---- the paper's view-culled final level: 512 depth nodes at 512^2 -------
    culled = None
    if prec != 0 and not args.no_culled:
        culled = time_form(fr, prec, args.steps, args.warmup, world, form=form, final_level=1)
        culled["snap"] = snapshot(fr, culled["vol"])
        fr_depth_culled = fr.depth.cpu().numpy().astype(np.float64)
        culled_plain = time_form(fr, 0, 2, 1, world, final_level=1)
        culled["plain"] = culled_plain
    # ---- the precision form at 512^3 (five levels from 32^3) ----------------
    p512 = {}
    if prec != 0 and not args.no_512:
        L5 = w.num_levels + 1
        for name in ("mixed", "fp8_mixed"):
            r = time_form(fr, PREC[name], side_steps, 2, world, form=form, levels=L5)
            p512[name] = (r, snapshot(fr, r["vol"]))
        fp32_512 = time_form(fr, 0, 2, 1, world, levels=L5)
        p512["fp32"] = (fp32_512, snapshot(fr, fp32_512["vol"]))

    # ---- Fig. 3: the method against the two octree baselines -----------------
    fig3 = None
    if not args.no_octree:
        fig3 = octree_tradeoff(fr, prec)
    # ---- the paper's final f_O: CBN + SoftZ -------------------------------------
    cbn = None
    fitted = None
    if prec != 0 and not args.no_fitted:
        fitted = fitted_form(fr, args, world)
    if prec != 0 and not args.no_cbn:
        cbn = cbn_form(fr, args, world)
    # ---- the video stream in lockstep batches ----------------------------------
    stream_out, stream_inputs = None, None
    if prec != 0 and not args.no_stream:
        stream_out, stream_inputs = run_stream(fr, args, world, sur_margin)
        if rank == 0 and not args.no_cpu_baseline:
            stream_out["accuracy_samples"] = stream_accuracy(fr, args, stream_inputs,
                                                             sur_margin)

    # ---- query points/s (raw field, inputs resident) -----------------------
    Q = args.query_points
    with torch.cuda.stream(stream):
        pts = torch.from_numpy(synth.query_points(Q, seed=123)).to(dev)
        qout = torch.empty(Q, dtype=torch.float32, device=dev)
    stream.synchronize()

    def query_rate(qprec):
        pifu.pifu_query_ex(fr.ctx, fr.occ, w.calib, pts, qout, precision=qprec, stream=stream)
        qe = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        n_q = 3
        with torch.cuda.stream(stream):
            fr.flush.zero_()
        qe[0].record(stream)
        for _ in range(n_q):
            pifu.pifu_query_ex(fr.ctx, fr.occ, w.calib, pts, qout, precision=qprec, stream=stream)
        qe[1].record(stream)
        stream.synchronize()
        return world * Q * n_q / (qe[0].elapsed_time(qe[1]) / 1000.0)

    q_head = query_rate(prec)
    q_plain = query_rate(0) if prec != 0 else q_head

    # ---- end to end through the public API with host buffers ---------------
    h_occ = torch.from_numpy(w.occ_map).pin_memory()
    h_col = torch.from_numpy(w.col_map).pin_memory()
    h_depth = torch.empty((R, R), dtype=torch.float32).pin_memory()
    h_rgb = torch.empty((R, R, 3), dtype=torch.float32).pin_memory()
    h_mask = torch.empty((R, R), dtype=torch.uint8).pin_memory()
    e2e_steps = max(3, min(args.steps, 30))

    def e2e_serial():
        # each step: copy the maps in, run the frame, copy the outputs out, wait
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            with torch.cuda.stream(stream):
                fr.occ.copy_(h_occ, non_blocking=True)
                fr.col.copy_(h_col, non_blocking=True)
            fr.run(prec, form)
            with torch.cuda.stream(stream):
                h_depth.copy_(fr.depth, non_blocking=True)
                h_rgb.copy_(fr.rgb, non_blocking=True)
                h_mask.copy_(fr.mask, non_blocking=True)
            stream.synchronize()
        return time.perf_counter() - t0

    def e2e_pipelined():
        # The same copies on a second stream, overlapping the frames: while
        # frame i runs, step i+1's maps come in from pinned host memory and
        # step i-1's outputs go out, through device staging buffers (one
        # device-to-device copy each way on the frame's stream, so the
        # frame's own buffers and graph stay the same).  Graph frames go out
        # through pifu_frame_async: the host enqueues step i+1 while frame i
        # runs, and pifu_frame_wait at the end reports the frames' errors.
        graph = form == "graph" and prec != 0
        cs = torch.cuda.Stream(device=dev)
        s_occ, s_col = torch.empty_like(fr.occ), torch.empty_like(fr.col)
        s_depth, s_rgb, s_mask = (torch.empty_like(fr.depth), torch.empty_like(fr.rgb),
                                  torch.empty_like(fr.mask))
        ev_in = torch.cuda.Event()
        ev_out = torch.cuda.Event()
        ev_d2h = torch.cuda.Event()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(cs):
            s_occ.copy_(h_occ, non_blocking=True)
            s_col.copy_(h_col, non_blocking=True)
        stream.wait_stream(cs)
        for i in range(e2e_steps):
            with torch.cuda.stream(stream):
                fr.occ.copy_(s_occ, non_blocking=True)
                fr.col.copy_(s_col, non_blocking=True)
                ev_in.record(stream)
            with torch.cuda.stream(cs):
                if i + 1 < e2e_steps:
                    cs.wait_event(ev_in)                    # staging read by this step
                    s_occ.copy_(h_occ, non_blocking=True)   # step i+1's maps
                    s_col.copy_(h_col, non_blocking=True)
                if i > 0:
                    cs.wait_event(ev_out)                   # step i-1's outputs staged
                    h_depth.copy_(s_depth, non_blocking=True)
                    h_rgb.copy_(s_rgb, non_blocking=True)
                    h_mask.copy_(s_mask, non_blocking=True)
                    ev_d2h.record(cs)
            fr.run(prec, form, wait=not graph)
            with torch.cuda.stream(stream):
                if i > 0:
                    stream.wait_event(ev_d2h)               # staging free again
                s_depth.copy_(fr.depth, non_blocking=True)
                s_rgb.copy_(fr.rgb, non_blocking=True)
                s_mask.copy_(fr.mask, non_blocking=True)
                ev_out.record(stream)
            stream.wait_stream(cs)                          # step i+1's maps are in
        with torch.cuda.stream(cs):
            cs.wait_event(ev_out)
            h_depth.copy_(s_depth, non_blocking=True)
            h_rgb.copy_(s_rgb, non_blocking=True)
            h_mask.copy_(s_mask, non_blocking=True)
        if graph:
            fr.pifu.pifu_frame_wait(fr.ctx, stream)
        cs.synchronize()
        return time.perf_counter() - t0

    def over_ranks(sec):
        if world > 1:
            t = torch.tensor([sec], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            sec = float(t.item())
        return sec

    e2e_serial_s = over_ranks(e2e_serial())
    e2e_s = over_ranks(e2e_pipelined())
    e2e_value = world * e2e_steps / e2e_s
    e2e_serial_value = world * e2e_steps / e2e_serial_s
    h2d = h_occ.numel() * 4 + h_col.numel() * 4
    d2h = h_depth.numel() * 4 + h_rgb.numel() * 4 + h_mask.numel()
    fr.close()
    if rank != 0:
        return

    # ---- roofline of the dominant kernel class of the headline form --------
    prof = prof_run["prof"]
    peaks, peak_src = measured_peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    dk = prof["mlp_hidden"] if prec != 0 else prof["mlp_f32"]
    achieved = dk["flops"] / (dk["ms"] / 1000.0) / 1e12 if dk["ms"] > 0 else 0.0
    if prec == 0:
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = fp32_simt_peak_tflops(sm_mhz)
        kname, bound, src = "sgemm_bias_lrelu", "alu", "paper_2007_13988_gb300/csrc/mlp_f32.cu"
        peak_note = (f"FP32 SIMT: 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz "
                     f"(sm_max_mhz, {peak_src})")
    else:
        peak = peaks.get("bf16_tflops", 1900.0)
        kname, bound, src = "tc_linear_kernel", "tensor", "paper_2007_13988_gb300/csrc/mlp_tc.cu"
        peak_note = f"dense BF16 cuBLAS burst, MEASURED_PEAKS.json ({peak_src})"
    traffic = recorded_traffic(kname, source_digest([src]))
    roofline = {"bound": bound, "kernel": kname + " (hidden MLP layers)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": peak_note, "traffic": traffic,
                "avg_launch_ms": dk["ms"] / max(1, dk["launches"]),
                "flops_per_launch": dk["flops"] / max(1, dk["launches"]),
                "share_of_step": dk["ms"] / max(1e-9, sum(prof_run["step_ms"])),
                "dominant_class": dom,
                "measured_on": ("host-driven frames of the same workload (same kernels and "
                                "shapes; a CUDA graph has no per-launch events), "
                                f"{len(prof_run['step_ms'])} steps")
                               if form == "graph" else "the timed steps"}
    nprof = max(1, len(prof_run["step_ms"]))
    kernels = {k: {"launches": v["launches"] // nprof,
                   "ms_per_step": v["ms"] / nprof,
                   "achieved_gbs": (v["bytes"] / (v["ms"] / 1000.0) / 1e9) if v["ms"] > 0 else None}
               for k, v in prof.items()}
    # the bookkeeping classes against HBM: their algorithmic bytes (bitsets
    # read and written, 4 B per listed or evaluated node, the render's outputs)
    # over their device time; the gather against L2 (4 taps x C x 4 B per point)
    # and, for HBM, the maps read once per frame plus the BF16 rows written
    hbm = peaks.get("hbm_gbs", 6800.0)
    book = {}
    for k in ("level", "select", "render"):
        v = prof[k]
        if v["ms"] <= 0:
            continue
        gbs = v["bytes"] / (v["ms"] / 1000.0) / 1e9
        book[k] = {"bound": "hbm", "bytes_per_frame": v["bytes"] / nprof,
                   "ms_per_frame": v["ms"] / nprof, "launches_per_frame": v["launches"] / nprof,
                   "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}
    g = prof["gather"]
    if g["ms"] > 0:
        map_bytes = (w.occ_map.nbytes + (w.col_map.nbytes if w.col_map is not None else 0))
        ldx_o = (w.occ_net.d_in + 7) // 8 * 8
        ldx_t = (w.col_net.d_in + 7) // 8 * 8
        rows = 2.0 * (head["evals"] * ldx_o + head["hits"] * ldx_t)
        hbm_bytes = map_bytes + rows
        sec = g["ms"] / nprof / 1000.0
        book["gather"] = {"bound": "l2", "l2_bytes_per_frame": g["bytes"] / nprof,
                          "achieved_l2": g["bytes"] / nprof / sec / 1e9,
                          "hbm_bytes_per_frame": hbm_bytes, "achieved": hbm_bytes / sec / 1e9,
                          "peak": hbm, "unit": "GB/s", "frac": hbm_bytes / sec / 1e9 / hbm,
                          "ms_per_frame": g["ms"] / nprof,
                          "launches_per_frame": g["launches"] / nprof}
    for k in book:
        book[k]["measured_on"] = roofline["measured_on"]
        book[k]["peak_source"] = f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"
    launches = sum(v["launches"] for v in head["prof"].values())
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": workload_config(w, head["evals"], head["hits"], args.precision),
            "query_pts_per_s": q_head,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "form": "pipelined: step i+1's maps in and step i-1's outputs out on a "
                            "second stream during frame i (pinned host memory, device "
                            "staging), every step's copies inside the timed loop; frames "
                            "through pifu_frame_async, errors read by pifu_frame_wait inside "
                            "the timed region",
                    "serial": {"value": e2e_serial_value,
                               "form": "copy in, frame, copy out, wait: one step at a time"}},
            "gpu_launches": launches, "roofline": roofline, "kernels": kernels,
            "bookkeeping_roofline": book,
            "step_ms": {"min": min(head["step_ms"]), "median": statistics.median(head["step_ms"]),
                        "max": max(head["step_ms"])}}
    line["config"]["form"] = ("one CUDA graph per frame, enqueued by pifu_frame_async (the host "
                              "does not wait between frames; pifu_frame_wait after the timed "
                              "steps)" if form == "graph"
                              else "host-driven (pifu_localize + pifu_render)")
    line["config"]["layer_schedule"] = args.schedule
    if form == "graph":
        line["host_driven"] = {"value": prof_run["value"], "ms_per_step": prof_run["ms_per_step"]}
        line["sync_call"] = {"value": sync_call["value"], "ms_per_step": sync_call["ms_per_step"],
                             "form": "the same graph through pifu_frame, which waits for each "
                                     "frame: the events then also hold the host's wait and "
                                     "relaunch"}
    if prec in (2, 3):
        line["config"]["margin"] = 0.02
        line["config"]["rechecked_per_frame"] = head["rechecked"]
    line["config"]["surrogate"] = False
    line["config"]["evals_per_level"] = head["evals_per_level"]
    line["config"]["conflict_rounds"] = head["rounds"]
    if sur is not None:
        sur_report.update({
            "value": sur["value"], "unit": UNIT, "ms_per_step": sur["ms_per_step"],
            "form": "the headline form with f_S at every level but the finest",
            "speedup_over_headline": sur["value"] / head["value"],
            "evals_per_level": sur["evals_per_level"], "conflict_rounds": sur["rounds"],
            "fallback_per_frame": sur["fallback"], "coarse_evals_per_frame": sur["coarse_evals"],
            "fallback_fraction": sur["fallback"] / max(1, sur["coarse_evals"]),
            "coarse_f_O_evals_saved": head["coarse_evals"] - sur["fallback"]})
        line["surrogate"] = sur_report
    if plain is not None:
        line["plain_fp32"] = {"value": plain["value"], "ms_per_step": plain["ms_per_step"],
                              "query_pts_per_s": q_plain,
                              "speedup_of_headline": head["value"] / plain["value"]}
        if sur is not None:
            line["surrogate"]["speedup_over_plain_fp32"] = sur["value"] / plain["value"]
        d = plain_rgb.astype(np.float64) - head_snap["rgb"].astype(np.float64)
        mse = float(np.mean(d * d))
        line["accuracy"] = {"colour_psnr_vs_fp32_db": float("inf") if mse == 0 else
                            10 * np.log10(1.0 / mse)}
    if others:
        line["other_forms"] = {
            name: {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                   "dtype": DTYPE[name], "rechecked_per_frame": r["rechecked"],
                   "evals_per_frame": r["evals"], "conflict_rounds": r["rounds"],
                   "speedup_over_headline": r["value"] / head["value"],
                   "speedup_over_plain_fp32": r["value"] / plain["value"] if plain else None}
            for name, (r, _) in others.items()}
    if simt_rc is not None:
        r, rh = simt_rc
        nr = max(1, len(rh["step_ms"]))
        line["recheck_forms"] = {
            "note": "the FP32-accurate pass of the MIXED forms (re-check of occupancies within "
                    "the margin of 0.5, batches of <= 256 points) in the headline: passes of "
                    "more than 192 points in split TF32 on the tensor cores (hi*hi + hi*lo + "
                    "lo*hi, FP32 accumulation), passes of at most 64 points in FP32 FFMA as "
                    "one cooperative launch over every SM, the others on the FP32 form's "
                    "cluster network; against every pass on that cluster network; ms per "
                    "frame of that class on the host-driven form (its host launch gaps "
                    "included)",
            "tensor": {"value": head["value"], "ms_per_step": head["ms_per_step"],
                       "pass_ms_per_frame": prof["mlp_f32"]["ms"] / nprof,
                       "pass_launches_per_frame": prof["mlp_f32"]["launches"] // nprof},
            "simt": {"value": r["value"], "ms_per_step": r["ms_per_step"],
                     "pass_ms_per_frame": rh["prof"]["mlp_f32"]["ms"] / nr,
                     "pass_launches_per_frame": rh["prof"]["mlp_f32"]["launches"] // nr,
                     "rechecked_per_frame": r["rechecked"]}}
    if head["clocks"] is not None:
        line["clocks"] = head["clocks"]
    if world == 1 and not args.no_cpu_baseline:
        t, cnt, (lv, o_rgb, o_hit) = oracle_frame(w, keep=True)
        t_all, t_one, _ = oracle_tiny_times()
        line["cpu_baseline"] = {"value": 1.0 / t, "unit": UNIT, "cores": cpu_threads(),
                                "kind": "oracle",
                                "sample": f"one full frame of the FP64 oracle (numpy): "
                                          f"{cnt['evals']} f_O + {cnt['hits']} f_T evaluations, "
                                          f"localization bookkeeping and ray scan; {t:.1f} s",
                                "tiny_workload_frame_s": {
                                    "all_cores": t_all, "one_thread": t_one,
                                    "workload": "16^3 -> 64^3 + 64^2 render, 33-128-64-1 MLP"}}
        # colour at the pixels both renders hit (silhouette pixels that one of
        # them misses are counted apart)
        line.setdefault("accuracy", {}).update(accuracy(head_snap, lv, o_rgb, o_hit))
        if sur is not None:
            line["surrogate"]["accuracy"] = accuracy(sur_snap, lv, o_rgb, o_hit)
        for name, (r, snap) in others.items():
            line["other_forms"][name]["accuracy"] = accuracy(snap, lv, o_rgb, o_hit,
                                                             plain_rgb if plain else None)
    if culled is not None:
        L = w.num_levels
        cv = culled["vol"]
        line["culled_final_level"] = {
            "form": "the paper's view-culled final level (Sec. 3.2): 32^3 -> 256^3 localized, "
                    "then 513 depth nodes per pixel column of the 512^2 image, shadow nodes "
                    "culled, ambiguous nodes evaluated, no conflict loop; graph form",
            "value": culled["value"], "unit": UNIT, "ms_per_step": culled["ms_per_step"],
            "localized_evals_per_frame": int(sum(cv.evals_per_level[i] for i in range(L))),
            "culled_level_evals_per_frame": int(cv.evals_per_level[L]),
            "plain_fp32": {"value": culled["plain"]["value"],
                           "ms_per_step": culled["plain"]["ms_per_step"]},
            "speedup_over_plain_fp32": culled["value"] / culled["plain"]["value"]}
        if world == 1 and not args.no_cpu_baseline:
            from oracle import field, render as orender
            f = lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P)
            t0 = time.perf_counter()
            o_rgb2, o_depth2, o_hit2, res = orender.render_culled(f, lv[-1].binary, w.render,
                                                                  w.col_net, w.occ_map, w.col_map,
                                                                  w.calib)
            sn = culled["snap"]
            both = sn["mask"] & o_hit2
            d = sn["rgb"].astype(np.float64)[both] - o_rgb2[both]
            mse = float(np.mean(d * d)) if d.size else 0.0
            line["culled_final_level"]["accuracy"] = {
                "iou_vs_oracle": accuracy(sn, lv, o_rgb, o_hit)["iou_vs_oracle"],
                "mask_agreement_vs_oracle_culled": float(np.mean(sn["mask"] == o_hit2)),
                "depth_max_abs_vs_oracle_culled": float(np.nanmax(np.abs(
                    fr_depth_culled[both] - o_depth2[both]))) if both.any() else None,
                "colour_psnr_vs_oracle_culled_db": float("inf") if mse == 0 else
                10 * np.log10(1.0 / mse),
                "oracle_culled_evals": res["n_eval"], "oracle_s": time.perf_counter() - t0}
    if fig3 is not None:
        line["fig3_octree_baselines"] = fig3
    if cbn is not None:
        wc, cg, cm, cp = cbn
        ck = cm["prof"]["cbn_tc"]
        c_ach = ck["flops"] / (ck["ms"] / 1000.0) / 1e12 if ck["ms"] > 0 else 0.0
        c_peak = peaks.get("bf16_tflops", 1900.0)
        out = {"form": "the paper's final f_O, CBN + SoftZ (SoftZ 64 -> 128, five CBN blocks "
                       "of 128 channels conditioned on the 256-channel feature), "
                       "32^3 -> 256^3 + 512^2 render, MIXED, one CUDA graph per frame",
               "value": cg["value"], "unit": UNIT, "ms_per_step": cg["ms_per_step"],
               "host_driven": {"value": cm["value"], "ms_per_step": cm["ms_per_step"]},
               "evals_per_frame": cg["evals"], "rechecked_per_frame": cg["rechecked"],
               "conflict_rounds": cg["rounds"],
               "f_O_gflop_per_frame": cm["evals"] * wc.occ_net.flops_per_point() / 1e9,
               "plain_fp32": {"value": cp["value"], "ms_per_step": cp["ms_per_step"]},
               "speedup_over_plain_fp32": cg["value"] / cp["value"],
               "speedup_over_headline": cg["value"] / head["value"],
               "kernel_roofline": {
                   "kernel": "cbn_tc_kernel (whole f_O per 128-point tile)", "bound": "tensor",
                   "achieved": c_ach, "peak": c_peak, "unit": "TFLOP/s",
                   "frac": c_ach / c_peak, "peak_source": "dense BF16 cuBLAS burst, "
                   "MEASURED_PEAKS.json",
                   "launches_per_step": ck["launches"] / max(1, len(cm["step_ms"])),
                   "ms_per_step": ck["ms"] / max(1, len(cm["step_ms"])),
                   "measured_on": "host-driven frames (a CUDA graph has no per-launch events)"},
               "kernels": {k: {"launches": v["launches"] // max(1, len(cm["step_ms"])),
                               "ms_per_step": v["ms"] / max(1, len(cm["step_ms"]))}
                           for k, v in cm["prof"].items() if v["launches"]}}
        if world == 1 and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            _, _, (lvc, o_rgbc, o_hitc) = oracle_frame(wc, keep=True)
            out["accuracy"] = accuracy(cg["snap"], lvc, o_rgbc, o_hitc)
            out["oracle_s"] = time.perf_counter() - t0
        line["cbn_softz"] = out
    if fitted is not None:
        wf, fg, fm, fp = fitted
        nprof_f = max(1, len(fm["step_ms"]))
        out = {"form": "the headline frame and form (32^3 -> 256^3 + 512^2 render, MIXED, one "
                       "CUDA graph per frame) with f_O fitted to the figure: 2000 Adam steps of "
                       "BCE on 65,536 points (half uniform, half near the capsule surfaces), "
                       "fitted once by the oracle's trainer (tests/golden/fit_occupancy.py)",
               "value": fg["value"], "unit": UNIT, "ms_per_step": fg["ms_per_step"],
               "host_driven": {"value": fm["value"], "ms_per_step": fm["ms_per_step"]},
               "evals_per_frame": fg["evals"], "evals_per_level": fg["evals_per_level"],
               "rechecked_per_frame": fg["rechecked"], "conflict_rounds": fg["rounds"],
               "hits_per_frame": fg["hits"],
               "plain_fp32": {"value": fp["value"], "ms_per_step": fp["ms_per_step"]},
               "speedup_over_plain_fp32": fg["value"] / fp["value"],
               "speedup_over_headline": fg["value"] / head["value"],
               "kernels": {k: {"launches": v["launches"] // nprof_f,
                               "ms_per_step": v["ms"] / nprof_f}
                           for k, v in fm["prof"].items() if v["launches"]}}
        if world == 1 and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            _, cnt_f, (lvf, o_rgbf, o_hitf) = oracle_frame(wf, keep=True)
            out["accuracy"] = accuracy(fg["snap"], lvf, o_rgbf, o_hitf)
            out["oracle_s"] = time.perf_counter() - t0
            out["oracle_evals_per_frame"] = cnt_f["evals"]
        line["fitted_weights"] = out
    if stream_out is not None:
        line["stream"] = stream_out
    if p512:
        out = {"workload": "the same frame at 512^3 effective resolution: 32^3 -> 512^3 "
                           "(five levels) + 512^2 render, graph form",
               "margin": 0.02}
        base = p512["fp32"][0]
        out["plain_fp32"] = {"value": base["value"], "ms_per_step": base["ms_per_step"],
                             "form": "host-driven FP32", "evals_per_frame": base["evals"]}
        for name in ("mixed", "fp8_mixed"):
            r, _ = p512[name]
            out[name] = {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                         "dtype": DTYPE[name], "speedup_over_plain_fp32": r["value"] / base["value"],
                         "evals_per_frame": r["evals"], "rechecked_per_frame": r["rechecked"],
                         "conflict_rounds": r["rounds"]}
        if rank == 0:
            t0 = time.perf_counter()
            _, _, (lv5, o_rgb5, o_hit5) = oracle_frame(w, keep=True, levels=w.num_levels + 1)
            out["oracle_s"] = time.perf_counter() - t0
            for name in ("mixed", "fp8_mixed"):
                out[name]["accuracy"] = accuracy(p512[name][1], lv5, o_rgb5, o_hit5,
                                                 p512["fp32"][1]["rgb"])
        line["precision_512"] = out
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
