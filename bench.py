"""Benchmark of the SEU-injection hot path on GB300.

Default workload (one GPU): 2,000,000 Gaussians (4 clusters, SH degree 3, fp32
storage), four 1600x1040 views on a ring, 20,000 single-bit upsets with 70% on
bits 24-31 of log-scale and opacity.  A step is one launch of the batched
dirty-tile engine over B variants (B picked by the library's autotuner from
{8, 16, ..., 2048}), replayed as a CUDA graph: inject + guard-ready preprocess
of the flipped primitives, the two plan kernels, dirty-tile re-blend fused with
the comparison against the clean frames, finalisation of the per-(variant,
view) records.  Reported beside it: the plain one-variant-per-launch
full-render loop on the same flips and the stage split of a full render, the
end-to-end rate through host buffers, contamination and SSIM campaigns, the
support-guard clamp bandwidth on a 66,000,000-Gaussian scene, Table 2 and the
scaling law, the serving loop, and the CPU oracle on bounded samples.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "injections/s and Mpix/s vs plain loop on 1 GB300; p99 frame latency; guard GB/s"
UNIT = "injections/s"
WORKLOAD = ("2M Gaussians (4 clusters, SH degree 3, fp32), 4 ring views 1600x1040, 20k upsets "
            "(70% on bits 24-31 of log-scale/opacity), guard off")
ENGINE = "batched dirty-tile engine (inject, plan, re-blend + compare, finalise), replayed as a CUDA graph"
FLOP_PER_EVAL = 20          # FP32 ops per pixel-primitive evaluation of the blend (FMA = 2)
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_k_dirty_2M_4views_batch2048.txt")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 2000; the reference arm: 4, each step is seconds of CPU work)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default 5; the reference arm: 1)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-guard-stress", action="store_true", help="skip the 66M-Gaussian guard measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--guard-n", type=int, default=66_000_000)
    ap.add_argument("--only-guard", action="store_true", help="run only the guard measurement (profiling)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop latency measurement")
    ap.add_argument("--no-analytics", action="store_true", help="skip the Table 2 / scaling-law campaigns")
    ap.add_argument("--batch", type=int, default=0,
                    help="variants per launch (default: the library's autotuner picks); for small profiling cases")
    ap.add_argument("--tile", default="",
                    help="render tile shape WxH (default: the library's autotuner picks with the batch)")
    ap.add_argument("--gaussians", type=int, default=2_000_000,
                    help="scene size (the 2M default is the benchmark; smaller only for profiling captures)")
    args = ap.parse_args()
    ref = args.impl == "reference"
    if args.steps is None:
        args.steps = 4 if ref else 2000
    if args.warmup is None:
        args.warmup = 1 if ref else 5
    return args


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def traffic_record():
    """Per-launch DRAM bytes of kernels from the committed ncu summary (key value lines)."""
    out = {}
    try:
        for line in open(TRAFFIC_FILE):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(None, 1)
            out[k] = v.strip()
    except FileNotFoundError:
        pass
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (rank 0, N = 1)
# ---------------------------------------------------------------------------
def workload_config(n, cams, nflips, world=1):
    """The `config` of both arms: the workload only (no engine settings)."""
    W, H = int(cams[0]["width"]), int(cams[0]["height"])
    name = WORKLOAD if n == 2_000_000 else f"profiling case: {n} Gaussians, otherwise " + WORKLOAD
    return {"workload": name, "gaussians": n, "sh_degree": 3, "storage": "fp32", "resolution": f"{W}x{H}",
            "views": len(cams), "upsets": nflips, "guard": "off",
            "l2": "GPU steps: a 256 MB buffer is written between timed steps (outside the step events)",
            "parallelism": f"replicas x{world}, upset list sharded"}


def clean_views(scene, cams):
    """Clean renders of every view by the oracle, one thread per view (its C calls
    release the GIL); returns (images, seconds)."""
    import concurrent.futures as cf
    import oracle as O
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=len(cams)) as ex:
        imgs = list(ex.map(lambda c: O.render(scene.planes, scene.fmt, scene.sh_degree, c), list(cams)))
    return imgs, time.perf_counter() - t0


def oracle_steps(scene, cams, flips, clean, steps, warmup):
    """The oracle as it stands on the host cores, in steps: a step is one upset
    per core rendered at full resolution in one view and compared with it
    (OpenMP over upsets); the view rotates over the ring views from step to
    step and the upsets walk the list.  Returns (seconds of each timed step,
    cores); K steps cover K * cores (upset, view) pairs = K * cores / views
    injections."""
    import oracle as O
    cores = O.max_threads()
    nv = len(cams)
    times = []
    for i in range(warmup + steps):
        sl = flips[(i * cores) % (len(flips) - cores):][:cores]
        k = i % nv
        t0 = time.perf_counter()
        O.campaign(scene.planes, scene.fmt, scene.sh_degree, cams[k:k + 1], sl, clean_imgs=clean[k:k + 1],
                   nthreads=cores)
        if i >= warmup:
            times.append(time.perf_counter() - t0)
    return times, cores


def cpu_baseline(scene, cams, flips, clean, t_clean):
    """The oracle on the benchmark workload, the same steps as the reference
    arm: one step per view (four), one upset per core each, whole 1600x1040
    views, nothing extrapolated."""
    nv = steps = len(cams)
    times, cores = oracle_steps(scene, cams, flips, clean, steps, 0)
    t = sum(times)
    W, H = int(cams[0]["width"]), int(cams[0]["height"])
    return {"value": steps * cores / nv / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nv} steps of {cores} upsets x 1 full {W}x{H} view (one step per ring view; OpenMP over "
                      f"upsets), {t:.1f} s; value = {cores} upsets x {nv} views / {nv} / seconds, not extrapolated; "
                      f"clean views rendered untimed ({t_clean:.1f} s)"}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_timing(scene3, cams3, flips3, c3_all, clean3, t_clean3):
    """Per-injection cost of the oracle, as it stands, single-threaded and with
    OpenMP over upsets on all host cores, on the three campaign workloads: the
    5,000-Gaussian 256x256 one (bounded samples of its 200 upsets), the
    134,826-Gaussian 800x800 stratified one (samples of 100 upsets) and the
    benchmark's (one upset single-threaded in view 0, extrapolated to 4 views;
    the all-cores figure is `cpu_baseline`; `clean3` are its clean views).
    Clean frames are rendered first and timed on their own.  Context for the
    GPU numbers, never a target."""
    import oracle as O
    from paper_2606_21791_gb300 import synth as S
    cores = O.max_threads()

    def clean_of(sc, cams):
        t0 = time.perf_counter()
        imgs = [O.render(sc.planes, sc.fmt, sc.sh_degree, c) for c in cams]
        return imgs, time.perf_counter() - t0

    def per_inj(sc, cams, fl, clean, nthreads):
        t0 = time.perf_counter()
        O.campaign(sc.planes, sc.fmt, sc.sh_degree, cams, fl, clean_imgs=clean, nthreads=nthreads)
        return (time.perf_counter() - t0) / len(fl)

    out = {"cores": cores, "cpu": cpu_model(), "unit": "s per injection (all views of the workload)"}
    sc, cams, fl = S.tiny_workload()
    clean, tc = clean_of(sc, cams)
    out["c1"] = {"workload": "5,000 Gaussians (SH 0, fp32), 256x256, 1 view", "clean_frame_s": tc,
                 "single_thread": per_inj(sc, cams, fl[:20], clean, 1), "all_cores": per_inj(sc, cams, fl, clean, cores),
                 "sample": "20 of the 200 upsets single-threaded, all 200 on all cores"}
    sc, cams, fl = S.batching_workload(S.FP32)
    clean, tc = clean_of(sc, cams)
    nall = max(cores, 16)
    out["c2"] = {"workload": "134,826 Gaussians (4 clusters, SH 3, fp32), 800x800, 1 view", "clean_frame_s": tc,
                 "single_thread": per_inj(sc, cams, fl[:2], clean, 1),
                 "all_cores": per_inj(sc, cams, fl[:nall], clean, cores),
                 "sample": f"2 of 100 upsets single-threaded, {nall} on all cores"}
    single = per_inj(scene3, cams3[0:1], flips3[:1], clean3[0:1], 1) * len(cams3)
    out["c3"] = {"workload": "2M Gaussians (4 clusters, SH 3, fp32), 4 views 1600x1040",
                 "clean_frames_s": t_clean3, "single_thread": single, "all_cores": 1.0 / c3_all,
                 "sample": "1 upset in view 0 single-threaded, extrapolated to 4 views; all cores: cpu_baseline",
                 "campaign_of_20000_single_thread_days": single * 20000 / 86400.0}
    return out


def run_reference(args):
    """The oracle, as it stands, on the host cores (there is no other
    implementation of this path to install).  A step is one upset per core,
    rendered at full resolution in one view and compared with it; the view
    rotates over the four ring views from step to step, so K steps cover
    K * cores (upset, view) pairs = K * cores / 4 injections.  Only rank 0 runs."""
    rank, local, world = dist_info()
    if rank != 0:
        return
    from paper_2606_21791_gb300 import synth as S
    import oracle as O
    O.build()
    scene, cams, flips = S.scale_workload(n=args.gaussians)
    K, Wu = args.steps, args.warmup
    nv = len(cams)
    clean, t_clean = clean_views(scene, cams)
    times, cores = oracle_steps(scene, cams, flips, clean, K, Wu)
    total = sum(times)
    value = K * cores / nv / total
    W, H = int(cams[0]["width"]), int(cams[0]["height"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": K, "warmup": Wu,
            "ms_per_step": 1000 * total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": workload_config(scene.n, cams, len(flips), args.gpus),
            "engine": "CPU oracle (plain C, fp32 render math, OpenMP over upsets)",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step {cores} upsets x 1 full {W}x{H} view, the view rotating over the "
                                       f"{nv} ring views; value = steps x {cores} / {nv} / seconds (not "
                                       f"extrapolated in pixels); clean views rendered untimed ({t_clean:.1f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import paper_2606_21791_gb300 as P
    P.build()
    from paper_2606_21791_gb300 import gs as G
    from paper_2606_21791_gb300 import replicas as R
    from paper_2606_21791_gb300 import synth as S

    rank, local, world = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pk, pk_kind = peaks()
    if args.only_guard:
        print(json.dumps({"guard": guard_stress(args, G, S, dev, pk, pk_kind)}), flush=True)
        return

    t_setup = time.perf_counter()
    scene, cams, flips = S.scale_workload(n=args.gaussians)
    K_views = len(cams)
    Wd, Hd = int(cams[0]["width"]), int(cams[0]["height"])
    h = G.gs_load_scene(scene.planes, scene.n, scene.sh_degree, scene.fmt)
    G.gs_set_views(h, cams)
    mask = S.GUARD_WORDS_DEFAULT
    # each rank takes its own slice of the upset list (independent units, no collective)
    d_flips = G.to_device(flips, dev)
    nflips = len(flips)
    if args.tile:
        G.gs_set_tile(h, *(int(x) for x in args.tile.lower().split("x")))
    if args.batch > 0:
        G.gs_set_batch(h, args.batch)
        B = args.batch
        tile = G.gs_get_tile(h)
        log(f"[bench] setup {time.perf_counter() - t_setup:.1f}s; batch B={B} (set)")
    elif args.tile:
        tile = G.gs_get_tile(h)
        B, us_per = G.gs_autotune(h, d_flips, 8192, G.GS_GUARD_OFF, mask)
        log(f"[bench] setup {time.perf_counter() - t_setup:.1f}s; tile {tile[0]}x{tile[1]} (set), autotuned batch "
            f"B={B} ({us_per:.2f} us/variant)")
    else:
        tile, B, us_per = G.gs_autotune_tile(h, d_flips, 8192, G.GS_GUARD_OFF, mask)
        log(f"[bench] setup {time.perf_counter() - t_setup:.1f}s; autotuned tile {tile[0]}x{tile[1]}, batch B={B} "
            f"({us_per:.2f} us/variant)")

    out = G.device_bytes(B * K_views * 24, dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def flips_at(i):
        a, b = R.step_slice(i, rank, world, B, nflips)
        return d_flips[a * 8:b * 8]

    def step(i):
        G.gs_inject_and_render(h, flips_at(i), B, 1, G.GS_GUARD_OFF, mask, out)

    # work per step (untimed pass with counters on; the engine is deterministic)
    G.gs_count_work(h, True)
    for i in range(args.warmup, args.warmup + args.steps):
        step(i)
    work = G.gs_read_work(h)
    G.gs_count_work(h, False)

    G.gs_time_kernels(h, True)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        wall0 = time.perf_counter()
        for j in range(args.steps):
            flush.zero_()
            ev[j][0].record(stream)
            step(args.warmup + j)
            ev[j][1].record(stream)
            kern_ms.append(G.gs_read_kernel_ms(h))   # (plan, blend + compare)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        torch.cuda.nvtx.range_pop()
        if world > 1:
            torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    G.gs_time_kernels(h, False)
    t_total, inj = R.aggregate(sum(step_ms) / 1000.0, B * args.steps, dev)
    value = inj / t_total
    lat = sorted(step_ms)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]

    # end to end through the C-ABI call with host buffers (pinned): the library
    # copies the step's upsets in and its records out inside the call
    host_flips = torch.from_numpy(flips.view(np.uint8).copy()).pin_memory()
    host_out = torch.empty(B * K_views * 24, dtype=torch.uint8).pin_memory()
    for i in range(2):
        a, b = R.step_slice(i, rank, world, B, nflips)
        G.gs_inject_and_render_host(h, host_flips[a * 8:b * 8], B, 1, G.GS_GUARD_OFF, mask, host_out)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for j in range(args.steps):
        a, b = R.step_slice(args.warmup + j, rank, world, B, nflips)
        G.gs_inject_and_render_host(h, host_flips[a * 8:b * 8], B, 1, G.GS_GUARD_OFF, mask, host_out)
    e2e_t, e2e_units = R.aggregate(time.perf_counter() - e0, B * args.steps, dev)
    # the last step's records of every rank on rank 0, in list order (untimed): the
    # ranks' slices of one step are consecutive, rank by rank
    last = host_out.numpy().view(G.RESULT_DTYPE).reshape(B, K_views)
    gathered = R.gather_records(rank * B + np.arange(B), last, world * B, dev)
    e2e = {"value": e2e_units / e2e_t, "unit": UNIT, "h2d_bytes_per_step": B * 8,
           "d2h_bytes_per_step": B * K_views * 24,
           "how": "per step: gs_inject_and_render_host with pinned host upsets and records (the copies in and out "
                  "and a stream sync inside the call)"}

    # the same workload at batches of 8-64 variants per launch (graph replay each)
    small_b = {}
    nsb = min(2048, nflips)
    for b in (8, 16, 32, 64):
        G.gs_set_batch(h, b)
        G.gs_inject_and_render(h, d_flips[:8 * b], b, 1, G.GS_GUARD_OFF, mask, out)   # capture
        torch.cuda.synchronize()
        sb0, sb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sbo = G.device_bytes(nsb * K_views * 24, dev)
        flush.zero_()
        sb0.record(stream)
        G.gs_inject_and_render(h, d_flips[:8 * nsb], nsb, 1, G.GS_GUARD_OFF, mask, sbo)
        sb1.record(stream)
        torch.cuda.synchronize()
        small_b[str(b)] = nsb / (sb0.elapsed_time(sb1) / 1000.0)
    best_small = max(small_b, key=small_b.get)
    small_batches = {"injections_s": small_b, "best_batch": int(best_small), "best_injections_s": small_b[best_small],
                     "sample": f"the first {nsb} upsets per batch size, one call each (launches of B variants)"}
    G.gs_set_batch(h, B)

    # plain loop: one variant per launch, full preprocess + sort + blend + compare, no graphs
    nplain = 16
    G.gs_inject_and_render_full(h, d_flips[:8 * 2], 2, 1, G.GS_GUARD_OFF, mask, out)
    torch.cuda.synchronize()
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_out = G.device_bytes(nplain * K_views * 24, dev)
    torch.cuda.nvtx.range_push("plain_loop")
    pe0.record(stream)
    G.gs_inject_and_render_full(h, flips_at(args.warmup)[: 8 * nplain] if B >= nplain else d_flips[:8 * nplain],
                                nplain, 1, G.GS_GUARD_OFF, mask, plain_out)
    pe1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    plain_s = pe0.elapsed_time(pe1) / 1000.0
    plain = {"value": nplain / plain_s, "unit": UNIT, "sample": f"{nplain} upsets, {K_views} views each",
             "mpix_s": nplain * K_views * Wd * Hd / plain_s / 1e6}

    # sort-first contamination (nodes a scale-sign upset corrupts), guard off / FIELD guard
    contam = contamination(G, S, h, scene, K_views, dev)
    # SSIM of every (variant, view) from the re-blended pixels
    ssim_line = ssim_campaign(G, S, h, d_flips, nflips, K_views, dev)
    # stage split of the full render (preprocess / binning + radix sort / blend)
    stages = render_stages(G, S, h, cams, flush, dev, pk, pk_kind)

    # roofline of the dominant kernel (dirty-tile blend): FP32-pipe bound
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or pk.get("sm_max_mhz", 2070.0)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = nsm * 128 * 2 * sm_mhz * 1e6 / 1e12
    kavg = sum(k[1] for k in kern_ms) / len(kern_ms) / 1000.0
    plan_avg = sum(k[0] for k in kern_ms) / len(kern_ms) / 1000.0
    evals_per_launch = work["evaluations"] / args.steps
    achieved = evals_per_launch * FLOP_PER_EVAL / kavg / 1e12
    tr = traffic_record()
    traffic = float(tr["k_dirty_bytes_per_launch"]) if "k_dirty_bytes_per_launch" in tr else None
    roofline = {"kernel": "k_dirty (dirty-tile blend + compare)", "bound": "alu", "achieved": achieved,
                "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                "peak_source": f"{nsm} SMs x 128 FP32 lanes x 2 x median SM clock {sm_mhz:.0f} MHz under load",
                "work_per_launch": {"evaluations": evals_per_launch, "flop_per_eval": FLOP_PER_EVAL,
                                    "tiles": work["tiles"] / args.steps, "entries": work["entries"] / args.steps,
                                    "tiles_dropped_by_plan": work["tiles_unchanged"] / args.steps,
                                    "blocks_blended": work["blocks_blended"] / args.steps,
                                    "warp_steps": work["warp_steps"] / args.steps,
                                    "warp_steps_blending": work["warp_steps_blending"] / args.steps,
                                    "warp_cycle_share": phase_shares(work),
                                    # of a walk step's 64 pixel slots: those the plan left active, and
                                    # those still blending (active and not yet stopped)
                                    "slots_active_per_step": work["active_pixel_steps"] / max(work["warp_steps"], 1),
                                    "slots_live_per_step": work["evaluations"] / max(work["warp_steps"], 1),
                                    "plan_drops": {k: work[k] / args.steps for k in
                                                   ("dropped_stop_key", "dropped_tile_reach", "dropped_no_reach",
                                                    "dropped_pixel_stop")}},
                "kernel_ms_avg": kavg * 1000.0, "kernel_share_of_step": kavg * 1000.0 / (sum(step_ms) / len(step_ms)),
                "plan_kernel_ms_avg": plan_avg * 1000.0}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(scene.n, cams, nflips, world),
        "engine": {"name": ENGINE, "batch": B, "tile": f"{tile[0]}x{tile[1]}",
                   "batch_and_tile_from": ("set" if args.batch > 0 else
                                           "tile set, batch autotuned" if args.tile else
                                           "autotuner (tiles 16x16, 8x8, 32x8; batches 8-2048)")},
        "e2e": e2e,
        # per step: injector, item scan, two plan kernels, dirty-tile blend, finalise
        "gpu_launches": 6 * args.steps,
        "records_gathered_on_rank0": None if gathered is None else int(gathered.shape[0]),
        "mpix_s_effective": value * K_views * Wd * Hd / 1e6,
        "mpix_s_blended": work["blocks_blended"] * 64 * world / t_total / 1e6,   # 8x8 blocks
        "plain_loop": plain,
        "render_stages": stages,
        "contamination": contam,
        "ssim": ssim_line,
        "speedup_vs_plain_loop": value / plain["value"],
        "batches_8_to_64": small_batches,
        "batch_latency_ms": {"p50": p50, "p99": p99, "what": f"one launch of {B} variants x {K_views} views"},
        "wall_s_timed_region": wall,
        "roofline": roofline,
        "clocks": clocks,
        "peaks": {"source": pk_kind, "hbm_gbs": pk.get("hbm_gbs")},
    }
    G.gs_free_scene(h)
    del d_flips, flush
    torch.cuda.empty_cache()

    if not args.no_guard_stress:
        line["guard"] = guard_stress(args, G, S, dev, pk, pk_kind)
    if world == 1 and not args.no_analytics:
        line["campaign_analytics"] = campaign_analytics(G, S, dev)
        line["formats_134k"] = batching_formats(G, S, dev)
    if not args.no_serving:
        line["serving"] = serving(args, G, S, dev)
        st = line["serving"]["storm"]
        line["p99_frame_latency_ms"] = {"storm_field_guard": st["guard_field"]["p99_ms"],
                                        "storm_prim_guard": st["guard_prim"]["p99_ms"],
                                        "storm_guard_off": st["guard_off"]["p99_ms"],
                                        "poisson_80pct": line["serving"]["poisson"][1]["p99_ms"],
                                        "poisson_80pct_budget_bound": line["serving"]["budget_bound"]["p99_ms"]}
    if rank == 0 and world == 1 and not args.no_cpu:
        clean3, t_clean3 = clean_views(scene, cams)
        line["cpu_baseline"] = cpu_baseline(scene, cams, flips, clean3, t_clean3)
        try:
            line["oracle_timing"] = oracle_timing(scene, cams, flips, line["cpu_baseline"]["value"], clean3, t_clean3)
        except Exception as e:   # context only: report the failure, keep the measured line
            line["oracle_timing"] = {"error": repr(e)}
    line["summary"] = summary(line)   # last, so a cut-off tail of the line still holds it
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def phase_shares(work):
    """Shares of the dirty-tile blend's warp cycles (measurement build) spent
    setting up a block, walking its entries and comparing."""
    keys = ("cycles_setup", "cycles_walk", "cycles_compare")
    tot = sum(work.get(k, 0) for k in keys)
    return {k.split("_", 1)[1]: (work[k] / tot if tot else None) for k in keys}


def summary(line):
    """The secondary targets of the line in one small object."""
    def get(*path):
        d = line
        for k in path:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d
    return {"injections_s": line["value"], "e2e_injections_s": get("e2e", "value"),
            "plain_loop_injections_s": get("plain_loop", "value"),
            "speedup_vs_plain_loop": line.get("speedup_vs_plain_loop"),
            "k_dirty_roofline_frac": get("roofline", "frac"),
            "guard_field_frac_of_hbm": get("guard", "field", "frac"),
            "guard_prim_frac_of_hbm": get("guard", "prim", "frac"),
            "p99_frame_latency_ms": line.get("p99_frame_latency_ms"),
            "cpu_baseline_injections_s": get("cpu_baseline", "value")}


def contamination(G, S, h, scene, K_views, dev, count=256):
    """Sort-first partition of the screen into 4-64 nodes: the fraction of nodes
    that log-scale sign-bit upsets contaminate (actual: nodes whose pixels
    change; predicted: nodes the primitive's footprint reaches), with the guard
    off and with the FIELD guard, and the IoU of predicted and actual."""
    import torch
    from paper_2606_21791_gb300 import contamination as CT
    rng = np.random.default_rng(S.SEED_BASE + 110)
    fl = S.flips_at(rng.integers(0, scene.n, count).astype(np.uint32), rng.integers(3, 6, count), 31)
    d = G.to_device(fl, dev)
    out = G.device_bytes(count * K_views * 24, dev)
    reg = torch.zeros(count * K_views * 2, dtype=torch.int64, device=dev)
    res = {"upsets": f"{count} log-scale sign-bit upsets (words 3-5, bit 31), {K_views} views each",
           "cells": "8x8 screen grid; partitions 2x2, 4x2, 4x4, 8x4, 8x8"}
    for name, mode in (("no_guard", G.GS_GUARD_OFF), ("field_guard", G.GS_GUARD_FIELD)):
        G.gs_inject_and_render_regions(h, d, count, mode, S.GUARD_WORDS_DEFAULT, out, reg)
        torch.cuda.synchronize()
        r = reg.cpu().numpy().view(np.uint64).reshape(count * K_views, 2)
        res[name] = {str(k): v for k, v in CT.summary(r[:, 0], r[:, 1]).items()}
    return res


def campaign_analytics(G, S, dev):
    """Table 2 on the 134,826-Gaussian stratified campaign (50,000 upsets, fp32,
    800x800), with the campaign's own injection rate, and the scaling law of the
    median / mean single-upset error (MSE) over model sizes 5k-300k (20,000
    upsets each on the log-scale sign and exponent bits), guard off and FIELD
    guard."""
    import torch
    from paper_2606_21791_gb300 import analytics as AN
    res = {}
    sc, cams, fl = S.batching_workload(S.FP32)
    h = G.gs_load_scene(sc.planes, sc.n, 3, S.FP32)
    G.gs_set_views(h, cams)
    d = G.to_device(fl, dev)
    out = G.device_bytes(len(fl) * 24, dev)
    G.gs_inject_and_render(h, d[:8 * 512], 512, 1, G.GS_GUARD_OFF, S.GUARD_WORDS_DEFAULT, out)   # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    G.gs_inject_and_render(h, d, len(fl), 1, G.GS_GUARD_OFF, S.GUARD_WORDS_DEFAULT, out)
    e1.record()
    torch.cuda.synchronize()
    rec = G.from_device(out, G.RESULT_DTYPE).reshape(len(fl), 1)
    G.gs_free_scene(h)
    res["table2"] = {"workload": "134,826 Gaussians (4 clusters, SH 3, fp32), 800x800, 50,000 stratified upsets",
                     "injections_per_s": len(fl) / (e0.elapsed_time(e1) / 1000.0),
                     "fields": AN.severity_table(fl, rec, 800 * 800)}
    sizes = [5_000, 20_000, 80_000, 300_000]
    med = {"no_guard": [], "field_guard": []}
    mean = {"no_guard": [], "field_guard": []}
    zero = {"no_guard": [], "field_guard": []}
    for n in sizes:
        sc = S.make_scene(n, 3, S.FP32, S.SEED_BASE + 120 + n % 97, layout="clusters")
        cams = S.ring_cameras(1, 800, 800)
        # the cells that carry the error: log-scale sign and exponent bits
        rng = np.random.default_rng(S.SEED_BASE + 121)
        fl = S.flips_at(rng.integers(0, sc.n, 20_000).astype(np.uint32), rng.integers(3, 6, 20_000),
                        rng.integers(23, 32, 20_000))
        h = G.gs_load_scene(sc.planes, sc.n, 3, S.FP32)
        G.gs_set_views(h, cams)
        d = G.to_device(fl, dev)
        out = G.device_bytes(len(fl) * 24, dev)
        for name, mode in (("no_guard", G.GS_GUARD_OFF), ("field_guard", G.GS_GUARD_FIELD)):
            G.gs_inject_and_render(h, d, len(fl), 1, mode, S.GUARD_WORDS_DEFAULT, out)
            torch.cuda.synchronize()
            mse = G.from_device(out, G.RESULT_DTYPE)["sse"] / (800 * 800 * 3)
            med[name].append(float(np.median(mse)))
            mean[name].append(float(mse.mean()))
            zero[name].append(float((mse == 0).mean()))
        G.gs_free_scene(h)
    fits = {}
    for name in med:
        a, _, r2 = AN.loglog_fit(sizes, med[name])
        am, _, r2m = AN.loglog_fit(sizes, mean[name])
        fits[name] = {"median_mse": med[name], "mean_mse": mean[name], "zero_error_frac": zero[name],
                      "alpha_median": a, "r2_median": r2, "alpha_mean": am, "r2_mean": r2m}
    res["scaling"] = {"sizes": sizes, "upsets_per_size": "20,000 on log-scale sign/exponent bits (words 3-5, bits 23-31)",
                      "error": "per-variant MSE (800x800x3)", **fits,
                      "guard_mean_error_factor_at_largest": mean["no_guard"][-1] / max(mean["field_guard"][-1], 1e-30)}
    return res


def batching_formats(G, S, dev):
    """The 134,826-Gaussian campaign (4 clusters, SH 3, 800x800, one view, 50,000
    upsets stratified over every (word, bit) cell of the format) in each storage
    format, fp32, fp16 and bf16, with the guard off and with per-primitive (PRIM)
    boxes on the 14 non-SH-rest words: injections/s of the whole campaign at
    32 variants per launch and at the batch the autotuner picks."""
    import torch
    res = {"workload": "134,826 Gaussians (4 clusters, SH 3), 800x800, 1 view, 50,000 stratified upsets"}
    for fmt, fname in ((S.FP32, "fp32"), (S.FP16, "fp16"), (S.BF16, "bf16")):
        sc, cams, fl = S.batching_workload(fmt, count=50_000)
        h = G.gs_load_scene(sc.planes, sc.n, 3, fmt)
        lo, hi = S.prim_boxes(sc, 14, S.SEED_BASE + 60)
        G.gs_set_prim_box(h, lo, hi, 14)
        G.gs_set_views(h, cams)
        d = G.to_device(fl, dev)
        out = G.device_bytes(len(fl) * 24, dev)
        b_auto, _ = G.gs_autotune(h, d, 8192, G.GS_GUARD_OFF, S.GUARD_WORDS_DEFAULT)
        row = {"autotuned_batch": b_auto}
        for gname, gmode in (("guard_off", G.GS_GUARD_OFF), ("prim_guard", G.GS_GUARD_PRIM)):
            for bname, b in (("batch_32", 32), ("batch_auto", b_auto)):
                G.gs_set_batch(h, b)
                G.gs_inject_and_render(h, d[:8 * 512], 512, 1, gmode, S.GUARD_WORDS_DEFAULT, out)   # warm, capture
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                G.gs_inject_and_render(h, d, len(fl), 1, gmode, S.GUARD_WORDS_DEFAULT, out)
                e1.record()
                torch.cuda.synchronize()
                row[f"{gname}_{bname}"] = len(fl) / (e0.elapsed_time(e1) / 1000.0)
        res[fname] = row
        G.gs_free_scene(h)
        del d, out
    torch.cuda.empty_cache()
    return res


def ssim_campaign(G, S, h, d_flips, nflips, K_views, dev, count=1024):
    """The campaign with the per-(variant, view) SSIM on and off (same upsets):
    injections/s of each, and the SSIM distribution.  The dirty-tile SSIM runs
    on 16x16 tiles: another tuned shape is set aside for this section and put
    back after it."""
    tile = G.gs_get_tile(h)
    if tile != (16, 16):
        G.gs_set_tile(h, 16, 16)
    try:
        res = _ssim_campaign(G, S, h, d_flips, nflips, K_views, dev, count)
    finally:
        if tile != (16, 16):
            G.gs_set_tile(h, *tile)
    res["tiles"] = "16x16"
    return res


def _ssim_campaign(G, S, h, d_flips, nflips, K_views, dev, count):
    import torch
    count = min(count, nflips)
    out = G.device_bytes(count * K_views * 24, dev)
    ss = torch.zeros(count * K_views, dtype=torch.float64, device=dev)
    d = d_flips[:8 * count]
    res = {}
    for name, arg in (("with_ssim", ss), ("without", None)):
        G.gs_inject_and_render_ex(h, d, count, G.GS_GUARD_OFF, S.GUARD_WORDS_DEFAULT, out, None, arg)   # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            G.gs_inject_and_render_ex(h, d, count, G.GS_GUARD_OFF, S.GUARD_WORDS_DEFAULT, out, None, arg)
        e1.record()
        torch.cuda.synchronize()
        res[name + "_injections_per_s"] = 3 * count / (e0.elapsed_time(e1) / 1000.0)
    v = ss.cpu().numpy()
    res.update({"upsets": f"{count} of the benchmark's upsets, {K_views} views each",
                "mean_ssim": float(v.mean()), "min_ssim": float(v.min()),
                "frac_below_0.99": float((v < 0.99).mean())})
    return res


def render_stages(G, S, h, cams, flush, dev, pk, pk_kind, reps=10):
    """Stage split of one full render of view 0 (the pipeline the plain loop runs
    per variant): CUDA events inside gs_render bracket the preprocess, the
    binning with its radix sorts and the blend; medians over `reps` renders, L2
    flushed before each.  Algorithmic bytes: the preprocess reads every word of
    every primitive and writes its 48-B blend record, 8-B tile rect and 8-B
    depth-sort pair; the tile lists are 8-B (tile, primitive) pairs written once
    and read once.  The radix passes move 20 B per element (the histogram reads
    the 4-B key, the scatter reads and writes key and value), the tile count and
    emit read 20 B per primitive and write 8 B per pair, the range pass reads 4 B
    per pair."""
    import torch
    cam = cams[:1]
    W, H = int(cam[0]["width"]), int(cam[0]["height"])
    img = torch.empty(H * W * 3, dtype=torch.float32, device=dev)
    G.gs_time_kernels(h, True)
    rows = []
    for i in range(3 + reps):
        flush.zero_()
        if i == 3:
            torch.cuda.nvtx.range_push("render_stages")
        G.gs_render(h, cam, img)
        if i >= 3:
            rows.append(G.gs_read_render_ms(h))
    torch.cuda.nvtx.range_pop()
    G.gs_time_kernels(h, False)
    pre_ms, sort_ms, blend_ms = (sorted(r[0][j] for r in rows)[len(rows) // 2] for j in range(3))
    n, pairs, passes_depth, passes_pairs = rows[-1][1]
    _, _, fmt, nwords = G.gs_scene_info(h)
    wbytes = 4 if fmt == S.FP32 else 2
    pre_bytes = n * (nwords * wbytes + 64)
    sort_alg = pairs * 16
    sort_moved = 20 * (n * passes_depth + pairs * passes_pairs) + 20 * n + 12 * pairs
    hbm = pk.get("hbm_gbs")
    gbs = lambda b, ms: b / (ms * 1e-3) / 1e9
    frame = pre_ms + sort_ms + blend_ms
    return {
        "what": f"full render of one {W}x{H} view of the benchmark scene, stage medians of {reps} (CUDA events)",
        "frame_ms": frame,
        "preprocess": {"ms": pre_ms, "share": pre_ms / frame, "bytes": pre_bytes,
                       "gbs": gbs(pre_bytes, pre_ms), "frac_of_hbm_peak": gbs(pre_bytes, pre_ms) / hbm,
                       "bytes_per_primitive": nwords * wbytes + 64},
        "bin_sort": {"ms": sort_ms, "share": sort_ms / frame, "primitives": n, "pairs": pairs,
                     "radix_passes": {"depth_keys": passes_depth, "pair_tile_keys": passes_pairs},
                     "algorithmic_bytes": sort_alg, "gbs_algorithmic": gbs(sort_alg, sort_ms),
                     "bytes_moved_by_passes": sort_moved, "gbs_passes": gbs(sort_moved, sort_ms),
                     "frac_of_hbm_peak_passes": gbs(sort_moved, sort_ms) / hbm},
        "blend": {"ms": blend_ms, "share": blend_ms / frame, "mpix_s": W * H / (blend_ms * 1e-3) / 1e6,
                  "pairs_per_us": pairs / (blend_ms * 1e3)},
        "peak": {"hbm_gbs": hbm, "source": pk_kind},
    }


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


def serving(args, G, S, dev):
    """Serving loop: 4 resident scenes (6,741 / 134,826 / 300,000 / 2,000,000
    Gaussians, SH 3, fp16 storage), mixed 800x800 and 1600x1040 render requests
    with Poisson arrivals at 50/80/95% of the measured capacity plus interleaved
    1,000-upset campaigns, and an upset storm (1,000 upsets per frame, 300 frames)
    on the largest scene with the guard on and off."""
    import torch
    rng = np.random.default_rng(S.SEED_BASE + 40)
    sizes = (6_741, 134_826, 300_000, 2_000_000)
    t0 = time.perf_counter()
    scenes = [S.make_scene(n, 3, S.FP16, S.SEED_BASE + 41 + i, layout="clusters") for i, n in enumerate(sizes)]
    handles = [G.gs_load_scene(sc.planes, sc.n, 3, S.FP16) for sc in scenes]
    G.gs_set_views(handles[1], S.ring_cameras(1, 800, 800))          # campaign target
    camp_flips = S.flips_stratified(1000, sizes[1], 59, S.FP16, S.SEED_BASE + 42)
    d_camp = G.to_device(camp_flips, dev)
    camp_out = G.device_bytes(1000 * 24, dev)
    slots = 4
    srv = G.gs_server_create(200 << 30, slots)
    ids = [G.gs_server_add_scene(srv, h) for h in handles]
    res = [(800, 800), (1600, 1040)]
    pool = [torch.empty(1600 * 1040 * 3, dtype=torch.float32, device=dev) for _ in range(48)]

    def make(i):
        if i % 10 == 9:
            return G.make_request(G.GS_REQ_CAMPAIGN, ids[1], dev_flips=d_camp, nflips=1000, dev_results=camp_out)
        W, H = res[int(rng.integers(0, 2))]
        cam = S.ring_cameras(1, W, H, elevation_deg=float(rng.uniform(-30, 30)))[0]
        return G.make_request(G.GS_REQ_RENDER, ids[int(rng.integers(0, 4))], cam, dev_rgb=pool[i % len(pool)])

    # warm every path (scratch growth, graph capture)
    for i in range(12):
        G.gs_server_wait(srv, G.gs_server_submit(srv, make(i)))
    # capacity: closed loop, `slots` requests in flight
    n_cap = 120
    reqs = [make(i) for i in range(n_cap)]
    c0 = time.perf_counter()
    inflight = []
    for i, r in enumerate(reqs):
        inflight.append(G.gs_server_submit(srv, r))
        if len(inflight) >= 2 * slots:
            G.gs_server_wait(srv, inflight.pop(0))
    for t in inflight:
        G.gs_server_wait(srv, t)
    cap_rps = n_cap / (time.perf_counter() - c0)
    # open loop: Poisson arrivals at fractions of capacity; latency = scheduled
    # arrival -> done (the arrival time is passed to the server, so a submitter
    # that falls behind does not hide queueing)
    def open_loop(server, rate, n, seed_off):
        gaps = rng.exponential(1000.0 / rate, size=n)   # ms
        reqs = [make(seed_off + i) for i in range(n)]
        off = G.gs_server_now(server) - time.perf_counter() * 1000.0   # server ms = perf ms + off
        t_first = G.gs_server_now(server) + 2.0
        arrivals = t_first + np.cumsum(gaps)
        tickets = []
        for i in range(n):
            while time.perf_counter() * 1000.0 + off < arrivals[i]:
                time.sleep(0.0001)
            tickets.append(G.gs_server_submit(server, reqs[i], float(arrivals[i])))
        lat, last = [], 0.0
        for t in tickets:
            r = G.gs_server_wait(server, t)
            lat.append(r["t_done_ms"] - r["t_submit_ms"])
            last = max(last, r["t_done_ms"])
        span_s = (last - t_first) / 1000.0
        return {"requests": n, "offered_rps": rate, "throughput_rps": n / span_s, "p50_ms": _pct(lat, 0.5),
                "p99_ms": _pct(lat, 0.99), "mean_ms": sum(lat) / n}

    n_open = 2000
    poisson = []
    for j, load in enumerate((0.5, 0.8, 0.95)):
        row = open_loop(srv, load * cap_rps, n_open, 1000 + j * n_open)
        row["load"] = load
        poisson.append(row)
    G.gs_server_destroy(srv)
    # the same mix at 80% load under a budget that holds the resident scenes and
    # the render scratch of two requests at most: admission has to wait for memory
    srv = G.gs_server_create(1 << 50, 1)   # one slot: the scratch of the largest request alone
    big = [G.gs_server_add_scene(srv, hh) for hh in handles][-1]
    cam_big = S.ring_cameras(1, 1600, 1040)[0]
    G.gs_server_wait(srv, G.gs_server_submit(srv, G.make_request(G.GS_REQ_RENDER, big, cam_big, dev_rgb=pool[0])))
    st0 = G.gs_server_stats(srv)
    G.gs_server_destroy(srv)
    scratch_big = st0["scratch"]
    budget = st0["resident"] + 2 * scratch_big + (64 << 20)
    srv = G.gs_server_create(budget, slots)
    ids = [G.gs_server_add_scene(srv, hh) for hh in handles]
    for i in range(8):
        G.gs_server_wait(srv, G.gs_server_submit(srv, make(i)))
    tight = open_loop(srv, 0.8 * cap_rps, n_open, 20000)
    stt = G.gs_server_stats(srv)
    G.gs_server_destroy(srv)
    tight.update({"load": 0.8, "budget_bytes": budget, "resident_bytes": st0["resident"],
                  "scratch_bytes_largest_request": scratch_big,
                  "delayed_by_budget_frac": stt["mem_delayed"] / (n_open + 8), "refused": 0})
    # upset storm on the largest scene: 1,000 upsets accumulate per frame
    storm = {}
    lo3, hi3 = S.prim_boxes(scenes[3], 14, S.SEED_BASE + 44)
    for name, guard in (("guard_prim", G.GS_GUARD_PRIM), ("guard_field", G.GS_GUARD_FIELD),
                        ("guard_off", G.GS_GUARD_OFF)):
        h = G.gs_load_scene(scenes[3].planes, scenes[3].n, 3, S.FP16)
        if guard == G.GS_GUARD_PRIM:
            G.gs_set_prim_box(h, lo3, hi3, 14)
        srv = G.gs_server_create(200 << 30, 1)
        sid = G.gs_server_add_scene(srv, h)
        cam = S.ring_cameras(1, 1600, 1040)[0]
        img = torch.empty(1600 * 1040 * 3, dtype=torch.float32, device=dev)
        frames = 300
        fl = S.flips_multi(1000 * frames, scenes[3].n, 59, S.FP16, S.SEED_BASE + 43)
        d_fl = G.to_device(fl, dev)
        lat = []
        for f in range(frames + 5):
            fi = f % frames
            r = G.make_request(G.GS_REQ_STORM, sid, cam, guard_mode=guard,
                               word_mask=S.GUARD_WORDS_DEFAULT, dev_flips=d_fl[fi * 8000:(fi + 1) * 8000], nflips=1000,
                               dev_rgb=img)
            resp = G.gs_server_wait(srv, G.gs_server_submit(srv, r))
            if f >= 5:
                lat.append(resp["t_done_ms"] - resp["t_submit_ms"])
        finite = bool(torch.isfinite(img).all().item())
        G.gs_server_destroy(srv)
        G.gs_free_scene(h)
        storm[name] = {
            "frames": frames, "upsets_per_frame": 1000, "p50_ms": _pct(lat, 0.5), "p99_ms": _pct(lat, 0.99),
            "mean_ms": sum(lat) / len(lat), "last_frame_finite": finite}
    for h in handles:
        G.gs_free_scene(h)
    torch.cuda.empty_cache()
    log(f"[bench] serving measured in {time.perf_counter() - t0:.1f}s")
    return {"scenes": list(sizes), "storage": "fp16", "slots": slots, "capacity_rps": cap_rps,
            "mix": "90% renders (random scene, 800x800 or 1600x1040, random view), 10% 1,000-upset campaigns on the "
                   "134,826-Gaussian scene (800x800)",
            "poisson": poisson, "budget_bound": tight, "storm": storm,
            "latency": "host ms from the scheduled arrival (open loop, passed to the server) or submission (storm) "
                       "to completion of the request's stream"}


def guard_frame(G, S, h, n, dev, guard_ms):
    """One 2592x1944 frame of the guard-stress scene, the guard's share of a
    guarded frame, and k simultaneous upsets (k = 1, 1,000, 20,000) rendered
    without and with the FIELD guard: PSNR against the clean frame."""
    import torch
    W, H = 2592, 1944
    cam = S.look_at_camera((0.0, 0.0, 15.0), width=W, height=H)
    stream = torch.cuda.current_stream()
    clean = torch.empty(W * H * 3, dtype=torch.float32, device=dev)
    img = torch.empty_like(clean)
    G.gs_render(h, cam, clean)                       # sizes the scratch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.nvtx.range_push("frame_66M")
    ev[0].record(stream)
    G.gs_render(h, cam, clean)
    ev[1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    frame_ms = ev[0].elapsed_time(ev[1])
    saved = torch.empty(n * 59, dtype=torch.int32, device=dev)
    G.gs_read_planes(h, saved)
    out = G.device_bytes(24, dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    dose = []
    for k in (1, 1000, 20000):
        fl = S.flips_multi(k, n, 59, S.FP32, S.SEED_BASE + 50 + k)
        d = G.to_device(fl, dev)
        row = {"k": k}
        for guard in (False, True):
            G.gs_write_planes(h, saved)
            G.gs_apply_flips(h, d, k)
            if guard:
                cnt.zero_()
                G.gs_guard(h, 0, S.GUARD_WORDS_DEFAULT, cnt)
            G.gs_render(h, cam, img)
            G.gs_compare(img, clean, H, W, 1, out)
            r = G.from_device(out, G.RESULT_DTYPE)[0]
            mse = max(float(r["sse"]) / (W * H * 3), 1e-10)
            key = "guard" if guard else "no_guard"
            row[key] = {"psnr_db": 10 * math.log10(1 / mse), "footprint": float(r["footprint"]) / (W * H),
                        "nonfinite_px": int(r["nonfinite"])}
            if guard:
                row[key]["clamps"] = int(cnt.item())
        dose.append(row)
    G.gs_write_planes(h, saved)
    del saved
    return {"resolution": f"{W}x{H}", "render_ms": frame_ms, "guard_ms": guard_ms,
            "guard_share_of_guarded_frame": guard_ms / (guard_ms + frame_ms), "dose": dose}


def guard_stress(args, G, S, dev, pk, pk_kind):
    """Support-guard clamp (Algorithm 1) over a 66M-Gaussian SH-3 fp32 scene:
    FIELD boxes (56 B/primitive read) and per-primitive boxes (168 B read)."""
    import torch
    n = args.guard_n
    t0 = time.perf_counter()
    planes = S.make_scene_torch(n, 3, S.FP32, S.SEED_BASE + 4, device=dev)
    h = G.gs_load_scene(planes, n, 3, S.FP32)
    lo, hi = S.prim_boxes_torch(planes, S.FP32, 14, S.SEED_BASE + 5)
    del planes
    torch.cuda.empty_cache()
    G.gs_set_prim_box(h, lo, hi, 14)
    del lo, hi
    torch.cuda.empty_cache()
    log(f"[bench] guard scene {n} ready in {time.perf_counter() - t0:.1f}s")
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    res = {"gaussians": n, "words_guarded": 14, "peak_hbm_gbs": pk["hbm_gbs"], "peak_source": pk_kind}
    for mode, name, bytes_per in ((0, "field", 14 * 4), (1, "prim", 14 * 4 * 3)):
        for _ in range(3):
            G.gs_guard(h, mode, S.GUARD_WORDS_DEFAULT, cnt)
        reps = 10
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.nvtx.range_push(f"guard_{name}")
        for a, b in evs:
            a.record(stream)
            G.gs_guard(h, mode, S.GUARD_WORDS_DEFAULT, cnt)
            b.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = [a.elapsed_time(b) for a, b in evs]
        t = statistics.median(ms) / 1000.0
        gbs = n * bytes_per / t / 1e9
        res[name] = {"ms": t * 1000, "gb_s": gbs, "frac": gbs / pk["hbm_gbs"], "bytes_per_launch": n * bytes_per,
                     "clamps": int(cnt.item())}
    if not args.only_guard:
        res["frame"] = guard_frame(G, S, h, n, dev, res["field"]["ms"])
    G.gs_free_scene(h)
    torch.cuda.empty_cache()
    return res


if __name__ == "__main__":
    main()
