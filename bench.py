"""Throughput of the multi-hypothesis featuremetric LM pose solver on GB300.

Metric: hypothesis x LM-iterations per second on the full single-frame workload
(256^2-anchor TDOM/DSM crop at 0.5 m, C = 32 FP32 descriptors, 3-level query pyramid
480x640 / 240x320 / 120x160, 64 hypotheses, 10 LM iterations per level, gravity and
laser-range priors on).  One step = one whole solve of one frame: every level, every
iteration, every hypothesis, the priors, the damped solves and the final selection.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`value` is measured with the frame resident in device memory (CUDA events around each
solve on the solve's stream, L2 flushed by a 512 MiB write between steps, outside the
events).  `e2e` is the same metric through the C-ABI with page-locked HOST buffers, the
host->device copies of the frame and the device->host copy of the results inside the
timed region.  `--impl reference` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.  Under torchrun every rank solves its own frame
(independent replicas, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
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

METRIC = "hypothesis·LM-iters/sec (256² crop, C=32)"
UNIT = "hyp*iter/s"
WORKLOAD = ("full single frame: 256x256 anchors at 0.5 m, C=32, 3 levels 480x640/240x320/120x160, "
            "64 hypotheses, 10 LM iterations per level, gravity + range priors")
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
BUILD_SRC = os.path.join(ROOT, "paper_2606_31098_gb300", "csrc", "pilot_build_impl.cuh")
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per (anchor, hypothesis) unit of the FP32 build pass at C = 32,
# from one ncu capture of a finest-level launch of the full frame (dram__bytes_read.sum +
# dram__bytes_write.sum = 15 055 104 B over its 2 097 152 units; a coarse-level launch: 4.86 B
# per unit), valid for the kernel source with this SHA-256 prefix; None otherwise.
BUILD_TRAFFIC = {"src_sha256_16": "9465498ff6a231dc", "dram_bytes_per_unit": 7.178}


def flops_per_unit(C: int) -> int:
    """Algorithmic FP32 flops of one (anchor, hypothesis) evaluation, as the scope table
    counts them: about 40 per channel (bilinear value and two gradients 28, dequantisation
    3, residual 1, the six sums 12... rounded to 40) plus about 150 per anchor (transform,
    projection, A, A^T M A, A^T b): 1430 at C = 32."""
    return 40 * C + 150


def executed_flops_per_unit(C: int) -> int:
    """FP32 flops the build pass actually executes per unit (FMA = 2): 25 per channel
    (bilinear value and gradients from shared tap differences 12, residual 1, six sums 12)
    plus 200 per anchor (transform 18, projection 10, Huber 6, Jacobian rows 12, M A 36,
    weights 12, 21 H entries 84, 6 g entries 24): 1000 at C = 32."""
    return 25 * C + 200


def gather_bytes_per_unit(C: int, elem: int) -> int:
    """Bytes of the 4-tap bilinear gather of one (anchor, hypothesis) evaluation."""
    return 4 * C * elem


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed-index", type=int, default=0)
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--pin-schedule", default="", metavar="TILE:STREAMS",
                    help="skip the autotuner: plain form with this tile and stream count, batched form with "
                         "this tile (for profiling runs, whose timings would mislead the autotuner)")
    ap.add_argument("--crop-only", action="store_true",
                    help="profiling entry point: only the reference-crop timing, printed as one JSON line")
    ap.add_argument("--batched-only", action="store_true",
                    help="profiling entry point: only the batched-form timings, printed as one JSON line")
    ap.add_argument("--served-only", action="store_true",
                    help="profiling entry point: only the served-form stream sweep, printed as one JSON line")
    ap.add_argument("--paper-schedule-only", action="store_true",
                    help="profiling entry point: only the plain paper-schedule solve (3 warm-up + 20 timed "
                         "solves of one frame), printed as one JSON line")
    return ap.parse_args()


def paper_schedule_only(B, S, torch):
    """The plain paper-schedule solve alone (see paper_schedule_form), for ncu captures."""
    f = S.make_frame(S.config_paper_schedule(), S.frame_seed(6, 0))
    solver = B.Solver(B.Options(iters=(4, 3, 2, 0), keep_top_k=(0, 0, 128, 0), max_points=500, max_hyps=1210))
    fa = B.FrameArgs(f, B.device_arrays(f), is_device=True)
    st = torch.cuda.current_stream()
    for _ in range(3):
        solver.solve(fa, st)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(20):
        r = solver.solve(fa, st)
    e1.record(st)
    e1.synchronize()
    print(json.dumps({"form": "paper_schedule_plain_f32", "ms_per_frame": e0.elapsed_time(e1) / 20,
                      "hyp_iters": r.hyp_iters, "schedule": solver.schedule([fa], batched=False)}), flush=True)
    solver.close()
    return 0


def max_over_ranks(values, world: int, device: str):
    """Element-wise maximum of a list of floats over all ranks (identity for one rank)."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_throughput(units_per_rank: int, max_ms: float, world: int) -> float:
    """Whole-job rate of independent replicas: every rank processed units_per_rank in at
    most max_ms (the slowest rank's time)."""
    return world * units_per_rank / (max_ms / 1e3)


def rank_seed_index(seed_index: int, rank: int) -> int:
    """Each replica solves its own frame (no data-path exchange)."""
    return seed_index + rank


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
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
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hw_thermal=parts[6], sw_thermal=parts[7], sw_power=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hw_thermal", "hw_thermal_slowdown"),
                              ("sw_thermal", "sw_thermal_slowdown"), ("sw_power", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


def load_peaks():
    try:
        return json.load(open(MEASURED_PEAKS))
    except Exception:
        return None


def build_src_hash() -> str:
    return hashlib.sha256(open(BUILD_SRC, "rb").read()).hexdigest()[:16]


def traffic_per_launch(units_per_launch: int):
    """DRAM bytes per build launch: BUILD_TRAFFIC's per-unit figure scaled to the units of
    one launch; None when the kernel source changed since the counters were taken."""
    if BUILD_TRAFFIC["dram_bytes_per_unit"] is None or BUILD_TRAFFIC["src_sha256_16"] != build_src_hash():
        return None
    return BUILD_TRAFFIC["dram_bytes_per_unit"] * units_per_launch


def frame_gather_ceiling(B, torch, frame, dev, C, elem, dtype, tile, stream):
    """Gather ceiling of the build pass on this frame: pilot_probe_gather_frame at every
    level with the hypotheses' start poses (the frame's own locality), combined over the
    levels as the solve weights them (equal units per level).  Returns units per second."""
    poses = torch.as_tensor(np.asarray(frame.T_hyps, np.float32).reshape(-1, 12), device="cuda")
    total_s = 0.0
    for level in range(frame.L):
        s = 2.0 ** -level
        rate = B.probe_gather_frame(dev.arrays["points"], dev.arrays["qry_feat"][level], dev.arrays["ref_feat"][level],
                                    dtype, frame.fx * s, frame.fy * s, frame.cx * s, frame.cy * s, poses, tile, stream)
        total_s += frame.N * frame.M / rate
    return frame.L * frame.N * frame.M / total_s


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def make_frames(S, specs):
    """Seeded synthetic frames built in parallel on the host cores (spawned workers: no
    CUDA state is inherited)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(16, cpu_cores(), len(specs)))) as pool:
        return pool.starmap(S.make_frame, specs)


def batched_and_served(args, B, S, torch, world, stream, served_too: bool = True, gmap=None):
    """The batched form (one persistent launch per level under a CUDA graph) on BF16
    storage, and the served form (served_streams).

    * uneven32_bf16: 32 independently generated scenes, crop sides drawn uniformly from
      {128, 192, 256, 384}^2 anchors, 16-144 hypotheses each, 3 levels, priors on.
    * crop256: 8 independently generated 256^2-anchor frames (64 hypotheses): the plain
      form solving them one at a time in FP32 and in BF16, and the batched BF16 form
      solving all 8 in one batch -- the comparison the metric is quoted on."""
    rng = np.random.default_rng(12345)
    sides_all = (128, 192, 256, 384)
    sides = [int(sides_all[k]) for k in rng.integers(0, 4, 32)]
    hyps = [int(m) for m in rng.integers(16, 145, 32)]
    specs = [(S.SceneConfig(crop_side=sd, n_hyps=m), S.frame_seed(3, 5000 + i)) for i, (sd, m) in enumerate(zip(sides, hyps))]
    specs += [(S.config_full_frame(), S.frame_seed(3, 6000 + i)) for i in range(8)]
    frames = make_frames(S, specs)
    uneven_frames, f256 = frames[:32], frames[32:40]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def bf16_args(f):
        return B.FrameArgs(f, B.quantized_device_arrays(f, B.BF16), is_device=True, dtype=B.BF16)

    def time_batch(fas, reps):
        solver = B.Solver(B.Options(max_points=384 * 384, max_hyps=sum(fa.M for fa in fas), max_frames=len(fas)))
        if args.pin_schedule:
            solver.set_schedule(fas, batched=True, tile=int(args.pin_schedule.split(":")[0]))
            sched = solver.schedule(fas, batched=True)
        else:
            sched, _ = solver.autotune(fas, batched=True, reps=1, stream=stream)
        solver.solve_batch(fas, stream)
        ts, units = [], 0
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = solver.solve_batch(fas, stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            units += sum(r.hyp_iters for r in res)
        solver.close()
        return world * units / (sum(ts) / 1e3), sum(ts) / reps, sched

    def time_plain(fas, reps):
        solver = B.Solver(B.Options(max_points=max(fa.c.N for fa in fas), max_hyps=max(fa.M for fa in fas)))
        if args.pin_schedule:
            tile, streams = (int(v) for v in args.pin_schedule.split(":"))
            solver.set_schedule(fas[:1], batched=False, tile=tile, streams=streams)
            sched = solver.schedule(fas[:1], batched=False)
        else:
            sched, _ = solver.autotune(fas[:1], batched=False, reps=2, stream=stream)
        for fa in fas:
            solver.solve(fa, stream)
        ts, units = [], 0
        for _ in range(reps):
            for fa in fas:
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = solver.solve(fa, stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
                units += r.hyp_iters
        solver.close()
        return world * units / (sum(ts) / 1e3), sched

    uneven = [bf16_args(f) for f in uneven_frames]
    v_uneven, ms_uneven, sc_uneven = time_batch(uneven, 3)
    v_uneven_plain_bf16, _ = time_plain(uneven, 1)
    del uneven
    uneven32 = [B.FrameArgs(f, B.device_arrays(f), is_device=True) for f in uneven_frames]
    v_uneven_plain_f32, _ = time_plain(uneven32, 1)
    del uneven32
    a256_bf16 = [bf16_args(f) for f in f256]
    a256_f32 = [B.FrameArgs(f, B.device_arrays(f), is_device=True) for f in f256]
    v_plain_f32, sc_pf = time_plain(a256_f32, 2)
    v_plain_bf16, sc_pb = time_plain(a256_bf16, 2)
    v_256, ms_256, sc_256 = time_batch(a256_bf16, 3)
    del a256_f32
    batched = {"uneven32_bf16": {"value": v_uneven, "unit": UNIT, "ms_per_batch": ms_uneven, "frames": 32,
                                 "distinct_scenes": 32, "crops": "128^2..384^2 (uniform over 4 sides)",
                                 "hypotheses": "16..144", "schedule": sc_uneven,
                                 "plain_bf16_same_frames": v_uneven_plain_bf16,
                                 "plain_f32_same_frames": v_uneven_plain_f32},
               "crop256": {"frames": 8, "distinct_scenes": 8, "hypotheses": 64, "unit": UNIT,
                           "plain_f32": v_plain_f32, "plain_bf16": v_plain_bf16, "batched_bf16": v_256,
                           "ms_per_batch_bf16": ms_256, "schedules": {"plain_f32": sc_pf, "plain_bf16": sc_pb,
                                                                      "batched_bf16": sc_256}}}

    if not served_too:
        return batched, {}
    return batched, served_streams(B, S, torch, gmap)


def served_streams(B, S, torch, g, counts=(1, 4, 16, 64), duration: float = 4.0, seed: int = 8_000_000,
                   reserved_sms: int = 8):
    """The served form on the serving workload: UAV streams at 30 Hz (exponential
    inter-arrival, mean 33 ms) over one 4096^2 map at 0.5 m, each a smooth trajectory
    (altitude 100-300 m, pitch 30-70 deg, heading rate up to 10 deg/s, 10 m/s); per frame a
    device crop of 128^2 .. 384^2 anchors around the stream's previous estimate, a grid of
    16-144 hypotheses around it, BF16 features, submitted to one server with a 16 GiB arena
    (admission by slots, hypotheses and arena memory); the newest arrived frame of a stream
    is taken when its previous result returns.  Swept over stream counts; each point
    `duration` s of arrivals.  Reports the sustainable rate and arrival-to-result latency."""
    from paper_2606_31098_gb300 import serving as SV
    from paper_2606_31098_gb300 import tracking as TK
    sc = S.StreamConfig(n_frames=int(duration * 30.0) + 30)
    n_max = max(counts)
    inputs = []
    for s_ in range(n_max):
        gt = S.stream_trajectory(g, sc, seed + s_)
        inputs.append((gt, S.stream_sensors(g, sc, gt, seed + 1000 + s_)))
    net = S.StreamNetwork(sc, seed + 99)
    dsm_dev = torch.as_tensor(g.dsm, device="cuda")
    H0, W0 = sc.levels[0]
    cam = TK.Camera(sc.f0, sc.f0, W0 / 2.0, H0 / 2.0, W0, H0)
    rng = np.random.default_rng(seed)
    arrivals = []
    for _ in range(n_max):
        a = rng.uniform(0.0, 1.0 / sc.rate_hz) + np.concatenate([[0.0], np.cumsum(rng.exponential(1.0 / sc.rate_hz, sc.n_frames - 1))])
        arrivals.append(a)
    budget = 16 << 30
    out = {"workload": "UAV streams at 30 Hz over a 4096^2 map at 0.5 m, per-frame device crop 128^2..384^2 "
                       "anchors around the previous estimate, 16-144 grid hypotheses, BF16, 3 levels",
           "hbm_budget_bytes": budget, "max_slots": 64, "reserved_sms": reserved_sms,
           "duration_s_per_point": duration, "sweep": []}
    # untimed warm-up: the first crops, network calls and solves load modules and kernels
    server = B.Server(B.Options(iters=(10, 10, 10, 0), max_points=384 * 384, max_hyps=64 * 144), budget, max_slots=64)
    SV.StreamClient(server, g, dsm_dev, sc, net, cam).run(
        [SV.StreamState(inputs[s][0], inputs[s][1], arrivals[s], inputs[s][0][0].copy()) for s in range(2)], 0.5)
    server.close()
    for iters, ns in [((10, 10, 10, 0), c) for c in counts] + [((4, 3, 2, 0), n_max)]:
        server = B.Server(B.Options(iters=iters, max_points=384 * 384, max_hyps=64 * 144), budget, max_slots=64)
        server.set_reserved_sms(reserved_sms)
        client = SV.StreamClient(server, g, dsm_dev, sc, net, cam)
        streams = [SV.StreamState(inputs[s][0], inputs[s][1], arrivals[s], inputs[s][0][0].copy()) for s in range(ns)]
        st = client.run(streams, duration)
        st["iters"] = list(iters[:3])
        ss = server.stats()
        st.update({k: v for k, v in ss.items() if k in ("rounds", "peak_active", "arena_bytes_peak")})
        # fraction of the run the server's rounds occupied the device / its worker
        st["round_device_busy"] = ss["round_device_ms"] / (1e3 * st["span_s"])
        st["round_wall_busy"] = ss["round_wall_ms"] / (1e3 * st["span_s"])
        # the server's own rate while its rounds run (the rest of the device time goes to the
        # clients' crops, network stand-in, quantisation and seeding)
        st["hyp_iter_per_round_s"] = st["hyp_iter_per_s"] / max(st["round_device_busy"], 1e-9)
        server.close()
        out["sweep"].append(st)
        if ns == n_max and iters[0] == 10:
            out["config5"] = st
    return out


def paper_schedule_form(args, B, S, torch, world, stream):
    """The paper's own refinement schedule (Sec. V-A, Supp. "Multi-Hypothesis Refinement"):
    500 sampled anchors, 1210 grid hypotheses, best 128 kept after the coarse level, 2 / 3 / 4
    iterations coarse to fine (3316 hyp*iter per frame), 384x512 / 192x256 / 96x128 levels,
    C = 32.  Plain FP32 solves one frame at a time; the batched form solves 8 frames per
    graph replay (the FP64 oracle's time for such a frame is in cpu_baseline)."""
    frames = [S.make_frame(S.config_paper_schedule(), S.frame_seed(6, i)) for i in range(2)]
    po = dict(iters=(4, 3, 2, 0), keep_top_k=(0, 0, 128, 0), max_points=500)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def timed(fn, reps):
        fn()
        fn()
        ts, units = [], 0
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            units += u
        return ts, units

    out = {}
    solver = B.Solver(B.Options(max_hyps=1210, **po))
    fas = [B.FrameArgs(f, B.device_arrays(f), is_device=True) for f in frames]
    k = [0]

    def plain():
        k[0] ^= 1
        return solver.solve(fas[k[0]], stream).hyp_iters
    ts, units = timed(plain, 6)
    out["plain_f32"] = {"ms_per_frame": sum(ts) / len(ts), "value": world * units / (sum(ts) / 1e3), "unit": UNIT}
    solver.close()
    # one frame through the batched form (one persistent launch per level: all 1210 FP64
    # steps of an iteration run at once, one per warp)
    bs = B.Solver(B.Options(max_hyps=1210, max_frames=1, **po))

    def batched1():
        k[0] ^= 1
        return bs.solve_batch([fas[k[0]]], stream)[0].hyp_iters
    ts, units = timed(batched1, 6)
    out["batched1_f32"] = {"ms_per_frame": sum(ts) / len(ts), "value": world * units / (sum(ts) / 1e3), "unit": UNIT}
    bs.close()
    for dt in (B.F32, B.BF16):
        bs = B.Solver(B.Options(max_hyps=1210 * 8, max_frames=8, **po))
        qa = [B.FrameArgs(f, B.quantized_device_arrays(f, dt), is_device=True, dtype=dt) for f in frames] * 4
        ts, units = timed(lambda: sum(r.hyp_iters for r in bs.solve_batch(qa, stream)), 3)
        out[f"batched8_{B.DTYPE_NAMES[dt]}"] = {"ms_per_frame": sum(ts) / len(ts) / 8,
                                                "value": world * units / (sum(ts) / 1e3), "unit": UNIT}
        bs.close()
    out["hyp_iter_per_frame"] = 1210 * 2 + 128 * 3 + 128 * 4
    out["workload"] = ("500 sampled anchors, 1210 grid hypotheses (11 x 11 x 10), top 128 after the coarse "
                       "level, 2/3/4 LM iterations, levels 384x512/192x256/96x128, C=32, priors on")
    out["paper_context"] = "optimiser 43.82 ms per frame on an RTX 5090 for this schedule (Supp. runtime table)"
    return out


def seeding_form(B, S, n_frames: int = 24):
    """Synthetic analogue of the seeding ablation (Supp. "Effect of Multi-hypothesis
    Sampling"): the paper's schedule on frames whose prior is 5-15 m / 5-15 deg off in
    (x, y, yaw), solved from four hypothesis sets around the prior (none: the prior alone;
    yaw: 10 yaw offsets; xy: the 11 x 11 grid; joint: all 1210).  Pose errors of the
    selected hypothesis against the ground truth: medians and Recall@1/3/5/10 (m and deg).
    An accuracy experiment on the CUDA path (batched FP32 solves), not a timed form."""
    import concurrent.futures as cf
    cfg = S.config_seeding_ablation()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        frames = list(ex.map(lambda i: S.make_frame(cfg, S.frame_seed(7, i)), range(n_frames)))
    po = dict(iters=(4, 3, 2, 0), keep_top_k=(0, 0, 128, 0), max_points=500)
    solver = B.Solver(B.Options(max_hyps=1210 * 8, max_frames=8, **po))
    out = {}
    for st in S.SEEDING_STRATEGIES:
        errs = []
        for b0 in range(0, n_frames, 8):
            group = frames[b0:b0 + 8]
            fas = []
            for f in group:
                hyps = S.seeding_hypotheses(f.meta["T_prior"], st, cfg)
                fas.append(B.FrameArgs(f, B.device_arrays(f, T_hyps=hyps), is_device=True))
            for f, r in zip(group, solver.solve_batch(fas)):
                T = r.T_cw[r.best]
                errs.append((S.translation_error_m(T, f.T_gt), S.rotation_error_deg(T, f.T_gt)))
        e = np.array(errs)
        out[st] = {"hypotheses": int(len(S.seeding_hypotheses(frames[0].meta["T_prior"], st, cfg))),
                   "median_t_m": float(np.median(e[:, 0])), "median_R_deg": float(np.median(e[:, 1])),
                   "recall_1_3_5_10": [float(100.0 * np.mean((e[:, 0] < th) & (e[:, 1] < th)))
                                       for th in (1.0, 3.0, 5.0, 10.0)]}
    solver.close()
    out["frames"] = n_frames
    out["workload"] = ("paper schedule (500 anchors, top 128 after coarse, 2/3/4 iterations), prior offset "
                       "5-15 m horizontal and 5-15 deg yaw, seeded frames 7000000..")
    return out


def crop_form(B, S, torch, stream, g=None):
    """The TDOM/DSM reference crop (Supp. "TDOM/DSM Reference Crop") on the serving workload's
    map (4096 x 4096 cells at 0.5 m): device time per crop (corner-ray footprint with 8000
    samples of 0.25 m per ray, homography, warp and geo-anchor lift) for 256^2 and 384^2 crops,
    over 16 seeded pose priors."""
    g = S.make_global_map(side=4096, seed=31) if g is None else g
    dm = B.MapArgs(torch.as_tensor(g.dsm, device="cuda"), torch.as_tensor(g.tdom, device="cuda"), g.x0, g.y0, g.gsd)
    priors = [S.crop_prior(g, k) for k in range(16)]
    out = {"map": "4096 x 4096 cells at 0.5 m (TDOM RGB + DSM)", "ray_samples": 8000, "ray_step_m": 0.25,
           "paper_context": "TDOM/DSM crop 13.17 ms per frame on the CPU (Supp. runtime table)"}
    for S_ in (256, 384):
        ps = [B.crop_params(pr["T_cw"], pr["fx"], pr["fy"], pr["cx"], pr["cy"], pr["img_w"], pr["img_h"],
                            0.0, 0.25, 8000, S_) for pr in priors]
        bufs = B.crop_reference(dm, ps[0], stream=stream)
        for p in ps:
            B.crop_reference(dm, p, out=bufs, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(4):
            for p in ps:
                B.crop_reference(dm, p, out=bufs, stream=stream)
        e1.record(stream)
        e1.synchronize()
        out[f"ms_per_crop_{S_}"] = e0.elapsed_time(e1) / (4 * len(ps))
    return out, g, priors


def tracking_form(B, S, gmap, n_frames: int = 60):
    """Sequential localisation (Supp. "Runtime Analysis"; Sec. V-A's Failure Recovery
    Count) of a seeded 60-frame flight over the 4096^2 map: constant-velocity priors, a
    256^2 reference crop per frame, the paper's 1210-seed grid and schedule, prior gates
    (gravity 0.1, range 3 m); 5 % of frames visually failed (random reference
    descriptors).  Serial and with the map preparation one frame ahead.  Accuracy and
    recoveries use the paper's 20 m / 20 deg rule; times are per frame: device time of the
    crop (map-preparation stream) and of seeding + solve (localisation stream), and the
    host wall time of a frame with the synthetic network (the feature extractor's stand-in,
    on the host) included."""
    from paper_2606_31098_gb300 import tracking as TK
    tc = S.TrackConfig(n_frames=n_frames)
    gt = S.make_trajectory(gmap, tc, seed=51)
    bank = S.query_bank(tc, seed=52)
    H0, W0 = tc.levels[0]
    cam = TK.Camera(tc.f0, tc.f0, W0 / 2.0, H0 / 2.0, W0, H0)
    grid_xy = tuple(float(v) for v in range(-10, 11, 2))
    grid_yaw = (-9.0, -7.0, -5.0, -3.0, -1.0, 1.0, 3.0, 5.0, 7.0, 9.0)
    opts = B.Options(iters=(4, 3, 2, 0), keep_top_k=(0, 0, 128, 0), max_hyps=1210, max_points=500,
                     gate_grav=0.1, gate_range=3.0)
    out = {"frames": n_frames, "rate_hz": tc.rate_hz,
           "workload": "60-frame synthetic flight, 256^2 crops on a 4096^2 map, 1210 seeds, 500 anchors, "
                       "2/3/4 iterations, 5 % visually failed frames"}
    for mode in ("serial", "lookahead"):
        tr = TK.SequentialTracker(gmap.dsm, None, gmap.x0, gmap.y0, gmap.gsd, cam,
                                  TK.CropSettings(tc.crop_side, 0.0, tc.ray_step, tc.ray_samples), opts,
                                  grid_xy, grid_yaw, mode=mode)
        net = S.SyntheticNetwork(gmap, tc, bank, gt, 53)
        res = TK.run_sequence(tr, gt, net)
        tr.close()
        e = res["err"]
        ok = ~res["failed"]
        tm = res["timings"][1:]                       # frame 0 includes first-use set-up
        out[mode] = {"frc": res["frc"], "median_t_m": float(np.median(e[:, 0])),
                     "median_R_deg": float(np.median(e[:, 1])),
                     "recall_1_3_5_10": [float(100.0 * np.mean((e[:, 0] < th) & (e[:, 1] < th)))
                                         for th in (1.0, 3.0, 5.0, 10.0)],
                     "median_t_m_tracked": float(np.median(e[ok, 0])) if ok.any() else None,
                     "crop_ms": float(np.mean([x.crop_ms for x in tm])),
                     "seed_solve_ms": float(np.mean([x.solve_ms for x in tm])),
                     "wall_ms": float(np.mean([x.wall_ms for x in tm])),
                     "crops_prepared_ahead": int(sum(x.prepared_ahead for x in tm))}
    return out


def run_oracle_sample(frame, n_hyps: int, threads: int):
    """Solve `n_hyps` hypotheses of the frame with the FP64 oracle; returns
    (hyp_iters, seconds)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    r = O.solve(frame, O.SolverOptions(iters=(10, 10, 10, 0)), T_hyps=frame.T_hyps[:n_hyps], n_threads=threads)
    return r.hyp_iters, time.perf_counter() - t0


def oracle_hyps_for(threads: int) -> int:
    # one hypothesis per thread (~1.7 s of CPU per hypothesis on one Grace core): one sample
    # is about 10-30 s of CPU work and under 3 s of wall time on 16 cores
    return max(2, threads)


# --------------------------------------------------------------------- reference arm

def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2606_31098_gb300 import scenes as S
    from oracle import build_oracle
    build_oracle.build()
    frame = S.make_frame(S.config_full_frame(), S.frame_seed(2, args.seed_index))
    threads = cpu_cores()
    nh = oracle_hyps_for(threads)
    for _ in range(args.warmup):
        run_oracle_sample(frame, nh, threads)
    total_units, total_s = 0, 0.0
    for _ in range(args.steps):
        u, s = run_oracle_sample(frame, nh, threads)
        total_units += u
        total_s += s
    value = total_units / total_s
    sample = f"{nh} of the 64 hypotheses of the full frame per step (all 3 levels x 10 iterations)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded scene generator)",
            "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (plain C, OpenMP over hypotheses)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)

    from paper_2606_31098_gb300 import binding as B
    from paper_2606_31098_gb300 import build_ext
    from paper_2606_31098_gb300 import scenes as S

    build_ext.build()
    B.load()
    if args.paper_schedule_only:
        return paper_schedule_only(B, S, torch)
    if args.crop_only:
        out, _, _ = crop_form(B, S, torch, torch.cuda.current_stream())
        print(json.dumps({"form": "crop", **out}), flush=True)
        return 0
    if args.served_only:
        out = served_streams(B, S, torch, S.make_global_map(side=4096, seed=31))
        print(json.dumps({"form": "served", **out}), flush=True)
        return 0
    if args.batched_only:
        out, _ = batched_and_served(args, B, S, torch, world, torch.cuda.current_stream(), served_too=False)
        print(json.dumps({"form": "batched", **out}), flush=True)
        return 0
    frame = S.make_frame(S.config_full_frame(), S.frame_seed(2, rank_seed_index(args.seed_index, rank)))
    opts = B.Options(iters=(10, 10, 10, 0), max_points=frame.N, max_hyps=frame.M, max_channels=32, profile=1)
    solver = B.Solver(opts)
    stream = torch.cuda.current_stream()
    dev = B.FrameArgs(frame, B.device_arrays(frame), is_device=True)
    host = B.FrameArgs(frame, B.host_arrays(frame, pinned=True), is_device=False)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(fa, steps):
        times, build_ms, build_n, launches, units = [], 0.0, 0, 0, 0
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = solver.solve(fa, stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            ms, nb, nt = solver.profile()
            build_ms += ms
            build_n += nb
            launches += nt
            units += r.hyp_iters
        return times, build_ms, build_n, launches, units, r

    if args.pin_schedule:
        tile, streams = (int(v) for v in args.pin_schedule.split(":"))
        solver.set_schedule([dev], batched=False, tile=tile, streams=streams)
        plain_schedule = solver.schedule([dev], batched=False)
    else:
        plain_schedule, _ = solver.autotune([dev], batched=False, reps=3, stream=stream)
    for _ in range(args.warmup):
        solver.solve(dev, stream)
        solver.solve(host, stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    times, build_ms, build_n, launches, units, res = timed(dev, args.steps)
    torch.cuda.synchronize()
    barrier()
    e2e_times, _, _, _, e2e_units, _ = timed(host, args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()

    # the same plain form on reduced-precision storage (GPU-quantised maps, FP32 math)
    precision = {}
    for dt in (B.BF16, B.F16, B.FP8E4M3):
        qa = B.FrameArgs(frame, B.quantized_device_arrays(frame, dt), is_device=True, dtype=dt)
        solver.set_schedule([qa], batched=False, tile=plain_schedule["tile"], streams=plain_schedule["streams"])
        for _ in range(2):
            solver.solve(qa, stream)
        qt, qb, qn, _, qu, _ = timed(qa, max(3, args.steps // 3))
        precision[B.DTYPE_NAMES[dt]] = {"value": world * qu / (sum(qt) / 1e3), "unit": UNIT,
                                        "ms_per_step": sum(qt) / len(qt), "build_avg_launch_ms": qb / max(qn, 1)}

    # the same plain form with a query confidence map per level weighting the photo term
    confidence = {}
    cframe = S.with_query_confidence(frame, rank_seed_index(args.seed_index, rank) + 17)
    for dt in (B.F32, B.BF16):
        ca = B.FrameArgs(cframe, B.quantized_device_arrays(cframe, dt), is_device=True, dtype=dt)
        solver.set_schedule([ca], batched=False, tile=plain_schedule["tile"], streams=plain_schedule["streams"])
        for _ in range(2):
            solver.solve(ca, stream)
        ct, _, _, _, cu, _ = timed(ca, max(3, args.steps // 3))
        confidence[B.DTYPE_NAMES[dt]] = {"value": world * cu / (sum(ct) / 1e3), "unit": UNIT,
                                         "ms_per_step": sum(ct) / len(ct)}
    solver.set_schedule([dev], batched=False, tile=plain_schedule["tile"], streams=plain_schedule["streams"])

    total_ms, e2e_ms = max_over_ranks([sum(times), sum(e2e_times)], world, "cuda")
    value = replica_throughput(units, total_ms, world)
    e2e_value = replica_throughput(e2e_units, e2e_ms, world)

    # roofline of the dominant kernel (the build pass).  The hypotheses run in `parts`
    # concurrent launches per LM iteration (one per stream), so launch durations overlap:
    # the rate is the build pass' units over the timed solves divided by their whole device
    # time (which also holds the ~1 % of small kernels: a lower bound).
    C, elem = frame.C, 4
    parts = min(plain_schedule["streams"] or 2, frame.M)
    units_per_launch = frame.N * (frame.M // parts)   # no pruning: equal parts every launch
    build_units = units_per_launch * build_n           # over the timed device-frame solves
    avg_launch_ms = build_ms / max(build_n, 1)
    units_per_s = build_units / (total_ms * 1e-3)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max = (clk or {}).get("sm_max_mhz") or (load_peaks() or {}).get("sm_max_mhz", 2070.0)
    # FP32 side: the scope table's algorithmic flops per unit against the FP32 FMA peak from
    # the SM count and clock (152 x 128 lanes x 2 flops x 2070 MHz = 80.5 TFLOP/s on GB300)
    achieved_tflops = units_per_s * flops_per_unit(C) / 1e12
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    frac_fp32 = achieved_tflops / peak_tflops
    # gather side: the tap bytes against the same loads' ceiling on this frame (the probe
    # runs the build pass' loads with the frame's own locality and no arithmetic)
    ceiling_units = frame_gather_ceiling(B, torch, frame, dev, C, elem, B.F32, plain_schedule["tile"], stream)
    tap_bytes = gather_bytes_per_unit(C, elem)
    achieved_gbps = units_per_s * tap_bytes / 1e9
    ceiling_gbps = ceiling_units * tap_bytes / 1e9
    frac_gather = units_per_s / ceiling_units
    traffic = traffic_per_launch(units_per_launch)
    # other measured ceilings on this GPU: FP32 FMA throughput, and 4-tap gathers at uniformly
    # random pixels of the finest map (no reuse between samples)
    probe_fma = B.probe_fma(stream)
    probe_gather = B.probe_gather(dev.arrays["qry_feat"][0], B.F32, 1 << 24, stream)
    if frac_fp32 >= frac_gather:
        bound, achieved, peak, unit = "alu", achieved_tflops, peak_tflops, "TFLOP/s"
    else:
        bound, achieved, peak, unit = "gather", achieved_gbps, ceiling_gbps, "GB/s"
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": traffic,
                "frac_fp32": frac_fp32, "frac_gather": frac_gather,
                "achieved_tflops": achieved_tflops, "peak_tflops": peak_tflops,
                "achieved_gather_GBps": achieved_gbps, "gather_ceiling_GBps": ceiling_gbps,
                "units_per_s": units_per_s, "gather_ceiling_units_per_s": ceiling_units,
                "kernel": "build pass with fused FP64 step (pilot::build_fused_kernel<f32, 32>)",
                "peak_basis": f"FP32 FMA derived: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz; "
                              "gather: pilot_probe_gather_frame on this frame (same grid, loads and locality)",
                "flops_per_unit": flops_per_unit(C), "flops_per_unit_executed": executed_flops_per_unit(C),
                "gather_bytes_per_unit": tap_bytes, "units_per_launch": units_per_launch,
                "avg_launch_ms": avg_launch_ms, "launches": build_n, "concurrent_launches": parts,
                "achieved_basis": "build-pass units of the timed solves / their device time",
                "traffic_basis": "ncu dram bytes per unit of a finest-level launch (cold cache) x units per "
                                 "launch (None: not measured for this kernel source)",
                "hbm_GBps_measured": (load_peaks() or {}).get("hbm_gbs"),
                "fma_probe_TFLOPs": probe_fma, "gather_random_pixels_GBps": probe_gather}

    gmap = S.make_global_map(side=4096, seed=31) if not args.no_forms else None
    batched, served = batched_and_served(args, B, S, torch, world, stream, gmap=gmap) if not args.no_forms else ({}, {})
    paper = paper_schedule_form(args, B, S, torch, world, stream) if not args.no_forms else {}
    crop, crop_map, crop_priors = crop_form(B, S, torch, stream, gmap) if not args.no_forms else ({}, None, None)
    seeding = seeding_form(B, S) if not args.no_forms else {}
    tracking = tracking_form(B, S, crop_map) if not args.no_forms else {}

    h2d = sum(a.nbytes for k, v in B.host_arrays(frame).items() for a in (v if isinstance(v, list) else [v]))
    d2h = frame.M * (12 * 8 + 8 + 4 + 4) + 16

    cpu = None
    if rank == 0:
        threads = cpu_cores()
        nh = oracle_hyps_for(threads)
        u, s = run_oracle_sample(frame, nh, threads)
        cpu = {"value": u / s, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{nh} of the 64 hypotheses of the same frame, all 3 levels x 10 iterations "
                         f"({u} hyp*iter in {s:.1f} s)"}
        # the same on one core (one hypothesis), per anchor as well, and the small plain
        # single-frame workload (4096 anchors, 1 hypothesis, one 120x160 level, 20 iterations)
        u1, s1 = run_oracle_sample(frame, 1, 1)
        cpu["value_1core"] = u1 / s1
        cpu["point_hyp_iter_per_s"] = frame.N * u / s
        cpu["point_hyp_iter_per_s_1core"] = frame.N * u1 / s1
        from oracle import oracle as O
        sf = S.make_frame(S.config_small_plain(), S.frame_seed(1, 0))
        t0 = time.perf_counter()
        rs = O.solve(sf, O.SolverOptions(iters=(20, 0, 0, 0)), n_threads=1)
        el = time.perf_counter() - t0
        cpu["small_plain_1core"] = {"hyp_iter_per_s": rs.hyp_iters / el, "point_hyp_iter_per_s": sf.N * rs.hyp_iters / el}
        try:
            cpu["cpu_model"] = next(l.split(":", 1)[1].strip() for l in open("/proc/cpuinfo")
                                    if l.lower().startswith(("model name", "cpu part")))
        except (OSError, StopIteration):
            cpu["cpu_model"] = None
        if paper:
            from oracle import oracle as O
            pf = S.make_frame(S.config_paper_schedule(), S.frame_seed(6, 0))
            t0 = time.perf_counter()
            O.solve(pf, O.SolverOptions(iters=(4, 3, 2, 0), keep_top_k=(0, 0, 128, 0)), n_threads=threads)
            cpu["paper_schedule_ms_per_frame"] = 1e3 * (time.perf_counter() - t0)
        if crop:
            from oracle import crop as OC
            om = OC.MapArgs(crop_map.dsm, crop_map.tdom, crop_map.x0, crop_map.y0, crop_map.gsd)
            pr = crop_priors[0]
            op = OC.params(pr["T_cw"], pr["fx"], pr["fy"], pr["cx"], pr["cy"], pr["img_w"], pr["img_h"],
                           0.0, 0.25, 8000, 256)
            t0 = time.perf_counter()
            OC.crop(om, op)
            cpu["crop_256_ms"] = 1e3 * (time.perf_counter() - t0)

    # kept short and printed last: the headline comparison of the forms, rates rounded
    headline = None
    if batched:
        c256, u32 = batched["crop256"], batched["uneven32_bf16"]
        r = lambda x: int(round(x))
        headline = {"what": "hyp*iter/s, batched BF16 form vs plain FP32 (the metric's form) and plain BF16, same frames",
                    "equal_accuracy": "f32, bf16, f16 (selected pose within 1e-3 deg / 1 mm of the FP64 oracle on 256 of "
                                      "256 seeds); not fp8e4m3",
                    "crop256_x8": {"plain_f32": r(c256["plain_f32"]), "plain_bf16": r(c256["plain_bf16"]),
                                   "batched_bf16": r(c256["batched_bf16"]),
                                   "vs_plain_f32": round(c256["batched_bf16"] / c256["plain_f32"], 3),
                                   "vs_plain_bf16": round(c256["batched_bf16"] / c256["plain_bf16"], 3)},
                    "uneven_x32": {"plain_f32": r(u32["plain_f32_same_frames"]),
                                   "plain_bf16": r(u32["plain_bf16_same_frames"]), "batched_bf16": r(u32["value"]),
                                   "vs_plain_f32": round(u32["value"] / u32["plain_f32_same_frames"], 3),
                                   "vs_plain_bf16": round(u32["value"] / u32["plain_bf16_same_frames"], 3)}}
        if served.get("config5"):
            c5 = served["config5"]
            headline["served_64_streams"] = {"hyp_iter_per_s": r(c5["hyp_iter_per_s"]),
                                             "completed_fps": round(c5["completed_fps"], 1),
                                             "offered_fps": round(c5["offered_fps"], 1),
                                             "p50_ms": round(c5["p50_ms"], 1), "p99_ms": round(c5["p99_ms"], 1)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scene generator)",
                "config": {"workload": WORKLOAD, "points": frame.N, "hypotheses": frame.M, "channels": C,
                           "levels": [list(q.shape[:2]) for q in frame.qry_feat], "iters_per_level": [10, 10, 10],
                           "feature_dtype": "f32",
                           "form": f"plain single frame, hypotheses in {parts} concurrent launches per iteration",
                           "schedule": plain_schedule,
                           "l2": "flushed between steps (512 MiB write)", "replicas": world},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms / args.steps},
                "gpu_launches": int(launches),
                "roofline": roofline,
                "precision_forms": precision, "confidence_form": confidence,
                "batched_form": batched,
                "served_form": served, "paper_schedule_form": paper, "crop_form": crop,
                "seeding_ablation": seeding, "tracking_form": tracking,
                "clocks": clk,
                "cpu_baseline": cpu,
                "headline": headline}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
