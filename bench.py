"""Benchmark: frames/s of the per-frame decomposition solve on a 640x480, K=6 video.

One step = one pass of the whole hot path over one synthetic 30-frame video:
every frame is ingested (chromaticity, soft-Retinex weight, pair weights), the
first is cold-started and the others warm-started from the previous frame, and
each frame runs 8 outer iterations of (Gauss-Newton step with 20 PCG steps,
then the base-colour step), temporal pairs on.  Inputs are resident in HBM;
L2 is flushed (256 MB write) before every step, outside the timed events.

Prints one JSON line (rank 0).  Under torchrun every rank solves its own video
(weak scaling, no data-path collective); the time is the max over ranks.
`--impl reference` times the FP64 CPU oracle instead, on a bounded sample.
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

from paper_1908_01961_b300 import synth  # noqa: E402

WORK = synth.VIDEO_640x480
METRIC = "frames/s at 640x480 K=6 (plain cold/warm solve, 8 GN x 20 PCG per frame)"
WORKLOAD = ("video_640x480_K6: 30 synthetic frames, 40 moving Voronoi cells, rotating light; "
            "frame 0 cold start, frames 1-29 warm start; 8 outer x (GN step of 20 PCG + base-colour step); "
            "temporal + 4 spatial consistency pairs")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gid", choices=["gid", "reference"])
    ap.add_argument("--frames", type=int, default=WORK["frames"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start comparison")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the editing, clustering, correction and preconditioner measurements (profiling runs)")
    ap.add_argument("--tile", type=int, default=None, choices=[-1, 0, 2, 4, 8, 16, 17, 258, 260, 264, 273],
                    help="PCG loop instead of autotuning: operator tile rows, 0 = persistent kernel, "
                         "-1 = resident kernel, rows + 256 = fused step; for profiling")
    ap.add_argument("--parity", action="store_true",
                    help="stream workload: after the timed run, per-layer error of 10 sampled frames against the "
                         "oracle (each solved from the GPU's state at the previous frame; minutes of host time)")
    ap.add_argument("--tile-cache", default=None,
                    help="batch workload: file of autotuned tile shapes to read and extend (default: none)")
    ap.add_argument("--l2-window", action="store_true",
                    help="video and stream workloads: the PCG launches mark the operator coefficients persisting "
                         "in L2 (gid_set_l2_window)")
    ap.add_argument("--batch-form", default="worklist", choices=["worklist", "persistent", "branch"],
                    help="batch workload: PCG steps as work-list launches over all videos of one K (default), the "
                         "work list as one cooperative launch per K and Gauss-Newton step, or one graph branch per "
                         "video with autotuned tile shapes")
    ap.add_argument("--workload", default="video", choices=["video", "batch", "stream"],
                    help="video: the 640x480 K=6 video (default); batch: 24 uneven videos in one graph per step")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_video(seed, frames):
    v = synth.SyntheticVideo(WORK["H"], WORK["W"], WORK["K"], WORK["n_cells"], seed=seed)
    fr = [v.frame(t) for t in range(frames)]
    b0 = synth.initial_base_colors(fr[0].I, fr[0].labels, WORK["K"]).astype(np.float32)
    return fr, b0


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash():
    """Hash of the sources that define and launch the solver kernels (the ones
    whose DRAM traffic profiles/traffic.json records)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1908_01961_b300", "csrc")
    for f in ("gid_kernels.cuh", "gid.cu"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        if t.get("source_hash") != source_hash():
            return None
        return t["kernels"][kernel]["dram_bytes_per_launch_full_size"]
    except Exception:
        return None


def algorithmic_bytes(kind, K, P, M, ns, nt, temporal, fused=False):
    """Minimum bytes each kernel kind moves per launch as designed (FP32 planes)."""
    V = K + 4
    NC = 10 + 3 * (K + 1) + 2 * ns  # operator coefficient planes written by k_linearize (pair weights included)
    t = 1 if temporal else 0
    if kind == "apply" and fused:  # k_pcg_step: read z, M^-1, coefficients (+ mq_old, p_old, delta after
        first = 5 * V + NC         # step 1); write z, mq, p (+ delta)
        rest = 9 * V + NC
        return 4.0 * P * ((M - 1) * rest + first) / M
    if kind == "update" and fused:  # the last step's update only: read delta, p, X; write X
        return 4.0 * P * 4 * V
    if kind == "apply":     # read z, coefficients (+ p_old, q_old after step 1); write p, q
        first = 3 * V + NC
        rest = 5 * V + NC
        return 4.0 * P * ((M - 1) * rest + first) / M
    if kind == "pcg":       # the persistent loop: M operator phases and M vector phases
        return M * (algorithmic_bytes("apply", K, P, M, ns, nt, temporal) +
                    algorithmic_bytes("update", K, P, M, ns, nt, temporal))
    if kind == "update":    # read delta, p, q, z, M^-1; write delta, z (last: read delta, p, X; write X)
        return 4.0 * P * ((M - 1) * 7 * V + 4 * V) / M
    if kind == "linearize":  # read X, I, w_SR, pairs (+ r_prev, temporal sum); write M^-1, z, delta, coefficients
        return 4.0 * P * (4 * V + 4 + ns + (nt + 3 + 1) * t + NC) + P
    if kind == "dense":     # read X and I
        return 4.0 * P * (V + 3)
    return None


# ---------------------------------------------------------------- reference arm (the oracle)

def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_frame(threads, seed=0):
    """The FP64 oracle's whole solve of frame 0 of the video (cold start, 8 outer
    iterations of a Gauss-Newton step of 20 PCG steps and the base-colour step),
    precompute included, on `threads` host threads (the oracle's loops are
    spread by OpenMP; its results do not depend on the thread count).
    Returns (seconds, X, b, energy history)."""
    import oracle as O
    O.set_threads(threads)
    fr, b0 = make_video(seed, 1)
    off_s, _ = synth.offsets_for(seed)
    I = fr[0].I.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    C, wsr, om, _ = O.precompute(I, off_s)
    pb = O.Problem(I, fr[0].labels, b0.astype(np.float64), wsr, om, off_s)
    X, bo, hist = O.solve_frame(pb, pb.init_cold(), WORK["N"], WORK["M"])
    return time.perf_counter() - t0, X, bo, hist


CPU_SAMPLE = ("one whole 640x480 K=6 frame (frame 0 of the video: precompute, cold start, 8 x (GN step of 20 PCG "
              "+ base-colour step)), FP64 oracle")


def cpu_baseline():
    """The oracle on the host: one whole frame on every host thread (the
    reported value) and on one thread; returns (record, X, b, history) of the
    all-thread run, whose result the parity block reuses."""
    import oracle
    oracle.build()
    n = host_threads()
    dt_n, X, bo, hist = oracle_frame(n)
    dt_1, _, _, _ = oracle_frame(1)
    rec = {"value": 1.0 / dt_n, "unit": "frames/s", "cores": n, "kind": "oracle", "sample": CPU_SAMPLE,
           "seconds_per_frame": dt_n, "cores_1": {"cores": 1, "value": 1.0 / dt_1, "seconds_per_frame": dt_1},
           "cores_nproc": {"cores": n, "value": 1.0 / dt_n, "seconds_per_frame": dt_n}, "cpu_model": cpu_model()}
    return rec, X, bo, hist


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    n = host_threads()
    for _ in range(args.warmup):
        oracle_frame(n)
    times = [oracle_frame(n)[0] for _ in range(args.steps)]
    tot = sum(times)
    value = args.steps / tot
    out = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "H": WORK["H"], "W": WORK["W"], "K": WORK["K"],
                      "step": "one whole frame (frame 0: cold start, 8 x 20), on every host thread"},
           "cpu_baseline": {"value": value, "unit": "frames/s", "cores": n, "kind": "oracle", "sample": CPU_SAMPLE,
                            "cpu_model": cpu_model()},
           "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def sub_bench(*argv):
    """Another workload of this file in a child process (its own CUDA context);
    the child's JSON line, reduced to the figures the main line reports."""
    try:
        p = subprocess.run([sys.executable, os.path.abspath(__file__), *argv], capture_output=True, text=True,
                           timeout=1200, env=dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0"))
        line = [l for l in p.stdout.strip().splitlines() if l.startswith("{")][-1]
        d = json.loads(line)
    except Exception as e:  # reported, never fatal for the main measurement
        return {"error": f"{type(e).__name__}: {e}"[:300]}
    keep = ("metric", "value", "unit", "ms_per_step", "pixels_per_s", "latency_ms", "frames_per_s", "gpu_launches",
            "clocks", "config")
    return {k: d[k] for k in keep if k in d}


def pcg_loop_name(s, rows):
    if rows == -1:
        _, (tw, th, nb) = s.pcg_layout()
        return f"resident PCG kernel ({nb} tiles of {tw}x{th}, one per SM)"
    if rows == 0:
        return "persistent PCG kernel"
    if rows > 0 and rows & 256:
        return f"128x{rows & 255} tiles, one fused kernel per PCG step (vector update folded into the operator)"
    return f"128x{rows} operator tiles, operator and vector kernels per PCG step"


def layer_errors(R, T, b, E, Xo, bo, Eo):
    """Per-layer error of the GPU solve against the oracle's (max-abs and RMS of
    R = exp(r) per channel set, T_0, each T_k, the base colours), the relative
    energy error, and the non-negativity branch flips: layer values whose sign
    (T > 0 or not, the branch of the non-negativity weight) differs."""
    Ro, To = np.exp(Xo[:3]), Xo[3:]

    def st(a, o):
        d = np.asarray(a, np.float64) - np.asarray(o, np.float64)
        return {"max_abs": float(np.abs(d).max()), "rms": float(np.sqrt(np.mean(d * d)))}

    out = {"R": st(R, Ro), "T_0": st(T[0], To[0])}
    for k in range(1, T.shape[0]):
        out[f"T_{k}"] = st(T[k], To[k])
    out["b"] = st(b, bo)
    out["energy_rel"] = float(abs(E - Eo) / abs(Eo))
    flip = (T > 0) != (To > 0)
    out["nonneg_branch_flips"] = int(np.count_nonzero(flip))
    # the largest layer error at pixels more than 2 pixels from any branch flip
    near = flip.any(axis=0)
    for _ in range(2):
        n = near.copy()
        n[1:] |= near[:-1]
        n[:-1] |= near[1:]
        n[:, 1:] |= near[:, :-1]
        n[:, :-1] |= near[:, 1:]
        near = n
    far = ~near
    d = np.concatenate([np.abs(R - Ro), np.abs(np.asarray(T, np.float64) - To)])
    out["max_abs_away_from_flips"] = float(d[:, far].max()) if far.any() else 0.0
    out["pixels_near_flips"] = int(near.sum())
    worst = max(v["max_abs"] for k, v in out.items() if isinstance(v, dict))
    out["meets_bar"] = bool(worst <= 1e-3 and out["energy_rel"] <= 1e-4)
    return out


# ---------------------------------------------------------------- CUDA arm

def run_gid(args, ws, rank, local):
    import torch

    from paper_1908_01961_b300 import gid

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, W, K, N, M, F = WORK["H"], WORK["W"], WORK["K"], WORK["N"], WORK["M"], args.frames
    P = H * W
    seed = rank
    frames, b0 = make_video(seed, F)
    off_s, off_t = synth.offsets_for(seed)
    rgb = [torch.from_numpy(f.I.astype(np.float32)).to(dev) for f in frames]
    lab = [torch.from_numpy(f.labels).to(dev) for f in frames]
    w = gid.default_weights(off_s, off_t, temporal=1)
    s = gid.Solver(H, W, K, w)
    s.set_base_colors(b0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > 126 MB L2

    def step():
        s.new_sequence()
        for t in range(F):
            s.set_frame(rgb[t], lab[t])
            s.init(0 if t == 0 else 1)
            s.run(N, M)

    step()
    if args.tile is None:
        tile_rows, tile_us = s.autotune(10)     # operator tile shape for this frame size (setup, untimed)
    else:
        s.set_apply_tile(args.tile)
        tile_rows, tile_us = args.tile, "fixed by --tile"
    if args.l2_window:
        s.set_l2_window(True)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    # timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    n0 = s.launch_count()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    launches = s.launch_count() - n0
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(ws, sum(ms))
    value = ws * args.steps * F / (total_ms / 1000.0)
    E, _ = s.energy()
    if not np.isfinite(E):
        raise RuntimeError("non-finite energy after the timed steps")

    # one profiled step (identical work): per-kernel CUDA-event durations on the ctx stream
    flush.fill_(0.0)
    s.profile(True)
    step()
    prof = s.profile_read()
    s.profile(False)
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms = kinds[dom][0] / kinds[dom][1]
    peak, peak_src = measured_peaks()
    fused = tile_rows > 0 and (tile_rows & 256) != 0
    kernel_name = {"apply": "k_pcg_step" if fused else "k_apply", "update": "k_update", "linearize": "k_linearize",
                   "dense": "k_dense", "pcg": "k_pcg_resident" if tile_rows == -1 else "k_pcg"}.get(dom)
    # The profiled step launches kernel by kernel with an event after each (no
    # graph replay, no programmatic overlap), so it runs slower than the timed
    # steps: a kind's time per step is its share of the profiled step times the
    # timed step's own duration.
    prof_total = sum(v[0] for v in kinds.values())
    step_ms = total_ms / args.steps
    scale = step_ms / prof_total
    # The roofline of the solver: one PCG step (operator + vector kernels, or its
    # share of the single-launch loop) against the algorithmic bytes of a textbook
    # PCG step, (8 V + 2 + S) x 4 B per pixel (read p twice, the state X for the
    # operator's coefficients, delta and r; write delta, r and p; w_SR and the S
    # pair weights)
    V = K + 4
    S_pairs = len(off_s) + len(off_t)
    pcg_bytes = 4.0 * (8 * V + 2 + S_pairs) * P
    pcg_ms = sum(kinds[k][0] for k in ("apply", "update", "pcg") if k in kinds) * scale
    n_pcg = F * N * M
    pcg_us = 1000.0 * pcg_ms / n_pcg
    ach = pcg_bytes / (pcg_us * 1e-6) / 1e9
    traffic = ncu_traffic("pcg_step")
    alg = algorithmic_bytes(dom, K, P, M, len(off_s), len(off_t), True, fused)
    design = None
    if alg and dom in ("apply", "update"):
        dom_scaled = dom_ms * scale
        design = {"kernel": kernel_name, "design_bytes_per_launch": alg, "avg_launch_ms": dom_scaled,
                  "achieved_GBps": alg / (dom_scaled / 1000.0) / 1e9, "frac": alg / (dom_scaled / 1000.0) / 1e9 / peak,
                  "note": "the kernel's own design bytes (stored coefficient planes) per launch"}
    roof = {"bound": "hbm", "kernel": "PCG step (" + ("k_pcg_resident" if "pcg" in kinds and tile_rows == -1 else
                                                      "k_pcg" if "pcg" in kinds else
                                                      "k_pcg_step, last step's k_update" if fused else
                                                      "k_apply + k_update") + ")",
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": traffic,
            "peak_source": peak_src, "algorithmic_bytes_per_step": pcg_bytes,
            "bytes_per_px": 4 * (8 * V + 2 + S_pairs), "pcg_step_us": pcg_us, "pcg_steps_per_video": n_pcg,
            "frac_survey_bytes": ach / peak, "dominant_kind": dom, "design_roofline": design,
            "method": "pcg_step_us = (time of the PCG kernels in a profiled step with a CUDA event after every "
                      "kernel) x (timed step / profiled step) / PCG steps; achieved = algorithmic bytes of one "
                      f"PCG step / pcg_step_us (profiled step {prof_total:.1f} ms vs timed step {step_ms:.1f} ms)"}
    shares = {k: {"ms_per_step": v[0], "launches": v[1]} for k, v in kinds.items()}

    # end to end: the host-buffer entry point, host<->device copies inside the timed region
    e2e = None
    if not args.no_e2e:
        # the whole video through the pipelined host-buffer entry point (page-locked buffers)
        rgb_h = torch.from_numpy(np.stack([f.I.astype(np.float32) for f in frames])).pin_memory().numpy()
        lab_h = torch.from_numpy(np.stack([f.labels for f in frames])).pin_memory().numpy()
        R_h = torch.empty((F, 3, H, W), dtype=torch.float32).pin_memory().numpy()
        T_h = torch.empty((F, K + 1, H, W), dtype=torch.float32).pin_memory().numpy()
        b_h = torch.empty((F, K, 3), dtype=torch.float32).pin_memory().numpy()

        def e2e_step():
            s.new_sequence()
            s.solve_video_host(rgb_h, lab_h, 0, N, M, R_h, T_h, b_h)

        e2e_step()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        dt = max_over_ranks(ws, time.perf_counter() - t0)
        e2e = {"value": ws * args.steps * F / dt, "unit": "frames/s",
               "h2d_bytes_per_step": F * (3 * P * 4 + P),
               "d2h_bytes_per_step": F * ((3 + K + 1) * P * 4 + K * 3 * 4)}

    # the measurements below run other contexts in this process and its children: the
    # headline context gives up its L2 set-aside so that they have the whole L2
    l2_window = s.l2_window()
    if l2_window:
        s.set_l2_window(False)

    # editing (Sec. 7.4): recombination of the last frame's layers with one recoloured
    # object, one re-keyed and one suppressed indirect layer
    editing = None
    if rank == 0 and not args.no_extras:
        bn = s.base_colors().copy()
        bn[0] = bn[0][::-1]
        gains = np.ones(K, np.float32)
        gains[1] = 0.0
        mask = (lab[F - 1] == 2).to(torch.uint8) * 3
        out = torch.empty((3, H, W), device=dev)
        for _ in range(3):
            s.recombine(bn, gains, mask, out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 50
        e0.record(stream)
        for _ in range(reps):
            s.recombine(bn, gains, mask, out)
        e1.record(stream)
        torch.cuda.synchronize()
        us = 1000.0 * e0.elapsed_time(e1) / reps
        eb = 4.0 * P * (K + 4) + P + 4.0 * 3 * P   # read X and the mask, write the image
        editing = {"kernel": "k_recombine", "us_per_frame": us, "algorithmic_bytes": eb,
                   "achieved_GBps": eb / (us * 1e-6) / 1e9, "note": "host call included (gains and colours "
                   "passed by value)"}

    # chromaticity clustering of frame 0 (Sec. 4.1), the step before the solve
    clustering = None
    if rank == 0 and not args.no_extras:
        for _ in range(3):
            gid.cluster(rgb[0])
        t0 = time.perf_counter()
        reps = 20
        for _ in range(reps):
            labs, bcl = gid.cluster(rgb[0])
        clustering = {"ms_per_frame": 1000.0 * (time.perf_counter() - t0) / reps, "clusters": int(bcl.shape[0]),
                      "note": "host wall time of gid_cluster (4 kernels, scratch allocation, synchronising)"}

    # misclustering correction (Sec. 4.2) of one region of frame 0: K candidate solves as one batch
    correction = None
    if rank == 0 and not args.no_extras:
        region = torch.zeros((H, W), dtype=torch.uint8, device=dev)
        region[H // 4:H // 2, W // 4:W // 2] = (lab[0][H // 4:H // 2, W // 4:W // 2] == int(lab[0][H // 3, W // 3]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best, sp, _ = gid.correct_region(rgb[0], lab[0], b0, region, gid.default_weights(off_s), N, M)
        correction = {"ms": 1000.0 * (time.perf_counter() - t0), "candidates": K, "region_pixels":
                      int(region.sum().item()), "winner": best, "note": "host wall time: K contexts created, "
                      "solved as one batch (8 GN x 20 PCG each), region energies, destroyed"}

    # preconditioners (Sec. 6.1 names none): Jacobi vs per-pixel block-Jacobi on frame 0,
    # cold start, 8 Gauss-Newton steps of M PCG steps; final energy against solve time
    preconditioners = None
    if rank == 0 and not args.no_extras:
        preconditioners = []
        sp = gid.Solver(H, W, K, gid.default_weights(off_s))
        sp.set_frame(rgb[0], lab[0])
        sp.set_apply_tile((tile_rows & 255) if tile_rows and tile_rows > 0 else 17)   # one operator kernel per PCG step in both arms
        for kind in ("jacobi", "block"):
            sp.set_preconditioner(kind)
            for Mi in (10, 15, 20):
                times = []
                for rep in range(4):
                    sp.set_base_colors(b0)
                    sp.init(0)
                    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    sp.run(N, Mi)
                    a1.record(stream)
                    torch.cuda.synchronize()
                    if rep > 0:
                        times.append(a0.elapsed_time(a1))
                Ei, _ = sp.energy()
                preconditioners.append({"preconditioner": kind, "N": N, "M": Mi, "ms": float(np.median(times)),
                                        "energy": Ei})
        # Jacobi with the single-reduction recurrence (one grid-wide reduction per PCG
        # step): the fused step at the same tile height
        sp.set_preconditioner("jacobi")
        rows_f = (tile_rows & 255) if tile_rows and tile_rows > 0 else 17
        sp.set_apply_tile((17 if rows_f == 16 else rows_f) | gid.FUSED)   # the fused step has no 16-row tile
        for Mi in (10, 15, 20):
            times = []
            for rep in range(4):
                sp.set_base_colors(b0)
                sp.init(0)
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                sp.run(N, Mi)
                a1.record(stream)
                torch.cuda.synchronize()
                if rep > 0:
                    times.append(a0.elapsed_time(a1))
            Ei, _ = sp.energy()
            preconditioners.append({"preconditioner": "jacobi, single-reduction recurrence (fused step)", "N": N,
                                    "M": Mi, "ms": float(np.median(times)), "energy": Ei})
        sp.close()

    # the same video with the block-Jacobi preconditioner at equal final energy: the
    # fewest PCG steps per Gauss-Newton step whose per-frame final energies are all
    # at or below the Jacobi 8 x 20 solve's (energies from untimed passes), then timed
    # like the headline (CUDA events, L2 flushed between steps)
    block_arm = None
    if rank == 0 and not args.no_extras:
        def video_energies(solver, Mi):
            solver.new_sequence()
            out = []
            for t in range(F):
                solver.set_frame(rgb[t], lab[t])
                solver.init(0 if t == 0 else 1)
                solver.run(N, Mi)
                out.append(solver.energy()[0])
            return np.array(out)

        sb = gid.Solver(H, W, K, w)
        sb.set_base_colors(b0)
        sb.set_apply_tile((tile_rows & 255) if tile_rows and tile_rows > 0 else 17)
        e_ref = video_energies(s, M)
        sb.set_preconditioner("block")
        ratios, Mb = {}, None
        for Mi in (6, 8, 10, 12, 14, 16, 20):
            sb.set_base_colors(b0)
            e_b = video_energies(sb, Mi)
            ratios[Mi] = {"video_total": float(e_b.sum() / e_ref.sum()), "worst_frame": float((e_b / e_ref).max()),
                          "best_frame": float((e_b / e_ref).min())}
            if ratios[Mi]["video_total"] <= 1.0:
                Mb = Mi
                break
        if Mb is not None:
            def step_b():
                sb.new_sequence()
                for t in range(F):
                    sb.set_frame(rgb[t], lab[t])
                    sb.init(0 if t == 0 else 1)
                    sb.run(N, Mb)

            for _ in range(3):
                flush.fill_(1.0)
                step_b()
            tb = []
            for i in range(max(args.steps, 3)):
                flush.fill_(float(i))
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                step_b()
                a1.record(stream)
                torch.cuda.synchronize()
                tb.append(a0.elapsed_time(a1))
            ms_b = float(np.mean(tb))
            block_arm = {"preconditioner": "block", "N": N, "M": Mb, "frames_per_s": F * 1000.0 / ms_b,
                         "ms_per_video": ms_b, "reference": f"jacobi {N} x {M}",
                         "criterion": "sum over the video's frames of the final energy <= the reference's",
                         "energy_ratio_by_M": ratios}
        else:
            block_arm = {"preconditioner": "block", "M": None, "energy_ratio_by_M": ratios,
                         "note": "no candidate reached the reference's summed final energy"}
        sb.close()

    learned = None
    if rank == 0 and not args.no_learned:
        learned = learned_arm(dev, flush)

    # the batch of 24 uneven videos and the 1080p stream, each in a process of its own
    batch_line, stream_line = None, None
    if rank == 0 and not args.no_extras:
        torch.cuda.synchronize()
        batch_line = sub_bench("--workload", "batch", "--steps", "1", "--warmup", "2")
        stream_line = sub_bench("--workload", "stream", "--warmup", "1")

    # the oracle on the host cores (one whole frame), and the per-layer error of the GPU's
    # solve of that frame (in the timed launch configuration) and of the 64 x 48 workload
    cpu, parity = None, None
    if rank == 0 and not args.no_cpu:
        cpu, Xo, bo, hist = cpu_baseline()
        s.new_sequence()
        s.set_frame(rgb[0], lab[0])
        s.init(0)
        s.run(N, M)
        R0, T0 = s.layers()
        E0, _ = s.energy()
        parity = {"bar": "every layer <= 1e-3 max-abs, energy <= 1e-4 relative, after the same N x M from the same "
                         "start",
                  "video_640x480_K6_frame0": dict(layer_errors(R0.cpu().numpy(), T0.cpu().numpy(), s.base_colors(),
                                                               E0, Xo, bo, hist[-1].sum()), N=N, M=M, start="cold"),
                  "single_64x48_K4": parity_64x48()}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD, "H": H, "W": W, "K": K, "frames_per_step": F, "N_outer": N,
                          "M_inner": M, "l2": "flushed before each step (256 MB write, outside the events)",
                          "parallelism": f"replicas x{ws} (one video per GPU)",
                          "operator_tile": pcg_loop_name(s, tile_rows) +
                          (f" (autotuned; us per PCG step {tile_us})" if args.tile is None else " (fixed)"),
                          "l2_window": l2_window},
               "gpu_launches": launches, "roofline": roof, "kernel_time_per_step": shares,
               "e2e": e2e, "cpu_baseline": cpu, "parity": parity, "clocks": clk, "final_energy": E,
               "learned_warm_start": learned, "editing": editing, "clustering": clustering,
               "misclustering_correction": correction, "preconditioners": preconditioners,
               "batch_24_videos": batch_line, "stream_1080p": stream_line,
               "block_jacobi_equal_energy": block_arm}
        print(json.dumps(out), flush=True)


def parity_64x48():
    """The 64 x 48 K = 4 workload (5 x 10, cold start, refinement on) on the GPU
    and in the oracle: per-layer errors."""
    import torch

    import oracle as O
    from paper_1908_01961_b300 import gid
    cfg = synth.SINGLE_64x48
    H, W, K = cfg["H"], cfg["W"], cfg["K"]
    f = synth.SyntheticVideo(H, W, K, cfg["n_cells"], seed=0).frame(0)
    b0 = synth.initial_base_colors(f.I, f.labels, K).astype(np.float32)
    off_s, _ = synth.offsets_for(0)
    s = gid.Solver(H, W, K, gid.default_weights(off_s))
    s.set_base_colors(b0)
    s.set_frame(torch.from_numpy(f.I.astype(np.float32)).cuda(), torch.from_numpy(f.labels).cuda())
    s.init(0)
    s.run(cfg["N"], cfg["M"])
    R, T = s.layers()
    E, _ = s.energy()
    I = f.I.astype(np.float32).astype(np.float64)
    C, wsr, om, _ = O.precompute(I, off_s)
    pb = O.Problem(I, f.labels, b0.astype(np.float64), wsr, om, off_s)
    Xo, bo, hist = O.solve_frame(pb, pb.init_cold(), cfg["N"], cfg["M"])
    out = layer_errors(R.cpu().numpy(), T.cpu().numpy(), s.base_colors(), E, Xo, bo, hist[-1].sum())
    s.close()
    return dict(out, N=cfg["N"], M=cfg["M"], start="cold")


# ---------------------------------------------------------------- learned warm start

LEARNED_FRAMES = 50
LEARNED_REPS = 5


def learned_arm(dev, flush):
    """Frames/s of a single 640x480 K=6 frame solved to the cold start's final
    energy: plain (cold start, 8 Gauss-Newton steps) against the learned start
    (network forward, T_0 refit, base-colour step, then as many Gauss-Newton
    steps as the held-out frames needed to reach that energy).  Step counts from
    energies after every step on LEARNED_FRAMES held-out frames; times from CUDA
    events over LEARNED_REPS solves of the first frame (L2 flushed between)."""
    import torch

    from paper_1908_01961_b300 import gid
    from paper_1908_01961_b300 import warmstart as WS
    if not os.path.exists(WS.DEFAULT_WEIGHTS):
        return {"unavailable": "no trained weights file"}
    net = WS.load_net()
    frames = WS.generate(range(WS.EVAL_SEED0, WS.EVAL_SEED0 + LEARNED_FRAMES), workers=1)
    ev = WS.evaluate(net, frames, zero_below=(WS.ZERO_BELOW,), learned_steps=2 * WS.N_OUTER)
    n_cold = [int(np.nonzero(np.array(e["E_cold"]) <= e["E_cold"][-1])[0][0]) for e in ev]
    n_learned = [e["learned"][str(WS.ZERO_BELOW)]["n"] for e in ev]
    nc, nl = max(n_cold), max(n_learned)
    I, lab, b = frames[0]
    rgb, lb = torch.from_numpy(I).to(dev), torch.from_numpy(lab).to(dev)
    s = gid.Solver(WS.H, WS.W, WS.K, WS.solver_weights())
    s.set_base_colors(b)
    stream = torch.cuda.current_stream()

    def timed(fn, reps=LEARNED_REPS):
        for _ in range(3):
            fn()
        out = []
        for i in range(reps):
            flush.fill_(float(i))
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            z.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(z))
        return statistics.median(out)

    def cold():
        s.new_sequence()
        s.set_frame(rgb, lb)
        s.init(0)
        s.run(nc, WS.M_INNER)

    def learned(n):
        s.new_sequence()
        s.set_frame(rgb, lb)
        s.init_learned(net, WS.ZERO_BELOW)
        if n:
            s.run(n, WS.M_INNER)

    ms_cold, ms_learned, ms_init = timed(cold), timed(lambda: learned(nl)), timed(lambda: learned(0))
    return {"eval_frames": LEARNED_FRAMES, "eval_seeds": f"{WS.EVAL_SEED0}..{WS.EVAL_SEED0 + LEARNED_FRAMES - 1}",
            "gn_steps_to_cold_final_energy": {"cold": n_cold, "learned": n_learned},
            "gn_steps_timed": {"cold": nc, "learned": nl}, "gn_step_ratio": nl / nc,
            "frames_per_s_cold": 1000.0 / ms_cold, "frames_per_s_learned": 1000.0 / ms_learned,
            "ms_cold": ms_cold, "ms_learned": ms_learned, "ms_learned_init": ms_init,
            "zero_below": WS.ZERO_BELOW, "weights": os.path.relpath(WS.DEFAULT_WEIGHTS, ROOT)}


# ---------------------------------------------------------------- batched workload

BATCH_SIZES = [(240, 320), (480, 640), (540, 960), (720, 1280)]
BATCH_FRAMES = 10


def batch_shapes():
    """24 videos: six of each size, K = 4, 6, 8 in turn."""
    return [(BATCH_SIZES[i % 4][0], BATCH_SIZES[i % 4][1], (4, 6, 8)[i % 3]) for i in range(24)]


def _batch_video(args):
    """Frames and initial colours of one batch video (runs in a worker process)."""
    H, W, K, seed = args
    v = synth.SyntheticVideo(H, W, K, max(12, W // 16), seed=seed)
    fr = [v.frame(t) for t in range(BATCH_FRAMES)]
    return ([f.I.astype(np.float32) for f in fr], [f.labels for f in fr],
            synth.initial_base_colors(fr[0].I, fr[0].labels, K).astype(np.float32))


def run_batch(args, ws, rank, local):
    import multiprocessing as mp
    shapes = batch_shapes()
    jobs = [(H, W, K, 1000 * rank + i) for i, (H, W, K) in enumerate(shapes)]
    with mp.get_context("spawn").Pool(min(len(jobs), max(1, os.cpu_count() or 1))) as pool:
        made = pool.map(_batch_video, jobs)   # before any CUDA call in this process

    import torch

    from paper_1908_01961_b300 import gid

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, M = WORK["N"], WORK["M"]
    vids, weights, rgb, lab = [], [], [], []
    for i, (H, W, K) in enumerate(shapes):
        seed = 1000 * rank + i
        frames_I, frames_lab, b0 = made[i]
        off_s, off_t = synth.offsets_for(seed)
        weights.append(gid.default_weights(off_s, off_t, temporal=1))
        vids.append(b0)
        rgb.append([torch.from_numpy(x).to(dev) for x in frames_I])
        lab.append([torch.from_numpy(x).to(dev) for x in frames_lab])
    batch = gid.Batch(shapes, weights)
    batch.set_worklist(args.batch_form != "branch", args.batch_form == "persistent")
    for v, b0 in zip(batch.videos, vids):
        v.set_base_colors(b0)

    def step():
        batch.new_sequence()
        for t in range(BATCH_FRAMES):
            batch.set_frames([r[t] for r in rgb], [l[t] for l in lab])
            batch.init(0 if t == 0 else 1)
            batch.run(N, M)

    step()
    if args.batch_form == "branch":
        batch.autotune(args.tile_cache, reps=5)   # the work-list form always uses 128 x 4 tiles
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    n0 = sum(v.launch_count() for v in batch.videos)
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    launches = sum(v.launch_count() for v in batch.videos) - n0
    clk = clocks.stop()
    total_ms = max_over_ranks(ws, sum(a.elapsed_time(b) for a, b in ev))
    frames = len(shapes) * BATCH_FRAMES
    px = sum(h * w for h, w, _ in shapes) * BATCH_FRAMES
    energies = [v.energy()[0] for v in batch.videos]
    if not all(np.isfinite(energies)):
        raise RuntimeError("non-finite energy in the batch")
    batch.close()
    seq_ms = time_sequential(shapes, weights, vids, rgb, lab, N, M, flush) if rank == 0 else None
    if rank == 0:
        out = {"metric": "frames/s over 24 uneven videos (6 each of 320x240, 640x480, 960x540, 1280x720; K 4/6/8), "
                         "8 GN x 20 PCG per frame", "value": ws * args.steps * frames / (total_ms / 1000.0),
               "unit": "frames/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"batch of 24 videos x {BATCH_FRAMES} frames, one CUDA graph launch per "
                                      "frame-step for all videos",
                          "pcg_launches": {"worklist": "one operator and one vector launch per K and PCG step "
                                                       "over all videos of that K (128 x 4 tiles)",
                                           "persistent": "one cooperative launch per K and Gauss-Newton step over "
                                                         "all videos of that K (128 x 4 tiles, grid barriers)",
                                           "branch": "one graph branch per video, tile shapes autotuned per frame "
                                                     "size"}[args.batch_form],
                          "megapixels_per_frame_step": px / BATCH_FRAMES / 1e6,
                          "l2": "flushed before each step (256 MB write, outside the events)"},
               "pixels_per_s": ws * args.steps * px / (total_ms / 1000.0), "gpu_launches": launches,
               "sequential": {"pixels_per_s": px / (seq_ms / 1000.0), "ms": seq_ms,
                              "how": "the same 24 videos x 10 frames on rank 0, one after another, each in its own "
                                     "context (graphs on, PCG loop autotuned per frame size, L2 flushed before each "
                                     "video), CUDA events around each video's 10 frames"},
               "e2e": None, "cpu_baseline": None, "clocks": clk}
        print(json.dumps(out), flush=True)


def time_sequential(shapes, weights, b0s, rgb, lab, N, M, flush):
    """The batch's videos solved one after another, each in its own context: one
    untimed pass (graph capture, autotuning once per frame size), then one timed
    pass per video.  Returns the summed device time in ms."""
    import torch

    from paper_1908_01961_b300 import gid
    stream = torch.cuda.current_stream()
    tiles, total = {}, 0.0
    for i, (H, W, K) in enumerate(shapes):
        s = gid.Solver(H, W, K, weights[i])
        s.set_base_colors(b0s[i])

        def solve():
            s.new_sequence()
            for t in range(BATCH_FRAMES):
                s.set_frame(rgb[i][t], lab[i][t])
                s.init(0 if t == 0 else 1)
                s.run(N, M)

        solve()
        if (H, W, K) in tiles:
            s.set_apply_tile(tiles[(H, W, K)])
        else:
            tiles[(H, W, K)] = s.autotune(5)[0]
        solve()
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        solve()
        b.record(stream)
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
        s.close()
    return total


# ---------------------------------------------------------------- long stream (1080p)

STREAM = synth.STREAM_1080P
STREAM_FRAMES = 60


def _stream_frame(args):
    seed, t = args
    v = synth.SyntheticVideo(STREAM["H"], STREAM["W"], STREAM["K"], STREAM["n_cells"], seed=seed)
    f = v.frame(t)
    return f.I.astype(np.float32), f.labels


def run_stream(args, ws, rank, local):
    """Per-frame latency of a 1920x1080 K=8 stream: frame 0 cold, then warm
    starts with temporal pairs, 8 GN x 20 PCG per frame.  Every frame's solve
    (ingest, initialisation, run) is bracketed by CUDA events on the solver's
    stream; the inputs are resident in HBM."""
    import multiprocessing as mp
    F = args.frames if args.frames != WORK["frames"] else STREAM_FRAMES
    seed = 7 + rank
    with mp.get_context("spawn").Pool(max(1, min(F, (os.cpu_count() or 2) - 1))) as pool:
        made = pool.map(_stream_frame, [(seed, t) for t in range(F)])   # before any CUDA call

    import torch

    from paper_1908_01961_b300 import gid

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, W, K, N, M = STREAM["H"], STREAM["W"], STREAM["K"], STREAM["N"], STREAM["M"]
    b0 = synth.initial_base_colors(made[0][0].astype(np.float64), made[0][1], K).astype(np.float32)
    off_s, off_t = synth.offsets_for(seed)
    rgb = [torch.from_numpy(I).to(dev) for I, _ in made]
    lab = [torch.from_numpy(l).to(dev) for _, l in made]
    s = gid.Solver(H, W, K, gid.default_weights(off_s, off_t, temporal=1))
    s.set_base_colors(b0)
    stream = torch.cuda.current_stream()
    s.set_frame(rgb[0], lab[0])
    s.init(0)
    if args.tile is None:
        tile_rows, tile_us = s.autotune(5)
    else:
        s.set_apply_tile(args.tile)
        tile_rows, tile_us = args.tile, "fixed by --tile"
    if args.l2_window:
        s.set_l2_window(True)

    def frame(t):
        s.set_frame(rgb[t], lab[t])
        s.init(0 if t == 0 else 1)
        s.run(N, M)

    for _ in range(args.warmup):
        s.new_sequence()
        frame(0)
    torch.cuda.synchronize()
    s.new_sequence()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(F)]
    barrier(ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    n0 = s.launch_count()
    for t in range(F):
        ev[t][0].record(stream)
        frame(t)
        ev[t][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    launches = s.launch_count() - n0
    clk = clocks.stop()
    lat = np.array([a.elapsed_time(b) for a, b in ev])
    total_ms = max_over_ranks(ws, float(lat.sum()))
    E, _ = s.energy()
    if not np.isfinite(E):
        raise RuntimeError("non-finite energy after the stream")
    parity = stream_parity(s, made, rgb, lab, off_s, off_t, b0, frame) if args.parity and rank == 0 else None
    if rank == 0:
        out = {"metric": "per-frame latency of a 1920x1080 K=8 stream (8 GN x 20 PCG per frame)",
               "value": float(np.percentile(lat, 50)), "unit": "ms", "n_gpus": ws, "steps": 1,
               "warmup": args.warmup, "ms_per_step": total_ms, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"stream_1920x1080_K8: {F} frames, 80 moving Voronoi cells, rotating light; "
                                      "frame 0 cold, then warm starts with temporal pairs", "H": H, "W": W, "K": K,
                          "frames": F, "N_outer": N, "M_inner": M,
                          "operator_tile": pcg_loop_name(s, tile_rows) + (f" (autotuned; us per PCG step {tile_us})"
                                                                          if args.tile is None else " (fixed)"),
                          "l2_window": s.l2_window(),
                          "l2": "inputs (20 MB per frame of planes, 190 MB per PCG vector set) exceed the L2"},
               "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                              "max": float(lat.max()), "first_frame": float(lat[0])},
               "frames_per_s": ws * F / (total_ms / 1000.0), "gpu_launches": launches, "e2e": None,
               "cpu_baseline": None, "clocks": clk, "final_energy": E, "parity": parity}
        print(json.dumps(out), flush=True)


def stream_parity(s, made, rgb, lab, off_s, off_t, b0, frame):
    """Per-layer error of the stream's frames 0, 33, 66, ... against the FP64
    oracle.  The stream is replayed from its start; at a sampled frame t the
    GPU's state and colours after frame t - 1 are read, the GPU solves frame t
    (N x M, warm start, temporal pairs) and the oracle solves the same frame
    from the same state, cast to FP64 (frame 0: both from the cold start)."""
    import oracle as O
    O.build()
    O.set_threads(host_threads())
    N, M, K = STREAM["N"], STREAM["M"], STREAM["K"]
    F = len(made)
    sample = list(range(0, F, 33))
    out, gpu = {}, {}
    s.new_sequence()
    for t in range(F):
        if t in sample:
            Xp = s.state().cpu().numpy().astype(np.float64) if t > 0 else None
            bp = s.base_colors().astype(np.float64) if t > 0 else None
        frame(t)
        if t in sample:
            R, T = s.layers()
            E, _ = s.energy()
            gpu[t] = (R.cpu().numpy(), T.cpu().numpy(), s.base_colors(), E, Xp, bp)
    t0 = time.perf_counter()
    for t in sample:
        R, T, bg, E, Xp, bp = gpu[t]
        I = made[t][0].astype(np.float64)
        if t == 0:
            C, wsr, om, _ = O.precompute(I, off_s)
            pb = O.Problem(I, made[t][1], b0.astype(np.float64), wsr, om, off_s)
            X0 = pb.init_cold()
        else:
            Ip = made[t - 1][0].astype(np.float64)
            C, wsr, om, omt = O.precompute(I, off_s, off_t, Iprev=Ip)
            pb = O.Problem(I, made[t][1], b0.astype(np.float64), wsr, om, off_s, omega_t=omt, off_t=off_t,
                           rprev=Xp[:3], b=bp)
            X0 = Xp
        Xo, bo, hist = O.solve_frame(pb, X0, N, M)
        out[str(t)] = layer_errors(R, T, bg, E, Xo, bo, hist[-1].sum())
    worst = {}
    for rec in out.values():
        for k, v in rec.items():
            if isinstance(v, dict):
                worst[k] = max(worst.get(k, 0.0), v["max_abs"])
    return {"frames": sample, "per_frame": out, "worst_max_abs": worst,
            "worst_energy_rel": max(r["energy_rel"] for r in out.values()),
            "nonneg_branch_flips": {t: r["nonneg_branch_flips"] for t, r in out.items()},
            "meets_bar": all(r["meets_bar"] for r in out.values()), "oracle_seconds": time.perf_counter() - t0,
            "oracle_threads": host_threads(), "start": "each sampled frame from the GPU's state after the previous "
            "frame (frame 0: cold start); N x M = 8 x 20"}


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batch":
        run_batch(args, ws, rank, local)
    elif args.workload == "stream":
        run_stream(args, ws, rank, local)
    else:
        run_gid(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
