"""Benchmark: online IS-NMF frames/s at F=513, K=100 on GB300.

Workload (the long-stream configuration): F=513, K=100, minibatch beta=1000,
10 inner h iterations, fresh restarts, one pass over a seeded gamma-model
stream generated on the device. One step = one onmf_push_frames call of
1,000,000 frames (1000 minibatches) already resident in HBM; 10 steps are
the full 10^7-frame pass. Inputs are larger than L2 (2.05 GB per step), so no
L2 flush is needed between steps.

Reported: frames/s of the mixed-precision path (value), the plain FP32 GPU
path on the same workload, their objective agreement, the roofline of the
step kernel, an end-to-end number through the C ABI with host buffers (and
the host link's own rate), the FP64 oracle on the host cores
(cpu_baseline), SM clocks during the timed region, the library's kernel
launch count, the drift of each arithmetic of A and B, batch IS-NMF on the
same stream, the objective-vs-time comparison, the parameter study and the
serving replay.

--impl reference times the FP64 CPU oracle as the reference arm.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

F, K, BETA, N_IN = 513, 100, 1000, 10
FLOP_PER_FRAME = (6 * N_IN + 6) * F * K  # algorithmic flops of one frame
METRIC = "online IS-NMF frames/s (F=513,K=100)"
WORKLOAD = "online IS-NMF long stream F=513 K=100 beta=1000 n_inner=10, %s frames/step"


def workload(fps):
    return WORKLOAD % ("1e6" if fps == 1_000_000 else "{:,}".format(fps))


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--frames-per-step", type=int, default=1_000_000)
    p.add_argument("--hsolve", default="auto", choices=["auto", "mma", "tc", "cluster"],
                   help="h-solve kernel of the mixed path; auto: the autotuner's choice")
    p.add_argument("--skip-fp32", action="store_true")
    p.add_argument("--accumulate", default="auto",
                   choices=["auto", "fp64", "fp32", "fp32_compensated"],
                   help="arithmetic of A, B on the mixed path; auto: measure the drift of "
                        "each over one pass and take the fastest within bounds")
    p.add_argument("--skip-e2e", action="store_true")
    p.add_argument("--skip-batch-long", action="store_true",
                   help="skip the batch cycles over the whole long stream")
    p.add_argument("--skip-cpu", action="store_true")
    p.add_argument("--cpu-sample-minibatches", type=int, default=120)
    p.add_argument("--skip-c2", action="store_true",
                   help="skip the objective-vs-time comparison (online vs batch)")
    p.add_argument("--skip-study", action="store_true",
                   help="skip the forgetting-factor / init / warm-restart study")
    p.add_argument("--serve-seconds", type=float, default=30.0,
                   help="wall window of the serving replay (0 skips serving)")
    p.add_argument("--serve-direct-seconds", type=float, default=10.0,
                   help="window of a second replay with direct launches (0 skips it)")
    p.add_argument("--serve-fork-seconds", type=float, default=10.0,
                   help="window of a replay whose h-solve is one launch per dictionary size "
                        "(0 skips it)")
    p.add_argument("--phase-timing", action="store_true",
                   help="measurement build of the library (clock64 stamps at the phase "
                        "boundaries of the online step): print the per-phase table and exit")
    p.add_argument("--phase-dump", default=None,
                   help="with --phase-timing: also save the raw stamps "
                        "[minibatch][CTA][point] to this .npy file")
    p.add_argument("--probe-tcgen05", action="store_true",
                   help="build and run the tcgen05 issue-cost probe "
                        "(paper_1106_4198_gb300/probes/tcgen05_issue.cu) and exit")
    p.add_argument("--stats-ranges", type=int, default=-1,
                   help="statistics schedule of the mma path (onmf_config.stats_ranges); "
                        "-1: the autotuner's choice (or automatic with --hsolve given)")
    p.add_argument("--serve-streams", type=int, default=256)
    p.add_argument("--serve-budget", type=int, default=1 << 30)
    return p.parse_args()


# ------------------------------------------------------------- distributed


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


DRIFT_W, DRIFT_AB = 1e-6, 1e-9
BATCH_LONG_CYCLES = 3


def choose_accumulate(drift):
    """The fastest arithmetic of A, B whose drift against the FP64 sums over
    the measured pass stays within DRIFT_W (W) and DRIFT_AB (A, B); FP64
    itself always qualifies."""
    ok = [n for n in ("fp64", "fp32", "fp32_compensated") if n in drift and (
        n == "fp64" or (drift[n]["W_rel"] <= DRIFT_W and drift[n]["A_rel"] <= DRIFT_AB
                        and drift[n]["B_rel"] <= DRIFT_AB))]
    return min(ok, key=lambda n: drift[n]["ms_per_1e6_frames"])


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, x, device="cpu"):
    """Max of a float over all ranks (x itself at world size 1)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x, device="cpu"):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        import statistics
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- peaks


# DRAM bytes (read + write) per frame of the step kernel, from one ncu
# capture of each h-solve variant (64,000 frames, scaled per frame: the
# traffic is proportional to the frames processed). A variant that changed
# since its capture is absent here and reports traffic = null.
NCU_TRAFFIC_PER_FRAME = {"mma": 2166.3}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# -------------------------------------------------------------- our arm


def run_ours(args):
    import numpy as np
    import torch

    import paper_1106_4198_gb300 as onmf
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    fps = args.frames_per_step
    seed = synth.DATA_SEED + 7919 * rank  # each rank: its own stream
    Wstar = torch.as_tensor(synth.dictionary(F, K, seed), dtype=torch.float32,
                            device=dev)
    W0 = synth.init_dictionary(F, K)
    # inputs resident in HBM before the timed region
    chunks = [synth.device_frames(F, K, fps, seed=seed, chunk=c, Wstar=Wstar)
              for c in range(args.steps)]
    torch.cuda.synchronize()

    # the mixed path runs the h-solve kernel the autotuner measures fastest,
    # unless --hsolve names one
    tune_cfg = onmf.onmf_config_default(F, K, precision=onmf.ONMF_MIXED, beta=BETA,
                                        n_inner=N_IN)
    ranges, tune_ranges_us = max(0, args.stats_ranges), None
    if args.hsolve == "auto":
        hsolve, tuned, tune_us, tune_ranges_us, _ = onmf.onmf_autotune(tune_cfg, stream=stream)
        ranges = tuned if args.stats_ranges < 0 else args.stats_ranges
    else:
        hsolve = [k for k, v in onmf.HSOLVE_NAMES.items() if v == args.hsolve][0]
        tune_us = None
    hname = onmf.HSOLVE_NAMES[hsolve]

    # drift of the running statistics A, B over the whole stream in each
    # arithmetic (FP64 sums as the reference); one pass of all the chunks
    drift = None
    acc = {v: k for k, v in onmf.ACC_NAMES.items()}.get(args.accumulate, onmf.ONMF_ACC_FP64)
    if rank == 0 and args.accumulate == "auto":
        runs = {}
        # two rounds, the modes interleaved; the time of a mode is its faster
        # pass (the results are deterministic, the same in both rounds)
        for _ in range(2):
            for mode in (onmf.ONMF_ACC_FP64, onmf.ONMF_ACC_FP32, onmf.ONMF_ACC_FP32_COMP):
                m = onmf.OnlineISNMF(F, K, W0, stream=stream, beta=BETA, n_inner=N_IN,
                                     precision=onmf.ONMF_MIXED, hsolve=hsolve, accumulate=mode,
                                     stats_ranges=ranges)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for c in chunks:
                    m.push(c)
                e1.record(stream)
                m.sync()
                A, B, t, ls = m.stats()
                name = onmf.ACC_NAMES[mode]
                ms = e0.elapsed_time(e1)
                if name in runs:
                    ms = min(ms, runs[name]["ms"])
                runs[name] = dict(W=m.W(), A=A, B=B, t=t, loss=ls, ms=ms)
                m.close()
        ref = runs["fp64"]

        def rel(a, b):
            return float(np.linalg.norm(a - b) / np.linalg.norm(b))
        drift = {"frames": int(ref["t"]), "minibatches": int(ref["t"]) // BETA,
                 "reference": "the same pass with FP64 sums"}
        for name, r in runs.items():
            drift[name] = {"ms_per_1e6_frames": r["ms"] / (r["t"] / 1e6)}
            if name != "fp64":
                drift[name].update(W_rel=rel(r["W"], ref["W"]), A_rel=rel(r["A"], ref["A"]),
                                   B_rel=rel(r["B"], ref["B"]),
                                   loss_rel=abs(r["loss"] - ref["loss"]) / ref["loss"])
        drift["rule"] = ("fastest arithmetic whose W drifts <= %g and A, B <= %g "
                         "relative to FP64 sums" % (DRIFT_W, DRIFT_AB))
        name = choose_accumulate(drift)
        drift["choice"] = name
        acc = {v: k for k, v in onmf.ACC_NAMES.items()}[name]
    acc = int(max_over_ranks(dist, float(acc) if rank == 0 else -1.0, dev))

    def timed_pass(precision, record_launch_times=False):
        m = onmf.OnlineISNMF(F, K, W0, stream=stream, beta=BETA, n_inner=N_IN,
                             precision=precision,
                             hsolve=hsolve if precision == onmf.ONMF_MIXED else 0,
                             accumulate=acc if precision == onmf.ONMF_MIXED else 0,
                             stats_ranges=ranges if precision == onmf.ONMF_MIXED else 0)
        for w in range(args.warmup):
            m.push(chunks[w % len(chunks)])
        m.sync()
        zero = np.zeros((K, F))
        m.set_state(W0, zero, zero, 0, 0.0)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        barrier(dist, local)
        torch.cuda.synchronize()
        l0 = onmf.onmf_kernel_launches()
        with ClockSampler(local) as clk:
            evs[0].record(stream)
            for i in range(args.steps):
                m.push(chunks[i])
                evs[i + 1].record(stream)
            torch.cuda.synchronize()
        barrier(dist, local)
        launches = onmf.onmf_kernel_launches() - l0
        per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
        total_ms = evs[0].elapsed_time(evs[-1])
        _, _, t, ls = m.stats()
        W_end = m.W()
        m.close()
        return dict(ms=total_ms, per_step_ms=per, launches=launches,
                    frames=t, loss=ls / max(t, 1), clocks=clk.summary(), W=W_end)

    mixed = timed_pass(onmf.ONMF_MIXED)

    # end to end through the C ABI with pinned host buffers, right after the
    # device-resident pass (before the FP32 comparison, whose seconds of
    # FMA load would leave the GPU in another clock state)
    e2e = None
    if not args.skip_e2e:
        host = [torch.empty((fps, F), dtype=torch.float32, pin_memory=True)
                for _ in range(2)]
        host[0].copy_(chunks[0])
        host[1].copy_(chunks[1 % len(chunks)])
        m = onmf.OnlineISNMF(F, K, W0, stream=stream, beta=BETA, n_inner=N_IN,
                             precision=onmf.ONMF_MIXED, hsolve=hsolve, accumulate=acc,
                             stats_ranges=ranges)
        for w in range(args.warmup):
            m.push(host[w % 2].numpy())
        m.sync()
        # the copy engine's rate from the same pinned buffer (one step of
        # frames), for context: the library pulls pinned frames with a kernel
        scratch = torch.empty_like(chunks[0])
        l0e, l1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(2):
            l0e.record(stream)
            scratch.copy_(host[0], non_blocking=True)
            l1e.record(stream)
            torch.cuda.synchronize()
        link_gbs = fps * F * 4 / (l0e.elapsed_time(l1e) * 1e6)
        del scratch
        res = np.zeros(1)
        barrier(dist, local)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            for i in range(args.steps):
                m.push(host[i % 2].numpy())
                _, res[0] = onmf.onmf_get_stats(m.state)  # device->host read of the result
            torch.cuda.synchronize()
            e2e_s = max_over_ranks(dist, time.perf_counter() - t0, dev)
        m.close()
        e2e = {"value": sum_over_ranks(dist, fps * args.steps, dev) / e2e_s,
               "unit": "frames/s", "h2d_bytes_per_step": fps * F * 4,
               "d2h_bytes_per_step": 8, "clocks": clk.summary(),
               "h2d_copy_engine_gbs": link_gbs}
        del host

    fp32 = None if args.skip_fp32 else timed_pass(onmf.ONMF_FP32)
    unfused = None if (args.skip_fp32 or rank != 0) else run_unfused_fp32(chunks, W0)

    # batch IS-NMF on the same long stream, which fits in HBM here: a few
    # cycles over every frame, and both dictionaries scored alike (h of every
    # frame re-solved with W fixed, mean d_IS per frame)
    batch_long = None
    if rank == 0 and not args.skip_batch_long:
        Vall = torch.cat(chunks)
        N_all = Vall.shape[0]
        Wb = torch.as_tensor(W0, device=dev).contiguous()
        Hb = torch.empty((N_all, K), device=dev)

        def score_long(W):
            sc = onmf.OnlineISNMF(F, K, W, stream=stream, beta=BETA, n_inner=N_IN,
                                  precision=onmf.ONMF_MIXED)
            o = sc.project(Vall, Hb, n_inner=N_IN, want_obj=True)
            sc.close()
            return o / N_all

        s_init = score_long(W0)
        s_online = score_long(mixed["W"])
        onmf.nmf_batch_init_H(Vall, Wb, Hb, stream=stream)
        plan = onmf.BatchPlan(F, K, N_all, onmf.ONMF_MIXED)  # scratch outside the timing
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        obj = plan.step(Vall, Wb, Hb, n_iter=BATCH_LONG_CYCLES, stream=stream)
        b1.record(stream)
        torch.cuda.synchronize()
        plan.close()
        batch_ms = b0.elapsed_time(b1)
        s_batch = score_long(Wb.cpu().numpy())
        batch_long = {
            "frames": int(N_all), "cycles": BATCH_LONG_CYCLES,
            "ms_per_cycle": batch_ms / BATCH_LONG_CYCLES,
            "batch_own_objective_per_cycle": [float(x) for x in obj],
            "score": "mean d_IS per frame, every frame's h re-solved with W fixed "
                     "(%d iterations)" % N_IN,
            "score_initial_W": s_init, "score_online_pass_W": s_online,
            "score_batch_W": s_batch, "online_pass_ms": mixed["ms"]}
        del Vall, Hb, Wb
        torch.cuda.empty_cache()

    ms = max_over_ranks(dist, mixed["ms"], dev)
    total_frames = sum_over_ranks(dist, fps * args.steps, dev)
    value = total_frames / (ms / 1e3)
    out = None
    if rank == 0:
        peaks = measured_peaks()
        launch_ms = sum(mixed["per_step_ms"]) / len(mixed["per_step_ms"])
        achieved = FLOP_PER_FRAME * fps / (launch_ms / 1e3) / 1e12
        peak = peaks.get("bf16_tflops_sustained") or 1700.0
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": (NCU_TRAFFIC_PER_FRAME[hname] * fps
                            if hname in NCU_TRAFFIC_PER_FRAME else None),
                "traffic_note": "DRAM bytes per launch of %d frames, scaled from an ncu "
                                "capture of 64,000 frames" % fps,
                "kernel": "online step kernel, mixed precision, %s h-solve" % hname,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained"
                if peaks else "fallback"}
        out = {
            "metric": METRIC, "value": value, "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic gamma-model spectrogram generated on device",
            "config": {"workload": workload(fps), "F": F, "K": K, "beta": BETA,
                       "n_inner": N_IN, "frames_per_step": fps,
                       "global_batch": fps * world,
                       "l2": "inputs 2.05 GB/step > L2, no flush",
                       "hsolve": hname,
                       "accumulate": onmf.ACC_NAMES[acc],
                       "autotune_us_per_minibatch": tune_us,
                       "stats_ranges": ranges,
                       "autotune_stats_ranges_us": ({str(k): v for k, v in tune_ranges_us.items()}
                                                    if tune_ranges_us else None),
                       "parallelism": "replicas" if world > 1 else "single"},
            "fp32_value": (total_frames / (fp32["ms"] / 1e3)) if fp32 else None,
            "fp32_clocks": fp32["clocks"] if fp32 else None,
            "fp32_unfused_torch": unfused,
            "speedup_vs_fp32": (fp32["ms"] / mixed["ms"]) if fp32 else None,
            "objective": mixed["loss"],
            "objective_fp32": fp32["loss"] if fp32 else None,
            "objective_rel_diff": (abs(mixed["loss"] - fp32["loss"]) / fp32["loss"])
            if fp32 else None,
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": mixed["launches"],
            "clocks": mixed["clocks"],
            "accumulator_drift": drift,
            "batch_long_stream": batch_long,
        }
    return out, dist


# ------------------------------------- unfused FP32 (cuBLAS + elementwise)


def unfused_minibatch(Vmb, W, A, B, eps=1e-12, n_in=10):
    """One step of Algorithm 1 written out with PyTorch ops on any device and
    dtype: Vmb (n, F) frames, W, A, B (F, K). Fresh-restart start point
    h0 = sum_f y_f / sum W for every k, n_in multiplicative h updates with
    exponent 1/2, X from the final h, A += (P H^T) o W^2, B += Q H^T,
    W = sqrt(A/B), then the L1 column rescale of W, A, B."""
    import torch
    Y = Vmb.t() + eps  # F x n
    H = (Y.sum(0) / W.sum()).expand(W.shape[1], Y.shape[1]).contiguous()
    for _ in range(n_in):
        X = W @ H + eps
        H = H * torch.sqrt((W.t() @ (Y / (X * X))) / (W.t() @ (1.0 / X)))
    X = W @ H + eps
    P, Q = Y / (X * X), 1.0 / X
    A = A + (P @ H.t()) * W * W
    B = B + Q @ H.t()
    W = torch.sqrt(A / B)
    s = W.sum(0)
    return W / s, A / s, B * s


def run_unfused_fp32(chunks, W0, n_mb=20, warm=3):
    """The plain FP32 GPU form written out with PyTorch CUDA ops (cuBLAS SGEMM
    with TF32 off, one elementwise kernel per step, FP32 everywhere): the
    same Algorithm 1 step per minibatch, on the first n_mb minibatches of the
    stream after `warm` untimed ones. A comparison leg of the benchmark, not
    part of the library."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        V = chunks[0]
        eps = 1e-12
        W = torch.as_tensor(W0, device=V.device).t().contiguous()  # F x K
        A = torch.zeros_like(W)
        B = torch.zeros_like(W)

        def minibatch(j, W, A, B):
            return unfused_minibatch(V[j * BETA:(j + 1) * BETA], W, A, B, eps, N_IN)

        for j in range(warm):
            W, A, B = minibatch(j, W, A, B)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for j in range(warm, warm + n_mb):
            W, A, B = minibatch(j, W, A, B)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return {"value": n_mb * BETA / (ms / 1e3), "unit": "frames/s",
            "us_per_minibatch": 1e3 * ms / n_mb,
            "sample": "%d minibatches after %d untimed ones" % (n_mb, warm),
            "what": "Algorithm 1 in PyTorch FP32 ops: cuBLAS SGEMM (TF32 off) and "
                    "elementwise kernels, about 8 launches per inner iteration"}


# ----------------------------------------------------------------- serving

HOP_S = 0.032         # 32 ms hop
SPEEDUP = 4.0         # arrivals at 4x real time
SERVE_KS = (16, 32, 64, 128)


def serving_schedule(n_streams, window_s, rng):
    """Per-stream chunk arrivals: K ~ U{16,32,64,128}; stream length
    log-uniform over 10 s .. 2 h of 32 ms frames; chunk length log-uniform
    integer in [8, 512]; chunks of a stream arrive as a Poisson process whose
    frame rate is 4x real time; stream starts uniform over the first 60 s of
    the replay (scaled into the window). Returns (streams, events) with
    events = [(t, stream, n)] sorted by time."""
    streams = []
    events = []
    rate = SPEEDUP / HOP_S  # frames per second per stream
    start_span = min(60.0, window_s / 2)
    for i in range(n_streams):
        K = int(rng.choice(SERVE_KS))
        length = int(np.exp(rng.uniform(np.log(10 / HOP_S), np.log(7200 / HOP_S))))
        t = rng.uniform(0, start_span)
        left = length
        while left > 0 and t < window_s:
            n = int(min(left, np.floor(np.exp(rng.uniform(np.log(8), np.log(513))))))
            t += rng.exponential(n / rate)
            if t >= window_s:
                break
            events.append((t, i, n))
            left -= n
        streams.append(K)
    events.sort()
    return streams, events


SUBMIT_THREADS = 8


def run_serving(args, precision, launch=0, window_s=None):
    """launch: 0 = each batch one captured CUDA graph, 1 = direct launches."""
    import paper_1106_4198_gb300 as onmf
    import synth
    window_s = window_s or args.serve_seconds
    rng = np.random.default_rng(4321)
    Ks, events = serving_schedule(args.serve_streams, window_s, rng)
    pool = synth.spectrogram(F, 64, 65536, seed=synth.DATA_SEED + 17)  # gamma-model frames
    srv = onmf.onmf_server_create(F, max_chunk=512, max_batch=256, slots=2,
                                  budget_bytes=args.serve_budget, precision=precision,
                                  launch=launch)
    lat, frames_done = [], 0
    try:
        ids = []
        for i, K in enumerate(Ks):
            cfg = onmf.onmf_config_default(F, K, precision=precision, n_inner=N_IN)
            ids.append(onmf.onmf_server_open_stream(srv, cfg, synth.init_dictionary(F, K)))
        # warm-up: one chunk per stream
        for sid in ids:
            onmf.onmf_server_submit(srv, sid, pool[:32], tag=-1)
        got = 0
        while got < len(ids):
            got += len(onmf.onmf_server_poll(srv, 1024, wait_ms=1000))
        # timed replay at the scheduled arrival times
        t0 = time.perf_counter()
        k = 0
        pending = 0
        while k < len(events) or pending:
            now = time.perf_counter() - t0
            while k < len(events) and events[k][0] <= now:
                _, i, n = events[k]
                off = int(rng.integers(0, pool.shape[0] - n))
                onmf.onmf_server_submit(srv, ids[i], pool[off:off + n], tag=k)
                pending += 1
                k += 1
            wait = 0 if k < len(events) else 50
            for cp in onmf.onmf_server_poll(srv, 1024, wait_ms=wait):
                lat.append(cp.t_done - cp.t_submit)
                frames_done += cp.frames
                pending -= 1
            if k < len(events):
                nxt = events[k][0] - (time.perf_counter() - t0)
                if nxt > 0.0005:
                    time.sleep(min(nxt, 0.002))
        replay_s = time.perf_counter() - t0
        st_replay = onmf.onmf_server_get_stats(srv)
        # saturation: the same chunks submitted at once by SUBMIT_THREADS
        # client threads, each one onmf_server_submit_many call over its
        # share of the streams (each stream's chunks in order; the copies run
        # without the GIL)
        offs = [int(rng.integers(0, pool.shape[0] - n)) for _, _, n in events]
        sat_frames = sum(n for _, _, n in events)
        shares = []
        for t in range(SUBMIT_THREADS):
            ks = [k for k, (_, i, _) in enumerate(events) if i % SUBMIT_THREADS == t]
            shares.append(([ids[events[k][1]] for k in ks],
                           [pool[offs[k]:offs[k] + events[k][2]] for k in ks], ks))

        def submitter(t):
            sids, vs, tags = shares[t]
            onmf.onmf_server_submit_many(srv, sids, vs, tags)

        def saturate():
            threads = [threading.Thread(target=submitter, args=(t,))
                       for t in range(SUBMIT_THREADS)]
            t1 = time.perf_counter()
            for th in threads:
                th.start()
            for th in threads:
                th.join()
            submit_s = time.perf_counter() - t1
            got = 0
            while got < len(events):
                got += len(onmf.onmf_server_poll(srv, 4096, wait_ms=1000))
            return submit_s, time.perf_counter() - t1

        saturate()  # warm-up: grows the server's pinned chunk arena to the queue depth
        st_replay = onmf.onmf_server_get_stats(srv)
        submit_s, sat_s = saturate()
        st = onmf.onmf_server_get_stats(srv)
    finally:
        onmf.onmf_server_destroy(srv)
    lat_ms = np.array(lat) * 1e3
    offered = sum(n for _, _, n in events) / window_s
    return {
        "workload": "%d streams, K in {16,32,64,128}, F=513, chunks 8-512 frames, "
                    "Poisson arrivals at 4x real time, %.0f s replay" % (len(Ks), window_s),
        "launch": "cuda graph per batch" if launch == 0 else "direct kernel launches",
        "hsolve_launches": ("one per dictionary size" if os.environ.get("ONMF_SERVE_FORK") == "1"
                            else "one over all dictionary sizes"),
        "chunks": len(events), "frames": int(frames_done),
        "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat) else None,
        "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat) else None,
        "max_ms": float(lat_ms.max()) if len(lat) else None,
        "offered_frames_per_s": offered,
        "achieved_frames_per_s": frames_done / replay_s,
        "saturation_frames_per_s": sat_frames / sat_s,
        "saturation_submit_s": submit_s, "saturation_s": sat_s,
        "saturation_client_threads": SUBMIT_THREADS,
        "saturation_host_batch_s": (st["host_batch_ns"] - st_replay["host_batch_ns"]) * 1e-9,
        "saturation_device_s": (st["device_ns"] - st_replay["device_ns"]) * 1e-9,
        "saturation_kernel_launches": st["launches"] - st_replay["launches"],
        "launches": st["launches"], "batches_overlapped": st["batches_overlapped"],
        "budget_bytes": args.serve_budget, "precision": "mixed" if precision else "fp32",
    }


# ----------------------------------------------------------- oracle (CPU)


# ------------------------------------- objective vs time: online vs batch

C2_F, C2_K, C2_N, C2_ITERS = 513, 50, 112_500, 200


def run_c2(precision):
    """Objective against device time for one online pass (beta = 1000 and
    100, n_inner = 10, fresh restarts) and 200 batch multiplicative-update
    cycles on the same 112,500 x 513 gamma-model spectrogram, K = 50.

    Both methods are scored alike: at each checkpoint the current W is held
    fixed and every frame's h is solved from the fresh-restart start point
    (onmf_project, 10 iterations); the score is the mean d_IS per frame.
    Batch also reports its own objective (with its current H). Times are
    CUDA-event device times of the updates only (scoring excluded)."""
    import torch

    import paper_1106_4198_gb300 as onmf
    import synth

    F_, K_, N_ = C2_F, C2_K, C2_N
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    seed = synth.DATA_SEED + 2
    Wstar = torch.as_tensor(synth.dictionary(F_, K_, seed), dtype=torch.float32, device=dev)
    V = synth.device_frames(F_, K_, N_, seed=seed, chunk=0, Wstar=Wstar)
    W0 = synth.init_dictionary(F_, K_)
    Hs = torch.empty((N_, K_), device=dev)

    def score(W):
        s = onmf.OnlineISNMF(F_, K_, W, stream=stream, beta=1000, n_inner=N_IN,
                             precision=precision)
        obj = s.project(V, Hs, n_inner=N_IN, want_obj=True)
        s.close()
        return obj / N_

    curves = {}
    for beta in (1000, 100):
        m = onmf.OnlineISNMF(F_, K_, W0, stream=stream, beta=beta, n_inner=N_IN,
                             precision=precision)
        pts = [(0.0, score(W0))]
        t = 0.0
        seg = N_ // 10
        for a in range(0, N_, seg):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.push(V[a:a + seg])
            if a + seg >= N_:
                m.flush()
            e1.record(stream)
            e1.synchronize()
            t += e0.elapsed_time(e1)
            pts.append((t, score(m.W())))
        m.close()
        curves["online_beta%d" % beta] = pts

    W = torch.as_tensor(np.asarray(W0, dtype=np.float32), device=dev).contiguous()
    H = torch.zeros((N_, K_), device=dev)
    onmf.nmf_batch_init_H(V, W, H, stream=stream)
    pts = [(0.0, score(W0))]
    own = []
    t = 0.0
    plan = onmf.BatchPlan(F_, K_, N_, precision)  # the cycles below allocate nothing
    for c in range(C2_ITERS // 10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obj = plan.step(V, W, H, n_iter=10, stream=stream)
        e1.record(stream)
        e1.synchronize()
        t += e0.elapsed_time(e1)
        own.extend(obj.tolist())
        pts.append((t, score(W.cpu().numpy())))
    plan.close()
    curves["batch"] = pts

    def first_time_below(pts, target):
        for tt, v in pts:
            if v <= target:
                return tt
        return None

    b_final = curves["batch"][-1][1]
    out = {"workload": "F=513 K=50 N=112,500 gamma-model spectrogram; online one pass "
                       "(beta 1000 and 100, n_inner 10) vs 200 batch MU cycles",
           "precision": "mixed" if precision == onmf.ONMF_MIXED else "fp32",
           "score": "mean d_IS per frame, h re-solved with W fixed (10 iterations)",
           "curves_ms_score": {k: [[round(a, 4), b] for a, b in v] for k, v in curves.items()},
           "batch_own_objective_first_last": [own[0], own[-1]]}
    for k in ("online_beta1000", "online_beta100"):
        t_end, s_end = curves[k][-1]
        out[k] = {"pass_ms": t_end, "final_score": s_end,
                  "batch_ms_to_same_score": first_time_below(curves["batch"], s_end),
                  "batch_score_at_same_time": min(
                      [v for tt, v in curves["batch"] if tt <= t_end] or [curves["batch"][0][1]])}
    out["batch"] = {"ms_200_cycles": curves["batch"][-1][0], "final_score": b_final}
    return out


# ------------------------------------------------ study: r, beta, init, passes

STUDY_R = (0.5, 0.7, 0.9, 1.0)
STUDY_BETA = (1, 10, 100, 1000)


def run_study(precision):
    """The parameter study of the paper's experiments (Section 3) on the
    112,500 x 513 gamma-model spectrogram with K = 50, split into 100,000
    training frames and 12,500 held-out frames. Every score is the mean
    d_IS per held-out frame with W fixed and h re-solved from the fresh
    restart (10 iterations); times are CUDA-event device times of training.
      - forgetting factor: one pass for every r in {0.5, 0.7, 0.9, 1} and
        beta in {1, 10, 100, 1000}, rho = r^(beta / 100,000);
      - initial dictionary: random Gamma(1,1) columns against 50 training
        frames (normalized), at beta = 1000, r = 0.7;
      - warm restarts: 5 passes with a new permutation each, one h update
        per visit, kept activations started at the batch start point;
      - forgetting factor over several passes (the small-set protocol of
        Section 3: warm restarts, one h update per visit, W drawn from the
        training frames): 2,000 training and 500 held-out frames, 10 passes
        with a new permutation each, r in {0.1, 0.3, 0.5, 0.7, 0.9, 1} x beta
        in {1, 10, 100, 1000}, rho = r^(beta / 2,000) (the past scaled by r
        per pass), and the literal placement of rho (on the new statistics)
        at r in {0.1, 0.5}; the held-out score after every pass."""
    import torch

    import paper_1106_4198_gb300 as onmf
    import synth

    F_, K_, N_ = C2_F, C2_K, C2_N
    n_train = 100_000
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    seed = synth.DATA_SEED + 2
    Wstar = torch.as_tensor(synth.dictionary(F_, K_, seed), dtype=torch.float32, device=dev)
    V = synth.device_frames(F_, K_, N_, seed=seed, chunk=0, Wstar=Wstar)
    Vtr, Vte = V[:n_train], V[n_train:]
    Hte = torch.empty((N_ - n_train, K_), device=dev)
    W0 = synth.init_dictionary(F_, K_)

    def score(W):
        s = onmf.OnlineISNMF(F_, K_, W, stream=stream, beta=1000, n_inner=N_IN,
                             precision=precision)
        obj = s.project(Vte, Hte, n_inner=N_IN, want_obj=True)
        s.close()
        return obj / (N_ - n_train)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def one_pass(W_init, beta, r):
        m = onmf.OnlineISNMF(F_, K_, W_init, stream=stream, beta=beta, n_inner=N_IN,
                             precision=precision, r=r, n_ref=n_train)
        ms = timed(lambda: (m.push(Vtr), m.flush()))
        W = m.W()
        m.close()
        return W, ms

    grid = []
    for r in STUDY_R:
        for beta in STUDY_BETA:
            W, ms = one_pass(W0, beta, r)
            sc = score(W)
            grid.append({"r": r, "beta": beta, "score": sc if np.isfinite(sc) else None,
                         "ms": ms})
    # initial dictionary from training frames (the paper's protocol)
    pick = np.random.default_rng(8).choice(n_train, K_, replace=False)
    Wd = Vtr[torch.as_tensor(pick, device=dev)].cpu().numpy().astype(np.float64)
    Wd /= Wd.sum(axis=1, keepdims=True)
    init = {}
    for name, Wi in (("gamma", W0), ("training_frames", Wd.astype(np.float32))):
        W, ms = one_pass(Wi, 1000, 0.7)
        init[name] = {"score_start": score(Wi), "score": score(W), "ms": ms}
    # warm restarts: several permuted passes, one h update per visit
    m = onmf.OnlineISNMF(F_, K_, W0, stream=stream, beta=1000, n_inner=1,
                         precision=precision, r=0.7, n_ref=n_train)
    Wt = torch.as_tensor(np.asarray(W0, dtype=np.float32), device=dev).contiguous()
    Hk = torch.zeros((n_train, K_), device=dev)
    onmf.nmf_batch_init_H(Vtr, Wt, Hk, stream=stream)
    rng = np.random.default_rng(9)
    warm, t = [], 0.0
    for p in range(5):
        order = torch.as_tensor(rng.permutation(n_train), dtype=torch.int64, device=dev)
        t += timed(lambda: (m.push_warm(Vtr, Hk, order), m.flush()))
        warm.append({"pass": p + 1, "ms": t, "score": score(m.W())})
    m.close()
    best = min((g for g in grid if g["score"] is not None), key=lambda g: g["score"])
    multipass = run_multipass_study(precision)
    return {"workload": "F=513 K=50 gamma-model spectrogram, 100,000 training and 12,500 "
                        "held-out frames; score = mean d_IS per held-out frame",
            "precision": "mixed" if precision == onmf.ONMF_MIXED else "fp32",
            "score_of_initial_W": score(W0),
            "r_beta_grid": grid, "best": best, "init": init, "warm_passes": warm,
            "r_beta_grid_multipass": multipass}


MP_TRAIN, MP_TEST, MP_PASSES = 2000, 500, 10
MP_R = (0.1, 0.3, 0.5, 0.7, 0.9, 1.0)


def run_multipass_study(precision):
    """Forgetting factor r and minibatch size beta over several passes of a
    small training set (Section 3, small data set: warm restarts, one update
    of h per visit, W initialized with training frames). rho = r^(beta/N)
    with N the training-set size (reading R19), so one pass scales the past
    by r. A setting is marked unstable when a pass leaves a non-finite W or
    the held-out score rises by more than 1 % over the best pass before it."""
    import torch

    import paper_1106_4198_gb300 as onmf
    import synth

    F_, K_ = C2_F, C2_K
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    seed = synth.DATA_SEED + 5
    Wstar = torch.as_tensor(synth.dictionary(F_, K_, seed), dtype=torch.float32, device=dev)
    V = synth.device_frames(F_, K_, MP_TRAIN + MP_TEST, seed=seed, chunk=0, Wstar=Wstar)
    Vtr, Vte = V[:MP_TRAIN].contiguous(), V[MP_TRAIN:].contiguous()
    Hte = torch.empty((MP_TEST, K_), device=dev)
    pick = np.random.default_rng(11).choice(MP_TRAIN, K_, replace=False)
    W0 = Vtr[torch.as_tensor(pick, device=dev)].cpu().numpy().astype(np.float64)
    W0 = (W0 / W0.sum(axis=1, keepdims=True)).astype(np.float32)

    def score(W):
        if not np.all(np.isfinite(W)):
            return None
        s = onmf.OnlineISNMF(F_, K_, W, stream=stream, beta=1000, n_inner=N_IN,
                             precision=precision)
        obj = s.project(Vte, Hte, n_inner=N_IN, want_obj=True)
        s.close()
        return obj / MP_TEST if np.isfinite(obj) else None

    out = {"workload": "F=513 K=50 gamma-model spectrogram, %d training and %d held-out "
                       "frames, %d permuted passes, warm restarts, one h update per visit, "
                       "W0 = normalized training frames" % (MP_TRAIN, MP_TEST, MP_PASSES),
           "score_of_initial_W": score(W0), "settings": []}
    cases = [(r, beta, 0) for r in MP_R for beta in STUDY_BETA]
    cases += [(r, beta, 1) for r in (0.1, 0.5) for beta in STUDY_BETA]
    for r, beta, on_new in cases:
        m = onmf.OnlineISNMF(F_, K_, W0, stream=stream, beta=beta, n_inner=1,
                             precision=precision, r=r, n_ref=MP_TRAIN, rho_on_new=on_new)
        Wt = torch.as_tensor(W0, device=dev).contiguous()
        Hk = torch.zeros((MP_TRAIN, K_), device=dev)
        onmf.nmf_batch_init_H(Vtr, Wt, Hk, stream=stream)
        rng = np.random.default_rng(12)
        scores, ms, err = [], 0.0, None
        for p in range(MP_PASSES):
            order = torch.as_tensor(rng.permutation(MP_TRAIN), dtype=torch.int64, device=dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            try:
                m.push_warm(Vtr, Hk, order)
                m.flush()
                e1.record(stream)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
                scores.append(score(m.W()))
            except onmf.OnmfError as x:  # a non-finite W stops the run
                err = str(x)
                break
        m.close()

        def rose(i):
            before = [x for x in scores[:i] if x is not None]
            return scores[i] is not None and bool(before) and scores[i] > 1.01 * min(before)

        unstable = (err is not None or any(x is None for x in scores)
                    or any(rose(i) for i in range(1, len(scores))))
        out["settings"].append({"r": r, "beta": beta, "rho_on_new": on_new,
                                "scores_per_pass": scores,
                                "ms_total": ms, "error": err, "unstable": bool(unstable),
                                "final": scores[-1] if scores else None})
    return out


def cpu_oracle_rate(n_mb, threads):
    """Frames/s of the FP64 oracle on a bounded sample of the workload."""
    import numpy as np

    import oracle
    import synth
    V = synth.spectrogram(F, K, n_mb * BETA)
    W0 = synth.init_dictionary(F, K)
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.online_pass(V, W0, beta=BETA, n_in=N_IN, want_H=False)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return n_mb * BETA / dt, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    threads = os.cpu_count() or 1
    import oracle
    if not oracle.have_openmp():
        threads = 1
    n_mb = 2
    for _ in range(args.warmup):
        cpu_oracle_rate(1, threads)
    times = []
    for _ in range(args.steps):
        rate, dt = cpu_oracle_rate(n_mb, threads)
        times.append(dt)
    total = n_mb * BETA * args.steps
    value = total / sum(times)
    sample = "%d minibatches (%d frames) of the workload per step" % (n_mb, n_mb * BETA)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic gamma-model spectrogram (host)",
        "config": {"workload": workload(getattr(args, "frames_per_step", 1_000_000)),
                   "F": F, "K": K, "beta": BETA, "n_inner": N_IN,
                   "frames_per_step": getattr(args, "frames_per_step", 1_000_000),
                   "global_batch": getattr(args, "frames_per_step", 1_000_000),
                   "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


PHASE_NAMES = ["h-solve", "wait after the h-solve", "statistics (tcgen05)",
               "barrier before the column pass", "column pass + loss", "barrier before the next minibatch"]
STAMP_PTS = 48  # points per (minibatch, CTA) record of the measurement build
UNIT_NAMES = ["range wait -> first chunk in shared memory", "first chunk -> MMAs issued",
              "MMAs done", "accumulators to shared memory", "partial-sum stores", "unit end"]


def run_phase_timing(args):
    """Per-phase timing of the online step (F=513, K=100, beta=1000, 10 inner
    iterations, mixed, mma h-solve, compensated sums) from the measurement
    build: 100 minibatches in one launch after a warm-up launch; per phase
    the mean over all CTAs of the launch and the slowest CTA (averaged over
    minibatches 1-98), in us at the SM clock measured from the launch's
    CUDA-event time; the steps of the statistics units averaged over the
    CTAs that run one."""
    import ctypes

    import torch

    import paper_1106_4198_gb300 as onmf
    import synth
    L = onmf.lib()
    L.onmf_phase_stamps.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int32)]
    ranges = max(0, args.stats_ranges)
    nmb = 100
    Wstar = torch.as_tensor(synth.dictionary(F, K, synth.DATA_SEED), dtype=torch.float32,
                            device="cuda")
    V = synth.device_frames(F, K, nmb * BETA, seed=synth.DATA_SEED, chunk=0, Wstar=Wstar)
    m = onmf.OnlineISNMF(F, K, synth.init_dictionary(F, K), beta=BETA, n_inner=N_IN,
                         precision=onmf.ONMF_MIXED, hsolve=onmf.ONMF_HSOLVE_MMA,
                         accumulate=onmf.ONMF_ACC_FP32_COMP, stats_ranges=ranges)
    buf = np.zeros(128 * 256 * STAMP_PTS, dtype=np.int64)
    grid = ctypes.c_int32(0)
    m.push(V)
    assert L.onmf_phase_stamps(m.state, buf.ctypes.data, buf.size, ctypes.byref(grid)) == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    m.push(V)
    e1.record()
    m.sync()
    ms = e0.elapsed_time(e1)
    assert L.onmf_phase_stamps(m.state, buf.ctypes.data, buf.size, ctypes.byref(grid)) == 0
    m.close()
    G = grid.value
    st = buf[:nmb * G * STAMP_PTS].reshape(nmb, G, STAMP_PTS)
    if args.phase_dump:
        np.save(args.phase_dump, st)
    mb = slice(1, nmb - 1)
    ns = st[:, :, :7]   # %globaltimer, ns
    clk = st[:, :, 8:15]  # clock64 of the statistics units
    # SM clock: CTA 0's unit clock against its globaltimer over the units
    has = clk[mb, :, 0] != 0
    out = {"workload": "F=513 K=100 beta=1000 n_inner=10, mixed, mma h-solve, compensated A/B, "
                       "100 minibatches in one launch", "stats_ranges": ranges, "grid": G,
           "us_per_minibatch": 1e3 * ms / nmb, "critical_path_us": {}, "per_cta_mean_us": {},
           "statistics_unit_us": {}}
    # critical path of a minibatch (all CTAs on one clock): the h-solve from
    # the first CTA's start to the last CTA's end, then each later step from
    # the end of the one before it (the last CTA) to its own end (the last
    # CTA), the barriers from the last arrival to the first CTA through
    first = lambda i: ns[mb, :, i].min(axis=1)
    last = lambda i: ns[mb, :, i].max(axis=1)
    nxt = ns[2:nmb, :, 0].min(axis=1)  # start of the next minibatch
    cp = {"h-solve": last(1) - first(0),
          "statistics (tcgen05, after the last h-solve)": last(3) - last(1),
          "barrier before the column pass": first(4) - last(3),
          "column pass + loss": last(5) - first(4),
          "barrier before the next minibatch": nxt - last(5)}
    for k, v in cp.items():
        out["critical_path_us"][k] = float(np.mean(v)) / 1e3
    out["critical_path_us"]["sum"] = float(sum(np.mean(v) for v in cp.values())) / 1e3
    for i, nm in enumerate(PHASE_NAMES):
        d = (ns[mb, :, i + 1] - ns[mb, :, i]) / 1e3
        out["per_cta_mean_us"][nm] = float(d.mean())
    # the window of the barrier before the column pass, per CTA: statistics
    # done (point 3) -> arrived, column loaded (32) -> next frames staged (33)
    # -> through (4)
    win = st[mb, :, 32:34]
    out["barrier_window_us"] = {
        "arrival (its release waits for the partial-sum stores), column W, A, B loads":
            float(np.mean(win[:, :, 0] - ns[mb, :, 3])) / 1e3,
        "next minibatch's frames staged": float(np.mean(win[:, :, 1] - win[:, :, 0])) / 1e3,
        "wait for the last arrival": float(np.mean(ns[mb, :, 4] - win[:, :, 1])) / 1e3,
        "last CTA out of the window after the last arrival":
            float(np.mean(win[:, :, 1].max(axis=1) - last(3))) / 1e3}
    span_clk = clk[mb, :, 6] - clk[mb, :, 0]
    span_ns = st[mb, :, 15] - st[mb, :, 7]
    ghz = float(np.median(span_clk[has] / np.maximum(span_ns[has], 1)))
    out["sm_ghz_estimate"] = ghz
    tl = st[mb, :, 38:40]
    has_t = tl[:, :, 0] != 0
    out["hsolve_outside_tile_us"] = {
        "minibatch start -> tile start (sum of W, W^T image copy issued)":
            float(np.mean((tl[:, :, 0] - ns[mb, :, 0])[has_t])) / 1e3,
        "tile end -> frame range released, next frames requested":
            float(np.mean((ns[mb, :, 1] - tl[:, :, 1])[has_t])) / 1e3}
    cs = st[mb, :, 40:45]
    okc = cs[:, :, 0] != 0
    out["column_step_us"] = {}
    for nm, (i, j) in {"partial sums of the ranges loaded and added": (0, 1),
                       "A, B, W' = sqrt(A/B)": (1, 2), "column sum (block reduction)": (2, 3),
                       "rescale, W, A, B and image stores": (3, 4)}.items():
        out["column_step_us"][nm] = float(np.mean((cs[:, :, j] - cs[:, :, i])[okc])) / ghz / 1e3
    sg = st[mb, :, 34:38]
    ok = sg[:, :, 0] != 0
    for nm, (i, j) in {"staging: frames in shared memory": (0, 1),
                       "staging: frame sums and input check": (1, 2),
                       "staging: f-major copy y = eps + v": (2, 3)}.items():
        out["barrier_window_us"][nm] = float(np.mean((sg[:, :, j] - sg[:, :, i])[ok])) / ghz / 1e3
    for i, nm in enumerate(UNIT_NAMES):
        d = np.where(has, (clk[mb, :, i + 1] - clk[mb, :, i]) / ghz / 1e3, np.nan)
        out["statistics_unit_us"][nm] = float(np.nanmean(d))
    # the h-solve tile of every CTA that has one (clock64)
    hs = st[mb, :, 16:32]
    hh = hs[:, :, 0] != 0
    steps = {"frames staged and converted": (0, 1), "W^T image in shared memory": (1, 2),
             "inner iteration 1": (2, 3), "inner iterations 2-10 (mean)": None,
             "inner iteration 10, step A (x = W h, ratios)": (11, 15),
             "inner iteration 10, step B (W^T [p q], h update)": (15, 12),
             "final ratios and loss": (12, 13), "P, Q, H rows written": (13, 14)}
    out["hsolve_tile_us"] = {}
    for nm, ij in steps.items():
        if ij is None:
            d = (hs[:, :, 12] - hs[:, :, 3]) / 9.0
        else:
            d = hs[:, :, ij[1]] - hs[:, :, ij[0]]
        out["hsolve_tile_us"][nm] = float(np.mean(d[hh])) / ghz / 1e3
    out["hsolve_tile_us"]["clocks per inner iteration 2-10"] = float(
        np.mean(((hs[:, :, 12] - hs[:, :, 3]) / 9.0)[hh]))
    return out


def run_probe_tcgen05():
    """Compile the tcgen05 issue-cost probe for sm_103a and run it; one JSON
    object per configuration."""
    here = os.path.dirname(os.path.abspath(__file__))
    pkg = os.path.join(here, "paper_1106_4198_gb300")
    src = os.path.join(pkg, "probes", "tcgen05_issue.cu")
    exe = os.path.join(pkg, "probes", "tcgen05_issue")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I" + os.path.join(pkg, "csrc"), "-I" + os.path.join(here, "include"),
                    src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, check=True)
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def main():
    args = parse()
    if args.probe_tcgen05:
        print(json.dumps({"probe": "tcgen05.mma issue cost and mma.sync throughput, one CTA",
                          "rows": run_probe_tcgen05()}),
              flush=True)
        return
    if args.phase_timing:
        os.environ["ONMF_LIB_VARIANT"] = "phase"
        print(json.dumps(run_phase_timing(args)), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out, dist = run_ours(args)
    rank, world, _ = dist_env()
    if rank == 0:
        if not args.skip_cpu and world == 1:
            threads = os.cpu_count() or 1
            import oracle
            if not oracle.have_openmp():
                threads = 1
            rate, dt = cpu_oracle_rate(args.cpu_sample_minibatches, threads)
            out["cpu_baseline"] = {
                "value": rate, "unit": "frames/s", "cores": threads, "kind": "oracle",
                "sample": "%d minibatches (%d frames) of the workload, %.1f s"
                          % (args.cpu_sample_minibatches,
                             args.cpu_sample_minibatches * BETA, dt)}
        if not args.skip_c2 and world == 1:
            import paper_1106_4198_gb300 as onmf
            out["objective_vs_time"] = run_c2(onmf.ONMF_MIXED)
        if not args.skip_study and world == 1:
            import paper_1106_4198_gb300 as onmf
            out["study"] = run_study(onmf.ONMF_MIXED)
        if args.serve_seconds > 0 and world == 1:
            import paper_1106_4198_gb300 as onmf
            out["serving"] = run_serving(args, onmf.ONMF_MIXED)
            if args.serve_direct_seconds > 0:
                d = run_serving(args, onmf.ONMF_MIXED, launch=onmf.ONMF_SERVE_DIRECT,
                                window_s=args.serve_direct_seconds)
                out["serving"]["direct_launch"] = {
                    k: d[k] for k in ("workload", "p50_ms", "p99_ms", "max_ms",
                                      "saturation_frames_per_s", "saturation_submit_s",
                                      "saturation_s", "launches")}
            if args.serve_fork_seconds > 0:
                # the h-solve as one launch per dictionary size on forked
                # streams (the library's earlier form), for comparison
                os.environ["ONMF_SERVE_FORK"] = "1"
                try:
                    d = run_serving(args, onmf.ONMF_MIXED, window_s=args.serve_fork_seconds)
                finally:
                    del os.environ["ONMF_SERVE_FORK"]
                out["serving"]["hsolve_launch_per_size"] = {
                    k: d[k] for k in ("workload", "p50_ms", "p99_ms", "max_ms",
                                      "saturation_frames_per_s", "saturation_s", "launches",
                                      "saturation_device_s")}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
