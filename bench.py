#!/usr/bin/env python3
"""Benchmark of the TT-rounding hot path on one GB300 (or N replicas).

Workload (one step): the rank-concatenating sum of 20 random TT tensors
(order 10, mode size 64, ranks 20, iid N(0,1) cores, coefficients U(-1,1);
concatenated rank 400) followed by TT-round at delta = 1e-6, through the C ABI
(tt_add + tt_round).  Inputs are uploaded once and stay resident in HBM; a
256 MB buffer is written between timed steps to flush the 129 MB L2.

Prints one JSON line (rank 0).  --impl reference times the CPU FP64 oracle on
the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TT-roundings/s at δ-accuracy, mixed vs FP64 on one GB300; serve p50/p99 latency"
UNIT = "roundings/s"
DELTA = 1e-6
WORKLOAD = "sum of 20 random TTs (d=10, n=64, ranks 20, N(0,1) cores, alpha~U(-1,1); concatenated rank 400) + TT-round at delta=1e-6"

# nominal / measured peaks (MEASURED_PEAKS.json when present)
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25
FP32_LANES_PER_SM = 128
SM_COUNT = None  # read from the device (cudaDevAttrMultiProcessorCount) by run_ours


def fp32_alu_peak(peaks):
    """FP32 CUDA-core peak in TFLOP/s: SMs x 128 FP32 lanes x 2 (FMA) x the
    maximum SM clock, with the SM count queried from the device."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return j, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def roofline_for(fam, prof, peaks, src):
    """bound, achieved, peak, unit for one kernel family."""
    secs = prof["total_ms"] / 1e3
    if fam == "gram_tf32_tc" or fam.startswith("gemm_tf32"):
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * NOMINAL_TF32_OVER_BF16
        return "tensor", prof["flops"] / secs / 1e12, peak, "TFLOP/s", (
            "%s sustained bf16 x nominal tf32/bf16 ratio 1.1/2.25" % src)
    if fam in ("gemm_f32", "gram_f32", "sgemm_f32", "sgram_f32"):
        return "alu", prof["flops"] / secs / 1e12, fp32_alu_peak(peaks), "TFLOP/s", (
            "%d SMs (queried) x 128 FP32 lanes x 2 x max SM clock" % SM_COUNT)
    if fam in ("gemm_f64", "gram_f64"):
        return "alu", prof["flops"] / secs / 1e12, 1.25, "TFLOP/s", "nominal GB300 FP64 rate"
    if fam == "chol_inv":
        # the r x r Cholesky + inverse: single-CTA (latency-bound) factors of the
        # diagonal blocks plus CUDA-core GEMMs; the roofline is the FP32 ALU of the GPU
        return "alu", prof["flops"] / secs / 1e12, fp32_alu_peak(peaks), "TFLOP/s", (
            "%d SMs (queried) x 128 FP32 lanes x 2 x max SM clock (the kernel is latency-bound on few SMs)"
            % SM_COUNT)
    return "hbm", prof["bytes"] / secs / 1e9, peaks["hbm_gbs"], "GB/s", "%s HBM copy bandwidth" % src


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of the ranks' values (every rank gets it): the slowest
    replica sets the job's time.  Without a process group, the value."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, local_seconds, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time.  Returns (value, max_seconds)."""
    tmax = max_over_ranks(local_seconds, dist, device)
    return world * units_per_rank / tmax, tmax


def oracle_step(al, xs):
    import oracle as O
    return O.tt_round(O.tt_add(list(al), xs), DELTA)


def cpu_baseline_sample(al, xs, budget_s=30.0):
    """The oracle (unchanged) on the host cores: whole rounding steps of the
    same workload until about budget_s seconds have elapsed (at least one)."""
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle_step(al, xs)
        n += 1
        el = time.perf_counter() - t0
        if el + el / n > budget_s:
            break
    return {"value": n / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d full rounding(s) of the workload (NumPy/LAPACK FP64, default BLAS threads)" % n}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from ttinputs import cfg_round_sum
    al, xs = cfg_round_sum(0)
    for _ in range(args.warmup):
        oracle_step(al, xs)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(al, xs)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = args.steps / tot
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "delta": DELTA, "implementation": "CPU FP64 oracle (NumPy/LAPACK)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "one full rounding of the workload per step"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    global SM_COUNT
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    SM_COUNT = torch.cuda.get_device_properties(local).multi_processor_count
    dist = None
    dev = "cuda:%d" % local
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2211_08770_gb300 import build as B
    B.build()
    from paper_2211_08770_gb300 import ttgb as T
    from ttinputs import cfg_round_sum

    peaks, peak_src = load_peaks()
    al, xs = cfg_round_sum(0)
    stream = torch.cuda.Stream(device=local)

    def time_path(precision, steps, warmup, profile):
        ctx = T.Ctx(local, precision, stream=stream.cuda_stream)
        X = [T.tt_tensor_create(ctx, c) for c in xs]
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda:%d" % local)

        def step():
            s = T.tt_add(ctx, al, X)
            y, err = T.tt_round(ctx, s, DELTA)
            r = y.ranks
            s.free()
            y.free()
            return r, err

        for _ in range(warmup):
            ranks, err = step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ctx.reset_stats()
        ctx.reset_profile()
        ctx.set_profiling(bool(profile), family=profile if isinstance(profile, str) else None)
        evs = []
        clocks = ClockSampler(local)
        clocks.start()
        wall0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(steps):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ranks, err = step()
                e1.record(stream)
                evs.append((e0, e1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        ck = clocks.stop()
        ms = [a.elapsed_time(b) for a, b in evs]
        stats = ctx.stats()
        prof = ctx.profile() if profile else {}
        ctx.set_profiling(False)
        tot_ms = 1e3 * job_throughput(world, steps, sum(ms) / 1e3, dist, dev)[1]
        for x in X:
            x.free()
        ctx.close()
        return dict(ms=ms, tot_ms=tot_ms, wall=wall, clocks=ck, stats=stats, prof=prof, ranks=ranks, err=err)

    def time_e2e(precision, steps):
        """The public API end to end from page-locked host memory: upload of
        the 20 input TTs (storage dtype), tt_add, and tt_round_to_host (the
        rounded cores copied into page-locked buffers as the sweep finishes
        them); every step."""
        ctx = T.Ctx(local, precision, stream=stream.cuda_stream)
        dt = torch.float64 if precision == "fp64" else torch.float32
        es = 8 if precision == "fp64" else 4
        hin = []
        for x in xs:
            cs = []
            for c in x:
                b = torch.empty(c.shape, dtype=dt, pin_memory=True)
                b.numpy()[...] = c
                cs.append(b.numpy())
            hin.append(cs)
        h2d = sum(c.size for x in xs for c in x) * es
        # output buffers sized by the concatenated ranks (rounding never grows them)
        rs = [1] + [sum(x[k].shape[2] for x in xs) for k in range(len(xs[0]) - 1)] + [1]
        hout = [torch.empty(rs[k] * xs[0][k].shape[1] * rs[k + 1], dtype=dt, pin_memory=True).numpy()
                for k in range(len(xs[0]))]
        times, d2h = [], 0
        for i in range(steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            X = [T.tt_tensor_create_storage(ctx, c) for c in hin]
            s = T.tt_add(ctx, al, X)
            y, _, cores = T.tt_round_to_host(ctx, s, DELTA, hout)
            t1 = time.perf_counter()
            d2h = sum(c.size for c in cores) * es
            for v in X + [s, y]:
                v.free()
            if i > 0:
                times.append(t1 - t0)
        ctx.close()
        value, _ = job_throughput(world, len(times), sum(times), dist, dev)
        return dict(value=value, unit=UNIT, h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h),
                    host_memory="page-locked, storage dtype (tt_tensor_create_storage / tt_round_to_host)")

    def accuracy(precision):
        """||x - round(x)|| / ||x|| of one rounding of the workload on the
        given path (outside the timed region), x being the exact FP64 sum of
        the FP64 inputs.  Measured with the FP64 GPU path (TT sum with -1 and
        the norm by right-to-left orthogonalization, no cancellation)."""
        ctx = T.Ctx(local, precision, stream=stream.cuda_stream)
        X = [T.tt_tensor_create(ctx, c) for c in xs]
        s = T.tt_add(ctx, al, X)
        y, est = T.tt_round(ctx, s, DELTA)
        cores = y.cores()
        st = ctx.stats()
        for v in X + [s, y]:
            v.free()
        ctx.close()
        c64 = T.Ctx(local, "fp64", stream=stream.cuda_stream)
        X64 = [T.tt_tensor_create(c64, c) for c in xs]
        x64 = T.tt_add(c64, al, X64)
        y64 = T.tt_tensor_create(c64, cores)
        diff = T.tt_add(c64, [1.0, -1.0], [x64, y64])
        err = T.tt_norm(c64, diff) / T.tt_norm(c64, x64)
        for v in X64 + [x64, y64, diff]:
            v.free()
        c64.close()
        return {"rel_error": err, "rel_error_over_delta": err / DELTA, "err_est": est,
                "bound": "delta + 1e-6 (FP32 storage)" if precision != "fp64" else "delta",
                "second_pass_skips": int(st["second_pass_skips"]), "series_passes": int(st["series_passes"]),
                "measured_by": "FP64 GPU path: ||x - x~|| from the TT sum x - x~ and its norm"}

    prec = args.precision
    # Every family's launches are timed on a short separate pass (two events
    # per launch cost host time, which shows in a step of ~300 launches); the
    # timed pass then times only the dominant family's launches, for the
    # roofline, in the timed region itself.
    allprof, dom = {}, None
    if not args.no_profile:
        allprof = time_path(prec, max(3, args.steps // 2), 1, profile=True)["prof"]
        dom = max(allprof, key=lambda k: allprof[k]["total_ms"]) if allprof else None
    main = time_path(prec, args.steps, args.warmup, profile=dom or False)
    value = world * args.steps / (main["tot_ms"] / 1e3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": main["tot_ms"] / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"mixed_tf32": "f32 storage, tf32 tensor-core Gram", "fp32": "f32", "fp64": "f64"}[prec],
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "delta": DELTA, "precision": prec, "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": "256 MB buffer written between timed steps (working set ~0.5 GB > 129 MB L2)",
                      "sweeps": "pipelined (three bonds in flight; tt_ctx_set_pipeline)",
                      "output_ranks": main["ranks"]},
           "gpu_launches": int(main["stats"]["kernel_launches"]),
           "host_syncs": int(main["stats"]["host_syncs"]),
           "path_stats": {k: int(main["stats"][k]) for k in ("svd_calls", "certified_bonds", "fallback_orth", "series_passes",
                                                                          "second_pass_skips")},
           "clocks": main["clocks"],
           "accuracy": accuracy(prec)}
    # roofline of the dominant kernel family
    prof = main["prof"]
    if prof and dom in prof:
        fam = dom
        bound, ach, peak, unit, how = roofline_for(fam, prof[fam], peaks, peak_src)
        traffic = None
        tp = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tp):
            with open(tp) as f:
                tj = json.load(f)
            ent = tj.get(fam)
            if ent and ent.get("workload") == WORKLOAD and ent.get("source_hash") == _src_hash(ent.get("source")):
                traffic = ent.get("bytes_per_launch")
        out["roofline"] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                           "traffic": traffic, "kernel": fam, "peak_source": how,
                           "launches": prof[fam]["launches"],
                           "avg_launch_ms": prof[fam]["total_ms"] / max(1, prof[fam]["launches"]),
                           "share_of_step": prof[fam]["total_ms"] / max(1e-9, sum(main["ms"]))}
        nprof = max(3, args.steps // 2)
        out["kernel_profile"] = {"steps": nprof, "note": "separate pass, every launch timed with CUDA events "
                                 "(includes host enqueue gaps of short launches)",
                                 "families": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 4)} for k, v in
                                              sorted(allprof.items(), key=lambda kv: -kv[1]["total_ms"])}}
    if prec != "fp64" and not args.no_fp64:
        f = time_path("fp64", args.fp64_steps, 1, profile=False)
        fv = world * args.fp64_steps / (f["tot_ms"] / 1e3)
        out["fp64_path"] = {"value": fv, "unit": UNIT, "ms_per_step": f["tot_ms"] / args.fp64_steps,
                            "steps": args.fp64_steps, "output_ranks": f["ranks"], "clocks": f["clocks"],
                            "accuracy": accuracy("fp64")}
        out["speedup_vs_fp64"] = value / fv
    out["e2e"] = time_e2e(prec, args.e2e_steps)

    def leg(key, f):
        # an optional leg that fails is reported in its key; the line still prints
        try:
            out[key] = f()
        except Exception as e:  # noqa: BLE001
            out[key] = {"error": "%s: %s" % (type(e).__name__, e)}

    if args.batch_count > 0:
        leg("batched", lambda: time_batched(T, local, prec, args.batch_count, not args.no_fp64))
    if args.orth_budget > 0:
        leg("orth", lambda: time_orth(T, local, args.orth_m, args.orth_budget))
    if args.paper_budget > 0:
        leg("paper_experiments", lambda: time_paper_experiments(T, local, args.paper_budget))
    if not args.no_variants:
        leg("variants", lambda: time_variants(T, local, al, xs, stream))
    if args.serve_count > 0:
        leg("serve", lambda: time_serve(T, local, prec, args.serve_count, args.serve_rate, args.serve_workers))
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline_sample(al, xs, budget_s=args.cpu_budget)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def time_batched(T, dev, prec, count, with_fp64):
    """Batched rounding of `count` uneven instances (orders 4-12, modes
    16-128, ranks 8-256, unit-scaled Gaussian cores, delta 1e-6): the lane
    count is tuned on a held-out draw of the same distribution (seed 1, a
    quarter of the count), then one timed pass over the seed-0 draw; the
    fixed-lane baseline (8 lanes, the library default) is timed too."""
    import torch
    from ttinputs import cfg_batched
    xs = cfg_batched(0, count=count)
    held = cfg_batched(1, count=max(16, count // 4))
    res = {"workload": "batched rounding, %d instances: d 4-12, n 16-128, r 8-256, delta 1e-6" % count,
           "unit": "roundings/s", "count": count, "tuned_on": "held-out draw (seed 1, %d instances)" % len(held)}

    def run(precision, lanes_list):
        ctx = T.Ctx(dev, precision)
        hs = [T.tt_tensor_create(ctx, x) for x in xs]
        hh = [T.tt_tensor_create(ctx, x) for x in held]
        torch.cuda.synchronize()
        rates = {}
        for lanes in lanes_list:
            ctx.concurrency = lanes
            ys = T.tt_round_batched(ctx, hh, [DELTA] * len(hh))  # warm
            for y in ys:
                y.free()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ys = T.tt_round_batched(ctx, hh, [DELTA] * len(hh))
            torch.cuda.synchronize()
            rates[lanes] = len(hh) / (time.perf_counter() - t0)
            for y in ys:
                y.free()
        for h in hh:
            h.free()
        best = max(rates, key=rates.get)
        ctx.concurrency = best
        ctx.reset_stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ys = T.tt_round_batched(ctx, hs, [DELTA] * count)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = ctx.stats()
        for y in ys + hs:
            y.free()
        ctx.close()
        return dict(value=count / dt, seconds=dt, lanes=best, tuning={str(k): round(v, 2) for k, v in rates.items()},
                    gpu_launches=int(st["kernel_launches"]), host_syncs=int(st["host_syncs"]),
                    peak_bytes=int(st["peak_bytes"]))

    m = run(prec, (4, 8, 16, 32))
    res.update(m)
    res["fixed_8_lanes_value"] = run(prec, (8,))["value"]
    if with_fp64:
        f = run("fp64", (m["lanes"],))
        res["fp64_value"] = f["value"]
        res["speedup_vs_fp64"] = m["value"] / f["value"]
    return res


def _gpu_loo(T, ctx, Q):
    """||I - Q^T Q||_2 per basis prefix from GPU TT dots (host eigenvalues)."""
    import numpy as np
    m = len(Q)
    G = np.zeros((m, m))
    for i in range(m):
        v = T.tt_dot_many(ctx, Q[i], Q[: i + 1])
        G[i, : i + 1] = v
        G[: i + 1, i] = v
    return [float(np.max(np.abs(np.linalg.eigvalsh(np.eye(k) - G[:k, :k])))) for k in range(1, m + 1)]


def time_orth(T, dev, m, budget_s):
    """The recursive ill-conditioned family (order 8, mode 32, rank-10 f_k,
    a_k = c a_{k-1} + (1 - c) f_k with c = 0.999, formed on the GPU by TT
    sums) orthogonalized by TT-MGS2 and TT-CGS2 (rounding after every update,
    delta = 1e-6), mixed and FP64, within a time budget: each arm runs on the
    first 10, 20, ... inputs (up to m) while the next run is predicted to fit
    (the cost grows like m^5: m^2 roundings of ranks ~10 m)."""
    import numpy as np
    import torch
    from ttinputs import cfg_orth_recursive
    t_start = time.perf_counter()
    F = cfg_orth_recursive(0, m=m)
    res = {"workload": "recursive family a_k = 0.999 a_(k-1) + 0.001 f_k, d=8, n=32, f_k rank 10 N(0,1); "
                       "round after every update, delta=1e-6", "runs": []}
    arms = [(p, s) for p in ("mixed_tf32", "fp64") for s in ("mgs2", "cgs2")]
    for ai, (prec, scheme) in enumerate(arms):
        ctx = T.Ctx(dev, prec)
        Fg = [T.tt_tensor_create(ctx, f) for f in F]
        A = [Fg[0]]
        for k in range(1, m):
            A.append(T.tt_add(ctx, [0.999, 0.001], [A[-1], Fg[k]]))
        sizes, last, prev = [], None, None
        for mm in [v for v in (10, 20, 30, 40, 50, 60, 80, 100) if v <= m]:
            left = budget_s - (time.perf_counter() - t_start)
            share = left / (len(arms) - ai)  # what this arm may still spend
            if prev and prev[1] * (mm / prev[0]) ** 5 > share:
                break
            ctx.reset_stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Q, R, nr = T.tt_orthogonalize(ctx, scheme, A[:mm], 1e-6, "every_update")
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            prev = (mm, dt)
            sizes.append({"m": mm, "seconds": round(dt, 3)})
            if last:
                for q in last[0]:
                    q.free()
            last = (Q, nr, dt, ctx.stats(), mm)
        if last:
            Q, nr, dt, st, mm = last
            loo = _gpu_loo(T, ctx, Q)
            c64 = T.Ctx(dev, "fp64")
            Ah = [T.tt_tensor_create(c64, a.cores()) for a in A[:mm]]
            G = np.array([T.tt_dot_many(c64, a, Ah) for a in Ah])
            ev = np.linalg.eigvalsh(0.5 * (G + G.T))
            c64.close()
            res["runs"].append({"precision": prec, "scheme": scheme, "m": mm, "seconds": dt, "roundings": nr,
                                "roundings_per_s": nr / dt, "loo": loo[-1],
                                "loo_curve_every_5": [float("%.3g" % v) for v in loo[4::5]],
                                "kappa": float(np.sqrt(max(ev[-1], 0) / max(ev[0], 1e-300))),
                                "max_rank": max(max(q.ranks) for q in Q), "svd_calls": int(st["svd_calls"]),
                                "fallback_orth": int(st["fallback_orth"]), "fallback_fp32": int(st["fallback_fp32"]),
                                "gpu_launches": int(st["kernel_launches"]),
                                "host_syncs": int(st["host_syncs"]), "sizes_timed": sizes})
            for q in Q:
                q.free()
        ctx.close()
    res["seconds_total"] = time.perf_counter() - t_start
    return res


def time_paper_experiments(T, dev, budget_s):
    """The paper's own inputs (Section 4): Krylov vectors of the ones tensor
    under the Dirichlet Laplacian TT-matrix, each rounded to TT-rank 1 and
    normalised, generated on the GPU; the six schemes at delta in {1e-3,
    1e-5, 1e-8}, FP64 and mixed, order 3 (n = 15, m = 20) and order 6
    (n = 15, m = 35, within the budget); the loss of orthogonality at the
    last basis size, its curve, and the largest TT-rank of the basis."""
    import torch
    t_start = time.perf_counter()
    out = {"inputs": "Krylov: x_1 = ones, a_j = normalised rank-1 TT-round of x_j, x_(j+1) = -Laplacian a_j", "runs": []}
    for d, n, m in ((3, 15, 20), (6, 15, 35)):
        for prec in ("fp64", "mixed_tf32"):
            ctx = T.Ctx(dev, prec)
            op = T.tt_operator_laplacian(ctx, d, n)
            ones = T.tt_tensor_create(ctx, [__import__("numpy").ones((1, n, 1)) for _ in range(d)])
            t0 = time.perf_counter()
            A = T.tt_krylov_basis(ctx, op, ones, m, 0.0, 1)
            torch.cuda.synchronize()
            t_gen = time.perf_counter() - t0
            for delta in (1e-3, 1e-5, 1e-8):
                for scheme in ("cgs", "mgs", "cgs2", "mgs2", "gram", "householder"):
                    if time.perf_counter() - t_start > budget_s:
                        out["truncated_by_budget"] = True
                        break
                    k = m
                    t0 = time.perf_counter()
                    while True:
                        try:
                            Q, R, nr = T.tt_orthogonalize(ctx, scheme, A[:k], delta)
                            break
                        except T.TTError as e:
                            if e.name != "TT_ERR_NOT_SPD" or k <= 1:
                                raise
                            k -= 1
                    dt = time.perf_counter() - t0
                    loo = _gpu_loo(T, ctx, Q)
                    out["runs"].append({"d": d, "n": n, "m": k, "precision": prec, "delta": delta, "scheme": scheme,
                                        "seconds": dt, "roundings": nr, "loo_last": loo[-1],
                                        "loo_curve": [float("%.3g" % v) for v in loo],
                                        "max_rank": max(max(q.ranks) for q in Q), "krylov_seconds": t_gen})
                    for q in Q:
                        q.free()
            ctx.close()
    out["seconds_total"] = time.perf_counter() - t_start
    return out


def time_variants(T, dev, al, xs, stream):
    """Rounding variants on the single-rounding workload: Gram-SVD rounding
    (FP64), randomized rounding with a Gaussian sketch of ranks 400 (mixed,
    exact at that rank), both against tt_round on the same input; and the
    TT matrix-vector product of the Dirichlet Laplacian (d = 10, n = 64)
    with the rank-400 sum (mixed), against the HBM roofline."""
    import numpy as np
    import torch
    from ttinputs import random_tt
    peaks, _ = load_peaks()
    out = {}
    d, n = len(xs[0]), xs[0][0].shape[1]

    def timed(f, reps):
        f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            y = f()
            torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps, y

    c64 = T.Ctx(dev, "fp64", stream=stream.cuda_stream)
    X64 = [T.tt_tensor_create(c64, c) for c in xs]
    x64 = T.tt_add(c64, al, X64)
    t_g, yg = timed(lambda: T.tt_round_gram_svd(c64, x64, DELTA)[0], 2)
    t_r, yr = timed(lambda: T.tt_round(c64, x64, DELTA)[0], 2)
    diff = T.tt_add(c64, [1.0, -1.0], [yg, yr])
    out["gram_svd_fp64"] = {"roundings_per_s": 1.0 / t_g, "tt_round_fp64_roundings_per_s": 1.0 / t_r,
                            "rel_diff_vs_tt_round": T.tt_norm(c64, diff) / T.tt_norm(c64, x64),
                            "output_ranks": yg.ranks}
    cm = T.Ctx(dev, "mixed_tf32", stream=stream.cuda_stream)
    Xm = [T.tt_tensor_create(cm, c) for c in xs]
    xm = T.tt_add(cm, al, Xm)
    # rank-100 approximations of the rank-400 sum: the randomized sketch
    # (ranks 100 + 10 oversampling) against the deterministic rounding capped
    # at rank 100 (the quasi-optimal TT-SVD truncation), on time and error
    target, over = 100, 10
    om = T.tt_tensor_create(cm, random_tt(np.random.default_rng(77), [n] * d,
                                          [1] + [target + over] * (d - 1) + [1]))
    t_rand, yrand = timed(lambda: T.tt_round_randomized(cm, xm, om), 3)
    t_cap, ycap = timed(lambda: T.tt_round_capped(cm, xm, 0.0, target)[0], 3)

    def rel_err(y):
        yd = T.tt_tensor_create(c64, y.cores())
        diff = T.tt_add(c64, [1.0, -1.0], [x64, yd])
        return T.tt_norm(c64, diff) / T.tt_norm(c64, x64)

    er, ec = rel_err(yrand), rel_err(ycap)
    out["randomized_mixed"] = {"target_rank": target, "sketch_ranks": target + over,
                               "roundings_per_s": 1.0 / t_rand, "capped_tt_round_roundings_per_s": 1.0 / t_cap,
                               "rel_error": er, "capped_rel_error": ec, "error_ratio": er / ec,
                               "output_ranks": yrand.ranks}
    op = T.tt_operator_laplacian(cm, d, n)
    cm.reset_profile()
    cm.set_profiling(True, family="matvec_f32")
    t_mv, ymv = timed(lambda: T.tt_matvec(cm, op, xm), 5)
    prof = cm.profile().get("matvec_f32")
    cm.set_profiling(False)
    if prof:
        gbs = prof["bytes"] / (prof["total_ms"] / 1e3) / 1e9
        out["matvec_mixed"] = {"operator": "Dirichlet Laplacian TT-matrix (ranks 2), d=10, n=64",
                               "input_ranks": xm.ranks, "output_ranks": ymv.ranks, "seconds": t_mv,
                               "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                            "frac": gbs / peaks["hbm_gbs"], "launches": prof["launches"],
                                            "avg_launch_ms": prof["total_ms"] / max(1, prof["launches"])}}
    c64.close()
    cm.close()
    return out


def time_serve(T, dev, prec, count, rate, workers, rates=(100, 300, 1000, 3000, 5000)):
    """Serving: roundings and CGS2/MGS2 outer iterations against resident
    orthonormal bases (orders 6-12, modes 32/64, ranks 10-60, basis size
    1-64, delta 1e-5/1e-7), mixed and FP64.  Per precision: the capacity
    (every request submitted at once, completed requests per second), then
    open-loop Poisson arrivals at each rate of the sweep up to twice the
    capacity (beyond it the queue grows without bound: reported as
    saturated), and at `rate` (0: 70% of the capacity) for the headline
    percentiles."""
    from paper_2211_08770_gb300.serve import poisson_load
    from ttinputs import cfg_serving
    bases, reqs = cfg_serving(0, count=count)
    out = {"workload": "rounding or CGS2/MGS2 step vs resident basis (50/50); d 6-12, n 32/64, r 10-60, "
                       "k 1-64, delta 1e-5/1e-7; %d requests per run" % count, "workers": workers}
    for p in (prec, "fp64"):
        ctx = T.Ctx(dev, p)
        srv = T.Server(ctx, workers=workers)
        bids = {}
        for key, B in bases.items():
            hs = [T.tt_tensor_create(ctx, q) for q in B]
            bids[key] = srv.add_basis(hs)
            for h in hs:
                h.free()
        # warm the lanes outside the measurement
        poisson_load(srv, ctx, reqs[: min(8, count)], rate=1e6, basis_ids=bids, seed=99)
        sat = poisson_load(srv, ctx, reqs, rate=1e9, basis_ids=bids, seed=2)
        cap = sat["throughput"] or 0.0
        res = {"capacity": cap, "capacity_p50_ms": sat["p50_ms"], "sweep": []}
        for r in rates:
            if r > 2.0 * cap:
                res["sweep"].append({"offered_rate": r, "saturated": True})
                continue
            o = poisson_load(srv, ctx, reqs, rate=float(r), basis_ids=bids, seed=3)
            res["sweep"].append({k: o[k] for k in ("offered_rate", "throughput", "p50_ms", "p99_ms", "completed")})
        offered = rate if rate > 0 else max(0.7 * cap, 1e-3)
        o = poisson_load(srv, ctx, reqs, rate=offered, basis_ids=bids, seed=1)
        st = srv.stats()
        res.update(offered_rate=offered, throughput=o["throughput"], p50_ms=o["p50_ms"], p99_ms=o["p99_ms"],
                   service_p50_ms=o["service_p50_ms"], queue_p99_ms=o["queue_p99_ms"],
                   footprint_peak=int(st["footprint_peak"]), gpu_launches=int(st["kernel_launches"]),
                   roundings=int(st["roundings"]), errors=len(o["errors"]) + len(sat["errors"]))
        srv.close()
        ctx.close()
        out[p] = res
    # the headline percentiles: the served precision at 70% of its capacity
    for k in ("capacity", "offered_rate", "throughput", "p50_ms", "p99_ms"):
        out[k] = out[prec][k]
    return out


def _src_hash(source=None):
    """sha1 (12 hex digits) of some files of the CUDA sources (a name or a
    list of names), or of all."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2211_08770_gb300", "csrc")
    names = sorted(os.listdir(csrc)) if source is None else ([source] if isinstance(source, str) else list(source))
    for fn in names:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_tf32", choices=["mixed_tf32", "fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=25.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-profile", action="store_true",
                    help="time without the per-launch CUDA events (no roofline / kernel profile)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--serve-count", type=int, default=64)
    ap.add_argument("--serve-rate", type=float, default=0.0)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--orth-m", type=int, default=50, help="inputs of the recursive-family orthogonalization")
    ap.add_argument("--orth-budget", type=float, default=90.0, help="seconds for the orthogonalization runs (0: skip)")
    ap.add_argument("--paper-budget", type=float, default=60.0, help="seconds for the paper's experiments (0: skip)")
    ap.add_argument("--no-variants", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
