#!/usr/bin/env python3
"""Throughput benchmark of the MDS hot path on GB300.

Default workload: divide-and-conquer MDS (Section 3.2) of n=100,000 points in
d=100 (5 dominant directions of variance 15, 95 of variance 1), parts of
800-1,200 own points plus c=20 shared connecting points, r=10, FP32 distance
arithmetic and FP64 eigen-solves; one step = one mds_divide_conquer call over
the whole set (norms, all parts' distance tiles and double centering, the
batched Lanczos eigen-solve, Procrustes alignment and the aligned scatter).
Metric: points embedded per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload dc|interp|interp_f32|image|image_dc|serve]

Every line also carries a short serving leg ("serve"): three resident BF16
models (l, r) = (500, 2), (1000, 5), (2000, 10) over d=100 Gaussian data,
Poisson arrivals of embed requests of 1-50,000 points (log-uniform) at a
fixed fraction of the measured capacity, continuous batching in the
library's server; p50/p99 latency from submit to results in host memory.

Under torchrun every rank runs its own independent problem of the same size
(weak scaling, no data-path collective); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "points embedded/sec at stated Procrustes error vs oracle"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal dense FP64 rate of a GB300 (the eigen-solver's arithmetic):
# 1.25 TFLOP/s = 152 SMs x 2 FP64 FMA/clk x 2 flop x ~2.06 GHz.
FP64_PEAK_TFLOPS = 1.25
# DRAM traffic per launch of the dominant kernel from an ncu capture, valid
# only while the kernel source is unchanged (sha256 of the .cu file).
NCU_TRAFFIC = {
    # ncu DRAM bytes (read + write) of one launch on a smaller case, per unit
    # of work, scaled to the full launch: per row of Y for the projection
    # kernels (profiles/k_gower_tck_image_fp8_n814255.md,
    # profiles/k_gower_tc_interp_bf16_n1000000.md), per byte of Q streamed for
    # the batched D&C eigen-solver (profiles/k_lanczos_dc_f32_n100000.md; the
    # landmark problems of the interpolation workloads are L2-resident and
    # the image-like D&C parts stream whole rows, so neither uses it)
    "k_gower_tck.cu": {"sha": "54d0c9db6af3e843", "per": "row", "bytes": 1688.6},
    "k_gower_tc.cu": {"sha": "a89affadd1612472", "per": "row", "bytes": 452.0},
    "k_lanczos.cu": {"sha": "2b3722bfea4ec539", "per": "streamed byte", "bytes": 0.8287, "workloads": ("dc",)},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["dc", "interp", "interp_f32", "image", "image_dc", "serve"], default="dc")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-parts", type=int, default=4, help="parts in the bounded oracle sample")
    ap.add_argument("--cluster", type=int, default=0,
                    help="CTAs per eigenproblem (default: the library's choice; for profiling)")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests per serving run (the serving leg of every line; per step for --workload serve)")
    ap.add_argument("--serve-load", type=float, default=0.8, help="offered load as a fraction of measured capacity")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg (for launch lists)")
    ap.add_argument("--full-matvec", action="store_true",
                    help="D&C eigen-solver: stream whole rows of Q instead of the symmetric ranges")
    ap.add_argument("--n", type=int, default=0,
                    help="points per GPU (default: the workload's full size; smaller sizes are for profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(seed, rank):
    """Each rank embeds its own independent workload of the same size."""
    return seed + 1000 * rank


def max_over_ranks(x, device=None):
    """Max of a per-rank float over the default process group (identity
    when there is none): the job is as slow as its slowest rank."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_per_rank, ms_per_step):
    """Points embedded by all ranks per second of the slowest rank's step."""
    return world * n_per_rank / (ms_per_step / 1e3)


def emit(obj):
    print(json.dumps(obj), flush=True)


def file_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# ---------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------- CPU oracle leg


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_dc_sample(Y, part, r, nparts):
    """Oracle divide-and-conquer on parts 0..nparts-1 (each aligned to part 0).
    Returns (rows, X rows, seconds, points)."""
    import oracle as O
    t0 = time.perf_counter()
    rows, xs = [], []
    for j in range(min(nparts, part.p)):
        rj, Xj, _ = O.divide_conquer_part(Y, part.anchors, part.ptr, part.own, j, r)
        rows.append(rj)
        xs.append(Xj)
    dt = time.perf_counter() - t0
    rows = np.concatenate(rows)
    return rows, np.vstack(xs), dt, len(rows)


def oracle_interp_sample(Y, idx, r, m):
    """Oracle interpolation MDS: landmark MDS + Eq. (2) for the first m
    non-landmark rows.  Returns (rows, X rows, seconds, points)."""
    import oracle as O
    t0 = time.perf_counter()
    L = Y[idx].astype(np.float64)
    D1 = O.sq_dist(L, L)
    X1, lam, _, _ = O.classical_mds(D1, r)
    is_lm = np.zeros(len(Y), dtype=bool)
    is_lm[idx] = True
    rest = np.nonzero(~is_lm)[0][:m]
    Xs = O.gower_interpolate(X1, lam, D1, O.sq_dist(Y[rest].astype(np.float64), L))
    dt = time.perf_counter() - t0
    return np.concatenate([idx, rest]), np.vstack([X1, Xs]), dt, len(rest) + len(idx)


# ---------------------------------------------------------------- workloads


WORKLOADS = {"dc": W.DC_F32, "interp": W.INTERP_BF16, "interp_f32": W.INTERP_F32, "image": W.IMAGE_FP8,
             "image_dc": W.IMAGE_DC}


def is_dc(name):
    return WORKLOADS[name].kind == "dc"


def oracle_sample(name, Y, aux, r, cpu_parts):
    """Bounded oracle sample of a workload: a few parts (D&C) or the landmark
    MDS plus a block of interpolated rows (interpolation)."""
    wide = Y.shape[1] > 200
    if is_dc(name):
        k = min(cpu_parts, 2) if wide else cpu_parts
        rows, Xo, dt, npts = oracle_dc_sample(Y, aux, r, k)
        return rows, Xo, dt, npts, f"parts 0..{k - 1} ({npts} points) of the same workload, each part's classical MDS + Procrustes to part 0"
    m = 2_000 if wide else 20_000
    rows, Xo, dt, npts = oracle_interp_sample(Y, aux, r, m)
    return rows, Xo, dt, npts, f"landmark MDS + Eq. (2) for {npts - len(aux)} rows of the same workload"


def make_workload(name, seed, n=0):
    import dataclasses
    base = WORKLOADS[name]
    w = base
    if n:
        w = dataclasses.replace(base, n=n, name=base.name.replace(f"n{base.n}", f"n{n}"))
    Y = W.make_data(base, seed, n=w.n)
    if name == "dc":
        return w, Y, W.partitions_uneven(w.n, w.c, w.own_lo, w.own_hi, seed)
    if name == "image_dc":
        return w, Y, W.partitions_equal(w.n, w.l, w.c, seed)
    return w, Y, W.landmarks(w.n, w.l, seed)


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w, Y, aux = make_workload(args.workload, args.seed, args.n)
    times, pts = [], 0
    for i in range(args.warmup + args.steps):
        _, _, dt, npts, sample = oracle_sample(args.workload, Y, aux, w.r, args.cpu_parts)
        if i >= args.warmup:
            times.append(dt)
            pts += npts
    value = pts / sum(times)
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic", "config": {"workload": w.name, "n": w.n, "d": w.d, "r": w.r},
          "cpu_baseline": {"value": value, "unit": "points/s", "cores": cpu_threads(), "kind": "oracle",
                           "sample": sample},
          "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# --------------------------------------------------------------- serving leg


def serve_leg(dev, seed, n_req, warm_req, load, slots):
    """Embed requests arriving as a Poisson process onto three resident
    models through the library's continuous-batching server.  Returns the
    served points/s over the timed requests, their p50/p99 latency, and the
    capacity the arrival rate was derived from."""
    import torch
    from paper_2007_11919_gb300 import mds as M

    w = W.SERVE_BF16
    base = torch.from_numpy(W.make_data(w, seed, n=max(l for l, _ in W.SERVE_MODELS) * 3)).to(dev)
    models = []
    for k, (l, r) in enumerate(W.SERVE_MODELS):
        idx = torch.from_numpy(W.landmarks(base.shape[0], l, seed + 11 * k)).to(dev)
        models.append(M.mds_interpolate(base, idx, r, "bf16", want_model=True)[2])
    total = warm_req + n_req
    _, sizes = W.serve_requests(total, *W.SERVE_SIZES, rate_per_s=1.0, seed=seed)
    which = np.random.default_rng(seed).integers(0, len(models), size=total)
    pool_rows = int(min(sizes.sum(), 400_000))
    pool = torch.from_numpy(W.make_data(w, seed + 1, n=pool_rows)).pin_memory()
    starts = np.random.default_rng(seed + 2).integers(0, pool_rows - sizes + 1)
    outs = torch.empty(int(sizes.sum()) * max(r for _, r in W.SERVE_MODELS), dtype=torch.float32).pin_memory()
    ooff = np.concatenate([[0], np.cumsum(sizes * np.array([W.SERVE_MODELS[k][1] for k in which]))])

    def req(i):
        r = W.SERVE_MODELS[which[i]][1]
        return (int(which[i]), pool[starts[i]:starts[i] + sizes[i]],
                outs[ooff[i]:ooff[i + 1]].view(int(sizes[i]), r))

    with M.Server(models, slots=slots) as srv:
        # capacity: every request of the warm-up set submitted at once
        t0 = time.perf_counter()
        tk = [srv.submit(*req(i)) for i in range(warm_req)]
        for t in tk:
            srv.wait(t)
        cap = float(sizes[:warm_req].sum()) / (time.perf_counter() - t0)
        # timed: Poisson arrivals at `load` x capacity
        rate = load * cap / float(sizes.mean())
        gaps = np.random.default_rng(seed + 3).exponential(1.0 / rate, size=n_req)
        due = np.cumsum(gaps)
        sub, tk = [], []
        t0 = time.perf_counter()
        for j in range(n_req):
            while time.perf_counter() - t0 < due[j]:
                pass
            sub.append(time.perf_counter() - t0)
            tk.append(srv.submit(*req(warm_req + j)))
        lat = np.array([srv.wait(t)[1] for t in tk])
        st = srv.stats()
    done = np.array(sub) + lat / 1e3
    pts = float(sizes[warm_req:].sum())
    tw = which[warm_req:]
    lr = np.array(W.SERVE_MODELS, dtype=np.float64)[tw]            # (l, r) per timed request
    flops = float(np.sum(sizes[warm_req:] * (2.0 * lr[:, 0] * w.d + 2.0 * lr[:, 0] * lr[:, 1])))
    d2h = int(np.sum(sizes[warm_req:] * lr[:, 1] * 4))
    for m in models:
        m.free()
    return {"points_per_s": pts / float(done.max()), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "load": load, "capacity_points_per_s": cap,
            "requests": n_req, "points": int(pts), "slots": slots, "batches": int(st["batches"]),
            "max_in_flight": int(st["max_in_flight"]), "wall_s": float(done.max()),
            "h2d_bytes": int(pts * w.d * 4), "d2h_bytes": d2h, "tensor_flops": flops,
            "batches_timed_and_warm": int(st["batches"]),
            "models": [f"l{l}_r{r}_bf16" for l, r in W.SERVE_MODELS],
            "timing": "host clock, submit to results in pinned host memory"}


# --------------------------------------------------------------- our arm


def ours(args):
    import torch
    import torch.distributed as tdist

    rank, world, local = dist_env()
    if world > 1:
        tdist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2007_11919_gb300 import build as gbuild
    gbuild.build()
    import paper_2007_11919_gb300 as G
    from paper_2007_11919_gb300 import mds as M

    seed = rank_seed(args.seed, rank)
    if args.workload == "serve":
        return serve_main(args, rank, world, dev)
    w, Y, aux = make_workload(args.workload, seed, args.n)
    Yd = torch.from_numpy(Y).to(dev)
    L = M._lib()
    if is_dc(args.workload):
        part = aux
        anc = torch.from_numpy(part.anchors).to(dev)
        own = torch.from_numpy(part.own).to(dev)
        # the whole divide-and-conquer call as one autotuned, graph-captured plan
        plan = M.DcPlan(w.n, w.d, Yd.dtype, part.ptr, w.c, w.r, w.prec, tune=args.cluster == 0,
                        cluster=args.cluster, device=dev, full_matvec=args.full_matvec)
        Xbuf = torch.zeros((w.n, w.r), dtype=torch.float64 if w.prec == "f64" else torch.float32, device=dev)
        vbuf = torch.empty(w.r, dtype=torch.float64, device=dev)

        def step(Yin=Yd, a=anc, o=own):
            return plan.execute(Yin, a, o, X=Xbuf, var=vbuf)
    else:
        idx = torch.from_numpy(aux).to(dev)
        wsb = L.mds_interpolate_workspace_size(w.n, w.d, w.l, w.r, M.PREC[w.prec])
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)

        def step(Yin=Yd, a=idx, o=None):
            X, var, _ = G.mds_interpolate(Yin, a, w.r, w.prec, workspace=ws, cluster=args.cluster)
            return X, var

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    M.mds_set_timing(True)
    for _ in range(args.warmup):
        X, var = step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps, CUDA events per step
    clocks = ClockSampler(local)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    stream = torch.cuda.current_stream(dev)
    step_ms, stats = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        X, var = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats.append(M.mds_last_stats())
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    clk = clocks.stop()
    ms_per_step = max_over_ranks(sum(step_ms), dev) / args.steps
    value = job_throughput(world, w.n, ms_per_step)

    # ---- roofline of the dominant kernel: the Lanczos eigensolve (stage "eig")
    # or, for interpolation, the fused distance + projection kernel (stage
    # "post"), whichever takes longer per step; the other is reported beside it
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    eig_ms = statistics.mean(s["stage_ms"]["eig"] for s in stats)

    def lanczos_roof():
        # Algorithmic bytes: all n^2 entries of Q (4 bytes each in FP32
        # storage) once per Lanczos step, summed over the parts' steps.
        flops = statistics.mean(s["eig_flops"] for s in stats)
        qbytes = statistics.mean(s["eig_qbytes"] for s in stats)
        qread = statistics.mean(s["eig_qread"] for s in stats)
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = qbytes / (eig_ms * 1e-3) / 1e9
        kind = "batched Lanczos, one cluster per part" if is_dc(args.workload) else \
            "Lanczos of the landmark problem, one team of clusters; Q is L2-resident, the steps are latency-bound"
        roof = {"kernel": f"k_lanczos ({kind})", "bound": "hbm",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "launch_ms": eig_ms, "bytes_per_launch": qbytes,
                # what the kernel streams: the symmetric ranges read each
                # off-diagonal block of Q once for both triangles
                "streamed_bytes_per_launch": qread, "streamed_gbs": qread / (eig_ms * 1e-3) / 1e9,
                "fp64_equiv_flops_per_launch": flops,
                "fp64_equiv_tflops": flops / (eig_ms * 1e-3) / 1e12, "traffic": None}
        src = os.path.join(ROOT, "paper_2007_11919_gb300", "csrc", "k_lanczos.cu")
        tr = NCU_TRAFFIC["k_lanczos.cu"]
        if tr["sha"] == file_sha(src) and args.workload in tr["workloads"]:
            roof["traffic"] = tr["bytes"] * qread
        return roof

    def projection_roof():
        kms = statistics.mean(s["stage_ms"]["post"] for s in stats)
        flops = w.n * (2.0 * w.l * w.d + 2.0 * w.l * w.r)
        pk = peaks.get("bf16_tflops", 1900.0)
        src_note = "MEASURED_PEAKS.json bf16_tflops (burst, of measured)" if peaks else "fallback 1.9 PFLOP/s"
        if w.prec == "fp8":
            # FP8 dense rate = measured BF16 x the nominal 4.5 / 2.25 ratio
            pk *= 2.0
            src_note += " x 2 (nominal FP8 / BF16 ratio)"
        byte_rows = Y.dtype == np.uint8
        if w.prec in ("f32", "f64"):
            # SIMT distance tiles and projection on the FP32 pipe: peak from the
            # unit counts, 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
            pk = 152 * 128 * 2 * 2.07e9 / 1e12
            achieved = flops / (kms * 1e-3) / 1e12
            return {"kernel": "k_gower (SIMT distance tiles fused with the Gower projection)", "bound": "alu",
                    "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                    "peak_source": "derived: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2.07 GHz", "launch_ms": kms,
                    "flops_per_launch": flops, "traffic": None}
        kname = ("k_gower_tck (tcgen05 distance tiles of byte rows, K streamed, fused with the Gower projection)"
                 if byte_rows else "k_gower_tc (tcgen05 distance tiles and Gower projection, A^2 kept in TMEM)")
        achieved = flops / (kms * 1e-3) / 1e12
        roof = {"kernel": kname, "bound": "tensor",
                "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                "peak_source": src_note, "launch_ms": kms, "flops_per_launch": flops}
        src = os.path.join(ROOT, "paper_2007_11919_gb300", "csrc", "k_gower_tck.cu" if byte_rows else "k_gower_tc.cu")
        tr = NCU_TRAFFIC.get(os.path.basename(src))
        roof["traffic"] = tr["bytes"] * w.n if tr and tr["sha"] == file_sha(src) else None
        return roof

    roof_other = None
    if is_dc(args.workload):
        roof = lanczos_roof()
    else:
        post_ms = statistics.mean(s["stage_ms"]["post"] for s in stats)
        roof, roof_other = lanczos_roof(), projection_roof()
        if post_ms > eig_ms:
            roof, roof_other = roof_other, roof

    # ---- end to end through the public API: pinned host input, host output
    Yh = torch.from_numpy(Y).pin_memory()
    if is_dc(args.workload):
        anc_h = torch.from_numpy(part.anchors).pin_memory()
        own_h = torch.from_numpy(part.own).pin_memory()
        h2d = Yh.numel() * Yh.element_size() + anc_h.numel() * 8 + own_h.numel() * 8
    else:
        anc_h = torch.from_numpy(aux).pin_memory()
        own_h = None
        h2d = Yh.numel() * Yh.element_size() + anc_h.numel() * 8
    # the step's own device buffers receive the host copies (a plan keeps its
    # captured graph for the same buffers)
    Ybuf = Yd
    abuf = anc if is_dc(args.workload) else idx
    obuf = own if is_dc(args.workload) else None
    e2e_ms = []
    d2h = w.n * w.r * 4 + w.r * 8
    if not is_dc(args.workload):
        # interpolation takes host rows directly: the library overlaps their
        # transfer with the landmark eigenproblem and the projection
        idx_h = torch.from_numpy(aux)
        hws = torch.empty(L.mds_interpolate_host_workspace_size(w.n, w.d, w.l, w.r, M.PREC[w.prec],
                                                                M.DTYPE[Yh.dtype]), dtype=torch.uint8, device=dev)
        Xout = torch.empty((w.n, w.r), dtype=torch.float32, pin_memory=True)
        # untimed warm-up of the host path (its streams, pinned buffers and launches)
        for _ in range(max(1, args.warmup)):
            G.mds_interpolate_host(Yh, idx_h, w.r, w.prec, out=Xout, workspace=hws, cluster=args.cluster)
        torch.cuda.synchronize()
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if is_dc(args.workload):
            Ybuf.copy_(Yh, non_blocking=True)
            abuf.copy_(anc_h, non_blocking=True)
            obuf.copy_(own_h, non_blocking=True)
            X, var = step(Ybuf, abuf, obuf)
            Xh = X.cpu()
            _ = var.cpu()
        else:
            Xh, var, _ = G.mds_interpolate_host(Yh, idx_h, w.r, w.prec, out=Xout, workspace=hws,
                                                cluster=args.cluster)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = job_throughput(world, w.n, max_over_ranks(statistics.mean(e2e_ms), dev))

    # ---- CPU oracle leg (rank 0, N = 1 only) and the error against it
    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        rows, Xo, dt, npts, sample = oracle_sample(args.workload, Y, aux, w.r, args.cpu_parts)
        err = O.aligned_rel_error(Xh.double().numpy()[rows], Xo)
        cpu = {"value": npts / dt, "unit": "points/s", "cores": cpu_threads(), "kind": "oracle", "sample": sample}

    serve = (serve_leg(dev, seed, args.serve_requests, 50, args.serve_load, args.serve_slots)
             if rank == 0 and not args.no_serve else None)

    if rank == 0:
        peaks_note = None
        emit({"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": w.prec, "data": "synthetic",
              "config": {"workload": w.name, "n_per_gpu": w.n, "d": w.d, "r": w.r,
                         "parts": (part.p if is_dc(args.workload) else None),
                         "c": (w.c if is_dc(args.workload) else None),
                         "l": (w.l if not is_dc(args.workload) else None),
                         "eigensolve": "Lanczos (FP64 scalars, double-FP32 working vectors, FP32 basis)",
                         "matvec": ("whole rows of Q" if args.full_matvec or w.prec == "f64" or not is_dc(args.workload)
                                    else "symmetric ranges of Q where every CTA's range is at most 1,024 columns"
                                         " (cluster of 3+ CTAs), else whole rows"),
                         "cluster": stats[-1]["cluster"],
                         "plan": (dict(plan.info(), graph=True, autotuned=args.cluster == 0)
                                  if is_dc(args.workload) else None),
                         "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas{world}"},
              "procrustes_rel_err_vs_oracle": err,
              "stage_ms": {k: statistics.mean(s["stage_ms"][k] for s in stats) for k in stats[0]["stage_ms"]},
              "eig_steps_per_call": stats[-1]["eig_steps"],
              "roofline": roof, "roofline_other_kernel": roof_other, "cpu_baseline": cpu,
              "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_steps": [round(t, 3) for t in e2e_ms]},
              "gpu_launches": int(sum(s["launches"] for s in stats)),
              "clocks": clk, "gpu": torch.cuda.get_device_name(dev), "note": peaks_note, "serve": serve})
    if world > 1:
        tdist.destroy_process_group()


def serve_main(args, rank, world, dev):
    """--workload serve: the serving run is the measurement; one step is a
    window of --serve-requests arrivals."""
    import torch
    import torch.distributed as tdist

    seed = rank_seed(args.seed, rank)
    clocks = ClockSampler(dev.index)
    if world > 1:
        tdist.barrier()
    clocks.start()
    res = serve_leg(dev, seed, args.steps * args.serve_requests, max(args.warmup, 1) * 50, args.serve_load,
                    args.serve_slots)
    clk = clocks.stop()
    wall = max_over_ranks(res["wall_s"], dev)
    pts = -max_over_ranks(-res["points"], dev) if world > 1 else res["points"]
    value = world * pts / wall
    w = W.SERVE_BF16
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        base = W.make_data(w, seed, n=6000)
        l, r = W.SERVE_MODELS[-1]
        idx = W.landmarks(len(base), l, seed + 22)
        t0 = time.perf_counter()
        _, _, ex = O.interpolation_mds(base[idx], np.arange(l), r)
        ex["L"] = base[idx].astype(np.float64)
        Ynew = W.make_data(w, seed + 5, n=10_000)
        O.embed_new(ex, Ynew)
        dt = time.perf_counter() - t0
        cpu = {"value": 10_000 / dt, "unit": "points/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"landmark MDS (l={l}, r={r}) + Eq. (2) for 10,000 new points"}
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    pk = peaks.get("bf16_tflops", 1900.0)
    achieved = res["tensor_flops"] / res["wall_s"] / 1e12
    roof = {"kernel": "k_gower_tc (served batches)", "bound": "tensor", "achieved": achieved, "peak": pk,
            "unit": "TFLOP/s", "frac": achieved / pk,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured)" if peaks else "fallback 1.9 PFLOP/s",
            "traffic": None,
            "note": "algorithmic flops of the served points over the serving wall time at the offered load "
                    "(idle gaps and copies included), a lower bound on the kernel's own rate"}
    if rank == 0:
        emit({"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
              "config": {"workload": w.name, "d": w.d, "models": res["models"],
                         "request_sizes": "log-uniform 1-50,000", "arrivals": "Poisson",
                         "load": args.serve_load, "slots": args.serve_slots,
                         "l2": "not flushed: requests stream from host memory", "parallelism": f"replicas{world}"},
              "serve": res, "roofline": roof, "cpu_baseline": cpu,
              "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": res["h2d_bytes"] // args.steps,
                      "d2h_bytes_per_step": res["d2h_bytes"] // args.steps},
              "gpu_launches": 2 * res["batches"], "clocks": clk, "gpu": torch.cuda.get_device_name(dev)})


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
