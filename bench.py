#!/usr/bin/env python3
"""Throughput benchmark of the MDS hot path on GB300.

Default workload (``image_all``): the image-like set, n = 814,255 rows of
d = 784 byte pixels (80% zeros, the rest round(clip(N(180, 60), 1, 255))),
embedded by BOTH of the paper's big-data methods in every step:
  * interpolation MDS (Section 3.1): l = 2,000 random landmarks, r = 10, the
    n x l landmark distances on tcgen05 in FP8 E4M3 (exact nibble planes of
    the bytes) fused with Gower's projection, Eq. (2); the landmark
    eigenproblem in FP64;
  * divide-and-conquer MDS (Section 3.2): parts of 2,000 points (c = 50
    connecting points + 1,950 own), r = 10, every part's Gram on tcgen05 in
    FP8, Q stored in FP32, all parts' Lanczos eigen-solves in one persistent
    launch, Procrustes alignment; the whole call replayed as an autotuned
    CUDA graph.
One step = one call of each method over all n rows (device-resident inputs);
value = n / step time (points embedded per second by the two methods in
turn).  The same line carries, under "configs", the other workloads, each
timed alone on its own inputs: interpolation FP64 (n = 2,000), divide-and-
conquer FP32 (n = 100,000), interpolation BF16 (n = 1,000,000), the plain
FP32 form of the same interpolation, and its affine pass, MaxMin landmark
selection at n = 1,000,000 and l = 1,000, pivot MDS and fast MDS; and under "serve"
the serving run (three resident BF16 models, Poisson arrivals of 1-50,000
point requests, continuous batching, p50/p99 latency).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload image_all|image|image_dc|dc|interp|interp_f32|affine|interp_f64|maxmin|pivot|fast|serve]

Under torchrun every rank runs its own independent problem of the same size
(weak scaling, no data-path collective); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import dataclasses
import hashlib
import json
import os
import platform
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
# DRAM traffic per launch of a kernel from an ncu capture, valid only while
# the kernel source is unchanged (sha256 prefix of the .cu file): ncu DRAM
# bytes (read + write) of one launch on a smaller case, per unit of work,
# scaled to the full launch -- per row of Y for the projection kernels
# (profiles/k_gower_tck_image_fp8_n814255.md,
# profiles/k_gower_tc_interp_bf16_n1000000.md), per byte of Q streamed for the
# batched divide-and-conquer eigen-solver (profiles/k_lanczos_dc_f32_n100000.md).
# The landmark problems of the interpolation workloads are L2-resident.
NCU_TRAFFIC = {
    "k_gower_tck.cu": {"sha": "54d0c9db6af3e843", "per": "row", "bytes": 1688.6},
    "k_gower_tc.cu": {"sha": "a89affadd1612472", "per": "row", "bytes": 452.0},
    # per byte of Q streamed, per workload
    # (profiles/k_lanczos_image_dc_fp8_n814255.md, profiles/k_lanczos_dc_f32_n100000.md)
    "k_lanczos.cu": {"sha": "8a15a9c67c457db5", "per": "streamed byte", "bytes": {"image_dc": 1.0325, "dc": 0.8305}},
    # per row of Y per round (profiles/k_maxmin_tiles_maxmin_f32_n1000000.md)
    "k_maxmin.cu": {"sha": "ea7609f60cd2d721", "per": "row per round", "bytes": 411.5},
    # per row of Y (profiles/k_affine_project_bulk_affine_f32_n1000000.md)
    "k_affine.cu": {"sha": "f592f8bbd752a734", "per": "row", "bytes": 432.2},
}

# name -> (workload, method)
LEGS = {
    "image": (W.IMAGE_FP8, "interp"),
    "image_dc": (W.IMAGE_DC, "dc"),
    "dc": (W.DC_F32, "dc"),
    "interp": (W.INTERP_BF16, "interp"),
    "interp_f32": (W.INTERP_F32, "interp"),
    "affine": (W.INTERP_AFFINE_F32, "affine"),
    "interp_f64": (W.CLASSICAL_INTERP_F64, "interp"),
    "maxmin": (W.MAXMIN_F32, "maxmin"),
    "pivot": (W.PIVOT_F32, "pivot"),
    "fast": (W.FAST_F32, "fast"),
}
HEADLINE = ("image", "image_dc")          # the image-like set, both methods
SUB_CONFIGS = ("interp_f64", "dc", "interp", "interp_f32", "affine", "maxmin", "pivot", "fast")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["image_all", "serve", *LEGS], default="image_all")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="image_all: skip the other workloads")
    ap.add_argument("--config-steps", type=int, default=5, help="timed steps of each workload under 'configs'")
    ap.add_argument("--cluster", type=int, default=0,
                    help="CTAs per eigenproblem (default: the library's choice; for profiling)")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests per serving run (the serving leg of every line; per step for --workload serve)")
    ap.add_argument("--serve-load", type=float, default=0.8, help="offered load as a fraction of measured capacity")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg (for launch lists)")
    ap.add_argument("--eig-tol", type=float, default=0.0,
                    help="D&C eigen-solver residual tolerance (relative to lambda_1); 0 = the library default")
    ap.add_argument("--full-matvec", action="store_true",
                    help="divide-and-conquer eigen-solver: stream whole rows of Q instead of the symmetric ranges")
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


def load_peaks():
    return json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}


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
            return
        # nvidia-smi's start-up (NVML initialisation) can hold up this
        # process's CUDA calls for up to a second: the timed region starts
        # only once its first sample is written
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

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


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{platform.machine()} {platform.processor()}".strip()


def oracle_job(method, payload):
    """One bounded oracle sample; returns (X of the sampled rows, seconds).

    interp:  landmark MDS (Section 2) + Eq. (2) for a block of rows.
    affine:  the affine form of Eq. (2) for the landmarks and a block of rows.
    dc:      classical MDS of the listed parts (the first one solved once),
             each aligned to the first by Procrustes (Section 3.2)."""
    import oracle as O
    t0 = time.perf_counter()
    if method == "interp":
        L = payload["L"].astype(np.float64)
        D1 = O.sq_dist(L, L)
        X1, lam, _, _ = O.classical_mds(D1, payload["r"])
        Xs = O.gower_interpolate(X1, lam, D1, O.sq_dist(payload["rows"].astype(np.float64), L))
        X = np.vstack([X1, Xs])
    elif method == "affine":
        X, _, _ = O.affine_interpolation(payload["Y"], np.arange(payload["l"]), payload["r"])
    else:
        got = O.divide_conquer_parts(payload["Y"], payload["anchors"], payload["ptr"], payload["own"],
                                     list(range(len(payload["ptr"]) - 1)), payload["r"])
        X = np.vstack([g[1] for g in got])
    return X, time.perf_counter() - t0


def oracle_payload(method, Y, aux, r, n_rows):
    """The sampled rows of a workload, re-indexed locally, for oracle_job:
    returns (global row indices in the order of oracle_job's X, payload,
    description)."""
    if method == "dc":
        part = aux
        k = min(n_rows, part.p)
        own = part.own[:part.ptr[k]]
        rows = np.concatenate([part.anchors, own])
        c = part.c
        payload = {"Y": Y[rows], "anchors": np.arange(c), "ptr": part.ptr[:k + 1].copy(),
                   "own": np.arange(c, c + len(own)), "r": r}
        return rows, payload, (f"parts 0..{k - 1} ({len(rows)} points) of the same workload: each part's "
                               "classical MDS once, Procrustes of parts 1.. to part 0")
    idx = aux
    is_lm = np.zeros(len(Y), dtype=bool)
    is_lm[idx] = True
    rest = np.nonzero(~is_lm)[0][:n_rows]
    rows = np.concatenate([idx, rest])
    if method == "affine":
        return rows, {"Y": Y[rows], "l": len(idx), "r": r}, \
            f"landmark MDS + the affine form of Eq. (2) for the {len(idx)} landmarks and {len(rest)} rows"
    return rows, {"L": Y[idx], "rows": Y[rest], "r": r}, \
        f"landmark MDS (l={len(idx)}) + Eq. (2) for {len(rest)} rows of the same workload"


def oracle_seconds_one_thread(method, payload):
    """The same oracle sample in a fresh spawned process whose BLAS runs on
    one thread (the thread count is fixed when numpy loads)."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(1) as pool:
            return pool.apply(oracle_job, (method, payload))[1]
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


# Sample sizes (rows or parts) of the bounded oracle samples, per workload:
# about 5-25 s of CPU work each on the machine's host.
SAMPLE = {"image": 1000, "image_dc": 2, "dc": 4, "interp": 20_000, "interp_f32": 20_000, "affine": 20_000,
          "interp_f64": 1700}


def make_workload(name, seed, n=0):
    w, method = LEGS[name]
    if n:
        w = dataclasses.replace(w, n=n, name=w.name.replace(f"n{w.n}", f"n{n}"))
    Y = W.make_data(LEGS[name][0], seed, n=w.n)
    if method == "dc":
        if w.own_lo:
            return w, method, Y, W.partitions_uneven(w.n, w.c, w.own_lo, w.own_hi, seed)
        return w, method, Y, W.partitions_equal(w.n, w.l, w.c, seed)
    if method == "maxmin":
        return w, method, Y, None
    if method == "fast":
        return w, method, Y, W.fast_mds_tree(w.n, w.l, w.c, seed)
    return w, method, Y, W.landmarks(w.n, w.l, seed)


def reference_arm(args):
    """The oracle, as it stands, on the host cores: each step one bounded
    sample of the workload (for image_all the two methods in turn)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    names = HEADLINE if args.workload == "image_all" else (args.workload,)
    if args.workload == "serve":
        names = ("interp",)
    legs = []
    for nm in names:
        w, method, Y, aux = make_workload(nm, args.seed, args.n)
        k = 1 if method == "dc" and w.d > 200 else (120 if w.d > 200 else SAMPLE[nm])
        rows, payload, desc = oracle_payload(method, Y, aux, w.r, k)
        legs.append((nm, w, method, payload, len(rows), desc))
    times, pts = [], 0
    for i in range(args.warmup + args.steps):
        nm, w, method, payload, npts, _ = legs[i % len(legs)]
        _, dt = oracle_job(method, payload)
        if i >= args.warmup:
            times.append(dt)
            pts += npts
    value = pts / sum(times)
    wname = (f"image_all_fp8_n{legs[0][1].n}_d784_l2000_parts2000_c50_r10" if args.workload == "image_all"
             else legs[0][1].name)
    sample = "; ".join(f"{nm}: {desc}" for nm, _, _, _, _, desc in legs) + \
        (" (steps alternate between the methods)" if len(legs) > 1 else "")
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic", "config": {"workload": wname, "n": legs[0][1].n, "d": legs[0][1].d,
                                          "r": legs[0][1].r},
          "cpu_baseline": {"value": value, "unit": "points/s", "cores": cpu_threads(), "kind": "oracle",
                           "sample": sample, "cpu_model": cpu_model()},
          "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# --------------------------------------------------------------- serving leg


def serve_leg(dev, seed, n_req, warm_req, cap_req, load, slots):
    """Embed requests arriving as a Poisson process onto three resident
    models through the library's continuous-batching server.  Returns the
    served points/s over the timed requests, their p50/p99 latency, and the
    capacity the arrival rate was derived from (cap_req requests submitted
    at once, after warm_req untimed ones)."""
    import torch
    from paper_2007_11919_gb300 import mds as M

    w = W.SERVE_BF16
    base = torch.from_numpy(W.make_data(w, seed, n=max(l for l, _ in W.SERVE_MODELS) * 3)).to(dev)
    models = []
    for k, (l, r) in enumerate(W.SERVE_MODELS):
        idx = torch.from_numpy(W.landmarks(base.shape[0], l, seed + 11 * k)).to(dev)
        models.append(M.mds_interpolate(base, idx, r, "bf16", want_model=True)[2])
    total = warm_req + cap_req + n_req
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
        for t in [srv.submit(*req(i)) for i in range(warm_req)]:      # streams, pinned paths warmed up
            srv.wait(t)
        # capacity: cap_req requests submitted at once
        t0 = time.perf_counter()
        tk = [srv.submit(*req(warm_req + i)) for i in range(cap_req)]
        for t in tk:
            srv.wait(t)
        cap = float(sizes[warm_req:warm_req + cap_req].sum()) / (time.perf_counter() - t0)
        # timed: Poisson arrivals at `load` x capacity
        first = warm_req + cap_req
        rate = load * cap / float(sizes.mean())
        gaps = np.random.default_rng(seed + 3).exponential(1.0 / rate, size=n_req)
        due = np.cumsum(gaps)
        sub, tk = [], []
        t0 = time.perf_counter()
        for j in range(n_req):
            while time.perf_counter() - t0 < due[j]:
                pass
            sub.append(time.perf_counter() - t0)
            tk.append(srv.submit(*req(first + j)))
        lat = np.array([srv.wait(t)[1] for t in tk])
        st = srv.stats()
    done = np.array(sub) + lat / 1e3
    pts = float(sizes[first:].sum())
    tw = which[first:]
    lr = np.array(W.SERVE_MODELS, dtype=np.float64)[tw]            # (l, r) per timed request
    flops = float(np.sum(sizes[first:] * (2.0 * lr[:, 0] * w.d + 2.0 * lr[:, 0] * lr[:, 1])))
    d2h = int(np.sum(sizes[first:] * lr[:, 1] * 4))
    for m in models:
        m.free()
    return {"points_per_s": pts / float(done.max()), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "load": load, "capacity_points_per_s": cap,
            "capacity_requests": cap_req, "requests": n_req, "points": int(pts), "slots": slots,
            "batches": int(st["batches"]), "max_in_flight": int(st["max_in_flight"]), "wall_s": float(done.max()),
            "h2d_bytes": int(pts * w.d * 4), "d2h_bytes": d2h, "tensor_flops": flops,
            "models": [f"l{l}_r{r}_bf16" for l, r in W.SERVE_MODELS],
            "timing": "host clock, submit to results in pinned host memory"}


# --------------------------------------------------------------- our arm


class Leg:
    """One workload: its inputs on the device, the device call a step runs,
    the host-buffer call of the end-to-end measurement, and the roofline of
    its dominant kernel."""

    def __init__(self, name, dev, seed, args, n=0):
        import torch
        from paper_2007_11919_gb300 import mds as M
        self.name, self.args, self.dev = name, args, dev
        self.w, self.method, self.Y, self.aux = make_workload(name, seed, n)
        w = self.w
        self.Yd = torch.from_numpy(self.Y).to(dev)
        self.xdt = torch.float64 if w.prec == "f64" else torch.float32
        L = M._lib()
        if self.method == "dc":
            part = self.aux
            self.anc = torch.from_numpy(part.anchors).to(dev)
            self.own = torch.from_numpy(part.own).to(dev)
            # the whole divide-and-conquer call as one autotuned, graph-captured plan
            self.plan = M.DcPlan(w.n, w.d, self.Yd.dtype, part.ptr, w.c, w.r, w.prec, tune=args.cluster == 0,
                                 cluster=args.cluster, device=dev, full_matvec=args.full_matvec,
                                 eig_tol=args.eig_tol)
            self.X = torch.zeros((w.n, w.r), dtype=self.xdt, device=dev)
            self.var = torch.empty(w.r, dtype=torch.float64, device=dev)
        elif self.method == "maxmin":
            self.ws = torch.empty(L.mds_landmarks_maxmin_workspace_size(w.n, w.d), dtype=torch.uint8, device=dev)
        elif self.method == "fast":
            perm, self.rng, self.par = W.flatten_fast_tree(self.aux)
            self.perm = torch.from_numpy(perm).to(dev)
            rng = np.ascontiguousarray(self.rng.reshape(-1))
            self.ws = torch.empty(L.mds_fast_workspace_size(w.n, w.d, len(self.par), rng.ctypes.data_as(ctypes.c_void_p),
                                                            self.par.ctypes.data_as(ctypes.c_void_p), w.c, w.r,
                                                            M.PREC[w.prec]), dtype=torch.uint8, device=dev)
        else:
            self.idx = torch.from_numpy(self.aux).to(dev)
            size = {"affine": L.mds_interpolate_affine_workspace_size, "pivot": L.mds_pivot_workspace_size}.get(
                self.method, L.mds_interpolate_workspace_size)
            self.ws = torch.empty(size(w.n, w.d, w.l, w.r, M.PREC[w.prec]), dtype=torch.uint8, device=dev)

    def step(self):
        import paper_2007_11919_gb300 as G
        w = self.w
        if self.method == "dc":
            return self.plan.execute(self.Yd, self.anc, self.own, X=self.X, var=self.var)
        if self.method == "affine":
            return G.mds_interpolate_affine(self.Yd, self.idx, w.r, w.prec, workspace=self.ws)
        if self.method == "maxmin":
            return G.mds_landmarks_maxmin(self.Yd, w.l, 0, workspace=self.ws), None
        if self.method == "pivot":
            return G.mds_pivot(self.Yd, self.idx, w.r, w.prec, workspace=self.ws)
        if self.method == "fast":
            return G.mds_fast(self.Yd, self.perm, self.rng, self.par, w.c, w.r, w.prec, workspace=self.ws,
                              cluster=self.args.cluster)
        X, var, _ = G.mds_interpolate(self.Yd, self.idx, w.r, w.prec, workspace=self.ws, cluster=self.args.cluster)
        return X, var

    # ---- end to end: the library's host-buffer calls (or copies + device call)
    def host_setup(self):
        import torch
        from paper_2007_11919_gb300 import mds as M
        w = self.w
        self.Yh = torch.from_numpy(self.Y).pin_memory()
        self.h2d = self.Yh.numel() * self.Yh.element_size()
        self.d2h = w.n * w.r * (8 if w.prec == "f64" else 4) + w.r * 8
        self.Xh = torch.empty((w.n, w.r), dtype=self.xdt, pin_memory=True)
        if self.method == "dc":
            self.anc_h = torch.from_numpy(self.aux.anchors).pin_memory()
            self.own_h = torch.from_numpy(self.aux.own).pin_memory()
            self.h2d += 8 * (self.anc_h.numel() + self.own_h.numel())
            self.e2e_how = "mds_dc_plan_execute_host: host buffers in, plan-owned device copies, graph replay, results out"
        elif self.method == "interp":
            self.idx_h = torch.from_numpy(self.aux)
            self.h2d += 8 * self.idx_h.numel()
            L = M._lib()
            self.hws = torch.empty(L.mds_interpolate_host_workspace_size(w.n, w.d, w.l, w.r, M.PREC[w.prec],
                                                                         M.DTYPE[self.Yh.dtype]),
                                   dtype=torch.uint8, device=self.dev)
            self.e2e_how = "mds_interpolate_host: chunked copies of the rows overlap the landmark eigenproblem"
        else:
            self.idx_h = (torch.from_numpy(self.aux).pin_memory() if self.method in ("affine", "pivot") else
                          torch.from_numpy(W.flatten_fast_tree(self.aux)[0]).pin_memory() if self.method == "fast"
                          else None)
            self.h2d += 8 * (self.idx_h.numel() if self.idx_h is not None else 0)
            if self.method == "maxmin":
                self.d2h = 8 * w.l
            self.e2e_how = f"copies of the rows and indices, then the {self.method} call, then the result back"

    def host_step(self):
        import paper_2007_11919_gb300 as G
        w = self.w
        if self.method == "dc":
            X, _ = self.plan.execute_host(self.Yh, self.anc_h, self.own_h, X=self.Xh)
            return X
        if self.method == "interp":
            X, _, _ = G.mds_interpolate_host(self.Yh, self.idx_h, w.r, w.prec, out=self.Xh, workspace=self.hws,
                                             cluster=self.args.cluster)
            return X
        self.Yd.copy_(self.Yh, non_blocking=True)
        if self.method in ("affine", "pivot"):
            self.idx.copy_(self.idx_h, non_blocking=True)
        elif self.method == "fast":
            self.perm.copy_(self.idx_h, non_blocking=True)
        X, var = self.step()
        if self.method == "maxmin":
            return X.cpu()
        self.Xh.copy_(X, non_blocking=True)
        _ = var.cpu()
        return self.Xh

    # ---- roofline of the leg's dominant kernel from the library's stage events
    def roofline(self, stats):
        peaks = load_peaks()
        eig_ms = statistics.mean(s["stage_ms"]["eig"] for s in stats)
        post_ms = statistics.mean(s["stage_ms"]["post"] for s in stats)
        if self.method == "maxmin":
            return self._maxmin_roof(stats, peaks), None
        lan = self._lanczos_roof(stats, eig_ms, peaks)
        if self.method in ("dc", "fast"):
            return lan, None
        if self.method == "pivot":
            dist_ms = statistics.mean(s["stage_ms"]["dist"] for s in stats)
            other = self._scatter_roof(dist_ms)
            return (other, lan) if dist_ms > eig_ms else (lan, other)
        other = self._affine_roof(post_ms, peaks) if self.method == "affine" else self._projection_roof(post_ms, peaks)
        return (other, lan) if post_ms > eig_ms else (lan, other)

    def _lanczos_roof(self, stats, eig_ms, peaks):
        # Algorithmic bytes: all n^2 entries of Q (4 bytes each in FP32
        # storage, 8 in FP64) once per Lanczos step, summed over the problems'
        # steps (a landmark problem is a single one, solved in FP64).
        flops = statistics.mean(s["eig_flops"] for s in stats)
        qbytes = statistics.mean(s["eig_qbytes"] for s in stats)
        qread = statistics.mean(s["eig_qread"] for s in stats)
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = qbytes / (eig_ms * 1e-3) / 1e9
        kind = ("batched Lanczos, one cluster per part, FP32 Q, double-FP32 vectors" if self.method == "dc" else
                "FP64 Lanczos of the landmark problem, one team of clusters; Q is L2-resident, the steps are "
                "latency-bound")
        roof = {"kernel": f"k_lanczos ({kind})", "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "launch_ms": eig_ms, "bytes_per_launch": qbytes,
                # what the kernel streams: the symmetric ranges read each
                # off-diagonal block of Q once for both triangles
                "streamed_bytes_per_launch": qread, "streamed_gbs": qread / (eig_ms * 1e-3) / 1e9,
                "fp64_equiv_flops_per_launch": flops, "traffic": None}
        src = os.path.join(ROOT, "paper_2007_11919_gb300", "csrc", "k_lanczos.cu")
        tr = NCU_TRAFFIC["k_lanczos.cu"]
        if tr["sha"] == file_sha(src) and self.name in tr["bytes"]:
            roof["traffic"] = tr["bytes"][self.name] * qread
        return roof

    def _projection_roof(self, kms, peaks):
        w = self.w
        flops = w.n * (2.0 * w.l * w.d + 2.0 * w.l * w.r)
        pk = peaks.get("bf16_tflops", 1900.0)
        src_note = "MEASURED_PEAKS.json bf16_tflops (burst, of measured)" if peaks else "fallback 1.9 PFLOP/s"
        if w.prec == "fp8":
            # FP8 dense rate = measured BF16 x the nominal 4.5 / 2.25 ratio
            pk *= 2.0
            src_note += " x 2 (nominal FP8 / BF16 ratio)"
        byte_rows = self.Y.dtype == np.uint8
        achieved = flops / (kms * 1e-3) / 1e12
        if w.prec in ("f32", "f64"):
            # SIMT distance tiles and projection: peak from the unit counts,
            # 152 SMs x 128 FP32 (or 2 FP64) FMA lanes x 2 flop x 2.07 GHz
            lanes = 2 if w.prec == "f64" else 128
            pk = 152 * lanes * 2 * 2.07e9 / 1e12
            return {"kernel": "k_gower (SIMT distance tiles fused with the Gower projection)", "bound": "alu",
                    "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                    "peak_source": f"derived: 152 SMs x {lanes} {w.prec.upper()} FMA lanes x 2 flop x 2.07 GHz",
                    "launch_ms": kms, "flops_per_launch": flops, "traffic": None}
        kname = ("k_gower_tck (tcgen05 distance tiles of byte rows, K streamed, fused with the Gower projection)"
                 if byte_rows else "k_gower_tc (tcgen05 distance tiles and Gower projection, A^2 kept in TMEM)")
        roof = {"kernel": kname, "bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk, "peak_source": src_note, "launch_ms": kms, "flops_per_launch": flops}
        src = os.path.join(ROOT, "paper_2007_11919_gb300", "csrc", "k_gower_tck.cu" if byte_rows else "k_gower_tc.cu")
        tr = NCU_TRAFFIC.get(os.path.basename(src))
        roof["traffic"] = tr["bytes"] * w.n if tr and tr["sha"] == file_sha(src) else None
        return roof

    def _affine_roof(self, kms, peaks):
        # Algorithmic bytes of the affine pass: every row of Y read once and
        # X written once (the landmark mean and axes are l x d, negligible)
        w = self.w
        nbytes = w.n * w.d * self.Y.dtype.itemsize + w.n * w.r * (8 if w.prec == "f64" else 4)
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = nbytes / (kms * 1e-3) / 1e9
        tr = NCU_TRAFFIC["k_affine.cu"]
        src = os.path.join(ROOT, "paper_2007_11919_gb300", "csrc", "k_affine.cu")
        traffic = tr["bytes"] * w.n if (tr["sha"] == file_sha(src) and self.Y.dtype == np.float32) else None
        return {"kernel": "k_affine_project_bulk (one pass over Y: X = (Y - y_L) U_r; the stage holds this "
                          "launch alone)",
                "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "launch_ms": kms, "bytes_per_launch": nbytes, "traffic": traffic}

    def _maxmin_roof(self, stats, peaks):
        # Algorithmic bytes: every round streams all n rows once (l - 1 rounds)
        w = self.w
        kms = statistics.mean(s["stage_ms"]["dist"] for s in stats)
        nbytes = (w.l - 1) * w.n * w.d * self.Y.dtype.itemsize
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = nbytes / (kms * 1e-3) / 1e9
        tr = NCU_TRAFFIC["k_maxmin.cu"]
        src = os.path.join(ROOT, "paper_2007_11919_gb300", "csrc", "k_maxmin.cu")
        traffic = tr["bytes"] * w.n * (w.l - 1) if tr["sha"] == file_sha(src) else None
        return {"kernel": "k_maxmin_tiles (one streaming pass over Y per landmark, running minima, argmax; "
                          "all l - 1 rounds)",
                "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "launch_ms": kms, "bytes_per_launch": nbytes, "traffic": traffic}

    def _scatter_roof(self, kms):
        # Pivot MDS's scatter matrix S = Y_c^T Y_c: FP32 products (double-FP32
        # sums), d (d + 1) / 2 distinct products per row; bound by the FP32 FMA
        # pipe: SMs x 128 lanes x 2 flops x the 2,070 MHz maximum SM clock.
        import torch
        w = self.w
        flops = 2.0 * w.n * w.d * (w.d + 1) / 2
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        peak = sms * 128 * 2 * 2.070e9 / 1e12
        achieved = flops / (kms * 1e-3) / 1e12
        return {"kernel": "k_scatter_tri (scatter matrix of all n rows, upper triangle of 4 x 4 thread tiles, "
                          "FP32 FMA)",
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"FP32 FMA pipe: {sms} SMs x 128 lanes x 2 flops x 2.07 GHz (derived)",
                "launch_ms": kms, "flops_per_launch": flops, "traffic": None}

    def describe(self):
        w = self.w
        d = {"workload": w.name, "method": self.method, "n": w.n, "d": w.d, "r": w.r, "prec": w.prec}
        if self.method == "dc":
            d.update(parts=self.aux.p, c=w.c, plan=dict(self.plan.info(), graph=True,
                                                        autotuned=self.args.cluster == 0))
        elif self.method == "fast":
            d.update(l=w.l, s=w.c, nodes=len(self.par), leaves=int(sum(1 for _ in self.aux.leaves())))
        else:
            d.update(l=w.l)
        return d

    def variant_check(self, X):
        """Error against the oracle and the oracle's rate for the paper's other
        variants, on a bounded sample: MaxMin's first picks on the full rows
        (a MaxMin sequence's prefix is the sequence of that length) and the
        oracle on 20,000 rows; pivot MDS on a 3,000-row sample (both sides);
        fast MDS on the first top-level subset's subtree."""
        import oracle as O
        import paper_2007_11919_gb300 as G
        import torch
        w = self.w
        out = {}
        if self.method == "maxmin":
            got = X.cpu().numpy()
            out["prefix_bit_exact"] = bool(np.array_equal(got[:8], O.maxmin_landmarks(self.Y, 8, 0)))
            m = 20_000
            t0 = time.perf_counter()
            O.maxmin_landmarks(self.Y[:m], w.l, 0)
            sec = time.perf_counter() - t0
            desc = f"MaxMin of l={w.l} landmarks among the first {m} rows"
        elif self.method == "pivot":
            m = 3000
            Ys = self.Y[:m]
            piv = W.landmarks(m, w.l, 1)
            t0 = time.perf_counter()
            Xo, _, _ = O.pivot_mds(Ys, piv, w.r)
            sec = time.perf_counter() - t0
            Xs, _ = G.mds_pivot(torch.from_numpy(Ys).to(self.dev), torch.from_numpy(piv).to(self.dev), w.r, w.prec)
            out["procrustes_rel_err_vs_oracle"] = O.aligned_rel_error(Xs.double().cpu().numpy(), Xo)
            out["err_sample"] = f"both sides on the first {m} rows with {w.l} pivots among them"
            desc = f"pivot MDS of the first {m} rows, l={w.l} pivots"
        else:
            sub = self.aux.children[0]
            loc = {int(g): i for i, g in enumerate(sub.idx)}

            def local(node):
                return W.FastNode(np.array([loc[int(g)] for g in node.idx], dtype=np.int64),
                                  [local(ch) for ch in node.children])
            t0 = time.perf_counter()
            Xo, _, _ = O.fast_mds(self.Y[sub.idx], local(sub), w.r, w.c)
            sec = time.perf_counter() - t0
            m = len(sub.idx)
            out["procrustes_rel_err_vs_oracle"] = O.aligned_rel_error(X.double().cpu().numpy()[sub.idx], Xo)
            desc = f"fast MDS of the first top-level subset ({m} rows, its own subtree)"
        out["cpu_baseline"] = {"value": m / sec, "unit": "points/s", "cores": cpu_threads(), "kind": "oracle",
                               "sample": desc, "seconds": sec}
        return out


PHASES = ("exchange", "checks", "matvec", "pass_newest", "publish", "finish")


def lanczos_phases(reset=False):
    """The eigen-solver's phase cycles (a library built with
    GBMDS_PHASE_TIMERS=1), or None."""
    from paper_2007_11919_gb300 import mds as M
    L = M._lib()
    L.mds_lanczos_phase_cycles.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.mds_lanczos_phase_cycles.restype = ctypes.c_int
    out = (ctypes.c_double * 7)()
    if L.mds_lanczos_phase_cycles(out if not reset else None, 1 if reset else 0) != 0:
        return None
    if reset:
        return {}
    tot = sum(out[:6]) or 1.0
    return {"cta_steps": out[6], "cycles_per_cta_step": {k: out[i] / max(out[6], 1.0) for i, k in enumerate(PHASES)},
            "share": {k: out[i] / tot for i, k in enumerate(PHASES)}}


def time_legs(legs, steps, flush, stream):
    """Steps of all legs in turn, the L2 flushed before each call; per leg the
    CUDA-event time of every call and the library's stats of that call."""
    import torch
    from paper_2007_11919_gb300 import mds as M
    ms = {lg.name: [] for lg in legs}
    stats = {lg.name: [] for lg in legs}
    for _ in range(steps):
        for lg in legs:
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lg.step()
            e1.record(stream)
            e1.synchronize()
            ms[lg.name].append(e0.elapsed_time(e1))
            stats[lg.name].append(M.mds_last_stats())
    return ms, stats


def leg_report(lg, ms, stats, world, dev, cpu_on, one_thread):
    """Value, stage times, roofline, error against the oracle sample, CPU
    baseline and end-to-end figures of one leg."""
    import torch
    import oracle as O
    w = lg.w
    rank = dist_env()[0]
    mean_ms = max_over_ranks(statistics.mean(ms), dev)
    roof, other = lg.roofline(stats)
    X = lg.step()[0]
    torch.cuda.synchronize()
    rep = {"config": lg.describe(), "value": job_throughput(world, w.n, mean_ms), "unit": "points/s",
           "ms_per_step": mean_ms,
           "stage_ms": {k: statistics.mean(s["stage_ms"][k] for s in stats) for k in stats[0]["stage_ms"]},
           "eig_steps_per_call": stats[-1]["eig_steps"], "cluster": stats[-1]["cluster"],
           "launches_per_call": stats[-1]["launches"], "roofline": roof, "roofline_other_kernel": other}
    # end to end through the host-buffer call
    lg.host_setup()
    lg.host_step()                       # untimed: streams, pinned paths, the plan's own buffers
    torch.cuda.synchronize()
    e2e = []
    for _ in range(len(ms)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xh = lg.host_step()
        torch.cuda.synchronize()
        e2e.append(1e3 * (time.perf_counter() - t0))
    rep["e2e"] = {"value": job_throughput(world, w.n, max_over_ranks(statistics.mean(e2e), dev)), "unit": "points/s",
                  "h2d_bytes_per_step": int(lg.h2d), "d2h_bytes_per_step": int(lg.d2h),
                  "ms_steps": [round(t, 3) for t in e2e], "how": lg.e2e_how,
                  "equals_device_result": bool(torch.equal(Xh.to(X.device), X))}
    if lg.method in ("maxmin", "pivot", "fast"):
        if rank == 0 and world == 1 and cpu_on:
            rep.update(lg.variant_check(X))
        return rep
    if rank == 0 and world == 1 and cpu_on:
        rows, payload, desc = oracle_payload(lg.method, lg.Y, lg.aux, w.r, SAMPLE[lg.name])
        Xo, sec = oracle_job(lg.method, payload)
        rep["procrustes_rel_err_vs_oracle"] = O.aligned_rel_error(X.double().cpu().numpy()[rows], Xo)
        cpu = {"value": len(rows) / sec, "unit": "points/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": desc, "seconds": sec}
        if one_thread:
            sec1 = oracle_seconds_one_thread(lg.method, payload)
            cpu["one_thread"] = {"value": len(rows) / sec1, "seconds": sec1, "cores": 1}
        rep["cpu_baseline"] = cpu
    return rep


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
    from paper_2007_11919_gb300 import mds as M

    seed = rank_seed(args.seed, rank)
    if args.workload == "serve":
        return serve_main(args, rank, world, dev)
    names = HEADLINE if args.workload == "image_all" else (args.workload,)
    legs = [Leg(nm, dev, seed, args, args.n) for nm in names]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    M.mds_set_timing(True)
    stream = torch.cuda.current_stream(dev)
    time_legs(legs, args.warmup, flush, stream)
    torch.cuda.synchronize()

    # ---- timed region: K steps (every leg once per step), L2 flushed between calls
    clocks = ClockSampler(local)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    have_phases = lanczos_phases(reset=True) is not None
    ms, stats = time_legs(legs, args.steps, flush, stream)
    torch.cuda.synchronize()
    phases = lanczos_phases() if have_phases else None
    if world > 1:
        tdist.barrier()
    clk = clocks.stop()
    step_ms = [sum(ms[lg.name][i] for lg in legs) for i in range(args.steps)]
    ms_per_step = max_over_ranks(statistics.mean(step_ms), dev)
    n = legs[0].w.n
    value = job_throughput(world, n, ms_per_step)
    launches = int(sum(s["launches"] for lg in legs for s in stats[lg.name]))

    cpu_on = not args.no_cpu_baseline
    reps = {lg.name: leg_report(lg, ms[lg.name], stats[lg.name], world, dev, cpu_on,
                                one_thread=lg.method in ("interp", "dc"))
            for lg in legs}
    # the step's roofline: the dominant kernel of the longest leg
    top = max(legs, key=lambda lg: reps[lg.name]["ms_per_step"])
    roof = reps[top.name]["roofline"]
    e2e_ms = sum(lg.w.n / reps[lg.name]["e2e"]["value"] * world * 1e3 for lg in legs)
    e2e = {"value": job_throughput(world, n, e2e_ms), "unit": "points/s",
           "h2d_bytes_per_step": sum(reps[lg.name]["e2e"]["h2d_bytes_per_step"] for lg in legs),
           "d2h_bytes_per_step": sum(reps[lg.name]["e2e"]["d2h_bytes_per_step"] for lg in legs),
           "how": "; ".join(f"{lg.name}: {reps[lg.name]['e2e']['how']}" for lg in legs)}
    cpu = None
    if all("cpu_baseline" in reps[lg.name] for lg in legs):
        # the oracle's rate for a step of the same composition: n points through every leg
        sec = sum(n / reps[lg.name]["cpu_baseline"]["value"] for lg in legs)
        cpu = {"value": n / sec, "unit": "points/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": "; ".join(f"{lg.name}: {reps[lg.name]['cpu_baseline']['sample']}" for lg in legs),
               "cpu_model": cpu_model(), "host_cpus": os.cpu_count()}
        if all("one_thread" in reps[lg.name]["cpu_baseline"] for lg in legs):
            sec1 = sum(n / reps[lg.name]["cpu_baseline"]["one_thread"]["value"] for lg in legs)
            cpu["one_thread"] = {"value": n / sec1, "cores": 1}
    err = max((reps[lg.name].get("procrustes_rel_err_vs_oracle") or 0.0) for lg in legs) if cpu else None

    configs = None
    if args.workload == "image_all" and not args.no_configs:
        configs = {}
        for nm in SUB_CONFIGS:
            lg = Leg(nm, dev, seed, args)
            time_legs([lg], args.warmup, flush, stream)
            torch.cuda.synchronize()
            cms, cst = time_legs([lg], args.config_steps, flush, stream)
            configs[nm] = leg_report(lg, cms[nm], cst[nm], world, dev, cpu_on, one_thread=False)
            del lg
            torch.cuda.empty_cache()

    serve = (serve_leg(dev, seed, args.serve_requests, 100, 500, args.serve_load, args.serve_slots)
             if rank == 0 and not args.no_serve else None)

    if rank == 0:
        wname = ("image_all_fp8_n%d_d784_l2000_parts2000_c50_r10" % n if args.workload == "image_all"
                 else legs[0].w.name)
        emit({"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": legs[0].w.prec, "data": "synthetic",
              "config": {"workload": wname, "n_per_gpu": n, "legs": [lg.describe() for lg in legs],
                         "step": "one call of each leg over all n rows, device-resident inputs",
                         "l2": "flushed before every call (256 MB write)", "parallelism": f"replicas{world}"},
              "procrustes_rel_err_vs_oracle": err, "legs": reps, "roofline": roof, "cpu_baseline": cpu,
              "e2e": e2e, "gpu_launches": launches, "clocks": clk, "gpu": torch.cuda.get_device_name(dev),
              "configs": configs, "serve": serve,
              **({"lanczos_phases": dict(phases, build="GBMDS_PHASE_TIMERS=1 (instrumented)")} if phases else {})})
    if world > 1:
        tdist.destroy_process_group()


def serve_main(args, rank, world, dev):
    """--workload serve: the serving run is the measurement; one step is a
    window of --serve-requests arrivals."""
    import torch

    seed = rank_seed(args.seed, rank)
    clocks = ClockSampler(dev.index)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
    clocks.start()
    res = serve_leg(dev, seed, args.steps * args.serve_requests, max(args.warmup, 1) * 50, 500, args.serve_load,
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
    peaks = load_peaks()
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
