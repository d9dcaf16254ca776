#!/usr/bin/env python
"""Throughput of the fast Basic SSA hot path on one or more GB300s.

One step = one whole pass of the hot path on the long-series workload:
spectrum of the series (Algorithm 2 steps 1-2), thick-restart Lanczos SVD of
the N = 2^20, L = 2^19 trajectory matrix for k = 50 triples (Algorithms 1-3),
and Hankelization of all k elementary components (Algorithm 4).  The metric
is decompositions per second (each including its reconstruction).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f64|f32c]
  python bench.py --impl reference ...   # the CPU oracle on this host's cores

Multi-GPU (torchrun, one rank per GPU) runs independent replicas: the path
does not shard within one series (a dependent chain of products), so each rank
decomposes its own series and value = all ranks' decompositions / max rank time.
"""
from __future__ import annotations

import argparse
import csv
import io
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

METRIC = "SSA decomps/sec & matvec HBM GB/s vs peak at stated sigma error; p50/p99 latency"
UNIT = "decomps/s"

WORKLOADS = {
    # long series: 20 sinusoids (periods log-uniform in [5, 5000], amplitudes 1/i) + trend + N(0, 0.1^2)
    "many_sines_N1M": dict(N=1 << 20, L=1 << 19, k=50, gen="many_sines", seed=1,
                           golden="tests/golden/sigma_many_sines_N1048576_L524288_k50.txt"),
    # half-length variant, used for profiling captures (bases ~0.9 GB, still larger than L2)
    "many_sines_N512K": dict(N=1 << 19, L=1 << 18, k=50, gen="many_sines", seed=1, golden=None),
    # N = 1000 three-sine series (the paper-sized small case)
    "three_sines_N1000": dict(N=1000, L=500, k=10, gen="three_sines", seed=0, golden=None),
    # shapes of the paper's section 7 real-data runs (daily temperatures, monthly births), three-sine stand-ins
    "standin_N86867_k50": dict(N=86867, L=43433, k=50, gen="three_sines", seed=8,
                               golden="tests/golden/sigma_three_sines_N86867_L43433_k50.txt"),
    "standin_N5113_k100": dict(N=5113, L=2556, k=100, gen="three_sines", seed=7,
                               golden="tests/golden/sigma_three_sines_N5113_L2556_k100.txt"),
    # 4096 ragged series in one persistent launch: N ~ U{500..20000}, L alternating round(N/3) and N//2,
    # k ~ U{4..32}, three-sine generator with per-series seeds; FP32-compensated products
    "batch_4096": dict(kind="batch", count=4096, seed=2),
    # the first 512 series of the same generator (profiling captures: one launch of ~0.2 s)
    "batch_512": dict(kind="batch", count=512, seed=2),
    # Poisson arrivals at 2000 requests/s into the request server: N log-uniform in [1e3, 1e6], L = N//2,
    # k ~ U{2..64}, 40 GiB admission budget; each step is one arrival window of --window seconds
    "serving_2000rps": dict(kind="serving", rate=2000.0, seed=4),
    # trajectory-matrix products X v (Algorithm 2) at the long-series size: the library's kernels in
    # both precisions, with cuFFT (torch.fft) doing the same product beside them as a timed comparison
    "matvec_N1M": dict(kind="products", N=1 << 20, L=1 << 19, gen="many_sines", seed=1),
    # section 6.4 timing setup: Q = N/2, B = T = N/4, L = B/2, I = {1, 2}; unit = whole H-matrices
    "hmatrix_N4000": dict(kind="hmatrix", N=4000, seed=0),
    # section 6.3: replicas of the rank-5 series + N(0, 5^2), L = N/2, rank-5 reconstruction each
    "bootstrap_N4000_R64": dict(kind="bootstrap", N=4000, R=64),
    # precision stress: N = 2^22, L = 2^21, k = 100, exact-rank-40 damped cosines + N(0, 1e-6^2);
    # both precisions, per-sigma errors
    "damped_N4M_k100": dict(kind="precision", N=1 << 22, L=1 << 21, k=100, gen="damped_sines", seed=3,
                            golden="tests/golden/sigma_damped_sines_N4194304_L2097152_k100.txt"),
}

# ncu DRAM traffic of the dominant kernel as a ratio to its algorithmic bytes
# (dram__bytes_read.sum + dram__bytes_write.sum over launches of the bench
# size), keyed by the kernel class; valid only while the kernel source is
# unchanged (sha256 of the file that holds it), else the line reports traffic null.
NCU_TRAFFIC = {
    "cgs_update_proj": {"ratio": 0.983, "file": "paper_0911_4498_gb300/csrc/cgs_lanes.cuh",
                        "sha256": "50cd82553364e561ab037eafa03b2172b9570d6313defe12e3e522694e98f435",
                        "profile": "profiles/cgs_lanes_many_sines_N1M_dram.md"},
    # projection launches 2402 and 2405 of the same capture: (423.8 / 427.8 + 256.3 / 260.0) / 2
    "cgs_proj": {"ratio": 0.988, "file": "paper_0911_4498_gb300/csrc/cgs_lanes.cuh",
                 "sha256": "50cd82553364e561ab037eafa03b2172b9570d6313defe12e3e522694e98f435",
                 "profile": "profiles/cgs_lanes_many_sines_N1M_dram.md"},
    # one launch of the 512-series batch: (328.48 + 36.62) GB of DRAM traffic / 524.91 GB algorithmic
    "k_batch_ssa": {"ratio": 0.696, "file": "paper_0911_4498_gb300/csrc/batch.cu",
                    "sha256": "219ee73bceec3bff1faf08d4a2df1ca7ac97d161158a9b4862b991c05ba461a5",
                    "profile": "profiles/batch_ssa_batch512.md"},
}


def ncu_traffic(kernel, bytes_per_launch):
    import hashlib
    t = NCU_TRAFFIC.get(kernel)
    if not t:
        return None
    with open(os.path.join(ROOT, t["file"]), "rb") as fh:
        if hashlib.sha256(fh.read()).hexdigest() != t["sha256"]:
            return None
    return t["ratio"] * bytes_per_launch


def series(w):
    from paper_0911_4498_gb300 import synth
    return getattr(synth, w["gen"])(w["N"], seed=w["seed"])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def read_golden(path):
    if not path or not os.path.exists(os.path.join(ROOT, path)):
        return None
    out = {}
    with open(os.path.join(ROOT, path)) as fh:
        for line in fh:
            if line.startswith("#") or ":" not in line:
                continue
            k, _, v = line.partition(":")
            out[k.strip()] = np.array([float(t) for t in v.split()])
    return out


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.dev is not None:
            cmd += ["-i", str(self.dev)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = list(csv.reader(io.StringIO(open(self.path).read())))
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for_smi(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


def aggregate(elapsed_s, units, dist=None, device=None):
    """Whole-job throughput over ranks: (sum of units) / (max rank time).

    Each rank passes its own timed-region length and unit count; with a
    process group the max time and the summed units are all-reduced.
    """
    if dist is None:
        return units / elapsed_s, elapsed_s, units
    import torch
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())


# ----------------------------------------------------------------- CPU oracle sample
def cpu_worker(args):
    """Unit costs of the CPU oracle on this workload (own process, 1 thread): one product of
    each kind (Algorithms 2/3 on the oracle's radix-2 FFT), MGS-twice reorthogonalisation
    against 64 basis columns of each length, one restart product, one projected SVD of size d
    and one rank-1 Hankelization (Algorithm 4)."""
    from oracle import fast_hankel, jacobi, lanczos
    w = WORKLOADS[args.workload]
    f = series(w)
    N, L, k = w["N"], w["L"], w["k"]
    K = N - L + 1
    Lw, Kw = min(L, K), max(L, K)
    d, kk = lanczos.default_dims(Lw, Kw, k)
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    M = fast_hankel.fft_length(N)
    chat = fast_hankel.spectrum(f, L, M)
    t_spec = time.perf_counter() - t0
    u, v = rng.standard_normal(L), rng.standard_normal(K)
    t = time.perf_counter()
    fast_hankel.hankel_matvec(chat, N, L, v)
    fast_hankel.hankel_rmatvec(chat, N, L, u)
    t_mv = (time.perf_counter() - t) / 2
    C0 = 64
    t_col = {}
    for dim in sorted({Lw, Kw}):
        Q = np.asfortranarray(rng.standard_normal((dim, C0)))
        x = rng.standard_normal(dim)
        t = time.perf_counter()
        lanczos._mgs_twice(Q, C0, x)
        t_col[dim] = (time.perf_counter() - t) / C0
    Q = np.asfortranarray(rng.standard_normal((Kw, d)))
    P = rng.standard_normal((d, kk))
    t = time.perf_counter()
    _ = Q @ P
    t_ritz = (time.perf_counter() - t) * (Lw + Kw) / Kw
    Bm = np.triu(np.tril(rng.standard_normal((d + 1, d)), 0), -1)
    t = time.perf_counter()
    jacobi.svd(Bm)
    t_svd = time.perf_counter() - t
    t = time.perf_counter()
    fast_hankel.rank1_hankelization(1.0, u, v)
    t_hank = time.perf_counter() - t
    print(json.dumps({"seconds": time.perf_counter() - t0, "t_spec": t_spec, "t_mv": t_mv,
                      "t_col": {str(a): b for a, b in t_col.items()}, "t_ritz": t_ritz, "t_svd": t_svd,
                      "t_hank": t_hank, "d": d, "kk": kk}))


def cpu_sample(workload):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", workload],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("cpu worker failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_restarts(workload):
    """Thick restarts the oracle's own Lanczos took on this workload (header of its stored
    values), or None."""
    path = WORKLOADS[workload].get("golden")
    if not path or not os.path.exists(os.path.join(ROOT, path)):
        return None
    with open(os.path.join(ROOT, path)) as fh:
        for line in fh:
            if line.startswith("#") and "restarts" in line:
                try:
                    return int(line.split("restarts")[1].split(",")[0])
                except ValueError:
                    return None
    return None


def cpu_decomp_seconds(workload, s, restarts):
    """Seconds one oracle decomposition + reconstruction takes on one core, from the measured
    unit costs over the oracle's own schedule (its restart rule, d and kk; restarts as it ran
    them): spectrum + every half-step (a product and MGS twice against that half-step's basis)
    + the projected SVD of every cycle + the restart and final Ritz products + k Hankelizations."""
    w = WORKLOADS[workload]
    N, L, k = w["N"], w["L"], w["k"]
    K = N - L + 1
    Lw, Kw = min(L, K), max(L, K)
    tcol = {int(a): b for a, b in s["t_col"].items()}
    tot = s["t_spec"]
    sched = side_schedule(Lw, Kw, s["d"], s["kk"], restarts)
    for ncols, dim in sched:
        tot += s["t_mv"] + ncols * tcol[dim]
    tot += (restarts + 1) * (s["t_svd"] + s["t_ritz"]) + k * s["t_hank"]
    return tot, len(sched)


def cpu_baseline(workload, gpu_restarts):
    s = cpu_sample(workload)
    rs = oracle_restarts(workload)
    rs = gpu_restarts if rs is None else rs
    sec, halfsteps = cpu_decomp_seconds(workload, s, rs)
    return {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"unit costs of the oracle measured here in {s['seconds']:.1f} s (one product "
                       f"{s['t_mv']:.2f} s, MGS twice per basis column, projected SVD, Ritz product, one "
                       f"Hankelization {s['t_hank']:.2f} s) over the oracle's schedule of {halfsteps} half-steps "
                       f"and {rs} restarts, plus the reconstruction of all k components: {sec:.0f} s per "
                       "decomposition")}


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    if "N" not in w or "k" not in w or w.get("kind") is not None:
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm covers the single-series "
                                                              "workloads (the oracle has no batched or served path)"}))
        return 0
    rs = oracle_restarts(args.workload)
    secs, walls = [], []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        s = cpu_sample(args.workload)
        wall = time.perf_counter() - t
        sec, halfsteps = cpu_decomp_seconds(args.workload, s, rs if rs is not None else 4)
        if i >= args.warmup:
            secs.append(sec)
            walls.append(wall)
    sec = statistics.median(secs)
    value = 1.0 / sec
    sample = (f"each step measures the oracle's unit costs on this host (one product each way, MGS twice "
              f"against 64 columns, a projected SVD, a Ritz product, a Hankelization; {statistics.median(walls):.1f} s)"
              f" and prices one decomposition + reconstruction over the oracle's own schedule "
              f"({halfsteps} half-steps, {rs if rs is not None else 4} restarts): {sec:.0f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": w["N"], "L": w["L"], "k": w["k"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- many-series workloads
def side_schedule(dimL, dimK, d, kk, restarts):
    """(basis columns, vector length) of every reorthogonalisation of one
    thick-restart Lanczos run, in the order the engine runs them."""
    out = [(0, dimL), (0, dimK)]            # p_0 and the first v
    r, c = 1, 1
    for cyc in range(restarts + 1):
        while c < d + 1:
            out.append((r, dimL))
            r += 1
            out.append((c, dimK))
            c += 1
        if cyc < restarts:
            r, c = kk, kk + 1
    return out


def lanczos_bytes(N, L, k, d, kk, restarts, M, s=8):
    """Algorithmic bytes of one decomposition by the per-unit figures: each
    product s(N + M) (input, output, half spectrum at 16 B per complex), each
    CGS2 reorthogonalisation 3 passes over its basis plus the vector, each
    restart the Ritz products."""
    K = N - L + 1
    Lw, Kw = min(L, K), max(L, K)
    mv = s * (Lw + Kw) + 16 * (M // 2 + 1)
    tot = 0.0
    for ncols, dim in side_schedule(Lw, Kw, d, kk, restarts):
        tot += mv + 8.0 * (3 * ncols * dim + 5 * dim)
    tot += restarts * 8.0 * ((d + kk) * Lw + (d + kk) * Kw)
    tot += 8.0 * ((d + k) * (Lw + Kw))
    return tot


def default_dims(L, K, k):
    mn = min(L, K)
    d = min(max(2 * k, k + 32), mn)
    d = max(d, k)
    kk = min(max(k + (d - k + 4) // 5, k), max(d - 1, k))
    return d, kk


def cpu_sample_series(specs, halfsteps=6, budget_s=20.0):
    """Oracle Lanczos on a bounded sample of series, one process per core
    (spawned before any GPU work in the pool): seconds per half-step each."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    cores = os.cpu_count() or 1
    with ctx.Pool(min(cores, len(specs))) as pool:
        t = time.perf_counter()
        res = pool.map(_cpu_one, [(N, L, k, seed, halfsteps) for (N, L, k, seed) in specs])
        wall = time.perf_counter() - t
    return res, wall, min(cores, len(specs))


def _cpu_one(a):
    N, L, k, seed, halfsteps = a
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle import ssa as ossa
    from paper_0911_4498_gb300 import synth
    f = synth.three_sines(N, seed=seed)
    t = time.perf_counter()
    out = ossa.decompose(f, L, k, method="lanczos", max_steps=halfsteps)
    return (time.perf_counter() - t) / max(1, int(out.get("steps", halfsteps)))


def run_gpu_batch(args, w):
    import torch
    from paper_0911_4498_gb300 import build, synth
    build.build()
    import paper_0911_4498_gb300 as ssa
    series_l, Ls, ks = synth.batch_workload(w["count"], seed=w["seed"])
    n = len(series_l)
    Ns = np.array([f.size for f in series_l], dtype=np.int64)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(Ns)
    f_host = np.concatenate(series_l)
    Ls = Ls.astype(np.int64)
    ks32 = ks.astype(np.int32)
    prec = ssa.SSA_PREC_F32C if args.precision_batch == "f32c" else ssa.SSA_PREC_F64
    stream = torch.cuda.current_stream()
    opts = ssa.make_opts(precision=prec, stream=stream.cuda_stream)
    f_dev = torch.from_numpy(f_host).cuda()
    off_d = torch.from_numpy(off).cuda()
    L_d = torch.from_numpy(Ls).cuda()
    k_d = torch.from_numpy(ks32).cuda()
    sig_all = np.empty(int(ks.sum()))

    def step(fin, offs, Lsx, ksx, collect=False):
        b, rc = ssa.ssa_decompose_batch(fin, offs, Lsx, ksx, opts)
        infos = None
        try:
            if collect:
                infos = [ssa.ssa_batch_info(b, i) for i in range(n)]
                pos = 0
                for i in range(n):
                    ssa.ssa_batch_get(b, i, sig_all[pos:pos + ks[i]])
                    pos += ks[i]
        finally:
            ssa.ssa_batch_destroy(b)
        return rc, infos

    rc, infos = step(f_dev, off_d, L_d, k_d, collect=True)
    # the timed runs: one batch plan, its run captured once in a CUDA graph and replayed
    side = torch.cuda.Stream()
    plan = ssa.ssa_batch_plan(off, Ls, ks32, ssa.make_opts(precision=prec, stream=side.cuda_stream))
    torch.cuda.synchronize()
    ssa.ssa_batch_run(plan, f_dev)
    ssa.ssa_batch_wait(plan)
    graph = torch.cuda.CUDAGraph()
    l0 = ssa.ssa_kernel_launches()
    with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
        ssa.ssa_batch_run(plan, f_dev)
    kernels_per_run = ssa.ssa_kernel_launches() - l0
    for _ in range(max(0, args.warmup - 1)):
        graph.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = sampler.stop()
    assert ssa.ssa_batch_wait(plan) in (ssa.SSA_OK, ssa.SSA_ENOCONV)
    ssa.ssa_batch_destroy(plan)
    launches = kernels_per_run * args.steps
    value = n / (ms / 1000.0)
    # end to end with host arrays: H2D of all series inside the call, D2H of every sigma
    f_pin = torch.from_numpy(f_host).pin_memory()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        b, _ = ssa.ssa_decompose_batch(f_pin.numpy(), off, Ls, ks32, opts)
        pos = 0
        for i in range(n):
            ssa.ssa_batch_get(b, i, sig_all[pos:pos + ks[i]])
            pos += ks[i]
        ssa.ssa_batch_destroy(b)
    e2e_dt = (time.perf_counter() - t) / args.steps
    # accuracy on a sample of series against the oracle
    from oracle import ssa as ossa
    sample = list(range(0, n, max(1, n // 6)))[:6]
    errs = []
    starts = np.concatenate([[0], np.cumsum(ks)])
    for i in sample:
        ref = ossa.decompose(series_l[i], int(Ls[i]), int(ks[i]), method="jacobi" if Ns[i] <= 1500 else "lanczos")
        got = sig_all[starts[i]:starts[i + 1]]
        errs.append(float(np.max(np.abs(got - ref["sigma"]) / ref["sigma"])))
    # algorithmic bytes of the launch by the per-unit figures and the engine's restart schedule
    tot_bytes = 0.0
    for i in range(n):
        K = int(Ns[i] - Ls[i] + 1)
        d, kk = default_dims(int(Ls[i]), K, int(ks[i]))
        M = 4
        while M < Ns[i]:
            M *= 2
        tot_bytes += lanczos_bytes(int(Ns[i]), int(Ls[i]), int(ks[i]), d, kk, infos[i]["restarts"], M,
                                   s=4 if prec == ssa.SSA_PREC_F32C else 8)
    hbm, peak_kind = peaks()
    achieved = tot_bytes / (ms / 1000.0) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": ncu_traffic("k_batch_ssa", tot_bytes), "kernel": "k_batch_ssa", "bytes_per_launch": tot_bytes,
            "ms_per_launch": ms, "launches": args.steps, "peak_source": peak_kind,
            "note": "algorithmic bytes of all series by the per-unit formulas; ncu measured DRAM traffic at 70 % of "
                    "them (the rest hits L2 and shared memory); the kernel is latency-bound, one 16-warp CTA per "
                    "SM with long-scoreboard stalls on the streamed bases, not bandwidth-bound"}
    cpu = None
    if not args.no_cpu_baseline:
        pick = list(range(0, n, max(1, n // 32)))[:32]
        per_half, wall, cores = cpu_sample_series([(int(Ns[i]), int(Ls[i]), int(ks[i]), 2 * 1_000_003 + i)
                                                   for i in pick], args.sample_halfsteps)
        est = [per_half[j] * infos[i]["matvecs"] for j, i in enumerate(pick)]
        cpu = {"value": (os.cpu_count() or 1) / statistics.mean(est), "unit": UNIT, "cores": os.cpu_count() or 1,
               "kind": "oracle",
               "sample": f"oracle Lanczos, first {args.sample_halfsteps} half-steps of {len(pick)} of the series "
                         f"(one per core, {wall:.1f} s), scaled to each series' half-step count on the GPU; all "
                         "cores busy"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+df64" if prec == ssa.SSA_PREC_F32C else "df64", "data": "synthetic",
            "config": {"workload": args.workload, "series": n, "N": "U{500..20000}", "L": "round(N/3) | N//2",
                       "k": "U{4..32}", "total_samples": int(Ns.sum()), "precision": args.precision_batch,
                       "launch": "ssa_batch_run captured once in a CUDA graph, replayed per step",
                       "l2": (f"inputs {8 * Ns.sum() / 1e9:.2f} GB, larger than the 129 MB L2; no flush"
                              if 8 * Ns.sum() > 129e6 else
                              f"inputs {8 * Ns.sum() / 1e6:.0f} MB fit in L2 and are not flushed")},
            "sigma_rel_err_max_sample": max(errs), "converged": all(i["converged"] for i in infos),
            "matvecs_mean": float(np.mean([i["matvecs"] for i in infos])), "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": n / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": int(8 * Ns.sum()),
                    "d2h_bytes_per_step": int(8 * ks.sum())},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line))
    return 0


def run_gpu_serving(args, w):
    """Request server under the workload's Poisson stream (N log-uniform [1e3, 1e6], L = N//2,
    k U{2..64}, seeded series).

    Capacity: the first --serve-queue arrivals of the 2000 req/s stream (about a second of it,
    far above what one GPU serves) are submitted on their arrival times and the server runs until
    every one has finished; capacity = their number / (last completion - first submission): the
    offered mix, every request counted once.  Latency: a continuous Poisson stream at 0.7 x that
    capacity for --warmup + --steps seconds with no drain in between; p50/p99 over the requests
    that finish after the warm-up seconds, with the offered and completed counts so that a stream
    the server could not keep up with shows.  Series come from a pool of pre-generated ones (request
    i uses pool entry i mod P: its N, L, k and series)."""
    import threading
    import torch
    from paper_0911_4498_gb300 import build, synth
    build.build()
    import paper_0911_4498_gb300 as ssa
    prec = ssa.SSA_PREC_F32C if args.precision_batch == "f32c" else ssa.SSA_PREC_F64
    P = args.serve_pool
    pool_arr = synth.serving_arrivals(w["rate"], P / w["rate"] * 1.2 + 1.0, seed=w["seed"])[:P]
    pool = [(N, L, k, synth.three_sines(N, seed=sd)) for (_, N, L, k, sd) in pool_arr]

    def server():
        return ssa.ssa_serve_create(ssa.make_serve_opts(precision=prec, workers=args.serve_workers,
                                                        batch_workers=args.serve_batch_workers,
                                                        max_batch=args.serve_max_batch,
                                                        grid_cap=args.serve_grid_cap))

    def submit_stream(srv, arrivals, t0, on_submit):
        for ta, pi in arrivals:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            N, L, k, f = pool[pi]
            on_submit(ssa.ssa_serve_submit(srv, f, L, k, 0), k)

    # ---- capacity
    arr = synth.serving_arrivals(w["rate"], args.serve_queue / w["rate"] * 1.5 + 1.0, seed=w["seed"] + 1)
    arr = [(t, i % P) for i, (t, *_r) in enumerate(arr)][:args.serve_queue]
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = ssa.ssa_kernel_launches()
    srv = server()
    ids = []
    t0 = time.perf_counter()
    submit_stream(srv, arr, t0, lambda rid, k: ids.append((rid, k)))
    t_last, batched, n_big = 0.0, 0, 0
    for (rid, k), (_, pi) in zip(ids, arr):
        while not ssa.ssa_serve_poll(srv, rid, 1.0):
            pass
        rc, info = ssa.ssa_serve_take(srv, rid, np.empty(k))
        t_last = max(t_last, info["t_done"])
        batched += info["batched"]
        n_big += pool[pi][0] > args.serve_batch_n
    stats = ssa.ssa_serve_stats(srv)
    ssa.ssa_serve_destroy(srv)
    capacity = len(ids) / t_last
    # ---- latency under a sustainable stream
    rate2 = 0.7 * capacity
    dur = float(args.warmup + args.steps)
    arr2 = synth.serving_arrivals(rate2, dur, seed=w["seed"] + 2)
    arr2 = [(t, i % P) for i, (t, *_r) in enumerate(arr2)]
    srv = server()
    pending, lock, res2 = [], threading.Lock(), []
    state = {"done": False}

    def collector():
        while True:
            with lock:
                item = pending[0] if pending else None
            if item is None:
                if state["done"]:
                    return
                time.sleep(0.0005)
                continue
            rid, k = item
            if ssa.ssa_serve_poll(srv, rid, 0.05):
                rc, info = ssa.ssa_serve_take(srv, rid, np.empty(k))
                res2.append((info["t_submit"], info["t_done"] - info["t_submit"]))
                with lock:
                    pending.pop(0)

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()

    def add(rid, k):
        with lock:
            pending.append((rid, k))

    submit_stream(srv, arr2, t0, add)
    state["done"] = True
    th.join()
    ssa.ssa_serve_destroy(srv)
    clocks = sampler.stop()
    launches = ssa.ssa_kernel_launches() - launches0
    lat = [l for (ts, l) in res2 if ts >= args.warmup]
    # the same mix (every pool entry once; the capacity sample cycles through the pool) one request
    # after another through the plain FP64 single-series path; plans of every FFT size class are
    # made first, untimed (the four-step tiling autotuner runs once per size class and process)
    seq = pool[:args.seq_sample] if args.seq_sample > 0 else pool
    for N, L, k, f in {int(np.ceil(np.log2(e[0]))): e for e in seq}.values():
        ssa.ssa_plan_destroy(ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=ssa.SSA_PREC_F64)))
    t = time.perf_counter()
    for (N, L, k, f) in seq:
        plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=ssa.SSA_PREC_F64))
        d, _ = ssa.ssa_decompose(plan, f, k)
        sg = np.empty(k)
        ssa.ssa_decomp_get(d, sg, None, None, None)
        ssa.ssa_decomp_destroy(d)
        ssa.ssa_plan_destroy(plan)
    seq_rate = len(seq) / (time.perf_counter() - t)
    pct = lambda a, q: float(np.percentile(a, q)) if a else None
    line = {"metric": METRIC, "value": capacity, "unit": "requests/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64" if prec == ssa.SSA_PREC_F32C else "df64",
            "data": "synthetic",
            "config": {"workload": args.workload, "arrival_rate": w["rate"], "N": "log-uniform [1e3, 1e6]",
                       "L": "N//2", "k": "U{2..64}", "mem_budget_GiB": 40, "precision": args.precision_batch,
                       "outputs": "sigma and residuals", "workers": args.serve_workers,
                       "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8 (default)"),
                       "batch_workers": args.serve_batch_workers, "max_batch": args.serve_max_batch,
                       "grid_cap": args.serve_grid_cap,
                       "series_pool": P, "capacity_sample": len(ids),
                       "latency_stream_s": dur, "latency_warmup_s": args.warmup},
            "capacity": {"requests": len(ids), "seconds": t_last, "batched": batched,
                         "share_N_above_batch_limit": n_big / len(ids)},
            "latency_s": {"p50": pct(lat, 50), "p99": pct(lat, 99), "offered_rps": rate2,
                          "offered": len(arr2), "completed": len(res2), "counted": len(lat)},
            "sequential_f64": {"value": seq_rate, "requests": len(seq)},
            "speedup_vs_sequential_f64": capacity / seq_rate, "mem_peak_GiB": stats["mem_peak"] / 2**30,
            "roofline": None, "cpu_baseline": None,
            "e2e": {"value": capacity, "unit": "requests/s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line))
    return 0


def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, sampler.stop()


def fft_product(f, L, M, dtype, device="cpu"):
    """X x (Algorithm 2) through a library FFT (torch.fft: cuFFT on a GPU), for timed comparison.

    The circulant column c = (f_{N-L+1..N}, 0 x (M-N), f_{1..N-L}) is transformed once; returns a
    function mapping x (K values, a tensor) to X x (L values).  Not part of the library's path.
    """
    import torch
    N = f.size
    K = N - L + 1
    c = np.zeros(M)
    c[:L] = f[N - L:]
    c[L + (M - N):] = f[:N - L]
    chat = torch.fft.rfft(torch.from_numpy(c).to(device=device, dtype=dtype))
    wbuf = torch.zeros(M, dtype=dtype, device=device)

    def prod(xx):
        wbuf[:K].copy_(xx.flip(0))
        return torch.fft.irfft(torch.fft.rfft(wbuf) * chat, n=M)[:L]

    return prod


def run_gpu_products(args, w):
    """Products per second of X v at N = 2^20 through the C ABI (device buffers), beside cuFFT."""
    import math as _m
    import torch
    from paper_0911_4498_gb300 import build
    build.build()
    import paper_0911_4498_gb300 as ssa
    N, L = w["N"], w["L"]
    K = N - L + 1
    f = series(w)
    stream = torch.cuda.current_stream()
    R = 20          # products per step
    NV = 40         # input/output vectors the products rotate through (2 x 168 MB > L2)
    rng = np.random.default_rng(7)
    xs = torch.from_numpy(rng.standard_normal((NV, K))).cuda()
    ys = torch.empty((NV, L), dtype=torch.float64, device="cuda")
    rows = np.linspace(0, L - 1, 8).astype(np.int64)
    xh = xs[0].cpu().numpy()
    exact = np.array([_m.fsum(f[i:i + K] * xh) for i in rows])
    scale = float(np.linalg.norm(f) * np.linalg.norm(xh))
    res, M = {}, None
    for name, prec in (("ssa_f64", ssa.SSA_PREC_F64), ("ssa_f32c", ssa.SSA_PREC_F32C)):
        plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=prec, stream=stream.cuda_stream))
        ssa.ssa_set_series(plan, f)
        M, _ = ssa.ssa_plan_info(plan)
        cnt = [0]

        def step():
            for _ in range(R):
                i = cnt[0] % NV
                ssa.ssa_matvec(plan, 0, xs[i], ys[i], 1)
                cnt[0] += 1

        ms, clocks = _timed(step, args.steps, args.warmup)
        ssa.ssa_matvec(plan, 0, xs[0], ys[0], 1)
        torch.cuda.synchronize()
        err = float(np.max(np.abs(ys[0].cpu().numpy()[rows] - exact)) / scale)
        res[name] = {"ms_per_product": ms / R, "products_per_s": 1000.0 * R / ms, "max_err_normwise": err,
                     "clocks": clocks}
        ssa.ssa_plan_destroy(plan)
    for name, dt in (("cufft_f64", torch.float64), ("cufft_f32", torch.float32)):
        prod = fft_product(f, L, M, dt, "cuda")
        xin = xs.to(dt)
        outs = [None] * NV
        cnt = [0]

        def step():
            for _ in range(R):
                i = cnt[0] % NV
                outs[i] = prod(xin[i])
                cnt[0] += 1

        ms, clocks = _timed(step, args.steps, args.warmup)
        y0 = prod(xin[0]).double().cpu().numpy()
        err = float(np.max(np.abs(y0[rows] - exact)) / scale)
        res[name] = {"ms_per_product": ms / R, "products_per_s": 1000.0 * R / ms, "max_err_normwise": err,
                     "clocks": clocks}
    # algorithmic bytes of one product (input, output and the half spectrum, 8-byte values)
    mv_bytes = 8.0 * (K + L) + 16.0 * (M // 2 + 1)
    hbm, peak_kind = peaks()
    ours = res["ssa_f64"]
    achieved = mv_bytes / (ours["ms_per_product"] / 1000.0) / 1e9
    line = {"metric": METRIC, "value": ours["products_per_s"], "unit": "products/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ours["ms_per_product"] * R,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "df64",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "L": L, "K": K, "M": M, "products_per_step": R,
                       "l2": "inputs and outputs rotate through 40 vectors each (2 x 168 MB), larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": "X v (three four-step kernels)", "bytes_per_launch": mv_bytes,
                         "peak_source": peak_kind},
            "products": {k2: {kk: v for kk, v in r.items() if kk != "clocks"} for k2, r in res.items()},
            "accuracy_reference": "8 sampled rows of X x summed exactly (math.fsum) on the host",
            "cpu_baseline": None, "e2e": None, "gpu_launches": None,
            "clocks": ours["clocks"]}
    print(json.dumps(line))
    return 0


def _oracle_rows(a):
    f, L, B, T, rows = a
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle import hmatrix as ohm
    t = time.perf_counter()
    for i in rows:
        U = ohm.base_vectors(f[i:i + B], L, [1, 2])
        for j in range(f.size - T + 1):
            from oracle import trajectory
            X = trajectory.trajectory_matrix(f[j:j + T], L)
            R = X - U @ (U.T @ X)
            float(np.sum(R * R)) / float(np.sum(X * X))
    return time.perf_counter() - t


def run_gpu_hmatrix(args, w):
    import torch
    from paper_0911_4498_gb300 import build, synth
    build.build()
    import paper_0911_4498_gb300 as ssa
    N = w["N"]
    Q, B = N // 2, N // 4
    T, L = B, B // 2
    f = synth.hmatrix_series(N, Q, seed=w["seed"])
    prec = ssa.SSA_PREC_F32C if args.precision_batch == "f32c" else ssa.SSA_PREC_F64
    stream = torch.cuda.current_stream()
    opts = ssa.make_opts(precision=prec, stream=stream.cuda_stream)
    fd = torch.from_numpy(f).cuda()
    G = torch.empty((N - B + 1, N - T + 1), dtype=torch.float64, device="cuda")
    launches0 = ssa.ssa_kernel_launches()
    ms, clocks = _timed(lambda: ssa.ssa_hmatrix(fd, L, B, T, [1, 2], opts, out=G), args.steps, args.warmup)
    launches = (ssa.ssa_kernel_launches() - launches0) // (args.steps + args.warmup)
    value = 1000.0 / ms
    # end to end: host series in, host H-matrix out
    Gh = np.empty((N - B + 1, N - T + 1))
    t = time.perf_counter()
    for _ in range(args.steps):
        ssa.ssa_hmatrix(f, L, B, T, [1, 2], opts, out=Gh)
    e2e = args.steps / (time.perf_counter() - t)
    # parity on sampled rows against the oracle's definition
    from oracle import hmatrix as ohm
    from oracle import trajectory
    Gc = G.cpu().numpy()
    err = 0.0
    for i in (0, (N - B) // 2, N - B):
        U = ohm.base_vectors(f[i:i + B], L, [1, 2])
        for j in range(0, N - T + 1, 97):
            X = trajectory.trajectory_matrix(f[j:j + T], L)
            R = X - U @ (U.T @ X)
            err = max(err, abs(Gc[i, j] - float(np.sum(R * R)) / float(np.sum(X * X))))
    cpu = None
    if not args.no_cpu_baseline:
        import multiprocessing as mp
        cores = os.cpu_count() or 1
        rows = [[i] for i in range(0, N - B + 1, max(1, (N - B + 1) // cores))][:cores]
        with mp.get_context("spawn").Pool(len(rows)) as pool:
            t = time.perf_counter()
            secs = pool.map(_oracle_rows, [(f, L, B, T, r) for r in rows])
            wall = time.perf_counter() - t
        per_row = statistics.mean(secs)
        cpu = {"value": cores / (per_row * (N - B + 1)), "unit": "hmatrix/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(rows)} full rows of G by the oracle's definition (one per core, {wall:.1f} s), "
                         f"scaled to all {N - B + 1} rows with every core busy"}
    line = {"metric": METRIC, "value": value, "unit": "hmatrix/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+df64" if prec == ssa.SSA_PREC_F32C else "df64", "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "Q": Q, "B": B, "T": T, "L": L, "I": [1, 2],
                       "base_decompositions": N - B + 1, "products": 2 * (N - B + 1),
                       "precision": args.precision_batch},
            "base_decomps_per_s": (N - B + 1) * value, "g_abs_err_max_sample": err,
            "roofline": None, "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "hmatrix/s", "h2d_bytes_per_step": 8 * N,
                    "d2h_bytes_per_step": 8 * (N - B + 1) * (N - T + 1)},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line))
    return 0


def run_gpu_bootstrap(args, w):
    import torch
    from paper_0911_4498_gb300 import build, synth
    build.build()
    import paper_0911_4498_gb300 as ssa
    N, R = w["N"], w["R"]
    L, k = N // 2, 5
    reps = [synth.bootstrap_series(N, seed=100 + r) for r in range(R)]
    clean = synth.bootstrap_series(N, seed=0, sigma=0.0)
    prec = ssa.SSA_PREC_F32C if args.precision_batch == "f32c" else ssa.SSA_PREC_F64
    stream = torch.cuda.current_stream()
    opts = ssa.make_opts(precision=prec, stream=stream.cuda_stream)
    off = np.arange(R + 1, dtype=np.int64) * N
    Ls = np.full(R, L, dtype=np.int64)
    ks = np.full(R, k, dtype=np.int32)
    fd = torch.from_numpy(np.concatenate(reps)).cuda()
    goff, gidx = ssa.groups_csr([list(range(k))])
    out = torch.empty(R * N, dtype=torch.float64, device="cuda")

    def step(fin, o):
        b, _ = ssa.ssa_decompose_batch(fin, off, Ls, ks, opts)
        try:
            ssa.ssa_batch_reconstruct(b, goff, gidx, 1, o)
        finally:
            ssa.ssa_batch_destroy(b)

    launches0 = ssa.ssa_kernel_launches()
    ms, clocks = _timed(lambda: step(fd, out), args.steps, args.warmup)
    launches = (ssa.ssa_kernel_launches() - launches0) // (args.steps + args.warmup)
    value = R / (ms / 1000.0)
    G = out.cpu().numpy().reshape(R, N)
    fh = np.concatenate(reps)
    oh = np.empty(R * N)
    t = time.perf_counter()
    for _ in range(args.steps):
        step(fh, oh)
    e2e = R * args.steps / (time.perf_counter() - t)
    from oracle import ssa as ossa
    err = 0.0
    for r in (0, R // 2):
        ref = ossa.decompose(reps[r], L, k, method="lanczos")
        rec = ossa.reconstruct(N, L, ref["sigma"], ref["U"], ref["V"], [list(range(k))], method="fft")[0]
        err = max(err, float(np.linalg.norm(G[r] - rec) / np.linalg.norm(rec)))
    cpu = None
    if not args.no_cpu_baseline:
        per_half, wall, cores = cpu_sample_series([(N, L, k, 0)] * min(os.cpu_count() or 1, 16), args.sample_halfsteps)
        b, _ = ssa.ssa_decompose_batch(fh, off, Ls, ks, opts)
        mv = statistics.mean(ssa.ssa_batch_info(b, i)["matvecs"] for i in range(R))
        ssa.ssa_batch_destroy(b)
        cpu = {"value": (os.cpu_count() or 1) / (statistics.mean(per_half) * mv), "unit": "reconstructions/s",
               "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"oracle Lanczos half-steps on {cores} replicas-sized series (one per core, {wall:.1f} s), "
                         f"scaled to the GPU's {mv:.0f} half-steps per replica; reconstruction not included"}
    bias = G.mean(axis=0) - clean
    line = {"metric": METRIC, "value": value, "unit": "reconstructions/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+df64" if prec == ssa.SSA_PREC_F32C else "df64", "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "L": L, "replicas": R, "rank": k, "noise_sigma": 5.0,
                       "precision": args.precision_batch},
            "rec_rel_l2_err_max_sample": err,
            "bootstrap": {"bias_rms": float(np.sqrt(np.mean(bias ** 2))),
                          "std_mean": float(np.mean(G.std(axis=0, ddof=1))),
                          "mse_rec": float(np.mean((G - clean) ** 2)),
                          "mse_input": float(np.mean((np.stack(reps) - clean) ** 2))},
            "roofline": None, "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "reconstructions/s", "h2d_bytes_per_step": 8 * R * N,
                    "d2h_bytes_per_step": 8 * R * N},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line))
    return 0


def run_gpu_precision(args, w):
    import torch
    from paper_0911_4498_gb300 import build
    build.build()
    import paper_0911_4498_gb300 as ssa
    N, L, k = w["N"], w["L"], w["k"]
    f = series(w)
    fd = torch.from_numpy(f).cuda()
    stream = torch.cuda.current_stream()
    signal = 40
    groups = [list(range(signal)), list(range(signal, k))]   # disjoint: signal, the rest
    goff, gidx = ssa.groups_csr(groups)
    res = {}
    for name, prec in (("f64", ssa.SSA_PREC_F64), ("f32c", ssa.SSA_PREC_F32C)):
        plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=prec, stream=stream.cuda_stream))
        sig = torch.empty(k, dtype=torch.float64, device="cuda")
        rec = torch.empty((2, N), dtype=torch.float64, device="cuda")
        info = {}

        def step():
            d, rc = ssa.ssa_decompose(plan, fd, k)
            try:
                ssa.ssa_reconstruct(d, goff, gidx, 2, rec)
                ssa.ssa_decomp_get(d, sig, None, None, None)
                info.update(ssa.ssa_decomp_info(d))
                info["rc"] = rc
            finally:
                ssa.ssa_decomp_destroy(d)

        ms, clocks = _timed(step, args.steps, args.warmup)
        res[name] = {"ms": ms, "sigma": sig.cpu().numpy(), "rec": rec.cpu().numpy(), "info": dict(info),
                     "clocks": clocks}
        ssa.ssa_plan_destroy(plan)
    a, b = res["f64"]["sigma"], res["f32c"]["sigma"]
    gold = read_golden(w.get("golden"))

    def errs(x, ref):
        return {"rel_sigma_i": [float(v) for v in np.abs(x - ref) / np.abs(ref)],
                "rel_sigma_1": [float(v) for v in np.abs(x - ref) / abs(ref[0])],
                "max_rel_signal": float(np.max(np.abs(x[:signal] - ref[:signal]) / ref[:signal])),
                "max_rel_sigma_1": float(np.max(np.abs(x - ref)) / abs(ref[0]))}

    out = {"f32c_vs_f64": errs(b, a)}
    if gold is not None:
        out["f64_vs_oracle"] = errs(a, gold["sigma"][:k])
        out["f32c_vs_oracle"] = errs(b, gold["sigma"][:k])
    r64, r32 = res["f64"]["rec"], res["f32c"]["rec"]
    rec_err = {"signal_group_f32c_vs_f64": float(np.linalg.norm(r32[0] - r64[0]) / np.linalg.norm(r64[0])),
               "all_k_f32c_vs_f64": float(np.linalg.norm(r32.sum(0) - r64.sum(0)) / np.linalg.norm(r64.sum(0))),
               "signal_group_f64_vs_series": float(np.linalg.norm(r64[0] - f) / np.linalg.norm(f))}
    line = {"metric": METRIC, "value": 1000.0 / res["f64"]["ms"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["f64"]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "df64", "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "L": L, "k": k, "signal_rank": signal,
                       "groups": "first 40 (signal) and the other 60", "l2": "bases ~13 GB, larger than L2"},
            "modes": {m: {"value": 1000.0 / res[m]["ms"], "ms": res[m]["ms"], "restarts": res[m]["info"]["restarts"],
                          "matvecs": res[m]["info"]["matvecs"], "converged": res[m]["info"]["rc"] == 0}
                      for m in res},
            "sigma_errors": out, "reconstruction_rel_l2": rec_err,
            "oracle_reference": "present" if gold is not None else "not yet computed",
            "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": res["f64"]["clocks"]}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_0911_4498_gb300 import build
    build.build()
    import paper_0911_4498_gb300 as ssa

    w = WORKLOADS[args.workload]
    if w.get("kind") == "batch":
        return run_gpu_batch(args, w)
    if w.get("kind") == "serving":
        return run_gpu_serving(args, w)
    if w.get("kind") == "hmatrix":
        return run_gpu_hmatrix(args, w)
    if w.get("kind") == "bootstrap":
        return run_gpu_bootstrap(args, w)
    if w.get("kind") == "precision":
        return run_gpu_precision(args, w)
    if w.get("kind") == "products":
        return run_gpu_products(args, w)
    N, L, k = w["N"], w["L"], w["k"]
    K = N - L + 1
    prec = ssa.SSA_PREC_F32C if args.precision == "f32c" else ssa.SSA_PREC_F64
    skip = args.reorth_skip if prec == ssa.SSA_PREC_F64 else 0.0
    stream = torch.cuda.current_stream()
    opts = ssa.make_opts(precision=prec, seed=rank, stream=stream.cuda_stream, reorth_skip=skip)
    f_host = series(w)
    plan = ssa.ssa_embed_plan(N, L, opts)
    f_dev = torch.from_numpy(f_host).cuda()
    groups = [[i] for i in range(k)]
    off, idx = ssa.groups_csr(groups)
    off_dev = torch.from_numpy(off).cuda()
    idx_dev = torch.from_numpy(idx).cuda()
    out_dev = torch.empty((k, N), dtype=torch.float64, device="cuda")
    sig_dev = torch.empty(k, dtype=torch.float64, device="cuda")
    info = {}

    def step(fin, out, sig):
        d, rc = ssa.ssa_decompose(plan, fin, k)
        try:
            ssa.ssa_reconstruct(d, off_dev, idx_dev, k, out)
            ssa.ssa_decomp_get(d, sig, None, None, None)
            info.update(ssa.ssa_decomp_info(d))
            info["rc"] = rc
        finally:
            ssa.ssa_decomp_destroy(d)

    for _ in range(args.warmup):
        step(f_dev, out_dev, sig_dev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(gpu_index_for_smi(local))
    sampler.start()
    launches0 = ssa.ssa_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat = []
    for _ in range(args.steps):
        t = time.perf_counter()
        step(f_dev, out_dev, sig_dev)
        lat.append(time.perf_counter() - t)
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed_ms = e0.elapsed_time(e1)
    launches = ssa.ssa_kernel_launches() - launches0
    # per-kernel accounting: the same K steps again with the library's CUDA events around every
    # launch (they cost host and device time per launch, so they stay out of the number above)
    ssa.ssa_stats_enable(True)
    for _ in range(args.steps):
        step(f_dev, out_dev, sig_dev)
    stats = ssa.ssa_stats_get()
    ssa.ssa_stats_enable(False)
    clocks = sampler.stop()
    value, elapsed_s, _ = aggregate(elapsed_ms / 1000.0, args.steps, dist, "cuda")
    elapsed_ms = elapsed_s * 1000.0
    if dist:
        dist.barrier()

    # accuracy against the oracle's stored values
    sig = sig_dev.cpu().numpy()
    gold = read_golden(w.get("golden"))
    sig_err = None
    if gold is not None:
        ref = gold["sigma"][:k]
        sig_err = float(np.max(np.abs(sig - ref) / ref))

    # roofline of the kernel with the most device time
    hbm, peak_kind = peaks()
    # the HBM roofline applies to the kernels that stream HBM bytes; the projected SVD (no HBM
    # traffic, one cluster of CTAs) is named beside it when it takes more time
    cand = [s for s in stats if s["name"] not in ("misc", "skipped") and s["launches"] > 0 and s["bytes"] > 0]
    dom = max(cand, key=lambda s: s["ms"]) if cand else None
    top = max((s for s in stats if s["name"] not in ("misc", "skipped") and s["launches"] > 0),
              key=lambda s: s["ms"], default=None)
    roof = None
    if dom:
        achieved = dom["bytes"] / (dom["ms"] / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": ncu_traffic(dom["name"], dom["bytes"] / dom["launches"]), "kernel": dom["name"],
                "bytes_per_launch": dom["bytes"] / dom["launches"], "ms_per_launch": dom["ms"] / dom["launches"],
                "launches": dom["launches"], "peak_source": peak_kind}
        if top is not None and top["name"] != dom["name"]:
            roof["top_kernel_overall"] = {"kernel": top["name"], "ms_per_launch": top["ms"] / top["launches"],
                                          "bound": "no HBM traffic (latency or arithmetic)"
                                          if top["bytes"] == 0 else "hbm"}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        f_pin = torch.from_numpy(f_host).pin_memory()
        out_pin = torch.empty((k, N), dtype=torch.float64).pin_memory()
        sig_pin = torch.empty(k, dtype=torch.float64).pin_memory()
        n_e2e = max(1, args.steps)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(n_e2e):
            step(f_pin, out_pin, sig_pin)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        e2e_value, _, _ = aggregate(dt, n_e2e, dist, "cuda")
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * N,
               "d2h_bytes_per_step": 8 * k + 8 * k * N}

    # the other settings on the same workload (decomposition + reconstruction): the other precision,
    # and in FP64 the full reorthogonalisation (no skip test) beside the skip test
    name_main = ("f64" if skip == 0 else f"f64_skip{skip:g}") if prec == ssa.SSA_PREC_F64 else "f32c"
    modes = {name_main: {"value": value, "sigma_rel_err_max": sig_err}}
    if not args.no_modes:
        alts = [("f32c", ssa.SSA_PREC_F32C, 0.0, 0), ("f64", ssa.SSA_PREC_F64, 0.0, 0)]
        if args.reorth_skip > 0:
            alts.append((f"f64_skip{args.reorth_skip:g}", ssa.SSA_PREC_F64, args.reorth_skip, 0))
        for name, other, sk, ro in alts:
            if name in modes:
                continue
            plan2 = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=other, seed=rank, stream=stream.cuda_stream,
                                                           reorth_skip=sk, reorth=ro))
            sig2 = torch.empty(k, dtype=torch.float64, device="cuda")

            def step2():
                d, rc = ssa.ssa_decompose(plan2, f_dev, k)
                try:
                    ssa.ssa_reconstruct(d, off_dev, idx_dev, k, out_dev)
                    ssa.ssa_decomp_get(d, sig2, None, None, None)
                finally:
                    ssa.ssa_decomp_destroy(d)

            for _ in range(max(1, args.warmup)):
                step2()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                step2()
            e1.record(stream)
            torch.cuda.synchronize()
            v2, _, _ = aggregate(e0.elapsed_time(e1) / 1000.0, args.steps, dist, "cuda")
            err2 = None
            if gold is not None:
                err2 = float(np.max(np.abs(sig2.cpu().numpy() - gold["sigma"][:k]) / gold["sigma"][:k]))
            ssa.ssa_plan_destroy(plan2)
            modes[name] = {"value": v2, "sigma_rel_err_max": err2}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, int(info.get("restarts", 4)))

    ssa.ssa_plan_destroy(plan)
    dd = min(max(2 * k, k + 32), min(L, K))
    ws_bytes = 2 * (L + K) * (dd + 2) * 8
    l2_note = (f"working set (Lanczos bases, {ws_bytes / 2**30:.2f} GiB) is larger than the 129 MB L2; no flush"
               if ws_bytes > 129e6 else
               f"working set ({ws_bytes / 2**20:.1f} MiB) fits in L2 and is not flushed: an L2-warm small-case timing")
    if rank == 0:
        per_kernel = {s["name"]: {"launches": s["launches"], "ms": round(s["ms"], 3),
                                  "GBps": round(s["bytes"] / (s["ms"] / 1e3) / 1e9, 1) if s["ms"] > 0 else None}
                      for s in stats if s["launches"]}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "df64" if prec == ssa.SSA_PREC_F64 else "f32+df64", "data": "synthetic",
                "config": {"workload": args.workload, "N": N, "L": L, "K": K, "k": k, "groups": "k elementary",
                           "precision": args.precision, "reorth_skip": skip,
                           "parallelism": f"replicas x{world}",
                           "l2": l2_note},
                "sigma_rel_err_max": sig_err, "converged": bool(info.get("converged")),
                "restarts": info.get("restarts"), "matvecs_per_decomp": info.get("matvecs"),
                "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                "modes": modes, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "kernels": per_kernel}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="many_sines_N1M", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="f64", choices=["f64", "f32c"])
    ap.add_argument("--reorth-skip", type=float, default=1e-12,
                    help="FP64: skip level of the reorthogonalisation (0 = full Gram-Schmidt every step)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-modes", action="store_true")
    ap.add_argument("--sample-halfsteps", type=int, default=6)
    ap.add_argument("--cpu-worker", action="store_true")
    ap.add_argument("--precision-batch", default="f32c", choices=["f64", "f32c"],
                    help="precision of the batch and serving workloads")
    ap.add_argument("--serve-pool", type=int, default=256, help="serving: pre-generated series the stream cycles")
    ap.add_argument("--serve-queue", type=int, default=2000, help="serving: most requests outstanding at once")
    ap.add_argument("--serve-latency-s", type=float, default=6.0, help="serving: length of the sustainable-load run")
    ap.add_argument("--serve-batch-n", type=int, default=32768, help="serving: N limit of the batched engine")
    ap.add_argument("--serve-max-batch", type=int, default=128, help="serving: requests per batched launch at most")
    ap.add_argument("--seq-sample", type=int, default=0,
                    help="serving: pool entries timed one after another in FP64 (0 = all of them)")
    ap.add_argument("--serve-workers", type=int, default=16, help="serving: single-series workers (streams)")
    ap.add_argument("--serve-connections", type=int, default=32,
                    help="serving: CUDA_DEVICE_MAX_CONNECTIONS (hardware work queues) unless already set")
    ap.add_argument("--serve-grid-cap", type=int, default=0,
                    help="serving: CTAs per persistent kernel of a request (0 = the whole device)")
    ap.add_argument("--serve-batch-workers", type=int, default=1, help="serving: batched-launch workers")
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS[args.workload].get("kind") == "serving":
        # 16 single-series streams share 8 hardware work queues by default; read when the CUDA
        # context is created, so set before the first CUDA call of this process
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", str(args.serve_connections))
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
