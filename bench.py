#!/usr/bin/env python3
"""CPAA PageRank benchmark on one GB300 per rank.

Workload (default): Chung-Lu power-law undirected graph, n = 2^24 vertices,
256M distinct undirected edges (the first 2.56e8 distinct pairs drawn,
exponent 2.1, seed 0) plus a Hamiltonian ring, symmetric int32 CSR (about
545M entries); damping c = 0.85; uniform p = 1/n; stop when the rigorous L1
bound is below 1e-6.  One step = one full cpaa_solve in FP64, the paper's
arithmetic (prep, kappa, M fused recurrence rounds, finalisation), on inputs
already resident in HBM.  The CSR (about 2.2 GB of column indices) is far
larger than the 126 MB L2, so no extra L2 flush is needed between steps.
The same solve in FP32 and in double-float (DF64) is timed as named legs of
the same line.

Printed: one JSON line (rank 0).  ``value`` is GTEPS = nnz x rounds / s over
all ranks; ``e2e`` is the same through the C ABI with host buffers (H2D of p
and D2H of pi inside the timed region); ``roofline`` is for the step kernel,
timed live with CUDA events on the solve's stream; ``cpu_baseline`` is the
FP64 oracle on the host cores on a bounded sample of the same graph.

``--impl reference`` times the FP64 CPU oracle alone (this method has no
other reference implementation) on the same workload and prints its line.
Multi-GPU runs (torchrun) are independent replicas: the method's rounds need
the whole graph, and one graph fits one GPU.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CPAA GTEPS (% HBM roofline); time to 1e-6 L1 vs plain FP64 on same GB300"

WORKLOADS = {
    "chung_lu_16M": dict(n=1 << 24, edges=256_000_000, distinct=True, gamma=2.1, seed=0, c=0.85, tol=1e-6,
                         desc="Chung-Lu power-law graph (exponent 2.1, seed 0), n=2^24 (16.7M) vertices, "
                              "256M distinct undirected edges + ring; c=0.85, uniform p, tol 1e-6 L1"),
    "chung_lu_10k": dict(n=10_000, edges=100_000, gamma=2.1, seed=0, c=0.85, tol=1e-10,
                         desc="Chung-Lu n=10000, 1e5 pair draws, gamma=2.1, seed 0, + ring; "
                              "c=0.85, uniform p, tol 1e-10"),
    "chung_lu_4M": dict(n=1 << 22, edges=64_000_000, distinct=True, gamma=2.1, seed=0, c=0.85, tol=1e-6,
                        desc="Chung-Lu n=2^22, 64M distinct undirected edges, gamma=2.1, seed 0, + ring; "
                             "c=0.85, uniform p, tol 1e-6 L1"),
    "chung_lu_1M": dict(n=1 << 20, edges=16_000_000, gamma=2.1, seed=0, c=0.85, tol=1e-6,
                        desc="Chung-Lu n=2^20, 1.6e7 pair draws, gamma=2.1, seed 0, + ring; "
                             "c=0.85, uniform p, tol 1e-6 L1"),
    "chung_lu_16M_shuffled": dict(n=1 << 24, edges=256_000_000, distinct=True, gamma=2.1, seed=0, c=0.85,
                                  tol=1e-6, shuffle=1,
                                  desc="Chung-Lu n=2^24 as chung_lu_16M, vertex ids randomly permuted "
                                       "(seed 1); c=0.85, uniform p, tol 1e-6 L1"),
    "grid_4096": dict(rows=4096, cols=4096, frac=0.2, seed=0, c=0.85, tol=1e-6,
                      desc="4096x4096 lattice, 20% of edges deleted (seed 0, spanning tree kept); "
                           "c=0.85, uniform p, tol 1e-6 L1"),
}

PREC = {"f64": 0, "f32": 1, "bf16": 2, "df64": 3}
VB = {"f64": 8, "f32": 4, "bf16": 2, "df64": 8}


def alg_bytes_per_round(n, nnz, prec):
    """Algorithmic bytes one round must move: column indices 4 nnz, row
    pointers 4 (n+1), one degree word 4 n, the gathered vector once (vb n),
    the old iterate read and the new one written (2 vb n), the accumulator
    read-modify-write (2 vr n) and, for the FP32/BF16 forms, the Kahan
    compensation read-modify-write (8 n)."""
    vb = VB[prec]
    vr = 8 if prec in ("f64", "df64") else 4
    kahan = 0 if prec in ("f64", "df64") else 8
    return 4 * nnz + 4 * (n + 1) + 4 * n + 3 * vb * n + 2 * vr * n + kahan * n


# -- distributed plumbing (replicas) --------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world, use_cuda):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if use_cuda else "gloo")


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world, device="cpu"):
    """Max of a float over all ranks (identity when world == 1)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, world, device="cpu"):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# -- clocks ----------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
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
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -- inputs -----------------------------------------------------------------------

def make_graph(wl, device):
    import cpaa_inputs as ci
    w = WORKLOADS[wl]
    t = time.time()
    if "rows" in w:
        g = ci.grid_deleted(w["rows"], w["cols"], w["frac"], seed=w["seed"], device=device)
    else:
        g = ci.chung_lu(w["n"], w["edges"], gamma=w["gamma"], seed=w["seed"], device=device,
                        distinct=w.get("distinct", False))
        if w.get("shuffle"):
            g = ci.shuffled(g, seed=w["shuffle"])
    return g, time.time() - t


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def step_kernel_hash():
    """Hash of the round kernel's source (its implementation header and the
    per-row arithmetic it includes)."""
    h = hashlib.sha256()
    for name in ("step_impl.cuh", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_2112_01743_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(prec, wl):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when there is none or the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "cheb_step_%s_%s.md" % (prec, wl))
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_src_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != step_kernel_hash():
        return None
    return float(m.group(1))


# -- CPU oracle leg ------------------------------------------------------------------

def oracle_sample(rp, cx, rounds, threads):
    """Time the FP64 oracle for ``rounds`` rounds on the full graph."""
    from oracle import oracle as O
    n = len(rp) - 1
    p = np.full(n, 1.0 / n)
    O.lib()
    t = time.perf_counter()
    O.cpaa(rp, cx, p, 0.85, rounds, nthreads=threads)
    dt = time.perf_counter() - t
    return dt


# -- main arms ----------------------------------------------------------------------

def run_batch(pkg, args, stream):
    """256 personalised vectors (1-16 uniform seeds each) on the 4M-vertex
    Chung-Lu graph, c = 0.85, tol 1e-6: cpaa_solve_batch in FP32 against the
    plain FP64 single-vector solve, per query (time to the same L1 bound)."""
    import torch
    import cpaa_inputs as ci
    g = ci.chung_lu(1 << 22, 64_000_000, seed=0, device="cuda", distinct=True)
    n, nnz = g.n, g.nnz
    G = pkg.Graph(g.row_ptr, g.col_idx, n=n, autotune=not args.no_autotune,
                  layout={"tune_precision": pkg.CPAA_F32})
    blayout = {k: v for k, v in G.layout().items()
               if k in ("hub_degree", "hub_tile", "long_chunk", "sort_window", "tuned", "tune_candidates")}
    del g
    B = 256
    seeds = ci.seed_vectors(n, B, max_seeds=16, seed=0)
    P = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    for b, (s, w) in enumerate(seeds):
        P[b, torch.as_tensor(s.astype(np.int64), device="cuda")] = torch.as_tensor(w, device="cuda")
    PI = torch.empty_like(P)
    cs = np.full(B, 0.85)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = G.solve_batch(B, P, cs, 1e-6, PI, precision=pkg.CPAA_F32)  # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    infos = G.solve_batch(B, P, cs, 1e-6, PI, precision=pkg.CPAA_F32)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1)
    # the same batch under the a-posteriori stopping rule
    PI2 = torch.empty_like(P)
    G.solve_batch(B, P, cs, 1e-6, PI2, precision=pkg.CPAA_F32, stop_rule=pkg.CPAA_STOP_POSTERIORI)
    torch.cuda.synchronize()
    e0.record(stream)
    infos2 = G.solve_batch(B, P, cs, 1e-6, PI2, precision=pkg.CPAA_F32, stop_rule=pkg.CPAA_STOP_POSTERIORI)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch2 = e0.elapsed_time(e1)
    d12 = float((PI2 - PI).abs().sum(dim=1).max().item())
    del PI2
    # plain FP64 single-vector form on a sample of the same queries
    sample = list(range(0, B, 16))
    pi = torch.empty((n,), dtype=torch.float64, device="cuda")
    G.solve(P[0], 0.85, 1e-6, pi, precision=pkg.CPAA_F64)
    torch.cuda.synchronize()
    e0.record(stream)
    for b in sample:
        G.solve(P[b], 0.85, 1e-6, pi, precision=pkg.CPAA_F64)
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1) / len(sample)
    l1 = float((PI[sample[-1]] - pi).abs().sum().item())
    G.close()
    rounds = [i.rounds for i in infos]
    rounds2 = [i.rounds for i in infos2]
    return {"workload": "Chung-Lu n=2^22, 64M distinct undirected edges, gamma=2.1, seed 0, + ring; 256 "
                        "vectors uniform over 1-16 seeds; c=0.85; tol 1e-6 L1",
            "n": n, "nnz": nnz, "B": B, "precision": "f32", "layout": blayout,
            "ms_batch": t_batch, "ms_per_query_batched_f32": t_batch / B,
            "ms_per_query_single_f64": t_single,
            "speedup_batched_f32_vs_single_f64": t_single / (t_batch / B),
            "effective_gteps": nnz * sum(rounds) / (t_batch * 1e-3) / 1e9,
            "rounds_min_max": [min(rounds), max(rounds)],
            "l1_batched_f32_vs_single_f64_last_sample": l1,
            "posteriori": {"ms_per_query_batched_f32": t_batch2 / B,
                           "speedup_vs_single_f64": t_single / (t_batch2 / B),
                           "rounds_min_max": [min(rounds2), max(rounds2)],
                           "rounds_mean": float(np.mean(rounds2)), "rigorous_rounds_mean": float(np.mean(rounds)),
                           "max_l1_vs_rigorous": d12}}


def run_small(pkg, args, stream):
    """The 10,000-vertex Chung-Lu graph in FP64, uniform p, run until Eq. 41's
    ERR_M < 1e-10 (39 rounds at c = 0.85): it fits in L2, so this is a latency
    figure (time per solve and per round), not a bandwidth one."""
    import torch
    import cpaa_inputs as ci
    g = ci.chung_lu(10_000, 100_000, seed=0, device="cuda")
    G = pkg.Graph(g.row_ptr, g.col_idx, n=g.n)
    n, nnz = g.n, g.nnz
    p = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    pi = torch.empty_like(p)
    M = 39
    for _ in range(5):
        G.solve(p, 0.85, 0.0, pi, fixed_rounds=M, precision=pkg.CPAA_F64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    infos = [G.solve(p, 0.85, 0.0, pi, fixed_rounds=M, precision=pkg.CPAA_F64, time_rounds=True)
             for _ in range(reps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    G.close()
    return {"workload": "Chung-Lu n=10000, 1e5 pair draws, gamma 2.1, seed 0, + ring; FP64; c=0.85; "
                        "uniform p; 39 rounds (ERR_M < 1e-10)", "n": n, "nnz": nnz, "rounds": M,
            "ms_per_solve": ms, "us_per_round": 1e3 * sum(i.rounds_ms for i in infos) / (M * reps),
            "gteps": nnz * M / (ms * 1e-3) / 1e9}


def run_grid(pkg, args, stream):
    """Precision study on the 4096 x 4096 lattice with 20% of its edges deleted
    (spanning tree kept), c = 0.85, uniform p, tol 1e-6: FP64, FP32 and BF16
    storage, each timed and compared with the FP64 result."""
    import torch
    import cpaa_inputs as ci
    g = ci.grid_deleted(4096, 4096, 0.2, seed=0, device="cuda")
    n, nnz = g.n, g.nnz
    G = pkg.Graph(g.row_ptr, g.col_idx, n=n)
    del g
    p = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    out = {}
    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, prec in (("f64", pkg.CPAA_F64), ("f32", pkg.CPAA_F32), ("bf16", pkg.CPAA_BF16),
                       ("df64", pkg.CPAA_DF64)):
        pi = torch.empty_like(p)
        for _ in range(3):
            G.solve(p, 0.85, 1e-6, pi, precision=prec)
        torch.cuda.synchronize()
        e0.record(stream)
        infos = [G.solve(p, 0.85, 1e-6, pi, precision=prec, time_rounds=True) for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        rms = sum(i.rounds_ms for i in infos) / sum(i.rounds for i in infos)
        res[name] = pi
        out[name] = {"ms_per_solve": ms, "rounds": infos[0].rounds, "round_ms": rms,
                     "gteps": nnz * infos[0].rounds / (ms * 1e-3) / 1e9,
                     "hbm_frac_of_measured": alg_bytes_per_round(n, nnz, name) / (rms * 1e-3) / 1e9
                     / measured_peak_gbs()[0]}
    for name in ("f32", "bf16", "df64"):
        out[name]["l1_vs_f64"] = float((res[name] - res["f64"]).abs().sum().item())
    out["frontier_one_seed_f64"] = one_seed_frontier(pkg, G, n, pkg.CPAA_F64, reps=10)
    G.close()
    del G
    torch.cuda.empty_cache()
    # the series on [lambda_lo, 1]: the same lattice with a self-loop on every
    # vertex certifies lambda_lo = -1 + 2/d_max = -0.6
    gl = ci.with_self_loops(ci.grid_deleted(4096, 4096, 0.2, seed=0, device="cuda"))
    GL = pkg.Graph(gl.row_ptr, gl.col_idx, n=gl.n)
    del gl
    iv = {"workload": "the same lattice with a self-loop on every vertex; c=0.85, uniform p, tol 1e-6",
          "lambda_lo_certified": GL.spectrum_bound()}
    for prec_name in ("f64", "f32", "df64"):
        ivp = {}
        piv = {}
        for name, cert in (("plain", False), ("interval", True)):
            pi = torch.empty_like(p)
            for _ in range(3):
                GL.solve(p, 0.85, 1e-6, pi, precision=PREC[prec_name], certify_interval=cert)
            torch.cuda.synchronize()
            e0.record(stream)
            infos = [GL.solve(p, 0.85, 1e-6, pi, precision=PREC[prec_name], certify_interval=cert, time_rounds=True)
                     for _ in range(args.steps)]
            e1.record(stream)
            torch.cuda.synchronize()
            ivp[name] = {"rounds": infos[0].rounds, "ms_per_solve": e0.elapsed_time(e1) / args.steps,
                         "round_ms": sum(i.rounds_ms for i in infos) / sum(i.rounds for i in infos),
                         "bound": infos[0].bound, "lambda_lo": infos[0].lambda_lo}
            piv[name] = pi
        ivp["l1_interval_vs_plain"] = float((piv["interval"] - piv["plain"]).abs().sum().item())
        ivp["speedup"] = ivp["plain"]["ms_per_solve"] / ivp["interval"]["ms_per_solve"]
        iv[prec_name] = ivp
    out["interval_looped"] = iv
    GL.close()
    return {"workload": "4096x4096 lattice, 20% of edges deleted (seed 0, spanning tree kept); "
                        "c=0.85, uniform p, tol 1e-6", "n": n, "nnz": nnz, **out}


def one_seed_frontier(pkg, G, n, precision, reps=20, c=0.85, tol=1e-6):
    """Mean device time of one-seed solves (seeds spread over the id range)
    with and without CPAA_SPARSE_FRONTIER, and whether the results agree bit
    for bit."""
    import torch
    seeds = np.linspace(0, n - 1, reps).astype(np.int64)
    out = {}
    res = {}
    for fr in (False, True):
        p = torch.zeros(n, dtype=torch.float64, device="cuda")
        pi = torch.empty_like(p)
        p[int(seeds[0])] = 1.0
        G.solve(p, c, tol, pi, precision=precision, frontier=fr)  # warm-up (and graph capture)
        torch.cuda.synchronize()
        ms = []
        last = None
        for sd in seeds:
            p.zero_()
            p[int(sd)] = 1.0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            info = G.solve(p, c, tol, pi, precision=precision, frontier=fr)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            last = info.rounds
        res[fr] = pi.clone()
        out["frontier" if fr else "plain"] = {"ms_per_solve_mean": float(np.mean(ms)),
                                             "ms_per_solve_median": float(np.median(ms)), "rounds_last": last}
    out["same_bits"] = bool(torch.equal(res[False], res[True]))
    out["speedup"] = out["plain"]["ms_per_solve_mean"] / out["frontier"]["ms_per_solve_mean"]
    return out


def run_serving(pkg, args):
    """Continuous-batching server over 8 resident Chung-Lu graphs (10k..8M
    vertices, mean degree 16).  Queries: a uniform graph, 1-16 distinct uniform
    seeds, c uniform over {0.5, 0.85, 0.95}, tol 1e-6.  First a closed loop with
    512 queries outstanding gives the saturated rate; then an open-loop Poisson
    stream at 0.7 x that rate, and shorter streams at 0.3, 0.5 and 0.9 x it;
    latency = submit -> result ready (server side)."""
    import threading
    import torch
    import cpaa_inputs as ci
    sizes = [10_000, 50_000, 200_000, 500_000, 1_000_000, 2_000_000, 4_000_000, 8_000_000]
    G = []
    for i, n in enumerate(sizes):
        g = ci.chung_lu(n, 8 * n, seed=100 + i, device="cuda")
        G.append(pkg.Graph(g.row_ptr, g.col_idx, n=g.n))
        del g
    torch.cuda.empty_cache()
    nnz_total = sum(x.nnz for x in G)
    rng = np.random.default_rng(0)

    def make(count):
        out = []
        for _ in range(count):
            gi = int(rng.integers(len(sizes)))
            k = int(rng.integers(1, 17))
            seeds = rng.choice(sizes[gi], size=k, replace=False).astype(np.int32)
            out.append((gi, seeds, float(rng.choice([0.5, 0.85, 0.95]))))
        return out

    def run(queries, rate, stop_rule=pkg.CPAA_STOP_RIGOROUS, fused=False, frontier=False):
        S = pkg.Server(64 << 30, stop_rule=stop_rule, fused=fused, frontier=frontier)
        ids = [S.add_graph(x, 16) for x in G]
        tickets = []
        lock = threading.Condition()
        done = {"n": 0, "t_last": 0.0, "entries": 0}

        def consumer():
            i = 0
            while i < len(queries):
                with lock:
                    while i >= len(tickets):
                        lock.wait()
                    t = tickets[i]
                _, info = S.wait(t, None)
                done["entries"] += G[queries[i][0]].nnz * info.rounds
                i += 1
                done["n"] = i
                done["t_last"] = time.perf_counter()

        th = threading.Thread(target=consumer)
        th.start()
        t0 = time.perf_counter()
        if rate is None:  # closed loop: at most 512 outstanding
            for q in queries:
                while len(tickets) - done["n"] >= 512:
                    time.sleep(50e-6)
                t = S.submit(ids[q[0]], q[1], None, q[2], 1e-6)
                with lock:
                    tickets.append(t)
                    lock.notify()
        else:
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(queries)))
            for q, ta in zip(queries, arrivals):
                dt = t0 + ta - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                t = S.submit(ids[q[0]], q[1], None, q[2], 1e-6)
                with lock:
                    tickets.append(t)
                    lock.notify()
        th.join()
        st = S.stats()
        S.close()
        st["effective_gteps"] = done["entries"] / (done["t_last"] - t0) / 1e9
        st["mean_width"] = st["round_columns"] / max(1, st["rounds"])
        return len(queries) / (done["t_last"] - t0), st

    sat_queries = make(args.serve_queries // 4)
    sat_qps, sat_st = run(sat_queries, None)
    post_qps, post_st = run(sat_queries, None, pkg.CPAA_STOP_POSTERIORI)
    fused_qps, fused_st = run(sat_queries, None, pkg.CPAA_STOP_RIGOROUS, True)
    rate = 0.7 * sat_qps
    qps, st = run(make(args.serve_queries), rate)
    sweep = []
    for load in (0.3, 0.5, 0.7, 0.9):
        if load == 0.7:
            q, s = qps, st
            count = args.serve_queries
        else:
            count = max(1, args.serve_queries // 8)
            q, s = run(make(count), load * sat_qps)
        sweep.append({"load": load, "rate_qps": load * sat_qps, "queries": count, "achieved_qps": q,
                      "p50_ms": s["p50_us"] / 1e3, "p99_ms": s["p99_us"] / 1e3,
                      "mean_width": s["mean_width"], "relayouts": s["relayouts"],
                      "failed": s["failed"]})
    # the sparse frontier (early rounds on the seeds' k-hop balls) at low load,
    # where tiles often start from empty
    frontier_sweep = []
    for load in (0.3, 0.5):
        count = max(1, args.serve_queries // 8)
        q, s_ = run(make(count), load * sat_qps, frontier=True)
        frontier_sweep.append({"load": load, "rate_qps": load * sat_qps, "queries": count, "achieved_qps": q,
                               "p50_ms": s_["p50_us"] / 1e3, "p99_ms": s_["p99_us"] / 1e3,
                               "mean_width": s_["mean_width"], "failed": s_["failed"]})
    # one-seed solves on the 8M-vertex graph with and without the frontier
    frontier_solve = one_seed_frontier(pkg, G[-1], sizes[-1], pkg.CPAA_F32)
    for x in G:
        x.close()
    return {"workload": "8 Chung-Lu graphs (n = 10k..8M, mean degree 16, gamma 2.1) resident; "
                        "queries: uniform graph, 1-16 seeds, c in {0.5, 0.85, 0.95}, tol 1e-6; "
                        "FP32, 16 slots per graph",
            "nnz_total": nnz_total, "queries": args.serve_queries,
            "saturated_qps": sat_qps, "poisson_rate_qps": rate, "achieved_qps": qps,
            "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3, "mean_ms": st["mean_us"] / 1e3,
            "admit_p50_ms": st["admit_p50_us"] / 1e3, "saturated_p50_ms": sat_st["p50_us"] / 1e3,
            "saturated_p99_ms": sat_st["p99_us"] / 1e3,
            "saturated_effective_gteps": sat_st["effective_gteps"],
            "saturated_mean_width": sat_st["mean_width"], "completed": st["completed"],
            "failed": st["failed"],
            "posteriori_saturated_qps": post_qps, "posteriori_saturated_p50_ms": post_st["p50_us"] / 1e3,
            "posteriori_saturated_p99_ms": post_st["p99_us"] / 1e3,
            "fused_saturated_qps": fused_qps, "fused_saturated_p50_ms": fused_st["p50_us"] / 1e3,
            "fused_saturated_p99_ms": fused_st["p99_us"] / 1e3,
            "fused_saturated_effective_gteps": fused_st["effective_gteps"],
            "poisson_sweep": sweep, "frontier_poisson_sweep": frontier_sweep,
            "frontier_one_seed_8M_f32": frontier_solve}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    if dev == "cuda":
        torch.cuda.set_device(local)
    g, _ = make_graph(args.workload, dev)
    rp, cx = g.numpy()
    n, nnz = g.n, g.nnz
    del g
    threads = os.cpu_count() or 1
    rounds = args.ref_rounds
    for _ in range(args.warmup):
        oracle_sample(rp, cx, rounds, threads)
    times = [oracle_sample(rp, cx, rounds, threads) for _ in range(args.steps)]
    tot = sum(times)
    value = nnz * rounds * len(times) / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "n": n, "nnz": nnz,
                   "rounds_per_step": rounds},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": threads, "kind": "oracle",
                         "sample": "%d round(s) of the FP64 oracle recurrence on the full graph "
                                   "per step" % rounds},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dist_init(world, True)
    import paper_2112_01743_gb300 as pkg
    wl = WORKLOADS[args.workload]
    prec = args.precision

    g, gen_s = make_graph(args.workload, "cuda")
    n, nnz = g.n, g.nnz
    t = time.time()
    # layout parameters picked by the library's autotuner, timed in the main precision
    G = pkg.Graph(g.row_ptr, g.col_idx, n=n, validate=True, autotune=not args.no_autotune,
                  layout={"tune_precision": PREC[prec]})
    create_s = time.time() - t
    layout = G.layout()
    cpu_graph = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_graph = g.numpy()
    del g
    torch.cuda.empty_cache()

    p = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    pi = torch.empty_like(p)
    stream = torch.cuda.current_stream()

    def solve(precision, time_rounds=True):
        return G.solve(p, wl["c"], wl["tol"], pi, precision=PREC[precision],
                       time_rounds=time_rounds)

    # ---- main timed region (device-resident inputs).  The clock sampler starts
    # before the warm-up so that its own start-up is not inside the timed region.
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    for _ in range(max(args.warmup, 3)):
        solve(prec)
    torch.cuda.synchronize()
    clocks.lines.clear()  # keep only the samples taken during the timed region
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0.record(stream)
    infos = []
    for i in range(args.steps):
        marks[i].record(stream)
        infos.append(solve(prec))
    marks[-1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)]
    barrier(world)
    clk = clocks.stop()
    local_ms = e0.elapsed_time(e1)
    ms_total = reduce_max(local_ms, world, "cuda")
    rounds = infos[0].rounds
    units = reduce_sum(sum(nnz * i.rounds for i in infos), world, "cuda")
    value = units / (ms_total * 1e-3) / 1e9
    pi_main = pi.clone()
    round_ms = sum(i.rounds_ms for i in infos) / sum(i.rounds for i in infos)
    ab = alg_bytes_per_round(n, nnz, prec)
    peak, peak_kind = measured_peak_gbs()
    achieved = ab / (round_ms * 1e-3) / 1e9

    # ---- the other number formats on the same graph and tolerance: FP32 (the
    # 1e-6-relative path, time to the same L1 bound as the plain FP64 form) and
    # DF64 (FP64-class accuracy on the FP32 pipes); FP64 when the main line is not
    legs = {}
    if not args.skip_legs:
        for name in ("f64", "f32", "df64"):
            if name == prec:
                continue
            out = torch.empty_like(p)
            for _ in range(3):
                G.solve(p, wl["c"], wl["tol"], out, precision=PREC[name])
            torch.cuda.synchronize()
            e0.record(stream)
            inf = [G.solve(p, wl["c"], wl["tol"], out, precision=PREC[name], time_rounds=True)
                   for _ in range(args.steps)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            r = sum(i.rounds_ms for i in inf) / sum(i.rounds for i in inf)
            legs[name] = {"ms_per_solve": ms, "rounds": inf[0].rounds, "round_ms": r,
                          "gteps": nnz * inf[0].rounds / (ms * 1e-3) / 1e9,
                          "hbm_frac_of_measured": alg_bytes_per_round(n, nnz, name) / (r * 1e-3) / 1e9 / peak,
                          "l1_vs_%s" % prec: float((out - pi_main).abs().sum().item()),
                          "speedup_vs_%s" % prec: (ms_total / args.steps) / ms}
            del out

    # ---- the paper's comparison: power method (SPI) on the same kernels, same L1 bound
    power = None
    if not args.skip_power:
        power = {}
        for name in ("f64", "f32"):
            pp = torch.empty_like(p)
            G.power_solve(p, wl["c"], wl["tol"], pp, precision=PREC[name])
            torch.cuda.synchronize()
            e0.record(stream)
            pinf = [G.power_solve(p, wl["c"], wl["tol"], pp, precision=PREC[name]) for _ in range(args.steps)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms_pow = e0.elapsed_time(e1) / args.steps
            ms_cheb = (ms_total / args.steps) if name == prec else (legs[name]["ms_per_solve"] if name in legs
                                                                   else None)
            power[name] = {"rounds": pinf[0].rounds, "ms_per_solve": ms_pow,
                           "cpaa_rounds": rounds if name == prec else (legs[name]["rounds"] if name in legs
                                                                       else None),
                           "cpaa_ms_per_solve": ms_cheb,
                           "cpaa_speedup": (ms_pow / ms_cheb) if ms_cheb else None,
                           "l1_vs_cpaa_same_precision": float((pp - pi_main).abs().sum().item()) if name == prec else None}

    # ---- end to end through the C ABI with host buffers (pinned)
    hp = torch.full((n,), 1.0 / n, dtype=torch.float64).pin_memory()
    hpi = torch.empty((n,), dtype=torch.float64).pin_memory()
    for _ in range(2):
        G.solve(hp, wl["c"], wl["tol"], hpi, precision=PREC[prec])
    barrier(world)
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2e_units = 0
    for _ in range(args.steps):
        ii = G.solve(hp, wl["c"], wl["tol"], hpi, precision=PREC[prec])
        e2e_units += nnz * ii.rounds
    e2e_s = reduce_max(time.perf_counter() - t, world, "cuda")
    e2e_units = reduce_sum(e2e_units, world, "cuda")
    e2e = {"value": e2e_units / e2e_s / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n}

    # ---- batched personalised queries (the 4M-vertex, 256-vector configuration)
    batch = None
    if not args.skip_batch:
        del G
        torch.cuda.empty_cache()
        batch = run_batch(pkg, args, stream)
        G = None

    # ---- the 10k-vertex FP64 configuration (latency)
    small = None
    if not args.skip_grid:
        small = run_small(pkg, args, stream)

    # ---- precision study on the lattice
    grid = None
    if not args.skip_grid:
        if G is not None:
            del G
            G = None
        torch.cuda.empty_cache()
        grid = run_grid(pkg, args, stream)

    # ---- serving: continuous batching over 8 resident graphs
    serving = None
    if not args.skip_serve:
        if G is not None:
            del G
            G = None
        torch.cuda.empty_cache()
        serving = run_serving(pkg, args)

    # ---- CPU oracle baseline on a bounded sample
    cpu = None
    if cpu_graph is not None:
        rp, cx = cpu_graph
        threads = os.cpu_count() or 1
        dt = oracle_sample(rp, cx, args.ref_rounds, threads)
        cpu = {"value": nnz * args.ref_rounds / dt / 1e9, "unit": "GTEPS", "cores": threads,
               "kind": "oracle",
               "sample": "%d round(s) of the FP64 oracle recurrence on the full graph (%.1f s)"
                         % (args.ref_rounds, dt)}

    if G is not None:
        G.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
        "data": "synthetic",
        "config": {"workload": wl["desc"], "n": n, "nnz": nnz, "rounds": rounds,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (col_idx %.2f GB), no flush" % (4 * nnz / 1e9),
                   "graph_gen_s": round(gen_s, 2), "graph_create_s": round(create_s, 2),
                   "layout": {k: layout[k] for k in ("hub_degree", "hub_tile", "long_chunk", "sort_window",
                                                     "tuned", "tune_candidates")},
                   "step_ms": [round(x, 3) for x in step_ms]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(prec, args.workload),
                     "kernel": "cheb_step_kernel<%s>" % prec, "alg_bytes_per_launch": ab,
                     "avg_launch_ms": round_ms, "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        # per solve: stats + its block sum, prep, the rounds, the last round's two
        # fixed-order sum kernels, the normaliser's two kernels and the finalisation
        "gpu_launches": sum(i.rounds + 8 for i in infos),
        "legs": legs,
        "power": power,
        "batch": batch,
        "small": small,
        "grid": grid,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="chung_lu_16M")
    ap.add_argument("--precision", choices=sorted(PREC), default="f64",
                    help="number format of the main line (default: FP64, the paper's)")
    ap.add_argument("--ref-rounds", type=int, default=2,
                    help="oracle rounds per CPU sample (bounded CPU work)")
    ap.add_argument("--skip-legs", action="store_true", help="skip the other number formats")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-grid", action="store_true")
    ap.add_argument("--skip-power", action="store_true")
    ap.add_argument("--serve-queries", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default layout parameters")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
