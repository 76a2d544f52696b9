#!/usr/bin/env python
"""Throughput of BSGD-TV epochs on one GB300 (or N independent ones).

A step is one epoch of Algorithm 1 (fused block products, reductions, step and
the FGP TV prox) on the 512x512 workload: 30-ellipse phantom, parallel beam
with 360 angles x 727 bins (A has 1.2e8 nonzeros, 0.96 GB as FP32 values +
int32 indices), M = N = 8 blocks, lambda = 0.02, 50 FGP iterations.  The
inputs (A) are larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  With torchrun (N > 1) every rank reconstructs its own
slice (weak scaling, no data exchange); the elapsed time is the max over
ranks.  --impl reference times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "BSGD-TV epochs/s + HBM GB/s (fused Ax,Aᵀr,TV-prox); served p50/p99 latency"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "products_ellipse512.md")
TRAFFIC_SOURCES = ["paper_1812_01307_gb300/csrc/products.cu", "paper_1812_01307_gb300/csrc/products_common.cuh",
                   "paper_1812_01307_gb300/csrc/layout.cpp", "paper_1812_01307_gb300/csrc/layout.h"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ellipse512")
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-slices", type=int, default=64,
                    help="slices of the batched variant (many slices sharing one A); 0 skips it")
    ap.add_argument("--served-requests", type=int, default=400,
                    help="requests of the served stream (0 skips it); the configuration's stream has "
                         "2000, the default times its first 400")
    ap.add_argument("--served-small", action="store_true",
                    help="leave the 1024x1024 requests (p = 0.1) out of the served stream")
    ap.add_argument("--served-budget-gb", type=float, default=64.0)
    ap.add_argument("--served-pack", type=int, default=1,
                    help="geometries a server group may pack into one set of launches (1: none)")
    ap.add_argument("--served-pack-ratio", type=float, default=4.0,
                    help="largest ratio of nonzeros between geometries packed into one group")
    ap.add_argument("--served-tick", type=int, default=10, help="max epochs between admissions")
    ap.add_argument("--served-rate", type=float, default=0.0,
                    help="Poisson arrival rate of the served stream, requests/s (0: 0.7x the saturated rate)")
    ap.add_argument("--served-priority", type=int, default=1,
                    help="1: groups of smaller geometries on higher-priority streams; 0: all equal")
    ap.add_argument("--served-slots", type=int, default=0,
                    help="slots per group for every geometry (0: the L2 rule, 32 at most)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip every variant (stored formats and the batch)")
    ap.add_argument("--variants", default="f32_i16,f16_i16,bf16_i16,batch,batch_f16,matrix_free,stochastic",
                    help="comma-separated variants to run: f32_i16, f16_i16, bf16_i16, batch, batch_f16, "
                         "matrix_free, stochastic")
    ap.add_argument("--mf-n", type=int, default=2048, help="image size of the matrix-free variant")
    ap.add_argument("--batch-tuning", default="",
                    help="FGP iterations per launch and slices per FGP group for the batch, "
                         "e.g. 5,9 (default: autotune)")
    return ap.parse_args()


def workload_desc(wl):
    return (f"{wl.name}: {wl.n}x{wl.n} image, {wl.n_ellipses} ellipses, parallel beam "
            f"{wl.n_angles} angles x {wl.n_bins} bins, M=N={wl.M}, lambda={wl.lam}, "
            f"{wl.fgp_iters} FGP iterations per epoch, x0=0")


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def samples(self):
        """Rows written so far (0 if the sampler is not running)."""
        if self.proc is None or not self.path:
            return 0
        try:
            self.f.flush()
            with open(self.path) as f:
                return sum(1 for line in f if line.count(",") >= 8)
        except OSError:
            return 0

    def wait_samples(self, n, limit_s, work=None):
        """Until at least n rows exist (at most limit_s seconds), calling
        work() meanwhile (e.g. untimed epochs that keep the GPU loaded)."""
        t0 = time.perf_counter()
        while self.proc is not None and self.samples() < n and time.perf_counter() - t0 < limit_s:
            if work is not None:
                work()
            else:
                time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, fl in enumerate(flags)
                          if fl.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profiled_traffic():
    """DRAM bytes per launch of the product kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    prof = {}
    try:
        with open(PROFILE_TRAFFIC) as f:
            for line in f:
                if ":" in line and not line.startswith(("#", "|", " ")):
                    k, v = line.split(":", 1)
                    prof[k.strip()] = v.strip()
    except OSError:
        return None
    if prof.get("source_sha256") != kernel_source_hash() or "dram_bytes_per_launch" not in prof:
        return None
    return int(prof["dram_bytes_per_launch"])


def kernel_source_hash():
    """sha256 of the product kernel's sources with comments and blank space
    removed (a comment-only edit does not change the kernel)."""
    import re
    h = hashlib.sha256()
    for p in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, p)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()


# ------------------------------------------------------------- served stream
def served_stream(args, B, synth):
    """Continuous batching under a Poisson stream of reconstruction requests:
    image n in {128, 256, 512, 1024} with p = .4, .3, .2, .1 (1024 left out,
    the rest renormalised, under --served-small), angles = round(0.7 n), bins =
    ceil(sqrt(2) n) + 1, lambda ~ U(0.01, 0.1), epochs ~ U{100..300}, 30 FGP
    iterations, FP16 weights, A cached per geometry.  Phase 1 submits every
    request at once (saturated throughput); phase 2 replays them with Poisson
    arrivals at 0.7x that rate.  Latency = submit -> x in host memory."""
    import math
    import threading

    import numpy as np
    full = not getattr(args, "served_small", False)
    sizes = [128, 256, 512] + ([1024] if full else [])
    probs = np.array([0.4, 0.3, 0.2] + ([0.1] if full else []))
    probs = probs / probs.sum()
    ellipses = {128: 10, 256: 20, 512: 30, 1024: 40}
    K, N, pool = 30, args.served_requests, 8
    rng = np.random.default_rng(2024)
    budget = int(args.served_budget_gb * 2 ** 30)
    t_setup = time.perf_counter()
    geoms = {}
    slots_of = {}

    def slot_cap(n, rows):
        # slots per group: the server's own rule (0) unless --served-slots
        # fixes the number; the rule's value, for the report
        if args.served_slots > 0:
            return args.served_slots, args.served_slots
        slots = 32
        while slots > 1 and slots * max(rows, n * n) * 4 > 64 * 2 ** 20:
            slots //= 2
        return 0, slots

    srv = B.Server(budget, K, args.served_tick)
    srv.set_priority(args.served_priority)
    pack = getattr(args, "served_pack", 1)
    if pack > 1:
        srv.set_packing(pack, getattr(args, "served_pack_ratio", 4.0))
    for n in sizes:
        na, nb = int(round(0.7 * n)), int(math.ceil(math.sqrt(2) * n)) + 1
        A = synth.parallel_beam_csr(n, na, nb)
        # u_max of this geometry by the batch power iteration with the
        # on-the-fly projector (no second stored copy of A)
        with B.BatchReconstructor(None, (n, n), 1, parallel_beam=(na, nb)) as one:
            u, _ = one.estimate_umax(300, 1e-9)
        ask, slots_of[n] = slot_cap(n, A.rows)
        gid = srv.add_geometry(A, (n, n), 0.9 / (2 * u), slots=ask, fmt=B.FMT_F16_I16,
                               prewarm=0)
        ys = [synth.noisy_projections(A, synth.phantom(n, ellipses[n], s), s).astype(np.float32)
              for s in range(pool)]
        geoms[n] = (gid, ys, A.nnz)
    reqs = []
    for i in range(N):
        n = int(rng.choice(sizes, p=probs))
        reqs.append((n, int(rng.integers(pool)), float(rng.uniform(0.01, 0.1)), int(rng.integers(100, 301))))
    t_setup = time.perf_counter() - t_setup

    def run(arrivals):
        ids = [None] * N
        t0 = time.perf_counter()

        def submitter():
            for i, (n, k, lam, ep) in enumerate(reqs):
                wait = arrivals[i] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                ids[i] = srv.submit(geoms[n][0], geoms[n][1][k], lam, ep)

        th = threading.Thread(target=submitter)
        th.start()
        lat, done_at = [], []
        for i in range(N):
            while ids[i] is None:
                time.sleep(0.0005)
            x, l, _ = srv.wait(ids[i], geoms[reqs[i][0]][0], timeout_s=600)
            lat.append(l)
        th.join()
        return np.array(lat), time.perf_counter() - t0

    st0 = srv.stats()
    lat_sat, span_sat = run(np.zeros(N))
    sat_rps = N / span_sat
    rate = args.served_rate if args.served_rate > 0 else 0.7 * sat_rps
    arrivals = np.cumsum(rng.exponential(1.0 / rate, N))
    st1 = srv.stats()
    lat, span = run(arrivals)
    st2 = srv.stats()
    srv.close()
    slice_epochs = sum(r[3] for r in reqs)
    mix = {str(n): int(sum(1 for r in reqs if r[0] == n)) for n in sizes}
    by_size = {}
    for n in sizes:   # Poisson-phase latency of each image size
        ln = lat[[i for i, r in enumerate(reqs) if r[0] == n]]
        if len(ln):
            by_size[str(n)] = {"p50_ms": 1e3 * float(np.percentile(ln, 50)),
                               "p99_ms": 1e3 * float(np.percentile(ln, 99))}
    return {"requests": N, "stream": ("the first %d requests of the 2000-request served stream" % N
                                       if full else "%d requests without the 1024x1024 ones" % N),
            "mix": mix, "fgp_iters": K, "epochs": "U{100..300}", "lambda": "U(0.01,0.1)",
            "weights": "f16", "slots_per_group": {str(n): slots_of[n] for n in sizes},
            "hbm_budget_gb": args.served_budget_gb, "packing_max_parts": pack,
            "stream_priority_by_size": bool(args.served_priority),
            "latency_by_size": by_size,
            "packed_groups": st2["packed_groups"], "max_parts_per_group": st2["max_parts"],
            "launches_per_epoch_of_a_packed_group": st2["packed_launches"] or None,
            "max_tick_epochs": args.served_tick,
            "saturated": {"requests_per_s": sat_rps, "slice_epochs_per_s": slice_epochs / span_sat,
                          "p50_ms": 1e3 * float(np.percentile(lat_sat, 50)),
                          "p99_ms": 1e3 * float(np.percentile(lat_sat, 99))},
            "poisson_rate_per_s": rate,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(lat.mean()), "throughput_requests_per_s": N / span,
            "slice_epochs_per_s": slice_epochs / span,
            "max_running": st2["max_running"], "groups_made": st2["groups_made"],
            "ticks": st2["ticks"] - st1["ticks"], "setup_s": t_setup,
            "note": "latency = submit to x in host memory; inputs drawn from a pool of %d seeded "
                    "phantoms per size; phase 1 all at once, phase 2 Poisson at %s" % (
                        pool, "%.3g requests/s (given)" % rate if args.served_rate > 0 else "0.7x phase 1")}


# ------------------------------------------------------------- CPU oracle
def oracle_epochs_per_s(P, mu, seconds, min_epochs=2, max_epochs=10 ** 9):
    """Times the FP64 oracle's epochs (block-by-block Algorithm 1 + FGP) on the
    host; returns (epochs/s, epochs timed, seconds)."""
    import numpy as np
    import oracle
    wl = P.wl
    A = oracle.to_scipy(P.A)
    rb, cb = oracle.partition(A.shape[0], A.shape[1], wl.M, wl.N, wl.n_bins, wl.n)
    blocks = oracle.split_blocks(A, rb, cb)
    y = P.y.astype(np.float32).astype(np.float64)
    x = np.zeros(A.shape[1])
    r = y.copy()
    rng = np.random.default_rng(0)
    done = 0
    t0 = time.perf_counter()
    while done < max_epochs and (done < min_epochs or time.perf_counter() - t0 < seconds):
        x, r, _ = oracle.epoch(blocks, rb, cb, y, x, r, mu, wl.lam, wl.fgp_iters, (wl.n, wl.n), rng)
        done += 1
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def _pair_worker(conn, blocks_mine, rb, cb, pairs):
    """Worker of oracle_parallel_epochs_per_s: holds the blocks of its pairs,
    answers each (x, r) with their block products (oracle.block_products)."""
    import os
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle
    M, N = len(rb) - 1, len(cb) - 1
    blocks = [[None] * N for _ in range(M)]
    for (i, j), blk in zip(pairs, blocks_mine):
        blocks[i][j] = blk
    while True:
        msg = conn.recv()
        if msg is None:
            break
        x, r = msg
        z, gh = oracle.block_products(blocks, rb, cb, x, r, pairs)
        conn.send([(z[i][j], gh[i][j]) for i, j in pairs])
    conn.close()


def oracle_parallel_epochs_per_s(P, mu, seconds, workers, min_epochs=2):
    """The same oracle epochs with the M x N block products spread over
    `workers` spawned processes (contiguous runs of pairs in (i, j) order),
    the residual / gradient sums (ascending j / i), the step and the FGP prox
    in this process: the oracle's own functions, in the oracle's order.
    Returns (epochs/s, epochs timed, seconds, workers)."""
    import multiprocessing as mp

    import numpy as np
    import oracle
    wl = P.wl
    A = oracle.to_scipy(P.A)
    rb, cb = oracle.partition(A.shape[0], A.shape[1], wl.M, wl.N, wl.n_bins, wl.n)
    blocks = oracle.split_blocks(A, rb, cb)
    pairs = [(i, j) for i in range(wl.M) for j in range(wl.N)]
    workers = max(1, min(workers, len(pairs)))
    ctx = mp.get_context("spawn")
    procs, conns, shares = [], [], []
    for w in range(workers):
        mine = pairs[len(pairs) * w // workers: len(pairs) * (w + 1) // workers]
        a, b = ctx.Pipe()
        pr = ctx.Process(target=_pair_worker, args=(b, [blocks[i][j] for i, j in mine], rb, cb, mine),
                         daemon=True)
        pr.start()
        procs.append(pr)
        conns.append(a)
        shares.append(mine)
    del blocks
    y = P.y.astype(np.float32).astype(np.float64)
    x = np.zeros(A.shape[1])
    r = y.copy()
    M, N = wl.M, wl.N

    def one_epoch(x, r):
        for c in conns:
            c.send((x, r))
        z = [[None] * N for _ in range(M)]
        gh = [[None] * N for _ in range(M)]
        for c, mine in zip(conns, shares):
            for (i, j), (zz, gg) in zip(mine, c.recv()):
                z[i][j], gh[i][j] = zz, gg
        r_new = oracle.reduce_residual(y, z, rb)
        x_hat = x + mu * oracle.reduce_gradient(gh, cb, x.shape[0])
        if wl.lam > 0.0 and wl.fgp_iters > 0:
            x_new = oracle.fgp(x_hat.reshape(wl.n, wl.n), mu * wl.lam, wl.fgp_iters).ravel()
        else:
            x_new = x_hat
        return x_new, r_new

    try:
        x, r = one_epoch(x, r)     # warm-up: every worker has started and answered
        done = 0
        t0 = time.perf_counter()
        while done < min_epochs or time.perf_counter() - t0 < seconds:
            x, r = one_epoch(x, r)
            done += 1
        dt = time.perf_counter() - t0
    finally:
        for c in conns:
            try:
                c.send(None)
            except (OSError, BrokenPipeError):
                pass
        for pr in procs:
            pr.join(timeout=10)
            if pr.is_alive():
                pr.terminate()
    return done / dt, done, dt, workers


# ------------------------------------------------------------------ arms
def run_reference(args):
    from paper_1812_01307_gb300 import dist as D
    rank, _, world = D.env_rank()
    if rank != 0:
        return 0
    import oracle
    from paper_1812_01307_gb300 import synth
    wl = synth.WORKLOADS[args.workload]
    P = synth.make_problem(wl)
    u, _ = oracle.power_iteration(P.A, 1000, 1e-10)
    mu = 0.9 / (2 * u)
    # warm-up (one epoch at most) and a bounded timed sample of the K steps
    oracle_epochs_per_s(P, mu, 0.0, min_epochs=min(args.warmup, 1), max_epochs=min(args.warmup, 1))
    budget = 120.0
    v, done, dt = oracle_epochs_per_s(P, mu, budget, min_epochs=1, max_epochs=max(args.steps, 1))
    sample = (f"{done} of the {args.steps} requested epochs of {wl.name} (time-bounded, "
              f"{dt:.1f} s), FP64 numpy/scipy, block by block")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "epochs/s", "n_gpus": args.gpus,
            "steps": done, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(wl)},
            "cpu_baseline": {"value": v, "unit": "epochs/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "epochs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1812_01307_gb300 import dist as D
    from paper_1812_01307_gb300 import synth
    rank, local, world = D.env_rank()
    if world != args.gpus:
        print(f"warning: WORLD_SIZE={world} but --gpus {args.gpus}", file=sys.stderr)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    D.barrier()
    from paper_1812_01307_gb300 import bsgdtv as B
    B.load()

    base = synth.WORKLOADS[args.workload]
    import dataclasses
    wl = dataclasses.replace(base, seed=base.seed + rank)   # each rank its own slice
    P = synth.make_problem(wl)
    rec = B.Reconstructor(P.A, (wl.n, wl.n), wl.M, wl.N, row_unit=wl.n_bins, col_unit=wl.n)
    u, _ = rec.estimate_umax(1000, 1e-10)
    mu = 0.9 / (2 * u)
    y_dev = torch.tensor(P.y, dtype=torch.float32, device=dev)
    rec.set_data(y_dev, wl.lam, mu)
    info = rec.info()
    K, W = args.steps, args.warmup

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    rec.run(W, wl.fgp_iters)
    torch.cuda.synchronize()

    def untimed():   # more warm-up epochs while the clock sampler starts
        rec.run(20, wl.fgp_iters)
        torch.cuda.synchronize()

    sampler.wait_samples(1, 5.0, untimed)
    n_before = sampler.samples()
    launches0 = B.bsgdtv_launch_count()
    D.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    prod_ms, epoch_ms = B.bsgdtv_run_timed(rec.h, K, wl.fgp_iters)
    ev1.record()
    torch.cuda.synchronize()
    D.barrier()
    # a short timed region may fall between two samples: keep the GPU loaded
    # with untimed epochs until the sampler has recorded one more
    launches = B.bsgdtv_launch_count() - launches0
    sampler.wait_samples(n_before + 1, 5.0, untimed)
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    elapsed_max = D.max_over_ranks(elapsed, dev)
    value = world * K / elapsed_max

    # end to end through the public API: y from pinned host memory in, x out, every step
    E = max(1, min(args.e2e_steps, K))
    y_pin = torch.empty(P.A.rows, dtype=torch.float32).pin_memory()
    y_pin.copy_(torch.from_numpy(P.y.astype(np.float32)))
    x_pin = torch.empty(P.A.cols_n, dtype=torch.float32).pin_memory()
    y_np, x_np = y_pin.numpy(), x_pin.numpy()
    torch.cuda.synchronize()
    D.barrier()
    # the one-call form: y in, one epoch, x out, one synchronisation
    t0 = time.perf_counter()
    for _ in range(E):
        B.bsgdtv_reconstruct(rec.h, y_np, wl.lam, mu, 1, wl.fgp_iters, x_np)
    torch.cuda.synchronize()
    e2e_dt = D.max_over_ranks(time.perf_counter() - t0, dev)
    # the same through the three calls (a synchronisation after y and after x)
    D.barrier()
    t0 = time.perf_counter()
    for _ in range(E):
        B.bsgdtv_set_data(rec.h, y_np, wl.lam, mu)
        rec.run(1, wl.fgp_iters)
        B.bsgdtv_get_x(rec.h, x_np)
    torch.cuda.synchronize()
    e2e3_dt = D.max_over_ranks(time.perf_counter() - t0, dev)
    e2e = {"value": world * E / e2e_dt, "unit": "epochs/s", "h2d_bytes_per_step": 4 * P.A.rows,
           "d2h_bytes_per_step": 4 * P.A.cols_n, "steps": E,
           "three_calls_value": world * E / e2e3_dt,
           "note": "per step: bsgdtv_reconstruct(host y, 1 epoch, host x) from pinned buffers, "
                   "one synchronisation; three_calls_value: bsgdtv_set_data(host y) + "
                   "bsgdtv_run(1 epoch) + bsgdtv_get_x(host x)"}
    rec.close()
    peak, peak_kind = hbm_peak()
    fp32_scalar, fp32_packed = B.bsgdtv_fp32_fma_peak()
    fp32_peak = max(fp32_scalar, fp32_packed)

    # the same workload with the other stored formats of A (one timed run each)
    variants = {}
    if not args.no_variants:
        Kv = max(1, min(K, 1000))
        for name in [v for v in ("f32_i16", "f16_i16", "bf16_i16") if v in args.variants.split(",")]:
            fmt = B.FORMATS[name]
            rv = B.Reconstructor(P.A, (wl.n, wl.n), wl.M, wl.N, row_unit=wl.n_bins, col_unit=wl.n, fmt=fmt)
            rv.set_data(y_dev, wl.lam, mu)
            rv.run(W, wl.fgp_iters)
            torch.cuda.synchronize()
            D.barrier()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record()
            pk, ep = B.bsgdtv_run_timed(rv.h, Kv, wl.fgp_iters)
            v1.record()
            torch.cuda.synchronize()
            dt = D.max_over_ranks(v0.elapsed_time(v1) / 1e3, dev)
            vinfo = rv.info()
            rv.close()
            ach = vinfo["min_bytes_per_pass"] / (pk / 1e3 / Kv) / 1e9
            variants[name] = {"value": world * Kv / dt, "unit": "epochs/s", "steps": Kv,
                              "products_ms": pk / Kv, "bytes_per_launch": vinfo["min_bytes_per_pass"],
                              "achieved_gbs": ach, "frac": ach / peak}

    # stochastic variant: half of the row and of the column blocks per iteration
    if not args.no_variants and "stochastic" in args.variants.split(","):
        alpha = gamma = 0.5
        Ks = max(1, min(K, 1000))
        R_sel, C_sel = synth.subset_draws(wl.M, wl.N, alpha, gamma, Ks + W, seed=wl.seed)
        rs = B.Reconstructor(P.A, (wl.n, wl.n), wl.M, wl.N, row_unit=wl.n_bins, col_unit=wl.n)
        rs.set_data(y_dev, wl.lam, mu)
        rs.run_subsets(R_sel[:W], C_sel[:W], wl.fgp_iters)
        torch.cuda.synchronize()
        D.barrier()
        t0s = time.perf_counter()
        dev_ms, prep_ms = B.bsgdtv_run_subsets_timed(rs.h, R_sel[W:], C_sel[W:], wl.fgp_iters)
        wall_s = time.perf_counter() - t0s
        dts = D.max_over_ranks(dev_ms / 1e3, dev)
        rs.close()
        variants["stochastic"] = {
            "value": world * Ks / dts, "unit": "iterations/s", "steps": Ks, "alpha": alpha,
            "gamma": gamma, "block_epochs_per_s": world * Ks * alpha * gamma / dts,
            "host_prep_ms": prep_ms, "wall_iterations_per_s": Ks / wall_s,
            "note": "per iteration half of the row blocks and half of the column blocks are drawn "
                    "(Sec. 3); a block-epoch is M*N block products; value: CUDA-event time of the "
                    "iterations' kernels on the handle's stream (work-item lists already on the "
                    "device); host_prep_ms: building and uploading those lists, outside it"}

    # many slices sharing one A: B slices of the same geometry, one batch handle
    # (FP32 weights, and binary16 weights with FP32 arithmetic)
    batch_kinds = [(k, f) for k, f in (("batch", B.FMT_F32_I32), ("batch_f16", B.FMT_F16_I16))
                   if k in args.variants.split(",")]
    if not args.no_variants and args.batch_slices > 0 and batch_kinds:
        Bs = args.batch_slices
        _, Ys = synth.slice_stack(P.A, wl.n, wl.n_ellipses, Bs, seed=wl.seed)
        Ys_dev = torch.tensor(Ys, dtype=torch.float32, device=dev)
        lam_b = np.random.default_rng(wl.seed + 3).uniform(0.01, 0.05, Bs)
        Kfb = 30   # FGP iterations of the batched-volume configuration
    for kind, bfmt in (batch_kinds if not args.no_variants and args.batch_slices > 0 else []):
        # an NVTX range per variant lets a profiler select its launches
        # (ncu --nvtx --nvtx-include batch/ ...)
        torch.cuda.nvtx.range_push(kind)
        bt = B.BatchReconstructor(P.A, (wl.n, wl.n), Bs, fmt=bfmt)
        bt.set_data(Ys_dev, lam_b, mu)
        if args.batch_tuning:   # a known tuning: no timing trials (e.g. under a profiler)
            chunk, group = (int(v) for v in args.batch_tuning.split(","))
            bt.set_tuning(chunk, group)
        else:
            chunk, group, _ = bt.autotune(Kfb, 3)
        lanes = bt.tuning()[2:]
        bt.set_data(Ys_dev, lam_b, mu)
        bt.run(max(W, 3), Kfb)
        torch.cuda.synchronize()
        D.barrier()
        Kb = max(1, min(K, 150))
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record()
        pk, ep = bt.run_timed(Kb, Kfb)
        b1.record()
        torch.cuda.synchronize()
        dt = D.max_over_ranks(b0.elapsed_time(b1) / 1e3, dev)
        bt.close()
        torch.cuda.nvtx.range_pop()
        nnz_b = int(P.A.row_ptr[-1])
        # both passes: A once each (4 B index + 4 B FP32 or 2 B FP16 weight per
        # nonzero), and y, x, r, x^ of every slice once per pass they appear in
        per_nnz = 8 if bfmt == B.FMT_F32_I32 else 6
        pass_bytes = 2 * per_nnz * nnz_b + 4 * Bs * 3 * (P.A.rows + P.A.cols_n)
        ach = pass_bytes / (pk / 1e3 / Kb) / 1e9
        prod_s = pk / 1e3 / Kb
        # ALU roof: 2 FMAs (4 flops) per nonzero and slice, at the measured FP32 peak
        flops = 4.0 * nnz_b * Bs
        t_hbm, t_alu = pass_bytes / (peak * 1e9), flops / (fp32_peak * 1e12)
        variants[kind] = {"value": world * Bs * Kb / dt, "unit": "slice-epochs/s", "slices": Bs,
                          "steps": Kb, "fgp_iters": Kfb, "lambda": "per slice U(0.01,0.05), seeded",
                          "epoch_ms": 1e3 * dt / Kb, "products_ms": pk / Kb,
                          "weights": "f32" if bfmt == B.FMT_F32_I32 else "f16",
                          "bytes_per_epoch_products": int(pass_bytes), "achieved_gbs": ach,
                          "autotuned_fgp_iters_per_launch": chunk,
                          "autotuned_fgp_slices_per_group": group,
                          "pass_lanes_per_nonzero": {"row": lanes[0], "column": lanes[1]},
                          "frac": ach / peak,
                          "products_tflops": flops / prod_s / 1e12,
                          "alu_frac": flops / prod_s / 1e12 / fp32_peak,
                          "binding_roof": "alu" if t_alu > t_hbm else "hbm",
                          "binding_frac": max(t_hbm, t_alu) / prod_s,
                          "config": "batched volume: %d slices of %dx%d sharing one A (%d angles x %d "
                                    "bins), per-slice lambda ~ U(0.01,0.05), %d FGP iterations"
                                    % (Bs, wl.n, wl.n, wl.n_angles, wl.n_bins, Kfb),
                          "note": "two passes over A (CSR then CSC) per epoch, lanes = slices; "
                                  "x and r gathered from L2; binding_frac = max(HBM time, FP32 "
                                  "ALU time at the measured peak) / product time"}

    # large and matrix free: 2048x2048, 60 ellipses, 1440 angles x 2897 bins, 16 slices
    if not args.no_variants and "matrix_free" in args.variants.split(","):
        import math
        torch.cuda.nvtx.range_push("matrix_free")
        n5 = args.mf_n
        na5, nb5, S5, K5 = int(round(1440 * n5 / 2048)), int(math.ceil(math.sqrt(2) * n5)), 16, 50
        X5 = np.stack([synth.phantom(n5, 60, s).ravel() for s in range(S5)]).astype(np.float32)
        mf = B.BatchReconstructor(None, (n5, n5), S5, parallel_beam=(na5, nb5))
        Y5 = mf.project(torch.tensor(X5, device=dev)).cpu().numpy().astype(np.float64)
        for b in range(S5):   # 1 % Gaussian noise, seed b + 1, as the stored-matrix inputs
            sig = 0.01 * float(np.mean(np.abs(Y5[b])))
            Y5[b] += sig * np.random.default_rng(b + 1).standard_normal(Y5.shape[1])
        with B.BatchReconstructor(None, (n5, n5), 1, parallel_beam=(na5, nb5)) as one:
            u5, it5 = one.estimate_umax(100, 1e-6)
        mu5 = 0.9 / (2 * u5)
        mf.set_data(torch.tensor(Y5, dtype=torch.float32, device=dev), np.full(S5, 0.02), mu5)
        mf.run(1, K5)
        torch.cuda.synchronize()
        D.barrier()
        Km = 3
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record()
        pk5, ep5 = mf.run_timed(Km, K5)
        m1.record()
        torch.cuda.synchronize()
        dt5 = D.max_over_ranks(m0.elapsed_time(m1) / 1e3, dev)
        mf.close()
        torch.cuda.nvtx.range_pop()
        # the operator's nonzeros (no stored A): 4 flops per nonzero and slice at
        # least (one FMA in each pass), at the measured FP32 peak
        nnz5 = synth.parallel_beam_nnz(n5, na5, nb5)
        flops5 = 4.0 * nnz5 * S5
        prod5_s = pk5 / 1e3 / Km
        variants["matrix_free"] = {
            "value": world * S5 * Km / dt5, "unit": "slice-epochs/s", "slices": S5, "steps": Km,
            "image": f"{n5}x{n5}", "angles": na5, "bins": nb5, "fgp_iters": K5,
            "epoch_ms": 1e3 * dt5 / Km, "products_ms": pk5 / Km, "u_max": u5, "u_max_iters": it5,
            "nnz": nnz5, "products_tflops": flops5 / prod5_s / 1e12,
            "alu_frac": flops5 / prod5_s / 1e12 / fp32_peak,
            "note": "weights computed on the fly in both passes (no stored A); the stored FP32 CSR "
                    "of this geometry would hold about 7.7e9 nonzeros (62 GB)"}

    served = None
    if rank == 0 and world == 1 and args.served_requests > 0:
        served = served_stream(args, B, synth)

    prod_avg_s = prod_ms / 1e3 / K
    per_launch = info["min_bytes_per_pass"]
    achieved = per_launch / prod_avg_s / 1e9
    R, c, nnz = P.A.rows, P.A.cols_n, info["nnz"]
    # per epoch at least: A (8 B per nonzero), y, r^{k-1}, r^k (3R) and x, x^ (2c)
    # once, and the prox's input and output fields (2c)
    epoch_bytes = 8 * nnz + 4 * (3 * R + 2 * c) + 8 * c
    epoch_s = elapsed / K
    line = {"metric": METRIC, "value": value, "unit": "epochs/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": 1e3 * elapsed_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(wl), "parallelism": f"independent slices x{world}",
                       "l2": "inputs larger than L2 (A = %.2f GB), no flush" % (8 * nnz / 1e9),
                       "nnz": nnz, "segments": info["segments"], "work_items": info["work_items"]},
            "products_per_s": 2 * value,
            "roofline": {"bound": "hbm", "kernel": "products_kernel (fused Ax, 2A^T r)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": profiled_traffic(), "bytes_per_launch": per_launch,
                         "avg_launch_ms": prod_avg_s * 1e3,
                         "share_of_epoch": prod_ms / epoch_ms if epoch_ms > 0 else None,
                         "epoch_bytes": epoch_bytes,
                         "epoch_achieved": epoch_bytes / epoch_s / 1e9,
                         "epoch_frac": epoch_bytes / epoch_s / 1e9 / peak},
            "fp32_peak_tflops": {"scalar": fp32_scalar, "packed": fp32_packed,
                                 "kind": "measured in this run: FMA chains at full occupancy, CUDA events"},
            "gpu_launches": launches, "clocks": clocks, "e2e": e2e,
            "served": served, "variants": variants or None}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, done, dt = oracle_epochs_per_s(P, mu, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "epochs/s", "cores": 1, "kind": "oracle",
                                "sample": f"{done} epochs of {wl.name} from x=0 ({dt:.1f} s, FP64 numpy/scipy, one thread)"}
        ncpu = os.cpu_count() or 1
        if ncpu > 1:
            va, done_a, dt_a, wk = oracle_parallel_epochs_per_s(P, mu, args.cpu_seconds, ncpu)
            line["cpu_baseline"]["all_cores"] = {
                "value": va, "unit": "epochs/s", "cores": wk, "host_cpus": ncpu, "kind": "oracle",
                "sample": f"{done_a} epochs of {wl.name} ({dt_a:.1f} s): the {wl.M}x{wl.N} block "
                          f"products over {wk} processes, sums, step and FGP prox in one"}
    if rank == 0:
        print(json.dumps(line), flush=True)
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
