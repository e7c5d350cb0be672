"""Benchmark of the rank-Greville recursive least-squares update on GB300.

Workload (one "step" = one pass of the whole hot path over one synthetic stream):
  single large FP64 stream, A = G1 G2 with G1 (65536 x 64), G2 (64 x 1024) Gaussian,
  n = 65536 rows, m = 1024, r = 64, targets Y = A x_true + N(0, 1e-3); the rows arrive in
  blocks of k = 32 rows (2048 rg_add_rows calls), then rg_solution materialises X.
  Each step starts from an empty state (rg_reset), so every step solves the stream from
  scratch. Inputs (512 MiB) are resident in HBM and larger than L2.

Prints ONE JSON line (rank 0). Extra per-configuration numbers (k = 1/8/32/all rows per
call, FP64 and mixed) go under "extra".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--quick]

--impl reference times the CPU oracle (oracle/rg_oracle.c, plain FP64 Algorithm 1) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ROWS, M, R = 65536, 1024, 64
K_CALL = 32
METRIC = ("row updates/sec (device-timed, batched & single) at stated rel. error vs FP64 "
          "oracle; % HBM roofline")
WORKLOAD = f"single FP64 stream n={N_ROWS} m={M} r={R}, k={K_CALL} rows per rg_add_rows call"


# DRAM bytes (read + write) of one 32-row stream_kernel<false, false> launch, from the ncu
# capture of that kernel summarised under profiles/, and the hash of the kernel sources it
# was taken on: once the sources change the figure no longer applies (null).
TRAFFIC_BYTES_PER_LAUNCH = 1465600
TRAFFIC_SOURCES_SHA = "5083b1f17f1c9ba7"


STREAM_KERNEL_SOURCES = ("rg_stream.cu", "rg_core.cuh", "rg_internal.cuh", "rg_tc.cuh")


def kernel_sources_sha() -> str:
    """Hash of the sources compiled into stream_kernel."""
    import hashlib
    h = hashlib.sha256()
    for f in STREAM_KERNEL_SOURCES:
        h.update(f.encode())
        h.update(open(os.path.join(ROOT, "paper_2106_11594_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic():
    return TRAFFIC_BYTES_PER_LAUNCH if kernel_sources_sha() == TRAFFIC_SOURCES_SHA else None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp64_peak_tflops(sm_mhz: float, nsm: int = 152) -> float:
    """FP64 vector peak: 2 DFMA per clock per SM on GB300 (1/64 of FP32), i.e.
    152 SMs x 4 flop/clk x clock. At the 2070 MHz maximum this is 1.26 TFLOP/s, the
    nominal GB300 FP64 figure."""
    return nsm * 4.0 * sm_mhz * 1e6 / 1e12


def flops_per_row(m: int, r: int) -> float:
    """Algorithmic flops of one dependent row as the library computes it: gamma = Ct Gamma
    (2rm), rejection Gamma - C^T gamma (2rm), ||Gamma_r||^2 and ||Gamma||^2 (4m), the
    rank-one update of P = B^T B (2r^2), the a-priori error and the correction u (4r).
    (Algorithm 1's Sherman-Morrison form would count 4r^2 for zeta and P^-1.)"""
    return 4.0 * r * m + 4.0 * m + 2.0 * r * r + 4.0 * r


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while active."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
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
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

def run_gpu(args):
    import torch

    from paper_2106_11594_gb300 import dist as rgdist
    from paper_2106_11594_gb300 import inputs, rg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = N_ROWS if not args.quick else 8192
    s = inputs.large_stream(n, M, R)
    A = torch.from_numpy(s.A).to(dev)
    Y = torch.from_numpy(s.Y).to(dev)
    X = torch.empty(M, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def one_step(st, k, ev=None):
        st.reset()
        for c, j0 in enumerate(range(0, n, k)):
            # launch durations are sampled on every 16th call: an event pair around every
            # launch would itself slow the timed region by ~15 %. The sample starts at call
            # 15, past the two rank-growth calls (0, 1) whose section scan makes them ~20x
            # longer: counted once per 16 calls they would weigh 8x their share of the step
            sample = ev is not None and c % 16 == 15
            if sample:
                ev[0].append(torch.cuda.Event(enable_timing=True))
                ev[0][-1].record(stream)
            st.add_rows(A[j0:j0 + k], Y[j0:j0 + k])
            if sample:
                ev[1].append(torch.cuda.Event(enable_timing=True))
                ev[1][-1].record(stream)
        st.solution(X, with_rank=False)

    def timed(mode, k, steps, warmup, launch_events=False):
        st = rg.RankGreville(M, 1e-10, mode)
        for _ in range(warmup):
            one_step(st, k)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ev = ([], []) if launch_events else None
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(steps):
            one_step(st, k, ev)
        t1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ms = t0.elapsed_time(t1)
        st.sync()
        r = st.rank()
        launch_ms = None
        if ev is not None:
            launch_ms = sum(a.elapsed_time(b) for a, b in zip(ev[0], ev[1])) / len(ev[0])
        st.close()
        return ms, r, launch_ms

    # --- headline: FP64, k = 32, with per-launch events and clock sampling
    with ClockSampler(local) as clk:
        ms, rk, launch_ms = timed(rg.RG_FP64, K_CALL, args.steps, args.warmup, launch_events=True)
    clocks = clk.summary()
    # one replica of the stream per rank (a single stream does not shard): whole-job rows
    # over the slowest rank's time
    value, ms, _ = rgdist.job_throughput(n * args.steps, ms, dev)
    ms_per_step = ms / args.steps
    # parity of the last step against the oracle is covered by the tests; report the rank
    # --- e2e through host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.skip_e2e:
        Ah = torch.from_numpy(s.A).pin_memory().numpy()
        Yh = torch.from_numpy(s.Y).pin_memory().numpy()
        Xh = torch.empty(M, dtype=torch.float64).pin_memory().numpy()
        st = rg.RankGreville(M, 1e-10, rg.RG_FP64)

        def e2e_step():
            st.reset()
            for j0 in range(0, n, K_CALL):
                st.add_rows_host(Ah[j0:j0 + K_CALL], Yh[j0:j0 + K_CALL])
            st.solution_host(Xh)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st.close()
        e2e = {"value": n * args.steps / dt, "unit": "rows/s",
               "h2d_bytes_per_step": int(n * (M + 1) * 8), "d2h_bytes_per_step": int(M * 8)}
    # --- extra configurations (fewer steps)
    extra = {}
    if not args.headline_only:
        for mode, mname in ((rg.RG_FP64, "fp64"), (rg.RG_MIXED, "mixed")):
            for k in (1, 8, 32, n):
                if k == 1 and mode == rg.RG_FP64 and args.quick:
                    continue
                steps = 1 if k <= 8 else 2
                ms_k, r_k, _ = timed(mode, k, steps, 1)
                extra[f"{mname}_k{k if k < n else 'all'}"] = {
                    "rows_per_s": n * steps / (ms_k / 1e3), "ms_per_step": ms_k / steps, "rank": r_k}
        for k in (32, n):  # the FP64 orthonormal variant (Section 2.2)
            ms_k, r_k, _ = timed(rg.RG_FP64 | rg.RG_ORTHONORMAL, k, 2, 1)
            extra[f"fp64_orthonormal_k{k if k < n else 'all'}"] = {
                "rows_per_s": n * 2 / (ms_k / 1e3), "ms_per_step": ms_k / 2, "rank": r_k}
    # --- pseudoinverse of the whole stream from its factorization (rg_pinv), FP64 and the
    # orthonormal variant: 4 n m r flop per call
    if not args.headline_only:
        for flags, pname in ((rg.RG_FP64, "fp64"), (rg.RG_FP64 | rg.RG_ORTHONORMAL, "fp64_orthonormal")):
            st = rg.RankGreville(M, 1e-10, flags)
            st.add_rows(A, Y)
            Ap = torch.empty((M, n), dtype=torch.float64, device=dev)
            for _ in range(3):
                st.pinv(A, Ap)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            reps = 3
            t0.record(stream)
            for _ in range(reps):
                st.pinv(A, Ap)
            t1.record(stream)
            torch.cuda.synchronize()
            ms_p = t0.elapsed_time(t1) / reps
            rk = st.rank()
            tflops = 4.0 * n * M * rk / (ms_p / 1e3) / 1e12
            extra[f"pinv_{pname}_n{n}"] = {"ms_per_call": ms_p, "rank": rk, "tflops": tflops,
                                          "frac_fp64_peak": tflops / fp64_peak_tflops(clocks.get("sm_mhz") or 2070.0)}
            st.close()
            del Ap
            torch.cuda.empty_cache()
    # --- batched workloads
    if not args.headline_only and not args.quick:
        from paper_2106_11594_gb300 import inputs as _inp
        n3, m3, r3 = _inp.uneven_batch_shapes()
        shapes3 = [(int(a), int(b), int(c)) for a, b, c in zip(n3, m3, r3)]
        shapes4 = [(2048, 256, 32)] * 1024
        for mode, mname in ((rg.RG_MIXED, "mixed"), (rg.RG_FP64, "fp64")):
            extra[f"batch_uneven4096_{mname}"] = run_batched("uneven", shapes3, 3, 1e-4, mode, 2, 1, dev, ws, rank)
            extra[f"batch_uniform1024_{mname}"] = run_batched("uniform", shapes4, 4, 1e-3, mode, 2, 1, dev, ws, rank)
            extra[f"adjoint_uniform1024_{mname}"] = run_batched("uniform", shapes4, 4, 1e-3, mode, 2, 1, dev, ws, rank,
                                                               backward=True)
        # the orthonormal variant of Section 2.2 with every step in FP64
        extra["batch_uniform1024_fp64_orthonormal"] = run_batched(
            "uniform", shapes4, 4, 1e-3, rg.RG_FP64 | rg.RG_ORTHONORMAL, 2, 1, dev, ws, rank)
    # --- roofline of the dominant kernel (the stream kernel, one launch per 32-row call)
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = fp64_peak_tflops(sm_mhz)
    achieved = K_CALL * flops_per_row(M, R) / (launch_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": measured_traffic(),
                "peak_source": f"FP64 vector peak derived: 152 SMs x 4 flop/clk x {sm_mhz:.0f} MHz "
                               "(median SM clock sampled during the timed region)",
                "kernel": "rg::stream_kernel<false, false> (one launch per 32-row call)",
                "avg_launch_ms": launch_ms}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "rows_per_step": n, "m": M, "r": R,
                           "rows_per_call": K_CALL, "l2": "inputs larger than L2 (512 MiB)",
                           "parallelism": "replicas only" if ws > 1 else "single GPU"},
                "rank_after_step": rk, "gpu_launches": args.steps * (2 + n // K_CALL),
                "clocks": clocks, "e2e": e2e, "roofline": roofline}
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(args, n)
        line["extra"] = extra
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------------------
# Batched workloads (extra lines): matrices formed on the GPU from the seeded factors
# (inputs.factor_stream_factors draws G1, G2, x_true, noise in the generator's order)
# ---------------------------------------------------------------------------------------

def make_batch_on_gpu(shapes, workload_id, noise, dev, ids=None):
    import torch

    from paper_2106_11594_gb300 import inputs
    n = np.array([s[0] for s in shapes], dtype=np.int64)
    m = np.array([s[1] for s in shapes], dtype=np.int64)
    ro = np.zeros(len(shapes) + 1, dtype=np.int64)
    ro[1:] = np.cumsum(n)
    eo = np.zeros(len(shapes) + 1, dtype=np.int64)
    eo[1:] = np.cumsum(n * m)
    A = torch.empty(int(eo[-1]), dtype=torch.float64, device=dev)
    Y = torch.empty(int(ro[-1]), dtype=torch.float64, device=dev)
    ids = range(len(shapes)) if ids is None else ids
    for b, ((nb, mb, rb), inst) in enumerate(zip(shapes, ids)):
        G1, G2, x, e = inputs.factor_stream_factors(nb, mb, rb, noise, inputs.rng_for(workload_id, int(inst)))
        G1t = torch.from_numpy(G1).to(dev)
        G2t = torch.from_numpy(G2).to(dev)
        Ab = G1t @ G2t
        A[eo[b]:eo[b + 1]] = Ab.reshape(-1)
        Y[ro[b]:ro[b + 1]] = Ab @ torch.from_numpy(x).to(dev) + torch.from_numpy(e).to(dev)
    return A, Y, torch.from_numpy(ro).to(dev), torch.from_numpy(eo).to(dev), m


def run_batched(name, shapes, workload_id, noise, mode, steps, warmup, dev, ws=1, rank=0, backward=False):
    """Times one batched workload. With several ranks the instances are partitioned by
    LPT on their cost (each rank keeps the seeded draws of its own instance ids) and the
    rate is all ranks' rows over the slowest rank's time. backward=True times the
    differentiable form instead: forward, the loss L = sum_b ||X_b - x_target,b||^2 and
    the adjoint (dL/dA, dL/dy of every instance) per step."""
    import torch

    from paper_2106_11594_gb300 import dist as rgdist
    from paper_2106_11594_gb300 import inputs, rg
    ids = np.arange(len(shapes))
    if ws > 1:
        ns, ms_, rs = (np.array([s[i] for s in shapes]) for i in range(3))
        ids = rgdist.lpt_partition(rgdist.instance_cost(ns, ms_, rs), ws)[rank]
    all_shapes = shapes
    shapes = [all_shapes[i] for i in ids]
    A, Y, ro, eo, m = make_batch_on_gpu(shapes, workload_id, noise, dev, ids)
    bt = rg.RankGrevilleBatch(m, 1e-10, mode)
    X = torch.empty(int(m.sum()), dtype=torch.float64, device=dev)
    ranks = torch.empty(len(shapes), dtype=torch.int64, device=dev)
    if backward:
        xt = torch.cat([torch.from_numpy(inputs.rng_for(workload_id, 1 << 20 | int(i)).standard_normal(int(mb)))
                        for i, mb in zip(ids, m)]).to(dev)
        gA = torch.empty_like(A)
        gY = torch.empty_like(Y)
        gX = torch.empty_like(X)

    def step():
        bt.reset()
        bt.add_rows(A, ro, eo, Y)
        bt.solution(X, None, ranks)
        if backward:
            torch.sub(X, xt, out=gX)
            gX.mul_(2.0)
            bt.adjoint(A, ro, eo, Y, Y.numel(), gX, gA, gY)

    # autotune the per-block row cap on this batch (outside the timed region)
    from paper_2106_11594_gb300 import autotune
    kb, kb_times = autotune.tune_block_rows(bt, A, ro, eo, Y, X)
    # capture one step into a CUDA graph on a side stream and replay it
    graph = None
    cap_stream = torch.cuda.Stream()
    cap_stream.wait_stream(torch.cuda.current_stream())
    bt.set_stream(cap_stream)
    with torch.cuda.stream(cap_stream):
        for _ in range(warmup):
            step()
    cap_stream.synchronize()
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap_stream):
            step()
        graph = g
    except Exception as exc:  # capture unsupported here: time direct launches instead
        print(f"[bench] graph capture failed ({exc}); timing direct launches", file=sys.stderr)
        torch.cuda.synchronize()
    stream = cap_stream
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0.record(stream)
        for _ in range(steps):
            if graph is not None:
                graph.replay()
            else:
                step()
        t1.record(stream)
    torch.cuda.synchronize()
    bt.sync()
    ms = t0.elapsed_time(t1) / steps
    rows_mine = int(sum(s[0] for s in shapes))
    expect = np.array([min(s2) for s2 in shapes])
    rk = ranks.cpu().numpy()
    rate, ms, rows = rgdist.job_throughput(rows_mine, ms, dev)
    match = rgdist.sum_over_ranks(float((rk == expect).sum()), dev)
    out = {"rows_per_s": rate, "ms_per_step": ms, "rows": int(rows),
           "instances": len(all_shapes), "rank_match_generator": int(match),
           "cuda_graph": graph is not None, "block_rows": kb,
           "autotune_ms": {str(k): round(v, 3) for k, v in kb_times.items()}}
    bt.close()
    del A, Y
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------------------

def cpu_baseline(args, n_full):
    from oracle import fp64
    from paper_2106_11594_gb300 import inputs
    n = min(n_full, args.cpu_rows)
    s = inputs.large_stream(N_ROWS if not args.quick else 8192, M, R)
    A, Y = s.A[:n], s.Y[:n]
    fp64.build()
    t0 = time.perf_counter()
    fp64.solve(A, Y, tol=1e-10)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "rows/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} rows of the stream (includes the 64 rank-growth rows), "
                      "plain C FP64 Algorithm 1, one thread"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import fp64
    from paper_2106_11594_gb300 import inputs
    n = min(N_ROWS, args.cpu_rows)
    s = inputs.large_stream(N_ROWS, M, R)
    A, Y = s.A[:n], s.Y[:n]
    fp64.build()
    for _ in range(args.warmup):
        fp64.solve(A[:256], Y[:256], tol=1e-10)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fp64.solve(A, Y, tol=1e-10)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "rows/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "rows_per_step": n, "m": M, "r": R},
        "cpu_baseline": {"value": v, "unit": "rows/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n} rows of the stream per step, plain C FP64 "
                                   "Algorithm 1, one thread"},
        "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def profile_case(name):
    """One untimed run of a small case of the hot path, for profilers (ncu -k/-c):
    stream-k32 / stream-kall (FP64 stream n=4096, m=1024, r=64 in 32-row calls / one
    call), stream-kall-mixed, batch-uniform-{mixed,fp64} (152 instances of n=2048, m=256,
    r=32), batch-uneven-mixed (the first 512 shapes of the 4096-instance batch), pinv
    (rg_pinv of an FP64 stream n=16384, m=1024, r=64 after one call)."""
    import torch

    from paper_2106_11594_gb300 import inputs, rg
    dev = torch.device("cuda")
    if name == "pinv":
        s = inputs.large_stream(16384, M, R)
        A = torch.from_numpy(s.A).to(dev)
        Y = torch.from_numpy(s.Y).to(dev)
        st = rg.RankGreville(M, 1e-10, rg.RG_FP64)
        st.add_rows(A, Y)
        Ap = torch.empty((M, s.n), dtype=torch.float64, device=dev)
        st.pinv(A, Ap)
        torch.cuda.synchronize()
        print(name, "rank", st.rank())
        st.close()
        return
    if name.startswith("stream"):
        mode = rg.RG_MIXED if name.endswith("mixed") else rg.RG_FP64
        k = 32 if name == "stream-k32" else 4096
        s = inputs.large_stream(4096, M, R)
        A = torch.from_numpy(s.A).to(dev)
        Y = torch.from_numpy(s.Y).to(dev)
        st = rg.RankGreville(M, 1e-10, mode)
        for j0 in range(0, s.n, k):
            st.add_rows(A[j0:j0 + k], Y[j0:j0 + k])
        X = torch.empty(M, dtype=torch.float64, device=dev)
        print(name, "rank", st.solution(X))
        st.close()
        return
    mode = rg.RG_MIXED if name.endswith("mixed") else rg.RG_FP64
    if name.startswith("batch-uniform"):
        shapes, wid, noise = [(2048, 256, 32)] * 152, 4, 1e-3
    else:
        n3, m3, r3 = inputs.uneven_batch_shapes()
        shapes, wid, noise = [(int(a), int(b), int(c)) for a, b, c in zip(n3, m3, r3)][:512], 3, 1e-4
    A, Y, ro, eo, m = make_batch_on_gpu(shapes, wid, noise, dev)
    bt = rg.RankGrevilleBatch(m, 1e-10, mode)
    bt.add_rows(A, ro, eo, Y)
    X = torch.empty(int(m.sum()), dtype=torch.float64, device=dev)
    ranks = torch.empty(len(shapes), dtype=torch.int64, device=dev)
    bt.solution(X, None, ranks)
    bt.sync()
    print(name, "ranks match", int((ranks.cpu().numpy() == np.array([min(x) for x in shapes])).sum()),
          "of", len(shapes))
    bt.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--quick", action="store_true", help="small stream (8192 rows)")
    ap.add_argument("--cpu-rows", type=int, default=16384)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--headline-only", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    choices=["stream-k32", "stream-kall", "stream-kall-mixed", "batch-uniform-mixed",
                             "batch-uniform-fp64", "batch-uneven-mixed", "pinv"],
                    help="run one small untimed case for a profiler and exit")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
