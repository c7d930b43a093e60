"""Benchmark of the batched differentiable MPC layer on GB300.

One step = one forward (box-constrained iLQR, <= 8 iterations, tol 1e-6) plus
one backward (adjoint LQR: dL/dQ, dL/dx_ref, dL/dx0) over B = 4096 race-track
instances of horizon N = 20 in FP32, inputs resident in HBM, replayed from two
CUDA graphs (forward, backward) with L2 flushed between steps.

Besides the headline value the JSON line carries the forward latency
distribution, the three-launches-per-iteration form on the same inputs, the
end-to-end number through the public API with host buffers, the roofline of
the dominant kernel, the FP64 CPU oracle on a bounded sample, and the SM clocks
sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own B instances (a different seed
per rank; instances are independent, so there is no collective on the data
path) and the slowest rank's time is reported: weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

B, N, MAX_ITER, TOL = 4096, 20, 8, 1e-6
METRIC = "DiffMPC fwd+bwd solves/s at B=4096,N=20 FP32 vs plain; p50/p99 fwd latency"
UNIT = "solves/s"
WORKLOAD = "race-track MPC batch: B=4096 instances, N=20, <=8 iLQR iterations (tol 1e-6), forward + adjoint backward"
# Algorithmic FP32 flops (FMA = 2), fixed from the method's steps:
#   per stage and executed iteration: RK4 rollout 0.53k + RK4 Jacobian 10.5k
#   + Riccati with box QP 11.9k + line search 4 x 0.72k  = 25.8k
#   final linearization + factorization at x* (store-all): 10.5k + 11.9k = 22.4k per stage
#   adjoint sweeps from the tape: 1.2k per stage
FLOP_STAGE_ITER = 25.8e3
FLOP_STAGE_FINAL = 22.4e3
FLOP_STAGE_BWD = 1.2e3
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20


# the sources the MPC kernel (k_mpc) is compiled from
KERNEL_SOURCES = ("camp_device.cuh", "camp_internal.h", "camp_kernels.cu")


def _kernel_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2605_29155_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic():
    """DRAM bytes per forward launch from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "k_mpc_forward_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    return d.get("bytes_per_launch") if d.get("kernel_hash") == _kernel_hash() else None


# ------------------------------------------------------------------ oracle --

def _oracle_chunk(args):
    prob, idx, gu = args
    from oracle import adjoint, ilqr
    from oracle.model import Quadrotor
    quad = Quadrotor(W.DEFAULT_MODEL)
    for i in idx:
        pr = ilqr.problem_from_batch(prob, i)
        so = ilqr.solve(quad, pr, MAX_ITER, TOL)
        if so.status in (ilqr.CONVERGED, ilqr.STALLED, ilqr.MAX_ITER):
            adjoint.adjoint(pr, so, np.zeros((pr.x_ref.shape[0], 13)), gu[i])
    return len(idx)


def oracle_rate(n_inst, seed=0, pool=None, cores=1):
    """Solves/s of the FP64 oracle (forward + backward) on n_inst track instances."""
    prob = W.cfg_track(seed=seed, B=n_inst)
    gu = W.loss_weights_u0(n_inst, N, seed=1)
    chunks = [list(range(k, n_inst, cores)) for k in range(cores)]
    t0 = time.perf_counter()
    if pool is None:
        _oracle_chunk((prob, list(range(n_inst)), gu))
    else:
        sum(pool.map(_oracle_chunk, [(prob, c, gu) for c in chunks if c]))
    return n_inst / (time.perf_counter() - t0)


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    per_step = max(cores, 32)
    with _oracle_pool(cores) as pool:
        for _ in range(args.warmup):
            oracle_rate(cores, seed=99, pool=pool, cores=cores)
        rates, t_all = [], time.perf_counter()
        for k in range(args.steps):
            rates.append(oracle_rate(per_step, seed=k, pool=pool, cores=cores))
        wall = time.perf_counter() - t_all
    value = per_step * args.steps / wall
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * wall / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD + " (FP64 CPU oracle, one instance at a time per process)",
                            B=B, N=N, sample=f"{per_step} instances per step"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                  sample=f"{per_step} race-track instances per step, fwd+bwd, {args.steps} steps"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


_BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_pool(cores):
    """A spawned pool of `cores` oracle processes with one BLAS thread each:
    the workers inherit the environment when they start, before they import
    numpy."""
    old = {v: os.environ.get(v) for v in _BLAS_VARS}
    for v in _BLAS_VARS:
        os.environ[v] = "1"
    try:
        return mp.get_context("spawn").Pool(cores)
    finally:
        for v, val in old.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi sampled every 100 ms in the background; mark() brackets the
    timed region, and the summary keeps the samples taken inside it (all
    samples when the region is shorter than the sampling interval)."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.out, self.marks = index, None, None, []

    def mark(self):
        self.marks.append(self._lines())

    def _lines(self):
        if self.out is None:
            return 0
        self.out.flush()
        self.out.seek(0)
        return len(self.out.read().strip().splitlines())

    def __enter__(self):
        try:
            self.out = open(os.path.join("/tmp", f"camp_clocks_{os.getpid()}.csv"), "w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.out is None:
            return None
        self.out.seek(0)
        lines = self.out.read().strip().splitlines()
        if len(self.marks) == 2 and self.marks[1] - self.marks[0] >= 3:
            lines = lines[self.marks[0]:self.marks[1]]
        rows = [r.split(",") for r in lines if r.count(",") >= 7]
        if not rows:
            return None
        sm = [float(r[0]) for r in rows]
        mx = max(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[4 + j].strip().lower() == "active"})
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=mx, reasons=reasons, samples=len(rows),
                    power_w_max=max(float(r[2]) for r in rows))


# ------------------------------------------------------------- GPU arm -----

def fp32_fma_peak(dev, local_rank):
    """Measured FP32 multiply-add throughput (mpc_fp32_fma_probe: 2 blocks of
    1024 threads per SM, 8 independent FMA chains per thread): `burst` is the
    best of 10 single launches of about 2 ms (the denominator for a kernel
    timed alone); `sustained` is 1 s of back-to-back launches, with the SM
    clocks sampled during it."""
    import torch
    from paper_2605_29155_gb300 import camp
    sink = torch.zeros(1, device=dev)
    stream = torch.cuda.current_stream()
    code, fl = camp.mpc_fp32_fma_probe(64, sink.data_ptr(), stream.cuda_stream)
    camp.check(code, "mpc_fp32_fma_probe")
    torch.cuda.synchronize()
    trips = 2000
    best = 0.0
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        code, fl = camp.mpc_fp32_fma_probe(trips, sink.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    reps = max(1, int(1.0 / max(fl / (best * 1e12), 1e-6)))
    with ClockSampler(local_rank) as clk:
        clk.mark()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        total = 0.0
        for _ in range(reps):
            code, fl = camp.mpc_fp32_fma_probe(trips, sink.data_ptr(), stream.cuda_stream)
            total += fl
        e1.record(stream)
        e1.synchronize()
        clk.mark()
    sustained = total / (e0.elapsed_time(e1) * 1e-3) / 1e12
    return dict(burst_tflops=best, sustained_tflops=sustained, clocks_sustained=clk.summary(),
                how="mpc_fp32_fma_probe: 2 x 1024 threads per SM, 8 FMA chains per thread; burst = best of 10 "
                    f"launches of {trips} x 16 FMA per chain, sustained = {reps} launches back to back")


def run_ours(args, rank, world, local_rank):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_29155_gb300 import DiffMPC, Problem

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    # CPU baseline first (spawned pools, before any further GPU work), rank 0 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        sample = max(4 * cores, 64)
        with _oracle_pool(cores) as pool:
            oracle_rate(cores, seed=99, pool=pool, cores=cores)
            rate = oracle_rate(sample, seed=0, pool=pool, cores=cores)
        with _oracle_pool(1) as pool:
            rate1 = oracle_rate(16, seed=0, pool=pool, cores=1)
        cpu = dict(value=rate, unit=UNIT, cores=cores, kind="oracle",
                   sample=f"first {sample} instances of the race-track workload, fwd+bwd, FP64, {cores} processes",
                   one_thread=dict(value=rate1, unit=UNIT, cores=1,
                                   sample="first 16 instances of the same workload, one process"))

    fma_peak = fp32_fma_peak(dev, local_rank)

    prob = W.cfg_track(seed=rank)
    gu_np = W.loss_weights_u0(B, N, seed=1 + rank)
    p = Problem.from_numpy(prob, device=dev)
    gu = torch.as_tensor(gu_np, dtype=torch.float32, device=dev)

    solver = DiffMPC(N_max=N, B_max=B, max_iter=MAX_ITER, tol=TOL, device=dev)
    s = solver.alloc_solution(B, N)
    grads = (torch.empty_like(p.Q), torch.empty_like(p.x_ref), torch.empty_like(p.x0))
    ipb = solver.autotune(p, s)
    tpi, ipb, grid = solver.launch_shape(B, N)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # capture forward and backward graphs
    for _ in range(3):
        solver.solve(p, s)
        solver.backward(p, s, gu, out=grads)
    torch.cuda.synchronize()
    g_fwd, g_bwd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g_fwd):
            solver.solve(p, s)
        with torch.cuda.graph(g_bwd):
            solver.backward(p, s, gu, out=grads)
    torch.cuda.current_stream().wait_stream(side)
    stream = torch.cuda.current_stream()

    def step(ev):
        flush.fill_(1.0)
        ev[0].record(stream)
        g_fwd.replay()
        ev[1].record(stream)
        g_bwd.replay()
        ev[2].record(stream)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        for _ in range(args.warmup):
            step([torch.cuda.Event(enable_timing=True) for _ in range(3)])
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clk.mark()
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(evs[k])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk.mark()
    if dist:
        dist.barrier()
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    fwd_ms = [e[0].elapsed_time(e[1]) for e in evs]
    ms = statistics.fmean(step_ms)
    ms_fwd = statistics.fmean(fwd_ms)
    if dist:
        t = torch.tensor([ms, ms_fwd], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_fwd = float(t[0]), float(t[1])
    status = s.status.cpu().numpy()
    iters = s.iters.cpu().numpy()

    # forward latency distribution (graph replays, cold L2)
    lat = []
    for _ in range(args.latency_reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        g_fwd.replay()
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    lat.sort()
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]

    # plain form (one launch per phase of every iteration, eager, as Sec. IV structures it)
    plain = DiffMPC(N_max=N, B_max=B, max_iter=MAX_ITER, tol=TOL, exec_mode="plain", tpi=tpi, ipb=ipb, device=dev)
    sp = plain.alloc_solution(B, N)
    gp = (torch.empty_like(p.Q), torch.empty_like(p.x_ref), torch.empty_like(p.x0))
    for _ in range(2):
        plain.solve(p, sp)
        plain.backward(p, sp, gu, out=gp)
    torch.cuda.synchronize()
    pms = []
    for _ in range(max(3, args.steps // 2)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        plain.solve(p, sp)
        plain.backward(p, sp, gu, out=gp)
        e1.record(stream)
        e1.synchronize()
        pms.append(e0.elapsed_time(e1))
    plain_ms = statistics.fmean(pms)
    same = bool(torch.equal(sp.u, s.u) and torch.equal(gp[0], grads[0]))
    plain_launches = plain.launch_count(False)
    plain.close()

    # end to end through the public API with pinned host buffers
    names = ("x0", "Q", "x_ref", "R", "u_ref", "u_lo", "u_hi")
    host_in = {k: torch.as_tensor(prob[k], dtype=torch.float32).pin_memory() for k in names}
    host_gu = torch.as_tensor(gu_np, dtype=torch.float32).pin_memory()
    host_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (s.u, grads[0], grads[1], grads[2])]
    dev_in = {k: getattr(p, k) for k in names}
    h2d = sum(t.numel() * 4 for t in host_in.values()) + host_gu.numel() * 4
    d2h = sum(t.numel() * t.element_size() for t in host_out)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        for n_ in names:
            dev_in[n_].copy_(host_in[n_], non_blocking=True)
        gu.copy_(host_gu, non_blocking=True)
        solver.solve(p, s)
        solver.backward(p, s, gu, out=grads)
        for h, d in zip(host_out, (s.u, grads[0], grads[1], grads[2])):
            h.copy_(d, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e = statistics.fmean(e2e_ms)
    side = side_configs(dev, flush) if (rank == 0 and world == 1 and not args.no_side) else None

    # roofline of the dominant kernel (the persistent forward launch)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    clocks = clk.summary()
    sm_max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    nominal_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    peak_tflops = fma_peak["burst_tflops"]
    hz = np.full(B, N)
    fwd_flops = float(np.sum(iters * (hz - 1)) * FLOP_STAGE_ITER + np.sum(hz - 1) * FLOP_STAGE_FINAL)
    achieved = fwd_flops / (ms_fwd * 1e-3) / 1e12
    fwd_launches, bwd_launches = solver.launch_count(False)
    solver.close()

    if rank != 0:
        return
    value = B * world / (ms * 1e-3)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        config=dict(workload=WORKLOAD, B_per_gpu=B, N=N, max_iter=MAX_ITER, tol=TOL,
                    exec="persistent forward + adjoint backward, each one CUDA graph replay",
                    launch=dict(threads_per_instance=tpi, instances_per_block=ipb, blocks=grid),
                    l2="flushed between steps (256 MiB write, outside the timed events)",
                    inputs="seeded synthetic race track (7 gates, 30 m loop, 0-20 m/s)"),
        p50_fwd_ms=p50, p99_fwd_ms=p99, fwd_ms=ms_fwd, bwd_ms=ms - ms_fwd,
        fwd_solves_per_s=B * world / (ms_fwd * 1e-3),
        plain=dict(value=B * world / (plain_ms * 1e-3), unit=UNIT, ms_per_step=plain_ms,
                   launches_per_step=plain_launches[0] + plain_launches[1],
                   exec="eager, one launch per phase: rollout, then per iteration Riccati (linearization fused) and line search",
                   bit_identical_to_persistent=same),
        speedup_vs_plain=plain_ms / ms,
        iters_mean=float(iters.mean()), status_counts=np.bincount(status, minlength=5).tolist(),
        e2e=dict(value=B * world / (e2e * 1e-3), unit=UNIT, ms_per_step=e2e, h2d_bytes_per_step=int(h2d),
                 d2h_bytes_per_step=int(d2h), api="paper_2605_29155_gb300.DiffMPC.solve/backward (ctypes C ABI), eager"),
        roofline=dict(kernel="k_mpc<float> persistent forward", bound="alu", achieved=achieved, peak=peak_tflops,
                      unit="TFLOP/s", frac=achieved / peak_tflops, traffic=_traffic(),
                      peak_note="of measured: FP32 FMA throughput, burst (mpc_fp32_fma_probe); nominal "
                                f"{sms} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_max_mhz:.0f} MHz = "
                                f"{nominal_tflops:.1f} TFLOP/s",
                      fp32_peak=fma_peak, flops_per_launch=fwd_flops),
        cpu_baseline=cpu,
        side_configs=side,
        clocks=clocks,
        gpu_launches=(fwd_launches + bwd_launches) * args.steps,
        wall_s_timed=wall,
    )
    print(json.dumps(line), flush=True)


def _time_fwd_bwd(solver, p, s, gu, reps, flush, stream):
    """Mean ms of eager forward + backward steps (L2 flushed before each)."""
    import torch
    grads = (torch.empty_like(p.Q), torch.empty_like(p.x_ref), torch.empty_like(p.x0))
    for _ in range(2):
        solver.solve(p, s)
        solver.backward(p, s, gu, out=grads)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        solver.solve(p, s)
        solver.backward(p, s, gu, out=grads)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.fmean(ms)


def side_configs(dev, flush, reps=3):
    """The other two batch shapes of the workload, measured beside the headline:
    uneven horizons (persistent form with the work queue, autotuned, against
    the plain form) and memory-heavy gradients (store-all tape against
    recompute: solves/s and device memory held by the torch allocator, tape
    included)."""
    import torch
    from paper_2605_29155_gb300 import DiffMPC, Problem
    stream = torch.cuda.current_stream()
    out = {}
    prob = W.cfg_uneven()
    Bu, Nu = prob["x0"].shape[0], prob["x_ref"].shape[1]
    p = Problem.from_numpy(prob, device=dev)
    gu = torch.as_tensor(W.loss_weights_u0(Bu, Nu, seed=1), dtype=torch.float32, device=dev)
    per = DiffMPC(N_max=Nu, B_max=Bu, max_iter=prob["max_iter"], tol=prob["tol"], device=dev)
    s = per.alloc_solution(Bu, Nu)
    per.autotune(p, s)
    tpi, ipb, grid = per.launch_shape(Bu, Nu)
    ms_p = _time_fwd_bwd(per, p, s, gu, reps, flush, stream)
    per.close()
    pl = DiffMPC(N_max=Nu, B_max=Bu, max_iter=prob["max_iter"], tol=prob["tol"], exec_mode="plain", tpi=tpi,
                 ipb=ipb, device=dev)
    ms_l = _time_fwd_bwd(pl, p, pl.alloc_solution(Bu, Nu), gu, reps, flush, stream)
    pl.close()
    out["uneven"] = dict(workload=f"B={Bu}, horizons U{{5..40}}, <= {prob['max_iter']} iterations, u_hi x U(0.8, 1.2)",
                         persistent_solves_per_s=Bu / (ms_p * 1e-3), plain_solves_per_s=Bu / (ms_l * 1e-3),
                         launch=dict(threads_per_instance=tpi, instances_per_block=ipb, blocks=grid))
    prob = W.cfg_mem()
    Bm, Nm = prob["x0"].shape[0], prob["x_ref"].shape[1]
    p = Problem.from_numpy(prob, device=dev)
    gu = torch.as_tensor(W.loss_weights_u0(Bm, Nm, seed=1), dtype=torch.float32, device=dev)
    mem = {}
    for mode in ("store_all", "recompute"):
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        sol = DiffMPC(N_max=Nm, B_max=Bm, max_iter=prob["max_iter"], tol=prob["tol"], store_mode=mode, device=dev)
        s = sol.alloc_solution(Bm, Nm)
        ms = _time_fwd_bwd(sol, p, s, gu, reps, flush, stream)
        tape = 0 if s.tape is None else s.tape.numel() * s.tape.element_size()
        mem[mode] = dict(solves_per_s=Bm / (ms * 1e-3), ms_per_step=ms, tape_bytes=tape,
                         torch_peak_bytes=int(torch.cuda.max_memory_allocated() - base))
        del s
        sol.close()
    out["mem"] = dict(workload=f"B={Bm}, N={Nm}, per-stage Q and x_ref, fwd+bwd", **mem)
    out["hover_latency"] = hover_latency(dev, flush)
    out["policy_latency"] = policy_latency(dev, flush)
    out["closed_loop_track"] = closed_loop_track(dev)
    out["general_cost"] = general_cost_track(dev, flush, reps)
    out["costmap_fused"] = costmap_fused_track(dev, flush)
    return out


def costmap_fused_track(dev, flush, B=4096, N=20, reps=20):
    """The actor's cost map fused with the solve (Sec. V-A, Algorithm 2's
    (C, c) <- pi(x)): observation -> 2 x 512 ReLU -> sigmoid-scaled Q_t written
    straight into the solve's Q buffer -> MPC forward -> adjoint dL/dQ ->
    cost-map backward to the weights, all four in one CUDA graph; the MLP's
    layers run on the tensor cores (tcgen05, 3xTF32).  Random-init weights of
    that architecture; L2 flushed between replays.  Also the MLP's forward
    and backward alone, each its own graph."""
    import torch
    from paper_2605_29155_gb300 import CostMap, DiffMPC, Problem
    prob = W.race_track(B, N, seed=0)
    params = W.costmap_weights(26, N * 13, seed=0)
    p = Problem.from_numpy(dict(prob, Q=np.ones((B, N, 13))), device=dev)
    gu = torch.as_tensor(W.loss_weights_u0(B, N, seed=1), dtype=torch.float32, device=dev)
    cm = CostMap(params, N, B, device=dev)
    sol = DiffMPC(N_max=N, B_max=B, max_iter=MAX_ITER, tol=TOL, device=dev)
    s = sol.alloc_solution(B, N)
    cm.forward(p.x0, p.x_ref, Q=p.Q)
    sol.autotune(p, s)
    grads = (torch.empty_like(p.Q), torch.empty_like(p.x_ref), torch.empty_like(p.x0))
    wg = [torch.empty_like(t) for t in (cm.W1, cm.b1, cm.W2, cm.b2, cm.W3, cm.b3)]

    def whole():
        cm.forward(p.x0, p.x_ref, Q=p.Q)
        sol.solve(p, s)
        sol.backward(p, s, gu, out=grads)
        cm.backward(p.x0, p.x_ref, grads[0], out=wg)

    def mlp_fwd():
        cm.forward(p.x0, p.x_ref, Q=p.Q)

    def mlp_bwd():
        cm.backward(p.x0, p.x_ref, grads[0], out=wg)

    graphs = {}
    side = torch.cuda.Stream(device=dev)
    for name, fn in (("fused", whole), ("mlp_fwd", mlp_fwd), ("mlp_bwd", mlp_bwd)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        graphs[name] = g
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms = {}
    for name, g in graphs.items():
        t = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(1.0)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        ms[name] = statistics.median(t)
    flops_fwd = 2.0 * B * (26 * 512 + 512 * 512 + 512 * N * 13)
    flag = cm.wait_flag()
    res = dict(workload=f"race track B={B}, N={N}: cost map (26 -> 512 -> 512 -> {N * 13}, random init) -> "
                        "MPC fwd+bwd -> cost-map bwd, one CUDA graph",
               solves_per_s=B / (ms["fused"] * 1e-3), ms_fused=ms["fused"], ms_mlp_fwd=ms["mlp_fwd"],
               ms_mlp_bwd=ms["mlp_bwd"], mlp_share=(ms["mlp_fwd"] + ms["mlp_bwd"]) / ms["fused"],
               mlp_fwd_tflops_3xtf32=3 * flops_fwd / (ms["mlp_fwd"] * 1e-3) / 1e12,
               mlp_fwd_flops=flops_fwd, device_wait_flag=flag, iters_mean=float(s.iters.float().mean()))
    sol.close()
    return res


def general_cost_track(dev, flush, reps, B=4096, N=20):
    """The benchmark batch with the general stage cost of Eq. (2): a dense C
    per instance (diag(Q, R) + 0.05 M'M / 17, M ~ N(0, 1), shared over the
    stages) and c_t = -C z_ref,t per stage; forward + backward (dL/dC, dL/dc,
    dL/dx0), eager, L2 flushed before each step."""
    import torch
    from paper_2605_29155_gb300 import DiffMPC, Problem
    prob = W.race_track(B, N, seed=0)
    rng = np.random.default_rng(21)
    M = rng.normal(size=(B, 17, 17))
    diag = np.concatenate([prob["Q"][:, 0], prob["R"]], axis=1)
    C = np.einsum("bi,ij->bij", diag, np.eye(17)) + 0.05 * np.einsum("bki,bkj->bij", M, M) / 17
    zr = np.concatenate([prob["x_ref"], np.repeat(prob["u_ref"][:, None], N, axis=1)], axis=2)
    c = -np.einsum("bij,btj->bti", C, zr)
    p = Problem.from_numpy(dict(prob, C=C[:, None], c=c), device=dev)
    gu = torch.as_tensor(W.loss_weights_u0(B, N, seed=1), dtype=torch.float32, device=dev)
    sol = DiffMPC(N_max=N, B_max=B, max_iter=MAX_ITER, tol=TOL, device=dev)
    s = sol.alloc_solution(B, N)
    sol.autotune(p, s)
    out = (torch.empty_like(p.C), torch.empty_like(p.c), torch.empty_like(p.x0))
    for _ in range(2):
        sol.solve(p, s)
        sol.backward_general(p, s, gu, out=out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms, fw = [], []
    for _ in range(max(reps, 5)):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        flush.fill_(1.0)
        e0.record(stream)
        sol.solve(p, s)
        e1.record(stream)
        sol.backward_general(p, s, gu, out=out)
        e2.record(stream)
        e2.synchronize()
        ms.append(e0.elapsed_time(e2))
        fw.append(e0.elapsed_time(e1))
    res = dict(workload=f"race track B={B}, N={N}, dense C (shared) and per-stage c, fwd+bwd",
               solves_per_s=B / (statistics.fmean(ms) * 1e-3), fwd_ms=statistics.fmean(fw),
               bwd_ms=statistics.fmean(ms) - statistics.fmean(fw), iters_mean=float(s.iters.float().mean()),
               launch=list(sol.launch_shape(B, N)))
    sol.close()
    return res


def policy_latency(dev, flush, reps=30):
    """Per-call latency of a policy inference in the setting of the paper's
    Table IV: one observation -> cost map (26 -> 512 -> 512 -> T * 13, random
    init) writing Q_t -> MPC forward with exactly K iterations (tol 0), for T
    in {2, 5, 10} and K in {1, 5, 10}, one race-track instance.  Eager calls,
    CUDA events around the cost map and the solve on their stream, L2 flushed
    before each; medians of `reps` calls."""
    import torch
    from paper_2605_29155_gb300 import CostMap, DiffMPC, Problem
    stream = torch.cuda.current_stream()
    rows = []
    for Th in (2, 5, 10):
        prob = W.race_track(1, Th, seed=5)
        p = Problem.from_numpy(dict(prob, Q=np.ones((1, Th, 13))), device=dev)
        cm = CostMap(W.costmap_weights(26, Th * 13, seed=6), Th, 1)
        for Kh in (1, 5, 10):
            sol = DiffMPC(N_max=Th, B_max=1, max_iter=Kh, tol=0.0, device=dev)
            s = sol.alloc_solution(1, Th)
            for _ in range(3):
                cm.forward(p.x0, p.x_ref, Q=p.Q)
                sol.solve(p, s)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                cm.forward(p.x0, p.x_ref, Q=p.Q)
                sol.solve(p, s)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            rows.append(dict(T=Th, K=Kh, device_ms=statistics.median(ts), iters=int(s.iters[0]),
                             wait_flag=cm.wait_flag()))
            sol.close()
    return dict(workload="one race-track observation -> cost map -> MPC forward with exactly K iterations, "
                         "eager calls, medians of %d" % reps, rows=rows)


def closed_loop_track(dev, B=4096, N=20, K=50):
    """Receding-horizon control on the race-track batch (the loop of
    Algorithm 2 around the solve): each of K environment steps solves the
    forward problem, moves every instance to its predicted x_1, slides the
    reference window by one stage and warm-starts the next solve from the
    shifted controls.  Timed with CUDA events over all K steps (eager calls;
    the shifts are device copies)."""
    import torch
    from paper_2605_29155_gb300 import DiffMPC, Problem
    prob = W.race_track(B, N + K, seed=0)
    full_ref = torch.as_tensor(prob["x_ref"], dtype=torch.float32, device=dev)
    p = Problem.from_numpy(dict(prob, x_ref=np.ascontiguousarray(prob["x_ref"][:, :N])), device=dev)
    x0_start = p.x0.clone()
    sol = DiffMPC(N_max=N, B_max=B, max_iter=MAX_ITER, tol=TOL, device=dev)
    s = sol.alloc_solution(B, N)
    sol.autotune(p, s)
    u_init = torch.empty(B, N, 4, dtype=torch.float32, device=dev)
    iters = torch.zeros(B, dtype=torch.int64, device=dev)

    def run():
        p.x0.copy_(x0_start)
        p.u_init = None
        iters.zero_()
        for k in range(K):
            p.x_ref.copy_(full_ref[:, k:k + N])
            sol.solve(p, s)
            iters.add_(s.iters)
            p.x0.copy_(s.x[:, 1])
            u_init[:, :-1].copy_(s.u[:, 1:])
            u_init[:, -1].copy_(s.u[:, -1])
            p.u_init = u_init

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    err = torch.linalg.norm(p.x0[:, 0:3] - full_ref[:, K, 0:3], dim=1)
    out = dict(workload=f"race track B={B}, N={N}, {K} receding-horizon steps, <= {MAX_ITER} iterations each, "
                        "warm start from the shifted solution",
               instance_steps_per_s=B * K / (ms * 1e-3), ms_per_env_step=ms / K,
               iters_per_solve=float(iters.float().mean()) / K,
               final_position_error_m_median=float(err.median()))
    sol.close()
    return out


def hover_latency(dev, flush, reps=30):
    """Per-call latency in the setting of the paper's solver-latency comparison
    (Sec. V, Table II): hover stabilisation at random targets, B in {1, 256},
    horizon N in {2, 10, 50}.  Each call runs exactly 5 iterations (tol 0),
    the upper bound of a control update.  Eager API calls (what a control loop
    issues), L2 flushed before each; medians of `reps` calls:
      device_ms  CUDA events around the call on its stream (host launch
                 overhead included, since the GPU waits for it)
      wall_ms    host clock around the call plus a synchronize."""
    import torch
    from paper_2605_29155_gb300 import DiffMPC, Problem
    stream = torch.cuda.current_stream()
    rows = []
    for Bh in (1, 256):
        for Nh in (2, 10, 50):
            prob = W.hover_targets(Bh, Nh, seed=4)
            p = Problem.from_numpy(prob, device=dev)
            gu = torch.as_tensor(W.loss_weights_u0(Bh, Nh, seed=1), dtype=torch.float32, device=dev)
            sol = DiffMPC(N_max=Nh, B_max=Bh, max_iter=5, tol=0.0, device=dev)
            s = sol.alloc_solution(Bh, Nh)
            grads = (torch.empty_like(p.Q), torch.empty_like(p.x_ref), torch.empty_like(p.x0))
            sol.autotune(p, s)
            for _ in range(3):
                sol.solve(p, s)
                sol.backward(p, s, gu, out=grads)
            torch.cuda.synchronize()
            t = {k: [] for k in ("fwd_dev", "bwd_dev", "fwd_wall", "bwd_wall")}
            for _ in range(reps):
                for part in ("fwd", "bwd"):
                    flush.fill_(1.0)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    w0 = time.perf_counter()
                    e0.record(stream)
                    if part == "fwd":
                        sol.solve(p, s)
                    else:
                        sol.backward(p, s, gu, out=grads)
                    e1.record(stream)
                    e1.synchronize()
                    t[part + "_wall"].append((time.perf_counter() - w0) * 1e3)
                    t[part + "_dev"].append(e0.elapsed_time(e1))
            med = {k: statistics.median(v) for k, v in t.items()}
            row = dict(B=Bh, N=Nh, fwd_device_ms=med["fwd_dev"], bwd_device_ms=med["bwd_dev"],
                       fwd_wall_ms=med["fwd_wall"], bwd_wall_ms=med["bwd_wall"],
                       iters=float(s.iters.float().mean()), launch=list(sol.launch_shape(Bh, Nh)))
            sol.close()
            # the stage-parallel Riccati form (one instance per block; its
            # final factorization writes the tape the backward replays)
            sc = DiffMPC(N_max=Nh, B_max=Bh, max_iter=5, tol=0.0, device=dev, exec_mode="scan")
            ss = sc.alloc_solution(Bh, Nh)
            for _ in range(3):
                sc.solve(p, ss)
                sc.backward(p, ss, gu, out=grads)
            torch.cuda.synchronize()
            tf, tb = [], []
            for _ in range(reps):
                for part, acc in (("fwd", tf), ("bwd", tb)):
                    flush.fill_(1.0)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    if part == "fwd":
                        sc.solve(p, ss)
                    else:
                        sc.backward(p, ss, gu, out=grads)
                    e1.record(stream)
                    e1.synchronize()
                    acc.append(e0.elapsed_time(e1))
            row.update(scan_fwd_device_ms=statistics.median(tf), scan_bwd_device_ms=statistics.median(tb))
            sc.close()
            rows.append(row)
    return dict(workload="hover stabilisation at random targets, exactly 5 iterations (tol 0), fwd and bwd "
                         "per eager API call, medians of %d; scan_*: exec_mode scan (stage-parallel Riccati)" % reps,
                rows=rows)


def run_kernels_only(args):
    """W + K eager forward+backward steps on the benchmark workload, nothing
    else: the command the committed ncu summaries were taken with."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_29155_gb300 import DiffMPC, Problem

    Bk = args.batch
    prob = W.cfg_track(B=Bk)
    p = Problem.from_numpy(prob)
    gu = torch.as_tensor(W.loss_weights_u0(Bk, N, seed=1), dtype=torch.float32, device="cuda")
    solver = DiffMPC(N_max=N, B_max=Bk, max_iter=MAX_ITER, tol=TOL, tpi=args.tpi, ipb=args.ipb)
    s = solver.alloc_solution(Bk, N)
    grads = (torch.empty_like(p.Q), torch.empty_like(p.x_ref), torch.empty_like(p.x0))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.warmup + args.steps):
        if k == args.warmup:
            torch.cuda.synchronize()
            e0.record()
        solver.solve(p, s)
        solver.backward(p, s, gu, out=grads)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps(dict(mode="kernels", B=Bk, N=N, steps=args.steps, ms_per_step=e0.elapsed_time(e1) / args.steps,
                          launch=solver.launch_shape(Bk, N), iters_mean=float(s.iters.float().mean()))))
    solver.close()


def run_costmap_only(args):
    """W + K eager cost-map forward + backward passes (B instances, N = 20,
    random-init weights), nothing else: the command the committed ncu summary
    of the tensor-core kernel was taken with."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_29155_gb300 import CostMap
    Bk = args.batch
    prob = W.race_track(Bk, N, seed=0)
    cm = CostMap(W.costmap_weights(26, N * 13, seed=0), N, Bk)
    x0 = torch.as_tensor(prob["x0"], dtype=torch.float32, device="cuda")
    xr = torch.as_tensor(prob["x_ref"], dtype=torch.float32, device="cuda")
    dQ = torch.as_tensor(np.random.default_rng(1).normal(size=(Bk, N, 13)), dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.warmup + args.steps):
        if k == args.warmup:
            torch.cuda.synchronize()
            e0.record()
        cm.forward(x0, xr)
        cm.backward(x0, xr, dQ)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps(dict(mode="costmap", B=Bk, N=N, steps=args.steps, ms_per_step=e0.elapsed_time(e1) / args.steps,
                          wait_flag=cm.wait_flag())))


def run_scan_only(args):
    """W + K eager forward solves in the stage-parallel Riccati form (hover
    stabilisation, B instances, N = 50, exactly 5 iterations), nothing else:
    the command the committed ncu summary of k_scan_ric was taken with."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_29155_gb300 import DiffMPC, Problem
    Bk, Nh = args.batch, 50
    p = Problem.from_numpy(W.hover_targets(Bk, Nh, seed=4))
    solver = DiffMPC(N_max=Nh, B_max=Bk, max_iter=5, tol=0.0, exec_mode="scan", store_mode="recompute")
    s = solver.alloc_solution(Bk, Nh)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.warmup + args.steps):
        if k == args.warmup:
            torch.cuda.synchronize()
            e0.record()
        solver.solve(p, s)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps(dict(mode="scan", B=Bk, N=Nh, steps=args.steps, ms_per_step=e0.elapsed_time(e1) / args.steps,
                          iters_mean=float(s.iters.float().mean()))))
    solver.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--latency-reps", type=int, default=200)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-side", action="store_true", help="skip the uneven-horizon and memory-heavy batches")
    ap.add_argument("--mode", default="full", choices=["full", "kernels", "costmap", "scan"],
                    help="kernels: only W + K eager forward+backward steps of the workload (for profilers); "
                         "costmap: only W + K cost-map forward+backward passes; "
                         "scan: only W + K stage-parallel forward solves (hover, N = 50)")
    ap.add_argument("--batch", type=int, default=B, help="instances (kernels, costmap and scan modes)")
    ap.add_argument("--tpi", type=int, default=0, help="threads per instance, 0 = default (kernels mode only)")
    ap.add_argument("--ipb", type=int, default=0, help="instances per block, 0 = default (kernels mode only)")
    args = ap.parse_args()
    if args.mode == "kernels":
        run_kernels_only(args)
        return
    if args.mode == "costmap":
        run_costmap_only(args)
        return
    if args.mode == "scan":
        run_scan_only(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus == 1 else 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
