"""Benchmark of the GB300 ellsolve library on the cubed-sphere workload.

Default workload (one GPU): equiangular cubed sphere 6 x 512 x 512 cells x 128
quadratically graded levels on r in [1, 1.01] (201,326,592 unknowns),
omega^2 = 0.01, lambda = 1, right-hand side N(0, 1) smoothed by three in-panel
Jacobi sweeps; FP32 V-cycles (2/2 line-Jacobi sweeps, damping 0.8, coarsened to
4 x 4 per panel) inside FP64 iterative refinement, each refinement step replayed
as one CUDA graph.  One step = one solve from x = 0 to a 1e-5 relative residual
reduction.  Metric: unknowns x V-cycles per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload sphere512|sphere128|box256]

Under torchrun every rank solves its own instance of the workload (the solve
itself is not split across GPUs); value = all ranks' unknowns x V-cycles / the
slowest rank's time.  --impl reference times the FP64 CPU oracle instead, on a
bounded sample of the same workload (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "unknowns*V-cycles/s"
WORKLOADS = {
    # name: (kind, n, nz, graded, omega2, lambda2, rhs, rtol)
    "sphere512": (1, 512, 128, True, 0.01, 1.0, "smooth_gauss", 1e-5),
    "sphere256": (1, 256, 128, True, 0.01, 1.0, "smooth_gauss", 1e-5),
    "sphere128": (1, 128, 128, True, 0.01, 1.0, "smooth_gauss", 1e-5),
    "box256": (0, 256, 64, True, 0.01, 1.0, "uniform", 1e-5),
}
# bounded oracle sample for the CPU baseline: the same sphere at 1/16 of the columns
ORACLE_SAMPLE = (1, 128, 128, True, 0.01, 1.0)


def rhs_for(kind, n, nz, how, member=0):
    from paper_1307_2036_gb300 import inputs
    shape = (nz, 1 if kind == 0 else 6, n, n)
    if how == "uniform":
        return inputs.uniform_pm1(shape, member=member)
    return inputs.smooth_per_panel(inputs.gaussian(shape, member=member), sweeps=3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        out = os.environ.get("ELLSOLVE_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out, f"clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


_oracle_barrier = None
# every CPU this process may use, taken before the process is bound to the CPUs
# local to its GPU: the oracle's CPU baseline runs on all of them
HOST_CPUS_ALL = sorted(os.sched_getaffinity(0))


def _oracle_init(barrier, cpus):
    global _oracle_barrier
    _oracle_barrier = barrier
    os.sched_setaffinity(0, cpus)


def _oracle_one(job):
    """One worker of the parallel oracle timing: set up the sample problem
    (member `m`), wait for every worker, then time the V-cycles and residual."""
    import numpy as np

    import oracle
    from paper_1307_2036_gb300 import inputs
    sample, vcycles, m = job
    kind, n, nz, graded, w2, l2 = sample
    og = oracle.Grid(kind, n, nz, inputs.radial_levels(nz, graded=graded), w2, l2)
    f = rhs_for(kind, n, nz, "smooth_gauss" if kind == 1 else "uniform", member=m)
    b = og.volumes() * f
    u = np.zeros_like(b)
    _oracle_barrier.wait()
    t0 = time.perf_counter()
    for _ in range(vcycles):
        u = og.vcycle(b, u)
    og.residual(b, u)
    return b.size * vcycles, time.perf_counter() - t0


def oracle_rate_parallel(sample, vcycles, procs=None):
    """The oracle as it stands, one single-threaded process per host core, all
    timed together (the processes are spawned: this process may hold a CUDA
    context).  Returns (unknowns * V-cycles / s over the slowest process,
    seconds, processes, description)."""
    import multiprocessing as mp
    if procs is None:
        procs = max(1, len(HOST_CPUS_ALL))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    with ctx.Pool(procs, initializer=_oracle_init, initargs=(barrier, HOST_CPUS_ALL)) as pool:
        res = pool.map(_oracle_one, [(sample, vcycles, m) for m in range(procs)])
    work = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    kind, n, nz = sample[0], sample[1], sample[2]
    desc = (f"oracle (plain C, FP64, one thread per process) on {procs} processes at once "
            f"(host CPUs {HOST_CPUS_ALL[0]}-{HOST_CPUS_ALL[-1]}), "
            f"each {vcycles} V-cycle(s) + residual on the {'sphere 6x' if kind == 1 else 'box '}"
            f"{n}x{n}x{nz} graded grid ({work // (procs * vcycles)} unknowns, its own "
            f"right-hand side)")
    return work / dt, dt, procs, desc


def run_reference(args, rank, world):
    if rank != 0:
        return
    works, times, desc, procs = [], [], "", 1
    for i in range(args.warmup + args.steps):
        r, dt, procs, desc = oracle_rate_parallel(ORACLE_SAMPLE, 1)
        if i >= args.warmup:
            works.append(r * dt)
            times.append(dt)
    value = sum(works) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns*V-cycles/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "unknowns*V-cycles/s", "cores": procs,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "unknowns*V-cycles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_ranks(dist, ms, ms_e2e, cycles, e2e_cycles, device="cpu"):
    """Whole-job figures over the ranks: the slowest rank's times, the summed
    V-cycles (each rank solves its own problem of N unknowns)."""
    import torch
    t = torch.tensor([ms, ms_e2e, float(cycles), float(e2e_cycles)], dtype=torch.float64,
                     device=device)
    tmax, tsum = t.clone(), t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tmax[1]), float(tsum[2]), float(tsum[3])


def bind_host_to_gpu(torch, dev):
    """Run this process on the CPUs next to the GPU (its PCI device's
    local_cpulist), so that pinned host buffers allocated afterwards sit in
    that NUMA node and the copies do not cross sockets.  Returns the CPU list,
    or None when the system does not say."""
    try:
        props = torch.cuda.get_device_properties(dev)
        dom = getattr(props, "pci_domain_id", 0)
        bus = getattr(props, "pci_bus_id", None)
        slot = getattr(props, "pci_device_id", None)
        if bus is None or slot is None:
            return None
        path = f"/sys/bus/pci/devices/{dom:04x}:{bus:02x}:{slot:02x}.0/local_cpulist"
        with open(path) as fh:
            text = fh.read().strip()
        cpus = set()
        for part in text.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return text
    except (OSError, ValueError, AttributeError):
        return None


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1307_2036_gb300 import ellsolve, inputs

    torch.cuda.set_device(local_rank)
    host_cpus = bind_host_to_gpu(torch, local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    kind, n, nz, graded, w2, l2, rhs_kind, rtol = WORKLOADS[args.workload]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sv = ellsolve.Solver(kind, n, nz, inputs.radial_levels(nz, graded=graded), w2, l2,
                             precision=1, use_graph=1, inner_cycles=args.inner_cycles,
                             stream=stream.cuda_stream)
        f_host = torch.from_numpy(rhs_for(kind, n, nz, rhs_kind, member=rank)).pin_memory()
        f = f_host.to("cuda", non_blocking=True)
        x = torch.zeros_like(f)
        x_host = torch.empty_like(f_host).pin_memory()
    stream.synchronize()
    N = sv.N
    if args.shapes_in:
        # the launch shapes an earlier run's autotuner chose (for a profiled
        # rerun of the same launches: timing under a profiler is distorted)
        with open(args.shapes_in) as fh:
            for l, shp in enumerate(json.load(fh)):
                sv.set_level_tuning(l, *shp)
        tuned_ctas = sv.level_tuning(0)[0]
    else:
        tuned_ctas, tuned_ms = sv.autotune()
    level_shapes = [list(sv.level_tuning(l)) for l in range(sv.nlevels)]
    if args.shapes_out:
        with open(args.shapes_out, "w") as fh:
            json.dump(level_shapes, fh)

    def solve():
        st, res = sv.solve(f, x, rtol=rtol, maxit=60)
        if st < 0:
            raise RuntimeError(f"solve failed: {st}")
        return res

    for _ in range(args.warmup):
        res = solve()
    vcycles_per_solve = res.iterations

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # device-timed region: K solves with inputs resident in HBM
    sampler = ClockSampler(local_rank)
    barrier()
    sampler.start()
    l0 = sv.launch_count()
    sv.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cycles = 0
    e0.record(stream)
    for _ in range(args.steps):
        cycles += solve().iterations
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    launches = sv.launch_count() - l0
    ms = e0.elapsed_time(e1)
    prof_ms, prof_n, prof_bytes = sv.profile_read()
    sv.profile(False)
    final_rel = res.rel_residual

    # End-to-end region: every step copies its right-hand side from pinned host
    # memory to the device, solves through the C ABI and copies the solution
    # back to pinned host memory.  The copies run on their own streams into
    # double buffers, so that step i+1's input and step i-1's output move while
    # step i solves (the copy engines work beside the kernels); all of them lie
    # inside the timed region.
    barrier()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        fd = [f, torch.empty_like(f)]
        xd = [x, torch.zeros_like(x)]
    stream.synchronize()
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    # the copy bandwidth of this machine, alone (outside the timed region; one
    # untimed copy each way first, so that first-touch costs are not counted)
    with torch.cuda.stream(h2d):
        fd[1].copy_(f_host, non_blocking=True)
        x_host.copy_(xd[1], non_blocking=True)
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0.record(h2d)
    with torch.cuda.stream(h2d):
        fd[1].copy_(f_host, non_blocking=True)
    c1.record(h2d)
    with torch.cuda.stream(h2d):
        x_host.copy_(xd[1], non_blocking=True)
    c2.record(h2d)
    h2d.synchronize()
    copy_gbs = (N * 8 / (c0.elapsed_time(c1) * 1e6), N * 8 / (c1.elapsed_time(c2) * 1e6))
    solve_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_solved = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e2e_cycles = 0
    K = args.steps
    cin = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    cout = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(K)]
    h0.record(stream)
    h2d.wait_event(h0)
    with torch.cuda.stream(h2d):
        fd[0].copy_(f_host, non_blocking=True)
        ev_in[0].record(h2d)
    for i in range(K):
        j = i % 2
        if i + 1 < K:  # the next step's input, into the other buffer once it is free
            if i >= 1:
                h2d.wait_event(ev_solved[1 - j])
            with torch.cuda.stream(h2d):
                cin[i][0].record(h2d)
                fd[1 - j].copy_(f_host, non_blocking=True)
                cin[i][1].record(h2d)
                ev_in[1 - j].record(h2d)
        stream.wait_event(ev_in[j])
        if i >= 2:
            stream.wait_event(ev_out[j])  # the solution of step i-2 has left this buffer
        solve_ev[i][0].record(stream)
        st, res = sv.solve(fd[j], xd[j], rtol=rtol, maxit=60)
        solve_ev[i][1].record(stream)
        if st < 0:
            raise RuntimeError(f"solve failed: {st}")
        e2e_cycles += res.iterations
        ev_solved[j].record(stream)
        d2h.wait_event(ev_solved[j])
        with torch.cuda.stream(d2h):
            cout[i][0].record(d2h)
            x_host.copy_(xd[j], non_blocking=True)
            cout[i][1].record(d2h)
            ev_out[j].record(d2h)
    for j in range(min(2, K)):
        stream.wait_event(ev_out[j])
    h1.record(stream)
    barrier()
    ms_e2e = h0.elapsed_time(h1)
    e2e_solve_ms = sum(a.elapsed_time(b) for a, b in solve_ev) / max(1, len(solve_ev))
    # the copies' own durations inside the loop (beside the solves)
    cin_ms = [a.elapsed_time(b) for a, b in cin[:max(0, K - 1)]]
    cout_ms = [a.elapsed_time(b) for a, b in cout[:K]]
    del fd, xd

    if dist is not None:
        ms, ms_e2e, cycles, e2e_cycles = aggregate_ranks(dist, ms, ms_e2e, cycles, e2e_cycles,
                                                         device="cuda")
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    value = N * cycles / (ms * 1e-3)
    e2e = N * e2e_cycles / (ms_e2e * 1e-3)
    peak, peak_kind = measured_peaks()
    achieved = (prof_bytes / (prof_ms * 1e-3) / 1e9) if prof_ms > 0 else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "smoother_traffic.txt")
    if os.path.exists(tfile):
        with open(tfile) as fh:
            tinfo = json.load(fh)
        if tinfo.get("workload") == args.workload and tinfo.get("kernel_rev") == KERNEL_REV:
            traffic = tinfo.get("dram_bytes_per_launch")
    # the oracle's CPU baseline: rank 0 of a single-GPU run only
    cpu_rate, cpu_s, cpu_cores, cpu_desc = (oracle_rate_parallel(ORACLE_SAMPLE, 1)
                                            if not args.no_cpu and world == 1
                                            else (None, 0, 1, ""))
    extras = {}
    if not args.no_extras:
        del sv
        torch.cuda.empty_cache()
        extras["ensemble"] = run_ensemble(torch, stream)
        extras["serving"] = run_serving(torch, stream, args.serve_requests)
        extras["smoothers"] = run_smoothers(torch, stream, args.workload)
        extras["configs"] = run_configs(torch, stream)
        extras["accuracy"] = run_accuracy(torch, stream, args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": "unknowns*V-cycles/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {
            "workload": args.workload, "grid": ("cubed sphere 6x" if kind == 1 else "box ") +
            f"{n}x{n}", "nz": nz, "unknowns": N, "omega2": w2, "lambda": l2 ** 0.5,
            "solver": ("FP32 V-cycle (2/2 line-Jacobi, rho 0.8) in FP64 refinement with the "
                       "tracked residual, CUDA graph"),
            "inner_cycles": args.inner_cycles,
            "autotuned_smoother_ctas_per_sm": tuned_ctas,
            "autotuned_level_shapes": {
                "fields": "smoother CTAs/SM, ring steps, tmem (0 auto, 1 on, 2 off), staged "
                          "(0 auto, 1 on, 2 off), restrict chunk blocks, prolong chunk blocks",
                "levels": level_shapes},
            "rtol": rtol, "vcycles_per_solve": vcycles_per_solve,
            "final_rel_residual": final_rel, "time_to_rtol_ms": ms / args.steps,
            "rel_error_est": res.rel_error_est,
            "l2_policy": "inputs larger than L2 (FP32 hierarchy %.1f GB)" % (N * 16 / 3 * 4 / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": "k_smooth_tw finest level (FP32 line-Jacobi sweep, twisted elimination)",
                     "launches_timed": prof_n, "peak_source": peak_kind},
        "cpu_baseline": {"value": cpu_rate, "unit": "unknowns*V-cycles/s", "cores": cpu_cores,
                         "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": e2e, "unit": "unknowns*V-cycles/s", "h2d_bytes_per_step": N * 8,
                "d2h_bytes_per_step": N * 8,
                "copies": "pinned host <-> device on copy streams, double-buffered: step i+1's "
                          "input and step i-1's output move during step i's solve",
                "copy_gbs_alone": {"h2d": copy_gbs[0], "d2h": copy_gbs[1]},
                "host_cpus": host_cpus,
                "solve_ms_in_loop": e2e_solve_ms,
                "copy_ms_in_loop": {
                    "h2d": sum(cin_ms) / len(cin_ms) if cin_ms else None,
                    "d2h": sum(cout_ms) / len(cout_ms) if cout_ms else None}},
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_accuracy(torch, stream, workload):
    """The benchmark workload solved to 1e-10 in mixed precision and to 1e-12
    by the FP64 multigrid (whose results match the oracle's to 1e-10 in the
    parity tests): relative L2 difference of the two solutions, with times."""
    from paper_1307_2036_gb300 import ellsolve, inputs
    kind, n, nz, graded, w2, l2, rhs_kind, _ = WORKLOADS[workload]
    r = inputs.radial_levels(nz, graded=graded)
    with torch.cuda.stream(stream):
        f = torch.from_numpy(rhs_for(kind, n, nz, rhs_kind)).to("cuda")
        xm = torch.zeros_like(f)
        x64 = torch.zeros_like(f)
    stream.synchronize()
    out = {"workload": f"{workload}: mixed precision to 1e-10 against FP64 multigrid to 1e-12"}
    for name, x, kw, rtol in (("mixed", xm, dict(precision=1, use_graph=1), 1e-10),
                              ("fp64", x64, dict(precision=0), 1e-12)):
        sv = ellsolve.Solver(kind, n, nz, r, w2, l2, stream=stream.cuda_stream, **kw)
        if name == "mixed":
            sv.autotune()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        st, res = sv.solve(f, x, rtol=rtol, maxit=100)
        e1.record(stream)
        stream.synchronize()
        out[name] = {"ms": e0.elapsed_time(e1), "vcycles": res.iterations,
                     "rel_residual": res.rel_residual, "status": int(st)}
        if name == "mixed":
            out[name]["rel_error_est"] = res.rel_error_est
        sv.close()
    with torch.cuda.stream(stream):
        err = float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64))
    stream.synchronize()
    out["rel_l2_mixed_vs_fp64"] = err
    del f, xm, x64
    torch.cuda.empty_cache()
    return out


def run_configs(torch, stream):
    """The small workloads beside the benchmark workload.  box32: box 32x32,
    n_z = 32 uniform on [1, 1.01], omega^2 = 0.01, lambda = 1, seeded uniform
    and manufactured (3, 5) x cos m = 2 right-hand sides, time to 1e-5 for FP64
    multigrid, mixed precision and PCG (latency-bound: time to solution, not a
    roofline).  box256_sweep: box 256x256, n_z = 64 graded, the 9 cases omega^2 x lambda
    with a uniform right-hand side: FP64 multigrid and PCG to 1e-5, mixed
    precision to 1e-10 (V-cycles or iterations, time, status)."""
    import numpy as np

    from paper_1307_2036_gb300 import ellsolve, inputs

    def timed(sv, f, x, rtol, maxit):
        sv.solve(f, x, rtol=rtol, maxit=maxit)  # warm-up (graph capture)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        st, res = sv.solve(f, x, rtol=rtol, maxit=maxit)
        e1.record(stream)
        stream.synchronize()
        return {"ms": e0.elapsed_time(e1), "iterations": res.iterations,
                "rel_residual": res.rel_residual, "status": int(st)}

    solvers = (("fp64 multigrid", dict(precision=0), 1e-5, 100),
               ("mixed multigrid", dict(precision=1, use_graph=1), 1e-5, 100),
               ("fp64 pcg", dict(precision=0, solver=1), 1e-5, 2000))
    out = {"box32": {"workload": "box 32x32x32 uniform, omega2 0.01, lambda 1, rtol 1e-5"}}
    r1 = inputs.radial_levels(32)
    for rhs_name, fh in (("uniform", inputs.uniform_pm1((32, 1, 32, 32))),
                         ("manufactured", inputs.fourier_cos_mode(32, 32))):
        with torch.cuda.stream(stream):
            f = torch.from_numpy(np.ascontiguousarray(fh)).to("cuda")
            x = torch.zeros_like(f)
        stream.synchronize()
        for name, kw, rtol, maxit in solvers:
            sv = ellsolve.Solver(0, 32, 32, r1, 0.01, 1.0, stream=stream.cuda_stream, **kw)
            out["box32"][f"{rhs_name}, {name}"] = timed(sv, f, x, rtol, maxit)
            sv.close()
    nb, nzb = 256, 64
    rb = inputs.radial_levels(nzb, graded=True)
    with torch.cuda.stream(stream):
        fb = torch.from_numpy(rhs_for(0, nb, nzb, "uniform")).to("cuda")
        xb = torch.zeros_like(fb)
    stream.synchronize()
    out["box256_sweep"] = {"workload": "box 256x256x64 graded, uniform RHS; multigrid and PCG to 1e-5, "
                             "mixed precision to 1e-10", "cases": []}
    for w2 in (1e-3, 1e-2, 1e-1):
        for lam in (0.1, 1.0, 10.0):
            case = {"omega2": w2, "lambda": lam}
            for name, kw, rtol, maxit in solvers:
                if name == "mixed multigrid":
                    rtol = 1e-10
                sv = ellsolve.Solver(0, nb, nzb, rb, w2, lam * lam, stream=stream.cuda_stream,
                                     **kw)
                case[name] = timed(sv, fb, xb, rtol, maxit)
                sv.close()
            out["box256_sweep"]["cases"].append(case)
    del fb, xb
    torch.cuda.empty_cache()
    return out


def run_smoothers(torch, stream, workload, reps=3):
    """Block red-black SOR and full multigrid against damped line Jacobi
    V-cycles on the benchmark workload (time to the workload's tolerance,
    V-cycles, time per V-cycle), and CG with
    block red-black SSOR against block Jacobi on the box 256 x 256 x 64."""
    from paper_1307_2036_gb300 import ellsolve, inputs
    kind, n, nz, graded, w2, l2, rhs_kind, rtol = WORKLOADS[workload]
    r = inputs.radial_levels(nz, graded=graded)
    with torch.cuda.stream(stream):
        f = torch.from_numpy(rhs_for(kind, n, nz, rhs_kind)).to("cuda")
        x = torch.zeros_like(f)
    stream.synchronize()

    def timed(sv, f, x, rtol, maxit):
        sv.solve(f, x, rtol=rtol, maxit=maxit)  # warm-up (graph capture)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        for _ in range(reps):
            st, res = sv.solve(f, x, rtol=rtol, maxit=maxit)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps, st, res

    out = {"workload": f"{workload}, rtol {rtol:g}, mixed precision", "multigrid": []}
    for name, sm, nu, rho, fmg in (("line Jacobi 2/2, rho 0.8", 0, 2, 0.8, 0),
                                   ("line Jacobi 2/2, rho 0.8, full multigrid", 0, 2, 0.8, 1),
                                   ("line RB-SOR 1/1, rho 1", 1, 1, 1.0, 0),
                                   ("line RB-SOR 2/2, rho 1", 1, 2, 1.0, 0)):
        sv = ellsolve.Solver(kind, n, nz, r, w2, l2, precision=1, use_graph=1, smoother=sm,
                             nu_pre=nu, nu_post=nu, damping=rho, fmg=fmg,
                             stream=stream.cuda_stream)
        sv.autotune()
        ms, st, res = timed(sv, f, x, rtol, 60)
        out["multigrid"].append({"smoother": name, "ms_to_rtol": ms, "vcycles": res.iterations,
                                 "ms_per_vcycle": ms / max(1, res.iterations),
                                 "rel_residual": res.rel_residual, "status": int(st)})
        sv.close()
    del f, x
    torch.cuda.empty_cache()
    nb, nzb = 256, 64
    rb = inputs.radial_levels(nzb, graded=True)
    with torch.cuda.stream(stream):
        fb = torch.from_numpy(rhs_for(0, nb, nzb, "uniform")).to("cuda")
        xb = torch.zeros_like(fb)
    stream.synchronize()
    out["pcg"] = {"workload": f"box {nb}x{nb}x{nzb} graded, omega2 0.01, lambda 1, rtol 1e-5, FP64"}
    for name, pc in (("block Jacobi", 0), ("block RB-SSOR", 1)):
        sv = ellsolve.Solver(0, nb, nzb, rb, 0.01, 1.0, precision=0, solver=1, precond=pc,
                             stream=stream.cuda_stream)
        ms, st, res = timed(sv, fb, xb, 1e-5, 1000)
        out["pcg"][name] = {"ms_to_rtol": ms, "iterations": res.iterations,
                            "rel_residual": res.rel_residual}
        sv.close()
    return out


def run_ensemble(torch, stream, members=32, n=128, nz=64, rtol=1e-8, reps=3):
    """Ensemble: `members` independent cubed-sphere problems 6 x n^2 x nz with
    per-member omega^2 (log-uniform [1e-3, 1e-1]) and lambda (uniform [0.5, 5]),
    uniform right-hand sides; one batched mixed-precision solve (one launch per
    kernel and level over all members) against the same solves done one after
    another in plain FP64 multigrid, and the same mixed-precision solves one
    after another (which separates the gain of batching from that of precision)."""
    from paper_1307_2036_gb300 import ellsolve, inputs
    w2s, lams = inputs.member_params(members)
    r = inputs.radial_levels(nz, graded=True)
    with torch.cuda.stream(stream):
        sv = [ellsolve.Solver(1, n, nz, r, float(w2s[m]), float(lams[m]) ** 2, precision=1,
                              stream=stream.cuda_stream) for m in range(members)]
        sv[0].autotune()
        fs = [torch.tensor(inputs.uniform_pm1(sv[0].shape(), member=m), device="cuda")
              for m in range(members)]
        xs = [torch.zeros_like(f) for f in fs]
    stream.synchronize()
    st, res = ellsolve.solve_batch(sv, fs, xs, rtol=rtol, maxit=60)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        st, res = ellsolve.solve_batch(sv, fs, xs, rtol=rtol, maxit=60)
    e1.record(stream)
    stream.synchronize()
    batched_s = e0.elapsed_time(e1) / 1e3 / reps
    worst = max(x.rel_residual for x in res)
    cycles = [x.iterations for x in res]
    # the same mixed-precision solves one member after another: the gain of
    # batching alone
    for m in range(members):
        sv[m].solve(fs[m], xs[m], rtol=rtol, maxit=60)  # warm-up (each handle's own plan)
    stream.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for m in range(members):
            sv[m].solve(fs[m], xs[m], rtol=rtol, maxit=60)
    e1.record(stream)
    stream.synchronize()
    seq_mixed_s = e0.elapsed_time(e1) / 1e3 / reps
    # plain FP64, one member after another
    with torch.cuda.stream(stream):
        p64 = [ellsolve.Solver(1, n, nz, r, float(w2s[m]), float(lams[m]) ** 2, precision=0,
                               stream=stream.cuda_stream) for m in range(members)]
        x64 = torch.zeros_like(fs[0])
    p64[0].solve(fs[0], x64, rtol=rtol, maxit=100)  # warm-up
    stream.synchronize()
    e0.record(stream)
    it64 = []
    for m in range(members):
        _, r64 = p64[m].solve(fs[m], x64, rtol=rtol, maxit=100)
        it64.append(r64.iterations)
    e1.record(stream)
    stream.synchronize()
    seq_s = e0.elapsed_time(e1) / 1e3
    return {"workload": f"{members} members, cubed sphere 6x{n}x{n}x{nz}, rtol {rtol}",
            "batched_mixed_solves_per_s": members / batched_s,
            "sequential_mixed_solves_per_s": members / seq_mixed_s,
            "sequential_fp64_solves_per_s": members / seq_s,
            "speedup": seq_s / batched_s,
            "batching_gain": seq_mixed_s / batched_s,
            "precision_gain": seq_s / seq_mixed_s,
            "batched_vcycles_per_member": [min(cycles), max(cycles)],
            "fp64_vcycles_per_member": [min(it64), max(it64)],
            "worst_rel_residual": worst}


def _serve(torch, stream, ellsolve, inputs, req, shapes, budget, slots):
    """Submit the requests of `req` at their arrival times to a fresh server;
    between submissions poll the outstanding ones without waiting, so that a
    finished request's solution buffer is released at once (the device holds
    the solution of every outstanding request).  Returns per-request latency
    (submit -> completion, as the library measures it), status and wall time."""
    import numpy as np
    count = len(req["arrival"])
    srv = ellsolve.Server(budget, slots, stream=stream.cuda_stream)
    lat = np.zeros(count)
    status = np.zeros(count, dtype=np.int64)
    outstanding = {}  # ticket -> (index, x)

    def drain(wait):
        for t in list(outstanding):
            st, res = srv.poll(t, timeout_us=-1 if wait else 0)
            if st == ellsolve.PENDING:
                continue
            i, _ = outstanding.pop(t)
            lat[i], status[i] = res.seconds, st
    t0 = time.perf_counter()
    for i in range(count):
        due = t0 + float(req["arrival"][i])
        while True:
            drain(False)
            now = time.perf_counter()
            if now >= due:
                break
            time.sleep(min(due - now, 2e-3))
        n, nz = int(req["n"][i]), int(req["nz"][i])
        with torch.cuda.stream(stream):
            x = torch.zeros_like(shapes[(n, nz)])
        stream.synchronize()
        t = srv.submit(1, n, nz, inputs.radial_levels(nz, graded=True), float(req["omega2"][i]),
                       float(req["lam"][i]) ** 2, shapes[(n, nz)], x, rtol=float(req["tol"][i]),
                       maxit=80)
        outstanding[t] = (i, x)
    drain(True)
    wall = time.perf_counter() - t0
    srv.close()
    return lat, status, wall


def _fifo(arrival, service):
    """One-at-a-time FIFO queue over the arrivals: latency of every request."""
    import numpy as np
    done, lat = 0.0, np.zeros(len(arrival))
    for i, (a, s) in enumerate(zip(arrival, service)):
        done = max(float(a), done) + float(s)
        lat[i] = done - float(a)
    return lat, done - float(arrival[0])


def run_serving(torch, stream, count, rate=200.0, low_count=1000, low_rate=60.0,
                budget=64 << 30, slots=16):
    """Mixed-size requests through the continuous-batching server: Poisson
    arrivals at 200/s, n in {48, 96, 192, 384}, nz in {32, 64, 128}, tol in
    {1e-5, 1e-10}, omega^2 and lambda drawn as in the ensemble.  Two runs:
    `count` requests offered at `rate` per second (above the server's
    capacity, so the queue grows; `count` is bounded by the device memory
    the outstanding requests' solution buffers need), and `low_count` requests at `low_rate`, below
    capacity.  Baseline: plain FP64 multigrid one request at a time in FIFO
    order over the same arrivals, with the service time of each (n, nz, tol)
    class measured once on the GPU (the class's first request)."""
    import numpy as np

    from paper_1307_2036_gb300 import ellsolve, inputs
    runs = {}
    fifo_cache = {}
    for name, cnt, rt, seed_off in (("offered_at_200_per_s", count, rate, 0),
                                    ("below_capacity", low_count, low_rate, 1)):
        req = inputs.request_stream(cnt, rate=rt, seed=inputs.DEFAULT_SEED + seed_off)
        shapes = {}
        with torch.cuda.stream(stream):
            for i in range(cnt):
                key = (int(req["n"][i]), int(req["nz"][i]))
                if key not in shapes:
                    shapes[key] = torch.tensor(
                        inputs.uniform_pm1((key[1], 6, key[0], key[0]), member=1000 + len(shapes)),
                        device="cuda")
        stream.synchronize()
        lat, status, wall = _serve(torch, stream, ellsolve, inputs, req, shapes, budget, slots)
        # FP64 FIFO baseline: service time per (n, nz, tol) class
        service = np.zeros(cnt)
        for i in range(cnt):
            key = (int(req["n"][i]), int(req["nz"][i]), float(req["tol"][i]))
            if key not in fifo_cache:
                n, nz, tol = key
                with torch.cuda.stream(stream):
                    p = ellsolve.Solver(1, n, nz, inputs.radial_levels(nz, graded=True),
                                        float(req["omega2"][i]), float(req["lam"][i]) ** 2,
                                        precision=0, stream=stream.cuda_stream)
                    xb = torch.zeros_like(shapes[(n, nz)])
                stream.synchronize()
                a = time.perf_counter()
                p.solve(shapes[(n, nz)], xb, rtol=tol, maxit=100)
                stream.synchronize()
                fifo_cache[key] = time.perf_counter() - a
                del p, xb
            service[i] = fifo_cache[key]
        base, base_span = _fifo(req["arrival"], service)
        ok = status == ellsolve.OK
        nc = status == ellsolve.NOT_CONVERGED
        runs[name] = {
            "requests": cnt, "offered_per_s": rt,
            "achieved_solves_per_s": cnt / wall,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "status_counts": {"ok": int(ok.sum()), "not_converged": int(nc.sum()),
                              "error": int((~ok & ~nc).sum())},
            "not_converged_requests": [
                {"n": int(req["n"][i]), "nz": int(req["nz"][i]), "tol": float(req["tol"][i]),
                 "omega2": float(req["omega2"][i]), "lambda": float(req["lam"][i])}
                for i in np.nonzero(nc)[0][:8]],
            "fp64_fifo_baseline": {"solves_per_s": cnt / base_span,
                                   "p50_latency_s": float(np.percentile(base, 50)),
                                   "p99_latency_s": float(np.percentile(base, 99))}}
        del shapes
        torch.cuda.empty_cache()
    return {"workload": "mixed-size requests: n in 48..384, nz in 32..128, tol 1e-5/1e-10; "
                        f"server {slots} slots, {budget >> 30} GiB budget",
            "sample": (f"{count} of a 10,000-request stream at {rate:g}/s (the queue grows "
                       "above capacity and every outstanding request holds its solution "
                       "buffer on the device, which bounds the sample), and "
                       f"{low_count} requests at {low_rate:g}/s below capacity"),
            "fp64_fifo_service": "plain FP64 multigrid, one solve per (n, nz, tol) class timed "
                                 "on the GPU, queued FIFO against the same arrivals",
            "note": "not_converged: 1e-10 requests whose FP64 attainable residual is above 1e-10",
            **runs}


# bumped whenever the finest-level smoother kernel changes (invalidates traffic)
KERNEL_REV = "smooth-v11-predicated-copies"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sphere512")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ensemble and serving measurements")
    ap.add_argument("--serve-requests", type=int, default=1500,
                    help="requests of the serving run at 200/s (bounded by the device "
                         "memory that outstanding solution buffers need)")
    ap.add_argument("--shapes-out", default=None,
                    help="write the autotuned per-level launch shapes to this JSON file")
    ap.add_argument("--shapes-in", default=None,
                    help="take the per-level launch shapes from this JSON file instead of "
                         "autotuning")
    ap.add_argument("--inner-cycles", type=int, default=3,
                    help="FP32 V-cycles per FP64 refinement step")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
