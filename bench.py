"""Benchmark: LSRK(5,4) time steps of the nodal DG TM-Maxwell solver.

One step = five fused stage kernels (right-hand side + 2N-storage update)
over the whole mesh.  Default workload: seeded jittered-grid Delaunay mesh of
the unit square with n = 707 (K = 999,698 triangles), order N = 5 (Np = 21),
FP32 fields, Gaussian pulse (width 0.05) at (0.5, 0.5).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica of the workload on its own GPU (the solver does not
shard); value = all ranks' element-stage updates / max over ranks of the
timed region.
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

METRIC = ("DG element-stage updates/s and RHS GFLOP/s (% roofline) at N=5; "
          "served solves/s + p99 latency")
UNIT = "element-stage updates/s"

# algorithmic HBM bytes per element for one fused stage (FP32): q in/out and
# residual in/out (12 Np floats) + 13 geometry floats + 6 int32 connectivity;
# the first stage of a step does not read the residual (a_1 = 0).
STAGE_BYTES = {1: 220, 2: 364, 3: 556, 4: 796, 5: 1084, 6: 1420, 7: 1804}

# element-local products of the FP32-field tensor-core variants
PRODUCTS = {"fp32": "3xTF32", "tf32": "1xTF32", "bf16": "1xBF16", "bf16x3": "3xBF16"}


def rhs_flops_per_element(N):
    Np = (N + 1) * (N + 2) // 2
    Nafp = 3 * (N + 1)
    return 6 * 2 * Np * Np + 2 * Np * 13 + 3 * (2 * Np * Nafp + Np) + Nafp * 18


def step_bytes_per_element(N):
    Np = (N + 1) * (N + 2) // 2
    first = STAGE_BYTES[N] - 3 * Np * 4
    return 4 * STAGE_BYTES[N] + first


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id, period_ms=100):
        self.gpu_id = gpu_id
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.error = None

    def start(self):
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                   "-lms", str(self.period_ms)]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception as ex:  # no nvidia-smi
            self.error = str(ex)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"error": self.error or "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"error": "no samples", "raw": self.lines[:3]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- oracle
def oracle_sample_rate(n, N, seconds, steps=None, warmup=0):
    """Time the FP64 oracle's LSRK(5,4) steps on the n-mesh; returns
    (element-stage updates/s, steps run, K)."""
    import numpy as np

    import oracle as O
    from synth import gaussian_pulse, jittered_delaunay_mesh

    mesh = jittered_delaunay_mesh(n, seed=2024)
    d = O.Discretization(*mesh, N)
    q = np.stack(gaussian_pulse(d.x, d.y))
    dt = O.cfl_dt(d)
    for _ in range(warmup):
        q = O.lsrk_step(d, q, 0.0, dt)
    t0 = time.perf_counter()
    done = 0
    while True:
        q = O.lsrk_step(d, q, done * dt, dt)
        done += 1
        el = time.perf_counter() - t0
        if steps is not None and done >= steps:
            break
        if steps is None and el >= seconds:
            break
    return d.K * 5 * done / el, done, d.K, el


def oracle_timings():
    """The oracle's own timings on this host, in the calling process: per
    right-hand side and per LSRK(5,4) step on the three configurations
    (bounded samples of the two large ones), and the whole cavity solve of
    the small one.  Returns a dict (seconds and element-stage updates/s)."""
    import numpy as np

    import oracle as O
    from synth import cavity_mode, gaussian_pulse, jittered_delaunay_mesh, square_grid_mesh

    def per_call(fn, min_s=2.0):
        fn()
        t0, k = time.perf_counter(), 0
        while True:
            fn()
            k += 1
            el = time.perf_counter() - t0
            if el >= min_s:
                return el / k, k

    out = {}
    # cavity: [-1,1]^2, 8x8 squares x 2, N = 4, T = 1 at the CFL step
    d = O.Discretization(*square_grid_mesh(8, 8), 4)
    q0 = np.stack(cavity_mode(d.x, d.y, 0.0))
    rhs_s, _ = per_call(lambda: O.maxwell_rhs(d, q0))
    t0 = time.perf_counter()
    qT, t = O.solve(d, q0, 1.0, O.cfl_dt(d))
    solve_s = time.perf_counter() - t0
    nsteps = int(np.ceil(1.0 / O.cfl_dt(d) - 1e-12))
    out["cavity_N4_K128"] = {"K": d.K, "N": 4, "rhs_s": rhs_s, "solve_s": solve_s,
                             "steps": nsteps, "max_error_vs_exact": float(
                                 np.abs(qT - np.stack(cavity_mode(d.x, d.y, t))).max()),
                             "element_stage_per_s": d.K * 5 * nsteps / solve_s}
    # samples of the large configurations
    for name, n, N in (("jittered_N5_sample", 100, 5), ("jittered_N7_sample", 50, 7)):
        d = O.Discretization(*jittered_delaunay_mesh(n, seed=2024), N)
        q = np.stack(gaussian_pulse(d.x, d.y))
        dt = O.cfl_dt(d)
        rhs_s, _ = per_call(lambda: O.maxwell_rhs(d, q))
        step_s, k = per_call(lambda: O.lsrk_step(d, q, 0.0, dt))
        out[name] = {"K": d.K, "N": N, "n": n, "rhs_s": rhs_s, "step_s": step_s, "steps_timed": k,
                     "element_stage_per_s": d.K * 5 / step_s}
    return out


def run_oracle_study(args):
    """The oracle timed on the host cores, one thread (child process with
    the BLAS / OpenMP thread counts pinned to 1) and the default threads.
    One JSON line."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--_oracle-timings"]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1200)
    one = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else {
        "error": r.stderr[-500:]}
    return {"study": "oracle timings", "kind": "oracle", "host_cores": os.cpu_count(),
            "one_thread": one, "default_threads": oracle_timings()}


def cpu_baseline(n=100, N=5, seconds=10.0):
    """The oracle on one host core (BLAS/OpenMP threads pinned to 1), in a
    child process so the thread limit applies before numpy loads."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--_oracle-sample", str(n), str(N), str(seconds)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-500:]}
    v = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": v["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "FP64 numpy oracle, %d LSRK(5,4) steps on the n=%d jittered mesh "
                      "(K=%d, N=%d), 1 thread, %.1f s" % (v["steps"], n, v["K"], N, v["seconds"])}


# ------------------------------------------------------------- replicas
def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (the timed
    region of the slowest replica decides the whole job's time)."""
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def replica_throughput(world, K, steps, ms):
    """Whole-job element-stage updates/s: every rank advances its own copy
    of the K-element mesh by `steps` five-stage steps; `ms` is the maximum
    over ranks of the timed region."""
    return world * K * 5 * steps / (ms / 1e3)


# ------------------------------------------------------------- our arm
def measure_host_link(nbytes, dev, reps=5, rounds=4):
    """Host <-> device copy bandwidth of pinned memory through torch copies
    (copy engines): host to device alone, device to host alone, and both at
    once on two streams; `rounds` copies of `nbytes` per direction, GB/s of
    the bytes moved, best of `reps`."""
    import torch
    h_in = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    main = torch.cuda.current_stream(dev)
    sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(h2d, d2h):
        best = float("inf")
        for r in range(reps + 1):
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(main)
            sa.wait_stream(main)
            sb.wait_stream(main)
            for _ in range(rounds):
                if h2d:
                    with torch.cuda.stream(sa):
                        d_in.copy_(h_in, non_blocking=True)
                if d2h:
                    with torch.cuda.stream(sb):
                        h_out.copy_(d_out, non_blocking=True)
            main.wait_stream(sa)
            main.wait_stream(sb)
            e1.record(main)
            e1.synchronize()
            if r > 0:
                best = min(best, e0.elapsed_time(e1))
        return rounds * (h2d + d2h) * nbytes / (best / 1e3) / 1e9

    out = {"h2d_gbs": timed(1, 0), "d2h_gbs": timed(0, 1), "both_gbs": timed(1, 1)}
    del h_in, h_out, d_in, d_out
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_1304_5546_gb300 as P
    from synth import gaussian_pulse, jittered_delaunay_mesh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if dist is not None:
            dist.barrier()

    N = args.order
    mesh = jittered_delaunay_mesh(args.n, seed=2024)
    s = P.Solver(*mesh, N=N, precision=args.precision, device=dev, simt=args.simt)
    x, y = s.nodes()
    q0 = np.stack(gaussian_pulse(x, y))
    q = s.from_numpy(q0)
    res = s.new_fields()
    dt = s.cfl_dt()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        s.step(q, res, dt, nsteps=1)
    P.dg_sync_check(s.op)

    clocks = ClockSampler(dev if world > 1 else None) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    launches0 = P.dg_launch_count(s.op)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    start.record(stream)
    s.step(q, res, dt, nsteps=args.steps)
    end.record(stream)
    end.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = start.elapsed_time(end)
    launches = P.dg_launch_count(s.op) - launches0
    clk = clocks.stop() if clocks else None
    P.dg_check_finite(s.op, q)

    # end to end through the C ABI with host buffers: every step copies its
    # fields in from pinned host memory and its result back out.
    # dg_step_host_jobs: e2e_steps independent jobs (three pinned host field
    # sets, reused in turn), one step each, copies overlapping the steps of
    # the neighbouring jobs; dg_step_host: the same one job at a time
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    hs = [s.from_numpy(q0).cpu().pin_memory() for _ in range(3)]
    work = torch.empty(P.dg_step_host_jobs_work_bytes(s.op), dtype=torch.uint8, device=dev)
    P.dg_step_host_jobs(s.op, hs, work, 0.0, dt, 1)  # warm
    jobs = [hs[j % 3] for j in range(e2e_steps)]
    barrier()
    t0 = time.perf_counter()
    P.dg_step_host_jobs(s.op, jobs, work, 0.0, dt, 1)
    e2e_s = time.perf_counter() - t0
    barrier()
    del work
    h = hs[0]
    dq, dres = s.new_fields(), s.new_fields()
    P.dg_step_host(s.op, h, dq, dres, 0.0, dt, 1)  # warm
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.dg_step_host(s.op, h, dq, dres, 0.0, dt, 1)
    e2e_serial_s = time.perf_counter() - t0
    barrier()
    field_bytes = 3 * s.fstride * (8 if args.precision == "fp64" else 4)
    link = measure_host_link(field_bytes, dev)

    ms, e2e_s, e2e_serial_s = max_over_ranks([ms, e2e_s, e2e_serial_s], dist, device="cuda")
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None

    K = s.K
    kernel_kind = s.kernel()[0]
    value = replica_throughput(world, K, args.steps, ms)
    peaks, peak_kind = measured_peaks()
    bytes_step = K * step_bytes_per_element(N) * (2 if args.precision == "fp64" else 1)
    achieved = bytes_step * args.steps / (ms / 1e3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    if os.path.exists(tpath):
        try:
            from paper_1304_5546_gb300.build import kernel_source_hash
            t = json.load(open(tpath))
            key = "N%d_%s" % (N, args.precision)
            fam = t.get("kernel_family")
            if t.get("kernel_hash") == kernel_source_hash(fam) and key in t.get("per_element", {}):
                traffic = t["per_element"][key] * K * 5 * args.steps / launches
        except Exception:
            traffic = None
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {
            "workload": "single large mesh: jittered Delaunay unit square n=%d (K=%d), N=%d, "
                        "Gaussian pulse w=0.05, LSRK(5,4) steps" % (args.n, K, N),
            "K": K, "N": N, "Np": s.Np, "precision": args.precision,
            "products": {"tensor cores": "tensor cores (tcgen05, %s)" % PRODUCTS.get(
                             args.precision, "3xTF32"),
                         "cuda cores": "CUDA cores, one thread per node",
                         "element threads": "CUDA cores, one thread per element"}[kernel_kind],
            "mesh_seed": 2024,
            "l2": "inputs larger than L2 (q, q_tmp, res: %.0f MB)" % (
                3 * 3 * s.fstride * (8 if args.precision == "fp64" else 4) / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "rhs_gflops": world * K * rhs_flops_per_element(N) * 5 * args.steps / (ms / 1e3) / 1e9,
        "roofline": {
            "bound": "hbm",
            "achieved": achieved,
            "peak": peaks["hbm_gbs"],
            "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"],
            "traffic": traffic,
            "peak_kind": peak_kind,
            "kernel": {"tensor cores": "dg_stage_tc_kernel", "cuda cores": "dg_stage_kernel",
                       "element threads": "dg_stage_ept_kernel"}[kernel_kind]
                      + " (fused RHS + LSRK stage)",
            "bytes_per_element_step": step_bytes_per_element(N),
        },
        "e2e": {
            "value": replica_throughput(world, K, e2e_steps, e2e_s * 1e3),
            "unit": UNIT,
            "h2d_bytes_per_step": 3 * s.fstride * (8 if args.precision == "fp64" else 4),
            "d2h_bytes_per_step": 3 * s.fstride * (8 if args.precision == "fp64" else 4),
            "steps": e2e_steps,
            "api": "dg_step_host_jobs: per step, pinned host fields -> device, 1 LSRK step, "
                   "device -> host; one job's copies overlap the neighbouring jobs' steps",
            "serial": {"value": replica_throughput(world, K, e2e_steps, e2e_serial_s * 1e3),
                       "api": "dg_step_host, one job at a time (copy in, step, copy out)"},
            # the end-to-end bound: a step cannot take less than its copies
            # at the host link's two-way rate, nor less than the device step
            "host_link": dict(link, **{
                "bound_value": replica_throughput(
                    world, K, 1, 1e3 * max(2 * field_bytes / (link["both_gbs"] * 1e9),
                                           ms / args.steps / 1e3)),
                "how": "pinned torch copies of one job's fields (copy engines), 4 per direction, best of 5; "
                       "bound = K * 5 / max(copy-in + copy-out bytes / two-way GB/s, "
                       "device ms per step)"}),
        },
        "gpu_launches": launches,
        "clocks": clk,
    }
    hl = out["e2e"]["host_link"]
    hl["frac"] = out["e2e"]["value"] / hl["bound_value"]
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    if world == 1 and not args.no_workloads:
        # the metric's other half: batched solves and served solves/s + p99
        # (their own seeded workloads, timed after the main measurement)
        s.close()
        del q, res, hs, h, dq, dres
        torch.cuda.empty_cache()
        out["batched"] = run_batched(args)
        sargs = argparse.Namespace(**vars(args))
        sargs.serve_rates = [300.0]
        sargs.serve_requests = 60
        out["serving"] = run_serving(sargs)
    if dist is not None:
        dist.destroy_process_group()
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    n, N = 100, args.order
    value, steps, K, seconds = oracle_sample_rate(n, N, None, steps=args.steps, warmup=args.warmup)
    sample = ("FP64 numpy oracle on the n=%d jittered mesh (K=%d, N=%d), %d timed LSRK(5,4) "
              "steps after %d warm-up, default BLAS threads" % (n, K, N, steps, args.warmup))
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": seconds * 1e3 / steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "single large mesh workload, bounded sample: jittered Delaunay "
                               "unit square n=%d (K=%d), N=%d, LSRK(5,4) steps" % (n, K, N),
                   "K": K, "N": N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_precision_study(args):
    """Precision path of the element-local contractions: each FP32-field
    tensor-core variant against an FP64 run of the same solve (jittered
    unit-square mesh, Gaussian pulse, LSRK(5,4) steps).  One JSON line with
    max and L2 errors relative to the FP64 run per variant."""
    import numpy as np
    import torch

    import paper_1304_5546_gb300 as P
    from synth import gaussian_pulse, jittered_delaunay_mesh

    torch.cuda.set_device(0)
    N, n, steps = args.order, args.n, args.study_steps

    mesh = jittered_delaunay_mesh(n, seed=2024)
    runs = {}
    for v in ("fp64", "fp32", "bf16x3", "tf32", "bf16"):
        s = P.Solver(*mesh, N=N, precision=v)
        x, y = s.nodes()
        q0 = np.stack(gaussian_pulse(x, y))
        if v == "fp64":
            q0 = q0.astype(np.float32).astype(np.float64)  # same start as the FP32 runs
        q = s.from_numpy(q0)
        res = s.new_fields()
        dt = s.cfl_dt()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(q, res, dt, steps)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        P.dg_sync_check(s.op)
        runs[v] = (s.to_numpy(q), el, s.K)
        s.close()
    ref = runs["fp64"][0]
    scale = np.abs(ref).max()
    table = {}
    for v, (qv, el, K) in runs.items():
        e = qv - ref
        table[v] = {"max_err": float(np.abs(e).max() / scale),
                    "l2_err": float(np.sqrt((e ** 2).mean() / (ref ** 2).mean())),
                    "seconds": el, "element_stage_per_s": K * 5 * steps / el}
    return {"study": "precision", "N": N, "K": runs["fp64"][2], "steps": steps,
            "reference": "FP64 run of the same solve (the FP64 path matches the FP64 oracle "
                         "to 1e-12 in the GPU parity tests)",
            "errors_relative_to": "max|q| (max_err) and rms(q) (l2_err) of the FP64 run",
            "variants": table}


def run_sweep_study(args):
    """Order sweep of the single-mesh path at about 10M nodal values per
    field (K ~ 1e7 / Np): for N = 1..7, the FP32 tensor-core kernel (face
    pairs off and on: dg_operator_set_face_pairs), the FP32 CUDA-core kernel
    and, at N <= 5, the element-thread kernel (median of three runs),
    `--study-steps` LSRK steps each timed with CUDA events (the two
    tensor-core settings alternate three times on one operator; medians).
    With --sweep-media every operator has a seeded per-element permittivity
    (wave speeds drawn from {0.5, 1, 2}) and the algorithmic bytes are those
    of its 20-value records (media_step_bytes_per_element).  One JSON line: ms/step, element-stage updates/s, RHS
    GFLOP/s and achieved HBM bandwidth (algorithmic bytes) per order and
    kernel, and the share of interior faces whose two elements lie in one
    tensor-core block."""
    import numpy as np
    import torch

    import paper_1304_5546_gb300 as P
    from synth import gaussian_pulse, jittered_delaunay_mesh, n_for_target_elements
    from synth import random_permittivity

    torch.cuda.set_device(0)
    peaks, peak_kind = measured_peaks()
    steps = args.study_steps
    media = args.sweep_media
    sweep_bytes = media_step_bytes_per_element if media else step_bytes_per_element
    rows = []

    def timed(s, q, res, dt):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        s.step(q, res, dt, steps)
        b.record()
        b.synchronize()
        P.dg_sync_check(s.op)
        return a.elapsed_time(b) / steps

    def row(N, K, kernel, ms, **extra):
        gbs = K * sweep_bytes(N) / (ms / 1e3) / 1e9
        r = {"N": N, "K": K, "kernel": kernel, "ms_per_step": ms,
             "element_stage_per_s": K * 5 / (ms / 1e3),
             "rhs_gflops": K * rhs_flops_per_element(N) * 5 / (ms / 1e3) / 1e9,
             "hbm_gbs": gbs, "frac_hbm": gbs / peaks["hbm_gbs"]}
        r.update(extra)
        return r

    for N in args.sweep_orders:
        Np = (N + 1) * (N + 2) // 2
        n = n_for_target_elements(1e7 / Np)
        mesh = jittered_delaunay_mesh(n, seed=2024)
        eps = random_permittivity(mesh[2].shape[0], seed=5) if media else None
        kinds = ("fp32tc", "fp32simt") + (("fp32ept",) if N <= 5 else ())
        for kind in kinds:
            s = P.Solver(*mesh, N=N, precision=kind, eps=eps)
            x, y = s.nodes()
            q = s.from_numpy(np.stack(gaussian_pulse(x, y)))
            res = s.new_fields()
            dt = s.cfl_dt()
            s.step(q, res, dt, 3)
            torch.cuda.synchronize()
            if kind == "fp32simt":
                rows.append(row(N, s.K, "cuda cores", timed(s, q, res, dt)))
            elif kind == "fp32ept":
                rows.append(row(N, s.K, "element threads",
                                float(np.median([timed(s, q, res, dt) for _ in range(3)]))))
            else:
                times = {0: [], 1: []}
                for _ in range(3):
                    for pairs in (0, 1):
                        P.dg_operator_set_face_pairs(s.op, pairs)
                        times[pairs].append(timed(s, q, res, dt))
                E = 80 if N <= 3 else 40
                EToE = P.dg_mesh_connectivity(s.mesh)[0]
                k = np.arange(s.K)[:, None]
                interior = EToE != k
                same = interior & (EToE // E == k // E)
                share = float(same.sum() / max(interior.sum(), 1))
                rows.append(row(N, s.K, "tensor cores (3xTF32)", float(np.median(times[0]))))
                rows.append(row(N, s.K, "tensor cores (3xTF32), face pairs",
                                float(np.median(times[1])), faces_in_block=share))
            s.close()
    return {"study": "order sweep", "nodal_values_per_field": "~1e7", "steps": steps,
            "media": "per-element permittivity, seed 5" if media else None,
            "peak_hbm_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind,
            "bytes_per_element_step": {str(N): sweep_bytes(N) for N in range(1, 8)},
            "rows": rows}


def _longrun_oracle_worker(name, n, N, steps, snaps, conn, threads):
    """Spawned process (no CUDA): the FP64 oracle's run of one long-run
    configuration.  Makes the FP32-rounded Gaussian start on the oracle's
    nodes, hands it over, takes the time step from the parent, steps, and
    hands over the fields at the snapshot steps (as .npy files in /tmp)."""
    import os as _os
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        _os.environ[v] = str(threads)
    import time as _time

    import numpy as np

    import oracle as O
    from synth import gaussian_pulse, jittered_delaunay_mesh

    t0 = _time.perf_counter()
    d = O.Discretization(*jittered_delaunay_mesh(n, seed=2024), N)
    q = np.stack(gaussian_pulse(d.x, d.y)).astype(np.float32).astype(np.float64)
    path = "/tmp/longrun_%s_q0.npy" % name
    np.save(path, q)
    conn.send(("q0", path))
    dt = conn.recv()
    for k in range(steps):
        q = O.lsrk_step(d, q, k * dt, dt)
        if k + 1 in snaps:
            path = "/tmp/longrun_%s_oracle_%d.npy" % (name, k + 1)
            np.save(path, q)
            conn.send(("snap", k + 1, path, _time.perf_counter() - t0))
    conn.send(("done", _time.perf_counter() - t0))


def run_longrun_study(args):
    """Long-run accuracy against the FP64 oracle at the configured sizes:
    the single large mesh (K = 999,698, N = 5) for 100 LSRK steps and the
    precision-path mesh (K = 262,088, N = 7) for 500 steps, from the
    FP32-rounded Gaussian pulse (width 0.05 at (0.5, 0.5)) and the library's
    CFL time step.  The oracle runs in spawned processes on the host cores
    (started before any CUDA call); every FP32 variant runs on the GPU from
    the same start.  At each snapshot step: max nodal error relative to
    max |q| of the oracle, and L2 (rms) error relative to the oracle's rms.
    One JSON line; writes gpurun_out/longrun_gpu_done once the GPU part is
    over (the oracle may still be running)."""
    import multiprocessing as mp

    import numpy as np

    configs = [
        {"name": "large_N5", "n": 707, "N": 5, "steps": 100, "snaps": [1, 10, 100],
         "variants": ["fp32", "fp32simt"]},
        {"name": "precision_N7", "n": 362, "N": 7, "steps": 500, "snaps": [1, 10, 100, 500],
         "variants": ["fp32", "bf16x3", "tf32", "bf16", "fp32simt"]},
    ]
    if args.longrun_quick:  # small sizes, for a check of the machinery
        configs = [dict(c, n=c["n"] // 8, steps=c["steps"] // 10,
                        snaps=[x for x in c["snaps"] if x <= c["steps"] // 10]) for c in configs]
    ctx = mp.get_context("spawn")
    workers = []
    for c in configs:
        a, b = ctx.Pipe()
        pr = ctx.Process(target=_longrun_oracle_worker,
                         args=(c["name"], c["n"], c["N"], c["steps"], set(c["snaps"]), b,
                               args.longrun_threads))
        pr.start()
        workers.append((pr, a))

    import torch

    import paper_1304_5546_gb300 as P
    from synth import jittered_delaunay_mesh

    torch.cuda.set_device(0)
    results = []
    for c, (pr, conn) in zip(configs, workers):
        tag, q0_path = conn.recv()
        q0 = np.load(q0_path)
        mesh = jittered_delaunay_mesh(c["n"], seed=2024)
        gpu = {}
        dt = None
        for v in c["variants"]:
            s = P.Solver(*mesh, N=c["N"], precision=v)
            if dt is None:
                dt = s.cfl_dt()
                conn.send(dt)
            q, res = s.from_numpy(q0), s.new_fields()
            snaps, done, ms = {}, 0, 0.0
            for k in c["snaps"]:
                a_ev = torch.cuda.Event(enable_timing=True)
                b_ev = torch.cuda.Event(enable_timing=True)
                a_ev.record()
                s.step(q, res, dt, nsteps=k - done, t0=done * dt)
                b_ev.record()
                b_ev.synchronize()
                ms += a_ev.elapsed_time(b_ev)
                done = k
                snaps[k] = s.to_numpy(q)
            P.dg_sync_check(s.op)
            gpu[v] = (snaps, ms / c["steps"])
            s.close()
        results.append((c, gpu, dt))
    os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
    open(os.path.join(ROOT, "gpurun_out", "longrun_gpu_done"), "w").write("done\n")
    out = []
    for (c, gpu, dt), (pr, conn) in zip(results, workers):
        rows = {v: {"steps": [], "max_rel": [], "l2_rel": []} for v in c["variants"]}
        oracle_s = None
        while True:
            msg = conn.recv()
            if msg[0] == "done":
                oracle_s = msg[1]
                break
            _, k, path, _el = msg
            ref = np.load(path)
            scale_max = np.abs(ref).max()
            scale_l2 = np.sqrt(np.mean(ref ** 2))
            for v in c["variants"]:
                e = gpu[v][0][k] - ref
                rows[v]["steps"].append(k)
                rows[v]["max_rel"].append(float(np.abs(e).max() / scale_max))
                rows[v]["l2_rel"].append(float(np.sqrt(np.mean(e ** 2)) / scale_l2))
            os.remove(path)
        pr.join()
        for v in c["variants"]:
            rows[v]["gpu_ms_per_step"] = gpu[v][1]
        out.append({"config": c["name"], "K": 2 * c["n"] ** 2, "N": c["N"], "steps": c["steps"],
                    "dt": dt, "oracle_seconds": oracle_s,
                    "oracle_threads": args.longrun_threads, "variants": rows})
    return {"study": "long-run error against the FP64 oracle",
            "start": "FP32-rounded Gaussian pulse w=0.05 at (0.5, 0.5), H = 0",
            "error": "max |gpu - oracle| / max |oracle| and rms(gpu - oracle) / rms(oracle) "
                     "over all nodal values of the three fields",
            "configs": out}


def run_partition_study(args):
    """The mesh-partition path on one device (dg_partition_*): the default
    workload (order `--order`, K = 2 n^2) split into P parts by recursive
    coordinate bisection and stepped with one halo exchange per LSRK stage,
    for P in `--partition-parts`.  Per P: ms/step against the unpartitioned
    operator, the exchange alone (pack, transfer, unpack) per stage, the traces exchanged per stage, and whether the
    result equals the unpartitioned one bit for bit.  One JSON line."""
    import numpy as np
    import torch

    import paper_1304_5546_gb300 as P
    from synth import gaussian_pulse, jittered_delaunay_mesh

    torch.cuda.set_device(0)
    N, n, steps = args.order, args.n, args.study_steps
    s = P.Solver(*jittered_delaunay_mesh(n, seed=2024), N=N, precision=args.precision)
    x, y = s.nodes()
    q0 = s.from_numpy(np.stack(gaussian_pulse(x, y)))
    dt = s.cfl_dt()

    def timed(fn, reps):
        fn(3)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn(reps)
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    q, res = q0.clone(), s.new_fields()
    ms_single = timed(lambda k: s.step(q, res, dt, k), steps)
    want, wres = q0.clone(), s.new_fields()
    s.step(want, wres, dt, 10)
    rows = []
    for nparts in args.partition_parts:
        part = P.Partition(s, nparts)
        part.set_fields(q0)
        ms = timed(lambda k: part.step(dt, k), steps)
        ms_x = timed(lambda k: [part.exchange() for _ in range(k)], 200)
        part.set_fields(q0)
        part.step(dt, 10)
        got = s.new_fields()
        part.get_fields(got)
        part.sync_check()
        torch.cuda.synchronize()
        info = [part.info(p) for p in range(nparts)]
        values = sum(i[4] for i in info)  # node values per field per exchange
        pairs = sum(i[2] for i in info)
        rows.append({"parts": nparts, "ms_per_step": ms, "vs_unpartitioned": ms / ms_single,
                     "exchange_ms_per_stage": ms_x, "part_pairs": pairs,
                     "trace_values_per_stage": 3 * values,
                     "trace_bytes_per_stage": 3 * values * s.view(q).element_size(),
                     "elements_per_part": [i[0] for i in info],
                     "ghosts_per_part": [i[1] for i in info],
                     "bitwise_equal_after_10_steps": bool(torch.equal(s.view(got), s.view(want)))})
        part.close()
    return {"study": "partition", "N": N, "K": s.K, "precision": args.precision, "steps": steps,
            "ms_per_step_unpartitioned": ms_single, "rows": rows}


def batched_workload(n_problems=256, seed=4242, k_lo=500, k_hi=50000, orders=(3, 5, 7),
                     speeds=(0.5, 1.0, 2.0)):
    """Seeded batch of independent problems: K log-uniform in [k_lo, k_hi]
    (jittered Delaunay unit-square meshes with 2 n^2 ~ K triangles), N drawn
    from `orders`, per-element wave speed drawn from `speeds` (eps = 1/c^2),
    Gaussian pulse (width 0.1) at a seeded centre.  Returns a list of dicts
    with mesh, N, eps, pulse centre."""
    import numpy as np

    from synth import jittered_delaunay_mesh, n_for_target_elements, random_permittivity

    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        k = float(np.exp(rng.uniform(np.log(k_lo), np.log(k_hi))))
        N = int(rng.choice(orders))
        n = n_for_target_elements(k)
        mesh = jittered_delaunay_mesh(n, seed=seed + 1 + i)
        K = mesh[2].shape[0]
        out.append({"mesh": mesh, "N": N, "eps": random_permittivity(K, seed=seed + 10007 + i,
                                                                     speeds=speeds),
                    "x0": float(rng.uniform(0.3, 0.7)), "y0": float(rng.uniform(0.3, 0.7))})
    return out


def media_step_bytes_per_element(N):
    """Algorithmic HBM bytes per element per LSRK step with per-element
    permittivity records (20 floats) in FP32: four fused stages
    (12 Np floats + 20 record floats + 3 int32) and a first stage that does
    not read the residual (9 Np floats + records + codes)."""
    Np = (N + 1) * (N + 2) // 2
    stage = 12 * Np * 4 + 20 * 4 + 12
    return 4 * stage + (stage - 3 * Np * 4)


def run_batched(args):
    """Batched workload: every problem advanced `--batch-steps` LSRK steps
    (its own CFL dt) by one multi-order persistent launch per stage replayed
    from CUDA graphs, after the autotuner; against the same problems solved
    one after another with dg_step on the same GPU.  One JSON line."""
    import numpy as np
    import torch

    import paper_1304_5546_gb300 as P
    from synth import gaussian_pulse

    torch.cuda.set_device(0)
    steps = args.batch_steps
    specs = batched_workload(args.batch_problems, seed=args.batch_seed,
                             orders=tuple(args.batch_orders))
    solvers, q0s, dts = [], [], []
    for sp in specs:
        s = P.Solver(*sp["mesh"], N=sp["N"], precision="fp32", eps=sp["eps"])
        x, y = s.nodes()
        q0s.append(np.stack(gaussian_pulse(x, y, sp["x0"], sp["y0"], 0.1)).astype(np.float32))
        dts.append(s.cfl_dt())
        solvers.append(s)
    Ks = np.array([s.K for s in solvers])
    Ns = np.array([s.N for s in solvers])
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # ---- sequential plain solves: each problem alone, one after another
    qs = [s.from_numpy(q) for s, q in zip(solvers, q0s)]
    rs = [s.new_fields() for s in solvers]
    for s, q, r, dt in zip(solvers, qs, rs, dts):  # warm every kernel instance
        s.step(q, r, dt, 1)
    qs = [s.from_numpy(q) for s, q in zip(solvers, q0s)]
    launches0 = sum(P.dg_launch_count(s.op) for s in solvers)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    for s, q, r, dt in zip(solvers, qs, rs, dts):
        s.step(q, r, dt, steps)
    b.record(stream)
    b.synchronize()
    seq_ms = a.elapsed_time(b)
    seq_launches = sum(P.dg_launch_count(s.op) for s in solvers) - launches0
    seq_out = [s.to_numpy(q) for s, q in zip(solvers, qs)]

    # ---- sequential plain solves replayed from CUDA graphs: each problem's
    # `steps` steps captured once into a graph of its own (outside the timed
    # region), the graphs replayed one after another: no launch overhead
    graph = {"how": "dg_step per problem, its %d steps captured into one CUDA graph, "
                    "graphs replayed one after another" % steps}
    try:
        qg = [s.from_numpy(q) for s, q in zip(solvers, q0s)]
        rg = [s.new_fields() for s in solvers]
        side = torch.cuda.Stream()
        graphs = []
        for s, q, r, dt in zip(solvers, qg, rg, dts):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                s.step(q, r, dt, steps)  # recorded, not run
            graphs.append(g)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        for g in graphs:
            g.replay()
        b.record(stream)
        b.synchronize()
        graph_ms = a.elapsed_time(b)
        same = all(np.array_equal(s.to_numpy(q), ref) for s, q, ref in zip(solvers, qg, seq_out))
        graph.update({"value": len(solvers) / (graph_ms / 1e3), "unit": "solves/s",
                      "ms": graph_ms, "bit_equal_to_sequential": bool(same)})
        del graphs, qg, rg
    except Exception as e:  # capture refused: report it, keep the rest of the line
        graph["unavailable"] = repr(e)[:200]

    # ---- batched
    cap = [0] * 7
    for K, N in zip(Ks, Ns):
        cap[N - 1] += (int(K) + 3) // 4 * 4
    B = P.Batch(cap)
    slots = [B.add(s, dt) for s, dt in zip(solvers, dts)]
    for slot, q in zip(slots, q0s):
        B.set_fields(slot, q)
    t0 = time.perf_counter()
    B.tune(reps=3)
    tune_s = time.perf_counter() - t0
    B.step(1)  # warm (tables, graphs)
    B.sync_check()
    for slot, q in zip(slots, q0s):
        B.set_fields(slot, q)
    clocks = ClockSampler(None) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    l0 = B.launch_count()
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    B.step(steps)
    b.record(stream)
    b.synchronize()
    bat_ms = a.elapsed_time(b)
    clk = clocks.stop() if clocks else None
    bat_launches = B.launch_count() - l0
    B.sync_check()
    diff = 0.0
    for slot, ref in zip(slots, seq_out):
        got = B.get_fields(slot).astype(np.float64)
        diff = max(diff, float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30)))
    cta, nblk, cost = B.plan()
    mode, tuned_split_ms, tuned_conc_ms = B.launch_mode()
    elems, ms_def, ms_alt = B.block_elems()
    B.close()
    for s in solvers:
        s.close()

    n = len(specs)
    el_stage = float(np.sum(Ks)) * 5 * steps
    bytes_total = float(sum(int(K) * media_step_bytes_per_element(int(N)) for K, N in zip(Ks, Ns))) * steps
    peaks, peak_kind = measured_peaks()
    achieved = bytes_total / (bat_ms / 1e3) / 1e9
    return {
        "workload": "batched",
        "metric": "batched solves/s (independent problems x LSRK steps, mixed orders)",
        "value": n / (bat_ms / 1e3),
        "unit": "solves/s",
        "higher_is_better": True,
        "ms": bat_ms,
        "steps_per_solve": steps,
        "element_stage_updates_per_s": el_stage / (bat_ms / 1e3),
        "sequential": {"value": n / (seq_ms / 1e3), "unit": "solves/s", "ms": seq_ms,
                       "gpu_launches": seq_launches,
                       "how": "dg_step per problem, one problem after another, one stream"},
        "speedup_vs_sequential": seq_ms / bat_ms,
        "sequential_graphs": graph,
        "speedup_vs_sequential_graphs": (graph["ms"] / bat_ms) if "ms" in graph else None,
        "max_rel_diff_vs_sequential": diff,
        "gpu_launches": bat_launches,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"problems": n, "K_total": int(Ks.sum()), "K_min": int(Ks.min()),
                   "K_max": int(Ks.max()),
                   "per_order_K": {str(N): int(Ks[Ns == N].sum()) for N in sorted(set(Ns.tolist()))},
                   "orders": sorted(set(Ns.tolist())), "wave_speeds": [0.5, 1.0, 2.0],
                   "seed": args.batch_seed, "products": "tensor cores (tcgen05, 3xTF32)",
                   "graph": "one-step CUDA graphs (concurrent mode: each order's 5 stage "
                            "launches on its own branch, then the step counter; split mode: 5 "
                            "stage launches over all orders, then the step counter)"},
        "launch_mode": {"chosen": mode, "tuned_split_ms": tuned_split_ms,
                        "tuned_concurrent_ms": tuned_conc_ms,
                        "how": "dg_batch_tune: 3 stage launches in each mode, the faster kept"},
        "block_elems": {str(g + 1): {"elems": int(elems[g]), "tuned_ms_default": float(ms_def[g]),
                                     "tuned_ms_alternative": float(ms_alt[g])}
                        for g in range(7) if nblk[g]},
        "plan": {"cta_per_order": {str(g + 1): int(cta[g]) for g in range(7) if nblk[g]},
                 "blocks_per_order": {str(g + 1): int(nblk[g]) for g in range(7) if nblk[g]},
                 "cost_us_per_block_iter": {str(g + 1): float(cost[g]) * 1e6 for g in range(7)
                                            if nblk[g]},
                 "tune_seconds": tune_s},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "peak_kind": peak_kind,
                     "kernel": "dg_batch_tc_kernel (fused RHS + LSRK stage, all orders)"},
        "clocks": clk,
    }


def serving_requests(n_requests=120, seed=777, k_lo=1000, k_hi=200000, orders=(3, 4, 5, 6, 7),
                     t_lo=0.5, t_hi=2.0, f=10.0, time_scale=0.01):
    """Seeded solve requests: K log-uniform in [k_lo, k_hi] (jittered
    Delaunay unit-square meshes), N uniform over `orders`, final time
    uniform in [t_lo, t_hi], Ricker source of peak frequency f at a seeded
    location, zero initial fields.  Times are scaled by `time_scale` (final
    time and wavelet period alike: T -> T s, f -> f / s, t0 = 1.2 / f) so
    that a solve takes tens to hundreds of steps.  Returns dicts with mesh, N,
    T and source (x, y, f, t0, amplitude)."""
    import numpy as np

    from synth import jittered_delaunay_mesh, n_for_target_elements

    rng = np.random.default_rng(seed)
    out = []
    fs = f / time_scale
    for i in range(n_requests):
        k = float(np.exp(rng.uniform(np.log(k_lo), np.log(k_hi))))
        N = int(rng.choice(orders))
        T = float(rng.uniform(t_lo, t_hi)) * time_scale
        xs, ys = rng.uniform(0.2, 0.8, size=2)
        mesh = jittered_delaunay_mesh(n_for_target_elements(k), seed=seed + 1 + i)
        out.append({"mesh": mesh, "N": N, "T": T,
                    "source": (float(xs), float(ys), fs, 1.2 / fs, 1.0)})
    return out


def _percentile(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def serve_plain_sequential(P, reqs, dev_solvers, arrivals):
    """Requests served one at a time, in arrival order, by plain dg_solve on
    each request's own device operator (operator resident in HBM beforehand,
    its point source attached with dg_operator_set_source, fields and
    residual allocated beforehand): per request, zero the fields, solve to
    T, copy the result into pinned host memory, wait for it.  Latency runs
    from the arrival time to the result in host memory."""
    import numpy as np
    import torch

    stream = torch.cuda.current_stream()
    bufs = [(s.new_fields(), s.new_fields(), torch.empty((3, s.fstride), pin_memory=True))
            for s in dev_solvers]
    t_start = P.Server.clock() + 0.01
    rec = []
    launches0 = sum(P.dg_launch_count(s.op) for s in dev_solvers)
    for i, (r, s) in enumerate(zip(reqs, dev_solvers)):
        t_arr = t_start + arrivals[i]
        while P.Server.clock() < t_arr:
            pass
        q, res, h = bufs[i]
        q.zero_()
        nsteps, _ = s.solve(q, res, r["T"])
        h.copy_(q, non_blocking=True)
        stream.synchronize()
        rec.append((t_arr, P.Server.clock(), s.K, nsteps))
    lat = [d - a for a, d, _, _ in rec]
    span = rec[-1][1] - rec[0][0]
    out = {"solves_per_s": len(rec) / span, "p50_ms": 1e3 * _percentile(lat, 50),
           "p99_ms": 1e3 * _percentile(lat, 99), "mean_ms": 1e3 * float(np.mean(lat)),
           "makespan_s": span, "failed": 0,
           "gpu_launches": sum(P.dg_launch_count(s.op) for s in dev_solvers) - launches0,
           "element_stage_updates_per_s": 5.0 * sum(K * n for _, _, K, n in rec) / span}
    results = [s.to_numpy(b[0]) for s, b in zip(dev_solvers, bufs)]
    return out, results


def run_serving(args):
    """Serving workload: Poisson arrivals at each rate in --serve-rates of
    the same seeded requests, served by the continuous-batching server, by
    the same server with each work limit of --serve-work-limits (nodal values
    per field stepped together, first come first served), and by the server
    admitting one request at a time (sequential plain solves).  Latency =
    result in host memory - submission.  One JSON line."""
    import numpy as np
    import torch

    import paper_1304_5546_gb300 as P

    torch.cuda.set_device(0)
    reqs = serving_requests(args.serve_requests, seed=args.serve_seed,
                            time_scale=args.serve_time_scale)
    solvers = [P.Solver(*r["mesh"], N=r["N"], precision="fp32", host_only=True) for r in reqs]
    outs = [np.zeros((3, s.K, s.Np), np.float32) for s in solvers]
    # memory budget -> element capacity per order: 36 Np + 92 bytes per
    # element (two field buffers and the residual, records, face codes),
    # split evenly over the orders
    budget = args.serve_budget_gb * 1e9
    orders = sorted({r["N"] for r in reqs})
    cap = [0] * 7
    for N in orders:
        Np = (N + 1) * (N + 2) // 2
        cap[N - 1] = int(budget / len(orders) / (36 * Np + 92))
    rng = np.random.default_rng(args.serve_seed + 1)
    # plain sequential solves: device operators with the request's source
    dev = []
    if not args.serve_no_plain:
        for r in reqs:
            d = P.Solver(*r["mesh"], N=r["N"], precision="fp32")
            P.dg_operator_set_source(d.op, r["source"])
            dev.append(d)
        warm = dev[0].new_fields()
        dev[0].solve(warm, dev[0].new_fields(), reqs[0]["T"])  # warm the kernels
        torch.cuda.synchronize()
    clocks = ClockSampler(None) if not args.no_clocks else None
    if clocks:
        clocks.start()
    # warm: one request through each mode (kernels, graphs, staging)
    for seq in (False, True):
        srv = P.Server(cap, sequential=seq)
        srv.wait(srv.submit(solvers[0], reqs[0]["T"], source=reqs[0]["source"], out=outs[0]))
        srv.close()
    rows = []
    for lam in args.serve_rates:
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(reqs)))
        arrivals -= arrivals[0]
        row = {"rate_per_s": lam}
        modes = ([("batched", False, 0)]
                 + [("limited_%g" % w, False, int(w)) for w in args.serve_work_limits]
                 + [("sequential", True, 0)])
        for mode, seq, limit in modes:
            srv = P.Server(cap, sequential=seq, work_limit=limit)
            t_start = P.Server.clock() + 0.01
            ids = []
            for i, (r, s, o) in enumerate(zip(reqs, solvers, outs)):
                while P.Server.clock() < t_start + arrivals[i]:
                    pass
                ids.append(srv.submit(s, r["T"], source=r["source"], out=o))
            infos = [srv.wait(i) for i in ids]
            st = srv.stats()
            srv.close()
            lat = [i["t_done"] - i["t_submit"] for i in infos if i["state"] == 2]
            span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
            el_steps = sum(i["K"] * i["nsteps"] for i in infos if i["state"] == 2)
            row[mode] = {"solves_per_s": len(lat) / span, "p50_ms": 1e3 * _percentile(lat, 50),
                         "p99_ms": 1e3 * _percentile(lat, 99), "mean_ms": 1e3 * float(np.mean(lat)),
                         "makespan_s": span, "failed": st["failed"], "gpu_launches": st["launches"],
                         "batched_steps": st["steps"],
                         "element_stage_updates_per_s": 5.0 * el_steps / span}
        if dev:
            row["plain_sequential"], plain_out = serve_plain_sequential(P, reqs, dev, arrivals)
            # the served results against the plain solves of the same requests
            row["max_rel_diff_served_vs_plain"] = max(
                float(np.abs(o - p).max() / max(np.abs(p).max(), 1e-30))
                for o, p in zip(outs, plain_out))
        row["speedup_solves_per_s"] = row["batched"]["solves_per_s"] / row["sequential"]["solves_per_s"]
        row["p99_ratio_seq_over_batched"] = row["sequential"]["p99_ms"] / row["batched"]["p99_ms"]
        if dev:
            base = row["plain_sequential"]
            for mode, _, _ in modes:
                row[mode]["vs_plain_sequential"] = {
                    "solves_per_s": row[mode]["solves_per_s"] / base["solves_per_s"],
                    "p50": row[mode]["p50_ms"] / base["p50_ms"],
                    "p99": row[mode]["p99_ms"] / base["p99_ms"]}
        for mode, _, limit in modes:
            if limit:
                row[mode]["speedup_solves_per_s"] = (row[mode]["solves_per_s"]
                                                     / row["sequential"]["solves_per_s"])
                row[mode]["p99_ratio_seq_over_this"] = (row["sequential"]["p99_ms"]
                                                        / row[mode]["p99_ms"])
        rows.append(row)
    clk = clocks.stop() if clocks else None
    for d in dev:
        d.close()
    Ks = np.array([s.K for s in solvers])
    return {
        "workload": "serving",
        "metric": "served solves/s and p50/p99 latency (continuous batching vs sequential)",
        "unit": "solves/s",
        "higher_is_better": True,
        "rates": rows,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"requests_per_rate": len(reqs), "K_min": int(Ks.min()), "K_max": int(Ks.max()),
                   "K_mean": float(Ks.mean()), "orders": orders,
                   "T_range": [0.5 * args.serve_time_scale, 2.0 * args.serve_time_scale],
                   "time_scale": args.serve_time_scale,
                   "source": "Ricker, peak frequency %g, t0 = 1.2 / f, seeded location"
                             % (10.0 / args.serve_time_scale),
                   "initial_fields": "zero", "memory_budget_gb": args.serve_budget_gb,
                   "capacity_elements": {str(N): cap[N - 1] for N in orders},
                   "latency": "submission to result in host memory",
                   "sequential": "same server, one request admitted at a time",
                   "plain_sequential": "dg_solve per request in arrival order on its own "
                                       "resident device operator (point source attached), "
                                       "result copied to pinned host memory"},
        "clocks": clk,
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--order", type=int, default=5)
    ap.add_argument("--n", type=int, default=707, help="mesh resolution (K = 2 n^2)")
    ap.add_argument("--precision", default="fp32",
                    choices=["fp32", "fp64", "tf32", "bf16", "bf16x3", "fp32tc", "fp32ept"],
                    help="fp32: the default FP32 kernel of the order (3xTF32 tensor-core "
                         "products at N = 5); fp32tc / fp32ept: the tensor-core / "
                         "element-thread kernel; tf32 / bf16 / bf16x3: the precision-path "
                         "variants (FP32 fields and accumulation)")
    ap.add_argument("--simt", action="store_true", help="FP32 products on CUDA cores")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--_oracle-sample", nargs=3, default=None)
    ap.add_argument("--_oracle-timings", action="store_true")
    ap.add_argument("--study", choices=["precision", "sweep", "partition", "oracle", "longrun"],
                    default=None,
                    help="instead of the benchmark line: the precision-path study "
                         "(use with --order 7 --n 362 for K = 262,088)")
    ap.add_argument("--study-steps", type=int, default=500)
    ap.add_argument("--longrun-threads", type=int, default=4,
                    help="numpy threads of each oracle process of --study longrun")
    ap.add_argument("--longrun-quick", action="store_true",
                    help="--study longrun on small meshes and few steps")
    ap.add_argument("--sweep-orders", type=int, nargs="+", default=list(range(1, 8)))
    ap.add_argument("--sweep-media", action="store_true",
                    help="--study sweep with a seeded per-element permittivity")
    ap.add_argument("--partition-parts", type=int, nargs="+", default=[1, 2, 4, 8])
    ap.add_argument("--workload", choices=["single", "batched", "serving"], default="single",
                    help="single: the large-mesh benchmark line (default); batched: many "
                         "mixed-order problems in one launch per stage vs sequential solves")
    ap.add_argument("--batch-problems", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--batch-seed", type=int, default=4242)
    ap.add_argument("--batch-orders", type=int, nargs="+", default=[3, 5, 7])
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[10, 30, 100, 300, 1000])
    ap.add_argument("--serve-seed", type=int, default=777)
    ap.add_argument("--serve-time-scale", type=float, default=0.01)
    ap.add_argument("--serve-budget-gb", type=float, default=4.0)
    ap.add_argument("--serve-work-limits", type=float, nargs="*", default=[3e6, 1e7],
                    help="work limits (nodal values per field stepped together) to serve with")
    ap.add_argument("--serve-no-plain", action="store_true",
                    help="leave out the plain sequential dg_solve baseline")
    ap.add_argument("--no-workloads", action="store_true",
                    help="main line only: without its batched and serving objects")
    args = ap.parse_args(argv)
    if args._oracle_sample:
        n, N, sec = int(args._oracle_sample[0]), int(args._oracle_sample[1]), float(args._oracle_sample[2])
        v, steps, K, el = oracle_sample_rate(n, N, sec)
        print(json.dumps({"value": v, "steps": steps, "K": K, "seconds": el}))
        return 0
    if args.study == "precision":
        print(json.dumps(run_precision_study(args)), flush=True)
        return 0
    if args.study == "sweep":
        print(json.dumps(run_sweep_study(args)), flush=True)
        return 0
    if args.study == "partition":
        print(json.dumps(run_partition_study(args)), flush=True)
        return 0
    if args.study == "longrun":
        print(json.dumps(run_longrun_study(args)), flush=True)
        return 0
    if args._oracle_timings:
        print(json.dumps(oracle_timings()), flush=True)
        return 0
    if args.study == "oracle":
        print(json.dumps(run_oracle_study(args)), flush=True)
        return 0
    if args.workload == "serving" and args.impl == "ours":
        print(json.dumps(run_serving(args)), flush=True)
        return 0
    if args.workload == "batched" and args.impl == "ours":
        print(json.dumps(run_batched(args)), flush=True)
        return 0
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
