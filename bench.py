"""Benchmark of the state-vector hot path.

One step = reset to |0...0>, the 32-qubit random U3 + CNOT brickwork of depth
40 (seed 8091) applied through the C ABI, flush, P(q=1) for every qubit,
<sum_i Z_i Z_{i+1}> and a full-register sample.  The default arm runs
complex64 with greedy fusion into <=5-qubit blocks (the fast path); a bounded
sample of the same circuit on the plain complex128 path (one launch per
gate) is timed beside it.

Printed: one JSON line (rank 0).  ``value`` is amplitude-updates/s over the
whole job: sum over all gates of 2^(n - #controls), divided by the device
time of the K timed steps (CUDA events on the library's stream, max over
ranks).  ``e2e`` is the same metric on the host clock around the public API
calls, including the host->device gate data and the device->host results.

``--impl reference`` times the FP64 CPU oracle instead, on a bounded sample of
the same workload on the host cores.
"""
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import circuitgen as cg  # noqa: E402

METRIC = "amplitude-updates/s & HBM-roofline fraction, fused c64 vs plain c128, infid≤1e-5"
UNIT = "amp-updates/s"
SEED = 8091


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--depth", type=int, default=40)
    ap.add_argument("--precision", default="c64")
    ap.add_argument("--fusion", default="greedy")
    ap.add_argument("--kmax", type=int, default=6)
    ap.add_argument("--plain-layers", type=int, default=2, help="layers of the plain c128 comparison sample")
    ap.add_argument("--grover-iterations", type=int, default=20,
                    help="Grover iterations timed (0: the full r = floor(pi/4 sqrt(2^n)) search)")
    ap.add_argument("--cpu-gates", type=int, default=6, help="gates of the oracle CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--fused-c128-layers", type=int, default=6,
                    help="layers of the circuit timed as complex128 double-float fused blocks (0: skip)")
    ap.add_argument("--vqe-uniform", default=None, metavar="COUNT,QUBITS,LAYERS",
                    help="vqe workload: COUNT circuits of QUBITS qubits and LAYERS layers (seeded angles) "
                         "instead of the 4096-circuit mix")
    ap.add_argument("--vqe-config", default=None, metavar="THREADS,M",
                    help="vqe workload: fixed launch configuration instead of the autotuner's")
    ap.add_argument("--workload", default="random",
                    choices=["random", "vqe", "planner", "qft", "grover", "fig7", "adder", "plain", "sharded"],
                    help="random: the headline line; vqe / planner: secondary measurements")
    return ap.parse_args()


def workload(n, depth):
    ops = cg.random_u3_brickwork(n, depth, SEED)
    terms = cg.zz_chain_terms(n)
    u = float(cg.uniform_draws(SEED + 1, 1)[0])
    return ops, terms, u


def amp_updates(ops, n):
    return float(sum(1 << (n - len(o.controls)) for o in ops))


def workload_name(n, depth):
    return ("%d-qubit random circuit, depth %d: U3 on every qubit + CNOT brickwork per layer (seed %d); "
            "then P(q=1) for all q, <sum Z_i Z_i+1>, measure-all" % (n, depth, SEED))


# ---------------------------------------------------------------------------
# distributed plumbing (replicas: each rank runs its own register)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device=None):
    """Max of a host scalar over all ranks (the timed region of the slowest
    rank).  Works with the nccl (device tensor) and gloo (CPU) backends."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds_per_rank, world, device=None):
    """Replicas: every rank processes the same number of units; the job's
    throughput is all ranks' units over the slowest rank's time."""
    t = max_over_ranks(seconds_per_rank, world, device)
    return units_per_rank * world / t, t


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


# profiling class of the library -> kernel name in profiles/traffic.json
TRAFFIC_KERNEL = {"block_tc": "k_block_tmem5", "block_tc6": "k_block_tmem6"}


def kernel_traffic(kernel, n):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.json), scaled from the captured register size to n
    (the block kernels' traffic is proportional to 2^n); with n None, the
    capture's DRAM bytes per algorithmic byte.  None if there is
    no capture or the kernel's sources changed since it was taken (SHA-256
    over the listed source files, in order)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[kernel]
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, KeyError, ValueError, TypeError):
        return None
    if h.hexdigest() != rec["sha256"]:
        return None
    if n is None:  # the captured DRAM bytes per algorithmic byte
        return rec["bytes_per_launch"] / rec["alg_bytes_per_launch"]
    return rec["bytes_per_launch"] * 2.0 ** (n - rec["n"])


def measure_ops(sim, n, terms, u, stream, peak, b, reps=3):
    """CUDA-event time (median of reps, after one warm call) and HBM
    bandwidth of each read or measurement on the current register.  Bytes
    are algorithmic: what the operation must read and write, counted in
    whole 32-byte sectors (DRAM's access granularity)."""
    import torch

    N = 2.0 ** n
    # the half of the amplitudes with bit q set spans every 32-byte sector
    # when q < log2(32 / b): then the least traffic is the whole state
    def half(q):
        return N * b if (1 << q) * b < 32 else N / 2 * b
    ops = [
        ("probs_all", lambda: sim.probs_all(), N * b, "P(q=1) for every q and the norm: one read"),
        ("prob_q0", lambda: sim.prob(0), half(0), "P(q0=1): the amplitudes with bit 0 set (every sector)"),
        ("prob_top", lambda: sim.prob(n - 1), half(n - 1), "P(q%d=1): reads the half with the top bit set" % (n - 1)),
        ("expect_zz", lambda: sim.expect(terms), N * b, "sum_i Z_i Z_i+1 (%d terms): one read" % len(terms)),
        ("measure_q0", lambda: sim.measure(0, u), 2 * N * b + half(0),
         "measure qubit 0 and collapse: read all (sums), read the kept amplitudes (every sector), write all"),
        ("measure_all", lambda: sim.measure_all(u), 2 * N * b,
         "sample all qubits and collapse to the basis state: read all, write all"),
    ]
    out = {}
    for name, fn, nbytes, what in ops:
        fn()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        out[name] = {"ms": ms, "GB/s": nbytes / ms / 1e6, "frac": nbytes / ms / 1e6 / peak, "bytes": nbytes,
                     "what": what}

    # a diagonal block: every controlled phase and RZ among 12 qubits, fused
    # by the planner into one pass (timed by the library's per-launch events,
    # so the host's table build is not counted)
    dq = list(range(n - 12, n))
    diag_ops = [cg.op("R", (j,), (k,), (0.1 * (j + k),)) for j in dq for k in dq if k < j]
    diag_ops += [cg.op("RZ", (j,), (), (0.3 + 0.01 * j,)) for j in dq]
    sim.flush()
    sim.set_profiling(True)
    times, passes = [], []
    for rep in range(reps + 1):
        sim.reset_stats()
        sim.run(diag_ops)
        sim.flush()
        kt = sim.kernel_times()
        passes.append(sim.stats()["passes"])
        if rep and "block_diag" in kt:
            times.append(kt["block_diag"]["total_ms"] / kt["block_diag"]["launches"])
    sim.set_profiling(False)
    if times:
        ms = statistics.median(times)
        out["diag_block_12q"] = {"ms": ms, "GB/s": 2 * N * b / ms / 1e6, "frac": 2 * N * b / ms / 1e6 / peak,
                                 "bytes": 2 * N * b, "passes": passes[-1],
                                 "what": "%d diagonal gates on qubits %d..%d (controlled phases, RZ) as one "
                                         "multiply-by-table pass: read all, write all" % (len(diag_ops), dq[0], dq[-1])}

    # an emulated classical function: x -> 7x mod 1021 on 10 qubits (identity
    # above 1020), one pass; its algorithmic bytes are those of the register
    # values that move (1020 of 1024: 0 and 1021..1023 are fixed points)
    perm = [(7 * x) % 1021 if x < 1021 else x for x in range(1024)]
    moved = sum(1 for x in range(1024) if perm[x] != x) / 1024.0
    for name, qs in (("permute_low10", list(range(10))), ("permute_high10", list(range(n - 10, n)))):
        def fn(qs=qs):
            sim.apply_permutation(perm, qs)
            sim.flush()
        fn()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        pb = 2 * N * b * moved
        out[name] = {"ms": ms, "GB/s": pb / ms / 1e6, "frac": pb / ms / 1e6 / peak, "bytes": pb,
                     "what": "x -> 7x mod 1021 on qubits %d..%d: read and write the amplitudes of the 1020 "
                             "register values that move" % (qs[0], qs[-1])}
    return out


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.machine()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle sample (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(n, ops, gates):
    """Time the FP64 oracle on the first `gates` gates of the workload, after
    one untimed gate that touches every page of the register."""
    import oracle

    oracle.build()
    sim = oracle.OracleSim(n)
    sim.apply_op(ops[0])
    sample = ops[1:1 + gates]
    t0 = time.perf_counter()
    for o in sample:
        sim.apply_op(o)
    dt = time.perf_counter() - t0
    upd = amp_updates(sample, n)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = int(os.environ.get("OMP_NUM_THREADS", cores))
    return upd / dt, dt, threads, len(sample)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = args.n
    ops, _, _ = workload(n, args.depth)
    vals = []
    t_all = []
    steps_total = args.warmup + args.steps
    import oracle

    oracle.build()
    sim = oracle.OracleSim(n)
    sim.apply_op(ops[0])  # touch all pages once
    g = max(1, args.cpu_gates // 2)
    for s in range(steps_total):
        sample = ops[1 + s * g: 1 + (s + 1) * g]
        t0 = time.perf_counter()
        for o in sample:
            sim.apply_op(o)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            vals.append(amp_updates(sample, n) / dt)
            t_all.append(dt)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    v = statistics.median(vals)
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(t_all),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": workload_name(n, args.depth), "n_qubits": n, "precision": "c128",
                   "fusion": "none", "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                         "sample": "%d gates of the workload per step on the FP64 oracle, %d qubits" % (g, n)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    import paper_1612_08091_gb300 as q

    q.load()
    n = args.n
    ops, terms, u = workload(n, args.depth)
    upd_step = amp_updates(ops, n)
    stream = torch.cuda.current_stream(device)
    sim = q.Simulator(n, precision=args.precision, fusion=args.fusion, kmax=args.kmax, stream=stream)

    h2d_bytes = sum(16 * (1 << (2 * len(o.targets))) + 4 * (len(o.targets) + len(o.controls)) for o in ops)
    d2h_bytes = 8 * (n + 1) + 8 + 8 * 4096 + 32  # probabilities, expectation, measure-all sums and result

    def step():
        sim.reset(0)
        sim.run(ops)
        sim.flush()
        p1, nrm = sim.probs_all()
        e = sim.expect(terms)
        j = sim.measure_all(u)
        return p1, nrm, e, j

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sim.reset_stats()
    sim.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    dev_s = ev0.elapsed_time(ev1) / 1e3
    host_s = t1 - t0
    kt = sim.kernel_times()
    st = sim.stats()
    sim.set_profiling(False)
    value, dev_s = job_throughput(upd_step * args.steps, dev_s, world, device)
    e2e, host_s = job_throughput(upd_step * args.steps, host_s, world, device)

    peak, peak_kind = measured_peaks()
    dom_name, dom = max(kt.items(), key=lambda kv: kv[1]["total_ms"]) if kt else (None, None)
    roof = None
    if dom:
        per_launch_bytes = dom["alg_bytes"] / dom["launches"]
        per_launch_s = dom["total_ms"] / dom["launches"] / 1e3
        achieved = per_launch_bytes / per_launch_s / 1e9
        step_ms_total = sum(v["total_ms"] for v in kt.values())
        traffic = kernel_traffic(TRAFFIC_KERNEL[dom_name], n) if dom_name in TRAFFIC_KERNEL else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind, "traffic": traffic, "kernel": dom_name,
                "alg_bytes_per_launch": per_launch_bytes, "launches_per_step": dom["launches"] / args.steps,
                "share_of_gate_time": dom["total_ms"] / step_ms_total if step_ms_total else None}

    # the reads and measurements of the step, one at a time on the same
    # register (outside the timed region): each against the HBM roofline
    # with its algorithmic bytes
    measurements = measure_ops(sim, n, terms, u, stream, peak, 8 if args.precision == "c64" else 16) \
        if rank == 0 else None

    plain = plain_df = fused_df = None
    if not args.no_plain and rank == 0 and args.plain_layers > 0:
        sim.close()
        torch.cuda.empty_cache()
        def layers_prefix(nl):
            cnt = 0
            for layer in range(nl):
                cnt += n + len(range(layer % 2, n - 1, 2))
            return ops[:cnt]

        def plain_sample(df, sample, fusion="none", kmax=6):
            with q.Simulator(n, precision="c128", fusion=fusion, kmax=kmax, stream=stream, c128_df=df) as ps:
                ps.run(sample[: n])  # warm-up on the same register
                ps.flush()
                torch.cuda.synchronize()
                ps.reset_stats()
                ps.set_profiling(True)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ps.run(sample)
                ps.flush()
                b.record(stream)
                torch.cuda.synchronize()
                pkt = ps.kernel_times()
                pst = ps.stats()
            ps_s = a.elapsed_time(b) / 1e3
            torch.cuda.empty_cache()
            rate = amp_updates(sample, n) / ps_s
            # every logical amplitude update of a plain complex128 gate reads
            # and writes 16 bytes: roofline = HBM bandwidth / 32 bytes
            roof = None
            if fusion == "none":
                roof = {"value": peak * 1e9 / 32.0, "unit": UNIT, "frac": rate * 32.0 / (peak * 1e9),
                        "what": "measured HBM bandwidth / 32 bytes per logical amplitude update"}
            if roof is not None:
                roof["note"] = ("double-float arithmetic: the plain complex128 >= 80% target is met in this "
                                "arithmetic only" if df else
                                "fp64 arithmetic: the dense gate is bound by the FP64 pipe (~2.1 TB/s), not HBM")
            return {"value": rate, "unit": UNIT, "precision": "c128", "hbm_roofline": roof,
                    "arithmetic": "double-float (fp32 pairs, ~2^-45 relative)" if df else "fp64",
                    "fusion": fusion if fusion == "none" else "%s, kmax %d" % (fusion, kmax),
                    "sample": "first %d gates of the same %d-qubit circuit, %s (the whole circuit: "
                              "bench.py --workload plain)"
                              % (len(sample), n, "one launch per gate" if fusion == "none"
                                 else "%d fused passes" % pst["passes"]),
                    "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"],
                                    "GB/s": v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9} for k, v in pkt.items()}}

        # the first `plain_layers` layers of the same circuit, one launch per
        # gate; and complex128 fused blocks in double-float arithmetic over
        # the first `fused_c128_layers` layers (4-qubit blocks: the block
        # arithmetic, not HBM, bounds complex128 blocks)
        plain = plain_sample(False, layers_prefix(args.plain_layers))
        plain_df = plain_sample(True, layers_prefix(args.plain_layers))
        if args.fused_c128_layers > 0:
            fused_df = plain_sample(True, layers_prefix(args.fused_c128_layers), "greedy", 4)

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        v, dt, threads, g = oracle_sample(n, ops, args.cpu_gates)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": cpu_model(),
               "sample": "%d gates of the %d-qubit workload on the FP64 oracle (%.1f s)" % (g, n, dt)}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "compute": ("bf16x3 tensor-core blocks, fp32 accumulate; fp64 reductions" if args.precision == "c64"
                        else "fp64"),
            "data": "synthetic",
            "config": {"workload": workload_name(n, args.depth), "n_qubits": n, "depth": args.depth,
                       "precision": args.precision, "fusion": args.fusion, "kmax": args.kmax,
                       "gates_per_step": len(ops), "amp_updates_per_step": upd_step,
                       "passes_per_step": st["passes"] / args.steps,
                       "l2": "inputs larger than L2 (state %.2f GiB vs 126 MiB L2)" % (
                           (8 if args.precision == "c64" else 16) * 2.0 ** n / 2 ** 30),
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roof,
            "kernel_times": kt,
            "measurements": measurements,
            "plain_c128": plain,
            "plain_c128_double_float": plain_df,
            "fused_c128_double_float": fused_df,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes},
            "clocks": clk,
            "gpu_launches": int(st["launches"]),
            "check": {"norm2": results[-1][1], "zz": results[-1][2], "sample": results[-1][3]},
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# secondary workloads (their own JSON lines; not the headline)
# ---------------------------------------------------------------------------
def run_vqe(args):
    """4096 hardware-efficient-ansatz circuits (n uniform 10..20, L 2..8),
    TFIM energies, one persistent launch replayed from a CUDA graph."""
    import torch

    import paper_1612_08091_gb300 as q

    torch.cuda.set_device(0)
    if args.vqe_uniform:
        count, nqu, lay = (int(v) for v in args.vqe_uniform.split(","))
        circuits = cg.hea_batch(count, seed=2016, nmin=nqu, nmax=nqu, lmin=lay, lmax=lay)
        workload = "%d ansatz circuits of %d qubits, %d layers, RY/RZ + CNOT ladder, TFIM energy (seed 2016)" % (
            count, nqu, lay)
    else:
        circuits = cg.hea_batch(4096, seed=2016)
        workload = ("4096 ansatz circuits, n uniform in 10..20, L in 2..8, RY/RZ + CNOT ladder, "
                    "TFIM energy (seed 2016)")
    nq = [c["n"] for c in circuits]
    nl = [c["L"] for c in circuits]
    angles = q.hea_angles(circuits)
    upd = float(sum((1 << c["n"]) * (c["L"] * (3 * c["n"] - 1)) for c in circuits))
    with q.Batch(nq, nl) as b:
        t0 = time.perf_counter()
        if args.vqe_config:
            cfg = tuple(int(v) for v in args.vqe_config.split(","))
            b.set_config(*cfg)
        else:
            cfg = b.autotune(angles, reps=3)
        tune_s = time.perf_counter() - t0
        for _ in range(args.warmup):
            b.run(angles)
        ts = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            e = b.run(angles)
            ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)

    # the two classes alone, same launch configuration: circuits held in
    # shared memory (n <= m) and circuits in global memory (n > m)
    def class_time(sel):
        cs = [c for c in circuits if sel(c)]
        if not cs:
            return None, 0
        ang = q.hea_angles(cs)
        with q.Batch([c["n"] for c in cs], [c["L"] for c in cs]) as bb:
            bb.set_config(*cfg)
            for _ in range(args.warmup):
                bb.run(ang)
            tt = []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                bb.run(ang)
                tt.append(time.perf_counter() - t0)
        return statistics.median(tt), len(cs)

    t_res, n_res = class_time(lambda c: c["n"] <= cfg[1])
    t_glob, n_glob = class_time(lambda c: c["n"] > cfg[1])
    # HBM bytes of the circuits above the shared-memory size m: the initial
    # |0> write, per layer a pair pass and a top-qubit pass (each reads and
    # writes the state), the final permutation pass and the energy read
    m = cfg[1]
    hbm = float(sum(8.0 * (1 << c["n"]) * (4 * c["L"] + 4) for c in circuits if c["n"] > m))
    peak, peak_kind = measured_peaks()
    # DRAM bytes: the ncu capture's ratio to the algorithmic bytes (the
    # global-memory kernel's traffic grows with the state passes it makes)
    ratio = kernel_traffic("k_vqe_batch_global", None)
    out = {"metric": "variational batch throughput", "value": upd / t, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
           "dtype": "c64", "data": "synthetic",
           "config": {"workload": workload, "circuits_per_s": len(circuits) / t,
                      "amp_updates_per_step": upd, "autotuned": {"threads": cfg[0], "smem_qubits": cfg[1]},
                      "autotune_s": tune_s, "timing": "host clock around sim_batch_run (graph replay: angles "
                                                      "H2D, persistent kernel, energies D2H)"},
           "classes": {
               "shared_memory": {"circuits": n_res, "ms": None if t_res is None else 1e3 * t_res,
                                 "bound": "on chip (shared memory, FP32)"},
               "global_memory": {"circuits": n_glob, "ms": None if t_glob is None else 1e3 * t_glob,
                                 "GB/s": None if not t_glob else hbm / t_glob / 1e9,
                                 "frac": None if not t_glob else hbm / t_glob / 1e9 / peak},
               "timing": "each class alone as its own batch, same launch configuration"},
           "roofline": {"bound": "hbm", "achieved": hbm / t / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": hbm / t / 1e9 / peak, "peak_source": peak_kind,
                        "traffic": None if ratio is None else ratio * hbm,
                        "bytes_per_step": hbm,
                        "what": "global-memory traffic of the circuits above the shared-memory size (n > %d): "
                                "4L + 4 state passes each; the rest stays on chip" % m},
           "check": {"energy_mean": float(np.mean(e))}}
    print(json.dumps(out), flush=True)
    return 0


def run_planner(args):
    """Learned fusion planning as configured: the cost model trained on this
    GPU's timings of 26-30 qubit random, QFT and H / controlled-Rz circuits
    (complex64), evaluated on a held-out 33-qubit complex64 random circuit of
    depth 30 against greedy fusion with kmax 5 and kmax 6 (each the median of
    `steps` timed runs) and against the unfused complex128 path over the
    whole circuit (one run; 128 GiB).  A second model, trained on complex128
    double-float timings (26-28 qubits), is evaluated on a held-out 30-qubit
    circuit, where blocks are bound by arithmetic and plans differ."""
    import torch

    import paper_1612_08091_gb300 as q
    from paper_1612_08091_gb300 import costmodel

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sizes = (26, 27, 28, 29, 30)
    t0 = time.perf_counter()
    X, ms = costmodel.collect(sizes=sizes, precisions=("c64",), seed=2018)
    collect_s = time.perf_counter() - t0
    params, loss = costmodel.train(X, ms, hidden=32, epochs=300)
    n = 33
    ops = cg.random_u3_brickwork(n, 30, seed=2018)
    upd = amp_updates(ops, n)

    def timed(fusion, model=None, n=n, ops=ops, precision="c64", df=False, kmax=6, steps=None):
        steps = args.steps if steps is None else steps
        with q.Simulator(n, precision=precision, fusion=fusion, c128_df=df, kmax=kmax, stream=stream) as sim:
            if model is not None:
                sim.set_cost_model(*model)
            res = []
            for _ in range(args.warmup + steps):
                sim.reset(0)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                sim.run(ops)
                sim.flush()
                torch.cuda.synchronize()
                res.append(time.perf_counter() - t1)
            st = sim.stats()
            p1, nrm = sim.probs_all()
        torch.cuda.empty_cache()
        return {"s": statistics.median(res[args.warmup:]), "passes": st["passes"] / (args.warmup + steps),
                "runs": steps, "p1": np.asarray(p1), "norm2": nrm}

    g5 = timed("greedy", kmax=5)
    g6 = timed("greedy", kmax=6)
    ml = timed("mlp", (params, 32))
    # the unfused complex128 path over the whole circuit, FP64 arithmetic,
    # one timed run (warm-up: the circuit's first layer)
    with q.Simulator(n, precision="c128", fusion="none", stream=stream) as ps:
        ps.run(ops[:n])
        ps.flush()
        ps.reset(0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ps.run(ops)
        ps.flush()
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t1
        p1_plain, _ = ps.probs_all()
    torch.cuda.empty_cache()

    # complex128 in double-float arithmetic, where fused blocks are bound by
    # FP32 arithmetic rather than HBM: a second model trained on this GPU's
    # complex128 double-float timings (26-28 qubits), held out at 30 qubits
    t0 = time.perf_counter()
    X2, ms2 = costmodel.collect(sizes=(26, 27, 28), precisions=("c128",), kmaxes=(1, 2, 3, 4, 5), seed=2018,
                                df=True)
    collect2_s = time.perf_counter() - t0
    params2, loss2 = costmodel.train(X2, ms2, hidden=32, epochs=300)
    n2 = 30
    ops2 = cg.random_u3_brickwork(n2, 10, seed=2018)
    upd2 = amp_updates(ops2, n2)
    g2 = timed("greedy", n=n2, ops=ops2, precision="c128", df=True)
    m2 = timed("mlp", (params2, 32), n=n2, ops=ops2, precision="c128", df=True)

    def arm(r, u):
        return {"ms": 1e3 * r["s"], "passes": r["passes"], "value": u / r["s"], "runs": r["runs"],
                "timing": "host clock around run + flush (median)"}

    out = {"metric": "learned fusion planner, held-out 33-qubit circuit", "value": upd / ml["s"], "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * ml["s"],
           "higher_is_better": True, "dtype": "c64", "data": "synthetic",
           "config": {"workload": "33-qubit random U3 + CNOT brickwork, depth 30 (seed 2018), complex64",
                      "training": {"samples": int(len(ms)), "sizes": list(sizes), "collect_s": collect_s,
                                   "train_mse_log_ms": loss,
                                   "circuits": "random depth 4, QFT of a basis state, H / controlled-Rz chain"}},
           "learned": dict(arm(ml, upd), gain_over_greedy_k5=g5["s"] / ml["s"], gain_over_greedy_k6=g6["s"] / ml["s"]),
           "greedy_k5": arm(g5, upd),
           "greedy_k6": arm(g6, upd),
           "plain_c128": {"ms": 1e3 * t_plain, "value": upd / t_plain, "runs": 1, "arithmetic": "fp64",
                          "what": "whole circuit, one launch per gate, complex128",
                          "learned_speedup": t_plain / ml["s"]},
           "check": {"max_p1_difference_learned_vs_plain_c128": float(np.max(np.abs(ml["p1"] - np.asarray(p1_plain)))),
                     "learned_norm2": ml["norm2"]},
           "c128_double_float": {
               "workload": "30-qubit random U3 + CNOT brickwork, depth 10 (seed 2018), complex128 in "
                           "double-float arithmetic",
               "training": {"samples": int(len(ms2)), "sizes": [26, 27, 28], "collect_s": collect2_s,
                            "train_mse_log_ms": loss2},
               "greedy_k5": arm(g2, upd2),
               "learned": dict(arm(m2, upd2), gain_over_greedy=g2["s"] / m2["s"])}}
    print(json.dumps(out), flush=True)
    return 0


def run_circuit(args):
    """The structured circuits of the method's examples, fused complex64
    (greedy, kmax 6) against plain complex128 (one launch per gate, timed on
    a sample of the first gates and extrapolated per amplitude update):
      qft    -- QFT on 30 qubits applied to a seeded basis state x; checked
                against 2^{-n/2} exp(2 pi i x y / 2^n) on sampled amplitudes;
      grover -- Grover search on 28 qubits: 20 iterations timed, the full
                r = floor(pi/4 sqrt(2^n)) extrapolated; the marked amplitude
                checked against (-1)^r sin((2r+1) theta) for the 20;
      fig7   -- the paper's benchmark circuit on 30 qubits: H on all, the
                controlled-Rz chain, H on all; checked by its norm."""
    import math

    import torch

    import paper_1612_08091_gb300 as q

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    w = args.workload
    basis = 0
    if w == "qft":
        n = 30
        basis = int(cg.random_basis_state(n, SEED))
        ops = cg.qft_ops(n)
        what = "QFT on %d qubits of the basis state x = %d (seed %d)" % (n, basis, SEED)
        full_iters = None
    elif w == "grover":
        n = 28
        marked = int(cg.grover_marked(n, 2017))
        full_iters = cg.grover_iterations(n)
        iters = args.grover_iterations if args.grover_iterations > 0 else full_iters
        ops = cg.grover_ops(n, marked, iterations=iters)
        what = ("Grover search on %d qubits, marked item %d (seed 2017): %d of the r = %d iterations timed"
                % (n, marked, iters, full_iters))
    elif w == "adder":
        m = 15
        n = 2 * m + 2
        rng = np.random.default_rng(SEED)
        a_in, b_in = (int(v) for v in rng.integers(0, 1 << m, 2))
        reps = 4
        ops = cg.ripple_adder_ops(m, reps=reps)
        basis = cg.adder_basis_index(m, a_in, b_in)
        what = ("ripple-carry adder (CNOT / Toffoli) of two %d-bit registers on %d qubits, %d times, basis input "
                "a = %d, b = %d (seed %d)" % (m, n, reps, a_in, b_in, SEED))
        full_iters = None
    else:
        n = 30
        ops = cg.hadamard_crz_chain(n, SEED)
        what = "H on all %d qubits, controlled-Rz chain (angles seed %d), H on all" % (n, SEED)
        full_iters = None
    upd = amp_updates(ops, n)

    def timed(sim, ops_, reps):
        ts = []
        for _ in range(args.warmup + reps):
            sim.reset(basis)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.run(ops_)
            sim.flush()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return statistics.median(ts[args.warmup:])

    classes = None
    with q.Simulator(n, precision="c64", fusion="greedy", stream=stream) as sim:
        t_fused = timed(sim, ops, args.steps)
        # the register holds the last timed run's result; passes per run
        passes = sim.stats()["passes"] / (args.warmup + args.steps)
        if t_fused < 10.0:
            # one more run with events around every launch: time and HBM
            # bandwidth (algorithmic bytes) per kernel class
            peak, _ = measured_peaks()
            sim.reset(basis)
            sim.set_profiling(True)
            sim.run(ops)
            sim.flush()
            kt = sim.kernel_times()
            sim.set_profiling(False)
            classes = {k: {"launches": v["launches"], "ms": v["total_ms"],
                           "GB/s": v["alg_bytes"] / v["total_ms"] / 1e6 if v["total_ms"] else None,
                           "frac": v["alg_bytes"] / v["total_ms"] / 1e6 / peak if v["total_ms"] else None}
                       for k, v in kt.items()}
            # the register again holds the circuit's result for the checks below
        check = {}
        if w == "qft":
            rng = np.random.default_rng(SEED + 1)
            rnd = [int(i) for i in rng.integers(0, 1 << n, 256)]
            got = np.array([sim.get_amplitudes(i, 1)[0] for i in rnd] + list(sim.get_amplitudes(0, 4096)))
            ys = rnd + list(range(4096))
            # exact integer phase x*y mod 2^n, then to an angle
            want = np.array([np.exp(2j * math.pi * ((basis * y) % (1 << n)) / float(1 << n)) for y in ys])
            want *= 2.0 ** (-n / 2)
            check = {"max_abs_error": float(np.max(np.abs(got - want))), "amplitude": 2.0 ** (-n / 2),
                     "sampled": int(len(ys))}
        elif w == "grover":
            theta = math.asin(2.0 ** (-n / 2))
            a = sim.get_amplitudes(marked, 1)[0]
            want = (-1) ** iters * math.sin((2 * iters + 1) * theta)
            p1, nrm = sim.probs_all()
            check = {"marked_amplitude": [float(a.real), float(a.imag)], "closed_form": want,
                     "abs_error": float(abs(a - want)),
                     "success_probability_raw": float(abs(a) ** 2),
                     "success_probability_normalised": float(abs(a) ** 2 / nrm),
                     "success_closed_form": math.sin((2 * iters + 1) * theta) ** 2, "norm2": nrm,
                     "norm2_error": abs(nrm - 1.0)}
        elif w == "adder":
            bb, z = b_in, 0
            for _ in range(reps):
                z ^= (a_in + bb) >> m
                bb = (a_in + bb) % (1 << m)
            want_idx = cg.adder_basis_index(m, a_in, bb, z)
            amp = sim.get_amplitudes(want_idx, 1)[0]
            check = {"result_index": want_idx, "amplitude": [float(amp.real), float(amp.imag)]}
        else:
            _, nrm = sim.probs_all()
            check = {"norm2": nrm}
    torch.cuda.empty_cache()
    no_perm = None
    no_prod = None
    if w == "grover":
        # the same iterations with the one-qubit layers as 6-qubit blocks
        with q.Simulator(n, precision="c64", fusion="greedy", stream=stream, product_passes=False) as sim:
            t_np = timed(sim, ops, args.steps)
            no_prod = {"ms": 1e3 * t_np, "passes": sim.stats()["passes"] / (args.warmup + args.steps),
                       "value": upd / t_np, "what": "greedy 6-qubit blocks only (product_passes=False)"}
        torch.cuda.empty_cache()
    if w == "adder":
        # the same circuit with dense blocks only (no permutation blocks)
        with q.Simulator(n, precision="c64", fusion="greedy", stream=stream, perm_blocks=False) as sim:
            t_np = timed(sim, ops, args.steps)
            sim.reset_stats()
            sim.reset(basis)
            sim.run(ops)
            sim.flush()
            no_perm = {"ms": 1e3 * t_np, "passes": sim.stats()["passes"], "value": upd / t_np,
                       "what": "greedy dense blocks only (perm_blocks=False)"}
        torch.cuda.empty_cache()

    # plain complex128 on a sample of the first gates
    sample = ops[: min(len(ops), 64)]
    with q.Simulator(n, precision="c128", fusion="none", stream=stream) as ps:
        t_plain_sample = timed(ps, sample, 1)
    rate_plain = amp_updates(sample, n) / t_plain_sample
    out = {"metric": "%s: fused complex64 vs plain complex128" % w, "value": upd / t_fused, "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_fused,
           "higher_is_better": True, "dtype": "c64", "data": "synthetic",
           "config": {"workload": what, "n_qubits": n, "gates": len(ops), "passes": passes,
                      "amp_updates": upd, "fusion": "greedy", "kmax": 6},
           "plain_c128": {"value": rate_plain, "unit": UNIT, "sample": "first %d gates, one launch per gate, fp64"
                          % len(sample), "extrapolated_ms": 1e3 * upd / rate_plain,
                          "speedup_of_fused": (upd / t_fused) / rate_plain},
           "check": check}
    if no_perm is not None:
        out["dense_blocks_only"] = no_perm
    if no_prod is not None:
        out["blocks_only"] = no_prod
    if classes is not None:
        out["classes"] = classes
    if full_iters:
        out["config"]["extrapolated_full_search_s"] = t_fused * full_iters / iters
    print(json.dumps(out), flush=True)
    return 0


def run_plain(args):
    """The plain complex128 path (one launch per gate) over the WHOLE
    32-qubit depth-40 circuit of the headline, in FP64 arithmetic and in
    double-float arithmetic (FP32 pairs, about 2^-45 relative per product),
    each run once after a warm-up on the circuit's first layer; the two
    results are compared with each other."""
    import torch

    import paper_1612_08091_gb300 as q

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.n
    ops, terms, _ = workload(n, args.depth)
    upd = amp_updates(ops, n)
    peak, peak_kind = measured_peaks()
    arms = {}
    probs = {}
    for name, df in (("fp64", False), ("double_float", True)):
        with q.Simulator(n, precision="c128", fusion="none", stream=stream, c128_df=df) as sim:
            sim.run(ops[:n])
            sim.flush()
            sim.reset(0)
            torch.cuda.synchronize()
            sim.reset_stats()
            sim.set_profiling(True)
            clocks = ClockSampler(0)
            clocks.start()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.run(ops)
            sim.flush()
            e1.record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop()
            t = e0.elapsed_time(e1) / 1e3
            kt = sim.kernel_times()
            st = sim.stats()
            sim.set_profiling(False)
            p1, nrm = sim.probs_all()
            zz = sim.expect(terms)
            probs[name] = np.asarray(p1)
        torch.cuda.empty_cache()
        rate = upd / t
        arms[name] = {
            "value": rate, "unit": UNIT, "s": t, "gates": len(ops), "launches": int(st["launches"]),
            "hbm_roofline": {"value": peak * 1e9 / 32.0, "frac": rate * 32.0 / (peak * 1e9), "peak": peak,
                             "peak_source": peak_kind,
                             "what": "measured HBM bandwidth / 32 bytes per logical amplitude update"},
            "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"],
                            "GB/s": v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9,
                            "frac": v["alg_bytes"] / (v["total_ms"] / 1e3) / 1e9 / peak} for k, v in kt.items()},
            "check": {"norm2": nrm, "zz": zz}, "clocks": clk}
    out = {"metric": "plain complex128 path, whole circuit", "value": arms["double_float"]["value"], "unit": UNIT,
           "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * arms["double_float"]["s"],
           "higher_is_better": True, "dtype": "c128", "data": "synthetic",
           "config": {"workload": workload_name(n, args.depth), "n_qubits": n, "fusion": "none",
                      "amp_updates": upd, "l2": "state %.0f GiB, larger than L2" % (16 * 2.0 ** n / 2 ** 30)},
           "fp64": arms["fp64"], "double_float": arms["double_float"],
           "check": {"max_prob_difference_fp64_vs_double_float":
                     float(np.max(np.abs(probs["fp64"] - probs["double_float"])))}}
    print(json.dumps(out), flush=True)
    return 0


def run_sharded(args):
    """The headline circuit (32 qubits, depth 40, complex64 fused) on a
    register split into 2 shards of 31 qubits on one GPU: the exchange
    planner moves the top qubit into the shards whenever a gate targets it
    (sim_swap_halves), the shards run their own fused queues.  Reported
    beside the same circuit on one handle, with the exchange kernel timed on
    its own (CUDA events, median of 3) against the HBM roofline (it reads and
    writes half of each shard)."""
    import torch

    import paper_1612_08091_gb300 as q
    from paper_1612_08091_gb300.sharded import ShardedSimulator

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n, g = args.n, 1
    ops, terms, u = workload(n, args.depth)
    upd = amp_updates(ops, n)
    peak, peak_kind = measured_peaks()

    def timed(run):
        ts = []
        for _ in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return statistics.median(ts[args.warmup:])

    with q.Simulator(n, precision="c64", fusion="greedy", stream=stream) as one:
        def run_one():
            one.reset(0)
            one.run(ops)
            one.flush()
        t_one = timed(run_one)
        p1_one, _ = one.probs_all()
    torch.cuda.empty_cache()
    with ShardedSimulator(n, global_qubits=g, precision="c64", fusion="greedy", stream=stream) as sh:
        def run_sh():
            sh.reset(0)
            sh.run(ops)
            sh.flush()
        t_sh = timed(run_sh)
        ex = sh.exchanges / (args.warmup + args.steps)
        p1_sh, nrm = sh.probs_all()
        # the exchange kernel alone: one swap of the top qubit with local 30
        a, b = sh.shards[0], sh.shards[1]
        ts = []
        for _ in range(4):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            a.swap_halves(b, n - g - 1)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t_swap = statistics.median(ts[1:])
    torch.cuda.empty_cache()
    swap_bytes = 2.0 * 2 * 8 * 2.0 ** (n - g - 1)  # half of each shard read and written
    out = {"metric": "sharded register: 2 shards on one GPU", "value": upd / t_sh, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_sh, "higher_is_better": True,
           "dtype": "c64", "data": "synthetic",
           "config": {"workload": workload_name(n, args.depth) + " (circuit only)", "shards": 1 << g,
                      "exchanges_per_run": ex, "fusion": "greedy", "kmax": args.kmax},
           "single_handle": {"ms": 1e3 * t_one, "value": upd / t_one},
           "exchange_kernel": {"ms": 1e3 * t_swap, "bytes": swap_bytes, "GB/s": swap_bytes / t_swap / 1e9,
                               "frac": swap_bytes / t_swap / 1e9 / peak, "peak_source": peak_kind,
                               "what": "sim_swap_halves of two 31-qubit complex64 shards on qubit 30: "
                                       "half of each shard read and written"},
           "check": {"max_p1_difference_vs_single_handle": float(np.max(np.abs(np.asarray(p1_sh) - p1_one))),
                     "norm2": nrm}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "vqe":
        return run_vqe(args)
    if args.workload == "planner":
        return run_planner(args)
    if args.workload == "plain":
        return run_plain(args)
    if args.workload == "sharded":
        return run_sharded(args)
    if args.workload in ("qft", "grover", "fig7", "adder"):
        return run_circuit(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
