"""Benchmark: QFactor gate-updates/s at 12 qubits on one GB300.

Workload: 12-qubit linear brickwork of 12 layers (66 general U(4) gates),
target reachable from seeded Haar-random gates, 8 seeded Haar starts, circuit
tensors in complex64 (4x4 updates in FP64).  One step = one TwoSidedSweep of
all 8 starts = 8 x 132 = 1056 gate updates; the tensors are rebuilt from the
target every 40 sweeps as in Qfactor.  The 8 tensors hold 1.07 GB, far more
than L2, so no L2 flush is needed between steps.

Prints one JSON line (see the repository's benchmark contract).  With
``--impl reference`` it times the FP64 CPU oracle instead, on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import qf_inputs as qi  # noqa: E402

N_QUBITS = 12
LAYERS = 12
STARTS = 8
SEED = 2024
RESET_ITER = 40  # Sec. III-A2 reset_iter
METRIC = "gate-updates/s at 12 qubits (% HBM roofline)"
UNIT = "gate-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["c64", "c128"], default="c64")
    ap.add_argument("--starts", type=int, default=STARTS)
    ap.add_argument("--qubits", type=int, default=N_QUBITS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="timed CPU work of the oracle baseline sample")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-c128", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=4096)
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--no-lookahead", action="store_true")
    ap.add_argument("--no-kqubit", action="store_true")
    ap.add_argument("--no-spec", action="store_true")
    ap.add_argument("--oracle-1core", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--profile-case", choices=["k4", "k3", "pair", "pass", "batched", "batched_k"], default=None,
                    help="run one small case of a kernel family for a profiler capture and exit: "
                         "k4/k3/pair/pass: 12 qubits, 2 starts, complex64, one live sweep after one "
                         "warm-up sweep; batched/batched_k: the first 512/256 instances of the "
                         "benchmark's batches, an autotuning call then one run")
    return ap.parse_args()


def workload(n, starts):
    locs = qi.brickwork_locations(n, LAYERS)
    inst = qi.make_problem(n, locs, starts, seed=SEED)
    return inst


def config_dict(args, inst):
    prec = "complex64 tensor, FP64 4x4 update" if args.precision == "c64" else "complex128 tensor, FP64"
    return {
        "workload": f"{inst.n}-qubit linear brickwork, {LAYERS} layers ({inst.p} U(4) gates), "
                    f"{inst.n_starts} starts per GPU, reachable Haar target, {prec}",
        "n_qubits": inst.n,
        "n_gates": inst.p,
        "starts_per_gpu": inst.n_starts,
        "precision": args.precision,
        "updates_per_step_per_gpu": inst.n_starts * 2 * inst.p,
        "step": "one TwoSidedSweep of every start; after every 40th sweep of the plan the gates "
                "are re-unitarised and the tensors rebuilt (the timed region starts at such a sweep, "
                "so it holds ceil(steps/40) rebuilds)",
        "l2": "no flush: the circuit tensors (%.2f GB) exceed L2" % (
            inst.n_starts * 4**inst.n * (8 if args.precision == "c64" else 16) / 1e9),
        "parallelism": "replicas (independent starts per GPU)",
    }


# ------------------------------------------------------------------ ranks


def replica_seed(rank):
    """Each rank runs its own seeded starts (replicas: no data exchange)."""
    return SEED + 1000 * int(rank)


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (the job's time is its slowest rank)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, steps, ms_max):
    """Whole-job units per second: every rank's units over the slowest
    rank's time."""
    return units_per_rank * world * steps / (ms_max / 1e3)


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        try:
            sm = [float(r[1]) for r in rows]
            smax = max(float(r[2]) for r in rows)
        except ValueError:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("[N/A]", ""))
                if any(r[3] not in ("[N/A]", "") for r in rows) else None}


# ------------------------------------------------------------------ helpers


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_tf32_peak():
    """Dense TF32 tensor rate: the measured sustained BF16 GEMM rate (the
    pass is timed inside long sweeps) times the nominal TF32 / BF16 ratio;
    the fallback's sustained BF16 figure without the file."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if d.get("bf16_tflops_sustained"):
            return float(d["bf16_tflops_sustained"]) * TF32_PER_BF16, \
                "measured bf16_tflops_sustained x nominal TF32/BF16 (1.1/2.25)"
    return 1700.0 * TF32_PER_BF16, "fallback sustained BF16 1.7 PFLOP/s x nominal TF32/BF16 (1.1/2.25)"


_ALU_PEAKS = {}


def measured_alu_peaks(torch, dev):
    """Dense FP64 and FP32 throughput of this GPU, measured in this run: the
    best of 5 cuBLAS DGEMM (4096^3) and SGEMM (8192^3, TF32 off) products,
    2 n^3 flops each, CUDA events.  Denominators for the complex128 pass
    (bound by the FP64 pipe) and the double-FP32 pass (FP32 pipe)."""
    if _ALU_PEAKS:
        return _ALU_PEAKS
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for key, dt, m in (("fp64_gflops", torch.float64, 4096), ("fp32_gflops", torch.float32, 8192)):
            a = torch.randn(m, m, dtype=dt, device=dev)
            b = torch.randn(m, m, dtype=dt, device=dev)
            c = a @ b
            best = float("inf")
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            _ALU_PEAKS[key] = 2.0 * m**3 / (best / 1e3) / 1e9
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    _ALU_PEAKS["how"] = ("cuBLAS DGEMM 4096^3 and SGEMM 8192^3 (TF32 off) through torch.matmul, "
                         "best of 5, 2 n^3 flops, CUDA events, in this run")
    return _ALU_PEAKS


def batched_pipes(name="batched_kernel_pipes.json"):
    """Pipe fractions of a batched kernel from a committed ncu summary
    (profiles/<name>), if it was taken on the current kernel sources; else
    None."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    for src, h in d.get("kernel_sources", {}).items():
        with open(os.path.join(ROOT, src), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != h:
                return None
    return d


def kernel_traffic(precision, starts, n):
    """DRAM bytes per pass launch from a committed ncu summary, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_2306_08152_gb300", "csrc", "qf_pass.cu")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()
    if d.get("kernel_sha256") != h:
        return None
    key = f"{precision}"
    entry = d.get("per_launch", {}).get(key)
    if not entry:
        return None
    # scale a capture of a smaller case by the entries processed
    scale = (starts * 4**n) / float(entry["entries"])
    return entry["dram_bytes"] * scale


def oracle_setup(inst):
    """The oracle's circuit tensor of start 0 (untimed setup of a sample)."""
    import oracle as orc

    V = orc.circuit_unitary(inst.target_gates, inst.locs, inst.n)
    return orc.init_circuit_tensor(V, inst.starts[0], inst.locs, inst.n)


def oracle_updates(T, gates, locs, n, seconds, max_updates=None):
    """Time the oracle's gate updates (Alg. 1 TwoSidedSweep backward steps,
    ApplyRight, CalcEnvMat, OptimizeGate, ApplyLeft) from tensor T for about
    `seconds`; returns (updates, wall s, CPU s)."""
    import oracle as orc

    gates = gates.copy()
    p = len(locs)
    done = 0
    w0 = time.perf_counter()
    c0 = time.process_time()
    k = p - 1
    while True:
        a, b = int(locs[k][0]), int(locs[k][1])
        T = orc.apply_right(T, gates[k].conj().T, a, b, n)
        E = orc.calc_env_mat(T, a, b, n)
        u, _ = orc.optimize_gate(E)
        gates[k] = u
        T = orc.apply_left(T, u, a, b, n)
        done += 1
        k = (k - 1) % p
        el = time.perf_counter() - w0
        if el >= seconds or (max_updates and done >= max_updates):
            break
    wall = time.perf_counter() - w0
    cpu = time.process_time() - c0
    return done, wall, cpu


def oracle_sample(inst, seconds, max_updates=None):
    """The oracle's gate updates on start 0 of the workload, on every host
    core NumPy uses."""
    T = oracle_setup(inst)
    return oracle_updates(T, inst.starts[0], inst.locs, inst.n, seconds, max_updates), T


def oracle_single_core(inst, T, seconds):
    """The same oracle updates in a child process pinned to one host core
    with one BLAS/OpenMP thread (the tensor is handed over in a file, so the
    child only times updates)."""
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "oracle_state.npz")
        np.savez(path, T=T, gates=inst.starts[0], locs=inst.locs, n=inst.n)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-1core", path,
               "--cpu-seconds", str(seconds)]
        res = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        return {"error": res.stderr.strip().splitlines()[-1] if res.stderr.strip() else "failed"}
    return json.loads(res.stdout.strip().splitlines()[-1])


def run_oracle_1core(args):
    """Child of oracle_single_core: pin to one core, time the updates."""
    cpus = sorted(os.sched_getaffinity(0))
    os.sched_setaffinity(0, {cpus[-1]})
    st = np.load(args.oracle_1core)
    done, wall, cpu = oracle_updates(st["T"], st["gates"], st["locs"], int(st["n"]), args.cpu_seconds)
    print(json.dumps({"updates": done, "wall_s": wall, "cpu_s": cpu, "core": cpus[-1]}))
    return 0


# ------------------------------------------------------------------ reference arm


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    inst = workload(args.qubits, 1)
    import oracle as orc  # noqa: F401

    # warm-up samples of one update each, then K timed samples of 2 updates
    for _ in range(args.warmup):
        oracle_sample_cached(inst, 1)
    total_updates = 0
    total_wall = 0.0
    total_cpu = 0.0
    for _ in range(args.steps):
        d, w, c = oracle_sample_cached(inst, 2)
        total_updates += d
        total_wall += w
        total_cpu += c
    value = total_updates / total_wall
    cores = round(total_cpu / total_wall, 2)
    # the arm's configuration; the oracle samples start 0 of it (starts are
    # independent, so its per-update rate is the workload's)
    cfg = config_dict(args, workload(args.qubits, args.starts))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{total_updates} gate updates (ApplyRight, CalcEnvMat, "
                                   f"OptimizeGate, ApplyLeft) of the FP64 NumPy oracle on start 0 "
                                   f"of the {inst.n}-qubit workload (starts are independent); "
                                   f"2 updates per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


_ORACLE_STATE = {}


def oracle_sample_cached(inst, updates):
    """Like oracle_sample, but keeps the oracle's tensor between calls so
    that each reference step times only its own updates."""
    import oracle as orc

    st = _ORACLE_STATE.get(id(inst))
    n, locs = inst.n, inst.locs
    if st is None:
        V = orc.circuit_unitary(inst.target_gates, locs, n)
        T = orc.init_circuit_tensor(V, inst.starts[0], locs, n)
        st = {"T": T, "gates": inst.starts[0].copy(), "k": len(locs) - 1}
        _ORACLE_STATE[id(inst)] = st
    w0 = time.perf_counter()
    c0 = time.process_time()
    for _ in range(updates):
        k = st["k"]
        a, b = int(locs[k][0]), int(locs[k][1])
        T = orc.apply_right(st["T"], st["gates"][k].conj().T, a, b, n)
        E = orc.calc_env_mat(T, a, b, n)
        u, _ = orc.optimize_gate(E)
        st["gates"][k] = u
        st["T"] = orc.apply_left(T, u, a, b, n)
        st["k"] = (k - 1) % len(locs)
    return updates, time.perf_counter() - w0, time.process_time() - c0


# ------------------------------------------------------------------ extra lines


def run_batched(args, qf, torch, dev):
    """Batched uneven instantiation: 4096 reachable instances of 3, 4 and 5
    qubits (2:1:1), 5-40 U(4) gates on random adjacent pairs, 4 starts each,
    complex64 sweeps with FP64 refinement in one persistent launch; metric:
    instances whose best start reaches cost <= 1e-10 per second.  The plain
    FP64 per-instance GPU path (qf_instantiate_ex per instance, complex128)
    runs on a sample of the same instances for comparison."""
    insts = qi.batched_instances(args.batch_instances, 4, seed=SEED)
    probs = []
    for inst in insts:
        V = qf.circuit_unitary(inst.n, inst.locs, torch.from_numpy(inst.target_gates), device=dev)
        probs.append((V.cpu().numpy(), inst.locs, inst.starts))
    opts = dict(dist_tol=1e-10, max_sweeps=500)
    qf.instantiate_batched(probs[:64], precision=qf.QF_C64_REFINE64, **opts)  # warm-up + tuning
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = qf.instantiate_batched(probs, precision=qf.QF_C64_REFINE64, **opts)
    wall = time.perf_counter() - t0
    best = res["costs"][np.arange(len(probs)), res["best"]]
    ok = int((best <= 1e-10).sum())
    # the same instances with complex128 tensors throughout (no complex64
    # phase): do the complex64 sweeps lose successes?
    qf.instantiate_batched(probs[:64], precision=qf.QF_C128, **opts)  # tuning
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res128 = qf.instantiate_batched(probs, precision=qf.QF_C128, **opts)
    wall128 = time.perf_counter() - t0
    best128 = res128["costs"][np.arange(len(probs)), res128["best"]]
    ok128 = int((best128 <= 1e-10).sum())
    both = int(((best <= 1e-10) & (best128 <= 1e-10)).sum())
    # plain FP64 per-instance path on a sample
    sample = probs[: max(1, min(64, len(probs)))]
    t1 = time.perf_counter()
    ok_plain = 0
    for V, L, G in sample:
        r = qf.instantiate_ex(torch.from_numpy(V).to(dev), L, torch.from_numpy(G).to(dev), **opts)
        ok_plain += int(r["best_cost"] <= 1e-10)
    wall_plain = time.perf_counter() - t1
    return {
        "metric": "batched instantiations/s at cost<=1e-10", "unit": "instantiations/s",
        "value": ok / wall, "success": ok, "instances": len(probs), "starts": 4,
        "wall_s": wall, "kernel_ms": res["kernel_ms"], "warps_per_cta": res["warps_per_cta"],
        "ctas": res["ctas"], "sweeps": res["total_sweeps"], "c64_sweeps": res["total_c64_sweeps"],
        "precision": "complex64 sweeps, FP64 4x4 updates, complex128 refinement",
        "workload": f"{len(probs)} reachable instances, 3/4/5 qubits 2:1:1, 5-40 U(4) gates on random "
                    "adjacent pairs, 4 Haar starts, tol 1e-10, <=500 sweeps",
        "roofline": batched_roofline(),
        "success_c128": {"success": ok128, "value": ok128 / wall128, "wall_s": wall128,
                         "kernel_ms": res128["kernel_ms"], "sweeps": res128["total_sweeps"],
                         "success_in_both": both,
                         "note": "the same instances, starts and options with complex128 tensors "
                                 "throughout the batched kernel"},
        "success_plain_sample_c64refine": int((best[: len(sample)] <= 1e-10).sum()),
        "plain_fp64_per_instance": {"value": ok_plain / wall_plain, "unit": "instantiations/s",
                                    "success": ok_plain, "sample": len(sample), "wall_s": wall_plain,
                                    "path": "qf_instantiate_ex per instance, complex128, 4 starts"},
    }


def run_batched_k(args, qf, torch, dev):
    """Batched instantiation of circuits of 2- and 3-qubit gates
    (qf_instantiate_batched_k): 1024 reachable instances of 3, 4 and 5
    qubits (2:1:1), 4-16 gates on random qubit sets (each three-qubit with
    probability 1/2), 4 starts each, complex64 sweeps with FP64 refinement
    in one persistent launch; metric: instances whose best start reaches
    cost <= 1e-10 per second."""
    insts = qi.batched_instances_k(1024, 4, seed=SEED + 9)
    probs = []
    for inst in insts:
        V = qf.circuit_unitary_k(inst.n, inst.locs, inst.target_gates, device=dev)
        probs.append((V.cpu().numpy(), inst.locs, inst.starts))
    opts = dict(dist_tol=1e-10, max_sweeps=500)
    qf.instantiate_batched_k(probs[:64], precision=qf.QF_C64_REFINE64, **opts)  # warm-up + tuning
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = qf.instantiate_batched_k(probs, precision=qf.QF_C64_REFINE64, **opts)
    wall = time.perf_counter() - t0
    best = res["costs"][np.arange(len(probs)), res["best"]]
    ok = int((best <= 1e-10).sum())
    n3 = sum(sum(1 for q in x.locs if len(q) == 3) for x in insts)
    ng = sum(len(x.locs) for x in insts)
    return {
        "metric": "batched instantiations/s at cost<=1e-10, 2- and 3-qubit gates",
        "unit": "instantiations/s", "value": ok / wall, "success": ok, "instances": len(probs),
        "starts": 4, "wall_s": wall, "kernel_ms": res["kernel_ms"], "warps_per_cta": res["warps_per_cta"],
        "ctas": res["ctas"], "sweeps": res["total_sweeps"], "c64_sweeps": res["total_c64_sweeps"],
        "three_qubit_gates": n3, "gates": ng, "roofline": batched_roofline("batched_k_kernel_pipes.json"),
        "precision": "complex64 sweeps, FP64 4x4 and 8x8 updates, complex128 refinement",
        "workload": f"{len(probs)} reachable instances, 3/4/5 qubits 2:1:1, 4-16 gates on random qubit "
                    "sets (three-qubit with probability 1/2), 4 Haar starts, tol 1e-10, <=500 sweeps"}


def batched_roofline(name="batched_kernel_pipes.json"):
    """The batched kernels run whole small problems per warp with the
    tensors in shared memory: no HBM bound; the FP64 pipe (the updates'
    refinement) is the busiest unit.  Fractions from the committed capture
    of the same kernel source (null if the source changed since)."""
    d = batched_pipes(name)
    if d is None:
        return None
    return {"bound": "alu", "unit": "fraction of pipe cycles", "peak": 1.0,
            "achieved": d["fp64_pipe_active_frac"], "frac": d["fp64_pipe_active_frac"],
            "pipe": "FP64", "fp64_pipe_active_frac": d["fp64_pipe_active_frac"],
            "fp64_pipe_elapsed_frac": d["fp64_pipe_elapsed_frac"],
            "fp32_fma_pipe_active_frac": d["fma_pipe_active_frac"],
            "sm_active_frac_of_elapsed": d["sm_active_frac_of_elapsed"],
            "source": f"ncu capture (profiles/{name}): " + d["capture"]}


def run_c128(args, qf, torch, dev, inst, V, starts):
    """12-qubit sweep on complex128 tensors: bound by the FP64 pipe (64 FP64
    flops per entry per update)."""
    plan = qf.Plan(inst.n, inst.locs, inst.n_starts, qf.QF_C128)
    stream = torch.cuda.current_stream(dev)
    plan.load(V, starts, stream=stream)
    plan.sweep(1, reset_iter=0)
    plan.costs()
    plan.pass_stats()
    plan.enable_pass_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps = 2
    e0.record(stream)
    plan.sweep(steps, reset_iter=0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pass_ms, launches, _, pbytes = plan.pass_stats()
    plan.close()
    updates = inst.n_starts * 2 * inst.p * steps
    flops = pbytes / max(launches, 1) / 32 * 64  # 16-byte entries, read + write
    achieved = flops / ((pass_ms / 1e3) / max(launches, 1)) / 1e9
    peaks = measured_alu_peaks(torch, dev)
    return {"metric": "gate-updates/s at 12 qubits, complex128", "unit": "gate-updates/s",
            "value": updates / (ms / 1e3), "ms_per_sweep": ms / steps, "dtype": "c128",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fp64_gflops"],
                         "unit": "GFLOP/s", "frac": achieved / peaks["fp64_gflops"],
                         "peak_source": "measured FP64: " + peaks["how"],
                         "nominal_peak": 1250.0, "frac_of_nominal": achieved / 1250.0,
                         "flops_per_launch": flops}}


# FP32 pipe operations per tensor entry of a df64 pass (both operators):
# 8 complex multiply-adds of 48 operations (two TwoProd, two TwoSum and the
# lo-part gathering per real part) and 2 renormalisations of 6.
DF64_OPS_PER_ENTRY = 8 * 48 + 2 * 6
# FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz (maximum SM clock), one
# operation per lane per cycle (an FMA counts once)
FP32_PIPE_GOPS = 152 * 128 * 2.07


def run_df64(args, qf, torch, dev, inst, V, starts):
    """12-qubit sweep on double-FP32 tensors (QF_DF64): complex128-class
    accuracy from FP32 error-free arithmetic, bound by the FP32 pipe."""
    plan = qf.Plan(inst.n, inst.locs, inst.n_starts, qf.QF_DF64)
    stream = torch.cuda.current_stream(dev)
    plan.load(V, starts, stream=stream)
    plan.sweep(1, reset_iter=0)
    plan.costs()
    plan.pass_stats()
    plan.enable_pass_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps = 3
    e0.record(stream)
    plan.sweep(steps, reset_iter=0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pass_ms, launches, _, pbytes = plan.pass_stats()
    costs = plan.costs()
    plan.close()
    updates = inst.n_starts * 2 * inst.p * steps
    entries = pbytes / max(launches, 1) / 32  # 16-byte entries, read + write
    ops = entries * DF64_OPS_PER_ENTRY
    avg_s = (pass_ms / 1e3) / max(launches, 1)
    achieved = ops / avg_s / 1e9
    peak, _ = measured_peaks()
    peaks = measured_alu_peaks(torch, dev)
    return {"metric": "gate-updates/s at 12 qubits, df64 (double-FP32 complex tensor)",
            "unit": "gate-updates/s", "value": updates / (ms / 1e3), "ms_per_sweep": ms / steps,
            "dtype": "df64",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PIPE_GOPS,
                         "unit": "Gop/s", "frac": achieved / FP32_PIPE_GOPS,
                         "peak_source": "FP32 pipe from unit counts and clock: 152 SMs x 128 lanes "
                                        "x 2.07 GHz, one operation per lane per cycle",
                         "measured_sgemm_gflops": peaks["fp32_gflops"],
                         "frac_of_measured_sgemm_flops": 2 * achieved / peaks["fp32_gflops"],
                         "ops_per_entry": DF64_OPS_PER_ENTRY, "avg_launch_ms": avg_s * 1e3,
                         "hbm_gbs": pbytes / max(launches, 1) / avg_s / 1e9,
                         "hbm_frac": pbytes / max(launches, 1) / avg_s / 1e9 / peak},
            "final_costs": [float(c) for c in costs]}


def run_lookahead(args, qf, torch, dev, inst, V, starts, one_update_costs):
    """The same sweeps with look-ahead windows: two consecutive updates on
    disjoint pairs share one pass (complex64).  Gate updates per second
    count every update, as in the headline."""
    n, locs = inst.n, inst.locs
    stream = torch.cuda.current_stream(dev)
    plan = qf.Plan(n, locs, inst.n_starts, qf.QF_C64)
    windows = plan.set_lookahead(True)
    plan.load(V, starts, stream=stream)
    for _ in range(args.warmup):
        plan.sweep(1, reset_iter=40)
    plan.costs()
    plan.pass_stats()
    plan.enable_pass_timing(True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.sweep(1, reset_iter=40)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pass_ms, pass_launches, all_launches, pass_bytes = plan.pass_stats()
    plan.enable_pass_timing(False)
    plan.sweep(1, reset_iter=40)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        plan.sweep(1, reset_iter=40)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1) / args.steps
    if plan.status() != 0:
        raise RuntimeError("device status reports a non-finite update")
    costs = plan.costs()
    plan.close()
    peak, peak_kind = measured_peaks()
    alg_bytes = pass_bytes / max(pass_launches, 1)
    avg_pass_s = (pass_ms / 1e3) / max(pass_launches, 1)
    achieved = alg_bytes / avg_pass_s / 1e9
    updates = inst.n_starts * 2 * inst.p
    value = updates * args.steps / (ms / 1e3)
    # the one-update-per-pass roofline: one read and one write of a start's
    # tensor per gate update at the measured copy bandwidth
    one_pass_bytes = 2 * 8 * 4**n
    one_pass_roofline = peak * 1e9 / one_pass_bytes
    return {"value": value, "unit": UNIT,
            "effective": {"frac_of_one_pass_roofline": value / one_pass_roofline,
                          "one_pass_roofline_updates_per_s": one_pass_roofline,
                          "effective_gbs": value * one_pass_bytes / 1e9,
                          "note": "updates/s against the bytes one update per pass would move"},
            "value_graph": updates / (ms_graph / 1e3),
            "ms_per_step": ms / args.steps, "ms_per_step_graph": ms_graph,
            "pair_windows_per_sweep": windows,
            "passes_per_sweep": pass_launches / args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "kernel": "pass kernels of the look-ahead sweep (two-update pair pass; "
                                   "single passes where a window holds one update)",
                         "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                         "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_pass_s * 1e3},
            "gpu_launches": int(all_launches),
            "final_costs": [float(c) for c in costs],
            "max_cost_diff_vs_one_update": float(np.max(np.abs(np.asarray(costs) -
                                                               np.asarray(one_update_costs))))}


def run_kqubit(args, qf, torch, dev):
    """Three-qubit gates: 12 qubits, layers of gates on consecutive triples
    (offsets 0, 1, 2 in turn, 20 gates), 8 starts, complex64 tensors, one
    sweep per step; the 8x8 pass reads and writes the tensor once per update."""
    n, S = 12, 8
    locs = []
    for layer in range(6):
        o = layer % 3
        locs += [(q, q + 1, q + 2) for q in range(o, n - 2, 3)]
    gen = qi.rng(SEED + 33)
    tgt = [qi.haar_unitary(8, gen) for _ in locs]
    V = qf.circuit_unitary_k(n, locs, tgt, device=dev)
    starts = qf.flatten_gates([[qi.haar_unitary(8, qi.rng(SEED + 34 + s)) for _ in locs]
                               for s in range(S)]).to(dev)
    stream = torch.cuda.current_stream(dev)
    plan = qf.Plan(n, locs, S, qf.QF_C64)
    plan.load(V, starts, stream=stream)
    plan.sweep(2, reset_iter=0)  # the second sweep captures the graph
    plan.costs()
    steps = 5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # value: CUDA-graph replay of each sweep
    e0.record(stream)
    plan.sweep(steps, reset_iter=0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1)
    # roofline: the same sweeps as live launches with CUDA events around every pass
    plan.pass_stats()
    plan.enable_pass_timing(True)
    e0.record(stream)
    plan.sweep(steps, reset_iter=0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pass_ms, launches, _, pbytes = plan.pass_stats()
    costs = plan.costs()
    plan.close()
    peak, peak_kind = measured_peaks()
    avg_s = (pass_ms / 1e3) / max(launches, 1)
    alg = pbytes / max(launches, 1)
    achieved = alg / avg_s / 1e9
    updates = S * 2 * len(locs) * steps
    return {"metric": "gate-updates/s at 12 qubits, three-qubit gates, complex64",
            "unit": "gate-updates/s", "value": updates / (ms_graph / 1e3),
            "ms_per_sweep": ms_graph / steps, "ms_per_sweep_live": ms / steps,
            "timing": "value: CUDA-graph replay of each sweep; roofline: live launches with CUDA "
                      "events around every pass",
            "workload": f"12 qubits, {len(locs)} three-qubit gates on consecutive triples (6 layers, "
                        "offsets 0/1/2), 8 starts, reachable Haar target, complex64 tensor, FP64 8x8 update",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "kernel": "pass8_kernel (B <- L B R on 8x8 blocks)",
                         "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                         "alg_bytes_per_launch": alg, "avg_launch_ms": avg_s * 1e3,
                         "pass_share_of_step": pass_ms / ms if ms > 0 else None},
            "final_costs": [float(c) for c in costs]}


# Tensor-core flops per tensor entry of the complex64 16x16 pass (both
# operators, tcgen05 in 3xTF32 form): two stages of a real K = 32 dot
# product per real output value (2 per entry), three TF32 products each.
K4_TC_FLOPS_PER_ENTRY = 2 * 2 * 32 * 2 * 3
# nominal dense TF32 / BF16 tensor rate on GB300 (1.1 / 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def run_k4(args, qf, torch, dev):
    """Four-qubit gates: 12 qubits, layers of gates on consecutive quadruples
    (offsets 0 and 2 in turn, 15 gates), 8 starts, complex64 tensors, one
    sweep per step.  The 16x16 pass reads and writes the tensor once per
    update and runs its 128 complex-FMA-equivalents per entry on the tensor
    cores (768 TF32 flops per entry in 3xTF32 form), so HBM is its
    roofline (48 flop/byte, below the TF32 ridge of about 120)."""
    n, S = 12, 8
    locs = []
    for layer in range(6):
        o = 0 if layer % 2 == 0 else 2
        locs += [(q, q + 1, q + 2, q + 3) for q in range(o, n - 3, 4)]
    gen = qi.rng(SEED + 44)
    tgt = [qi.haar_unitary(16, gen) for _ in locs]
    V = qf.circuit_unitary_k(n, locs, tgt, device=dev)
    starts = qf.flatten_gates([[qi.haar_unitary(16, qi.rng(SEED + 45 + s)) for _ in locs]
                               for s in range(S)]).to(dev)
    stream = torch.cuda.current_stream(dev)
    plan = qf.Plan(n, locs, S, qf.QF_C64)
    plan.load(V, starts, stream=stream)
    plan.sweep(2, reset_iter=0)  # the second sweep captures the graph
    plan.costs()
    steps = 3
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.sweep(steps, reset_iter=0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1)
    plan.pass_stats()
    plan.enable_pass_timing(True)
    e0.record(stream)
    plan.sweep(steps, reset_iter=0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pass_ms, launches, _, pbytes = plan.pass_stats()
    costs = plan.costs()
    if plan.status() != 0:
        raise RuntimeError("device status reports a non-finite update")
    plan.close()
    peak, peak_kind = measured_peaks()
    avg_s = (pass_ms / 1e3) / max(launches, 1)
    alg = pbytes / max(launches, 1)
    entries = alg / 16  # 8-byte entries, read + write
    tc_tflops = entries * K4_TC_FLOPS_PER_ENTRY / avg_s / 1e12
    tf32_peak, tf32_kind = measured_tf32_peak()
    updates = S * 2 * len(locs) * steps
    return {"metric": "gate-updates/s at 12 qubits, four-qubit gates, complex64",
            "unit": "gate-updates/s", "value": updates / (ms_graph / 1e3),
            "ms_per_sweep": ms_graph / steps, "ms_per_sweep_live": ms / steps,
            "workload": f"12 qubits, {len(locs)} four-qubit gates on consecutive quadruples (6 layers, "
                        "offsets 0/2), 8 starts, reachable Haar target, complex64 tensor, FP64 16x16 update",
            "roofline": {"bound": "hbm", "achieved": alg / avg_s / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / avg_s / 1e9 / peak,
                         "kernel": "pass16tc_kernel (B <- L B R on 16x16 blocks, tcgen05 3xTF32)",
                         "peak_source": peak_kind,
                         "hbm_gbs": alg / avg_s / 1e9, "hbm_frac": alg / avg_s / 1e9 / peak,
                         "tensor": {"achieved_tflops": tc_tflops, "peak_tflops": tf32_peak,
                                    "frac": tc_tflops / tf32_peak if tf32_peak else None,
                                    "peak_source": tf32_kind},
                         "alg_bytes_per_launch": alg, "avg_launch_ms": avg_s * 1e3,
                         "pass_share_of_step": pass_ms / ms if ms > 0 else None},
            "final_costs": [float(c) for c in costs]}


def run_spec(args, qf, torch, dev):
    """Specialised gate set (a trapped-ion native set: GPI and Rz on every
    qubit, Moelmer-Soerensen on brickwork pairs): 12 qubits, 8 starts,
    complex64, one sweep per step; the updates are the closed-form argmax of
    Re Tr(E G(theta)) and one-qubit gates run as G (x) I in a 4x4 slot."""
    n, S = 12, 8
    specs = []
    for layer in range(4):
        specs += [("gpi", q) for q in range(n)]
        specs += [("ms", q, q + 1) for q in range(layer % 2, n - 1, 2)]
    specs += [("rz", q) for q in range(n)]
    p = len(specs)
    gen = qi.rng(SEED + 41)
    # reachable target: the circuit at random angles, multiplied out on the device
    one = qf.Plan(n, specs, 1, qf.QF_C128)
    one.load_params(torch.eye(1 << n, dtype=torch.complex128, device=dev),
                    torch.from_numpy(gen.uniform(-np.pi, np.pi, (1, p, 2))).to(dev))
    slots = qf.spec_slots(specs, n)
    V = qf.circuit_unitary_k(n, slots, one.gates(device=dev)[0].unsqueeze(0), device=dev)
    one.close()
    params = torch.from_numpy(gen.uniform(-np.pi, np.pi, (S, p, 2))).to(dev)
    stream = torch.cuda.current_stream(dev)
    plan = qf.Plan(n, specs, S, qf.QF_C64)
    plan.load_params(V, params, stream=stream)
    plan.sweep(2, reset_iter=0)  # the second sweep captures the graph
    plan.costs()
    steps = 5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.sweep(steps, reset_iter=0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1)
    plan.pass_stats()
    plan.enable_pass_timing(True)
    e0.record(stream)
    plan.sweep(steps, reset_iter=0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pass_ms, launches, _, pbytes = plan.pass_stats()
    costs = plan.costs()
    plan.close()
    peak, peak_kind = measured_peaks()
    avg_s = (pass_ms / 1e3) / max(launches, 1)
    alg = pbytes / max(launches, 1)
    updates = S * 2 * p * steps
    return {"metric": "gate-updates/s at 12 qubits, GPI/Rz/MS gate set, complex64",
            "unit": "gate-updates/s", "value": updates / (ms_graph / 1e3),
            "ms_per_sweep": ms_graph / steps, "ms_per_sweep_live": ms / steps,
            "timing": "value: CUDA-graph replay of each sweep; roofline: live launches with CUDA "
                      "events around every pass",
            "workload": f"12 qubits, {p} gates (4 layers of GPI on every qubit and MS on brickwork "
                        "pairs, then Rz on every qubit), 8 starts, reachable target, complex64 tensor, "
                        "closed-form FP64 updates",
            "roofline": {"bound": "hbm", "achieved": alg / avg_s / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / avg_s / 1e9 / peak, "kernel": "pass kernels (4x4 slots)",
                         "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                         "alg_bytes_per_launch": alg, "avg_launch_ms": avg_s * 1e3,
                         "pass_share_of_step": pass_ms / ms if ms > 0 else None},
            "final_costs": [float(c) for c in costs]}


def config_oracle_costs():
    """The FP64 oracle's final costs on the 3- and 6-qubit workloads, stored
    by tests/golden/make_config_costs.py (read here, not recomputed)."""
    path = os.path.join(ROOT, "tests", "golden", "config_oracle_costs.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def run_configs(args, qf, torch, dev):
    """Correctness and time per sweep of the smaller workloads:
    3-qubit alternating circuit (6 U(4) gates, 1 start, to 1e-10 or 500
    sweeps); 6-qubit brickwork (30 gates, 16 starts) on a Haar-random target
    and on a reachable one, complex128 vs complex64 with FP64 refinement, on
    the plan engine and on the batched kernel; the 8-qubit differentiable
    cost (56 gates, 32 gate sets); the 13-qubit complex64 sweep (72 gates,
    8 starts)."""
    out = {}
    sync = torch.cuda.synchronize

    # 3 qubits, 6 gates alternating on (0,1),(1,2)
    locs = np.array([[0, 1], [1, 2]] * 3, dtype=np.int32)
    inst = qi.make_problem(3, locs, 1, seed=SEED)
    V = qf.circuit_unitary(3, locs, torch.from_numpy(inst.target_gates), device=dev)
    t = time.perf_counter()
    r = qf.instantiate_ex(V, locs, torch.from_numpy(inst.starts).to(dev), dist_tol=1e-10, max_sweeps=500)
    w = time.perf_counter() - t
    gold = config_oracle_costs()
    out["3q_6gates"] = {"cost": r["best_cost"], "sweeps": r["sweeps"], "reason": r["reason"],
                        "ms_per_sweep": 1e3 * w / max(r["sweeps"], 1), "path": "qf_instantiate_ex, complex128",
                        "oracle": gold.get("3q_6gates", {}).get("start0")}

    # 6 qubits, brickwork of 30 gates, 16 starts
    locs = qi.brickwork_locations(6, 12)
    inst = qi.make_problem(6, locs, 16, seed=SEED)
    Vr = qf.circuit_unitary(6, locs, torch.from_numpy(inst.target_gates), device=dev)
    Vh = torch.from_numpy(qi.haar_unitary(64, qi.rng(SEED))).to(dev)
    starts = torch.from_numpy(inst.starts).to(dev)
    rows = {}
    for tname, V in (("haar", Vh), ("reachable", Vr)):
        for pname, prec in (("c128", qf.QF_C128), ("c64_refine64", qf.QF_C64_REFINE64)):
            t = time.perf_counter()
            r = qf.instantiate_ex(V, locs, starts, dist_tol=1e-10, max_sweeps=500, precision=prec)
            w = time.perf_counter() - t
            t = time.perf_counter()
            rb = qf.instantiate_batched([(V.cpu().numpy(), locs, inst.starts)], dist_tol=1e-10,
                                        max_sweeps=500, precision=prec)
            wb = time.perf_counter() - t
            rows[f"{tname}/{pname}"] = {
                "engine": {"best_cost": r["best_cost"], "sweeps": r["sweeps"], "c64_sweeps": r["c64_sweeps"],
                           "reason": r["reason"], "s": w, "ms_per_sweep": 1e3 * w / max(r["sweeps"], 1)},
                "batched": {"best_cost": float(rb["costs"][0].min()), "max_sweeps": int(rb["sweeps"].max()),
                            "s": wb, "kernel_ms": rb["kernel_ms"]}}
    # starts 0 and 1 alone, next to the oracle's final cost for the same start
    per_start = {}
    for tname, V in (("haar", Vh), ("reachable", Vr)):
        for st in (0, 1):
            r = qf.instantiate_ex(V, locs, starts[st:st + 1], dist_tol=1e-10, max_sweeps=500,
                                  precision=qf.QF_C128)
            per_start[f"{tname}/start{st}"] = {
                "gpu_c128": {"cost": r["best_cost"], "sweeps": r["sweeps"]},
                "oracle": gold.get("6q_30gates", {}).get(tname, {}).get(f"start{st}")}
    rows["per_start_vs_oracle"] = per_start
    out["6q_30gates_16starts"] = rows

    # 8 qubits, 56 gates, 32 gate sets: differentiable cost (forward + backward)
    locs = qi.brickwork_locations(8, 16)
    g = qi.rng(SEED)
    gates = torch.from_numpy(np.stack([qi.haar_gates(len(locs), g) for _ in range(32)])).to(dev)
    V = torch.from_numpy(qi.haar_unitary(256, g)).to(dev)
    x = gates.clone().requires_grad_(True)
    qf.QFactorCost.apply(x, V, locs).sum().backward()
    sync()
    t = time.perf_counter()
    reps = 5
    for _ in range(reps):
        x.grad = None
        qf.QFactorCost.apply(x, V, locs).sum().backward()
    sync()
    out["8q_56gates_32sets_grad"] = {"ms_per_forward_backward": 1e3 * (time.perf_counter() - t) / reps,
                                     "gradients_per_call": 32 * len(locs)}

    # 13 qubits, 72 gates, 8 starts, complex64
    locs = qi.brickwork_locations(13, LAYERS)
    inst = qi.make_problem(13, locs, 8, seed=SEED)
    V = qf.circuit_unitary(13, locs, torch.from_numpy(inst.target_gates), device=dev)
    plan = qf.Plan(13, locs, 8, qf.QF_C64)
    stream = torch.cuda.current_stream(dev)
    plan.load(V, torch.from_numpy(inst.starts).to(dev), stream=stream)
    plan.sweep(1, reset_iter=0)
    plan.costs()
    plan.pass_stats()
    plan.enable_pass_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.sweep(2, reset_iter=0)
    e1.record(stream)
    sync()
    ms = e0.elapsed_time(e1)
    pass_ms, launches, _, pbytes = plan.pass_stats()
    plan.close()
    alg = pbytes / max(launches, 1)
    peak, _ = measured_peaks()
    gbs = alg / ((pass_ms / 1e3) / max(launches, 1)) / 1e9
    out["13q_72gates_8starts_c64"] = {"value": 8 * 2 * len(locs) * 2 / (ms / 1e3), "unit": "gate-updates/s",
                                      "pass_gbs": gbs, "frac": gbs / peak, "ms_per_sweep": ms / 2}
    return out


# ------------------------------------------------------------------ our arm


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2306_08152_gb300 as qf

    qf._native.load()
    inst = workload(args.qubits, args.starts)
    n, locs = inst.n, inst.locs
    # replicas: rank r runs its own seeded starts (seed offset by rank)
    if rank > 0:
        inst = qi.make_problem(n, locs, args.starts, seed=replica_seed(rank))
    prec = qf.QF_C64 if args.precision == "c64" else qf.QF_C128
    stream = torch.cuda.current_stream(dev)
    V = qf.circuit_unitary(n, locs, torch.from_numpy(inst.target_gates), device=dev)
    starts = torch.from_numpy(inst.starts).to(dev)
    plan = qf.Plan(n, locs, inst.n_starts, prec)
    plan.load(V, starts, stream=stream)
    for _ in range(args.warmup):
        plan.sweep(1, reset_iter=40)
    # untimed sweeps up to the next rebuild sweep: the first timed sweep is
    # a multiple of RESET_ITER, so every RESET_ITER timed sweeps hold one
    # re-unitarisation and rebuild
    align = (RESET_ITER - 1 - args.warmup) % RESET_ITER
    for _ in range(align):
        plan.sweep(1, reset_iter=RESET_ITER)
    first_timed = args.warmup + align + 1
    rebuilds_timed = sum(1 for k in range(first_timed, first_timed + args.steps) if k % RESET_ITER == 0)
    plan.costs()
    plan.pass_stats()  # reset counters

    # the timed steps: each sweep replays the plan's captured CUDA graph (the
    # production path of qf_plan_sweep); inputs stay resident in HBM
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.sweep(1, reset_iter=RESET_ITER)
    e1.record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    ms = e0.elapsed_time(e1)
    _, _, all_launches, _ = plan.pass_stats()
    # the same steps as live launches with CUDA events around every pass, for
    # the per-launch roofline
    plan.enable_pass_timing(True)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        plan.sweep(1, reset_iter=40)
    g1.record(stream)
    torch.cuda.synchronize()
    ms_live = g0.elapsed_time(g1) / args.steps
    pass_ms, pass_launches, _, pass_bytes = plan.pass_stats()
    plan.enable_pass_timing(False)
    if plan.status() != 0:
        raise RuntimeError("device status reports a non-finite update")
    costs = plan.costs()
    ms = max_over_ranks(ms, dist, dev)
    updates_per_step = inst.n_starts * 2 * inst.p * world
    value = job_throughput(inst.n_starts * 2 * inst.p, world, args.steps, ms)

    # roofline of the dominant kernel (the fused pass): algorithmic bytes of
    # every timed pass launch (one read + one write of the tensors it covers)
    # over the summed launch durations
    eb = 8 if args.precision == "c64" else 16
    alg_bytes = pass_bytes / max(pass_launches, 1)
    avg_pass_s = (pass_ms / 1e3) / max(pass_launches, 1)
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / avg_pass_s / 1e9
    traffic = kernel_traffic(args.precision, inst.n_starts, n)
    if traffic is not None:
        traffic *= alg_bytes / (inst.n_starts * 4**n * 2 * eb)  # per launch of this size
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "pass kernels (fused B <- L B R over every 4x4 block)",
                "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_pass_s * 1e3,
                "pass_launches": pass_launches,
                "pass_share_of_step": (pass_ms / (ms_live * args.steps)) if ms_live > 0 else None}
    if args.precision == "c128":
        fp64_peak = 1250.0  # GFLOP/s nominal FP64 (no measured FP64 peak on this machine)
        flops = alg_bytes / (2 * eb) * 64
        roofline_fp64 = flops / avg_pass_s / 1e9
        roofline = {"bound": "alu", "achieved": roofline_fp64, "peak": fp64_peak, "unit": "GFLOP/s",
                    "frac": roofline_fp64 / fp64_peak, "traffic": traffic,
                    "kernel": roofline["kernel"],
                    "peak_source": "nominal FP64 1.25 TFLOP/s (64 FP64 flops per entry)",
                    "hbm_gbs": achieved, "hbm_frac": achieved / peak, "avg_launch_ms": avg_pass_s * 1e3}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        V_h = V.cpu().pin_memory()
        starts_h = starts.cpu().pin_memory()
        opts = qf.Options(dist_tol=0.0, max_sweeps=1,
                          precision=qf.QF_C64 if args.precision == "c64" else qf.QF_C128)
        e2e_steps = max(1, min(args.steps, 10))
        qf.instantiate_ex(V_h, locs, starts_h, options=opts, stream=stream)  # warm-up
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            r = qf.instantiate_ex(V_h, locs, starts_h, options=opts, stream=stream)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, dist, dev)
        h2d = V_h.numel() * 16 + starts_h.numel() * 16 + locs.size * 4
        d2h = starts_h.numel() * 16 + inst.n_starts * 8
        e2e = {"value": updates_per_step * e2e_steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": e2e_steps,
               "call": "qf_instantiate_ex(host target, host starts, max_sweeps=1): "
                       "allocation, H2D, InitCircuitTensor, one sweep, D2H"}
        del r

    kqubit = k4 = None
    if not args.no_kqubit and world == 1:
        kqubit = run_kqubit(args, qf, torch, dev)
        k4 = run_k4(args, qf, torch, dev)
    spec = None
    if not args.no_spec and world == 1:
        spec = run_spec(args, qf, torch, dev)
    lookahead = None
    if not args.no_lookahead and args.precision == "c64" and n >= 8 and world == 1:
        lookahead = run_lookahead(args, qf, torch, dev, inst, V, starts, costs)
    extra_c128 = extra_df64 = None
    if not args.no_c128 and args.precision == "c64" and world == 1:
        extra_c128 = run_c128(args, qf, torch, dev, inst, V, starts)
        extra_df64 = run_df64(args, qf, torch, dev, inst, V, starts)
    batched = None
    if not args.no_batched and world == 1:
        batched = run_batched(args, qf, torch, dev)
        batched["mixed_2_3_qubit"] = run_batched_k(args, qf, torch, dev)
    configs = None
    if not args.no_configs and world == 1:
        configs = run_configs(args, qf, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        (done, wall, cput), T0 = oracle_sample(inst, args.cpu_seconds)
        one = oracle_single_core(inst, T0, args.cpu_seconds)
        del T0
        single = ({"value": one["updates"] / one["wall_s"], "unit": UNIT, "cores": 1,
                   "sample": f"{one['updates']} gate updates, {one['wall_s']:.1f} s wall, one process "
                             f"pinned to core {one['core']} with one BLAS/OpenMP thread"}
                  if "updates" in one else one)
        cpu = {"value": done / wall, "unit": UNIT, "cores": round(cput / wall, 2), "kind": "oracle",
               "sample": f"{done} gate updates (ApplyRight, CalcEnvMat, OptimizeGate, ApplyLeft) "
                         f"of the FP64 NumPy oracle on start 0 of the same {n}-qubit workload, "
                         f"{wall:.1f} s wall; cores = CPU time / wall time",
               "single_core": single, "nproc": os.cpu_count(),
               "cores_available": len(os.sched_getaffinity(0))}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c64" if args.precision == "c64" else "c128",
            "data": "synthetic", "config": dict(config_dict(args, inst),
                                                rebuilds_in_timed_region=rebuilds_timed,
                                                first_timed_sweep=first_timed),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(all_launches), "clocks": clock_info,
            "ms_per_step_live": ms_live,
            "timing": "value: CUDA-graph replay of each sweep (qf_plan_sweep); roofline: the same "
                      "sweeps as live launches with CUDA events around every pass",
            "lookahead": lookahead, "kqubit": kqubit, "k4": k4, "spec": spec, "c128": extra_c128, "df64": extra_df64, "batched": batched, "configs": configs,
            "final_costs": [float(c) for c in costs],
        }
        print(json.dumps(line))
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """A small case of one kernel family for ncu captures: 12 qubits, 2
    starts (the tensors, 268 MB in complex64, exceed L2), complex64, a
    warm-up sweep and one live sweep (no graph).  k4: four-qubit gates on
    consecutive quadruples (pass16c_kernel, env16_kernel); k3: three-qubit
    gates on consecutive triples (pass8a/pass8c/pass8f kernels); pair: the
    look-ahead brickwork (pass_pair_kernel); pass: the plain brickwork
    (pass_block/window/lane kernels)."""
    import torch

    import paper_2306_08152_gb300 as qf

    qf._native.load()
    dev = torch.device("cuda", 0)
    if args.profile_case == "batched":
        # the first 512 instances of the benchmark's uneven batch: a warm-up
        # call (autotuning: 4 trial launches, then its run), then one run
        insts = qi.batched_instances(4096, 4, seed=SEED)[:512]
        probs = [(qf.circuit_unitary(i.n, i.locs, torch.from_numpy(i.target_gates), device=dev).cpu().numpy(),
                  i.locs, i.starts) for i in insts]
        opts = dict(dist_tol=1e-10, max_sweeps=500, precision=qf.QF_C64_REFINE64)
        qf.instantiate_batched(probs, **opts)
        res = qf.instantiate_batched(probs, **opts)
        best = res["costs"].min(axis=1)
        print(json.dumps({"case": "batched", "instances": len(probs), "kernel_ms": res["kernel_ms"],
                          "success": int((best <= 1e-10).sum()), "warps_per_cta": res["warps_per_cta"],
                          "sweeps": res["total_sweeps"]}))
        return 0
    if args.profile_case == "batched_k":
        # the first 256 instances of the benchmark's batch of 2- and 3-qubit
        # circuits: a warm-up call (autotuning: 4 trial launches, then its
        # run), then one run
        insts = qi.batched_instances_k(1024, 4, seed=SEED + 9)[:256]
        probs = [(qf.circuit_unitary_k(i.n, i.locs, i.target_gates, device=dev).cpu().numpy(), i.locs, i.starts)
                 for i in insts]
        opts = dict(dist_tol=1e-10, max_sweeps=500, precision=qf.QF_C64_REFINE64)
        qf.instantiate_batched_k(probs, **opts)
        res = qf.instantiate_batched_k(probs, **opts)
        best = res["costs"].min(axis=1)
        print(json.dumps({"case": "batched_k", "instances": len(probs), "kernel_ms": res["kernel_ms"],
                          "success": int((best <= 1e-10).sum()), "warps_per_cta": res["warps_per_cta"],
                          "sweeps": res["total_sweeps"]}))
        return 0
    n, S = 12, 2
    if args.profile_case == "k4":
        locs = []
        for layer in range(6):
            o = 0 if layer % 2 == 0 else 2
            locs += [(q, q + 1, q + 2, q + 3) for q in range(o, n - 3, 4)]
    elif args.profile_case == "k3":
        locs = []
        for layer in range(6):
            o = layer % 3
            locs += [(q, q + 1, q + 2) for q in range(o, n - 2, 3)]
    else:
        locs = [tuple(int(x) for x in q) for q in qi.brickwork_locations(n, LAYERS)]
    gen = qi.rng(SEED + 55)
    tgt = [qi.haar_unitary(2 ** len(q), gen) for q in locs]
    V = qf.circuit_unitary_k(n, locs, tgt, device=dev)
    starts = qf.flatten_gates([[qi.haar_unitary(2 ** len(q), qi.rng(SEED + 56 + s)) for q in locs]
                               for s in range(S)]).to(dev)
    plan = qf.Plan(n, locs, S, qf.QF_C64)
    if args.profile_case == "pair":
        plan.set_lookahead(True)
    plan.enable_pass_timing(True)  # live launches
    plan.load(V, starts)
    plan.sweep(1, reset_iter=0)
    plan.pass_stats()
    plan.sweep(1, reset_iter=0)
    ms, launches, all_launches, pbytes = plan.pass_stats()
    costs = plan.costs()
    plan.close()
    print(json.dumps({"case": args.profile_case, "n_qubits": n, "starts": S, "gates": len(locs),
                      "pass_ms": ms, "pass_launches": launches, "launches": all_launches,
                      "pass_gbs": pbytes / (ms / 1e3) / 1e9 if ms > 0 else None,
                      "costs": [float(c) for c in costs]}))
    return 0


def main():
    args = parse()
    if args.oracle_1core:
        return run_oracle_1core(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
