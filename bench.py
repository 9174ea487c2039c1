"""Benchmark: 30-qubit layered-circuit throughput (gates/s) and HBM roofline.

One step = one pass of the hot path over the single-large-state workload:
|0...0> initialisation of the 2^n complex64 state, 500 gates of alternating
U3-on-every-qubit / CZ-even / CZ-odd layers (seeded angles), the paper's QFT
command sequence on all n qubits (H, CPHASE pi/2^(i+1), SWAPs), then sampling the
output by measuring all n qubits in order with seeded uniforms (the outcome is
read back).  gates/s counts the 500 + QFT gate commands (980 at n = 30).

JSON line keys follow the harness contract; ``value`` is timed on the device with
CUDA events on the engine's stream, ``e2e`` through the public API from the host
(gate descriptors in, measured outcome out), ``roofline`` for the kernel class with
the largest share of device time, ``cpu_baseline`` the complex128 CPU oracle on a
bounded sample of the same circuit.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--n 30] [--mode fused|plain]
       python bench.py --impl reference ...   (the CPU oracle arm)
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from paper_1908_07187_gb300 import shor  # noqa: E402

METRIC = "30-qubit gates/s & % HBM peak; served circuits/s + p99 vs plain, TV err<=1e-5"
UNIT = "gates/s"
FALLBACK_HBM_GBS = 6800.0


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (the whole job is as
    slow as its slowest replica); the values themselves on one rank."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(units_per_step: int, steps: int, world: int, seconds: float) -> float:
    """Units processed by all ranks (each rank runs its own replica of the step)
    divided by the slowest rank's time."""
    return world * units_per_step * steps / seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--mode", default="fused", choices=["fused", "plain"])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-pass-per-gate comparison")
    ap.add_argument("--no-kitaev", action="store_true", help="skip the Kitaev order-finding measurement")
    ap.add_argument("--no-3nx1", dest="no_3nx1", action="store_true", help="skip the conventional (3nx1) order-finding run")
    ap.add_argument("--no-33q", dest="no_33q", action="store_true", help="skip the 33-qubit run of the layered workload")
    ap.add_argument("--no-block", action="store_true", help="skip the dense 5-qubit block measurement")
    ap.add_argument("--no-precision", action="store_true", help="skip the complex64-vs-complex128 precision check")
    ap.add_argument("--batch-circuits", type=int, default=4096, help="circuits in the batched measurement (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=1000, help="requests in the serving measurement (0: skip)")
    return ap.parse_args()


def workload(n: int, seed: int):
    return workloads.layered_circuit(n, seed=seed, n_gates=500, qft=True, measure=n)


def gate_ops(circ):
    return [op for op in circ.ops if op.kind != "measure"]


DIAGONAL = {"z", "s", "sdg", "t", "tdg", "p", "rz"}


def tile_fp32_ops(ops, n: int, tile_launches: float) -> float:
    """FP32 lane operations the fused tile passes execute for a gate list (an
    FMA counts as one): an uncontrolled non-diagonal 1-qubit gate is a pivot-form
    butterfly, 8 FMAs per amplitude pair; a
    controlled one a full complex 2x2 product on the pairs where the controls
    hold, 16 per pair; diagonal gates are folded into pending phases (no
    per-gate arithmetic); each pass ends with one complex factor per amplitude
    (4 operations).  Flushes at transposes are left out (sign flips are integer
    work; general phase flushes occur only in the QFT passes), so this is a
    lower bound."""
    f = 0.0
    for op in ops:
        if op.kind == "swap" or op.kind in DIAGONAL:
            continue
        c = len(op.controls)
        f += (8.0 if c == 0 else 16.0) * 2.0 ** (n - c - 1)
    return f + 4.0 * 2.0 ** n * tile_launches


def fp32_lane_peak(sm_count: int, sm_mhz: float) -> float:
    """FP32 lane operations per second: SMs x 128 FP32 lanes x clock (the packed
    f32x2 forms issue at the same lane rate, measured)."""
    return sm_count * 128 * sm_mhz * 1e6


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources that decide each kernel class's memory traffic
KERNEL_SOURCES = {"tile": ("kernels_tile.cu", "qk_kernels.cuh", "qk_plan.cu")}


_C_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|//[^\n]*|/\*.*?\*/', re.S)


def code_only(src: str) -> str:
    """C/C++/CUDA source without comments, whitespace runs collapsed: what the
    compiler sees, so that editing a comment does not read as a kernel change."""
    out = _C_TOKENS.sub(lambda m: m.group(0) if m.group(0)[0] in "\"'" else " ", src)
    return " ".join(out.split())


def kernel_source_sha(kernel_class: str = "tile"):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1908_07187_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel_class, sorted(os.listdir(csrc))):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, f), encoding="utf-8") as fh:
                h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_class: str, n: int):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        rec = d.get(f"{kernel_class}_n{n}")
        if rec and rec.get("src_sha") == kernel_source_sha(kernel_class):
            return float(rec["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
def host_mem_gib():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable"):
                    return int(line.split()[1]) / 2 ** 20
    except Exception:
        pass
    return 0.0


def oracle_size(n: int):
    """Largest qubit count <= n whose complex128 state fits comfortably in host RAM."""
    m = n
    while m > 20 and host_mem_gib() < (16 << m) / 2 ** 30 * 1.3:
        m -= 1
    return m


# CPU part numbers of Arm cores (MIDR part field), for hosts whose lscpu is missing
ARM_PARTS = {"0xd0c": "Neoverse-N1", "0xd40": "Neoverse-V1", "0xd49": "Neoverse-N2", "0xd4f": "Neoverse-V2",
             "0xd8e": "Neoverse-N3", "0xd84": "Neoverse-V3"}


def host_info():
    """The host the oracle is timed on: logical CPUs and the CPU model (lscpu's
    model name, else /proc/cpuinfo's model name or Arm CPU part)."""
    import platform

    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    part = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":", 1)[0].strip().lower()
                if not model and key == "model name":
                    model = line.split(":", 1)[1].strip()
                if key == "cpu part" and not part:
                    part = line.split(":", 1)[1].strip().lower()
    except OSError:
        pass
    if not model and part:
        model = ARM_PARTS.get(part, f"Arm CPU part {part}")
    return {"nproc": os.cpu_count(), "cpu": model or platform.machine(), "arch": platform.machine()}


def oracle_gate_rate(m: int, circ, first: int, count: int, openmp: bool, budget_s: float = 1e9):
    """Time the complex128 oracle on gate ops first..first+count-1 of an m-qubit
    workload circuit (gate op 0 applied untimed, which also touches every page of
    the state), stopping early once budget_s has passed.  Returns (gates, s)."""
    import oracle

    st = oracle.OracleState(m, openmp=openmp)
    ops = gate_ops(circ)
    st.apply_op(ops[0])
    t0 = time.perf_counter()
    done = 0
    for op in ops[first:first + count]:
        st.apply_op(op)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0


def cpu_baseline(n: int, circ):
    """The oracle as it stands on the host: one thread on 20 gates of the
    layered circuit at min(n, 26) qubits (per-gate cost scales with 2^n, so the
    rate is scaled to n), and the all-core build on the n-qubit state (or the
    largest that fits in host RAM) for up to about 10 s of gates."""
    hi = host_info()
    m1 = min(n, 26)
    g1, t1 = oracle_gate_rate(m1, workload(m1, 2), 1, 20, openmp=False)
    single = g1 / t1 * 2.0 ** (m1 - n)
    m2 = oracle_size(n)
    g2, t2 = oracle_gate_rate(m2, circ if m2 == n else workload(m2, 2), 1, 200, openmp=True, budget_s=10.0)
    allc = g2 / t2 * 2.0 ** (m2 - n)
    sample = (f"gate ops 2..{g2 + 1} of the {m2}-qubit layered circuit (gate 1 untimed) on the complex128 oracle's "
              f"all-core build, {hi['nproc']} threads, {t2:.1f} s")
    if m2 != n:
        sample += f", scaled by 2^{m2 - n} to {n} qubits"
    return {"value": allc, "unit": UNIT, "cores": hi["nproc"], "kind": "oracle", "sample": sample,
            "single_thread": {"value": single, "unit": UNIT, "cores": 1, "ms_per_gate_at_n": 1000.0 / single,
                              "sample": f"gate ops 2..21 of the {m1}-qubit layered circuit, 1 thread, {t1:.1f} s"
                                        + (f", scaled by 2^{m1 - n} to {n} qubits" if m1 != n else "")},
            "host": hi}


def run_reference(args):
    """The CPU oracle arm: the complex128 oracle (all-core build) on the host,
    each step two gate ops of the n-qubit layered circuit (or of the largest
    that fits in host RAM, scaled by the state size), timed as run."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    hi = host_info()
    n = args.n
    m = oracle_size(n)
    circ = workload(m, 2)
    ops = gate_ops(circ)
    st = oracle.OracleState(m, openmp=True)
    st.apply_op(ops[0])             # untimed: touches every page
    per_step = 2
    ms, pos = [], 1
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for op in ops[pos:pos + per_step]:
            st.apply_op(op)
        dt = time.perf_counter() - t0
        pos += per_step
        if s >= args.warmup:
            ms.append(1000.0 * dt)
    ms_step = statistics.median(ms)
    value = per_step / (ms_step / 1000.0) * 2.0 ** (m - n)
    sample = f"{per_step} gate ops per step of the {m}-qubit layered circuit on the complex128 oracle, {hi['nproc']} threads"
    if m != n:
        sample += f", rate scaled by 2^{m - n} to {n} qubits (ms_per_step is as timed at {m} qubits)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": f"layered U3/CZ-brickwork 500 gates + QFT({n}) + measure all, {n} qubits",
                       "n_qubits": n, "gate_ops_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": hi["nproc"], "kind": "oracle", "sample": sample,
                             "host": hi},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def layered_33q_measurement(qk, torch, stream, n: int = 33, steps: int = 2):
    """The metric's workload at its largest configuration: the same layered
    U3/CZ + QFT + measure-all step at 33 qubits (64 GiB of complex64), device
    time with CUDA events over `steps` steps after one warm-up step."""
    circ = workload(n, 2)
    gops = gate_ops(circ)
    meas = [op for op in circ.ops if op.kind == "measure"]
    ctx = qk.Context("c64", "fused", stream=stream.cuda_stream, profile=True)
    ctx.add_qubits(n)
    ctx.add_cbits(circ.n_cbits)

    def step():
        ctx.reset()
        qk.run_ops(ctx, gops)
        for op in meas:
            ctx.measure(op.targets, op.uniforms, op.cbits, wait=False)
        ctx.flush()

    step()
    ctx.sync()
    ctx.profile()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = ctx.profile()
    ctx.close()
    tile = prof.get("tile", {"launches": 0, "ms": 0.0})
    return {"n_qubits": n, "gates_per_step": len(gops), "ms_per_step": round(ms, 3),
            "gates_per_s": round(len(gops) / (ms / 1000.0), 1),
            "tile_passes_per_step": tile["launches"] / steps,
            "tile_ms_per_step": round(tile["ms"] / steps, 3),
            "state_bytes": 8 << n}


def shor_3nx1_measurement(qk, torch, stream, b: int = 11, reps: int = 2):
    """The conventional order-finding circuit (3nx1 branch of Appendix A) for a
    seeded b-bit N: t = bit_length(N^2 - 1) control qubits and b work qubits (33
    qubits at b = 11), H on the controls, t controlled mul-mod gathers, the work
    register measured, the QFT sequence, the control register measured.  Device
    time of the whole run with CUDA events, then the order and factors from the
    control register's value by continued fractions."""
    N, a = workloads.kitaev_parameters(b, seed=4)
    circ = workloads.shor_3nx1_circuit(N, a, seed=3)
    t = circ.n_qubits - N.bit_length()
    res = {"b": b, "N": N, "a": a, "qubits": circ.n_qubits, "control_qubits": t,
           "gate_ops": circ.gate_count(), "state_bytes": 8 << circ.n_qubits}
    ctx = qk.Context("c64", "fused", stream=stream.cuda_stream)
    ctx.add_qubits(circ.n_qubits)
    ctx.add_cbits(circ.n_cbits)
    qk.run_ops(ctx, circ.ops)            # defines the gates, allocates the gather buffer
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.reset()
        qk.run_ops(ctx, circ.ops)
    e1.record(stream)
    torch.cuda.synchronize()
    res["ms_per_run"] = round(e0.elapsed_time(e1) / reps, 3)
    bits = [int(x) for x in ctx.read_cbits()]
    ctx.close()
    res["work_value"] = shor.register_from_bits(bits[:N.bit_length()])
    res["y"] = shor.register_from_bits(bits[N.bit_length():])
    r = shor.order_from_outcome(res["y"], t, a, N)
    res["order"] = r
    res["factors"] = shor.factors_from_order(a, r, N) if r else None
    res["paper_context"] = "the paper runs 3nx1 for N = 8189 (39 qubits) on a desktop (Fig. 5); 39 qubits need 4 TiB of complex64, beyond one GPU"
    return res


# ---------------------------------------------------------------------------
# dense 5-qubit block (secondary measurement)
# ---------------------------------------------------------------------------
def block_measurement(qk, torch, stream, n: int, reps: int = 10, k: int = 5):
    """One dense k-qubit unitary on the lowest qubits of an n-qubit complex64
    state, tensor cores (3xTF32; k < 5 as the 5-qubit block U (x) I) vs CUDA
    cores; device time per pass with CUDA events.  Flops count the k-qubit
    product (2^(n-k) groups x (2^(k+1))^2 x 2)."""
    import numpy as np

    d = 1 << k
    g = np.random.Generator(np.random.PCG64(5))
    z = (g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    U = q * (np.diag(r) / np.abs(np.diag(r)))
    low = list(range(k - 1, -1, -1))
    other = list(range(10 + k - 1, 9, -1))
    out = {"n": n, "k": k, "alg_bytes_per_pass": 2 * 8 * 2 ** n,
           "alg_flops_per_pass": 2 ** (n - k) * (2 * d) * (2 * d) * 2}
    for tc in (True, False):
        ctx = qk.Context("c64", "plain", stream=stream.cuda_stream, tensor_cores=tc)
        ctx.add_qubits(n)
        gid = ctx.define_gate_matrix(U)
        ctx.apply_gate("h", [0])
        for _ in range(2):
            ctx.apply_gate(gid, low)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.apply_gate(gid, low)
        e1.record(stream)
        ctx.sync()
        ms = e0.elapsed_time(e1) / reps
        key = "tensor_core" if tc else "cuda_core"
        out[key] = {"ms_per_pass": round(ms, 4), "GBps": round(out["alg_bytes_per_pass"] / ms / 1e6, 1),
                    "TFLOPs": round(out["alg_flops_per_pass"] / ms / 1e9, 2)}
        if tc:
            # blocks alternating between the lowest qubits and qubits 10..: every
            # application first gathers its targets onto the lowest physical qubits
            groups = (low, other)
            for g in groups:
                ctx.apply_gate(gid, g)
            ctx.sync()
            e0.record(stream)
            for r in range(reps):
                ctx.apply_gate(gid, groups[r % 2])
            e1.record(stream)
            ctx.sync()
            ms = e0.elapsed_time(e1) / reps
            out["tensor_core_any_qubits"] = {"ms_per_gate": round(ms, 4),
                                             "note": "one relabelling gather + one tensor-core pass per gate"}
        ctx.close()
    return out


# ---------------------------------------------------------------------------
# Kitaev order finding (secondary measurement)
# ---------------------------------------------------------------------------
def kitaev_measurement(qk, torch, stream, b: int = 20, reps: int = 5):
    """Time one whole order-finding run (t = 2b stages) on a seeded b-bit N:
    the generic op sequence in fused mode and the fused-stage entry point.
    Device time with CUDA events; measured bits must agree."""
    N, a = workloads.kitaev_parameters(b, seed=3)
    circ = workloads.kitaev_circuit(N, a, seed=5)
    res = {"b": b, "N": N, "a": a, "qubits": circ.n_qubits, "stages": circ.n_cbits}
    bits = {}
    for name, runner in (("generic", lambda c: qk.run_ops(c, circ.ops)), ("fused_stage", lambda c: qk.run_kitaev_fused(c, circ))):
        ctx = qk.Context("c64", "fused", stream=stream.cuda_stream)
        ctx.add_qubits(circ.n_qubits)
        ctx.add_cbits(circ.n_cbits)
        for _ in range(2):
            ctx.reset()
            runner(ctx)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.reset()
            runner(ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        res[f"ms_per_run_{name}"] = round(e0.elapsed_time(e1) / reps, 4)
        bits[name] = [int(x) for x in ctx.read_cbits()]
        ctx.close()
    # the fused-stage run captured once into a CUDA graph and replayed
    ctx = qk.Context("c64", "fused", stream=stream.cuda_stream)
    ctx.add_qubits(circ.n_qubits)
    ctx.add_cbits(circ.n_cbits)
    qk.run_kitaev_fused(ctx, circ)
    ctx.sync()
    ctx.capture_begin()
    ctx.reset()
    qk.run_kitaev_fused(ctx, circ)
    graph = ctx.capture_end()
    for _ in range(2):
        graph.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.launch()
    e1.record(stream)
    torch.cuda.synchronize()
    res["ms_per_run_graph"] = round(e0.elapsed_time(e1) / reps, 4)
    bits["graph"] = [int(x) for x in ctx.read_cbits()]
    graph.close()
    ctx.close()
    res["bits_match"] = bits["generic"] == bits["fused_stage"] == bits["graph"]
    res["y"] = shor.outcome_from_bits(bits["fused_stage"])
    # the paper's classical step: continued fractions of y / 2^t, then gcds
    r = shor.order_from_outcome(res["y"], circ.n_cbits, a, N)
    res["order"] = r
    res["factors"] = shor.factors_from_order(a, r, N) if r else None
    res["paper_context"] = "21-qubit Kitaev run of the 20-bit N = 961307 took 139 s on one i5-7400T core (Abstract)"
    return res


# ---------------------------------------------------------------------------
# batched uneven small circuits (secondary measurement)
# ---------------------------------------------------------------------------
def _wait_batch(b):
    while not b.done():
        time.sleep(0.0005)


def batch_measurement(qk, torch, stream, count: int = 4096, seq_every: int = 16, oracle_per_n: int = 3):
    """The batched configuration: `count` independent U3 + CZ layer circuits of
    10..20 qubits (uniform) and 50..300 layers.  Circuits of at most 13 qubits run
    whole in shared memory; 14..20-qubit circuits as batched tile passes (states
    in HBM, pass k of every circuit in one launch).  Measured two ways, as the
    one-circuit-per-context path beside it: end to end (wall time from the gate
    lists to the finished run: marshalling, host planning, upload, device) and
    device time.  The per-context path runs every `seq_every`-th circuit on its
    own fused context fed by one bulk gate-list call, scaled to `count`.  Final
    states of the `oracle_per_n` shallowest circuits of each size are compared
    with the complex128 oracle (all-core build)."""
    import numpy as np
    import oracle

    specs = [workloads.batch_layer_spec(i) for i in range(count)]
    lists = [qk.layer_gate_ops(*sp) for sp in specs]
    gates = int(sum(len(x) for x in lists))
    b = qk.Batch(stream=stream.cuda_stream)

    def fill():
        for sp, ops in zip(specs, lists):
            b.add_circuit(sp[0], 0)
            b.apply_gates(ops)

    fill()
    b.run(store_states=True)                      # warm-up: allocations
    _wait_batch(b)
    b.clear()
    t0 = time.perf_counter()
    fill()
    t_fill = time.perf_counter() - t0
    b.run(store_states=True)
    _wait_batch(b)
    t_e2e = time.perf_counter() - t0
    st = b.stats()
    dev_ms = st["device_ms"]
    # the oracle on the shallowest circuits of each size
    by_n = {}
    for i, (n, depth, _) in enumerate(specs):
        by_n.setdefault(n, []).append((depth, i))
    pick = [i for n in sorted(by_n) for _, i in sorted(by_n[n])[:oracle_per_n]]
    tv_max, mx_max, t_or = 0.0, 0.0, time.perf_counter()
    for i in pick:
        n, depth, ang = specs[i]
        ref = oracle.OracleState(n, openmp=True)
        for op in workloads.layer_spec_circuit(n, depth, ang).ops:
            ref.apply_op(op)
        got = b.read(i)[1].astype(np.complex128)
        tv_max = max(tv_max, 0.5 * float(np.abs(np.abs(got) ** 2 - np.abs(ref.psi) ** 2).sum()))
        mx_max = max(mx_max, float(np.abs(got - ref.psi).max()))
    t_or = time.perf_counter() - t_or
    b.close()
    # one circuit per context (fused engine), bulk gate list, every seq_every-th circuit
    sel = list(range(0, count, seq_every))
    ctxs = []
    for i in sel:
        ctx = qk.Context("c64", "fused", stream=stream.cuda_stream)
        ctx.add_qubits(specs[i][0])
        ctxs.append(ctx)
    for ctx, i in zip(ctxs[:8], sel[:8]):         # warm-up
        ctx.apply_gates(lists[i])
        ctx.flush()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t1 = time.perf_counter()
    p0.record(stream)
    for ctx, i in zip(ctxs, sel):
        ctx.reset()
        ctx.apply_gates(lists[i])
        ctx.flush()
    p1.record(stream)
    torch.cuda.synchronize()
    seq_wall = time.perf_counter() - t1
    seq_dev = p0.elapsed_time(p1)
    for ctx in ctxs:
        ctx.close()
    scale = count / len(sel)
    n_large = sum(1 for sp in specs if sp[0] > qk.Batch.SMEM_QUBITS)
    return {"circuits": count, "qubits": "10..20 (uniform)", "layers": "50..300 (uniform)", "gates": gates,
            "large_circuits": n_large,
            "batched": {"e2e_s": round(t_e2e, 3), "e2e_circuits_per_s": round(count / t_e2e, 1),
                        "device_ms": round(dev_ms, 2), "device_circuits_per_s": round(count / (dev_ms / 1000.0), 1),
                        "device_gates_per_s": round(gates / (dev_ms / 1000.0), 1),
                        "host_fill_s": round(t_fill, 3), "host_plan_ms": round(st["plan_ms"], 1),
                        "tile_launches": st["tile_launches"]},
            "per_context": {"circuits_run": len(sel), "every": seq_every,
                            "e2e_s_scaled": round(seq_wall * scale, 3),
                            "e2e_circuits_per_s": round(len(sel) / seq_wall, 1),
                            "device_ms_scaled": round(seq_dev * scale, 2),
                            "device_circuits_per_s": round(len(sel) / (seq_dev / 1000.0), 1),
                            "note": "one fused context per circuit, one bulk gate-list call each, one stream"},
            "speedup_e2e": round((seq_wall * scale) / t_e2e, 2),
            "speedup_device": round((seq_dev * scale) / dev_ms, 2),
            "precision": {"circuits_checked": len(pick), "tv_max": tv_max, "max_abs": mx_max,
                          "reference": "complex128 CPU oracle", "oracle_s": round(t_or, 1)}}


def dense_block_measurement(qk, torch, stream, n: int = 20, depth: int = 30):
    """One n-qubit U3 + CZ layer circuit three ways: the fused tile path (FP32
    CUDA cores, pivot-form butterflies), and every layer as dense
    5-qubit blocks (the layer's U3s on five neighbouring qubits and the CZs among
    them multiplied into one 32 x 32 unitary on the host) on the tensor cores
    (3xTF32; a block elsewhere is first gathered onto the five lowest physical
    qubits) and on CUDA cores, with the CZs between blocks as phase passes.  Device time
    and error against the complex128 oracle for each."""
    import numpy as np
    import oracle

    _, _, ang = workloads.batch_layer_spec(7, n_min=n, n_max=n, d_min=depth, d_max=depth)
    circ = workloads.layer_spec_circuit(n, depth, ang)
    ref = oracle.OracleState(n, openmp=True)
    for op in circ.ops:
        ref.apply_op(op)
    groups = [list(range(g, min(g + 5, n))) for g in range(0, n, 5)]

    def block_matrix(L, qs):
        u = np.array([[1.0 + 0j]])
        for q in reversed(qs):                    # first target (highest qubit) = MSB
            u = np.kron(u, oracle.u3(*ang[L][q]))
        d = np.ones(1 << len(qs), dtype=np.complex128)
        for q in range(L % 2, n - 1, 2):
            if q in qs and q + 1 in qs:
                a, b2 = qs.index(q), qs.index(q + 1)
                for x in range(1 << len(qs)):
                    if (x >> a) & 1 and (x >> b2) & 1:
                        d[x] = -d[x]
        return d[:, None] * u

    mats = [[block_matrix(L, qs) for qs in groups] for L in range(depth)]

    def run_dense(ctx, gids):
        for L in range(depth):
            for g, qs in enumerate(groups):
                ctx.apply_gate(gids[L][g], list(reversed(qs)))
            for q in range(L % 2, n - 1, 2):
                if q // 5 != (q + 1) // 5:
                    ctx.apply_gate("z", [q + 1], controls=[q])

    def timed(make, runner):
        ctx = make()
        runner(ctx)
        ctx.sync()
        ctx.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        runner(ctx)
        ctx.flush()
        e1.record(stream)
        torch.cuda.synchronize()
        got = ctx.get_state().astype(np.complex128)
        ctx.close()
        return {"ms": round(e0.elapsed_time(e1), 3),
                "tv": 0.5 * float(np.abs(np.abs(got) ** 2 - np.abs(ref.psi) ** 2).sum()),
                "max_abs": float(np.abs(got - ref.psi).max())}

    out = {"n": n, "layers": depth, "gates": len(circ.ops)}
    ops = qk.layer_gate_ops(n, depth, ang)

    def mk_fused():
        c = qk.Context("c64", "fused", stream=stream.cuda_stream)
        c.add_qubits(n)
        return c

    out["fused_tile_fp32"] = timed(mk_fused, lambda c: c.apply_gates(ops))
    for tc in (True, False):
        holder = {}

        def mk(tc=tc, holder=holder):
            c = qk.Context("c64", "plain", stream=stream.cuda_stream, tensor_cores=tc)
            c.add_qubits(n)
            holder["gids"] = [[c.define_gate_matrix(m) for m in row] for row in mats]
            return c

        out["dense_blocks_3xtf32" if tc else "dense_blocks_fp32"] = timed(mk, lambda c: run_dense(c, holder["gids"]))
    return out


# ---------------------------------------------------------------------------
# precision of the measured path (the metric's TV bound)
# ---------------------------------------------------------------------------
def precision_measurement(qk, torch, stream, n: int, gops):
    """Total-variation distance and max |a - b| between the complex64 fused state
    and the complex128 one-pass-per-gate state after the step's gates (before the
    measurement), both on the GPU at the full size.  The complex128 path is itself
    checked element by element against the CPU oracle in the parity tests.  The
    QFT's closing SWAPs are left out: they only relabel qubits, and without them
    neither state needs a relabelling gather (which would not fit beside both
    states at 33 qubits)."""
    gops = [op for op in gops if op.kind != "swap"]
    a = qk.Context("c64", "fused", stream=stream.cuda_stream)
    a.add_qubits(n)
    qk.run_ops(a, gops)
    va = a.torch_view()
    a.sync()
    b = qk.Context("c128", "plain", stream=stream.cuda_stream)
    b.add_qubits(n)
    qk.run_ops(b, gops)
    vb = b.torch_view()
    b.sync()
    torch.cuda.synchronize()
    tv, mx, norm = 0.0, 0.0, 0.0
    chunk = 1 << 25
    for s0 in range(0, 1 << n, chunk):
        x = va[s0:s0 + chunk].to(torch.complex128)
        y = vb[s0:s0 + chunk]
        px = x.real * x.real + x.imag * x.imag
        py = y.real * y.real + y.imag * y.imag
        tv += float((px - py).abs().sum())
        norm += float(px.sum())
        mx = max(mx, float((x - y).abs().max()))
    a.close()
    b.close()
    return {"n": n, "tv": 0.5 * tv, "max_abs": mx, "norm2_c64": norm, "tv_bound": 1e-5, "max_abs_bound": 1e-4,
            "reference": "complex128 one-pass-per-gate path on the GPU, same gates"}


# ---------------------------------------------------------------------------
# serving (secondary measurement)
# ---------------------------------------------------------------------------
def serving_measurement(torch, count: int, rate: float = 200.0):
    """Seeded requests of 8..33 qubits (log-uniform) arriving as a Poisson process,
    served with continuous batching vs one at a time on the plain sequential path.
    Measured bits of the two paths must agree."""
    from paper_1908_07187_gb300 import qk, serve

    reqs = [workloads.serving_request(10_000 + i) for i in range(count)]
    arr = workloads.poisson_arrivals(count, rate, seed=11)
    # each request marshalled once, before its arrival, for both paths
    calls = [serve.marshal(qk, c) for c in reqs]
    warm = [workloads.serving_request(20_000 + i, n_min=8, n_max=20) for i in range(8)]
    serve.Server(qk, torch).run(warm, [0.0] * len(warm))
    served = serve.Server(qk, torch).run(reqs, arr, calls)
    plain = serve.serve_plain(qk, torch, reqs, arr, calls=calls)
    agree = sum(list(a.cbits) == list(b.cbits) for a, b in zip(served, plain))
    out = {"requests": count, "arrival_rate_per_s": rate, "qubits": "log-uniform 8..33",
           "served": serve.summarize(served), "plain": serve.summarize(plain),
           "small_batched": sum(r.path == "batch" for r in served), "bits_agree": agree,
           "hbm_budget_bytes": 160 * 10**9}
    out["speedup_circuits_per_s"] = out["served"]["circuits_per_s"] / out["plain"]["circuits_per_s"]
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1908_07187_gb300 import qk

    n = args.n
    circ = workload(n, 2 + rank)          # independent replica per rank
    gops = gate_ops(circ)
    meas = [op for op in circ.ops if op.kind == "measure"]
    n_gates = len(gops)
    stream = torch.cuda.Stream()
    ctx = qk.Context("c64", args.mode, stream=stream.cuda_stream, profile=True)
    ctx.add_qubits(n)
    ctx.add_cbits(n)

    def step():
        ctx.reset()
        qk.run_ops(ctx, gops)
        for op in meas:
            ctx.measure(op.targets, op.uniforms, op.cbits, wait=False)
        ctx.flush()

    for _ in range(args.warmup):
        step()
    ctx.sync()
    ctx.profile()                      # drop warm-up launch records
    ctx.reset_counters()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    counters = ctx.counters()
    prof = ctx.profile()
    if dist:
        dist.barrier()
    ms = max_over_ranks([ms], dist, "cuda")[0]
    ms_per_step = ms / args.steps
    value = job_throughput(n_gates, args.steps, world, ms / 1000.0)

    # end to end through the public API: host gate descriptors in, outcome out
    h2d = 0
    for op in gops:
        h2d += 4 * (len(op.targets) + len(op.controls) + len(op.cond)) + 8 * len(op.params)
    for op in meas:
        h2d += 4 * (len(op.targets) + len(op.cbits)) + 8 * len(op.uniforms)
    d2h = 8
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.reset()
        qk.run_ops(ctx, gops)
        for op in meas:
            outcome = ctx.measure(op.targets, op.uniforms, op.cbits, wait=True)
    t_e2e = max_over_ranks([time.perf_counter() - t0], dist, "cuda")[0]
    e2e_value = job_throughput(n_gates, e2e_steps, world, t_e2e)
    _ = outcome
    ctx.close()                        # frees the state before the secondary measurements

    # one-pass-per-gate comparison (fused vs plain), a short run
    plain = None
    if args.mode == "fused" and not args.no_plain:
        pctx = qk.Context("c64", "plain", stream=stream.cuda_stream)
        pctx.add_qubits(n)
        pctx.add_cbits(n)
        qk.run_ops(pctx, gops)  # warm
        pctx.sync()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        pctx.reset()
        qk.run_ops(pctx, gops)
        for op in meas:
            pctx.measure(op.targets, op.uniforms, op.cbits, wait=False)
        pctx.flush()
        p1.record(stream)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1)
        plain = {"value": n_gates / (pms / 1000.0), "unit": UNIT, "ms_per_step": pms}
        pctx.close()

    # roofline for the kernel class with the largest device-time share: HBM,
    # the algorithmic bytes of one launch (a tile pass reads and writes the state
    # once: 2^n x 8 B x 2) over the launch's average CUDA-event time
    top = max(prof, key=lambda k: prof[k]["ms"])
    rec = prof[top]
    peak, peak_kind = peaks()
    per_launch_s = rec["ms"] / rec["launches"] / 1000.0 if rec["launches"] else 0.0
    alg_bytes = rec["bytes"] / rec["launches"] if rec["launches"] else 0.0
    achieved = alg_bytes / per_launch_s / 1e9 if per_launch_s else 0.0
    traffic = recorded_traffic(top, n)
    tot_ms = sum(v["ms"] for v in prof.values())
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": top,
                "peak_kind": f"{peak_kind} (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)",
                "launches_per_step": rec["launches"] / args.steps,
                "share_of_device_time": round(rec["ms"] / tot_ms, 4) if tot_ms else None,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": round(1000.0 * per_launch_s, 4)}
    roofline_fp32 = None
    if top == "tile":
        # the same passes against the FP32 lane rate, counting what the kernel executes
        sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        sm_mhz = clk.get("sm_mhz") or 2070.0
        launches_step = rec["launches"] / args.steps
        ops_step = tile_fp32_ops(gops, n, launches_step)
        lane_peak = fp32_lane_peak(sm_count, sm_mhz)
        rate = ops_step / (rec["ms"] / args.steps / 1000.0)
        roofline_fp32 = {"bound": "alu", "achieved": round(rate / 1e12, 3), "peak": round(lane_peak / 1e12, 3),
                         "unit": "T FP32 lane-ops/s", "frac": round(rate / lane_peak, 4),
                         "ops_per_step": ops_step,
                         "peak_kind": f"derived: {sm_count} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (median SM clock "
                                      "sampled during the timed region)",
                         "count": "8 per amplitude pair per uncontrolled non-diagonal gate, 16 per acting pair per "
                                  "controlled one, 4 per amplitude per pass (final phase and scale); lower bound"}

    # secondary measurements: a failure in one is recorded under its key and
    # the line is still printed
    def guarded(name, fn, *a, **kw):
        try:
            return fn(*a, **kw)
        except Exception as e:  # noqa: BLE001
            print(f"bench: {name} failed: {type(e).__name__}: {e}", file=sys.stderr)
            return {"error": f"{type(e).__name__}: {str(e)[:300]}"}

    kitaev = None
    big = None
    if not args.no_33q and n < 33:
        big = guarded("layered_33q", layered_33q_measurement, qk, torch, stream)
    shor3 = None
    if not args.no_3nx1:
        shor3 = guarded("shor_3nx1", shor_3nx1_measurement, qk, torch, stream)
    if not args.no_kitaev:
        kitaev = guarded("kitaev", kitaev_measurement, qk, torch, stream)
    block = block4 = None
    if not args.no_block:
        block = guarded("block5", block_measurement, qk, torch, stream, n)
        block4 = guarded("block4", block_measurement, qk, torch, stream, n, k=4)
    batch = None
    if args.batch_circuits > 0 and world == 1:
        batch = guarded("batched", batch_measurement, qk, torch, stream, args.batch_circuits)
        if "error" not in batch:
            batch["dense_blocks_vs_tile"] = guarded("dense_blocks_vs_tile", dense_block_measurement, qk, torch,
                                                    stream)
    precision = None
    if not args.no_precision and args.mode == "fused":
        precision = guarded("precision", precision_measurement, qk, torch, stream, n, gops)
    serving = None
    if args.serve_requests > 0 and world == 1:
        serving = guarded("serving", serving_measurement, torch, args.serve_requests)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = guarded("cpu_baseline", cpu_baseline, n, circ)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": f"layered U3/CZ-brickwork 500 gates + QFT({n}) + measure all, {n} qubits complex64",
                       "n_qubits": n, "gates_per_step": n_gates, "mode": args.mode,
                       "l2": "state (%.1f GiB) larger than L2" % ((8 << n) / 2 ** 30), "parallelism": f"replicas{world}"},
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": counters["launches"],
            "state_passes_per_step": counters["state_passes"] / args.steps,
            "roofline": roofline,
            "roofline_fp32": roofline_fp32,
            # what one-pass-per-gate execution would have to stream for the same gates/s
            "gate_equivalent_bandwidth": {
                "GBps": round(value * 2 * 8 * (1 << n) / 1e9, 1),
                "x_measured_hbm_peak": round(value * 2 * 8 * (1 << n) / 1e9 / peak, 2),
                "unfused_plain_path_GBps": round(plain["value"] * 2 * 8 * (1 << n) / 1e9, 1) if plain else None},
            "cpu_baseline": cpu,
            "plain_path": plain,
            "precision": precision,
            "kitaev": kitaev,
            "shor_3nx1": shor3,
            "layered_33q": big,
            "block4": block4,
            "block5": block,
            "batched": batch,
            "serving": serving,
            "launch_profile": {k: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k, v in prof.items() if v["launches"]},
            "clocks": clk,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
