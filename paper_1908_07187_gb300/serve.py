"""Continuous-batching request loop over one GPU (argument marshalling and
scheduling only; every amplitude operation runs in libqk's kernels).

Requests are circuits (``workloads.Circuit``) with arrival times.  Small requests
(at most ``Batch.SMEM_QUBITS`` qubits) are served by batched launches: while one
batch runs, newly arrived small requests collect into the next batch, which is
launched as soon as the running one finishes (two batch objects alternate).  Larger
requests each get a context on a stream of their own and run concurrently (up to
24 qubits, like the batches, on high-priority streams; mid-size and big requests
queue apart and at most four big ones run at once), admitted
while the sum of their state footprints (2^n x 8 bytes, twice that when the circuit
holds a permutation oracle, which gathers out of place) fits the HBM budget; freed
memory admits the next request.  Results are the measured classical bits (and, on
request, the final state).

A large request is handed to a worker thread that creates its context and
enqueues its work (the library calls release the interpreter lock), so the
scheduling loop keeps harvesting finished batches and admitting arrivals while
a big circuit is being planned.  Each request's ops are marshalled once into
runs of plain gates (one bulk gate-list call per run) and the calls that take
other arguments (permutation gates, measurements, phase corrections).

``serve_plain`` is the comparison path: the same requests one after another in
arrival order, each on one context and stream through the same marshalled
calls, with no batching and no overlap.
"""
from __future__ import annotations

import queue
import threading
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np


def marshal(qk, circ):
    """A circuit's ops as a list of library calls: ("gates", GATE_OP array) for
    each run of built-in 1-target gates, ("op", Op) for anything else."""
    out, run = [], []

    def close_run():
        if run:
            arr = np.zeros(len(run), dtype=qk.GATE_OP_DTYPE)
            for j, op in enumerate(run):
                arr[j]["gate_id"] = qk.GATE[op.kind]
                arr[j]["target"] = op.targets[0]
                arr[j]["nc"] = len(op.controls)
                arr[j]["controls"][:len(op.controls)] = op.controls
                arr[j]["ncc"] = len(op.cond)
                arr[j]["cond"][:len(op.cond)] = op.cond
                arr[j]["np"] = len(op.params)
                arr[j]["params"][:len(op.params)] = op.params
            out.append(("gates", arr))
            run.clear()

    for op in circ.ops:
        simple = (op.kind in qk.GATE and op.kind != "swap" and len(op.targets) == 1 and len(op.controls) <= 4
                  and len(op.cond) <= 4 and len(op.params) <= 3)
        if simple:
            run.append(op)
        else:
            close_run()
            out.append(("op", op))
    close_run()
    return out


def enqueue(qk, ctx, calls):
    """Enqueue a marshalled request on its context (no waiting)."""
    for kind, x in calls:
        if kind == "gates":
            ctx.apply_gates(x)
        else:
            qk.run_ops(ctx, [x])


@dataclass
class Result:
    index: int
    n: int
    arrival: float
    start: float = 0.0
    finish: float = 0.0
    cbits: Optional[np.ndarray] = None
    state: Optional[np.ndarray] = None
    path: str = ""

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def footprint(circ) -> int:
    """Device bytes a request holds while it runs."""
    has_perm = any(op.kind == "mulmod" for op in circ.ops)
    return (8 << circ.n_qubits) * (2 if has_perm else 1)


@dataclass
class _Active:
    res: Result
    ctx: object
    stream: object
    event: object
    mem: int


@dataclass
class Server:
    qk: object                         # the paper_1908_07187_gb300.qk module
    torch: object
    hbm_budget_bytes: int = 160 * 10**9
    max_active: int = 16               # concurrent requests above 13 qubits (streams)
    max_big: int = 4                   # of those, above priority_max_qubits
    batch_max: int = 4096              # small requests per batched launch
    keep_states: bool = False
    # requests up to this many qubits (and every batch) run on high-priority
    # streams, so that their short kernels are not queued behind the passes of
    # much larger states
    priority_max_qubits: int = 24
    stats: Dict[str, float] = field(default_factory=dict)

    def run(self, circuits: List, arrivals: List[float], calls: Optional[List] = None) -> List[Result]:
        qk, torch = self.qk, self.torch
        small_max = qk.Batch.SMEM_QUBITS
        if calls is None:
            calls = [marshal(qk, c) if c.n_qubits > small_max else None for c in circuits]
        order = sorted(range(len(circuits)), key=lambda i: arrivals[i])
        results = [Result(i, circuits[i].n_qubits, arrivals[i]) for i in range(len(circuits))]
        pending_small: deque = deque()
        # above 13 qubits: mid-size requests and big ones queue apart, so that a
        # big request waiting for memory does not hold up the small states behind it
        pending_mid: deque = deque()
        pending_big: deque = deque()
        hi_prio = torch.cuda.Stream(priority=-1)
        batches = [qk.Batch(stream=hi_prio.cuda_stream), qk.Batch(stream=hi_prio.cuda_stream)]
        inflight = None                 # (batch, [result indices])
        active: List[_Active] = []
        started: "queue.Queue" = queue.Queue()   # large requests whose work is enqueued
        pool = ThreadPoolExecutor(max_workers=self.max_active)
        starting = 0
        big_running = 0                 # big requests admitted and not finished
        mem = 0
        done = 0
        nxt = 0
        n_batches = 0
        t0 = time.perf_counter()
        now = 0.0

        def start_large(i, need):
            c = circuits[i]
            stream = torch.cuda.Stream(priority=-1 if c.n_qubits <= self.priority_max_qubits else 0)
            ctx = qk.Context("c64", "fused", stream=stream.cuda_stream)
            ctx.add_qubits(c.n_qubits)
            if c.n_cbits:
                ctx.add_cbits(c.n_cbits)
            enqueue(qk, ctx, calls[i])
            ctx.flush()
            ev = torch.cuda.Event()
            ev.record(stream)
            started.put(_Active(results[i], ctx, stream, ev, need))
        while done < len(circuits):
            now = time.perf_counter() - t0
            while nxt < len(order) and arrivals[order[nxt]] <= now:
                i = order[nxt]
                nq = circuits[i].n_qubits
                (pending_small if nq <= small_max else
                 pending_mid if nq <= self.priority_max_qubits else pending_big).append(i)
                nxt += 1
            progressed = False
            # -- small requests: one batched launch at a time, the next one fills meanwhile
            if inflight is not None and inflight[0].done():
                b, idx = inflight
                cbits = b.read_all_cbits()
                off = 0
                for pos, i in enumerate(idx):
                    r = results[i]
                    r.finish = time.perf_counter() - t0
                    k = circuits[i].n_cbits
                    r.cbits = cbits[off:off + k].copy()
                    off += k
                    if self.keep_states:
                        r.state = b.read(pos)[1]
                    done += 1
                inflight = None
                progressed = True
            if inflight is None and pending_small:
                b = batches[n_batches % 2]
                b.clear()
                idx = []
                while pending_small and len(idx) < self.batch_max:
                    i = pending_small.popleft()
                    c = circuits[i]
                    b.add_ops(c.n_qubits, c.n_cbits, c.ops)
                    results[i].start = time.perf_counter() - t0
                    results[i].path = "batch"
                    idx.append(i)
                b.run(store_states=self.keep_states)
                inflight = (b, idx)
                n_batches += 1
                progressed = True
            # -- large requests: admit while memory and streams allow; a worker
            # thread creates the context and enqueues the work
            for q, big in ((pending_big, True), (pending_mid, False)):
                while q and len(active) + starting < self.max_active and (not big or big_running < self.max_big):
                    i = q[0]
                    need = footprint(circuits[i])
                    if mem + need > self.hbm_budget_bytes and (active or starting):
                        break
                    q.popleft()
                    results[i].start = time.perf_counter() - t0
                    results[i].path = "stream"
                    mem += need
                    starting += 1
                    big_running += int(big)
                    pool.submit(start_large, i, need)
                    progressed = True
            while True:
                try:
                    a = started.get_nowait()
                except queue.Empty:
                    break
                starting -= 1
                active.append(a)
                progressed = True
            still = []
            for a in active:
                if a.event.query():
                    a.res.finish = time.perf_counter() - t0
                    a.res.cbits = a.ctx.read_cbits()
                    if self.keep_states:
                        a.res.state = a.ctx.get_state()
                    a.ctx.close()
                    mem -= a.mem
                    big_running -= int(a.res.n > self.priority_max_qubits)
                    done += 1
                    progressed = True
                else:
                    still.append(a)
            active = still
            if not progressed:
                time.sleep(0.0001)
        pool.shutdown(wait=True)
        for b in batches:
            b.close()
        self.stats = {"batches": n_batches, "makespan_s": max(r.finish for r in results) - min(arrivals)}
        return results


def serve_plain(qk, torch, circuits: List, arrivals: List[float], keep_states: bool = False,
                calls: Optional[List] = None) -> List[Result]:
    """One request at a time in arrival order on one stream (no batching, no overlap)."""
    if calls is None:
        calls = [marshal(qk, c) for c in circuits]
    results = [Result(i, circuits[i].n_qubits, arrivals[i]) for i in range(len(circuits))]
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    for i in sorted(range(len(circuits)), key=lambda i: arrivals[i]):
        while time.perf_counter() - t0 < arrivals[i]:
            time.sleep(0.0001)
        c = circuits[i]
        r = results[i]
        r.start = time.perf_counter() - t0
        ctx = qk.Context("c64", "fused", stream=stream.cuda_stream)
        ctx.add_qubits(c.n_qubits)
        if c.n_cbits:
            ctx.add_cbits(c.n_cbits)
        enqueue(qk, ctx, calls[i])
        r.cbits = ctx.read_cbits()
        if keep_states:
            r.state = ctx.get_state()
        r.finish = time.perf_counter() - t0
        r.path = "plain"
        ctx.close()
    return results


SIZE_CLASSES = (("8-13", 8, 13), ("14-24", 14, 24), ("25-29", 25, 29), ("30-33", 30, 33))


def summarize(results: List[Result]) -> Dict[str, object]:
    lat = np.array([r.latency for r in results])
    span = max(r.finish for r in results) - min(r.arrival for r in results)
    out = {"requests": len(results), "circuits_per_s": len(results) / span, "makespan_s": span,
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "mean_ms": float(lat.mean() * 1e3), "by_qubits": {}}
    for name, lo, hi in SIZE_CLASSES:
        sub = np.array([r.latency for r in results if lo <= r.n <= hi])
        if len(sub):
            out["by_qubits"][name] = {"requests": int(len(sub)), "p50_ms": float(np.percentile(sub, 50) * 1e3),
                                      "p99_ms": float(np.percentile(sub, 99) * 1e3)}
    return out
