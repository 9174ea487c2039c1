"""Continuous-batching request loop over one GPU (argument marshalling and
scheduling only; every amplitude operation runs in libqk's kernels).

Requests are circuits (``workloads.Circuit``) with arrival times.  Small requests
(at most ``Batch.SMEM_QUBITS`` qubits) are served by batched launches: while one
batch runs, newly arrived small requests collect into the next batch, which is
launched as soon as the running one finishes (two batch objects alternate).  Larger
requests each get a context on a stream of their own and run concurrently, admitted
while the sum of their state footprints (2^n x 8 bytes, twice that when the circuit
holds a permutation oracle, which gathers out of place) fits the HBM budget; freed
memory admits the next request.  Results are the measured classical bits (and, on
request, the final state).

``serve_plain`` is the comparison path: the same requests one after another in
arrival order, each on one context and stream through the per-gate engine, with no
batching and no overlap.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np


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
    max_active: int = 16               # concurrent large requests (streams)
    batch_max: int = 4096              # small requests per batched launch
    keep_states: bool = False
    stats: Dict[str, float] = field(default_factory=dict)

    def run(self, circuits: List, arrivals: List[float]) -> List[Result]:
        qk, torch = self.qk, self.torch
        small_max = qk.Batch.SMEM_QUBITS
        order = sorted(range(len(circuits)), key=lambda i: arrivals[i])
        results = [Result(i, circuits[i].n_qubits, arrivals[i]) for i in range(len(circuits))]
        pending_small: deque = deque()
        pending_large: deque = deque()
        batches = [qk.Batch(), qk.Batch()]
        inflight = None                 # (batch, [result indices])
        active: List[_Active] = []
        mem = 0
        done = 0
        nxt = 0
        n_batches = 0
        t0 = time.perf_counter()
        now = 0.0
        while done < len(circuits):
            now = time.perf_counter() - t0
            while nxt < len(order) and arrivals[order[nxt]] <= now:
                i = order[nxt]
                (pending_small if circuits[i].n_qubits <= small_max else pending_large).append(i)
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
            # -- large requests: admit while memory and streams allow
            while pending_large and len(active) < self.max_active:
                i = pending_large[0]
                need = footprint(circuits[i])
                if mem + need > self.hbm_budget_bytes and active:
                    break
                pending_large.popleft()
                c = circuits[i]
                stream = torch.cuda.Stream()
                ctx = qk.Context("c64", "fused", stream=stream.cuda_stream)
                ctx.add_qubits(c.n_qubits)
                if c.n_cbits:
                    ctx.add_cbits(c.n_cbits)
                results[i].start = time.perf_counter() - t0
                results[i].path = "stream"
                qk.run_ops(ctx, c.ops)
                ctx.flush()
                ev = torch.cuda.Event()
                ev.record(stream)
                active.append(_Active(results[i], ctx, stream, ev, need))
                mem += need
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
                    done += 1
                    progressed = True
                else:
                    still.append(a)
            active = still
            if not progressed:
                time.sleep(0.0001)
        for b in batches:
            b.close()
        self.stats = {"batches": n_batches, "makespan_s": max(r.finish for r in results) - min(arrivals)}
        return results


def serve_plain(qk, torch, circuits: List, arrivals: List[float], keep_states: bool = False) -> List[Result]:
    """One request at a time in arrival order on one stream (no batching, no overlap)."""
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
        qk.run_ops(ctx, c.ops)
        r.cbits = ctx.read_cbits()
        if keep_states:
            r.state = ctx.get_state()
        r.finish = time.perf_counter() - t0
        r.path = "plain"
        ctx.close()
    return results


def summarize(results: List[Result]) -> Dict[str, float]:
    lat = np.array([r.latency for r in results])
    span = max(r.finish for r in results) - min(r.arrival for r in results)
    return {"requests": len(results), "circuits_per_s": len(results) / span, "makespan_s": span,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
