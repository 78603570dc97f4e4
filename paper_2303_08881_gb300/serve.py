"""Serving runtime: a stream of FGMRES solve requests through one GPU.

Requests arrive with a matrix (host CSR + subdomain partition), a right-hand side and an
arrival time. A pool of worker threads serves them in arrival order, each worker on its own
CUDA stream, so several requests' setups (host analysis in C++, which releases the GIL) and
solves run concurrently. Factors are cached per matrix: a request that repeats an earlier
matrix reuses its handle and only solves. Device memory is bounded by an admission cap: a
new handle is admitted only when its estimated footprint fits under the cap together with
every live and cached handle; idle cached handles are evicted least recently used first, and
otherwise the request waits for memory to be released.

The latency of a request is the time from its arrival to its solution being back in host
memory. Nothing here computes any part of the method: every numerical step runs through
the library's C ABI (``ilu_setup`` / ``gmres_solve``).
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np


def estimate_bytes(n: int, nnz: int, restart: int, pc_bytes: int = 4) -> int:
    """Device footprint of a handle before it exists: the CSR in two orders, the FP64
    local values (three factor regions), the streamed programs, the inner workspaces and
    the FGMRES basis V, Z ((2 restart + 1) vectors of n doubles) with slack."""
    factors = nnz * (12 + 12 + 3 * 8) + nnz * (8 + 2 * pc_bytes)
    krylov = (2 * restart + 6) * 8 * ((n + 63) // 64 * 64)
    return int(1.2 * (factors + krylov + 64 * n)) + (4 << 20)


@dataclass
class CacheEntry:
    handle: object
    bytes: int
    busy: int = 0
    last: float = 0.0


class HandleCache:
    """Handles keyed by matrix, with an admission cap on their summed device bytes.
    Thread-safe. `reserve` blocks until the request fits (evicting idle entries, least
    recently used first) or raises MemoryError if it can never fit."""

    def __init__(self, cap_bytes: int, free_fn=None, clock=time.perf_counter):
        self.cap = int(cap_bytes)
        self.entries: "collections.OrderedDict[str, CacheEntry]" = collections.OrderedDict()
        self.reserved = 0          # bytes of handles being built
        self.building = set()      # keys whose handle a request is building
        self.cv = threading.Condition()
        self.free_fn = free_fn or (lambda h: h.close())
        self.clock = clock
        self.evictions = 0
        self.hits = 0
        self.peak = 0

    def held(self) -> int:
        return sum(e.bytes for e in self.entries.values()) + self.reserved

    def acquire(self, key: str, timeout: float = 600.0):
        """The cached handle for `key`, marked busy, once no other request uses it (a
        handle serves one thread at a time). None when `key` is neither cached nor being
        built; the caller then builds it and must call `insert` or `abandon`."""
        deadline = self.clock() + timeout
        with self.cv:
            while True:
                e = self.entries.get(key)
                if e is not None and e.busy == 0:
                    e.busy = 1
                    e.last = self.clock()
                    self.entries.move_to_end(key)
                    self.hits += 1
                    return e.handle
                if e is None and key not in self.building:
                    self.building.add(key)
                    return None
                left = deadline - self.clock()
                if left <= 0:
                    raise TimeoutError(f"handle {key} stayed busy")
                self.cv.wait(left)

    def abandon(self, key: str) -> None:
        """A build of `key` failed: let the next request build it."""
        with self.cv:
            self.building.discard(key)
            self.cv.notify_all()

    def reserve(self, nbytes: int, timeout: float = 600.0) -> None:
        if nbytes > self.cap:
            raise MemoryError(f"request needs {nbytes} bytes, above the {self.cap}-byte cap")
        deadline = self.clock() + timeout
        with self.cv:
            while self.held() + nbytes > self.cap:
                idle = [k for k, e in self.entries.items() if e.busy == 0]
                if idle:
                    k = idle[0]  # least recently used (entries are kept in use order)
                    e = self.entries.pop(k)
                    self.free_fn(e.handle)
                    self.evictions += 1
                    continue
                left = deadline - self.clock()
                if left <= 0:
                    raise MemoryError("admission wait timed out")
                self.cv.wait(left)
            self.reserved += nbytes
            self.peak = max(self.peak, self.held())

    def insert(self, key: str, handle, reserved: int, actual: int) -> None:
        """Turn the caller's reservation into a cached entry of `actual` bytes, busy
        with the caller's request."""
        with self.cv:
            self.reserved -= reserved
            self.building.discard(key)
            self.entries[key] = CacheEntry(handle, int(actual), busy=1, last=self.clock())
            self.peak = max(self.peak, self.held())
            self.cv.notify_all()

    def cancel(self, reserved: int) -> None:
        with self.cv:
            self.reserved -= reserved
            self.cv.notify_all()

    def update_bytes(self, key: str, actual: int) -> None:
        with self.cv:
            e = self.entries.get(key)
            if e is not None:
                e.bytes = int(actual)
                self.peak = max(self.peak, self.held())

    def release(self, key: str) -> None:
        with self.cv:
            e = self.entries.get(key)
            if e is not None:
                e.busy -= 1
                e.last = self.clock()
            self.cv.notify_all()

    def close(self) -> None:
        with self.cv:
            for e in self.entries.values():
                self.free_fn(e.handle)
            self.entries.clear()


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the trace starts
    key: str                # matrix identity; repeats share it
    problem: object         # paper_2303_08881_gb300.problems.Problem (host CSR, partition, b)


@dataclass
class Record:
    rid: int
    arrival: float
    start: float = 0.0
    done: float = 0.0
    iters: int = 0
    status: int = -1
    reused: bool = False
    rel_res: float = float("nan")
    device_bytes: int = 0
    setup_s: float = 0.0     # handle build (host analysis + device factorisation); 0 when reused
    solve_s: float = 0.0     # right-hand side in, FGMRES, solution out
    host_ms: float = 0.0     # the handle's host analysis, device setup and graph build (library clocks)
    device_ms: float = 0.0
    graph_ms: float = 0.0
    escalations: int = 0     # continuations with a longer restart after maxit (see serve)
    x: object = None         # the solution (host numpy) when serve(keep_solutions=True)


@dataclass
class Report:
    records: list
    wall: float
    cache_hits: int
    evictions: int
    peak_bytes: int
    workers: int
    cap_bytes: int
    stats: dict = field(default_factory=dict)


def serve(requests, workers: int = 8, cap_bytes: int = 120 << 30, restart: int = 50, rtol: float = 1e-8,
          maxit: int = 5000, opts: dict | None = None, check_residual: bool = True,
          keep_solutions: bool = False, escalate: tuple = (200, 256)) -> Report:
    """Run the requests (sorted by arrival) in real time and return per-request records.

    A solve that reaches maxit without meeting rtol continues from its last iterate with
    each restart length in `escalate` in turn (a longer Krylov space per cycle for the
    hardest, most anisotropic requests), each with a fresh maxit; a request that still does
    not converge is reported with status ILU_ERR_NOT_CONVERGED."""
    import torch
    import paper_2303_08881_gb300 as ilu

    opts = dict(opts or {})
    cache = HandleCache(cap_bytes)
    pending: "queue.Queue[Request | None]" = queue.Queue()
    records = {r.rid: Record(r.rid, r.arrival) for r in requests}
    errors = []
    t0 = [0.0]

    def now():
        return time.perf_counter() - t0[0]

    def worker():
        stream = torch.cuda.Stream()
        while True:
            req = pending.get()
            if req is None:
                return
            rec = records[req.rid]
            rec.start = now()
            pr = req.problem
            key = req.key
            held = False  # whether this request holds a busy mark on the entry `key`
            try:
                h = cache.acquire(key)
                rec.reused = held = h is not None
                if h is None:
                    est = estimate_bytes(pr.n, pr.nnz, restart, 4 if opts.get("pc_precision", "fp32") == "fp32" else 8)
                    try:
                        cache.reserve(est)
                    except Exception:
                        cache.abandon(key)
                        raise
                    ts = time.perf_counter()
                    try:
                        h = ilu.ilu_setup_problem(pr, ilu.Opts(stream=stream.cuda_stream, **opts))
                        rec.setup_s = time.perf_counter() - ts
                    except Exception:
                        cache.cancel(est)
                        cache.abandon(key)
                        raise
                    cache.insert(key, h, est, max(est, h.stats()["device_bytes"]))
                    held = True
                ts = time.perf_counter()
                with torch.cuda.stream(stream):
                    b = torch.from_numpy(pr.b).to("cuda", non_blocking=True)
                    x = torch.zeros_like(b)
                # a reused handle solves on the stream it was created with
                stream.synchronize()
                info = ilu.gmres_solve(h, b, x, rtol=rtol, restart=restart, maxit=maxit)
                iters = info["iters"]
                for m in escalate:
                    if info["status"] != ilu.ILU_ERR_NOT_CONVERGED:
                        break
                    rec.escalations += 1
                    info = ilu.gmres_solve(h, b, x, rtol=rtol, restart=m, maxit=maxit)  # x: the last iterate
                    iters += info["iters"]
                info["iters"] = iters
                xs = x.cpu().numpy()
                rec.done = now()
                rec.solve_s = time.perf_counter() - ts
                rec.iters, rec.status = info["iters"], info["status"]
                if keep_solutions:
                    rec.x = xs
                rec.device_bytes = h.stats()["device_bytes"]
                tm = h.times()
                if not rec.reused:
                    rec.host_ms, rec.device_ms = tm["host_ms"], tm["device_ms"]
                rec.graph_ms = tm["graph_ms"]
                cache.update_bytes(key, rec.device_bytes)
                if check_residual:
                    r = pr.b - pr.scipy() @ xs
                    rec.rel_res = float(np.linalg.norm(r) / max(np.linalg.norm(pr.b), 1e-300))
            except Exception as e:  # recorded, the trace goes on
                rec.done = now()
                rec.status = -2
                errors.append((req.rid, repr(e)))
            finally:
                if held:
                    cache.release(key)

    threads = [threading.Thread(target=worker, daemon=True) for _ in range(workers)]
    for t in threads:
        t.start()
    t0[0] = time.perf_counter()
    for r in sorted(requests, key=lambda q: q.arrival):
        wait = r.arrival - now()
        if wait > 0:
            time.sleep(wait)
        pending.put(r)
    for _ in threads:
        pending.put(None)
    for t in threads:
        t.join()
    wall = now()
    cache.close()
    rep = Report([records[r.rid] for r in requests], wall, cache.hits, cache.evictions, cache.peak, workers,
                 cap_bytes)
    rep.stats = summarize(rep.records, wall)
    rep.stats["errors"] = errors[:5]
    return rep


def summarize(records, wall: float) -> dict:
    ok = [r for r in records if r.status in (0, 5)]
    lat = np.array([r.done - r.arrival for r in ok]) if ok else np.zeros(1)
    return {
        "requests": len(records),
        "completed": len(ok),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "throughput_rps": len(ok) / max(wall, 1e-9),
        "reused": sum(r.reused for r in ok),
        "max_rel_res": float(max((r.rel_res for r in ok if r.rel_res == r.rel_res), default=float("nan"))),
        "converged": sum(r.status == 0 for r in ok),
        "escalated": sum(r.escalations > 0 for r in ok),
        "max_iters": int(max((r.iters for r in ok), default=0)),
        "mean_wait_ms": float(np.mean([r.start - r.arrival for r in ok]) * 1e3) if ok else 0.0,
        "mean_setup_ms": float(np.mean([r.setup_s for r in ok if not r.reused]) * 1e3) if ok else 0.0,
        "mean_solve_ms": float(np.mean([r.solve_s for r in ok]) * 1e3) if ok else 0.0,
        "mean_host_analysis_ms": float(np.mean([r.host_ms for r in ok if not r.reused])) if ok else 0.0,
        "mean_device_setup_ms": float(np.mean([r.device_ms for r in ok if not r.reused])) if ok else 0.0,
        "mean_graph_ms": float(np.mean([r.graph_ms for r in ok])) if ok else 0.0,
        "busy_setup_s": float(sum(r.setup_s for r in ok)),
        "busy_solve_s": float(sum(r.solve_s for r in ok)),
    }
