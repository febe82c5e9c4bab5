"""Continuous-batching MPHF build server.

Requests (a key set and a hash seed) arrive over time.  A request is
admitted as soon as a slot is free *and* the device memory it adds fits the
remaining budget, so requests that arrive while others are on the GPU start
without waiting for a batch to drain; admitted builds run concurrently, one
CUDA stream per slot, and overlap on the device.  Each slot keeps its
workspace between requests (grown when a larger request needs more), and
the built function (g values and rank directory) stays on the device.  A
build whose hypergraph keeps a 2-core is retried with the next hash seeds
(inside hpeel_mphf_build).  Latency is measured from a request's arrival to
its completion.

The budget bounds what the server holds on the device, not only what is in
flight: every slot's retained workspace, the keys and outputs of running
builds, and the outputs of finished builds kept for the caller (until
release()) are all counted.  When a pending request does not fit, idle
slots give their workspaces back.

The scheduling never changes a result: a request gets the same g values and
rank directory alone and in any mix.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import mphf_build, mphf_workspace_size, num_vertices


@dataclass
class Request:
    rid: int
    keys: object            # host (numpy uint64 / torch int64) or device int64 tensor
    seed: int = 1
    arrival: float = 0.0    # seconds, on the server's clock
    footprint: int = 0      # device bytes while in flight (filled at submit)


@dataclass
class Result:
    rid: int
    n: int
    m: int
    G: object = None
    rank_dir: object = None
    stats: dict = field(default_factory=dict)
    error: str | None = None
    arrival: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    held: int = 0           # device bytes of G and rank_dir the server still counts

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def output_bytes(n: int, gamma_milli: int = 1230) -> int:
    """Device bytes of a built function: g values and rank directory."""
    m = num_vertices(n, gamma_milli, 3)
    return 8 * max((m + 31) // 32, 1) + 8 * ((m + 511) // 512 + 1)


def footprint_bytes(n: int, gamma_milli: int = 1230) -> int:
    """Device bytes one build holds: workspace, keys, g values, rank directory."""
    return mphf_workspace_size(n, gamma_milli) + 8 * n + output_bytes(n, gamma_milli)


class MphfServer:
    def __init__(self, slots: int = 4, hbm_budget: int = 16 << 30, gamma_milli: int = 1230,
                 max_tries: int = 8, device: int = 0, keep_results: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.gamma = gamma_milli
        self.max_tries = max_tries
        self.budget = hbm_budget
        self.keep = keep_results
        self.in_use = 0       # device bytes held: workspaces, running builds, kept outputs
        self.max_in_use = 0   # largest in_use seen
        self.max_running = 0  # most requests on the device at once
        self.running = 0
        self.pending: deque[Request] = deque()
        self.results: dict[int, Result] = {}
        self.cv = threading.Condition()
        self.stop = False
        self.t0 = time.perf_counter()
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(slots)]
        for w in self.workers:
            w.start()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ---------------------------------------------------------------- API --
    def submit(self, req: Request) -> None:
        n = int(req.keys.shape[0])
        req.footprint = footprint_bytes(n, self.gamma)
        if req.footprint > self.budget:
            with self.cv:
                self.results[req.rid] = Result(req.rid, n, num_vertices(n, self.gamma, 3),
                                               error="footprint exceeds the memory budget",
                                               arrival=req.arrival, finished=self.now())
                self.cv.notify_all()
            return
        with self.cv:
            self.pending.append(req)
            self.cv.notify_all()

    def release(self, rid: int) -> Result | None:
        """Drop the server's copy of a finished result (its g values and rank
        directory leave the budget); returns the result."""
        with self.cv:
            res = self.results.pop(rid, None)
            if res is not None and res.held:
                self.in_use -= res.held
                res.held = 0
                self.cv.notify_all()
            return res

    def wait(self, count: int, timeout: float = 600.0) -> None:
        deadline = time.perf_counter() + timeout
        with self.cv:
            while len(self.results) < count:
                left = deadline - time.perf_counter()
                if left <= 0:
                    raise TimeoutError(f"{len(self.results)} of {count} requests finished")
                self.cv.wait(left)

    def close(self) -> None:
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for w in self.workers:
            w.join()

    # ---------------------------------------------------------- scheduling --
    def _take(self, ws_bytes: int):
        """Under the lock: the first pending request that fits the budget
        (first come first served, smaller requests may pass a large one that
        does not fit yet), for a slot that holds a workspace of ws_bytes.
        Returns (request, workspace bytes to allocate) or (None, 0)."""
        for i, req in enumerate(self.pending):
            n = int(req.keys.shape[0])
            need_ws = mphf_workspace_size(n, self.gamma)
            grow = need_ws if need_ws > ws_bytes else 0  # the old one is freed first
            cost = 8 * n + output_bytes(n, self.gamma) + grow - (ws_bytes if grow else 0)
            if self.in_use + cost <= self.budget:
                del self.pending[i]
                self.in_use += cost
                self.running += 1
                self.max_in_use = max(self.max_in_use, self.in_use)
                self.max_running = max(self.max_running, self.running)
                return req, grow
        return None, 0

    def _worker(self, slot: int):
        torch = self.torch
        stream = torch.cuda.Stream(device=self.device)
        ws = None
        ws_bytes = 0  # counted in in_use while the slot keeps it
        while True:
            with self.cv:
                req = None
                while not self.stop:
                    req, grow = self._take(ws_bytes)
                    if req is not None:
                        break
                    if ws is not None and self.pending:
                        # a waiting request does not fit: give the idle
                        # workspace back and look again
                        ws = None
                        self.in_use -= ws_bytes
                        ws_bytes = 0
                        self.cv.notify_all()
                        continue
                    self.cv.wait()
                if req is None:
                    if ws is not None:
                        ws = None
                        self.in_use -= ws_bytes
                    return
                admitted = self.now()
                if grow:
                    ws = None  # freed before the larger one is taken
                    ws_bytes = grow
            n = int(req.keys.shape[0])
            io = 8 * n + output_bytes(n, self.gamma)
            res = Result(req.rid, n, num_vertices(n, self.gamma, 3), arrival=req.arrival,
                         admitted=admitted)
            keys = out = None
            try:
                with torch.cuda.device(self.device), torch.cuda.stream(stream):
                    if ws is None:
                        ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=self.device)
                    keys = req.keys
                    if not (isinstance(keys, torch.Tensor) and keys.is_cuda):
                        if isinstance(keys, np.ndarray):
                            keys = torch.from_numpy(keys.view(np.int64))
                        keys = keys.to(self.device, non_blocking=True)
                    out = mphf_build(keys, req.seed, self.gamma, self.max_tries, workspace=ws)
                    if self.keep:
                        res.G, res.rank_dir = out.G, out.rank_dir
                        res.held = output_bytes(n, self.gamma)
                    res.stats = out.stats
            except Exception as exc:  # a failed build is reported, not raised
                res.error = str(exc)
            finally:
                keys = out = None  # the device copies leave with the accounting
            res.finished = self.now()
            with self.cv:
                self.in_use -= io - res.held
                self.running -= 1
                self.results[req.rid] = res
                self.cv.notify_all()


def run_stream(server: MphfServer, key_sets, arrivals, seeds=None) -> list[Result]:
    """Submit request i at server time arrivals[i] (seconds from now) and wait
    for all of them.  Returns the results in request order."""
    base = server.now()
    for i, (keys, t) in enumerate(zip(key_sets, arrivals)):
        delay = base + t - server.now()
        if delay > 0:
            time.sleep(delay)
        server.submit(Request(i, keys, 1 if seeds is None else int(seeds[i]),
                              arrival=server.now()))
    server.wait(len(key_sets))
    return [server.results[i] for i in range(len(key_sets))]


def latency_summary(results) -> dict:
    lat = np.array([r.latency for r in results if r.error is None])
    keys = sum(r.n for r in results if r.error is None)
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    return {"requests": len(results), "failed": sum(r.error is not None for r in results),
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "keys_per_s": keys / span if span > 0 else None,
            "retried": sum(1 for r in results if r.stats.get("attempts", 1) > 1)}
