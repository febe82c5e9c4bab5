"""Continuous-batching MPHF build server.

Requests (a key set and a hash seed) arrive over time.  A request is
admitted as soon as a slot is free *and* its device-memory footprint fits the
remaining budget, so requests that arrive while others are on the GPU start
without waiting for a batch to drain; admitted builds run concurrently, one
CUDA stream per slot, and overlap on the device.  Each slot keeps its
workspace between requests (grown when a larger request needs more), and
the built function (g values and rank directory) stays on the device.  A
build whose hypergraph keeps a 2-core is retried with the next hash seeds
(inside hpeel_mphf_build).  Latency is measured from a request's arrival to
its completion.

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

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def footprint_bytes(n: int, gamma_milli: int = 1230) -> int:
    """Device bytes one build holds: workspace, keys, g values, rank directory."""
    m = num_vertices(n, gamma_milli, 3)
    return (mphf_workspace_size(n, gamma_milli) + 8 * n + 8 * ((m + 31) // 32)
            + 8 * ((m + 511) // 512 + 1))


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
        self.in_use = 0
        self.max_in_use = 0   # largest admitted footprint total seen
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
    def _take(self):
        """Under the lock: the first pending request that fits the budget
        (first come first served, smaller requests may pass a large one that
        does not fit yet)."""
        for i, req in enumerate(self.pending):
            if self.in_use + req.footprint <= self.budget:
                del self.pending[i]
                self.in_use += req.footprint
                self.running += 1
                self.max_in_use = max(self.max_in_use, self.in_use)
                self.max_running = max(self.max_running, self.running)
                return req
        return None

    def _worker(self, slot: int):
        torch = self.torch
        stream = torch.cuda.Stream(device=self.device)
        ws = None
        while True:
            with self.cv:
                req = None
                while not self.stop:
                    req = self._take()
                    if req is not None:
                        break
                    self.cv.wait()
                if req is None:
                    return
                admitted = self.now()
            n = int(req.keys.shape[0])
            res = Result(req.rid, n, num_vertices(n, self.gamma, 3), arrival=req.arrival,
                         admitted=admitted)
            try:
                with torch.cuda.device(self.device), torch.cuda.stream(stream):
                    need = mphf_workspace_size(n, self.gamma)
                    if ws is None or ws.numel() < need:
                        ws = None
                        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=self.device)
                    keys = req.keys
                    if not (isinstance(keys, torch.Tensor) and keys.is_cuda):
                        if isinstance(keys, np.ndarray):
                            keys = torch.from_numpy(keys.view(np.int64))
                        keys = keys.to(self.device, non_blocking=True)
                    out = mphf_build(keys, req.seed, self.gamma, self.max_tries, workspace=ws)
                    res.G, res.rank_dir, res.stats = (out.G, out.rank_dir, out.stats) \
                        if self.keep else (None, None, out.stats)
            except Exception as exc:  # a failed build is reported, not raised
                res.error = str(exc)
            res.finished = self.now()
            with self.cv:
                self.in_use -= req.footprint
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
