#!/usr/bin/env python3
"""Benchmark of the GB300 hypergraph peeling hot path.

One step = one whole pass of the hot path over one hypergraph: the plain
peel (hpeel_peel) of the n = 1e9, r = 3, gamma = 1.23 workload -- edge
records and packed incidence build, round-synchronous peel, canonical order,
claim words and layer offsets out -- with the edges (hashed from SplitMix64
keys, seed 1, hash seed 1) resident in device memory.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--legs LIST] [--n N]

The line also carries the end-to-end figure (edges from pinned host memory,
order and claims back to it, every step), the CPU oracle on a sample, and the
other workloads as sub-legs (--legs picks them; "none" times the step alone,
e.g. under a profiler): the n = 1e8 MPHF build, lookups, the device-driven
forms, the stress configurations (n = 1e9 at gamma 1.222 and 1.20, r = 4),
the batched form, serving, static functions, general hypergraphs and the
random-access ceiling of the rounds.

N > 1 runs under torch.distributed.run, one rank per GPU: every rank peels
its own independent hypergraph (key seed 1 + rank) -- weak scaling, no
collective on the data path; a barrier and a max-reduction of the timings
only.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEEL_N = 10**9                 # the headline: plain peel of 1e9 edges
MPHF_N = 10**8                 # the MPHF build leg
GAMMA_MILLI = 1230
R = 3
KEY_SEED = 1
HASH_SEED = 1
METRIC = "peeled edges/sec (Medges/s)"
UNIT = "Medges/s"
CPU_SAMPLE_EDGES = 10**7       # cpu_baseline: one oracle peel of this many edges
REF_STEP_EDGES = 2 * 10**6     # --impl reference: edges per oracle step
ALL_LEGS = ("e2e", "cpu", "mphf", "lookup", "async", "peel_async", "stress", "batched",
            "serving", "sf", "general", "random_access", "large")
LARGE_N = 7_600_000_000        # the paper's largest key set (sec. 5: 7.6e9 n-grams)

# Algorithmic bytes per unit of work, per step of the path (r = 3).  "sector"
# charges one 32-byte sector per random access (64 bytes for a read-modify-
# write), "word" charges only the bytes the method reads and writes.  Units:
# edges (hash, build, extract, emit, assign), vertices (fill), peeled edges
# (rounds).  Every peeled edge is appended to the layer list once (16 B) and
# read back once by the round that deletes it, which updates its r-1 other
# vertices; a vertex that falls to degree 1 marks its record and claims its
# last edge (one random read-modify-write; the mark and the read of the
# claimed edge's vertices hit the sectors those atomics just fetched).
def byte_model(step, n, m, st):
    L0, peeled = st["first_layer"], st["n_peeled"]
    cross, moves = st["frontier"], st["hinge_moves"]
    if step == "hash_bucket":
        # key read, edge record write, r incidences written to the buckets
        w = (8 + 16 + R * 8) * n
        return {"units": n, "word": w, "sector": w}
    if step == "apply_buckets":
        # refine: incidences read, written to their sub-buckets; apply: read
        # again, accumulated in shared memory, each vertex record written once
        w = 3 * R * 8 * n + 8 * m
        return {"units": n, "word": w, "sector": w}
    if step == "hash_edges":
        return {"units": n, "word": 24 * n, "sector": 24 * n}
    if step == "records_bucket":
        # edge rows read, edge record write, r incidences written to the buckets
        w = (4 * R + 16 + R * 8) * n
        return {"units": n, "word": w, "sector": w}
    if step == "fill":
        return {"units": m, "word": 8 * m, "sector": 8 * m}
    if step == "build_incidence":
        return {"units": n, "word": (16 + R * 16) * n, "sector": (16 + R * 64) * n}
    if step == "rounds":
        # round 0: scan of the vertex records, mark + claim per degree-1
        # vertex; then per peeled edge: entry append and read, r-1 DeleteEdge
        # atomics; per fall to degree 1: mark, claim, vertex read; per moved
        # hinge: entry rewrite
        word = (8 * m + L0 * (8 + 8 + 16) + peeled * (32 + (R - 1) * 16)
                + cross * (4 + 8 + 16) + 16 * moves)
        sector = (8 * m + L0 * (32 + 64) + peeled * (32 + (R - 1) * 64)
                  + cross * 64 + 16 * moves)
        return {"units": peeled, "word": word, "sector": sector}
    if step == "extract_claim":
        # edge records read, claims written (the first pass's counts are
        # taken on the way)
        return {"units": n, "word": 20 * n, "sector": 20 * n}
    if step == "emit_scatter":
        return {"units": n, "word": 12 * n, "sector": 12 * n}
    if step == "emit_hist":
        return {"units": n, "word": 4 * n, "sector": 4 * n}
    if step == "assign":
        # entry stream, two g reads and one g update per edge (G is L2-resident)
        return {"units": n, "word": (16 + 2 * 8 + 16) * n, "sector": (16 + 2 * 32 + 64) * n}
    return None


# DRAM bytes per unit measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# for a kernel version, keyed by the sha256 of the source files its kernels
# live in; stale entries are ignored.  Filled from the summaries in profiles/.
NCU_TRAFFIC = {
    # step: (source files, sha256 prefix, bytes per unit, where measured)
    "rounds": (("paper_1312_0526_gb300/csrc/peel.cu",
                "paper_1312_0526_gb300/csrc/rounds_bucketed.cu",
                "paper_1312_0526_gb300/csrc/build.cu"), "9df1550ecb748c40", 339.63,
               "every round kernel (sorted round 0 and L_0..L_2, random k_round) of one peel at "
               "n = 3e7 (host round loop), scaled by peeled edges"),
}


def src_hash(rels):
    h = hashlib.sha256()
    for rel in rels:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x: float, dist=None, device="cpu") -> float:
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_medges(n_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank peels its own n-edge hypergraph."""
    return n_per_rank * world / (ms / 1e3) / 1e6


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_cpu():
    """Core count and CPU model of the host the CPU legs run on."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if model and not model.isdigit():
                    break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def cpu_baseline():
    """The oracle, as it stands, on a bounded sample of the workload: the
    first 1e7 keys of the same stream hashed (r = 3, gamma = 1.23, hash seed
    1) and peeled round by round with the canonical order, single-threaded.
    Beside it the paper's in-memory baseline form: the greedy LIFO peel with
    the XOR trick ("Standard+XOR"), hashing included."""
    import oracle
    from paper_1312_0526_gb300 import inputs
    oracle.build()
    n = CPU_SAMPLE_EDGES
    keys = inputs.keys(n, KEY_SEED)
    m = oracle.num_vertices(n, GAMMA_MILLI, R)
    t0 = time.perf_counter()
    res = oracle.peel_rounds(oracle.hash_edges(keys, m, R, HASH_SEED), m)
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    oracle.peel_greedy(oracle.hash_edges(keys, m, R, HASH_SEED), m)
    dg = time.perf_counter() - t1
    hc = host_cpu()
    return {"value": n / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one single-threaded oracle peel (hash + round-synchronous peel + "
                      f"canonical order) of the first {n:.0e} edges of the same workload, "
                      f"{dt:.2f} s, {res.rounds} rounds; host {hc['nproc']} cores, "
                      f"{hc['model']}",
            "host": hc,
            "greedy_peel": {"value": n / dg / 1e6, "unit": UNIT,
                            "sample": f"hash + greedy LIFO peel of the same edges, {dg:.2f} s"}}


def roofline_of(prof, steps, n, m, st, round_loop):
    """Roofline of the step with the largest live CUDA-event total."""
    peak, peak_kind = measured_peaks()
    prof = dict(prof)
    # the host loop times round 0, the sorted rounds and the random rounds
    # apart; the byte model covers all of them, as the graph loop's one scope
    for part in ("round0", "rounds_sorted"):
        if part in prof and "rounds" in prof:
            c, t = prof.pop(part)[:2]
            prof["rounds"] = [prof["rounds"][0] + c, prof["rounds"][1] + t]
    ranked = sorted(((v[1], k) for k, v in prof.items()), reverse=True)
    for tot_ms, name in ranked:
        model = byte_model(name, n, m, st)
        if model is None:
            continue
        per_step_ms = tot_ms / steps
        launches_per_step = prof[name][0] / steps
        if name == "rounds" and round_loop == "graph":
            # one launch of the CUDA graph that holds round 0 and both loops
            # of rounds (sorted, random); its kernels run back to back
            launches_per_step = 1
        achieved = model["sector"] / (per_step_ms / 1e3) / 1e9
        traffic = traffic_step = source = None
        if name in NCU_TRAFFIC:
            src, h, per_unit, where = NCU_TRAFFIC[name]
            if src_hash(src) == h:
                traffic_step = per_unit * model["units"]
                traffic = traffic_step / max(launches_per_step, 1)
                source = f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {where}"
        return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "model": "sector", "peak_kind": peak_kind,
                "algorithmic_bytes_per_step": model["sector"],
                "units_per_step": model["units"],
                "word_model_gbs": model["word"] / (per_step_ms / 1e3) / 1e9,
                "launches_per_step": launches_per_step,
                "traffic_per_step": traffic_step,
                "traffic_gbs": traffic_step / (per_step_ms / 1e3) / 1e9 if traffic_step else None,
                "traffic_source": source,
                "ms_per_step": per_step_ms,
                "share": tot_ms / sum(v[1] for v in prof.values())}
    return None


def peel_e2e(edges, m, ws, ref, steps, sync_all, max_over_ranks):
    """The headline through the public API with host buffers: every step's
    edges (12 B per edge) come from pinned host memory and its order and
    claim words (8 B per edge) go back to pinned host memory.  A copy stream
    moves step i+1's edges into one of two device buffers while step i
    peels (a buffer is refilled only after the peel that read it); the
    results go back on another stream into double host buffers."""
    import torch

    import paper_1312_0526_gb300 as hp

    n = edges.shape[0]
    stream = torch.cuda.current_stream()
    edges_h = torch.empty(edges.shape, dtype=edges.dtype, pin_memory=True)
    edges_h.copy_(edges)
    ed = [edges, torch.empty_like(edges)]
    outs = [(torch.empty(n, dtype=torch.int32, device="cuda"),
             torch.empty(n, dtype=torch.int32, device="cuda"),
             torch.empty(4097, dtype=torch.int64, device="cuda")) for _ in range(2)]
    host = [(torch.empty(n, dtype=torch.int32, pin_memory=True),
             torch.empty(n, dtype=torch.int32, pin_memory=True)) for _ in range(2)]
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    read, built_ev, copied = [None, None], [None, None], [None, None]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def enqueue_copy(i):
        b = i & 1
        with torch.cuda.stream(h2d):
            h2d.wait_event(e0)
            if built_ev[b] is not None:
                h2d.wait_event(built_ev[b])
            ed[b].copy_(edges_h, non_blocking=True)
            copied[b] = torch.cuda.Event()
            copied[b].record(h2d)

    sync_all()
    e0.record(stream)
    enqueue_copy(0)
    for i in range(steps):
        b = i & 1
        # the peel call returns when its step is done, so the next step's
        # copy is queued first and runs while this one peels
        if i + 1 < steps:
            enqueue_copy(i + 1)
        stream.wait_event(copied[b])
        if read[b] is not None:
            stream.wait_event(read[b])  # step i-2's results are on the host
        hp.peel(ed[b], m, workspace=ws, out=outs[b])
        built = torch.cuda.Event()
        built.record(stream)
        built_ev[b] = built
        with torch.cuda.stream(d2h):
            d2h.wait_event(built)
            host[b][0].copy_(outs[b][0], non_blocking=True)
            host[b][1].copy_(outs[b][1], non_blocking=True)
            read[b] = torch.cuda.Event()
            read[b].record(d2h)
    stream.wait_stream(d2h)
    stream.wait_stream(h2d)
    e1.record(stream)
    sync_all()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps)
    ro, rc = ref[0].cpu(), ref[1].cpu()
    same = all(torch.equal(host[b][0], ro) and torch.equal(host[b][1], rc)
               for b in range(min(2, steps)))
    del ed[1], outs, host, edges_h
    torch.cuda.empty_cache()
    return ms, same


def mphf_leg(n, steps, warmup, rank):
    """The MWHC MPHF build (hpeel_mphf_build: hash, incidence, peel,
    canonical order, g assignment, rank directory) of n = 1e8 keys, keys
    device-resident; and end to end with each step's keys
    copied from pinned host memory (double-buffered on a copy stream) and
    the g values and rank directory read back."""
    import numpy as np
    import torch

    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import inputs

    m = hp.num_vertices(n, GAMMA_MILLI, R)
    keys_h = torch.from_numpy(inputs.keys(n, KEY_SEED + rank).view(np.int64)).pin_memory()
    keys = keys_h.to("cuda", non_blocking=False)
    ws = torch.empty(hp.mphf_workspace_size(n, GAMMA_MILLI), dtype=torch.uint8, device="cuda")
    G = torch.empty((m + 31) // 32, dtype=torch.int64, device="cuda")
    D = torch.empty((m + 511) // 512 + 1, dtype=torch.int64, device="cuda")
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(src, g, d):
        return hp.mphf_build(src, HASH_SEED, GAMMA_MILLI, workspace=ws, G=g, rank_dir=d,
                             order=order)

    for _ in range(max(warmup, 1)):
        res = step(keys, G, D)
    torch.cuda.synchronize()
    hp.profile_reset()
    hp.profile_enable(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        res = step(keys, G, D)
    b.record(stream)
    torch.cuda.synchronize()
    hp.profile_enable(False)
    prof = hp.profile_read()
    ms = a.elapsed_time(b) / steps
    # end to end: keys from pinned host memory, results back to it
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    Gb, Db = [G, torch.empty_like(G)], [D, torch.empty_like(D)]
    G_h = [torch.empty_like(G, device="cpu").pin_memory() for _ in range(2)]
    D_h = [torch.empty_like(D, device="cpu").pin_memory() for _ in range(2)]
    kd = [keys, torch.empty_like(keys)]
    read, built_ev, copied = [None, None], [None, None], [None, None]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def enqueue_copy(i):
        bb = i & 1
        with torch.cuda.stream(h2d):
            h2d.wait_event(e0)
            if built_ev[bb] is not None:
                h2d.wait_event(built_ev[bb])
            kd[bb].copy_(keys_h, non_blocking=True)
            copied[bb] = torch.cuda.Event()
            copied[bb].record(h2d)

    torch.cuda.synchronize()
    e0.record(stream)
    enqueue_copy(0)
    for i in range(steps):
        bb = i & 1
        if i + 1 < steps:
            enqueue_copy(i + 1)
        stream.wait_event(copied[bb])
        if read[bb] is not None:
            stream.wait_event(read[bb])
        step(kd[bb], Gb[bb], Db[bb])
        built = torch.cuda.Event()
        built.record(stream)
        built_ev[bb] = built
        with torch.cuda.stream(d2h):
            d2h.wait_event(built)
            G_h[bb].copy_(Gb[bb], non_blocking=True)
            D_h[bb].copy_(Db[bb], non_blocking=True)
            read[bb] = torch.cuda.Event()
            read[bb].record(d2h)
    stream.wait_stream(d2h)
    stream.wait_stream(h2d)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / steps
    same = all(torch.equal(G_h[x], G.cpu()) and torch.equal(D_h[x], D.cpu())
               for x in range(min(2, steps)))
    del kd, ws, order, Gb, Db
    torch.cuda.empty_cache()
    st = res.stats
    out = {"value": n / ms / 1e3, "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "rounds": st["rounds"], "seed_used": st["seed_used"],
           "steps_ms": {k: v[1] / steps for k, v in sorted(prof.items())},
           "roofline": roofline_of(prof, steps, n, m, st, "graph"),
           "e2e": {"value": n / e2e_ms / 1e3, "unit": UNIT, "ms_per_step": e2e_ms,
                   "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * (G.numel() + D.numel()),
                   "same_as_device_resident": same},
           "config": {"workload": f"mphf-build n={n:.0e} r=3 gamma=1.23, SplitMix64 keys seed "
                                  "1+rank, hash seed 1 (hash, incidence, peel, canonical "
                                  "order, g assignment, rank)"}}
    return out, keys, G, D, m, st["seed_used"]


def stress_leg(steps=2, warmup=1):
    """The other plain-peel stress configurations: n =
    1e9 at gamma 1.222 (near the threshold, many rounds) and 1.20 (below it:
    a 2-core is left), and r = 4 at n = 1e8, gamma 1.30; hpeel_peel from
    device-resident edges."""
    import torch

    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import inputs

    out = {}
    for name, n, g, r in (("n1e9_g1222", 10**9, 1222, 3), ("n1e9_g1200", 10**9, 1200, 3),
                          ("n1e8_g1300_r4", 10**8, 1300, 4)):
        m = hp.num_vertices(n, g, r)
        keys = inputs.keys_torch(n, KEY_SEED)
        edges = hp.hash_edges(keys, m, r, HASH_SEED)
        del keys
        torch.cuda.empty_cache()
        ws = torch.empty(hp.peel_workspace_size(n, m, r), dtype=torch.uint8, device="cuda")
        po = (torch.empty(n, dtype=torch.int32, device="cuda"),
              torch.empty(n, dtype=torch.int32, device="cuda"),
              torch.empty(1 << 16 | 1, dtype=torch.int64, device="cuda"))
        for _ in range(warmup):
            res = hp.peel(edges, m, workspace=ws, max_layers=1 << 16, out=po)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            res = hp.peel(edges, m, workspace=ws, max_layers=1 << 16, out=po)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[name] = {"value": n / ms / 1e3, "unit": UNIT, "ms_per_step": ms, "steps": steps,
                     "n": n, "gamma": g / 1000, "r": r, "rounds": res.rounds,
                     "n_peeled": res.n_peeled, "core_nonempty": res.core_nonempty}
        del edges, ws, po, res
        torch.cuda.empty_cache()
    return out


def peel_async_leg(edges, m, ws, ref, steps=5, warmup=2):
    """The headline peel through hpeel_peel_async (one cached CUDA graph, the
    rounds and the order sort's passes driven by the device, no host
    synchronisation), on the same edges and workspace; outputs checked equal
    to hpeel_peel's."""
    import torch

    import paper_1312_0526_gb300 as hp

    out = hp.peel_async(edges, m, workspace=ws)
    for _ in range(warmup - 1):
        hp.peel_async(edges, m, workspace=ws, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        hp.peel_async(edges, m, workspace=ws, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    st = hp.stats_from_device(out.stats)
    same = bool(torch.equal(out.order, ref[0]) and torch.equal(out.claim, ref[1]))
    n = edges.shape[0]
    del out
    torch.cuda.empty_cache()
    return {"value": n / ms / 1e3, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "async_status": st["async_status"], "rounds": st["rounds"],
            "same_as_hpeel_peel": same}


def lookup_leg(keys, G, D, m, seed):
    """MPHF lookups of the n build keys (hpeel_mphf_lookup), and the space of
    the built function."""
    import torch

    import paper_1312_0526_gb300 as hp

    out = torch.empty(keys.shape[0], dtype=torch.int32, device="cuda")
    hp.mphf_lookup(keys, seed, m, G, D, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    a.record()
    for _ in range(reps):
        hp.mphf_lookup(keys, seed, m, G, D, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    n = keys.shape[0]
    ok = bool(torch.equal(torch.sort(out)[0], torch.arange(n, dtype=torch.int32, device="cuda")))
    return {"value": n / ms / 1e3, "unit": "Mlookups/s", "ms": ms, "bijection": ok,
            "bits_per_key": hp.mphf_bits_per_key(n, GAMMA_MILLI)}


def random_access_leg(n, m, rounds_ms):
    """The random-access ceiling the rounds run against: random 64-bit atomics,
    random 8-byte loads and the access pattern of one peeled edge (a record
    claim and two vertex updates), over arrays the size of the build's edge
    records (n x 16 B) and vertex records (m x 8 B), timed with CUDA events
    (the measurement library's probe, measure/probe.cu)."""
    import torch

    from paper_1312_0526_gb300 import measure

    A = torch.zeros(n * 2, dtype=torch.int64, device="cuda")
    B = torch.zeros(m, dtype=torch.int64, device="cuda")
    out = {}
    # the loads run first, while the vertex words are still zero
    for kind, name, arg_b in ((1, "load64", None), (0, "rmw64", None), (2, "peeled_edge", B)):
        target = A if kind == 2 else B
        measure.random_access(kind, n, target, arg_b, seed=7)  # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        torch.cuda.synchronize()
        a.record()
        for r in range(reps):
            measure.random_access(kind, n, target, arg_b, seed=100 + r)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        out[name] = {"g_per_s": n / ms / 1e6, "ms": ms}
    del A, B
    torch.cuda.empty_cache()
    rounds_g = n / rounds_ms / 1e6
    out["rounds_g_edges_per_s"] = rounds_g
    out["rounds_vs_peeled_edge_pattern"] = rounds_g / out["peeled_edge"]["g_per_s"]
    out["arrays"] = (f"rmw64 and load64 over the vertex-record size ({m * 8 / 1e9:.2f} GB); "
                     f"peeled_edge: records {n * 16 / 1e9:.2f} GB + vertex words "
                     f"{m * 8 / 1e9:.2f} GB; {n:.0e} operations each")
    return out


SF_SIGMA = 256


def sf_leg(n, steps, warmup):
    """Static function (sec. 3, f: S -> [sigma]) of the n = 1e8 keys with
    sigma = 256 (8-bit values, uniform from SplitMix64 stream seed 5):
    hpeel_sf_build per step, keys and values device-resident; every key is
    looked up afterwards and must return its value."""
    import numpy as np
    import torch

    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import inputs

    keys = torch.from_numpy(inputs.keys(n, KEY_SEED).view(np.int64)).cuda()
    vals = torch.from_numpy((inputs.keys(n, 5) % np.uint64(SF_SIGMA)).astype(np.uint32)
                            .view(np.int32)).cuda()
    ws = torch.empty(hp.sf_workspace_size(n, GAMMA_MILLI), dtype=torch.uint8, device="cuda")
    res = None
    for _ in range(max(warmup, 1)):
        res = hp.sf_build(keys, vals, SF_SIGMA, HASH_SEED, GAMMA_MILLI, workspace=ws)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        res = hp.sf_build(keys, vals, SF_SIGMA, HASH_SEED, GAMMA_MILLI, workspace=ws,
                          U=res.U)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    out = hp.sf_lookup(keys, res.stats["seed_used"], res.m, SF_SIGMA, res.U)
    ok = bool(torch.equal(out, vals))
    r = {"value": n / ms / 1e3, "unit": "Mkeys/s", "ms_per_step": ms, "steps": steps,
         "sigma": SF_SIGMA, "bits_per_vertex": res.bits,
         "bits_per_key": res.bits * res.m / n, "every_key_maps_to_its_value": ok,
         "config": {"workload": f"static function n={n:.0e} sigma={SF_SIGMA} gamma=1.23 "
                                "(hash, incidence, peel, assignment mod sigma)"}}
    del keys, vals, ws, res, out
    torch.cuda.empty_cache()
    return r


def general_leg(n, steps, warmup):
    """Peel of a general (not r-partite) 3-hypergraph (hpeel_peel_general):
    n = 1e8 edges on m = ceil(1.23 n) vertices, vertex j of key k = mix64(k ^
    (1 + j)) mod m (any vertex in any position, repeats possible), edges
    device-resident, canonical order + claims + layer offsets out."""
    import numpy as np
    import torch

    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import inputs

    m = (n * GAMMA_MILLI + 999) // 1000
    keys = torch.from_numpy(inputs.keys(n, KEY_SEED).view(np.int64)).cuda()
    edges = hp.hash_edges(keys, m, R, HASH_SEED, general=True)
    del keys
    ws = torch.empty(hp.peel_workspace_size(n, m, R, general=True), dtype=torch.uint8,
                     device="cuda")
    res = None
    for _ in range(max(warmup, 1)):
        res = hp.peel(edges, m, workspace=ws, general=True)
    torch.cuda.synchronize()
    hp.profile_reset()
    hp.profile_enable(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        res = hp.peel(edges, m, workspace=ws, general=True)
    b.record()
    torch.cuda.synchronize()
    hp.profile_enable(False)
    prof = hp.profile_read()
    ms = a.elapsed_time(b) / steps
    out = {"value": n / ms / 1e3, "unit": UNIT, "ms_per_step": ms, "steps": steps, "n": n,
           "m": m, "rounds": res.rounds, "n_peeled": res.n_peeled,
           "steps_ms": {k: v[1] / steps for k, v in sorted(prof.items())},
           "config": {"workload": f"general 3-hypergraph peel n={n:.0e} m=ceil(1.23 n), "
                                  "edges on the device"}}
    del edges, ws, res
    torch.cuda.empty_cache()
    return out


def async_leg(keys, G_ref, D_ref, steps=5, warmup=2):
    """The device-driven MPHF build (hpeel_mphf_build_async: reseed loop,
    rounds and assignment as conditional nodes of one CUDA graph, no host
    synchronisation; no canonical order output) on the same keys, timed with
    CUDA events; G and rank directory checked equal to the host-driven build."""
    import torch

    import paper_1312_0526_gb300 as hp

    n = keys.shape[0]
    ws = torch.empty(hp.mphf_workspace_size(n, GAMMA_MILLI), dtype=torch.uint8, device="cuda")
    G, D, st = hp.mphf_build_async(keys, HASH_SEED, GAMMA_MILLI, workspace=ws)
    for _ in range(warmup - 1):
        hp.mphf_build_async(keys, HASH_SEED, GAMMA_MILLI, workspace=ws, G=G, rank_dir=D, stats=st)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        hp.mphf_build_async(keys, HASH_SEED, GAMMA_MILLI, workspace=ws, G=G, rank_dir=D, stats=st)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    stats = hp.stats_from_device(st)
    same = bool(torch.equal(G, G_ref) and torch.equal(D, D_ref))
    # two builds in flight: each of two streams has its own workspace and
    # outputs, and the builds alternate between them; one build's bandwidth-
    # bound passes run while the other's short rounds leave the GPU idle
    ws2 = torch.empty_like(ws)
    G2, D2, st2 = hp.mphf_build_async(keys, HASH_SEED, GAMMA_MILLI, workspace=ws2)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [(ws, G, D, st), (ws2, G2, D2, st2)]
    torch.cuda.synchronize()
    for i in range(2):  # warm-up of both graphs on their streams
        with torch.cuda.stream(streams[i]):
            w, g_, d_, s_ = outs[i]
            hp.mphf_build_async(keys, HASH_SEED, GAMMA_MILLI, workspace=w, G=g_, rank_dir=d_,
                                stats=s_)
    torch.cuda.synchronize()
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    a2.record(cur)
    for sm in streams:
        sm.wait_stream(cur)
    for i in range(2 * steps):
        with torch.cuda.stream(streams[i & 1]):
            w, g_, d_, s_ = outs[i & 1]
            hp.mphf_build_async(keys, HASH_SEED, GAMMA_MILLI, workspace=w, G=g_, rank_dir=d_,
                                stats=s_)
    for sm in streams:
        cur.wait_stream(sm)
    b2.record(cur)
    torch.cuda.synchronize()
    ms2 = a2.elapsed_time(b2) / (2 * steps)
    same2 = bool(torch.equal(G2, G_ref) and torch.equal(D2, D_ref) and torch.equal(G, G_ref))
    del ws, G, D, st, ws2, G2, D2, st2
    torch.cuda.empty_cache()
    return {"value": n / ms / 1e3, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "two_in_flight": {"value": n / ms2 / 1e3, "unit": UNIT, "ms_per_build": ms2,
                              "builds": 2 * steps, "same_as_host_driven": same2},
            "async_status": stats["async_status"], "seed_used": stats["seed_used"],
            "rounds": stats["rounds"], "same_as_host_driven": same,
            "config": {"workload": f"mphf-build n={n:.0e} r=3 gamma=1.23, device-driven (one "
                                   "CUDA graph per build, no host synchronisation), no "
                                   "canonical order"}}


MAX_N = 3_400_000_000


def max_scale_leg(steps=2, warmup=1):
    """The largest MPHF one GB300 builds: n = 3.4e9 keys (m = 4,182,000,000
    vertices, just below the 2^32 vertex ids of the ABI), keys on the device,
    the incidence build one part per pass.  Every key must peel and the
    lookups of all keys must be a bijection onto [0, n) (checked)."""
    import torch

    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import inputs

    n = MAX_N
    m = hp.num_vertices(n, GAMMA_MILLI, R)
    torch.cuda.empty_cache()
    keys = inputs.keys_torch(n, KEY_SEED)
    wsb = hp.mphf_workspace_size(n, GAMMA_MILLI)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    G = torch.empty((m + 31) // 32, dtype=torch.int64, device="cuda")
    D = torch.empty((m + 511) // 512 + 1, dtype=torch.int64, device="cuda")
    res = None
    for _ in range(warmup):
        res = hp.mphf_build(keys, HASH_SEED, GAMMA_MILLI, workspace=ws, G=G, rank_dir=D)
    torch.cuda.synchronize()
    hp.profile_reset()
    hp.profile_enable(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        res = hp.mphf_build(keys, HASH_SEED, GAMMA_MILLI, workspace=ws, G=G, rank_dir=D)
    b.record()
    torch.cuda.synchronize()
    hp.profile_enable(False)
    prof = hp.profile_read()
    ms = a.elapsed_time(b) / steps
    del ws
    torch.cuda.empty_cache()
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    step = 1 << 28
    out = torch.empty(step, dtype=torch.int32, device="cuda")
    ok = True
    for lo in range(0, n, step):
        hi = min(n, lo + step)
        hp.mphf_lookup(keys[lo:hi], res.stats["seed_used"], m, G, D, out=out[:hi - lo])
        idx = out[:hi - lo].to(torch.int64) & 0xFFFFFFFF
        if not bool((idx < n).all()):
            ok = False
            break
        flags.index_fill_(0, idx, 1)
    ok = ok and int(flags.sum(dtype=torch.int64)) == n
    del keys, flags, out, G, D
    torch.cuda.empty_cache()
    return {"value": n / ms / 1e3, "unit": "Mkeys/s", "ms_per_step": ms, "steps": steps,
            "n": n, "m": m, "rounds": res.stats["rounds"], "n_peeled": res.stats["n_peeled"],
            "workspace_gb": wsb / 1e9, "workspace_bytes_per_key": wsb / n,
            "lookup_bijection": ok,
            "steps_ms": {k: v[1] / steps for k, v in sorted(prof.items())},
            "config": {"workload": f"mphf-build n={n:.2e} r=3 gamma=1.23, keys on the device "
                                   f"(SplitMix64 seed {KEY_SEED}), incidence build one part "
                                   f"per pass"}}


def large_leg(n=LARGE_N, steps=2, warmup=1):
    """The MPHF of the paper's largest key set, 7.6e9 keys (sec. 5), on one
    GB300 through hpeel_mphf_build_large (64-bit ids, edges re-hashed from
    the keys), the layer list in pinned host memory; every key must peel and
    the lookups of all keys must be a bijection onto [0, n) (checked)."""
    import torch

    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import inputs

    m = hp.num_vertices(n, GAMMA_MILLI, R)
    torch.cuda.empty_cache()
    keys = inputs.keys_torch(n, KEY_SEED)
    wsb = hp.mphf_large_workspace_size(n, GAMMA_MILLI, True)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    hl = torch.empty(n, dtype=torch.int64, pin_memory=True)
    G = torch.empty((m + 31) // 32, dtype=torch.int64, device="cuda")
    D = torch.empty((m + 511) // 512 + 1, dtype=torch.int64, device="cuda")
    res = None
    for _ in range(warmup):
        res = hp.mphf_build_large(keys, HASH_SEED, GAMMA_MILLI, workspace=ws, G=G, rank_dir=D,
                                  host_list=hl)
    torch.cuda.synchronize()
    hp.profile_reset()
    hp.profile_enable(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        res = hp.mphf_build_large(keys, HASH_SEED, GAMMA_MILLI, workspace=ws, G=G, rank_dir=D,
                                  host_list=hl)
    b.record()
    torch.cuda.synchronize()
    hp.profile_enable(False)
    prof = hp.profile_read()
    ms = a.elapsed_time(b) / steps
    del ws, hl
    torch.cuda.empty_cache()
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    step = 1 << 28
    out = torch.empty(step, dtype=torch.int64, device="cuda")
    ok = True
    for lo in range(0, n, step):
        hi = min(n, lo + step)
        hp.mphf_lookup_large(keys[lo:hi], res.stats["seed_used"], m, G, D, out=out[:hi - lo])
        idx = out[:hi - lo]
        if not bool(((idx >= 0) & (idx < n)).all()):
            ok = False
            break
        flags.index_fill_(0, idx, 1)
    ok = ok and int(flags.sum(dtype=torch.int64)) == n
    del keys, flags, out, G, D
    torch.cuda.empty_cache()
    return {"value": n / ms / 1e3, "unit": "Mkeys/s", "ms_per_step": ms, "steps": steps,
            "n": n, "m": m, "rounds": res.stats["rounds"], "n_peeled": res.stats["n_peeled"],
            "seed_used": res.stats["seed_used"], "workspace_gb": wsb / 1e9,
            "host_list_gb": 8 * n / 1e9, "lookup_bijection": ok,
            "steps_ms": {k: v[1] / steps for k, v in sorted(prof.items())},
            "config": {"workload": f"mphf-build n={n:.2e} r=3 gamma=1.23 (the paper's 7.6e9-key "
                                   f"set, sec. 5), 64-bit ids, keys on the device (SplitMix64 "
                                   f"seed {KEY_SEED}), layer list in pinned host memory"}}


BATCH_B = 65536


def batched_leg(steps, warmup):
    """Batched form (65,536 lognormal buckets, median 2,000 keys, 64..65,536,
    hash seed = bucket id): one persistent launch per step, autotuned launch
    shape, replayed from a captured CUDA graph; beside it the plain path over
    the same keys taken as one hypergraph."""
    import numpy as np
    import torch

    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import autotune, inputs

    sizes = inputs.lognormal_bucket_sizes(BATCH_B, median=2000, sigma=0.92, lo=64, hi=65536,
                                          seed=3)
    keys, off = inputs.bucketed_keys(sizes, seed=2)
    total = int(off[-1])
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    do = torch.from_numpy(off.view(np.int64)).cuda()
    out = {}
    for with_g in (False, True):
        tun = autotune.tune(dk, do, GAMMA_MILLI, with_g=with_g)
        ws = torch.empty(hp.batched_workspace_size(BATCH_B, GAMMA_MILLI, tun), dtype=torch.uint8,
                         device="cuda")
        res = hp.peel_batched(dk, do, GAMMA_MILLI, with_g=with_g, tuning=tun, workspace=ws)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s):
                hp.peel_batched(dk, do, GAMMA_MILLI, tuning=tun, workspace=ws, out=res)
        torch.cuda.synchronize()
        for _ in range(max(warmup, 1)):
            graph.replay()
        torch.cuda.synchronize()
        l0 = hp.kernel_launches()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            graph.replay()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        st = res.status.cpu().numpy()
        out["with_g" if with_g else "peel"] = {
            "value": total / ms / 1e3, "unit": UNIT, "ms_per_step": ms, "tuning": tun,
            "buckets_peeled": int((st == 0).sum()), "buckets_with_core": int((st == 1).sum()),
            "graph_replays": steps, "hbm_gbs_context": total * (8 + 4) / ms / 1e6}
    # the plain path on the same keys as one hypergraph of all 2.01e8 edges
    # (hash seed 1, gamma 1.23): hpeel_hash_edges + hpeel_peel per step
    m = hp.num_vertices(total, GAMMA_MILLI, 3)
    del ws
    torch.cuda.empty_cache()
    pws = torch.empty(hp.peel_workspace_size(total, m, 3), dtype=torch.uint8, device="cuda")
    edges = torch.empty((total, 3), dtype=torch.int32, device="cuda")
    pout = (torch.empty(total, dtype=torch.int32, device="cuda"),
            torch.empty(total, dtype=torch.int32, device="cuda"),
            torch.empty(4097, dtype=torch.int64, device="cuda"))
    for _ in range(max(warmup, 1)):
        hp.hash_edges(dk, m, 3, HASH_SEED, out=edges)
        hp.peel(edges, m, workspace=pws, out=pout)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        hp.hash_edges(dk, m, 3, HASH_SEED, out=edges)
        hp.peel(edges, m, workspace=pws, out=pout)
    b.record()
    torch.cuda.synchronize()
    pms = a.elapsed_time(b) / steps
    out["plain_one_graph"] = {"value": total / pms / 1e3, "unit": UNIT, "ms_per_step": pms,
                              "steps": steps,
                              "workload": f"the same {total} keys as one 3-hypergraph (hash "
                                          "seed 1, gamma 1.23): hpeel_hash_edges + hpeel_peel"}
    out["speedup_vs_plain"] = out["peel"]["value"] / out["plain_one_graph"]["value"]
    del pws, edges, pout
    torch.cuda.empty_cache()
    out["config"] = {"workload": "65,536 bucket 3-hypergraphs, lognormal sizes (median 2,000, "
                                 "sigma 0.92, clipped 64..65,536), gamma 1.23, hash seed = "
                                 "bucket id, SplitMix64 keys seed 2",
                     "total_edges": total}
    return out


SERVE_REQUESTS = 200


def serving_leg():
    """Serving: MPHF build requests with Poisson arrivals, key-set sizes
    log-uniform 1e3..1e7 (SplitMix64 keys, seed 1000 + request), gamma 1.23;
    4 slots, 32 GiB admission budget, keys uploaded from pinned host memory
    inside each request's latency.  The arrival rate is swept as a fraction
    of the capacity measured with one slot and every request queued at once."""
    import numpy as np
    import torch

    from paper_1312_0526_gb300 import inputs, serve

    unit_arrivals, sizes, seeds = inputs.request_stream(SERVE_REQUESTS, rate_per_s=1.0, seed=4)
    keysets = [torch.from_numpy(inputs.keys(int(s), int(k)).view(np.int64)).pin_memory()
               for s, k in zip(sizes, seeds)]
    srv = serve.MphfServer(slots=1, hbm_budget=32 << 30, keep_results=False, max_tries=32)
    try:
        serve.run_stream(srv, keysets[:8], [0.0] * 8)  # warm-up (workspace, graphs)
        srv.results.clear()
        res = serve.run_stream(srv, keysets, [0.0] * len(keysets))
    finally:
        srv.close()
    span = max(r.finished for r in res) - min(r.arrival for r in res)
    capacity = len(res) / span
    out = {"requests": SERVE_REQUESTS, "mean_keys": float(np.mean(sizes)),
           "capacity_req_per_s": capacity, "isolated": serve.latency_summary(res), "rates": []}
    for frac in (0.25, 0.5, 0.75, 0.9, 1.1):
        rate = frac * capacity
        srv = serve.MphfServer(slots=4, hbm_budget=32 << 30, keep_results=False,
                               max_tries=32)
        try:
            res = serve.run_stream(srv, keysets, list(unit_arrivals / rate))
            summ = serve.latency_summary(res)
            summ.update({"load": frac, "rate_req_per_s": rate,
                         "max_concurrent": srv.max_running})
            out["rates"].append(summ)
        finally:
            srv.close()
    return out


def run_reference(args, world, rank):
    """The oracle (there is no reference code to install: the paper ships
    none), timed as it stands on the host cores: each step hashes and peels
    (round-synchronous, canonical order) the first 2e6 edges of the same
    workload."""
    if rank != 0:
        return 0
    import oracle
    from paper_1312_0526_gb300 import inputs
    oracle.build()
    n = REF_STEP_EDGES
    keys = inputs.keys(n, KEY_SEED)
    m = oracle.num_vertices(n, GAMMA_MILLI, R)

    def step():
        oracle.peel_rounds(oracle.hash_edges(keys, m, R, HASH_SEED), m)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = n / dt / 1e6
    hc = host_cpu()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"plain peel r=3 gamma=1.23, SplitMix64 keys seed 1, hash "
                               f"seed 1; oracle steps on the first {n:.0e} edges",
                   "n": PEEL_N, "gamma": GAMMA_MILLI / 1000, "r": R},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step one single-threaded oracle hash + round-"
                                   f"synchronous peel with canonical order of {n:.0e} edges; "
                                   f"host {hc['nproc']} cores, {hc['model']}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched_shape_call(shape: str):
    """The batched workload with one fixed launch shape ("THREADSxCTAS", no
    autotuning, no g values): one warm-up and one timed call -- a short,
    fixed launch sequence for a profiler.  Prints its own small JSON line."""
    import numpy as np
    import torch

    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import inputs

    t, c = (int(x) for x in shape.split("x"))
    tun = {"threads": t, "ctas_per_sm": c}
    sizes = inputs.lognormal_bucket_sizes(BATCH_B, median=2000, sigma=0.92, lo=64, hi=65536,
                                          seed=3)
    keys, off = inputs.bucketed_keys(sizes, seed=2)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    do = torch.from_numpy(off.view(np.int64)).cuda()
    ws = torch.empty(hp.batched_workspace_size(BATCH_B, GAMMA_MILLI, tun), dtype=torch.uint8,
                     device="cuda")
    res = hp.peel_batched(dk, do, GAMMA_MILLI, tuning=tun, workspace=ws)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    hp.peel_batched(dk, do, GAMMA_MILLI, tuning=tun, workspace=ws, out=res)
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"batched_ms": a.elapsed_time(b), "tuning": tun, "edges": int(off[-1])}),
          flush=True)


def summary_of(line):
    """The headline figures of every leg in one small object, placed last in
    the line so that a truncated copy of the line still shows them."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or d.get(k) is None:
                return None
            d = d[k]
        return round(d, 3) if isinstance(d, float) else d
    s = {"peel_1e9_ms": g(line, "ms_per_step"), "peel_1e9_medges_s": g(line, "value"),
         "peel_1e9_e2e_ms": g(line, "e2e", "ms_per_step"),
         "rounds_ms": g(line, "roofline", "ms_per_step"),
         "rounds_frac_sector_model": g(line, "roofline", "frac"),
         "rounds_vs_random_access_ceiling": g(line, "roofline", "random_access_ceiling", "frac"),
         "peel_async_ms": g(line, "peel_async", "ms_per_step"),
         "mphf_1e8_ms": g(line, "mphf_1e8", "ms_per_step"),
         "mphf_1e8_e2e_ms": g(line, "mphf_1e8", "e2e", "ms_per_step"),
         "mphf_1e8_device_driven_ms": g(line, "device_driven", "ms_per_step"),
         "lookup_mlookups_s": g(line, "lookup", "value"),
         "batched_ms": g(line, "batched", "peel", "ms_per_step"),
         "batched_medges_s": g(line, "batched", "peel", "value"),
         "batched_with_g_ms": g(line, "batched", "with_g", "ms_per_step"),
         "batched_plain_one_graph_ms": g(line, "batched", "plain_one_graph", "ms_per_step"),
         "batched_vs_plain": g(line, "batched", "speedup_vs_plain"),
         "serving_capacity_req_s": g(line, "serving", "capacity_req_per_s"),
         "sf_1e8_ms": g(line, "static_function", "ms_per_step"),
         "general_1e8_ms": g(line, "general_peel", "ms_per_step"),
         "cpu_oracle_medges_s": g(line, "cpu_baseline", "value"),
         "large_7_6e9_mphf_s": (round(line["large_7_6e9"]["ms_per_step"] / 1e3, 3)
                                if line.get("large_7_6e9") else None),
         "large_7_6e9_bijection": g(line, "large_7_6e9", "lookup_bijection")}
    for name in ("n1e9_g1222", "n1e9_g1200", "n1e8_g1300_r4"):
        s[f"stress_{name}_ms"] = g(line, "stress", name, "ms_per_step")
    rates = g(line, "serving", "rates") or []
    s["serving_p50_p99_ms_by_load"] = [[r.get("load"), round(r.get("p50_ms") or 0, 2),
                                        round(r.get("p99_ms") or 0, 2)] for r in rates]
    return s


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=PEEL_N,
                    help="edges of the headline peel (smaller cases for profilers)")
    ap.add_argument("--legs", default="all",
                    help="comma-separated sub-legs to run besides the timed step: "
                         + ",".join(ALL_LEGS) + "; 'all' (default) or 'none'")
    ap.add_argument("--max-scale", action="store_true",
                    help="also build the largest MPHF one GB300 holds (n = 3.4e9)")
    ap.add_argument("--round-loop", default="graph", choices=["graph", "host"],
                    help="graph: rounds in a CUDA graph (default); host: one launch per round "
                         "(same kernels; for profilers that cannot see inside the graph)")
    ap.add_argument("--batched-shape", default=None,
                    help="THREADSxCTAS: only one call of the batched form with this launch "
                         "shape (a fixed launch sequence for a profiler)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    legs = (set(ALL_LEGS) if args.legs == "all"
            else {x for x in args.legs.split(",") if x and x != "none"})
    unknown = legs - set(ALL_LEGS)
    if unknown:
        raise SystemExit(f"unknown legs: {sorted(unknown)}")

    import torch
    import paper_1312_0526_gb300 as hp
    from paper_1312_0526_gb300 import build as hpbuild
    from paper_1312_0526_gb300 import inputs

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if dist.is_nccl_available() else "gloo")
    if rank == 0:
        hpbuild.build()
    if dist:
        dist.barrier()
    hp.lib()
    if args.batched_shape:
        batched_shape_call(args.batched_shape)
        return 0
    if args.round_loop == "host":
        hp.set_tuning(host_round_loop=1)

    def sync_all():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, dist, "cuda" if dist and dist.get_backend() == "nccl" else "cpu")

    # ---- the headline: plain peel of n edges, edges device-resident
    n = args.n
    m = hp.num_vertices(n, GAMMA_MILLI, R)
    keys = inputs.keys_torch(n, KEY_SEED + rank)
    edges = hp.hash_edges(keys, m, R, HASH_SEED)
    del keys
    torch.cuda.empty_cache()
    ws = torch.empty(hp.peel_workspace_size(n, m, R), dtype=torch.uint8, device="cuda")
    out = (torch.empty(n, dtype=torch.int32, device="cuda"),
           torch.empty(n, dtype=torch.int32, device="cuda"),
           torch.empty(4097, dtype=torch.int64, device="cuda"))
    stream = torch.cuda.current_stream()

    def step():
        return hp.peel(edges, m, workspace=ws, out=out)

    for _ in range(max(args.warmup, 0)):
        res = step()
    sync_all()
    hp.profile_reset()
    hp.profile_enable(True)
    l0 = hp.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        sync_all()
        ev0.record(stream)
        for _ in range(args.steps):
            res = step()
        ev1.record(stream)
        sync_all()
    launches = hp.kernel_launches() - l0
    hp.profile_enable(False)
    prof = hp.profile_read()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    st = dict(res.stats)
    value = aggregate_medges(n, world, ms)
    roof = roofline_of(prof, args.steps, n, m, st, args.round_loop)
    ref = (out[0].clone(), out[1].clone())

    e2e = None
    if "e2e" in legs:
        e2e_steps = max(1, min(args.steps, 30))  # the copy pipeline fills once per run
        e2e_ms, same = peel_e2e(edges, m, ws, ref, e2e_steps, sync_all, max_over_ranks)
        e2e = {"value": aggregate_medges(n, world, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": 4 * R * n, "d2h_bytes_per_step": 8 * n,
               "ms_per_step": e2e_ms, "steps": e2e_steps, "same_as_device_resident": same,
               "copies": "every step's edges (12 B each) copied from pinned host memory into "
                         "one of two device buffers on a copy stream while the previous step "
                         "peels (the first copy is not overlapped); order and claim words "
                         "(8 B per edge) copied back to pinned host buffers on a second stream"}
    peel_async = None
    if "peel_async" in legs and world == 1:
        peel_async = peel_async_leg(edges, m, ws, ref)
    del edges, ws, out, ref
    torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = cpu_baseline() if world == 1 and "cpu" in legs else None
    mphf = lookup = device_driven = None
    if world == 1 and "mphf" in legs:
        mphf, mkeys, G, D, mm, seed_used = mphf_leg(MPHF_N, args.steps, args.warmup, rank)
        if "lookup" in legs:
            lookup = lookup_leg(mkeys, G, D, mm, seed_used)
        if "async" in legs:
            device_driven = async_leg(mkeys, G, D)
        del mkeys, G, D
        torch.cuda.empty_cache()
    stress = stress_leg() if world == 1 and "stress" in legs else None
    batched = batched_leg(args.steps, args.warmup) if world == 1 and "batched" in legs else None
    serving = serving_leg() if world == 1 and "serving" in legs else None
    sf = sf_leg(MPHF_N, steps=3, warmup=1) if world == 1 and "sf" in legs else None
    general = general_leg(MPHF_N, steps=3, warmup=1) if world == 1 and "general" in legs else None
    random_access = None
    if world == 1 and "random_access" in legs and "rounds" in prof:
        random_access = random_access_leg(n, m, prof["rounds"][1] / args.steps)
        if roof is not None and roof["kernel"] == "rounds":
            # the rounds against the rate the memory system serves their own
            # access pattern alone (one record claim + two vertex updates per
            # peeled edge), next to the copy-bandwidth fraction
            roof["random_access_ceiling"] = {
                "g_edges_per_s": random_access["peeled_edge"]["g_per_s"],
                "achieved_g_edges_per_s": random_access["rounds_g_edges_per_s"],
                "frac": random_access["rounds_vs_peeled_edge_pattern"],
                "source": "random_access leg (measurement library probe, kind 2)"}
    max_scale = max_scale_leg() if world == 1 and args.max_scale else None
    large = large_leg() if world == 1 and "large" in legs else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"plain peel n={n:.0e} r=3 gamma=1.23, edges hashed from "
                               f"SplitMix64 keys seed 1+rank with hash seed 1, device-resident; "
                               f"records + incidence build, round-synchronous peel, canonical "
                               f"order + claim words + layer offsets out (hpeel_peel)",
                   "n": n, "m": m, "gamma": GAMMA_MILLI / 1000, "r": R,
                   "parallelism": f"{world} independent hypergraphs (one per GPU)",
                   "l2": f"inputs larger than L2: {12 * n / 1e9:.1f} GB edges, "
                         f"{8 * m / 1e9:.1f} GB vertex records, {16 * n / 1e9:.1f} GB edge "
                         f"records per step"},
        "stats": {k: st[k] for k in ("rounds", "n_peeled", "core_nonempty", "first_layer",
                                     "frontier", "hinge_moves")},
        "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "clocks": clk.summary(),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "steps_ms": {k: v[1] / args.steps for k, v in sorted(prof.items())},
        "peel_async": peel_async,
        "mphf_1e8": mphf,
        "lookup": lookup,
        "device_driven": device_driven,
        "stress": stress,
        "batched": batched,
        "serving": serving,
        "static_function": sf,
        "general_peel": general,
        "random_access": random_access,
        "max_scale": max_scale,
        "large_7_6e9": large,
    }
    line["summary"] = summary_of(line)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
