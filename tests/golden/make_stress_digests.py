"""Writes tests/golden/stress_digests.json: the oracle's results on the large
workloads (n = 1e9 at gamma 1.23, 1.222, 1.20; r = 4, n = 1e8, gamma 1.30;
the batched workload of 65,536 lognormal buckets, about 2e8 keys), stored as
SHA-256 digests of the output arrays plus the layer sizes, so the GPU test
can compare full outputs without running the oracle for minutes.

Calls only the oracle (oracle/) and the seeded input generator.  Run once:
    python tests/golden/make_stress_digests.py [name ...]
It needs about 55 GB of host memory for the n = 1e9 workloads.
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1312_0526_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "stress_digests.json")

CONFIGS = {
    "n1e9_g1230_r3": (10**9, 1230, 3, True),
    "n1e9_g1222_r3": (10**9, 1222, 3, False),
    "n1e9_g1200_r3": (10**9, 1200, 3, False),
    "n1e8_g1300_r4": (10**8, 1300, 4, False),
}


def digest(a: np.ndarray) -> str:
    h = hashlib.sha256()
    mv = memoryview(np.ascontiguousarray(a)).cast("B")
    step = 1 << 28
    for i in range(0, len(mv), step):
        h.update(mv[i:i + step])
    return h.hexdigest()


# The batched workload (sec. 3 "Practical workarounds (HEM)": one small MWHC
# hypergraph per bucket): 65,536 buckets of clip(round(exp(ln 2000 + 0.92 Z)),
# 64, 65,536) keys (Z from SplitMix64 stream 3), keys from stream 2 cut into
# consecutive buckets, bucket b hashed with seed b at gamma 1.23.
BATCHED = {"batched_65536": (65536, 2000, 0.92, 64, 65536, 3, 2, 1230)}


def run_batched(name):
    B, median, sigma, lo, hi, size_seed, key_seed, g = BATCHED[name]
    t0 = time.time()
    sizes = inputs.lognormal_bucket_sizes(B, median=median, sigma=sigma, lo=lo, hi=hi,
                                          seed=size_seed)
    keys, off = inputs.bucketed_keys(sizes, seed=key_seed)
    h_order, h_g = hashlib.sha256(), hashlib.sha256()
    rounds = np.zeros(B, dtype=np.uint32)
    status = np.zeros(B, dtype=np.uint32)
    for b in range(B):
        k = keys[int(off[b]):int(off[b + 1])]
        m = oracle.num_vertices(len(k), g, 3)
        e = oracle.hash_edges(k, m, 3, b)
        res = oracle.peel_rounds(e, m)
        rounds[b] = res.rounds
        status[b] = 1 if res.core_nonempty else 0
        h_order.update(np.ascontiguousarray(res.order, dtype=np.uint32).tobytes())
        # g values of the bucket (all zero when it keeps a 2-core), in the
        # layout of the MPHF's G: ceil(m / 32) words per bucket, concatenated
        G = (oracle.mphf_assign(e, m, res) if not res.core_nonempty
             else np.zeros((m + 31) // 32, dtype=np.uint64))
        h_g.update(np.ascontiguousarray(G, dtype=np.uint64).tobytes())
    return {"B": B, "median": median, "sigma": sigma, "lo": lo, "hi": hi,
            "size_seed": size_seed, "key_seed": key_seed, "gamma_milli": g,
            "total_keys": int(off[-1]), "buckets_with_core": int(status.sum()),
            "order_sha256": h_order.hexdigest(), "rounds_sha256": digest(rounds),
            "status_sha256": digest(status), "G_sha256": h_g.hexdigest(),
            "max_rounds": int(rounds.max()), "oracle_seconds": round(time.time() - t0, 1)}


def run(name):
    if name in BATCHED:
        return run_batched(name)
    n, g, r, mphf = CONFIGS[name]
    t0 = time.time()
    keys = inputs.keys(n, 1)
    m = oracle.num_vertices(n, g, r)
    edges = oracle.hash_edges(keys, m, r, 1)
    del keys
    res = oracle.peel_rounds(edges, m)
    rec = {"n": n, "gamma_milli": g, "r": r, "m": m, "hash_seed": 1, "key_seed": 1,
           "rounds": res.rounds, "n_peeled": res.n_peeled,
           "layer_sizes": np.diff(res.layer_off.astype(np.int64)).tolist(),
           "order_sha256": digest(res.order), "claim_sha256": digest(res.claim),
           "edges_sha256": digest(edges)}
    if mphf and not res.core_nonempty:
        G = oracle.mphf_assign(edges, m, res)
        rec["G_sha256"] = digest(G)
        rec["rank_dir_sha256"] = digest(oracle.rank_dir(G, m))
    rec["oracle_seconds"] = round(time.time() - t0, 1)
    return rec


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names or list(CONFIGS) + list(BATCHED):
        print("running", name, flush=True)
        data[name] = run(name)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        print(name, {k: v for k, v in data[name].items() if k != "layer_sizes"}, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
