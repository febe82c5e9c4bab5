"""Writes tests/golden/stress_digests.json: the oracle's results on the large
workloads (n = 1e9 at gamma 1.23, 1.222, 1.20; r = 4, n = 1e8, gamma 1.30),
stored as SHA-256 digests of the output arrays plus the layer sizes, so the
GPU test can compare full outputs without running the oracle for minutes.

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


def run(name):
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
    for name in names or list(CONFIGS):
        print("running", name, flush=True)
        data[name] = run(name)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        print(name, {k: v for k, v in data[name].items() if k != "layer_sizes"}, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
