"""Reader for the hand-derived fixtures in tests/golden/."""
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
UNCLAIMED = 0xFFFFFFFF


def load(name):
    fields = {"edge": []}
    with open(os.path.join(GOLDEN_DIR, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, _, val = line.partition(":")
            key, val = key.strip(), val.strip()
            if key == "edge":
                fields["edge"].append([int(t) for t in val.split()])
            else:
                fields[key] = val
    r, P = int(fields["r"]), int(fields["P"])
    g = {"r": r, "P": P, "m": r * P,
         "edges": np.array(fields["edge"], dtype=np.uint32).reshape(-1, r)}
    g["order"] = np.array([int(t) for t in fields["order"].split()], dtype=np.uint32)
    claim = []
    for tok in fields["claim"].split():
        if tok == "-":
            claim.append(UNCLAIMED)
        else:
            t, h = tok.split(":")
            claim.append((int(t) << 2) | int(h))
    g["claim"] = np.array(claim, dtype=np.uint32)
    g["layer_off"] = np.array([int(t) for t in fields["layer_off"].split()], dtype=np.uint64)
    g["n_peeled"] = int(fields["n_peeled"])
    if "g" in fields:
        g["g"] = {int(a): int(b) for a, b in (t.split("=") for t in fields["g"].split())}
    if "rank" in fields:
        g["rank"] = [int(t) for t in fields["rank"].split()]
    return g


def all_names():
    return sorted(f for f in os.listdir(GOLDEN_DIR) if f.endswith(".txt") and f != "README.txt")
