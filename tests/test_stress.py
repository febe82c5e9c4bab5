"""Full-size parity: n = 1e9 (gamma 1.23, 1.222, 1.20) and r = 4, n = 1e8,
gamma 1.30, in the launch configuration bench.py uses.

The oracle's complete outputs for these workloads were computed once by
tests/golden/make_stress_digests.py (oracle/ only) and stored as SHA-256
digests of the arrays plus the layer sizes; here the GPU outputs are
digested the same way.  A digest match means the arrays are equal bit for
bit.  Each case holds tens of GB on the device and takes about a minute.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1312_0526_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import paper_1312_0526_gb300 as hp  # noqa: E402

DIGESTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                       "stress_digests.json")


def _load():
    if not os.path.exists(DIGESTS):
        return {}
    with open(DIGESTS) as f:
        return json.load(f)


CASES = _load()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_0526_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _digest_dev(t) -> str:
    """SHA-256 of a device tensor's bytes, copied to the host in slices."""
    h = hashlib.sha256()
    flat = t.reshape(-1).view(torch.uint8)
    step = 1 << 30
    for i in range(0, flat.numel(), step):
        h.update(flat[i:i + step].cpu().numpy().tobytes())
    return h.hexdigest()


@pytest.mark.parametrize("name", sorted(CASES))
def test_full_size_parity(name):
    c = CASES[name]
    n, g, r, m = c["n"], c["gamma_milli"], c["r"], c["m"]
    assert hp.num_vertices(n, g, r) == m
    torch.cuda.empty_cache()
    keys = torch.from_numpy(inputs.keys(n, c["key_seed"]).view(np.int64)).cuda()
    edges = hp.hash_edges(keys, m, r, c["hash_seed"])
    assert _digest_dev(edges) == c["edges_sha256"]
    res = hp.peel(edges, m, max_layers=1 << 16)
    assert res.rounds == c["rounds"] and res.n_peeled == c["n_peeled"]
    sizes = np.diff(res.layer_off.cpu().numpy().astype(np.int64)).tolist()
    assert sizes == c["layer_sizes"]
    assert _digest_dev(res.order) == c["order_sha256"]
    assert _digest_dev(res.claim) == c["claim_sha256"]
    del edges, res
    torch.cuda.empty_cache()
    if "G_sha256" in c:
        got = hp.mphf_build(keys, seed=c["hash_seed"], gamma_milli=g)
        assert got.stats["seed_used"] == c["hash_seed"]
        assert _digest_dev(got.G) == c["G_sha256"]
        assert _digest_dev(got.rank_dir) == c["rank_dir_sha256"]
    del keys
    torch.cuda.empty_cache()
