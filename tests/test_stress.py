"""Full-size parity: n = 1e9 (gamma 1.23, 1.222, 1.20) and r = 4, n = 1e8,
gamma 1.30, in the launch configuration bench.py uses; and the batched
workload (65,536 lognormal buckets, about 2e8 keys) with the autotuned launch
shape, once called directly and once replayed from a captured CUDA graph.

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


CASES = {k: v for k, v in _load().items() if "n" in v}
BATCHED_CASES = {k: v for k, v in _load().items() if "B" in v}


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
    keys = inputs.keys_torch(n, c["key_seed"])
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


def test_full_size_parity_one_part_per_pass():
    # the same n = 1e9 workload with the incidence build run one part per
    # pass (the mode graphs of more than 2^30 edges take by default)
    c = CASES.get("n1e9_g1230_r3")
    if c is None:
        pytest.skip("no digests")
    n, g, r, m = c["n"], c["gamma_milli"], c["r"], c["m"]
    torch.cuda.empty_cache()
    hp.set_tuning(bucket_part_passes=2)
    try:
        keys = inputs.keys_torch(n, c["key_seed"])
        edges = hp.hash_edges(keys, m, r, c["hash_seed"])
        res = hp.peel(edges, m, max_layers=1 << 16)
        assert res.rounds == c["rounds"] and res.n_peeled == c["n_peeled"]
        assert _digest_dev(res.order) == c["order_sha256"]
        assert _digest_dev(res.claim) == c["claim_sha256"]
        del edges, res
        torch.cuda.empty_cache()
        if "G_sha256" in c:
            got = hp.mphf_build(keys, seed=c["hash_seed"], gamma_milli=g)
            assert _digest_dev(got.G) == c["G_sha256"]
            assert _digest_dev(got.rank_dir) == c["rank_dir_sha256"]
            del got
        del keys
    finally:
        hp.set_tuning()
        torch.cuda.empty_cache()


def test_largest_mphf_on_one_gpu():
    # n = 3.4e9 keys: m = 4,182,000,000 vertices, just below the 2^32 vertex
    # ids of the ABI; the build runs one part per pass (automatic above 2^30
    # edges).  No oracle output exists at this size: the properties checked
    # are the ones any size must have -- every key peeled, and the lookups of
    # all keys a bijection onto [0, n).
    n = 3_400_000_000
    m = hp.num_vertices(n)
    assert m < 2**32
    free, total = torch.cuda.mem_get_info()
    need = 8 * n + hp.mphf_workspace_size(n) + (m // 4) + (8 << 30)
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    torch.cuda.empty_cache()
    keys = inputs.keys_torch(n, 21)
    ws = torch.empty(hp.mphf_workspace_size(n), dtype=torch.uint8, device="cuda")
    got = hp.mphf_build(keys, seed=1, max_tries=4, workspace=ws)
    del ws
    torch.cuda.empty_cache()
    assert got.stats["n_peeled"] == n and got.stats["core_nonempty"] == 0
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    step = 1 << 28
    out = torch.empty(step, dtype=torch.int32, device="cuda")
    for a in range(0, n, step):
        b = min(n, a + step)
        hp.mphf_lookup(keys[a:b], got.stats["seed_used"], m, got.G, got.rank_dir,
                       out=out[:b - a])
        idx = out[:b - a].to(torch.int64) & 0xFFFFFFFF
        assert bool((idx < n).all())  # checked before it indexes anything
        flags.index_fill_(0, idx, 1)
    assert int(flags.sum(dtype=torch.int64)) == n
    del keys, flags, out, got
    torch.cuda.empty_cache()


def _batched_digests(res):
    return {"order_sha256": _digest_dev(res.order), "rounds_sha256": _digest_dev(res.rounds),
            "status_sha256": _digest_dev(res.status), "G_sha256": _digest_dev(res.G)}


@pytest.mark.parametrize("name", sorted(BATCHED_CASES))
def test_batched_full_size_parity(name):
    from paper_1312_0526_gb300 import autotune
    c = BATCHED_CASES[name]
    g = c["gamma_milli"]
    sizes = inputs.lognormal_bucket_sizes(c["B"], median=c["median"], sigma=c["sigma"],
                                          lo=c["lo"], hi=c["hi"], seed=c["size_seed"])
    keys, off = inputs.bucketed_keys(sizes, seed=c["key_seed"])
    assert int(off[-1]) == c["total_keys"]
    torch.cuda.empty_cache()
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    do = torch.from_numpy(off.view(np.int64)).cuda()
    tun = autotune.tune(dk, do, g, with_g=True)
    ws = torch.empty(hp.batched_workspace_size(c["B"], g, tun), dtype=torch.uint8,
                     device="cuda")
    res = hp.peel_batched(dk, do, g, with_g=True, tuning=tun, workspace=ws)
    torch.cuda.synchronize()
    want = {k: c[k] for k in ("order_sha256", "rounds_sha256", "status_sha256", "G_sha256")}
    assert _batched_digests(res) == want
    assert int((res.status == 1).sum()) == c["buckets_with_core"]
    # the same launch captured into a CUDA graph and replayed into cleared
    # outputs
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            hp.peel_batched(dk, do, g, tuning=tun, workspace=ws, out=res)
    torch.cuda.synchronize()
    for t in (res.order, res.rounds, res.status):
        t.fill_(-1)
    res.G.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    assert _batched_digests(res) == want
    del dk, do, ws, res, graph
    torch.cuda.empty_cache()


def test_large_path_matches_the_1e9_digests():
    # the MPHF build beyond 32-bit ids, on the n = 1e9 workload: g values and
    # rank directory equal the oracle's (its digests), the layer list once in
    # device memory and once in pinned host memory
    c = CASES.get("n1e9_g1230_r3")
    if c is None or "G_sha256" not in c:
        pytest.skip("no digests")
    n, g = c["n"], c["gamma_milli"]
    torch.cuda.empty_cache()
    keys = inputs.keys_torch(n, c["key_seed"])
    for on_host in (False, True):
        hl = torch.empty(n, dtype=torch.int64, pin_memory=True) if on_host else None
        got = hp.mphf_build_large(keys, seed=c["hash_seed"], gamma_milli=g, host_list=hl)
        assert got.stats["seed_used"] == c["hash_seed"] and got.stats["rounds"] == c["rounds"]
        assert _digest_dev(got.G) == c["G_sha256"]
        assert _digest_dev(got.rank_dir) == c["rank_dir_sha256"]
        del got, hl
        torch.cuda.empty_cache()
    del keys
    torch.cuda.empty_cache()


def test_large_path_5e9_keys_layer_list_on_host():
    # beyond the 32-bit ids: n = 5e9 keys (m = 6.15e9 vertices), the layer
    # list in pinned host memory.  No oracle output exists at this size: every
    # key must peel and the lookups of all keys must be a bijection onto [0, n)
    n = 5_000_000_000
    m = hp.num_vertices(n)
    free, total = torch.cuda.mem_get_info()
    need = 8 * n + hp.mphf_large_workspace_size(n, 1230, True) + m // 4 + n + (8 << 30)
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    torch.cuda.empty_cache()
    keys = inputs.keys_torch(n, 23)
    hl = torch.empty(n, dtype=torch.int64, pin_memory=True)
    got = hp.mphf_build_large(keys, seed=1, max_tries=4, host_list=hl)
    del hl
    assert got.stats["n_peeled"] == n and got.stats["core_nonempty"] == 0
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    step = 1 << 28
    out = torch.empty(step, dtype=torch.int64, device="cuda")
    for a in range(0, n, step):
        b = min(n, a + step)
        hp.mphf_lookup_large(keys[a:b], got.stats["seed_used"], m, got.G, got.rank_dir,
                             out=out[:b - a])
        idx = out[:b - a]
        assert bool(((idx >= 0) & (idx < n)).all())  # checked before it indexes anything
        flags.index_fill_(0, idx, 1)
    assert int(flags.sum(dtype=torch.int64)) == n
    del keys, flags, out, got
    torch.cuda.empty_cache()
