"""Device-driven MPHF build (hpeel_mphf_build_async): the reseed loop, the
rounds and the reverse-layer assignment as conditional nodes of one CUDA
graph.  Its output is compared with the host-driven build and the oracle,
element by element (bit-exact: all integer work)."""
import numpy as np
import pytest

import oracle
from paper_1312_0526_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1312_0526_gb300 as hp  # noqa: E402

ASYNC_PEELED, ASYNC_EXHAUSTED = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_0526_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a.view(np.int64))).cuda()


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _same_as_host_build(keys_np, max_tries=32, seed=1):
    k = _dev(keys_np)
    want = hp.mphf_build(k, seed=seed, max_tries=max_tries)
    G, D, st = hp.mphf_build_async(k, seed=seed, max_tries=max_tries)
    torch.cuda.synchronize()
    got = hp.stats_from_device(st)
    assert got["async_status"] == ASYNC_PEELED
    # (hinge_moves is left out: how often a later claim lowers a hinge
    # depends on the order the claims arrive in, not on the result)
    for f in ("seed_used", "attempts", "rounds", "n_peeled", "first_layer", "frontier"):
        assert got[f] == want.stats[f], f
    assert got["core_nonempty"] == 0 and got["device_err"] == 0
    assert torch.equal(G, want.G) and torch.equal(D, want.rank_dir)
    return got, G, D


@pytest.mark.parametrize("n", [1, 3, 17, 1000, 4097, 100_000, 250_000])
def test_async_equals_host_build(n):
    keys = inputs.keys(n, 1)
    got, G, D = _same_as_host_build(keys)
    want = oracle.mphf_build(keys, seed=1, max_tries=32)
    assert got["seed_used"] == want.seed_used
    assert np.array_equal(_u64(G), want.G) and np.array_equal(_u64(D), want.dir)


def test_async_reseeds_on_the_device():
    # key sets whose first seed leaves a 2-core: the retry loop runs inside
    # the graph and lands on the oracle's seed
    found = 0
    for s in range(300):
        k = inputs.keys(60, 2000 + s)
        m = oracle.num_vertices(60, 1230, 3)
        if oracle.peel_rounds(oracle.hash_edges(k, m, 3, 1), m).core_nonempty:
            want = oracle.mphf_build(k, seed=1, max_tries=64)
            G, D, st = hp.mphf_build_async(_dev(k), seed=1, max_tries=64)
            got = hp.stats_from_device(st)
            assert got["async_status"] == ASYNC_PEELED
            assert got["seed_used"] == want.seed_used > 1
            assert got["attempts"] == want.seed_used
            assert np.array_equal(_u64(G), want.G) and np.array_equal(_u64(D), want.dir)
            found += 1
            if found == 3:
                break
    assert found == 3


def test_async_retries_exhausted_leaves_G_untouched():
    keys = np.array([5, 5, 6, 7], dtype=np.uint64)
    m = hp.num_vertices(4)
    G = torch.full((max((m + 31) // 32, 1),), 0x1234, dtype=torch.int64, device="cuda")
    G0 = G.clone()
    _, _, st = hp.mphf_build_async(_dev(keys), seed=9, max_tries=3, G=G)
    got = hp.stats_from_device(st)
    assert got["async_status"] == ASYNC_EXHAUSTED
    assert got["core_nonempty"] == 1 and got["attempts"] == 3 and got["seed_used"] == 0
    assert got["n_peeled"] < 4
    assert torch.equal(G, G0)


def test_async_empty_input():
    G, D, st = hp.mphf_build_async(torch.empty(0, dtype=torch.int64, device="cuda"), seed=4)
    got = hp.stats_from_device(st)
    assert got["async_status"] == ASYNC_PEELED and got["seed_used"] == 4
    assert int(D[0]) == 0


@pytest.fixture
def small_buckets():
    hp.set_tuning(bucket_shift=10, bucket_min_vertices=0)
    yield
    hp.set_tuning()


@pytest.mark.parametrize("n", [100_000, 250_001])
def test_async_equals_host_build_bucketed(small_buckets, n):
    _same_as_host_build(inputs.keys(n, 5))


def test_async_bucket_overflow_redone_direct(small_buckets):
    # 90,000 copies of one key put all their incidences in three buckets and
    # overflow both the buckets and the overflow list; the graph's if-node
    # redoes the build with direct updates (no device error) and the peel of
    # every seed stops at the duplicates' 2-core, where the oracle stops
    base = inputs.keys(10_000, 10)
    keys = np.concatenate([base, np.full(90_000, base[0], dtype=np.uint64)])
    n = keys.shape[0]
    m = oracle.num_vertices(n, 1230, 3)
    _, _, st = hp.mphf_build_async(_dev(keys), seed=3, max_tries=2)
    got = hp.stats_from_device(st)
    assert got["async_status"] == ASYNC_EXHAUSTED and got["device_err"] == 0
    assert got["attempts"] == 2
    want = oracle.peel_rounds(oracle.hash_edges(keys, m, 3, 4), m)
    assert got["n_peeled"] == want.n_peeled < n
    assert got["rounds"] == want.rounds


def test_async_graph_replayed_with_new_key_contents():
    # the cached graph is keyed by pointers: new contents in the same buffers
    # give the new build
    n = 50_000
    k = _dev(inputs.keys(n, 21))
    ws = torch.empty(hp.mphf_workspace_size(n), dtype=torch.uint8, device="cuda")
    G, D, st = hp.mphf_build_async(k, seed=1, max_tries=32, workspace=ws)
    for s in (22, 23):
        k.copy_(_dev(inputs.keys(n, s)))
        hp.mphf_build_async(k, seed=1, max_tries=32, workspace=ws, G=G, rank_dir=D, stats=st)
        want = oracle.mphf_build(inputs.keys(n, s), seed=1, max_tries=32)
        got = hp.stats_from_device(st)
        assert got["seed_used"] == want.seed_used
        assert np.array_equal(_u64(G), want.G) and np.array_equal(_u64(D), want.dir)


def test_async_captured_into_a_torch_graph():
    # the build's conditional nodes join a graph the caller captures; each
    # replay rebuilds from the keys' current contents
    n = 30_000
    k = _dev(inputs.keys(n, 31))
    ws = torch.empty(hp.mphf_workspace_size(n), dtype=torch.uint8, device="cuda")
    G, D, st = hp.mphf_build_async(k, seed=1, max_tries=32, workspace=ws)  # warm-up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        hp.mphf_build_async(k, seed=1, max_tries=32, workspace=ws, G=G, rank_dir=D, stats=st)
    for s in (32, 33):
        k.copy_(_dev(inputs.keys(n, s)))
        g.replay()
        torch.cuda.synchronize()
        want = oracle.mphf_build(inputs.keys(n, s), seed=1, max_tries=32)
        got = hp.stats_from_device(st)
        assert got["async_status"] == ASYNC_PEELED and got["seed_used"] == want.seed_used
        assert np.array_equal(_u64(G), want.G) and np.array_equal(_u64(D), want.dir)


def test_async_lookup_after_build_is_a_bijection():
    n = 200_000
    k = _dev(inputs.keys(n, 41))
    G, D, st = hp.mphf_build_async(k, seed=1, max_tries=32)
    got = hp.stats_from_device(st)
    h = hp.mphf_lookup(k, got["seed_used"], hp.num_vertices(n), G, D)
    v = torch.sort(h.to(torch.int64)).values.cpu().numpy()
    assert np.array_equal(v, np.arange(n))
