"""Device-driven peel and static-function build (hpeel_peel_async,
hpeel_peel_general_async, hpeel_sf_build_async): the whole path as one CUDA
graph with no host round trip, stats in device memory.  Outputs are compared
with the oracle element by element (bit-exact: all integer work) and with the
synchronous calls; the graphs are also captured into a caller's
torch.cuda.CUDAGraph and replayed on new input contents."""
import numpy as np
import pytest

import oracle
from paper_1312_0526_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1312_0526_gb300 as hp  # noqa: E402

DONE, EXHAUSTED, DEVICE_ERROR, LAYERS_FULL = 1, 2, 3, 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_0526_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _dev64(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _check_against_oracle(got: hp.AsyncPeel, want, max_layers=4096, general=False):
    torch.cuda.synchronize()
    st = hp.stats_from_device(got.stats)
    assert st["async_status"] == DONE and st["device_err"] == 0
    assert st["rounds"] == want.rounds and st["n_peeled"] == want.n_peeled
    assert st["core_nonempty"] == (1 if want.core_nonempty else 0)
    assert np.array_equal(_u32(got.order), want.order)
    assert np.array_equal(_u32(got.claim), want.claim)
    R = want.rounds
    assert np.array_equal(got.layer_off[:R + 1].cpu().numpy().astype(np.uint64),
                          want.layer_off[:R + 1].astype(np.uint64))
    return st


@pytest.mark.parametrize("n,gamma,r", [(1, 1230, 3), (17, 1230, 3), (1000, 1230, 3),
                                       (100_000, 1230, 3), (60_000, 1200, 3),
                                       (50_000, 1300, 4), (30_000, 1100, 3)])
def test_peel_async_matches_oracle_and_sync_peel(n, gamma, r):
    m = oracle.num_vertices(n, gamma, r)
    e = oracle.hash_edges(inputs.keys(n, 5), m, r, 1)
    want = oracle.peel_rounds(e, m)
    de = _dev32(e)
    got = hp.peel_async(de, m)
    st = _check_against_oracle(got, want)
    sync = hp.peel(de, m)
    for f in ("first_layer", "frontier", "n_peeled", "rounds"):
        assert st[f] == sync.stats[f], f


def _chain(n):
    """A band-shaped 3-hypergraph that peels a few edges per round from both
    ends: more rounds (> 300) than one pass of the order sort has bins."""
    P = n
    e = np.zeros((n, 3), dtype=np.uint32)
    for i in range(n):
        k, q = divmod(i, 4)
        e[i] = ((i + 1) // 2, P + i // 2, 2 * P + 2 * k + (q % 2))
    return e, 3 * P


@pytest.mark.parametrize("n", [1203, 2500, 12_000])
def test_peel_async_many_rounds_device_driven_sort_passes(n):
    e, m = _chain(n)
    want = oracle.peel_rounds(e, m)
    assert want.rounds > 300
    _check_against_oracle(hp.peel_async(_dev32(e), m, max_layers=8192), want)


def test_peel_async_layer_table_too_small():
    e, m = _chain(1200)
    want = oracle.peel_rounds(e, m)
    got = hp.peel_async(_dev32(e), m, max_layers=8)
    torch.cuda.synchronize()
    st = hp.stats_from_device(got.stats)
    assert st["async_status"] == LAYERS_FULL and st["rounds"] == want.rounds
    assert np.array_equal(_u32(got.order), want.order)
    assert np.array_equal(_u32(got.claim), want.claim)


def test_peel_async_device_check():
    e = np.array([[0, 3, 6], [1, 1, 7]], dtype=np.uint32)  # vertex 1 at position 1
    got = hp.peel_async(_dev32(e), 9)
    torch.cuda.synchronize()
    st = hp.stats_from_device(got.stats)
    assert st["async_status"] == DEVICE_ERROR and st["device_err"] == 1


def test_peel_async_empty():
    got = hp.peel_async(torch.empty((0, 3), dtype=torch.int32, device="cuda"), 0)
    torch.cuda.synchronize()
    st = hp.stats_from_device(got.stats)
    assert st["async_status"] == DONE and st["rounds"] == 0 and st["n_peeled"] == 0
    assert int(got.layer_off[0]) == 0


@pytest.fixture
def small_buckets():
    hp.set_tuning(bucket_shift=10, bucket_min_vertices=0)
    yield
    hp.set_tuning()


@pytest.mark.parametrize("n,gamma,r", [(100_000, 1230, 3), (60_000, 1200, 4)])
def test_peel_async_bucketed_build(small_buckets, n, gamma, r):
    m = oracle.num_vertices(n, gamma, r)
    e = oracle.hash_edges(inputs.keys(n, 6), m, r, 1)
    _check_against_oracle(hp.peel_async(_dev32(e), m), oracle.peel_rounds(e, m))


@pytest.mark.parametrize("span", [1024, 30_000])
def test_peel_async_bucket_overflow_redone_in_the_graph(small_buckets, span):
    # vertices confined to the first `span` of each part: the buckets
    # overflow and the graph's if node redoes the build with direct updates
    n, P = 60_000, 40_000
    rng = np.random.default_rng(9)
    e = np.stack([rng.integers(0, span, n) + j * P for j in range(3)], axis=1).astype(np.uint32)
    _check_against_oracle(hp.peel_async(_dev32(e), 3 * P), oracle.peel_rounds(e, 3 * P))


@pytest.mark.parametrize("n,gamma,r", [(1000, 1230, 3), (100_000, 1300, 3), (40_000, 1500, 4),
                                       (50_000, 1230, 2)])
def test_peel_general_async_matches_oracle(n, gamma, r):
    m = (n * gamma + 999) // 1000
    e = oracle.hash_edges_general(inputs.keys(n, 8), m, r, 1)
    want = oracle.peel_rounds_general(e, m)
    _check_against_oracle(hp.peel_async(_dev32(e), m, general=True), want, general=True)


def test_peel_async_captured_in_torch_graph_and_replayed_on_new_edges():
    n, gamma = 50_000, 1230
    m = oracle.num_vertices(n, gamma, 3)
    graphs = [oracle.hash_edges(inputs.keys(n, s), m, 3, 1) for s in (21, 22, 23)]
    de = _dev32(graphs[0])
    ws = torch.empty(hp.peel_workspace_size(n, m, 3), dtype=torch.uint8, device="cuda")
    out = hp.peel_async(de, m, workspace=ws)   # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            hp.peel_async(de, m, workspace=ws, out=out)
    torch.cuda.synchronize()
    for e in graphs[1:] + graphs[:1]:
        de.copy_(_dev32(e))
        out.order.fill_(-1)
        g.replay()
        _check_against_oracle(out, oracle.peel_rounds(e, m))


def test_peel_async_replays_its_cached_graph_on_new_edges():
    n = 20_000
    m = oracle.num_vertices(n, 1230, 3)
    de = _dev32(oracle.hash_edges(inputs.keys(n, 31), m, 3, 1))
    ws = torch.empty(hp.peel_workspace_size(n, m, 3), dtype=torch.uint8, device="cuda")
    out = hp.peel_async(de, m, workspace=ws)
    for seed in (32, 33):
        e = oracle.hash_edges(inputs.keys(n, seed), m, 3, 1)
        de.copy_(_dev32(e))
        hp.peel_async(de, m, workspace=ws, out=out)
        _check_against_oracle(out, oracle.peel_rounds(e, m))


# ------------------------------------------------------- static functions --

def _values(n, sigma, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, sigma, n, dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("n,sigma", [(1, 2), (1000, 5), (100_000, 256), (60_000, 2**32)])
def test_sf_build_async_matches_oracle_and_sync_build(n, sigma):
    keys = inputs.keys(n, 41)
    vals = _values(n, sigma, n + 3)
    want = oracle.sf_build(keys, vals, sigma, seed=1, max_tries=64)
    dk, dv = _dev64(keys), _dev32(vals)
    U, st = hp.sf_build_async(dk, dv, sigma, seed=1, max_tries=64)
    torch.cuda.synchronize()
    s = hp.stats_from_device(st)
    assert s["async_status"] == DONE and s["seed_used"] == want.seed_used
    words = len(want.U)
    assert np.array_equal(U[:words].cpu().numpy().view(np.uint64), want.U)
    sync = hp.sf_build(dk, dv, sigma, seed=1, max_tries=64)
    assert torch.equal(sync.U, U[:words])
    out = hp.sf_lookup(dk, want.seed_used, sync.m, sigma, U)
    assert np.array_equal(_u32(out), vals)


def test_sf_build_async_value_check_and_exhausted_seeds():
    n, sigma = 5000, 100
    keys = inputs.keys(n, 43)
    vals = _values(n, sigma, 7)
    vals[1234] = sigma  # not below sigma
    _, st = hp.sf_build_async(_dev64(keys), _dev32(vals), sigma)
    torch.cuda.synchronize()
    s = hp.stats_from_device(st)
    assert s["async_status"] == DEVICE_ERROR and s["device_err"] == 7
    dup = np.concatenate([keys[:100], keys[:100]])  # duplicates never peel
    _, st = hp.sf_build_async(_dev64(dup), _dev32(np.zeros(200, np.uint32)), 3, max_tries=3)
    torch.cuda.synchronize()
    s = hp.stats_from_device(st)
    assert s["async_status"] == EXHAUSTED and s["attempts"] == 3


def test_sf_build_async_captured_in_torch_graph_and_replayed_on_new_values():
    n, sigma = 30_000, 1000
    keys = inputs.keys(n, 45)
    dk = _dev64(keys)
    dv = _dev32(_values(n, sigma, 1))
    ws = torch.empty(hp.sf_workspace_size(n), dtype=torch.uint8, device="cuda")
    U, st = hp.sf_build_async(dk, dv, sigma, workspace=ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            hp.sf_build_async(dk, dv, sigma, workspace=ws, U=U, stats=st)
    torch.cuda.synchronize()
    for vs in (2, 3):
        vals = _values(n, sigma, vs)
        dv.copy_(_dev32(vals))
        g.replay()
        torch.cuda.synchronize()
        want = oracle.sf_build(keys, vals, sigma, seed=1, max_tries=8)
        assert hp.stats_from_device(st)["seed_used"] == want.seed_used
        assert np.array_equal(U[:len(want.U)].cpu().numpy().view(np.uint64), want.U)
