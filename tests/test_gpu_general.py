"""General (not r-partite) hypergraphs (sec. 2: edges are r-subsets of the
vertex set; rows may repeat a vertex) through hpeel_peel_general, against
the oracle's general peel: order, claim words (hinge = smallest position in
the row) and layer offsets, element by element."""
import numpy as np
import pytest

import oracle
from paper_1312_0526_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1312_0526_gb300 as hp  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_0526_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _check(edges, m):
    want = oracle.peel_rounds_general(edges, m)
    got = hp.peel(_dev(edges), m, max_layers=8192, general=True)
    assert got.rounds == want.rounds and got.n_peeled == want.n_peeled
    assert np.array_equal(_u32(got.order), want.order)
    assert np.array_equal(_u32(got.claim), want.claim)
    assert np.array_equal(got.layer_off.cpu().numpy().view(np.uint64), want.layer_off)
    return want, got


@pytest.mark.parametrize("n,gamma,r", [
    (1, 1230, 3), (5, 1230, 3), (4097, 1230, 3), (100_000, 1230, 3), (100_000, 1300, 3),
    (100_000, 1100, 3), (60_000, 1400, 4), (40_000, 2300, 2), (300_000, 1230, 3)])
def test_general_peel_parity_hashed(n, gamma, r):
    m = max(1, (n * gamma + 999) // 1000)  # any m, not a multiple of r
    edges = oracle.hash_edges_general(inputs.keys(n, 3), m, r, 1)
    want, got = _check(edges, m)
    if gamma <= 1100 and n > 1000:
        assert want.n_peeled < n


def test_general_peel_random_small_graphs_with_repeats():
    rng = np.random.default_rng(17)
    repeats = 0
    for trial in range(60):
        r = int(rng.integers(2, 5))
        m = int(rng.integers(1, 12))
        n = int(rng.integers(1, 40))
        edges = rng.integers(0, m, (n, r)).astype(np.uint32)
        repeats += int((np.sort(edges, axis=1)[:, 1:] == np.sort(edges, axis=1)[:, :-1]).any())
        _check(edges, m)
    assert repeats > 20


def test_general_peel_of_a_partite_graph_equals_the_partite_peel():
    n = 200_000
    m = hp.num_vertices(n, 1230, 3)
    edges = oracle.hash_edges(inputs.keys(n, 8), m, 3, 1)
    a = hp.peel(_dev(edges), m)
    b = hp.peel(_dev(edges), m, general=True)
    assert torch.equal(a.order, b.order) and torch.equal(a.claim, b.claim)


@pytest.fixture
def small_buckets():
    hp.set_tuning(bucket_shift=10, bucket_min_vertices=0)
    yield
    hp.set_tuning()


@pytest.mark.parametrize("n,r", [(150_000, 3), (50_000, 4), (30_000, 2)])
def test_general_peel_parity_bucketed(small_buckets, n, r):
    m = (n * 1250 + 999) // 1000
    _check(oracle.hash_edges_general(inputs.keys(n, 12), m, r, 1), m)


@pytest.fixture
def host_round_loop():
    hp.set_tuning(host_round_loop=1)
    yield
    hp.set_tuning()


def test_general_peel_parity_host_round_loop(host_round_loop):
    n = 120_000
    m = 150_001
    _check(oracle.hash_edges_general(inputs.keys(n, 14), m, 3, 1), m)


@pytest.mark.slow
def test_general_peel_parity_1e7():
    n = 10_000_000
    m = 12_300_001
    _check(oracle.hash_edges_general(inputs.keys(n, 1), m, 3, 1), m)


def test_general_peel_errors():
    e = np.array([[0, 1, 7]], dtype=np.uint32)
    with pytest.raises(hp.HpeelError, match="DEVICE_CHECK"):
        hp.peel(_dev(e), 7, general=True)
    # n >= 2^30 is refused before anything touches the (absent) buffers
    rc = hp.lib().hpeel_peel_general(None, 1 << 30, 1 << 31, 3, None, None, None, 0, None,
                                     None, 0, None)
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp._check(rc)
    ok = np.array([[0, 1, 2], [2, 3, 4]], dtype=np.uint32)
    _check(ok, 5)


@pytest.mark.parametrize("n,m,r", [(1, 1, 3), (1000, 7, 2), (100_000, 123_001, 3),
                                   (65_537, 2**32 - 5, 4), (100_000, 3, 3)])
def test_general_hash_matches_oracle(n, m, r):
    keys = inputs.keys(n, 21)
    got = hp.hash_edges(torch.from_numpy(keys.view(np.int64)).cuda(), m, r, 9, general=True)
    assert np.array_equal(_u32(got).reshape(n, r), oracle.hash_edges_general(keys, m, r, 9))
