"""Rounds in sorted form (claims bucketed by edge, DeleteEdge updates bucketed
by vertex and applied in shared memory; sec. 4.2's sorting) against the
oracle, element by element.  The tuning's sorted_round_min = 1 runs every
round in sorted form; larger values switch to the random round kernel once a
layer is smaller; both loop modes (graph and host) are covered, and the
device-driven calls as well."""
import numpy as np
import pytest

import oracle
from paper_1312_0526_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1312_0526_gb300 as hp  # noqa: E402

NEVER = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_0526_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev(a: np.ndarray):
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(params=[(1, 0), (1, 1), (500, 0), (500, 1), (0, 0)],
                ids=["all_sorted_graph", "all_sorted_host", "min500_graph", "min500_host",
                     "automatic_graph"])
def sorted_tuning(request):
    mn, host = request.param
    hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, sorted_round_min=mn,
                  host_round_loop=host)
    yield request.param
    hp.set_tuning()


def _check(e, m, tun):
    want = oracle.peel_rounds(e, m)
    got = hp.peel(_dev(e), m)
    assert got.rounds == want.rounds and got.n_peeled == want.n_peeled
    assert np.array_equal(_u32(got.order), want.order)
    assert np.array_equal(_u32(got.claim), want.claim)
    assert np.array_equal(_u64(got.layer_off), want.layer_off)
    if got.stats["sorted_rounds"] == want.rounds:
        # every round sorted: exact hinges, nothing to correct
        assert got.stats["hinge_moves"] == 0
    return got, want


@pytest.mark.parametrize("n,gamma", [(1, 1230), (2, 1230), (100, 1230), (4097, 1230),
                                     (100_000, 1230), (100_003, 1200), (50_000, 1300),
                                     (30_001, 1100), (200_000, 1222), (60_000, 1600)])
def test_peel_sorted_rounds_parity(sorted_tuning, n, gamma):
    m = oracle.num_vertices(n, gamma, 3)
    got, want = _check(oracle.hash_edges(inputs.keys(n, 8), m, 3, 1), m, sorted_tuning)
    if sorted_tuning[0] == 1 and gamma <= 1300:
        # L_0 (at most 0.3 n edges at these sparsities) and every later
        # layer are deleted in sorted form
        assert got.stats["sorted_rounds"] == want.rounds


def test_sorted_rounds_run_where_expected():
    n = 200_000
    m = oracle.num_vertices(n, 1230, 3)
    e = _dev(oracle.hash_edges(inputs.keys(n, 9), m, 3, 1))
    try:
        hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, sorted_round_min=1)
        every = hp.peel(e, m)
        hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, sorted_round_min=0)  # n / 20
        auto = hp.peel(e, m)
        hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, sorted_round_min=NEVER)
        never = hp.peel(e, m)
    finally:
        hp.set_tuning()
    assert every.stats["sorted_rounds"] == every.rounds
    assert 0 < auto.stats["sorted_rounds"] < auto.rounds
    assert never.stats["sorted_rounds"] == 0
    for x in (auto, never):
        assert torch.equal(x.order, every.order) and torch.equal(x.claim, every.claim)


def test_sorted_rounds_many_rounds_chain(sorted_tuning):
    # a band graph peeled a few edges per round: > 300 rounds, tiny layers
    n = 1203
    P = n
    e = np.zeros((n, 3), dtype=np.uint32)
    for i in range(n):
        k, q = divmod(i, 4)
        e[i] = ((i + 1) // 2, P + i // 2, 2 * P + 2 * k + (q % 2))
    _check(e, 3 * P, sorted_tuning)


def test_sorted_round_claim_list_overflow_is_redone():
    # every vertex has degree 1 (three fresh vertices per edge): round 0's
    # claims exceed the claim list, the peel is redone with random rounds
    n = 30_000
    P = n
    e = np.stack([np.arange(n) + j * P for j in range(3)], axis=1).astype(np.uint32)
    try:
        hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, sorted_round_min=1)
        for host in (0, 1):
            hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, sorted_round_min=1,
                          host_round_loop=host)
            _check(e, 3 * P, (0, host))
        out = hp.peel_async(_dev(e), 3 * P)
        torch.cuda.synchronize()
        want = oracle.peel_rounds(e, 3 * P)
        assert hp.stats_from_device(out.stats)["async_status"] == 1
        assert np.array_equal(_u32(out.order), want.order)
        assert np.array_equal(_u32(out.claim), want.claim)
    finally:
        hp.set_tuning()


@pytest.mark.parametrize("span", [1024, 30_000])
def test_sorted_rounds_on_skewed_graphs(span):
    n, P = 60_000, 40_000
    rng = np.random.default_rng(21)
    e = np.stack([rng.integers(0, span, n) + j * P for j in range(3)], axis=1).astype(np.uint32)
    try:
        hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, sorted_round_min=1)
        _check(e, 3 * P, (0, 0))
    finally:
        hp.set_tuning()


@pytest.mark.parametrize("n", [1000, 100_000, 250_000])
def test_mphf_sorted_rounds_parity(sorted_tuning, n):
    keys = inputs.keys(n, 14)
    want = oracle.mphf_build(keys, seed=1, max_tries=32)
    got = hp.mphf_build(_dev(keys), seed=1, max_tries=32)
    assert got.stats["seed_used"] == want.seed_used
    assert np.array_equal(_u64(got.G), want.G)
    assert np.array_equal(_u64(got.rank_dir), want.dir)
    G, D, st = hp.mphf_build_async(_dev(keys), seed=1, max_tries=32)
    torch.cuda.synchronize()
    s = hp.stats_from_device(st)
    assert s["async_status"] == 1 and s["seed_used"] == want.seed_used
    assert np.array_equal(_u64(G), want.G) and np.array_equal(_u64(D), want.dir)


@pytest.mark.parametrize("n,gamma", [(100_000, 1230), (60_000, 1200)])
def test_peel_async_sorted_rounds(sorted_tuning, n, gamma):
    m = oracle.num_vertices(n, gamma, 3)
    e = oracle.hash_edges(inputs.keys(n, 15), m, 3, 1)
    want = oracle.peel_rounds(e, m)
    out = hp.peel_async(_dev(e), m)
    torch.cuda.synchronize()
    s = hp.stats_from_device(out.stats)
    assert s["async_status"] == 1 and s["rounds"] == want.rounds
    assert np.array_equal(_u32(out.order), want.order)
    assert np.array_equal(_u32(out.claim), want.claim)
    R = want.rounds
    assert np.array_equal(_u64(out.layer_off[:R + 1]), want.layer_off)


def test_sf_sorted_rounds_parity():
    n, sigma = 100_000, 1000
    keys = inputs.keys(n, 16)
    vals = (inputs.keys(n, 17) % np.uint64(sigma)).astype(np.uint32)
    want = oracle.sf_build(keys, vals, sigma, seed=1, max_tries=64)
    try:
        hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, sorted_round_min=1)
        got = hp.sf_build(_dev(keys), _dev(vals), sigma, seed=1, max_tries=64)
        U, st = hp.sf_build_async(_dev(keys), _dev(vals), sigma, seed=1, max_tries=64)
        torch.cuda.synchronize()
    finally:
        hp.set_tuning()
    assert np.array_equal(_u64(got.U), want.U)
    assert np.array_equal(_u64(U[:len(want.U)]), want.U)
