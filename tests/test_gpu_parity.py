"""GPU path vs CPU oracle, element by element (bit-exact: all integer work).

Every call goes through the C ABI (via the ctypes binding).  Inputs come from
the seeded generators in paper_1312_0526_gb300.inputs; expected values come
only from the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1312_0526_gb300 import inputs
from tests import golden_io

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1312_0526_gb300 as hp  # noqa: E402


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


# ------------------------------------------------------------------- hash --

@pytest.mark.parametrize("n", [1, 2, 3, 255, 256, 257, 4095, 4097, 100_000, 1_000_003])
@pytest.mark.parametrize("r", [3, 4])
def test_hash_edges_parity(n, r):
    keys = inputs.keys(n, 1)
    m = oracle.num_vertices(n, 1230, r)
    want = oracle.hash_edges(keys, m, r, 1)
    got = _u32(hp.hash_edges(_dev(keys), m, r, 1)).reshape(n, r)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("P", [1, 2, 3, 1000, 41_000, 1_000_000_007, 1_431_655_765])
def test_hash_edges_fastmod_extreme_divisors(P):
    # keys that push mix64 outputs over the whole 64-bit range, with part
    # sizes up to the largest m < 2^32 allows
    keys = np.concatenate([inputs.keys(20_000, 77),
                           np.array([0, 1, 2**63, 2**64 - 1, 2**64 - 2], dtype=np.uint64)])
    m = 3 * P
    want = oracle.hash_edges(keys, m, 3, 12345)
    got = _u32(hp.hash_edges(_dev(keys), m, 3, 12345)).reshape(-1, 3)
    assert np.array_equal(got, want)


# ------------------------------------------------------------------- peel --

def _check_peel(edges: np.ndarray, m: int, max_layers=4096):
    want = oracle.peel_rounds(edges, m)
    got = hp.peel(_dev(edges), m, max_layers=max_layers)
    assert got.rounds == want.rounds
    assert got.n_peeled == want.n_peeled
    assert np.array_equal(_u32(got.order), want.order)
    assert np.array_equal(_u32(got.claim), want.claim)
    assert np.array_equal(_u64(got.layer_off), want.layer_off)
    return want


@pytest.mark.parametrize("name", [n for n in golden_io.all_names()
                                  if golden_io.load(n)["edges"].shape[0] > 0])
def test_peel_goldens(name):
    g = golden_io.load(name)
    got = hp.peel(_dev(g["edges"]), g["m"])
    assert np.array_equal(_u32(got.order), g["order"])
    assert np.array_equal(_u32(got.claim), g["claim"])
    assert np.array_equal(_u64(got.layer_off), g["layer_off"])
    assert got.n_peeled == g["n_peeled"]


@pytest.mark.parametrize("n,gamma,r", [
    (1, 1230, 3), (2, 1230, 3), (5, 1230, 3), (100, 1230, 3), (4095, 1230, 3),
    (4097, 1230, 3), (8192, 1230, 3), (12_288, 1200, 3), (100_000, 1230, 3), (100_000, 1222, 3), (100_000, 1200, 3),
    (100_000, 1300, 4), (54_321, 1400, 3), (30_001, 1100, 3), (300_000, 1230, 3),
])
def test_peel_parity(n, gamma, r):
    m = oracle.num_vertices(n, gamma, r)
    edges = oracle.hash_edges(inputs.keys(n, 1), m, r, 1)
    want = _check_peel(edges, m)
    if gamma <= 1200 and n > 1000:
        assert want.core_nonempty


def test_peel_random_small_graphs_with_cores():
    rng = np.random.default_rng(5)
    for trial in range(40):
        r = 3 if trial % 2 == 0 else 4
        P = int(rng.integers(1, 6))
        n = int(rng.integers(1, 40))
        edges = np.stack([rng.integers(0, P, n) + j * P for j in range(r)], axis=1).astype(np.uint32)
        _check_peel(edges, r * P)


def _chain(n):
    """A band-shaped 3-hypergraph where every vertex has degree 2 except near
    the ends: it peels from the two ends inwards, a few edges per round."""
    P = n
    e = np.zeros((n, 3), dtype=np.uint32)
    for i in range(n):
        k, q = divmod(i, 4)
        e[i] = ((i + 1) // 2, P + i // 2, 2 * P + 2 * k + (q % 2))
    return e, 3 * P


@pytest.mark.parametrize("n", [1200, 1203, 2500, 12_000])
def test_peel_many_rounds_multi_pass_emit(n):
    # more rounds than one emit pass has bins (256): the canonical order
    # needs the multi-pass sort (at n = 12,000: 4,500 rounds, 18 passes, the
    # later ones over several full tiles of ids read back from the order)
    e, m = _chain(n)
    want = oracle.peel_rounds(e, m)
    assert want.rounds > 300
    _check_peel(e, m, max_layers=8192)


def test_peel_deterministic_across_runs():
    n = 200_000
    m = oracle.num_vertices(n, 1230, 3)
    edges = _dev(oracle.hash_edges(inputs.keys(n, 3), m, 3, 1))
    a = hp.peel(edges, m)
    for _ in range(3):
        b = hp.peel(edges, m)
        assert torch.equal(a.order, b.order) and torch.equal(a.claim, b.claim)


def test_peel_empty_input():
    got = hp.peel(torch.empty((0, 3), dtype=torch.int32, device="cuda"), 0)
    assert got.rounds == 0 and got.n_peeled == 0 and got.order.numel() == 0
    assert _u64(got.layer_off).tolist() == [0]


def test_peel_rejects_vertex_outside_its_part():
    e = np.array([[0, 3, 6], [1, 1, 7]], dtype=np.uint32)  # vertex 1 at position 1
    with pytest.raises(hp.HpeelError, match="DEVICE_CHECK"):
        hp.peel(_dev(e), 9)


def test_peel_rejects_small_workspace():
    e = np.array([[0, 3, 6]], dtype=np.uint32)
    ws = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(hp.HpeelError, match="WORKSPACE"):
        hp.peel(_dev(e), 9, workspace=ws)


def test_peel_layer_capacity_error():
    e, m = _chain(1200)
    with pytest.raises(hp.HpeelError, match="CAPACITY"):
        hp.peel(_dev(e), m, max_layers=8)


# ------------------------------------------------------------------- MPHF --

@pytest.mark.parametrize("n", [1, 17, 1000, 4097, 100_000, 250_000])
def test_mphf_parity(n):
    keys = inputs.keys(n, 1)
    want = oracle.mphf_build(keys, seed=1, max_tries=32)
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    got = hp.mphf_build(_dev(keys), seed=1, max_tries=32, order=order)
    assert got.stats["seed_used"] == want.seed_used
    assert got.stats["rounds"] == want.rounds
    assert np.array_equal(_u64(got.G), want.G)
    assert np.array_equal(_u64(got.rank_dir), want.dir)
    # the whole path: the canonical order of the successful attempt's graph
    m = oracle.num_vertices(n, 1230, 3)
    pw = oracle.peel_rounds(oracle.hash_edges(keys, m, 3, want.seed_used), m)
    assert np.array_equal(_u32(order), pw.order)


def test_mphf_retries_exhausted_on_duplicate_keys():
    keys = np.array([5, 5, 6, 7], dtype=np.uint64)
    with pytest.raises(hp.HpeelError, match="RETRIES_EXHAUSTED"):
        hp.mphf_build(_dev(keys), seed=1, max_tries=3)


def test_mphf_reseed_matches_oracle():
    # find key sets whose first hash seed leaves a 2-core; both sides retry
    found = 0
    for s in range(300):
        k = inputs.keys(60, 2000 + s)
        m = oracle.num_vertices(60, 1230, 3)
        if oracle.peel_rounds(oracle.hash_edges(k, m, 3, 1), m).core_nonempty:
            want = oracle.mphf_build(k, seed=1, max_tries=64)
            got = hp.mphf_build(_dev(k), seed=1, max_tries=64)
            assert got.stats["seed_used"] == want.seed_used > 1
            assert np.array_equal(_u64(got.G), want.G)
            assert np.array_equal(_u64(got.rank_dir), want.dir)
            found += 1
            if found == 3:
                break
    assert found == 3


# ----------------------------------------------- L2-blocked incidence build --

@pytest.fixture
def small_buckets():
    """Route small graphs through the L2-blocked build with 1024-vertex
    chunks (many buckets), restoring the defaults afterwards."""
    hp.set_tuning(bucket_shift=10, bucket_min_vertices=0)
    yield
    hp.set_tuning()


@pytest.mark.parametrize("n,gamma,r", [(100_000, 1230, 3), (100_003, 1200, 3),
                                       (50_000, 1300, 4), (20_000, 1500, 2), (1, 1230, 3),
                                       (1025, 1230, 3)])
def test_peel_parity_bucketed(small_buckets, n, gamma, r):
    m = oracle.num_vertices(n, gamma, r)
    edges = oracle.hash_edges(inputs.keys(n, 5), m, r, 1)
    _check_peel(edges, m)


@pytest.mark.parametrize("shift,sub", [(10, 10), (14, 2), (12, 3), (16, 4)])
def test_peel_parity_extreme_sub_buckets(shift, sub):
    # one sub-bucket per chunk (S = 1) up to 4,096 of them (the refine's scan
    # then keeps most cursors in shared memory instead of registers)
    hp.set_tuning(bucket_shift=shift, bucket_sub_shift=sub, bucket_min_vertices=0)
    try:
        n = 50_000
        m = oracle.num_vertices(n, 1230, 3)
        _check_peel(oracle.hash_edges(inputs.keys(n, 12), m, 3, 1), m)
    finally:
        hp.set_tuning()


@pytest.mark.parametrize("span", [1024, 4096, 30_000])
def test_peel_bucket_overflow_falls_back(small_buckets, span):
    # every vertex in the first `span` of its part: buckets sized for a
    # uniform spread overflow; overflowing incidences go to the overflow
    # list, and when that is full too the peel is redone with direct updates
    n, P = 60_000, 40_000
    rng = np.random.default_rng(9)
    edges = np.stack([rng.integers(0, span, n) + j * P for j in range(3)], axis=1).astype(np.uint32)
    _check_peel(edges, 3 * P)


@pytest.mark.parametrize("n", [1000, 100_000])
def test_mphf_parity_bucketed(small_buckets, n):
    keys = inputs.keys(n, 4)
    want = oracle.mphf_build(keys, seed=1, max_tries=32)
    got = hp.mphf_build(_dev(keys), seed=1, max_tries=32)
    assert got.stats["seed_used"] == want.seed_used
    assert np.array_equal(_u64(got.G), want.G)
    assert np.array_equal(_u64(got.rank_dir), want.dir)


@pytest.fixture
def part_passes():
    """The L2-blocked build with small chunks, one part per pass (the mode
    graphs of more than 2^30 edges take by default)."""
    hp.set_tuning(bucket_shift=10, bucket_min_vertices=0, bucket_part_passes=2)
    yield
    hp.set_tuning()


@pytest.mark.parametrize("n,gamma,r", [(100_000, 1230, 3), (100_003, 1200, 3),
                                       (50_000, 1300, 4), (20_000, 1500, 2), (1, 1230, 3),
                                       (1025, 1230, 3)])
def test_peel_parity_one_part_per_pass(part_passes, n, gamma, r):
    m = oracle.num_vertices(n, gamma, r)
    edges = oracle.hash_edges(inputs.keys(n, 6), m, r, 1)
    _check_peel(edges, m)


@pytest.mark.parametrize("span", [1024, 30_000])
def test_peel_bucket_overflow_one_part_per_pass(part_passes, span):
    n, P = 60_000, 40_000
    rng = np.random.default_rng(10)
    edges = np.stack([rng.integers(0, span, n) + j * P for j in range(3)], axis=1).astype(np.uint32)
    _check_peel(edges, 3 * P)


def test_mphf_parity_one_part_per_pass(part_passes):
    keys = inputs.keys(100_000, 7)
    want = oracle.mphf_build(keys, seed=1, max_tries=32)
    got = hp.mphf_build(_dev(keys), seed=1, max_tries=32)
    assert got.stats["seed_used"] == want.seed_used
    assert np.array_equal(_u64(got.G), want.G)
    assert np.array_equal(_u64(got.rank_dir), want.dir)
    G, D, st = hp.mphf_build_async(_dev(keys), seed=1, max_tries=32)
    assert hp.stats_from_device(st)["seed_used"] == want.seed_used
    assert np.array_equal(_u64(G), want.G) and np.array_equal(_u64(D), want.dir)


def test_tuning_rejects_bad_values():
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp.set_tuning(bucket_shift=3)
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp.set_tuning(bucket_sub_shift=15)
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp.set_tuning(bucket_part_passes=3)
    hp.set_tuning()
    assert hp.get_tuning()["bucket_shift"] == 22


@pytest.mark.slow
def test_peel_and_mphf_parity_1e7_default_tuning():
    # default tuning: m = 12.3M vertices takes the L2-blocked build; the
    # whole output is compared with the oracle
    n = 10_000_000
    keys = inputs.keys(n, 1)
    m = oracle.num_vertices(n, 1230, 3)
    edges = oracle.hash_edges(keys, m, 3, 1)
    _check_peel(edges, m)
    want = oracle.mphf_build(keys, seed=1)
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    got = hp.mphf_build(_dev(keys), seed=1, order=order)
    assert np.array_equal(_u64(got.G), want.G)
    assert np.array_equal(_u64(got.rank_dir), want.dir)


# ----------------------------------------------------- round-loop drivers --

@pytest.fixture
def host_round_loop():
    """The host launches every round instead of the device-side graph loop."""
    hp.set_tuning(host_round_loop=1)
    yield
    hp.set_tuning()


@pytest.mark.parametrize("n,gamma,r", [(100_000, 1230, 3), (100_000, 1200, 3),
                                       (50_000, 1300, 4), (3, 1230, 3)])
def test_peel_parity_host_round_loop(host_round_loop, n, gamma, r):
    m = oracle.num_vertices(n, gamma, r)
    edges = oracle.hash_edges(inputs.keys(n, 6), m, r, 1)
    _check_peel(edges, m)


def test_mphf_parity_host_round_loop(host_round_loop):
    keys = inputs.keys(200_000, 8)
    want = oracle.mphf_build(keys, seed=1)
    got = hp.mphf_build(_dev(keys), seed=1)
    assert np.array_equal(_u64(got.G), want.G)
    assert np.array_equal(_u64(got.rank_dir), want.dir)


@pytest.mark.parametrize("r,gamma", [(2, 2300), (3, 1230), (4, 1300)])
def test_peel_parity_moved_hinges(r, gamma):
    # An edge often gains two degree-1 vertices in the same round, and the
    # claim of the larger position can land first: the layer-list entry then
    # names the wrong hinge until the round that deletes the edge moves it.
    # Exact claim words (hinges included) and MPHF g values show the moved
    # entries end right; hinge_moves shows the path ran.
    n = 200_000
    m = oracle.num_vertices(n, gamma, r)
    edges = oracle.hash_edges(inputs.keys(n, 12), m, r, 1)
    want = _check_peel(edges, m)
    got = hp.peel(_dev(edges), m, max_layers=4096)
    assert got.stats["hinge_moves"] > 0
    assert got.stats["hinge_moves"] <= want.n_peeled
    if r == 3:
        keys = inputs.keys(n, 13)
        wm = oracle.mphf_build(keys, seed=1)
        gm = hp.mphf_build(_dev(keys), seed=1)
        assert gm.stats["hinge_moves"] > 0
        assert np.array_equal(_u64(gm.G), wm.G)
        assert np.array_equal(_u64(gm.rank_dir), wm.dir)


# ------------------------------------------------------------------ lookup --

@pytest.mark.parametrize("n", [1, 1000, 100_000])
def test_mphf_lookup_is_a_bijection_and_matches_oracle(n):
    keys = inputs.keys(n, 21)
    dk = _dev(keys)
    res = hp.mphf_build(dk, seed=1, max_tries=32)
    seed = res.stats["seed_used"]
    vals = hp.mphf_lookup(dk, seed, res.m, res.G, res.rank_dir)
    got = _u32(vals)
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint32))
    Gh, Dh = _u64(res.G), _u64(res.rank_dir)
    for i in range(0, n, max(1, n // 500)):
        assert got[i] == oracle.lookup(int(keys[i]), seed, res.m, Gh, Dh)
    # keys outside the set map into [0, n]
    other = _u32(hp.mphf_lookup(_dev(inputs.keys(5000, 99)), seed, res.m, res.G, res.rank_dir))
    assert other.max() <= n


def test_bits_per_key_matches_table_space():
    assert round(hp.mphf_bits_per_key(10**8), 2) == 2.61


def test_mphf_and_sf_from_pinned_host_keys_equal_device_keys():
    # keys (and values) in pinned host memory are read in place by the GPU;
    # the results are those of the device-resident build
    n = 300_000
    kh = torch.from_numpy(inputs.keys(n, 77).view(np.int64)).pin_memory()
    a = hp.mphf_build(kh.cuda(), seed=1, max_tries=32)
    b = hp.mphf_build(kh, seed=1, max_tries=32)
    assert a.stats["seed_used"] == b.stats["seed_used"]
    assert torch.equal(a.G, b.G) and torch.equal(a.rank_dir, b.rank_dir)
    vh = torch.from_numpy((inputs.keys(n, 78) % np.uint64(1000)).astype(np.uint32)
                          .view(np.int32)).pin_memory()
    c = hp.sf_build(kh.cuda(), vh.cuda(), 1000, seed=1, max_tries=32)
    d = hp.sf_build(kh, vh, 1000, seed=1, max_tries=32)
    assert torch.equal(c.U, d.U)
    with pytest.raises(ValueError):
        hp.mphf_build(kh.clone(), seed=1)  # pageable host memory is refused
