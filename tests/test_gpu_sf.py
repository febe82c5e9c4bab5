"""Static functions (sec. 3: f: S -> [sigma] stored as u with f(x) = u[h0] +
u[h1] + u[h2] mod sigma) on the GPU against the oracle: the b-bit values u
bit for bit, the seed used, and the lookups of every key."""
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


def _values(n, sigma, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, sigma, n, dtype=np.uint64).astype(np.uint32)


def _dev64(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _check(n, sigma, key_seed=31):
    keys = inputs.keys(n, key_seed)
    vals = _values(n, sigma, n + 1)
    want = oracle.sf_build(keys, vals, sigma, seed=1, max_tries=64)
    dk = _dev64(keys)
    got = hp.sf_build(dk, _dev32(vals), sigma, seed=1, max_tries=64)
    assert got.stats["seed_used"] == want.seed_used
    assert got.bits == want.bits == (sigma - 1).bit_length()
    assert np.array_equal(got.U.cpu().numpy().view(np.uint64), want.U)
    out = hp.sf_lookup(dk, want.seed_used, got.m, sigma, got.U)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), vals)


@pytest.mark.parametrize("n,sigma", [
    (1, 2), (17, 3), (1000, 5), (4097, 100), (30_000, 2), (100_000, 2**13 - 1),
    (100_000, 2**16 + 1), (250_000, 2**31 + 11), (120_000, 2**32), (200_000, 255)])
def test_sf_parity_and_lookup(n, sigma):
    _check(n, sigma)


@pytest.fixture
def small_buckets():
    """The L2-blocked build on small graphs (tiny chunks)."""
    hp.set_tuning(bucket_shift=12, bucket_min_vertices=1)
    yield
    hp.set_tuning()


@pytest.mark.parametrize("sigma", [7, 2**20 + 3])
def test_sf_parity_bucketed_build(small_buckets, sigma):
    _check(150_000, sigma, key_seed=8)


@pytest.mark.slow
def test_sf_parity_1e7():
    # default tuning: the L2-blocked build at m = 12.3M vertices
    _check(10_000_000, 1000, key_seed=1)


def test_sf_sigma3_hinge_values_equal_the_mphf_g():
    # the MPHF is the static function x -> hinge position with sigma = 3
    n = 200_000
    keys = inputs.keys(n, 5)
    dk = _dev64(keys)
    mp = hp.mphf_build(dk, seed=1, max_tries=32)
    seed = mp.stats["seed_used"]
    edges = oracle.hash_edges(keys, mp.m, 3, seed)
    hinges = (oracle.peel_rounds(edges, mp.m).claim & 3).astype(np.uint32)
    sf = hp.sf_build(dk, _dev32(hinges), 3, seed=seed, max_tries=1)
    g = mp.G.cpu().numpy().view(np.uint64)
    u = sf.U.cpu().numpy().view(np.uint64)
    three = (g & (g >> np.uint64(1))) & np.uint64(0x5555555555555555)  # pairs holding 3
    assert np.array_equal(u, g & ~(three | (three << np.uint64(1))))  # 3 -> 0, pairwise


def test_sf_rejects_bad_values_and_sigma():
    keys = _dev64(inputs.keys(500, 3))
    vals = _values(500, 10, 1)
    vals[77] = 10
    with pytest.raises(hp.HpeelError, match="DEVICE_CHECK"):
        hp.sf_build(keys, _dev32(vals), 10, seed=1, max_tries=64)
    ok = _dev32(_values(500, 10, 1))
    for sigma in (0, 1, 2**32 + 1):
        with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
            hp.sf_build(keys, ok, sigma, seed=1)
    # the library stays usable after the failures
    _check(1000, 10)
