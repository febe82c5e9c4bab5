"""MPHF build beyond 32-bit ids (hpeel_mphf_build_large) against the oracle
and the 32-bit build: the same function bit for bit (g values, rank
directory, seed), with the layer list in device or in pinned host memory,
in both round-loop modes; lookups a bijection onto [0, n)."""
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
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("n", [1, 3, 17, 1000, 4097, 100_000, 1_000_003])
@pytest.mark.parametrize("on_host", [False, True])
def test_large_build_matches_oracle(n, on_host):
    keys = inputs.keys(n, 51)
    want = oracle.mphf_build(keys, seed=1, max_tries=32)
    hl = torch.empty(n, dtype=torch.int64, pin_memory=True) if on_host else None
    got = hp.mphf_build_large(_dev(keys), seed=1, max_tries=32, host_list=hl)
    assert got.stats["seed_used"] == want.seed_used
    assert np.array_equal(_u64(got.G), want.G)
    assert np.array_equal(_u64(got.rank_dir), want.dir)
    small = hp.mphf_build(_dev(keys), seed=1, max_tries=32)
    for f in ("rounds", "n_peeled", "first_layer", "frontier", "attempts"):
        assert got.stats[f] == small.stats[f], f


@pytest.mark.parametrize("gamma", [1222, 1230, 1300, 1500])
def test_large_build_other_gamma(gamma):
    n = 200_000
    keys = inputs.keys(n, 52)
    want = oracle.mphf_build(keys, seed=1, gamma_milli=gamma, max_tries=64)
    got = hp.mphf_build_large(_dev(keys), seed=1, gamma_milli=gamma, max_tries=64)
    assert got.stats["seed_used"] == want.seed_used
    assert np.array_equal(_u64(got.G), want.G)
    assert np.array_equal(_u64(got.rank_dir), want.dir)


def test_large_build_host_round_loop():
    n = 300_000
    keys = inputs.keys(n, 53)
    want = oracle.mphf_build(keys, seed=1, max_tries=32)
    try:
        hp.set_tuning(host_round_loop=1)
        got = hp.mphf_build_large(_dev(keys), seed=1, max_tries=32)
    finally:
        hp.set_tuning()
    assert np.array_equal(_u64(got.G), want.G)


def test_large_build_reseeds():
    # a key set whose first hash seed leaves a 2-core
    for s in range(300):
        k = inputs.keys(60, 4000 + s)
        m = oracle.num_vertices(60, 1230, 3)
        if oracle.peel_rounds(oracle.hash_edges(k, m, 3, 1), m).core_nonempty:
            break
    want = oracle.mphf_build(k, seed=1, max_tries=64)
    got = hp.mphf_build_large(_dev(k), seed=1, max_tries=64)
    assert got.stats["attempts"] > 1 and got.stats["seed_used"] == want.seed_used
    assert np.array_equal(_u64(got.G), want.G)
    dup = np.concatenate([k, k[:5]])
    with pytest.raises(hp.HpeelError, match="RETRIES_EXHAUSTED"):
        hp.mphf_build_large(_dev(dup), seed=1, max_tries=3)


@pytest.mark.parametrize("n", [1000, 250_000])
def test_large_lookup_is_a_bijection_and_equals_the_32_bit_lookup(n):
    keys = inputs.keys(n, 54)
    dk = _dev(keys)
    got = hp.mphf_build_large(dk, seed=1, max_tries=32)
    out = hp.mphf_lookup_large(dk, got.stats["seed_used"], got.m, got.G, got.rank_dir)
    vals = out.cpu().numpy()
    assert np.array_equal(np.sort(vals), np.arange(n))
    small = hp.mphf_lookup(dk, got.stats["seed_used"], got.m, got.G, got.rank_dir)
    assert np.array_equal(small.cpu().numpy().astype(np.int64) & 0xFFFFFFFF, vals)
    for i in (0, n // 2, n - 1):
        assert vals[i] == oracle.lookup(int(keys[i]), got.stats["seed_used"], got.m,
                                        _u64(got.G), _u64(got.rank_dir))


def test_large_rejects_bad_arguments():
    k = _dev(inputs.keys(100, 55))
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp.mphf_build_large(k, max_tries=0)
    with pytest.raises(hp.HpeelError, match="WORKSPACE"):
        hp.mphf_build_large(k, workspace=torch.empty(256, dtype=torch.uint8, device="cuda"))
