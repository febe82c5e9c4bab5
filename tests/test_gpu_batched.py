"""Batched bucket peel (hpeel_peel_batched) vs the oracle, bucket by bucket.

Every bucket b is its own hypergraph: keys off[b]..off[b+1], hash seed b,
m_b = num_vertices(n_b).  The oracle peels each bucket separately; the GPU
peels all of them in one launch.  Bit-exact on order, rounds, 2-core status
and g values.
"""
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


def _workload(extra_sizes=(), B=240, median=600, seed=3, key_seed=2):
    sizes = np.concatenate([inputs.lognormal_bucket_sizes(B, median=median, lo=1, hi=30000,
                                                          seed=seed),
                            np.array(extra_sizes, dtype=np.int64)])
    keys, off = inputs.bucketed_keys(sizes, seed=key_seed)
    return sizes, keys, off


def _oracle_bucket(keys, off, b, gamma=1230):
    k = keys[int(off[b]):int(off[b + 1])]
    n = len(k)
    m = oracle.num_vertices(n, gamma, 3)
    e = oracle.hash_edges(k, m, 3, b) if n else np.zeros((0, 3), np.uint32)
    return e, m, oracle.peel_rounds(e, m)


def _run(keys, off, with_g=False, tuning=None, gamma=1230):
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    do = torch.from_numpy(off.view(np.int64)).cuda()
    res = hp.peel_batched(dk, do, gamma_milli=gamma, with_g=with_g, tuning=tuning)
    torch.cuda.synchronize()
    return res


def _check_all(keys, off, res, with_g=False, gamma=1230):
    order = res.order.cpu().numpy().view(np.uint32)
    rounds = res.rounds.cpu().numpy().view(np.uint32)
    status = res.status.cpu().numpy().view(np.uint32)
    G = res.G.cpu().numpy().view(np.uint64) if with_g else None
    G_off = res.G_off.cpu().numpy() if with_g else None
    B = len(off) - 1
    for b in range(B):
        n = int(off[b + 1] - off[b])
        if n > 65536:
            assert status[b] == 2
            continue
        e, m, want = _oracle_bucket(keys, off, b, gamma)
        assert rounds[b] == want.rounds, b
        assert status[b] == (1 if want.core_nonempty else 0), b
        assert np.array_equal(order[int(off[b]):int(off[b + 1])], want.order), b
        if with_g:
            words = (m + 31) // 32
            assert int(G_off[b + 1] - G_off[b]) == words
            got_g = G[int(G_off[b]):int(G_off[b]) + words]
            if want.core_nonempty:
                assert not got_g.any()
            else:
                assert np.array_equal(got_g, oracle.mphf_assign(e, m, want)), b


def test_batched_parity_lognormal_buckets():
    # lognormal sizes plus edge cases: empty, 1..3 keys (tiny m, 2-cores),
    # buckets beyond shared memory (global path, 32-bit records below 65,535
    # keys, 64-bit from there), the 65,536-key maximum and one bucket over
    # the limit
    sizes, keys, off = _workload(extra_sizes=[0, 1, 2, 3, 64, 4097, 20000, 65534, 65535, 65536,
                                              70000])
    res = _run(keys, off)
    _check_all(keys, off, res)


def test_batched_parity_with_g():
    sizes, keys, off = _workload(B=160, median=900, seed=5, key_seed=7,
                                 extra_sizes=[17, 30000])
    res = _run(keys, off, with_g=True)
    _check_all(keys, off, res, with_g=True)


@pytest.mark.parametrize("tuning", [
    {"threads": 128, "ctas_per_sm": 1},
    {"threads": 512, "ctas_per_sm": 4},
    {"threads": 256, "ctas_per_sm": 2, "smem_bytes": 4096},   # nearly all on the global path
    {"threads": 64, "ctas_per_sm": 8},
    # a layer table of 3 entries in shared memory: every bucket of more than
    # one round is peeled again in the workspace
    {"threads": 256, "ctas_per_sm": 8, "smem_rounds": 3},
    # and 3 entries on the 32-bit global path as well: every bucket of more
    # than one round ends on the 64-bit path (64-bit records, 32-bit claims)
    {"threads": 256, "ctas_per_sm": 8, "smem_rounds": 3, "global16_rounds": 3},
])
def test_batched_results_do_not_depend_on_tuning(tuning):
    sizes, keys, off = _workload(B=120, median=700, seed=11, key_seed=13, extra_sizes=[25000])
    ref = _run(keys, off, with_g=True)
    got = _run(keys, off, with_g=True, tuning=tuning)
    for a in ("order", "rounds", "status", "G"):
        assert torch.equal(getattr(ref, a), getattr(got, a)), a
    _check_all(keys, off, got, with_g=True)


def test_batched_other_gamma():
    # near and below the threshold: many rounds, frequent 2-cores
    for gamma in (1200, 1222, 1400):
        sizes, keys, off = _workload(B=100, median=1500, seed=gamma, key_seed=gamma + 1)
        res = _run(keys, off, gamma=gamma)
        _check_all(keys, off, res, gamma=gamma)


def test_batched_captured_in_cuda_graph():
    sizes, keys, off = _workload(B=200, median=800, seed=17, key_seed=19)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    do = torch.from_numpy(off.view(np.int64)).cuda()
    B = len(off) - 1
    ws = torch.empty(hp.batched_workspace_size(B), dtype=torch.uint8, device="cuda")
    G_off = hp.batched_g_offsets(do, workspace=ws)
    out = hp.BatchedResult(torch.empty(len(keys), dtype=torch.int32, device="cuda"),
                           torch.empty(B, dtype=torch.int32, device="cuda"),
                           torch.empty(B, dtype=torch.int32, device="cuda"),
                           torch.empty(int(G_off[-1].item()), dtype=torch.int64, device="cuda"),
                           G_off)
    # warm-up outside the graph (first launch sets the kernel attributes)
    hp.peel_batched(dk, do, workspace=ws, out=out)
    torch.cuda.synchronize()
    ref = [out.order.clone(), out.rounds.clone(), out.G.clone()]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out.order.fill_(-1)
        with torch.cuda.graph(g, stream=s):
            hp.peel_batched(dk, do, workspace=ws, out=out)
    torch.cuda.synchronize()
    for _ in range(2):
        out.order.fill_(-1)
        out.G.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out.order, ref[0]) and torch.equal(out.rounds, ref[1])
        assert torch.equal(out.G, ref[2])


def test_batched_rejects_bad_arguments():
    keys = torch.zeros(4, dtype=torch.int64, device="cuda")
    off = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp.peel_batched(keys, off, gamma_milli=2100)
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp.peel_batched(keys, off, tuning={"threads": 100})
    with pytest.raises(hp.HpeelError, match="WORKSPACE"):
        hp.peel_batched(keys, off, workspace=torch.empty(256, dtype=torch.uint8, device="cuda"))
