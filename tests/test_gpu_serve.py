"""Continuous-batching MPHF server: results are identical alone and in the
mix, admission respects the device-memory budget, failed/oversized requests
are reported, reseeding works inside the server."""
import numpy as np
import pytest

import oracle
from paper_1312_0526_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1312_0526_gb300 as hp  # noqa: E402
from paper_1312_0526_gb300 import serve  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_0526_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _stream(num, seed=4, lo=3.0, hi=5.0):
    arr, sizes, seeds = inputs.request_stream(num, rate_per_s=1e9, seed=seed, lo_exp=lo, hi_exp=hi)
    return [inputs.keys(int(s), int(k)) for s, k in zip(sizes, seeds)]


def _same(a, b):
    assert a.error is None and b.error is None
    assert a.stats["seed_used"] == b.stats["seed_used"]
    assert torch.equal(a.G, b.G) and torch.equal(a.rank_dir, b.rank_dir)


def test_results_same_alone_and_in_the_mix():
    keysets = _stream(30)
    mix = serve.MphfServer(slots=4, hbm_budget=8 << 30)
    try:
        got = serve.run_stream(mix, keysets, [0.0] * len(keysets))
        assert mix.max_running > 1  # the builds really overlapped
    finally:
        mix.close()
    alone = serve.MphfServer(slots=1, hbm_budget=8 << 30)
    try:
        for i, ks in enumerate(keysets):
            alone.results.clear()
            alone.submit(serve.Request(0, ks, 1))
            alone.wait(1)
            _same(got[i], alone.results[0])
    finally:
        alone.close()
    # and against the oracle for a few of them
    for i in (0, 7, 19):
        want = oracle.mphf_build(keysets[i], seed=1)
        assert np.array_equal(got[i].G.cpu().numpy().view(np.uint64), want.G)
        assert np.array_equal(got[i].rank_dir.cpu().numpy().view(np.uint64), want.dir)


def test_admission_respects_the_budget():
    keysets = _stream(16, seed=9, lo=4.0, hi=5.0)
    budget = max(serve.footprint_bytes(len(k)) for k in keysets) * 2
    srv = serve.MphfServer(slots=8, hbm_budget=budget)
    try:
        res = serve.run_stream(srv, keysets, [0.0] * len(keysets))
    finally:
        srv.close()
    assert all(r.error is None for r in res)
    assert srv.max_in_use <= budget


@pytest.mark.parametrize("keep", [False, True])
def test_admission_bounds_the_allocated_device_memory(keep):
    # mixed 1e5..1e7-key requests on 4 slots: the memory torch's allocator
    # hands out while the server runs (retained slot workspaces, key copies,
    # outputs, kept results) stays within the budget plus a small slack for
    # the allocator's rounding
    arr, sizes, seeds = inputs.request_stream(12, rate_per_s=1e9, seed=13, lo_exp=5.0,
                                              hi_exp=7.0)
    keysets = [torch.from_numpy(inputs.keys(int(s), int(k)).view(np.int64)).pin_memory()
               for s, k in zip(sizes, seeds)]
    budget = int(1.5 * max(serve.footprint_bytes(len(k)) for k in keysets))
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    srv = serve.MphfServer(slots=4, hbm_budget=budget, keep_results=keep)
    try:
        res = serve.run_stream(srv, keysets, [0.0] * len(keysets))
        assert all(r.error is None for r in res)
        assert srv.max_in_use <= budget
        torch.cuda.synchronize()
        peak = torch.cuda.max_memory_allocated() - base
        assert peak <= budget + (16 << 20), (peak, budget)
        for i in range(len(keysets)):
            srv.release(i)
        res = None  # the caller's references to the outputs go too
    finally:
        srv.close()
    assert srv.in_use == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_large_requests_same_alone_and_in_the_mix():
    # a mix that reaches 1e6..1e7 keys per request (the top of the serving
    # workload's log-uniform range): each result equals the same build alone
    arr, sizes, seeds = inputs.request_stream(8, rate_per_s=1e9, seed=17, lo_exp=6.0,
                                              hi_exp=7.0)
    keysets = [inputs.keys(int(s), int(k)) for s, k in zip(sizes, seeds)]
    assert max(sizes) > 3_000_000
    mix = serve.MphfServer(slots=4, hbm_budget=32 << 30)
    try:
        got = serve.run_stream(mix, keysets, [0.0] * len(keysets))
        assert mix.max_running > 1
    finally:
        mix.close()
    alone = serve.MphfServer(slots=1, hbm_budget=32 << 30)
    try:
        for i, ks in enumerate(keysets):
            alone.results.clear()
            alone.submit(serve.Request(0, ks, 1))
            alone.wait(1)
            _same(got[i], alone.results[0])
    finally:
        alone.close()
    # the largest request against the oracle
    i = int(np.argmax(sizes))
    want = oracle.mphf_build(keysets[i], seed=1, max_tries=8)
    assert got[i].stats["seed_used"] == want.seed_used
    assert np.array_equal(got[i].G.cpu().numpy().view(np.uint64), want.G)
    assert np.array_equal(got[i].rank_dir.cpu().numpy().view(np.uint64), want.dir)


def test_oversized_request_is_reported_and_others_finish():
    keysets = _stream(5, seed=11)
    big = inputs.keys(3_000_000, 5)
    srv = serve.MphfServer(slots=2, hbm_budget=serve.footprint_bytes(200_000))
    try:
        res = serve.run_stream(srv, keysets + [big], [0.0] * 6)
    finally:
        srv.close()
    assert res[-1].error and "budget" in res[-1].error
    assert all(r.error is None for r in res[:-1])


def test_reseed_inside_the_server():
    # a key set whose first hash seed leaves a 2-core
    for s in range(300):
        k = inputs.keys(60, 3000 + s)
        m = oracle.num_vertices(60, 1230, 3)
        if oracle.peel_rounds(oracle.hash_edges(k, m, 3, 1), m).core_nonempty:
            break
    srv = serve.MphfServer(slots=2, max_tries=64)
    try:
        res = serve.run_stream(srv, [k, inputs.keys(5000, 1)], [0.0, 0.0])
    finally:
        srv.close()
    want = oracle.mphf_build(k, seed=1, max_tries=64)
    assert res[0].stats["attempts"] > 1 and res[0].stats["seed_used"] == want.seed_used
    assert np.array_equal(res[0].G.cpu().numpy().view(np.uint64), want.G)
    summary = serve.latency_summary(res)
    assert summary["requests"] == 2 and summary["failed"] == 0
