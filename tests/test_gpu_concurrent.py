"""Concurrent builds: several host threads, each with its own CUDA stream and
workspace, run MPHF builds at the same time (the serving pattern).  The
kernels of one build then share the GPU with other builds' kernels, so the
blocks of one launch can start far apart in time; the round-synchronous peel
must give exactly what it gives alone.  Every concurrent result is compared
bit for bit with the same build run by itself, and a sample with the oracle.
"""
import threading

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


def _key_sets(count, seed):
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(500), np.log(400_000), count)).astype(np.int64)
    return [inputs.keys(int(s), 7000 + i) for i, s in enumerate(sizes)]


def _alone(key_sets):
    out = []
    for k in key_sets:
        r = hp.mphf_build(torch.from_numpy(k.view(np.int64)).cuda(), seed=1, max_tries=32)
        out.append((r.G.cpu(), r.rank_dir.cpu(), r.stats["seed_used"]))
    return out


def _together(key_sets, threads):
    results = [None] * len(key_sets)
    errors = []
    nxt = [0]
    lock = threading.Lock()

    def worker():
        stream = torch.cuda.Stream()
        ws = None
        try:
            with torch.cuda.stream(stream):
                while True:
                    with lock:
                        i = nxt[0]
                        nxt[0] += 1
                    if i >= len(key_sets):
                        return
                    n = key_sets[i].shape[0]
                    need = hp.mphf_workspace_size(n)
                    if ws is None or ws.numel() < need:  # grows like a server slot's
                        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
                    keys = torch.from_numpy(key_sets[i].view(np.int64)).pin_memory().to(
                        "cuda", non_blocking=True)
                    r = hp.mphf_build(keys, seed=1, max_tries=32, workspace=ws)
                    results[i] = (r.G.cpu(), r.rank_dir.cpu(), r.stats["seed_used"])
        except Exception as e:  # reported by the main thread
            errors.append(e)

    ts = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in ts), "a build did not finish"
    assert not errors, errors[0]
    return results


@pytest.mark.parametrize("loop", ["graph", "host"])
def test_concurrent_builds_match_alone(loop):
    if loop == "host":
        hp.set_tuning(host_round_loop=1)
    try:
        key_sets = _key_sets(48, 11)
        want = _alone(key_sets)
        for rep in range(3):
            got = _together(key_sets, threads=4)
            for i, (g, w) in enumerate(zip(got, want)):
                assert g[2] == w[2], (rep, i)
                assert torch.equal(g[0], w[0]) and torch.equal(g[1], w[1]), (rep, i)
    finally:
        hp.set_tuning()
    # the sequential builds themselves agree with the oracle (a sample)
    for i in (0, 7, 23):
        o = oracle.mphf_build(key_sets[i], seed=1, max_tries=32)
        assert want[i][2] == o.seed_used
        assert np.array_equal(want[i][0].numpy().view(np.uint64), o.G)
        assert np.array_equal(want[i][1].numpy().view(np.uint64), o.dir)
