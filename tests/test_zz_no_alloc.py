"""hpeel_peel_noalloc against hpeel_peel.

The no-allocation entry point serves callers that cannot allocate device
memory when they peel (code inside another runtime's memory pool, fixed
memory budgets, plugins barred from the allocator).  It must give exactly the
results of the workspace entry point, call after call, even though every
call reuses the one scratch array compiled into the library, and it must
leave the device's free memory where it was.  This file is collected last so
that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1312_0526_gb300 as hp  # noqa: E402
from paper_1312_0526_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_0526_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(params=[0, 1], ids=["graph_loop_tuning", "host_loop_tuning"])
def round_loop(request):
    # the no-allocation call always launches its rounds from the host; the
    # workspace call it is compared with follows the tuning
    before = hp.get_tuning()
    hp.set_tuning(host_round_loop=request.param)
    yield request.param
    hp.set_tuning(**before)


def _edges(n, gamma, seed):
    m = hp.num_vertices(n, gamma, 3)
    keys = torch.from_numpy(inputs.keys(n, seed).view(np.int64)).cuda()
    return hp.hash_edges(keys, m, 3, 1), m


def _chain(n):
    """A band-shaped 3-hypergraph that peels a few edges per round from both
    ends: more rounds (> 300) than one pass of the order sort has bins."""
    P = n
    e = np.zeros((n, 3), dtype=np.uint32)
    for i in range(n):
        k, q = divmod(i, 4)
        e[i] = ((i + 1) // 2, P + i // 2, 2 * P + 2 * k + (q % 2))
    return torch.from_numpy(e.view(np.int32)).cuda(), 3 * P


def _same(a, b):
    assert a.rounds == b.rounds and a.n_peeled == b.n_peeled
    assert torch.equal(a.order, b.order)
    assert torch.equal(a.claim, b.claim)
    assert torch.equal(a.layer_off, b.layer_off)


def test_noalloc_matches_workspace_peel_on_two_calls_in_a_row(round_loop):
    # first a larger graph that fills most of the scratch, then a smaller one
    # with a 2-core: stale contents of the first call must not leak into the
    # second
    e1, m1 = _edges(400_000, 1230, 1)
    e2, m2 = _edges(60_000, 1200, 2)
    want1 = hp.peel(e1, m1)
    want2 = hp.peel(e2, m2)
    got1 = hp.peel_noalloc(e1, m1)
    got2 = hp.peel_noalloc(e2, m2)
    torch.cuda.synchronize()
    _same(got1, want1)
    _same(got2, want2)
    assert want2.core_nonempty and not want1.core_nonempty


def test_noalloc_many_rounds_multi_pass_order(round_loop):
    # > 256 rounds: the canonical order takes the multi-pass sort (its tail
    # re-sorted inside the scratch)
    e, m = _chain(1203)
    want = hp.peel(e, m)
    assert want.rounds > 300
    _same(hp.peel_noalloc(e, m), want)
    _same(hp.peel_noalloc(e, m), want)


def _host(res):
    # host copies only: a comparison on the device could make torch's
    # allocator take a new block while free memory is being watched
    return (res.rounds, res.n_peeled, res.order.cpu(), res.claim.cpu(), res.layer_off.cpu())


def test_noalloc_leaves_free_device_memory_unchanged():
    sizes = [(400_000, 1230, 1), (5_000, 1230, 4), (60_000, 1200, 2)]
    graphs = [_edges(*s) for s in sizes]
    wants = [_host(hp.peel(e, m)) for e, m in graphs]
    outs = [(torch.empty(e.shape[0], dtype=torch.int32, device="cuda"),
             torch.empty(e.shape[0], dtype=torch.int32, device="cuda"),
             torch.empty(4097, dtype=torch.int64, device="cuda")) for e, _ in graphs]
    # one call of each size first: the driver loads the device code and
    # reserves the kernels' local memory on first use
    for (e, m), o in zip(graphs, outs):
        hp.peel_noalloc(e, m, out=o)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for (e, m), o, want in zip(graphs, outs, wants):
            got = _host(hp.peel_noalloc(e, m, out=o))
            assert got[:2] == want[:2]
            assert all(torch.equal(a, b) for a, b in zip(got[2:], want[2:]))
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_noalloc_rejects_graphs_beyond_the_scratch():
    n = 600_000
    m = hp.num_vertices(n, 1230, 3)
    assert hp.peel_workspace_size(n, m, 3) > hp.NOALLOC_SCRATCH_BYTES
    e = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(hp.HpeelError, match="WORKSPACE_TOO_SMALL"):
        hp.peel_noalloc(e, m)
    # the library stays usable after the refusal
    e2, m2 = _edges(1000, 1230, 3)
    _same(hp.peel_noalloc(e2, m2), hp.peel(e2, m2))
