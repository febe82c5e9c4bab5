"""hpeel_peel_noalloc against hpeel_peel.

The no-allocation entry point serves callers that cannot allocate device
memory when they peel (code inside another runtime's memory pool, fixed
memory budgets, plugins barred from the allocator).  It must give exactly the
results of the workspace entry point, call after call, even though every
call reuses the one scratch array compiled into the library.  This file is
collected last so that a failure here leaves every other test already run.
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


def _edges(n, gamma, seed):
    m = hp.num_vertices(n, gamma, 3)
    keys = torch.from_numpy(inputs.keys(n, seed).view(np.int64)).cuda()
    return hp.hash_edges(keys, m, 3, 1), m


def _same(a, b):
    assert a.rounds == b.rounds and a.n_peeled == b.n_peeled
    assert torch.equal(a.order, b.order)
    assert torch.equal(a.claim, b.claim)
    assert torch.equal(a.layer_off, b.layer_off)


def test_noalloc_matches_workspace_peel_on_two_calls_in_a_row():
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
