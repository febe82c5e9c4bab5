"""The benchmark's random-access probe (measure/probe.cu, a library of its
own) does the operations it states: every atomicAdd lands (the words sum to
the operation count) and every claim lowers a record's claim word to an
operation number."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1312_0526_gb300 import measure  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_0526_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_probe_rmw_and_load():
    words = torch.zeros(1001, dtype=torch.int64, device="cuda")
    measure.random_access(1, 50_000, words)
    assert int(words.sum()) == 0
    measure.random_access(0, 50_000, words, seed=3)
    assert int(words.sum()) == 50_000
    assert int((words > 0).sum()) > 900  # spread over the words


def test_probe_peeled_edge():
    n_ops, n_rec = 40_000, 3001
    rec = torch.full((n_rec, 4), -1, dtype=torch.int32, device="cuda")
    words = torch.zeros(777, dtype=torch.int64, device="cuda")
    measure.random_access(2, n_ops, rec, words, seed=5)
    assert int(words.sum()) == 2 * n_ops
    # records read 0xFFFFFFFF in their first word, so the claim hit word 2
    claim = rec[:, 2].cpu().numpy().view("uint32")
    touched = claim != 0xFFFFFFFF
    assert touched.sum() > 0.9 * n_rec
    assert (claim[touched] < n_ops).all()
    assert (rec[:, [0, 1, 3]] == -1).all()


def test_probe_rejects_bad_kind():
    words = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError, match="refused"):
        measure.random_access(3, 10, words)
