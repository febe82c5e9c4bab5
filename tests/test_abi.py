"""The C ABI library builds, loads without a GPU and exports every symbol the
headers in include/ declare.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

import paper_1312_0526_gb300 as hp
from paper_1312_0526_gb300 import build as hpbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(hpeel_\w+)\s*\(", src):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    hpbuild.build()
    return hp.lib()


def test_headers_declare_the_boundary():
    names = _declared_functions()
    for want in ("hpeel_hash_edges", "hpeel_peel", "hpeel_mphf_build",
                 "hpeel_peel_workspace_size", "hpeel_mphf_workspace_size",
                 "hpeel_num_vertices", "hpeel_status_str", "hpeel_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(hp.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(raw, n)]
    assert missing == []


def test_host_only_calls(lib):
    assert lib.hpeel_version() >= 100
    assert lib.hpeel_status_str(0) == b"ok"
    assert b"2-core" in lib.hpeel_status_str(6)
    # vertex counts of the workloads (hand-computed, see the oracle pins)
    assert hp.num_vertices(100_000, 1230, 3) == 123_000
    assert hp.num_vertices(10**9, 1222, 3) == 1_222_000_002
    assert hp.num_vertices(10**8, 1300, 4) == 130_000_000
    assert hp.num_vertices(0, 1230, 3) == 0


def test_workspace_sizes_grow_with_n(lib):
    a = hp.peel_workspace_size(1000, 1230, 3)
    b = hp.peel_workspace_size(100_000, 123_000, 3)
    assert 0 < a < b
    # 8 B record + 4 B frontier per vertex, 4 B claim + 4 B layer per edge
    assert b >= 12 * 123_000 + 8 * 100_000
    assert hp.mphf_workspace_size(100_000) > b


def test_host_side_argument_checks(lib):
    # refused on the host before any device work (no GPU needed)
    INVALID = 1
    raw = ctypes.CDLL(hp.LIB_PATH)
    u64, u32, vp, sz = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t
    for fn in (raw.hpeel_peel_async, raw.hpeel_peel_general_async):
        fn.restype = ctypes.c_int
        fn.argtypes = [vp, u64, u64, u32, vp, vp, vp, u32, vp, vp, sz, vp]
        assert fn(None, 10, 30, 5, None, None, None, 0, None, None, 0, None) == INVALID  # r
        assert fn(None, 10, 30, 3, None, None, None, 0, None, None, 0, None) == INVALID  # stats
        assert fn(None, 2**32, 30, 3, None, None, None, 0, None, None, 0, None) == INVALID
    raw.hpeel_sf_build_async.restype = ctypes.c_int
    raw.hpeel_sf_build_async.argtypes = [vp, vp, u64, u64, u64, u32, u32, vp, vp, vp, sz, vp]
    assert raw.hpeel_sf_build_async(None, None, 10, 1, 1, 1230, 8, None, None, None, 0,
                                    None) == INVALID  # sigma < 2
    assert raw.hpeel_sf_build_async(None, None, 10, 5, 1, 1230, 0, None, None, None, 0,
                                    None) == INVALID  # max_tries
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp.set_tuning(bucket_part_passes=3)
    with pytest.raises(hp.HpeelError, match="INVALID_ARG"):
        hp.set_tuning(bucket_sub_shift=15)
    hp.set_tuning()
    assert hp.get_tuning()["bucket_part_passes"] == 0
    # an invalid batched launch shape has no workspace size (0)
    assert hp.batched_workspace_size(4, 1230, {"threads": 256, "ctas_per_sm": 2,
                                               "smem_rounds": 1}) == 0
    assert hp.batched_workspace_size(4, 1230, {"threads": 256, "ctas_per_sm": 2,
                                               "smem_rounds": 2}) > 0
    # the 16-bit claim words of the global path hold at most 16,383 rounds
    assert hp.batched_workspace_size(4, 1230, {"global16_rounds": 1}) == 0
    assert hp.batched_workspace_size(4, 1230, {"global16_rounds": 16384}) == 0
    assert hp.batched_workspace_size(4, 1230, {"global16_rounds": 16383}) > 0


def test_one_part_per_pass_takes_a_smaller_workspace(lib):
    # sec. 4.3's one part at a time: the L2-blocked build's buckets hold one
    # incidence per edge instead of r
    n = 10**6
    m = hp.num_vertices(n)
    try:
        hp.set_tuning(bucket_shift=14, bucket_min_vertices=0, bucket_part_passes=1)
        one = hp.peel_workspace_size(n, m)
        hp.set_tuning(bucket_shift=14, bucket_min_vertices=0, bucket_part_passes=2)
        per_part = hp.peel_workspace_size(n, m)
    finally:
        hp.set_tuning()
    assert per_part < one - 20 * n
    # automatic above 2^30 edges: about 51 B per edge at gamma = 1.23
    n = 3 * 10**9
    assert hp.peel_workspace_size(n, hp.num_vertices(n)) < 52 * n


def test_binding_rejects_host_tensors(lib):
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        hp.hash_edges(torch.zeros(4, dtype=torch.int64), 6, 3, 1)
    with pytest.raises(ValueError):
        hp.peel(torch.zeros((4, 3), dtype=torch.int32), 6)


def test_oracle_is_not_imported_by_the_product():
    # the product package never imports the oracle
    for f in glob.glob(os.path.join(ROOT, "paper_1312_0526_gb300", "**", "*.py"), recursive=True):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
    for f in glob.glob(os.path.join(ROOT, "paper_1312_0526_gb300", "csrc", "*")):
        assert "hpeel_oracle" not in open(f).read(), f


def test_measurement_probe_is_a_separate_library(lib):
    # the benchmark's random-access probe lives in its own library: the
    # peeling library exports no probe symbol
    from paper_1312_0526_gb300 import measure
    raw = ctypes.CDLL(hp.LIB_PATH)
    assert not hasattr(raw, "hpeel_measure_random_access")
    ml = measure.lib()
    assert ml.hpeel_measure_random_access(3, 10, None, 0, None, 0, 1, None) == 1
    assert ml.hpeel_measure_random_access(2, 10, None, 0, None, 0, 1, None) == 1
