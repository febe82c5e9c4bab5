"""GB300 (sm_103a) hypergraph peeling and MWHC minimal perfect hashing.

Thin Python binding over the C ABI in ``include/hpeel.h`` (library
``_build/libhpeel.so``, built by ``paper_1312_0526_gb300.build``).  The
functions here only marshal arguments: torch tensors provide device memory
and the current CUDA stream, and every step runs in the library's kernels.
There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.

Tensor conventions (torch has no full unsigned support, so unsigned data is
carried in signed tensors of the same width, bit for bit):
  keys      int64 [n]       (uint64 keys)
  edges     int32 [n, r]    (uint32 vertex ids)
  order     int32 [n]       (uint32 edge ids)
  claim     int32 [n]       (uint32 claim words, -1 = HPEEL_UNCLAIMED)
  layer_off int64 [R + 1]
  G         int64 [ceil(m/32)], rank_dir int64 [ceil(m/512) + 1]
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhpeel.so")


def _build_dir() -> str:
    d = os.path.join(_HERE, "_build")
    os.makedirs(d, exist_ok=True)
    return d
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "hpeel.h")

UNCLAIMED = 0xFFFFFFFF
MAX_ROUNDS = 1 << 20

STATUS = {
    0: "HPEEL_OK", 1: "HPEEL_ERR_INVALID_ARG", 2: "HPEEL_ERR_CUDA",
    3: "HPEEL_ERR_WORKSPACE_TOO_SMALL", 4: "HPEEL_ERR_TIMEOUT", 5: "HPEEL_ERR_DEVICE_CHECK",
    6: "HPEEL_ERR_CORE_NONEMPTY", 7: "HPEEL_ERR_RETRIES_EXHAUSTED", 8: "HPEEL_ERR_CAPACITY",
}


class HpeelError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Tuning(ctypes.Structure):
    _fields_ = [("bucket_shift", ctypes.c_uint32), ("bucket_min_vertices", ctypes.c_uint32),
                ("host_round_loop", ctypes.c_uint32), ("bucket_sub_shift", ctypes.c_uint32),
                ("bucket_part_passes", ctypes.c_uint32), ("sorted_round_min", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 2)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("smem_bytes", ctypes.c_uint32), ("smem_rounds", ctypes.c_uint32),
                ("global16_rounds", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 3)]


class Stats(ctypes.Structure):
    _fields_ = [("n_peeled", ctypes.c_uint64), ("rounds", ctypes.c_uint32),
                ("core_nonempty", ctypes.c_uint32), ("seed_used", ctypes.c_uint64),
                ("attempts", ctypes.c_uint32), ("device_err", ctypes.c_uint32),
                ("first_layer", ctypes.c_uint64), ("frontier", ctypes.c_uint64),
                ("hinge_moves", ctypes.c_uint64), ("async_status", ctypes.c_uint32),
                ("sorted_rounds", ctypes.c_uint32), ("reserved", ctypes.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_
                if k != "reserved"}


_lib = None
_lib_lock = threading.Lock()


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1312_0526_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        u64, u32, p, sz = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t
        st = ctypes.c_int
        L.hpeel_status_str.restype = ctypes.c_char_p
        L.hpeel_status_str.argtypes = [st]
        L.hpeel_last_error.restype = ctypes.c_char_p
        L.hpeel_last_error.argtypes = []
        L.hpeel_version.restype = ctypes.c_int
        L.hpeel_num_vertices.restype = u64
        L.hpeel_num_vertices.argtypes = [u64, u32, u32]
        L.hpeel_hash_edges.restype = st
        L.hpeel_hash_edges.argtypes = [p, u64, u64, u32, u64, p, p]
        L.hpeel_peel_workspace_size.restype = sz
        L.hpeel_peel_workspace_size.argtypes = [u64, u64, u32]
        L.hpeel_peel.restype = st
        L.hpeel_peel.argtypes = [p, u64, u64, u32, p, p, p, u32, ctypes.POINTER(Stats), p, sz, p]
        L.hpeel_mphf_workspace_size.restype = sz
        L.hpeel_mphf_workspace_size.argtypes = [u64, u32]
        L.hpeel_mphf_build.restype = st
        L.hpeel_mphf_build.argtypes = [p, u64, u64, u32, u32, p, p, p, ctypes.POINTER(Stats), p,
                                       sz, p]
        L.hpeel_peel_noalloc.restype = st
        L.hpeel_peel_noalloc.argtypes = [p, u64, u64, u32, p, p, p, u32, ctypes.POINTER(Stats), p]
        L.hpeel_set_tuning.restype = st
        L.hpeel_set_tuning.argtypes = [ctypes.POINTER(Tuning)]
        L.hpeel_get_tuning.restype = None
        L.hpeel_get_tuning.argtypes = [ctypes.POINTER(Tuning)]
        L.hpeel_batched_workspace_size.restype = sz
        L.hpeel_batched_workspace_size.argtypes = [u32, u32, ctypes.POINTER(BatchTuning)]
        L.hpeel_batched_g_offsets.restype = st
        L.hpeel_batched_g_offsets.argtypes = [p, u32, u32, p, p, sz, p]
        L.hpeel_peel_batched.restype = st
        L.hpeel_peel_batched.argtypes = [p, p, u32, u32, p, p, p, p, p,
                                         ctypes.POINTER(BatchTuning), p, sz, p]
        L.hpeel_mphf_lookup.restype = st
        L.hpeel_mphf_lookup.argtypes = [p, u64, u64, u64, p, p, p, p]
        L.hpeel_hash_edges_general.restype = st
        L.hpeel_hash_edges_general.argtypes = [p, u64, u64, u32, u64, p, p]
        L.hpeel_peel_general_workspace_size.restype = sz
        L.hpeel_peel_general_workspace_size.argtypes = [u64, u64, u32]
        L.hpeel_peel_general.restype = st
        L.hpeel_peel_general.argtypes = [p, u64, u64, u32, p, p, p, u32, ctypes.POINTER(Stats),
                                         p, sz, p]
        L.hpeel_mphf_large_workspace_size.restype = sz
        L.hpeel_mphf_large_workspace_size.argtypes = [u64, u32, ctypes.c_int]
        L.hpeel_mphf_build_large.restype = st
        L.hpeel_mphf_build_large.argtypes = [p, u64, u64, u32, u32, p, p, ctypes.POINTER(Stats),
                                             p, sz, p, p]
        L.hpeel_mphf_lookup_large.restype = st
        L.hpeel_mphf_lookup_large.argtypes = [p, u64, u64, u64, p, p, p, p]
        L.hpeel_peel_async.restype = st
        L.hpeel_peel_async.argtypes = [p, u64, u64, u32, p, p, p, u32, p, p, sz, p]
        L.hpeel_peel_general_async.restype = st
        L.hpeel_peel_general_async.argtypes = [p, u64, u64, u32, p, p, p, u32, p, p, sz, p]
        L.hpeel_sf_build_async.restype = st
        L.hpeel_sf_build_async.argtypes = [p, p, u64, u64, u64, u32, u32, p, p, p, sz, p]
        L.hpeel_mphf_build_async.restype = st
        L.hpeel_mphf_build_async.argtypes = [p, u64, u64, u32, u32, p, p, p, p, sz, p]
        L.hpeel_sf_bits.restype = u32
        L.hpeel_sf_bits.argtypes = [u64]
        L.hpeel_sf_words.restype = u64
        L.hpeel_sf_words.argtypes = [u64, u32, u64]
        L.hpeel_sf_workspace_size.restype = sz
        L.hpeel_sf_workspace_size.argtypes = [u64, u32]
        L.hpeel_sf_build.restype = st
        L.hpeel_sf_build.argtypes = [p, p, u64, u64, u64, u32, u32, p, ctypes.POINTER(Stats),
                                     p, sz, p]
        L.hpeel_sf_lookup.restype = st
        L.hpeel_sf_lookup.argtypes = [p, u64, u64, u64, u64, p, p, p]
        L.hpeel_kernel_launches.restype = u64
        L.hpeel_kernel_launches.argtypes = []
        L.hpeel_profile_enable.restype = None
        L.hpeel_profile_enable.argtypes = [ctypes.c_int]
        L.hpeel_profile_reset.restype = None
        L.hpeel_profile_reset.argtypes = []
        L.hpeel_profile_read.restype = sz
        L.hpeel_profile_read.argtypes = [ctypes.c_char_p, sz]
        _lib = L
        return L


def _check(rc: int):
    if rc != 0:
        raise HpeelError(rc, lib().hpeel_last_error().decode())


def _torch():
    import torch
    return torch


def _dev_ptr(t, name, dtype=None, ndim=None, host_ok=False):
    """Address of a contiguous CUDA tensor (or, with host_ok, of a tensor in
    pinned host memory, which the kernels read in place over the host link)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or (host_ok and t.is_pinned())):
        raise ValueError(f"{name} must be a CUDA tensor" +
                         (" or a pinned host tensor" if host_ok else ""))
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _workspace(nbytes: int, device):
    torch = _torch()
    # 256-byte alignment: the caching allocator hands out 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def num_vertices(n: int, gamma_milli: int = 1230, r: int = 3) -> int:
    """m = r * ceil(ceil(gamma n) / r) (sec. 3, sec. 4.3)."""
    return int(lib().hpeel_num_vertices(n, gamma_milli, r))


def hash_edges(keys, m: int, r: int = 3, seed: int = 1, out=None, general: bool = False):
    """Edges int32[n, r] of the keys (sec. 3 hashing, sec. 4.3 r parts; with
    general=True every vertex in [0, m), see hpeel_hash_edges_general)."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1)
    n = keys.shape[0]
    if out is None:
        out = torch.empty((n, r), dtype=torch.int32, device=keys.device)
    ep = _dev_ptr(out, "out", torch.int32)
    if out.numel() != n * r:
        raise ValueError("out must hold n * r entries")
    fn = lib().hpeel_hash_edges_general if general else lib().hpeel_hash_edges
    _check(fn(kp, n, m, r, seed, ep, _stream()))
    return out


@dataclass
class PeelResult:
    order: object      # int32 [n]
    claim: object      # int32 [n]
    layer_off: object  # int64 [rounds + 1]
    rounds: int
    n_peeled: int

    @property
    def core_nonempty(self) -> bool:
        return self.n_peeled < self.order.shape[0]


def peel_workspace_size(n: int, m: int, r: int = 3, general: bool = False) -> int:
    if general:
        return int(lib().hpeel_peel_general_workspace_size(n, m, r))
    return int(lib().hpeel_peel_workspace_size(n, m, r))


def peel(edges, m: int, workspace=None, max_layers: int = 4096,
         general: bool = False, out=None) -> PeelResult:
    """Round-synchronous peel with canonical order (sec. 4.2); see hpeel_peel,
    or hpeel_peel_general for a general (not r-partite) hypergraph.  out:
    None, or a tuple (order int32 [n], claim int32 [n], layer_off int64
    [max_layers + 1]) of buffers to write."""
    torch = _torch()
    ep = _dev_ptr(edges, "edges", torch.int32, 2)
    n, r = edges.shape
    dev = edges.device
    if out is None:
        order = torch.empty(n, dtype=torch.int32, device=dev)
        claim = torch.empty(n, dtype=torch.int32, device=dev)
        loff = torch.empty(max_layers + 1, dtype=torch.int64, device=dev)
    else:
        order, claim, loff = out
        if order.numel() < n or claim.numel() < n or loff.numel() < max_layers + 1:
            raise ValueError("out buffers too small: need n, n and max_layers + 1 entries")
    need = peel_workspace_size(n, m, r, general)
    ws = workspace if workspace is not None else _workspace(need, dev)
    wp = _dev_ptr(ws, "workspace", torch.uint8)
    st = Stats()
    fn = lib().hpeel_peel_general if general else lib().hpeel_peel
    _check(fn(ep, n, m, r, _dev_ptr(order, "order"), _dev_ptr(claim, "claim"),
              _dev_ptr(loff, "layer_off"), max_layers, ctypes.byref(st), wp, ws.numel(),
              _stream()))
    R = int(st.rounds)
    res = PeelResult(order, claim, loff[:R + 1], R, int(st.n_peeled))
    res.stats = st.as_dict()
    return res


@dataclass
class AsyncPeel:
    order: object      # int32 [n]
    claim: object      # int32 [n]
    layer_off: object  # int64 [max_layers + 1]: entries 0..rounds written
    stats: object      # uint8 [sizeof(hpeel_stats)] device memory


def peel_async(edges, m: int, workspace=None, max_layers: int = 4096, general: bool = False,
               out=None) -> AsyncPeel:
    """Device-driven peel (hpeel_peel_async, or hpeel_peel_general_async):
    enqueued as one CUDA graph on the current stream, no host
    synchronisation.  Read the stats with stats_from_device once the stream
    is done.  out: an AsyncPeel of buffers to reuse (the graph is cached by
    the set of pointers)."""
    torch = _torch()
    ep = _dev_ptr(edges, "edges", torch.int32, 2)
    n, r = edges.shape
    dev = edges.device
    if out is None:
        out = AsyncPeel(torch.empty(n, dtype=torch.int32, device=dev),
                        torch.empty(n, dtype=torch.int32, device=dev),
                        torch.empty(max_layers + 1, dtype=torch.int64, device=dev),
                        torch.zeros(ctypes.sizeof(Stats), dtype=torch.uint8, device=dev))
    elif out.layer_off.numel() < max_layers + 1:
        raise ValueError("layer_off must hold max_layers + 1 entries")
    ws = workspace if workspace is not None else _workspace(
        peel_workspace_size(n, m, r, general), dev)
    fn = lib().hpeel_peel_general_async if general else lib().hpeel_peel_async
    _check(fn(ep, n, m, r, _dev_ptr(out.order, "order"), _dev_ptr(out.claim, "claim"),
              _dev_ptr(out.layer_off, "layer_off"), max_layers,
              _dev_ptr(out.stats, "stats", torch.uint8), _dev_ptr(ws, "workspace", torch.uint8),
              ws.numel(), _stream()))
    return out


def mphf_lookup(keys, seed: int, m: int, G, rank_dir, out=None):
    """MPHF values of the query keys (hpeel_mphf_lookup): int32 [nq]."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1)
    if out is None:
        out = torch.empty(keys.shape[0], dtype=torch.int32, device=keys.device)
    _check(lib().hpeel_mphf_lookup(kp, keys.shape[0], seed, m, _dev_ptr(G, "G", torch.int64),
                                   _dev_ptr(rank_dir, "rank_dir", torch.int64),
                                   _dev_ptr(out, "out", torch.int32), _stream()))
    return out


@dataclass
class SfResult:
    U: object     # torch.int64 [hpeel_sf_words]: the b-bit values u, one bit string
    m: int
    sigma: int
    bits: int
    stats: dict


def sf_bits(sigma: int) -> int:
    """ceil(log2 sigma): bits per vertex of a static function."""
    return int(lib().hpeel_sf_bits(sigma))


def sf_workspace_size(n: int, gamma_milli: int = 1230) -> int:
    return int(lib().hpeel_sf_workspace_size(n, gamma_milli))


def sf_build(keys, values, sigma: int, seed: int = 1, gamma_milli: int = 1230,
             max_tries: int = 8, workspace=None, U=None) -> SfResult:
    """Static function f(keys[i]) = values[i] in [0, sigma) (sec. 3); see
    hpeel_sf_build."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1, host_ok=True)
    vp = _dev_ptr(values, "values", torch.int32, 1, host_ok=True)
    n = keys.shape[0]
    if values.shape[0] != n:
        raise ValueError("values must hold n entries")
    dev = keys.device if keys.is_cuda else torch.device("cuda", torch.cuda.current_device())
    m = num_vertices(n, gamma_milli, 3)
    words = int(lib().hpeel_sf_words(n, gamma_milli, sigma))
    if U is None:
        U = torch.empty(max(words, 1), dtype=torch.int64, device=dev)
    elif U.numel() < words:
        raise ValueError("U must hold hpeel_sf_words entries")
    ws = workspace if workspace is not None else _workspace(sf_workspace_size(n, gamma_milli), dev)
    st = Stats()
    _check(lib().hpeel_sf_build(kp, vp, n, sigma, seed, gamma_milli, max_tries,
                                _dev_ptr(U, "U", torch.int64), ctypes.byref(st),
                                _dev_ptr(ws, "workspace", torch.uint8), ws.numel(), _stream()))
    return SfResult(U[:words], m, sigma, sf_bits(sigma), st.as_dict())


def sf_build_async(keys, values, sigma: int, seed: int = 1, gamma_milli: int = 1230,
                   max_tries: int = 8, workspace=None, U=None, stats=None):
    """Device-driven static-function build (hpeel_sf_build_async): one CUDA
    graph on the current stream, no host synchronisation.  Returns (U,
    stats), stats a device uint8 tensor holding an hpeel_stats."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1, host_ok=True)
    vp = _dev_ptr(values, "values", torch.int32, 1, host_ok=True)
    n = keys.shape[0]
    if values.shape[0] != n:
        raise ValueError("values must hold n entries")
    dev = keys.device if keys.is_cuda else torch.device("cuda", torch.cuda.current_device())
    words = int(lib().hpeel_sf_words(n, gamma_milli, sigma))
    if U is None:
        U = torch.empty(max(words, 1), dtype=torch.int64, device=dev)
    elif U.numel() < words:
        raise ValueError("U must hold hpeel_sf_words entries")
    if stats is None:
        stats = torch.zeros(ctypes.sizeof(Stats), dtype=torch.uint8, device=dev)
    ws = workspace if workspace is not None else _workspace(sf_workspace_size(n, gamma_milli), dev)
    _check(lib().hpeel_sf_build_async(kp, vp, n, sigma, seed, gamma_milli, max_tries,
                                      _dev_ptr(U, "U", torch.int64),
                                      _dev_ptr(stats, "stats", torch.uint8),
                                      _dev_ptr(ws, "workspace", torch.uint8), ws.numel(),
                                      _stream()))
    return U, stats


def sf_lookup(keys, seed: int, m: int, sigma: int, U, out=None):
    """f of the query keys (hpeel_sf_lookup): int32 [nq] holding uint32 values."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1)
    if out is None:
        out = torch.empty(keys.shape[0], dtype=torch.int32, device=keys.device)
    _check(lib().hpeel_sf_lookup(kp, keys.shape[0], seed, m, sigma, _dev_ptr(U, "U", torch.int64),
                                 _dev_ptr(out, "out", torch.int32), _stream()))
    return out


def mphf_bits_per_key(n: int, gamma_milli: int = 1230) -> float:
    """Space of the built function: 2 bits per vertex plus a 64-bit rank count
    per 512 vertices (Table "space" of the paper: 2.61 bits/key at 1.23)."""
    m = num_vertices(n, gamma_milli, 3)
    return (64 * ((m + 31) // 32) + 64 * ((m + 511) // 512 + 1)) / max(n, 1)


NOALLOC_SCRATCH_BYTES = 24 << 20


def peel_noalloc(edges, m: int, max_layers: int = 4096, out=None) -> PeelResult:
    """hpeel_peel_noalloc: the peel of ``peel`` with no workspace and no device
    allocation inside the call (the library's built-in scratch is used; graphs
    up to NOALLOC_SCRATCH_BYTES of scratch).  out: None (the output tensors
    are allocated here by torch, before the call), or a tuple (order int32
    [n], claim int32 [n], layer_off int64 [max_layers + 1]) of the caller's
    buffers, so that nothing is allocated at call time."""
    torch = _torch()
    ep = _dev_ptr(edges, "edges", torch.int32, 2)
    n, r = edges.shape
    dev = edges.device
    if out is None:
        order = torch.empty(n, dtype=torch.int32, device=dev)
        claim = torch.empty(n, dtype=torch.int32, device=dev)
        loff = torch.empty(max_layers + 1, dtype=torch.int64, device=dev)
    else:
        order, claim, loff = out
        if order.numel() < n or claim.numel() < n or loff.numel() < max_layers + 1:
            raise ValueError("out buffers too small: need n, n and max_layers + 1 entries")
    st = Stats()
    _check(lib().hpeel_peel_noalloc(ep, n, m, r, _dev_ptr(order, "order"),
                                    _dev_ptr(claim, "claim"), _dev_ptr(loff, "layer_off"),
                                    max_layers, ctypes.byref(st), _stream()))
    R = int(st.rounds)
    res = PeelResult(order, claim, loff[:R + 1], R, int(st.n_peeled))
    res.stats = st.as_dict()
    return res


@dataclass
class MphfResult:
    G: object
    rank_dir: object
    m: int
    stats: dict


def mphf_workspace_size(n: int, gamma_milli: int = 1230) -> int:
    return int(lib().hpeel_mphf_workspace_size(n, gamma_milli))


def mphf_build(keys, seed: int = 1, gamma_milli: int = 1230, max_tries: int = 8,
               workspace=None, G=None, rank_dir=None, order=None) -> MphfResult:
    """MWHC MPHF build (sec. 3) with reseed-and-retry; see hpeel_mphf_build.
    keys: a CUDA tensor, or a pinned host tensor read in place by the GPU."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1, host_ok=True)
    n = keys.shape[0]
    dev = keys.device if keys.is_cuda else torch.device("cuda", torch.cuda.current_device())
    m = num_vertices(n, gamma_milli, 3)
    if G is None:
        G = torch.empty(max((m + 31) // 32, 1), dtype=torch.int64, device=dev)
    if rank_dir is None:
        rank_dir = torch.empty((m + 511) // 512 + 1, dtype=torch.int64, device=dev)
    ws = workspace if workspace is not None else _workspace(mphf_workspace_size(n, gamma_milli), dev)
    st = Stats()
    op = None
    if order is not None:
        op = _dev_ptr(order, "order", torch.int32, 1)
        if order.numel() != n:
            raise ValueError("order must hold n entries")
    _check(lib().hpeel_mphf_build(kp, n, seed, gamma_milli, max_tries,
                                  _dev_ptr(G, "G", torch.int64), _dev_ptr(rank_dir, "rank_dir",
                                                                          torch.int64),
                                  op, ctypes.byref(st), _dev_ptr(ws, "workspace", torch.uint8),
                                  ws.numel(), _stream()))
    res = MphfResult(G[:(m + 31) // 32], rank_dir, m, st.as_dict())
    res.order = order
    return res


def mphf_large_workspace_size(n: int, gamma_milli: int = 1230, list_on_host: bool = False) -> int:
    return int(lib().hpeel_mphf_large_workspace_size(n, gamma_milli, 1 if list_on_host else 0))


def mphf_build_large(keys, seed: int = 1, gamma_milli: int = 1230, max_tries: int = 8,
                     workspace=None, G=None, rank_dir=None, host_list=None) -> MphfResult:
    """MPHF build beyond 32-bit ids (hpeel_mphf_build_large): the function of
    mphf_build, for key sets up to about 1e10 keys.  host_list: None, or a
    pinned host int64 tensor of n entries that holds the layer list."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1, host_ok=True)
    n = keys.shape[0]
    dev = keys.device if keys.is_cuda else torch.device("cuda", torch.cuda.current_device())
    m = num_vertices(n, gamma_milli, 3)
    if G is None:
        G = torch.empty(max((m + 31) // 32, 1), dtype=torch.int64, device=dev)
    if rank_dir is None:
        rank_dir = torch.empty((m + 511) // 512 + 1, dtype=torch.int64, device=dev)
    hp_list = None
    if host_list is not None:
        if not (isinstance(host_list, torch.Tensor) and host_list.is_pinned()
                and host_list.dtype == torch.int64 and host_list.numel() >= n):
            raise ValueError("host_list must be a pinned int64 host tensor of n entries")
        hp_list = ctypes.c_void_p(host_list.data_ptr())
    ws = workspace if workspace is not None else _workspace(
        mphf_large_workspace_size(n, gamma_milli, host_list is not None), dev)
    st = Stats()
    _check(lib().hpeel_mphf_build_large(kp, n, seed, gamma_milli, max_tries,
                                        _dev_ptr(G, "G", torch.int64),
                                        _dev_ptr(rank_dir, "rank_dir", torch.int64),
                                        ctypes.byref(st), _dev_ptr(ws, "workspace", torch.uint8),
                                        ws.numel(), hp_list, _stream()))
    return MphfResult(G[:(m + 31) // 32], rank_dir, m, st.as_dict())


def mphf_lookup_large(keys, seed: int, m: int, G, rank_dir, out=None):
    """MPHF values of the query keys for a function mphf_build_large built:
    int64 [nq]."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1)
    if out is None:
        out = torch.empty(keys.shape[0], dtype=torch.int64, device=keys.device)
    _check(lib().hpeel_mphf_lookup_large(kp, keys.shape[0], seed, m,
                                         _dev_ptr(G, "G", torch.int64),
                                         _dev_ptr(rank_dir, "rank_dir", torch.int64),
                                         _dev_ptr(out, "out", torch.int64), _stream()))
    return out


def mphf_build_async(keys, seed: int = 1, gamma_milli: int = 1230, max_tries: int = 8,
                     workspace=None, G=None, rank_dir=None, stats=None):
    """Device-driven MPHF build (hpeel_mphf_build_async): enqueued as one CUDA
    graph on the current stream, no host synchronisation.  Returns (G,
    rank_dir, stats) where stats is a device uint8 tensor holding an
    hpeel_stats; read it with stats_from_device after the stream is done."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1, host_ok=True)
    n = keys.shape[0]
    dev = keys.device if keys.is_cuda else torch.device("cuda", torch.cuda.current_device())
    m = num_vertices(n, gamma_milli, 3)
    if G is None:
        G = torch.empty(max((m + 31) // 32, 1), dtype=torch.int64, device=dev)
    if rank_dir is None:
        rank_dir = torch.empty((m + 511) // 512 + 1, dtype=torch.int64, device=dev)
    if stats is None:
        stats = torch.zeros(ctypes.sizeof(Stats), dtype=torch.uint8, device=dev)
    ws = workspace if workspace is not None else _workspace(mphf_workspace_size(n, gamma_milli), dev)
    _check(lib().hpeel_mphf_build_async(kp, n, seed, gamma_milli, max_tries,
                                        _dev_ptr(G, "G", torch.int64),
                                        _dev_ptr(rank_dir, "rank_dir", torch.int64),
                                        _dev_ptr(stats, "stats", torch.uint8),
                                        _dev_ptr(ws, "workspace", torch.uint8), ws.numel(),
                                        _stream()))
    return G, rank_dir, stats


def stats_from_device(stats) -> dict:
    """The hpeel_stats a device-driven call wrote (copies to the host)."""
    raw = bytes(stats.cpu().numpy().tobytes())
    return Stats.from_buffer_copy(raw[:ctypes.sizeof(Stats)]).as_dict()


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().hpeel_kernel_launches())


def profile_enable(on: bool = True) -> None:
    """Per-step CUDA-event timing of every later call (see hpeel.h)."""
    lib().hpeel_profile_enable(1 if on else 0)


def profile_reset() -> None:
    lib().hpeel_profile_reset()


def profile_read() -> dict:
    """{step name: (launch groups, total ms)} accumulated since the last reset."""
    need = int(lib().hpeel_profile_read(None, 0))
    buf = ctypes.create_string_buffer(need + 16)
    lib().hpeel_profile_read(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def get_tuning() -> dict:
    t = Tuning()
    lib().hpeel_get_tuning(ctypes.byref(t))
    return {"bucket_shift": t.bucket_shift, "bucket_min_vertices": t.bucket_min_vertices,
            "host_round_loop": t.host_round_loop,
            "bucket_sub_shift": t.bucket_sub_shift, "bucket_part_passes": t.bucket_part_passes,
            "sorted_round_min": t.sorted_round_min}


def set_tuning(**kw) -> None:
    """Set tuning knobs (see hpeel_set_tuning); no arguments restores defaults."""
    if not kw:
        _check(lib().hpeel_set_tuning(None))
        return
    cur = get_tuning()
    cur.update(kw)
    t = Tuning(cur["bucket_shift"], cur["bucket_min_vertices"], cur["host_round_loop"],
               cur["bucket_sub_shift"], cur["bucket_part_passes"], cur["sorted_round_min"])
    _check(lib().hpeel_set_tuning(ctypes.byref(t)))


def _batch_tuning(tuning):
    if tuning is None:
        return None
    t = BatchTuning(int(tuning.get("threads", 0)), int(tuning.get("ctas_per_sm", 0)),
                    int(tuning.get("smem_bytes", 0)), int(tuning.get("smem_rounds", 0)),
                    int(tuning.get("global16_rounds", 0)))
    return ctypes.byref(t)


def batched_workspace_size(B: int, gamma_milli: int = 1230, tuning=None) -> int:
    return int(lib().hpeel_batched_workspace_size(B, gamma_milli, _batch_tuning(tuning)))


@dataclass
class BatchedResult:
    order: object     # int32 [total]: per-bucket canonical orders (local ids)
    rounds: object    # int32 [B]
    status: object    # int32 [B]: 0 peeled, 1 2-core left, 2 too large
    G: object         # int64 [G_off[B]] or None
    G_off: object     # int64 [B + 1] or None


def batched_g_offsets(bucket_off, gamma_milli: int = 1230, workspace=None):
    """Word offsets of the per-bucket g arrays (hpeel_batched_g_offsets)."""
    torch = _torch()
    op = _dev_ptr(bucket_off, "bucket_off", torch.int64, 1)
    B = bucket_off.shape[0] - 1
    ws = workspace if workspace is not None else _workspace(
        batched_workspace_size(B, gamma_milli), bucket_off.device)
    G_off = torch.empty(B + 1, dtype=torch.int64, device=bucket_off.device)
    _check(lib().hpeel_batched_g_offsets(op, B, gamma_milli, _dev_ptr(G_off, "G_off"),
                                         _dev_ptr(ws, "workspace", torch.uint8), ws.numel(),
                                         _stream()))
    return G_off


def peel_batched(keys, bucket_off, gamma_milli: int = 1230, with_g: bool = False,
                 tuning=None, workspace=None, out=None) -> BatchedResult:
    """Peel every bucket of keys (bucket b = keys[off[b]:off[b+1]], hash seed b)
    in one persistent launch (hpeel_peel_batched).  Asynchronous."""
    torch = _torch()
    kp = _dev_ptr(keys, "keys", torch.int64, 1)
    op = _dev_ptr(bucket_off, "bucket_off", torch.int64, 1)
    B = bucket_off.shape[0] - 1
    dev = keys.device
    need = batched_workspace_size(B, gamma_milli, tuning)
    ws = workspace if workspace is not None else _workspace(need, dev)
    if out is None:
        out = BatchedResult(torch.empty(keys.shape[0], dtype=torch.int32, device=dev),
                            torch.empty(B, dtype=torch.int32, device=dev),
                            torch.empty(B, dtype=torch.int32, device=dev), None, None)
        if with_g:
            out.G_off = batched_g_offsets(bucket_off, gamma_milli, ws)
            words = int(out.G_off[-1].item())
            out.G = torch.empty(max(words, 1), dtype=torch.int64, device=dev)
    gp = _dev_ptr(out.G, "G") if out.G is not None else None
    gop = _dev_ptr(out.G_off, "G_off") if out.G_off is not None else None
    _check(lib().hpeel_peel_batched(kp, op, B, gamma_milli, _dev_ptr(out.order, "order"),
                                    _dev_ptr(out.rounds, "rounds"), _dev_ptr(out.status, "status"),
                                    gp, gop, _batch_tuning(tuning),
                                    _dev_ptr(ws, "workspace", torch.uint8), ws.numel(), _stream()))
    return out
