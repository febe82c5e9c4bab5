"""CPU oracle for hypergraph peeling and MWHC minimal perfect hashing.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library (``paper_1312_0526_gb300``) never imports it and shares no code with
it: the oracle is plain single-threaded C in ``hpeel_oracle.c`` (built here
with gcc), wrapped with ctypes over numpy arrays.

Each wrapper names the passage of "Cache-Oblivious Peeling of Random
Hypergraphs" it follows; the C source states the definitions and the readings
taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpeel_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNCLAIMED = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, u32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.orc_mix64.restype = u64
        lib.orc_mix64.argtypes = [u64]
        lib.orc_num_vertices.restype = u64
        lib.orc_num_vertices.argtypes = [u64, u32, u32]
        lib.orc_hash_edges.restype = ctypes.c_int
        lib.orc_hash_edges.argtypes = [p, u64, u64, u32, u64, p]
        lib.orc_incidence.restype = ctypes.c_int
        lib.orc_incidence.argtypes = [p, u64, u64, u32, p, p]
        lib.orc_peel_rounds.restype = ctypes.c_int
        lib.orc_peel_rounds.argtypes = [p, u64, u64, u32, p, p, p, u64,
                                        ctypes.POINTER(u32), ctypes.POINTER(u64)]
        lib.orc_peel_greedy.restype = ctypes.c_int
        lib.orc_peel_greedy.argtypes = [p, u64, u64, u32, p, p, ctypes.POINTER(u64)]
        lib.orc_validate.restype = ctypes.c_int
        lib.orc_validate.argtypes = [p, u64, u64, u32, p, u64, p]
        lib.orc_mphf_assign.restype = ctypes.c_int
        lib.orc_mphf_assign.argtypes = [p, u64, u64, p, p, p, u32, p]
        lib.orc_rank_dir.restype = ctypes.c_int
        lib.orc_rank_dir.argtypes = [p, u64, p]
        lib.orc_lookup.restype = u64
        lib.orc_lookup.argtypes = [u64, u64, u64, p, p]
        lib.orc_mphf_build.restype = ctypes.c_int
        lib.orc_mphf_build.argtypes = [p, u64, u64, u32, u32, p, p,
                                       ctypes.POINTER(u64), ctypes.POINTER(u32)]
        lib.orc_peel_rounds_general.restype = ctypes.c_int
        lib.orc_peel_rounds_general.argtypes = [p, u64, u64, u32, p, p, p, u64,
                                                ctypes.POINTER(u32), ctypes.POINTER(u64)]
        lib.orc_hash_edges_general.restype = ctypes.c_int
        lib.orc_hash_edges_general.argtypes = [p, u64, u64, u32, u64, p]
        lib.orc_sf_bits.restype = u32
        lib.orc_sf_bits.argtypes = [u64]
        lib.orc_sf_words.restype = u64
        lib.orc_sf_words.argtypes = [u64, u32]
        lib.orc_sf_assign.restype = ctypes.c_int
        lib.orc_sf_assign.argtypes = [p, u64, u64, p, p, p, u32, p, u64, p]
        lib.orc_sf_lookup.restype = u64
        lib.orc_sf_lookup.argtypes = [u64, u64, u64, u64, p]
        lib.orc_sf_build.restype = ctypes.c_int
        lib.orc_sf_build.argtypes = [p, p, u64, u64, u64, u32, u32, p,
                                     ctypes.POINTER(u64), ctypes.POINTER(u32)]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def mix64(z: int) -> int:
    """SplitMix64 output function (hash mixer of the edge hashing)."""
    return int(_load().orc_mix64(ctypes.c_uint64(z & (2**64 - 1))))


def num_vertices(n: int, gamma_milli: int, r: int) -> int:
    """m = r * ceil(ceil(gamma n) / r), gamma = gamma_milli / 1000 (sec. 4.3)."""
    return int(_load().orc_num_vertices(n, gamma_milli, r))


def hash_edges(keys: np.ndarray, m: int, r: int, seed: int) -> np.ndarray:
    """Edges uint32[n, r]: vertex j = (mix64(k ^ (seed + j)) mod m/r) + j m/r
    (sec. 3 hash functions, sec. 4.3 tripartition)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.shape[0]
    edges = np.zeros((n, r), dtype=np.uint32)
    _check(_load().orc_hash_edges(_ptr(keys), n, m, r, seed, _ptr(edges)), "hash")
    return edges


def incidence(edges: np.ndarray, m: int):
    """(deg, x): degree and XOR of incident edge ids per vertex (sec. 4.1)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    n, r = edges.shape
    deg = np.zeros(max(m, 1), dtype=np.uint32)
    x = np.zeros(max(m, 1), dtype=np.uint32)
    _check(_load().orc_incidence(_ptr(edges), n, m, r, _ptr(deg), _ptr(x)), "incidence")
    return deg[:m], x[:m]


@dataclass
class PeelResult:
    order: np.ndarray      # uint32[n]: layers ascending, then core ascending
    claim: np.ndarray      # uint32[n]: (round << 2) | hinge, or UNCLAIMED
    layer_off: np.ndarray  # uint64[rounds + 1]
    rounds: int
    n_peeled: int

    @property
    def core_nonempty(self) -> bool:
        return self.n_peeled < self.order.shape[0]


def peel_rounds(edges: np.ndarray, m: int) -> PeelResult:
    """Round-synchronous (layered) peel with canonical order (sec. 4.2)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    n, r = edges.shape
    order = np.zeros(max(n, 1), dtype=np.uint32)
    claim = np.zeros(max(n, 1), dtype=np.uint32)
    # a layer table of n + 1 entries always suffices; 2^24 covers every graph
    # these tests build without an n-sized table for the largest ones
    max_layers = min(n + 1, 1 << 24)
    loff = np.zeros(max_layers + 1, dtype=np.uint64)
    rounds = ctypes.c_uint32(0)
    peeled = ctypes.c_uint64(0)
    _check(_load().orc_peel_rounds(_ptr(edges), n, m, r, _ptr(order), _ptr(claim),
                                   _ptr(loff), max_layers, ctypes.byref(rounds),
                                   ctypes.byref(peeled)), "peel_rounds")
    R = rounds.value
    return PeelResult(order[:n], claim[:n], loff[:R + 1].copy(), R, peeled.value)


def peel_rounds_general(edges: np.ndarray, m: int) -> PeelResult:
    """Round-synchronous peel of a general (not r-partite) hypergraph on [0, m):
    positions are read off the edge rows (sec. 2, sec. 4.2)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    n, r = edges.shape
    order = np.zeros(max(n, 1), dtype=np.uint32)
    claim = np.zeros(max(n, 1), dtype=np.uint32)
    max_layers = min(n + 1, 1 << 24)
    loff = np.zeros(max_layers + 1, dtype=np.uint64)
    rounds = ctypes.c_uint32(0)
    peeled = ctypes.c_uint64(0)
    _check(_load().orc_peel_rounds_general(_ptr(edges), n, m, r, _ptr(order), _ptr(claim),
                                           _ptr(loff), max_layers, ctypes.byref(rounds),
                                           ctypes.byref(peeled)), "peel_rounds_general")
    R = rounds.value
    return PeelResult(order[:n], claim[:n], loff[:R + 1].copy(), R, peeled.value)


def hash_edges_general(keys: np.ndarray, m: int, r: int, seed: int) -> np.ndarray:
    """Edges uint32[n, r] of a general hypergraph: vertex j = mix64(k ^ (seed + j)) mod m."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.shape[0]
    edges = np.zeros((n, r), dtype=np.uint32)
    _check(_load().orc_hash_edges_general(_ptr(keys), n, m, r, seed, _ptr(edges)),
           "hash_edges_general")
    return edges


def peel_greedy(edges: np.ndarray, m: int):
    """Standard greedy peel with a LIFO stack and the XOR trick (sec. 1, sec. 3,
    'Standard+XOR' of sec. 5).  Returns (removal order, peeled mask)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    n, r = edges.shape
    order = np.zeros(max(n, 1), dtype=np.uint32)
    peeled = np.zeros(max(n, 1), dtype=np.uint8)
    cnt = ctypes.c_uint64(0)
    _check(_load().orc_peel_greedy(_ptr(edges), n, m, r, _ptr(order), _ptr(peeled),
                                   ctypes.byref(cnt)), "peel_greedy")
    return order[:cnt.value].copy(), peeled[:n].astype(bool)


def validate(edges: np.ndarray, m: int, order: np.ndarray, n_peeled: int,
             claim: np.ndarray | None = None) -> int:
    """0 if order is a peeling order followed by a 2-core (sec. 1) and, given
    claim, if the layers and hinges follow sec. 4.2; else a failure code."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    n, r = edges.shape
    order = np.ascontiguousarray(order, dtype=np.uint32)
    cp = None
    if claim is not None:
        claim = np.ascontiguousarray(claim, dtype=np.uint32)
        cp = _ptr(claim)
    return int(_load().orc_validate(_ptr(edges), n, m, r, _ptr(order), n_peeled, cp))


def mphf_assign(edges: np.ndarray, m: int, res: PeelResult) -> np.ndarray:
    """2-bit packed g (uint64[ceil(m/32)]), reverse layer order (sec. 3, sec. 4.3)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    n = edges.shape[0]
    G = np.zeros(max((m + 31) // 32, 1), dtype=np.uint64)
    loff = np.ascontiguousarray(res.layer_off, dtype=np.uint64)
    _check(_load().orc_mphf_assign(_ptr(edges), n, m, _ptr(res.order), _ptr(res.claim),
                                   _ptr(loff), res.rounds, _ptr(G)), "mphf_assign")
    return G[:(m + 31) // 32]


def rank_dir(G: np.ndarray, m: int) -> np.ndarray:
    """dir[b] = number of non-zero g among vertices [0, 512 b) (sec. 3, sec. 5)."""
    G = np.ascontiguousarray(G, dtype=np.uint64)
    d = np.zeros((m + 511) // 512 + 1, dtype=np.uint64)
    _check(_load().orc_rank_dir(_ptr(G), m, _ptr(d)), "rank_dir")
    return d


def lookup(key: int, seed: int, m: int, G: np.ndarray, d: np.ndarray) -> int:
    """MPHF value of a key: rank of h_i(key), i = sum of g mod 3 (sec. 3, sec. 5)."""
    return int(_load().orc_lookup(key, seed, m, _ptr(G), _ptr(d)))


@dataclass
class MphfResult:
    G: np.ndarray
    dir: np.ndarray
    seed_used: int
    rounds: int
    m: int


def mphf_build(keys: np.ndarray, seed: int, gamma_milli: int = 1230,
               max_tries: int = 8) -> MphfResult:
    """Full MPHF build with reseed-and-retry on a non-empty core (sec. 3)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.shape[0]
    m = num_vertices(n, gamma_milli, 3)
    G = np.zeros(max((m + 31) // 32, 1), dtype=np.uint64)
    d = np.zeros((m + 511) // 512 + 1, dtype=np.uint64)
    su = ctypes.c_uint64(0)
    rounds = ctypes.c_uint32(0)
    rc = _load().orc_mphf_build(_ptr(keys), n, seed, gamma_milli, max_tries, _ptr(G),
                                _ptr(d), ctypes.byref(su), ctypes.byref(rounds))
    _check(rc, "mphf_build")
    return MphfResult(G[:(m + 31) // 32], d, su.value, rounds.value, m)


# ------------------------------------------------------ static functions --

def sf_bits(sigma: int) -> int:
    """ceil(log2 sigma): bits per stored value of a static function."""
    return int(_load().orc_sf_bits(sigma))


def sf_words(m: int, sigma: int) -> int:
    return int(_load().orc_sf_words(m, sf_bits(sigma)))


def sf_assign(edges: np.ndarray, m: int, res: PeelResult, values: np.ndarray,
              sigma: int) -> np.ndarray:
    """u with u[h0] + u[h1] + u[h2] = f(x) (mod sigma), reverse layer order,
    ceil(log2 sigma) bits per vertex (sec. 3)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    values = np.ascontiguousarray(values, dtype=np.uint32)
    n = edges.shape[0]
    U = np.zeros(max(sf_words(m, sigma), 1), dtype=np.uint64)
    loff = np.ascontiguousarray(res.layer_off, dtype=np.uint64)
    _check(_load().orc_sf_assign(_ptr(edges), n, m, _ptr(res.order), _ptr(res.claim),
                                 _ptr(loff), res.rounds, _ptr(values), sigma, _ptr(U)),
           "sf_assign")
    return U[:sf_words(m, sigma)]


def sf_lookup(key: int, seed: int, m: int, sigma: int, U: np.ndarray) -> int:
    """f(key) = (u[h0] + u[h1] + u[h2]) mod sigma (sec. 3)."""
    U = np.ascontiguousarray(U, dtype=np.uint64)
    return int(_load().orc_sf_lookup(key, seed, m, sigma, _ptr(U)))


@dataclass
class SfResult:
    U: np.ndarray
    seed_used: int
    rounds: int
    m: int
    bits: int


def sf_build(keys: np.ndarray, values: np.ndarray, sigma: int, seed: int = 1,
             gamma_milli: int = 1230, max_tries: int = 8) -> SfResult:
    """Static function f(keys[i]) = values[i] in [0, sigma), with
    reseed-and-retry on a non-empty core (sec. 3)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    values = np.ascontiguousarray(values, dtype=np.uint32)
    n = keys.shape[0]
    m = num_vertices(n, gamma_milli, 3)
    U = np.zeros(max(sf_words(m, sigma), 1), dtype=np.uint64)
    su = ctypes.c_uint64(0)
    rounds = ctypes.c_uint32(0)
    rc = _load().orc_sf_build(_ptr(keys), _ptr(values), n, sigma, seed, gamma_milli, max_tries,
                              _ptr(U), ctypes.byref(su), ctypes.byref(rounds))
    _check(rc, "sf_build")
    return SfResult(U[:sf_words(m, sigma)], su.value, rounds.value, m, sf_bits(sigma))

