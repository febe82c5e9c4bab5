"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these compares the oracle with itself: the expected values are
published test vectors, closed forms, hand-derived fixtures (tests/golden/),
brute force over all edge subsets, an independent validator built on explicit
incidence lists, or statistical laws of random hypergraphs.
"""
import itertools
import math
import random

import numpy as np
import pytest

import oracle
from paper_1312_0526_gb300 import inputs
from tests import golden_io

U = oracle.UNCLAIMED


# ---------------------------------------------------------------- hashing --

def test_mix64_published_splitmix64_vectors():
    # SplitMix64 reference outputs (Steele/Lea/Flood generator, as published
    # with Vigna's splitmix64.c): seed 0 -> 0xE220A8397B1DCDAF; seed 1234567
    # -> 6457827717110365317, 3203168211198807973, 9817491932198370423.
    gamma = 0x9E3779B97F4A7C15
    assert oracle.mix64((0 + gamma) % 2**64) == 0xE220A8397B1DCDAF
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423]
    got = [oracle.mix64((1234567 + (i + 1) * gamma) % 2**64) for i in range(3)]
    assert got == want


def test_key_stream_published_vectors():
    assert int(inputs.splitmix64_stream(0, 1)[0]) == 0xE220A8397B1DCDAF
    assert [int(v) for v in inputs.splitmix64_stream(1234567, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]
    # chunked generation is the same stream
    a = inputs.splitmix64_stream(5, 1000)
    b = inputs.splitmix64_stream(5, 1000, chunk=7)
    assert np.array_equal(a, b)
    assert len(np.unique(inputs.keys(100000))) == 100000


def test_key_stream_torch_generator_is_the_same_stream():
    torch = pytest.importorskip("torch")
    t = inputs.keys_torch(3, 1234567, device="cpu").numpy().view(np.uint64)
    assert [int(v) for v in t] == [6457827717110365317, 3203168211198807973,
                                   9817491932198370423]
    for seed in (1, 0, 2**63 + 5, 2**64 - 1):
        a = inputs.keys(50_001, seed)
        b = inputs.keys_torch(50_001, seed, device="cpu", chunk=4099).numpy().view(np.uint64)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n,g,r,m", [
    (100_000, 1230, 3, 123_000),
    (10**8, 1230, 3, 123_000_000),
    (10**9, 1230, 3, 1_230_000_000),
    (10**9, 1222, 3, 1_222_000_002),
    (10**9, 1200, 3, 1_200_000_000),
    (10**8, 1300, 4, 130_000_000),
    (0, 1230, 3, 0),
    (1, 1230, 3, 3),
    (2, 1230, 3, 3),
    (3, 1230, 3, 6),
])
def test_num_vertices(n, g, r, m):
    # m = r * ceil(ceil(gamma n) / r): computed by hand for each row.
    assert oracle.num_vertices(n, g, r) == m


@pytest.mark.parametrize("r", [3, 4])
def test_hash_tripartition_no_degenerate_edges(r):
    # sec. 4.3: vertex j lies in [j m/r, (j+1) m/r), so the r vertices of an
    # edge are distinct.
    n = 50_000
    m = oracle.num_vertices(n, 1230, r)
    P = m // r
    e = oracle.hash_edges(inputs.keys(n, 1), m, r, 1)
    for j in range(r):
        assert e[:, j].min() >= j * P and e[:, j].max() < (j + 1) * P


def test_hash_degree_law_poisson():
    # Each part gets one endpoint of every edge, uniformly: the degree of a
    # vertex is Binomial(n, 1/P).  Expected number of degree-d vertices is
    # m * C(n,d) p^d (1-p)^(n-d); check d = 0, 1, 2 within 5 sigma.
    n = 200_000
    m = oracle.num_vertices(n, 1230, 3)
    P = m // 3
    e = oracle.hash_edges(inputs.keys(n, 11), m, 3, 1)
    deg, _ = oracle.incidence(e, m)
    p = 1.0 / P
    for d in range(3):
        mean = m * math.comb(n, d) * p**d * (1 - p) ** (n - d)
        got = int((deg == d).sum())
        assert abs(got - mean) < 5 * math.sqrt(mean), (d, got, mean)


# Published SplitMix64 (state, output) pairs: the generator's state after
# i steps of 0x9E3779B97F4A7C15 from seed s is s + i * 0x9E3779B97F4A7C15, and
# its output is mix64 of that state (seed 0, first output; seed 1234567,
# outputs 1..3).
_GOLDEN = 0x9E3779B97F4A7C15
_PUBLISHED = [
    (_GOLDEN, 0xE220A8397B1DCDAF),
    ((1234567 + 1 * _GOLDEN) % 2**64, 6457827717110365317),
    ((1234567 + 2 * _GOLDEN) % 2**64, 3203168211198807973),
    ((1234567 + 3 * _GOLDEN) % 2**64, 9817491932198370423),
]


@pytest.mark.parametrize("r", [3, 4])
@pytest.mark.parametrize("seed", [77, 2**64 - 2])
@pytest.mark.parametrize("P", [1_000_003, 1_431_655_765])
def test_hash_composition_from_published_vectors(r, seed, P):
    # Vertex j of key k is (mix64(k XOR (seed + j)) mod P) + j P (sec. 3
    # hash functions, sec. 4.3 parts).  Key j is chosen so that k XOR (seed +
    # j) is a published SplitMix64 state: its vertex j must be the published
    # output mod P, shifted into part j.  A misread composition -- mix64((k
    # XOR seed) + j), mix64(k) XOR (seed + j), mix64(k XOR seed XOR j), or a
    # missing part offset -- misses for some j.  The seed 2^64 - 2 makes seed
    # + j wrap to 0 at j = 2.
    if r == 4 and P > (2**32 - 1) // 4:
        P = 1_000_000_007
    keys = np.array([st ^ ((seed + j) % 2**64) for j, (st, _) in enumerate(_PUBLISHED[:r])],
                    dtype=np.uint64)
    e = oracle.hash_edges(keys, r * P, r, seed)
    for j, (_, out) in enumerate(_PUBLISHED[:r]):
        assert int(e[j, j]) == out % P + j * P, (j, int(e[j, j]))


def test_hash_seed_changes_edges():
    k = inputs.keys(1000, 1)
    m = oracle.num_vertices(1000, 1230, 3)
    a = oracle.hash_edges(k, m, 3, 1)
    b = oracle.hash_edges(k, m, 3, 2)
    assert (a != b).mean() > 0.9


# -------------------------------------------------------------- incidence --

def _xor_prefix(n):
    # XOR of 0..n-1, by n mod 4
    k = n - 1
    if n == 0:
        return 0
    return [k, 1, k + 1, 0][k % 4]


@pytest.mark.parametrize("n,r", [(0, 3), (1, 3), (2, 3), (3, 3), (4, 3), (99_999, 3),
                                 (100_000, 3), (100_001, 4), (100_002, 4)])
def test_incidence_closed_forms(n, r):
    # sec. 4.1: sum of degrees is r n; XOR over all vertices of x[v] is the XOR
    # of every edge id r times: XOR_{i<n} i if r is odd, else 0.
    m = max(oracle.num_vertices(n, 1230, r), r)
    e = oracle.hash_edges(inputs.keys(n, 3), m, r, 1)
    deg, x = oracle.incidence(e, m)
    assert int(deg.sum()) == r * n
    want = _xor_prefix(n) if r % 2 == 1 else 0
    assert int(np.bitwise_xor.reduce(x, initial=0)) == want


def test_incidence_retrieve_edge():
    # sec. 4.1 RetrieveEdge: at degree 1, x[v] is the only edge of v.
    n = 20_000
    m = oracle.num_vertices(n, 1230, 3)
    e = oracle.hash_edges(inputs.keys(n, 5), m, 3, 1)
    deg, x = oracle.incidence(e, m)
    ones = np.nonzero(deg == 1)[0]
    assert len(ones) > 0
    for v in ones[:2000]:
        ee = int(x[v])
        assert ee < n and v in set(int(t) for t in e[ee])


# ---------------------------------------------------------------- goldens --

@pytest.mark.parametrize("name", golden_io.all_names())
def test_golden_peel(name):
    g = golden_io.load(name)
    res = oracle.peel_rounds(g["edges"], g["m"])
    assert np.array_equal(res.order, g["order"])
    assert np.array_equal(res.claim, g["claim"])
    assert np.array_equal(res.layer_off, g["layer_off"])
    assert res.n_peeled == g["n_peeled"]
    assert res.rounds == len(g["layer_off"]) - 1
    assert oracle.validate(g["edges"], g["m"], res.order, res.n_peeled, res.claim) == 0


@pytest.mark.parametrize("name", [n for n in golden_io.all_names()
                                  if "g" in golden_io.load(n) or "rank" in golden_io.load(n)])
def test_golden_mphf(name):
    g = golden_io.load(name)
    m = g["m"]
    res = oracle.peel_rounds(g["edges"], m)
    G = oracle.mphf_assign(g["edges"], m, res)
    vals = {v: (int(G[v >> 5]) >> (2 * (v & 31))) & 3 for v in range(m)}
    if "g" in g:
        assert {v: a for v, a in vals.items() if a} == g["g"]
    d = oracle.rank_dir(G, m)
    got = []
    for e in g["edges"]:
        i = sum(vals[int(v)] for v in e) % 3
        got.append(sum(1 for u in range(int(e[i])) if vals[u]))
    assert got == g["rank"]
    assert int(d[-1]) == len(g["rank"])


# ----------------------------------------------------- brute-force 2-core --

def _core_bruteforce(edges, m):
    """Union of all edge subsets whose touched vertices all have degree >= 2
    inside the subset; that union is the 2-core (sec. 1)."""
    n = len(edges)
    core = 0
    for mask in range(1 << n):
        deg = [0] * m
        for i in range(n):
            if mask >> i & 1:
                for v in edges[i]:
                    deg[v] += 1
        if all(deg[v] != 1 for v in range(m)):
            core |= mask
    return {i for i in range(n) if core >> i & 1}


def _random_small_graph(rng, n, r, P):
    return np.array([[rng.randrange(P) + j * P for j in range(r)] for _ in range(n)],
                    dtype=np.uint32).reshape(n, r)


@pytest.mark.parametrize("r", [3, 4])
def test_core_matches_bruteforce(r):
    rng = random.Random(1234 + r)
    cases = 0
    nonempty = 0
    for trial in range(160):
        n = rng.randint(1, 12 if r == 3 else 10)
        P = rng.choice([1, 2, 2, 3, 3, 4, 5])
        edges = _random_small_graph(rng, n, r, P)
        m = r * P
        want_core = _core_bruteforce(edges.tolist(), m)
        res = oracle.peel_rounds(edges, m)
        got_core = {int(e) for e in res.order[res.n_peeled:]}
        assert got_core == want_core, (edges.tolist(), got_core, want_core)
        assert {int(e) for e in np.nonzero(res.claim == U)[0]} == want_core
        _, peeled = oracle.peel_greedy(edges, m)
        assert {i for i in range(n) if not peeled[i]} == want_core
        assert oracle.validate(edges, m, res.order, res.n_peeled, res.claim) == 0
        cases += 1
        nonempty += bool(want_core)
    assert cases == 160 and 20 < nonempty < 150


# ------------------------------------------------- layered vs greedy peel --

@pytest.mark.parametrize("gamma", [1180, 1215, 1222, 1230, 1300])
def test_rounds_and_greedy_peel_the_same_set(gamma):
    # The 2-core is unique (sec. 1): the greedy peel and the layered peel
    # remove the same edges, whatever their order.
    n = 30_000
    m = oracle.num_vertices(n, gamma, 3)
    e = oracle.hash_edges(inputs.keys(n, 21), m, 3, 1)
    res = oracle.peel_rounds(e, m)
    go, gp = oracle.peel_greedy(e, m)
    assert set(res.order[:res.n_peeled].tolist()) == set(go.tolist())
    assert res.n_peeled == len(go)
    assert oracle.validate(e, m, res.order, res.n_peeled, res.claim) == 0
    full = np.concatenate([go, np.nonzero(~gp)[0].astype(np.uint32)])
    assert oracle.validate(e, m, full, len(go)) == 0


def test_intra_layer_order_is_free():
    # sec. 4.2: concatenated layers form a peeling order whatever the order
    # inside each layer.
    n = 20_000
    m = oracle.num_vertices(n, 1230, 3)
    e = oracle.hash_edges(inputs.keys(n, 8), m, 3, 1)
    res = oracle.peel_rounds(e, m)
    rng = np.random.default_rng(0)
    order = res.order.copy()
    for t in range(res.rounds):
        a, b = int(res.layer_off[t]), int(res.layer_off[t + 1])
        rng.shuffle(order[a:b])
    assert oracle.validate(e, m, order, res.n_peeled) == 0
    assert oracle.validate(e, m, order, res.n_peeled, res.claim) == 0


def test_canonical_order_shape():
    n = 20_000
    m = oracle.num_vertices(n, 1200, 3)  # below threshold: non-empty core
    e = oracle.hash_edges(inputs.keys(n, 9), m, 3, 1)
    res = oracle.peel_rounds(e, m)
    assert res.core_nonempty
    rounds = res.claim[res.order[:res.n_peeled]] >> 2
    assert np.all(np.diff(rounds.astype(np.int64)) >= 0)
    for t in range(res.rounds):
        seg = res.order[int(res.layer_off[t]):int(res.layer_off[t + 1])]
        assert len(seg) > 0 and np.all(np.diff(seg.astype(np.int64)) > 0)
    core = res.order[res.n_peeled:]
    assert np.all(np.diff(core.astype(np.int64)) > 0)
    assert np.all(res.claim[core] == U)


# --------------------------------------------------- the validator itself --

def _peeled_example():
    n = 5_000
    m = oracle.num_vertices(n, 1230, 3)
    e = oracle.hash_edges(inputs.keys(n, 4), m, 3, 1)
    return e, m, oracle.peel_rounds(e, m)


def test_validator_rejects_planted_mistakes():
    e, m, res = _peeled_example()
    assert res.rounds >= 3 and not res.core_nonempty
    L0, L1 = int(res.layer_off[1]), int(res.layer_off[2])
    # an edge of layer 1 moved before layer 0 (breaks the peeling order)
    bad = res.order.copy()
    bad[[0, L0]] = bad[[L0, 0]]
    assert oracle.validate(e, m, bad, res.n_peeled) != 0
    # a duplicate entry
    bad = res.order.copy()
    bad[1] = bad[0]
    assert oracle.validate(e, m, bad, res.n_peeled) != 0
    # a wrong hinge
    claim = res.claim.copy()
    ee = int(res.order[0])
    claim[ee] = (claim[ee] & ~np.uint32(3)) | np.uint32((int(claim[ee]) + 1) % 3)
    assert oracle.validate(e, m, res.order, res.n_peeled, claim) != 0
    # an edge of layer 1 labelled round 0 (layer not maximal / wrong round)
    claim = res.claim.copy()
    claim[int(res.order[L0])] = claim[int(res.order[L0])] & np.uint32(3)
    assert oracle.validate(e, m, res.order, res.n_peeled, claim) != 0
    # the last layer dropped: what is left is not a 2-core
    assert oracle.validate(e, m, res.order, L1) != 0
    # one layer-0 edge moved into layer 1: layer 0 is no longer maximal
    claim = res.claim.copy()
    order = res.order.copy()
    mv = int(order[L0 - 1])
    claim[mv] = (np.uint32(1) << np.uint32(2)) | (claim[mv] & np.uint32(3))
    assert oracle.validate(e, m, order, res.n_peeled, claim) != 0


# ------------------------------------------------------------- metamorphic --

def test_vertex_relabel_within_parts_is_invariant():
    # Renaming vertices inside a part leaves the rounds, hinges and order
    # unchanged (positions are kept, only names change).
    n = 10_000
    m = oracle.num_vertices(n, 1230, 3)
    P = m // 3
    e = oracle.hash_edges(inputs.keys(n, 12), m, 3, 1)
    rng = np.random.default_rng(1)
    perm = np.concatenate([rng.permutation(P) + j * P for j in range(3)]).astype(np.uint32)
    a = oracle.peel_rounds(e, m)
    b = oracle.peel_rounds(perm[e], m)
    assert np.array_equal(a.order, b.order) and np.array_equal(a.claim, b.claim)


def test_edge_relabel_permutes_rounds_and_hinges():
    n = 10_000
    m = oracle.num_vertices(n, 1230, 3)
    e = oracle.hash_edges(inputs.keys(n, 13), m, 3, 1)
    rng = np.random.default_rng(2)
    pi = rng.permutation(n)           # new id k holds old edge pi[k]
    a = oracle.peel_rounds(e, m)
    b = oracle.peel_rounds(e[pi], m)
    assert np.array_equal(b.claim, a.claim[pi])
    assert a.rounds == b.rounds and a.n_peeled == b.n_peeled


# ------------------------------------------------------ random-graph laws --

def test_threshold_c3():
    # sec. 1: above c_3 ~ 1.221 a random 3-hypergraph has an empty 2-core
    # w.h.p., below it a non-empty one.  With n = 2e4 the window is narrow
    # enough to see the switch between 1.215 and 1.23.
    n = 20_000
    freq = {}
    for g in (1190, 1205, 1215, 1230, 1250):
        m = oracle.num_vertices(n, g, 3)
        ok = 0
        for s in range(100):
            e = oracle.hash_edges(inputs.keys(n, 500 + s), m, 3, 1)
            ok += not oracle.peel_rounds(e, m).core_nonempty
        freq[g] = ok / 100
    assert freq[1190] <= 0.02 and freq[1205] <= 0.1
    assert freq[1215] < 0.5 < freq[1230]
    assert freq[1250] >= 0.97


def test_rounds_grow_slowly_above_threshold():
    # sec. 4.2: O(log log n) rounds w.h.p. above the threshold; far from it the
    # count is flat in n, and layers shrink quickly after the first.
    got = {}
    for n in (10_000, 100_000, 1_000_000):
        m = oracle.num_vertices(n, 1400, 3)
        res = oracle.peel_rounds(oracle.hash_edges(inputs.keys(n, 7), m, 3, 1), m)
        assert not res.core_nonempty
        got[n] = res.rounds
        sizes = np.diff(res.layer_off.astype(np.int64))
        assert sizes[0] > 0.25 * n and sizes[1] < 0.6 * sizes[0]
    assert max(got.values()) - min(got.values()) <= 2 and max(got.values()) < 20


# -------------------------------------------------------------------- MPHF --

@pytest.mark.parametrize("n", [1, 17, 1000, 50_000])
def test_mphf_bijection_and_mwhc_identity(n):
    keys = inputs.keys(n, 31)
    res = oracle.mphf_build(keys, seed=1, max_tries=32)
    m = res.m
    G, d = res.G, res.dir
    vals = np.array([(int(G[v >> 5]) >> (2 * (v & 31))) & 3 for v in range(m)])
    # exactly one assigned vertex per key (sec. 3: h_{f(x)} is a PHF)
    assert int((vals != 0).sum()) == n and int(d[-1]) == n
    out = [oracle.lookup(int(k), res.seed_used, m, G, d) for k in keys]
    assert sorted(out) == list(range(n))
    # MWHC equation: the g values of an edge sum (mod 3) to its hinge, which
    # is the position of an assigned vertex of the edge.
    e = oracle.hash_edges(keys, m, 3, res.seed_used)
    s = vals[e.astype(np.int64)].sum(axis=1) % 3
    assert np.all(vals[e[np.arange(n), s].astype(np.int64)] != 0)


def test_mphf_reseed_on_core_and_retry_exhaustion():
    # duplicate keys give identical edges under every seed: a 2-core always
    keys = np.array([5, 5, 6], dtype=np.uint64)
    with pytest.raises(RuntimeError, match="code 5"):
        oracle.mphf_build(keys, seed=1, max_tries=4)
    # two keys get m = 3 vertices: one possible edge, so never peelable
    with pytest.raises(RuntimeError, match="code 5"):
        oracle.mphf_build(inputs.keys(2, 1), seed=1, max_tries=4)
    # a tiny sparse set that fails on some seed is rebuilt with the next one
    tried = 0
    for s in range(200):
        k = inputs.keys(40, 900 + s)
        m = oracle.num_vertices(40, 1230, 3)
        if oracle.peel_rounds(oracle.hash_edges(k, m, 3, 1), m).core_nonempty:
            res = oracle.mphf_build(k, seed=1, max_tries=50)
            assert res.seed_used > 1
            tried += 1
            if tried == 3:
                break
    assert tried == 3


def test_space_bits_per_key_table_space():
    # Table "space": MWHC takes 2.61 bits/key at gamma = 1.23.  With 2 bits
    # per vertex and one 64-bit rank count per 512 vertices:
    for n in (10**6, 10**8, 10**9):
        m = oracle.num_vertices(n, 1230, 3)
        bits = 2 * m + 64 * ((m + 511) // 512 + 1)
        assert round(bits / n, 2) == 2.61


def test_rank_dir_blocks():
    # rank directory against an independent per-block count
    n = 30_000
    res = oracle.mphf_build(inputs.keys(n, 2), seed=1)
    m = res.m
    bits = np.unpackbits(res.G.view(np.uint8), bitorder="little")[:2 * m].reshape(m, 2)
    nz = bits.any(axis=1)
    blocks = (m + 511) // 512
    want = np.zeros(blocks + 1, dtype=np.int64)
    for b in range(blocks):
        want[b + 1] = want[b] + int(nz[b * 512:(b + 1) * 512].sum())
    assert np.array_equal(res.dir.astype(np.int64), want)


# ------------------------------------------------------- static functions --
# sec. 3: f: S -> [sigma] stored as u with f(x) = u[h0] + u[h1] + u[h2] mod
# sigma, ceil(log2 sigma) bits per value.

def _decode_u(U: np.ndarray, m: int, b: int) -> np.ndarray:
    """u[v] from the bit string: bits [v b, (v + 1) b), bit i = bit i % 64 of
    word i // 64 (numpy, independent of the oracle's C code)."""
    bits = np.unpackbits(U.view(np.uint8), bitorder="little")[: m * b]
    bits = bits.reshape(m, b).astype(np.uint64)
    return (bits << np.arange(b, dtype=np.uint64)).sum(axis=1)


@pytest.mark.parametrize("sigma", [2, 3, 4, 5, 31, 32, 33, 255, 256, 257, 2**16 + 1,
                                   2**31, 2**31 + 1, 2**32 - 1, 2**32])
def test_sf_bits_closed_form(sigma):
    assert oracle.sf_bits(sigma) == (sigma - 1).bit_length() == math.ceil(math.log2(sigma))


def _values(n, sigma, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, sigma, n, dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("n,sigma", [(1, 2), (7, 3), (500, 2), (2000, 5), (2000, 100),
                                     (3000, 2**13 - 1), (1500, 2**31 + 11), (1200, 2**32)])
def test_sf_every_key_maps_to_its_value(n, sigma):
    keys = inputs.keys(n, 40 + n % 7)
    vals = _values(n, sigma, n)
    r = oracle.sf_build(keys, vals, sigma, seed=1, max_tries=64)
    assert r.bits == (sigma - 1).bit_length()
    assert r.U.shape[0] == (r.m * r.bits + 63) // 64
    for k, v in zip(keys, vals):
        assert oracle.sf_lookup(int(k), r.seed_used, r.m, sigma, r.U) == int(v)


@pytest.mark.parametrize("sigma", [3, 7, 1000, 2**20 + 3])
def test_sf_solves_the_linear_system_from_the_edge_rows(sigma):
    # decode u independently and check every equation of the system on the
    # edge rows (no hashing in the check); only hinges are non-zero
    n = 4000
    keys = inputs.keys(n, 77)
    vals = _values(n, sigma, 5)
    r = oracle.sf_build(keys, vals, sigma, seed=1, max_tries=64)
    edges = oracle.hash_edges(keys, r.m, 3, r.seed_used).astype(np.int64)
    u = _decode_u(r.U, r.m, r.bits)
    assert (u < sigma).all()
    lhs = (u[edges[:, 0]] + u[edges[:, 1]] + u[edges[:, 2]]) % np.uint64(sigma)
    assert np.array_equal(lhs, vals.astype(np.uint64))
    res = oracle.peel_rounds(edges.astype(np.uint32), r.m)
    hinge_v = edges[np.arange(n), (res.claim & 3).astype(np.int64)]
    nonhinge = np.ones(r.m, dtype=bool)
    nonhinge[hinge_v] = False
    assert (u[nonhinge] == 0).all()
    assert len(np.unique(hinge_v)) == n  # each edge its own hinge


def test_sf_sigma3_with_hinge_values_is_the_mphf_g():
    # sec. 3: the MPHF is the static function x -> hinge position with
    # sigma = 3; its g differs only in storing an assigned 0 as 3
    n = 20000
    keys = inputs.keys(n, 9)
    mp = oracle.mphf_build(keys, seed=1, max_tries=32)
    edges = oracle.hash_edges(keys, mp.m, 3, mp.seed_used)
    res = oracle.peel_rounds(edges, mp.m)
    hinges = (res.claim & 3).astype(np.uint32)
    u = _decode_u(oracle.sf_assign(edges, mp.m, res, hinges, 3), mp.m, 2)
    g = _decode_u(mp.G, mp.m, 2)
    assert np.array_equal(u, g % 3)
    assert np.array_equal(u != 0, (g != 0) & (g != 3))


def test_sf_rejects_a_value_outside_sigma():
    keys = inputs.keys(300, 2)
    vals = _values(300, 10, 1)
    vals[123] = 10
    with pytest.raises(RuntimeError, match="code 1"):
        oracle.sf_build(keys, vals, 10, seed=1, max_tries=64)
    with pytest.raises(RuntimeError, match="code 1"):
        oracle.sf_build(keys, vals, 1, seed=1)


# ------------------------------------------- general (non-partite) graphs --
# sec. 2: edges are r-subsets of V with no part structure; a row may repeat a
# vertex (degrees count occurrences), positions are read off the rows.

def _random_general_graph(rng, n, r, m):
    return np.array([[rng.randrange(m) for _ in range(r)] for _ in range(n)],
                    dtype=np.uint32).reshape(n, r)


@pytest.mark.parametrize("r", [2, 3, 4])
def test_general_core_matches_bruteforce_and_greedy(r):
    rng = random.Random(99 + r)
    nonempty = 0
    for trial in range(150):
        n = rng.randint(1, 11)
        m = rng.randint(1, 9)
        edges = _random_general_graph(rng, n, r, m)
        want_core = _core_bruteforce(edges.tolist(), m)
        res = oracle.peel_rounds_general(edges, m)
        assert {int(e) for e in res.order[res.n_peeled:]} == want_core
        assert {int(e) for e in np.nonzero(res.claim == U)[0]} == want_core
        _, peeled = oracle.peel_greedy(edges, m)
        assert {i for i in range(n) if not peeled[i]} == want_core
        assert oracle.validate(edges, m, res.order, res.n_peeled, res.claim) == 0
        nonempty += bool(want_core)
    assert 10 < nonempty < 140


def test_general_peel_hand_examples():
    # (0,0,1), (1,2,3): in round 0 vertices 2 and 3 have degree 1 in edge 1,
    # smallest position 1; vertex 0 occurs twice (degree 2) and vertex 1 is
    # in both edges.  Deleting edge 1 leaves vertex 1 of degree 1 at position
    # 2 of edge 0: round 1, hinge 2.
    e = np.array([[0, 0, 1], [1, 2, 3]], dtype=np.uint32)
    res = oracle.peel_rounds_general(e, 4)
    assert res.order.tolist() == [1, 0]
    assert res.claim.tolist() == [(1 << 2) | 2, (0 << 2) | 1]
    assert res.layer_off.tolist() == [0, 1, 2]
    # a row repeating one vertex three times is a 2-core by itself
    e = np.array([[5, 5, 5], [1, 2, 5]], dtype=np.uint32)
    res = oracle.peel_rounds_general(e, 7)
    assert res.n_peeled == 1 and res.order.tolist() == [1, 0]
    assert res.claim.tolist() == [U, (0 << 2) | 0]
    # m need not be a multiple of r.  (0,1,2), (2,3,4): both edges peel in
    # round 0; vertex 2 has degree 2, so edge 1's smallest degree-1 position
    # is 1 (vertex 3) while edge 0's is 0 (vertex 0)
    e = np.array([[0, 1, 2], [2, 3, 4]], dtype=np.uint32)
    res = oracle.peel_rounds_general(e, 5)
    assert res.order.tolist() == [0, 1] and res.claim.tolist() == [0, 1]


def test_general_peel_of_a_partite_graph_is_the_partite_peel():
    # in an r-partite graph the row position of a vertex is its part
    for n, r, g in ((50_000, 3, 1230), (20_000, 4, 1300), (30_000, 3, 1200)):
        m = oracle.num_vertices(n, g, r)
        edges = oracle.hash_edges(inputs.keys(n, 4), m, r, 1)
        a = oracle.peel_rounds(edges, m)
        b = oracle.peel_rounds_general(edges, m)
        assert np.array_equal(a.order, b.order) and np.array_equal(a.claim, b.claim)
        assert np.array_equal(a.layer_off, b.layer_off)


def test_general_peel_is_invariant_under_vertex_relabelling():
    n, m = 40_000, 49_200
    edges = oracle.hash_edges_general(inputs.keys(n, 6), m, 3, 1)
    assert (edges < m).all() and len(np.unique(edges[:, 0])) < n  # no parts: any vertex anywhere
    a = oracle.peel_rounds_general(edges, m)
    perm = np.random.default_rng(3).permutation(m).astype(np.uint32)
    b = oracle.peel_rounds_general(perm[edges], m)
    assert np.array_equal(a.order, b.order) and np.array_equal(a.claim, b.claim)
    assert oracle.validate(edges, m, a.order, a.n_peeled, a.claim) == 0


def test_empty_graph_with_no_vertices():
    # an empty bucket: n = 0 edges on m = 0 vertices is the empty graph
    for peel in (oracle.peel_rounds, oracle.peel_rounds_general):
        res = peel(np.zeros((0, 3), dtype=np.uint32), 0)
        assert res.rounds == 0 and res.n_peeled == 0 and res.layer_off.tolist() == [0]
