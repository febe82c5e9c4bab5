// batched.cu -- many independent bucket hypergraphs in one persistent launch.
//
// The key set is cut into buckets (the HEM layout of sec. 3 "Practical
// workarounds": one small hypergraph per bucket); bucket b hashes its keys
// with seed b into a 3-partite hypergraph of m_b = 3 ceil(ceil(gamma n_b)/3)
// vertices and is peeled on its own.  One CTA takes one bucket at a time
// from a shared counter (work stealing over a largest-first schedule) and
// runs the whole path for it, block-synchronous:
//   hash + AddEdge (sec. 3, 4.1), round 0 scan, rounds with the claims of
//   round t+1 made by the deletions of round t (sec. 4.2; same scheme as the
//   single-graph path), the canonical order (layers ascending by round, edge
//   ids ascending inside a layer, 2-core edges last) by a stable one-warp
//   counting pass, and optionally the MWHC g values (sec. 3, layers last to
//   first).
// A bucket's state lives in shared memory when it fits: vertex records of 32
// bits (degree in the low 16, sum of incident local edge ids mod 2^16 in the
// high 16; a bucket in shared memory has far fewer than 2^16 edges, so the
// degree never carries into the sum), claim words, the layers as 16-bit local
// edge ids, the layer table and the g values -- no edge rows: an edge's
// vertices are hashed again from its key (read through the cache) when a
// round or the assignment needs them, which leaves about 11 bytes of shared
// memory per key.  Larger buckets use a per-CTA region of the workspace,
// with 32-bit records too unless the bucket has 2^16 - 1 edges or more.  No
// block waits on another; the only cross-block state is the bucket counter.
#include <algorithm>

#include "kernels.cuh"

namespace hp {

constexpr uint32_t kBatchMaxEdges = 65536;        // per bucket
constexpr uint32_t kBatchMaxVertices = (1u << 17) - 1;  // packed 17-bit local ids
// Claim words: (round << 2) | hinge, all ones while unclaimed.  16 bits in
// shared memory and in the 32-bit global path (layer tables of at most
// kClaim16Rounds entries, fewer if the tuning says so), 32 bits in the
// 64-bit path.
constexpr uint32_t kClaim16Rounds = 16383;

template <typename C>
__device__ __forceinline__ uint32_t unclaimed() { return (uint32_t)(C)~(C)0; }

// atomicMin on a claim word, returning the old value
__device__ __forceinline__ uint32_t claim_min(uint32_t *p, uint32_t v) { return atomicMin(p, v); }
__device__ __forceinline__ uint32_t claim_min(uint16_t *p, uint32_t v) {
    // the 32-bit word holding the half-word: compare-and-swap until the
    // half-word is at most v (every failed swap saw another claim succeed)
    uint32_t *w = reinterpret_cast<uint32_t *>(reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)3);
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(p) & 2u) * 8u;
    uint32_t old = *reinterpret_cast<volatile uint32_t *>(w);
    for (;;) {
        const uint32_t cur = (old >> sh) & 0xFFFFu;
        if (cur <= v) return cur;
        const uint32_t got = atomicCAS(w, old, (old & ~(0xFFFFu << sh)) | (v << sh));
        if (got == old) return cur;
        old = got;
    }
}

// Device copy of hpeel_num_vertices for r = 3.
__device__ __forceinline__ uint32_t bucket_vertices(uint32_t n, uint32_t gamma_milli) {
    const uint64_t gn = ((uint64_t)n * gamma_milli + 999u) / 1000u;
    return (uint32_t)((gn + 2) / 3 * 3);
}

// The three vertices of a bucket's edge: its key hashed with the bucket's
// seed into the three parts (the same hash as the single-graph path).
__device__ __forceinline__ void bucket_edge(uint64_t k, uint64_t seed, const FastMod &fm,
                                            uint32_t P, uint32_t (&v)[3]) {
#pragma unroll
    for (int j = 0; j < 3; j++)
        v[j] = (uint32_t)fastmod(mix64(k ^ (seed + (uint64_t)j)), fm) + (uint32_t)j * P;
}

// Vertex record arithmetic: degree in the low W bits, id sum in the rest.
template <typename T>
struct VRec;
template <>
struct VRec<uint32_t> {
    static constexpr int W = 16;
    __device__ static uint32_t deg(uint32_t r) { return r & 0xFFFFu; }
    __device__ static uint32_t sum(uint32_t r) { return r >> 16; }
    __device__ static uint32_t unit(uint32_t e) { return (e << 16) + 1u; }
    __device__ static uint32_t mask() { return 0xFFFFu; }
};
template <>
struct VRec<unsigned long long> {
    static constexpr int W = 32;
    __device__ static uint32_t deg(unsigned long long r) { return (uint32_t)r; }
    __device__ static uint32_t sum(unsigned long long r) { return (uint32_t)(r >> 32); }
    __device__ static unsigned long long unit(uint32_t e) {
        return ((unsigned long long)e << 32) + 1ull;
    }
    __device__ static uint32_t mask() { return 0xFFFFFFFFu; }
};

// Where one bucket's state lives (shared memory or the CTA's global region).
template <typename T, typename C>
struct BucketState {
    T *rec;          // [m]
    C *claim;        // [n] (round << 2) | hinge
    uint16_t *L;     // [n] layers appended (local edge ids < 2^16)
    uint32_t *loff;  // [rcap + 2] layer starts
    uint32_t *cnt;   // [rcap + 2] running starts of the order pass
    uint32_t *G;     // [ceil(m / 16)] 2-bit g values (MPHF)
    uint32_t rcap;   // rounds the loff table holds
};

struct BatchArgs {
    const uint64_t *keys;
    const uint64_t *off;  // [B + 1]
    uint32_t B;
    uint32_t gamma_milli;
    const uint32_t *sched;    // processing order of the buckets
    uint32_t *next;           // work-stealing counter
    uint32_t *order;          // [total] per-bucket canonical order (local ids)
    uint32_t *rounds;         // [B] or null
    uint32_t *status;         // [B] or null: 0 peeled, 1 2-core left, 2 too large
    uint64_t *G;              // or null
    const uint64_t *G_off;    // [B + 1] word offsets of the buckets' g arrays
    char *scratch;            // per-CTA global regions
    size_t scratch_bytes;     // bytes per CTA region
    uint32_t smem_bytes;      // dynamic shared memory per CTA
    uint32_t smem_rounds;     // layer-table entries of a bucket in shared memory
    uint32_t global16_rounds; // layer-table entries on the 32-bit global path
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// Bytes of one bucket's state with records of rec_bytes and a loff table of
// rcap + 2 entries.
__host__ __device__ inline size_t bucket_bytes(uint32_t n, uint32_t m, uint32_t rec_bytes,
                                               uint32_t claim_bytes, uint32_t rcap) {
    return a16((size_t)m * rec_bytes) + a16((size_t)n * claim_bytes) + a16((size_t)n * 2) +
           2 * a16(((size_t)rcap + 2) * 4) + a16(((size_t)m + 15) / 16 * 4);
}

template <typename T, typename C>
__device__ BucketState<T, C> carve(char *base, uint32_t n, uint32_t m, uint32_t rcap) {
    BucketState<T, C> s;
    size_t o = 0;
    s.rec = reinterpret_cast<T *>(base + o);
    o += a16((size_t)m * sizeof(T));
    s.claim = reinterpret_cast<C *>(base + o);
    o += a16((size_t)n * sizeof(C));
    s.L = reinterpret_cast<uint16_t *>(base + o);
    o += a16((size_t)n * 2);
    s.loff = reinterpret_cast<uint32_t *>(base + o);
    o += a16(((size_t)rcap + 2) * 4);
    s.cnt = reinterpret_cast<uint32_t *>(base + o);
    o += a16(((size_t)rcap + 2) * 4);
    s.G = reinterpret_cast<uint32_t *>(base + o);
    s.rcap = rcap;
    return s;
}

// Warp-aggregated append to a block-local list: slot list_base + the value
// of a shared counter.
__device__ __forceinline__ void cta_append(uint32_t *cursor, uint16_t *list, uint32_t list_base,
                                           bool pred, uint32_t v) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, pred);
    if (!ballot) return;
    const uint32_t leader = __ffs(ballot) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cursor, (uint32_t)__popc(ballot));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (pred) list[list_base + base + __popc(ballot & ((1u << lane) - 1u))] = (uint16_t)v;
}

// The whole path for one bucket.  Every thread of the block calls it.
// Returns false (writing nothing) when the bucket needs more rounds than its
// layer table holds; the caller reruns it with a larger table.
template <typename T, typename C>
__device__ bool run_bucket(const BatchArgs &a, uint32_t b, BucketState<T, C> s, uint32_t n,
                           uint32_t m, uint32_t *sh) {
    const uint32_t kUnc = unclaimed<C>();
    using V = VRec<T>;
    const uint32_t T_ = blockDim.x;
    const uint32_t tid = threadIdx.x;
    const uint32_t P = m / 3;
    const uint64_t key0 = a.off[b];
    uint32_t &lcur = sh[0];
    uint64_t &magic = *reinterpret_cast<uint64_t *>(sh + 2);
    if (tid == 0) {
        lcur = 0;
        magic = ~0ull / P;  // reciprocal for the remainder by P
    }
    for (uint32_t v = tid; v < m; v += T_) s.rec[v] = 0;
    for (uint32_t e = tid; e < n; e += T_) s.claim[e] = (C)kUnc;
    __syncthreads();
    const FastMod fm{P, magic};
    const uint64_t seed = b;
    // the bucket's keys, read through the cache: hashed here and again
    // whenever an edge's vertices are needed
    const uint64_t *keys = a.keys + key0;
    // hash + AddEdge
    for (uint32_t e = tid; e < n; e += T_) {
        uint32_t v[3];
        bucket_edge(__ldg(keys + e), seed, fm, P, v);
#pragma unroll
        for (int j = 0; j < 3; j++) atomicAdd(s.rec + v[j], V::unit(e));
    }
    __syncthreads();
    // round 0
    for (uint32_t v0 = 0; v0 < m; v0 += T_) {
        const uint32_t v = v0 + tid;
        bool take = false;
        uint32_t e = 0;
        if (v < m) {
            const T r = s.rec[v];
            if (V::deg(r) == 1u && V::sum(r) < n) {
                e = V::sum(r);
                const uint32_t j = (v >= P) + (v >= 2 * P);
                take = claim_min(s.claim + e, j) == kUnc;
            }
        }
        cta_append(&lcur, s.L, 0u, take, e);
    }
    // Rounds, one block barrier each: round t appends layer t + 1 from its
    // start le through counter t mod 3.  Every thread reads that counter just
    // after the round's barrier; the counter round t + 1 will use was last
    // read before the previous barrier, so thread 0 clears it during round t.
    uint32_t *cnt3 = sh + 4;  // sh[4..6]
    __syncthreads();
    if (tid == 0) {
        s.loff[0] = 0;
        s.loff[1] = lcur;
        cnt3[0] = cnt3[1] = cnt3[2] = 0;
    }
    __syncthreads();
    uint32_t t = 0, lb = 0, le = s.loff[1];
    bool too_many = false;
    while (le > lb) {
        if (t + 2 > s.rcap) {  // more rounds than the table holds (block-uniform)
            too_many = true;
            break;
        }
        uint32_t *cur = cnt3 + t % 3;
        if (tid == 0) cnt3[(t + 1) % 3] = 0;
        for (uint32_t i0 = lb; i0 < le; i0 += T_) {
            const uint32_t i = i0 + tid;
            bool take[2] = {false, false};
            uint32_t f[2] = {0, 0};
            if (i < le) {
                const uint32_t e = s.L[i];
                const uint32_t h = s.claim[e] & 3u;
                uint32_t v[3];
                bucket_edge(__ldg(keys + e), seed, fm, P, v);
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    const int j = k + ((uint32_t)k >= h ? 1 : 0);
                    const T old = atomicAdd(s.rec + v[j], (T)(0) - V::unit(e));
                    if (V::deg(old) == 2u) {
                        const uint32_t g = (V::sum(old) - e) & V::mask();
                        if (g < n) {
                            take[k] = claim_min(s.claim + g, ((t + 1) << 2) | (uint32_t)j) ==
                                      kUnc;
                            f[k] = g;
                        }
                    }
                }
            }
            cta_append(cur, s.L, le, take[0], f[0]);
            cta_append(cur, s.L, le, take[1], f[1]);
        }
        __syncthreads();
        const uint32_t next = le + *(volatile uint32_t *)cur;
        if (tid == 0) s.loff[t + 2] = next;
        lb = le;
        le = next;
        t++;
    }
    const uint32_t R = t;
    const uint32_t peeled = lb;  // loff[R]: the empty layer R starts where L ends
    __syncthreads();
    uint32_t *out = a.order + key0;
    if (too_many) return false;  // block-uniform
    // canonical order: one warp walks the edges in id order (stable), the
    // running start of every layer in cnt[0..R], the core after them
    if (tid < 32) {
        const uint32_t lane = tid;
        uint32_t *cnt = s.cnt;
        for (uint32_t r = lane; r <= R; r += 32) cnt[r] = r < R ? s.loff[r] : peeled;
        __syncwarp();
        for (uint32_t e0 = 0; e0 < n; e0 += 32) {
            const uint32_t e = e0 + lane;
            const bool valid = e < n;
            uint32_t key = 0xFFFFFFFFu;
            if (valid) {
                const uint32_t c = s.claim[e];
                key = c == kUnc ? R : (c >> 2);
            }
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
            if (valid) out[cnt[key] + __popc(peers & ((1u << lane) - 1u))] = e;
            __syncwarp();
            if (valid && lane == (uint32_t)(__ffs(peers) - 1)) cnt[key] += __popc(peers);
            __syncwarp();
        }
    }
    if (tid == 0) {
        if (a.status) a.status[b] = peeled < n ? 1u : 0u;
        if (a.rounds) a.rounds[b] = R;
    }
    __syncthreads();
    // MWHC g values (sec. 3), last layer first: layer r is L[loff[r],
    // loff[r + 1]).
    if (a.G && peeled == n) {
        const uint32_t words = (m + 15) / 16;
        for (uint32_t w = tid; w < words; w += T_) s.G[w] = 0;
        __syncthreads();
        for (int32_t r = (int32_t)R - 1; r >= 0; r--) {
            const uint32_t lo = s.loff[r], hi = s.loff[r + 1];
            for (uint32_t i = lo + tid; i < hi; i += T_) {
                const uint32_t e = s.L[i];
                const uint32_t h = s.claim[e] & 3u;
                uint32_t v[3];
                bucket_edge(__ldg(keys + e), seed, fm, P, v);
                uint32_t sum = 0;
#pragma unroll
                for (int j = 0; j < 3; j++)
                    if ((uint32_t)j != h)
                        sum += (((volatile uint32_t *)s.G)[v[j] >> 4] >> (2 * (v[j] & 15))) & 3u;
                const uint32_t val = (h + 6u - sum) % 3u;
                const uint32_t vh = v[h];
                atomicOr(s.G + (vh >> 4), (val ? val : 3u) << (2 * (vh & 15)));
            }
            __syncthreads();
        }
        uint64_t *dst = a.G + a.G_off[b];
        const uint32_t words64 = (m + 31) / 32;
        for (uint32_t w = tid; w < words64; w += T_) {
            const uint64_t lo32 = s.G[2 * w];
            const uint64_t hi32 = (2 * w + 1 < words) ? s.G[2 * w + 1] : 0u;
            dst[w] = lo32 | (hi32 << 32);
        }
    } else if (a.G) {
        uint64_t *dst = a.G + a.G_off[b];
        const uint32_t words64 = (m + 31) / 32;
        for (uint32_t w = tid; w < words64; w += T_) dst[w] = 0;
    }
    __syncthreads();
    return true;
}

__global__ void k_batched(BatchArgs a) {
    extern __shared__ __align__(16) char smem[];
    __shared__ __align__(16) uint32_t sh[8];  // sh[2..3] hold a 64-bit value
    __shared__ uint32_t s_b;
    char *region = a.scratch + (size_t)blockIdx.x * a.scratch_bytes;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t k = atomicAdd(a.next, 1u);
            s_b = k < a.B ? a.sched[k] : 0xFFFFFFFFu;
        }
        __syncthreads();
        const uint32_t b = s_b;
        __syncthreads();
        if (b == 0xFFFFFFFFu) break;
        const uint64_t n64 = a.off[b + 1] - a.off[b];
        if (n64 == 0 || n64 > kBatchMaxEdges) {
            if (threadIdx.x == 0) {
                if (a.status) a.status[b] = n64 == 0 ? 0u : 2u;
                if (a.rounds) a.rounds[b] = 0;
            }
            if (a.G && n64 == 0) {
                // nothing to write: an empty bucket has no g words
            }
            continue;
        }
        const uint32_t n = (uint32_t)n64;
        const uint32_t m = bucket_vertices(n, a.gamma_milli);
        const uint32_t rcap_s = min(n + 1, a.smem_rounds);
        bool done = false;
        if (n < 0xFFFFu && bucket_bytes(n, m, 4, 2, rcap_s) <= a.smem_bytes)
            done = run_bucket<uint32_t, uint16_t>(a, b, carve<uint32_t, uint16_t>(smem, n, m, rcap_s),
                                                  n, m, sh);
        // the global region: 32-bit records and 16-bit claims when the
        // 16-bit fields hold the bucket (fewer than 2^16 - 1 edges, at most
        // global16_rounds <= kClaim16Rounds rounds), as in shared memory;
        // else 64-bit records and 32-bit claims with room for every round
        // (n + 1 layer starts)
        if (!done && n < 0xFFFFu)
            done = run_bucket<uint32_t, uint16_t>(
                a, b, carve<uint32_t, uint16_t>(region, n, m, min(n + 1, a.global16_rounds)), n,
                m, sh);
        if (!done)
            run_bucket<unsigned long long, uint32_t>(
                a, b, carve<unsigned long long, uint32_t>(region, n, m, n + 1), n, m, sh);
    }
}

// Word offsets of the buckets' g arrays: G_off[b] = sum of ceil(m_c / 32)
// over c < b (the scan kernel turns counts into offsets).
__global__ void k_batch_g_words(const uint64_t *off, uint32_t B, uint32_t gamma_milli,
                                uint32_t *words) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const uint64_t n = off[b + 1] - off[b];
        words[b] = n <= kBatchMaxEdges ? (bucket_vertices((uint32_t)n, gamma_milli) + 31) / 32 : 0u;
    }
}

__global__ void k_widen_u32(const uint32_t *in, const uint32_t *cnt, uint32_t B, uint64_t *out) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= B; b += gridDim.x * blockDim.x)
        out[b] = b < B ? (uint64_t)in[b] : (B ? (uint64_t)in[B - 1] + cnt[B - 1] : 0ull);
}

void launch_batch_g_offsets(const Launch &L, const uint64_t *off, uint32_t B, uint32_t gamma_milli,
                            uint32_t *words, uint32_t *scanned, uint32_t *tmp, uint64_t *G_off) {
    count_launch();
    k_batch_g_words<<<grid_for(L, B ? B : 1, 1, 4), kThreads, 0, L.stream>>>(off, B, gamma_milli,
                                                                             words);
    launch_scan_u32(L, words, scanned, B, tmp);
    count_launch();
    k_widen_u32<<<grid_for(L, (uint64_t)B + 1, 1, 4), kThreads, 0, L.stream>>>(scanned, words, B,
                                                                               G_off);
}

// Largest-first schedule: buckets by size class (log2), classes descending.
__global__ void k_batch_schedule(const uint64_t *off, uint32_t B, uint32_t *sched,
                                 uint32_t *next) {
    __shared__ uint32_t cls[34];
    for (uint32_t c = threadIdx.x; c < 34; c += blockDim.x) cls[c] = 0;
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
        const uint64_t n = off[b + 1] - off[b];
        const uint32_t c = n ? 64 - __clzll(n) : 0;  // 0..33
        atomicAdd(&cls[c < 33 ? c : 33], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int c = 33; c >= 0; c--) {
            const uint32_t k = cls[c];
            cls[c] = s;
            s += k;
        }
        *next = 0;
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
        const uint64_t n = off[b + 1] - off[b];
        const uint32_t c = n ? 64 - __clzll(n) : 0;
        sched[atomicAdd(&cls[c < 33 ? c : 33], 1u)] = b;
    }
}

// Per-CTA global region: the largest bucket at this sparsity.
size_t batched_scratch_bytes(uint32_t gamma_milli) {
    const uint64_t gn = ((uint64_t)kBatchMaxEdges * gamma_milli + 999u) / 1000u;
    const uint32_t mmax = (uint32_t)((gn + 2) / 3 * 3);
    return (bucket_bytes(kBatchMaxEdges, mmax, 8, 4, kBatchMaxEdges + 1) + 255) & ~(size_t)255;
}

uint32_t batched_claim16_rounds() { return kClaim16Rounds; }

uint32_t batched_max_gamma_milli() {
    // largest gamma whose biggest bucket keeps its vertex ids within 17 bits
    uint32_t g = 1000;
    while (true) {
        const uint64_t gn = ((uint64_t)kBatchMaxEdges * (g + 1) + 999u) / 1000u;
        if ((gn + 2) / 3 * 3 > kBatchMaxVertices) return g;
        g++;
    }
}

void launch_batched(const Launch &L, const uint64_t *keys, const uint64_t *off, uint32_t B,
                    uint32_t gamma_milli, uint32_t *order, uint32_t *rounds, uint32_t *status,
                    uint64_t *G, const uint64_t *G_off, uint32_t threads, uint32_t ctas,
                    uint32_t smem_bytes, uint32_t smem_rounds, uint32_t global16_rounds,
                    uint32_t *sched, uint32_t *next, char *scratch) {
    count_launch();
    k_batch_schedule<<<1, 1024, 0, L.stream>>>(off, B, sched, next);
    BatchArgs a{keys, off, B, gamma_milli, sched, next, order, rounds, status, G, G_off,
                scratch, batched_scratch_bytes(gamma_milli), smem_bytes, smem_rounds,
                global16_rounds};
    smem_optin((const void *)k_batched);
    count_launch();
    k_batched<<<ctas, threads, smem_bytes, L.stream>>>(a);
}

}  // namespace hp
