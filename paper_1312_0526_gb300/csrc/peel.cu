// peel.cu -- packed incidence build and round-synchronous peeling.
//
// Edge records.  Edge e is one 16-byte record {v_0, v_1, v_2, claim} (r <= 3;
// 32 bytes with the claim in the second half for r = 4): one random access
// reads the vertices of an edge together with its claim word, where claim =
// (round << 2) | hinge once the edge is peeled and 0xFFFFFFFF before.
//
// Vertex records (sec. 4.1, packed incidence list with the edge id as label).
// The record of a vertex is one 64-bit word: degree in the low half, and in
// the high half the sum modulo 2^32 of the ids of its incident edges.  The
// paper combines the ids with XOR; any group operation has the property the
// XOR trick uses (with one edge left, the accumulator is that edge's id), and
// with addition one 64-bit atomicAdd updates degree and accumulator together
// and returns both.  AddEdge adds (e << 32) + 1, DeleteEdge subtracts it;
// the degree never goes below zero, so the low half never borrows from the
// high half.
//
// Rounds (sec. 4.2).  Layer L_t is the set of edges with a vertex of degree
// 1 after rounds 0..t-1.  The kernel of round t deletes every edge of L_t
// from its non-hinge vertices (the hinge keeps its record: its only edge is
// gone and no later round looks at it).  The atomic that takes a vertex from
// degree 2 to 1 returns the remaining edge f (old sum - e): that vertex is in
// the next frontier, and it claims f for round t+1 right away with atomicMin
// on f's claim word.  If f is itself in L_t, its claim already holds round t
// and the min leaves it unchanged; so the claims reaching an edge for round
// t+1 are exactly those of its degree-1 vertices after round t, the minimum
// is the hinge (smallest position) whatever the order of the atomics, and
// the single claimer that sees the unclaimed value appends f to L_{t+1} (the
// deduplication of D_i into P_i).  One kernel per round; the frontier is
// never stored.  (A vertex keeps its position j in every edge: the graph is
// r-partite, sec. 4.3.)
// Round 0 claims from a scan of all vertex records; a layer is deleted either
// from the list L (sparse) or by streaming all edge records and keeping those
// of the round (dense, for layers that are a large fraction of the edges).
#include "kernels.cuh"

namespace hp {

__global__ void k_fill_u32(uint32_t *__restrict__ p, uint64_t count, uint32_t value) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t head = (16u - ((uintptr_t)p & 15u)) / 4u % 4u;  // words to 16 B alignment
    if (((uintptr_t)p & 3u) == 0 && count > head + 4) {
        for (uint64_t k = i; k < head; k += stride) p[k] = value;
        uint4 *p4 = reinterpret_cast<uint4 *>(p + head);
        const uint64_t n4 = (count - head) / 4;
        const uint4 v4 = make_uint4(value, value, value, value);
        for (uint64_t k = i; k < n4; k += stride) p4[k] = v4;
        for (uint64_t k = head + n4 * 4 + i; k < count; k += stride) p[k] = value;
    } else {
        for (uint64_t k = i; k < count; k += stride) p[k] = value;
    }
}

void launch_fill_u32(const Launch &L, uint32_t *p, uint64_t count, uint32_t value) {
    if (count == 0) return;
    count_launch();
    k_fill_u32<<<grid_for(L, count, 16, 8), kThreads, 0, L.stream>>>(p, count, value);
}

// ------------------------------------------------------------ records --
// Row-major [n][R] edges -> records, with the r-partite check of sec. 4.3.
template <int R>
__global__ void __launch_bounds__(kThreads)
k_records(const uint32_t *__restrict__ edges, uint32_t n, uint32_t P, uint4 *__restrict__ rec,
          Ctl *ctl) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        uint32_t v[4] = {0, 0, 0, 0};
        bool ok = true;
#pragma unroll
        for (int j = 0; j < R; j++) {
            v[j] = edges[e * R + j];
            ok &= (v[j] - (uint32_t)j * P) < P;
        }
        if (!ok) raise_err(ctl, kDevBadVertex);
        store_record<R>(rec, e, v, ok);
    }
}

void launch_records(const Launch &L, const uint32_t *edges, uint32_t n, uint32_t r, uint32_t P,
                    uint4 *rec, Ctl *ctl) {
    if (n == 0) return;
    const unsigned grid = grid_for(L, n, 1, 8);
    switch (r) {
    case 2: count_launch(); k_records<2><<<grid, kThreads, 0, L.stream>>>(edges, n, P, rec, ctl); break;
    case 3: count_launch(); k_records<3><<<grid, kThreads, 0, L.stream>>>(edges, n, P, rec, ctl); break;
    case 4: count_launch(); k_records<4><<<grid, kThreads, 0, L.stream>>>(edges, n, P, rec, ctl); break;
    }
}

// ---------------------------------------------------------------- build --
// AddEdge of every edge on its r vertices: one 64-bit reduction each.
template <int R>
__global__ void __launch_bounds__(kThreads)
k_build(const uint4 *__restrict__ rec, uint32_t n, uint32_t m,
        unsigned long long *__restrict__ st, Ctl *ctl) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        uint32_t v[4];
        load_vertices<R>(rec, e, v);
        const unsigned long long add = ((unsigned long long)e << 32) | 1ull;
#pragma unroll
        for (int j = 0; j < R; j++) {
            if (v[j] < m)
                atomicAdd(st + v[j], add);
            else
                raise_err(ctl, kDevBadVertex);
        }
    }
}

void launch_build_incidence(const Launch &L, const uint4 *rec, uint32_t n, uint32_t r,
                            uint32_t m, unsigned long long *st, Ctl *ctl) {
    if (n == 0) return;
    const unsigned grid = grid_for(L, n, 1, 8);
    switch (r) {
    case 2: count_launch(); k_build<2><<<grid, kThreads, 0, L.stream>>>(rec, n, m, st, ctl); break;
    case 3: count_launch(); k_build<3><<<grid, kThreads, 0, L.stream>>>(rec, n, m, st, ctl); break;
    case 4: count_launch(); k_build<4><<<grid, kThreads, 0, L.stream>>>(rec, n, m, st, ctl); break;
    }
}

// ------------------------------------------------------- round epilogue --
// Every block adds its counts; the last block of the launch to finish
// closes round t: layer L_{t+1} is [loff[t+1], lcur) now that every append
// of the launch is done.  No block waits for another.  When the launch runs
// inside a CUDA graph's while node, the last block also sets the node's
// condition: 1 while the next layer is non-empty and the layer table has
// room (the loop ends after at most max_rounds launches whatever happens).
__device__ __forceinline__ void close_round(Ctl *ctl, uint32_t *loff, uint32_t t,
                                            uint32_t crossings, bool dense, uint32_t layer,
                                            uint32_t max_rounds, uint32_t active,
                                            cudaGraphConditionalHandle cond) {
    __shared__ uint32_t s_cross[kThreads / 32];
    const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, crossings);
    if ((threadIdx.x & 31u) == 0) s_cross[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t bsum = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; w++) bsum += s_cross[w];
        if (bsum) {
            atomicAdd(&ctl->cross, bsum);
            if (dense) atomicAdd(&ctl->dense_cross, bsum);
        }
        __threadfence();
        const uint32_t d = atomicAdd(&ctl->done, 1u);
        if (d == active - 1) {
            __threadfence();
            const uint32_t end = atomicAdd(&ctl->lcur, 0u);
            const uint32_t beg = loff[t + 1];
            loff[t + 2] = end;
            uint32_t more = end > beg ? 1u : 0u;
            if (more && t + 2 >= max_rounds) {  // round t+1 would overflow loff
                more = 0;
                atomicCAS(&ctl->err, 0u, (uint32_t)kDevCapacity);
            }
            if (dense) {
                ctl->dense_rounds += 1;
                ctl->dense_edges += layer;
            }
            ctl->next_size = end - beg;
            ctl->more = more;
            ctl->scur = beg;
            ctl->done = 0;
            ctl->round = t + 1;
            if (cond) cudaGraphSetConditional(cond, more);
        }
    }
}

// ---------------------------------------------------------------- round 0 --
// Claims of round 0 from a scan of all vertex records (F_0 is never stored).
// Layer 0 is not listed: the round-0 deletion pass is dense.  L_1 starts at
// index |L_0| of the layer list.
constexpr int kR0Items = 4;

template <int R>
__global__ void __launch_bounds__(kThreads)
k_round0(const RoundParams *__restrict__ prm, cudaGraphConditionalHandle cond) {
    const unsigned long long *__restrict__ st = prm->st;
    uint4 *__restrict__ rec = prm->rec;
    uint32_t *__restrict__ loff = prm->loff;
    Ctl *ctl = prm->ctl;
    const uint32_t m = prm->m, P = prm->P, n = prm->n;
    constexpr uint32_t kStep = kThreads * kR0Items;
    const uint64_t stride = (uint64_t)gridDim.x * kStep;
    uint32_t first = 0;
    for (uint64_t base = (uint64_t)blockIdx.x * kStep; base < m; base += stride) {
#pragma unroll
        for (int k = 0; k < kR0Items; k++) {
            const uint64_t v = base + (uint64_t)k * kThreads + threadIdx.x;
            if (v < m) {
                const unsigned long long s = __ldcs(st + v);
                if ((uint32_t)s == 1u) {
                    const uint32_t e = (uint32_t)(s >> 32);
                    if (e < n) {
                        const uint32_t j = part_of<R>((uint32_t)v, P);
                        first += atomicMin(claim_ptr<R>(rec, e), j) == kUnclaimed ? 1u : 0u;
                    } else {
                        raise_err(ctl, kDevBadEdge);
                    }
                }
            }
        }
    }
    // |L_0| = number of first claims; the last block publishes it as loff[1]
    __shared__ uint32_t s_first;
    if (threadIdx.x == 0) s_first = 0;
    __syncthreads();
    if (first) atomicAdd(&s_first, first);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_first) atomicAdd(&ctl->lcur, s_first);
        __threadfence();
        const uint32_t d = atomicAdd(&ctl->done, 1u);
        if (d == gridDim.x - 1) {
            __threadfence();
            const uint32_t end = atomicAdd(&ctl->lcur, 0u);
            loff[0] = 0;
            loff[1] = end;
            ctl->next_size = end;
            ctl->first_layer = end;
            ctl->more = end > 0 ? 1u : 0u;
            ctl->scur = 0;
            ctl->done = 0;
            ctl->round = 0;
            if (cond) cudaGraphSetConditional(cond, end > 0 ? 1u : 0u);
        }
    }
}

template <int R>
void *round0_fn() { return (void *)k_round0<R>; }

RoundLaunch round0_launch(const Launch &L, uint32_t r) {
    RoundLaunch k{};
    k.grid = grid_fixed(L, 8);
    k.block = kThreads;
    k.fn = r == 2 ? round0_fn<2>() : (r == 3 ? round0_fn<3>() : round0_fn<4>());
    return k;
}

void launch_round0(const Launch &L, uint32_t r, const RoundParams *prm) {
    const unsigned grid = grid_fixed(L, 8);
    const cudaGraphConditionalHandle c0 = 0;
    count_launch();
    switch (r) {
    case 2: k_round0<2><<<grid, kThreads, 0, L.stream>>>(prm, c0); break;
    case 3: k_round0<3><<<grid, kThreads, 0, L.stream>>>(prm, c0); break;
    case 4: k_round0<4><<<grid, kThreads, 0, L.stream>>>(prm, c0); break;
    }
}

// ---------------------------------------------------------------- rounds --
constexpr int kStageCap = 256;  // staged appends per warp

// Round t: delete layer L_t and list layer L_{t+1}.  A layer holding more
// than n / dense_div edges is read by streaming all edge records and keeping
// those claimed in round t (no solve records: such a layer is assigned from a
// record stream too); a smaller one is read from the list, and its solve
// record i goes to S[i].  Round 0 is always dense (L_0 is not listed).  The
// choice depends only on device values all blocks read alike.
// Each warp takes kRoundU * 32 consecutive entries per step, lane-strided,
// and issues every gather and atomic of its kRoundU edges before it consumes
// any result: more memory requests in flight per thread.
constexpr int kRoundU = 2;

template <int R, bool WITH_S>
__global__ void __launch_bounds__(kThreads)
k_round(const RoundParams *__restrict__ prm, cudaGraphConditionalHandle cond) {
    uint32_t *__restrict__ Llist = prm->Llist;
    uint32_t *__restrict__ loff = prm->loff;
    unsigned long long *__restrict__ st = prm->st;
    uint4 *__restrict__ rec = prm->rec;
    uint4 *__restrict__ S = prm->S;
    Ctl *ctl = prm->ctl;
    const uint32_t n = prm->n, dense_div = prm->dense_div, max_rounds = prm->max_rounds;
    __shared__ uint32_t stage_buf[kThreads / 32][kStageCap];
    WarpStage<kStageCap> stage{stage_buf[threadIdx.x >> 5], 0};
    const uint32_t t = *(volatile uint32_t *)&ctl->round;
    const uint32_t lb = loff[t], le = loff[t + 1];
    const bool dense = t == 0 || (le - lb) > n / dense_div;
    const uint64_t first = dense ? 0 : lb, last = dense ? n : le;
    constexpr uint32_t kBlockStep = kThreads * kRoundU;
    // blocks past the end of a small layer have nothing to do and take no
    // part in closing the round
    const uint64_t need = (last - first + kBlockStep - 1) / kBlockStep;
    const uint32_t active = (uint32_t)(need < gridDim.x ? (need ? need : 1) : gridDim.x);
    if (blockIdx.x >= active) return;
    const uint64_t stride = (uint64_t)active * kBlockStep;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t cross = 0;
    const unsigned long long one = 1ull;
    for (uint64_t base = first + (uint64_t)blockIdx.x * kBlockStep + (uint64_t)warp * 32 * kRoundU;
         base < last; base += stride) {
        uint32_t e[kRoundU], c[kRoundU], v[kRoundU][4];
        bool mine[kRoundU];
#pragma unroll
        for (int u = 0; u < kRoundU; u++) {
            const uint64_t i = base + (uint64_t)u * 32 + lane;
            mine[u] = false;
            c[u] = kUnclaimed;
            e[u] = 0;
            if (i < last) {
                if (dense) {
                    e[u] = (uint32_t)i;
                    c[u] = load_record_stream<R>(rec, i, v[u]);
                    mine[u] = c[u] != kUnclaimed && (c[u] >> 2) == t;
                } else {
                    e[u] = Llist[i];
                    mine[u] = true;
                }
            }
        }
        if (!dense) {
#pragma unroll
            for (int u = 0; u < kRoundU; u++)
                if (mine[u]) c[u] = load_record<R>(rec, e[u], v[u]);
        }
        // DeleteEdge on the non-hinge vertices of every edge (issued together)
        unsigned long long old[kRoundU][R - 1];
#pragma unroll
        for (int u = 0; u < kRoundU; u++) {
            const uint32_t h = c[u] & 3u;
            const unsigned long long sub = 0ull - (((unsigned long long)e[u] << 32) | one);
#pragma unroll
            for (int k = 0; k < R - 1; k++) {
                old[u][k] = 0;
                if (mine[u]) {
                    // k-th non-hinge position is k or k + 1 (static indices keep v in registers)
                    const uint32_t x = (uint32_t)k >= h ? v[u][k + 1] : v[u][k];
                    old[u][k] = atomicAdd(st + x, sub);
                }
            }
        }
        // vertices that fell to degree 1 claim their last edge for round t+1
        bool take[kRoundU][R - 1];
        uint32_t f[kRoundU][R - 1];
#pragma unroll
        for (int u = 0; u < kRoundU; u++) {
            const uint32_t h = c[u] & 3u;
#pragma unroll
            for (int k = 0; k < R - 1; k++) {
                take[u][k] = false;
                f[u][k] = 0;
                if (mine[u] && (uint32_t)old[u][k] == 2u) {
                    cross++;
                    const uint32_t j = (uint32_t)k + ((uint32_t)k >= h ? 1u : 0u);
                    const uint32_t g = (uint32_t)(old[u][k] >> 32) - e[u];  // the edge left
                    if (g < n) {
                        take[u][k] = atomicMin(claim_ptr<R>(rec, g), ((t + 1) << 2) | j) ==
                                     kUnclaimed;
                        f[u][k] = g;
                    } else {
                        raise_err(ctl, kDevBadEdge);
                    }
                }
            }
            if (WITH_S && !dense && mine[u]) S[base + (uint64_t)u * 32 + lane] = solve_record(c[u], v[u]);
        }
#pragma unroll
        for (int u = 0; u < kRoundU; u++)
#pragma unroll
            for (int k = 0; k < R - 1; k++) stage.push(take[u][k], f[u][k], &ctl->lcur, Llist);
    }
    stage.flush(&ctl->lcur, Llist);
    close_round(ctl, loff, t, cross, dense, le - lb, max_rounds, active, cond);
}

template <int R, bool WS>
void *round_fn() { return (void *)k_round<R, WS>; }

RoundLaunch round_launch(const Launch &L, bool with_s, uint32_t r) {
    RoundLaunch k{};
    k.grid = grid_fixed(L, 8);
    k.block = kThreads;
    if (with_s)
        k.fn = round_fn<3, true>();  // solve records exist for the r = 3 MPHF only
    else
        k.fn = r == 2 ? round_fn<2, false>() : (r == 3 ? round_fn<3, false>() : round_fn<4, false>());
    return k;
}

void launch_round(const Launch &L, bool with_s, uint32_t r, const RoundParams *prm) {
    const unsigned grid = grid_fixed(L, 8);
    const cudaGraphConditionalHandle c0 = 0;
    count_launch();
    if (with_s) {
        k_round<3, true><<<grid, kThreads, 0, L.stream>>>(prm, c0);
        return;
    }
    switch (r) {
    case 2: k_round<2, false><<<grid, kThreads, 0, L.stream>>>(prm, c0); break;
    case 3: k_round<3, false><<<grid, kThreads, 0, L.stream>>>(prm, c0); break;
    case 4: k_round<4, false><<<grid, kThreads, 0, L.stream>>>(prm, c0); break;
    }
}

// --------------------------------------------------------------- claims --
// Compact claim array: the API output and the key of the order sort.
template <int R>
__global__ void k_extract_claim(const uint4 *__restrict__ rec, uint32_t n,
                                uint32_t *__restrict__ claim) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        uint32_t v[4];
        claim[e] = load_record_stream<R>(rec, e, v);
    }
}

void launch_extract_claim(const Launch &L, const uint4 *rec, uint32_t n, uint32_t r,
                          uint32_t *claim) {
    if (n == 0) return;
    const unsigned grid = grid_for(L, n, 1, 8);
    switch (r) {
    case 2: count_launch(); k_extract_claim<2><<<grid, kThreads, 0, L.stream>>>(rec, n, claim); break;
    case 3: count_launch(); k_extract_claim<3><<<grid, kThreads, 0, L.stream>>>(rec, n, claim); break;
    case 4: count_launch(); k_extract_claim<4><<<grid, kThreads, 0, L.stream>>>(rec, n, claim); break;
    }
}

}  // namespace hp
