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
// t+1 are exactly those of its degree-1 vertices after round t, and the
// minimum is the hinge (smallest position) whatever the order of the
// atomics.  One kernel per round; the frontier is never stored.  (A vertex
// keeps its position j in every edge: the graph is r-partite, sec. 4.3.)
//
// Layer list.  The claimer that sees the unclaimed value (the deduplication
// of D_i into P_i) appends one entry for f: f's vertices, read from the
// record whose sector the claim atomic works on, rotated so
// that its own vertex comes first, and f's id.  Round t+1 then reads its
// layer as a sequential stream with no gather of edge records.  The first
// claimer need not be the hinge: a claimer of a smaller position may come
// later in the same round.  A later claimer whose atomicMin lowered the
// claim word therefore sets the mark bit of its vertex's record (kMark); the
// last of them holds the final minimum.  A vertex whose last edge is in L_t
// itself never marks (that claim holds round t and stays lower), so no
// deletion of round t sees a mark.  The round that deletes f takes as hinge
// the smallest position among the entry's first vertex and the marked
// vertices its DeleteEdge atomics return (all of them degree-1 vertices of f
// when round t+1 starts, and among them the true hinge), and rewrites the
// entry when the hinge moved, so each entry ends up as the solve record of
// its edge.  Round 0 claims from a scan of all vertex records and lists L_0
// the same way.
#include <mutex>
#include <set>
#include <utility>

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

// Round parameters written by a one-thread kernel (stream-ordered, no copy
// engine, no pageable host copy, which would synchronise the host).
__global__ void k_set_params(RoundParams *dst, RoundParams v) { *dst = v; }

void launch_set_params(const Launch &L, RoundParams *dst, const RoundParams &v) {
    count_launch();
    k_set_params<<<1, 1, 0, L.stream>>>(dst, v);
}

// ------------------------------------------------------------ records --
// Row-major [n][R] edges -> records, with the r-partite check of sec. 4.3.
// GEN: a general hypergraph (every vertex below P = m, any position).
template <int R, bool GEN>
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
            ok &= (v[j] - (GEN ? 0u : (uint32_t)j * P)) < P;
        }
        if (!ok) raise_err(ctl, kDevBadVertex);
        store_record<R>(rec, e, v, ok);
    }
}

void launch_records(const Launch &L, const uint32_t *edges, uint32_t n, uint32_t r, uint32_t P,
                    uint4 *rec, Ctl *ctl, bool gen) {
    if (n == 0) return;
    const unsigned grid = grid_for(L, n, 1, 8);
    count_launch();
#define HP_REC(RR)                                                                           \
    (gen ? k_records<RR, true><<<grid, kThreads, 0, L.stream>>>(edges, n, P, rec, ctl)       \
         : k_records<RR, false><<<grid, kThreads, 0, L.stream>>>(edges, n, P, rec, ctl))
    switch (r) {
    case 2: HP_REC(2); break;
    case 3: HP_REC(3); break;
    case 4: HP_REC(4); break;
    }
#undef HP_REC
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
// Every block of the launch adds its counts; the last block of the launch to
// finish closes round t: layer L_{t+1} is [loff[t+1], lcur) now that every
// append of the launch is done.  No block waits for another.  Every block
// takes part, including blocks with no entries: a block reads the round
// state (ctl->round, loff) when it starts, and a block of the same launch
// may start only after others have finished when the GPU is shared with
// other work, so the round may advance only once every block has read it.
// When the launch runs inside a CUDA graph's while node, the last block also
// sets the node's condition: 1 while the next layer is non-empty, the layer
// table has room and no kernel has raised an error (the loop ends after at
// most max_rounds launches whatever happens).
__device__ __forceinline__ void close_round(Ctl *ctl, uint32_t *loff, uint32_t t,
                                            uint32_t crossings, uint32_t moves,
                                            uint32_t max_rounds,
                                            cudaGraphConditionalHandle cond) {
    __shared__ uint32_t s_cnt[2][kThreads / 32];
    const uint32_t wc = __reduce_add_sync(0xFFFFFFFFu, crossings);
    const uint32_t wm = __reduce_add_sync(0xFFFFFFFFu, moves);
    if ((threadIdx.x & 31u) == 0) {
        s_cnt[0][threadIdx.x >> 5] = wc;
        s_cnt[1][threadIdx.x >> 5] = wm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t bc = 0, bm = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; w++) {
            bc += s_cnt[0][w];
            bm += s_cnt[1][w];
        }
        if (bc) atomicAdd(&ctl->cross, bc);
        if (bm) atomicAdd(&ctl->moves, bm);
        __threadfence();
        const uint32_t d = atomicAdd(&ctl->done, 1u);
        if (d == gridDim.x - 1) {
            __threadfence();
            const uint32_t end = atomicAdd(&ctl->lcur, 0u);
            const uint32_t beg = loff[t + 1];
            loff[t + 2] = end;
            uint32_t more = end > beg ? 1u : 0u;
            if (more && t + 2 >= max_rounds) {  // round t+1 would overflow loff
                more = 0;
                atomicCAS(&ctl->err, 0u, (uint32_t)kDevCapacity);
            }
            if (atomicAdd(&ctl->err, 0u) != 0u) more = 0;  // stop on any device error
            ctl->next_size = end - beg;
            ctl->more = more;
            ctl->done = 0;
            ctl->round = t + 1;
            if (cond) cudaGraphSetConditional(cond, more);
        }
    }
}

// Staged list entries: a per-warp buffer in dynamic shared memory, flushed
// to the list with one atomicAdd on the shared cursor per buffer-full.  The
// cursor is a single address, so its atomics serialise: the larger the
// buffer, the fewer of them (8 KiB per warp in the round kernel, 4 KiB in
// the round-0 scan).
#ifndef HPEEL_ROUND_STAGE_BYTES
#define HPEEL_ROUND_STAGE_BYTES 8192
#endif
#ifndef HPEEL_ROUND0_STAGE_BYTES
#define HPEEL_ROUND0_STAGE_BYTES 4096
#endif
template <int R, int BYTES>
constexpr int stage_cap() { return BYTES / (int)sizeof(Entry<R>); }

template <int R, int CAP>
__device__ __forceinline__ WarpStage<Entry<R>, CAP> warp_stage() {
    extern __shared__ uint4 dyn_smem[];
    return WarpStage<Entry<R>, CAP>{reinterpret_cast<Entry<R> *>(dyn_smem) + (threadIdx.x >> 5) * CAP,
                                    0};
}

// Grid (one resident wave) and dynamic shared memory of a staged kernel.
// Above 48 KiB a kernel needs the opt-in attribute, set once per kernel and
// device (not on every launch: other callers' graphs may be running).
inline RoundLaunch staged_launch(const Launch &L, void *fn, unsigned stage_bytes) {
    RoundLaunch k{};
    k.fn = fn;
    k.block = kThreads;
    k.smem = (kThreads / 32) * stage_bytes;
    if (k.smem > (48u << 10)) smem_optin(fn);
    k.grid = grid_resident(L, fn, 8, k.smem);
    return k;
}

// Claim of edge f with tag (atomicMin on its claim word, returns the old
// word), and f's vertices in position order.  The vertex words are read
// first, and the claim's address depends on the loaded word (the select is
// never taken: a vertex id is below m < 2^32 - 1), so the atomic reaches L2
// after the load has brought the record's sector in.  Issued independently,
// the two requests often fetched the same sector from DRAM twice.
//
// The claimer's position j goes into the tag (tag_hi | j): in an r-partite
// graph it is the part of the claiming vertex x (sec. 4.3); in a general
// graph (GEN) it is x's position in f's row, the first slot holding x (a
// vertex of degree 1 occurs once in its edge).
template <int R, bool GEN>
__device__ __forceinline__ uint32_t claim_and_read(uint4 *rec, uint32_t f, uint32_t tag_hi,
                                                   uint32_t x, uint32_t P, uint32_t (&p)[4],
                                                   uint32_t &j) {
    const uint4 q = __ldcg(rec + (R == 4 ? 2 * (uint64_t)f : (uint64_t)f));
    p[0] = q.x;
    p[1] = q.y;
    p[2] = R >= 3 ? q.z : 0u;
    p[3] = R == 4 ? q.w : 0u;
    if (GEN) {
        j = 0;
#pragma unroll
        for (int k = R - 1; k >= 1; k--) j = p[k] == x ? (uint32_t)k : j;
        j = p[0] == x ? 0u : j;
    } else {
        j = part_of<R>(x, P);
    }
    return atomicMin(claim_ptr<R>(rec, f) + (q.x == 0xFFFFFFFFu ? 1 : 0), tag_hi | j);
}

// The edge id field of a list entry: for a general graph it also keeps the
// hinge position in its two top bits (edge ids below 2^30).
constexpr uint32_t kGenPosShift = 30;
constexpr uint32_t kGenIdMask = (1u << kGenPosShift) - 1u;
template <bool GEN>
__device__ __forceinline__ uint32_t entry_id(uint32_t e, uint32_t h) {
    return GEN ? e | (h << kGenPosShift) : e;
}

// ---------------------------------------------------------------- round 0 --
// Claims of round 0 from a scan of all vertex records (F_0 is never stored):
// a vertex of degree 1 claims its edge with its position, and the first
// claimer of an edge lists it in L_0.  About a fifth of the vertices have
// degree 1, so each warp first queues its degree-1 vertices (vertex, edge)
// in shared memory and then claims them in full batches of 32, up to
// kR0Items batches in flight before any result is used.
constexpr int kR0Items = 4;
constexpr int kR0Queue = 32 * (kR0Items + 1);  // queued vertices per warp

template <int R, bool GEN>
__device__ __forceinline__ void round0_claims(int batches, const uint2 *q, uint32_t lane_limit,
                                              unsigned long long *st, uint4 *rec, uint32_t P,
                                              WarpStage<Entry<R>, stage_cap<R, HPEEL_ROUND0_STAGE_BYTES>()> &stage,
                                              Ctl *ctl, Entry<R> *Lst) {
    const uint32_t lane = threadIdx.x & 31u;
    bool first[kR0Items], have[kR0Items];
    uint32_t pv[kR0Items][4], jv[kR0Items], ev[kR0Items];
#pragma unroll
    for (int b = 0; b < kR0Items; b++) {
        first[b] = false;
        have[b] = false;
        jv[b] = 0;
        ev[b] = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) pv[b][k] = 0;
        if (b < batches) {
            const uint32_t slot = (uint32_t)b * 32u + lane;
            have[b] = slot < lane_limit;
            if (have[b]) {
                const uint2 it = q[slot];  // {vertex, edge}
                uint32_t j;
                const uint32_t c = claim_and_read<R, GEN>(rec, it.y, 0u, it.x, P, pv[b], j);
                first[b] = c == kUnclaimed;
                // a later claimer that lowered the claim marks its vertex;
                // this kernel is the record's only writer
                if (!first[b] && j < c) st[it.x] = ((unsigned long long)it.y << 32) | (1u | kMark);
                jv[b] = j;
                ev[b] = it.y;
            }
        }
    }
#pragma unroll
    for (int b = 0; b < kR0Items; b++) {
        if (b < batches) {
            uint32_t x[4];
            rotate_to<R>(pv[b], jv[b], x);
            stage.push(first[b], make_entry<R>(x, entry_id<GEN>(ev[b], jv[b])), &ctl->lcur, Lst);
        }
    }
}

template <int R, bool GEN>
__global__ void __launch_bounds__(kThreads)
k_round0(const RoundParams *__restrict__ prm, cudaGraphConditionalHandle cond) {
    unsigned long long *__restrict__ st = prm->st;
    uint4 *__restrict__ rec = prm->rec;
    Entry<R> *__restrict__ Lst = reinterpret_cast<Entry<R> *>(prm->L);
    uint32_t *__restrict__ loff = prm->loff;
    Ctl *ctl = prm->ctl;
    const uint32_t m = prm->m, P = prm->P, n = prm->n;
    constexpr int kCap = stage_cap<R, HPEEL_ROUND0_STAGE_BYTES>();
    auto stage = warp_stage<R, kCap>();
    __shared__ uint2 queue[kThreads / 32][kR0Queue];
    uint2 *q = queue[threadIdx.x >> 5];
    uint32_t qn = 0;  // warp-uniform queue length
    const uint32_t lane = threadIdx.x & 31u;
    constexpr uint32_t kStep = kThreads * kR0Items;
    const uint64_t stride = (uint64_t)gridDim.x * kStep;
    // whole warps step together: the trip count depends on blockIdx only
    for (uint64_t base = (uint64_t)blockIdx.x * kStep; base < m; base += stride) {
#pragma unroll
        for (int k = 0; k < kR0Items; k++) {
            const uint64_t v = base + (uint64_t)k * kThreads + threadIdx.x;
            bool one = false;
            uint32_t e = 0;
            if (v < m) {
                const unsigned long long s = __ldcs(st + v);
                const uint32_t deg = (uint32_t)s;
                if (deg & kMark) raise_err(ctl, kDevDegree);
                e = (uint32_t)(s >> 32);
                if (deg == 1u) {
                    one = e < n;
                    if (!one) raise_err(ctl, kDevBadEdge);
                }
            }
            const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, one);
            if (one) q[qn + __popc(ballot & ((1u << lane) - 1u))] = make_uint2((uint32_t)v, e);
            qn += __popc(ballot);
        }
        __syncwarp();
        const int full = (int)(qn >> 5);  // < kR0Items + 1 batches
        if (full) {
            round0_claims<R, GEN>(full, q, (uint32_t)full * 32u, st, rec, P, stage, ctl, Lst);
            // move the partial batch to the front
            const uint32_t rest = qn - (uint32_t)full * 32u;
            uint2 keep = make_uint2(0u, 0u);
            if (lane < rest) keep = q[(uint32_t)full * 32u + lane];
            __syncwarp();
            if (lane < rest) q[lane] = keep;
            qn = rest;
            __syncwarp();
        }
    }
    if (qn) round0_claims<R, GEN>(1, q, qn, st, rec, P, stage, ctl, Lst);
    stage.flush(&ctl->lcur, Lst);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&ctl->done, 1u);
        if (d == gridDim.x - 1) {
            __threadfence();
            const uint32_t end = atomicAdd(&ctl->lcur, 0u);
            // no round after a device error (the build's included)
            const uint32_t more = (end > 0 && atomicAdd(&ctl->err, 0u) == 0u) ? 1u : 0u;
            loff[0] = 0;
            loff[1] = end;
            ctl->next_size = end;
            ctl->first_layer = end;
            ctl->more = more;
            ctl->done = 0;
            ctl->round = 0;
            if (cond) cudaGraphSetConditional(cond, more);
        }
    }
}

template <int R>
void *round0_fn(bool gen) { return gen ? (void *)k_round0<R, true> : (void *)k_round0<R, false>; }

RoundLaunch round0_launch(const Launch &L, uint32_t r, bool gen) {
    return staged_launch(
        L, r == 2 ? round0_fn<2>(gen) : (r == 3 ? round0_fn<3>(gen) : round0_fn<4>(gen)),
        HPEEL_ROUND0_STAGE_BYTES);
}

void launch_round0(const Launch &L, uint32_t r, bool gen, const RoundParams *prm) {
    const RoundLaunch k = round0_launch(L, r, gen);
    cudaGraphConditionalHandle c0 = 0;
    void *args[] = {(void *)&prm, &c0};
    count_launch();
    cudaLaunchKernel(k.fn, dim3(k.grid), dim3(k.block), args, k.smem, L.stream);
}

// ---------------------------------------------------------------- rounds --
// Round t: delete layer L_t, read from the list as a stream, and list layer
// L_{t+1}.  Each warp takes kRoundU * 32 consecutive entries per step,
// lane-strided, and issues every atomic of its kRoundU edges before it
// consumes any result: more memory requests in flight per thread.
#ifndef HPEEL_ROUND_U
#define HPEEL_ROUND_U 2
#endif
// r = 4 carries more registers per edge: two edges per thread
template <int R>
constexpr int round_u() { return R == 4 ? 2 : HPEEL_ROUND_U; }

#ifndef HPEEL_ROUND_MIN_BLOCKS
#define HPEEL_ROUND_MIN_BLOCKS 3
#endif
template <int R, bool GEN>
__global__ void __launch_bounds__(kThreads, HPEEL_ROUND_MIN_BLOCKS)
k_round(const RoundParams *__restrict__ prm, cudaGraphConditionalHandle cond) {
    constexpr int kRoundU = round_u<R>();
    uint4 *__restrict__ Lw = prm->L;
    Entry<R> *__restrict__ Lst = reinterpret_cast<Entry<R> *>(prm->L);
    uint32_t *__restrict__ loff = prm->loff;
    unsigned long long *__restrict__ st = prm->st;
    uint4 *__restrict__ rec = prm->rec;
    Ctl *ctl = prm->ctl;
    const uint32_t n = prm->n, P = prm->P, max_rounds = prm->max_rounds;
    constexpr int kCap = stage_cap<R, HPEEL_ROUND_STAGE_BYTES>();
    auto stage = warp_stage<R, kCap>();
    const uint32_t t = *(volatile uint32_t *)&ctl->round;
    uint32_t lb = loff[t], le = loff[t + 1];
    if (lb > le || le > n) {  // inconsistent state: report, delete nothing
        raise_err(ctl, kDevCapacity);
        lb = le;
    }
    constexpr uint32_t kBlockStep = kThreads * kRoundU;
    // a small layer is spread over as many blocks as it fills; the others
    // skip the loop but still take part in closing the round
    const uint64_t need = ((uint64_t)(le - lb) + kBlockStep - 1) / kBlockStep;
    const uint32_t active = (uint32_t)(need < gridDim.x ? (need ? need : 1) : gridDim.x);
    const uint64_t stride = (uint64_t)active * kBlockStep;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t cross = 0, moves = 0;
    const unsigned long long one = 1ull;
    const uint64_t first = blockIdx.x < active ? lb + (uint64_t)blockIdx.x * kBlockStep +
                                                     (uint64_t)warp * 32 * kRoundU
                                               : (uint64_t)le;
    for (uint64_t base = first; base < le; base += stride) {
        uint32_t e[kRoundU], v[kRoundU][4], hg[kRoundU];
        bool mine[kRoundU];
#pragma unroll
        for (int u = 0; u < kRoundU; u++) {
            const uint64_t i = base + (uint64_t)u * 32 + lane;
            mine[u] = i < le;
            e[u] = 0;
            hg[u] = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) v[u][k] = 0;
            if (mine[u]) {
                const uint32_t w = load_entry<R>(Lw, i, v[u]);
                e[u] = GEN ? w & kGenIdMask : w;
                hg[u] = GEN ? w >> kGenPosShift : part_of<R>(v[u][0], P);
            }
        }
        // DeleteEdge on every vertex but the entry's first (issued together)
        unsigned long long old[kRoundU][R - 1];
#pragma unroll
        for (int u = 0; u < kRoundU; u++) {
            const unsigned long long sub = 0ull - (((unsigned long long)e[u] << 32) | one);
#pragma unroll
            for (int k = 0; k < R - 1; k++)
                old[u][k] = mine[u] ? atomicAdd(st + v[u][k + 1], sub) : 0ull;
        }
        // hinge: smallest position among the first vertex and the marked ones
#pragma unroll
        for (int u = 0; u < kRoundU; u++) {
            uint32_t h = hg[u];
#pragma unroll
            for (int k = R - 2; k >= 0; k--) {
                const uint32_t pos = (uint32_t)k + ((uint32_t)k >= hg[u] ? 1u : 0u);
                if (((uint32_t)old[u][k] & kMark) && pos < h) h = pos;
            }
            if (mine[u] && h != hg[u]) {
                uint32_t p[4], q[4];
                unrotate<R>(v[u], hg[u], p);
                rotate_to<R>(p, h, q);
                store_entry<R>(Lw, base + (uint64_t)u * 32 + lane,
                               make_entry<R>(q, entry_id<GEN>(e[u], h)));
                moves++;
            }
        }
        // vertices that fell to degree 1 mark themselves and claim their last
        // edge for round t+1; the vertex words of that edge come along
        bool take[kRoundU][R - 1];
        uint32_t f[kRoundU][R - 1], pf[kRoundU][R - 1][4], jf[kRoundU][R - 1];
#pragma unroll
        for (int u = 0; u < kRoundU; u++) {
#pragma unroll
            for (int k = 0; k < R - 1; k++) {
                take[u][k] = false;
                f[u][k] = 0;
                jf[u][k] = 0;
#pragma unroll
                for (int q = 0; q < 4; q++) pf[u][k][q] = 0;
                if (mine[u] && (uint32_t)old[u][k] == 2u) {
                    cross++;
                    const uint32_t g = (uint32_t)(old[u][k] >> 32) - e[u];  // the edge left
                    if (g < n) {
                        const uint32_t tag_hi = (t + 1) << 2;
                        uint32_t j;
                        const uint32_t c =
                            claim_and_read<R, GEN>(rec, g, tag_hi, v[u][k + 1], P, pf[u][k], j);
                        const uint32_t tag = tag_hi | j;
                        jf[u][k] = j;
                        take[u][k] = c == kUnclaimed;
                        f[u][k] = g;
                        // a later claimer that lowered the claim marks its
                        // vertex (never one whose last edge is in L_t: its
                        // claim holds round t and stays lower)
                        if (!take[u][k] && tag < c)
                            atomicOr(reinterpret_cast<unsigned int *>(st + v[u][k + 1]), kMark);
                    } else {
                        raise_err(ctl, kDevBadEdge);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kRoundU; u++)
#pragma unroll
            for (int k = 0; k < R - 1; k++) {
                uint32_t q[4];
                rotate_to<R>(pf[u][k], jf[u][k], q);
                stage.push(take[u][k], make_entry<R>(q, entry_id<GEN>(f[u][k], jf[u][k])),
                           &ctl->lcur, Lst);
            }
    }
    stage.flush(&ctl->lcur, Lst);
    close_round(ctl, loff, t, cross, moves, max_rounds, cond);
}

template <int R>
void *round_fn(bool gen) { return gen ? (void *)k_round<R, true> : (void *)k_round<R, false>; }

RoundLaunch round_launch(const Launch &L, uint32_t r, bool gen) {
    return staged_launch(
        L, r == 2 ? round_fn<2>(gen) : (r == 3 ? round_fn<3>(gen) : round_fn<4>(gen)),
        HPEEL_ROUND_STAGE_BYTES);
}

void launch_round(const Launch &L, uint32_t r, bool gen, const RoundParams *prm) {
    const RoundLaunch k = round_launch(L, r, gen);
    cudaGraphConditionalHandle c0 = 0;
    void *args[] = {(void *)&prm, &c0};
    count_launch();
    cudaLaunchKernel(k.fn, dim3(k.grid), dim3(k.block), args, k.smem, L.stream);
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
