// build.cu -- L2-blocked incidence build (sec. 4.1 AddEdge for every edge).
//
// AddEdge hits the vertex records in random order: with the records far
// larger than L2, every update is a DRAM sector read and write.  Here the
// updates are first bucketed by vertex range -- the paper's own remedy for
// random access (sec. 4.2 builds E_0 by sorting the orientations by vertex,
// sec. 4.3 part by part) -- and then applied range by range in shared
// memory, so every vertex record is written once:
//   pass 1 (fused with hashing, or with the row -> record conversion): each
//          block takes tiles of edges, writes their records, counting-sorts
//          a tile's (vertex, edge) incidences by chunk (2^shift vertices of
//          one part) in shared memory and appends each chunk's run to the
//          chunk's array (one atomicAdd per chunk and tile on its cursor),
//          so the pass writes at one moving front per chunk;
//   pass 2 (refine): a persistent kernel counting-sorts each chunk's pairs,
//          a tile at a time, into sub-buckets of 2^sub_shift vertices;
//   pass 3 (apply): one block per sub-bucket accumulates its vertices'
//          degrees and id sums in shared memory and writes the records.
// Large graphs run the three passes once per part (sec. 4.3 builds the
// incidence lists one part at a time): position j's incidences are bucketed
// and applied in pass j, so the buckets hold one incidence per edge instead
// of r.  Capacities cover the expected load with a wide margin; an incidence
// that finds its chunk's array full goes to an overflow list applied with direct
// updates, and when that list is full as well the build reports it and is
// redone with direct updates (same result), so any input is handled.
#include <algorithm>
#include <cmath>

#include "kernels.cuh"

namespace hp {

#ifndef HPEEL_RB_TILE
#define HPEEL_RB_TILE 2048
#endif
constexpr int kTileEdges = HPEEL_RB_TILE;  // edges per block step
#ifndef HPEEL_RB_THREADS
#define HPEEL_RB_THREADS 512
#endif
constexpr int kRbThreads = HPEEL_RB_THREADS;     // threads of a record-pass block
constexpr int kTileU = kTileEdges / kRbThreads;  // edges per thread and step

// Chunk of vertex v at position j: chunks never straddle the parts of an
// r-partite graph; a general graph (GEN) is one part [0, P = m).
template <bool GEN>
__device__ __forceinline__ uint32_t chunk_of(uint32_t v, uint32_t j, const BucketGeom &g) {
    const uint32_t part = GEN ? 0u : j;
    return part * g.chunks_per_part + ((v - part * g.P) >> g.shift);
}

// An incidence that finds its chunk's array full goes to the overflow list, applied
// after everything else; when the list itself is full the build fails with
// kDevBuildOverflow and the host redoes it with direct updates.
__device__ __forceinline__ void overflow_push(uint2 p, Overflow ov, Ctl *ctl) {
    const uint32_t k = ov.count ? atomicAdd(ov.count, 1u) : ov.cap;
    if (k < ov.cap)
        ov.list[k] = p;
    else
        atomicCAS(&ctl->err, 0u, ov.code);
}

#ifndef HPEEL_RB_MIN_BLOCKS
#define HPEEL_RB_MIN_BLOCKS 2
#endif
constexpr uint32_t kCurRegs = 2;  // chunk cursors per thread held in registers
template <int R, bool FROM_KEYS, bool GEN>
__global__ void __launch_bounds__(kRbThreads, HPEEL_RB_MIN_BLOCKS)
k_records_bucketed(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ rows,
                   uint32_t n, FastMod fm, uint64_t seed, const uint64_t *seed_dev, BucketGeom g,
                   uint4 *__restrict__ rec,
                   uint2 *__restrict__ pairs, uint32_t *__restrict__ fill, Overflow ov,
                   Ctl *ctl, int pass_part) {
    if (FROM_KEYS && seed_dev) seed = *seed_dev;  // the seed of a device-driven attempt
    extern __shared__ uint32_t smem[];
    // pass_part < 0: every position's incidences, chunks of all parts; else
    // only position pass_part's, chunks numbered inside that part
    const uint32_t C = pass_part >= 0 ? g.chunks_per_part
                                      : (GEN ? 1u : (uint32_t)R) * g.chunks_per_part;
    const bool write_rec = pass_part <= 0;  // records are written by the first pass
    auto in_pass = [&](int j) { return pass_part < 0 || j == pass_part; };
    auto chunk_here = [&](uint32_t v, int j) {
        return pass_part >= 0 ? (v - (uint32_t)j * g.P) >> g.shift : chunk_of<GEN>(v, j, g);
    };
    const uint32_t Cp = (C + 1) & ~1u;
    uint32_t *hist = smem;            // C: tile count per chunk
    uint32_t *cur = hist + Cp;        // C: the run's place in its chunk minus its stage slot
    uint32_t *toff = cur + Cp;        // C: start of the chunk's run in stage
    uint2 *stage = reinterpret_cast<uint2 *>(toff + Cp);  // R per edge (8-byte aligned: Cp even)

    const uint64_t tiles = ((uint64_t)n + kTileEdges - 1) / kTileEdges;
    // the next tile's input (keys, or rows) is loaded while this one is
    // hashed, sorted and written
    constexpr int kWords = FROM_KEYS ? 2 : R;  // 32-bit words of input per edge
    auto load_input = [&](uint64_t tile, uint32_t (&in)[kTileU][kWords]) {
#pragma unroll
        for (int q = 0; q < kTileU; q++) {
            const uint64_t e = tile * kTileEdges + (uint64_t)q * kRbThreads + threadIdx.x;
#pragma unroll
            for (int w = 0; w < kWords; w++) in[q][w] = 0;
            if (e < n) {
                if (FROM_KEYS) {
                    const uint64_t k = __ldcs(keys + e);
                    in[q][0] = (uint32_t)k;
                    in[q][kWords - 1] = (uint32_t)(k >> 32);
                } else {
#pragma unroll
                    for (int j = 0; j < kWords; j++)
                        if (write_rec || j == pass_part) in[q][j] = __ldcs(rows + e * R + j);
                }
            }
        }
    };
    uint32_t next_in[kTileU][kWords];
    if ((uint64_t)blockIdx.x < tiles) load_input(blockIdx.x, next_in);
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        uint32_t in[kTileU][kWords];
#pragma unroll
        for (int q = 0; q < kTileU; q++)
#pragma unroll
            for (int w = 0; w < kWords; w++) in[q][w] = next_in[q][w];
        if (tile + gridDim.x < tiles) load_input(tile + gridDim.x, next_in);
        for (uint32_t c = threadIdx.x; c < C; c += kRbThreads) hist[c] = 0;
        __syncthreads();
        uint32_t vv[kTileU][R], rank[kTileU][R];
        bool inc[kTileU];
#pragma unroll
        for (int q = 0; q < kTileU; q++) {
            const uint64_t e = tile * kTileEdges + (uint64_t)q * kRbThreads + threadIdx.x;
            uint32_t v[4] = {0, 0, 0, 0};
            bool ok = e < n;
            if (ok) {
                if (FROM_KEYS) {
                    const uint64_t k = ((uint64_t)in[q][kWords - 1] << 32) | in[q][0];
                    // a pass that writes no records needs only its own position
#pragma unroll
                    for (int j = 0; j < R; j++)
                        if (write_rec || j == pass_part)
                            v[j] = (uint32_t)fastmod(mix64(k ^ (seed + (uint64_t)j)), fm) +
                                   (uint32_t)j * g.P;
                } else {
#pragma unroll
                    for (int j = 0; j < R; j++) {
                        if (!write_rec && j != pass_part) continue;  // checked by pass 0
                        v[j] = in[q][j];
                        ok &= (v[j] - (GEN ? 0u : (uint32_t)j * g.P)) < g.P;
                    }
                    if (!ok) raise_err(ctl, kDevBadVertex);
                }
                if (write_rec) store_record<R>(rec, e, v, ok);
            }
            inc[q] = ok;  // an invalid row adds nothing (the call fails)
#pragma unroll
            for (int j = 0; j < R; j++) {
                vv[q][j] = v[j];
                rank[q][j] = ok && in_pass(j) ? atomicAdd(&hist[chunk_here(v[j], j)], 1u) : 0u;
            }
        }
        __syncthreads();
        // reserve each chunk's run with one atomicAdd on its cursor; the
        // results are awaited only after the staging below
        uint32_t gb[kCurRegs];
#pragma unroll
        for (uint32_t q = 0; q < kCurRegs; q++) {
            const uint32_t c = q * kRbThreads + threadIdx.x, h = c < C ? hist[c] : 0u;
            gb[q] = h ? atomicAdd(fill + ((size_t)c << g.fill_shift), h) : 0u;
        }
        for (uint32_t c = kCurRegs * kRbThreads + threadIdx.x; c < C; c += kRbThreads) {
            const uint32_t h = hist[c];
            cur[c] = h ? atomicAdd(fill + ((size_t)c << g.fill_shift), h) : 0u;
        }
        // exclusive scan of hist -> toff (warp 0, 32 chunks per step; the
        // other warps' cursor reservations are in flight meanwhile)
        if (threadIdx.x < 32) {
            const uint32_t lane = threadIdx.x;
            uint32_t run = 0;
            for (uint32_t c0 = 0; c0 < C; c0 += 32) {
                const uint32_t c = c0 + lane;
                const uint32_t h = c < C ? hist[c] : 0u;
                uint32_t x = h;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
                    if (lane >= (uint32_t)d) x += y;
                }
                if (c < C) toff[c] = run + x - h;
                run += __shfl_sync(0xFFFFFFFFu, x, 31);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kTileU; q++) {
            if (!inc[q]) continue;
            const uint32_t e = (uint32_t)(tile * kTileEdges + (uint64_t)q * kRbThreads + threadIdx.x);
#pragma unroll
            for (int j = 0; j < R; j++) {
                if (!in_pass(j)) continue;
                const uint32_t c = chunk_here(vv[q][j], j);
                const uint32_t slot = toff[c] + rank[q][j];
                stage[slot] = make_uint2(vv[q][j], e);
            }
        }
        // cur[c] = the run's first place in chunk c - its first stage slot
        // (mod 2^32): staged pair k of chunk c goes to place cur[c] + k
#pragma unroll
        for (uint32_t q = 0; q < kCurRegs; q++) {
            const uint32_t c = q * kRbThreads + threadIdx.x;
            if (c < C) cur[c] = gb[q] - toff[c];
        }
        for (uint32_t c = kCurRegs * kRbThreads + threadIdx.x; c < C; c += kRbThreads)
            cur[c] -= toff[c];
        __syncthreads();
        // write the staged runs: consecutive slots -> consecutive addresses
        const uint32_t total = toff[C - 1] + hist[C - 1];
        for (uint32_t k = threadIdx.x; k < total; k += kRbThreads) {
            const uint2 p = stage[k];
            // its chunk again, from the vertex (an r-partite graph's part
            // follows from the vertex id)
            const uint32_t c = pass_part >= 0 ? chunk_here(p.x, pass_part)
                                              : chunk_of<GEN>(p.x, GEN ? 0u : part_of<R>(p.x, g.P), g);
            const uint32_t pos = cur[c] + k;
            if (pos < g.cap)
                pairs[(uint64_t)c * g.cap + pos] = p;
            else
                overflow_push(p, ov, ctl);
        }
        __syncthreads();
    }
}

// Refine: the pairs of each chunk's array are counting-sorted in
// shared memory, a tile of kRefineTile slots at a time, into 2^(shift -
// sub_shift) sub-buckets of 2^sub_shift vertices; each tile's run of a
// sub-bucket is appended to it with one atomicAdd on its cursor.  One
// resident wave of blocks strides over the filled (chunk, tile) items; the next
// item's pairs are loaded into registers while the current one is sorted
// and written, so the load latency overlaps the work.
#ifndef HPEEL_REFINE_THREADS
#define HPEEL_REFINE_THREADS 512
#endif
#ifndef HPEEL_REFINE_ITEMS
#define HPEEL_REFINE_ITEMS 8
#endif
#ifndef HPEEL_REFINE_MIN_BLOCKS
#define HPEEL_REFINE_MIN_BLOCKS 2
#endif
constexpr int kRefThreads = HPEEL_REFINE_THREADS;
constexpr int kRefineItems = HPEEL_REFINE_ITEMS;
constexpr uint32_t kRefineTile = kRefThreads * kRefineItems;  // 4096 slots
constexpr uint32_t kRefWarps = kRefThreads / 32;
constexpr uint32_t kScanRegs = 4;  // sub-buckets per thread whose cursor stays in registers

__global__ void __launch_bounds__(kRefThreads, HPEEL_REFINE_MIN_BLOCKS)
k_refine_buckets(const uint2 *__restrict__ pairs, const uint32_t *__restrict__ fill, BucketGeom g,
                 uint32_t chunks, uint32_t chunk0, uint32_t sub_shift,
                 uint2 *__restrict__ pairs2, uint32_t *__restrict__ fill2, uint32_t cap2,
                 Overflow ov, Ctl *ctl) {
    extern __shared__ uint32_t smem[];
    const uint32_t S = 1u << (g.shift - sub_shift);
    uint32_t *hist = smem;          // S
    uint32_t *gbase = hist + S;     // S: sub-bucket cursor minus the run's first stage slot
    uint32_t *toff = gbase + S;     // S
    uint32_t *wsum = toff + S;      // kRefWarps: scan totals of the warps
    uint32_t *tstart = wsum + kRefWarps;  // chunks + 1: first item of each chunk
    // kRefineTile pairs, 8-byte aligned whatever S is
    uint2 *stage =
        reinterpret_cast<uint2 *>(smem + ((3 * S + kRefWarps + chunks + 1 + 1) & ~1u));
    // the scan gives each thread `per` consecutive sub-buckets
    const uint32_t per = (S + kRefThreads - 1) / kRefThreads, b0 = threadIdx.x * per;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    // items = the filled tiles of kRefineTile pairs of every chunk, numbered
    // chunk after chunk (a chunk's array may be far from full: a sorted
    // round's layer is a fraction of the largest one): tstart[c] = first
    // item of chunk c, from one block-wide scan of the tile counts
    auto chunk_fill = [&](uint32_t c) {
        return min(__ldg(fill + ((size_t)c << g.fill_shift)), g.cap);
    };
    {
        const uint32_t cper = (chunks + kRefThreads - 1) / kRefThreads, c0 = threadIdx.x * cper;
        uint32_t loc = 0;
        for (uint32_t q = 0; q < cper; q++)
            if (c0 + q < chunks) loc += (chunk_fill(c0 + q) + kRefineTile - 1) / kRefineTile;
        uint32_t x = loc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= (uint32_t)d) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t run = x - loc;
        for (uint32_t w = 0; w < warp; w++) run += wsum[w];
        for (uint32_t q = 0; q < cper; q++) {
            const uint32_t c = c0 + q;
            if (c < chunks) {
                tstart[c] = run;
                run += (chunk_fill(c) + kRefineTile - 1) / kRefineTile;
            }
        }
        if (threadIdx.x == kRefThreads - 1) tstart[chunks] = run;
        __syncthreads();
    }
    const uint32_t items = tstart[chunks];
    // the chunk of an item: a block's items only go up, so its chunk cursor
    // only moves forward (the last c with tstart[c] <= it)
    auto advance = [&](uint32_t it, uint32_t &c) {
        while (tstart[c + 1] <= it) c++;
    };
    auto load_item = [&](uint32_t it, uint32_t c, uint32_t &tn, uint2 (&p)[kRefineItems]) {
        const uint32_t t0 = (it - tstart[c]) * kRefineTile;
        tn = min(chunk_fill(c) - t0, kRefineTile);
        const uint2 *tsrc = pairs + (uint64_t)c * g.cap + t0;
#pragma unroll
        for (int q = 0; q < kRefineItems; q++) {
            const uint32_t i = (uint32_t)q * kRefThreads + threadIdx.x;
            p[q] = i < tn ? __ldcs(tsrc + i) : make_uint2(0u, 0u);
        }
    };
    uint32_t it = blockIdx.x, tn_next = 0, c_next = 0;
    uint2 pn[kRefineItems];
    if (it < items) {
        advance(it, c_next);
        load_item(it, c_next, tn_next, pn);
    }
    while (it < items) {
        const uint32_t c = c_next;  // chunk of this pass
        const uint32_t cg = chunk0 + c;              // chunk of the whole build
        const uint32_t part = cg / g.chunks_per_part;
        const uint32_t base_v = part * g.P + (cg % g.chunks_per_part) * (1u << g.shift);
        const uint32_t tn = tn_next;
        uint2 p[kRefineItems];
#pragma unroll
        for (int q = 0; q < kRefineItems; q++) p[q] = pn[q];
        const uint32_t nxt = it + gridDim.x;
        if (nxt < items) {
            advance(nxt, c_next);
            load_item(nxt, c_next, tn_next, pn);
        }
        for (uint32_t b = threadIdx.x; b < S; b += kRefThreads) hist[b] = 0;
        __syncthreads();
        uint32_t rk[kRefineItems];
        uint32_t bq[kRefineItems];  // sub-bucket of each pair, S for none
#pragma unroll
        for (int q = 0; q < kRefineItems; q++) {
            const uint32_t i = (uint32_t)q * kRefThreads + threadIdx.x;
            bq[q] = i < tn ? (p[q].x - base_v) >> sub_shift : S;
            // a pair outside the chunk (inconsistent input) is dropped with an error
            if (i < tn && bq[q] >= S) raise_err(ctl, kDevBadVertex);
            rk[q] = bq[q] < S ? atomicAdd(&hist[bq[q]], 1u) : 0u;
        }
        __syncthreads();
        // reserve each sub-bucket's run with one atomicAdd on its cursor;
        // the results are awaited only after the staging below
        uint32_t gb[kScanRegs];
#pragma unroll
        for (uint32_t q = 0; q < kScanRegs; q++) {
            const uint32_t b = b0 + q, h = q < per && b < S ? hist[b] : 0u;
            gb[q] = h ? atomicAdd(fill2 + (size_t)c * S + b, h) : 0u;
        }
        for (uint32_t q = kScanRegs; q < per; q++) {  // S > kRefThreads * kScanRegs
            const uint32_t b = b0 + q, h = b < S ? hist[b] : 0u;
            if (b < S) gbase[b] = h ? atomicAdd(fill2 + (size_t)c * S + b, h) : 0u;
        }
        {   // exclusive scan of hist -> toff over the whole block
            uint32_t loc = 0;
            for (uint32_t q = 0; q < per; q++)
                if (b0 + q < S) loc += hist[b0 + q];
            uint32_t x = loc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
                if (lane >= (uint32_t)d) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            // the totals of the warps before this one: a shuffle prefix
            uint32_t wx = lane < kRefWarps ? wsum[lane] : 0u;
#pragma unroll
            for (int d = 1; d < (int)kRefWarps; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wx, d);
                if (lane >= (uint32_t)d) wx += y;
            }
            const uint32_t before = __shfl_sync(0xFFFFFFFFu, wx, (warp + 31u) & 31u);
            uint32_t run = x - loc + (warp ? before : 0u);
            for (uint32_t q = 0; q < per; q++) {
                const uint32_t b = b0 + q;
                if (b < S) {
                    toff[b] = run;
                    run += hist[b];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kRefineItems; q++)
            if (bq[q] < S) stage[toff[bq[q]] + rk[q]] = p[q];
        // gbase[b] = cursor - first stage slot of the run: a staged pair at
        // slot k goes to position gbase[b] + k of its sub-bucket
#pragma unroll
        for (uint32_t q = 0; q < kScanRegs; q++)
            if (q < per && b0 + q < S) gbase[b0 + q] = gb[q] - toff[b0 + q];
        for (uint32_t q = kScanRegs; q < per; q++)
            if (b0 + q < S) gbase[b0 + q] -= toff[b0 + q];
        __syncthreads();
        const uint32_t total = toff[S - 1] + hist[S - 1];
        // this chunk's sub-buckets: S * cap2 slots, below 2^32 (the plans
        // check it), so a slot's index takes 32-bit arithmetic
        uint2 *const cdst = pairs2 + (size_t)c * S * cap2;
        for (uint32_t k = threadIdx.x; k < total; k += kRefThreads) {
            const uint2 q = stage[k];
            const uint32_t b = (q.x - base_v) >> sub_shift;  // its sub-bucket, again
            const uint32_t pos = gbase[b] + k;
            if (pos < cap2)
                cdst[b * cap2 + pos] = q;
            else
                overflow_push(q, ov, ctl);
        }
        __syncthreads();
        it = nxt;
    }
}

// One block per sub-bucket: degrees and id sums of its 2^sub_shift vertices
// accumulate in shared memory (two 32-bit atomics per incidence: the record's
// halves are independent, AddEdge never carries from one into the other),
// then every vertex record of the range is written once.
// Exclusive block-wide prefix sum of one value per thread (1024 threads);
// *total receives the sum.  Every thread calls it.
__device__ __forceinline__ uint32_t block_scan_1024(uint32_t v, uint32_t *total) {
    __shared__ uint32_t ws[32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = ws[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
            if (lane >= (uint32_t)d) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    const uint32_t before = (warp ? ws[warp - 1] : 0u) + x - v;
    *total = ws[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(1024)
k_apply_smem(const uint2 *__restrict__ pairs2, const uint32_t *__restrict__ fill2, uint32_t cap2,
             BucketGeom g, uint32_t sub_shift, uint32_t chunk0,
             unsigned long long *__restrict__ st, ClaimSink sink, Ctl *ctl) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t s_base;
    const uint32_t nv = 1u << sub_shift;
    uint32_t *deg = smem, *sum = smem + nv;
    const uint32_t S = 1u << (g.shift - sub_shift);
    const uint32_t s = blockIdx.x;
    const uint32_t c = chunk0 + s / S, b = s % S;  // chunk of the whole build
    const uint32_t part = c / g.chunks_per_part;
    const uint32_t base_v = part * g.P + (c % g.chunks_per_part) * (1u << g.shift) + b * nv;
    const uint32_t part_end = (part + 1) * g.P;
    if (base_v >= part_end) return;  // a sub-bucket past the end of its part
    for (uint32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        deg[k] = 0;
        sum[k] = 0;
    }
    __syncthreads();
    const uint32_t cnt = min(fill2[s], cap2);
    const uint2 *src = pairs2 + (size_t)s * cap2;
#ifndef HPEEL_APPLY_U
#define HPEEL_APPLY_U 4
#endif
    constexpr int kU = HPEEL_APPLY_U;  // loads in flight per thread
    for (uint32_t i0 = threadIdx.x; i0 < cnt; i0 += kU * blockDim.x) {
        uint2 p[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t i = i0 + (uint32_t)u * blockDim.x;
            p[u] = i < cnt ? __ldcs(src + i) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            if (i0 + (uint32_t)u * blockDim.x < cnt) {
                const uint32_t k = p[u].x - base_v;
                if (k < nv) {
                    atomicAdd(deg + k, 1u);
                    atomicAdd(sum + k, p[u].y);
                } else {
                    raise_err(ctl, kDevBadVertex);
                }
            }
        }
    }
    __syncthreads();
    const uint32_t lim = min(nv, part_end - base_v);
    for (uint32_t k = threadIdx.x; k < lim; k += blockDim.x)
        st[base_v + k] = (unsigned long long)deg[k] | ((unsigned long long)sum[k] << 32);
    if (!sink.claims) return;  // block-uniform
    // round 0's claims (sec. 4.2: F_0), one per vertex of degree 1: each
    // thread counts its own, one block-wide scan gives every thread its place
    // in the block's run, and the run is reserved with one atomic
    uint32_t mine = 0;
    for (uint32_t k = threadIdx.x; k < lim; k += blockDim.x) {
        if (deg[k] & kMark) raise_err(ctl, kDevDegree);
        if (deg[k] == 1u) {
            if (sum[k] < sink.n)
                mine++;
            else
                raise_err(ctl, kDevBadEdge);
        }
    }
    uint32_t total;
    uint32_t pos = block_scan_1024(mine, &total);
    if (threadIdx.x == 0) {
        const uint32_t q = total ? atomicAdd(&ctl->ccur, total) : 0u;
        if (total && (q + total > sink.cap || q + total < q)) raise_err(ctl, kDevRoundOverflow);
        s_base = q;
    }
    __syncthreads();
    pos += s_base;
    for (uint32_t k = threadIdx.x; k < lim; k += blockDim.x) {
        if (deg[k] == 1u && sum[k] < sink.n) {
            if (pos < sink.cap) sink.claims[pos] = make_uint2(sum[k], base_v + k);
            pos++;
        }
    }
}

// Incidences that found their bucket full, applied last with direct updates;
// with claims emitted by the apply, the list is complete only when there
// were none (ctl->cvalid).
__global__ void k_apply_overflow(const uint2 *__restrict__ list, const uint32_t *__restrict__ count,
                                 uint32_t cap, unsigned long long *__restrict__ st, Ctl *ctl,
                                 uint32_t emitted) {
    const uint32_t cnt = min(*count, cap);
    if (emitted && blockIdx.x == 0 && threadIdx.x == 0) ctl->cvalid = *count == 0 ? 1u : 0u;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const uint2 p = list[i];
        atomicAdd(st + p.x, ((unsigned long long)p.y << 32) | 1ull);
    }
}

BucketPlan bucket_plan(uint64_t n, uint64_t m, uint32_t r, uint32_t parts, uint32_t shift,
                       uint32_t sub_shift, int sms, uint32_t part_passes) {
    BucketPlan b{};
    // one part per pass: asked for (2), or automatic (0) above 2^30 edges;
    // a general graph has one part and always takes one pass
    const bool per_part = parts > 1 && (part_passes == 2 || (part_passes == 0 && n > (1ull << 30)));
    b.passes = per_part ? parts : 1;
    const uint64_t P = m / parts;
    b.shift = shift;
    b.chunks_per_part = (uint32_t)((P + (1ull << shift) - 1) >> shift);
    b.chunks = parts * b.chunks_per_part;
    b.chunks_pass = b.chunks / b.passes;
    // incidences per vertex of a part: one position per part when r-partite,
    // all r positions in the single part of a general graph
    const double per = (double)r / (double)parts;
    const uint64_t tiles = (n + kTileEdges - 1) / kTileEdges;
    // the record pass runs one resident wave; each chunk is one array
    b.blocks = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>(tiles, (uint64_t)sms * HPEEL_RB_MIN_BLOCKS));
    const double expect = P ? per * (double)n * (double)(1ull << shift) / (double)P : 0.0;
    uint64_t cap = (uint64_t)(expect + 8.0 * std::sqrt(expect + 1.0) + 64.0);
    b.cap = (uint32_t)std::min<uint64_t>(cap, per * (double)n + 64.0);
    b.pair_bytes = (uint64_t)b.chunks_pass * b.cap * 8;
    b.fill_words = (uint64_t)b.chunks_pass << kFillShift;
    // sub-buckets: 2^sub_shift vertices (default 2^13: 64 KiB of shared
    // memory for the apply's two 32-bit counters per vertex, 3 blocks per SM)
    b.sub_shift = sub_shift ? sub_shift : (shift > 9 ? shift - 9 : 0);
    if (b.sub_shift > 14) b.sub_shift = 14;
    if (!sub_shift && b.sub_shift > 13) b.sub_shift = 13;
    if (b.sub_shift > shift) b.sub_shift = shift;
    b.subs = b.chunks << (shift - b.sub_shift);
    b.subs_pass = b.subs / b.passes;
    const double expect2 = P ? per * (double)n * (double)(1ull << b.sub_shift) / (double)P : 0.0;
    uint64_t cap2 = (uint64_t)(expect2 + 8.0 * std::sqrt(expect2 + 1.0) + 256.0);
    b.cap2 = (uint32_t)std::min<uint64_t>(cap2, n);
    b.pair2_bytes = (uint64_t)b.subs_pass * b.cap2 * 8;
    b.ovf_cap = (uint32_t)std::max<uint64_t>(1u << 16, n / 16);
    b.smem = (size_t)(3 * ((b.chunks + 1) & ~1u)) * 4 + (size_t)kTileEdges * r * 8;
    // the refine indexes a chunk's sub-buckets with 32-bit arithmetic: a plan
    // beyond that asks for more shared memory than any block has, so the
    // caller builds without buckets
    if ((uint64_t)b.cap2 << (shift - b.sub_shift) >= (1ull << 32)) b.smem = ~(size_t)0;
    b.parts = parts;
    return b;
}

void launch_build_bucketed(const Launch &L, const BucketPlan &b, const uint64_t *keys,
                           const uint32_t *rows, uint32_t n, uint32_t r, FastMod fm,
                           uint64_t seed, uint32_t P, uint4 *rec, uint2 *pairs, uint32_t *fill,
                           Overflow ov, Ctl *ctl, bool gen, const uint64_t *seed_dev,
                           uint32_t pass) {
    if (n == 0) return;
    BucketGeom g{P, b.shift, b.chunks_per_part, b.cap, kFillShift};
    const unsigned grid = b.blocks;
    const int pass_part = b.passes > 1 ? (int)pass : -1;
    // the chunk cursors start at 0 every pass
    cudaMemsetAsync(fill, 0, 4 * b.fill_words, L.stream);
#define HP_BK(RR, FK)                                                                         \
    do {                                                                                      \
        auto kern = gen ? k_records_bucketed<RR, FK, true> : k_records_bucketed<RR, FK, false>; \
        smem_optin((const void *)kern);                                                      \
        count_launch();                                                                       \
        kern<<<grid, kRbThreads, b.smem, L.stream>>>(keys, rows, n, fm, seed, seed_dev, g, rec,\
                                                   pairs, fill, ov, ctl, pass_part);          \
    } while (0)
    if (keys) {
        switch (r) {
        case 2: HP_BK(2, true); break;
        case 3: HP_BK(3, true); break;
        case 4: HP_BK(4, true); break;
        }
    } else {
        switch (r) {
        case 2: HP_BK(2, false); break;
        case 3: HP_BK(3, false); break;
        case 4: HP_BK(4, false); break;
        }
    }
#undef HP_BK
}

void launch_refine(const Launch &L, const BucketGeom &g, uint32_t chunks, uint32_t chunk0,
                   uint32_t sub_shift, const uint2 *pairs, const uint32_t *fill,
                   uint2 *pairs2, uint32_t *fill2, uint32_t cap2, Overflow ov, Ctl *ctl) {
    const uint32_t S = 1u << (g.shift - sub_shift);
    const size_t smem1 = ((3 * (size_t)S + kRefWarps + chunks + 1 + 1) & ~(size_t)1) * 4 +
                         (size_t)kRefineTile * 8;
    smem_optin((const void *)k_refine_buckets);
    // items < 2^32: each holds up to 4096 of the pass's pairs, and the pair
    // storage of a pass is far below 2^44 pairs
    const uint64_t items = (uint64_t)chunks * ((g.cap + kRefineTile - 1) / kRefineTile);
    const unsigned grid = (unsigned)std::min<uint64_t>(
        std::max<uint64_t>(items, 1),
        grid_resident(L, (const void *)k_refine_buckets, 8, smem1, kRefThreads));
    count_launch();
    k_refine_buckets<<<grid, kRefThreads, smem1, L.stream>>>(pairs, fill, g, chunks, chunk0,
                                                            sub_shift, pairs2, fill2, cap2, ov,
                                                            ctl);
}

void launch_apply_buckets(const Launch &L, const BucketPlan &b, uint32_t P, const uint2 *pairs,
                          const uint32_t *fill, uint2 *pairs2, uint32_t *fill2, Overflow ov,
                          unsigned long long *st, Ctl *ctl, uint32_t pass, ClaimSink sink) {
    if (b.passes > 1) sink.claims = nullptr;  // claims need every part's degrees
    BucketGeom g{P, b.shift, b.chunks_per_part, b.cap, kFillShift};
    const uint32_t chunk0 = b.passes > 1 ? pass * b.chunks_per_part : 0u;
    launch_refine(L, g, b.chunks_pass, chunk0, b.sub_shift, pairs, fill, pairs2, fill2,
                  b.cap2, ov, ctl);
    const size_t smem2 = (size_t)8 << b.sub_shift;
    smem_optin((const void *)k_apply_smem);
    count_launch();
    k_apply_smem<<<b.subs_pass, 1024, smem2, L.stream>>>(pairs2, fill2, b.cap2, g, b.sub_shift,
                                                         chunk0, st, sink, ctl);
    count_launch();
    k_apply_overflow<<<grid_fixed(L, 4), kThreads, 0, L.stream>>>(ov.list, ov.count, ov.cap, st,
                                                                 ctl, sink.claims ? 1u : 0u);
}

}  // namespace hp
