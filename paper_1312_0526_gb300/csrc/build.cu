// build.cu -- L2-blocked incidence build (sec. 4.1 AddEdge for every edge).
//
// AddEdge hits the vertex records in random order: with the records far
// larger than L2, every update is a DRAM sector read and write.  Here the
// updates are first bucketed by vertex chunk -- the paper's own remedy for
// random access (sec. 4.2 builds E_0 by sorting the orientations by vertex,
// sec. 4.3 part by part), with the GPU's L2 as the fast memory -- and then
// applied chunk after chunk, so the records being updated stay in L2:
//   pass 1 (fused with hashing, or with the row -> record conversion): each
//          block takes a tile of edges, writes their records, counting-sorts
//          the tile's (vertex, edge) incidences by chunk in shared memory and
//          appends each chunk's run to that chunk's bucket;
//   pass 2: one kernel walks the buckets in chunk order and adds
//          (e << 32) + 1 to each vertex record (64-bit reductions, L2 hits).
// A chunk is 2^shift consecutive vertices of one part of the r-partite
// vertex set.  Bucket capacity covers the expected load of a chunk with a
// wide margin; an incidence that finds its bucket full is applied directly
// (same result, random access), so any input is handled.
#include <algorithm>
#include <cmath>

#include "kernels.cuh"

namespace hp {

constexpr int kTileEdges = 1024;  // edges per block step (4 per thread)

struct BucketGeom {
    uint32_t P;                // part size
    uint32_t shift;            // log2 of the vertices per chunk
    uint32_t chunks_per_part;
    uint32_t cap;              // bucket capacity (incidences)
};

__device__ __forceinline__ uint32_t chunk_of(uint32_t v, uint32_t j, const BucketGeom &g) {
    return j * g.chunks_per_part + ((v - j * g.P) >> g.shift);
}

template <int R, bool FROM_KEYS>
__global__ void __launch_bounds__(kThreads, 2)
k_records_bucketed(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ rows,
                   uint32_t n, FastMod fm, uint64_t seed, BucketGeom g, uint4 *__restrict__ rec,
                   uint2 *__restrict__ pairs, uint32_t *__restrict__ fill,
                   unsigned long long *__restrict__ st, Ctl *ctl) {
    constexpr int kInc = kTileEdges * R;
    extern __shared__ uint32_t smem[];
    const uint32_t C = R * g.chunks_per_part;
    const uint32_t Cp = (C + 1) & ~1u;
    uint32_t *hist = smem;            // C: tile count per chunk
    uint32_t *gbase = hist + Cp;      // C: bucket position of the tile's run
    uint32_t *toff = gbase + Cp;      // C: start of the chunk's run in stage
    uint32_t *sch = toff + Cp;        // kInc: chunk of each stage slot
    uint2 *stage = reinterpret_cast<uint2 *>(sch + kInc);  // kInc (8-byte aligned: Cp, kInc even)
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;

    const uint64_t tiles = ((uint64_t)n + kTileEdges - 1) / kTileEdges;
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        for (uint32_t c = threadIdx.x; c < C; c += kThreads) hist[c] = 0;
        __syncthreads();
        uint32_t vv[4][R], rank[4][R];
        bool inc[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint64_t e = tile * kTileEdges + (uint64_t)q * kThreads + threadIdx.x;
            uint32_t v[4] = {0, 0, 0, 0};
            bool ok = e < n;
            if (ok) {
                if (FROM_KEYS) {
                    const uint64_t k = __ldcs(keys + e);
#pragma unroll
                    for (int j = 0; j < R; j++)
                        v[j] = (uint32_t)fastmod(mix64(k ^ (seed + (uint64_t)j)), fm) +
                               (uint32_t)j * g.P;
                } else {
#pragma unroll
                    for (int j = 0; j < R; j++) {
                        v[j] = __ldcs(rows + e * R + j);
                        ok &= (v[j] - (uint32_t)j * g.P) < g.P;
                    }
                    if (!ok) raise_err(ctl, kDevBadVertex);
                }
                store_record<R>(rec, e, v, ok);
            }
            inc[q] = ok;  // an invalid row adds nothing (the call fails)
#pragma unroll
            for (int j = 0; j < R; j++) {
                vv[q][j] = v[j];
                rank[q][j] = ok ? atomicAdd(&hist[chunk_of(v[j], j, g)], 1u) : 0u;
            }
        }
        __syncthreads();
        // reserve each chunk's run in its bucket
        for (uint32_t c = threadIdx.x; c < C; c += kThreads)
            gbase[c] = hist[c] ? atomicAdd(fill + c, hist[c]) : 0u;
        // exclusive scan of hist -> toff (warp 0, 32 chunks per step)
        if (warp == 0) {
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
        for (int q = 0; q < 4; q++) {
            if (!inc[q]) continue;
            const uint32_t e = (uint32_t)(tile * kTileEdges + (uint64_t)q * kThreads + threadIdx.x);
#pragma unroll
            for (int j = 0; j < R; j++) {
                const uint32_t c = chunk_of(vv[q][j], j, g);
                const uint32_t slot = toff[c] + rank[q][j];
                stage[slot] = make_uint2(vv[q][j], e);
                sch[slot] = c;
            }
        }
        __syncthreads();
        // write the staged runs: consecutive slots -> consecutive addresses
        const uint32_t total = toff[C - 1] + hist[C - 1];
        for (uint32_t k = threadIdx.x; k < total; k += kThreads) {
            const uint32_t c = sch[k];
            const uint32_t pos = gbase[c] + (k - toff[c]);
            const uint2 p = stage[k];
            if (pos < g.cap)
                pairs[(uint64_t)c * g.cap + pos] = p;
            else  // bucket full: apply this incidence directly
                atomicAdd(st + p.x, ((unsigned long long)p.y << 32) | 1ull);
        }
        __syncthreads();
    }
}

// Apply the buckets in chunk order (every block walks chunk 0, then 1, ...):
// at any time the grid updates the records of about one chunk.
__global__ void __launch_bounds__(kThreads)
k_apply_buckets(const uint2 *__restrict__ pairs, const uint32_t *__restrict__ fill, uint32_t C,
                uint32_t cap, unsigned long long *__restrict__ st) {
    const uint32_t stride = gridDim.x * kThreads;
    for (uint32_t c = 0; c < C; c++) {
        const uint32_t cnt = min(fill[c], cap);
        const uint2 *b = pairs + (uint64_t)c * cap;
        for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < cnt; i += stride) {
            const uint2 p = __ldcs(b + i);
            atomicAdd(st + p.x, ((unsigned long long)p.y << 32) | 1ull);
        }
    }
}

BucketPlan bucket_plan(uint64_t n, uint64_t m, uint32_t r, uint32_t shift) {
    BucketPlan b{};
    const uint64_t P = m / r;
    b.shift = shift;
    b.chunks_per_part = (uint32_t)((P + (1ull << shift) - 1) >> shift);
    b.chunks = r * b.chunks_per_part;
    const double expect = P ? (double)n * (double)(1ull << shift) / (double)P : 0.0;
    uint64_t cap = (uint64_t)(expect + 16.0 * std::sqrt(expect + 1.0) + 1024.0);
    b.cap = (uint32_t)std::min<uint64_t>(cap, n);
    b.pair_bytes = (uint64_t)b.chunks * b.cap * 8;
    b.smem = (size_t)(3 * ((b.chunks + 1) & ~1u)) * 4 + (size_t)kTileEdges * r * (8 + 4);
    return b;
}

void launch_build_bucketed(const Launch &L, const BucketPlan &b, const uint64_t *keys,
                           const uint32_t *rows, uint32_t n, uint32_t r, FastMod fm,
                           uint64_t seed, uint32_t P, uint4 *rec, uint2 *pairs, uint32_t *fill,
                           unsigned long long *st, Ctl *ctl) {
    if (n == 0) return;
    BucketGeom g{P, b.shift, b.chunks_per_part, b.cap};
    const uint64_t tiles = ((uint64_t)n + kTileEdges - 1) / kTileEdges;
    const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)L.sms * 2);
#define HP_BK(RR, FK)                                                                         \
    do {                                                                                      \
        auto kern = k_records_bucketed<RR, FK>;                                               \
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem); \
        count_launch();                                                                       \
        kern<<<grid, kThreads, b.smem, L.stream>>>(keys, rows, n, fm, seed, g, rec, pairs,    \
                                                   fill, st, ctl);                            \
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
    count_launch();
    k_apply_buckets<<<grid_fixed(L, 8), kThreads, 0, L.stream>>>(pairs, fill, b.chunks, b.cap,
                                                                  st);
}

}  // namespace hp
