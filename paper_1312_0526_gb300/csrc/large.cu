// large.cu -- MWHC MPHF build for key sets beyond 32-bit ids (sec. 3, 4.2,
// 4.3; sec. 5 builds 7.6e9 keys).
//
// With n above 2^32 the edge ids and the vertex ids of m = gamma n vertices
// need more than 32 bits; a part of m/3 vertices still has 32-bit local ids
// (n up to about 1.05e10 at gamma = 1.23).  The state is kept compact so
// that the paper's largest instance fits one GPU:
//   keys           8 B per key (the caller's);
//   vertex records 8 B per vertex: degree in the low 24 bits, the sum of the
//                  ids of the incident edges modulo 2^40 above it (the label
//                  form of the XOR trick, sec. 4.1, with addition: at degree
//                  1 the sum is the last edge's id; AddEdge adds (e << 24) +
//                  1, DeleteEdge subtracts it);
//   claim words    4 B per edge: (round << 2) | hinge, all ones while
//                  unclaimed -- atomicMin keeps the smallest claiming
//                  position of the edge's round (the hinge);
//   layer list     8 B per peeled edge: the edge id and, in the top two bits,
//                  the position of its first claimer -- appended as the
//                  rounds find the layers (L_0 | L_1 | ...), read back as a
//                  stream; it may live in pinned host memory, where the
//                  kernels write and read it over the host link (the
//                  paper's layer lists live on disk);
//   g values       2 bits per vertex, rank directory 8 B per 512 vertices.
// No edge is stored: whenever an edge's vertices are needed (the rounds, the
// assignment) its key is read and hashed again.  The round that deletes an
// edge decrements every position but its first claimer's (that vertex has
// degree 1 and is never read again, whether or not it is the hinge), so no
// hinge correction is needed; the assignment reads the hinge from the claim
// word.
#include <algorithm>

#include "kernels.cuh"

namespace hp {

constexpr uint32_t kLDegBits = 24;
constexpr unsigned long long kLDegMask = (1ull << kLDegBits) - 1ull;
constexpr unsigned long long kLSumMask = (1ull << 40) - 1ull;
constexpr int kLPosShift = 62;
constexpr unsigned long long kLIdMask = (1ull << kLPosShift) - 1ull;

__device__ __forceinline__ unsigned long long lunit(uint64_t e) {
    return ((unsigned long long)e << kLDegBits) + 1ull;
}
__device__ __forceinline__ uint64_t lsum(unsigned long long r) { return (r >> kLDegBits) & kLSumMask; }

// Vertex j of a key: (mix64(k ^ (seed + j)) mod P) + j P, 64-bit.
__device__ __forceinline__ uint64_t lvertex(uint64_t k, uint64_t seed, int j, const FastMod &fm) {
    return fastmod(mix64(k ^ (seed + (uint64_t)j)), fm) + (uint64_t)j * fm.P;
}

// ----------------------------------------------------------------- build --
__global__ void __launch_bounds__(kThreads)
k_large_build(const uint64_t *__restrict__ keys, uint64_t n, uint64_t seed, FastMod fm,
              unsigned long long *__restrict__ st, uint32_t *__restrict__ claim, LargeCtl *ctl) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const uint64_t k = keys[e];
        claim[e] = kUnclaimed;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const unsigned long long old = atomicAdd(st + lvertex(k, seed, j, fm), lunit(e));
            if ((old & kLDegMask) >= kLDegMask - 1) atomicCAS(&ctl->err, 0u, (uint32_t)kDevDegree);
        }
    }
}

// -------------------------------------------------------------- appends --
// Per-warp staging of list appends (8 B entries): one 64-bit atomicAdd on
// the list cursor per buffer-full.
constexpr int kLStage = 512;

struct LStage {
    unsigned long long *buf;
    uint32_t cnt;
    __device__ __forceinline__ void flush(unsigned long long *cursor, unsigned long long *list) {
        __syncwarp();
        if (cnt == 0) return;
        const uint32_t lane = threadIdx.x & 31u;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)cnt);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (uint32_t i = lane; i < cnt; i += 32) list[base + i] = buf[i];
        cnt = 0;
        __syncwarp();
    }
    __device__ __forceinline__ void push(bool pred, unsigned long long v,
                                         unsigned long long *cursor, unsigned long long *list) {
        const uint32_t lane = threadIdx.x & 31u;
        const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, pred);
        if (ballot == 0) return;
        const uint32_t k = __popc(ballot);
        if (cnt + k > kLStage) flush(cursor, list);
        if (pred) buf[cnt + __popc(ballot & ((1u << lane) - 1u))] = v;
        cnt += k;
        __syncwarp();
    }
};

// Last block of a launch closes the round: layer t+1 is [loff[t+1], lcur).
__device__ __forceinline__ void large_close(LargeCtl *ctl, unsigned long long *loff, uint32_t t,
                                            bool first, uint64_t cross, uint32_t max_rounds,
                                            cudaGraphConditionalHandle cond) {
    __shared__ unsigned long long s_cross[kThreads / 32];
    unsigned long long wc = cross;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) wc += __shfl_down_sync(0xFFFFFFFFu, wc, d);
    if ((threadIdx.x & 31u) == 0) s_cross[threadIdx.x >> 5] = wc;
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned long long bc = 0;
    for (int w = 0; w < kThreads / 32; w++) bc += s_cross[w];
    if (bc) atomicAdd(&ctl->cross, bc);
    __threadfence();
    const uint32_t d = atomicAdd(&ctl->done, 1u);
    if (d != gridDim.x - 1) return;
    __threadfence();
    const unsigned long long end = atomicAdd(&ctl->lcur, 0ull);
    unsigned long long beg;
    uint32_t more;
    if (first) {
        loff[0] = 0;
        loff[1] = end;
        ctl->first_layer = end;
        beg = 0;
        more = end > 0 ? 1u : 0u;
        ctl->round = 0;
    } else {
        beg = loff[t + 1];
        loff[t + 2] = end;
        more = end > beg ? 1u : 0u;
        if (more && t + 2 >= max_rounds) {
            more = 0;
            atomicCAS(&ctl->err, 0u, (uint32_t)kDevCapacity);
        }
        ctl->round = t + 1;
    }
    if (atomicAdd(&ctl->err, 0u) != 0u) more = 0;
    ctl->more = more;
    ctl->done = 0;
    if (cond) cudaGraphSetConditional(cond, more);
}

// --------------------------------------------------------------- round 0 --
// Every vertex of degree 1 claims its edge; the first claimer lists it.
__global__ void __launch_bounds__(kThreads)
k_large_round0(const LargeParams *__restrict__ prm, cudaGraphConditionalHandle cond) {
    __shared__ unsigned long long sbuf[kThreads / 32][kLStage];
    LStage stage{sbuf[threadIdx.x >> 5], 0};
    const LargeParams p = *prm;
    const uint64_t P = p.fm.P;
    constexpr int kU = 4;
    const uint64_t step = (uint64_t)kThreads * kU;
    // whole warps iterate together (the trip count depends on blockIdx only)
    for (uint64_t base = (uint64_t)blockIdx.x * step; base < p.m; base += (uint64_t)gridDim.x * step) {
        unsigned long long r[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint64_t v = base + (uint64_t)u * kThreads + threadIdx.x;
            r[u] = v < p.m ? __ldcs(p.st + v) : 0ull;
        }
        uint32_t c[kU];
        bool one[kU];
        uint64_t e[kU];
        uint32_t j[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint64_t v = base + (uint64_t)u * kThreads + threadIdx.x;
            one[u] = v < p.m && (r[u] & kLDegMask) == 1ull;
            e[u] = lsum(r[u]);
            j[u] = (uint32_t)((v >= P) + (v >= 2 * P));
            if (one[u] && e[u] >= p.n) {
                atomicCAS(&p.ctl->err, 0u, (uint32_t)kDevBadEdge);
                one[u] = false;
            }
            c[u] = one[u] ? atomicMin(p.claim + e[u], j[u]) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kU; u++)
            stage.push(one[u] && c[u] == kUnclaimed,
                       (unsigned long long)e[u] | ((unsigned long long)j[u] << kLPosShift),
                       &p.ctl->lcur, p.L);
    }
    stage.flush(&p.ctl->lcur, p.L);
    large_close(p.ctl, p.loff, 0, true, 0, p.max_rounds, cond);
}

// ----------------------------------------------------------------- rounds --
// Round t: delete layer L_t (read as a stream) and claim layer L_{t+1}.
__global__ void __launch_bounds__(kThreads)
k_large_round(const LargeParams *__restrict__ prm, cudaGraphConditionalHandle cond) {
    __shared__ unsigned long long sbuf[kThreads / 32][kLStage];
    LStage stage{sbuf[threadIdx.x >> 5], 0};
    const LargeParams p = *prm;
    const uint32_t t = *(volatile uint32_t *)&p.ctl->round;
    uint64_t lb = p.loff[t], le = p.loff[t + 1];
    if (lb > le || le > p.n) {
        atomicCAS(&p.ctl->err, 0u, (uint32_t)kDevCapacity);
        lb = le;
    }
    constexpr int kU = 4;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t block_step = (uint64_t)kThreads * kU;
    uint64_t cross = 0;
    const uint32_t tag_hi = (t + 1) << 2;
    for (uint64_t base = lb + (uint64_t)blockIdx.x * block_step + (uint64_t)warp * 32 * kU; base < le;
         base += (uint64_t)gridDim.x * block_step) {
        uint64_t e[kU], k[kU];
        uint32_t jf[kU];
        bool mine[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint64_t i = base + (uint64_t)u * 32 + lane;
            mine[u] = i < le;
            const unsigned long long x = mine[u] ? __ldcs(p.L + i) : 0ull;
            e[u] = x & kLIdMask;
            jf[u] = (uint32_t)(x >> kLPosShift);
            if (mine[u] && e[u] >= p.n) {
                atomicCAS(&p.ctl->err, 0u, (uint32_t)kDevBadEdge);
                mine[u] = false;
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) k[u] = mine[u] ? __ldg(p.keys + e[u]) : 0ull;
        // DeleteEdge on the two positions other than the first claimer's
        unsigned long long old[kU][2];
        uint64_t w[kU][2];
        uint32_t pos[kU][2];
#pragma unroll
        for (int u = 0; u < kU; u++) {
#pragma unroll
            for (int q = 0; q < 2; q++) {
                pos[u][q] = (uint32_t)q + ((uint32_t)q >= jf[u] ? 1u : 0u);
                w[u][q] = lvertex(k[u], p.seed, (int)pos[u][q], p.fm);
                old[u][q] = mine[u] ? atomicAdd(p.st + w[u][q], 0ull - lunit(e[u])) : 0ull;
            }
        }
        bool take[kU][2];
        uint64_t g[kU][2];
#pragma unroll
        for (int u = 0; u < kU; u++) {
#pragma unroll
            for (int q = 0; q < 2; q++) {
                take[u][q] = false;
                g[u][q] = 0;
                if (mine[u] && (old[u][q] & kLDegMask) == 2ull) {
                    cross++;
                    const uint64_t gg = (lsum(old[u][q]) - e[u]) & kLSumMask;
                    if (gg < p.n) {
                        take[u][q] =
                            atomicMin(p.claim + gg, tag_hi | pos[u][q]) == kUnclaimed;
                        g[u][q] = gg;
                    } else {
                        atomicCAS(&p.ctl->err, 0u, (uint32_t)kDevBadEdge);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++)
#pragma unroll
            for (int q = 0; q < 2; q++)
                stage.push(take[u][q],
                           (unsigned long long)g[u][q] |
                               ((unsigned long long)pos[u][q] << kLPosShift),
                           &p.ctl->lcur, p.L);
    }
    stage.flush(&p.ctl->lcur, p.L);
    large_close(p.ctl, p.loff, t, false, cross, p.max_rounds, cond);
}

RoundLaunch large_round_launch(const Launch &L, bool first) {
    RoundLaunch k{};
    k.fn = first ? (void *)k_large_round0 : (void *)k_large_round;
    k.block = kThreads;
    k.smem = 0;
    k.grid = grid_resident(L, k.fn, 4, 0);
    return k;
}

__global__ void k_large_set_params(LargeParams *dst, LargeParams v) { *dst = v; }

void launch_large_set_params(const Launch &L, LargeParams *dst, const LargeParams &v) {
    count_launch();
    k_large_set_params<<<1, 1, 0, L.stream>>>(dst, v);
}

void launch_large_build(const Launch &L, const uint64_t *keys, uint64_t n, uint64_t seed,
                        FastMod fm, unsigned long long *st, uint32_t *claim, LargeCtl *ctl) {
    if (n == 0) return;
    count_launch();
    k_large_build<<<grid_fixed(L, 8), kThreads, 0, L.stream>>>(keys, n, seed, fm, st, claim, ctl);
}

// ----------------------------------------------------------- assignment --
// MWHC g values of layer t (sec. 3; sec. 4.3 layers last to first): for each
// edge of the layer, the hinge h from its claim word, s = the g values of
// the other two vertices, and g[v_h] = (h - s) mod 3 (stored as 3 for 0).
__global__ void __launch_bounds__(kThreads)
k_large_assign(const LargeParams *__restrict__ prm, uint32_t t, uint64_t *G) {
    const LargeParams p = *prm;
    const uint64_t lb = p.loff[t], le = p.loff[t + 1];
    constexpr int kU = 4;
    const uint64_t stride = (uint64_t)gridDim.x * kThreads * kU;
    for (uint64_t i0 = lb + (uint64_t)blockIdx.x * kThreads * kU + threadIdx.x; i0 < le; i0 += stride) {
        uint64_t e[kU], k[kU];
        uint32_t c[kU];
        bool ok[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint64_t i = i0 + (uint64_t)u * kThreads;
            ok[u] = i < le;
            e[u] = ok[u] ? (__ldcs(p.L + i) & kLIdMask) : 0ull;
            ok[u] = ok[u] && e[u] < p.n;
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            k[u] = ok[u] ? __ldg(p.keys + e[u]) : 0ull;
            c[u] = ok[u] ? __ldcg(p.claim + e[u]) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            if (!ok[u]) continue;
            const uint32_t h = c[u] & 3u;
            uint64_t v[3];
            uint32_t s = 0;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                v[j] = lvertex(k[u], p.seed, j, p.fm);
                if ((uint32_t)j != h)
                    s += (uint32_t)(__ldcg(G + (v[j] >> 5)) >> (2u * (uint32_t)(v[j] & 31u))) & 3u;
            }
            const uint32_t val = (h + 6u - s) % 3u;
            const uint64_t vh = h == 0 ? v[0] : (h == 1 ? v[1] : v[2]);
            atomicOr((unsigned long long *)(G + (vh >> 5)),
                     (unsigned long long)(val ? val : 3u) << (2u * (uint32_t)(vh & 31u)));
        }
    }
}

void launch_large_assign(const Launch &L, const LargeParams *prm, uint32_t t, uint64_t *G) {
    count_launch();
    k_large_assign<<<grid_fixed(L, 8), kThreads, 0, L.stream>>>(prm, t, G);
}

// ------------------------------------------------------------------- rank --
// dir[b] = non-zero 2-bit values among vertices [0, 512 b), as 64-bit counts:
// per-block counts (uint32), then a scan of 64-bit partial sums.
__device__ __forceinline__ uint32_t nz_pairs(uint64_t w) {
    return (uint32_t)__popcll((w | (w >> 1)) & 0x5555555555555555ull);
}

__global__ void k_large_rank_counts(const uint64_t *__restrict__ G, uint64_t words, uint64_t blocks,
                                    uint32_t *__restrict__ cnt) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < blocks; b += stride) {
        uint32_t c = 0;
        for (uint64_t w = b * 16; w < words && w < b * 16 + 16; w++) c += nz_pairs(G[w]);
        cnt[b] = c;
    }
}

// Segments of kRankSeg blocks: segment sums, their exclusive scan (one
// thread: few segments), then every block's prefix inside its segment.
constexpr uint64_t kRankSeg = 4096;

__global__ void k_large_rank_segsum(const uint32_t *__restrict__ cnt, uint64_t blocks,
                                    unsigned long long *__restrict__ seg) {
    const uint64_t nseg = (blocks + kRankSeg - 1) / kRankSeg;
    for (uint64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        unsigned long long acc = 0;
        for (uint64_t b = s * kRankSeg + threadIdx.x; b < blocks && b < (s + 1) * kRankSeg;
             b += blockDim.x)
            acc += cnt[b];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, d);
        __shared__ unsigned long long ws[32];
        if ((threadIdx.x & 31u) == 0) ws[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (uint32_t w = 0; w < blockDim.x / 32; w++) t += ws[w];
            seg[s] = t;
        }
        __syncthreads();
    }
}

__global__ void k_large_rank_segscan(unsigned long long *seg, uint64_t nseg) {
    unsigned long long run = 0;
    for (uint64_t s = 0; s < nseg; s++) {
        const unsigned long long c = seg[s];
        seg[s] = run;
        run += c;
    }
    seg[nseg] = run;
}

__global__ void k_large_rank_dir(const uint32_t *__restrict__ cnt, uint64_t blocks,
                                 const unsigned long long *__restrict__ seg, uint64_t *__restrict__ dir) {
    // one warp per segment, sequential over its blocks in chunks of 32
    const uint64_t nseg = (blocks + kRankSeg - 1) / kRankSeg;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t s = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); s < nseg;
         s += warps) {
        unsigned long long run = seg[s];
        for (uint64_t b0 = s * kRankSeg; b0 < blocks && b0 < (s + 1) * kRankSeg; b0 += 32) {
            const uint64_t b = b0 + lane;
            const uint32_t c = b < blocks ? cnt[b] : 0u;
            uint32_t x = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
                if (lane >= (uint32_t)d) x += y;
            }
            if (b < blocks) dir[b] = run + x - c;
            run += __shfl_sync(0xFFFFFFFFu, x, 31);
        }
        if (lane == 0 && s == nseg - 1) dir[blocks] = run;
    }
}

void launch_large_rank(const Launch &L, const uint64_t *G, uint64_t m, uint32_t *cnt,
                       unsigned long long *seg, uint64_t *dir) {
    const uint64_t words = (m + 31) / 32, blocks = (m + 511) / 512;
    if (blocks == 0) {
        cudaMemsetAsync(dir, 0, 8, L.stream);
        return;
    }
    const uint64_t nseg = (blocks + kRankSeg - 1) / kRankSeg;
    count_launch(4);
    k_large_rank_counts<<<grid_for(L, blocks, 1, 8), kThreads, 0, L.stream>>>(G, words, blocks, cnt);
    k_large_rank_segsum<<<(unsigned)std::min<uint64_t>(nseg, 65535), kThreads, 0, L.stream>>>(
        cnt, blocks, seg);
    k_large_rank_segscan<<<1, 1, 0, L.stream>>>(seg, nseg);
    k_large_rank_dir<<<grid_for(L, nseg * 32, 1, 8), kThreads, 0, L.stream>>>(cnt, blocks, seg,
                                                                              dir);
}

// ----------------------------------------------------------------- lookup --
__global__ void __launch_bounds__(kThreads)
k_large_lookup(const uint64_t *__restrict__ keys, uint64_t nq, FastMod fm, uint64_t seed,
               const uint64_t *__restrict__ G, const uint64_t *__restrict__ dir,
               uint64_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t q = (uint64_t)blockIdx.x * kThreads + threadIdx.x; q < nq; q += stride) {
        const uint64_t k = __ldcs(keys + q);
        uint64_t v[3];
        uint32_t g = 0;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            v[j] = lvertex(k, seed, j, fm);
            g += (uint32_t)(__ldg(G + (v[j] >> 5)) >> (2u * (uint32_t)(v[j] & 31u))) & 3u;
        }
        const uint32_t i = g % 3u;
        const uint64_t x = i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
        const uint64_t blk = x >> 9, w_end = x >> 5;
        uint64_t rank = __ldg(dir + blk);
        for (uint64_t w = blk << 4; w < w_end; w++) rank += nz_pairs(__ldg(G + w));
        const uint32_t sh = 2u * (uint32_t)(x & 31u);
        if (sh) rank += nz_pairs(__ldg(G + w_end) & ((1ull << sh) - 1ull));
        out[q] = rank;
    }
}

void launch_large_lookup(const Launch &L, const uint64_t *keys, uint64_t nq, FastMod fm,
                         uint64_t seed, const uint64_t *G, const uint64_t *dir, uint64_t *out) {
    if (nq == 0) return;
    count_launch();
    k_large_lookup<<<grid_for(L, nq, 1, 8), kThreads, 0, L.stream>>>(keys, nq, fm, seed, G, dir,
                                                                     out);
}

}  // namespace hp
