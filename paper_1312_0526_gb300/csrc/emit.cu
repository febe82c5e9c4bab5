// emit.cu -- canonical peeling order: a stable counting sort of edge ids by
// the round in their claim word, layers in round order and ascending id
// inside a layer (sec. 4.2 leaves the intra-layer order free; ascending id
// makes it unique), then the 2-core edges ascending.
//
// One pass sorts by up to kEmitBins keys: key k of an edge (round, or
// core_key for an unclaimed edge) goes to bin min(k - base, nbins - 1).
// Further passes sort the last bin again when there are more rounds; the
// host decides on them, or, for a graph that never returns to the host, the
// device (the *_dev kernels at the end of this file).
//   hist    -- per tile of kEmitTile consecutive inputs, bin counts, stored
//              bin-major: hist[b * tiles + tile] (the first pass's counts
//              are taken while the claims are extracted from the records);
//   scan    -- one exclusive prefix sum over hist gives, for every (bin,
//              tile), where that tile's edges of that bin start;
//   scatter -- each warp ranks its 512 inputs in input order (the lanes
//              holding the same bin, found with one ballot per bit of the
//              bin, plus per-warp running counts), so equal keys keep the
//              input order: the sort is stable.  The tile's inputs are
//              staged in shared memory in (bin, input) order, so each bin's
//              run of the tile leaves as one contiguous, coalesced stretch.
#include "kernels.cuh"

namespace hp {

__device__ __forceinline__ uint32_t emit_bin(uint32_t c, uint32_t base, uint32_t core_key,
                                             uint32_t nbins) {
    const uint32_t k = (c == kUnclaimed) ? core_key : (c >> 2);
    const uint32_t d = k - base;  // k >= base for every input of the pass
    return d < nbins - 1 ? d : nbins - 1;
}

// Lanes of the warp holding the same bin (valid lanes only): one ballot per
// bit of the bin index, for a bin below 2^PLANES, instead of a match.  More
// planes than the bins need give the same mask (the extra bits are 0 in
// every lane).
template <int PLANES, bool FULL>
__device__ __forceinline__ uint32_t bin_peers(uint32_t bin, bool valid) {
    uint32_t m = FULL ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
    for (int b = 0; b < PLANES; b++) {
        const bool bit = (bin >> b) & 1u;
        const uint32_t x = __ballot_sync(0xFFFFFFFFu, bit);
        m &= bit ? x : ~x;
    }
    return FULL || valid ? m : 0u;
}

__device__ __forceinline__ void emit_hist(const uint32_t *__restrict__ src, uint32_t count,
                                          const uint32_t *__restrict__ claim, uint32_t base,
                                          uint32_t core_key, uint32_t nbins,
                                          uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kEmitBins];
    const uint32_t tiles = (count + kEmitTile - 1) / kEmitTile;
    for (uint32_t b = threadIdx.x; b < nbins; b += kThreads) h[b] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * kEmitTile;
#pragma unroll 4
    for (uint32_t q = 0; q < kEmitItems; q++) {
        const uint64_t i = t0 + (uint64_t)q * kThreads + threadIdx.x;
        if (i < count) {
            const uint32_t e = src ? src[i] : (uint32_t)i;
            atomicAdd(&h[emit_bin(claim[e], base, core_key, nbins)], 1u);
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nbins; b += kThreads)
        hist[(uint64_t)b * tiles + blockIdx.x] = h[b];
}

__global__ void __launch_bounds__(kThreads)
k_emit_hist(const uint32_t *__restrict__ src, uint32_t count, const uint32_t *__restrict__ claim,
            uint32_t base, uint32_t core_key, uint32_t nbins, uint32_t *__restrict__ hist) {
    emit_hist(src, count, claim, base, core_key, nbins, hist);
}

// The first pass's histogram taken while the claims are extracted from the
// edge records (one block per tile of kEmitTile consecutive edges): the
// claim array is written once and not read back for the counts.
template <int R>
__device__ __forceinline__ void extract_claim_hist(const uint4 *__restrict__ rec, uint32_t n,
                                                   uint32_t *__restrict__ claim,
                                                   uint32_t core_key, uint32_t nbins,
                                                   uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kEmitBins];
    const uint32_t tiles = (n + kEmitTile - 1) / kEmitTile;
    for (uint32_t b = threadIdx.x; b < nbins; b += kThreads) h[b] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * kEmitTile;
    uint32_t c[kEmitItems];
#pragma unroll
    for (uint32_t q = 0; q < kEmitItems; q++) {
        const uint64_t e = t0 + (uint64_t)q * kThreads + threadIdx.x;
        uint32_t v[4];
        c[q] = e < n ? load_record_stream<R>(rec, e, v) : 0u;
    }
#pragma unroll
    for (uint32_t q = 0; q < kEmitItems; q++) {
        const uint64_t e = t0 + (uint64_t)q * kThreads + threadIdx.x;
        if (e < n) {
            claim[e] = c[q];
            atomicAdd(&h[emit_bin(c[q], 0u, core_key, nbins)], 1u);
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nbins; b += kThreads)
        hist[(uint64_t)b * tiles + blockIdx.x] = h[b];
}

template <int R>
__global__ void __launch_bounds__(kThreads)
k_extract_claim_hist(const uint4 *__restrict__ rec, uint32_t n, uint32_t *__restrict__ claim,
                     uint32_t core_key, uint32_t nbins, uint32_t *__restrict__ hist) {
    extract_claim_hist<R>(rec, n, claim, core_key, nbins, hist);
}

void launch_extract_claim_hist(const Launch &L, const uint4 *rec, uint32_t n, uint32_t r,
                               uint32_t *claim, uint32_t core_key, uint32_t nbins,
                               uint32_t *hist) {
    if (n == 0) return;
    const uint32_t tiles = (n + kEmitTile - 1) / kEmitTile;
    count_launch();
    switch (r) {
    case 2: k_extract_claim_hist<2><<<tiles, kThreads, 0, L.stream>>>(rec, n, claim, core_key, nbins, hist); break;
    case 3: k_extract_claim_hist<3><<<tiles, kThreads, 0, L.stream>>>(rec, n, claim, core_key, nbins, hist); break;
    case 4: k_extract_claim_hist<4><<<tiles, kThreads, 0, L.stream>>>(rec, n, claim, core_key, nbins, hist); break;
    }
}

void launch_emit_hist(const Launch &L, const uint32_t *src, uint32_t count, const uint32_t *claim,
                      uint32_t base, uint32_t core_key, uint32_t nbins, uint32_t *hist) {
    if (count == 0) return;
    const uint32_t tiles = (count + kEmitTile - 1) / kEmitTile;
    count_launch();
    k_emit_hist<<<tiles, kThreads, 0, L.stream>>>(src, count, claim, base, core_key, nbins, hist);
}

#ifndef HPEEL_SCATTER_MIN_BLOCKS
#define HPEEL_SCATTER_MIN_BLOCKS 6
#endif
struct ScatterSmem {
    uint32_t wc[kEmitWarps][kEmitBins];  // per warp and bin: count, then first slot
    uint32_t obase[kEmitBins];           // output index of tile slot 0 of the bin
    uint32_t stage[kEmitTile];           // (bin << 16) | tile index, ordered by bin
};
static_assert(kEmitTile <= 65536u && kEmitBins <= 65536u, "stage word packs bin and index");

// One tile: each warp ranks its 512 inputs in input order.  The count pass
// gives every input its rank among the warp's inputs of its bin (the warp's
// running count of the bin before its group of 32, plus the peers in lower
// lanes); after the scan the input goes to its bin's first slot for the
// warp plus that rank, so equal keys keep the input order.  FULL: the tile
// holds kEmitTile inputs (every tile but the last).
template <int PLANES, bool SRC, bool FULL>
__device__ __forceinline__ void emit_scatter_t(ScatterSmem &sm, const uint32_t *__restrict__ src,
                                               uint32_t count, const uint32_t *__restrict__ claim,
                                               uint32_t base, uint32_t core_key, uint32_t nbins,
                                               const uint32_t *__restrict__ offs,
                                               uint32_t *__restrict__ out) {
    const uint32_t tiles = (count + kEmitTile - 1) / kEmitTile;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    // bins past nbins hold no input: the counts and the scan stop at the
    // first multiple of 32 at or above nbins
    const uint32_t nb32 = (nbins + 31u) & ~31u;
    uint32_t *wc = sm.wc[warp];
    for (uint32_t b = lane; b < nb32; b += 32) wc[b] = 0;
    __syncwarp();
    // this warp's contiguous run of the tile, kEmitItems groups of 32
    const uint64_t t0 = (uint64_t)blockIdx.x * kEmitTile;
    const uint32_t w0 = warp * 32u * kEmitItems;  // index in the tile
    // br[g]: the input's bin, then (bin << 16) | rank; ~0 past the end
    uint32_t br[kEmitItems];
#pragma unroll
    for (int g = 0; g < kEmitItems; g++) {
        const uint64_t i = t0 + w0 + (uint32_t)g * 32u + lane;
        const bool valid = FULL || i < count;
        const uint32_t e = valid ? (SRC ? src[i] : (uint32_t)i) : 0u;
        br[g] = valid ? emit_bin(claim[e], base, core_key, nbins) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int g = 0; g < kEmitItems; g++) {
        const uint32_t bin = br[g];
        const bool valid = bin != 0xFFFFFFFFu;
        const uint32_t peers = bin_peers<PLANES, FULL>(valid ? bin : 0u, valid);
        const uint32_t below = __popc(peers & lt);
        const uint32_t before = valid ? wc[bin] : 0u;
        if (valid) br[g] = (bin << 16) | (before + below);  // rank < 512
        __syncwarp();
        // the lowest lane of each bin moves the bin's running count
        if (valid && below == 0u) wc[bin] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // bin totals of the tile -> first stage slot of each bin (warp 0 scans),
    // then each warp's first slot in each bin (earlier warps first: stable)
    if (warp == 0) {
        uint32_t run = 0;
        for (uint32_t b0 = 0; b0 < nb32; b0 += 32) {
            const uint32_t b = b0 + lane;
            uint32_t tot = 0;
#pragma unroll
            for (int w = 0; w < kEmitWarps; w++) {
                const uint32_t c = sm.wc[w][b];
                sm.wc[w][b] = tot;  // exclusive over warps, relative to the bin start
                tot += c;
            }
            uint32_t x = tot;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
                if (lane >= (uint32_t)d) x += y;
            }
            const uint32_t start = run + x - tot;
#pragma unroll
            for (int w = 0; w < kEmitWarps; w++) sm.wc[w][b] += start;
            sm.obase[b] = b < nbins ? offs[(uint64_t)b * tiles + blockIdx.x] - start : 0u;
            run += __shfl_sync(0xFFFFFFFFu, x, 31);
        }
    }
    __syncthreads();
    // stage the inputs in bin order, input order inside a bin
#pragma unroll
    for (int g = 0; g < kEmitItems; g++)
        if (br[g] != 0xFFFFFFFFu)
            sm.stage[wc[br[g] >> 16] + (br[g] & 0xFFFFu)] =
                (br[g] & 0xFFFF0000u) | (w0 + (uint32_t)g * 32u + lane);
    __syncthreads();
    // each bin's run of the tile is one contiguous stretch of the output:
    // consecutive threads write consecutive addresses
    const uint64_t left = (uint64_t)count - t0;
    const uint32_t tn = left < kEmitTile ? (uint32_t)left : kEmitTile;
#pragma unroll 4
    for (int q = 0; q < kEmitItems; q++) {
        const uint32_t k = (uint32_t)q * kThreads + threadIdx.x;
        if (FULL || k < tn) {
            const uint32_t s = sm.stage[k];
            const uint64_t i = t0 + (s & 0xFFFFu);
            out[sm.obase[s >> 16] + k] = SRC ? src[i] : (uint32_t)i;
        }
    }
}

// Ballot planes for the pass's bins (2, 4, 6, 7 or 8), whether the inputs
// are edge ids read from src or the tile's own indices, and whether the
// tile is full.
template <bool SRC, bool FULL>
__device__ __forceinline__ void emit_scatter_src(ScatterSmem &sm, const uint32_t *src,
                                                 uint32_t count, const uint32_t *claim,
                                                 uint32_t base, uint32_t core_key, uint32_t nbins,
                                                 const uint32_t *offs, uint32_t *out) {
    if (nbins <= 4)
        emit_scatter_t<2, SRC, FULL>(sm, src, count, claim, base, core_key, nbins, offs, out);
    else if (nbins <= 16)
        emit_scatter_t<4, SRC, FULL>(sm, src, count, claim, base, core_key, nbins, offs, out);
    else if (nbins <= 64)
        emit_scatter_t<6, SRC, FULL>(sm, src, count, claim, base, core_key, nbins, offs, out);
    else if (nbins <= 128)
        emit_scatter_t<7, SRC, FULL>(sm, src, count, claim, base, core_key, nbins, offs, out);
    else
        emit_scatter_t<8, SRC, FULL>(sm, src, count, claim, base, core_key, nbins, offs, out);
}

__device__ __forceinline__ void emit_scatter(const uint32_t *__restrict__ src, uint32_t count,
                                             const uint32_t *__restrict__ claim, uint32_t base,
                                             uint32_t core_key, uint32_t nbins,
                                             const uint32_t *__restrict__ offs,
                                             uint32_t *__restrict__ out) {
    __shared__ ScatterSmem sm;
    const bool full = (uint64_t)(blockIdx.x + 1) * kEmitTile <= count;
    if (src) {
        if (full)
            emit_scatter_src<true, true>(sm, src, count, claim, base, core_key, nbins, offs, out);
        else
            emit_scatter_src<true, false>(sm, src, count, claim, base, core_key, nbins, offs, out);
    } else {
        if (full)
            emit_scatter_src<false, true>(sm, src, count, claim, base, core_key, nbins, offs, out);
        else
            emit_scatter_src<false, false>(sm, src, count, claim, base, core_key, nbins, offs,
                                           out);
    }
}

__global__ void __launch_bounds__(kThreads, HPEEL_SCATTER_MIN_BLOCKS)
k_emit_scatter(const uint32_t *__restrict__ src, uint32_t count,
               const uint32_t *__restrict__ claim, uint32_t base, uint32_t core_key,
               uint32_t nbins, const uint32_t *__restrict__ offs, uint32_t *__restrict__ out) {
    emit_scatter(src, count, claim, base, core_key, nbins, offs, out);
}

void launch_emit_scatter(const Launch &L, const uint32_t *src, uint32_t count,
                         const uint32_t *claim, uint32_t base, uint32_t core_key, uint32_t nbins,
                         const uint32_t *offs, uint32_t *out) {
    if (count == 0) return;
    const uint32_t tiles = (count + kEmitTile - 1) / kEmitTile;
    count_launch();
    k_emit_scatter<<<tiles, kThreads, 0, L.stream>>>(src, count, claim, base, core_key, nbins,
                                                     offs, out);
}

__global__ void k_layer_off(const uint32_t *__restrict__ loff, uint32_t rounds,
                            uint64_t *__restrict__ out) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= rounds;
         t += gridDim.x * blockDim.x)
        out[t] = loff[t];
}

void launch_layer_off(const Launch &L, const uint32_t *loff, uint32_t rounds, uint64_t *out) {
    count_launch();
    k_layer_off<<<grid_for(L, (uint64_t)rounds + 1, 1, 4), kThreads, 0, L.stream>>>(loff, rounds,
                                                                                   out);
}

// ------------------------------------------------------------------ scan --
// Exclusive prefix sum, reduce-then-scan: level sums of 4096-element blocks
// are scanned recursively, then each block rescans its elements.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint64_t kScanBlock = (uint64_t)kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t ws[kScanThreads / 32];
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
        uint32_t s = ws[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, d);
            if (lane >= (uint32_t)d) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    const uint32_t before = (warp ? ws[warp - 1] : 0u) + x - v;
    if (total) *total = ws[kScanThreads / 32 - 1];
    __syncthreads();
    return before;
}

__device__ __forceinline__ void scan_reduce_block(const uint32_t *__restrict__ in, uint64_t count,
                                                  uint32_t *__restrict__ sums) {
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (b0 + k < count) s += in[b0 + k];
    uint32_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t *__restrict__ in, uint64_t count, uint32_t *__restrict__ sums) {
    scan_reduce_block(in, count, sums);
}

__device__ __forceinline__ void scan_down_block(const uint32_t *in, uint32_t *out, uint64_t count,
                                                const uint32_t *__restrict__ offs) {
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = (b0 + k < count) ? in[b0 + k] : 0u;
        s += v[k];
    }
    uint32_t run = block_excl_scan(s, nullptr) + (offs ? offs[blockIdx.x] : 0u);
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (b0 + k < count) out[b0 + k] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_down(const uint32_t *in, uint32_t *out, uint64_t count, const uint32_t *__restrict__ offs) {
    scan_down_block(in, out, count, offs);
}

size_t scan_tmp_words(uint64_t count) {
    size_t words = 0;
    while (count > kScanBlock) {
        count = (count + kScanBlock - 1) / kScanBlock;
        words += count;
    }
    return words + 1;
}

void launch_scan_u32(const Launch &L, const uint32_t *in, uint32_t *out, uint64_t count,
                     uint32_t *tmp) {
    if (count == 0) return;
    if (count <= kScanBlock) {
        count_launch();
        k_scan_down<<<1, kScanThreads, 0, L.stream>>>(in, out, count, nullptr);
        return;
    }
    const uint64_t blocks = (count + kScanBlock - 1) / kScanBlock;
    uint32_t *sums = tmp;
    count_launch();
    k_scan_reduce<<<(unsigned)blocks, kScanThreads, 0, L.stream>>>(in, count, sums);
    launch_scan_u32(L, sums, sums, blocks, tmp + blocks);
    count_launch();
    k_scan_down<<<(unsigned)blocks, kScanThreads, 0, L.stream>>>(in, out, count, sums);
}

}  // namespace hp

// ------------------------------------------------- device-driven passes --
// The same passes with their parameters in an EmitState in device memory,
// for a CUDA graph that runs them as the body of a while node: the number
// of rounds (and so of passes) is never read back to the host.  Every kernel
// is launched with the grid of the largest pass (the first, over all n
// edges); blocks past the current pass's tiles return at once.
namespace hp {

__global__ void k_emit_init(const Ctl *__restrict__ ctl, uint32_t n, EmitState *es,
                            cudaGraphConditionalHandle h) {
    EmitState e;
    e.n = n;
    e.R = ctl->more ? ctl->round + 1 : ctl->round;
    e.nkeys = e.R + 1;
    e.base = 0;
    e.seg = 0;
    e.count = n;
    e.nb = e.nkeys < kEmitBins ? e.nkeys : kEmitBins;
    e.more = 1;
    *es = e;
    cudaGraphSetConditional(h, 1u);
}

template <int R>
__global__ void __launch_bounds__(kThreads)
k_extract_claim_hist_dev(const uint4 *__restrict__ rec, uint32_t n, uint32_t *__restrict__ claim,
                         const EmitState *__restrict__ es, uint32_t *__restrict__ hist) {
    extract_claim_hist<R>(rec, n, claim, es->R, es->nb, hist);
}

// the histogram of a later pass (the first pass's comes with the claims)
__global__ void __launch_bounds__(kThreads)
k_emit_hist_dev(const uint32_t *__restrict__ tail, const uint32_t *__restrict__ claim,
                const EmitState *__restrict__ es, uint32_t *__restrict__ hist) {
    const EmitState e = *es;
    if (e.base == 0 || blockIdx.x >= (e.count + kEmitTile - 1) / kEmitTile) return;
    emit_hist(tail + e.seg, e.count, claim, e.base, e.R, e.nb, hist);
}

__global__ void __launch_bounds__(kThreads, HPEEL_SCATTER_MIN_BLOCKS)
k_emit_scatter_dev(const uint32_t *__restrict__ tail, const uint32_t *__restrict__ claim,
                   const EmitState *__restrict__ es, const uint32_t *__restrict__ offs,
                   uint32_t *__restrict__ order) {
    const EmitState e = *es;
    if (blockIdx.x >= (e.count + kEmitTile - 1) / kEmitTile) return;
    emit_scatter(e.base ? tail + e.seg : nullptr, e.count, claim, e.base, e.R, e.nb, offs,
                 order + e.seg);
}

// After a pass: stop, or move to the last bin's keys (they start at the
// layer offset of their first round).
__global__ void k_emit_advance(EmitState *es, const uint32_t *__restrict__ loff,
                               cudaGraphConditionalHandle h) {
    EmitState e = *es;
    if (e.nkeys - e.base <= kEmitBins) {
        es->more = 0;
        cudaGraphSetConditional(h, 0u);
        return;
    }
    e.base += e.nb - 1;
    e.seg = loff[e.base];
    e.count = e.n - e.seg;
    e.nb = e.nkeys - e.base < kEmitBins ? e.nkeys - e.base : kEmitBins;
    e.more = 1;
    *es = e;
    cudaGraphSetConditional(h, 1u);
}

// The next pass reads its inputs from a copy of the order's tail.
__global__ void k_emit_copy_tail(const uint32_t *__restrict__ order, uint32_t *__restrict__ tail,
                                 const EmitState *__restrict__ es) {
    const EmitState e = *es;
    if (!e.more) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = e.seg + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < e.n; i += stride)
        tail[i] = order[i];
}

// Scan of the pass's histogram: count = nb x tiles, level l of the reduce-
// then-scan hierarchy holds ceil(count / 4096^l) values.
__device__ __forceinline__ uint64_t emit_scan_count(const EmitState *es, int level) {
    uint64_t c = (uint64_t)es->nb * ((es->count + kEmitTile - 1) / kEmitTile);
    for (int l = 0; l < level; l++) c = (c + kScanBlock - 1) / kScanBlock;
    return c;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce_dev(const uint32_t *__restrict__ in, const EmitState *__restrict__ es, int level,
                  uint32_t *__restrict__ sums) {
    const uint64_t count = emit_scan_count(es, level);
    if ((uint64_t)blockIdx.x * kScanBlock >= count) return;
    scan_reduce_block(in, count, sums);
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_down_dev(const uint32_t *in, uint32_t *out, const EmitState *__restrict__ es, int level,
                const uint32_t *__restrict__ offs) {
    const uint64_t count = emit_scan_count(es, level);
    if ((uint64_t)blockIdx.x * kScanBlock >= count) return;
    scan_down_block(in, out, count, offs);
}

// Launch structure of the largest count; smaller counts leave blocks idle.
void launch_scan_dev(const Launch &L, const uint32_t *in, uint32_t *out, uint64_t max_count,
                     const EmitState *es, int level, uint32_t *tmp) {
    if (max_count <= kScanBlock) {
        count_launch();
        k_scan_down_dev<<<1, kScanThreads, 0, L.stream>>>(in, out, es, level, nullptr);
        return;
    }
    const uint64_t blocks = (max_count + kScanBlock - 1) / kScanBlock;
    count_launch();
    k_scan_reduce_dev<<<(unsigned)blocks, kScanThreads, 0, L.stream>>>(in, es, level, tmp);
    launch_scan_dev(L, tmp, tmp, blocks, es, level + 1, tmp + blocks);
    count_launch();
    k_scan_down_dev<<<(unsigned)blocks, kScanThreads, 0, L.stream>>>(in, out, es, level, tmp);
}

// layer_off[t] = loff[t] for t <= R, when R fits the caller's table.
__global__ void k_layer_off_dev(const uint32_t *__restrict__ loff, const Ctl *__restrict__ ctl,
                                uint32_t max_layers, uint64_t *__restrict__ out) {
    const uint32_t R = ctl->more ? ctl->round + 1 : ctl->round;
    if (R > max_layers) return;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= R; t += gridDim.x * blockDim.x)
        out[t] = loff[t];
}

void launch_emit_init(const Launch &L, const Ctl *ctl, uint32_t n, EmitState *es,
                      cudaGraphConditionalHandle h) {
    count_launch();
    k_emit_init<<<1, 1, 0, L.stream>>>(ctl, n, es, h);
}

void launch_extract_claim_hist_dev(const Launch &L, const uint4 *rec, uint32_t n, uint32_t r,
                                   uint32_t *claim, const EmitState *es, uint32_t *hist) {
    if (n == 0) return;
    const uint32_t tiles = (n + kEmitTile - 1) / kEmitTile;
    count_launch();
    switch (r) {
    case 2: k_extract_claim_hist_dev<2><<<tiles, kThreads, 0, L.stream>>>(rec, n, claim, es, hist); break;
    case 3: k_extract_claim_hist_dev<3><<<tiles, kThreads, 0, L.stream>>>(rec, n, claim, es, hist); break;
    case 4: k_extract_claim_hist_dev<4><<<tiles, kThreads, 0, L.stream>>>(rec, n, claim, es, hist); break;
    }
}

void launch_emit_pass_dev(const Launch &L, uint32_t n, const uint32_t *tail, const uint32_t *claim,
                          const EmitState *es, uint32_t *hist, uint32_t *scantmp,
                          uint32_t *order) {
    const uint32_t tiles = (n + kEmitTile - 1) / kEmitTile;
    count_launch();
    k_emit_hist_dev<<<tiles, kThreads, 0, L.stream>>>(tail, claim, es, hist);
    launch_scan_dev(L, hist, hist, (uint64_t)kEmitBins * tiles, es, 0, scantmp);
    count_launch();
    k_emit_scatter_dev<<<tiles, kThreads, 0, L.stream>>>(tail, claim, es, hist, order);
}

void launch_emit_advance(const Launch &L, EmitState *es, const uint32_t *loff, uint32_t *order,
                         uint32_t *tail, cudaGraphConditionalHandle h) {
    count_launch();
    k_emit_advance<<<1, 1, 0, L.stream>>>(es, loff, h);
    count_launch();
    k_emit_copy_tail<<<grid_fixed(L, 4), kThreads, 0, L.stream>>>(order, tail, es);
}

void launch_layer_off_dev(const Launch &L, const uint32_t *loff, const Ctl *ctl,
                          uint32_t max_layers, uint64_t *out) {
    count_launch();
    k_layer_off_dev<<<grid_for(L, (uint64_t)max_layers + 1, 1, 4), kThreads, 0, L.stream>>>(
        loff, ctl, max_layers, out);
}

}  // namespace hp
