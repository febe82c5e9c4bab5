// kernels.cuh -- host launchers of the hpeel kernels (one per hot-path step).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace hp {

constexpr int kThreads = 256;

// Stable counting sort of edges by round (canonical order) -- tile geometry.
constexpr int kEmitItems = 16;                                  // edges per thread
constexpr int kEmitWarps = kThreads / 32;
constexpr uint32_t kEmitTile = (uint32_t)kThreads * kEmitItems;  // 4096 edges
constexpr uint32_t kEmitBins = 256;                             // bins per pass

struct Launch {
    cudaStream_t stream;
    int sms;  // multiprocessors of the current device
};

// Instrumentation (prof.cu): every kernel launch is counted; when profiling
// is on, a ProfScope brackets a step with CUDA events on its stream.
void count_launch(uint32_t kernels = 1);
// While one lives on this thread, launches are not counted (graph capture).
struct LaunchCountPause {
    LaunchCountPause();
    ~LaunchCountPause();
};
struct ProfScope {
    ProfScope(const Launch &L, const char *name);
    ~ProfScope();
    const Launch &L;
    const char *name;
    void *a;
};
void prof_flush();  // after a stream synchronisation: accumulate timings

// Let fn take up to the device's opt-in maximum of dynamic shared memory.
// Set once per (device, kernel) under a lock and never lowered: the limit is
// process-wide state, and a per-launch value that another host thread lowers
// in between would make that thread's launch fail.
void smem_optin(const void *fn);

// Persistent grid size for grid-stride kernels over device-sized ranges.
inline unsigned grid_fixed(const Launch &L, int per_sm) { return (unsigned)(L.sms * per_sm); }
// One wave: as many blocks of kThreads as fit on the device at once (at most
// cap_per_sm per SM), for grid-stride kernels.
inline unsigned grid_resident(const Launch &L, const void *fn, int cap_per_sm,
                              size_t dyn_smem = 0, int threads = kThreads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, dyn_smem) != cudaSuccess ||
        nb <= 0) {
        cudaGetLastError();
        nb = 1;
    }
    if (nb > cap_per_sm) nb = cap_per_sm;
    return (unsigned)(L.sms * nb);
}
inline unsigned grid_for(const Launch &L, uint64_t work, int per_thread, int per_sm) {
    uint64_t blocks = (work + (uint64_t)kThreads * per_thread - 1) / ((uint64_t)kThreads * per_thread);
    uint64_t cap = (uint64_t)L.sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    return (unsigned)blocks;
}

// a1: keys -> r-partite edges (row-major rows, or edge records).
void launch_hash_edges(const Launch &L, const uint64_t *keys, uint64_t n, uint32_t r,
                       FastMod fm, uint64_t seed, uint32_t *edges,
                       bool gen = false);
// seed_dev (or NULL): the seed is read from device memory when the kernel
// runs (device-driven retries), else the seed argument.
void launch_hash_records(const Launch &L, const uint64_t *keys, uint64_t n, uint32_t r,
                         FastMod fm, uint64_t seed, uint4 *rec,
                         const uint64_t *seed_dev = nullptr);

// fill count 32-bit words with value.
void launch_fill_u32(const Launch &L, uint32_t *p, uint64_t count, uint32_t value);

// Row-major edges -> edge records (checks the r-partite ranges; gen: every
// vertex below P = m).
void launch_records(const Launch &L, const uint32_t *edges, uint32_t n, uint32_t r, uint32_t P,
                    uint4 *rec, Ctl *ctl, bool gen);

// a2: vertex records {deg, sum of incident edge ids} from the edge records.
void launch_build_incidence(const Launch &L, const uint4 *rec, uint32_t n, uint32_t r,
                            uint32_t m, unsigned long long *st, Ctl *ctl);

// a2, L2-blocked (build.cu): records + incidences bucketed by vertex chunk,
// then the buckets applied chunk by chunk.
struct BucketPlan {
    uint32_t shift;            // log2 vertices per chunk
    uint32_t chunks_per_part;
    uint32_t chunks;
    uint32_t blocks;           // blocks of the bucketing kernel
    uint32_t cap;              // incidences per chunk (one array each)
    uint64_t pair_bytes;       // bucket storage
    uint64_t fill_words;       // fill counters (one per chunk, 2^kFillShift words apart)
    size_t smem;               // dynamic shared memory of the bucketing kernel
    uint32_t sub_shift;        // log2 vertices per sub-bucket
    uint32_t subs;             // sub-buckets in all
    uint32_t cap2;             // incidences per sub-bucket
    uint64_t pair2_bytes;      // sub-bucket storage
    uint32_t ovf_cap;          // overflow list entries
    uint32_t parts;            // r (r-partite) or 1 (general graph)
    uint32_t passes;           // 1, or parts (one part per pass)
    uint32_t chunks_pass;      // chunks of one pass
    uint32_t subs_pass;        // sub-buckets of one pass
};
// Incidences that found their bucket full (applied last).  Without a list
// (count == nullptr) a full bucket raises code instead.
struct Overflow {
    uint2 *list;
    uint32_t *count;
    uint32_t cap;
    uint32_t code = kDevBuildOverflow;
};

// Exclusive prefix sum of h[0 .. count) into out[0 .. count) by the whole
// block (THREADS threads, each taking ceil(count / THREADS) consecutive
// entries: a warp shuffle scan, then one over the warps' totals).  Every
// thread calls it; the block is synchronised on return.
template <int THREADS>
__device__ __forceinline__ void block_scan_counts(const uint32_t *h, uint32_t *out,
                                                  uint32_t count) {
    constexpr int kW = THREADS / 32;
    __shared__ uint32_t ws[kW];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t per = (count + THREADS - 1) / THREADS, c0 = threadIdx.x * per;
    uint32_t loc = 0;
    for (uint32_t q = 0; q < per; q++)
        if (c0 + q < count) loc += h[c0 + q];
    uint32_t x = loc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    uint32_t wx = lane < (uint32_t)kW ? ws[lane] : 0u;
#pragma unroll
    for (int d = 1; d < kW; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wx, d);
        if (lane >= (uint32_t)d) wx += y;
    }
    const uint32_t before = __shfl_sync(0xFFFFFFFFu, wx, (warp + 31u) & 31u);
    uint32_t run = x - loc + (warp ? before : 0u);
    for (uint32_t q = 0; q < per; q++) {
        const uint32_t c = c0 + q;
        if (c < count) {
            out[c] = run;
            run += h[c];
        }
    }
    __syncthreads();
}

// Geometry of one bucketing: part size, log2 of the keys per chunk, chunks
// per part, chunk capacity, fill-counter stride.
struct BucketGeom {
    uint32_t P;                // part size
    uint32_t shift;            // log2 of the vertices per chunk
    uint32_t chunks_per_part;
    uint32_t cap;              // chunk capacity (incidences per chunk)
    uint32_t fill_shift;       // chunk c's fill counter is fill[c << fill_shift]
};
// The build's chunk cursors sit one 128-byte line apart: every block of the
// bucketing pass advances them, and cursors sharing a line would serialise.
constexpr uint32_t kFillShift = 5;
// parts: r for an r-partite graph (chunks never straddle parts), 1 for a
// general graph (one part [0, m)).
// part_passes: the tuning's bucket_part_passes (0 automatic, 1 one pass,
// 2 one part per pass).  pair_bytes, pair2_bytes: the storage of one pass.
BucketPlan bucket_plan(uint64_t n, uint64_t m, uint32_t r, uint32_t parts, uint32_t shift,
                       uint32_t sub_shift, int sms, uint32_t part_passes);
// Pass `pass` (0 .. passes - 1) of the bucketing; records are written by pass 0.
void launch_build_bucketed(const Launch &L, const BucketPlan &b, const uint64_t *keys,
                           const uint32_t *rows, uint32_t n, uint32_t r, FastMod fm,
                           uint64_t seed, uint32_t P, uint4 *rec, uint2 *pairs, uint32_t *fill,
                           Overflow ov, Ctl *ctl, bool gen, const uint64_t *seed_dev,
                           uint32_t pass);
// Refine only: the pairs of `chunks` chunks (from chunk0) counting-sorted
// into sub-buckets of 2^sub_shift keys (pair.x is the key); fill2 zeroed
// before.
void launch_refine(const Launch &L, const BucketGeom &g, uint32_t chunks, uint32_t chunk0,
                   uint32_t sub_shift, const uint2 *pairs, const uint32_t *fill,
                   uint2 *pairs2, uint32_t *fill2, uint32_t cap2, Overflow ov, Ctl *ctl);
// Round 0's claims emitted by the incidence build itself (the shared-memory
// apply sees every final degree): claims == nullptr for none.
struct ClaimSink {
    uint2 *claims;
    uint32_t cap;
    uint32_t n;
};
// Refine and apply of the same pass (fill2 and the overflow count zeroed
// before the pass's bucketing).  With a sink, every vertex of degree 1 appends
// its claim {edge, vertex} (ctl->cvalid tells round 0 whether the list is
// complete: not when overflowed incidences were applied afterwards).
void launch_apply_buckets(const Launch &L, const BucketPlan &b, uint32_t P, const uint2 *pairs,
                          const uint32_t *fill, uint2 *pairs2, uint32_t *fill2, Overflow ov,
                          unsigned long long *st, Ctl *ctl, uint32_t pass,
                          ClaimSink sink = ClaimSink{nullptr, 0, 0});

// Rounds in sorted form (rounds_bucketed.cu): the plan of a peel and the
// buffers it uses in the workspace.
struct SortedPlan {
    bool enabled;
    uint32_t min_edges, max_edges;  // layers deleted in sorted form
    uint32_t claim_cap;             // claims one round may make
    uint32_t bucket_blocks;         // blocks of the bucketing pass (list entries)
    uint32_t claim_bucket_blocks;   // blocks of the bucketing pass (claims)
    BucketGeom vg;                  // updates by vertex (parts, chunks)
    uint32_t vchunks, vsub_shift, vsubs, vcap2;
    BucketGeom eg;                  // claims by edge (one part of n edges)
    uint32_t eshift, esub, echunks, esubs, ecap2;
    size_t bucket_smem, claim_bucket_smem;
    uint64_t pairs_bytes, fill_bytes, pairs2_bytes, fill2_bytes, claims_bytes;
};
struct SortedBufs {
    uint2 *pairs;
    uint32_t *fill;
    uint2 *pairs2;
    uint32_t *fill2;
    uint2 *claims;
};
// min_edges: 0 automatic (n / 24), 0xFFFFFFFF never; b: the incidence
// build's bucket plan (its vertex chunks are reused).
SortedPlan sorted_plan(uint64_t n, uint64_t m, uint32_t r, const BucketPlan &b, uint32_t min_edges,
                       int sms);
// Round 0 (claims of the degree-1 vertices, L_0 listed) and one sorted round
// t = ctl->round (layer t deleted, layer t+1 claimed and listed); each ends
// by closing the round and setting the conditions (h_sorted: the next round
// is sorted; h_random: a round follows).
void launch_sorted_round0(const Launch &L, const SortedPlan &p, const SortedBufs &w,
                          const unsigned long long *st, uint32_t n, uint32_t m, uint4 *rec,
                          uint4 *Lst, uint32_t *loff, Ctl *ctl, uint32_t max_rounds,
                          cudaGraphConditionalHandle h_sorted,
                          cudaGraphConditionalHandle h_random);
void launch_sorted_round(const Launch &L, const SortedPlan &p, const SortedBufs &w,
                         unsigned long long *st, uint32_t n, uint4 *rec, uint4 *Lst,
                         uint32_t *loff, Ctl *ctl, uint32_t max_rounds,
                         cudaGraphConditionalHandle h_sorted, cudaGraphConditionalHandle h_random);

// A kernel of the round loop and its launch shape, for graph nodes.
struct RoundLaunch {
    void *fn;
    unsigned grid, block;
    unsigned smem;  // dynamic shared memory bytes per block
};

// a3 + a4 of round 0: scan all vertices, claim the edge of every degree-1
// vertex; publishes loff[0..1].
// *dst = v, in stream order.
void launch_set_params(const Launch &L, RoundParams *dst, const RoundParams &v);

// gen: a general (not r-partite) hypergraph, positions read off the rows.
void launch_round0(const Launch &L, uint32_t r, bool gen, const RoundParams *prm);
RoundLaunch round0_launch(const Launch &L, uint32_t r, bool gen);

// a5 + a4 of the next round + a6: delete layer t (t read on the device),
// claim and list layer t+1, close the round.
void launch_round(const Launch &L, uint32_t r, bool gen, const RoundParams *prm);
RoundLaunch round_launch(const Launch &L, uint32_t r, bool gen);

// claim[e] = claim word of record e.
void launch_extract_claim(const Launch &L, const uint4 *rec, uint32_t n, uint32_t r,
                          uint32_t *claim);

// a7: one pass of the stable counting sort of edge ids by round.
void launch_extract_claim_hist(const Launch &L, const uint4 *rec, uint32_t n, uint32_t r,
                               uint32_t *claim, uint32_t core_key, uint32_t nbins,
                               uint32_t *hist);
void launch_emit_hist(const Launch &L, const uint32_t *src, uint32_t count, const uint32_t *claim,
                      uint32_t base, uint32_t core_key, uint32_t nbins, uint32_t *hist);
void launch_emit_scatter(const Launch &L, const uint32_t *src, uint32_t count,
                         const uint32_t *claim, uint32_t base, uint32_t core_key, uint32_t nbins,
                         const uint32_t *offs, uint32_t *out);
void launch_layer_off(const Launch &L, const uint32_t *loff, uint32_t rounds, uint64_t *out);

// a7 driven by the device (EmitState in device memory): init (sets the
// pass loop's condition), the claims with the first histogram, one pass
// (later histogram, scan, scatter), advance to the next pass (sets the
// condition, copies the order's tail for the next pass), layer offsets.
void launch_emit_init(const Launch &L, const Ctl *ctl, uint32_t n, EmitState *es,
                      cudaGraphConditionalHandle h);
void launch_extract_claim_hist_dev(const Launch &L, const uint4 *rec, uint32_t n, uint32_t r,
                                   uint32_t *claim, const EmitState *es, uint32_t *hist);
void launch_emit_pass_dev(const Launch &L, uint32_t n, const uint32_t *tail, const uint32_t *claim,
                          const EmitState *es, uint32_t *hist, uint32_t *scantmp,
                          uint32_t *order);
void launch_emit_advance(const Launch &L, EmitState *es, const uint32_t *loff, uint32_t *order,
                         uint32_t *tail, cudaGraphConditionalHandle h);
void launch_layer_off_dev(const Launch &L, const uint32_t *loff, const Ctl *ctl,
                          uint32_t max_layers, uint64_t *out);

// f4: MPHF build beyond 32-bit ids (large.cu).
RoundLaunch large_round_launch(const Launch &L, bool first);
void launch_large_set_params(const Launch &L, LargeParams *dst, const LargeParams &v);
void launch_large_build(const Launch &L, const uint64_t *keys, uint64_t n, uint64_t seed,
                        FastMod fm, unsigned long long *st, uint32_t *claim, LargeCtl *ctl);
void launch_large_assign(const Launch &L, const LargeParams *prm, uint32_t t, uint64_t *G);
void launch_large_rank(const Launch &L, const uint64_t *G, uint64_t m, uint32_t *cnt,
                       unsigned long long *seg, uint64_t *dir);
void launch_large_lookup(const Launch &L, const uint64_t *keys, uint64_t nq, FastMod fm,
                         uint64_t seed, const uint64_t *G, const uint64_t *dir, uint64_t *out);

// a10: batched bucket peel (batched.cu).
size_t batched_scratch_bytes(uint32_t gamma_milli);
uint32_t batched_max_gamma_milli();
// Most layer-table entries of a bucket with 16-bit claim words.
uint32_t batched_claim16_rounds();
void launch_batched(const Launch &L, const uint64_t *keys, const uint64_t *off, uint32_t B,
                    uint32_t gamma_milli, uint32_t *order, uint32_t *rounds, uint32_t *status,
                    uint64_t *G, const uint64_t *G_off, uint32_t threads, uint32_t ctas,
                    uint32_t smem_bytes, uint32_t smem_rounds, uint32_t global16_rounds,
                    uint32_t *sched,
                    uint32_t *next, char *scratch);
void launch_batch_g_offsets(const Launch &L, const uint64_t *off, uint32_t B, uint32_t gamma_milli,
                            uint32_t *words, uint32_t *scanned, uint32_t *tmp, uint64_t *G_off);

// Exclusive prefix sum of count 32-bit values (out may alias in).
size_t scan_tmp_words(uint64_t count);
void launch_scan_u32(const Launch &L, const uint32_t *in, uint32_t *out, uint64_t count,
                     uint32_t *tmp);

// a8: MWHC assignment of one layer t from its solve records (host loop runs
// t = R-1 .. 0).
void launch_assign_layer(const Launch &L, const uint4 *Lst, const uint32_t *loff, uint32_t t,
                         uint32_t P, uint64_t *G);
// Static function (sec. 3): assignment of layer t mod sigma, b-bit values;
// lookup of nq keys.
void launch_sf_assign_layer(const Launch &L, const uint4 *Lst, const uint32_t *loff, uint32_t t,
                            const uint32_t *values, uint64_t sigma, uint32_t b, uint64_t *U,
                            Ctl *ctl);
void launch_sf_assign_layer_at(const Launch &L, const uint4 *Lst, const uint32_t *loff,
                               const int32_t *t, const uint32_t *values, uint64_t sigma,
                               uint32_t b, uint64_t *U, Ctl *ctl);
void launch_sf_lookup(const Launch &L, const uint64_t *keys, uint64_t nq, FastMod fm,
                      uint64_t seed, uint64_t sigma, uint32_t b, const uint64_t *U,
                      uint32_t *out);
// Assignment of the layer whose index the device holds at *t (device-driven
// build).
void launch_assign_layer_at(const Launch &L, const uint4 *Lst, const uint32_t *loff,
                            const int32_t *t, uint32_t P, uint64_t *G);
// Device-driven build control (async.cu): one-thread kernels that set the
// conditions of the graph's loops.
void launch_async_empty(const Launch &L, hpeel_stats *out, uint64_t seed, uint64_t *D);
void launch_async_init(const Launch &L, AsyncState *s, uint64_t seed, uint32_t max_tries,
                       uint32_t n);
void launch_async_check_overflow(const Launch &L, const Ctl *ctl, cudaGraphConditionalHandle h);
void launch_async_check_code(const Launch &L, const Ctl *ctl, uint32_t code,
                             cudaGraphConditionalHandle h);
void launch_async_decide(const Launch &L, AsyncState *s, const Ctl *ctl,
                         cudaGraphConditionalHandle h);
void launch_async_if_peeled(const Launch &L, const AsyncState *s, cudaGraphConditionalHandle h);
void launch_async_assign_init(const Launch &L, AsyncState *s, cudaGraphConditionalHandle h);
void launch_async_assign_step(const Launch &L, AsyncState *s, cudaGraphConditionalHandle h);
void launch_async_stats(const Launch &L, const AsyncState *s, const Ctl *ctl, hpeel_stats *out);
// Device-driven peel: the order runs only when no kernel raised an error;
// stats of the peel; the empty graph.
void launch_async_if_ok(const Launch &L, const Ctl *ctl, cudaGraphConditionalHandle h);
void launch_peel_async_stats(const Launch &L, const Ctl *ctl, uint32_t n, uint32_t max_layers,
                             bool want_layer_off, hpeel_stats *out);
void launch_peel_async_empty(const Launch &L, hpeel_stats *out, uint64_t *layer_off);
// a9: per-512-vertex counts of non-zero 2-bit values, then the directory.
void launch_rank_counts(const Launch &L, const uint64_t *G, uint64_t m, uint32_t *cnt);
void launch_widen_dir(const Launch &L, const uint32_t *scanned, const uint32_t *cnt,
                      uint64_t blocks, uint64_t *dir);
// MPHF lookup of nq keys.
void launch_lookup(const Launch &L, const uint64_t *keys, uint64_t nq, FastMod fm, uint64_t seed,
                   const uint64_t *G, const uint64_t *dir, uint32_t *out);

}  // namespace hp
