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
struct ProfScope {
    ProfScope(const Launch &L, const char *name);
    ~ProfScope();
    const Launch &L;
    const char *name;
    void *a;
};
void prof_flush();  // after a stream synchronisation: accumulate timings

// Persistent grid size for grid-stride kernels over device-sized ranges.
inline unsigned grid_fixed(const Launch &L, int per_sm) { return (unsigned)(L.sms * per_sm); }
inline unsigned grid_for(const Launch &L, uint64_t work, int per_thread, int per_sm) {
    uint64_t blocks = (work + (uint64_t)kThreads * per_thread - 1) / ((uint64_t)kThreads * per_thread);
    uint64_t cap = (uint64_t)L.sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    return (unsigned)blocks;
}

// a1: keys -> r-partite edges.
void launch_hash_edges(const Launch &L, const uint64_t *keys, uint64_t n, uint32_t r,
                       FastMod fm, uint64_t seed, uint32_t *edges);

// fill count 32-bit words with value.
void launch_fill_u32(const Launch &L, uint32_t *p, uint64_t count, uint32_t value);

// a2: degree / XOR-of-edge-ids records (state[2v] = deg, state[2v+1] = xor),
// claim[e] = unclaimed.
void launch_build_incidence(const Launch &L, const uint32_t *edges, uint32_t n, uint32_t r,
                            uint32_t P, uint32_t *state, uint32_t *claim, Ctl *ctl);

// a3 + a4 for round 0: scan all vertices, claim the edge of every degree-1
// vertex, append first claims to L.
void launch_round0(const Launch &L, const uint32_t *state, uint32_t m, uint32_t r, uint32_t P,
                   uint32_t n, uint32_t *claim, uint32_t *Llist, Ctl *ctl);

// a4 for round t >= 1 (t read on the device): claim edges of F_t.
void launch_claim(const Launch &L, const uint32_t *state, uint32_t r, uint32_t P, uint32_t n,
                  uint32_t *claim, const uint32_t *F, uint32_t *Llist, uint32_t *foff,
                  Ctl *ctl);

// a5 + a6: delete the edges of L_t from their non-hinge vertices, append
// vertices that fall to degree 1 to F_{t+1}; the last block advances t.
void launch_update(const Launch &L, const uint32_t *edges, uint32_t r, uint32_t m,
                   const uint32_t *claim, uint32_t *state, const uint32_t *Llist, uint32_t *F,
                   uint32_t *loff, const uint32_t *foff, Ctl *ctl);

// a7: one pass of the stable counting sort of edge ids by round.
void launch_emit_hist(const Launch &L, const uint32_t *src, uint32_t count, const uint32_t *claim,
                      uint32_t base, uint32_t core_key, uint32_t nbins, uint32_t *hist);
void launch_emit_scatter(const Launch &L, const uint32_t *src, uint32_t count,
                         const uint32_t *claim, uint32_t base, uint32_t core_key, uint32_t nbins,
                         const uint32_t *offs, uint32_t *out);
void launch_layer_off(const Launch &L, const uint32_t *loff, uint32_t rounds, uint64_t *out);

// Exclusive prefix sum of count 32-bit values (out may alias in).
size_t scan_tmp_words(uint64_t count);
void launch_scan_u32(const Launch &L, const uint32_t *in, uint32_t *out, uint64_t count,
                     uint32_t *tmp);

// a8: MWHC assignment of one layer t (host loop runs t = R-1 .. 0).
void launch_assign_layer(const Launch &L, const uint32_t *edges, const uint32_t *claim,
                         const uint32_t *order, const uint32_t *loff, uint32_t t, uint64_t *G);
// a9: per-512-vertex counts of non-zero 2-bit values, then the directory.
void launch_rank_counts(const Launch &L, const uint64_t *G, uint64_t m, uint32_t *cnt);
void launch_widen_dir(const Launch &L, const uint32_t *scanned, const uint32_t *cnt,
                      uint64_t blocks, uint64_t *dir);

}  // namespace hp
