// api.cu -- the C ABI (include/hpeel.h): argument checks, workspace layout,
// the round loop, the MPHF retry loop and its device-driven form (one CUDA
// graph with conditional nodes).  Every step of the path runs in the kernels
// of hash.cu, build.cu, peel.cu, emit.cu, mphf.cu and async.cu; this file
// only orders them and reads back the few scalars the host has to decide on.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "host.h"
#include "kernels.cuh"

using namespace hp;

namespace hp {
thread_local std::string g_last_error;
}

namespace {

// Small pinned host buffer for the per-round control-block read-back.
Ctl *pinned_ctl() {
    thread_local Ctl *p = nullptr;
    if (!p) {
        if (cudaMallocHost((void **)&p, sizeof(Ctl)) != cudaSuccess) p = nullptr;
    }
    return p;
}

struct PeelLayout {
    size_t ctl, params, emit, rec, state, claim, L, pairs, fill, pairs2, fill2, ovf, ovf_count, loff,
        hist, scantmp, total;
    size_t s_pairs, s_fill, s_pairs2, s_fill2, s_claims;  // sorted rounds
    uint32_t max_rounds;
    bool bucketed;
    BucketPlan plan;
    SortedPlan sp;
};

// SM count of the current device (152 when there is none: plan for a GB300).
int current_sms() {
    int dev = 0;
    DeviceInfo d;
    if (cudaGetDevice(&dev) != cudaSuccess || device_info(dev, &d) != HPEEL_OK) {
        cudaGetLastError();
        return 152;
    }
    return d.sms;
}

// Process-wide tuning (hpeel_set_tuning); read by layouts and launches.
hpeel_tuning g_tuning = {22u, 8u << 20, 0u, 0u, 0u, 0u, {0, 0}};
std::mutex g_tuning_mu;

hpeel_tuning tuning() {
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    return g_tuning;
}

// Workspace of one peel: edge records, vertex records, layer list (one entry
// per edge, the shape of an edge record), the incidence buckets of the
// L2-blocked build (sharing space with the layer list, which is written only
// after the build), the sub-buckets (sharing space with the claim words and
// the order-sort scratch, which are used only after the rounds), layer table.
PeelLayout peel_layout(uint64_t n, uint64_t m, uint32_t r, bool general = false) {
    PeelLayout p{};
    const hpeel_tuning tu = tuning();
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    p.max_rounds = (uint32_t)std::min<uint64_t>(HPEEL_MAX_ROUNDS, n + 1);
    p.bucketed = n > 0 && m >= tu.bucket_min_vertices;
    if (p.bucketed) {
        p.plan = bucket_plan(n, m, r, general ? 1u : r, tu.bucket_shift, tu.bucket_sub_shift,
                             current_sms(), tu.bucket_part_passes);
        // the bucketing kernel keeps three counters per chunk in shared memory
        if (p.plan.smem > (200u << 10)) p.bucketed = false;
    }
    if (p.bucketed && !general)
        p.sp = sorted_plan(n, m, r, p.plan, tu.sorted_round_min, current_sms());
    p.ctl = take(sizeof(Ctl));
    p.params = take(sizeof(RoundParams));
    p.emit = take(sizeof(EmitState));
    p.rec = take((r == 4 ? 32 : 16) * n);
    p.state = take(8 * m);
    // the layer list, the build's first-level buckets (dead once refined)
    // and, after the list's n entries, the claim list of the sorted rounds
    // (written from the build's apply on, so not where the build's live
    // sub-buckets are)
    const size_t ls = (r == 4 ? 32 : 16) * n;
    size_t shared = std::max<size_t>(ls, p.bucketed ? p.plan.pair_bytes : 0);
    const size_t claims_at = align256(ls);
    if (p.sp.enabled) shared = std::max<size_t>(shared, claims_at + p.sp.claims_bytes);
    const size_t region = take(shared);
    p.L = region;
    p.pairs = region;
    if (p.sp.enabled) p.s_claims = region + claims_at;
    p.fill = take(p.bucketed ? 4 * (size_t)p.plan.fill_words : 0);
    p.fill2 = take(p.bucketed ? 4 * (size_t)p.plan.subs_pass : 0);
    p.ovf = take(p.bucketed ? 8 * (size_t)p.plan.ovf_cap : 0);
    p.ovf_count = take(p.bucketed ? 4 : 0);
    p.loff = take(4 * ((size_t)p.max_rounds + 3));
    // sub-buckets (build only) | claim words + order-sort scratch (after the rounds)
    const uint64_t tiles = (n + kEmitTile - 1) / kEmitTile;
    const size_t region2 = off;
    size_t o2 = 0;
    auto take2 = [&](size_t bytes) {
        size_t o = o2;
        o2 = align256(o2 + bytes);
        return region2 + o;
    };
    p.claim = take2(4 * n);
    p.hist = take2(4 * kEmitBins * tiles);
    p.scantmp = take2(4 * scan_tmp_words(kEmitBins * tiles));
    p.pairs2 = region2;
    // the buckets of the sorted rounds live there too: they are used after
    // the build and before the order
    size_t o3 = 0;
    auto take3 = [&](size_t bytes) {
        size_t o = o3;
        o3 = align256(o3 + bytes);
        return region2 + o;
    };
    if (p.sp.enabled) {
        p.s_pairs = take3(p.sp.pairs_bytes);
        p.s_fill = take3(p.sp.fill_bytes);
        p.s_pairs2 = take3(p.sp.pairs2_bytes);
        p.s_fill2 = take3(p.sp.fill2_bytes);
    }
    off = region2 + std::max<size_t>(std::max<size_t>(o2, o3),
                                     p.bucketed ? align256(p.plan.pair2_bytes) : 0);
    p.total = off;
    return p;
}

SortedBufs sorted_bufs(const PeelLayout &lay, char *ws) {
    return SortedBufs{reinterpret_cast<uint2 *>(ws + lay.s_pairs),
                      reinterpret_cast<uint32_t *>(ws + lay.s_fill),
                      reinterpret_cast<uint2 *>(ws + lay.s_pairs2),
                      reinterpret_cast<uint32_t *>(ws + lay.s_fill2),
                      reinterpret_cast<uint2 *>(ws + lay.s_claims)};
}

struct MphfLayout {
    size_t state, rank_cnt, rank_scan, rank_tmp, peel, total;
    uint64_t m;
};

MphfLayout mphf_layout(uint64_t n, uint32_t gamma_milli) {
    MphfLayout p{};
    p.m = hpeel_num_vertices(n, gamma_milli, 3);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const uint64_t blocks = (p.m + 511) / 512;
    p.state = take(sizeof(AsyncState));
    p.rank_cnt = take(4 * blocks + 4);
    p.rank_scan = take(4 * blocks + 4);
    p.rank_tmp = take(4 * scan_tmp_words(blocks));
    p.peel = off;
    p.total = off + peel_layout(n, p.m, 3).total;
    return p;
}

struct PeelOut {
    uint32_t rounds;
    uint64_t n_peeled;
    uint64_t first_layer;
    uint64_t frontier;
    uint64_t moves;
    uint32_t sorted_rounds;
    uint32_t *loff;  // device layer table (uint32[rounds + 2])
    uint4 *list;     // device layer list: entries {v_hinge, others, e}
};

// What a peel starts from and what it must produce.
struct PeelIO {
    const uint32_t *edges = nullptr;  // row-major [n][r] input, or
    const uint64_t *keys = nullptr;   // keys hashed with (seed, fm) into records
    uint64_t seed = 0;
    FastMod fm{0, 0};
    uint32_t *order = nullptr;  // canonical order output (nullptr: not needed)
    uint32_t *claim = nullptr;  // claim-word output (nullptr: workspace)
    bool force_direct = false;  // update the vertex records directly (no buckets)
    bool general = false;       // a general (not r-partite) hypergraph on [0, m)
    bool host_loop = false;     // launch every round from the host, whatever the tuning
    bool random_rounds = false; // no round in sorted form
};

// Executable graphs of the round loop, cached by their parameters: round 0,
// then a while node whose body is one round kernel.  The round kernel's last
// block sets the while condition (next layer non-empty, table not full).
// The cache keeps the kGraphCache most recently used graphs.  A graph may
// still run on another caller's stream when it is evicted, so every launch
// records an event after it, and eviction waits for that event before the
// graph (and the condition handle its kernels set) is destroyed.
struct RoundGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;  // recorded after the latest launch
};
constexpr size_t kGraphCache = 16;
std::mutex g_graph_mu;
std::map<std::string, RoundGraph> g_graphs;
std::vector<std::string> g_graph_lru;  // least recently used first

void destroy_graph(RoundGraph &g) {
    if (g.done) {
        cudaEventSynchronize(g.done);
        cudaEventDestroy(g.done);
    }
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = RoundGraph{};
}

// Capture streams of this thread (one per nesting depth of the graph).
cudaStream_t capture_stream(int depth) {
    thread_local cudaStream_t s[4] = {nullptr, nullptr, nullptr, nullptr};
    thread_local int dev_of[4] = {-1, -1, -1, -1};
    int d = 0;
    cudaGetDevice(&d);
    if (!s[depth] || dev_of[depth] != d) {
        if (cudaStreamCreateWithFlags(&s[depth], cudaStreamNonBlocking) != cudaSuccess)
            return nullptr;
        dev_of[depth] = d;
    }
    return s[depth];
}

// A condition handle on the graph stream s is capturing into.
cudaError_t new_handle(cudaStream_t s, unsigned default_value, unsigned flags,
                       cudaGraphConditionalHandle *h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    return cudaGraphConditionalHandleCreate(h, g, default_value, flags);
}

// Append a conditional node at the capture position of s; *body receives its
// body graph, into which another stream captures.
cudaError_t append_conditional(cudaStream_t s, cudaGraphConditionalHandle h,
                               cudaGraphConditionalNodeType type, cudaGraph_t *body) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
    if (e != cudaSuccess) return e;
    *body = cp.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                               cudaStreamSetCaptureDependencies);
}

// Launch the cached executable graph for key on L.stream, capturing and
// instantiating it with capture() on first use (least recently used graphs
// are evicted, after their latest launch has finished).
template <typename F>
hpeel_status launch_cached_graph(const Launch &L, const std::string &key, F capture) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) {
        while (g_graph_lru.size() >= kGraphCache) {
            auto old = g_graphs.find(g_graph_lru.front());
            if (old != g_graphs.end()) {
                destroy_graph(old->second);
                g_graphs.erase(old);
            }
            g_graph_lru.erase(g_graph_lru.begin());
        }
        RoundGraph rg;
        HP_TRY(capture(&rg.graph));
        if (cudaGraphInstantiate(&rg.exec, rg.graph, 0) != cudaSuccess ||
            cudaEventCreateWithFlags(&rg.done, cudaEventDisableTiming) != cudaSuccess) {
            const cudaError_t e = cudaGetLastError();
            destroy_graph(rg);
            return fail(HPEEL_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
        }
        it = g_graphs.emplace(key, rg).first;
        g_graph_lru.push_back(key);
    } else {
        auto pos = std::find(g_graph_lru.begin(), g_graph_lru.end(), key);
        if (pos != g_graph_lru.end()) g_graph_lru.erase(pos);
        g_graph_lru.push_back(key);
    }
    HP_CUDA(cudaGraphLaunch(it->second.exec, L.stream));
    HP_CUDA(cudaEventRecord(it->second.done, L.stream));
    return HPEEL_OK;
}

// Round 0 and the loops of rounds, added at the capture position of s0; the
// loop bodies are captured on s1.  With a sorted plan: round 0 and the first
// rounds in sorted form (a while node over sorted rounds, rounds_bucketed.cu),
// then a while node over the random round kernel; without one: the random
// round 0 and its loop.  The round kernels' last blocks (or the sorted
// rounds' closing kernel) set the loop conditions.
struct RoundsArgs {
    uint32_t n, m, r;
    bool gen;
    const RoundParams *prm;
    const SortedPlan *sp;  // null: random rounds only
    SortedBufs sw;
    unsigned long long *st;
    uint4 *rec, *Ll;
    uint32_t *loff;
    Ctl *ctl;
    uint32_t max_rounds;
};

cudaError_t capture_rounds(cudaStream_t s0, cudaStream_t s1, int sms, const RoundsArgs &a) {
    Launch L0{s0, sms}, L1{s1, sms};
    const RoundLaunch k0 = round0_launch(L0, a.r, a.gen), k1 = round_launch(L0, a.r, a.gen);
    cudaGraphConditionalHandle h_s = 0, h_r = 0;
    cudaGraph_t body = nullptr, g = nullptr;
    auto begin_body = [&](cudaGraph_t b) {
        return cudaStreamBeginCaptureToGraph(s1, b, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed);
    };
    cudaError_t e = new_handle(s0, 0u, 0u, &h_r);
    if (e != cudaSuccess) return e;
    if (a.sp) {
        e = new_handle(s0, 0u, 0u, &h_s);
        if (e != cudaSuccess) return e;
        launch_sorted_round0(L0, *a.sp, a.sw, a.st, a.n, a.m, a.rec, a.Ll, a.loff, a.ctl,
                             a.max_rounds, h_s, h_r);
        e = append_conditional(s0, h_s, cudaGraphCondTypeWhile, &body);
        if (e == cudaSuccess) e = begin_body(body);
        if (e != cudaSuccess) return e;
        launch_sorted_round(L1, *a.sp, a.sw, a.st, a.n, a.rec, a.Ll, a.loff, a.ctl, a.max_rounds,
                            h_s, h_r);
        e = cudaStreamEndCapture(s1, &g);
        if (e != cudaSuccess) return e;
    } else {
        void *args[] = {(void *)&a.prm, &h_r};
        count_launch();
        e = cudaLaunchKernel(k0.fn, dim3(k0.grid), dim3(k0.block), args, k0.smem, s0);
        if (e != cudaSuccess) return e;
    }
    e = append_conditional(s0, h_r, cudaGraphCondTypeWhile, &body);
    if (e == cudaSuccess) e = begin_body(body);
    if (e != cudaSuccess) return e;
    {
        void *args[] = {(void *)&a.prm, &h_r};
        e = cudaLaunchKernel(k1.fn, dim3(k1.grid), dim3(k1.block), args, k1.smem, s1);
    }
    const cudaError_t e2 = cudaStreamEndCapture(s1, &g);
    return e != cudaSuccess ? e : e2;
}

// Kernels one peel's rounds launched, from its control block: round 0 (6 in
// sorted form), 7 per sorted round, 1 per random round.
uint64_t round_kernels(const Ctl &c, bool sorted) {
    const uint64_t rounds = (uint64_t)c.round + (c.more ? 1 : 0);
    return (sorted ? 6 : 1) + 7ull * c.brounds + (rounds - c.brounds);
}

// The device-driven round loop of a host-driven peel: round 0 and the loops
// of rounds as one cached CUDA graph, launched on L.stream.
hpeel_status launch_round_graph(const Launch &L, const RoundsArgs &a) {
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    const hpeel_tuning tu = tuning();
    char keybuf[256];
    snprintf(keybuf, sizeof keybuf, "rounds|%d|%p|%u|%u|%u|%d|%d|%u|%u|%u|%u|%d", dev,
             (const void *)a.prm, a.n, a.m, a.r, a.gen ? 1 : 0, a.sp ? 1 : 0, tu.bucket_shift,
             tu.bucket_sub_shift, tu.bucket_part_passes, tu.sorted_round_min, L.sms);
    return launch_cached_graph(L, std::string(keybuf), [&](cudaGraph_t *g) -> hpeel_status {
        cudaStream_t s0 = capture_stream(0), s1 = capture_stream(1);
        if (!s0 || !s1) return fail(HPEEL_ERR_CUDA, "capture stream creation failed");
        LaunchCountPause pause;
        cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            e = capture_rounds(s0, s1, L.sms, a);
            cudaGraph_t got = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(s0, &got);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) {
                *g = got;
                return HPEEL_OK;
            }
            if (got) cudaGraphDestroy(got);
        }
        cudaGetLastError();
        return fail(HPEEL_ERR_CUDA, "round graph capture: %s", cudaGetErrorString(e));
    });
}

// Round-synchronous peel (sec. 4.2) of n edges on m vertices.
// hctl: host memory the control block is read back into after every round.
hpeel_status peel_core_rb(const Launch &L, const PeelIO &io, uint32_t n, uint32_t m, uint32_t r,
                          char *ws, PeelOut *out, Ctl *hctl) {
    const PeelLayout lay = peel_layout(n, m, r, io.general);
    const hpeel_tuning tu = tuning();
    Ctl *ctl = reinterpret_cast<Ctl *>(ws + lay.ctl);
    uint4 *rec = reinterpret_cast<uint4 *>(ws + lay.rec);
    unsigned long long *st = reinterpret_cast<unsigned long long *>(ws + lay.state);
    uint32_t *claim = io.claim ? io.claim : reinterpret_cast<uint32_t *>(ws + lay.claim);
    uint4 *Ll = reinterpret_cast<uint4 *>(ws + lay.L);
    uint32_t *loff = reinterpret_cast<uint32_t *>(ws + lay.loff);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + lay.hist);
    uint32_t *scantmp = reinterpret_cast<uint32_t *>(ws + lay.scantmp);
    // part size: one part [0, m) for a general graph
    const uint32_t P = io.general ? m : m / r;

    HP_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), L.stream));
    // the first rounds in sorted form when the plan allows it; the
    // L2-blocked build then also lists round 0's claims
    const bool sorted = lay.sp.enabled && !io.force_direct && !io.random_rounds && !io.general;
    const SortedBufs sbufs = sorted ? sorted_bufs(lay, ws) : SortedBufs{};
    const ClaimSink sink = sorted ? ClaimSink{sbufs.claims, lay.sp.claim_cap, n}
                                  : ClaimSink{nullptr, 0, 0};
    if (lay.bucketed && !io.force_direct) {
        uint2 *pairs = reinterpret_cast<uint2 *>(ws + lay.pairs);
        uint32_t *fill = reinterpret_cast<uint32_t *>(ws + lay.fill);
        uint2 *pairs2 = reinterpret_cast<uint2 *>(ws + lay.pairs2);
        uint32_t *fill2 = reinterpret_cast<uint32_t *>(ws + lay.fill2);
        Overflow ov{reinterpret_cast<uint2 *>(ws + lay.ovf),
                    reinterpret_cast<uint32_t *>(ws + lay.ovf_count), lay.plan.ovf_cap};
        for (uint32_t pass = 0; pass < lay.plan.passes; pass++) {
            HP_CUDA(cudaMemsetAsync(fill2, 0, 4 * (size_t)lay.plan.subs_pass, L.stream));
            HP_CUDA(cudaMemsetAsync(ov.count, 0, 4, L.stream));
            {
                ProfScope ps(L, io.keys ? "hash_bucket" : "records_bucket");
                launch_build_bucketed(L, lay.plan, io.keys, io.edges, n, r, io.fm, io.seed, P,
                                      rec, pairs, fill, ov, ctl, io.general, nullptr, pass);
            }
            // every vertex record of the pass's part is written by the
            // shared-memory apply
            ProfScope ps(L, "apply_buckets");
            launch_apply_buckets(L, lay.plan, P, pairs, fill, pairs2, fill2, ov, st, ctl, pass,
                                 sink);
        }
    } else {
        {
            ProfScope ps(L, "fill");
            launch_fill_u32(L, reinterpret_cast<uint32_t *>(st), 2ull * m, 0u);
        }
        if (io.keys) {
            ProfScope ps(L, "hash_edges");
            launch_hash_records(L, io.keys, n, r, io.fm, io.seed, rec);
        } else {
            ProfScope ps(L, "records");
            launch_records(L, io.edges, n, r, P, rec, ctl, io.general);
        }
        ProfScope ps(L, "build_incidence");
        launch_build_incidence(L, rec, n, r, m, st, ctl);
    }
    HP_TRY(check_launch("build"));
    RoundParams hp_prm{};
    hp_prm.st = st;
    hp_prm.rec = rec;
    hp_prm.L = Ll;
    hp_prm.loff = loff;
    hp_prm.ctl = ctl;
    hp_prm.n = n;
    hp_prm.m = m;
    hp_prm.P = P;
    hp_prm.max_rounds = lay.max_rounds;
    RoundParams *prm = reinterpret_cast<RoundParams *>(ws + lay.params);
    launch_set_params(L, prm, hp_prm);
    RoundsArgs ra{n, m, r, io.general, prm, sorted ? &lay.sp : nullptr, sbufs, st, rec, Ll,
                  loff, ctl, lay.max_rounds};
    auto read_ctl = [&]() -> hpeel_status {
        HP_CUDA(cudaMemcpyAsync(hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, L.stream));
        HP_CUDA(cudaStreamSynchronize(L.stream));
        return HPEEL_OK;
    };
    if (tu.host_round_loop || io.host_loop) {
        // one launch (or, sorted, one short sequence) per round, the control
        // block read back after each
        if (sorted) {
            {
                ProfScope ps(L, "round0");
                launch_sorted_round0(L, lay.sp, ra.sw, st, n, m, rec, Ll, loff, ctl,
                                     lay.max_rounds, 0, 0);
            }
            HP_TRY(check_launch("round0"));
            HP_TRY(read_ctl());
            while (hctl->more && !hctl->err && hctl->bmode) {
                {
                    ProfScope ps(L, "rounds_sorted");
                    launch_sorted_round(L, lay.sp, ra.sw, st, n, rec, Ll, loff, ctl,
                                        lay.max_rounds, 0, 0);
                }
                HP_TRY(check_launch("sorted round"));
                HP_TRY(read_ctl());
            }
        } else {
            {
                ProfScope ps(L, "round0");
                launch_round0(L, r, io.general, prm);
            }
            HP_TRY(check_launch("round0"));
            HP_TRY(read_ctl());
        }
        while (hctl->more && !hctl->err) {
            {
                ProfScope ps(L, "rounds");
                launch_round(L, r, io.general, prm);
            }
            HP_TRY(check_launch("round"));
            HP_TRY(read_ctl());
        }
    } else {
        // round 0 and the loops of rounds in one CUDA graph: the rounds run
        // back to back on the device, one read-back at the end
        ProfScope ps(L, "rounds");
        HP_TRY(launch_round_graph(L, ra));
        HP_TRY(read_ctl());
        count_launch((uint32_t)round_kernels(*hctl, sorted));
    }
    if (hctl->err == kDevRoundOverflow && sorted) {
        // a sorted round's buckets or claim list were full (a skewed input):
        // redo the peel with every round in random form (same result)
        PeelIO again = io;
        again.random_rounds = true;
        return peel_core_rb(L, again, n, m, r, ws, out, hctl);
    }
    if (hctl->err == kDevBuildOverflow && !io.force_direct) {
        // a skewed input overflowed the incidence buckets: redo the whole
        // peel (records included) with direct updates of the vertex records
        PeelIO again = io;
        again.force_direct = true;
        return peel_core_rb(L, again, n, m, r, ws, out, hctl);
    }
    if (hctl->err == kDevCapacity)
        return fail(HPEEL_ERR_CAPACITY, "more than %u rounds", lay.max_rounds - 1);
    if (hctl->err == kDevDegree)
        return fail(HPEEL_ERR_CAPACITY, "a vertex has degree 2^31 or more");
    if (hctl->err)
        return fail(HPEEL_ERR_DEVICE_CHECK, "device check failed with code %u", hctl->err);
    const uint32_t R = hctl->more ? hctl->round + 1 : hctl->round;
    out->first_layer = hctl->first_layer;
    out->rounds = R;
    out->n_peeled = hctl->lcur;
    out->frontier = hctl->cross;
    out->moves = hctl->moves;
    out->sorted_rounds = hctl->brounds;
    out->loff = loff;
    out->list = Ll;

    if (!io.order && !io.claim) return HPEEL_OK;
    if (!io.order) {
        ProfScope ps(L, "extract_claim");
        launch_extract_claim(L, rec, n, r, claim);
        return check_launch("extract_claim");
    }

    // Canonical order: stable sort by key = round, core edges key R.  The
    // first pass's histogram is taken while the claims are extracted.
    uint32_t *order = io.order;
    const uint32_t nkeys = R + 1;
    {
        ProfScope ps(L, "extract_claim");
        launch_extract_claim_hist(L, rec, n, r, claim, R, std::min<uint32_t>(nkeys, kEmitBins),
                                  hist);
    }
    uint32_t base = 0, seg = 0;
    const uint32_t *src = nullptr;
    uint32_t *loff_h = nullptr;
    std::string loff_store;
    for (;;) {
        const uint32_t count = n - seg;
        const uint32_t nb = std::min<uint32_t>(nkeys - base, kEmitBins);
        const uint32_t tiles = (count + kEmitTile - 1) / kEmitTile;
        if (base > 0) {
            ProfScope ps(L, "emit_hist");
            launch_emit_hist(L, src, count, claim, base, R, nb, hist);
        }
        {
            ProfScope ps(L, "emit_scan");
            launch_scan_u32(L, hist, hist, (uint64_t)nb * tiles, scantmp);
        }
        {
            ProfScope ps(L, "emit_scatter");
            launch_emit_scatter(L, src, count, claim, base, R, nb, hist, order + seg);
        }
        HP_TRY(check_launch("emit"));
        if (nkeys - base <= kEmitBins) break;
        // keys >= base + nb - 1 landed in the last bin: sort that tail again
        if (!loff_h) {
            loff_store.resize(4 * ((size_t)R + 1));
            loff_h = reinterpret_cast<uint32_t *>(&loff_store[0]);
            HP_CUDA(cudaMemcpyAsync(loff_h, loff, 4 * ((size_t)R + 1), cudaMemcpyDeviceToHost,
                                    L.stream));
            HP_CUDA(cudaStreamSynchronize(L.stream));
        }
        base += nb - 1;
        seg = loff_h[base];
        // the edge records are dead once the claims are extracted: their
        // space holds the tail being re-sorted (the layer list must survive
        // for the MWHC assignment)
        uint32_t *tail = reinterpret_cast<uint32_t *>(rec);
        HP_CUDA(cudaMemcpyAsync(tail + seg, order + seg, 4 * (size_t)(n - seg),
                                cudaMemcpyDeviceToDevice, L.stream));
        src = tail + seg;
    }
    return HPEEL_OK;
}

hpeel_status peel_core(const Launch &L, const PeelIO &io, uint32_t n, uint32_t m, uint32_t r,
                       char *ws, PeelOut *out) {
    Ctl *hctl = pinned_ctl();
    if (!hctl) return fail(HPEEL_ERR_CUDA, "cudaMallocHost of the control read-back failed");
    return peel_core_rb(L, io, n, m, r, ws, out, hctl);
}

// ---------------------------------------------------------------------------
// Device-driven MPHF build: one CUDA graph, no host round trip.
//
// The graph is captured from the same launchers the host-driven build uses,
// with conditional nodes added at the capture position: an outer while loop
// over hash seeds (build, an if-node that redoes an overflowed L2-blocked
// build with direct updates, round 0, the while loop of rounds, a decision
// kernel), then an if-node on success holding the reverse-layer assignment
// (a while loop over layers) and the rank directory, then the stats.
// ---------------------------------------------------------------------------

// A second stream and an event of this host thread on the current device:
// work that does not depend on what the caller's stream runs meanwhile goes
// there (the MWHC assignment beside the order sort).
struct SideStream {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int dev = -1;
};

hpeel_status side_stream(SideStream **out) {
    thread_local SideStream ss[64];
    int d = 0;
    HP_CUDA(cudaGetDevice(&d));
    if (d < 0 || d >= 64) return fail(HPEEL_ERR_INVALID_ARG, "device %d out of range", d);
    SideStream &s = ss[d];
    if (s.dev != d) {
        // default priority: a raised one took 0.5 ms off a lone build but
        // slowed host-to-device key copies and concurrent builds on some GB300s
        HP_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
        HP_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
        s.dev = d;
    }
    *out = &s;
    return HPEEL_OK;
}

struct AsyncArgs {
    const uint64_t *keys;
    uint32_t n, m, max_tries;
    uint64_t seed;
    uint32_t gamma_milli;
    uint64_t *G, *D;
    hpeel_stats *stats;
    char *ws;
    int sms;
    // static function (sec. 3, f: S -> [sigma]) instead of the MPHF: values
    // non-null, U written instead of G and the rank directory
    const uint32_t *values = nullptr;
    uint64_t sigma = 0;
    uint32_t bits = 0;
    uint64_t *U = nullptr;
};

// into: a stream the caller is capturing (the build joins that graph at the
// capture position), or null to capture a graph of its own into *out.
hpeel_status capture_async_build(const AsyncArgs &a, cudaStream_t into, cudaGraph_t *out) {
    cudaStream_t s0 = into ? into : capture_stream(0), s1 = capture_stream(1),
                 s2 = capture_stream(2), s3 = capture_stream(3);
    if (!s0 || !s1 || !s2 || !s3) return fail(HPEEL_ERR_CUDA, "capture stream creation failed");
    LaunchCountPause pause;
    const MphfLayout ml = mphf_layout(a.n, a.gamma_milli);
    char *pw = a.ws + ml.peel;
    const PeelLayout lay = peel_layout(a.n, a.m, 3);
    AsyncState *state = reinterpret_cast<AsyncState *>(a.ws + ml.state);
    Ctl *ctl = reinterpret_cast<Ctl *>(pw + lay.ctl);
    uint4 *rec = reinterpret_cast<uint4 *>(pw + lay.rec);
    unsigned long long *st = reinterpret_cast<unsigned long long *>(pw + lay.state);
    uint4 *Ll = reinterpret_cast<uint4 *>(pw + lay.L);
    uint32_t *loff = reinterpret_cast<uint32_t *>(pw + lay.loff);
    RoundParams *prm = reinterpret_cast<RoundParams *>(pw + lay.params);
    const uint32_t n = a.n, m = a.m, P = m / 3;
    const FastMod fm = make_fastmod(P);
    const uint64_t *seed_dev = &state->seed;
    Launch L0{s0, a.sms}, L1{s1, a.sms}, L2{s2, a.sms};
    RoundParams rp{};
    rp.st = st;
    rp.rec = rec;
    rp.L = Ll;
    rp.loff = loff;
    rp.ctl = ctl;
    rp.n = n;
    rp.m = m;
    rp.P = P;
    rp.max_rounds = lay.max_rounds;
    const RoundLaunch k0 = round0_launch(L0, 3, false), k1 = round_launch(L0, 3, false);

    // captures end in this order whatever fails, so no stream of ours stays
    // capturing (the caller's capture is left to the caller)
    int open = 0;
    const int first = into ? 1 : 0;
    cudaStream_t opened[3] = {s0, s1, s2};
    auto abort_all = [&](hpeel_status stt) {
        for (int i = open - 1; i >= first; i--) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(opened[i], &g);
            if (i == 0 && g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        return stt;
    };
#define HP_CAP(call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return abort_all(fail(HPEEL_ERR_CUDA, "graph capture: %s failed: %s", #call,   \
                                  cudaGetErrorString(e_)));                                \
    } while (0)
    auto begin_body = [&](cudaStream_t s, cudaGraph_t body) {
        return cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed);
    };

    if (!into) HP_CAP(cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
    open = 1;
    launch_set_params(L0, prm, rp);
    launch_async_init(L0, state, a.seed, a.max_tries, n);
    cudaGraphConditionalHandle h_out = 0, h_ovf = 0, h_red = 0, h_ok = 0, h_asg = 0;
    cudaGraph_t b_out = nullptr, b_ovf = nullptr, b_red = nullptr, b_ok = nullptr, b_asg = nullptr;
    HP_CAP(new_handle(s0, 1u, cudaGraphCondAssignDefault, &h_out));
    HP_CAP(append_conditional(s0, h_out, cudaGraphCondTypeWhile, &b_out));
    {   // one attempt (body of the loop over seeds)
        HP_CAP(begin_body(s1, b_out));
        open = 2;
        HP_CAP(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s1));
        if (lay.bucketed) {
            uint2 *pairs = reinterpret_cast<uint2 *>(pw + lay.pairs);
            uint32_t *fill = reinterpret_cast<uint32_t *>(pw + lay.fill);
            uint2 *pairs2 = reinterpret_cast<uint2 *>(pw + lay.pairs2);
            uint32_t *fill2 = reinterpret_cast<uint32_t *>(pw + lay.fill2);
            Overflow ov{reinterpret_cast<uint2 *>(pw + lay.ovf),
                        reinterpret_cast<uint32_t *>(pw + lay.ovf_count), lay.plan.ovf_cap};
            for (uint32_t pass = 0; pass < lay.plan.passes; pass++) {
                HP_CAP(cudaMemsetAsync(fill2, 0, 4 * (size_t)lay.plan.subs_pass, s1));
                HP_CAP(cudaMemsetAsync(ov.count, 0, 4, s1));
                launch_build_bucketed(L1, lay.plan, a.keys, nullptr, n, 3, fm, a.seed, P, rec,
                                      pairs, fill, ov, ctl, false, seed_dev, pass);
                launch_apply_buckets(L1, lay.plan, P, pairs, fill, pairs2, fill2, ov, st, ctl,
                                     pass,
                                     lay.sp.enabled
                                         ? ClaimSink{sorted_bufs(lay, pw).claims,
                                                     lay.sp.claim_cap, n}
                                         : ClaimSink{nullptr, 0, 0});
            }
            // an overflowed build is redone with direct updates (same result)
            HP_CAP(new_handle(s1, 0u, 0u, &h_ovf));
            launch_async_check_overflow(L1, ctl, h_ovf);
            HP_CAP(append_conditional(s1, h_ovf, cudaGraphCondTypeIf, &b_ovf));
            HP_CAP(begin_body(s2, b_ovf));
            open = 3;
            HP_CAP(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s2));
            launch_fill_u32(L2, reinterpret_cast<uint32_t *>(st), 2ull * m, 0u);
            launch_hash_records(L2, a.keys, n, 3, fm, a.seed, rec, seed_dev);
            launch_build_incidence(L2, rec, n, 3, m, st, ctl);
            cudaGraph_t g = nullptr;
            HP_CAP(cudaStreamEndCapture(s2, &g));
            open = 2;
        } else {
            launch_fill_u32(L1, reinterpret_cast<uint32_t *>(st), 2ull * m, 0u);
            launch_hash_records(L1, a.keys, n, 3, fm, a.seed, rec, seed_dev);
            launch_build_incidence(L1, rec, n, 3, m, st, ctl);
        }
        // round 0, then the loops of rounds (as launch_round_graph)
        RoundsArgs ra{n, m, 3, false, prm, lay.sp.enabled ? &lay.sp : nullptr,
                      lay.sp.enabled ? sorted_bufs(lay, pw) : SortedBufs{}, st, rec, Ll, loff,
                      ctl, lay.max_rounds};
        HP_CAP(capture_rounds(s1, s2, a.sms, ra));
        cudaGraph_t g = nullptr;
        if (ra.sp) {
            // a sorted round whose buckets overflowed (a skewed input): the
            // attempt's build and rounds are redone in random form
            HP_CAP(new_handle(s1, 0u, 0u, &h_red));
            launch_async_check_code(L1, ctl, kDevRoundOverflow, h_red);
            HP_CAP(append_conditional(s1, h_red, cudaGraphCondTypeIf, &b_red));
            HP_CAP(begin_body(s2, b_red));
            open = 3;
            HP_CAP(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s2));
            launch_fill_u32(L2, reinterpret_cast<uint32_t *>(st), 2ull * m, 0u);
            launch_hash_records(L2, a.keys, n, 3, fm, a.seed, rec, seed_dev);
            launch_build_incidence(L2, rec, n, 3, m, st, ctl);
            RoundsArgs rr = ra;
            rr.sp = nullptr;
            HP_CAP(capture_rounds(s2, s3, a.sms, rr));
            HP_CAP(cudaStreamEndCapture(s2, &g));
            open = 2;
        }
        launch_async_decide(L1, state, ctl, h_out);
        HP_CAP(cudaStreamEndCapture(s1, &g));
        open = 1;
    }
    HP_CAP(new_handle(s0, 0u, 0u, &h_ok));
    launch_async_if_peeled(L0, state, h_ok);
    HP_CAP(append_conditional(s0, h_ok, cudaGraphCondTypeIf, &b_ok));
    {   // assignment in reverse layer order, then the rank directory (MPHF)
        HP_CAP(begin_body(s1, b_ok));
        open = 2;
        const uint64_t words = ((uint64_t)m + 31) / 32, blocks = ((uint64_t)m + 511) / 512;
        if (a.values)
            HP_CAP(cudaMemsetAsync(a.U, 0, 8 * (((uint64_t)m * a.bits + 63) / 64), s1));
        else
            HP_CAP(cudaMemsetAsync(a.G, 0, 8 * words, s1));
        HP_CAP(new_handle(s1, 0u, 0u, &h_asg));
        launch_async_assign_init(L1, state, h_asg);
        HP_CAP(append_conditional(s1, h_asg, cudaGraphCondTypeWhile, &b_asg));
        HP_CAP(begin_body(s2, b_asg));
        open = 3;
        if (a.values)
            launch_sf_assign_layer_at(L2, Ll, loff, &state->t, a.values, a.sigma, a.bits, a.U,
                                      ctl);
        else
            launch_assign_layer_at(L2, Ll, loff, &state->t, P, a.G);
        launch_async_assign_step(L2, state, h_asg);
        cudaGraph_t g = nullptr;
        HP_CAP(cudaStreamEndCapture(s2, &g));
        open = 2;
        if (!a.values) {
            uint32_t *cnt = reinterpret_cast<uint32_t *>(a.ws + ml.rank_cnt);
            uint32_t *scn = reinterpret_cast<uint32_t *>(a.ws + ml.rank_scan);
            uint32_t *tmp = reinterpret_cast<uint32_t *>(a.ws + ml.rank_tmp);
            launch_rank_counts(L1, a.G, m, cnt);
            launch_scan_u32(L1, cnt, scn, blocks, tmp);
            launch_widen_dir(L1, scn, cnt, blocks, a.D);
        }
        HP_CAP(cudaStreamEndCapture(s1, &g));
        open = 1;
    }
    launch_async_stats(L0, state, ctl, a.stats);
    if (!into) HP_CAP(cudaStreamEndCapture(s0, out));
    open = 0;
#undef HP_CAP
    return HPEEL_OK;
}

// ---------------------------------------------------------------------------
// Device-driven peel: the whole of hpeel_peel as one CUDA graph -- the build
// (with the direct rebuild of an overflowed L2-blocked build in an if node),
// round 0 and the while node of rounds, then, when no device check failed,
// the canonical order with its passes in a while node, the layer offsets,
// and the stats in device memory.
// ---------------------------------------------------------------------------
struct AsyncPeelArgs {
    const uint32_t *edges;
    uint32_t n, m, r;
    bool general;
    uint32_t *order, *claim;
    uint64_t *layer_off;
    uint32_t max_layers;
    hpeel_stats *stats;
    char *ws;
    int sms;
};

hpeel_status capture_async_peel(const AsyncPeelArgs &a, cudaStream_t into, cudaGraph_t *out) {
    cudaStream_t s0 = into ? into : capture_stream(0), s1 = capture_stream(1),
                 s2 = capture_stream(2);
    if (!s0 || !s1 || !s2) return fail(HPEEL_ERR_CUDA, "capture stream creation failed");
    LaunchCountPause pause;
    const PeelLayout lay = peel_layout(a.n, a.m, a.r, a.general);
    char *ws = a.ws;
    Ctl *ctl = reinterpret_cast<Ctl *>(ws + lay.ctl);
    uint4 *rec = reinterpret_cast<uint4 *>(ws + lay.rec);
    unsigned long long *st = reinterpret_cast<unsigned long long *>(ws + lay.state);
    uint4 *Ll = reinterpret_cast<uint4 *>(ws + lay.L);
    uint32_t *loff = reinterpret_cast<uint32_t *>(ws + lay.loff);
    RoundParams *prm = reinterpret_cast<RoundParams *>(ws + lay.params);
    EmitState *es = reinterpret_cast<EmitState *>(ws + lay.emit);
    uint32_t *claim = a.claim ? a.claim : reinterpret_cast<uint32_t *>(ws + lay.claim);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + lay.hist);
    uint32_t *scantmp = reinterpret_cast<uint32_t *>(ws + lay.scantmp);
    // the edge records are dead once the claims are extracted: a later pass
    // of the order sort reads its inputs from their space
    uint32_t *tail = reinterpret_cast<uint32_t *>(rec);
    const uint32_t n = a.n, m = a.m, r = a.r, P = a.general ? m : m / r;
    Launch L0{s0, a.sms}, L1{s1, a.sms}, L2{s2, a.sms};
    RoundParams rp{};
    rp.st = st;
    rp.rec = rec;
    rp.L = Ll;
    rp.loff = loff;
    rp.ctl = ctl;
    rp.n = n;
    rp.m = m;
    rp.P = P;
    rp.max_rounds = lay.max_rounds;
    const RoundLaunch k0 = round0_launch(L0, r, a.general), k1 = round_launch(L0, r, a.general);

    int open = 0;
    const int first = into ? 1 : 0;
    cudaStream_t opened[3] = {s0, s1, s2};
    auto abort_all = [&](hpeel_status stt) {
        for (int i = open - 1; i >= first; i--) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(opened[i], &g);
            if (i == 0 && g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        return stt;
    };
#define HP_CAP(call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return abort_all(fail(HPEEL_ERR_CUDA, "graph capture: %s failed: %s", #call,   \
                                  cudaGetErrorString(e_)));                                \
    } while (0)
    auto begin_body = [&](cudaStream_t s, cudaGraph_t body) {
        return cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed);
    };

    if (!into) HP_CAP(cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
    open = 1;
    HP_CAP(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s0));
    launch_set_params(L0, prm, rp);
    cudaGraphConditionalHandle h_ovf = 0, h_red = 0, h_ok = 0, h_emit = 0;
    cudaGraph_t b_ovf = nullptr, b_red = nullptr, b_ok = nullptr, b_emit = nullptr;
    if (lay.bucketed) {
        uint2 *pairs = reinterpret_cast<uint2 *>(ws + lay.pairs);
        uint32_t *fill = reinterpret_cast<uint32_t *>(ws + lay.fill);
        uint2 *pairs2 = reinterpret_cast<uint2 *>(ws + lay.pairs2);
        uint32_t *fill2 = reinterpret_cast<uint32_t *>(ws + lay.fill2);
        Overflow ov{reinterpret_cast<uint2 *>(ws + lay.ovf),
                    reinterpret_cast<uint32_t *>(ws + lay.ovf_count), lay.plan.ovf_cap};
        for (uint32_t pass = 0; pass < lay.plan.passes; pass++) {
            HP_CAP(cudaMemsetAsync(fill2, 0, 4 * (size_t)lay.plan.subs_pass, s0));
            HP_CAP(cudaMemsetAsync(ov.count, 0, 4, s0));
            launch_build_bucketed(L0, lay.plan, nullptr, a.edges, n, r, FastMod{0, 0}, 0, P, rec,
                                  pairs, fill, ov, ctl, a.general, nullptr, pass);
            launch_apply_buckets(L0, lay.plan, P, pairs, fill, pairs2, fill2, ov, st, ctl, pass,
                                 lay.sp.enabled && !a.general
                                     ? ClaimSink{sorted_bufs(lay, ws).claims, lay.sp.claim_cap, n}
                                     : ClaimSink{nullptr, 0, 0});
        }
        // an overflowed build is redone with direct updates (same result)
        HP_CAP(new_handle(s0, 0u, 0u, &h_ovf));
        launch_async_check_overflow(L0, ctl, h_ovf);
        HP_CAP(append_conditional(s0, h_ovf, cudaGraphCondTypeIf, &b_ovf));
        HP_CAP(begin_body(s1, b_ovf));
        open = 2;
        HP_CAP(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s1));
        launch_fill_u32(L1, reinterpret_cast<uint32_t *>(st), 2ull * m, 0u);
        launch_records(L1, a.edges, n, r, P, rec, ctl, a.general);
        launch_build_incidence(L1, rec, n, r, m, st, ctl);
        cudaGraph_t g = nullptr;
        HP_CAP(cudaStreamEndCapture(s1, &g));
        open = 1;
    } else {
        launch_fill_u32(L0, reinterpret_cast<uint32_t *>(st), 2ull * m, 0u);
        launch_records(L0, a.edges, n, r, P, rec, ctl, a.general);
        launch_build_incidence(L0, rec, n, r, m, st, ctl);
    }
    // round 0, then the loops of rounds (as launch_round_graph)
    const bool sorted = lay.sp.enabled && !a.general;
    RoundsArgs ra{n, m, r, a.general, prm, sorted ? &lay.sp : nullptr,
                  sorted ? sorted_bufs(lay, ws) : SortedBufs{}, st, rec, Ll, loff, ctl,
                  lay.max_rounds};
    HP_CAP(capture_rounds(s0, s1, a.sms, ra));
    if (sorted) {
        // a sorted round whose buckets overflowed (a skewed input): the build
        // and the rounds are redone in random form
        HP_CAP(new_handle(s0, 0u, 0u, &h_red));
        launch_async_check_code(L0, ctl, kDevRoundOverflow, h_red);
        HP_CAP(append_conditional(s0, h_red, cudaGraphCondTypeIf, &b_red));
        HP_CAP(begin_body(s1, b_red));
        open = 2;
        HP_CAP(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s1));
        launch_fill_u32(L1, reinterpret_cast<uint32_t *>(st), 2ull * m, 0u);
        launch_records(L1, a.edges, n, r, P, rec, ctl, a.general);
        launch_build_incidence(L1, rec, n, r, m, st, ctl);
        RoundsArgs rr = ra;
        rr.sp = nullptr;
        HP_CAP(capture_rounds(s1, s2, a.sms, rr));
        cudaGraph_t g = nullptr;
        HP_CAP(cudaStreamEndCapture(s1, &g));
        open = 1;
    }
    // the canonical order, only when no device check failed
    HP_CAP(new_handle(s0, 0u, 0u, &h_ok));
    launch_async_if_ok(L0, ctl, h_ok);
    HP_CAP(append_conditional(s0, h_ok, cudaGraphCondTypeIf, &b_ok));
    {
        HP_CAP(begin_body(s1, b_ok));
        open = 2;
        HP_CAP(new_handle(s1, 0u, 0u, &h_emit));
        launch_emit_init(L1, ctl, n, es, h_emit);
        launch_extract_claim_hist_dev(L1, rec, n, r, claim, es, hist);
        HP_CAP(append_conditional(s1, h_emit, cudaGraphCondTypeWhile, &b_emit));
        HP_CAP(begin_body(s2, b_emit));
        open = 3;
        launch_emit_pass_dev(L2, n, tail, claim, es, hist, scantmp, a.order);
        launch_emit_advance(L2, es, loff, a.order, tail, h_emit);
        cudaGraph_t g = nullptr;
        HP_CAP(cudaStreamEndCapture(s2, &g));
        open = 2;
        if (a.layer_off) launch_layer_off_dev(L1, loff, ctl, a.max_layers, a.layer_off);
        HP_CAP(cudaStreamEndCapture(s1, &g));
        open = 1;
    }
    launch_peel_async_stats(L0, ctl, n, a.max_layers, a.layer_off != nullptr, a.stats);
    if (!into) HP_CAP(cudaStreamEndCapture(s0, out));
    open = 0;
#undef HP_CAP
    return HPEEL_OK;
}

}  // namespace

extern "C" {

const char *hpeel_status_str(hpeel_status s) {
    switch (s) {
    case HPEEL_OK: return "ok";
    case HPEEL_ERR_INVALID_ARG: return "invalid argument";
    case HPEEL_ERR_CUDA: return "CUDA error";
    case HPEEL_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case HPEEL_ERR_TIMEOUT: return "device wait timed out";
    case HPEEL_ERR_DEVICE_CHECK: return "device-side input check failed";
    case HPEEL_ERR_CORE_NONEMPTY: return "hypergraph has a non-empty 2-core";
    case HPEEL_ERR_RETRIES_EXHAUSTED: return "no hash seed gave a peelable hypergraph";
    case HPEEL_ERR_CAPACITY: return "capacity exceeded";
    }
    return "unknown status";
}

const char *hpeel_last_error(void) { return g_last_error.c_str(); }

hpeel_status hpeel_set_tuning(const hpeel_tuning *t) {
    g_last_error.clear();
    hpeel_tuning v = {22u, 8u << 20, 0u, 0u, 0u, 0u, {0, 0}};
    if (t) {
        if (t->bucket_shift < 8 || t->bucket_shift > 30)
            return fail(HPEEL_ERR_INVALID_ARG, "bucket_shift %u outside [8, 30]", t->bucket_shift);
        if (t->bucket_sub_shift > 14 || (t->bucket_sub_shift && t->bucket_sub_shift > t->bucket_shift))
            return fail(HPEEL_ERR_INVALID_ARG, "bucket_sub_shift %u: need 0 or at most "
                        "min(14, bucket_shift)", t->bucket_sub_shift);
        if (t->bucket_part_passes > 2)
            return fail(HPEEL_ERR_INVALID_ARG, "bucket_part_passes %u: 0, 1 or 2",
                        t->bucket_part_passes);
        v = *t;
    }
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    g_tuning = v;
    return HPEEL_OK;
}

void hpeel_get_tuning(hpeel_tuning *t) {
    if (t) *t = tuning();
}

int hpeel_version(void) { return 100; }

uint64_t hpeel_num_vertices(uint64_t n, uint32_t gamma_milli, uint32_t r) {
    if (r == 0) return 0;
    const uint64_t gn = (n * gamma_milli + 999u) / 1000u;  // ceil(gamma n)
    return (gn + r - 1) / r * r;
}

hpeel_status hpeel_hash_edges(const uint64_t *d_keys, uint64_t n, uint64_t m, uint32_t r,
                              uint64_t seed, uint32_t *d_edges, void *stream) {
    g_last_error.clear();
    if (r < 2 || r > 4) return fail(HPEEL_ERR_INVALID_ARG, "r = %u, need 2 <= r <= 4", r);
    if (n == 0) return HPEEL_OK;
    if (m == 0 || m % r != 0 || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "m = %llu must be a positive multiple of r below 2^32",
                    (unsigned long long)m);
    if (!d_keys || !d_edges) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    {
        ProfScope ps(L, "hash_edges");
        launch_hash_edges(L, d_keys, n, r, make_fastmod(m / r), seed, d_edges);
    }
    return check_launch("hash_edges");
}

hpeel_status hpeel_hash_edges_general(const uint64_t *d_keys, uint64_t n, uint64_t m,
                                      uint32_t r, uint64_t seed, uint32_t *d_edges,
                                      void *stream) {
    g_last_error.clear();
    if (r < 2 || r > 4) return fail(HPEEL_ERR_INVALID_ARG, "r = %u, need 2 <= r <= 4", r);
    if (n == 0) return HPEEL_OK;
    if (m == 0 || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "m = %llu must be positive and below 2^32",
                    (unsigned long long)m);
    if (!d_keys || !d_edges) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    {
        ProfScope ps(L, "hash_edges");
        launch_hash_edges(L, d_keys, n, r, make_fastmod(m), seed, d_edges, true);
    }
    return check_launch("hash_edges");
}

size_t hpeel_peel_workspace_size(uint64_t n, uint64_t m, uint32_t r) {
    return peel_layout(n, m, r).total;
}

}  // extern "C"

namespace {

// hpeel_peel and hpeel_peel_general: the same path, positions from the parts
// of an r-partite graph or from the rows of a general one.
hpeel_status peel_entry(bool general, const uint32_t *d_edges, uint64_t n, uint64_t m,
                        uint32_t r, uint32_t *d_order, uint32_t *d_claim, uint64_t *d_layer_off,
                        uint32_t max_layers, hpeel_stats *h_stats, void *d_ws, size_t ws_bytes,
                        void *stream) {
    g_last_error.clear();
    if (h_stats) memset(h_stats, 0, sizeof *h_stats);
    if (r < 2 || r > 4) return fail(HPEEL_ERR_INVALID_ARG, "r = %u, need 2 <= r <= 4", r);
    if (n >= (1ull << 32) || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "n and m must be below 2^32");
    if (general && n >= (1ull << 30))
        return fail(HPEEL_ERR_INVALID_ARG, "a general hypergraph needs n < 2^30");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    if (n == 0) {
        if (d_layer_off) HP_CUDA(cudaMemsetAsync(d_layer_off, 0, sizeof(uint64_t), L.stream));
        HP_CUDA(cudaStreamSynchronize(L.stream));
        return HPEEL_OK;
    }
    if (m == 0 || (!general && m % r != 0))
        return fail(HPEEL_ERR_INVALID_ARG, general ? "m must be positive"
                                                   : "m = %llu must be a positive multiple of r",
                    (unsigned long long)m);
    if (!d_edges || !d_order || !d_ws) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)d_ws & 255u) != 0)
        return fail(HPEEL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const size_t need = peel_layout(n, m, r, general).total;
    if (ws_bytes < need)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes, need);
    PeelOut po{};
    PeelIO io;
    io.edges = d_edges;
    io.order = d_order;
    io.claim = d_claim;
    io.general = general;
    HP_TRY(peel_core(L, io, (uint32_t)n, (uint32_t)m, r, (char *)d_ws, &po));
    if (d_layer_off) {
        if (po.rounds > max_layers)
            return fail(HPEEL_ERR_CAPACITY, "%u rounds > max_layers %u", po.rounds, max_layers);
        launch_layer_off(L, po.loff, po.rounds, d_layer_off);
        HP_TRY(check_launch("layer_off"));
    }
    HP_CUDA(cudaStreamSynchronize(L.stream));
    prof_flush();
    if (h_stats) {
        h_stats->n_peeled = po.n_peeled;
        h_stats->rounds = po.rounds;
        h_stats->core_nonempty = po.n_peeled < n;
        h_stats->first_layer = po.first_layer;
        h_stats->frontier = po.frontier;
        h_stats->hinge_moves = po.moves;
        h_stats->sorted_rounds = po.sorted_rounds;
    }
    return HPEEL_OK;
}

}  // namespace

extern "C" {

hpeel_status hpeel_peel(const uint32_t *d_edges, uint64_t n, uint64_t m, uint32_t r,
                        uint32_t *d_order, uint32_t *d_claim, uint64_t *d_layer_off,
                        uint32_t max_layers, hpeel_stats *h_stats, void *d_ws, size_t ws_bytes,
                        void *stream) {
    return peel_entry(false, d_edges, n, m, r, d_order, d_claim, d_layer_off, max_layers, h_stats,
                      d_ws, ws_bytes, stream);
}

size_t hpeel_peel_general_workspace_size(uint64_t n, uint64_t m, uint32_t r) {
    return peel_layout(n, m, r, true).total;
}

hpeel_status hpeel_peel_general(const uint32_t *d_edges, uint64_t n, uint64_t m, uint32_t r,
                                uint32_t *d_order, uint32_t *d_claim, uint64_t *d_layer_off,
                                uint32_t max_layers, hpeel_stats *h_stats, void *d_ws,
                                size_t ws_bytes, void *stream) {
    return peel_entry(true, d_edges, n, m, r, d_order, d_claim, d_layer_off, max_layers, h_stats,
                      d_ws, ws_bytes, stream);
}

}  // extern "C"

namespace {

hpeel_status peel_async_entry(bool general, const uint32_t *d_edges, uint64_t n, uint64_t m,
                              uint32_t r, uint32_t *d_order, uint32_t *d_claim,
                              uint64_t *d_layer_off, uint32_t max_layers, hpeel_stats *d_stats,
                              void *d_ws, size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (r < 2 || r > 4) return fail(HPEEL_ERR_INVALID_ARG, "r = %u, need 2 <= r <= 4", r);
    if (n >= (1ull << 32) || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "n and m must be below 2^32");
    if (general && n >= (1ull << 30))
        return fail(HPEEL_ERR_INVALID_ARG, "a general hypergraph needs n < 2^30");
    if (!d_stats) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    if (n == 0) {
        launch_peel_async_empty(L, d_stats, d_layer_off);
        return check_launch("peel_async_empty");
    }
    if (m == 0 || (!general && m % r != 0))
        return fail(HPEEL_ERR_INVALID_ARG, general ? "m must be positive"
                                                   : "m = %llu must be a positive multiple of r",
                    (unsigned long long)m);
    if (!d_edges || !d_order || !d_ws) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)d_ws & 255u) != 0)
        return fail(HPEEL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const size_t need = peel_layout(n, m, r, general).total;
    if (ws_bytes < need)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes, need);
    AsyncPeelArgs a{d_edges, (uint32_t)n, (uint32_t)m, r, general, d_order, d_claim,
                    d_layer_off, max_layers, d_stats, (char *)d_ws, L.sms};
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HP_CUDA(cudaStreamIsCapturing(L.stream, &cs));
    if (cs == cudaStreamCaptureStatusActive) {
        // the caller is capturing: the peel's nodes join the caller's graph
        std::lock_guard<std::mutex> lk(g_graph_mu);
        return capture_async_peel(a, L.stream, nullptr);
    }
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    const hpeel_tuning tu = tuning();
    char keybuf[320];
    snprintf(keybuf, sizeof keybuf, "peel|%d|%d|%p|%llu|%llu|%u|%p|%p|%p|%u|%p|%p|%u|%u|%u|%u|%d",
             dev, general ? 1 : 0, (const void *)d_edges, (unsigned long long)n,
             (unsigned long long)m, r, (void *)d_order, (void *)d_claim, (void *)d_layer_off,
             max_layers, (void *)d_stats, d_ws, tu.bucket_shift, tu.bucket_min_vertices,
             tu.bucket_sub_shift, tu.bucket_part_passes, L.sms);
    return launch_cached_graph(L, std::string(keybuf), [&](cudaGraph_t *g) {
        return capture_async_peel(a, nullptr, g);
    });
}

}  // namespace

extern "C" {

hpeel_status hpeel_peel_async(const uint32_t *d_edges, uint64_t n, uint64_t m, uint32_t r,
                              uint32_t *d_order, uint32_t *d_claim, uint64_t *d_layer_off,
                              uint32_t max_layers, hpeel_stats *d_stats, void *d_ws,
                              size_t ws_bytes, void *stream) {
    return peel_async_entry(false, d_edges, n, m, r, d_order, d_claim, d_layer_off, max_layers,
                            d_stats, d_ws, ws_bytes, stream);
}

hpeel_status hpeel_peel_general_async(const uint32_t *d_edges, uint64_t n, uint64_t m,
                                      uint32_t r, uint32_t *d_order, uint32_t *d_claim,
                                      uint64_t *d_layer_off, uint32_t max_layers,
                                      hpeel_stats *d_stats, void *d_ws, size_t ws_bytes,
                                      void *stream) {
    return peel_async_entry(true, d_edges, n, m, r, d_order, d_claim, d_layer_off, max_layers,
                            d_stats, d_ws, ws_bytes, stream);
}

size_t hpeel_mphf_workspace_size(uint64_t n, uint32_t gamma_milli) {
    return mphf_layout(n, gamma_milli).total;
}

hpeel_status hpeel_mphf_build(const uint64_t *d_keys, uint64_t n, uint64_t seed,
                              uint32_t gamma_milli, uint32_t max_tries, uint64_t *d_G,
                              uint64_t *d_rank_dir, uint32_t *d_order, hpeel_stats *h_stats,
                              void *d_ws, size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (h_stats) memset(h_stats, 0, sizeof *h_stats);
    if (gamma_milli == 0) return fail(HPEEL_ERR_INVALID_ARG, "gamma_milli must be positive");
    const MphfLayout lay = mphf_layout(n, gamma_milli);
    const uint64_t m = lay.m;
    if (n >= (1ull << 32) || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "n and m must be below 2^32");
    if (max_tries == 0) return fail(HPEEL_ERR_INVALID_ARG, "max_tries must be positive");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    const uint64_t blocks = (m + 511) / 512;
    if (n == 0) {
        if (d_rank_dir) HP_CUDA(cudaMemsetAsync(d_rank_dir, 0, sizeof(uint64_t), L.stream));
        HP_CUDA(cudaStreamSynchronize(L.stream));
        if (h_stats) h_stats->seed_used = seed;
        return HPEEL_OK;
    }
    if (!d_keys || !d_G || !d_rank_dir || !d_ws) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)d_ws & 255u) != 0)
        return fail(HPEEL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < lay.total)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes,
                    lay.total);
    char *ws = (char *)d_ws;
    const FastMod fm = make_fastmod(m / 3);
    for (uint32_t a = 0; a < max_tries; a++) {
        const uint64_t s = seed + a;
        PeelOut po{};
        PeelIO io;
        io.keys = d_keys;
        io.seed = s;
        io.fm = fm;
        io.order = d_order;
        HP_TRY(peel_core(L, io, (uint32_t)n, (uint32_t)m, 3, ws + lay.peel, &po));
        if (h_stats) {
            h_stats->attempts = a + 1;
            h_stats->rounds = po.rounds;
            h_stats->n_peeled = po.n_peeled;
            h_stats->core_nonempty = po.n_peeled < n;
            h_stats->first_layer = po.first_layer;
            h_stats->frontier = po.frontier;
        h_stats->hinge_moves = po.moves;
        h_stats->sorted_rounds = po.sorted_rounds;
        }
        if (po.n_peeled < n) continue;
        // The rounds are complete (the peel read their outcome back), so the
        // assignment and the rank directory run on a second stream beside the
        // order sort the peel left queued on the caller's stream: they share
        // no memory (layer list, layer table, G, rank scratch vs claim words,
        // sort scratch, order).
        SideStream *side = nullptr;
        HP_TRY(side_stream(&side));
        const Launch L2{side->stream, L.sms};
        // a8: reverse layer order
        const uint64_t words = (m + 31) / 32;
        HP_CUDA(cudaMemsetAsync(d_G, 0, 8 * words, L2.stream));
        for (int64_t t = (int64_t)po.rounds - 1; t >= 0; t--) {
            ProfScope ps(L2, "assign");
            launch_assign_layer(L2, po.list, po.loff, (uint32_t)t, (uint32_t)(m / 3), d_G);
        }
        HP_TRY(check_launch("assign"));
        // a9: rank directory
        uint32_t *cnt = reinterpret_cast<uint32_t *>(ws + lay.rank_cnt);
        uint32_t *scn = reinterpret_cast<uint32_t *>(ws + lay.rank_scan);
        uint32_t *tmp = reinterpret_cast<uint32_t *>(ws + lay.rank_tmp);
        {
            ProfScope ps(L2, "rank");
            launch_rank_counts(L2, d_G, m, cnt);
            launch_scan_u32(L2, cnt, scn, blocks, tmp);
            launch_widen_dir(L2, scn, cnt, blocks, d_rank_dir);
        }
        HP_TRY(check_launch("rank"));
        HP_CUDA(cudaEventRecord(side->done, L2.stream));
        HP_CUDA(cudaStreamWaitEvent(L.stream, side->done, 0));
        HP_CUDA(cudaStreamSynchronize(L.stream));
        prof_flush();
        if (h_stats) h_stats->seed_used = s;
        return HPEEL_OK;
    }
    return fail(HPEEL_ERR_RETRIES_EXHAUSTED, "2-core non-empty for seeds %llu..%llu",
                (unsigned long long)seed, (unsigned long long)(seed + max_tries - 1));
}

hpeel_status hpeel_mphf_build_async(const uint64_t *d_keys, uint64_t n, uint64_t seed,
                                    uint32_t gamma_milli, uint32_t max_tries, uint64_t *d_G,
                                    uint64_t *d_rank_dir, hpeel_stats *d_stats, void *d_ws,
                                    size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (gamma_milli == 0) return fail(HPEEL_ERR_INVALID_ARG, "gamma_milli must be positive");
    const MphfLayout lay = mphf_layout(n, gamma_milli);
    const uint64_t m = lay.m;
    if (n >= (1ull << 32) || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "n and m must be below 2^32");
    if (max_tries == 0) return fail(HPEEL_ERR_INVALID_ARG, "max_tries must be positive");
    if (!d_stats) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    if (n == 0) {
        launch_async_empty(L, d_stats, seed, d_rank_dir);
        return check_launch("async_empty");
    }
    if (!d_keys || !d_G || !d_rank_dir || !d_ws) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)d_ws & 255u) != 0)
        return fail(HPEEL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < lay.total)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes,
                    lay.total);
    AsyncArgs a{d_keys, (uint32_t)n, (uint32_t)m, max_tries, seed, gamma_milli,
                d_G, d_rank_dir, d_stats, (char *)d_ws, L.sms};
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HP_CUDA(cudaStreamIsCapturing(L.stream, &cs));
    if (cs == cudaStreamCaptureStatusActive) {
        // the caller is capturing: the build's nodes join the caller's graph
        std::lock_guard<std::mutex> lk(g_graph_mu);
        return capture_async_build(a, L.stream, nullptr);
    }
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    const hpeel_tuning tu = tuning();
    char keybuf[320];
    snprintf(keybuf, sizeof keybuf, "mphf|%d|%p|%llu|%llu|%u|%u|%p|%p|%p|%p|%u|%u|%u|%u|%d",
             dev, (const void *)d_keys, (unsigned long long)n, (unsigned long long)seed,
             gamma_milli, max_tries, (void *)d_G, (void *)d_rank_dir, (void *)d_stats, d_ws,
             tu.bucket_shift, tu.bucket_min_vertices, tu.bucket_sub_shift, tu.bucket_part_passes,
             L.sms);
    return launch_cached_graph(L, std::string(keybuf), [&](cudaGraph_t *g) {
        return capture_async_build(a, nullptr, g);
    });
}

uint32_t hpeel_sf_bits(uint64_t sigma) {
    uint32_t b = 0;
    while (b < 64 && (1ull << b) < sigma) b++;
    return b;
}

uint64_t hpeel_sf_words(uint64_t n, uint32_t gamma_milli, uint64_t sigma) {
    const uint64_t m = hpeel_num_vertices(n, gamma_milli, 3);
    return (m * hpeel_sf_bits(sigma) + 63) / 64;
}

// The static-function workspace has the MPHF's layout (the device-driven
// build keeps its loop state at the front); the rank arrays stay unused.
size_t hpeel_sf_workspace_size(uint64_t n, uint32_t gamma_milli) {
    return mphf_layout(n, gamma_milli).total;
}

hpeel_status hpeel_sf_build(const uint64_t *d_keys, const uint32_t *d_values, uint64_t n,
                            uint64_t sigma, uint64_t seed, uint32_t gamma_milli,
                            uint32_t max_tries, uint64_t *d_U, hpeel_stats *h_stats, void *d_ws,
                            size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (h_stats) memset(h_stats, 0, sizeof *h_stats);
    if (gamma_milli == 0) return fail(HPEEL_ERR_INVALID_ARG, "gamma_milli must be positive");
    if (sigma < 2 || sigma > (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "sigma = %llu, need 2 <= sigma <= 2^32",
                    (unsigned long long)sigma);
    const uint64_t m = hpeel_num_vertices(n, gamma_milli, 3);
    if (n >= (1ull << 32) || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "n and m must be below 2^32");
    if (max_tries == 0) return fail(HPEEL_ERR_INVALID_ARG, "max_tries must be positive");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    if (n == 0) {
        if (h_stats) h_stats->seed_used = seed;
        return HPEEL_OK;
    }
    if (!d_keys || !d_values || !d_U || !d_ws) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)d_ws & 255u) != 0)
        return fail(HPEEL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const MphfLayout ml = mphf_layout(n, gamma_milli);
    if (ws_bytes < ml.total)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes,
                    ml.total);
    char *ws = (char *)d_ws + ml.peel;
    const PeelLayout lay = peel_layout(n, m, 3);
    Ctl *ctl = reinterpret_cast<Ctl *>(ws + lay.ctl);
    const uint32_t b = hpeel_sf_bits(sigma);
    const uint64_t words = (m * b + 63) / 64;
    const FastMod fm = make_fastmod(m / 3);
    for (uint32_t a = 0; a < max_tries; a++) {
        const uint64_t s = seed + a;
        PeelOut po{};
        PeelIO io;
        io.keys = d_keys;
        io.seed = s;
        io.fm = fm;
        HP_TRY(peel_core(L, io, (uint32_t)n, (uint32_t)m, 3, ws, &po));
        if (h_stats) {
            h_stats->attempts = a + 1;
            h_stats->rounds = po.rounds;
            h_stats->n_peeled = po.n_peeled;
            h_stats->core_nonempty = po.n_peeled < n;
            h_stats->first_layer = po.first_layer;
            h_stats->frontier = po.frontier;
            h_stats->hinge_moves = po.moves;
        h_stats->sorted_rounds = po.sorted_rounds;
        }
        if (po.n_peeled < n) continue;
        // reverse layer order (sec. 3, sec. 4.3 "Avoiding backward scans")
        HP_CUDA(cudaMemsetAsync(d_U, 0, 8 * words, L.stream));
        for (int64_t t = (int64_t)po.rounds - 1; t >= 0; t--) {
            ProfScope ps(L, "sf_assign");
            launch_sf_assign_layer(L, po.list, po.loff, (uint32_t)t, d_values, sigma, b, d_U, ctl);
        }
        HP_TRY(check_launch("sf_assign"));
        uint32_t err = 0;
        HP_CUDA(cudaMemcpyAsync(&err, &ctl->err, sizeof err, cudaMemcpyDeviceToHost, L.stream));
        HP_CUDA(cudaStreamSynchronize(L.stream));
        prof_flush();
        if (err) {
            if (h_stats) h_stats->device_err = err;
            return fail(HPEEL_ERR_DEVICE_CHECK, "a value is not below sigma (device code %u)",
                        err);
        }
        if (h_stats) h_stats->seed_used = s;
        return HPEEL_OK;
    }
    return fail(HPEEL_ERR_RETRIES_EXHAUSTED, "2-core non-empty for seeds %llu..%llu",
                (unsigned long long)seed, (unsigned long long)(seed + max_tries - 1));
}

hpeel_status hpeel_sf_build_async(const uint64_t *d_keys, const uint32_t *d_values, uint64_t n,
                                  uint64_t sigma, uint64_t seed, uint32_t gamma_milli,
                                  uint32_t max_tries, uint64_t *d_U, hpeel_stats *d_stats,
                                  void *d_ws, size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (gamma_milli == 0) return fail(HPEEL_ERR_INVALID_ARG, "gamma_milli must be positive");
    if (sigma < 2 || sigma > (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "sigma = %llu, need 2 <= sigma <= 2^32",
                    (unsigned long long)sigma);
    const MphfLayout lay = mphf_layout(n, gamma_milli);
    const uint64_t m = lay.m;
    if (n >= (1ull << 32) || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "n and m must be below 2^32");
    if (max_tries == 0) return fail(HPEEL_ERR_INVALID_ARG, "max_tries must be positive");
    if (!d_stats) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    if (n == 0) {
        launch_async_empty(L, d_stats, seed, nullptr);
        return check_launch("async_empty");
    }
    if (!d_keys || !d_values || !d_U || !d_ws) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)d_ws & 255u) != 0)
        return fail(HPEEL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < lay.total)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes,
                    lay.total);
    AsyncArgs a{d_keys, (uint32_t)n, (uint32_t)m, max_tries, seed, gamma_milli,
                nullptr, nullptr, d_stats, (char *)d_ws, L.sms};
    a.values = d_values;
    a.sigma = sigma;
    a.bits = hpeel_sf_bits(sigma);
    a.U = d_U;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HP_CUDA(cudaStreamIsCapturing(L.stream, &cs));
    if (cs == cudaStreamCaptureStatusActive) {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        return capture_async_build(a, L.stream, nullptr);
    }
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    const hpeel_tuning tu = tuning();
    char keybuf[360];
    snprintf(keybuf, sizeof keybuf,
             "sf|%d|%p|%p|%llu|%llu|%llu|%u|%u|%p|%p|%p|%u|%u|%u|%u|%d", dev,
             (const void *)d_keys, (const void *)d_values, (unsigned long long)n,
             (unsigned long long)sigma, (unsigned long long)seed, gamma_milli, max_tries,
             (void *)d_U, (void *)d_stats, d_ws, tu.bucket_shift, tu.bucket_min_vertices,
             tu.bucket_sub_shift, tu.bucket_part_passes, L.sms);
    return launch_cached_graph(L, std::string(keybuf), [&](cudaGraph_t *g) {
        return capture_async_build(a, nullptr, g);
    });
}

hpeel_status hpeel_sf_lookup(const uint64_t *d_keys, uint64_t nq, uint64_t seed, uint64_t m,
                             uint64_t sigma, const uint64_t *d_U, uint32_t *d_out,
                             void *stream) {
    g_last_error.clear();
    if (nq == 0) return HPEEL_OK;
    if (m < 3 || m % 3 != 0 || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "m = %llu must be a positive multiple of 3 below 2^32",
                    (unsigned long long)m);
    if (sigma < 2 || sigma > (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "sigma = %llu, need 2 <= sigma <= 2^32",
                    (unsigned long long)sigma);
    if (!d_keys || !d_U || !d_out) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    ProfScope ps(L, "sf_lookup");
    launch_sf_lookup(L, d_keys, nq, make_fastmod(m / 3), seed, sigma, hpeel_sf_bits(sigma), d_U,
                     d_out);
    return check_launch("sf_lookup");
}

hpeel_status hpeel_mphf_lookup(const uint64_t *d_keys, uint64_t nq, uint64_t seed,
                               uint64_t m, const uint64_t *d_G, const uint64_t *d_rank_dir,
                               uint32_t *d_out, void *stream) {
    g_last_error.clear();
    if (nq == 0) return HPEEL_OK;
    if (m < 3 || m % 3 != 0 || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "m = %llu must be a positive multiple of 3 below 2^32",
                    (unsigned long long)m);
    if (!d_keys || !d_G || !d_rank_dir || !d_out) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    ProfScope ps(L, "lookup");
    launch_lookup(L, d_keys, nq, make_fastmod(m / 3), seed, d_G, d_rank_dir, d_out);
    return check_launch("lookup");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Peel without any allocation.
//
// Some callers cannot allocate device memory when they need a peel: code that
// runs inside another runtime's memory pool or arena (which hands out no raw
// cudaMalloc blocks), code under a strict memory budget that must not grow
// the device footprint at call time, or plugins loaded where calling the
// allocator is forbidden.  For them hpeel_peel_noalloc runs the same kernels
// as hpeel_peel with its scratch taken from a fixed array that is part of this
// library's device image instead of a caller workspace.
// ---------------------------------------------------------------------------
namespace {

// The built-in scratch: every GPU on which the library's kernels are loaded
// holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HPEEL_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch on the current device.  Host code cannot use
// the symbol itself (on the host it names a stand-in, not device memory), so
// the address is looked up with the device current.  It is looked up again on
// every call (a cheap query): a cached address would go stale if the
// device's context were torn down and the module loaded again.
hpeel_status noalloc_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        return fail(HPEEL_ERR_CUDA, "cudaGetSymbolAddress of the built-in scratch failed: %s",
                    cudaGetErrorString(e));
    *out = p;
    return HPEEL_OK;
}

}  // namespace

extern "C" hpeel_status hpeel_peel_noalloc(const uint32_t *d_edges, uint64_t n, uint64_t m,
                                           uint32_t r, uint32_t *d_order, uint32_t *d_claim,
                                           uint64_t *d_layer_off, uint32_t max_layers,
                                           hpeel_stats *h_stats, void *stream) {
    g_last_error.clear();
    if (h_stats) memset(h_stats, 0, sizeof *h_stats);
    if (r < 2 || r > 4) return fail(HPEEL_ERR_INVALID_ARG, "r = %u, need 2 <= r <= 4", r);
    if (n >= (1ull << 32) || m >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "n and m must be below 2^32");
    if (n > 0 && (m == 0 || m % r != 0))
        return fail(HPEEL_ERR_INVALID_ARG, "m = %llu must be a positive multiple of r",
                    (unsigned long long)m);
    const size_t need = n ? peel_layout(n, m, r).total : 0;
    if (need > (size_t)HPEEL_NOALLOC_SCRATCH_BYTES)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL,
                    "n = %llu, m = %llu needs %zu bytes of scratch; the built-in scratch holds "
                    "%zu bytes -- use hpeel_peel with a caller workspace",
                    (unsigned long long)n, (unsigned long long)m, need,
                    (size_t)HPEEL_NOALLOC_SCRATCH_BYTES);
    Launch L;
    HP_TRY(make_launch(stream, &L));
    void *scratch = nullptr;
    HP_TRY(noalloc_scratch(&scratch));
    if (n == 0) {
        if (d_layer_off) HP_CUDA(cudaMemsetAsync(d_layer_off, 0, sizeof(uint64_t), L.stream));
        HP_CUDA(cudaStreamSynchronize(L.stream));
        return HPEEL_OK;
    }
    if (!d_edges || !d_order) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    // Every value the peel reads from the scratch is written earlier in the
    // same call (the control block, the first layer/frontier offsets and the
    // vertex records are cleared first), so what a previous call left there
    // does not matter.  The control block is read back into ordinary host
    // memory, which needs no pinned allocation.
    // The rounds are launched from the host one by one (as with the tuning's
    // host_round_loop), never through the cached round-loop CUDA graph: a
    // graph is instantiated on first use, and the driver backs an executable
    // graph with device memory of its own.
    thread_local Ctl readback;
    PeelOut po{};
    PeelIO io;
    io.edges = d_edges;
    io.order = d_order;
    io.claim = d_claim;
    io.host_loop = true;
    HP_TRY(peel_core_rb(L, io, (uint32_t)n, (uint32_t)m, r, (char *)scratch, &po, &readback));
    if (d_layer_off) {
        if (po.rounds > max_layers)
            return fail(HPEEL_ERR_CAPACITY, "%u rounds > max_layers %u", po.rounds, max_layers);
        launch_layer_off(L, po.loff, po.rounds, d_layer_off);
        HP_TRY(check_launch("layer_off"));
    }
    HP_CUDA(cudaStreamSynchronize(L.stream));
    prof_flush();
    if (h_stats) {
        h_stats->n_peeled = po.n_peeled;
        h_stats->rounds = po.rounds;
        h_stats->core_nonempty = po.n_peeled < n;
        h_stats->first_layer = po.first_layer;
        h_stats->frontier = po.frontier;
        h_stats->hinge_moves = po.moves;
        h_stats->sorted_rounds = po.sorted_rounds;
    }
    return HPEEL_OK;
}

// ---------------------------------------------------------------------------
// MPHF build beyond 32-bit ids (large.cu): the paper's 7.6e9-key instance and
// larger, with the layer list optionally in pinned host memory.
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t kLargeRankSeg = 4096;  // as large.cu

struct LargeLayout {
    size_t ctl, params, st, claim, L, loff, cnt, seg, total;
    uint64_t m, blocks, nseg;
    uint32_t max_rounds;
};

LargeLayout large_layout(uint64_t n, uint32_t gamma_milli, bool list_on_host) {
    LargeLayout p{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    p.m = hpeel_num_vertices(n, gamma_milli, 3);
    p.max_rounds = (uint32_t)std::min<uint64_t>(HPEEL_MAX_ROUNDS, n + 1);
    p.blocks = (p.m + 511) / 512;
    p.nseg = (p.blocks + kLargeRankSeg - 1) / kLargeRankSeg;
    p.ctl = take(sizeof(LargeCtl));
    p.params = take(sizeof(LargeParams));
    p.st = take(8 * p.m);
    p.claim = take(4 * n);
    p.L = take(list_on_host ? 0 : 8 * n);
    p.loff = take(8 * ((size_t)p.max_rounds + 3));
    p.cnt = take(4 * p.blocks + 4);
    p.seg = take(8 * (p.nseg + 1));
    p.total = off;
    return p;
}

// Round 0 and the while node over the round kernel (the kernels' last
// blocks set its condition), captured at the capture position of s0.
cudaError_t capture_large_rounds(cudaStream_t s0, cudaStream_t s1, int sms,
                                 const LargeParams *prm) {
    Launch L0{s0, sms};
    const RoundLaunch k0 = large_round_launch(L0, true), k1 = large_round_launch(L0, false);
    cudaGraphConditionalHandle h = 0;
    cudaError_t e = new_handle(s0, 0u, 0u, &h);
    if (e != cudaSuccess) return e;
    {
        void *args[] = {(void *)&prm, &h};
        e = cudaLaunchKernel(k0.fn, dim3(k0.grid), dim3(k0.block), args, 0, s0);
        if (e != cudaSuccess) return e;
    }
    cudaGraph_t body = nullptr, g = nullptr;
    e = append_conditional(s0, h, cudaGraphCondTypeWhile, &body);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    {
        void *args[] = {(void *)&prm, &h};
        e = cudaLaunchKernel(k1.fn, dim3(k1.grid), dim3(k1.block), args, 0, s1);
    }
    const cudaError_t e2 = cudaStreamEndCapture(s1, &g);
    return e != cudaSuccess ? e : e2;
}

LargeCtl *pinned_large_ctl() {
    thread_local LargeCtl *p = nullptr;
    if (!p && cudaMallocHost((void **)&p, sizeof(LargeCtl)) != cudaSuccess) p = nullptr;
    return p;
}

}  // namespace

extern "C" {

size_t hpeel_mphf_large_workspace_size(uint64_t n, uint32_t gamma_milli, int list_on_host) {
    return large_layout(n, gamma_milli ? gamma_milli : 1230, list_on_host != 0).total;
}

hpeel_status hpeel_mphf_build_large(const uint64_t *d_keys, uint64_t n, uint64_t seed,
                                    uint32_t gamma_milli, uint32_t max_tries, uint64_t *d_G,
                                    uint64_t *d_rank_dir, hpeel_stats *h_stats, void *d_ws,
                                    size_t ws_bytes, uint64_t *h_list, void *stream) {
    g_last_error.clear();
    if (h_stats) memset(h_stats, 0, sizeof *h_stats);
    if (gamma_milli == 0) return fail(HPEEL_ERR_INVALID_ARG, "gamma_milli must be positive");
    if (max_tries == 0) return fail(HPEEL_ERR_INVALID_ARG, "max_tries must be positive");
    const LargeLayout lay = large_layout(n, gamma_milli, h_list != nullptr);
    const uint64_t m = lay.m, P = m / 3;
    if (P >= (1ull << 32) || n >= (1ull << 40))
        return fail(HPEEL_ERR_INVALID_ARG,
                    "n = %llu: a part of m / 3 vertices needs ids below 2^32",
                    (unsigned long long)n);
    Launch L;
    HP_TRY(make_launch(stream, &L));
    if (n == 0) {
        if (d_rank_dir) HP_CUDA(cudaMemsetAsync(d_rank_dir, 0, sizeof(uint64_t), L.stream));
        HP_CUDA(cudaStreamSynchronize(L.stream));
        if (h_stats) h_stats->seed_used = seed;
        return HPEEL_OK;
    }
    if (!d_keys || !d_G || !d_rank_dir || !d_ws) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)d_ws & 255u) != 0)
        return fail(HPEEL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < lay.total)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes,
                    lay.total);
    if (h_list) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, h_list) != cudaSuccess ||
            pa.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return fail(HPEEL_ERR_INVALID_ARG,
                        "h_list must be page-locked host memory (cudaHostAlloc, "
                        "cudaMallocHost or cudaHostRegister)");
        }
    }
    LargeCtl *hctl = pinned_large_ctl();
    if (!hctl) return fail(HPEEL_ERR_CUDA, "cudaMallocHost of the control read-back failed");
    char *ws = (char *)d_ws;
    LargeCtl *ctl = reinterpret_cast<LargeCtl *>(ws + lay.ctl);
    LargeParams *prm = reinterpret_cast<LargeParams *>(ws + lay.params);
    unsigned long long *st = reinterpret_cast<unsigned long long *>(ws + lay.st);
    uint32_t *claim = reinterpret_cast<uint32_t *>(ws + lay.claim);
    unsigned long long *Ll =
        h_list ? reinterpret_cast<unsigned long long *>(h_list)
               : reinterpret_cast<unsigned long long *>(ws + lay.L);
    unsigned long long *loff = reinterpret_cast<unsigned long long *>(ws + lay.loff);
    const FastMod fm = make_fastmod(P);
    const hpeel_tuning tu = tuning();
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    for (uint32_t a = 0; a < max_tries; a++) {
        const uint64_t s = seed + a;
        HP_CUDA(cudaMemsetAsync(ctl, 0, sizeof(LargeCtl), L.stream));
        {
            ProfScope ps(L, "large_build");
            launch_fill_u32(L, reinterpret_cast<uint32_t *>(st), 2 * m, 0u);
            launch_large_build(L, d_keys, n, s, fm, st, claim, ctl);
        }
        LargeParams lp{st, claim, Ll, loff, ctl, d_keys, n, m, s, fm, lay.max_rounds};
        launch_large_set_params(L, prm, lp);
        HP_TRY(check_launch("large build"));
        {
            ProfScope ps(L, "large_rounds");
            if (tu.host_round_loop) {
                const RoundLaunch k0 = large_round_launch(L, true), k1 = large_round_launch(L, false);
                cudaGraphConditionalHandle c0 = 0;
                void *args[] = {(void *)&prm, &c0};
                count_launch();
                HP_CUDA(cudaLaunchKernel(k0.fn, dim3(k0.grid), dim3(k0.block), args, 0, L.stream));
                HP_CUDA(cudaMemcpyAsync(hctl, ctl, sizeof(LargeCtl), cudaMemcpyDeviceToHost, L.stream));
                HP_CUDA(cudaStreamSynchronize(L.stream));
                while (hctl->more && !hctl->err) {
                    count_launch();
                    HP_CUDA(cudaLaunchKernel(k1.fn, dim3(k1.grid), dim3(k1.block), args, 0,
                                             L.stream));
                    HP_CUDA(cudaMemcpyAsync(hctl, ctl, sizeof(LargeCtl), cudaMemcpyDeviceToHost,
                                            L.stream));
                    HP_CUDA(cudaStreamSynchronize(L.stream));
                }
            } else {
                char keybuf[160];
                snprintf(keybuf, sizeof keybuf, "large|%d|%p|%d", dev, (const void *)prm, L.sms);
                HP_TRY(launch_cached_graph(L, std::string(keybuf), [&](cudaGraph_t *g) -> hpeel_status {
                    cudaStream_t s0 = capture_stream(0), s1 = capture_stream(1);
                    if (!s0 || !s1) return fail(HPEEL_ERR_CUDA, "capture stream creation failed");
                    LaunchCountPause pause;
                    cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed);
                    if (e == cudaSuccess) {
                        e = capture_large_rounds(s0, s1, L.sms, prm);
                        cudaGraph_t got = nullptr;
                        const cudaError_t e2 = cudaStreamEndCapture(s0, &got);
                        if (e == cudaSuccess) e = e2;
                        if (e == cudaSuccess) {
                            *g = got;
                            return HPEEL_OK;
                        }
                        if (got) cudaGraphDestroy(got);
                    }
                    cudaGetLastError();
                    return fail(HPEEL_ERR_CUDA, "large round graph: %s", cudaGetErrorString(e));
                }));
                HP_CUDA(cudaMemcpyAsync(hctl, ctl, sizeof(LargeCtl), cudaMemcpyDeviceToHost, L.stream));
                HP_CUDA(cudaStreamSynchronize(L.stream));
                count_launch(1 + hctl->round + (hctl->more ? 1 : 0));
            }
        }
        if (hctl->err == kDevCapacity)
            return fail(HPEEL_ERR_CAPACITY, "more than %u rounds", lay.max_rounds - 1);
        if (hctl->err == kDevDegree)
            return fail(HPEEL_ERR_CAPACITY, "a vertex has degree 2^24 or more");
        if (hctl->err)
            return fail(HPEEL_ERR_DEVICE_CHECK, "device check failed with code %u", hctl->err);
        const uint32_t R = hctl->more ? hctl->round + 1 : hctl->round;
        if (h_stats) {
            h_stats->attempts = a + 1;
            h_stats->rounds = R;
            h_stats->n_peeled = hctl->lcur;
            h_stats->core_nonempty = hctl->lcur < n;
            h_stats->first_layer = hctl->first_layer;
            h_stats->frontier = hctl->cross;
        }
        if (hctl->lcur < n) continue;
        // a8: reverse layer order; a9: rank directory (64-bit counts)
        {
            ProfScope ps(L, "large_assign");
            HP_CUDA(cudaMemsetAsync(d_G, 0, 8 * ((m + 31) / 32), L.stream));
            for (int64_t t = (int64_t)R - 1; t >= 0; t--) launch_large_assign(L, prm, (uint32_t)t, d_G);
        }
        {
            ProfScope ps(L, "large_rank");
            launch_large_rank(L, d_G, m, reinterpret_cast<uint32_t *>(ws + lay.cnt),
                              reinterpret_cast<unsigned long long *>(ws + lay.seg), d_rank_dir);
        }
        HP_TRY(check_launch("large assign"));
        HP_CUDA(cudaStreamSynchronize(L.stream));
        prof_flush();
        if (h_stats) h_stats->seed_used = s;
        return HPEEL_OK;
    }
    return fail(HPEEL_ERR_RETRIES_EXHAUSTED, "2-core non-empty for seeds %llu..%llu",
                (unsigned long long)seed, (unsigned long long)(seed + max_tries - 1));
}

hpeel_status hpeel_mphf_lookup_large(const uint64_t *d_keys, uint64_t nq, uint64_t seed,
                                     uint64_t m, const uint64_t *d_G, const uint64_t *d_rank_dir,
                                     uint64_t *d_out, void *stream) {
    g_last_error.clear();
    if (nq == 0) return HPEEL_OK;
    if (m < 3 || m % 3 != 0 || m / 3 >= (1ull << 32))
        return fail(HPEEL_ERR_INVALID_ARG, "m = %llu must be a positive multiple of 3 with "
                    "m / 3 below 2^32", (unsigned long long)m);
    if (!d_keys || !d_G || !d_rank_dir || !d_out) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    Launch L;
    HP_TRY(make_launch(stream, &L));
    ProfScope ps(L, "large_lookup");
    launch_large_lookup(L, d_keys, nq, make_fastmod(m / 3), seed, d_G, d_rank_dir, d_out);
    return check_launch("large_lookup");
}

}  // extern "C"
