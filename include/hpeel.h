/*
 * hpeel.h -- C ABI of the GB300 (sm_103a) hypergraph peeling and MWHC
 * minimal-perfect-hash library.
 *
 * The operations follow "Cache-Oblivious Peeling of Random Hypergraphs"
 * (Belazzougui, Boldi, Ottaviano, Venturini, Vigna):
 *   - peeling order and 2-core ................. sec. 1 (Introduction)
 *   - hash functions, MWHC system, MPHF ........ sec. 3 (MWHC technique)
 *   - packed incidence lists (XOR trick) ....... sec. 4.1
 *   - layered (round-synchronous) peeling ...... sec. 4.2
 *   - r-partite hashing, reverse-layer assign .. sec. 4.3
 *   - broadword rank ........................... sec. 5
 *
 * Conventions for every call:
 *   - Pointers named d_* are device memory owned by the caller; the library
 *     never frees or keeps them after the call returns.  h_* pointers are
 *     host memory owned by the caller.
 *   - Work is issued on the caller's CUDA stream (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream).  Calls that decide on the
 *     host (how many rounds, whether to retry) synchronise that stream
 *     before returning and write their stats to host memory; each of them
 *     has an *_async form that decides on the device instead (stats in
 *     device memory, no synchronisation, capturable into a CUDA graph).
 *   - Scratch memory is a caller-provided workspace d_ws of at least the
 *     size the matching *_workspace_size() function returns, 256-byte
 *     aligned.  The library never calls cudaMalloc: every array of a call
 *     lives in the caller's buffers.  Two things still take device memory
 *     from the driver: loading the library's device code (on the first call
 *     on a device), and the CUDA graphs the library instantiates and caches
 *     for its device-side loops (the round loop of the default tuning, the
 *     device-driven calls), which the driver backs with memory of its own.
 *     hpeel_peel_noalloc uses neither kind of graph.
 *   - Every call returns an hpeel_status; no C++ exception crosses the ABI.
 *     On failure hpeel_last_error() (per host thread) holds a message.
 *   - Edge ids and vertex ids are uint32: n < 2^32 and m < 2^32, except in
 *     the *_large calls (64-bit ids, for key sets like the paper's 7.6e9).
 *   - All results are exact and deterministic: the same inputs give the
 *     same bytes on every run and in every launch configuration.
 */
#ifndef HPEEL_H
#define HPEEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hpeel_status {
    HPEEL_OK = 0,
    HPEEL_ERR_INVALID_ARG = 1,        /* bad size, NULL or misaligned pointer */
    HPEEL_ERR_CUDA = 2,               /* a CUDA runtime call failed */
    HPEEL_ERR_WORKSPACE_TOO_SMALL = 3,
    HPEEL_ERR_TIMEOUT = 4,            /* a bounded device-side wait gave up */
    HPEEL_ERR_DEVICE_CHECK = 5,       /* a kernel found an invalid input */
    HPEEL_ERR_CORE_NONEMPTY = 6,      /* MPHF: the hypergraph did not peel */
    HPEEL_ERR_RETRIES_EXHAUSTED = 7,  /* MPHF: no seed tried gave a peel */
    HPEEL_ERR_CAPACITY = 8            /* more rounds than the library supports */
} hpeel_status;

/* Per-call results, written to host memory by the calls that take one. */
typedef struct hpeel_stats {
    uint64_t n_peeled;      /* edges in the peeling order (sum of layer sizes) */
    uint32_t rounds;        /* R: number of non-empty layers */
    uint32_t core_nonempty; /* 1 if n_peeled < n (a 2-core is left) */
    uint64_t seed_used;     /* MPHF: hash seed of the successful attempt */
    uint32_t attempts;      /* MPHF: hash seeds tried */
    uint32_t device_err;    /* non-zero: code a kernel raised (see status) */
    uint64_t first_layer;   /* |L_0|: edges peeled in round 0 */
    uint64_t frontier;      /* vertices that fell from degree 2 to 1 in some
                               round (the frontiers F_1, F_2, ...) */
    uint64_t hinge_moves;   /* peeled edges whose first claim came from a
                               vertex other than the hinge (a vertex of
                               smaller position claimed later in the round) */
    uint32_t async_status;  /* the *_async calls: 1 done (outputs written),
                               2 no seed peeled (builds), 3 device check
                               failed (device_err holds the code), 4 more
                               rounds than max_layers (peels) */
    uint32_t sorted_rounds; /* rounds whose layer was deleted in sorted form
                               (see the tuning's sorted_round_min) */
    uint64_t reserved;
} hpeel_stats;

/* Largest number of rounds a single peel supports (claim words keep the
 * round in 30 bits; the layer tables are sized to this bound). */
#define HPEEL_MAX_ROUNDS (1u << 20)
/* Claim word of an edge that was not peeled (a 2-core edge). */
#define HPEEL_UNCLAIMED 0xFFFFFFFFu

/*
 * Tuning knobs (process-wide; no counterpart in the paper -- they pick among
 * equivalent schedules and never change a result).
 *   bucket_shift        log2 of the vertices per chunk of the L2-blocked
 *                       incidence build (default 22: 32 MiB of vertex
 *                       records per chunk, about a quarter of GB300's L2).
 *   bucket_min_vertices graphs with at least this many vertices use the
 *                       L2-blocked build (default 8 Mi); smaller ones update
 *                       the vertex records directly.
 *   host_round_loop     0 (default): the rounds run back to back on the
 *                       device (a CUDA graph whose while node repeats the
 *                       round kernel until a layer is empty); 1: the host
 *                       launches every round and reads the round's outcome
 *                       back before the next.
 *   bucket_sub_shift    log2 of the vertices one block accumulates in shared
 *                       memory in the L2-blocked build (0 = automatic:
 *                       min(13, bucket_shift - 9); at most 14).
 *   bucket_part_passes  0 (default): automatic -- r-partite graphs of more
 *                       than 2^30 edges run the L2-blocked build once per
 *                       part (sec. 4.3: one part at a time), so its buckets
 *                       hold one incidence per edge instead of r and the
 *                       workspace shrinks by about 2 x 16 (r - 1) bytes per
 *                       edge; 1: all parts in one pass; 2: one part per pass
 *                       (general graphs always take one pass).
 *   sorted_round_min    rounds whose layer holds at least this many edges
 *                       run in sorted form (sec. 4.2's sorting of the
 *                       orientations by edge and of the updates by vertex,
 *                       with shared memory as the fast tier) instead of with
 *                       atomics at random addresses -- the first rounds, until
 *                       one is smaller; 0 (default): automatic, n / 20, for
 *                       r = 3 r-partite graphs whose incidence build is
 *                       L2-blocked in one pass; 0xFFFFFFFF: never.  Results
 *                       are the same either way.
 * hpeel_set_tuning(NULL) restores the defaults.  Workspace sizes depend on
 * the tuning: query them after setting it.  Errors: HPEEL_ERR_INVALID_ARG.
 */
typedef struct hpeel_tuning {
    uint32_t bucket_shift;
    uint32_t bucket_min_vertices;
    uint32_t host_round_loop;
    uint32_t bucket_sub_shift;
    uint32_t bucket_part_passes;
    uint32_t sorted_round_min;
    uint32_t reserved[2];
} hpeel_tuning;
hpeel_status hpeel_set_tuning(const hpeel_tuning *t);
void hpeel_get_tuning(hpeel_tuning *t);

/* Static description of a status code. */
const char *hpeel_status_str(hpeel_status s);
/* Message of the last failure on this host thread ("" if none). */
const char *hpeel_last_error(void);
/* ABI version: major * 10000 + minor * 100 + patch. */
int hpeel_version(void);

/*
 * Number of vertices m for n edges at sparsity gamma = gamma_milli / 1000,
 * r-partite: m = r * ceil(ceil(gamma n) / r)  (sec. 3: gamma n vertices;
 * sec. 4.3: r equal parts).  Returns 0 for n == 0.  Pure host function.
 */
uint64_t hpeel_num_vertices(uint64_t n, uint32_t gamma_milli, uint32_t r);

/*
 * Key -> edge hashing (sec. 3 hash functions h_0..h_{r-1}; sec. 4.3 each h_j
 * maps into its own part [j m/r, (j+1) m/r)).
 *   d_keys  [n] uint64 keys.
 *   d_edges [n][r] uint32 output, row-major: d_edges[i*r + j] =
 *           (mix64(key_i ^ (seed + j)) mod (m/r)) + j*(m/r), mix64 being the
 *           SplitMix64 output function.
 *   2 <= r <= 4, m a positive multiple of r, m < 2^32.
 * Asynchronous on stream.  Errors: HPEEL_ERR_INVALID_ARG, HPEEL_ERR_CUDA.
 */
hpeel_status hpeel_hash_edges(const uint64_t *d_keys, uint64_t n, uint64_t m,
                              uint32_t r, uint64_t seed, uint32_t *d_edges,
                              void *stream);

/* General (not r-partite) form: d_edges[i*r + j] = mix64(key_i ^ (seed + j))
 * mod m, any vertex in any position (rows may repeat a vertex); 0 < m < 2^32.
 * For hpeel_peel_general.  Asynchronous on stream.  Errors as above. */
hpeel_status hpeel_hash_edges_general(const uint64_t *d_keys, uint64_t n, uint64_t m,
                                      uint32_t r, uint64_t seed, uint32_t *d_edges,
                                      void *stream);

/* Workspace bytes hpeel_peel needs for (n, m, r). */
size_t hpeel_peel_workspace_size(uint64_t n, uint64_t m, uint32_t r);

/*
 * Round-synchronous peel of an r-partite r-hypergraph (sec. 4.2, with the
 * packed incidence lists of sec. 4.1).  Round t removes every edge that has
 * a vertex of degree 1 in the graph left by rounds 0..t-1; an edge reached
 * from several degree-1 vertices is removed once.
 *   d_edges     [n][r] uint32, vertex j of every edge in [j m/r, (j+1) m/r)
 *               (what hpeel_hash_edges produces).  Not modified.
 *   d_order     [n] uint32 output: the canonical order -- layer 0 in
 *               ascending edge id, then layer 1 ascending, ..., then the
 *               2-core edges (not peeled) in ascending id.  The first
 *               n_peeled entries are a peeling order (sec. 1).
 *   d_claim     [n] uint32 output or NULL: (round << 2) | hinge for a peeled
 *               edge, hinge = smallest position j whose vertex had degree 1
 *               in that round; HPEEL_UNCLAIMED for a 2-core edge.
 *   d_layer_off [max_layers + 1] uint64 output or NULL: start of layer t in
 *               d_order for t < R, then n_peeled at index R.
 *   h_stats     host output or NULL: n_peeled, rounds, core_nonempty.
 *   2 <= r <= 4.  n = 0 is valid (empty order, no round).
 * Synchronises stream (the number of rounds is decided on the device and
 * read back); hpeel_peel_async is the form without a host round trip.
 * Errors: HPEEL_ERR_INVALID_ARG, HPEEL_ERR_WORKSPACE_TOO_SMALL,
 * HPEEL_ERR_CAPACITY (R > max_layers or R > HPEEL_MAX_ROUNDS, or a vertex
 * of degree 2^31 or more),
 * HPEEL_ERR_DEVICE_CHECK (a vertex id outside its part), HPEEL_ERR_CUDA.
 */
hpeel_status hpeel_peel(const uint32_t *d_edges, uint64_t n, uint64_t m,
                        uint32_t r, uint32_t *d_order, uint32_t *d_claim,
                        uint64_t *d_layer_off, uint32_t max_layers,
                        hpeel_stats *h_stats, void *d_ws, size_t ws_bytes,
                        void *stream);

/*
 * Round-synchronous peel of a general r-hypergraph: the same call as
 * hpeel_peel without the r-partite structure (sec. 2: an edge is any
 * r-subset of the vertex set; sec. 3's hash functions h_j map into all of
 * [gamma n]).
 *   d_edges  [n][r] uint32, every vertex below m, in any position; a row may
 *            repeat a vertex (its degree counts occurrences, so such a vertex
 *            can only leave with its edge through another vertex).
 *   The position of a degree-1 vertex in its edge is read off the edge's
 *   row; the hinge is again the smallest such position, so d_claim holds
 *   (round << 2) | position in the row.  m is any positive value below 2^32.
 *   n < 2^30 (the layer list keeps the hinge position in the top two bits of
 *   an edge id).  Other arguments, results and errors: as hpeel_peel, with
 *   HPEEL_ERR_DEVICE_CHECK for a vertex >= m.
 */
size_t hpeel_peel_general_workspace_size(uint64_t n, uint64_t m, uint32_t r);
hpeel_status hpeel_peel_general(const uint32_t *d_edges, uint64_t n, uint64_t m,
                                uint32_t r, uint32_t *d_order, uint32_t *d_claim,
                                uint64_t *d_layer_off, uint32_t max_layers,
                                hpeel_stats *h_stats, void *d_ws, size_t ws_bytes,
                                void *stream);

/*
 * hpeel_peel with no host round trip: the whole peel -- records, incidence
 * build, round 0 and the rounds (sec. 4.2, a while loop on the device),
 * the canonical order with as many passes of its sort as the rounds need,
 * the layer offsets -- is enqueued on stream as one CUDA graph, and the call
 * returns at once.  It can be captured into a caller's CUDA graph or
 * overlapped with other work on other streams.  hpeel_peel is its
 * synchronous form (same results, stats on the host).
 *   Arguments as hpeel_peel, except:
 *   d_stats   device memory (not host), written at the end of the graph:
 *             async_status 1 = peeled (d_order, d_claim and d_layer_off
 *             written; n_peeled, rounds, core_nonempty, first_layer,
 *             frontier, hinge_moves as hpeel_peel gives them), 3 = a device
 *             check failed (device_err holds the code: 1 a vertex outside its
 *             part, 3 more rounds than HPEEL_MAX_ROUNDS, 6 a vertex of degree
 *             2^31 or more; nothing else written), 4 = more rounds than
 *             max_layers (d_order and d_claim written, d_layer_off not).
 * The graph is built on the first call with a given set of pointers and
 * sizes and replayed by later calls with the same set (keep the workspace and
 * the output buffers to reuse it; the inputs' contents may change between
 * calls).  Returns HPEEL_OK once enqueued; errors found on the host:
 * HPEEL_ERR_INVALID_ARG, HPEEL_ERR_WORKSPACE_TOO_SMALL, HPEEL_ERR_CUDA.  When
 * stream is being captured (cudaStreamBeginCapture), the peel's nodes join
 * the caller's graph at the capture position instead.
 */
hpeel_status hpeel_peel_async(const uint32_t *d_edges, uint64_t n, uint64_t m, uint32_t r,
                              uint32_t *d_order, uint32_t *d_claim, uint64_t *d_layer_off,
                              uint32_t max_layers, hpeel_stats *d_stats, void *d_ws,
                              size_t ws_bytes, void *stream);

/* hpeel_peel_general with no host round trip: as hpeel_peel_async, for a
 * general r-hypergraph (arguments, results and limits of hpeel_peel_general;
 * device_err 1 for a vertex >= m).  Workspace:
 * hpeel_peel_general_workspace_size. */
hpeel_status hpeel_peel_general_async(const uint32_t *d_edges, uint64_t n, uint64_t m,
                                      uint32_t r, uint32_t *d_order, uint32_t *d_claim,
                                      uint64_t *d_layer_off, uint32_t max_layers,
                                      hpeel_stats *d_stats, void *d_ws, size_t ws_bytes,
                                      void *stream);

/*
 * hpeel_peel without any allocation./*
 * hpeel_peel without any allocation.  The paper has no counterpart: this is
 * a calling convenience of this library.
 *
 * For callers that cannot allocate device memory at the time they need a
 * peel -- code running inside another runtime's memory pool or arena, code
 * under a fixed memory budget, plugins where calling the allocator is not
 * allowed.  Same arguments, results and errors as hpeel_peel, without the
 * workspace: the scratch is an array of HPEEL_NOALLOC_SCRATCH_BYTES compiled
 * into this library's device image.  Every GPU on which the library's device
 * code is loaded holds that array until the process exits.
 *   - No allocation: the call makes no cudaMalloc, cudaFree or other
 *     allocating call, and it launches its rounds one by one from the host
 *     (whatever the tuning says), so no CUDA graph is instantiated either.
 *     What the driver does on its own is outside the call's control: the
 *     first call on a device loads the library's device code (and with it
 *     the scratch array) unless an earlier call of this library did, and the
 *     first launch of a kernel may reserve its local memory.  Make one call
 *     on each device at start-up to get both done before the budget counts.
 *   - Size limit: the call fails with HPEEL_ERR_WORKSPACE_TOO_SMALL (and
 *     launches nothing) when hpeel_peel_workspace_size(n, m, r) exceeds
 *     HPEEL_NOALLOC_SCRATCH_BYTES -- about 500,000 edges at gamma = 1.23,
 *     r = 3.  Larger graphs need hpeel_peel and a caller workspace.
 *   - Every call looks up the array's device address with the current device
 *     (host code cannot use the array's name as an address).
 *   - All calls in the process share the one array, which keeps the last
 *     call's contents.  Each call clears what it needs before use, so leftover
 *     contents never change a result, but two calls whose work overlaps on
 *     the GPU (different streams or host threads on the same device) race on
 *     the array: callers must order such calls.
 * Synchronises stream after every round (the host decides whether another
 * round follows), so the call cannot be captured into a CUDA graph.
 */
#define HPEEL_NOALLOC_SCRATCH_BYTES (24u << 20)
hpeel_status hpeel_peel_noalloc(const uint32_t *d_edges, uint64_t n, uint64_t m,
                                uint32_t r, uint32_t *d_order, uint32_t *d_claim,
                                uint64_t *d_layer_off, uint32_t max_layers,
                                hpeel_stats *h_stats, void *stream);

/* Workspace bytes hpeel_mphf_build needs for n keys at gamma_milli. */
size_t hpeel_mphf_workspace_size(uint64_t n, uint32_t gamma_milli);

/*
 * MWHC minimal perfect hash build, r = 3 (sec. 3): hash the keys into a
 * 3-partite hypergraph with m = hpeel_num_vertices(n, gamma_milli, 3)
 * vertices, peel it, solve g in reverse layer order (sec. 4.3 "Avoiding
 * backward scans") so that g[h_0(x)] + g[h_1(x)] + g[h_2(x)] = i (mod 3),
 * where h_i(x) is the hinge of x's edge, then build the rank directory
 * (sec. 3 ranking structure, sec. 5 broadword counting).  If the hypergraph
 * keeps a 2-core, the build is retried with hash seed seed+1, seed+2, ...
 * (at most max_tries seeds in total).
 *   d_keys    [n] uint64, distinct keys (duplicates can never peel), in
 *             device memory or in pinned host memory (cudaHostAlloc,
 *             cudaMallocHost or cudaHostRegister), which the hashing kernel
 *             reads in place over the host link (read again on a retry).
 *   d_G       [ceil(m/32)] uint64 output: 2 bits per vertex, vertex v at bits
 *             2(v mod 32), 2(v mod 32)+1 of word v/32; 0 = unassigned,
 *             1, 2 = g, 3 = g value 0 of an assigned (hinge) vertex.
 *   d_rank_dir [ceil(m/512) + 1] uint64 output: d_rank_dir[b] = number of
 *             non-zero 2-bit values among vertices [0, 512 b).
 *   MPHF(x) = d_rank_dir[v/512] + non-zero values in [512 (v/512), v), with
 *   v = h_i(x), i = (G[h_0(x)] + G[h_1(x)] + G[h_2(x)]) mod 3.
 *   d_order   [n] uint32 output or NULL: the canonical peeling order of the
 *             successful attempt's hypergraph (as hpeel_peel gives it), so
 *             the whole path can be checked; NULL skips that sort.
 *   h_stats   host output or NULL (seed_used, attempts, rounds).
 * Synchronises stream.  Errors: HPEEL_ERR_INVALID_ARG,
 * HPEEL_ERR_WORKSPACE_TOO_SMALL, HPEEL_ERR_RETRIES_EXHAUSTED,
 * HPEEL_ERR_CAPACITY, HPEEL_ERR_CUDA.
 */
hpeel_status hpeel_mphf_build(const uint64_t *d_keys, uint64_t n, uint64_t seed,
                              uint32_t gamma_milli, uint32_t max_tries,
                              uint64_t *d_G, uint64_t *d_rank_dir, uint32_t *d_order,
                              hpeel_stats *h_stats, void *d_ws, size_t ws_bytes,
                              void *stream);

/*
 * hpeel_mphf_build with no host round trip: the whole build is enqueued on
 * stream as one CUDA graph and the call returns at once.  The reseed-and-
 * retry loop (sec. 3: a hypergraph that keeps a 2-core is hashed again with
 * the next seed), the rounds and the reverse-layer assignment are loops on
 * the device (conditional nodes), so the call can be captured into a
 * caller's CUDA graph or overlapped with other work on other streams.
 *   Arguments as hpeel_mphf_build, except:
 *   d_stats   device memory (not host), written at the end of the graph:
 *             async_status 1 = peeled (G and rank directory written, seed_used
 *             set), 2 = no seed among max_tries peeled (G untouched), 3 = a
 *             device check failed (device_err); attempts, rounds, n_peeled
 *             and the other counts as hpeel_mphf_build gives them.
 *   No canonical order output.
 * The graph is built on the first call with a given set of pointers and
 * sizes and replayed by later calls with the same set (keep the workspace
 * and the output buffers to reuse it).  Returns HPEEL_OK once enqueued;
 * errors: HPEEL_ERR_INVALID_ARG, HPEEL_ERR_WORKSPACE_TOO_SMALL, HPEEL_ERR_CUDA.
 * When stream is being captured (cudaStreamBeginCapture), the build's nodes
 * join the caller's graph at the capture position instead.
 */
hpeel_status hpeel_mphf_build_async(const uint64_t *d_keys, uint64_t n, uint64_t seed,
                                    uint32_t gamma_milli, uint32_t max_tries, uint64_t *d_G,
                                    uint64_t *d_rank_dir, hpeel_stats *d_stats, void *d_ws,
                                    size_t ws_bytes, void *stream);

/*
 * MWHC MPHF build for key sets beyond 32-bit ids (sec. 3 and 4.2; sec. 5
 * builds 7.6e9 keys): the same function as hpeel_mphf_build -- the same
 * hashing, peel, hinges, g values and rank directory, bit for bit, for any n
 * both accept -- with 64-bit edge and vertex ids.  n may reach the size at
 * which a part of m / 3 vertices still has 32-bit local ids (about 1.05e10
 * keys at gamma = 1.23).  The state is compact: 8 bytes per vertex, 4 per
 * key of claim words, 8 per key of layer list; no edge is stored (an edge's
 * vertices are hashed again from its key when needed), so the keys must stay
 * readable by the device during the call.  No canonical order output.
 *   d_keys     [n] uint64 distinct keys in device memory (pinned host memory
 *              works but is read at random addresses over the host link).
 *   d_G        [ceil(m/32)] uint64 output, layout as hpeel_mphf_build's.
 *   d_rank_dir [ceil(m/512) + 1] uint64 output, as hpeel_mphf_build's.
 *   h_list     NULL (the layer list lives in the workspace), or n uint64
 *              entries of page-locked host memory (cudaHostAlloc,
 *              cudaMallocHost, cudaHostRegister): the kernels append the
 *              layers there and read them back as streams over the host
 *              link, which takes 8 bytes per key out of device memory.
 *   d_ws       hpeel_mphf_large_workspace_size(n, gamma_milli, h_list != NULL)
 *              bytes, 256-byte aligned.
 *   seed, gamma_milli, max_tries, h_stats: as hpeel_mphf_build (retries with
 *   seed + 1, ...; h_stats->seed_used is the seed lookups must use).
 * Synchronises stream.  Errors: HPEEL_ERR_INVALID_ARG (m / 3 >= 2^32, h_list
 * not page-locked), HPEEL_ERR_WORKSPACE_TOO_SMALL, HPEEL_ERR_RETRIES_EXHAUSTED,
 * HPEEL_ERR_CAPACITY (more than HPEEL_MAX_ROUNDS rounds, or a vertex of degree
 * 2^24 or more), HPEEL_ERR_DEVICE_CHECK, HPEEL_ERR_CUDA.
 */
size_t hpeel_mphf_large_workspace_size(uint64_t n, uint32_t gamma_milli, int list_on_host);
hpeel_status hpeel_mphf_build_large(const uint64_t *d_keys, uint64_t n, uint64_t seed,
                                    uint32_t gamma_milli, uint32_t max_tries, uint64_t *d_G,
                                    uint64_t *d_rank_dir, hpeel_stats *h_stats, void *d_ws,
                                    size_t ws_bytes, uint64_t *h_list, void *stream);
/* Lookup of the function hpeel_mphf_build_large built: as hpeel_mphf_lookup
 * with 64-bit results (the MPHF value of a key of the set, in [0, n)); m =
 * hpeel_num_vertices(n, gamma_milli, 3).  Asynchronous.  Errors:
 * HPEEL_ERR_INVALID_ARG, HPEEL_ERR_CUDA. */
hpeel_status hpeel_mphf_lookup_large(const uint64_t *d_keys, uint64_t nq, uint64_t seed,
                                     uint64_t m, const uint64_t *d_G, const uint64_t *d_rank_dir,
                                     uint64_t *d_out, void *stream);

/*
 * MPHF lookup (sec. 3; sec. 5 broadword rank): for each query key, hash it
 * with the build's seed into v_0, v_1, v_2 (as hpeel_hash_edges with r = 3),
 * take i = (g[v_0] + g[v_1] + g[v_2]) mod 3 (a stored 3 is 0) and return the
 * rank of v_i among the assigned vertices:
 *   d_rank_dir[v_i / 512] + non-zero 2-bit values in [512 (v_i / 512), v_i).
 * For a key of the build set the result is its MPHF value in [0, n) (a
 * bijection onto [0, n)); for any other key it is some value in [0, n].
 *   d_keys [nq] uint64; seed = hpeel_stats.seed_used of the build; m =
 *   hpeel_num_vertices(n, gamma_milli, 3); d_G, d_rank_dir as
 *   hpeel_mphf_build wrote them; d_out [nq] uint32 output.
 * Asynchronous.  Errors: HPEEL_ERR_INVALID_ARG, HPEEL_ERR_CUDA.
 */
hpeel_status hpeel_mphf_lookup(const uint64_t *d_keys, uint64_t nq, uint64_t seed,
                               uint64_t m, const uint64_t *d_G, const uint64_t *d_rank_dir,
                               uint32_t *d_out, void *stream);

/*
 * Static function (sec. 3): the paper's MWHC construction stores any
 * f: S -> [sigma], not only the MPHF.  It finds u[0..m) with values in
 * [0, sigma) such that f(x) = (u[h_0(x)] + u[h_1(x)] + u[h_2(x)]) mod sigma
 * for every key x (the same r = 3 hashing as hpeel_mphf_build), by peeling
 * and back-substitution in reverse layer order: the hinge of each peeled
 * edge takes the value that satisfies that edge's equation.  The MPHF is
 * the case sigma = 3, f(x) = hinge position.
 *   b = hpeel_sf_bits(sigma) = ceil(log2 sigma) bits per vertex; u[v] sits at
 *   bits [v b, (v + 1) b) of one bit string, bit i being bit (i mod 64) of
 *   word i / 64 (a value may straddle two words); vertices never a hinge
 *   hold 0.  2 <= sigma <= 2^32.
 */
uint32_t hpeel_sf_bits(uint64_t sigma);
/* uint64 words of u for n keys: ceil(m * b / 64), m = hpeel_num_vertices(n, gamma_milli, 3). */
uint64_t hpeel_sf_words(uint64_t n, uint32_t gamma_milli, uint64_t sigma);
/* Workspace bytes hpeel_sf_build needs. */
size_t hpeel_sf_workspace_size(uint64_t n, uint32_t gamma_milli);
/*
 *   d_keys    [n] uint64 keys (distinct, else every seed leaves a 2-core).
 *   d_values  [n] uint32: f(keys[i]) = d_values[i], each below sigma.
 *             Keys and values may be in pinned host memory (read in place,
 *             as for hpeel_mphf_build).
 *   d_U       [hpeel_sf_words(n, gamma_milli, sigma)] uint64 output.
 *   seed, gamma_milli, max_tries, h_stats, d_ws, ws_bytes: as for
 *             hpeel_mphf_build (retries with seed + 1, ... on a 2-core;
 *             h_stats->seed_used is the seed lookups must use).
 * Synchronises stream.  Errors: HPEEL_ERR_INVALID_ARG (sigma out of range,
 * n or m >= 2^32, NULL pointer), HPEEL_ERR_WORKSPACE_TOO_SMALL,
 * HPEEL_ERR_DEVICE_CHECK (a value >= sigma), HPEEL_ERR_RETRIES_EXHAUSTED,
 * HPEEL_ERR_CUDA.
 */
hpeel_status hpeel_sf_build(const uint64_t *d_keys, const uint32_t *d_values, uint64_t n,
                            uint64_t sigma, uint64_t seed, uint32_t gamma_milli,
                            uint32_t max_tries, uint64_t *d_U, hpeel_stats *h_stats,
                            void *d_ws, size_t ws_bytes, void *stream);
/*
 * hpeel_sf_build with no host round trip: the reseed-and-retry loop, the
 * rounds and the reverse-layer assignment run as loops on the device in one
 * CUDA graph (as hpeel_mphf_build_async does for the MPHF), so the call can
 * be captured into a caller's CUDA graph.  Arguments as hpeel_sf_build,
 * except d_stats, which is device memory written at the end of the graph:
 * async_status 1 = built (d_U written, seed_used set), 2 = no seed among
 * max_tries peeled (d_U untouched), 3 = a device check failed (device_err 7:
 * a value not below sigma; d_U incomplete).  Graph caching and capture as
 * hpeel_mphf_build_async.  Returns HPEEL_OK once enqueued; errors found on
 * the host: HPEEL_ERR_INVALID_ARG, HPEEL_ERR_WORKSPACE_TOO_SMALL,
 * HPEEL_ERR_CUDA.
 */
hpeel_status hpeel_sf_build_async(const uint64_t *d_keys, const uint32_t *d_values, uint64_t n,
                                  uint64_t sigma, uint64_t seed, uint32_t gamma_milli,
                                  uint32_t max_tries, uint64_t *d_U, hpeel_stats *d_stats,
                                  void *d_ws, size_t ws_bytes, void *stream);
/*
 * d_out[q] = f(d_keys[q]) = (u[h_0] + u[h_1] + u[h_2]) mod sigma for the u/*
 * d_out[q] = f(d_keys[q]) = (u[h_0] + u[h_1] + u[h_2]) mod sigma for the u
 * built with this seed (h_stats->seed_used), m and sigma.  For a key outside
 * the built set the result is some value in [0, sigma).  Asynchronous on
 * stream.  Errors: HPEEL_ERR_INVALID_ARG, HPEEL_ERR_CUDA.
 */
hpeel_status hpeel_sf_lookup(const uint64_t *d_keys, uint64_t nq, uint64_t seed, uint64_t m,
                             uint64_t sigma, const uint64_t *d_U, uint32_t *d_out,
                             void *stream);

/*
 * Batched peel of many independent bucket hypergraphs (the bucketed layout of
 * sec. 3 "Practical workarounds (HEM)": one small MWHC hypergraph per bucket),
 * r = 3.  Bucket b holds keys d_keys[off[b] .. off[b+1]) (n_b of them, at most
 * 65,536); it is hashed with seed b into m_b = hpeel_num_vertices(n_b,
 * gamma_milli, 3) vertices and peeled as hpeel_peel would (sec. 4.2).
 *   d_bucket_off    [B + 1] uint64, non-decreasing, off[0] = 0.
 *   d_order         [off[B]] uint32 output: for every bucket, at its keys'
 *                   positions, the canonical order of its edges in local ids
 *                   (edge i = key off[b] + i): layers ascending by round, ids
 *                   ascending inside a layer, then the 2-core edges ascending.
 *   d_bucket_rounds [B] uint32 output or NULL: rounds of each bucket.
 *   d_bucket_status [B] uint32 output or NULL: 0 = peeled completely, 1 = a
 *                   2-core is left, 2 = more than 65,536 keys (the bucket's
 *                   outputs are not written).
 *   d_G, d_G_off    both NULL, or: d_G_off [B + 1] word offsets (from
 *                   hpeel_batched_g_offsets) and d_G [d_G_off[B]] uint64 output,
 *                   the MWHC g values of bucket b at d_G + d_G_off[b] in the
 *                   layout of hpeel_mphf_build's d_G (all zero for a bucket that
 *                   kept a 2-core).
 *   tuning          NULL for the defaults, or the launch shape (see
 *                   hpeel_batch_tuning); results never depend on it.
 *   1000 <= gamma_milli <= 1999 (the largest bucket's vertex ids must fit 17
 *   bits).
 * Asynchronous: no host synchronisation, no allocation -- the call can be
 * captured into a CUDA graph.  Errors: HPEEL_ERR_INVALID_ARG,
 * HPEEL_ERR_WORKSPACE_TOO_SMALL, HPEEL_ERR_CUDA.
 */
typedef struct hpeel_batch_tuning {
    uint32_t threads;      /* threads per block (multiple of 32, 64..1024; 0: 256) */
    uint32_t ctas_per_sm;  /* blocks per SM (grid = SMs x this; 0: 2) */
    uint32_t smem_bytes;   /* shared memory per block for bucket state (0: the SM's
                              shared memory split between the blocks); buckets
                              that do not fit use the workspace instead */
    uint32_t smem_rounds;  /* layer-table entries of a bucket in shared memory
                              (0: 256; at least 2); a bucket that needs more
                              rounds is peeled again in the workspace */
    uint32_t global16_rounds;  /* layer-table entries of a bucket peeled in the
                              workspace with 32-bit vertex records and 16-bit
                              claim words (0: 16,383, the most a 16-bit claim
                              word holds; 2..16,383); a bucket that needs more
                              rounds is peeled again with 64-bit records and
                              32-bit claim words, which have room for every
                              round */
    uint32_t reserved[3];
} hpeel_batch_tuning;

size_t hpeel_batched_workspace_size(uint32_t B, uint32_t gamma_milli,
                                    const hpeel_batch_tuning *tuning);

/* d_G_off[b] = sum over c < b of ceil(m_c / 32): where bucket b's g words
 * start in d_G (B + 1 entries).  Uses the first part of a batched workspace
 * (hpeel_batched_workspace_size(B, gamma_milli, NULL) bytes suffice).
 * Asynchronous.  Errors: HPEEL_ERR_INVALID_ARG, HPEEL_ERR_WORKSPACE_TOO_SMALL,
 * HPEEL_ERR_CUDA. */
hpeel_status hpeel_batched_g_offsets(const uint64_t *d_bucket_off, uint32_t B,
                                     uint32_t gamma_milli, uint64_t *d_G_off,
                                     void *d_ws, size_t ws_bytes, void *stream);

hpeel_status hpeel_peel_batched(const uint64_t *d_keys, const uint64_t *d_bucket_off,
                                uint32_t B, uint32_t gamma_milli, uint32_t *d_order,
                                uint32_t *d_bucket_rounds, uint32_t *d_bucket_status,
                                uint64_t *d_G, const uint64_t *d_G_off,
                                const hpeel_batch_tuning *tuning, void *d_ws,
                                size_t ws_bytes, void *stream);

/*
 * Instrumentation (no counterpart in the paper; used to measure the path).
 *   hpeel_kernel_launches  total number of kernels this library has launched
 *                          in the process (all devices, all threads).
 *   hpeel_profile_enable   1: every step of every later call records a CUDA
 *                          event pair on the call's stream; the elapsed times
 *                          are added up per step name when the call returns.
 *                          0 (default): no events are recorded.
 *   hpeel_profile_reset    clears the per-step totals.
 *   hpeel_profile_read     writes "name launches total_ms" lines (one per
 *                          step name) into buf (at most len bytes, always
 *                          NUL-terminated when len > 0); returns the size
 *                          needed including the NUL.
 */
uint64_t hpeel_kernel_launches(void);
void hpeel_profile_enable(int on);
void hpeel_profile_reset(void);
size_t hpeel_profile_read(char *buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* HPEEL_H */
