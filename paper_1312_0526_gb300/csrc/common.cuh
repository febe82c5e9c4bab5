// common.cuh -- device helpers shared by the hpeel kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hpeel.h"

namespace hp {

constexpr uint32_t kUnclaimed = 0xFFFFFFFFu;

// Device error word codes (hpeel_stats.device_err).
enum : uint32_t {
    kDevOk = 0,
    kDevBadVertex = 1,   // a vertex id outside its part (input violates sec. 4.3)
    kDevBadEdge = 2,     // an edge id >= n read off a record (inconsistent state)
    kDevCapacity = 3,    // a round-table bound was exceeded
    kDevTimeout = 4,     // a bounded wait gave up
    kDevBuildOverflow = 5,  // the bucketed build's overflow list was full
    kDevDegree = 6,      // a vertex degree of 2^31 or more (no room for the mark bit)
    kDevBadValue = 7,    // a static-function value outside [0, sigma)
    kDevRoundOverflow = 8,  // a sorted round's buckets or claim list were full
};

// Device-side control block of one peel (lives in the workspace).
struct Ctl {
    uint32_t lcur;       // append cursor of the layer list L (L_0 | L_1 | ...)
    uint32_t round;      // index t of the round being run
    uint32_t done;       // blocks finished in the current update launch
    uint32_t err;        // first device error code (0 = none)
    uint32_t more;       // 1 while the next layer is non-empty
    uint32_t next_size;  // size of the layer the next round deletes
    uint32_t cross;      // vertices that fell from degree 2 to 1 (all rounds)
    uint32_t first_layer;   // |L_0|
    uint32_t moves;      // list entries whose first claimer was not the hinge
    uint32_t ccur;       // append cursor of the claim list of a sorted round
    uint32_t bmode;      // 1: the next round runs in sorted (bucketed) form
    uint32_t brounds;    // rounds run in sorted form
    uint32_t cvalid;     // 1: the incidence build left round 0's claims in the claim list
    uint32_t pad[3];
};

// State of a device-driven build (graph-resident reseed-and-retry).
enum : uint32_t {
    kAsyncRunning = 0,
    kAsyncPeeled = 1,
    kAsyncRetriesExhausted = 2,
    kAsyncDeviceError = 3,
};
struct AsyncState {
    uint64_t seed0, seed;  // first seed, seed of the current attempt
    uint32_t attempt;      // attempts made after the first
    uint32_t max_tries;
    uint32_t status;       // kAsync*
    uint32_t rounds;       // layers of the peeled attempt
    int32_t t;             // layer being assigned
    uint32_t n;
};

// Pass parameters of the canonical-order sort when the device drives it
// (the number of rounds is never read back to the host): pass k sorts the
// count inputs from seg on by keys base .. base + nb - 1 (the last bin takes
// every larger key); more = 1 while another pass follows.
struct EmitState {
    uint32_t n, R, nkeys, base, seg, count, nb, more;
};

// Arguments of the round-loop kernels, kept in the workspace so the CUDA
// graph of a round loop depends only on where the workspace is.
struct RoundParams {
    unsigned long long *st;  // vertex records [m]
    uint4 *rec;              // edge records [n]
    uint4 *L;                // layer list: one entry per peeled edge
    uint32_t *loff;          // layer starts
    Ctl *ctl;
    uint32_t n, m, P, max_rounds;
};

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014): two
// xorshift-multiply steps and a final xorshift, modulo 2^64.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Remainder by a runtime divisor P < 2^32 with a precomputed reciprocal
// (Barrett reduction, P. Barrett, CRYPTO 1986).  With M = floor((2^64-1)/P)
// the estimate q = floor(x M / 2^64) satisfies Q - 2 <= q <= Q for the true
// quotient Q = floor(x / P), so x - q P lies in [0, 3P) and at most two
// corrective subtractions give x mod P exactly.
struct FastMod {
    uint64_t P;
    uint64_t M;
};

inline FastMod make_fastmod(uint64_t P) { return FastMod{P, P ? (~0ull) / P : 0}; }

__device__ __forceinline__ uint64_t fastmod(uint64_t x, const FastMod f) {
    uint64_t q = __umul64hi(x, f.M);
    uint64_t r = x - q * f.P;
    if (r >= f.P) r -= f.P;
    if (r >= f.P) r -= f.P;
    return r;
}

// Control block and parameters of the large-n MPHF build (large.cu): 64-bit
// edge and vertex ids, 64-bit list cursors.
struct LargeCtl {
    unsigned long long lcur;         // append cursor of the layer list
    unsigned long long cross;        // vertices that fell from degree 2 to 1
    unsigned long long first_layer;  // |L_0|
    uint32_t round, done, err, more;
    uint32_t pad[8];
};
struct LargeParams {
    unsigned long long *st;    // vertex records [m]
    uint32_t *claim;           // claim words [n]
    unsigned long long *L;     // layer list [n] (device or pinned host memory)
    unsigned long long *loff;  // layer starts
    LargeCtl *ctl;
    const uint64_t *keys;
    uint64_t n, m, seed;
    FastMod fm;                // part size P = m / 3
    uint32_t max_rounds;
};

// Position (part index) of vertex v in an r-partite graph with part size P:
// the number of part boundaries at or below v.
template <int R>
__device__ __forceinline__ uint32_t part_of(uint32_t v, uint32_t P) {
    uint32_t j = 0;
#pragma unroll
    for (int k = 1; k < R; k++) j += (v >= (uint32_t)k * P) ? 1u : 0u;
    return j;
}

__device__ __forceinline__ void raise_err(Ctl *ctl, uint32_t code) {
    atomicCAS(&ctl->err, 0u, code);
}

// ------------------------------------------------------------ bulk copies --
// One-dimensional TMA copies (cp.async.bulk) from global into shared memory,
// completing on an mbarrier (one arrival: the thread that issues the copy
// and sets the byte count).  Source, destination and size are multiples of
// 16 bytes.  Waits are bounded: mbar_wait gives up after kMbarTries tries
// (each try suspends the thread for a short, hardware-chosen time).
constexpr uint32_t kMbarTries = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t arrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals)
                 : "memory");
}
// makes initialised mbarriers visible to the async proxy (before the first copy)
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier shared-memory accesses before its later
// async-proxy ones: a bulk copy into a buffer that the block just read
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// shared -> global bulk copy; the issuing thread waits with
// bulk_store_wait_read before the source buffer is reused or the block exits
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_store_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n"
        "  .reg .pred p;\n"
        "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "  selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}
// true once the phase with this parity has completed, false after kMbarTries
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < kMbarTries; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Mark bit in the degree half of a vertex record: set once the vertex has
// degree 1 with its last edge claimed (round 0 scan, or the fall from 2 to 1).
constexpr uint32_t kMark = 0x80000000u;

// Warp-aggregated append: every lane of the warp calls this (convergent);
// lanes with pred get consecutive slots of list, one atomicAdd per warp.
__device__ __forceinline__ void warp_append(uint32_t *cursor, uint32_t *list, bool pred,
                                            uint32_t value) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, pred);
    if (ballot == 0) return;
    uint32_t base = 0;
    const uint32_t leader = __ffs(ballot) - 1;
    if (lane == leader) base = atomicAdd(cursor, (uint32_t)__popc(ballot));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (pred) list[base + __popc(ballot & ((1u << lane) - 1u))] = value;
}

// ---- edge records ------------------------------------------------------
// Edge e: one uint4 {v_0, v_1, v_2, claim} for r <= 3 (v_2 = 0 when r = 2),
// two uint4 {v_0..v_3}, {claim, 0, 0, 0} for r = 4.
template <int R>
__device__ __forceinline__ uint32_t *claim_ptr(uint4 *rec, uint64_t e) {
    return R == 4 ? &rec[2 * e + 1].x : &rec[e].w;
}

template <int R>
__device__ __forceinline__ void store_record(uint4 *rec, uint64_t e, const uint32_t (&v)[4],
                                             bool valid) {
    // an invalid edge keeps vertex 0 everywhere: memory-safe, flagged by the caller
    const uint32_t a = valid ? v[0] : 0u, b = valid ? v[1] : 0u;
    const uint32_t c = valid ? v[2] : 0u, d = valid ? v[3] : 0u;
    if (R == 4) {
        rec[2 * e] = make_uint4(a, b, c, d);
        rec[2 * e + 1] = make_uint4(kUnclaimed, 0u, 0u, 0u);
    } else {
        rec[e] = make_uint4(a, b, R == 3 ? c : 0u, kUnclaimed);
    }
}

// Vertices only (immutable once written): streaming load.
template <int R>
__device__ __forceinline__ void load_vertices(const uint4 *rec, uint64_t e, uint32_t (&v)[4]) {
    const uint4 q = __ldcs(rec + (R == 4 ? 2 * e : e));
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}

// Vertices and claim word (random access).
template <int R>
__device__ __forceinline__ uint32_t load_record(const uint4 *rec, uint64_t e, uint32_t (&v)[4]) {
    if (R == 4) {
        const uint4 q = rec[2 * e], c = rec[2 * e + 1];
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        return c.x;
    }
    const uint4 q = rec[e];
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = 0u;
    return q.w;
}

// Same, for a pass that streams every record once.
template <int R>
__device__ __forceinline__ uint32_t load_record_stream(const uint4 *rec, uint64_t e,
                                                       uint32_t (&v)[4]) {
    if (R == 4) {
        const uint4 q = __ldcs(rec + 2 * e), c = __ldcs(rec + 2 * e + 1);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        return c.x;
    }
    const uint4 q = __ldcs(rec + e);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = 0u;
    return q.w;
}

// ---- layer-list entries --------------------------------------------------
// One entry per peeled edge, in the shape of its edge record with the
// vertices rotated: word 0 the hinge vertex, then the other vertices in
// position order, and the edge id where the record keeps its claim word
// ({v_h, v_a, v_b, e} for r = 3; {v_h, v_a, 0, e} for r = 2; two uint4
// {v_h, v_a, v_b, v_c}, {e, 0, 0, 0} for r = 4).  The hinge position is the
// part of word 0 (sec. 4.3), so an entry is also the MWHC solve record of
// its edge.
template <int R>
struct Entry {
    uint4 w[R == 4 ? 2 : 1];
};

template <int R>
__device__ __forceinline__ Entry<R> make_entry(const uint32_t (&v)[4], uint32_t e) {
    Entry<R> x;
    if (R == 4) {
        x.w[0] = make_uint4(v[0], v[1], v[2], v[3]);
        x.w[R == 4 ? 1 : 0] = make_uint4(e, 0u, 0u, 0u);
    } else {
        x.w[0] = make_uint4(v[0], v[1], R == 3 ? v[2] : 0u, e);
    }
    return x;
}

// v[0] = hinge vertex, v[1..R-1] = others in position order; returns e.
template <int R>
__device__ __forceinline__ uint32_t load_entry(const uint4 *L, uint64_t i, uint32_t (&v)[4]) {
    if (R == 4) {
        const uint4 a = __ldcs(L + 2 * i), b = __ldcs(L + 2 * i + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        return b.x;
    }
    const uint4 a = __ldcs(L + i);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = 0u;
    return a.w;
}

template <int R>
__device__ __forceinline__ void store_entry(uint4 *L, uint64_t i, const Entry<R> &x) {
    if (R == 4) {
        L[2 * i] = x.w[0];
        L[2 * i + 1] = x.w[R == 4 ? 1 : 0];
    } else {
        L[i] = x.w[0];
    }
}

// Rotation of the position-ordered vertices p[0..R-1] around position h:
// out[0] = p[h], out[1..R-1] = the others in position order.  Static indices
// only, so the arrays stay in registers.
template <int R>
__device__ __forceinline__ void rotate_to(const uint32_t (&p)[4], uint32_t h, uint32_t (&out)[4]) {
    uint32_t x = p[0];
#pragma unroll
    for (int q = 1; q < R; q++) x = h == (uint32_t)q ? p[q] : x;
    out[0] = x;
#pragma unroll
    for (int k = 0; k < R - 1; k++) out[k + 1] = (uint32_t)k >= h ? p[k + 1] : p[k];
#pragma unroll
    for (int k = R; k < 4; k++) out[k] = 0u;
}

// Inverse: position-ordered vertices of an entry whose hinge is at position h.
template <int R>
__device__ __forceinline__ void unrotate(const uint32_t (&v)[4], uint32_t h, uint32_t (&p)[4]) {
#pragma unroll
    for (int q = 0; q < R; q++) p[q] = (uint32_t)q == h ? v[0] : ((uint32_t)q < h ? v[q + 1] : v[q]);
#pragma unroll
    for (int k = R; k < 4; k++) p[k] = 0u;
}

// Block-aggregated append: every thread of the block calls this (it holds
// barriers) with K candidates; the block reserves all its slots with a single
// atomicAdd, so the shared cursor sees one atomic per K * blockDim items.
// The order of the appended values inside the list is unspecified.
template <int K, int THREADS>
__device__ __forceinline__ void block_append(uint32_t *cursor, uint32_t *list, const bool (&pred)[K],
                                             const uint32_t (&val)[K]) {
    __shared__ uint32_t warp_base[THREADS / 32];
    __shared__ uint32_t block_base;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < K; k++) cnt += pred[k] ? 1u : 0u;
    uint32_t x = cnt;  // inclusive warp scan
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) warp_base[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; w++) {
            const uint32_t c = warp_base[w];
            warp_base[w] = s;
            s += c;
        }
        block_base = s ? atomicAdd(cursor, s) : 0u;
    }
    __syncthreads();
    uint32_t pos = block_base + warp_base[warp] + x - cnt;
#pragma unroll
    for (int k = 0; k < K; k++)
        if (pred[k]) list[pos++] = val[k];
    __syncthreads();
}

// Per-warp staging buffer in shared memory for list appends: lanes push
// values (warp-synchronous), and the warp reserves space in the global list
// with one atomicAdd per CAP values (flush when full and at the end), so the
// shared list cursor sees few atomics however many values are appended.  The
// order of the values in the list is unspecified.
template <typename T, int CAP>
struct WarpStage {
    T *buf;        // this warp's CAP slots in shared memory
    uint32_t cnt;  // values staged (warp-uniform)

    __device__ __forceinline__ void flush(uint32_t *cursor, T *list) {
        __syncwarp();
        if (cnt == 0) return;
        const uint32_t lane = threadIdx.x & 31u;
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(cursor, cnt);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (uint32_t i = lane; i < cnt; i += 32) list[base + i] = buf[i];
        cnt = 0;
        __syncwarp();
    }
    // every lane of the warp calls push (convergent)
    __device__ __forceinline__ void push(bool pred, const T &val, uint32_t *cursor, T *list) {
        const uint32_t lane = threadIdx.x & 31u;
        const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, pred);
        if (ballot == 0) return;
        const uint32_t k = __popc(ballot);
        if (cnt + k > CAP) flush(cursor, list);
        if (pred) buf[cnt + __popc(ballot & ((1u << lane) - 1u))] = val;
        cnt += k;
        __syncwarp();
    }
};

// Block-aggregated reservation of one slot per thread with pred: returns the
// slot (unspecified order) for those threads; one atomicAdd per block call.
template <int THREADS>
__device__ __forceinline__ uint32_t block_reserve(uint32_t *cursor, bool pred) {
    __shared__ uint32_t warp_base[THREADS / 32];
    __shared__ uint32_t block_base;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, pred);
    if (lane == 0) warp_base[warp] = __popc(ballot);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; w++) {
            const uint32_t c = warp_base[w];
            warp_base[w] = s;
            s += c;
        }
        block_base = s ? atomicAdd(cursor, s) : 0u;
    }
    __syncthreads();
    const uint32_t pos = block_base + warp_base[warp] + __popc(ballot & ((1u << lane) - 1u));
    __syncthreads();
    return pos;
}

}  // namespace hp
