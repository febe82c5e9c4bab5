// rounds_bucketed.cu -- the dense rounds of sec. 4.2 in sorted form.
//
// The paper peels in rounds by sorting: the degree-1 orientations D_i are
// sorted by edge to keep one orientation per edge (the layer P_i), and the
// updates U_i are sorted by vertex and joined with the incidence lists.  The
// round kernel of peel.cu does the same work with atomics at random
// addresses, which is the cheapest form for the many small rounds; for the
// few large ones (the first rounds, where a quarter and then a tenth of the
// edges leave) the same random accesses are many times more than a pass over
// the arrays costs.  Those rounds here take the paper's sorted form, with
// shared memory as the fast tier:
//   claims  -- every vertex of degree 1 (all of them in round 0, those that
//              fall from 2 to 1 later) appends a claim {edge, vertex} to a
//              flat list; the claims are bucketed by edge range (two
//              counting-sort passes, as the incidence build does for
//              vertices), and one block per 2^esub edges gathers the
//              positions that claim each edge in a shared table, then goes
//              over its claims again: the claim of an edge's smallest
//              claiming position, if no earlier round took the edge, makes
//              that vertex the hinge and appends the list entry
//              {v_hinge, others, e}.  The hinge
//              is exact, so no entry of a sorted round is ever rewritten and
//              no vertex is marked.
//   updates -- the entries of the layer give their r - 1 DeleteEdge updates
//              {vertex, edge}, bucketed by vertex range (chunks of a part,
//              then sub-buckets of 2^sub_shift vertices); one block per
//              sub-bucket brings its vertex records into shared memory (all
//              of them by one bulk copy when it has many updates, else the
//              ones the round touches), applies the updates there with
//              64-bit shared atomics (degree and id sum in one word, as in
//              global memory), lets every vertex that falls from degree 2 to
//              1 claim its last edge for the next round, and writes the
//              records back.
// A round runs in sorted form when its layer holds at least a set number of
// edges; the rounds after the first one that does not run in random form.
// r = 3, r-partite graphs only.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "kernels.cuh"

namespace hp {

// ---------------------------------------------------------------- staging --
// Per-warp staging of appends to a list with a fixed capacity: lanes push
// values (warp-synchronous), the warp reserves space with one atomicAdd per
// buffer-full; values that find the list full are dropped and raise
// kDevRoundOverflow (the peel is then redone with random rounds).
template <typename T, int CAP>
struct CappedStage {
    T *buf;
    uint32_t cnt;

    __device__ __forceinline__ void flush(uint32_t *cursor, T *list, uint32_t cap, Ctl *ctl) {
        __syncwarp();
        if (cnt == 0) return;
        const uint32_t lane = threadIdx.x & 31u;
        uint32_t base = 0;
        if (lane == 0) {
            base = atomicAdd(cursor, cnt);
            if (base + cnt > cap || base + cnt < base) raise_err(ctl, kDevRoundOverflow);
        }
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (uint32_t i = lane; i < cnt; i += 32)
            if (base + i < cap && base + i >= base) list[base + i] = buf[i];
        cnt = 0;
        __syncwarp();
    }
    __device__ __forceinline__ void push(bool pred, const T &val, uint32_t *cursor, T *list,
                                         uint32_t cap, Ctl *ctl) {
        const uint32_t lane = threadIdx.x & 31u;
        const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, pred);
        if (ballot == 0) return;
        const uint32_t k = __popc(ballot);
        if (cnt + k > CAP) flush(cursor, list, cap, ctl);
        if (pred) buf[cnt + __popc(ballot & ((1u << lane) - 1u))] = val;
        cnt += k;
        __syncwarp();
    }
};

constexpr int kClaimStage = 512;  // claims staged per warp in round 0 (8 B each)

// ---------------------------------------------------------- round 0 claims --
// Every vertex of degree 1 claims its edge (F_0 of sec. 4.2, never stored):
// one claim {e, v} per such vertex, appended to the flat claim list.
constexpr int kR0EmitItems = 4;

// When the incidence build emitted round 0's claims (ctl->cvalid), the scan is
// skipped; otherwise k_round0_reset clears the list first.
__global__ void k_round0_reset(Ctl *ctl) {
    if (!ctl->cvalid) ctl->ccur = 0;
}

__global__ void __launch_bounds__(kThreads)
k_round0_emit(const unsigned long long *__restrict__ st, uint32_t m, uint32_t n,
              uint2 *__restrict__ claims, uint32_t claim_cap, Ctl *ctl) {
    if (*(volatile uint32_t *)&ctl->cvalid) return;  // the build emitted them
    __shared__ uint2 sbuf[kThreads / 32][kClaimStage];
    CappedStage<uint2, kClaimStage> stage{sbuf[threadIdx.x >> 5], 0};
    constexpr uint32_t kStep = kThreads * kR0EmitItems;
    // whole warps step together: the trip count depends on blockIdx only
    for (uint64_t base = (uint64_t)blockIdx.x * kStep; base < m;
         base += (uint64_t)gridDim.x * kStep) {
        unsigned long long s[kR0EmitItems];
#pragma unroll
        for (int k = 0; k < kR0EmitItems; k++) {
            const uint64_t v = base + (uint64_t)k * kThreads + threadIdx.x;
            s[k] = v < m ? __ldcs(st + v) : 0ull;
        }
#pragma unroll
        for (int k = 0; k < kR0EmitItems; k++) {
            const uint64_t v = base + (uint64_t)k * kThreads + threadIdx.x;
            const uint32_t deg = (uint32_t)s[k], e = (uint32_t)(s[k] >> 32);
            bool one = false;
            if (v < m) {
                if (deg & kMark) raise_err(ctl, kDevDegree);
                if (deg == 1u) {
                    one = e < n;
                    if (!one) raise_err(ctl, kDevBadEdge);
                }
            }
            stage.push(one, make_uint2(e, (uint32_t)v), &ctl->ccur, claims, claim_cap, ctl);
        }
    }
    stage.flush(&ctl->ccur, claims, claim_cap, ctl);
}

// -------------------------------------------------------------- bucketing --
// One counting-sort pass: each block takes tiles of input items, sorts their
// pairs by chunk in shared memory and appends each chunk's run to the chunk's
// array (one atomicAdd per chunk and tile on its cursor; cursors one 128-byte
// line apart, zeroed before the pass).  A tile's items are contiguous: one
// bulk copy (TMA) brings them into one of two shared-memory buffers while the
// block sorts the previous tile.  Items:
//   ENTRIES  -- the entries of layer t = ctl->round, each giving the pairs
//               {w, e} of its R - 1 non-hinge vertices; chunks by vertex
//               (part j, then 2^shift vertices of the part);
//   !ENTRIES -- the ctl->ccur claims {g, v} of the flat list; chunks by edge
//               (one part [0, P = n), 2^shift edges each).
#ifndef HPEEL_BUCKET_THREADS
#define HPEEL_BUCKET_THREADS 512
#endif
#ifndef HPEEL_BUCKET_BLOCKS
#define HPEEL_BUCKET_BLOCKS 2
#endif
// the claims' pass stages one pair per item from 8-byte items: more blocks fit
#ifndef HPEEL_CLAIM_BUCKET_BLOCKS
#define HPEEL_CLAIM_BUCKET_BLOCKS 3
#endif
constexpr int kBucketThreads = HPEEL_BUCKET_THREADS;
constexpr int kBucketItems = 4 * kBucketThreads;  // items per tile (4 per thread)
// words of each per-chunk counter array (a multiple of 4: the arrays after
// them stay 16-byte aligned)
__host__ __device__ constexpr uint32_t bucket_counters(uint32_t C) { return (C + 3) & ~3u; }

// shared memory of one pass: counters of every chunk, a tile's staged pairs
// and two tiles of input
__host__ __device__ constexpr size_t bucket_smem_bytes(uint32_t C, bool entries) {
    return (size_t)3 * bucket_counters(C) * 4 + (size_t)kBucketItems * (entries ? 2 : 1) * 8 +
           (size_t)2 * kBucketItems * (entries ? 16 : 8);
}

template <int R, bool ENTRIES>
__global__ void __launch_bounds__(kBucketThreads,
                                  ENTRIES ? HPEEL_BUCKET_BLOCKS : HPEEL_CLAIM_BUCKET_BLOCKS)
k_pairs_bucket(const uint4 *__restrict__ Lst, const uint32_t *__restrict__ loff,
               const uint2 *__restrict__ claims, uint32_t claim_cap, BucketGeom g, uint32_t C,
               uint2 *__restrict__ pairs, uint32_t *__restrict__ fill, Overflow ov, Ctl *ctl) {
    constexpr int kPer = ENTRIES ? R - 1 : 1;
    static_assert(kPer <= 2, "the stage holds two pairs per item (r = 3)");
    using In = typename std::conditional<ENTRIES, uint4, uint2>::type;  // one input item
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint64_t bar[2];
    const uint32_t Cq = bucket_counters(C);
    uint32_t *hist = smem;                                  // C: tile count per chunk
    uint32_t *cur = hist + Cq;                              // C: run's place - its stage slot
    uint32_t *toff = cur + Cq;                              // C: run's first stage slot
    uint2 *stage = reinterpret_cast<uint2 *>(toff + Cq);    // kPer per item (16-byte aligned)
    In *inbuf = reinterpret_cast<In *>(stage + kPer * kBucketItems);  // two tiles of input
    uint32_t i0, i1;
    if (ENTRIES) {
        const uint32_t t = *(volatile uint32_t *)&ctl->round;
        i0 = loff[t];
        i1 = loff[t + 1];
    } else {
        i0 = 0;
        i1 = min(*(volatile uint32_t *)&ctl->ccur, claim_cap);
    }
    if (i1 < i0) i1 = i0;
    const In *in = (ENTRIES ? reinterpret_cast<const In *>(Lst) : reinterpret_cast<const In *>(claims)) + i0;
    auto chunk_of_key = [&](uint32_t x) -> uint32_t {
        if (ENTRIES) {
            const uint32_t j = part_of<R>(x, g.P);
            return j * g.chunks_per_part + ((x - j * g.P) >> g.shift);
        }
        return x >> g.shift;
    };
    const uint64_t tiles = ((uint64_t)(i1 - i0) + kBucketItems - 1) / kBucketItems;
    auto tile_items = [&](uint64_t tile) -> uint32_t {
        const uint64_t left = (uint64_t)(i1 - i0) - tile * kBucketItems;
        return left < (uint64_t)kBucketItems ? (uint32_t)left : (uint32_t)kBucketItems;
    };
    // a tile's input arrives by one bulk copy of its first multiple of 16
    // bytes (every item but a claim tile's odd last one, read directly)
    auto bulk_bytes = [&](uint32_t tn) -> uint32_t { return (tn * (uint32_t)sizeof(In)) & ~15u; };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x < tiles) {
        const uint32_t bytes = bulk_bytes(tile_items(blockIdx.x));
        if (bytes) bulk_load(inbuf, in + (uint64_t)blockIdx.x * kBucketItems, bytes, &bar[0]);
    }
    uint32_t k = 0;  // this block's tiles so far: buffer k & 1, its use k >> 1
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, k++) {
        const uint32_t buf = k & 1u;
        // the next tile's input goes to the other buffer, which the block
        // read in the previous tile (ended by a barrier)
        const uint64_t next = tile + gridDim.x;
        if (threadIdx.x == 0 && next < tiles) {
            const uint32_t bytes = bulk_bytes(tile_items(next));
            if (bytes) {
                fence_proxy_async_smem();
                bulk_load(inbuf + (size_t)(buf ^ 1u) * kBucketItems, in + next * kBucketItems,
                          bytes, &bar[buf ^ 1u]);
            }
        }
        for (uint32_t c = threadIdx.x; c < C; c += kBucketThreads) hist[c] = 0;
        const uint32_t tn = tile_items(tile);
        const uint32_t nbulk = bulk_bytes(tn) / (uint32_t)sizeof(In);
        const bool landed = nbulk == 0 || mbar_wait(&bar[buf], (k >> 1) & 1u);
        if (!__syncthreads_and(landed)) {  // a copy that never lands: give up
            if (threadIdx.x == 0) {
                raise_err(ctl, kDevTimeout);
                mbar_wait(&bar[buf], (k >> 1) & 1u);
                if (next < tiles) mbar_wait(&bar[buf ^ 1u], ((k + 1) >> 1) & 1u);
            }
            __syncthreads();
            return;
        }
        const In *tin = inbuf + (size_t)buf * kBucketItems;
        const In *gin = in + tile * kBucketItems;
        uint2 pp[4][kPer];
        uint32_t ch[4][kPer], rank[4][kPer];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t li = (uint32_t)q * kBucketThreads + threadIdx.x;
            ok[q] = li < tn;
#pragma unroll
            for (int k2 = 0; k2 < kPer; k2++) pp[q][k2] = make_uint2(0u, 0u);
            if (ok[q]) {
                const In a = li < nbulk ? tin[li] : gin[li];
                if constexpr (ENTRIES) {  // {v_hinge, v_a, v_b, e}
                    pp[q][0] = make_uint2(a.y, a.w);
                    if (kPer > 1) pp[q][kPer - 1] = make_uint2(a.z, a.w);
                } else {
                    pp[q][0] = a;
                }
            }
#pragma unroll
            for (int k2 = 0; k2 < kPer; k2++) {
                ch[q][k2] = ok[q] ? chunk_of_key(pp[q][k2].x) : 0u;
                if (ch[q][k2] >= C) {  // a key outside the geometry: inconsistent state
                    raise_err(ctl, ENTRIES ? kDevBadVertex : kDevBadEdge);
                    ok[q] = false;
                }
            }
#pragma unroll
            for (int k2 = 0; k2 < kPer; k2++)
                rank[q][k2] = ok[q] ? atomicAdd(&hist[ch[q][k2]], 1u) : 0u;
        }
        __syncthreads();
        // reserve each chunk's run; the result is awaited after the staging
        const uint32_t h0 = threadIdx.x < C ? hist[threadIdx.x] : 0u;
        const uint32_t gb0 = h0 ? atomicAdd(fill + ((size_t)threadIdx.x << g.fill_shift), h0) : 0u;
        for (uint32_t c = kBucketThreads + threadIdx.x; c < C; c += kBucketThreads) {
            const uint32_t h = hist[c];
            cur[c] = h ? atomicAdd(fill + ((size_t)c << g.fill_shift), h) : 0u;
        }
        block_scan_counts<kBucketThreads>(hist, toff, C);  // exclusive scan of hist -> toff
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (!ok[q]) continue;
#pragma unroll
            for (int k2 = 0; k2 < kPer; k2++) {
                const uint32_t slot = toff[ch[q][k2]] + rank[q][k2];
                stage[slot] = pp[q][k2];
            }
        }
        // staged pair k of chunk c goes to place cur[c] + k (mod 2^32)
        if (threadIdx.x < C) cur[threadIdx.x] = gb0 - toff[threadIdx.x];
        for (uint32_t c = kBucketThreads + threadIdx.x; c < C; c += kBucketThreads)
            cur[c] -= toff[c];
        __syncthreads();
        const uint32_t total = toff[C - 1] + hist[C - 1];
        for (uint32_t k2 = threadIdx.x; k2 < total; k2 += kBucketThreads) {
            const uint2 p = stage[k2];
            const uint32_t c = chunk_of_key(p.x);  // its chunk again
            const uint32_t pos = cur[c] + k2;
            if (pos < g.cap)
                pairs[(uint64_t)c * g.cap + pos] = p;
            else
                raise_err(ctl, ov.code);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ updates --
// One block per vertex sub-bucket: the DeleteEdge updates of layer t applied
// in shared memory (see the file comment).  Every thread of the block runs
// every loop: the claim staging is warp-synchronous.
#ifndef HPEEL_DEL_CLAIMS
#define HPEEL_DEL_CLAIMS 1024
#endif
constexpr int kDelThreads = 512;
// claims a block gathers before one reservation: the expected number of
// vertices of a sub-bucket that fall to degree 1 in the first rounds is a
// few hundred; 1024 keeps the block at 74 KB of shared memory (3 per SM)
constexpr int kDelClaims = HPEEL_DEL_CLAIMS;
constexpr int kDelU = 8;          // loads in flight per thread
#ifndef HPEEL_DEL_PRE
#define HPEEL_DEL_PRE 4
#endif
constexpr int kDelPre = HPEEL_DEL_PRE;  // updates per thread loaded beside a bulk copy
static_assert(kDelPre >= 1 && kDelPre <= kDelU, "prefetched updates fit the first loop");
// updates from which a sub-bucket's records move by bulk copies
#ifndef HPEEL_DEL_BULK
#define HPEEL_DEL_BULK 512
#endif
constexpr uint32_t kDelBulk = HPEEL_DEL_BULK;

// three blocks per SM, as many as their shared memory allows
__global__ void __launch_bounds__(kDelThreads, 3)
k_delete_apply(const uint2 *__restrict__ pairs2, const uint32_t *__restrict__ fill2,
               uint32_t cap2, BucketGeom g, uint32_t sub_shift, unsigned long long *__restrict__ st,
               uint32_t n, uint2 *__restrict__ claims, uint32_t claim_cap, Ctl *ctl) {
    extern __shared__ unsigned long long srec[];  // 2^sub_shift records
    __shared__ uint32_t touched[(1u << 14) / 32];
    __shared__ uint2 cbuf[kDelClaims];
    __shared__ uint32_t s_cross[kDelThreads / 32];
    __shared__ uint32_t s_cnt, s_base;
    __shared__ uint64_t dbar;
    const uint32_t nv = 1u << sub_shift;
    const uint32_t S = 1u << (g.shift - sub_shift);
    const uint32_t s = blockIdx.x;
    const uint32_t c = s / S, b = s % S;
    const uint32_t part = c / g.chunks_per_part;
    const uint32_t base_v = part * g.P + (c % g.chunks_per_part) * (1u << g.shift) + b * nv;
    const uint32_t part_end = (part + 1) * g.P;
    if (base_v >= part_end) return;  // a sub-bucket past the end of its part
    const uint32_t cnt = min(fill2[s], cap2);
    if (cnt == 0) return;
    const uint32_t lim = min(nv, part_end - base_v);
    // a sub-bucket with kDelBulk updates or more (a whole one, its records
    // 16-byte aligned) takes all its records by one bulk copy and gives them
    // back by one, instead of loading and storing the touched ones that a
    // bitmap finds (which reads the updates twice)
    const bool bulk = cnt >= kDelBulk && lim == nv && (base_v & 1u) == 0u;  // block-uniform
    if (threadIdx.x == 0) {
        s_cnt = 0;
        if (bulk) {
            mbar_init(&dbar, 1);
            mbar_init_fence();
        }
    }
    if (!bulk)
        for (uint32_t k = threadIdx.x; k < (nv + 31) / 32; k += kDelThreads) touched[k] = 0;
    __syncthreads();
    const uint2 *src = pairs2 + (size_t)s * cap2;
    // the bulk form's first updates (kDelPre per thread) load while its
    // records arrive
    uint2 pv0[kDelPre];
    if (bulk) {
        if (threadIdx.x == 0) bulk_load(srec, st + base_v, nv * 8u, &dbar);
#pragma unroll
        for (int u = 0; u < kDelPre; u++) {
            const uint32_t i = threadIdx.x + (uint32_t)u * kDelThreads;
            pv0[u] = i < cnt ? __ldcs(src + i) : make_uint2(0xFFFFFFFFu, 0u);  // {w, e}
        }
        if (!__syncthreads_and(mbar_wait(&dbar, 0u))) {  // the copy never landed
            if (threadIdx.x == 0) {
                raise_err(ctl, kDevTimeout);
                mbar_wait(&dbar, 0u);
            }
            __syncthreads();
            return;
        }
    }
    if (!bulk) {
      // every loop keeps kDelU independent loads in flight per thread
      for (uint32_t i0 = threadIdx.x; i0 < cnt; i0 += kDelU * kDelThreads) {
          uint32_t k[kDelU];
#pragma unroll
          for (int u = 0; u < kDelU; u++) {
              const uint32_t i = i0 + (uint32_t)u * kDelThreads;
              k[u] = i < cnt ? __ldcg(src + i).x - base_v : 0xFFFFFFFFu;
          }
#pragma unroll
          for (int u = 0; u < kDelU; u++)
              if (k[u] < lim) atomicOr(&touched[k[u] >> 5], 1u << (k[u] & 31u));
      }
      __syncthreads();
      // only the touched records: a warp's loads cover 32 consecutive records
      for (uint32_t k0 = threadIdx.x; k0 < lim; k0 += kDelU * kDelThreads) {
          unsigned long long r[kDelU];
          bool t[kDelU];
#pragma unroll
          for (int u = 0; u < kDelU; u++) {
              const uint32_t k = k0 + (uint32_t)u * kDelThreads;
              t[u] = k < lim && ((touched[k >> 5] >> (k & 31u)) & 1u);
              r[u] = t[u] ? __ldcg(st + base_v + k) : 0ull;
          }
#pragma unroll
          for (int u = 0; u < kDelU; u++)
              if (t[u]) srec[k0 + (uint32_t)u * kDelThreads] = r[u];
      }
      __syncthreads();
    }
    // claims gather in shared memory and leave with one reservation on the
    // list cursor per block (a claim beyond the buffer reserves its own slot)
    uint32_t cross = 0;
    for (uint32_t i0 = threadIdx.x; i0 < cnt; i0 += kDelU * kDelThreads) {
      uint2 pv[kDelU];
      const bool loaded = bulk && i0 == threadIdx.x;
#pragma unroll
      for (int u = 0; u < kDelU; u++) {
          const uint32_t i = i0 + (uint32_t)u * kDelThreads;
          pv[u] = loaded && u < kDelPre ? pv0[u < kDelPre ? u : 0]
                  : i < cnt                 ? __ldcs(src + i)
                                            : make_uint2(0xFFFFFFFFu, 0u);  // {w, e}
      }
#pragma unroll
      for (int u = 0; u < kDelU; u++) {
        const uint2 p = pv[u];
        if (i0 + (uint32_t)u * kDelThreads >= cnt) continue;
        const uint32_t k = p.x - base_v;
        if (k < lim) {
            const unsigned long long sub = 0ull - (((unsigned long long)p.y << 32) | 1ull);
            const unsigned long long old = atomicAdd(srec + k, sub);
            if ((uint32_t)old == 2u) {  // w falls to degree 1: claim its last edge
                cross++;
                const uint32_t gl = (uint32_t)(old >> 32) - p.y;
                if (gl < n) {
                    const uint32_t slot = atomicAdd(&s_cnt, 1u);
                    if (slot < kDelClaims) {
                        cbuf[slot] = make_uint2(gl, p.x);
                    } else {
                        const uint32_t g = atomicAdd(&ctl->ccur, 1u);
                        if (g < claim_cap)
                            claims[g] = make_uint2(gl, p.x);
                        else
                            raise_err(ctl, kDevRoundOverflow);
                    }
                } else {
                    raise_err(ctl, kDevBadEdge);
                }
            }
        } else {
            raise_err(ctl, kDevBadVertex);
        }
      }
    }
    if (bulk) fence_proxy_async_smem();  // this thread's shared atomics before the copy back
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t k = min(s_cnt, (uint32_t)kDelClaims);
        const uint32_t b = k ? atomicAdd(&ctl->ccur, k) : 0u;
        if (k && (b + k > claim_cap || b + k < b)) raise_err(ctl, kDevRoundOverflow);
        s_base = b;
    }
    __syncthreads();
    {
        const uint32_t k = min(s_cnt, (uint32_t)kDelClaims), b = s_base;
        for (uint32_t i = threadIdx.x; i < k; i += kDelThreads)
            if (b + i < claim_cap && b + i >= b) claims[b + i] = cbuf[i];
    }
    if (bulk) {
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();  // the shared atomics before the copy's reads
            bulk_store(st + base_v, srec, nv * 8u);
            bulk_store_wait_read();
        }
    } else {
        for (uint32_t k = threadIdx.x; k < lim; k += kDelThreads)
            if ((touched[k >> 5] >> (k & 31u)) & 1u) st[base_v + k] = srec[k];
    }
    const uint32_t wc = __reduce_add_sync(0xFFFFFFFFu, cross);
    if ((threadIdx.x & 31u) == 0) s_cross[threadIdx.x >> 5] = wc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int q = 0; q < kDelThreads / 32; q++) tot += s_cross[q];
        if (tot) atomicAdd(&ctl->cross, tot);
    }
}

// ------------------------------------------------------------------- claims --
// One block per edge sub-chunk of 2^esub edges: the claims of round tr on
// the sub-chunk (see the file comment).  The shared table keeps 4 bits per
// edge, bit j set when the vertex at position j claims the edge.  The block
// then takes its claims in spans of kResThreads * kResU (small blocks,
// several per SM, so one block's loads overlap another's scans).
#ifndef HPEEL_RES_THREADS
#define HPEEL_RES_THREADS 256
#endif
constexpr int kResThreads = HPEEL_RES_THREADS;
constexpr int kResU = 8;  // claims per thread and span
constexpr uint32_t kResSpan = (uint32_t)kResThreads * kResU;
constexpr uint32_t kEsub = 13;

// Exclusive block-wide prefix sum of one value per thread; *total gets the
// sum.  Every thread calls it; it ends with the block synchronised.
__device__ __forceinline__ uint32_t res_block_scan(uint32_t v, uint32_t *total) {
    constexpr int kW = kResThreads / 32;
    __shared__ uint32_t ws[kW];
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
        uint32_t w = lane < (uint32_t)kW ? ws[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
            if (lane >= (uint32_t)d) w += y;
        }
        if (lane < (uint32_t)kW) ws[lane] = w;
    }
    __syncthreads();
    const uint32_t before = (warp ? ws[warp - 1] : 0u) + x - v;
    *total = ws[kW - 1];
    return before;
}

#ifndef HPEEL_RES_MIN_BLOCKS
#define HPEEL_RES_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(kResThreads, HPEEL_RES_MIN_BLOCKS)
k_claim_resolve(const uint2 *__restrict__ pairs2, const uint32_t *__restrict__ fill2,
                uint32_t cap2, uint32_t esub, uint32_t n, uint32_t P, uint32_t round_add,
                uint4 *__restrict__ rec, uint4 *__restrict__ Lst, Ctl *ctl) {
    extern __shared__ uint32_t mtab[];  // 2^esub / 8 words
    __shared__ uint32_t s_base;
    const uint32_t s = blockIdx.x;
    const uint64_t e0 = (uint64_t)s << esub;
    if (e0 >= n) return;
    const uint32_t cnt = min(fill2[s], cap2);
    if (cnt == 0) return;
    const uint64_t left = (uint64_t)n - e0;
    const uint32_t ne = (uint32_t)(left < (1ull << esub) ? left : (1ull << esub));
    const uint32_t words = (ne + 7) / 8;
    for (uint32_t k = threadIdx.x; k < words; k += kResThreads) mtab[k] = 0;
    __syncthreads();
    const uint2 *src = pairs2 + (size_t)s * cap2;
    for (uint32_t i0 = threadIdx.x; i0 < cnt; i0 += kResU * kResThreads) {
        uint2 pv[kResU];
#pragma unroll
        for (int u = 0; u < kResU; u++) {
            const uint32_t i = i0 + (uint32_t)u * kResThreads;
            pv[u] = i < cnt ? __ldcg(src + i) : make_uint2(0u, 0u);  // {g, v}
        }
#pragma unroll
        for (int u = 0; u < kResU; u++) {
            if (i0 + (uint32_t)u * kResThreads >= cnt) continue;
            const uint32_t el = (uint32_t)(pv[u].x - e0);
            if (el < ne) {
                const uint32_t j = part_of<3>(pv[u].y, P);
                atomicOr(&mtab[el >> 3], (1u << j) << (4u * (el & 7u)));
            } else {
                raise_err(ctl, kDevBadEdge);
            }
        }
    }
    __syncthreads();
    const uint32_t tr = *(volatile uint32_t *)&ctl->round + round_add;
    // the claims again, a span at a time: the claim of each edge's smallest
    // claiming position (read from the table) lists the edge, unless an
    // earlier round took it; the work follows the claims, not the 2^esub
    // edges of the sub-chunk.  The entries of a span are placed by one
    // block-wide scan and reserved with one atomic.
    for (uint32_t sp = 0; sp < cnt; sp += kResSpan) {
        uint2 pv[kResU];
        uint32_t hj[kResU];
        uint4 q[kResU];
        bool win[kResU];
        uint32_t mine = 0;
#pragma unroll
        for (int u = 0; u < kResU; u++) {
            const uint32_t i = sp + (uint32_t)u * kResThreads + threadIdx.x;
            pv[u] = i < cnt ? __ldcs(src + i) : make_uint2(0u, 0u);
            const uint32_t el = (uint32_t)(pv[u].x - e0);
            hj[u] = part_of<3>(pv[u].y, P);
            const uint32_t bits = el < ne ? (mtab[el >> 3] >> (4u * (el & 7u))) & 0xFu : 0u;
            win[u] = i < cnt && el < ne && (bits & ((1u << hj[u]) - 1u)) == 0u;
            q[u] = win[u] ? __ldcg(rec + pv[u].x) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kResU; u++) {
            if (win[u] && q[u].w != kUnclaimed) win[u] = false;  // claimed in an earlier round
            mine += win[u] ? 1u : 0u;
        }
        uint32_t total;
        uint32_t pos = res_block_scan(mine, &total);
        if (threadIdx.x == 0) s_base = total ? atomicAdd(&ctl->lcur, total) : 0u;
        __syncthreads();
        pos += s_base;
#pragma unroll
        for (int u = 0; u < kResU; u++) {
            if (!win[u]) continue;
            const uint32_t e = pv[u].x, h = hj[u];
            rec[e].w = (tr << 2) | h;
            const uint32_t p[4] = {q[u].x, q[u].y, q[u].z, 0u};
            uint32_t x[4];
            rotate_to<3>(p, h, x);
            Lst[pos++] = make_uint4(x[0], x[1], x[2], e);
        }
        __syncthreads();  // s_base and the scan's table are reused by the next span
    }
}

// ------------------------------------------------------------------- close --
// Close the sorted part of a round (one thread): layer t+1 (or L_0 after
// round 0's claims) is [loff[t+1], lcur); decide how the next round runs and
// set the loop conditions: h_sorted = next round in sorted form, h_random =
// another round follows (the random loop takes over once a round is not
// sorted).
__global__ void k_sorted_close(Ctl *ctl, uint32_t *loff, uint32_t max_rounds, uint32_t first,
                               uint32_t min_edges, uint32_t max_edges,
                               cudaGraphConditionalHandle h_sorted,
                               cudaGraphConditionalHandle h_random) {
    const uint32_t t = ctl->round;
    const uint32_t end = ctl->lcur;
    uint32_t next, more;
    uint32_t err = ctl->err;
    if (first) {
        loff[0] = 0;
        loff[1] = end;
        ctl->first_layer = end;
        next = end;
        more = end > 0 ? 1u : 0u;
    } else {
        const uint32_t beg = loff[t + 1];
        loff[t + 2] = end;
        next = end - beg;
        more = end > beg ? 1u : 0u;
        if (more && t + 2 >= max_rounds) {  // round t+1 would overflow loff
            more = 0;
            if (!err) ctl->err = err = kDevCapacity;
        }
        ctl->round = t + 1;
        ctl->brounds += 1;
    }
    if (err) more = 0;  // stop on any device error
    const uint32_t sorted = more && next >= min_edges && next <= max_edges ? 1u : 0u;
    ctl->next_size = next;
    ctl->more = more;
    ctl->bmode = sorted;
    ctl->ccur = 0;
    ctl->done = 0;
    if (h_sorted) cudaGraphSetConditional(h_sorted, sorted);
    if (h_random) cudaGraphSetConditional(h_random, more);
}

// ---------------------------------------------------------------- host side --
SortedPlan sorted_plan(uint64_t n, uint64_t m, uint32_t r, const BucketPlan &b, uint32_t min_edges,
                       int sms) {
    SortedPlan p{};
    if (r != 3 || b.parts != 3 || b.passes != 1 || n == 0 || min_edges == 0xFFFFFFFFu) return p;
    const uint64_t P = m / 3;
    // the largest layer deleted in sorted form: covers L_0 up to gamma 1.35
    p.max_edges = (uint32_t)std::min<uint64_t>(n, (n * 3) / 10 + 1024);
    // automatic: a sorted round costs a fixed few ms at n = 1e9 plus about
    // 40 ps per edge, a random one ~110 ps per edge: sorted from 1/20 of the
    // edges (L_0, L_1 and L_2 at gamma = 1.23)
    p.min_edges = min_edges ? min_edges : (uint32_t)std::max<uint64_t>(1, n / 20);
    if (p.min_edges > p.max_edges) return p;
    // claims of one round: at most the degree-1 vertices of round 0 (a
    // fraction lambda e^-lambda <= 1/e of the vertices for random graphs)
    p.claim_cap = (uint32_t)std::min<uint64_t>(0xFFFFFFF0u, m * 38 / 100 + 4096);
    p.bucket_blocks = (uint32_t)std::max<int>(1, sms * HPEEL_BUCKET_BLOCKS);  // one wave of blocks
    p.claim_bucket_blocks = (uint32_t)std::max<int>(1, sms * HPEEL_CLAIM_BUCKET_BLOCKS);
    // updates, by vertex: the build's chunks and sub-buckets
    p.vg = BucketGeom{(uint32_t)P, b.shift, b.chunks_per_part, 0, kFillShift};
    p.vchunks = b.chunks;
    p.vsub_shift = b.sub_shift;
    p.vsubs = b.subs;
    // a chunk's array holds its share of the pairs of the largest layer
    // (share: the part of the pairs that the largest chunk receives; a
    // part's last chunk is partial, so a full chunk gets more than an even
    // split)
    auto chunk_cap = [&](uint64_t items, uint32_t per_item, double share) {
        const uint64_t all = items * per_item;
        const double e = (double)all * std::min(1.0, share);
        return (uint32_t)std::min<uint64_t>((uint64_t)(e + 8.0 * std::sqrt(e + 1.0) + 64.0),
                                            all);
    };
    // a part holds about a third of the updates (0.4 leaves room for the
    // hinge positions' skew)
    p.vg.cap = chunk_cap(p.max_edges, 2, 0.4 * (double)(1ull << b.shift) / (double)P);
    const double e2 = 2.0 * p.max_edges * 0.4 * (double)(1ull << p.vsub_shift) / (double)P;
    p.vcap2 = (uint32_t)std::min<uint64_t>((uint64_t)(e2 + 8.0 * std::sqrt(e2 + 1.0) + 256.0),
                                           2ull * p.max_edges);
    // claims, by edge: chunks of 2^eshift edges, sub-chunks of 2^esub
    p.esub = kEsub;
    p.eshift = 22;
    while (p.eshift > p.esub && ((n - 1) >> p.eshift) == 0 && p.eshift > 14) p.eshift--;
    p.eg = BucketGeom{(uint32_t)n, p.eshift, (uint32_t)((n + (1ull << p.eshift) - 1) >> p.eshift), 0,
                      kFillShift};
    p.echunks = p.eg.chunks_per_part;
    p.esubs = p.echunks << (p.eshift - p.esub);
    p.eg.cap = chunk_cap(p.claim_cap, 1, (double)(1ull << p.eshift) / (double)n);
    const double c2 = (double)p.claim_cap * (double)(1ull << p.esub) / (double)n;
    p.ecap2 = (uint32_t)std::min<uint64_t>((uint64_t)(c2 + 8.0 * std::sqrt(c2 + 1.0) + 256.0),
                                           p.claim_cap);
    // the refine indexes a chunk's sub-buckets with 32-bit arithmetic
    if (((uint64_t)p.vcap2 << (p.vg.shift - p.vsub_shift)) >= (1ull << 32) ||
        ((uint64_t)p.ecap2 << (p.eshift - p.esub)) >= (1ull << 32))
        return SortedPlan{};
    const uint32_t C = std::max(p.vchunks, p.echunks);
    p.bucket_smem = bucket_smem_bytes(C, true);
    p.claim_bucket_smem = bucket_smem_bytes(C, false);
    if (p.bucket_smem > (200u << 10)) return SortedPlan{};
    p.pairs_bytes = 8 * std::max<uint64_t>((uint64_t)p.vchunks * p.vg.cap,
                                           (uint64_t)p.echunks * p.eg.cap);
    p.fill_bytes = 4 * ((uint64_t)std::max(p.vchunks, p.echunks) << kFillShift);
    p.pairs2_bytes = 8 * std::max<uint64_t>((uint64_t)p.vsubs * p.vcap2,
                                            (uint64_t)p.esubs * p.ecap2);
    p.fill2_bytes = 4 * (uint64_t)std::max(p.vsubs, p.esubs);
    p.claims_bytes = 8 * (uint64_t)p.claim_cap;
    p.enabled = true;
    return p;
}

namespace {
void set_smem(const void *fn, size_t) { smem_optin(fn); }
}  // namespace

void launch_sorted_claims(const Launch &L, const SortedPlan &p, const SortedBufs &w, uint32_t n,
                          uint4 *rec, uint4 *Lst, Ctl *ctl, uint32_t round_add) {
    Overflow none{nullptr, nullptr, 0, kDevRoundOverflow};
    cudaMemsetAsync(w.fill, 0, 4 * ((size_t)p.echunks << kFillShift), L.stream);
    cudaMemsetAsync(w.fill2, 0, 4 * (size_t)p.esubs, L.stream);
    BucketGeom eg = p.eg;
    set_smem((const void *)k_pairs_bucket<3, false>, p.claim_bucket_smem);
    count_launch();
    k_pairs_bucket<3, false><<<p.claim_bucket_blocks, kBucketThreads, p.claim_bucket_smem,
                               L.stream>>>(
        nullptr, nullptr, w.claims, p.claim_cap, eg, p.echunks, w.pairs, w.fill, none, ctl);
    launch_refine(L, eg, p.echunks, 0, p.esub, w.pairs, w.fill, w.pairs2, w.fill2,
                  p.ecap2, none, ctl);
    const size_t tsmem = ((size_t)1 << p.esub) / 2;
    set_smem((const void *)k_claim_resolve, tsmem);
    count_launch();
    k_claim_resolve<<<p.esubs, kResThreads, tsmem, L.stream>>>(w.pairs2, w.fill2, p.ecap2, p.esub, n,
                                                           p.vg.P, round_add, rec, Lst, ctl);
}

void launch_sorted_round0(const Launch &L, const SortedPlan &p, const SortedBufs &w,
                          const unsigned long long *st, uint32_t n, uint32_t m, uint4 *rec,
                          uint4 *Lst, uint32_t *loff, Ctl *ctl, uint32_t max_rounds,
                          cudaGraphConditionalHandle h_sorted,
                          cudaGraphConditionalHandle h_random) {
    count_launch(2);
    k_round0_reset<<<1, 1, 0, L.stream>>>(ctl);
    k_round0_emit<<<grid_fixed(L, 8), kThreads, 0, L.stream>>>(st, m, n, w.claims, p.claim_cap,
                                                               ctl);
    launch_sorted_claims(L, p, w, n, rec, Lst, ctl, 0u);
    count_launch();
    k_sorted_close<<<1, 1, 0, L.stream>>>(ctl, loff, max_rounds, 1u, p.min_edges, p.max_edges,
                                          h_sorted, h_random);
}

void launch_sorted_round(const Launch &L, const SortedPlan &p, const SortedBufs &w,
                         unsigned long long *st, uint32_t n, uint4 *rec, uint4 *Lst,
                         uint32_t *loff, Ctl *ctl, uint32_t max_rounds,
                         cudaGraphConditionalHandle h_sorted, cudaGraphConditionalHandle h_random) {
    Overflow none{nullptr, nullptr, 0, kDevRoundOverflow};
    cudaMemsetAsync(w.fill, 0, 4 * ((size_t)p.vchunks << kFillShift), L.stream);
    cudaMemsetAsync(w.fill2, 0, 4 * (size_t)p.vsubs, L.stream);
    BucketGeom vg = p.vg;
    set_smem((const void *)k_pairs_bucket<3, true>, p.bucket_smem);
    count_launch();
    k_pairs_bucket<3, true><<<p.bucket_blocks, kBucketThreads, p.bucket_smem, L.stream>>>(
        Lst, loff, nullptr, 0, vg, p.vchunks, w.pairs, w.fill, none, ctl);
    launch_refine(L, vg, p.vchunks, 0, p.vsub_shift, w.pairs, w.fill, w.pairs2, w.fill2,
                  p.vcap2, none, ctl);
    const size_t dsmem = (size_t)8 << p.vsub_shift;
    set_smem((const void *)k_delete_apply, dsmem);
    count_launch();
    k_delete_apply<<<p.vsubs, kDelThreads, dsmem, L.stream>>>(w.pairs2, w.fill2, p.vcap2, vg,
                                                              p.vsub_shift, st, n, w.claims,
                                                              p.claim_cap, ctl);
    launch_sorted_claims(L, p, w, n, rec, Lst, ctl, 1u);
    count_launch();
    k_sorted_close<<<1, 1, 0, L.stream>>>(ctl, loff, max_rounds, 0u, p.min_edges, p.max_edges,
                                          h_sorted, h_random);
}

}  // namespace hp
