// peel.cu -- packed incidence build and round-synchronous peeling.
//
// State: one 8-byte record per vertex, {deg, xor of incident edge ids}
// (sec. 4.1, the labelled packed incidence list with the edge id as label).
// Round t (sec. 4.2):
//   claim  -- every vertex v of the frontier F_t that still has degree 1
//             retrieves its edge e = xor[v] and writes (t << 2) | j into
//             claim[e] with atomicMin, j = position of v in the edge.  The
//             minimum is the hinge (smallest position), whatever the order
//             of the atomics; the one thread that sees the unclaimed value
//             appends e to the layer L_t, so an edge enters L_t once (the
//             deduplication of D_i into P_i).
//   update -- every edge of L_t is deleted (DeleteEdge) from its non-hinge
//             vertices: atomicSub on deg, atomicXor on xor.  The hinge keeps
//             its record: its only edge is gone and it is in no later
//             frontier, so nothing reads it again.  A vertex whose degree
//             drops from 2 to 1 is appended to F_{t+1}; each vertex crosses
//             that step at most once, so the frontiers F_1, F_2, ... fit in
//             one list of m entries and the layers in one list of n.
// Round 0 scans all m records instead of a list (F_0 is never stored).
// Kernels read t and the list bounds from the device control block, so the
// host loop needs no per-round arguments.
#include "kernels.cuh"

namespace hp {

__global__ void k_fill_u32(uint32_t *__restrict__ p, uint64_t count, uint32_t value) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t head = (16u - ((uintptr_t)p & 15u)) / 4u % 4u;  // words to 16 B alignment
    if (((uintptr_t)p & 3u) == 0 && count > head + 4) {
        for (uint64_t k = i; k < head; k += stride) p[k] = value;
        uint4 *p4 = reinterpret_cast<uint4 *>(p + head);
        const uint64_t n4 = (count - head) / 4;
        const uint4 v4 = make_uint4(value, value, value, value);
        for (uint64_t k = i; k < n4; k += stride) p4[k] = v4;
        for (uint64_t k = head + n4 * 4 + i; k < count; k += stride) p[k] = value;
    } else {
        for (uint64_t k = i; k < count; k += stride) p[k] = value;
    }
}

void launch_fill_u32(const Launch &L, uint32_t *p, uint64_t count, uint32_t value) {
    if (count == 0) return;
    count_launch();
    k_fill_u32<<<grid_for(L, count, 16, 8), kThreads, 0, L.stream>>>(p, count, value);
}

// ---------------------------------------------------------------- build --
// Four edges per thread: r uint4 loads hold 4 whole rows (coalesced).
template <int R>
__global__ void __launch_bounds__(kThreads)
k_build(const uint32_t *__restrict__ edges, uint32_t n, uint32_t P, uint32_t *__restrict__ st,
        uint32_t *__restrict__ claim, Ctl *ctl) {
    const uint64_t groups = ((uint64_t)n + 3) / 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const bool aligned = ((((uintptr_t)edges) | ((uintptr_t)claim)) & 15u) == 0;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
        const uint32_t e0 = (uint32_t)(g * 4);
        const uint32_t cnt = min(4u, n - e0);
        uint32_t w[4 * R];
        if (cnt == 4 && aligned) {
            const uint4 *p = reinterpret_cast<const uint4 *>(edges + (uint64_t)e0 * R);
#pragma unroll
            for (int q = 0; q < R; q++) {
                const uint4 t = __ldcs(p + q);
                w[4 * q + 0] = t.x;
                w[4 * q + 1] = t.y;
                w[4 * q + 2] = t.z;
                w[4 * q + 3] = t.w;
            }
            *reinterpret_cast<uint4 *>(claim + e0) =
                make_uint4(kUnclaimed, kUnclaimed, kUnclaimed, kUnclaimed);
        } else {
#pragma unroll
            for (int q = 0; q < 4 * R; q++)
                w[q] = (q / R < (int)cnt) ? edges[(uint64_t)e0 * R + q] : 0u;
            for (uint32_t k = 0; k < cnt; k++) claim[e0 + k] = kUnclaimed;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (k < (int)cnt) {
                const uint32_t e = e0 + k;
#pragma unroll
                for (int j = 0; j < R; j++) {
                    const uint32_t v = w[k * R + j];
                    if (v - (uint32_t)j * P >= P) {  // outside part j
                        raise_err(ctl, kDevBadVertex);
                        continue;
                    }
                    atomicAdd(st + 2ull * v, 1u);
                    atomicXor(st + 2ull * v + 1, e);
                }
            }
        }
    }
}

void launch_build_incidence(const Launch &L, const uint32_t *edges, uint32_t n, uint32_t r,
                            uint32_t P, uint32_t *state, uint32_t *claim, Ctl *ctl) {
    if (n == 0) return;
    const unsigned grid = grid_for(L, ((uint64_t)n + 3) / 4, 1, 8);
    switch (r) {
    case 2: count_launch(); k_build<2><<<grid, kThreads, 0, L.stream>>>(edges, n, P, state, claim, ctl); break;
    case 3: count_launch(); k_build<3><<<grid, kThreads, 0, L.stream>>>(edges, n, P, state, claim, ctl); break;
    case 4: count_launch(); k_build<4><<<grid, kThreads, 0, L.stream>>>(edges, n, P, state, claim, ctl); break;
    }
}

// ---------------------------------------------------------------- round 0 --
// kR0Items vertices per thread per block step, strided by the block size so
// every record load is coalesced; one block-aggregated append per step.
constexpr int kR0Items = 4;

template <int R>
__global__ void __launch_bounds__(kThreads)
k_round0(const uint2 *__restrict__ st, uint32_t m, uint32_t P, uint32_t n,
         uint32_t *__restrict__ claim, uint32_t *__restrict__ Llist, Ctl *ctl) {
    constexpr uint32_t kStep = kThreads * kR0Items;
    const uint64_t stride = (uint64_t)gridDim.x * kStep;
    for (uint64_t base = (uint64_t)blockIdx.x * kStep; base < m; base += stride) {
        bool take[kR0Items];
        uint32_t e[kR0Items];
#pragma unroll
        for (int k = 0; k < kR0Items; k++) {
            const uint64_t v = base + (uint64_t)k * kThreads + threadIdx.x;
            take[k] = false;
            e[k] = 0;
            if (v < m) {
                const uint2 s = __ldcs(st + v);
                if (s.x == 1u) {
                    e[k] = s.y;
                    if (s.y < n) {
                        const uint32_t j = part_of<R>((uint32_t)v, P);
                        take[k] = atomicMin(claim + s.y, j) == kUnclaimed;
                    } else {
                        raise_err(ctl, kDevBadEdge);
                    }
                }
            }
        }
        block_append<kR0Items, kThreads>(&ctl->lcur, Llist, take, e);
    }
}

void launch_round0(const Launch &L, const uint32_t *state, uint32_t m, uint32_t r, uint32_t P,
                   uint32_t n, uint32_t *claim, uint32_t *Llist, Ctl *ctl) {
    if (m == 0) return;
    const unsigned grid = grid_for(L, m, kR0Items, 8);
    const uint2 *st = reinterpret_cast<const uint2 *>(state);
    switch (r) {
    case 2: count_launch(); k_round0<2><<<grid, kThreads, 0, L.stream>>>(st, m, P, n, claim, Llist, ctl); break;
    case 3: count_launch(); k_round0<3><<<grid, kThreads, 0, L.stream>>>(st, m, P, n, claim, Llist, ctl); break;
    case 4: count_launch(); k_round0<4><<<grid, kThreads, 0, L.stream>>>(st, m, P, n, claim, Llist, ctl); break;
    }
}

// ---------------------------------------------------------------- claim --
constexpr int kClaimItems = 4;

template <int R>
__global__ void __launch_bounds__(kThreads)
k_claim(const uint2 *__restrict__ st, uint32_t P, uint32_t n, uint32_t *__restrict__ claim,
        const uint32_t *__restrict__ F, uint32_t *__restrict__ Llist, uint32_t *__restrict__ foff,
        Ctl *ctl) {
    constexpr uint32_t kStep = kThreads * kClaimItems;
    const uint32_t t = *(volatile uint32_t *)&ctl->round;
    const uint32_t fb = foff[t];
    const uint32_t fe = *(volatile uint32_t *)&ctl->fcur;
    if (blockIdx.x == 0 && threadIdx.x == 0) foff[t + 1] = fe;  // F_{t+1} starts here
    const uint64_t stride = (uint64_t)gridDim.x * kStep;
    for (uint64_t base = fb + (uint64_t)blockIdx.x * kStep; base < fe; base += stride) {
        bool take[kClaimItems];
        uint32_t e[kClaimItems];
#pragma unroll
        for (int k = 0; k < kClaimItems; k++) {
            const uint64_t i = base + (uint64_t)k * kThreads + threadIdx.x;
            take[k] = false;
            e[k] = 0;
            if (i < fe) {
                const uint32_t v = F[i];
                const uint2 s = st[v];
                if (s.x == 1u) {
                    e[k] = s.y;
                    if (s.y < n) {
                        const uint32_t tag = (t << 2) | part_of<R>(v, P);
                        take[k] = atomicMin(claim + s.y, tag) == kUnclaimed;
                    } else {
                        raise_err(ctl, kDevBadEdge);
                    }
                }
            }
        }
        block_append<kClaimItems, kThreads>(&ctl->lcur, Llist, take, e);
    }
}

void launch_claim(const Launch &L, const uint32_t *state, uint32_t r, uint32_t P, uint32_t n,
                  uint32_t *claim, const uint32_t *F, uint32_t *Llist, uint32_t *foff,
                  Ctl *ctl) {
    const unsigned grid = grid_fixed(L, 8);
    const uint2 *st = reinterpret_cast<const uint2 *>(state);
    switch (r) {
    case 2: count_launch(); k_claim<2><<<grid, kThreads, 0, L.stream>>>(st, P, n, claim, F, Llist, foff, ctl); break;
    case 3: count_launch(); k_claim<3><<<grid, kThreads, 0, L.stream>>>(st, P, n, claim, F, Llist, foff, ctl); break;
    case 4: count_launch(); k_claim<4><<<grid, kThreads, 0, L.stream>>>(st, P, n, claim, F, Llist, foff, ctl); break;
    }
}

// ---------------------------------------------------------------- update --
constexpr int kUpdItems = 2;  // edges per thread per block step

template <int R>
__global__ void __launch_bounds__(kThreads)
k_update(const uint32_t *__restrict__ edges, uint32_t m, const uint32_t *__restrict__ claim,
         uint32_t *__restrict__ st, const uint32_t *__restrict__ Llist, uint32_t *__restrict__ F,
         uint32_t *__restrict__ loff, const uint32_t *__restrict__ foff, Ctl *ctl) {
    constexpr uint32_t kStep = kThreads * kUpdItems;
    constexpr int K = kUpdItems * (R - 1);
    const uint32_t t = *(volatile uint32_t *)&ctl->round;
    const uint32_t lb = loff[t];
    const uint32_t le = *(volatile uint32_t *)&ctl->lcur;
    if (blockIdx.x == 0 && threadIdx.x == 0) loff[t + 1] = le;  // L_t = [lb, le)
    const uint64_t stride = (uint64_t)gridDim.x * kStep;
    for (uint64_t base = lb + (uint64_t)blockIdx.x * kStep; base < le; base += stride) {
        bool app[K];
        uint32_t wv[K];
#pragma unroll
        for (int q = 0; q < kUpdItems; q++) {
            const uint64_t i = base + (uint64_t)q * kThreads + threadIdx.x;
            uint32_t e = 0, h = 0xFFu;
            uint32_t w[R];
            if (i < le) {
                e = Llist[i];
                h = claim[e] & 3u;
#pragma unroll
                for (int j = 0; j < R; j++) w[j] = edges[(uint64_t)e * R + j];
            }
#pragma unroll
            for (int k = 0; k < R - 1; k++) {
                app[q * (R - 1) + k] = false;
                wv[q * (R - 1) + k] = 0;
                if (h == 0xFFu) continue;
                // k-th non-hinge position: positions after the hinge shift by one
                const int j = k + ((uint32_t)k >= h ? 1 : 0);
                const uint32_t x = w[j];
                if (x < m) {
                    const uint32_t old = atomicSub(st + 2ull * x, 1u);
                    atomicXor(st + 2ull * x + 1, e);
                    app[q * (R - 1) + k] = (old == 2u);
                    wv[q * (R - 1) + k] = x;
                } else {
                    raise_err(ctl, kDevBadVertex);
                }
            }
        }
        block_append<K, kThreads>(&ctl->fcur, F, app, wv);
    }
    // The last block to finish closes the round: F_{t+1} = [foff[t+1], fcur).
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&ctl->done, 1u);
        if (d == gridDim.x - 1) {
            __threadfence();
            const uint32_t fe = atomicAdd(&ctl->fcur, 0u);
            ctl->more = (fe > foff[t + 1] && le > lb) ? 1u : 0u;
            ctl->last_layer = le - lb;
            ctl->done = 0;
            ctl->round = t + 1;
        }
    }
}

void launch_update(const Launch &L, const uint32_t *edges, uint32_t r, uint32_t m,
                   const uint32_t *claim, uint32_t *state, const uint32_t *Llist, uint32_t *F,
                   uint32_t *loff, const uint32_t *foff, Ctl *ctl) {
    const unsigned grid = grid_fixed(L, 8);
    switch (r) {
    case 2: count_launch(); k_update<2><<<grid, kThreads, 0, L.stream>>>(edges, m, claim, state, Llist, F, loff, foff, ctl); break;
    case 3: count_launch(); k_update<3><<<grid, kThreads, 0, L.stream>>>(edges, m, claim, state, Llist, F, loff, foff, ctl); break;
    case 4: count_launch(); k_update<4><<<grid, kThreads, 0, L.stream>>>(edges, m, claim, state, Llist, F, loff, foff, ctl); break;
    }
}

}  // namespace hp
