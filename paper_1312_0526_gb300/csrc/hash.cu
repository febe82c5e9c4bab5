// hash.cu -- key -> edge hashing into r disjoint vertex ranges.
//
// sec. 3: each key x becomes the edge {h_0(x), ..., h_{r-1}(x)}; sec. 4.3:
// h_j has codomain [j m/r, (j+1) m/r), so the r vertices of an edge are
// distinct.  Here h_j(x) = (mix64(x ^ (seed + j)) mod P) + j P, P = m / r.
// For a general hypergraph every h_j maps into all of [0, m) (sec. 3's
// h_j: S -> [gamma n]): the same kernel with P = m and no part offset.
#include "kernels.cuh"

namespace hp {

// One key per thread: 8-byte coalesced key loads; the r ids of an edge are
// staged in shared memory so the block writes its whole edge tile with
// 16-byte coalesced stores.
// part_stride: P for the r-partite form, 0 for a general hypergraph.
template <int R>
__global__ void __launch_bounds__(kThreads)
k_hash_edges(const uint64_t *__restrict__ keys, uint64_t n, FastMod fm, uint64_t seed,
             uint32_t part_stride, uint32_t *__restrict__ edges) {
    __shared__ __align__(16) uint32_t tile[kThreads * R];
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    const uint32_t P = part_stride;
    for (uint64_t base = (uint64_t)blockIdx.x * kThreads; base < n; base += stride) {
        const uint64_t i = base + threadIdx.x;
        const uint32_t cnt = (n - base < (uint64_t)kThreads) ? (uint32_t)(n - base) : (uint32_t)kThreads;
        if (i < n) {
            const uint64_t k = keys[i];
#pragma unroll
            for (int j = 0; j < R; j++)
                tile[threadIdx.x * R + j] =
                    (uint32_t)fastmod(mix64(k ^ (seed + (uint64_t)j)), fm) + (uint32_t)j * P;
        }
        __syncthreads();
        uint32_t *dst = edges + base * R;
        const uint32_t words = cnt * R;
        if (cnt == kThreads && (((uintptr_t)dst) & 15u) == 0) {
            // kThreads * R words is a multiple of 4: whole uint4 stores
            const uint4 *src4 = reinterpret_cast<const uint4 *>(tile);
            uint4 *dst4 = reinterpret_cast<uint4 *>(dst);
            for (uint32_t q = threadIdx.x; q < words / 4; q += kThreads) dst4[q] = src4[q];
        } else {
            for (uint32_t q = threadIdx.x; q < words; q += kThreads) dst[q] = tile[q];
        }
        __syncthreads();
    }
}

void launch_hash_edges(const Launch &L, const uint64_t *keys, uint64_t n, uint32_t r,
                       FastMod fm, uint64_t seed, uint32_t *edges, bool gen) {
    if (n == 0) return;
    const unsigned grid = grid_for(L, n, 1, 8);
    const uint32_t ps = gen ? 0u : (uint32_t)fm.P;
    count_launch();
    switch (r) {
    case 2: k_hash_edges<2><<<grid, kThreads, 0, L.stream>>>(keys, n, fm, seed, ps, edges); break;
    case 3: k_hash_edges<3><<<grid, kThreads, 0, L.stream>>>(keys, n, fm, seed, ps, edges); break;
    case 4: k_hash_edges<4><<<grid, kThreads, 0, L.stream>>>(keys, n, fm, seed, ps, edges); break;
    }
}

// Keys -> edge records {v_0, v_1, v_2, unclaimed} (the MPHF path keeps its
// edges only as records): one 16-byte coalesced store per key.
template <int R>
__global__ void __launch_bounds__(kThreads)
k_hash_records(const uint64_t *__restrict__ keys, uint64_t n, FastMod fm, uint64_t seed,
               const uint64_t *seed_dev, uint4 *__restrict__ rec) {
    if (seed_dev) seed = *seed_dev;  // the seed of a device-driven attempt
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    const uint32_t P = (uint32_t)fm.P;
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        const uint64_t k = __ldcs(keys + i);
        uint32_t v[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < R; j++)
            v[j] = (uint32_t)fastmod(mix64(k ^ (seed + (uint64_t)j)), fm) + (uint32_t)j * P;
        store_record<R>(rec, i, v, true);
    }
}

void launch_hash_records(const Launch &L, const uint64_t *keys, uint64_t n, uint32_t r,
                         FastMod fm, uint64_t seed, uint4 *rec, const uint64_t *seed_dev) {
    if (n == 0) return;
    const unsigned grid = grid_for(L, n, 1, 8);
    count_launch();
    switch (r) {
    case 2: k_hash_records<2><<<grid, kThreads, 0, L.stream>>>(keys, n, fm, seed, seed_dev, rec); break;
    case 3: k_hash_records<3><<<grid, kThreads, 0, L.stream>>>(keys, n, fm, seed, seed_dev, rec); break;
    case 4: k_hash_records<4><<<grid, kThreads, 0, L.stream>>>(keys, n, fm, seed, seed_dev, rec); break;
    }
}

}  // namespace hp
