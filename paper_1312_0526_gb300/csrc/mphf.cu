// mphf.cu -- MWHC assignment and rank directory (r = 3).
//
// sec. 3: find u with u[h_0(x)] + u[h_1(x)] + u[h_2(x)] = f(x) (mod 3), where
// f(x) = i for the hinge h_i(x) of x's edge; then h_{f(x)} is a perfect hash
// and a rank over the non-zero u makes it minimal.  sec. 4.3 ("Avoiding
// backward scans"): layers are solved from the last to the first, and the
// order inside a layer is free.  Inside one layer no edge reads a 2-bit
// value another edge of the layer writes (a hinge has degree 1 in its round,
// so it belongs to no other edge alive then), so one launch per layer solves
// the whole layer in parallel; edges that share a 64-bit word of G combine
// their bits with atomicOr.
// sec. 5: the rank counts non-zero 2-bit pairs of a word with a broadword
// expression instead of a bit loop.
#include "kernels.cuh"

namespace hp {

// Solve the list entries [lb, le) of one layer: each {v_hinge, v_a, v_b, e}
// with the hinge position the part of v_hinge, read as a stream.  A thread
// takes kAssignU entries at a time and issues all their loads first.
#ifndef HPEEL_ASSIGN_U
#define HPEEL_ASSIGN_U 4
#endif
constexpr int kAssignU = HPEEL_ASSIGN_U;

__device__ __forceinline__ void assign_range(const uint4 *__restrict__ Lst, uint32_t lb,
                                             uint32_t le, uint32_t P, uint64_t *G) {
    const uint64_t stride = (uint64_t)gridDim.x * kThreads * kAssignU;
    for (uint64_t i0 = lb + (uint64_t)blockIdx.x * kThreads * kAssignU + threadIdx.x; i0 < le;
         i0 += stride) {
        uint4 s[kAssignU];
#pragma unroll
        for (int u = 0; u < kAssignU; u++) {
            const uint64_t i = i0 + (uint64_t)u * kThreads;
            s[u] = i < le ? __ldcs(Lst + i) : make_uint4(0u, 0u, 0u, 0u);
        }
        uint64_t wa[kAssignU], wb[kAssignU];
#pragma unroll
        for (int u = 0; u < kAssignU; u++) {
            const bool ok = i0 + (uint64_t)u * kThreads < le;
            wa[u] = ok ? __ldcg(G + (s[u].y >> 5)) : 0ull;
            wb[u] = ok ? __ldcg(G + (s[u].z >> 5)) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kAssignU; u++) {
            if (i0 + (uint64_t)u * kThreads >= le) continue;
            const uint32_t h = part_of<3>(s[u].x, P);
            const uint32_t sum = (uint32_t)(wa[u] >> (2u * (s[u].y & 31u)) & 3u) +
                                 (uint32_t)(wb[u] >> (2u * (s[u].z & 31u)) & 3u);
            const uint32_t val = (h + 6u - sum) % 3u;  // sum <= 6
            const uint64_t code = val ? val : 3u;
            atomicOr((unsigned long long *)(G + (s[u].x >> 5)),
                     (unsigned long long)(code << (2u * (s[u].x & 31u))));
        }
    }
}

// Layer t: list entries loff[t] .. loff[t+1].
__global__ void __launch_bounds__(kThreads)
k_assign(const uint4 *__restrict__ Lst, const uint32_t *__restrict__ loff, uint32_t t,
         uint32_t P, uint64_t *G) {
    assign_range(Lst, loff[t], loff[t + 1], P, G);
}

void launch_assign_layer(const Launch &L, const uint4 *Lst, const uint32_t *loff, uint32_t t,
                         uint32_t P, uint64_t *G) {
    count_launch();
    k_assign<<<grid_fixed(L, 8), kThreads, 0, L.stream>>>(Lst, loff, t, P, G);
}

// The same, for the layer whose index the device holds (the assignment loop
// of a device-driven build).
__global__ void __launch_bounds__(kThreads)
k_assign_at(const uint4 *__restrict__ Lst, const uint32_t *__restrict__ loff, const int32_t *t,
            uint32_t P, uint64_t *G) {
    const uint32_t tt = (uint32_t)*(volatile const int32_t *)t;
    assign_range(Lst, __ldcg(loff + tt), __ldcg(loff + tt + 1), P, G);
}

void launch_assign_layer_at(const Launch &L, const uint4 *Lst, const uint32_t *loff,
                            const int32_t *t, uint32_t P, uint64_t *G) {
    count_launch();
    k_assign_at<<<grid_fixed(L, 8), kThreads, 0, L.stream>>>(Lst, loff, t, P, G);
}

// Non-zero 2-bit values of a word: a pair is non-zero when either bit is set.
__device__ __forceinline__ uint32_t nonzero_pairs(uint64_t w) {
    return (uint32_t)__popcll((w | (w >> 1)) & 0x5555555555555555ull);
}

// One thread per 512 vertices (16 words of G, 32 vertices per word).
__global__ void k_rank_counts(const uint64_t *__restrict__ G, uint64_t words, uint64_t blocks,
                              uint32_t *__restrict__ cnt) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < blocks; b += stride) {
        uint32_t c = 0;
        const uint64_t w0 = b * 16;
        if (w0 + 16 <= words && ((((uintptr_t)G) & 15u) == 0)) {
            const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(G + w0);
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const ulonglong2 x = p[q];
                c += nonzero_pairs(x.x) + nonzero_pairs(x.y);
            }
        } else {
            for (uint64_t w = w0; w < words && w < w0 + 16; w++) c += nonzero_pairs(G[w]);
        }
        cnt[b] = c;
    }
}

void launch_rank_counts(const Launch &L, const uint64_t *G, uint64_t m, uint32_t *cnt) {
    const uint64_t words = (m + 31) / 32, blocks = (m + 511) / 512;
    if (blocks == 0) return;
    count_launch();
    k_rank_counts<<<grid_for(L, blocks, 1, 8), kThreads, 0, L.stream>>>(G, words, blocks, cnt);
}

__global__ void k_widen_dir(const uint32_t *__restrict__ scanned, const uint32_t *__restrict__ cnt,
                            uint64_t blocks, uint64_t *__restrict__ dir) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= blocks; b += stride) {
        if (b < blocks)
            dir[b] = scanned[b];
        else
            dir[b] = blocks ? (uint64_t)scanned[blocks - 1] + cnt[blocks - 1] : 0ull;
    }
}

void launch_widen_dir(const Launch &L, const uint32_t *scanned, const uint32_t *cnt,
                      uint64_t blocks, uint64_t *dir) {
    count_launch();
    k_widen_dir<<<grid_for(L, blocks + 1, 1, 8), kThreads, 0, L.stream>>>(scanned, cnt, blocks,
                                                                          dir);
}

// ------------------------------------------------------ static functions --
// sec. 3: any f: S -> [sigma] is stored as u with f(x) = u[h0] + u[h1] +
// u[h2] mod sigma, b = ceil(log2 sigma) bits per vertex in one bit string
// (vertex v at bits [v b, (v + 1) b), bit i in word i / 64): a value may
// straddle two words, so it is read from one or two words and set with one
// or two atomicOr.  The MPHF above is the case sigma = 3, f = hinge.
__device__ __forceinline__ uint64_t u_get(const uint64_t *U, uint32_t v, uint32_t b) {
    const uint64_t bit = (uint64_t)v * b;
    const uint64_t w = bit >> 6;
    const uint32_t sh = (uint32_t)(bit & 63u);
    uint64_t x = __ldcg(U + w) >> sh;
    if (sh + b > 64) x |= __ldcg(U + w + 1) << (64 - sh);
    return x & ((1ull << b) - 1ull);  // b <= 32
}

__device__ __forceinline__ void u_or(uint64_t *U, uint32_t v, uint32_t b, uint64_t x) {
    const uint64_t bit = (uint64_t)v * b;
    const uint64_t w = bit >> 6;
    const uint32_t sh = (uint32_t)(bit & 63u);
    atomicOr((unsigned long long *)(U + w), (unsigned long long)(x << sh));
    if (sh + b > 64) atomicOr((unsigned long long *)(U + w + 1), (unsigned long long)(x >> (64 - sh)));
}

// Layer t: for each entry {v_hinge, v_a, v_b, e}, u[v_hinge] = (values[e] -
// u[v_a] - u[v_b]) mod sigma.  Inside one layer no entry reads a value
// another entry of the layer writes (as for the MPHF), so the layer is one
// parallel launch.  A value >= sigma raises kDevBadValue.
__device__ __forceinline__ void sf_assign_range(const uint4 *__restrict__ Lst, uint32_t lb,
                                                uint32_t le, const uint32_t *__restrict__ values,
                                                FastMod fs, uint32_t b, uint64_t *U, Ctl *ctl) {
    const uint64_t sigma = fs.P;
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t i = lb + (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < le; i += stride) {
        const uint4 s = __ldcg(Lst + i);
        const uint32_t f = __ldg(values + s.w);
        if (f >= sigma) {
            raise_err(ctl, kDevBadValue);
            continue;
        }
        const uint64_t other = fastmod(u_get(U, s.y, b) + u_get(U, s.z, b), fs);
        const uint64_t val = fastmod((uint64_t)f + sigma - other, fs);
        if (val) u_or(U, s.x, b, val);
    }
}

__global__ void __launch_bounds__(kThreads)
k_sf_assign(const uint4 *__restrict__ Lst, const uint32_t *__restrict__ loff, uint32_t t,
            const uint32_t *__restrict__ values, FastMod fs, uint32_t b, uint64_t *U, Ctl *ctl) {
    sf_assign_range(Lst, __ldcg(loff + t), __ldcg(loff + t + 1), values, fs, b, U, ctl);
}

// The same, for the layer whose index the device holds (device-driven build).
__global__ void __launch_bounds__(kThreads)
k_sf_assign_at(const uint4 *__restrict__ Lst, const uint32_t *__restrict__ loff, const int32_t *t,
               const uint32_t *__restrict__ values, FastMod fs, uint32_t b, uint64_t *U,
               Ctl *ctl) {
    const uint32_t tt = (uint32_t)*(volatile const int32_t *)t;
    sf_assign_range(Lst, __ldcg(loff + tt), __ldcg(loff + tt + 1), values, fs, b, U, ctl);
}

void launch_sf_assign_layer_at(const Launch &L, const uint4 *Lst, const uint32_t *loff,
                               const int32_t *t, const uint32_t *values, uint64_t sigma,
                               uint32_t b, uint64_t *U, Ctl *ctl) {
    count_launch();
    k_sf_assign_at<<<grid_fixed(L, 8), kThreads, 0, L.stream>>>(Lst, loff, t, values,
                                                               make_fastmod(sigma), b, U, ctl);
}

void launch_sf_assign_layer(const Launch &L, const uint4 *Lst, const uint32_t *loff, uint32_t t,
                            const uint32_t *values, uint64_t sigma, uint32_t b, uint64_t *U,
                            Ctl *ctl) {
    count_launch();
    k_sf_assign<<<grid_fixed(L, 8), kThreads, 0, L.stream>>>(Lst, loff, t, values,
                                                            make_fastmod(sigma), b, U, ctl);
}

// f(key) = (u[h0] + u[h1] + u[h2]) mod sigma.
__global__ void __launch_bounds__(kThreads)
k_sf_lookup(const uint64_t *__restrict__ keys, uint64_t nq, FastMod fm, uint64_t seed,
            FastMod fs, uint32_t b, const uint64_t *__restrict__ U, uint32_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    const uint32_t P = (uint32_t)fm.P;
    for (uint64_t q = (uint64_t)blockIdx.x * kThreads + threadIdx.x; q < nq; q += stride) {
        const uint64_t k = __ldcs(keys + q);
        uint64_t s = 0;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const uint32_t v =
                (uint32_t)fastmod(mix64(k ^ (seed + (uint64_t)j)), fm) + (uint32_t)j * P;
            s += u_get(U, v, b);
        }
        out[q] = (uint32_t)fastmod(s, fs);
    }
}

void launch_sf_lookup(const Launch &L, const uint64_t *keys, uint64_t nq, FastMod fm,
                      uint64_t seed, uint64_t sigma, uint32_t b, const uint64_t *U,
                      uint32_t *out) {
    if (nq == 0) return;
    count_launch();
    k_sf_lookup<<<grid_for(L, nq, 1, 8), kThreads, 0, L.stream>>>(keys, nq, fm, seed,
                                                                  make_fastmod(sigma), b, U, out);
}

// ---------------------------------------------------------------- lookup --
// MPHF value of a key (sec. 3 and sec. 5): hash to h_0..h_2, i = (g[h_0] +
// g[h_1] + g[h_2]) mod 3 (a stored 3 counts as 0), v = h_i, and the value is
// the rank of v among the assigned vertices: the directory entry of v's
// 512-vertex block plus the non-zero pairs before v inside the block,
// counted a word at a time with the broadword expression.
__global__ void __launch_bounds__(kThreads)
k_lookup(const uint64_t *__restrict__ keys, uint64_t nq, FastMod fm, uint64_t seed,
         const uint64_t *__restrict__ G, const uint64_t *__restrict__ dir,
         uint32_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    const uint32_t P = (uint32_t)fm.P;
    for (uint64_t q = (uint64_t)blockIdx.x * kThreads + threadIdx.x; q < nq; q += stride) {
        const uint64_t k = __ldcs(keys + q);
        uint32_t v[3], g = 0;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            v[j] = (uint32_t)fastmod(mix64(k ^ (seed + (uint64_t)j)), fm) + (uint32_t)j * P;
            g += (uint32_t)(__ldg(G + (v[j] >> 5)) >> (2u * (v[j] & 31u))) & 3u;
        }
        const uint32_t i = g % 3u;
        const uint32_t x = i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
        const uint32_t blk = x >> 9, w_end = x >> 5;
        uint64_t rank = __ldg(dir + blk);
        for (uint32_t w = blk << 4; w < w_end; w++) rank += nonzero_pairs(__ldg(G + w));
        const uint32_t sh = 2u * (x & 31u);
        if (sh) rank += nonzero_pairs(__ldg(G + w_end) & ((1ull << sh) - 1ull));
        out[q] = (uint32_t)rank;
    }
}

void launch_lookup(const Launch &L, const uint64_t *keys, uint64_t nq, FastMod fm, uint64_t seed,
                   const uint64_t *G, const uint64_t *dir, uint32_t *out) {
    if (nq == 0) return;
    count_launch();
    k_lookup<<<grid_for(L, nq, 1, 8), kThreads, 0, L.stream>>>(keys, nq, fm, seed, G, dir, out);
}

}  // namespace hp
