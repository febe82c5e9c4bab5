// probe.cu -- random-access ceiling of the memory system (measurement only;
// built into its own library, libhpeel_measure.so, which only the benchmark
// and its test load: nothing of it is part of the peeling library).
//
// The peeling rounds (sec. 4.2) touch one vertex record per DeleteEdge and
// one edge record per claim, each at an address no other access predicts:
// their speed is the rate at which the memory system serves random 32-byte
// sector requests, not the copy bandwidth.  These kernels replay that access
// pattern on synthetic indices (SplitMix64 of the operation number) so that
// the rounds can be compared with the rate the same pattern reaches alone.
#include <cuda_runtime.h>

#include "common.cuh"
#include "probe.h"

namespace hp {

// kind 0: 64-bit atomicAdd at a random word of A
__global__ void k_probe_rmw(uint64_t n_ops, unsigned long long *A, FastMod fa, uint64_t seed) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops; i += stride)
        atomicAdd(A + fastmod(mix64(seed + i), fa), 1ull);
}

// kind 1: 8-byte load from a random word of A (summed so it is not dropped)
__global__ void k_probe_read(uint64_t n_ops, const unsigned long long *A, FastMod fa, uint64_t seed,
                             unsigned long long *sink) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long acc = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops; i += stride)
        acc += __ldcg(A + fastmod(mix64(seed + i), fa));
    if (acc == 0x5a5a5a5a5a5a5a5aull) *sink = acc;  // never true for zeroed words
}

// kind 2: one peeled edge -- the claim (a 16-byte record read, then an
// atomicMin on the record's last word, whose address depends on the read so
// that it hits L2) and the two DeleteEdge updates of vertex words of B
__global__ void k_probe_edge(uint64_t n_ops, uint4 *A, FastMod fa, unsigned long long *B,
                             FastMod fb, uint64_t seed) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops; i += stride) {
        const uint64_t h = mix64(seed + i);
        const uint64_t e = fastmod(h, fa);
        const uint4 r = __ldcg(A + e);
        uint32_t *claim = reinterpret_cast<uint32_t *>(A + e) + 3 - (r.x == 0xFFFFFFFFu ? 1 : 0);
        atomicMin(claim, (uint32_t)i);
        atomicAdd(B + fastmod(mix64(h ^ 1u), fb), 1ull);
        atomicAdd(B + fastmod(mix64(h ^ 2u), fb), 1ull);
    }
}

}  // namespace hp

using namespace hp;

extern "C" int hpeel_measure_random_access(uint32_t kind, uint64_t n_ops, void *d_a,
                                           size_t a_bytes, void *d_b, size_t b_bytes,
                                           uint64_t seed, void *stream) {
    if (kind > 2) return 1;
    const size_t unit = kind == 2 ? 16 : 8;
    if (!d_a || a_bytes < unit || ((uintptr_t)d_a & 15u)) return 1;
    if (kind == 2 && (!d_b || b_bytes < 8 || ((uintptr_t)d_b & 7u))) return 1;
    if (n_ops == 0) return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 2;
    const unsigned grid = (unsigned)sms * 8;
    const cudaStream_t s = (cudaStream_t)stream;
    const FastMod fa = make_fastmod(a_bytes / unit);
    if (kind == 0) {
        k_probe_rmw<<<grid, 256, 0, s>>>(n_ops, (unsigned long long *)d_a, fa, seed);
    } else if (kind == 1) {
        // the sink is the first word: written only for an impossible sum
        k_probe_read<<<grid, 256, 0, s>>>(n_ops, (const unsigned long long *)d_a, fa, seed,
                                          (unsigned long long *)d_a);
    } else {
        k_probe_edge<<<grid, 256, 0, s>>>(n_ops, (uint4 *)d_a, fa, (unsigned long long *)d_b,
                                          make_fastmod(b_bytes / 8), seed);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
