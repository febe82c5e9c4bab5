/*
 * probe.h -- random-access ceiling probe (measurement only; no counterpart in
 * the paper and not part of the peeling library's boundary).
 *
 * The rounds of sec. 4.2 touch vertex records and edge records at addresses
 * nothing predicts, so their speed limit is the rate at which the memory
 * system serves random sector requests, not the copy bandwidth.  The probe
 * runs n_ops operations of one kind at addresses drawn from SplitMix64 of
 * (seed + operation number), asynchronously on stream; time it with CUDA
 * events on that stream.
 *   kind 0: 64-bit atomicAdd of 1 to a random 8-byte word of d_a;
 *   kind 1: 8-byte load of a random word of d_a (d_a should hold zeros: the
 *           loaded values are summed and the first word of d_a is written
 *           only for one impossible sum);
 *   kind 2: one peeled edge: a 16-byte load of a random 16-byte record of
 *           d_a, then an atomicMin of the operation number (low 32 bits) into
 *           the record's last word (the claim), then a 64-bit atomicAdd of 1
 *           to each of two random 8-byte words of d_b (the two DeleteEdge
 *           updates).
 * d_a: a_bytes of device memory, 16-byte aligned; d_b: b_bytes, 8-byte
 * aligned (kind 2 only).  Returns 0 when enqueued, 1 for an invalid
 * argument, 2 for a CUDA error.
 */
#ifndef HPEEL_MEASURE_PROBE_H
#define HPEEL_MEASURE_PROBE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif
int hpeel_measure_random_access(uint32_t kind, uint64_t n_ops, void *d_a, size_t a_bytes,
                                void *d_b, size_t b_bytes, uint64_t seed, void *stream);
#ifdef __cplusplus
}
#endif
#endif
