// async.cu -- the device-driven MPHF build: the reseed-and-retry loop of
// sec. 3 (a hypergraph that keeps a 2-core is hashed again with the next
// seed) and the reverse-layer assignment loop run as conditional nodes of
// one CUDA graph, so a build needs no host round trip.  These one-thread
// kernels read what the previous kernels left in the control block and set
// the conditions of the loops around them.
#include "kernels.cuh"

namespace hp {

__global__ void k_async_init(AsyncState *s, uint64_t seed, uint32_t max_tries, uint32_t n) {
    s->seed0 = seed;
    s->seed = seed;
    s->attempt = 0;
    s->max_tries = max_tries;
    s->status = kAsyncRunning;
    s->rounds = 0;
    s->t = -1;
    s->n = n;
}

// After the build: 1 when the bucketed build overflowed (the attempt is
// redone with direct updates of the vertex records, as the host path does).
__global__ void k_async_check_overflow(const Ctl *ctl, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, ctl->err == kDevBuildOverflow ? 1u : 0u);
}

// 1 when the control block holds error code `code` (an if node redoes what
// raised it).
__global__ void k_async_check_code(const Ctl *ctl, uint32_t code, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, ctl->err == code ? 1u : 0u);
}

// After the round loop: stop on success, on a device error or when the
// seeds are used up; otherwise take the next seed and loop again.
__global__ void k_async_decide(AsyncState *s, const Ctl *ctl, cudaGraphConditionalHandle h) {
    uint32_t again = 0;
    if (ctl->err) {
        s->status = kAsyncDeviceError;
    } else if (ctl->lcur == s->n) {
        s->status = kAsyncPeeled;
        s->rounds = ctl->more ? ctl->round + 1 : ctl->round;
    } else if (s->attempt + 1 < s->max_tries) {
        s->attempt += 1;
        s->seed += 1;
        again = 1;
    } else {
        s->status = kAsyncRetriesExhausted;
    }
    cudaGraphSetConditional(h, again);
}

__global__ void k_async_if_peeled(const AsyncState *s, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, s->status == kAsyncPeeled ? 1u : 0u);
}

// Assignment loop: layers R-1 down to 0, one launch of k_assign_at each.
__global__ void k_async_assign_init(AsyncState *s, cudaGraphConditionalHandle h) {
    s->t = (int32_t)s->rounds - 1;
    cudaGraphSetConditional(h, s->t >= 0 ? 1u : 0u);
}

__global__ void k_async_assign_step(AsyncState *s, cudaGraphConditionalHandle h) {
    s->t -= 1;
    cudaGraphSetConditional(h, s->t >= 0 ? 1u : 0u);
}

__global__ void k_async_stats(const AsyncState *s, const Ctl *ctl, hpeel_stats *out) {
    hpeel_stats st{};
    // a check that fails after a successful peel (a static-function value
    // not below sigma) turns the outcome into a device error
    const uint32_t status =
        s->status == kAsyncPeeled && ctl->err ? (uint32_t)kAsyncDeviceError : s->status;
    st.n_peeled = ctl->lcur;
    st.rounds = ctl->more ? ctl->round + 1 : ctl->round;
    st.core_nonempty = status == kAsyncRetriesExhausted ? 1u : 0u;
    st.seed_used = status == kAsyncPeeled ? s->seed : 0ull;
    st.attempts = s->attempt + 1;
    st.device_err = status == kAsyncDeviceError ? ctl->err : 0u;
    st.first_layer = ctl->first_layer;
    st.frontier = ctl->cross;
    st.hinge_moves = ctl->moves;
    st.sorted_rounds = ctl->brounds;
    st.async_status = status;
    *out = st;
}

// ------------------------------------------------------ device-driven peel --
// 1 when no kernel raised a device error: the canonical order runs.
__global__ void k_async_if_ok(const Ctl *ctl, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, ctl->err == 0u ? 1u : 0u);
}

// Stats of a device-driven peel: async_status 1 = peeled (order and claims
// written; core_nonempty tells whether a 2-core is left), 3 = a device check
// failed (device_err holds the code; outputs not written), 4 = more rounds
// than the caller's layer table holds (order and claims written, layer
// offsets not).
__global__ void k_peel_async_stats(const Ctl *ctl, uint32_t n, uint32_t max_layers,
                                   uint32_t want_layer_off, hpeel_stats *out) {
    hpeel_stats st{};
    st.n_peeled = ctl->lcur;
    st.rounds = ctl->more ? ctl->round + 1 : ctl->round;
    st.core_nonempty = ctl->lcur < n ? 1u : 0u;
    st.attempts = 1;
    st.device_err = ctl->err;
    st.first_layer = ctl->first_layer;
    st.frontier = ctl->cross;
    st.hinge_moves = ctl->moves;
    st.sorted_rounds = ctl->brounds;
    st.async_status = ctl->err ? 3u : (want_layer_off && st.rounds > max_layers ? 4u : 1u);
    *out = st;
}

// No edges: an empty order, no round.
__global__ void k_peel_async_empty(hpeel_stats *out, uint64_t *layer_off) {
    hpeel_stats st{};
    st.attempts = 1;
    st.async_status = 1u;
    *out = st;
    if (layer_off) layer_off[0] = 0;
}

void launch_async_if_ok(const Launch &L, const Ctl *ctl, cudaGraphConditionalHandle h) {
    count_launch();
    k_async_if_ok<<<1, 1, 0, L.stream>>>(ctl, h);
}
void launch_peel_async_stats(const Launch &L, const Ctl *ctl, uint32_t n, uint32_t max_layers,
                             bool want_layer_off, hpeel_stats *out) {
    count_launch();
    k_peel_async_stats<<<1, 1, 0, L.stream>>>(ctl, n, max_layers, want_layer_off ? 1u : 0u, out);
}
void launch_peel_async_empty(const Launch &L, hpeel_stats *out, uint64_t *layer_off) {
    count_launch();
    k_peel_async_empty<<<1, 1, 0, L.stream>>>(out, layer_off);
}

// No keys: nothing to peel; the stats of a build that succeeded at once.
__global__ void k_async_empty(hpeel_stats *out, uint64_t seed, uint64_t *D) {
    hpeel_stats st{};
    st.seed_used = seed;
    st.attempts = 1;
    st.async_status = kAsyncPeeled;
    *out = st;
    if (D) D[0] = 0;
}

void launch_async_empty(const Launch &L, hpeel_stats *out, uint64_t seed, uint64_t *D) {
    count_launch();
    k_async_empty<<<1, 1, 0, L.stream>>>(out, seed, D);
}
void launch_async_init(const Launch &L, AsyncState *s, uint64_t seed, uint32_t max_tries,
                       uint32_t n) {
    count_launch();
    k_async_init<<<1, 1, 0, L.stream>>>(s, seed, max_tries, n);
}
void launch_async_check_overflow(const Launch &L, const Ctl *ctl, cudaGraphConditionalHandle h) {
    count_launch();
    k_async_check_overflow<<<1, 1, 0, L.stream>>>(ctl, h);
}
void launch_async_check_code(const Launch &L, const Ctl *ctl, uint32_t code,
                             cudaGraphConditionalHandle h) {
    count_launch();
    k_async_check_code<<<1, 1, 0, L.stream>>>(ctl, code, h);
}
void launch_async_decide(const Launch &L, AsyncState *s, const Ctl *ctl,
                         cudaGraphConditionalHandle h) {
    count_launch();
    k_async_decide<<<1, 1, 0, L.stream>>>(s, ctl, h);
}
void launch_async_if_peeled(const Launch &L, const AsyncState *s, cudaGraphConditionalHandle h) {
    count_launch();
    k_async_if_peeled<<<1, 1, 0, L.stream>>>(s, h);
}
void launch_async_assign_init(const Launch &L, AsyncState *s, cudaGraphConditionalHandle h) {
    count_launch();
    k_async_assign_init<<<1, 1, 0, L.stream>>>(s, h);
}
void launch_async_assign_step(const Launch &L, AsyncState *s, cudaGraphConditionalHandle h) {
    count_launch();
    k_async_assign_step<<<1, 1, 0, L.stream>>>(s, h);
}
void launch_async_stats(const Launch &L, const AsyncState *s, const Ctl *ctl, hpeel_stats *out) {
    count_launch();
    k_async_stats<<<1, 1, 0, L.stream>>>(s, ctl, out);
}

}  // namespace hp
