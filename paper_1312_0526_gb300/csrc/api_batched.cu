// api_batched.cu -- C ABI of the batched bucket peel (hpeel_peel_batched).
// Argument checks, tuning resolution and workspace layout; the work is the
// two kernels of batched.cu, issued without any host synchronisation, so a
// call can be captured into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "host.h"
#include "kernels.cuh"

using namespace hp;

namespace {

struct BatchPlan {
    uint32_t threads, ctas_per_sm, smem_bytes, smem_rounds, global16_rounds, grid;
    size_t sched, next, words, scanned, tmp, scratch, total;
};

hpeel_status batch_plan(uint32_t B, uint32_t gamma_milli, const hpeel_batch_tuning *tu,
                        BatchPlan *p) {
    int dev = 0;
    DeviceInfo d;
    if (cudaGetDevice(&dev) != cudaSuccess || device_info(dev, &d) != HPEEL_OK) {
        cudaGetLastError();
        d.sms = 152;  // no device: plan for one GB300
        d.smem_per_sm = 233472;
        d.smem_optin = 232448;
    }
    p->threads = tu && tu->threads ? tu->threads : 256u;
    p->ctas_per_sm = tu && tu->ctas_per_sm ? tu->ctas_per_sm : 2u;
    if (p->threads % 32 || p->threads < 64 || p->threads > 1024)
        return fail(HPEEL_ERR_INVALID_ARG, "threads = %u: need a multiple of 32 in [64, 1024]",
                    p->threads);
    if (p->ctas_per_sm > 32) return fail(HPEEL_ERR_INVALID_ARG, "ctas_per_sm > 32");
    p->smem_rounds = tu && tu->smem_rounds ? tu->smem_rounds : 256u;
    if (p->smem_rounds < 2 || p->smem_rounds > 16383)
        return fail(HPEEL_ERR_INVALID_ARG, "smem_rounds %u outside [2, 16383]", p->smem_rounds);
    p->global16_rounds = tu && tu->global16_rounds ? tu->global16_rounds : batched_claim16_rounds();
    if (p->global16_rounds < 2 || p->global16_rounds > batched_claim16_rounds())
        return fail(HPEEL_ERR_INVALID_ARG, "global16_rounds %u outside [2, %u]",
                    p->global16_rounds, batched_claim16_rounds());
    // default shared memory: fill the SM (1 KB per block is reserved by CUDA,
    // 64 B of static shared memory per block)
    const int per = d.smem_per_sm / (int)p->ctas_per_sm - 1024 - 64;
    uint32_t smem = tu && tu->smem_bytes ? tu->smem_bytes : (uint32_t)std::max(per, 0) & ~15u;
    smem = std::min<uint32_t>(smem, (uint32_t)d.smem_optin);
    p->smem_bytes = smem;
    p->grid = (uint32_t)d.sms * p->ctas_per_sm;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    p->sched = take(4 * (size_t)B + 4);
    p->next = take(4);
    p->words = take(4 * (size_t)B + 4);
    p->scanned = take(4 * (size_t)B + 4);
    p->tmp = take(4 * scan_tmp_words(B));
    p->scratch = take((size_t)p->grid * batched_scratch_bytes(gamma_milli));
    p->total = off;
    return HPEEL_OK;
}

hpeel_status check_gamma(uint32_t gamma_milli) {
    if (gamma_milli < 1000 || gamma_milli > batched_max_gamma_milli())
        return fail(HPEEL_ERR_INVALID_ARG, "gamma_milli = %u outside [1000, %u]", gamma_milli,
                    batched_max_gamma_milli());
    return HPEEL_OK;
}

}  // namespace

extern "C" {

size_t hpeel_batched_workspace_size(uint32_t B, uint32_t gamma_milli,
                                    const hpeel_batch_tuning *tuning) {
    BatchPlan p;
    if (batch_plan(B, gamma_milli ? gamma_milli : 1230, tuning, &p) != HPEEL_OK) return 0;
    return p.total;
}

hpeel_status hpeel_batched_g_offsets(const uint64_t *d_bucket_off, uint32_t B,
                                     uint32_t gamma_milli, uint64_t *d_G_off, void *d_ws,
                                     size_t ws_bytes, void *stream) {
    g_last_error.clear();
    HP_TRY(check_gamma(gamma_milli));
    if (!d_bucket_off || !d_G_off || !d_ws) return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    BatchPlan p;
    HP_TRY(batch_plan(B, gamma_milli, nullptr, &p));
    const size_t need = p.scratch;  // the offsets use only the regions before it
    if (ws_bytes < need)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes, need);
    Launch L;
    HP_TRY(make_launch(stream, &L));
    char *ws = (char *)d_ws;
    ProfScope ps(L, "batch_g_offsets");
    launch_batch_g_offsets(L, d_bucket_off, B, gamma_milli, reinterpret_cast<uint32_t *>(ws + p.words),
                           reinterpret_cast<uint32_t *>(ws + p.scanned),
                           reinterpret_cast<uint32_t *>(ws + p.tmp), d_G_off);
    return check_launch("batch_g_offsets");
}

hpeel_status hpeel_peel_batched(const uint64_t *d_keys, const uint64_t *d_bucket_off, uint32_t B,
                                uint32_t gamma_milli, uint32_t *d_order,
                                uint32_t *d_bucket_rounds, uint32_t *d_bucket_status,
                                uint64_t *d_G, const uint64_t *d_G_off,
                                const hpeel_batch_tuning *tuning, void *d_ws, size_t ws_bytes,
                                void *stream) {
    g_last_error.clear();
    HP_TRY(check_gamma(gamma_milli));
    if (B == 0) return HPEEL_OK;
    if (!d_keys || !d_bucket_off || !d_order || !d_ws)
        return fail(HPEEL_ERR_INVALID_ARG, "NULL pointer");
    if ((d_G == nullptr) != (d_G_off == nullptr))
        return fail(HPEEL_ERR_INVALID_ARG, "d_G and d_G_off go together");
    if (((uintptr_t)d_ws & 255u) != 0)
        return fail(HPEEL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    BatchPlan p;
    HP_TRY(batch_plan(B, gamma_milli, tuning, &p));
    if (ws_bytes < p.total)
        return fail(HPEEL_ERR_WORKSPACE_TOO_SMALL, "workspace %zu < %zu bytes", ws_bytes, p.total);
    Launch L;
    HP_TRY(make_launch(stream, &L));
    char *ws = (char *)d_ws;
    ProfScope ps(L, "batched");
    launch_batched(L, d_keys, d_bucket_off, B, gamma_milli, d_order, d_bucket_rounds,
                   d_bucket_status, d_G, d_G_off, p.threads, p.grid, p.smem_bytes,
                   p.smem_rounds, p.global16_rounds,
                   reinterpret_cast<uint32_t *>(ws + p.sched),
                   reinterpret_cast<uint32_t *>(ws + p.next), ws + p.scratch);
    return check_launch("batched");
}

}  // extern "C"
