// api.cu -- the C ABI of libtrmc: context lifetime, argument checks,
// launches.  Every entry point validates on the host, launches
// asynchronously on the caller's stream and returns a trmc_status.
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace trmc {

trmc_status set_error(trmc_ctx *ctx, trmc_status code, const std::string &msg)
{
    if (ctx) ctx->last_error = msg;
    return code;
}

trmc_status cuda_error(trmc_ctx *ctx, cudaError_t e, const char *where)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    return set_error(ctx, TRMC_ERR_CUDA, buf);
}

namespace {

constexpr size_t kControlBytes = 4096 + 32768;     // status, tickets; large-cell table

trmc_status check_state(trmc_ctx *ctx, const trmc_state *st)
{
    if (!st) return set_error(ctx, TRMC_ERR_ARG, "state is NULL");
    if (st->n_cells < 0) return set_error(ctx, TRMC_ERR_ARG, "n_cells < 0");
    if (st->n_cells > 0 && (!st->vx || !st->vy || !st->vz || !st->cell_start))
        return set_error(ctx, TRMC_ERR_ARG, "state velocity arrays or cell_start are NULL");
    if (st->capacity < 0) return set_error(ctx, TRMC_ERR_ARG, "capacity < 0");
    return TRMC_OK;
}

}  // namespace

const char *check_collide_args(const trmc_state *state, const trmc_collide_params *p)
{
    if (!state) return "state is NULL";
    if (state->n_cells < 0) return "n_cells < 0";
    if (state->n_cells > 0 && (!state->vx || !state->vy || !state->vz || !state->cell_start))
        return "state velocity arrays or cell_start are NULL";
    if (state->capacity < 0) return "capacity < 0";
    if (!p) return "params is NULL";
    if (p->trunc < TRMC_TRUNC_FIXED || p->trunc > TRMC_TRUNC_WB) return "bad trunc";
    if (p->trunc == TRMC_TRUNC_WB) {
        if (p->wb_length < TRMC_LEN_K || p->wb_length > TRMC_LEN_MEAN)
            return "TRMC-WB needs wb_length in {TRMC_LEN_K, TRMC_LEN_MIN, TRMC_LEN_MEAN}";
        if (p->m_fixed < 0) return "TRMC-WB needs m_fixed (m_max) >= 0";
    } else if (p->wb_length != 0) {
        return "params.wb_length must be 0 unless trunc is TRMC_TRUNC_WB";
    }
    if (p->m_cap < 1 || p->m_cap > TRMC_MCAP) return "m_cap outside [1, TRMC_MCAP]";
    if (p->trunc == TRMC_TRUNC_FIXED && (p->m_fixed < 1 || p->m_fixed > p->m_cap)) return "m_fixed outside [1, m_cap]";
    if (p->trunc == TRMC_TRUNC_RAD) {
        if (!state->m_max) return "TRMC-RAD needs state.m_max";
        if (p->m_min < 1 || p->m_min > p->m_cap) return "m_min outside [1, m_cap]";
        if (!(p->delta1 >= 0.0) || !(p->delta2 >= p->delta1)) return "need 0 <= delta1 <= delta2";
        if (p->indicator != TRMC_IND_PXX && p->indicator != TRMC_IND_M4) return "bad indicator";
    }
    if (!state->cell_param) {
        if (!(p->eps > 0.0)) return "eps must be > 0";
        if (!(p->dt >= 0.0)) return "dt must be >= 0";
        if (!(p->alpha >= 0.0 && p->alpha <= 1.0)) return "alpha outside [0, 1]";
        if (!(p->rho_scale >= 0.0)) return "rho_scale must be >= 0";
    }
    return nullptr;
}

}  // namespace trmc

using namespace trmc;

extern "C" {

trmc_status trmc_create(trmc_ctx **out, int32_t precision, uint64_t seed, size_t workspace_bytes)
{
    if (!out) return TRMC_ERR_ARG;
    *out = nullptr;
    if (precision != TRMC_FP64 && precision != TRMC_FP32_MIXED) return TRMC_ERR_ARG;
    trmc_ctx *ctx = new (std::nothrow) trmc_ctx();
    if (!ctx) return TRMC_ERR_NOMEM;
    ctx->precision = precision;
    ctx->seed = seed;
    cudaError_t e = cudaGetDevice(&ctx->device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, ctx->device);
    if (e != cudaSuccess) { delete ctx; return TRMC_ERR_CUDA; }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    if (workspace_bytes == 0) workspace_bytes = size_t(1) << 30;
    ctx->workspace_bytes = workspace_bytes + kControlBytes;
    e = cudaMalloc(&ctx->workspace, ctx->workspace_bytes);
    if (e != cudaSuccess) { delete ctx; return TRMC_ERR_NOMEM; }
    e = cudaMemset(ctx->workspace, 0, kControlBytes);
    if (e != cudaSuccess) { cudaFree(ctx->workspace); delete ctx; return TRMC_ERR_CUDA; }
    ctx->status = reinterpret_cast<int *>(ctx->workspace);
    ctx->tickets = reinterpret_cast<unsigned int *>(ctx->workspace + 64);
    ctx->big = reinterpret_cast<trmc::BigEntry *>(ctx->workspace + 4096);
    static_assert(sizeof(trmc::BigEntry) * trmc::kBigSlots <= 32768, "large-cell table");
    // the largest cell of the last collide launch, written by the device into
    // host-mapped memory and read by the next launch without a copy
    unsigned int *h = nullptr;
    e = cudaHostAlloc(reinterpret_cast<void **>(&h), sizeof(unsigned int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *h = ~0u;
        e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&ctx->n_max_dev), h, 0);
        if (e != cudaSuccess) { cudaFreeHost(h); h = nullptr; ctx->n_max_dev = nullptr; }
    }
    if (e != cudaSuccess) { cudaFree(ctx->workspace); delete ctx; return TRMC_ERR_CUDA; }
    ctx->n_max_host = h;
    ctx->slabs = ctx->workspace + kControlBytes;
    ctx->slabs_bytes = workspace_bytes;
    *out = ctx;
    return TRMC_OK;
}

trmc_status trmc_destroy(trmc_ctx *ctx)
{
    if (!ctx) return TRMC_ERR_ARG;
    if (ctx->workspace) cudaFree(ctx->workspace);
    if (ctx->n_max_host) cudaFreeHost(const_cast<unsigned int *>(ctx->n_max_host));
    if (ctx->tr_counts) cudaFree(ctx->tr_counts);
    if (ctx->tr_dom) cudaFree(ctx->tr_dom);
    delete ctx;
    return TRMC_OK;
}

const char *trmc_last_error(const trmc_ctx *ctx)
{
    if (!ctx) return "no context";
    return ctx->last_error.c_str();
}

trmc_status trmc_check(trmc_ctx *ctx, void *stream)
{
    if (!ctx) return TRMC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "trmc_check");
    int st[2] = {0, 0};
    e = cudaMemcpy(st, ctx->status, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(ctx, e, "trmc_check read");
    if (st[0] == 0) return TRMC_OK;
    e = cudaMemset(ctx->status, 0, 2 * sizeof(int));
    if (e != cudaSuccess) return cuda_error(ctx, e, "trmc_check clear");
    char buf[160];
    const char *what = st[0] == TRMC_ERR_CAPACITY ? "cell did not fit in the workspace (left unchanged)"
                       : st[0] == TRMC_ERR_STATE  ? "a particle moved more than one cell (dt too large)"
                       : st[0] == TRMC_ERR_TIMEOUT ? "device wait timed out"
                                                   : "device error";
    std::snprintf(buf, sizeof buf, "%s; first cell %d", what, st[1]);
    return set_error(ctx, static_cast<trmc_status>(st[0]), buf);
}

trmc_status trmc_set_collide_launch(trmc_ctx *ctx, int32_t threads, int32_t ctas_per_sm)
{
    if (!ctx) return TRMC_ERR_ARG;
    if (threads < 32 || threads > kThreadsDual || threads % 32 != 0)
        return set_error(ctx, TRMC_ERR_ARG, "threads must be a multiple of 32 in [32, 512]");
    if (ctas_per_sm < 1 || ctas_per_sm > 16) return set_error(ctx, TRMC_ERR_ARG, "ctas_per_sm outside [1, 16]");
    ctx->collide_threads = threads;
    ctx->collide_ctas_per_sm = ctas_per_sm;
    return TRMC_OK;
}

trmc_status trmc_set_collide_schedule(trmc_ctx *ctx, int32_t warp_particles, int32_t records_per_thread)
{
    if (!ctx) return TRMC_ERR_ARG;
    if (warp_particles != 0 && (warp_particles < 2 || warp_particles > 8192 || warp_particles % 2 != 0))
        return set_error(ctx, TRMC_ERR_ARG, "warp_particles must be 0 or even in [2, 8192]");
    if (records_per_thread < 0 || records_per_thread > 16)
        return set_error(ctx, TRMC_ERR_ARG, "records_per_thread must be 0 or in [1, 16]");
    ctx->collide_warp_particles = warp_particles;
    ctx->collide_records_per_thread = records_per_thread;
    return TRMC_OK;
}

trmc_status trmc_set_transport_launch(trmc_ctx *ctx, int32_t threads)
{
    if (!ctx) return TRMC_ERR_ARG;
    if (threads != 0 && (threads < 32 || threads > 256 || threads % 32 != 0))
        return set_error(ctx, TRMC_ERR_ARG, "transport threads must be 0 or a multiple of 32 in [32, 256]");
    ctx->transport_threads = threads;
    return TRMC_OK;
}

trmc_status trmc_init_cells(trmc_ctx *ctx, trmc_state *state, const double *cell_init_dev, void *stream)
{
    if (!ctx) return TRMC_ERR_ARG;
    trmc_status r = check_state(ctx, state);
    if (r != TRMC_OK) return r;
    if (state->n_cells > 0 && !cell_init_dev) return set_error(ctx, TRMC_ERR_ARG, "cell_init_dev is NULL");
    return launch_init(ctx, state, cell_init_dev, static_cast<cudaStream_t>(stream));
}

trmc_status trmc_collide(trmc_ctx *ctx, trmc_state *state, const trmc_collide_params *p, uint64_t step,
                         int64_t *report_dev, trmc_stats *stats_dev, void *stream)
{
    if (!ctx) return TRMC_ERR_ARG;
    trmc_status r = check_state(ctx, state);
    if (r != TRMC_OK) return r;
    const char *why = check_collide_args(state, p);
    if (why) return set_error(ctx, TRMC_ERR_ARG, why);
    if (state->n_cells == 0) return TRMC_OK;
    return launch_collide(ctx, state, p, step, report_dev, stats_dev, static_cast<cudaStream_t>(stream));
}

trmc_status trmc_transport(trmc_ctx *ctx, trmc_state *state, const trmc_domain *domains_dev, int32_t n_domains,
                           double cfl, double *dt_dev, uint64_t step, void *stream)
{
    if (!ctx) return TRMC_ERR_ARG;
    trmc_status r = check_state(ctx, state);
    if (r != TRMC_OK) return r;
    if (state->n_cells == 0) return TRMC_OK;
    if (!state->x || !state->x_alt || !state->vx_alt || !state->vy_alt || !state->vz_alt || !state->cell_start_alt)
        return set_error(ctx, TRMC_ERR_ARG, "transport needs x and the *_alt arrays");
    if (n_domains < 1 || !domains_dev) return set_error(ctx, TRMC_ERR_ARG, "need at least one domain");
    if (!dt_dev) return set_error(ctx, TRMC_ERR_ARG, "dt_dev is NULL");
    if (cfl > 1.0) return set_error(ctx, TRMC_ERR_ARG, "cfl > 1 would move particles more than one cell");
    if (cfl > 0.0 && !state->cell_vmax2) return set_error(ctx, TRMC_ERR_ARG, "CFL mode needs state.cell_vmax2");
    return launch_transport(ctx, state, domains_dev, n_domains, cfl, dt_dev, step, static_cast<cudaStream_t>(stream));
}

trmc_status trmc_moments(trmc_ctx *ctx, const trmc_state *state, double *out_dev, void *stream)
{
    if (!ctx) return TRMC_ERR_ARG;
    trmc_status r = check_state(ctx, state);
    if (r != TRMC_OK) return r;
    if (state->n_cells > 0 && !out_dev) return set_error(ctx, TRMC_ERR_ARG, "out_dev is NULL");
    return launch_moments(ctx, state, out_dev, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
