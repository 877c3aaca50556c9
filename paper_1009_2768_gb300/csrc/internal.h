// internal.h -- definitions shared by the translation units of libtrmc.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "trmc.h"

namespace trmc {
// A cell of at least kBigCell particles gets its moment sums from a pre-pass
// spread over eight CTAs (one per virtual warp of the canonical sums) instead
// of its own CTA alone: one table entry per slot, slot = cell mod kBigSlots.
constexpr int kBigCell = 32768;
constexpr int kBigSlots = 64;
struct BigEntry {
    int64_t cell;                     // the slot's cell in the launch that wrote it
    uint64_t stamp;                   // that launch's number
    double part[8 * 5];               // per virtual warp, its K partial sums as the CTA stores them
};
}  // namespace trmc

struct trmc_ctx {
    int precision = 0;
    uint64_t seed = 0;
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    // device workspace: [control block 4 KiB][collide slabs]
    char *workspace = nullptr;
    size_t workspace_bytes = 0;
    int *status = nullptr;            // [0] error code, [1] detail (cell), [2..3] spare
    unsigned int *tickets = nullptr;  // [0] next cell, [1] CTAs done, [2] largest cell (collide)
    trmc::BigEntry *big = nullptr;    // [kBigSlots] large cells' moment sums (control block)
    uint64_t big_stamp = 0;           // collide launches that ran the pre-pass
    // host-mapped word: the largest cell of the last collide launch (written by
    // its last CTA; UINT_MAX until the first launch), and its device address
    volatile unsigned int *n_max_host = nullptr;
    unsigned int *n_max_dev = nullptr;
    char *slabs = nullptr;
    size_t slabs_bytes = 0;
    // transport scratch, grown on demand
    int64_t *tr_counts = nullptr;     // [3 * cells] moves -1/0/+1 per old cell
    void *tr_dom = nullptr;           // per-domain mover set-up (transport), [tr_ndom]
    int tr_ndom = 0;
    int tr_cells = 0;
    // collide launch shape (trmc_set_collide_launch)
    int collide_threads = 128;
    int collide_ctas_per_sm = 4;
    // collide work schedule (trmc_set_collide_schedule; 0: the precision's default)
    int collide_warp_particles = 0;
    int collide_records_per_thread = 0;
    // transport sort launch shape (trmc_set_transport_launch; 0: by mean cell size)
    int transport_threads = 0;
    std::string last_error;
};

namespace trmc {

constexpr int kMC = TRMC_MCAP;
constexpr int kThreads = 256;         // collide CTA size, at most (whole-staging kernels)
constexpr int kThreadsDual = 512;     // the dual-mode kernels', and the most a context may set

trmc_status set_error(trmc_ctx *ctx, trmc_status code, const std::string &msg);
// Host checks of a collision step's state and parameters, shared by
// trmc_collide and trmc_collide_static: NULL if they are valid, else why not.
const char *check_collide_args(const trmc_state *state, const trmc_collide_params *p);
trmc_status cuda_error(trmc_ctx *ctx, cudaError_t e, const char *where);

trmc_status launch_collide(trmc_ctx *ctx, trmc_state *st, const trmc_collide_params *prm,
                           uint64_t step, int64_t *report, trmc_stats *stats, cudaStream_t s);
trmc_status launch_transport(trmc_ctx *ctx, trmc_state *st, const trmc_domain *domains,
                             int32_t n_domains, double cfl, double *dt, uint64_t step, cudaStream_t s);
trmc_status launch_init(trmc_ctx *ctx, trmc_state *st, const double *cell_init, cudaStream_t s);
trmc_status launch_moments(trmc_ctx *ctx, const trmc_state *st, double *out, cudaStream_t s);

}  // namespace trmc
