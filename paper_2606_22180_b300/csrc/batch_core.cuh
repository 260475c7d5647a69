// Job and plan structures of the multi-graph runtime (batching and serving
// forms), and the host calls that build and run plans.
#pragma once

#include <cstddef>
#include <vector>

#include "noise_core.cuh"

namespace felog {

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kBTile = 4096;
constexpr int kBTileItems = kBTile / kBThreads;  // 16 per thread

struct BJob {
    const int32_t *offsets, *cols;
    int64_t nnz;
    int32_t n, dim;
    uint64_t seed;
    void *phi_in, *phi_out;
    uint8_t *active[2];
    int32_t *starts, *walks;
    uint32_t *counts;
    uint64_t *thr;
    int32_t *alias;
    uint64_t *W;
    u128 *key;
    int32_t *rank;
    u128 *light_D;
    int32_t *heavy_idx;
    u128 *heavy_E;
    int32_t tile_base, n_tiles;
    long long *acc_in, *acc_out;           // MINIBATCH: fixed-point increments [n][dim]
    uint32_t *mark_in, *mark_out;          // MINIBATCH: touched rows [n]
    struct BState *st;                     // this job's state (in the job's own memory)
    int32_t *rec_n_active, *rec_n_next;    // [max_rounds]
    double *rec_loss;                      // [max_rounds]
};

struct BState {
    int32_t round, cur, n_active, n_next;
    int32_t done, phase;  // phase 0: tables and V_a not initialised yet
    int64_t clock, n_live;
    int64_t T_total;  // the learning-rate horizon (tokens)
    float inv_T, pad1;
    unsigned long long S;
    uint32_t cmax, pad2;
    NoiseAgg total;
    unsigned long long loss_acc;
};

struct BArgs {
    const BJob *jobs;
    int32_t n_jobs;
    const int64_t *slot_prefix;  // [n_jobs + 1]
    const int64_t *node_prefix;  // [n_jobs + 1]
    const int64_t *item_prefix;  // [n_jobs + 1]
    const int32_t *tile_job, *tile_start;
    int32_t *tile_count;
    NoiseAgg *tile_agg;
    int32_t n_tiles;
    int64_t n_slots, n_nodes;
    int32_t L, wpr, window, K, max_rounds, ks, enabled, reactivate, precision;
    double mu;
    float lr0;
    int64_t lr_total_tokens;
    // ranges of the jobs of dim 32, 64, 128 (jobs are ordered by dim): training
    // items, minibatch tokens (walk slots times L) and nodes
    int64_t item_lo[3], item_hi[3], tok_lo[3], tok_hi[3], node_lo[3], node_hi[3];
};

// Grid-wide barrier of the persistent batched kernel (device memory, zero
// before a launch): arrivals, generation, an error word set when a bounded
// wait ran out, and the tag of the barrier where that happened (phase index
// + 16 * round for the persistent kernel).
struct GridBarrier {
    unsigned int count, gen;
    int error, where;
};

struct BParams {
    int32_t L, wpr, window, K, max_rounds, ks, enabled, reactivate, precision;
    int32_t mode;  // FELOG_SGNS_HOGWILD or FELOG_SGNS_MINIBATCH (one synchronous batch per round)
    double mu;
    float lr0;
    int64_t lr_total_tokens, rows_per_warp;
};

struct HostTuning {
    int walk_block = 256;
    int sgns_blocks_per_sm = 2;
    int feedback_blocks_per_sm = 16;
    int sgns_form = 2;  // 2: two pairs per warp (16 lanes per row); 1: one pair per warp (32 lanes);
                        // 4: shape 2 with rows prefetched to shared memory
};

// Trainer shape before any tuning: the train parameters' hogwild_form where
// the batched trainer has it (1, 2, 4), else for the automatic form 0 the
// single-graph rule (4 for bf16 tables, which falls back to 2 for dims it
// does not cover; 2 for float tables), else 2.
inline int default_sgns_form(const felog_train_params *tp) {
    const int f = tp->hogwild_form;
    if (f == 1 || f == 2 || f == 4) return f;
    if (f == 0 && tp->precision == FELOG_BF16_SR) return 4;
    return 2;
}

// a membership of jobs on the device: job table, index-space prefixes, tiles
struct BatchPlan {
    int32_t n_jobs = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    size_t o_gst = 0, o_gna = 0, o_gnn = 0, o_gl = 0;  // gather staging
    size_t o_bar = 0;                                   // grid barrier of the persistent kernel
    BArgs args{};
    std::vector<int64_t> item_prefix;  // host copies
    std::vector<int64_t> slot_prefix, node_prefix;
    std::vector<int32_t> dims;         // host, plan order
    std::vector<BJob> jobs;            // host copy of the job table
};

size_t job_work_bytes(int32_t n, int32_t dim, const BParams &p);
void job_carve(BJob &jb, void *mem, int32_t n, const BParams &p);  // jb.dim set first
felog_status job_clear_state(const BJob &jb, const BParams &p, cudaStream_t s);
felog_status plan_build(BatchPlan &plan, const std::vector<BJob> &jobs, const BParams &p, cudaStream_t s);
void plan_release(BatchPlan &plan, cudaStream_t s);
felog_status plan_init_jobs(const BatchPlan &plan, const BParams &p, cudaStream_t s);
felog_status plan_step(const BatchPlan &plan, const BParams &p, const HostTuning &t, cudaStream_t s,
                       unsigned phases);
felog_status plan_gather(const BatchPlan &plan, const BParams &p, cudaStream_t s, std::vector<BState> &sts,
                         std::vector<int32_t> &rna, std::vector<int32_t> &rnn, std::vector<double> &rl);
BParams make_params(const felog_walk_params *wp, const felog_train_params *tp, const felog_feedback_params *fp);
felog_status check_params(const felog_walk_params *wp, const felog_train_params *tp, const felog_feedback_params *fp);
felog_status check_job(int32_t n, int64_t nnz, int32_t dim);
int sm_count();

}  // namespace felog
