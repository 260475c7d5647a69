// Host-only stand-ins for the CUDA runtime calls and the multi-graph plan
// functions used by the serving loop (server.cu).  Linked with
// -Wl,--wrap=<cuda call> so the server's calls land here: device memory is
// host memory, a step advances every unfinished job by one round, a job is
// done after max_rounds rounds.  Lets the server's queueing, admission and
// bookkeeping run under AddressSanitizer without a GPU.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>
#include <cuda_runtime.h>
#include "batch_core.cuh"

extern "C" {
cudaError_t __wrap_cudaMallocAsync(void **p, size_t n, cudaStream_t) { *p = malloc(n ? n : 1); return cudaSuccess; }
cudaError_t __wrap_cudaFreeAsync(void *p, cudaStream_t) { free(p); return cudaSuccess; }
cudaError_t __wrap_cudaMemcpyAsync(void *d, const void *s, size_t n, cudaMemcpyKind, cudaStream_t) { memcpy(d, s, n); return cudaSuccess; }
cudaError_t __wrap_cudaMemsetAsync(void *d, int v, size_t n, cudaStream_t) { memset(d, v, n); return cudaSuccess; }
cudaError_t __wrap_cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t __wrap_cudaStreamCreateWithFlags(cudaStream_t *s, unsigned) { *s = (cudaStream_t)0x1234; return cudaSuccess; }
cudaError_t __wrap_cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t __wrap_cudaGetDevice(int *d) { *d = 0; return cudaSuccess; }
cudaError_t __wrap_cudaSetDevice(int) { return cudaSuccess; }
}

namespace felog {
felog_status record_cuda_error(cudaError_t e, const char *) { return e == cudaSuccess ? FELOG_OK : FELOG_ERR_CUDA; }
felog_status check_launch(const char *) { return FELOG_OK; }
int sm_count() { return 148; }
size_t job_work_bytes(int32_t n, int32_t, const BParams &p) {
    size_t nn = n > 0 ? n : 1; size_t R = std::max(p.max_rounds, 1);
    return align_up(sizeof(BState), 256) + 2 * align_up(4 * R, 256) + align_up(8 * R, 256) + align_up(nn * 100, 256);
}
void job_carve(BJob &jb, void *mem, int32_t n, const BParams &p) {
    size_t R = std::max(p.max_rounds, 1);
    char *q = (char *)mem;
    jb.st = (BState *)q; q += align_up(sizeof(BState), 256);
    jb.rec_n_active = (int32_t *)q; q += align_up(4 * R, 256);
    jb.rec_n_next = (int32_t *)q; q += align_up(4 * R, 256);
    jb.rec_loss = (double *)q;
}
felog_status job_clear_state(const BJob &jb, const BParams &p, cudaStream_t) {
    size_t R = std::max(p.max_rounds, 1);
    memset(jb.st, 0, align_up(sizeof(BState), 256) + 2 * align_up(4 * R, 256) + 8 * R);
    return FELOG_OK;
}
felog_status plan_build(BatchPlan &plan, const std::vector<BJob> &jobs, const BParams &, cudaStream_t) {
    plan = BatchPlan{};
    plan.n_jobs = (int)jobs.size(); plan.jobs = jobs; plan.mem = malloc(16); plan.bytes = 16;
    for (auto &j : jobs) plan.dims.push_back(j.dim);
    return FELOG_OK;
}
void plan_release(BatchPlan &plan, cudaStream_t) { free(plan.mem); plan = BatchPlan{}; }
felog_status plan_init_jobs(const BatchPlan &plan, const BParams &p, cudaStream_t) {
    for (auto &j : plan.jobs) {
        if (j.st->phase) continue;
        j.st->n_live = j.n; j.st->done = j.n == 0 || p.max_rounds == 0; j.st->phase = 1;
        float *phi = (float *)j.phi_in;
        for (int64_t i = 0; i < (int64_t)j.n * j.dim; ++i) phi[i] = 0.5f;
    }
    return FELOG_OK;
}
felog_status plan_step(const BatchPlan &plan, const BParams &p, const HostTuning &, cudaStream_t, unsigned) {
    for (auto &j : plan.jobs) {
        BState &s = *j.st;
        if (s.done) continue;
        s.n_active = j.n;
        j.rec_n_active[s.round] = j.n; j.rec_loss[s.round] = 1.0;
        s.clock += (int64_t)j.n * p.L; s.round++;
        if (s.round >= p.max_rounds) s.done = 1;
    }
    return FELOG_OK;
}
felog_status plan_gather(const BatchPlan &plan, const BParams &p, cudaStream_t, std::vector<BState> &sts,
                         std::vector<int32_t> &rna, std::vector<int32_t> &rnn, std::vector<double> &rl) {
    int n = plan.n_jobs; size_t R = std::max(p.max_rounds, 1);
    sts.resize(n); rna.assign(R * n, 0); rnn.assign(R * n, 0); rl.assign(R * n, 0.0);
    for (int i = 0; i < n; ++i) {
        sts[i] = *plan.jobs[i].st;
        for (int r = 0; r < p.max_rounds; ++r) rl[r * n + i] = plan.jobs[i].rec_loss[r];
    }
    return FELOG_OK;
}
BParams make_params(const felog_walk_params *wp, const felog_train_params *tp, const felog_feedback_params *fp) {
    BParams p{}; p.L = wp->length; p.wpr = wp->walks_per_round; p.window = tp->window; p.K = tp->negatives;
    p.max_rounds = fp->max_rounds; p.precision = tp->precision; p.rows_per_warp = 16; return p;
}
felog_status check_params(const felog_walk_params *, const felog_train_params *, const felog_feedback_params *) { return FELOG_OK; }
felog_status check_job(int32_t n, int64_t nnz, int32_t dim) {  // same rules as the library
    if (n < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return FELOG_ERR_BAD_CSR;
    if (dim != 32 && dim != 64 && dim != 128) return FELOG_ERR_UNSUPPORTED;
    return FELOG_OK;
}
}
