// Round-interleaved pipeline (Section 5.3, RiPP) of Algorithm 1 on one GPU.
//
// The paper splits a round into operator groups that run as separate
// pipelines: sampling (R), corpus management, and training (T).  The
// sampling frontier of round r + 1 depends on the feedback after round r;
// Section 5.3 lets that feedback read the locally visible, possibly stale,
// embedding snapshot so that R_{r+1} need not wait.  On one GPU the two
// groups are two streams:
//
//   train stream   (the caller's): [snapshot of phi_in] T_r
//   sample stream  (the library's): Psi_r, V_a^{r+1}, compaction,
//                                   R_{r+1} (walk, counts), noise table r+1
//
// feedback_lag = 1: Psi_r reads the snapshot of phi_in taken as T_r starts
// (the table after round r - 1), so the sample stream's work of round r + 1
// runs while T_r trains.  feedback_lag = 0: Psi_r waits for T_r (Algorithm 1
// as printed) and the streams alternate.  Round buffers (walks, counts,
// alias table) are double-buffered: round r + 1's are written while T_r
// reads round r's.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace felog {

int sm_count();
bool csr_shape_ok(const felog_csr *g);
felog_status validate_csr_async(const felog_csr *g, const int32_t *starts, int32_t n_starts, int32_t *status,
                                cudaStream_t s);

__global__ void k_pipe_active_init(const int32_t *__restrict__ offsets, int32_t n, uint8_t *__restrict__ active,
                                   unsigned long long *__restrict__ n_live) {
    unsigned long long c = 0;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint8_t a = offsets[v + 1] > offsets[v];
        active[v] = a;
        c += a;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_live, c);
}

struct PipeWorkspace {
    uint8_t *active[2];
    int32_t *starts, *n_active, *n_next, *csr_status;
    unsigned long long *n_live;
    int32_t *walks[2];
    uint32_t *counts[2];
    uint64_t *thr[2];
    int32_t *alias[2];
    uint64_t *S[2];
    double *loss;  // [max_rounds]
    void *snap;    // phi_in snapshot (feedback_lag = 1)
    void *compact_ws, *noise_ws, *train_ws;
    size_t compact_bytes, noise_bytes, train_bytes;
};

static felog_train_params sizing(const felog_train_params *tp) {
    felog_train_params t = *tp;
    if (t.lr_total_tokens <= 0) t.lr_total_tokens = 1;
    return t;
}

static PipeWorkspace carve_pipe(Carver &c, int32_t n, const felog_walk_params *wp, const felog_train_params *tp_in,
                                int32_t max_rounds, int32_t lag) {
    const felog_train_params tpv = sizing(tp_in);
    PipeWorkspace w{};
    const size_t nn = n > 0 ? static_cast<size_t>(n) : 1;
    for (int b = 0; b < 2; ++b) w.active[b] = c.take<uint8_t>(nn);
    w.starts = c.take<int32_t>(nn);
    w.n_active = c.take<int32_t>(1);
    w.n_next = c.take<int32_t>(1);
    w.csr_status = c.take<int32_t>(1);
    w.n_live = c.take<unsigned long long>(1);
    for (int b = 0; b < 2; ++b) {
        w.walks[b] = c.take<int32_t>(nn * wp->walks_per_round * wp->length);
        w.counts[b] = c.take<uint32_t>(nn);
        w.thr[b] = c.take<uint64_t>(nn);
        w.alias[b] = c.take<int32_t>(nn);
        w.S[b] = c.take<uint64_t>(1);
    }
    w.loss = c.take<double>(std::max<int32_t>(max_rounds, 1));
    const size_t elem = tpv.precision == FELOG_FP32 ? 4 : 2;
    w.snap = lag ? c.take<char>(nn * tpv.dim * elem) : nullptr;
    w.compact_bytes = felog_compact_workspace_bytes(n);
    w.compact_ws = c.take<char>(w.compact_bytes);
    w.noise_bytes = felog_noise_workspace_bytes(n);
    w.noise_ws = c.take<char>(w.noise_bytes);
    w.train_bytes = felog_train_workspace_bytes(static_cast<int64_t>(nn) * wp->walks_per_round, wp->length, n, &tpv);
    w.train_ws = c.take<char>(w.train_bytes);
    return w;
}

// Events of the run: a base event, then per round the train stream's start
// and end and the sample stream's start and end of the work it does after T_r
// starts (Psi_r .. noise table r + 1).
struct PipeEvents {
    std::vector<cudaEvent_t> ev;
    bool ok = true;
    explicit PipeEvents(size_t count) : ev(count, nullptr) {
        for (auto &e : ev) ok &= cudaEventCreate(&e) == cudaSuccess;
    }
    ~PipeEvents() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    float since(int base, int i) const {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[base], ev[i]);
        return t;
    }
};

struct StreamGuard {
    cudaStream_t s = nullptr;
    ~StreamGuard() {
        if (s) cudaStreamDestroy(s);
    }
};

}  // namespace felog

using namespace felog;

extern "C" size_t felog_pipeline_workspace_bytes(int32_t n, const felog_walk_params *wp,
                                                 const felog_train_params *tp, int32_t max_rounds,
                                                 int32_t feedback_lag) {
    if (n < 0 || !wp || !tp || wp->length < 1 || wp->walks_per_round < 1 || max_rounds < 0) return 0;
    if (feedback_lag != 0 && feedback_lag != 1) return 0;
    const felog_train_params tpv = sizing(tp);
    if (felog_train_workspace_bytes(1, wp->length, n, &tpv) == 0) return 0;
    Carver c(nullptr, 0);
    carve_pipe(c, n, wp, tp, max_rounds, feedback_lag);
    return align_up(c.used, 256);
}

extern "C" felog_status felog_embed_pipelined(const felog_csr *g, const felog_walk_params *wp,
                                              const felog_train_params *tp_in, const felog_feedback_params *fp,
                                              int32_t feedback_lag, uint64_t seed, void *phi_in, void *phi_out,
                                              felog_round_stats *stats, felog_pipeline_stats *pstats,
                                              int32_t *rounds_run, void *workspace, size_t workspace_bytes,
                                              void *stream) {
    if (rounds_run) *rounds_run = 0;
    if (pstats) *pstats = felog_pipeline_stats{};
    if (!csr_shape_ok(g)) return FELOG_ERR_BAD_CSR;
    if (!wp || !tp_in || !fp || wp->length < 1 || wp->walks_per_round < 1 || fp->max_rounds < 0 ||
        fp->max_rounds >= 65536 || (feedback_lag != 0 && feedback_lag != 1))
        return FELOG_ERR_INVALID_ARG;
    if (g->n == 0 || fp->max_rounds == 0) return FELOG_OK;
    if (!phi_in || !phi_out) return FELOG_ERR_INVALID_ARG;
    const size_t need = felog_pipeline_workspace_bytes(g->n, wp, tp_in, fp->max_rounds, feedback_lag);
    if (need == 0) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < need) return FELOG_ERR_WORKSPACE;
    cudaStream_t sa = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    PipeWorkspace w = carve_pipe(c, g->n, wp, tp_in, fp->max_rounds, feedback_lag);
    const int32_t n = g->n, L = wp->length, wpr = wp->walks_per_round, R = fp->max_rounds;

    // the graph is checked on the device before any kernel gathers through it
    int32_t csr_status = 0;
    felog_status st = validate_csr_async(g, nullptr, 0, w.csr_status, sa);
    if (!st) st = record_cuda_error(cudaMemcpyAsync(&csr_status, w.csr_status, sizeof csr_status,
                                                    cudaMemcpyDeviceToHost, sa), "pipelined");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(sa), "pipelined");
    if (st) return st;
    if (csr_status) return FELOG_ERR_BAD_CSR;

    StreamGuard sb;
    st = record_cuda_error(cudaStreamCreateWithFlags(&sb.s, cudaStreamNonBlocking), "pipelined stream");
    if (st) return st;
    // events: 0 base, 1 end; per round r: 2 + 6r: train start, train end, snapshot taken,
    // sample start, sample end, sample ready (for the train stream to wait on)
    PipeEvents E(2 + 6 * static_cast<size_t>(R));
    if (!E.ok) return record_cuda_error(cudaGetLastError(), "pipelined events");
    auto ev = [&](int r, int k) { return E.ev[2 + 6 * r + k]; };

    st = felog_init_tables(n, tp_in->dim, tp_in->precision, seed, phi_in, phi_out, stream);
    if (!st) st = record_cuda_error(cudaMemsetAsync(w.n_live, 0, sizeof(unsigned long long), sa), "pipelined");
    if (st) return st;
    k_pipe_active_init<<<std::min(ceil_div(n, 256), sm_count() * 8), 256, 0, sa>>>(g->offsets, n, w.active[0],
                                                                                    w.n_live);
    if ((st = check_launch("pipelined init"))) return st;
    // round 0's sample on the train stream (nothing to overlap yet)
    int32_t n_act = 0;
    unsigned long long n_live = 0;
    st = felog_compact_active(w.active[0], n, w.starts, w.n_active, w.compact_ws, w.compact_bytes, stream);
    if (!st) st = record_cuda_error(cudaMemcpyAsync(&n_live, w.n_live, sizeof n_live, cudaMemcpyDeviceToHost, sa),
                                    "pipelined");
    if (!st) st = record_cuda_error(cudaMemcpyAsync(&n_act, w.n_active, sizeof n_act, cudaMemcpyDeviceToHost, sa),
                                    "pipelined");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(sa), "pipelined");
    if (st) return st;
    if (n_act == 0) return FELOG_OK;
    felog_train_params tp = *tp_in;
    if (tp.lr_total_tokens <= 0)
        tp.lr_total_tokens = std::max<int64_t>(1, static_cast<int64_t>(R) * wpr * static_cast<int64_t>(n_live) * L);
    cudaEventRecord(E.ev[0], sa);
    st = record_cuda_error(cudaMemsetAsync(w.counts[0], 0, sizeof(uint32_t) * n, sa), "pipelined");
    if (!st) st = felog_walk(g, w.starts, n_act, wp, seed, 0, w.walks[0], w.counts[0], stream);
    if (!st) st = felog_noise_table(w.counts[0], n, w.thr[0], w.alias[0], w.S[0], w.noise_ws, w.noise_bytes, stream);
    if (st) return st;

    std::vector<int32_t> n_active_of(R, 0), n_next_of(R, 0);
    const size_t snap_bytes = static_cast<size_t>(n) * tp.dim * (tp.precision == FELOG_FP32 ? 4 : 2);
    int64_t clock = 0;
    int32_t r = 0;
    for (; r < R; ++r) {
        const int b = r & 1;
        n_active_of[r] = n_act;
        const int64_t n_walks = static_cast<int64_t>(n_act) * wpr;
        // ---- train stream: [snapshot] T_r -------------------------------------
        if (feedback_lag) {
            st = record_cuda_error(cudaMemcpyAsync(w.snap, phi_in, snap_bytes, cudaMemcpyDeviceToDevice, sa),
                                   "pipelined snapshot");
            if (st) return st;
        }
        cudaEventRecord(ev(r, 2), sa);  // phi_in as T_r starts (the snapshot is taken)
        cudaEventRecord(ev(r, 0), sa);
        st = felog_train(w.walks[b], n_walks, L, n, &tp, w.thr[b], w.alias[b], w.S[b], seed, r, clock, phi_in,
                         phi_out, w.loss + r, w.train_ws, w.train_bytes, stream);
        if (st) return st;
        cudaEventRecord(ev(r, 1), sa);
        clock += n_walks * L;
        // ---- sample stream: Psi_r, V_a^{r+1}, compaction -------------------------
        // lag 1: after the snapshot; lag 0: after T_r.  Either way T_{r-1} is
        // done, so round r + 1's buffers (round r - 1's) are free.
        cudaStreamWaitEvent(sb.s, feedback_lag ? ev(r, 2) : ev(r, 1), 0);
        cudaEventRecord(ev(r, 3), sb.s);
        st = felog_feedback(g, feedback_lag ? w.snap : phi_in, tp.dim, tp.precision, fp, seed, r, w.active[b],
                            w.active[b ^ 1], nullptr, w.n_next, sb.s);
        if (!st) st = felog_compact_active(w.active[b ^ 1], n, w.starts, w.n_active, w.compact_ws,
                                           w.compact_bytes, sb.s);
        int32_t n_new = 0;
        if (!st) st = record_cuda_error(cudaMemcpyAsync(&n_new, w.n_active, sizeof n_new, cudaMemcpyDeviceToHost,
                                                        sb.s), "pipelined");
        if (!st) st = record_cuda_error(cudaStreamSynchronize(sb.s), "pipelined");  // T_r still runs on sa
        if (st) return st;
        n_next_of[r] = n_new;
        if (n_new == 0 || r + 1 == R) {
            cudaEventRecord(ev(r, 4), sb.s);
            cudaEventRecord(ev(r, 5), sb.s);
            ++r;
            break;
        }
        // ---- sample stream: R_{r+1} and its noise table ---------------------------
        st = record_cuda_error(cudaMemsetAsync(w.counts[b ^ 1], 0, sizeof(uint32_t) * n, sb.s), "pipelined");
        if (!st) st = felog_walk(g, w.starts, n_new, wp, seed, r + 1, w.walks[b ^ 1], w.counts[b ^ 1], sb.s);
        if (!st) st = felog_noise_table(w.counts[b ^ 1], n, w.thr[b ^ 1], w.alias[b ^ 1], w.S[b ^ 1], w.noise_ws,
                                        w.noise_bytes, sb.s);
        if (st) return st;
        cudaEventRecord(ev(r, 4), sb.s);
        cudaEventRecord(ev(r, 5), sb.s);
        cudaStreamWaitEvent(sa, ev(r, 5), 0);  // T_{r+1} (and its snapshot) after the sample
        n_act = n_new;
    }
    cudaStreamWaitEvent(sa, E.ev[2 + 6 * (r - 1) + 5], 0);
    cudaEventRecord(E.ev[1], sa);
    std::vector<double> loss(r);
    st = record_cuda_error(cudaMemcpyAsync(loss.data(), w.loss, sizeof(double) * r, cudaMemcpyDeviceToHost, sa),
                           "pipelined");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(sa), "pipelined");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(sb.s), "pipelined");
    if (st) return st;
    double train_busy = 0, sample_busy = 0, overlap = 0;
    for (int32_t k = 0; k < r; ++k) {
        const double a0 = E.since(0, 2 + 6 * k + 0), a1 = E.since(0, 2 + 6 * k + 1);
        const double b0 = E.since(0, 2 + 6 * k + 3), b1 = E.since(0, 2 + 6 * k + 4);
        train_busy += a1 - a0;
        sample_busy += b1 - b0;
        overlap += std::max(0.0, std::min(a1, b1) - std::max(a0, b0));
        if (stats) {
            felog_round_stats &rs = stats[k];
            rs.round = k;
            rs.n_active = n_active_of[k];
            rs.n_next = n_next_of[k];
            rs.reserved = 0;
            rs.tokens = static_cast<int64_t>(n_active_of[k]) * wpr * L;
            rs.walk_steps = static_cast<int64_t>(n_active_of[k]) * wpr * (L - 1);
            rs.loss = loss[k];
            rs.ms_walk = 0.f;  // the sample stream's time of round k + 1 is in ms_feedback
            rs.ms_noise = 0.f;
            rs.ms_train = static_cast<float>(a1 - a0);
            rs.ms_feedback = static_cast<float>(b1 - b0);
        }
    }
    if (pstats) {
        pstats->wall_ms = E.since(0, 1);
        pstats->train_busy_ms = train_busy;
        pstats->sample_busy_ms = sample_busy;
        pstats->overlap_ms = overlap;
        pstats->rounds = r;
        pstats->feedback_lag = feedback_lag;
    }
    if (rounds_run) *rounds_run = r;
    return FELOG_OK;
}
