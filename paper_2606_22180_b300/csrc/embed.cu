// Algorithm 1 on one GPU: V_a <- non-isolated nodes; while V_a is not empty
// and fewer than max_rounds rounds have run: Sample (walks from V_a, corpus
// counts fused), noise table, Train, Feedback (Psi and V_a^{r+1}).
//
// Every phase is a kernel on the caller's stream; the host reads |V_a| once
// per round (4 bytes) to size the next round's launches and to stop.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace felog {

constexpr int kInitThreads = 256;

__global__ void k_active_init(const int32_t *__restrict__ offsets, int32_t n, uint8_t *__restrict__ active,
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

int sm_count();
bool csr_shape_ok(const felog_csr *g);
felog_status validate_csr_async(const felog_csr *g, const int32_t *starts, int32_t n_starts, int32_t *status,
                                cudaStream_t s);

struct EmbedWorkspace {
    uint8_t *active[2];
    int32_t *starts;
    int32_t *n_active;
    int32_t *n_next;
    int32_t *csr_status;
    unsigned long long *n_live;
    int32_t *walks;
    uint32_t *counts;
    uint64_t *thr;
    int32_t *alias;
    uint64_t *S;
    double *loss;
    void *compact_ws;
    size_t compact_bytes;
    void *noise_ws;
    size_t noise_bytes;
    void *train_ws;
    size_t train_bytes;
};

// lr_total_tokens <= 0 means "derive it"; size and validate with a placeholder
static felog_train_params sizing_params(const felog_train_params *tp) {
    felog_train_params t = *tp;
    if (t.lr_total_tokens <= 0) t.lr_total_tokens = 1;
    return t;
}

static EmbedWorkspace carve_embed(Carver &c, int32_t n, const felog_walk_params *wp,
                                  const felog_train_params *tp_in) {
    const felog_train_params tpv = sizing_params(tp_in);
    const felog_train_params *tp = &tpv;
    EmbedWorkspace w{};
    const size_t nn = n > 0 ? static_cast<size_t>(n) : 1;
    w.active[0] = c.take<uint8_t>(nn);
    w.active[1] = c.take<uint8_t>(nn);
    w.starts = c.take<int32_t>(nn);
    w.n_active = c.take<int32_t>(1);
    w.n_next = c.take<int32_t>(1);
    w.csr_status = c.take<int32_t>(1);
    w.n_live = c.take<unsigned long long>(1);
    w.walks = c.take<int32_t>(nn * wp->walks_per_round * wp->length);
    w.counts = c.take<uint32_t>(nn);
    w.thr = c.take<uint64_t>(nn);
    w.alias = c.take<int32_t>(nn);
    w.S = c.take<uint64_t>(1);
    w.loss = c.take<double>(1);
    w.compact_bytes = felog_compact_workspace_bytes(n);
    w.compact_ws = c.take<char>(w.compact_bytes);
    w.noise_bytes = felog_noise_workspace_bytes(n);
    w.noise_ws = c.take<char>(w.noise_bytes);
    w.train_bytes = felog_train_workspace_bytes(static_cast<int64_t>(nn) * wp->walks_per_round,
                                                wp->length, n, tp);
    w.train_ws = c.take<char>(w.train_bytes);
    return w;
}

struct EventSet {
    cudaEvent_t e[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ok = false;
    EventSet() {
        ok = true;
        for (auto &x : e) ok &= cudaEventCreate(&x) == cudaSuccess;
    }
    ~EventSet() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
    float ms(int a, int b) const {
        float t = 0.f;
        cudaEventElapsedTime(&t, e[a], e[b]);
        return t;
    }
};

}  // namespace felog

using namespace felog;

extern "C" size_t felog_embed_workspace_bytes(int32_t n, const felog_walk_params *wp,
                                              const felog_train_params *tp) {
    if (n < 0 || !wp || !tp || wp->length < 1 || wp->walks_per_round < 1) return 0;
    const felog_train_params tpv = sizing_params(tp);
    if (felog_train_workspace_bytes(1, wp->length, n, &tpv) == 0) return 0;
    Carver c(nullptr, 0);
    carve_embed(c, n, wp, tp);
    return align_up(c.used, 256);
}

extern "C" felog_status felog_embed(const felog_csr *g, const felog_walk_params *wp,
                                    const felog_train_params *tp_in, const felog_feedback_params *fp,
                                    uint64_t seed, void *phi_in, void *phi_out,
                                    felog_round_stats *stats, int32_t *rounds_run, void *workspace,
                                    size_t workspace_bytes, void *stream) {
    if (rounds_run) *rounds_run = 0;
    if (!csr_shape_ok(g)) return FELOG_ERR_BAD_CSR;
    if (!wp || !tp_in || !fp || wp->length < 1 || wp->walks_per_round < 1 || fp->max_rounds < 0 ||
        fp->max_rounds >= 65536)
        return FELOG_ERR_INVALID_ARG;
    if (g->n == 0) return FELOG_OK;
    if (!phi_in || !phi_out) return FELOG_ERR_INVALID_ARG;
    const size_t need = felog_embed_workspace_bytes(g->n, wp, tp_in);
    if (need == 0) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < need) return FELOG_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    EmbedWorkspace w = carve_embed(c, g->n, wp, tp_in);
    const int32_t n = g->n, L = wp->length, wpr = wp->walks_per_round;

    // the graph is checked on the device before any kernel gathers through it
    int32_t csr_status = 0;
    felog_status st = validate_csr_async(g, nullptr, 0, w.csr_status, s);
    if (!st) st = record_cuda_error(cudaMemcpyAsync(&csr_status, w.csr_status, sizeof csr_status,
                                                    cudaMemcpyDeviceToHost, s), "embed");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "embed");
    if (st) return st;
    if (csr_status) return FELOG_ERR_BAD_CSR;
    st = felog_init_tables(n, tp_in->dim, tp_in->precision, seed, phi_in, phi_out, stream);
    if (st) return st;
    st = record_cuda_error(cudaMemsetAsync(w.n_live, 0, sizeof(unsigned long long), s), "embed");
    if (st) return st;
    k_active_init<<<std::min(ceil_div(n, kInitThreads), sm_count() * 8), kInitThreads, 0, s>>>(
        g->offsets, n, w.active[0], w.n_live);
    if ((st = check_launch("felog_embed init"))) return st;
    unsigned long long n_live = 0;
    st = record_cuda_error(cudaMemcpyAsync(&n_live, w.n_live, sizeof n_live, cudaMemcpyDeviceToHost, s), "embed");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "embed");
    if (st) return st;
    felog_train_params tp = *tp_in;
    if (tp.lr_total_tokens <= 0)
        tp.lr_total_tokens = std::max<int64_t>(1, static_cast<int64_t>(fp->max_rounds) * wpr *
                                                       static_cast<int64_t>(n_live) * L);

    EventSet ev;
    if (!ev.ok) return record_cuda_error(cudaGetLastError(), "embed events");
    int64_t clock = 0;
    int cur = 0;
    int32_t r = 0;
    for (; r < fp->max_rounds; ++r) {
        int32_t n_active = 0;
        st = felog_compact_active(w.active[cur], n, w.starts, w.n_active, w.compact_ws, w.compact_bytes, stream);
        if (!st) st = record_cuda_error(cudaMemcpyAsync(&n_active, w.n_active, sizeof n_active,
                                                        cudaMemcpyDeviceToHost, s), "embed");
        if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "embed");
        if (st) return st;
        if (n_active == 0) break;
        const int64_t n_walks = static_cast<int64_t>(n_active) * wpr;
        cudaEventRecord(ev.e[0], s);
        st = record_cuda_error(cudaMemsetAsync(w.counts, 0, sizeof(uint32_t) * n, s), "embed");
        if (!st) st = felog_walk(g, w.starts, n_active, wp, seed, r, w.walks, w.counts, stream);
        cudaEventRecord(ev.e[1], s);
        if (!st) st = felog_noise_table(w.counts, n, w.thr, w.alias, w.S, w.noise_ws, w.noise_bytes, stream);
        cudaEventRecord(ev.e[2], s);
        if (!st) st = felog_train(w.walks, n_walks, L, n, &tp, w.thr, w.alias, w.S, seed, r, clock,
                                  phi_in, phi_out, w.loss, w.train_ws, w.train_bytes, stream);
        cudaEventRecord(ev.e[3], s);
        if (!st) st = felog_feedback(g, phi_in, tp.dim, tp.precision, fp, seed, r, w.active[cur],
                                     w.active[cur ^ 1], nullptr, w.n_next, stream);
        cudaEventRecord(ev.e[4], s);
        if (st) return st;
        clock += n_walks * L;
        if (stats) {
            felog_round_stats &rs = stats[r];
            double loss = 0.0;
            int32_t n_next = 0;
            st = record_cuda_error(cudaMemcpyAsync(&loss, w.loss, sizeof loss, cudaMemcpyDeviceToHost, s), "embed");
            if (!st) st = record_cuda_error(cudaMemcpyAsync(&n_next, w.n_next, sizeof n_next,
                                                            cudaMemcpyDeviceToHost, s), "embed");
            if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "embed");
            if (st) return st;
            rs.round = r;
            rs.n_active = n_active;
            rs.n_next = n_next;
            rs.reserved = 0;
            rs.tokens = n_walks * L;
            rs.walk_steps = n_walks * (L - 1);
            rs.loss = loss;
            rs.ms_walk = ev.ms(0, 1);
            rs.ms_noise = ev.ms(1, 2);
            rs.ms_train = ev.ms(2, 3);
            rs.ms_feedback = ev.ms(3, 4);
        }
        cur ^= 1;
    }
    if (rounds_run) *rounds_run = r;
    return record_cuda_error(cudaStreamSynchronize(s), "embed");
}
