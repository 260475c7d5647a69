// Serving form: a request loop over embedding jobs with continuous batching.
//
// Clients submit jobs (a host CSR, dim, seed) at any time.  A worker thread
// owns the GPU work:
//   1. admission, first come first served: the queue head is admitted when
//      its device bytes (CSR, tables, work buffers) fit in the HBM budget
//      beside the resident jobs; a job larger than the whole budget is
//      rejected.  Memory is taken stream-ordered (cudaMallocAsync).
//   2. every iteration runs one round of Algorithm 1 for all resident jobs
//      together (the multi-graph step of batch.cu), each at its own round;
//      newly admitted jobs are initialised and join the next step.
//   3. jobs whose active set emptied or that reached max_rounds are
//      finished: their embedding is copied to host memory, their device
//      memory released, and the next queued jobs can be admitted.
// Latency of a request = completion time - submission time on the server's
// steady clock.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_core.cuh"

namespace felog {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    std::vector<int32_t> offsets, cols;
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t dim = 0;
    uint64_t seed = 0;
    size_t bytes = 0;  // device bytes while resident
};

struct Resident {
    std::unique_ptr<Request> req;
    void *mem = nullptr;
    BJob jb{};
};

struct Result {
    felog_result info{};
    std::vector<float> phi;  // [n][dim] once done
};

size_t table_bytes(int32_t n, int32_t dim, int32_t precision) {
    return static_cast<size_t>(n > 0 ? n : 1) * dim * (precision == FELOG_FP32 ? 4 : 2);
}

}  // namespace
}  // namespace felog

using namespace felog;

struct felog_server {
    felog_server_config cfg{};
    BParams p{};
    HostTuning tune;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable wake;     // submit / stop -> worker
    std::condition_variable changed;  // worker -> waiters
    bool stop = false;
    std::deque<std::unique_ptr<Request>> queue;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_id = 1;
    size_t resident_bytes = 0;        // guarded by mu
    int32_t resident_jobs = 0;        // guarded by mu
    Clock::time_point t0;
    felog_server_stats stats{};
    felog_status error = FELOG_OK;    // sticky failure of the worker
    // worker-private
    std::vector<Resident> resident;
    BatchPlan plan;
    std::vector<int32_t> plan_to_resident;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

felog_status upload_job(felog_server *sv, Resident &r) {
    Request &q = *r.req;
    cudaStream_t s = sv->stream;
    char *base = static_cast<char *>(r.mem);
    size_t off = 0;
    auto take = [&](size_t bytes) { char *x = base + off; off += align_up(bytes, 256); return x; };
    int32_t *offsets = reinterpret_cast<int32_t *>(take(4 * (static_cast<size_t>(q.n) + 1)));
    int32_t *cols = reinterpret_cast<int32_t *>(take(4 * std::max<size_t>(q.nnz, 1)));
    void *phi_in = take(table_bytes(q.n, q.dim, sv->p.precision));
    void *phi_out = take(table_bytes(q.n, q.dim, sv->p.precision));
    void *work = take(job_work_bytes(q.n, q.dim, sv->p));
    felog_status st = record_cuda_error(
        cudaMemcpyAsync(offsets, q.offsets.data(), 4 * (static_cast<size_t>(q.n) + 1), cudaMemcpyHostToDevice, s), "upload");
    if (!st && q.nnz)
        st = record_cuda_error(cudaMemcpyAsync(cols, q.cols.data(), 4 * static_cast<size_t>(q.nnz), cudaMemcpyHostToDevice, s),
                               "upload");
    if (st) return st;
    BJob &jb = r.jb;
    jb = BJob{};
    jb.offsets = offsets;
    jb.cols = cols;
    jb.nnz = q.nnz;
    jb.n = q.n;
    jb.dim = q.dim;
    jb.seed = q.seed;
    jb.phi_in = phi_in;
    jb.phi_out = phi_out;
    job_carve(jb, work, q.n, sv->p);
    return job_clear_state(jb, sv->p, s);
}

size_t job_device_bytes(const BParams &p, int32_t n, int64_t nnz, int32_t dim) {
    return align_up(4 * (static_cast<size_t>(n) + 1), 256) + align_up(4 * std::max<size_t>(nnz, 1), 256) +
           2 * align_up(table_bytes(n, dim, p.precision), 256) + job_work_bytes(n, dim, p);
}

felog_status rebuild_plan(felog_server *sv) {
    plan_release(sv->plan, sv->stream);
    std::vector<int32_t> idx(sv->resident.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = static_cast<int32_t>(i);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int32_t a, int32_t b) { return sv->resident[a].jb.dim < sv->resident[b].jb.dim; });
    std::vector<BJob> jobs;
    jobs.reserve(idx.size());
    for (int32_t i : idx) jobs.push_back(sv->resident[i].jb);
    sv->plan_to_resident = idx;
    return plan_build(sv->plan, jobs, sv->p, sv->stream);
}

felog_status finish_job(felog_server *sv, Resident &r, const BState &st, const std::vector<double> &rl,
                        int32_t plan_i) {
    const Request &q = *r.req;
    std::vector<float> phi(static_cast<size_t>(q.n) * q.dim);
    felog_status s;
    if (sv->p.precision == FELOG_FP32) {
        s = record_cuda_error(cudaMemcpyAsync(phi.data(), r.jb.phi_in, 4 * phi.size(), cudaMemcpyDeviceToHost, sv->stream),
                              "fetch");
        if (!s) s = record_cuda_error(cudaStreamSynchronize(sv->stream), "fetch");
    } else {
        std::vector<uint16_t> h(phi.size());
        s = record_cuda_error(cudaMemcpyAsync(h.data(), r.jb.phi_in, 2 * h.size(), cudaMemcpyDeviceToHost, sv->stream),
                              "fetch");
        if (!s) s = record_cuda_error(cudaStreamSynchronize(sv->stream), "fetch");
        for (size_t i = 0; i < h.size(); ++i) {
            const uint32_t b = static_cast<uint32_t>(h[i]) << 16;
            std::memcpy(&phi[i], &b, 4);
        }
    }
    if (s) return s;
    const double t = sv->now();
    std::lock_guard<std::mutex> lk(sv->mu);
    Result &res = sv->results[q.id];
    res.info.state = FELOG_JOB_DONE;
    res.info.rounds = st.round;
    res.info.tokens = st.clock;
    res.info.n_live = st.n_live;
    res.info.t_done = t;
    res.info.loss_last = st.round > 0 ? rl[static_cast<size_t>(st.round - 1) * sv->plan.n_jobs + plan_i] : 0.0;
    res.phi = std::move(phi);
    sv->stats.completed += 1;
    return FELOG_OK;
}

void fail_all(felog_server *sv, felog_status st) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->error = st;
    for (auto &kv : sv->results)
        if (kv.second.info.state == FELOG_JOB_QUEUED || kv.second.info.state == FELOG_JOB_RUNNING)
            kv.second.info.state = FELOG_JOB_FAILED;
    sv->queue.clear();
    sv->changed.notify_all();
}

void worker_main(felog_server *sv) {
    cudaSetDevice(sv->device);
    bool membership_changed = false;
    for (;;) {
        std::vector<std::unique_ptr<Request>> admit;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            while (sv->resident.empty() && sv->queue.empty() && !sv->stop) sv->wake.wait(lk);
            if (sv->stop && sv->resident.empty() && sv->queue.empty()) break;
            if (sv->stop && sv->cfg.drain_on_destroy == 0) break;
            while (!sv->queue.empty()) {
                Request &q = *sv->queue.front();
                if (q.bytes > sv->cfg.hbm_budget) {
                    sv->results[q.id].info.state = FELOG_JOB_REJECTED;
                    sv->stats.rejected += 1;
                    sv->queue.pop_front();
                    sv->changed.notify_all();
                    continue;
                }
                const bool slot_ok = sv->cfg.max_resident <= 0 ||
                                     sv->resident_jobs + static_cast<int32_t>(admit.size()) < sv->cfg.max_resident;
                if (!slot_ok || sv->resident_bytes + q.bytes > sv->cfg.hbm_budget) break;
                sv->resident_bytes += q.bytes;
                admit.push_back(std::move(sv->queue.front()));
                sv->queue.pop_front();
            }
        }
        // admission: memory, upload, initialisation of the new jobs
        std::vector<BJob> fresh;
        for (auto &q : admit) {
            Resident r;
            r.req = std::move(q);
            felog_status st = record_cuda_error(cudaMallocAsync(&r.mem, r.req->bytes, sv->stream), "admit");
            if (!st) st = upload_job(sv, r);
            if (st) {
                fail_all(sv, st);
                return;
            }
            fresh.push_back(r.jb);
            const double t = sv->now();
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                Result &res = sv->results[r.req->id];
                res.info.state = FELOG_JOB_RUNNING;
                res.info.t_admit = t;
                sv->stats.admitted += 1;
                sv->resident_jobs += 1;
                sv->stats.peak_resident_jobs = std::max(sv->stats.peak_resident_jobs, sv->resident_jobs);
                sv->stats.peak_resident_bytes = std::max(sv->stats.peak_resident_bytes, sv->resident_bytes);
            }
            sv->resident.push_back(std::move(r));
            membership_changed = true;
        }
        if (!fresh.empty()) {
            std::stable_sort(fresh.begin(), fresh.end(), [](const BJob &a, const BJob &b) { return a.dim < b.dim; });
            BatchPlan ip;
            felog_status st = plan_build(ip, fresh, sv->p, sv->stream);
            if (!st) st = plan_init_jobs(ip, sv->p, sv->stream);
            plan_release(ip, sv->stream);
            if (st) {
                fail_all(sv, st);
                return;
            }
        }
        if (sv->resident.empty()) continue;
        if (membership_changed) {
            felog_status st = rebuild_plan(sv);
            if (st) {
                fail_all(sv, st);
                return;
            }
            membership_changed = false;
        }
        const auto t_step = Clock::now();
        felog_status st = plan_step(sv->plan, sv->p, sv->tune, sv->stream, 0x3f);
        std::vector<BState> sts;
        std::vector<int32_t> rna, rnn;
        std::vector<double> rl;
        if (!st) st = plan_gather(sv->plan, sv->p, sv->stream, sts, rna, rnn, rl);
        if (st) {
            fail_all(sv, st);
            return;
        }
        sv->stats.steps += 1;
        sv->stats.busy_seconds += std::chrono::duration<double>(Clock::now() - t_step).count();
        // finish jobs that are done
        std::vector<char> gone(sv->resident.size(), 0);
        for (int32_t i = 0; i < sv->plan.n_jobs; ++i) {
            if (!sts[i].done) continue;
            Resident &r = sv->resident[sv->plan_to_resident[i]];
            st = finish_job(sv, r, sts[i], rl, i);
            if (st) {
                fail_all(sv, st);
                return;
            }
            cudaFreeAsync(r.mem, sv->stream);
            r.mem = nullptr;
            gone[sv->plan_to_resident[i]] = 1;
        }
        size_t freed = 0;
        int32_t n_gone = 0;
        for (size_t i = 0; i < sv->resident.size(); ++i) {
            if (gone[i]) {
                freed += sv->resident[i].req->bytes;
                ++n_gone;
            }
        }
        if (n_gone) {
            std::vector<Resident> keep;
            for (size_t i = 0; i < sv->resident.size(); ++i)
                if (!gone[i]) keep.push_back(std::move(sv->resident[i]));
            sv->resident = std::move(keep);
            membership_changed = true;
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->resident_bytes -= freed;
            sv->resident_jobs -= n_gone;
            sv->changed.notify_all();
        }
    }
    // shutting down: release what is still resident
    for (Resident &r : sv->resident)
        if (r.mem) cudaFreeAsync(r.mem, sv->stream);
    sv->resident.clear();
    plan_release(sv->plan, sv->stream);
    cudaStreamSynchronize(sv->stream);
}

bool csr_host_ok(const int32_t *offsets, const int32_t *cols, int32_t n, int64_t nnz) {
    if (n < 0 || nnz < 0 || !offsets || (nnz > 0 && !cols)) return false;
    if (offsets[0] != 0 || offsets[n] != nnz) return false;
    for (int32_t v = 0; v < n; ++v)
        if (offsets[v + 1] < offsets[v]) return false;
    for (int64_t e = 0; e < nnz; ++e)
        if (cols[e] < 0 || cols[e] >= n) return false;
    return true;
}

}  // namespace

extern "C" felog_status felog_server_create(const felog_server_config *cfg, felog_server **out) {
    if (!cfg || !out) return FELOG_ERR_INVALID_ARG;
    *out = nullptr;
    felog_status st = check_params(&cfg->walk, &cfg->train, &cfg->feedback);
    if (st) return st;
    felog_server *sv = new (std::nothrow) felog_server();
    if (!sv) return FELOG_ERR_INVALID_ARG;
    sv->cfg = *cfg;
    sv->p = make_params(&cfg->walk, &cfg->train, &cfg->feedback);
    sv->tune.sgns_form = default_sgns_form(&cfg->train);
    sv->t0 = Clock::now();
    st = record_cuda_error(cudaGetDevice(&sv->device), "felog_server_create");
    if (!st) st = record_cuda_error(cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking), "felog_server_create");
    if (st) {
        delete sv;
        return st;
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return FELOG_OK;
}

extern "C" double felog_server_now(const felog_server *sv) { return sv ? sv->now() : 0.0; }

extern "C" size_t felog_server_job_bytes(const felog_server *sv, int32_t n, int64_t nnz, int32_t dim) {
    if (!sv || check_job(n, nnz, dim)) return 0;
    return job_device_bytes(sv->p, n, nnz, dim);
}

extern "C" felog_status felog_server_submit(felog_server *sv, const int32_t *offsets, const int32_t *cols, int32_t n,
                                            int64_t nnz, int32_t dim, uint64_t seed, uint64_t *id) {
    if (!sv || !id) return FELOG_ERR_INVALID_ARG;
    felog_status st = check_job(n, nnz, dim);
    if (st) return st;
    if (!csr_host_ok(offsets, cols, n, nnz)) return FELOG_ERR_BAD_CSR;
    std::unique_ptr<Request> q(new (std::nothrow) Request());
    if (!q) return FELOG_ERR_INVALID_ARG;
    q->offsets.assign(offsets, offsets + n + 1);
    q->cols.assign(cols, cols + nnz);
    q->n = n;
    q->nnz = nnz;
    q->dim = dim;
    q->seed = seed;
    q->bytes = job_device_bytes(sv->p, n, nnz, dim);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->error) return sv->error;
    if (sv->stop) return FELOG_ERR_INVALID_ARG;
    q->id = sv->next_id++;
    Result &res = sv->results[q->id];
    res.info.state = FELOG_JOB_QUEUED;
    res.info.t_submit = sv->now();
    res.info.n = n;
    res.info.dim = dim;
    *id = q->id;
    sv->stats.submitted += 1;
    sv->queue.push_back(std::move(q));
    sv->wake.notify_one();
    return FELOG_OK;
}

extern "C" felog_status felog_server_poll(felog_server *sv, uint64_t id, felog_result *out) {
    if (!sv || !out) return FELOG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->results.find(id);
    if (it == sv->results.end()) return FELOG_ERR_INVALID_ARG;
    *out = it->second.info;
    return sv->error;
}

extern "C" felog_status felog_server_wait(felog_server *sv, uint64_t id, double timeout_s, felog_result *out) {
    if (!sv) return FELOG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    for (;;) {
        auto it = sv->results.find(id);
        if (it == sv->results.end()) return FELOG_ERR_INVALID_ARG;
        const int32_t s = it->second.info.state;
        if (s == FELOG_JOB_DONE || s == FELOG_JOB_REJECTED || s == FELOG_JOB_FAILED || sv->error) {
            if (out) *out = it->second.info;
            return sv->error;
        }
        if (sv->changed.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (out) *out = it->second.info;
            return FELOG_ERR_TIMEOUT;
        }
    }
}

extern "C" felog_status felog_server_fetch(felog_server *sv, uint64_t id, float *phi_in_host) {
    if (!sv) return FELOG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->results.find(id);
    if (it == sv->results.end() || it->second.info.state != FELOG_JOB_DONE) return FELOG_ERR_INVALID_ARG;
    if (phi_in_host && !it->second.phi.empty())
        std::memcpy(phi_in_host, it->second.phi.data(), sizeof(float) * it->second.phi.size());
    sv->results.erase(it);
    return FELOG_OK;
}

extern "C" felog_status felog_server_drain(felog_server *sv, double timeout_s) {
    if (!sv) return FELOG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!(sv->queue.empty() && sv->resident_jobs == 0) && !sv->error) {
        if (sv->changed.wait_until(lk, deadline) == std::cv_status::timeout) return FELOG_ERR_TIMEOUT;
    }
    return sv->error;
}

extern "C" felog_status felog_server_get_stats(felog_server *sv, felog_server_stats *out) {
    if (!sv || !out) return FELOG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->resident_jobs = sv->resident_jobs;
    out->resident_bytes = sv->resident_bytes;
    out->queued = static_cast<int32_t>(sv->queue.size());
    return sv->error;
}

extern "C" felog_status felog_server_destroy(felog_server *sv) {
    if (!sv) return FELOG_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->wake.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    felog_status st = sv->error;
    if (sv->stream) cudaStreamDestroy(sv->stream);
    delete sv;
    return st;
}
