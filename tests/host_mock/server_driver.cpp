// Scenarios for the serving loop on the mocked runtime (see runtime_mock.cpp).
// Usage: server_driver <scenario>; prints "ok" on success.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "felog.h"

static felog_server_config config(size_t budget, int32_t max_resident, int32_t drain) {
    felog_server_config cfg{};
    cfg.hbm_budget = budget;
    cfg.max_resident = max_resident;
    cfg.drain_on_destroy = drain;
    cfg.walk = {40, 1};
    cfg.train = {64, 5, 5, 0.025f, 0, 0, 4096, 0, 0, 0};
    cfg.feedback = {0, 0.65, 8, 6, 0};
    return cfg;
}

static void ring(int n, std::vector<int32_t> &off, std::vector<int32_t> &cols) {
    off.assign(n + 1, 0);
    cols.clear();
    for (int v = 0; v < n; ++v) {
        off[v] = static_cast<int32_t>(cols.size());
        cols.push_back((v + 1) % n);
        cols.push_back((v + n - 1) % n);
    }
    off[n] = static_cast<int32_t>(cols.size());
}

static uint64_t submit(felog_server *sv, int n, int *status = nullptr) {
    std::vector<int32_t> off, cols;
    ring(n, off, cols);
    uint64_t id = 0;
    const int st = felog_server_submit(sv, off.data(), cols.data(), n, static_cast<int64_t>(cols.size()), 64, 7, &id);
    if (status) *status = st;
    return id;
}

#define CHECK(c)                                                   \
    do {                                                           \
        if (!(c)) {                                                \
            std::printf("check failed: %s (line %d)\n", #c, __LINE__); \
            return 1;                                              \
        }                                                          \
    } while (0)

static int staggered() {
    auto cfg = config(size_t(1) << 30, 0, 0);
    felog_server *sv;
    CHECK(felog_server_create(&cfg, &sv) == FELOG_OK);
    std::vector<uint64_t> ids;
    for (int i = 0; i < 3; ++i) ids.push_back(submit(sv, 1000 + 600 * i));
    std::this_thread::sleep_for(std::chrono::milliseconds(2));
    for (int i = 3; i < 6; ++i) ids.push_back(submit(sv, 1000 + 600 * i));
    for (size_t i = 0; i < ids.size(); ++i) {
        felog_result r;
        CHECK(felog_server_wait(sv, ids[i], 30.0, &r) == FELOG_OK);
        CHECK(r.state == FELOG_JOB_DONE && r.rounds == 6);
        CHECK(r.tokens == 6LL * 40 * (1000 + 600 * static_cast<int64_t>(i)));
        CHECK(r.t_submit <= r.t_admit && r.t_admit <= r.t_done);
        std::vector<float> phi(static_cast<size_t>(r.n) * r.dim);
        CHECK(felog_server_fetch(sv, ids[i], phi.data()) == FELOG_OK);
        CHECK(phi[0] == 0.5f);
        CHECK(felog_server_fetch(sv, ids[i], nullptr) == FELOG_ERR_INVALID_ARG);  // forgotten
    }
    felog_server_stats s;
    CHECK(felog_server_get_stats(sv, &s) == FELOG_OK);
    CHECK(s.completed == 6 && s.admitted == 6 && s.resident_jobs == 0 && s.resident_bytes == 0);
    CHECK(felog_server_destroy(sv) == FELOG_OK);
    return 0;
}

static int budget() {
    felog_server *probe;
    auto cfg0 = config(size_t(1) << 30, 0, 0);
    CHECK(felog_server_create(&cfg0, &probe) == FELOG_OK);
    const size_t need = felog_server_job_bytes(probe, 2000, 4000, 64);
    CHECK(felog_server_destroy(probe) == FELOG_OK);
    auto cfg = config(need + need / 2, 0, 0);  // one job of 2000 nodes at a time
    felog_server *sv;
    CHECK(felog_server_create(&cfg, &sv) == FELOG_OK);
    std::vector<uint64_t> ids;
    for (int i = 0; i < 4; ++i) ids.push_back(submit(sv, 2000));
    const uint64_t big = submit(sv, 5000);
    felog_result rb;
    CHECK(felog_server_wait(sv, big, 30.0, &rb) == FELOG_OK && rb.state == FELOG_JOB_REJECTED);
    double prev_done = -1;
    for (uint64_t id : ids) {
        felog_result r;
        CHECK(felog_server_wait(sv, id, 30.0, &r) == FELOG_OK && r.state == FELOG_JOB_DONE);
        CHECK(r.t_admit >= prev_done);  // first come first served, one at a time
        prev_done = r.t_done;
    }
    felog_server_stats s;
    CHECK(felog_server_get_stats(sv, &s) == FELOG_OK);
    CHECK(s.peak_resident_jobs == 1 && s.rejected == 1 && s.peak_resident_bytes <= need + need / 2);
    CHECK(felog_server_destroy(sv) == FELOG_OK);
    return 0;
}

static int max_resident() {
    auto cfg = config(size_t(1) << 30, 2, 0);
    felog_server *sv;
    CHECK(felog_server_create(&cfg, &sv) == FELOG_OK);
    std::vector<uint64_t> ids;
    for (int i = 0; i < 7; ++i) ids.push_back(submit(sv, 500 + 100 * i));
    CHECK(felog_server_drain(sv, 30.0) == FELOG_OK);
    felog_server_stats s;
    CHECK(felog_server_get_stats(sv, &s) == FELOG_OK);
    CHECK(s.completed == 7 && s.peak_resident_jobs <= 2);
    CHECK(felog_server_destroy(sv) == FELOG_OK);
    return 0;
}

static int bad_input() {
    auto cfg = config(size_t(1) << 30, 0, 0);
    felog_server *sv;
    CHECK(felog_server_create(&cfg, &sv) == FELOG_OK);
    int32_t off[] = {0, 2, 1, 3}, cols[] = {1, 2, 0};
    uint64_t id;
    CHECK(felog_server_submit(sv, off, cols, 3, 3, 64, 1, &id) == FELOG_ERR_BAD_CSR);
    int32_t off2[] = {0, 1, 2}, cols2[] = {1, 5};
    CHECK(felog_server_submit(sv, off2, cols2, 2, 2, 64, 1, &id) == FELOG_ERR_BAD_CSR);
    int32_t off3[] = {0, 1, 2}, cols3[] = {1, 0};
    CHECK(felog_server_submit(sv, off3, cols3, 2, 2, 100, 1, &id) == FELOG_ERR_UNSUPPORTED);  // dim
    felog_result r;
    CHECK(felog_server_poll(sv, 12345, &r) == FELOG_ERR_INVALID_ARG);
    CHECK(felog_server_destroy(sv) == FELOG_OK);
    return 0;
}

static int concurrent_clients() {
    auto cfg = config(size_t(1) << 30, 0, 0);
    felog_server *sv;
    CHECK(felog_server_create(&cfg, &sv) == FELOG_OK);
    std::atomic<int> failures{0};
    std::vector<std::thread> ts;
    for (int t = 0; t < 4; ++t)
        ts.emplace_back([&, t] {
            for (int i = 0; i < 5; ++i) {
                int st = 0;
                const uint64_t id = submit(sv, 300 + 50 * t + i, &st);
                felog_result r;
                if (st || felog_server_wait(sv, id, 30.0, &r) || r.state != FELOG_JOB_DONE) failures++;
                if (felog_server_fetch(sv, id, nullptr)) failures++;
            }
        });
    for (auto &t : ts) t.join();
    CHECK(failures.load() == 0);
    felog_server_stats s;
    CHECK(felog_server_get_stats(sv, &s) == FELOG_OK && s.completed == 20);
    CHECK(felog_server_destroy(sv) == FELOG_OK);
    return 0;
}

static int destroy_with_pending(int drain) {
    auto cfg = config(size_t(1) << 30, 1, drain);
    felog_server *sv;
    CHECK(felog_server_create(&cfg, &sv) == FELOG_OK);
    for (int i = 0; i < 5; ++i) submit(sv, 3000);
    CHECK(felog_server_destroy(sv) == FELOG_OK);  // must return and release everything
    return 0;
}

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    int rc = 2;
    if (!std::strcmp(argv[1], "staggered")) rc = staggered();
    else if (!std::strcmp(argv[1], "budget")) rc = budget();
    else if (!std::strcmp(argv[1], "max_resident")) rc = max_resident();
    else if (!std::strcmp(argv[1], "bad_input")) rc = bad_input();
    else if (!std::strcmp(argv[1], "concurrent_clients")) rc = concurrent_clients();
    else if (!std::strcmp(argv[1], "destroy_abandon")) rc = destroy_with_pending(0);
    else if (!std::strcmp(argv[1], "destroy_drain")) rc = destroy_with_pending(1);
    if (rc == 0) std::printf("ok\n");
    return rc;
}
