/*
 * felog_cpu_baseline.c -- the timed CPU baseline: the oracle's own routines
 * spread over every host core with OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY, like the oracle it calls: the benchmark's CPU
 * baseline and reference legs load it, nothing on the CUDA path does.  No
 * arithmetic of the method is written here; every value is computed by a
 * function of felog_oracle.c, called on a part of the work:
 *
 *   walks     slices of the start list through oracle_walk.  A walk is keyed
 *             by its start and round alone, so the result is bit-identical
 *             to one oracle_walk call for any number of threads.
 *   SGNS      Hogwild in binary64: each thread trains chunks of walks with
 *             oracle_sgns_serial_range on the shared tables, without locks
 *             (the lock-free SGD of word2vec and DeepWalk).  Each chunk keeps
 *             its walks' corpus indices, so the negatives and learning rates
 *             are the serial oracle's; only the interleaving of updates
 *             differs between runs.
 *   Psi       nodes in parallel through oracle_psi_node (independent per
 *             node, bit-identical to oracle_feedback).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int32_t dim, window, negatives;
    double lr0;
    int64_t lr_total_tokens;
} oracle_train_params;

int oracle_walk(const int32_t *offsets, const int32_t *cols, int32_t n, const int32_t *starts,
                int32_t n_starts, int32_t L, int32_t wpr, uint64_t seed, int32_t round, int32_t *walks);
double oracle_sgns_serial_range(const int32_t *walks, int64_t w0, int64_t w1, int32_t L, int32_t n,
                                const oracle_train_params *tp, const uint64_t *thr, const int32_t *alias,
                                uint64_t S, uint64_t seed, int32_t round, int64_t clock_base,
                                double *phi_in, double *phi_out);
double oracle_psi_node(const int32_t *offsets, const int32_t *cols, const double *phi, int32_t d,
                       int32_t ks, uint64_t seed, int32_t round, int32_t v);

int baseline_threads(void) { return omp_get_max_threads(); }

/* one walk per start (wpr = 1), rows in start order */
int baseline_walk(const int32_t *offsets, const int32_t *cols, int32_t n, const int32_t *starts,
                  int32_t n_starts, int32_t L, uint64_t seed, int32_t round, int32_t *walks) {
    const int32_t chunk = 1024;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t i0 = 0; i0 < n_starts; i0 += chunk) {
        const int32_t cnt = n_starts - i0 < chunk ? n_starts - i0 : chunk;
        bad |= oracle_walk(offsets, cols, n, starts + i0, cnt, L, 1, seed, round, walks + (int64_t)i0 * L);
    }
    return bad;
}

/* walks [0, n_walks) of the round's corpus, chunks of 16 walks per thread */
double baseline_sgns_hogwild(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                             const oracle_train_params *tp, const uint64_t *thr, const int32_t *alias,
                             uint64_t S, uint64_t seed, int32_t round, int64_t clock_base, double *phi_in,
                             double *phi_out) {
    const int64_t chunk = 16;
    double loss = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : loss)
    for (int64_t w0 = 0; w0 < n_walks; w0 += chunk) {
        const int64_t w1 = w0 + chunk < n_walks ? w0 + chunk : n_walks;
        loss += oracle_sgns_serial_range(walks, w0, w1, L, n, tp, thr, alias, S, seed, round, clock_base,
                                         phi_in, phi_out);
    }
    return loss;
}

/* Psi of the listed nodes (psi[i] for nodes[i]) */
void baseline_psi(const int32_t *offsets, const int32_t *cols, const double *phi, int32_t d, int32_t ks,
                  uint64_t seed, int32_t round, const int32_t *nodes, int64_t m, double *psi) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < m; ++i)
        psi[i] = oracle_psi_node(offsets, cols, phi, d, ks, seed, round, nodes[i]);
}
