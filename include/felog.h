/*
 * felog.h -- C ABI of the FeLoG walk + SGNS hot path on one B300 (sm_103a).
 *
 * The calls follow the paper's Sample / Train / feedback decomposition
 * (Section 5.1, Algorithm 1; the unified Sample and Train interfaces of
 * Section 5.4):
 *
 *   felog_compact_active  active flags -> ascending start list   (Alg. 1, V_a)
 *   felog_walk            Sample: uniform truncated walks        (Section 2, Alg. 1 Sampling)
 *   felog_noise_table     Pn(u) of Eq. 2 as an integer alias table
 *   felog_init_tables     embedding tables phi_in, phi_out
 *   felog_train           Train: skip-gram negative sampling     (Eq. 1, Eq. 2; Alg. 1 Training)
 *   felog_feedback        Psi (Eq. 4) and the next active set (Eq. 5; Alg. 1 Feedback)
 *   felog_embed           Algorithm 1 end to end
 *
 * and around them: felog_validate_csr (the graph checked on the device),
 * felog_embed_pipelined (round-interleaved pipeline, Section 5.3),
 * felog_walk_node2vec (second-order walks, a Sample variant of Section 5.4),
 * felog_fabc_* (walk compression, Section 5.2.2, Eq. 7, Eq. 8),
 * felog_sr_bf16 (the bf16 stores' stochastic rounding on its own),
 * felog_batch_* (many graphs in one launch sequence) and felog_server_*
 * (a request loop with continuous batching), felog_compact_active_noalloc.
 *
 * Conventions (every call):
 *   - Pointers documented "device" point to CUDA device memory owned by the
 *     caller; the library never frees caller memory and allocates none of
 *     its own except where a call says so (felog_embed_host).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and asynchronous unless stated.
 *   - Argument errors are reported synchronously by the return status and
 *     nothing is launched.  FELOG_ERR_CUDA reports a launch or runtime error
 *     seen by the call (cudaGetLastError); the message is available from
 *     felog_last_cuda_error().
 *   - No C++ exception crosses this boundary.
 *   - Thread-compatible: distinct host threads may call concurrently on
 *     distinct streams and buffers.
 *
 * Random numbers: Philox4x32-10 keyed by the 64-bit seed with counter
 * (x0, x1, x2, stream); stream 0 = walks, 1 = Psi subsets, 2 = negatives,
 * 3 = table initialisation, 4 = stochastic rounding, 7 = shared tile
 * negatives, 8 = node2vec attempts.
 */
#ifndef FELOG_H_
#define FELOG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FELOG_OK = 0,
    FELOG_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
    FELOG_ERR_BAD_CSR = 2,     /* CSR fails validation (host shape checks or felog_validate_csr) */
    FELOG_ERR_WORKSPACE = 3,   /* workspace missing or smaller than required */
    FELOG_ERR_CUDA = 4,        /* CUDA launch / runtime error */
    FELOG_ERR_UNSUPPORTED = 5, /* a parameter combination with no kernel */
    FELOG_ERR_TIMEOUT = 6      /* a bounded wait ran out */
} felog_status;

/* Undirected, unweighted graph (Table 1) in CSR form, device pointers.
 * offsets[n+1] non-decreasing with offsets[0] = 0 and offsets[n] = nnz;
 * cols[nnz] in [0, n); each row sorted ascending, symmetric, loop-free. */
typedef struct {
    const int32_t *offsets;
    const int32_t *cols;
    int32_t n;
    int64_t nnz;
} felog_csr;

/* length: nodes per walk (L >= 1); walks_per_round: walks each active node
 * starts per round (>= 1). */
typedef struct {
    int32_t length;
    int32_t walks_per_round;
} felog_walk_params;

typedef enum {
    FELOG_SGNS_HOGWILD = 0,  /* lock-free asynchronous updates (fast form) */
    FELOG_SGNS_MINIBATCH = 1, /* synchronous minibatch, bitwise reproducible */
    FELOG_SGNS_TILE = 2       /* shared-negatives tiles on the tensor cores */
} felog_sgns_mode;

typedef enum {
    FELOG_FP32 = 0,   /* float tables */
    FELOG_BF16_SR = 1 /* bfloat16 tables, float math, stochastic rounding on store */
} felog_precision;

/* dim in {32, 64, 128, 256}; 1 <= window <= 16; 1 <= negatives <= 15;
 * learning rate lr0 * max(1e-4, 1 - t / lr_total_tokens) on the global token
 * clock t; minibatch = positions per synchronous batch (MINIBATCH mode);
 * hogwild_rows_per_warp (HOGWILD mode, <= 0 selects 16): at most
 * n / hogwild_rows_per_warp walks are trained concurrently, which bounds the
 * staleness of lock-free updates on small graphs; hogwild_form selects the
 * HOGWILD kernel: 1 = full warp per pair, 2 = two pairs per warp (half warp
 * each; dim <= 128, negatives <= 7), 3 = form 2 with each walk window's
 * phi_in increments summed in shared memory (window <= 15): a warp reads a
 * context row plus its own pending increments of that node, and a window
 * position's summed increment reaches memory when the position leaves the
 * window (other warps see it then; on power-law graphs hub rows collect many
 * warps' delayed increments, which costs link AUC), 4 = form 2 with the
 * next step's context and negative rows copied to shared memory (cp.async)
 * while the current step computes (float tables of dim 32, 64 or 128, bf16
 * tables of dim 64 or 128; other shapes run form 2), 5 = form 2 on float tables
 * with each step's row increments written to shared memory and added to the
 * tables by the bulk-copy engine (cp.reduce.async.bulk, one per row; other
 * precisions run form 2); 0 = automatic: form 4 for
 * bf16 tables of dim 128 with negatives <= 7, form 2 for other shapes with
 * dim <= 128 and negatives <= 7, form 1 otherwise.
 * TILE mode (dim in {32, 64, 128}): tile_negatives = shared negatives per
 * tile (128, 256, 384 or 512; 0 selects 512: each then stands for about 20
 * per-pair draws, fewer shared negatives let hub rows take oversized stale
 * steps and training can diverge); tile_ctas = concurrent tiles
 * (0 = min(SMs, max(1, n / 28000)), which bounds how many stale tile
 * updates meet on shared rows: more tiles at once train faster and reach a
 * lower link AUC; 1 = tiles strictly in order, the reproducible form). */
typedef struct {
    int32_t dim;
    int32_t window;
    int32_t negatives;
    float lr0;
    int64_t lr_total_tokens;
    int32_t mode;      /* felog_sgns_mode */
    int32_t minibatch; /* >= 1 */
    int32_t precision; /* felog_precision */
    int32_t hogwild_rows_per_warp;
    int32_t hogwild_form;
    int32_t tile_negatives;
    int32_t tile_ctas;
    int32_t stage_flush;  /* form 3: every stage_flush centers all staged increments
                             reach memory (0: a position's when it leaves the window) */
} felog_train_params;

/* enabled = 0 is the plain method (every non-isolated node stays active);
 * mu: threshold of Eq. 5 (a node stays active iff Psi < mu); ks: subset size
 * of Eq. 4 (1..32); max_rounds: cap on Algorithm 1's loop; reactivate = 1
 * evaluates every non-isolated node each round instead of only V_a. */
typedef struct {
    int32_t enabled;
    double mu;
    int32_t ks;
    int32_t max_rounds;
    int32_t reactivate;
} felog_feedback_params;

/* Per-round record filled by felog_embed (host memory). */
typedef struct {
    int32_t round;
    int32_t n_active;   /* |V_a^r| */
    int32_t n_next;     /* |V_a^{r+1}| */
    int32_t reserved;
    int64_t tokens;     /* corpus positions trained this round */
    int64_t walk_steps; /* walk transitions this round */
    double loss;        /* summed pair loss of the round */
    float ms_walk, ms_noise, ms_train, ms_feedback; /* CUDA-event phase times */
} felog_round_stats;

const char *felog_status_string(felog_status s);
/* Text of the last CUDA error seen by a call on this host thread. */
const char *felog_last_cuda_error(void);

/* Device-side check of a caller's CSR (the shape felog_csr documents) and,
 * optionally, of a start list.  status (device int32) is cleared and then
 * receives the OR of the FELOG_CSR_* bits of every problem found (0: valid).
 * Columns are only read where a row's offsets are in range, so a malformed
 * graph is reported without any out-of-range read.  Symmetry is not checked.
 * Asynchronous: read *status after the stream reaches it.  felog_embed and
 * felog_batch_create run this check themselves and return FELOG_ERR_BAD_CSR
 * before any kernel reads the graph; the single-step calls (felog_walk,
 * felog_feedback, ...) trust the graph but guard every index they derive
 * from it, so a malformed graph cannot make them read out of range. */
enum {
    FELOG_CSR_ENDS = 1,         /* offsets[0] != 0, offsets[n] != nnz, or a row outside [0, nnz] */
    FELOG_CSR_DECREASING = 2,   /* offsets[v+1] < offsets[v] */
    FELOG_CSR_COL_RANGE = 4,    /* a column outside [0, n) */
    FELOG_CSR_ORDER = 8,        /* a row not strictly ascending (unsorted or duplicate) */
    FELOG_CSR_SELF_LOOP = 16,   /* a column equal to its row */
    FELOG_CSR_START_RANGE = 32  /* a start outside [0, n) */
};
felog_status felog_validate_csr(const felog_csr *g, const int32_t *starts, int32_t n_starts, int32_t *status,
                                void *stream);

/* Stable compaction of the active set (Algorithm 1's V_a): starts[] receives
 * the indices v with active[v] != 0 in ascending order, *n_active (device
 * int32) their count.  active: device uint8[n]; starts: device int32[n].
 * Workspace: felog_compact_workspace_bytes(n) bytes of device memory. */
size_t felog_compact_workspace_bytes(int32_t n);
felog_status felog_compact_active(const uint8_t *active, int32_t n, int32_t *starts,
                                  int32_t *n_active, void *workspace, size_t workspace_bytes,
                                  void *stream);

/* Allocation-free compaction (the paper has no counterpart: this is a
 * deployment convenience).  Same result as felog_compact_active, but it needs
 * no workspace: its scratch (one int32 count per 4096-flag tile) is a
 * file-scope device array of 4096 entries (16 KiB) that every GPU loading
 * this library holds until the process exits.  It is meant for callers that
 * must not allocate device memory: code running where an allocation could
 * synchronise the device or break a memory budget (inside a serving loop
 * with a fixed memory plan, or a host framework that owns all device
 * allocation).
 *   - n may not exceed felog_compact_active_noalloc_max_n() = 2^24; larger n
 *     returns FELOG_ERR_INVALID_ARG and launches nothing.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept for later calls, which
 *     assumes the device's primary context lives as long as the process: after
 *     a cudaDeviceReset the kept address is stale.
 *   - All calls share the one array: calls that can overlap on the GPU (on
 *     different streams, or from different threads) race and must be
 *     serialised by the caller.  Every slot a call reads is written earlier
 *     by the same call, so no clearing is needed between calls.
 *   - No cudaMalloc, cudaFree or allocating library routine is called. */
int32_t felog_compact_active_noalloc_max_n(void);
felog_status felog_compact_active_noalloc(const uint8_t *active, int32_t n, int32_t *starts,
                                          int32_t *n_active, void *stream);

/* Sample (Section 2 "Sampling process"; Section 5.4 Sample interface):
 * uniform truncated walks.  Walk (round r, rep j, start s = starts[i]) is
 * written to row j*n_starts + i of walks[n_starts*wpr][L] (device int32,
 * row-major).  Step t >= 1 draws Philox(x0=t, x1=s, x2=r*wpr+j, 0) and moves
 * to neighbour floor(u64 * deg / 2^64) (u64 = word1:word0) in CSR order.  A
 * node without neighbours ends the walk; the rest of its row is -1.
 * counts (device uint32[n], may be NULL): every written node is added to it
 * (the corpus histogram used by felog_noise_table).  The CSR is validated on
 * the host only for its sizes; starts must lie in [0, n). */
felog_status felog_walk(const felog_csr *g, const int32_t *starts, int32_t n_starts,
                        const felog_walk_params *wp, uint64_t seed, int32_t round,
                        int32_t *walks, uint32_t *counts, void *stream);

/* node2vec second-order walks, a Sample variant (Section 5.4; the rule is
 * node2vec's, Grover and Leskovec, KDD 2016): having come from t to v, the
 * next node x has weight 1/p if x == t, 1 if x is a neighbour of t, 1/q
 * otherwise.  Step 1 is uniform.  Later steps use rejection: attempt a
 * draws Philox(x0 = t | a << 16, x1 = s, x2 = r*wpr + j, stream 8),
 * proposes neighbour floor(u64 * deg / 2^64) and accepts iff
 * (hi64 >> 11) * 2^-53 < alpha(x) / max(1/p, 1, 1/q) in binary64.  After
 * 64 rejected attempts it takes the last proposal.  Rows, padding and
 * counts as felog_walk; L <= 65535; p, q > 0 finite.  The CSR rows must be
 * sorted (a binary search decides "neighbour of t"). */
felog_status felog_walk_node2vec(const felog_csr *g, const int32_t *starts, int32_t n_starts,
                                 const felog_walk_params *wp, double p, double q, uint64_t seed,
                                 int32_t round, int32_t *walks, uint32_t *counts, void *stream);

/* Corpus histogram: counts[v] += occurrences of v in tokens[n_tokens]
 * (entries < 0 are skipped).  counts must be zeroed by the caller. */
felog_status felog_count(const int32_t *tokens, int64_t n_tokens, int32_t n, uint32_t *counts,
                         void *stream);

/* Noise distribution Pn(u) of Eq. 2: unigram counts raised to 0.75, as an
 * exact integer alias table.  W_v = c_v ? max(1, floor(c^0.75 / cmax^0.75 *
 * 2^32)) : 0 (c^0.75 = sqrt(c) * sqrt(sqrt(c)) in binary64); S = sum W_v.
 * thr (device uint64[n]), alias (device int32[n]) and *S (device uint64)
 * are written; the table equals, entry for entry, the sequential sweep that
 * pairs light buckets (n W < S) with heavy ones in ascending order.  A draw
 * takes b = mulhi64(u, n) and keeps b iff mulhi64(u', S) < thr[b], else
 * alias[b].  Workspace: felog_noise_workspace_bytes(n). */
size_t felog_noise_workspace_bytes(int32_t n);
felog_status felog_noise_table(const uint32_t *counts, int32_t n, uint64_t *thr, int32_t *alias,
                               uint64_t *S, void *workspace, size_t workspace_bytes, void *stream);

/* phi_in[v][i] = (u - 1/2) / dim with u = (Philox(x0=i/4, x1=v, 0, 3) word
 * i%4 >> 8) * 2^-24 in float; phi_out = 0.  Tables are device [n][dim] of
 * float (FELOG_FP32) or bfloat16 (FELOG_BF16_SR, rounded to nearest). */
felog_status felog_init_tables(int32_t n, int32_t dim, int32_t precision, uint64_t seed,
                               void *phi_in, void *phi_out, void *stream);

/* Train (Eq. 1, Eq. 2; Section 5.4 Train interface): skip-gram with negative
 * sampling over the corpus walks[n_walks][L] (device int32; -1 = padding).
 * For every center c = walks[w][p] and window offset o in [-W, W] \ {0}
 * with a context x = walks[w][p+o] >= 0, the pair maximises
 *   log sigma(phi_in[x] . phi_out[c]) + sum_k log sigma(-phi_in[x] . phi_out[n_k])
 * with K negatives n_k drawn from the alias table (thr, alias, *S) by
 * Philox(x0 = q<<8 | k, x1 = w, x2 = round<<16 | p, 2), q the slot of o;
 * a negative equal to c is skipped.  The learning rate of a position is
 * lr0 * max(1e-4, 1 - t / lr_total_tokens), t = clock_base + w*L + p.
 * HOGWILD applies updates immediately with no locking; MINIBATCH reads the
 * tables as they stood at the start of each batch of `minibatch` positions,
 * sums the increments per row exactly (fixed point, order independent) and
 * applies them at the end of the batch.  TILE replaces the per-pair draws
 * by Ns = tile_negatives draws shared by all pairs whose center lies in one
 * tile of Tc = 128 - 2W consecutive corpus positions (tile t: positions
 * [t*Tc, t*Tc + Tc)): draw j is Philox(x0 = j, x1 = t, x2 = round, 7) through
 * the alias table, each shared negative has weight K / Ns, one equal to the
 * pair's center is skipped; eta is that of the tile's first position; the
 * scores of a tile read the tables as gathered at its start and its summed
 * increments are added at its end; products run in bf16 on the tensor
 * cores with f32 accumulation.  *loss (device double) receives the summed
 * pair loss -log sigma(s+) - sum log sigma(-s_k) (TILE: negatives weighted
 * by K / Ns).  A TILE call waits for its launch (outside stream capture)
 * and returns FELOG_ERR_TIMEOUT if a wait for the tensor cores ran out; the
 * launch then stopped early, *loss is NaN and the tables are undefined.
 * During stream capture the NaN loss is the only report.
 * Workspace: felog_train_workspace_bytes(...). */
/* Stochastic rounding to bfloat16 (the precision form's rounding of every
 * bf16 table store): out[i] = the upper half of (bits of x[i]) + r16[i],
 * i.e. the 16 random bits r16[i] are added below the kept bits and the sum
 * is truncated.  The bf16 Hogwild trainers round with the same instruction.
 * x: device float[n]; r16: device uint16[n]; out: device uint16[n] (bf16
 * patterns).  n >= 0; pointers may be NULL only when n == 0.  Finite inputs
 * round as stated (a carry out of the largest finite value gives infinity);
 * infinities stay; a NaN gives a NaN. */
felog_status felog_sr_bf16(const float *x, const uint16_t *r16, int64_t n, uint16_t *out, void *stream);

size_t felog_train_workspace_bytes(int64_t n_walks, int32_t L, int32_t n,
                                   const felog_train_params *tp);
felog_status felog_train(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                         const felog_train_params *tp, const uint64_t *thr, const int32_t *alias,
                         const uint64_t *S, uint64_t seed, int32_t round, int64_t clock_base,
                         void *phi_in, void *phi_out, double *loss, void *workspace,
                         size_t workspace_bytes, void *stream);

/* Feedback (Eq. 4, Eq. 5): Psi(v) = mean cosine of phi_in[v] with a subset of
 * min(deg, ks) neighbours (all of them if deg <= ks, else ks distinct CSR
 * positions by Floyd's algorithm keyed Philox(x0=s, x1=v, x2=round, 1),
 * sorted ascending), in binary64 with a fixed summation order (partials over
 * i = l mod 32, then a xor butterfly 16..1).  Evaluated nodes: those with
 * active_in[v] and deg > 0 (every deg > 0 node when reactivate).
 * active_out[v] = evaluated && Psi < mu (feedback enabled) or deg > 0
 * (disabled).  psi (device double[n], may be NULL) gets Psi or NaN for
 * nodes not evaluated; *n_next (device int32) the size of the next set. */
felog_status felog_feedback(const felog_csr *g, const void *phi_in, int32_t dim, int32_t precision,
                            const felog_feedback_params *fp, uint64_t seed, int32_t round,
                            const uint8_t *active_in, uint8_t *active_out, double *psi,
                            int32_t *n_next, void *stream);

/* Algorithm 1 end to end on one GPU: V_a <- non-isolated nodes; for each
 * round: compact V_a, walk (counts fused), noise table, train, feedback,
 * until V_a is empty or max_rounds.  lr_total_tokens <= 0 selects
 * max_rounds * wpr * |non-isolated| * L.  phi_in / phi_out (device
 * [n][dim]) are initialised by the call; phi_in is the embedding.
 * stats (host, max_rounds entries, may be NULL) and *rounds_run (host, may be
 * NULL) are filled; the call synchronises `stream` once per round to read
 * |V_a|.  Workspace: felog_embed_workspace_bytes(...). */
size_t felog_embed_workspace_bytes(int32_t n, const felog_walk_params *wp,
                                   const felog_train_params *tp);
felog_status felog_embed(const felog_csr *g, const felog_walk_params *wp,
                         const felog_train_params *tp, const felog_feedback_params *fp,
                         uint64_t seed, void *phi_in, void *phi_out, felog_round_stats *stats,
                         int32_t *rounds_run, void *workspace, size_t workspace_bytes,
                         void *stream);

/* ------------------------------------------------------------------------
 * Round-interleaved pipeline (Section 5.3): Algorithm 1 with its operators
 * in two pipelines on one GPU.  The caller's stream trains (T_r); a stream
 * the library creates computes Psi_r and V_a^{r+1}, compacts it, samples
 * round r + 1 (walks, counts) and builds its noise table into a second set of
 * round buffers.  feedback_lag = 1 takes Section 5.3's stale-snapshot
 * reading: Psi_r reads a copy of phi_in taken as T_r starts (the table after
 * round r - 1), so round r + 1's sampling overlaps T_r; feedback_lag = 0 is
 * Algorithm 1 as printed (Psi_r after T_r; no overlap).  Results, per
 * round, equal those of a serial run with the same feedback rule (the
 * oracle's Algorithm 1 with the same lag).  The call synchronises once per
 * round, with the sample stream only.  Stats: per round as felog_embed, with
 * ms_train = T_r on the train stream and ms_feedback = the sample stream's
 * work after T_r starts (walk and noise times are folded into it).
 * TILE-mode training waits for its launch (see felog_train), which
 * serialises the two streams.
 * ------------------------------------------------------------------------ */
typedef struct {
    double wall_ms;        /* first sample to last round's end, CUDA events */
    double train_busy_ms;  /* sum of T_r */
    double sample_busy_ms; /* sum of the sample stream's work */
    double overlap_ms;     /* time both streams were busy */
    int32_t rounds;
    int32_t feedback_lag;
} felog_pipeline_stats;

size_t felog_pipeline_workspace_bytes(int32_t n, const felog_walk_params *wp, const felog_train_params *tp,
                                      int32_t max_rounds, int32_t feedback_lag);
felog_status felog_embed_pipelined(const felog_csr *g, const felog_walk_params *wp,
                                   const felog_train_params *tp, const felog_feedback_params *fp,
                                   int32_t feedback_lag, uint64_t seed, void *phi_in, void *phi_out,
                                   felog_round_stats *stats, felog_pipeline_stats *pstats, int32_t *rounds_run,
                                   void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * FaBC (Section 5.2.2, Eq. 7, Eq. 8): frequency-aware bitmap compression of
 * a walk corpus, to persist it or move it off the GPU.
 *
 * Selection: nodes ordered by frequency p = count / total (ties to the
 * smaller id); with c = 1/L + 1/32 and g(k) = 1 - F_k + k c (Eq. 7), k grows
 * from 0 while p(k+1) >= c + 0.1 g(k) (Eq. 8; the first node that fails
 * stops it) and k < k_max <= felog_fabc_max_k() = 32.
 *
 * Encoded layout for n_seq sequences of L ids, B = ceil(L / 8):
 *   n_seq*k int32      the k selected ids, stored with every sequence
 *   n_seq*k*B bytes    bitmap (s, j) at byte (s*k + j)*B: bit i (byte i/8,
 *                      bit i%8) is set iff walks[s][i] == ids[j]
 *   int32 tail         the ids of the positions no bitmap covers, sequence
 *                      by sequence in position order (little-endian, not
 *                      padded: it starts 4*n_seq*k + n_seq*k*B bytes in)
 * Its size is 4*n_seq*k + n_seq*k*B + 4*tail bytes, which for L a multiple
 * of 8 is g(k) * 4*n_seq*L with F_k the covered fraction of positions.
 * Any int32 value round-trips, -1 padding included.
 * ------------------------------------------------------------------------ */
int32_t felog_fabc_max_k(void);
/* Device workspace for n_seq sequences (selection needs felog_fabc_workspace_bytes(0)). */
size_t felog_fabc_workspace_bytes(int64_t n_seq);
/* Capacity an encode output needs: 4*n_seq*k + n_seq*k*B + 4*n_seq*L. */
size_t felog_fabc_max_bytes(int64_t n_seq, int32_t L, int32_t k);
/* counts: device uint32[n] (corpus frequencies, e.g. from felog_walk); ids:
 * host int32[k_max]; *k and *F (host; F may be NULL) receive k and F_k.
 * Synchronises `stream` to read the candidates. */
felog_status felog_fabc_select(const uint32_t *counts, int32_t n, int32_t L, int32_t k_max,
                               int32_t *ids, int32_t *k, double *F, void *workspace,
                               size_t workspace_bytes, void *stream);
/* walks: device int32[n_seq][L]; ids: device int32[k] (distinct); out:
 * device bytes, 4-byte aligned, out_bytes >= felog_fabc_max_bytes; *tail
 * (device int64) receives the number of tail ids.  A misaligned out or
 * walks returns FELOG_ERR_INVALID_ARG.  With k = 0 the encoding is the walks
 * verbatim. */
felog_status felog_fabc_encode(const int32_t *walks, int64_t n_seq, int32_t L, const int32_t *ids,
                               int32_t k, uint8_t *out, size_t out_bytes, int64_t *tail,
                               void *workspace, size_t workspace_bytes, void *stream);
/* in: device encoded bytes (4-byte aligned, else FELOG_ERR_INVALID_ARG),
 * in_bytes of them: reads stay below in_bytes, and a tail position past it
 * (a damaged buffer) decodes as -1; walks: device int32[n_seq][L]. */
felog_status felog_fabc_decode(const uint8_t *in, size_t in_bytes, int64_t n_seq, int32_t L, int32_t k,
                               int32_t *walks, void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Batching form: many independent embedding jobs (Algorithm 1 each) trained
 * together.  One round of every unfinished job runs as one fixed sequence
 * of launches with no host synchronisation, each job at its own round index,
 * so felog_batch_run can capture all rounds in one CUDA graph.  A job's walks,
 * alias tables and Psi are exactly those of the single-graph calls with the
 * same seed.  Training (dim <= 128, negatives <= 7): HOGWILD mode runs the
 * half-warp Hogwild step with at most n_j / hogwild_rows_per_warp warps on
 * job j at once; MINIBATCH mode (the deterministic form) runs one
 * synchronous batch per round and job (tp->minibatch is ignored), so every
 * job's tables, |V_a| and losses equal, bit for bit, felog_embed's for that
 * job alone with a minibatch covering the round; it needs 16 * dim + 8 more
 * bytes of device memory per node (fixed-point accumulators and marks).
 * ------------------------------------------------------------------------ */
typedef struct {
    felog_csr graph;          /* device CSR, node ids local to the job */
    uint64_t seed;
    int32_t dim;              /* 32, 64 or 128 */
    void *phi_in, *phi_out;   /* device [n][dim] tables in the batch precision */
} felog_job;

typedef struct {
    int32_t rounds;           /* rounds run */
    int32_t done;             /* 1 once V_a emptied or max_rounds was reached */
    int64_t tokens;           /* corpus positions trained */
    int64_t n_live;           /* non-isolated nodes */
    double loss_last;         /* summed pair loss of the last round */
} felog_job_stats;

typedef struct {              /* a job's device buffers (owned by the batch) */
    uint8_t *active[2];
    int32_t *starts, *walks;  /* walks of the last round: row i = walk of starts[i] */
    uint32_t *counts;
    uint64_t *thr;
    int32_t *alias;
} felog_job_buffers;

typedef struct {
    int32_t walk_block;             /* threads per block of the walk kernel */
    int32_t sgns_blocks_per_sm;     /* resident trainer blocks per SM */
    int32_t feedback_blocks_per_sm; /* Psi blocks per SM */
    int32_t from_cache;             /* 1 when read from the cache file */
    int32_t sgns_form;              /* trainer shape: 2 = two pairs per warp, 16 lanes per row;
                                       1 = one pair per warp, 32 lanes per row; 4 = shape 2 with
                                       each step's rows copied to shared memory one step ahead
                                       (jobs with rows of 256 or 512 bytes: float dim 64/128,
                                       bf16 dim 128; other jobs run shape 2) */
} felog_tuning;

typedef struct felog_batch felog_batch;

/* Allocates (cudaMalloc) the per-job buffers and tables; tp->dim is ignored
 * (each job has its own dim); lr_total_tokens <= 0 derives each job's
 * horizon from its own graph.  Jobs' graphs and tables stay caller-owned and
 * must outlive the batch. */
felog_status felog_batch_create(const felog_job *jobs, int32_t n_jobs, const felog_walk_params *wp,
                                const felog_train_params *tp, const felog_feedback_params *fp,
                                felog_batch **out);
felog_status felog_batch_destroy(felog_batch *b);
size_t felog_batch_device_bytes(const felog_batch *b);
/* initialise tables and V_a of every job (round 0) */
felog_status felog_batch_reset(felog_batch *b, void *stream);
/* one round of every unfinished job */
felog_status felog_batch_step(felog_batch *b, void *stream);
/* reset + max_rounds steps.  use_graph = 0: ordinary launches; 1: the
 * launches captured in one CUDA graph (instantiated on first use, relaunched
 * afterwards; needs a non-NULL stream); 2: one persistent kernel for all
 * rounds (every phase of every job, separated by grid-wide barriers; a
 * cooperative launch of as many blocks as can be resident, the trainer in
 * its two-pairs-per-warp shape).  Every form computes the same values.  A
 * barrier wait gives up once it has waited the batch's wait limit (60 s
 * unless felog_batch_set_wait_limit says otherwise); every block then leaves
 * at its next barrier and felog_batch_read returns FELOG_ERR_TIMEOUT. */
felog_status felog_batch_run(felog_batch *b, int32_t use_graph, void *stream);
/* budget of each grid-barrier wait of the persistent form, in seconds of the
 * GPU's global timer; 0 < seconds <= 3600, else FELOG_ERR_INVALID_ARG.  It
 * must exceed the longest phase (a round's training of every job). */
felog_status felog_batch_set_wait_limit(felog_batch *b, double seconds);
/* Check of the persistent form's grid barrier on its own: a cooperative
 * launch of as many blocks as can be resident passes `passes` (1..1024)
 * barriers that each expect `phantom` (0..1024) arrivals more than there are
 * blocks.  phantom = 0: returns FELOG_OK and *where = -1.  phantom > 0: the
 * first barrier never releases, every wait gives up after `seconds`
 * (0 < seconds <= 60) and the call returns FELOG_ERR_TIMEOUT with *where = 0,
 * the index of the barrier that ran out; the context stays usable.  Allocates
 * 16 bytes stream-ordered and synchronises `stream`. */
felog_status felog_grid_barrier_check(int32_t phantom, int32_t passes, double seconds, int32_t *where,
                                      void *stream);
/* synchronises `stream`; stats [n_jobs] (caller order), per-round |V_a| and
 * loss [max_rounds][n_jobs] (each may be NULL) */
felog_status felog_batch_read(felog_batch *b, felog_job_stats *stats, int32_t *rec_n_active,
                              double *rec_loss, void *stream);
felog_status felog_batch_job_buffers(const felog_batch *b, int32_t job, felog_job_buffers *out);
/* times the walk kernel's block size, the trainer's shape (pairs per warp,
 * lanes per row, rows prefetched or not: felog_tuning.sgns_form) with its
 * resident blocks per SM (HOGWILD mode), and Psi blocks per SM, each on
 * round 0, and keeps the fastest; shapes that would change the estimator
 * (the staged form) are not tried.  cache_path (may be NULL) is a text file
 * of earlier results keyed by GPU name and batch shape.  Leaves the batch
 * reset. */
felog_status felog_batch_autotune(felog_batch *b, const char *cache_path, felog_tuning *out, void *stream);
/* sets the launch shapes (from_cache ignored): walk_block a multiple of 32
 * in [32, 1024], sgns_blocks_per_sm 1..8, feedback_blocks_per_sm 1..32,
 * sgns_form 1, 2 or 4; else FELOG_ERR_INVALID_ARG.  Values are unchanged by
 * any shape. */
felog_status felog_batch_set_tuning(felog_batch *b, const felog_tuning *t);

/* ------------------------------------------------------------------------
 * Serving form: a request loop over embedding jobs with continuous batching.
 * Clients submit host CSRs at any time; a worker thread admits queued jobs
 * first come first served when their device bytes (CSR, tables, work
 * buffers; felog_server_job_bytes) fit in the HBM budget beside the
 * resident jobs, runs one round of Algorithm 1 for all resident jobs
 * together per iteration (each at its own round, the multi-graph step of the
 * batching form), and on completion copies the job's phi_in to host memory
 * and releases its device memory.  A job larger than the whole budget is
 * rejected.  Times are seconds on the server's steady clock.
 * ------------------------------------------------------------------------ */
enum {
    FELOG_JOB_QUEUED = 0,
    FELOG_JOB_RUNNING = 1,
    FELOG_JOB_DONE = 2,
    FELOG_JOB_REJECTED = 3,
    FELOG_JOB_FAILED = 4
};

typedef struct {
    size_t hbm_budget;          /* bytes of device memory for resident jobs */
    int32_t max_resident;       /* cap on resident jobs (<= 0: none) */
    int32_t drain_on_destroy;   /* 1: destroy finishes queued and resident jobs first */
    felog_walk_params walk;
    felog_train_params train;   /* dim ignored (per job); HOGWILD or MINIBATCH (as the batching form), negatives <= 7 */
    felog_feedback_params feedback;
} felog_server_config;

typedef struct {
    int32_t state;              /* FELOG_JOB_* */
    int32_t rounds;
    int32_t n, dim;
    int64_t tokens, n_live;
    double t_submit, t_admit, t_done;
    double loss_last;
} felog_result;

typedef struct {
    int64_t submitted, admitted, completed, rejected, steps;
    int32_t resident_jobs, peak_resident_jobs, queued, reserved;
    size_t resident_bytes, peak_resident_bytes;
    double busy_seconds;        /* time spent in rounds (device work + readback) */
} felog_server_stats;

typedef struct felog_server felog_server;

felog_status felog_server_create(const felog_server_config *cfg, felog_server **out);
/* finishes or abandons pending work (drain_on_destroy), frees everything */
felog_status felog_server_destroy(felog_server *sv);
double felog_server_now(const felog_server *sv);
size_t felog_server_job_bytes(const felog_server *sv, int32_t n, int64_t nnz, int32_t dim);
/* host CSR (validated: offsets monotone from 0 to nnz, cols in [0, n)),
 * copied by the call; returns the request id */
felog_status felog_server_submit(felog_server *sv, const int32_t *offsets, const int32_t *cols, int32_t n,
                                 int64_t nnz, int32_t dim, uint64_t seed, uint64_t *id);
felog_status felog_server_poll(felog_server *sv, uint64_t id, felog_result *out);
/* waits until the request is done, rejected or failed (FELOG_ERR_TIMEOUT
 * after timeout_s seconds) */
felog_status felog_server_wait(felog_server *sv, uint64_t id, double timeout_s, felog_result *out);
/* copies a finished request's phi_in ([n][dim] float, may be NULL) and
 * forgets the request */
felog_status felog_server_fetch(felog_server *sv, uint64_t id, float *phi_in_host);
/* waits until nothing is queued or resident */
felog_status felog_server_drain(felog_server *sv, double timeout_s);
felog_status felog_server_get_stats(felog_server *sv, felog_server_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* FELOG_H_ */
