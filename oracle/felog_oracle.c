/*
 * felog_oracle.c -- plain, slow, obviously-correct CPU oracle for the FeLoG
 * walk + skip-gram-negative-sampling hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA path shares
 * no code, header, table or helper with it.
 *
 * Floating point is IEEE binary64 throughout, compiled without FMA
 * contraction (-ffp-contract=off) so every sum and product is individually
 * rounded.  Each function names the passage of the paper it follows:
 *
 *   Section 2, Eq. 1 / Eq. 2  skip-gram objective with negative sampling
 *   Section 5.1, Eq. 4        neighbourhood-consistency score Psi
 *   Section 5.1, Eq. 5        next active set
 *   Algorithm 1               sample -> train -> feedback loop
 *   Section 6.4               link-prediction AUC
 *
 * Where the paper is silent, the reading taken is stated beside the code.
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel Random Numbers: As Easy as 1, 2, 3", SC 2011), keyed by the
 * 64-bit seed, with a 4-word counter (x0, x1, x2, stream).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define STREAM_WALK 0u
#define STREAM_PSI 1u
#define STREAM_NEG 2u
#define STREAM_INIT 3u
#define STREAM_SR 4u
#define STREAM_TILE 7u
#define STREAM_N2V 8u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC 2011): ten rounds of two 32x32->64 multiplies; the key  */
/* is bumped by the two Weyl constants between rounds.                       */
/* ------------------------------------------------------------------------ */
void oracle_philox(uint64_t seed, const uint32_t ctr_in[4], uint32_t out[4]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox4(uint64_t seed, uint32_t x0, uint32_t x1, uint32_t x2, uint32_t stream,
                    uint32_t out[4]) {
    uint32_t ctr[4] = {x0, x1, x2, stream};
    oracle_philox(seed, ctr, out);
}

/* floor(u * m / 2^64): an integer uniformly spread over [0, m) */
static uint64_t mulhi64(uint64_t u, uint64_t m) {
    return (uint64_t)(((unsigned __int128)u * (unsigned __int128)m) >> 64);
}

static uint64_t lo_word64(const uint32_t w[4]) { return ((uint64_t)w[1] << 32) | w[0]; }
static uint64_t hi_word64(const uint32_t w[4]) { return ((uint64_t)w[3] << 32) | w[2]; }

/* ------------------------------------------------------------------------ */
/* Uniform truncated random walks (Section 2 "Sampling process"; the Sample  */
/* interface of Section 5.1 and Section 5.4, Algorithm 1 step "Sampling").   */
/*                                                                           */
/* Readings: L counts nodes; each start issues wpr walks per round; walk     */
/* (round r, rep j, start s) draws step t from Philox(x0=t, x1=s,            */
/* x2=r*wpr+j, WALK); the next node is neighbour floor(u64*deg/2^64) of the  */
/* current node in CSR order.  A node with no neighbours ends the walk and   */
/* the rest of the row is -1.  Output row (j*n_starts + i) holds the walk of */
/* starts[i], rep j.                                                         */
/* ------------------------------------------------------------------------ */
int oracle_walk(const int32_t *offsets, const int32_t *cols, int32_t n, const int32_t *starts,
                int32_t n_starts, int32_t L, int32_t wpr, uint64_t seed, int32_t round,
                int32_t *walks) {
    if (L < 1 || wpr < 1 || n_starts < 0) return 1;
    for (int32_t j = 0; j < wpr; ++j) {
        for (int32_t i = 0; i < n_starts; ++i) {
            int32_t *row = walks + ((int64_t)j * n_starts + i) * L;
            int32_t s = starts[i];
            if (s < 0 || s >= n) return 2;
            int32_t v = s;
            row[0] = s;
            for (int32_t t = 1; t < L; ++t) {
                int64_t deg = (int64_t)offsets[v + 1] - offsets[v];
                if (deg == 0) {
                    for (int32_t q = t; q < L; ++q) row[q] = -1;
                    break;
                }
                uint32_t w[4];
                philox4(seed, (uint32_t)t, (uint32_t)s, (uint32_t)(round * wpr + j), STREAM_WALK, w);
                uint64_t idx = mulhi64(lo_word64(w), (uint64_t)deg);
                v = cols[offsets[v] + (int64_t)idx];
                row[t] = v;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* node2vec second-order walks (a Sample variant the paper names, Section   */
/* 5.4; the rule is node2vec's, Grover and Leskovec, KDD 2016): having come */
/* from t to v, the next node x, a neighbour of v, has unnormalised weight  */
/* 1/p if x == t, 1 if x is a neighbour of t, 1/q otherwise.                */
/* Reading (sampling procedure): step 1 is uniform; later steps use         */
/* rejection -- attempt a draws Philox(x0 = t | a << 16, x1 = s,            */
/* x2 = r*wpr + j, stream 8), proposes neighbour floor(u64 * deg / 2^64)    */
/* and accepts iff (hi64 >> 11) * 2^-53 < alpha(x) / alpha_max in binary64, */
/* alpha_max = max(1/p, 1, 1/q); after 64 rejected attempts the last        */
/* proposal is taken.  Rows, padding and start handling as in oracle_walk.  */
/* ------------------------------------------------------------------------ */
static int is_neighbour(const int32_t *offsets, const int32_t *cols, int32_t t, int32_t x) {
    for (int32_t e = offsets[t]; e < offsets[t + 1]; ++e)
        if (cols[e] == x) return 1;
    return 0;
}

int oracle_walk_node2vec(const int32_t *offsets, const int32_t *cols, int32_t n, const int32_t *starts,
                         int32_t n_starts, int32_t L, int32_t wpr, double p, double q, uint64_t seed,
                         int32_t round, int32_t *walks) {
    if (L < 1 || L > 65535 || wpr < 1 || n_starts < 0 || !(p > 0.0) || !(q > 0.0)) return 1;
    const double ap = 1.0 / p, aq = 1.0 / q;
    const double amax = ap > 1.0 ? (ap > aq ? ap : aq) : (1.0 > aq ? 1.0 : aq);
    for (int32_t j = 0; j < wpr; ++j) {
        for (int32_t i = 0; i < n_starts; ++i) {
            int32_t *row = walks + ((int64_t)j * n_starts + i) * L;
            int32_t s = starts[i];
            if (s < 0 || s >= n) return 2;
            int32_t prev = -1, v = s;
            row[0] = s;
            for (int32_t t = 1; t < L; ++t) {
                int64_t deg = (int64_t)offsets[v + 1] - offsets[v];
                if (deg == 0) {
                    for (int32_t r = t; r < L; ++r) row[r] = -1;
                    break;
                }
                int32_t x = -1;
                for (uint32_t a = 0; a < 64; ++a) {
                    uint32_t w[4];
                    philox4(seed, (uint32_t)t | (a << 16), (uint32_t)s, (uint32_t)(round * wpr + j),
                            STREAM_N2V, w);
                    x = cols[offsets[v] + (int64_t)mulhi64(lo_word64(w), (uint64_t)deg)];
                    if (prev < 0) break; /* first step: uniform */
                    double alpha = x == prev ? ap : (is_neighbour(offsets, cols, prev, x) ? 1.0 : aq);
                    double u = (double)(hi_word64(w) >> 11) * 0x1p-53;
                    if (u < alpha / amax) break;
                }
                prev = v;
                v = x;
                row[t] = v;
            }
        }
    }
    return 0;
}

/* occurrences of every node in a corpus (the round's walks) */
void oracle_counts(const int32_t *walks, int64_t n_tokens, int32_t n, uint32_t *counts) {
    memset(counts, 0, sizeof(uint32_t) * (size_t)n);
    for (int64_t p = 0; p < n_tokens; ++p)
        if (walks[p] >= 0) counts[walks[p]] += 1;
}

/* ------------------------------------------------------------------------ */
/* Noise distribution Pn(u) of Eq. 2 as an integer alias table.              */
/*                                                                           */
/* Reading: Pn is the unigram distribution of the round's corpus raised to   */
/* 0.75.  The weight c^0.75 is formed as sqrt(c)*sqrt(sqrt(c)) in binary64   */
/* (each step correctly rounded) and quantised to an integer                 */
/*   W_v = c_v ? max(1, floor(w_v / w_max * 2^32)) : 0.                      */
/* With S = sum W and masses m_v = n * W_v, a bucket b holds (thr[b],        */
/* alias[b]) with thr in [0, S]; a draw picks bucket b uniformly and keeps b */
/* when a second uniform integer in [0, S) is below thr[b], else alias[b].   */
/* The table is built by the sequential "sweep": a cursor i over light items */
/* (m < S) and a cursor j over heavy items (m >= S), both ascending, and the */
/* current heavy item's remaining mass rem:                                  */
/*   - if rem < S, heavy j is now light: thr[j] = rem, alias[j] = next heavy */
/*     j', and rem = m_j' - (S - rem), j = j'.  (Checked first.)             */
/*   - else the next light item i gets thr[i] = m_i, alias[i] = j, and       */
/*     rem -= S - m_i.                                                       */
/* Buckets never assigned keep thr = S (alias = itself).  All arithmetic is  */
/* exact in 64-bit integers, so the table is a pure function of the counts.  */
/* ------------------------------------------------------------------------ */
int oracle_noise_table(const uint32_t *counts, int32_t n, uint64_t *W, uint64_t *thr,
                       int32_t *alias, uint64_t *S_out) {
    double wmax = 0.0;
    for (int32_t v = 0; v < n; ++v) {
        if (counts[v] == 0) continue;
        double c = (double)counts[v];
        double w = sqrt(c) * sqrt(sqrt(c));
        if (w > wmax) wmax = w;
    }
    uint64_t S = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (counts[v] == 0) {
            W[v] = 0;
            continue;
        }
        double c = (double)counts[v];
        double w = sqrt(c) * sqrt(sqrt(c));
        double q = floor((w / wmax) * 4294967296.0);
        uint64_t Wv = (uint64_t)q;
        W[v] = Wv < 1 ? 1 : Wv;
        S += W[v];
    }
    *S_out = S;
    for (int32_t v = 0; v < n; ++v) {
        thr[v] = S;
        alias[v] = v;
    }
    if (S == 0) return 0; /* empty corpus: no draws are possible */
    const uint64_t nn = (uint64_t)n;
    int32_t i = 0, j = 0;
    while (i < n && nn * W[i] >= S) ++i; /* first light */
    while (j < n && nn * W[j] < S) ++j;  /* first heavy */
    if (j >= n) return 3;                /* cannot happen: some mass is >= the mean */
    uint64_t rem = nn * W[j];
    for (;;) {
        if (rem < S) {
            int32_t j2 = j + 1;
            while (j2 < n && nn * W[j2] < S) ++j2;
            if (j2 >= n) return 4; /* cannot happen with exact arithmetic */
            thr[j] = rem;
            alias[j] = j2;
            rem = nn * W[j2] - (S - rem);
            j = j2;
        } else if (i < n) {
            thr[i] = nn * W[i];
            alias[i] = j;
            rem -= S - nn * W[i];
            ++i;
            while (i < n && nn * W[i] >= S) ++i;
        } else {
            break;
        }
    }
    return 0;
}

/* negative draw for slot k of context slot q of the token at (walk, pos) */
int32_t oracle_draw_negative(const uint64_t *thr, const int32_t *alias, int32_t n, uint64_t S,
                             uint64_t seed, int32_t round, int64_t walk_idx, int32_t pos,
                             int32_t q, int32_t k) {
    uint32_t w[4];
    philox4(seed, ((uint32_t)q << 8) | (uint32_t)k, (uint32_t)walk_idx,
            ((uint32_t)round << 16) | (uint32_t)pos, STREAM_NEG, w);
    uint64_t b = mulhi64(lo_word64(w), (uint64_t)n);
    uint64_t coin = mulhi64(hi_word64(w), S);
    return coin < thr[b] ? (int32_t)b : alias[b];
}

/* ------------------------------------------------------------------------ */
/* Table initialisation (word2vec convention; the paper is silent):         */
/* phi_in[v][i] = (u - 1/2) / d with u a 24-bit uniform from                 */
/* Philox(x0=i/4, x1=v, 0, INIT) word i%4, computed in binary32; phi_out = 0.*/
/* ------------------------------------------------------------------------ */
void oracle_init_tables(int32_t n, int32_t d, uint64_t seed, double *phi_in, double *phi_out) {
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t i = 0; i < d; ++i) {
            uint32_t w[4];
            philox4(seed, (uint32_t)(i / 4), (uint32_t)v, 0u, STREAM_INIT, w);
            float u = (float)(w[i % 4] >> 8) * 0x1p-24f;
            float x = (u - 0.5f) / (float)d;
            phi_in[(int64_t)v * d + i] = (double)x;
            phi_out[(int64_t)v * d + i] = 0.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Stochastic rounding of a binary32 value to bfloat16 (precision form:      */
/* bf16 tables with float arithmetic and stochastic rounding on every        */
/* store).  Definition: a bfloat16 is the upper half of a binary32 pattern;  */
/* x lies between its truncation RD = x & 0xffff0000 and the next pattern    */
/* away from zero, at the fraction f = (x & 0xffff) / 2^16 of the way.  SR   */
/* returns the farther one with probability f: a uniform 16-bit r is added   */
/* to the lower half and the sum is truncated, which carries into the upper  */
/* half for exactly the f * 2^16 values r >= 2^16 - (x & 0xffff).  Carries   */
/* run through the exponent, so the rounding crosses binades and reaches     */
/* infinity from the largest finite values, as rounding away from zero      */
/* does.  Reading: infinities are returned unchanged; any NaN returns the    */
/* canonical quiet NaN 0x7fc0 (truncating could turn a NaN whose payload is  */
/* in the lower half into an infinity).  Returns the bf16 bit pattern.       */
/* ------------------------------------------------------------------------ */
uint32_t oracle_sr_bf16(uint32_t xbits, uint32_t r16) {
    uint32_t exponent = (xbits >> 23) & 0xffu, mantissa = xbits & 0x7fffffu;
    if (exponent == 0xffu) return mantissa ? 0x7fc0u : (xbits >> 16);
    return (uint32_t)(((uint64_t)xbits + (r16 & 0xffffu)) >> 16) & 0xffffu;
}

/* The keyed form: r16 is the low half of word (element % 4) of             */
/* Philox(seed; x0 = element / 4, x1 = row, x2 = counter, stream 4), the     */
/* rounding stream keyed by element, row and a per-row update counter.       */
uint32_t oracle_sr_bf16_keyed(uint32_t xbits, uint64_t seed, uint32_t element, uint32_t row,
                              uint32_t counter) {
    uint32_t w[4];
    philox4(seed, element / 4u, row, counter, STREAM_SR, w);
    return oracle_sr_bf16(xbits, w[element % 4u] & 0xffffu);
}

/* Stochastic rounding of an array with caller-supplied bits: out[i] =      */
/* SR(x[i]) with r16[i].                                                     */
void oracle_sr_bf16_array(const uint32_t *x, const uint16_t *r16, int64_t m, uint16_t *out) {
    for (int64_t i = 0; i < m; ++i) out[i] = (uint16_t)oracle_sr_bf16(x[i], r16[i]);
}

/* A row store with stochastic rounding: out[i] = SR(x[i]) with the bits of  */
/* element i of the rounding stream keyed (i / 4, row, counter).             */
void oracle_sr_bf16_row(const uint32_t *x, int64_t m, uint64_t seed, uint32_t row, uint32_t counter,
                        uint16_t *out) {
    for (int64_t i = 0; i < m; ++i)
        out[i] = (uint16_t)oracle_sr_bf16_keyed(x[i], seed, (uint32_t)i, row, counter);
}

/* linear learning-rate decay on the global token clock (reading: word2vec) */
double oracle_learning_rate(double lr0, int64_t t, int64_t T) {
    double f = 1.0 - (double)t / (double)T;
    return lr0 * (f < 1e-4 ? 1e-4 : f);
}

/* -log sigma(z) = log(1 + exp(-z)), evaluated without overflow */
static double neg_log_sigmoid(double z) {
    return z >= 0 ? log1p(exp(-z)) : -z + log1p(exp(z));
}

static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

static double dot(const double *a, const double *b, int32_t d) {
    double s = 0.0;
    for (int32_t i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}

/* slot q in [0, 2w) of window offset o in [-w, -1] U [1, w] */
static int32_t slot_of(int32_t o, int32_t w) { return o < 0 ? o + w : o + w - 1; }

/* ------------------------------------------------------------------------ */
/* One (center c, context x) pair of Eq. 2, gradient ascent on               */
/*   log sigma(phi_in[x] . phi_out[c]) + sum_k log sigma(-phi_in[x] . phi_out[n_k]).
 * Targets are visited in order (c, n_1 .. n_K); a negative equal to c is    */
/* skipped.  For each target t with label y: f = phi_in[x].phi_out[t],       */
/* g = eta (y - sigma(f)); the context's increment accumulates g phi_out[t]  */
/* (value before the update) and phi_out[t] += g phi_in[x] immediately; the  */
/* increment is added to phi_in[x] after the last target.  Returns the pair's*/
/* loss  -log sigma(s+) - sum log sigma(-s_k)  at the values it read.        */
/* `scratch` holds d doubles.                                                */
/* ------------------------------------------------------------------------ */
double oracle_pair_update(double *in_x, double *const *out_targets, int32_t n_targets,
                          int32_t d, double eta, double *scratch) {
    double loss = 0.0;
    for (int32_t i = 0; i < d; ++i) scratch[i] = 0.0;
    for (int32_t t = 0; t < n_targets; ++t) {
        double *o = out_targets[t];
        double label = t == 0 ? 1.0 : 0.0;
        double f = dot(in_x, o, d);
        loss += t == 0 ? neg_log_sigmoid(f) : neg_log_sigmoid(-f);
        double g = eta * (label - sigmoid(f));
        for (int32_t i = 0; i < d; ++i) scratch[i] += g * o[i];
        for (int32_t i = 0; i < d; ++i) o[i] += g * in_x[i];
    }
    for (int32_t i = 0; i < d; ++i) in_x[i] += scratch[i];
    return loss;
}

typedef struct {
    int32_t dim, window, negatives;
    double lr0;
    int64_t lr_total_tokens;
} oracle_train_params;

/* ------------------------------------------------------------------------ */
/* Serial SGNS over one round's corpus (Eq. 1 summed over the walks, Eq. 2   */
/* per pair), pairs in canonical order: walks in row order, centers by       */
/* position, window offsets -w..-1, 1..w.  eta is taken from the global      */
/* token clock  clock_base + walk*L + pos.  Returns the summed loss.         */
/* ------------------------------------------------------------------------ */
/* Walks [w0, w1) of the round's corpus, in order, with their indices in the */
/* whole corpus (which key the negatives and the token clock).               */
double oracle_sgns_serial_range(const int32_t *walks, int64_t w0, int64_t w1, int32_t L, int32_t n,
                                const oracle_train_params *tp, const uint64_t *thr,
                                const int32_t *alias, uint64_t S, uint64_t seed, int32_t round,
                                int64_t clock_base, double *phi_in, double *phi_out) {
    const int32_t d = tp->dim, w = tp->window, K = tp->negatives;
    double *scratch = (double *)malloc(sizeof(double) * (size_t)d);
    double **targets = (double **)malloc(sizeof(double *) * (size_t)(K + 1));
    double loss = 0.0;
    for (int64_t wi = w0; wi < w1; ++wi) {
        const int32_t *row = walks + wi * L;
        for (int32_t p = 0; p < L; ++p) {
            int32_t c = row[p];
            if (c < 0) continue;
            double eta = oracle_learning_rate(tp->lr0, clock_base + wi * L + p, tp->lr_total_tokens);
            for (int32_t o = -w; o <= w; ++o) {
                if (o == 0) continue;
                int32_t pp = p + o;
                if (pp < 0 || pp >= L || row[pp] < 0) continue;
                int32_t x = row[pp], q = slot_of(o, w);
                int32_t nt = 0;
                targets[nt++] = phi_out + (int64_t)c * d;
                for (int32_t k = 0; k < K; ++k) {
                    int32_t nk = oracle_draw_negative(thr, alias, n, S, seed, round, wi, p, q, k);
                    if (nk == c) continue;
                    targets[nt++] = phi_out + (int64_t)nk * d;
                }
                loss += oracle_pair_update(phi_in + (int64_t)x * d, targets, nt, d, eta, scratch);
            }
        }
    }
    free(scratch);
    free(targets);
    return loss;
}

double oracle_sgns_serial(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                          const oracle_train_params *tp, const uint64_t *thr,
                          const int32_t *alias, uint64_t S, uint64_t seed, int32_t round,
                          int64_t clock_base, double *phi_in, double *phi_out) {
    return oracle_sgns_serial_range(walks, 0, n_walks, L, n, tp, thr, alias, S, seed, round, clock_base,
                                    phi_in, phi_out);
}

/* ------------------------------------------------------------------------ */
/* Synchronous-minibatch SGNS (deterministic form).  A batch is B            */
/* consecutive corpus positions (walk*L + pos).  Every pair in the batch     */
/* reads the tables as they were when the batch began, eta is the rate of    */
/* the batch's first position, the per-pair gradient terms of Eq. 2 are      */
/* summed per row, and the sums are added at the end of the batch.           */
/* Optional per-batch losses go to batch_loss (may be NULL).                 */
/* ------------------------------------------------------------------------ */
double oracle_sgns_minibatch(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                             const oracle_train_params *tp, int64_t B, const uint64_t *thr,
                             const int32_t *alias, uint64_t S, uint64_t seed, int32_t round,
                             int64_t clock_base, double *phi_in, double *phi_out,
                             double *batch_loss) {
    const int32_t d = tp->dim, w = tp->window, K = tp->negatives;
    double *din = (double *)calloc((size_t)n * d, sizeof(double));
    double *dout = (double *)calloc((size_t)n * d, sizeof(double));
    uint8_t *touched_in = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *touched_out = (uint8_t *)calloc((size_t)n, 1);
    int32_t *list_in = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *list_out = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *tg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(K + 1));
    double *g = (double *)malloc(sizeof(double) * (size_t)(K + 1));
    const int64_t total = n_walks * L;
    double loss = 0.0;
    int64_t nb = 0;
    for (int64_t b0 = 0; b0 < total; b0 += B, ++nb) {
        int64_t b1 = b0 + B < total ? b0 + B : total;
        double eta = oracle_learning_rate(tp->lr0, clock_base + b0, tp->lr_total_tokens);
        int32_t n_in = 0, n_out = 0;
        double bl = 0.0;
        for (int64_t tok = b0; tok < b1; ++tok) {
            int64_t wi = tok / L;
            int32_t p = (int32_t)(tok % L);
            const int32_t *row = walks + wi * L;
            int32_t c = row[p];
            if (c < 0) continue;
            for (int32_t o = -w; o <= w; ++o) {
                if (o == 0) continue;
                int32_t pp = p + o;
                if (pp < 0 || pp >= L || row[pp] < 0) continue;
                int32_t x = row[pp], q = slot_of(o, w);
                int32_t nt = 0;
                tg[nt++] = c;
                for (int32_t k = 0; k < K; ++k) {
                    int32_t nk = oracle_draw_negative(thr, alias, n, S, seed, round, wi, p, q, k);
                    if (nk != c) tg[nt++] = nk;
                }
                const double *ix = phi_in + (int64_t)x * d;
                for (int32_t t = 0; t < nt; ++t) {
                    double f = dot(ix, phi_out + (int64_t)tg[t] * d, d);
                    bl += t == 0 ? neg_log_sigmoid(f) : neg_log_sigmoid(-f);
                    g[t] = eta * ((t == 0 ? 1.0 : 0.0) - sigmoid(f));
                }
                if (!touched_in[x]) { touched_in[x] = 1; list_in[n_in++] = x; }
                double *dx = din + (int64_t)x * d;
                for (int32_t t = 0; t < nt; ++t) {
                    const double *ot = phi_out + (int64_t)tg[t] * d;
                    double *dt = dout + (int64_t)tg[t] * d;
                    for (int32_t i = 0; i < d; ++i) dx[i] += g[t] * ot[i];
                    for (int32_t i = 0; i < d; ++i) dt[i] += g[t] * ix[i];
                    if (!touched_out[tg[t]]) { touched_out[tg[t]] = 1; list_out[n_out++] = tg[t]; }
                }
            }
        }
        for (int32_t a = 0; a < n_in; ++a) {
            int64_t r = list_in[a];
            for (int32_t i = 0; i < d; ++i) {
                phi_in[r * d + i] += din[r * d + i];
                din[r * d + i] = 0.0;
            }
            touched_in[r] = 0;
        }
        for (int32_t a = 0; a < n_out; ++a) {
            int64_t r = list_out[a];
            for (int32_t i = 0; i < d; ++i) {
                phi_out[r * d + i] += dout[r * d + i];
                dout[r * d + i] = 0.0;
            }
            touched_out[r] = 0;
        }
        if (batch_loss) batch_loss[nb] = bl;
        loss += bl;
    }
    free(din); free(dout); free(touched_in); free(touched_out);
    free(list_in); free(list_out); free(tg); free(g);
    return loss;
}

/* The Ns shared negatives of tile t (reading of the tile form below):       */
/* draw j takes Philox(x0 = j, x1 = t, x2 = round, stream 7) and the alias   */
/* table as a per-pair draw does.                                            */
void oracle_tile_negatives(const uint64_t *thr, const int32_t *alias, int32_t n, uint64_t S,
                           uint64_t seed, int32_t round, int64_t t, int32_t Ns, int32_t *out) {
    for (int32_t j = 0; j < Ns; ++j) {
        uint32_t r4[4];
        philox4(seed, (uint32_t)j, (uint32_t)t, (uint32_t)round, STREAM_TILE, r4);
        uint64_t b = mulhi64(lo_word64(r4), (uint64_t)n);
        uint64_t coin = mulhi64(hi_word64(r4), S);
        out[j] = coin < thr[b] ? (int32_t)b : alias[b];
    }
}

/* ------------------------------------------------------------------------ */
/* Shared-negatives tile form of Eq. 2 (an estimator variant; the paper      */
/* prescribes per-pair draws).  Reading taken:                               */
/*  - tile t holds the centers at corpus positions [t*T, min(t*T+T, N)),     */
/*    positions numbered walk*L + pos, pairs formed as in the serial form;  */
/*  - the tile draws Ns negatives once: draw j uses Philox(x0 = j,           */
/*    x1 = t, x2 = round, stream 7) and the alias table exactly like a      */
/*    per-pair draw; every pair of the tile uses all Ns of them, each with  */
/*    weight K/Ns, so the expected negative term of a pair equals that of   */
/*    K independent draws; a shared negative equal to the pair's center is   */
/*    skipped for that pair (the per-pair skip rule);                       */
/*  - eta is the rate of the tile's first center position;                   */
/*  - all scores of a tile read the tables as they stood when the tile       */
/*    began and the summed increments are added when it ends (tiles run in  */
/*    order);                                                               */
/*  - normalize != 0: a node's summed increment is divided by the number of  */
/*    the tile's rows that hold it in that table -- for phi_in the distinct */
/*    context positions that take part in a pair, for phi_out the distinct  */
/*    center positions that take part in a pair plus the negative slots    */
/*    drawn as that node.  Without it, a node that a walk revisits every    */
/*    other step (a hub between degree-1 neighbours) receives dozens of     */
/*    pair gradients computed from one stale value in one step, and         */
/*    training diverges on power-law graphs.                                */
/* Per pair (x, c): loss -log sigma(f+) - (K/Ns) sum_j log sigma(-f_j),       */
/* increments g+ = eta (1 - sigma(f+)), g_j = -eta (K/Ns) sigma(f_j) applied */
/* as phi_in[x] += g phi_out[target], phi_out[target] += g phi_in[x].         */
/* tile_loss (may be NULL) receives each tile's loss.                        */
/* ------------------------------------------------------------------------ */
double oracle_sgns_tile(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                        const oracle_train_params *tp, int32_t T, int32_t Ns, int32_t normalize,
                        const uint64_t *thr, const int32_t *alias, uint64_t S, uint64_t seed,
                        int32_t round, int64_t clock_base, double *phi_in, double *phi_out,
                        double *tile_loss) {
    const int32_t d = tp->dim, w = tp->window, K = tp->negatives;
    const double omega = (double)K / (double)Ns;
    double *din = (double *)calloc((size_t)n * d, sizeof(double));
    double *dout = (double *)calloc((size_t)n * d, sizeof(double));
    uint8_t *touched_in = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *touched_out = (uint8_t *)calloc((size_t)n, 1);
    int32_t *list_in = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *list_out = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *neg = (int32_t *)malloc(sizeof(int32_t) * (size_t)Ns);
    const int64_t total = n_walks * L;
    /* rows per node in the current tile, and the tile that last counted a */
    /* position as a context / as a center                                 */
    int32_t *rows_in = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *rows_out = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int64_t *ctx_tile = (int64_t *)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    int64_t *ctr_tile = (int64_t *)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    for (int64_t i = 0; i < total; ++i) ctx_tile[i] = ctr_tile[i] = -1;
    double loss = 0.0;
    int64_t t = 0;
    for (int64_t b0 = 0; b0 < total; b0 += T, ++t) {
        int64_t b1 = b0 + T < total ? b0 + T : total;
        double eta = oracle_learning_rate(tp->lr0, clock_base + b0, tp->lr_total_tokens);
        oracle_tile_negatives(thr, alias, n, S, seed, round, t, Ns, neg);
        int32_t n_in = 0, n_out = 0;
        double tl = 0.0;
        for (int64_t tok = b0; tok < b1; ++tok) {
            int64_t wi = tok / L;
            int32_t p = (int32_t)(tok % L);
            const int32_t *row = walks + wi * L;
            int32_t c = row[p];
            if (c < 0) continue;
            for (int32_t o = -w; o <= w; ++o) {
                if (o == 0) continue;
                int32_t pp = p + o;
                if (pp < 0 || pp >= L || row[pp] < 0) continue;
                int32_t x = row[pp];
                if (ctx_tile[wi * L + pp] != t) { ctx_tile[wi * L + pp] = t; rows_in[x] += 1; }
                if (ctr_tile[tok] != t) { ctr_tile[tok] = t; rows_out[c] += 1; }
                const double *ix = phi_in + (int64_t)x * d;
                double *dx = din + (int64_t)x * d;
                if (!touched_in[x]) { touched_in[x] = 1; list_in[n_in++] = x; }
                for (int32_t j = -1; j < Ns; ++j) {
                    int32_t target = j < 0 ? c : neg[j];
                    if (j >= 0 && target == c) continue;
                    const double *ot = phi_out + (int64_t)target * d;
                    double f = dot(ix, ot, d);
                    double g;
                    if (j < 0) {
                        tl += neg_log_sigmoid(f);
                        g = eta * (1.0 - sigmoid(f));
                    } else {
                        tl += omega * neg_log_sigmoid(-f);
                        g = -eta * omega * sigmoid(f);
                    }
                    double *dt = dout + (int64_t)target * d;
                    for (int32_t i = 0; i < d; ++i) dx[i] += g * ot[i];
                    for (int32_t i = 0; i < d; ++i) dt[i] += g * ix[i];
                    if (!touched_out[target]) { touched_out[target] = 1; list_out[n_out++] = target; }
                }
            }
        }
        for (int32_t j = 0; j < Ns; ++j) rows_out[neg[j]] += 1;
        for (int32_t a = 0; a < n_in; ++a) {
            int64_t r = list_in[a];
            double sc = normalize ? 1.0 / (double)rows_in[r] : 1.0;
            for (int32_t i = 0; i < d; ++i) {
                phi_in[r * d + i] += sc * din[r * d + i];
                din[r * d + i] = 0.0;
            }
            touched_in[r] = 0;
            rows_in[r] = 0;
        }
        for (int32_t a = 0; a < n_out; ++a) {
            int64_t r = list_out[a];
            double sc = normalize ? 1.0 / (double)rows_out[r] : 1.0;
            for (int32_t i = 0; i < d; ++i) {
                phi_out[r * d + i] += sc * dout[r * d + i];
                dout[r * d + i] = 0.0;
            }
            touched_out[r] = 0;
        }
        for (int32_t j = 0; j < Ns; ++j) rows_out[neg[j]] = 0;
        for (int32_t a = 0; a < n_out; ++a) rows_out[list_out[a]] = 0;
        if (tile_loss) tile_loss[t] = tl;
        loss += tl;
    }
    free(din); free(dout); free(touched_in); free(touched_out);
    free(list_in); free(list_out); free(neg);
    free(rows_in); free(rows_out); free(ctx_tile); free(ctr_tile);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Neighbourhood-consistency score Psi (Section 5.1, Eq. 4) and next active  */
/* set (Eq. 5).                                                              */
/*                                                                           */
/* Readings: the sampled subset of size ks is drawn without replacement; if  */
/* deg <= ks the whole neighbourhood is used in CSR order, else Floyd's      */
/* algorithm picks ks distinct CSR positions (step s draws from             */
/* Philox(x0=s, x1=v, x2=round, PSI), uniform in [0, j] by 64-bit multiply- */
/* high) and they are sorted ascending.  Each dot product and squared norm   */
/* is summed in a fixed order: partial sum l in [0,32) adds elements         */
/* i = l, l+32, ... ascending; the 32 partials are then combined pairwise by */
/* xor distance 16, 8, 4, 2, 1 and partial 0 is taken.  cos = dot /          */
/* (sqrt(|v|^2) sqrt(|u|^2)); a zero norm gives cos = 0.  Psi is the sum of  */
/* the cosines in ascending subset order divided by the subset size.         */
/* ------------------------------------------------------------------------ */
static double canonical_dot(const double *a, const double *b, int32_t d) {
    double lane[32], tmp[32];
    for (int l = 0; l < 32; ++l) {
        double s = 0.0;
        for (int32_t i = l; i < d; i += 32) {
            double prod = a[i] * b[i];
            s = s + prod;
        }
        lane[l] = s;
    }
    for (int off = 16; off >= 1; off >>= 1) {
        for (int l = 0; l < 32; ++l) tmp[l] = lane[l] + lane[l ^ off];
        memcpy(lane, tmp, sizeof lane);
    }
    return lane[0];
}

/* ks distinct positions in [0, deg), ascending (deg > ks) */
void oracle_psi_subset(int64_t deg, int32_t ks, uint64_t seed, int32_t v, int32_t round,
                       int64_t *out) {
    int32_t m = 0;
    for (int32_t s = 0; s < ks; ++s) {
        int64_t j = deg - ks + s;
        uint32_t w[4];
        philox4(seed, (uint32_t)s, (uint32_t)v, (uint32_t)round, STREAM_PSI, w);
        int64_t t = (int64_t)mulhi64(lo_word64(w), (uint64_t)(j + 1));
        int present = 0;
        for (int32_t a = 0; a < m; ++a) present |= out[a] == t;
        out[m++] = present ? j : t;
    }
    /* insertion sort, ascending */
    for (int32_t a = 1; a < m; ++a) {
        int64_t key = out[a];
        int32_t b = a - 1;
        while (b >= 0 && out[b] > key) { out[b + 1] = out[b]; --b; }
        out[b + 1] = key;
    }
}

double oracle_psi_node(const int32_t *offsets, const int32_t *cols, const double *phi, int32_t d,
                       int32_t ks, uint64_t seed, int32_t round, int32_t v) {
    int64_t deg = (int64_t)offsets[v + 1] - offsets[v];
    if (deg == 0) return 0.0;
    int64_t *sub = (int64_t *)malloc(sizeof(int64_t) * (size_t)(deg < ks ? deg : ks));
    int32_t m;
    if (deg <= ks) {
        m = (int32_t)deg;
        for (int32_t a = 0; a < m; ++a) sub[a] = a;
    } else {
        m = ks;
        oracle_psi_subset(deg, ks, seed, v, round, sub);
    }
    const double *pv = phi + (int64_t)v * d;
    double nv = canonical_dot(pv, pv, d);
    double sum = 0.0;
    for (int32_t a = 0; a < m; ++a) {
        int32_t u = cols[offsets[v] + sub[a]];
        const double *pu = phi + (int64_t)u * d;
        double nu = canonical_dot(pu, pu, d);
        double cs = 0.0;
        if (nv > 0.0 && nu > 0.0) cs = canonical_dot(pv, pu, d) / (sqrt(nv) * sqrt(nu));
        sum = sum + cs;
    }
    free(sub);
    return sum / (double)m;
}

typedef struct {
    int32_t enabled;
    double mu;
    int32_t ks;
    int32_t max_rounds;
    int32_t reactivate;
} oracle_feedback_params;

/* Psi for the evaluated nodes (active ones; every non-isolated node when   */
/* reactivating) and the next active set.  psi_out is NaN where not         */
/* evaluated.  Feedback disabled: every non-isolated node stays active.     */
/* Returns the size of the next active set.                                 */
int64_t oracle_feedback(const int32_t *offsets, const int32_t *cols, int32_t n, const double *phi,
                        int32_t d, const oracle_feedback_params *fp, uint64_t seed, int32_t round,
                        const uint8_t *active_in, uint8_t *active_out, double *psi_out) {
    int64_t count = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t deg = (int64_t)offsets[v + 1] - offsets[v];
        int evaluate = deg > 0 && (fp->reactivate || active_in[v]);
        double psi = NAN;
        if (evaluate) psi = oracle_psi_node(offsets, cols, phi, d, fp->ks, seed, round, v);
        if (psi_out) psi_out[v] = psi;
        uint8_t next;
        if (!fp->enabled) next = deg > 0;
        else next = evaluate && psi < fp->mu;
        active_out[v] = next;
        count += next;
    }
    return count;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: initialise V_a to the non-isolated nodes, then repeat        */
/* sample -> train -> feedback until V_a is empty or max_rounds is reached.  */
/* mode 0 = serial SGNS, mode 1 = synchronous minibatch of B positions,      */
/* mode 2 = the shared-negatives tile form, tiles of 128 - 2w centers in     */
/* corpus order with B shared negatives each and row averaging.              */
/* phi_in / phi_out are filled by the initialiser.  Per-round statistics:    */
/* stats[r*4 + 0] = |V_a^r|, +1 = tokens, +2 = loss, +3 = |V_a^{r+1}|.       */
/* Returns the number of rounds run.                                         */
/*                                                                           */
/* feedback_lag = 1 is the round-interleaved reading of Section 5.3: the    */
/* feedback that fixes V_a^{r+1} is computed on the embedding snapshot of   */
/* phi_in taken when round r's training starts (the table after round      */
/* r - 1), so sampling round r + 1 does not wait for round r's training.    */
/* feedback_lag = 0 is Algorithm 1 as printed (Psi after round r's         */
/* training).                                                                */
/* ------------------------------------------------------------------------ */
int32_t oracle_embed_lag(const int32_t *offsets, const int32_t *cols, int32_t n, int32_t L, int32_t wpr,
                         const oracle_train_params *tp_in, const oracle_feedback_params *fp,
                         int32_t mode, int64_t B, uint64_t seed, int32_t feedback_lag, double *phi_in,
                         double *phi_out, double *stats) {
    oracle_train_params tp = *tp_in;
    const int32_t d = tp.dim;
    oracle_init_tables(n, d, seed, phi_in, phi_out);
    uint8_t *active = (uint8_t *)malloc((size_t)n);
    uint8_t *next = (uint8_t *)malloc((size_t)n);
    int32_t *starts = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t *counts = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint64_t *thr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *alias = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *snap = feedback_lag ? (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * d) : NULL;
    int64_t n_live = 0;
    for (int32_t v = 0; v < n; ++v) {
        active[v] = offsets[v + 1] > offsets[v];
        n_live += active[v];
    }
    if (tp.lr_total_tokens <= 0) tp.lr_total_tokens = (int64_t)fp->max_rounds * wpr * n_live * L;
    if (tp.lr_total_tokens <= 0) tp.lr_total_tokens = 1;
    int64_t clock = 0;
    int32_t r = 0;
    for (; r < fp->max_rounds; ++r) {
        int32_t ns = 0;
        for (int32_t v = 0; v < n; ++v)
            if (active[v]) starts[ns++] = v;
        if (ns == 0) break;
        int64_t n_walks = (int64_t)ns * wpr;
        int32_t *walks = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_walks * L));
        oracle_walk(offsets, cols, n, starts, ns, L, wpr, seed, r, walks);
        oracle_counts(walks, n_walks * L, n, counts);
        uint64_t S;
        oracle_noise_table(counts, n, W, thr, alias, &S);
        if (snap) memcpy(snap, phi_in, sizeof(double) * (size_t)n * d);  /* the table as training starts */
        double loss;
        if (mode == 0)
            loss = oracle_sgns_serial(walks, n_walks, L, n, &tp, thr, alias, S, seed, r, clock,
                                      phi_in, phi_out);
        else if (mode == 1)
            loss = oracle_sgns_minibatch(walks, n_walks, L, n, &tp, B, thr, alias, S, seed, r,
                                         clock, phi_in, phi_out, NULL);
        else
            loss = oracle_sgns_tile(walks, n_walks, L, n, &tp, 128 - 2 * tp.window, (int32_t)B, 1,
                                    thr, alias, S, seed, r, clock, phi_in, phi_out, NULL);
        clock += n_walks * L;
        int64_t na = oracle_feedback(offsets, cols, n, snap ? snap : phi_in, d, fp, seed, r, active, next, NULL);
        if (stats) {
            stats[r * 4 + 0] = ns;
            stats[r * 4 + 1] = (double)(n_walks * L);
            stats[r * 4 + 2] = loss;
            stats[r * 4 + 3] = (double)na;
        }
        memcpy(active, next, (size_t)n);
        free(walks);
    }
    free(active); free(next); free(starts); free(counts); free(W); free(thr); free(alias); free(snap);
    return r;
}

int32_t oracle_embed(const int32_t *offsets, const int32_t *cols, int32_t n, int32_t L, int32_t wpr,
                     const oracle_train_params *tp_in, const oracle_feedback_params *fp,
                     int32_t mode, int64_t B, uint64_t seed, double *phi_in, double *phi_out,
                     double *stats) {
    return oracle_embed_lag(offsets, cols, n, L, wpr, tp_in, fp, mode, B, seed, 0, phi_in, phi_out, stats);
}

/* ------------------------------------------------------------------------ */
/* Link-prediction AUC (Section 6.4) by its definition: the fraction of      */
/* (positive, negative) score pairs ordered correctly, ties counting 1/2.    */
/* O(P * N).                                                                 */
/* ------------------------------------------------------------------------ */
double oracle_auc_pairs(const double *pos, int64_t P, const double *neg, int64_t N) {
    double wins = 0.0;
    for (int64_t a = 0; a < P; ++a)
        for (int64_t b = 0; b < N; ++b)
            wins += pos[a] > neg[b] ? 1.0 : (pos[a] == neg[b] ? 0.5 : 0.0);
    return wins / ((double)P * (double)N);
}

/* dot-product link scores phi[u] . phi[v] in binary64 */
void oracle_link_scores(const double *phi, int32_t d, const int32_t *pairs, int64_t m,
                        double *scores) {
    for (int64_t a = 0; a < m; ++a)
        scores[a] = dot(phi + (int64_t)pairs[2 * a] * d, phi + (int64_t)pairs[2 * a + 1] * d, d);
}

/* ------------------------------------------------------------------------ */
/* FaBC, frequency-aware bitmap compression of walk sequences (Section      */
/* 5.2.2).  Selection (Eq. 7, Eq. 8): nodes ordered by frequency p (count / */
/* total, ties to the smaller id); with c = 1/L + 1/32 and                  */
/* g(k) = 1 - F_k + k c, k grows from 0 while p(k+1) >= c + 0.1 g(k)         */
/* (reading: stop at the first node that fails, k <= k_max).  Returns k;     */
/* ids[0..k) receive the nodes and *F the covered fraction F_k.             */
/* ------------------------------------------------------------------------ */
int32_t oracle_fabc_select(const uint32_t *counts, int32_t n, int32_t L, int32_t k_max,
                           int32_t *ids, double *F) {
    uint64_t total = 0;
    for (int32_t v = 0; v < n; ++v) total += counts[v];
    const double c = 1.0 / (double)L + 1.0 / 32.0;
    double Fk = 0.0, g = 1.0;
    int32_t k = 0;
    while (k < k_max && total > 0) {
        /* the (k+1)-th most frequent node: largest count, smallest id, not yet taken */
        int32_t best = -1;
        for (int32_t v = 0; v < n; ++v) {
            int taken = 0;
            for (int32_t j = 0; j < k; ++j) taken |= ids[j] == v;
            if (taken) continue;
            if (best < 0 || counts[v] > counts[best]) best = v;
        }
        if (best < 0) break;
        const double p = (double)counts[best] / (double)total;
        if (!(p >= c + 0.1 * g)) break;
        ids[k] = best;
        k += 1;
        Fk += p;
        g = 1.0 - Fk + (double)k * c;
    }
    if (F) *F = Fk;
    return k;
}

/* Encoded layout for N sequences of L ids, B = ceil(L / 8) bytes per bitmap: */
/*   N*k int32   the k selected ids, stored with every sequence (Eq. 7 counts */
/*               4Nk bytes for them)                                          */
/*   N*k*B bytes bitmap (s, j) at (s*k + j)*B: bit i (byte i/8, bit i%8) set  */
/*               iff walks[s][i] == ids[j]                                    */
/*   int32 tail  ids of the positions no bitmap covers, in sequence order    */
/* Returns the encoded size in bytes; out must hold 4Nk + NkB + 4NL bytes.    */
int64_t oracle_fabc_encode(const int32_t *walks, int64_t N, int32_t L, const int32_t *ids,
                           int32_t k, uint8_t *out) {
    const int64_t B = (L + 7) / 8;
    uint8_t *idreg = out, *bm = out + 4 * N * k, *tail = bm + N * k * B;
    int64_t t = 0;
    for (int64_t s = 0; s < N; ++s) {
        for (int32_t j = 0; j < k; ++j) memcpy(idreg + 4 * (s * k + j), &ids[j], 4);
        for (int32_t j = 0; j < k; ++j) memset(bm + (s * k + j) * B, 0, (size_t)B);
        for (int32_t i = 0; i < L; ++i) {
            int32_t v = walks[s * L + i];
            int covered = 0;
            for (int32_t j = 0; j < k; ++j) {
                if (v == ids[j]) {
                    bm[(s * k + j) * B + i / 8] |= (uint8_t)(1u << (i % 8));
                    covered = 1;
                }
            }
            if (!covered) memcpy(tail + 4 * t++, &v, 4);
        }
    }
    return 4 * N * k + N * k * B + 4 * t;
}

/* Inverse of oracle_fabc_encode: a position covered by bitmap j takes the */
/* sequence's j-th id, the others take the tail ids in order.               */
void oracle_fabc_decode(const uint8_t *in, int64_t N, int32_t L, int32_t k, int32_t *walks) {
    const int64_t B = (L + 7) / 8;
    const uint8_t *idreg = in, *bm = in + 4 * N * k, *tail = bm + N * k * B;
    int64_t t = 0;
    for (int64_t s = 0; s < N; ++s) {
        for (int32_t i = 0; i < L; ++i) {
            int32_t v = 0;
            int found = 0;
            for (int32_t j = 0; j < k && !found; ++j) {
                if (bm[(s * k + j) * B + i / 8] >> (i % 8) & 1u) {
                    memcpy(&v, idreg + 4 * (s * k + j), 4);
                    found = 1;
                }
            }
            if (!found) memcpy(&v, tail + 4 * t++, 4);
            walks[s * L + i] = v;
        }
    }
}
