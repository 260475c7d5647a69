// Batching form: many independent graph-embedding jobs (Algorithm 1 each)
// trained together on one GPU.
//
// Every job keeps its own device buffers (active flags, start list, walks,
// counts, alias table and its scratch); a device table of jobs and a device
// array of per-job states (round, token clock, |V_a|, done flag, sums) let one
// fixed sequence of launches run one round of every unfinished job, each at
// its own round index, with no host synchronisation.  The rounds can
// therefore be captured in one CUDA graph.
//
// Work is mapped onto flat index spaces, each with a prefix over jobs:
//   tiles  - 4096-node pieces of one job (compaction, alias-table build);
//   slots  - n_j * wpr walk rows of job j (walk kernel);
//   nodes  - n_j nodes of job j (alias finish, Psi);
//   items  - max(1, n_j / rows_per_warp) training workers of job j; each
//            trains every c_j-th walk of its job, so at most c_j warps touch
//            one job's rows at once (the staleness bound of the single-graph
//            kernel, per job).
// A job's walks, alias table and Psi are those of the single-graph calls on
// the same seed (same Philox keys, same integer table); its training is the
// same half-warp Hogwild step.
#include <algorithm>
#include <cstring>
#include <fstream>
#include <sstream>
#include <new>
#include <string>
#include <vector>

#include "batch_core.cuh"
#include "feedback_core.cuh"
#include "noise_core.cuh"
#include "sgns_core.cuh"
#include "walk_core.cuh"

namespace felog {

bool csr_shape_ok(const felog_csr *g);
felog_status validate_csr_async(const felog_csr *g, const int32_t *starts, int32_t n_starts, int32_t *status,
                                cudaStream_t s);

// largest j with prefix[j] <= x (x < prefix[n_jobs])
__device__ __forceinline__ int find_job(const int64_t *__restrict__ prefix, int n_jobs, int64_t x) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// set-up: per-job state, tables, V_a^0, learning-rate horizon
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_b_init(BArgs a) {
    for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < a.n_nodes;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int j = find_job(a.node_prefix, a.n_jobs, x);
        const BJob &jb = a.jobs[j];
        if (jb.st->phase != 0) continue;
        const int32_t v = static_cast<int32_t>(x - a.node_prefix[j]);
        T *pin = static_cast<T *>(jb.phi_in) + static_cast<int64_t>(v) * jb.dim;
        T *pout = static_cast<T *>(jb.phi_out) + static_cast<int64_t>(v) * jb.dim;
        const float fd = static_cast<float>(jb.dim);
        for (int i4 = 0; i4 < jb.dim / 4; ++i4) {
            const u32x4 r = philox(jb.seed, static_cast<uint32_t>(i4), static_cast<uint32_t>(v), 0u, kStreamInit);
            const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float u = static_cast<float>(w[k] >> 8) * 5.9604644775390625e-08f;  // 2^-24
                const float val = __fdiv_rn(u - 0.5f, fd);
                if constexpr (std::is_same<T, float>::value) {
                    pin[i4 * 4 + k] = val;
                    pout[i4 * 4 + k] = 0.f;
                } else {
                    pin[i4 * 4 + k] = __float2bfloat16_rn(val);
                    pout[i4 * 4 + k] = __float2bfloat16_rn(0.f);
                }
            }
        }
        const uint8_t live = jb.offsets[v + 1] > jb.offsets[v];
        jb.active[0][v] = live;
        // one add per group of lanes on the same job
        const unsigned act = __activemask();
        const unsigned grp = __match_any_sync(act, j);
        const unsigned mine = grp & __ballot_sync(act, live);
        if (mine && (__ffs(mine) - 1) == static_cast<int>(threadIdx.x & 31))
            atomicAdd(reinterpret_cast<unsigned long long *>(&jb.st->n_live),
                      static_cast<unsigned long long>(__popc(mine)));
    }
}

__global__ void k_b_lr(BArgs a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n_jobs) return;
    BState &st = *a.jobs[j].st;
    if (st.phase != 0) return;
    int64_t T = a.lr_total_tokens;
    if (T <= 0) T = static_cast<int64_t>(a.max_rounds) * a.wpr * st.n_live * a.L;
    if (T <= 0) T = 1;
    st.T_total = T;
    st.inv_T = static_cast<float>(1.0 / static_cast<double>(T));
    st.done = st.n_live == 0 || a.max_rounds == 0;
    st.phase = 1;
}

// ---------------------------------------------------------------------------
// compaction of each job's V_a (tiles never span jobs)
// ---------------------------------------------------------------------------
// Every per-round kernel of the batch is a phase function over (block b of
// g blocks) with a thin kernel around it, so that one persistent kernel can
// run all phases of all rounds (k_b_persistent) with the same arithmetic.
__device__ __forceinline__ void ph_compact_count(const BArgs &a, int b, int g) {
    __shared__ int32_t warp_sum[kBWarps];
    for (int t = b; t < a.n_tiles; t += g) {
        const int j = a.tile_job[t];
        const BJob &jb = a.jobs[j];
        const BState &st = *a.jobs[j].st;
        int32_t c = 0;
        if (!st.done) {
            const int32_t start = a.tile_start[t];
            const uint8_t *act = jb.active[st.cur];
            for (int i = threadIdx.x; i < kBTile; i += kBThreads) {
                const int32_t v = start + i;
                if (v < jb.n) {
                    c += act[v] != 0;
                    jb.counts[v] = 0u;
                }
            }
        }
        c = __reduce_add_sync(kFull, c);
        if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t s = 0;
            for (int w = 0; w < kBWarps; ++w) s += warp_sum[w];
            a.tile_count[t] = s;
        }
        __syncthreads();
    }
}
__global__ void __launch_bounds__(kBThreads) k_b_compact_count(BArgs a) { ph_compact_count(a, blockIdx.x, gridDim.x); }

// one thread per job: exclusive scan of its tile counts, |V_a|, round reset
__device__ __forceinline__ void ph_compact_scan(const BArgs &a, int b, int g) {
    for (int j = b * blockDim.x + threadIdx.x; j < a.n_jobs; j += g * blockDim.x) {
        BState &st = *a.jobs[j].st;
        st.S = 0;
        st.cmax = 0;
        st.loss_acc = 0;
        st.n_next = 0;
        if (st.done) {
            st.n_active = 0;
            continue;
        }
        const BJob &jb = a.jobs[j];
        int32_t run = 0;
        for (int32_t t = jb.tile_base; t < jb.tile_base + jb.n_tiles; ++t) {
            const int32_t c = a.tile_count[t];
            a.tile_count[t] = run;
            run += c;
        }
        st.n_active = run;
        if (run == 0 || st.round >= a.max_rounds) {
            st.done = 1;
            st.n_active = 0;
        }
    }
}
__global__ void k_b_compact_scan(BArgs a) { ph_compact_scan(a, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void ph_compact_scatter(const BArgs &a, int b, int g) {
    __shared__ int32_t warp_tot[kBWarps];
    for (int t = b; t < a.n_tiles; t += g) {
        const int j = a.tile_job[t];
        const BJob &jb = a.jobs[j];
        const BState &st = *a.jobs[j].st;
        if (st.done) continue;  // uniform over the block
        const uint8_t *act = jb.active[st.cur];
        const int32_t my = a.tile_start[t] + threadIdx.x * kBTileItems;
        uint32_t bits = 0;
#pragma unroll
        for (int k = 0; k < kBTileItems; ++k) {
            const int32_t v = my + k;
            if (v < jb.n && act[v]) bits |= 1u << k;
        }
        const int32_t c = __popc(bits);
        int32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if ((threadIdx.x & 31) >= o) incl += y;
        }
        if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = incl;
        __syncthreads();
        int32_t warp_excl = 0;
        for (int w = 0; w < (threadIdx.x >> 5); ++w) warp_excl += warp_tot[w];
        int32_t pos = a.tile_count[t] + warp_excl + incl - c;
        while (bits) {
            const int k = __ffs(bits) - 1;
            bits &= bits - 1;
            jb.starts[pos++] = my + k;
        }
        __syncthreads();
    }
}
__global__ void __launch_bounds__(kBThreads) k_b_compact_scatter(BArgs a) {
    ph_compact_scatter(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// walks (counts fused); walk row o of job j = rep * |V_a| + i, as in felog_walk
// ---------------------------------------------------------------------------
template <bool VEC>
__device__ __forceinline__ void ph_walk(const BArgs &a, int b, int g) {
    for (int64_t x = static_cast<int64_t>(b) * blockDim.x + threadIdx.x; x < a.n_slots;
         x += static_cast<int64_t>(g) * blockDim.x) {
        const int j = find_job(a.slot_prefix, a.n_jobs, x);
        const BState &st = *a.jobs[j].st;
        const int64_t o = x - a.slot_prefix[j];
        if (st.done || o >= static_cast<int64_t>(st.n_active) * a.wpr) continue;
        const BJob &jb = a.jobs[j];
        const int32_t rep = static_cast<int32_t>(o / st.n_active);
        const int32_t i = static_cast<int32_t>(o - static_cast<int64_t>(rep) * st.n_active);
        const int32_t s = jb.starts[i];
        const uint32_t x2 = static_cast<uint32_t>(st.round) * static_cast<uint32_t>(a.wpr) + static_cast<uint32_t>(rep);
        walk_fill_row<true, VEC>(jb.offsets, jb.cols, jb.n, jb.nnz, s, a.L, jb.seed, x2, jb.walks + o * a.L,
                                 jb.counts);
    }
}
template <bool VEC>
__global__ void k_b_walk(BArgs a) { ph_walk<VEC>(a, blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// per-job alias tables of the round's corpus (same integers as felog_noise_table)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ph_noise_max(const BArgs &a, int b, int g) {
    for (int t = b; t < a.n_tiles; t += g) {
        const int j = a.tile_job[t];
        if (a.jobs[j].st->done) continue;
        const BJob &jb = a.jobs[j];
        uint32_t m = 0;
        const int32_t start = a.tile_start[t];
        for (int i = threadIdx.x; i < kBTile; i += kBThreads)
            if (start + i < jb.n) m = max(m, jb.counts[start + i]);
        m = __reduce_max_sync(kFull, m);
        if ((threadIdx.x & 31) == 0 && m) atomicMax(&a.jobs[j].st->cmax, m);
    }
}
__global__ void __launch_bounds__(kBThreads) k_b_noise_max(BArgs a) { ph_noise_max(a, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void ph_noise_weights(const BArgs &a, int b, int g) {
    for (int t = b; t < a.n_tiles; t += g) {
        const int j = a.tile_job[t];
        if (a.jobs[j].st->done) continue;
        const BJob &jb = a.jobs[j];
        const uint32_t cm = a.jobs[j].st->cmax;
        const double wmax = cm ? three_quarter_power(cm) : 1.0;
        unsigned long long local = 0;
        const int32_t start = a.tile_start[t];
        for (int i = threadIdx.x; i < kBTile; i += kBThreads) {
            const int32_t v = start + i;
            if (v >= jb.n) break;
            const uint32_t c = jb.counts[v];
            uint64_t w = 0;
            if (c) {
                const double q = floor(__dmul_rn(__ddiv_rn(three_quarter_power(c), wmax), 4294967296.0));
                w = static_cast<uint64_t>(q);
                if (w < 1) w = 1;
            }
            jb.W[v] = w;
            local += w;
        }
        for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
        if ((threadIdx.x & 31) == 0 && local) atomicAdd(&a.jobs[j].st->S, local);
    }
}
__global__ void __launch_bounds__(kBThreads) k_b_noise_weights(BArgs a) { ph_noise_weights(a, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void ph_noise_agg(const BArgs &a, int b, int gb) {
    __shared__ NoiseAgg part[kBThreads];
    for (int t = b; t < a.n_tiles; t += gb) {
        const int j = a.tile_job[t];
        if (a.jobs[j].st->done) continue;
        const BJob &jb = a.jobs[j];
        const uint64_t S = a.jobs[j].st->S;
        const int32_t my = a.tile_start[t] + threadIdx.x * kBTileItems;
        NoiseAgg g{0, 0, 0, 0};
        for (int k = 0; k < kBTileItems; ++k) {
            const int32_t v = my + k;
            if (v >= jb.n) break;
            bool light;
            uint64_t amt;
            classify(jb.W[v], static_cast<uint64_t>(jb.n), S, light, amt);
            if (light) { g.D += amt; g.nL += 1; }
            else { g.E += amt; g.nH += 1; }
        }
        part[threadIdx.x] = g;
        __syncthreads();
        if (threadIdx.x == 0) {
            NoiseAgg s{0, 0, 0, 0};
            for (int i = 0; i < kBThreads; ++i) {
                s.D += part[i].D; s.E += part[i].E; s.nL += part[i].nL; s.nH += part[i].nH;
            }
            a.tile_agg[t] = s;
        }
        __syncthreads();
    }
}
__global__ void __launch_bounds__(kBThreads) k_b_noise_agg(BArgs a) { ph_noise_agg(a, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void ph_noise_scan(const BArgs &a, int b, int g) {
    for (int j = b * blockDim.x + threadIdx.x; j < a.n_jobs; j += g * blockDim.x) {
        if (a.jobs[j].st->done) continue;
        const BJob &jb = a.jobs[j];
        NoiseAgg run{0, 0, 0, 0};
        for (int32_t t = jb.tile_base; t < jb.tile_base + jb.n_tiles; ++t) {
            const NoiseAgg x = a.tile_agg[t];
            a.tile_agg[t] = run;
            run.D += x.D; run.E += x.E; run.nL += x.nL; run.nH += x.nH;
        }
        a.jobs[j].st->total = run;
    }
}
__global__ void k_b_noise_scan(BArgs a) { ph_noise_scan(a, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void ph_noise_scatter(const BArgs &a, int b, int gb) {
    __shared__ NoiseAgg part[kBThreads];
    for (int t = b; t < a.n_tiles; t += gb) {
        const int j = a.tile_job[t];
        if (a.jobs[j].st->done) continue;
        const BJob &jb = a.jobs[j];
        const uint64_t S = a.jobs[j].st->S;
        const int32_t my = a.tile_start[t] + threadIdx.x * kBTileItems;
        NoiseAgg g{0, 0, 0, 0};
        for (int k = 0; k < kBTileItems; ++k) {
            const int32_t v = my + k;
            if (v >= jb.n) break;
            bool light;
            uint64_t amt;
            classify(jb.W[v], static_cast<uint64_t>(jb.n), S, light, amt);
            if (light) { g.D += amt; g.nL += 1; }
            else { g.E += amt; g.nH += 1; }
        }
        part[threadIdx.x] = g;
        __syncthreads();
        if (threadIdx.x == 0) {
            NoiseAgg run = a.tile_agg[t];
            for (int i = 0; i < kBThreads; ++i) {
                const NoiseAgg x = part[i];
                part[i] = run;
                run.D += x.D; run.E += x.E; run.nL += x.nL; run.nH += x.nH;
            }
        }
        __syncthreads();
        NoiseAgg run = part[threadIdx.x];
        for (int k = 0; k < kBTileItems; ++k) {
            const int32_t v = my + k;
            if (v >= jb.n) break;
            bool light;
            uint64_t amt;
            classify(jb.W[v], static_cast<uint64_t>(jb.n), S, light, amt);
            if (light) {
                jb.key[v] = run.D;
                jb.light_D[run.nL] = run.D;
                jb.rank[v] = run.nL;
                run.D += amt;
                run.nL += 1;
            } else {
                run.E += amt;
                jb.key[v] = run.E;
                jb.heavy_idx[run.nH] = v;
                jb.heavy_E[run.nH] = run.E;
                jb.rank[v] = run.nH;
                run.nH += 1;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBThreads) k_b_noise_scatter(BArgs a) { ph_noise_scatter(a, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void ph_noise_finish(const BArgs &a, int b, int g) {
    for (int64_t x = static_cast<int64_t>(b) * blockDim.x + threadIdx.x; x < a.n_nodes;
         x += static_cast<int64_t>(g) * blockDim.x) {
        const int j = find_job(a.node_prefix, a.n_jobs, x);
        const BState &st = *a.jobs[j].st;
        if (st.done) continue;
        const BJob &jb = a.jobs[j];
        const int32_t v = static_cast<int32_t>(x - a.node_prefix[j]);
        if (st.S == 0) {
            jb.thr[v] = 0;
            jb.alias[v] = v;
            continue;
        }
        alias_entry(v, jb.W[v], static_cast<uint64_t>(jb.n), st.S, jb.key[v], jb.rank[v], jb.light_D,
                    st.total.nL, jb.heavy_idx, jb.heavy_E, st.total.nH, st.total.D, jb.thr + v, jb.alias + v);
    }
}
__global__ void k_b_noise_finish(BArgs a) { ph_noise_finish(a, blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// SGNS over training items of the jobs whose dim is D
// ---------------------------------------------------------------------------
// FORM 2: two pairs per warp (a half warp each, 16 lanes per row); FORM 1:
// one pair per warp (32 lanes per row); FORM 4: FORM 2 with each step's rows
// copied to shared memory one step ahead (cp.async; used for rows of 256 or
// 512 bytes: float dim 64/128, bf16 dim 128).  Same estimator, different
// shapes.
template <int D, class T, int KFIX, int FORM, bool NC>
__device__ __forceinline__ void ph_sgns(const BArgs &a, int64_t item_lo, int64_t item_hi, int b, int g) {
    extern __shared__ __align__(16) int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int K = KFIX > 0 ? KFIX : a.K;
    int32_t *wk;
    char *rows = nullptr;
    if constexpr (FORM == 4) {
        char *base = reinterpret_cast<char *>(smem) +
                     wib * pf_bytes_per_warp(a.L, a.window, K, D, static_cast<int>(sizeof(T)));
        wk = reinterpret_cast<int32_t *>(base);
        rows = base + 4 * ((a.L + 2 * a.window * K + 3) & ~3);
    } else {
        wk = smem + wib * (a.L + 2 * a.window * K);
    }
    int32_t *negs = wk + a.L;
    const int64_t warps = static_cast<int64_t>(g) * kWarps;
    for (int64_t it = item_lo + static_cast<int64_t>(b) * kWarps + wib; it < item_hi; it += warps) {
        const int j = find_job(a.item_prefix, a.n_jobs, it);
        const BState &st = *a.jobs[j].st;
        if (st.done) continue;
        const BJob &jb = a.jobs[j];
        const int64_t c_j = a.item_prefix[j + 1] - a.item_prefix[j];
        const int64_t walks = static_cast<int64_t>(st.n_active) * a.wpr;
        TrainView<T> v{static_cast<T *>(jb.phi_in), static_cast<T *>(jb.phi_out), jb.thr, jb.alias,
                       static_cast<uint64_t>(jb.n), st.S, jb.seed, static_cast<uint32_t>(st.round), a.lr0,
                       st.inv_T, st.clock, a.window, a.K, a.L};
        long long loss_fx = 0;
        for (int64_t wl = it - a.item_prefix[j]; wl < walks; wl += c_j) {
            if constexpr (FORM == 1)
                loss_fx += fw_train_walk<D, T, 8, KFIX, NC>(v, jb.walks + wl * a.L, wl, wk, negs);
            else if constexpr (FORM == 4)
                loss_fx += hw_train_walk_pf<D, T, KFIX>(v, jb.walks + wl * a.L, wl, wk, negs, rows);
            else
                loss_fx += hw_train_walk<D, T, KFIX, false, NC>(v, jb.walks + wl * a.L, wl, wk, negs);
        }
        for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
        if (lane == 0 && loss_fx != 0)
            atomicAdd(&jb.st->loss_acc, static_cast<unsigned long long>(loss_fx));
    }
}
template <int D, class T, int KFIX, int FORM>
__global__ void __launch_bounds__(kSgnsThreads, 2) k_b_sgns(BArgs a, int64_t item_lo, int64_t item_hi) {
    ph_sgns<D, T, KFIX, FORM, true>(a, item_lo, item_hi, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// MINIBATCH (the deterministic form): one synchronous batch per round and
// job.  Token x of the flat space over the jobs of one dim (a job's span is
// its n * wpr walk slots times L) is center position p of walk slot wi; slots
// past the job's active walks are idle.  eta is that of the round's first
// position, formed in binary64 as felog_train does for a batch; the per-center
// and per-row routines are the single-graph kernels' own, so a job's round
// equals felog_train's minibatch form over the round with minibatch >= its
// tokens, bit for bit.
// ---------------------------------------------------------------------------
template <int D, class T, bool NC>
__device__ __forceinline__ void ph_mb_grad(const BArgs &a, int64_t tok_lo, int64_t tok_hi, int b, int g) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t *negs = smem + wib * (2 * a.window * a.K);
    const int64_t warps = static_cast<int64_t>(g) * kWarps;
    for (int64_t x = tok_lo + static_cast<int64_t>(b) * kWarps + wib; x < tok_hi; x += warps) {
        const int j = find_job(a.slot_prefix, a.n_jobs, x / a.L);
        const BState &st = *a.jobs[j].st;
        if (st.done) continue;
        const BJob &jb = a.jobs[j];
        const int64_t t = x - a.slot_prefix[j] * a.L;
        const int64_t wi = t / a.L;
        if (wi >= static_cast<int64_t>(st.n_active) * a.wpr) continue;
        const int p = static_cast<int>(t - wi * a.L);
        const double f = 1.0 - static_cast<double>(st.clock) / static_cast<double>(st.T_total);
        const float eta = static_cast<float>(static_cast<double>(a.lr0) * (f < 1e-4 ? 1e-4 : f));
        const MbView v{jb.thr, jb.alias, static_cast<uint64_t>(jb.n), st.S, jb.seed, static_cast<uint32_t>(st.round),
                       a.window, a.K, a.L};
        const MbState ms{jb.acc_in, jb.acc_out, jb.mark_in, jb.mark_out, nullptr, nullptr, nullptr};
        const float closs = mb_grad_center<D, T, 8, NC>(v, jb.walks + wi * a.L, wi, p, eta,
                                                    static_cast<const T *>(jb.phi_in),
                                                    static_cast<const T *>(jb.phi_out), ms, negs);
        long long loss_fx = __float2ll_rn(closs * kLossScaleF);
        for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
        if (lane == 0 && loss_fx != 0) atomicAdd(&jb.st->loss_acc, static_cast<unsigned long long>(loss_fx));
    }
}
template <int D, class T>
__global__ void __launch_bounds__(kSgnsThreads) k_b_mb_grad(BArgs a, int64_t tok_lo, int64_t tok_hi) {
    ph_mb_grad<D, T, true>(a, tok_lo, tok_hi, blockIdx.x, gridDim.x);
}

// every marked row of the jobs [node_lo, node_hi) of one dim, both tables
template <int D, class T>
__device__ __forceinline__ void ph_mb_apply(const BArgs &a, int64_t node_lo, int64_t node_hi, int b, int g) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(g) * (blockDim.x / 32);
    for (int64_t i = node_lo * 2 + static_cast<int64_t>(b) * (blockDim.x / 32) + (threadIdx.x >> 5);
         i < node_hi * 2; i += warps) {
        const int64_t x = i >> 1;
        const bool is_in = (i & 1) == 0;
        const int j = find_job(a.node_prefix, a.n_jobs, x);
        const BState &st = *a.jobs[j].st;
        if (st.done) continue;
        const BJob &jb = a.jobs[j];
        const int32_t r = static_cast<int32_t>(x - a.node_prefix[j]);
        uint32_t *mark = is_in ? jb.mark_in : jb.mark_out;
        if (!mark[r]) continue;
        mb_apply_row<D, T>(static_cast<T *>(is_in ? jb.phi_in : jb.phi_out), is_in ? jb.acc_in : jb.acc_out, mark, r,
                           is_in, jb.seed, static_cast<uint32_t>(st.round) << 20, lane);
    }
}
template <int D, class T>
__global__ void __launch_bounds__(256) k_b_mb_apply(BArgs a, int64_t node_lo, int64_t node_hi) {
    ph_mb_apply<D, T>(a, node_lo, node_hi, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Psi and V_a^{r+1} (same values as felog_feedback)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void ph_feedback(const BArgs &a, int b, int g) {
    __shared__ PsiScratch scratch[kBWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    PsiScratch &w = scratch[wib];
    const int GN = psi_group_size(a.ks);
    const int64_t warps = static_cast<int64_t>(g) * kBWarps;
    // groups of GN consecutive flat nodes (they may span jobs): totals node
    // by node, then cosines and means lane-parallel, as felog_feedback does
    for (int64_t base = (static_cast<int64_t>(b) * kBWarps + wib) * GN; base < a.n_nodes; base += warps * GN) {
        const int cnt = static_cast<int>(a.n_nodes - base < GN ? a.n_nodes - base : GN);
        for (int i = 0; i < cnt; ++i) {
            const int64_t x = base + i;
            const int j = find_job(a.node_prefix, a.n_jobs, x);
            const BState &st = *a.jobs[j].st;
            const BJob &jb = a.jobs[j];
            const int32_t v = static_cast<int32_t>(x - a.node_prefix[j]);
            const int32_t lo = jb.offsets[v], hi = jb.offsets[v + 1];
            const int64_t deg = lo >= 0 && hi <= jb.nnz ? static_cast<int64_t>(hi) - lo : 0;
            const bool evaluate = !st.done && deg > 0 && (a.reactivate || jb.active[st.cur][v]);
            if (evaluate)
                psi_node_totals<T>(jb.cols, static_cast<const T *>(jb.phi_in), jb.n, jb.dim, a.ks, jb.seed,
                                   static_cast<uint32_t>(st.round), v, lo, deg, w, i);
            else if (lane == 0) w.m[i] = 0;
        }
        const double psi = psi_group_finish(w, cnt, a.ks);
        if (lane < cnt) {
            const int64_t x = base + lane;
            const int j = find_job(a.node_prefix, a.n_jobs, x);
            const BState &st = *a.jobs[j].st;
            if (!st.done) {
                const BJob &jb = a.jobs[j];
                const int32_t v = static_cast<int32_t>(x - a.node_prefix[j]);
                const int32_t lo = jb.offsets[v], hi = jb.offsets[v + 1];
                const bool live = lo >= 0 && hi <= jb.nnz && hi > lo;
                const bool evaluated = w.m[lane] > 0;
                const uint8_t next = a.enabled ? static_cast<uint8_t>(evaluated && psi < a.mu)
                                               : static_cast<uint8_t>(live);
                jb.active[st.cur ^ 1][v] = next;
                if (next) atomicAdd(&jb.st->n_next, 1);
            }
        }
        __syncwarp();
    }
}
template <class T>
__global__ void __launch_bounds__(kBThreads) k_b_feedback(BArgs a) { ph_feedback<T>(a, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void ph_round_end(const BArgs &a, int b, int g) {
    for (int j = b * blockDim.x + threadIdx.x; j < a.n_jobs; j += g * blockDim.x) {
        BState &st = *a.jobs[j].st;
        if (st.done) continue;
        const int r = st.round;
        const BJob &jb = a.jobs[j];
        jb.rec_n_active[r] = st.n_active;
        jb.rec_n_next[r] = st.n_next;
        jb.rec_loss[r] = static_cast<double>(static_cast<long long>(st.loss_acc)) / kLossScale;
        st.clock += static_cast<int64_t>(st.n_active) * a.wpr * a.L;
        st.round = r + 1;
        st.cur ^= 1;
        if (st.n_next == 0 || st.round >= a.max_rounds) st.done = 1;
    }
}
__global__ void k_b_round_end(BArgs a) { ph_round_end(a, blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// One persistent kernel for a whole run: every phase of every round of every
// job, the phases separated by a grid-wide barrier.  The grid is launched
// cooperatively (all blocks resident), so a barrier only waits for blocks
// that are running.  Each wait is still bounded: it gives up once the
// nanosecond global timer has advanced by the run's budget (60 s unless the
// caller sets another), or after kGridPollLimit polls about a microsecond
// apart, whichever comes first; it then sets the error word (and the tag of
// the barrier) and every block returns at its next barrier.  Phase data
// written by other blocks is read after the barrier's release/acquire
// fences; the alias table, rebuilt every round, is read through L2 rather
// than the read-only cache (NC = false), which a kernel only refreshes at
// its launch.
// ---------------------------------------------------------------------------
constexpr unsigned kGridPollLimit = 1u << 31;
constexpr double kDefaultGridWaitS = 60.0;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// `expected` arrivals release the barrier (gridDim.x in the persistent
// kernel); returns false once any wait of this barrier has run out.
__device__ __forceinline__ bool grid_sync(GridBarrier *bar, unsigned expected, unsigned long long budget_ns,
                                          int tag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &bar->gen;
        volatile int *verr = &bar->error;
        const unsigned g0 = *vgen;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == expected - 1) {
            bar->count = 0;  // every block has arrived: reset, then release them
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned it = 0;
            while (*vgen == g0 && !*verr) {
                if (++it > kGridPollLimit || global_ns() - t0 > budget_ns) {
                    if (atomicCAS(&bar->error, 0, 1) == 0) bar->where = tag;
                    break;
                }
                __nanosleep(1000);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *reinterpret_cast<volatile int *>(&bar->error) == 0;
}

template <class T, int KFIX, bool MB>
__global__ void __launch_bounds__(kBThreads, 2)
    k_b_persistent(BArgs a, GridBarrier *bar, unsigned long long budget_ns) {
    const int b = blockIdx.x, g = gridDim.x;
    int tag = 0;
    auto sync = [&]() { return grid_sync(bar, gridDim.x, budget_ns, tag++); };
    for (int r = 0; r < a.max_rounds; ++r) {
        tag = 16 * r;
        ph_compact_count(a, b, g);
        if (!sync()) return;
        ph_compact_scan(a, b, g);
        if (!sync()) return;
        ph_compact_scatter(a, b, g);
        if (!sync()) return;
        if (a.L % 4 == 0) ph_walk<true>(a, b, g);
        else ph_walk<false>(a, b, g);
        if (!sync()) return;
        ph_noise_max(a, b, g);
        if (!sync()) return;
        ph_noise_weights(a, b, g);
        if (!sync()) return;
        ph_noise_agg(a, b, g);
        if (!sync()) return;
        ph_noise_scan(a, b, g);
        if (!sync()) return;
        ph_noise_scatter(a, b, g);
        if (!sync()) return;
        ph_noise_finish(a, b, g);
        if (!sync()) return;
        if constexpr (MB) {
            ph_mb_grad<32, T, false>(a, a.tok_lo[0], a.tok_hi[0], b, g);
            ph_mb_grad<64, T, false>(a, a.tok_lo[1], a.tok_hi[1], b, g);
            ph_mb_grad<128, T, false>(a, a.tok_lo[2], a.tok_hi[2], b, g);
            if (!sync()) return;
            ph_mb_apply<32, T>(a, a.node_lo[0], a.node_hi[0], b, g);
            ph_mb_apply<64, T>(a, a.node_lo[1], a.node_hi[1], b, g);
            ph_mb_apply<128, T>(a, a.node_lo[2], a.node_hi[2], b, g);
        } else {
            ph_sgns<32, T, KFIX, 2, false>(a, a.item_lo[0], a.item_hi[0], b, g);
            ph_sgns<64, T, KFIX, 2, false>(a, a.item_lo[1], a.item_hi[1], b, g);
            ph_sgns<128, T, KFIX, 2, false>(a, a.item_lo[2], a.item_hi[2], b, g);
        }
        if (!sync()) return;
        ph_feedback<T>(a, b, g);
        if (!sync()) return;
        ph_round_end(a, b, g);
        if (!sync()) return;
    }
}

// The persistent kernel's barrier on its own: `passes` barriers of a
// resident grid that expects `phantom` arrivals more than it has blocks.
// With phantom = 0 every barrier releases; with phantom > 0 the first one
// never does, and every wait runs out after budget_ns.
__global__ void __launch_bounds__(kBThreads) k_grid_barrier_check(GridBarrier *bar, unsigned phantom, int passes,
                                                                   unsigned long long budget_ns) {
    for (int k = 0; k < passes; ++k)
        if (!grid_sync(bar, gridDim.x + phantom, budget_ns, k)) return;
}

// gathers every job's state and round records into contiguous arrays
__global__ void k_b_gather(BArgs a, BState *st_out, int32_t *rna, int32_t *rnn, double *rl) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n_jobs) return;
    const BJob &jb = a.jobs[j];
    st_out[j] = *jb.st;
    for (int r = 0; r < a.max_rounds; ++r) {
        rna[static_cast<int64_t>(r) * a.n_jobs + j] = jb.rec_n_active[r];
        rnn[static_cast<int64_t>(r) * a.n_jobs + j] = jb.rec_n_next[r];
        rl[static_cast<int64_t>(r) * a.n_jobs + j] = jb.rec_loss[r];
    }
}

// ---------------------------------------------------------------------------
// host side: job memory, plans (a membership of jobs), init and step
// ---------------------------------------------------------------------------
size_t job_work_bytes(int32_t n, int32_t dim, const BParams &p) {
    const size_t nn = n > 0 ? static_cast<size_t>(n) : 1;
    const size_t R = static_cast<size_t>(std::max(p.max_rounds, 1));
    size_t b = 0;
    auto add = [&](size_t x) { b += align_up(x, 256); };
    if (p.mode == FELOG_SGNS_MINIBATCH) {
        add(8 * nn * dim);  // acc_in
        add(8 * nn * dim);  // acc_out
        add(4 * nn);        // mark_in
        add(4 * nn);        // mark_out
    }
    add(sizeof(BState));
    add(4 * R);                                            // rec_n_active
    add(4 * R);                                            // rec_n_next
    add(8 * R);                                            // rec_loss
    add(nn);                                               // active[0]
    add(nn);                                               // active[1]
    add(4 * nn);                                           // starts
    add(4 * nn * static_cast<size_t>(p.wpr) * p.L);        // walks
    add(4 * nn);                                           // counts
    add(8 * nn);                                           // thr
    add(4 * nn);                                           // alias
    add(8 * nn);                                           // W
    add(16 * nn);                                          // key
    add(4 * nn);                                           // rank
    add(16 * nn);                                          // light_D
    add(4 * nn);                                           // heavy_idx
    add(16 * nn);                                          // heavy_E
    return b;
}

void job_carve(BJob &jb, void *mem, int32_t n, const BParams &p) {
    const size_t nn = n > 0 ? static_cast<size_t>(n) : 1;
    const size_t R = static_cast<size_t>(std::max(p.max_rounds, 1));
    char *q = static_cast<char *>(mem);
    auto take = [&](size_t bytes) { char *r = q; q += align_up(bytes, 256); return r; };
    if (p.mode == FELOG_SGNS_MINIBATCH) {
        jb.acc_in = reinterpret_cast<long long *>(take(8 * nn * jb.dim));
        jb.acc_out = reinterpret_cast<long long *>(take(8 * nn * jb.dim));
        jb.mark_in = reinterpret_cast<uint32_t *>(take(4 * nn));
        jb.mark_out = reinterpret_cast<uint32_t *>(take(4 * nn));
    }
    jb.st = reinterpret_cast<BState *>(take(sizeof(BState)));
    jb.rec_n_active = reinterpret_cast<int32_t *>(take(4 * R));
    jb.rec_n_next = reinterpret_cast<int32_t *>(take(4 * R));
    jb.rec_loss = reinterpret_cast<double *>(take(8 * R));
    jb.active[0] = reinterpret_cast<uint8_t *>(take(nn));
    jb.active[1] = reinterpret_cast<uint8_t *>(take(nn));
    jb.starts = reinterpret_cast<int32_t *>(take(4 * nn));
    jb.walks = reinterpret_cast<int32_t *>(take(4 * nn * p.wpr * p.L));
    jb.counts = reinterpret_cast<uint32_t *>(take(4 * nn));
    jb.thr = reinterpret_cast<uint64_t *>(take(8 * nn));
    jb.alias = reinterpret_cast<int32_t *>(take(4 * nn));
    jb.W = reinterpret_cast<uint64_t *>(take(8 * nn));
    jb.key = reinterpret_cast<u128 *>(take(16 * nn));
    jb.rank = reinterpret_cast<int32_t *>(take(4 * nn));
    jb.light_D = reinterpret_cast<u128 *>(take(16 * nn));
    jb.heavy_idx = reinterpret_cast<int32_t *>(take(4 * nn));
    jb.heavy_E = reinterpret_cast<u128 *>(take(16 * nn));
}

// state and records of a job must start at zero (phase 0 = not initialised)
felog_status job_clear_state(const BJob &jb, const BParams &p, cudaStream_t s) {
    const size_t R = static_cast<size_t>(std::max(p.max_rounds, 1));
    const size_t bytes = align_up(sizeof(BState), 256) + 2 * align_up(4 * R, 256) + 8 * R;
    if (p.mode == FELOG_SGNS_MINIBATCH) {
        // the accumulators and marks lie in front of the state, contiguous
        const size_t nn = jb.n > 0 ? static_cast<size_t>(jb.n) : 1;
        const size_t mb = 2 * align_up(8 * nn * jb.dim, 256) + 2 * align_up(4 * nn, 256);
        felog_status st = record_cuda_error(cudaMemsetAsync(jb.acc_in, 0, mb, s), "job accumulators");
        if (st) return st;
    }
    return record_cuda_error(cudaMemsetAsync(jb.st, 0, bytes, s), "job state");
}

felog_status plan_build(BatchPlan &plan, const std::vector<BJob> &jobs_in, const BParams &p, cudaStream_t s) {
    plan = BatchPlan{};
    const int32_t n_jobs = static_cast<int32_t>(jobs_in.size());
    if (n_jobs == 0) return FELOG_OK;
    std::vector<BJob> jobs = jobs_in;
    std::vector<int64_t> slot_prefix(n_jobs + 1, 0), node_prefix(n_jobs + 1, 0), item_prefix(n_jobs + 1, 0);
    std::vector<int32_t> tile_job, tile_start;
    plan.dims.resize(n_jobs);
    int32_t tile = 0;
    for (int32_t i = 0; i < n_jobs; ++i) {
        BJob &jb = jobs[i];
        plan.dims[i] = jb.dim;
        slot_prefix[i + 1] = slot_prefix[i] + static_cast<int64_t>(jb.n) * p.wpr;
        node_prefix[i + 1] = node_prefix[i] + jb.n;
        item_prefix[i + 1] = item_prefix[i] + std::max<int64_t>(1, jb.n / p.rows_per_warp);
        const int32_t nt = std::max(1, ceil_div(std::max(jb.n, 1), kBTile));
        jb.tile_base = tile;
        jb.n_tiles = nt;
        for (int32_t t = 0; t < nt; ++t) {
            tile_job.push_back(i);
            tile_start.push_back(t * kBTile);
        }
        tile += nt;
    }
    const int32_t R = std::max(p.max_rounds, 1);
    size_t off = 0;
    auto slot = [&](size_t bytes) { size_t o = off; off += align_up(bytes, 256); return o; };
    const size_t o_jobs = slot(sizeof(BJob) * n_jobs);
    const size_t o_sp = slot(sizeof(int64_t) * (n_jobs + 1));
    const size_t o_np = slot(sizeof(int64_t) * (n_jobs + 1));
    const size_t o_ip = slot(sizeof(int64_t) * (n_jobs + 1));
    const size_t o_tj = slot(sizeof(int32_t) * tile);
    const size_t o_ts = slot(sizeof(int32_t) * tile);
    const size_t o_tc = slot(sizeof(int32_t) * tile);
    const size_t o_ta = slot(sizeof(NoiseAgg) * tile);
    plan.o_gst = slot(sizeof(BState) * n_jobs);
    plan.o_gna = slot(sizeof(int32_t) * R * n_jobs);
    plan.o_gnn = slot(sizeof(int32_t) * R * n_jobs);
    plan.o_gl = slot(sizeof(double) * R * n_jobs);
    plan.o_bar = slot(sizeof(GridBarrier));
    felog_status st = record_cuda_error(cudaMallocAsync(&plan.mem, off, s), "plan");
    if (st) return st;
    plan.bytes = off;
    char *base = static_cast<char *>(plan.mem);
    st = record_cuda_error(cudaMemsetAsync(base + plan.o_bar, 0, sizeof(GridBarrier), s), "plan");
    if (!st)
        st = record_cuda_error(cudaMemcpyAsync(base + o_jobs, jobs.data(), sizeof(BJob) * n_jobs, cudaMemcpyHostToDevice, s), "plan");
    if (!st) st = record_cuda_error(cudaMemcpyAsync(base + o_sp, slot_prefix.data(), sizeof(int64_t) * (n_jobs + 1), cudaMemcpyHostToDevice, s), "plan");
    if (!st) st = record_cuda_error(cudaMemcpyAsync(base + o_np, node_prefix.data(), sizeof(int64_t) * (n_jobs + 1), cudaMemcpyHostToDevice, s), "plan");
    if (!st) st = record_cuda_error(cudaMemcpyAsync(base + o_ip, item_prefix.data(), sizeof(int64_t) * (n_jobs + 1), cudaMemcpyHostToDevice, s), "plan");
    if (!st) st = record_cuda_error(cudaMemcpyAsync(base + o_tj, tile_job.data(), sizeof(int32_t) * tile, cudaMemcpyHostToDevice, s), "plan");
    if (!st) st = record_cuda_error(cudaMemcpyAsync(base + o_ts, tile_start.data(), sizeof(int32_t) * tile, cudaMemcpyHostToDevice, s), "plan");
    // pageable sources: the copies above have consumed them once the stream reaches this point
    if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "plan");
    if (st) {
        cudaFreeAsync(plan.mem, s);
        plan.mem = nullptr;
        return st;
    }
    plan.n_jobs = n_jobs;
    plan.item_prefix = item_prefix;
    plan.slot_prefix = slot_prefix;
    plan.node_prefix = node_prefix;
    plan.jobs = jobs;
    BArgs &a = plan.args;
    a.jobs = reinterpret_cast<const BJob *>(base + o_jobs);
    a.n_jobs = n_jobs;
    a.slot_prefix = reinterpret_cast<const int64_t *>(base + o_sp);
    a.node_prefix = reinterpret_cast<const int64_t *>(base + o_np);
    a.item_prefix = reinterpret_cast<const int64_t *>(base + o_ip);
    a.tile_job = reinterpret_cast<const int32_t *>(base + o_tj);
    a.tile_start = reinterpret_cast<const int32_t *>(base + o_ts);
    a.tile_count = reinterpret_cast<int32_t *>(base + o_tc);
    a.tile_agg = reinterpret_cast<NoiseAgg *>(base + o_ta);
    a.n_tiles = tile;
    a.n_slots = slot_prefix[n_jobs];
    a.n_nodes = node_prefix[n_jobs];
    a.L = p.L;
    a.wpr = p.wpr;
    a.window = p.window;
    a.K = p.K;
    a.max_rounds = p.max_rounds;
    a.ks = p.ks;
    a.enabled = p.enabled;
    a.reactivate = p.reactivate;
    a.precision = p.precision;
    a.mu = p.mu;
    a.lr0 = p.lr0;
    a.lr_total_tokens = p.lr_total_tokens;
    for (int k = 0; k < 3; ++k) {
        const int32_t d = 32 << k;
        int32_t j0 = 0;
        while (j0 < n_jobs && plan.dims[j0] < d) ++j0;
        int32_t j1 = j0;
        while (j1 < n_jobs && plan.dims[j1] == d) ++j1;
        a.item_lo[k] = item_prefix[j0];
        a.item_hi[k] = item_prefix[j1];
        a.tok_lo[k] = slot_prefix[j0] * p.L;
        a.tok_hi[k] = slot_prefix[j1] * p.L;
        a.node_lo[k] = node_prefix[j0];
        a.node_hi[k] = node_prefix[j1];
    }
    return FELOG_OK;
}

void plan_release(BatchPlan &plan, cudaStream_t s) {
    if (plan.mem) cudaFreeAsync(plan.mem, s);
    plan = BatchPlan{};
}

namespace {

int grid_for(int64_t work, int block, int per_sm) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((work + block - 1) / block,
                                                                    static_cast<int64_t>(per_sm) * sm_count())));
}

template <int D, class T>
void launch_b_sgns(const BatchPlan &plan, const BParams &p, const HostTuning &t, int64_t lo, int64_t hi,
                   cudaStream_t s) {
    if (hi <= lo) return;
    // form 4 for rows of 256 bytes or more (bf16 dim 128, float dim 64 and 128), else form 2: on the
    // 512-graph mix the dim-64 bf16 jobs (128-byte rows) trained no faster prefetched
    // (2.40e8 against 2.44e8 tokens/s for the whole batch)
    constexpr bool kPfHere = kPfSupported<D, T> && D * sizeof(T) >= 256;
    const int form = t.sgns_form == 1 ? 1 : (t.sgns_form == 4 && kPfHere ? 4 : 2);
    size_t smem = sizeof(int32_t) * kWarps * (p.window * 2 * p.K + p.L);
    void (*kern)(BArgs, int64_t, int64_t) = form == 1 ? (p.K == 5 ? k_b_sgns<D, T, 5, 1> : k_b_sgns<D, T, 0, 1>)
                                                      : (p.K == 5 ? k_b_sgns<D, T, 5, 2> : k_b_sgns<D, T, 0, 2>);
    if constexpr (kPfHere) {
        const size_t pf_smem =
            static_cast<size_t>(kWarps) * pf_bytes_per_warp(p.L, p.window, p.K, D, static_cast<int>(sizeof(T)));
        if (form == 4 && pf_smem <= 200 * 1024) {  // longer walks than fit run shape 2
            smem = pf_smem;
            kern = p.K == 5 ? k_b_sgns<D, T, 5, 4> : k_b_sgns<D, T, 0, 4>;
        }
    }
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    const int64_t want = (hi - lo + kWarps - 1) / kWarps;
    const int blocks = static_cast<int>(
        std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(t.sgns_blocks_per_sm) * sm_count())));
    kern<<<blocks, kSgnsThreads, smem, s>>>(plan.args, lo, hi);
}

template <int D, class T>
void launch_b_mb(const BatchPlan &plan, const BParams &p, int32_t j0, int32_t j1, cudaStream_t s) {
    const int64_t tok_lo = plan.slot_prefix[j0] * p.L, tok_hi = plan.slot_prefix[j1] * p.L;
    if (tok_hi <= tok_lo) return;
    const size_t smem = sizeof(int32_t) * kWarps * (2 * p.window * p.K);
    k_b_mb_grad<D, T><<<grid_for((tok_hi - tok_lo + kWarps - 1) / kWarps, 1, 16), kSgnsThreads, smem, s>>>(
        plan.args, tok_lo, tok_hi);
    const int64_t node_lo = plan.node_prefix[j0], node_hi = plan.node_prefix[j1];
    k_b_mb_apply<D, T><<<grid_for((2 * (node_hi - node_lo) + 7) / 8, 1, 16), 256, 0, s>>>(plan.args, node_lo,
                                                                                          node_hi);
}

template <class T>
void launch_mb_all(const BatchPlan &plan, const BParams &p, cudaStream_t s) {
    int32_t j = 0;
    while (j < plan.n_jobs) {
        int32_t k = j;
        while (k < plan.n_jobs && plan.dims[k] == plan.dims[j]) ++k;
        switch (plan.dims[j]) {
            case 32: launch_b_mb<32, T>(plan, p, j, k, s); break;
            case 64: launch_b_mb<64, T>(plan, p, j, k, s); break;
            case 128: launch_b_mb<128, T>(plan, p, j, k, s); break;
        }
        j = k;
    }
}

template <class T>
void launch_sgns_all(const BatchPlan &plan, const BParams &p, const HostTuning &t, cudaStream_t s) {
    // items are ordered by job and jobs by dim: one launch per dim range
    int32_t j = 0;
    while (j < plan.n_jobs) {
        int32_t k = j;
        while (k < plan.n_jobs && plan.dims[k] == plan.dims[j]) ++k;
        const int64_t lo = plan.item_prefix[j], hi = plan.item_prefix[k];
        switch (plan.dims[j]) {
            case 32: launch_b_sgns<32, T>(plan, p, t, lo, hi, s); break;
            case 64: launch_b_sgns<64, T>(plan, p, t, lo, hi, s); break;
            case 128: launch_b_sgns<128, T>(plan, p, t, lo, hi, s); break;
        }
        j = k;
    }
}

}  // namespace

// tables and V_a^0 of the plan's jobs still in phase 0 (the caller clears
// their state first)
felog_status plan_init_jobs(const BatchPlan &plan, const BParams &p, cudaStream_t s) {
    if (plan.n_jobs == 0) return FELOG_OK;
    const BArgs &a = plan.args;
    if (p.precision == FELOG_FP32) k_b_init<float><<<grid_for(a.n_nodes, 256, 16), 256, 0, s>>>(a);
    else k_b_init<__nv_bfloat16><<<grid_for(a.n_nodes, 256, 16), 256, 0, s>>>(a);
    k_b_lr<<<ceil_div(plan.n_jobs, 256), 256, 0, s>>>(a);
    return check_launch("felog init jobs");
}

// phases: bit 0 compaction, 1 walk, 2 noise, 3 sgns, 4 feedback, 5 round end
felog_status plan_step(const BatchPlan &plan, const BParams &p, const HostTuning &t, cudaStream_t s,
                       unsigned phases) {
    if (plan.n_jobs == 0) return FELOG_OK;
    const BArgs &a = plan.args;
    const int jg = ceil_div(plan.n_jobs, 256);
    if (phases & 1) {
        k_b_compact_count<<<a.n_tiles, kBThreads, 0, s>>>(a);
        k_b_compact_scan<<<jg, 256, 0, s>>>(a);
        k_b_compact_scatter<<<a.n_tiles, kBThreads, 0, s>>>(a);
    }
    if (phases & 2) {
        const int wb = t.walk_block;
        if (a.L % 4 == 0) k_b_walk<true><<<grid_for(a.n_slots, wb, 2048 / wb), wb, 0, s>>>(a);
        else k_b_walk<false><<<grid_for(a.n_slots, wb, 2048 / wb), wb, 0, s>>>(a);
    }
    if (phases & 4) {
        k_b_noise_max<<<a.n_tiles, kBThreads, 0, s>>>(a);
        k_b_noise_weights<<<a.n_tiles, kBThreads, 0, s>>>(a);
        k_b_noise_agg<<<a.n_tiles, kBThreads, 0, s>>>(a);
        k_b_noise_scan<<<jg, 256, 0, s>>>(a);
        k_b_noise_scatter<<<a.n_tiles, kBThreads, 0, s>>>(a);
        k_b_noise_finish<<<grid_for(a.n_nodes, 256, 8), 256, 0, s>>>(a);
    }
    if (phases & 8) {
        if (p.mode == FELOG_SGNS_MINIBATCH) {
            if (p.precision == FELOG_FP32) launch_mb_all<float>(plan, p, s);
            else launch_mb_all<__nv_bfloat16>(plan, p, s);
        } else if (p.precision == FELOG_FP32) {
            launch_sgns_all<float>(plan, p, t, s);
        } else {
            launch_sgns_all<__nv_bfloat16>(plan, p, t, s);
        }
    }
    if (phases & 16) {
        const int grid = static_cast<int>(std::max<int64_t>(
            1, std::min<int64_t>((a.n_nodes + kBWarps * psi_group_size(p.ks) - 1) / (kBWarps * psi_group_size(p.ks)),
                                 static_cast<int64_t>(sm_count()) * t.feedback_blocks_per_sm)));
        if (p.precision == FELOG_FP32) k_b_feedback<float><<<grid, kBThreads, 0, s>>>(a);
        else k_b_feedback<__nv_bfloat16><<<grid, kBThreads, 0, s>>>(a);
    }
    if (phases & 32) k_b_round_end<<<jg, 256, 0, s>>>(a);
    return check_launch("felog batch step");
}

// copies states and records of the plan's jobs to the host (synchronises s)
felog_status plan_gather(const BatchPlan &plan, const BParams &p, cudaStream_t s, std::vector<BState> &sts,
                         std::vector<int32_t> &rna, std::vector<int32_t> &rnn, std::vector<double> &rl) {
    const int n = plan.n_jobs;
    const size_t R = static_cast<size_t>(std::max(p.max_rounds, 1));
    sts.resize(n);
    rna.assign(R * n, 0);
    rnn.assign(R * n, 0);
    rl.assign(R * n, 0.0);
    if (n == 0) return FELOG_OK;
    char *base = static_cast<char *>(plan.mem);
    k_b_gather<<<ceil_div(n, 256), 256, 0, s>>>(plan.args, reinterpret_cast<BState *>(base + plan.o_gst),
                                                reinterpret_cast<int32_t *>(base + plan.o_gna),
                                                reinterpret_cast<int32_t *>(base + plan.o_gnn),
                                                reinterpret_cast<double *>(base + plan.o_gl));
    felog_status st = check_launch("gather");
    if (!st) st = record_cuda_error(cudaMemcpyAsync(sts.data(), base + plan.o_gst, sizeof(BState) * n, cudaMemcpyDeviceToHost, s), "gather");
    if (!st && p.max_rounds > 0) {
        st = record_cuda_error(cudaMemcpyAsync(rna.data(), base + plan.o_gna, 4 * R * n, cudaMemcpyDeviceToHost, s), "gather");
        if (!st) st = record_cuda_error(cudaMemcpyAsync(rnn.data(), base + plan.o_gnn, 4 * R * n, cudaMemcpyDeviceToHost, s), "gather");
        if (!st) st = record_cuda_error(cudaMemcpyAsync(rl.data(), base + plan.o_gl, 8 * R * n, cudaMemcpyDeviceToHost, s), "gather");
    }
    if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "gather");
    return st;
}

BParams make_params(const felog_walk_params *wp, const felog_train_params *tp, const felog_feedback_params *fp) {
    BParams p;
    p.L = wp->length;
    p.wpr = wp->walks_per_round;
    p.window = tp->window;
    p.K = tp->negatives;
    p.max_rounds = fp->max_rounds;
    p.ks = fp->ks;
    p.enabled = fp->enabled;
    p.reactivate = fp->reactivate;
    p.precision = tp->precision;
    p.mu = fp->mu;
    p.lr0 = tp->lr0;
    p.lr_total_tokens = tp->lr_total_tokens;
    p.rows_per_warp = tp->hogwild_rows_per_warp > 0 ? tp->hogwild_rows_per_warp : 16;
    p.mode = tp->mode;
    return p;
}

felog_status check_params(const felog_walk_params *wp, const felog_train_params *tp, const felog_feedback_params *fp) {
    if (!wp || !tp || !fp) return FELOG_ERR_INVALID_ARG;
    if (wp->length < 1 || wp->walks_per_round < 1) return FELOG_ERR_INVALID_ARG;
    if (tp->window < 1 || tp->window > 16 || tp->negatives < 1 || tp->negatives > 7)
        return FELOG_ERR_UNSUPPORTED;  // the batched trainer is the half-warp form
    if (tp->mode != FELOG_SGNS_HOGWILD && tp->mode != FELOG_SGNS_MINIBATCH) return FELOG_ERR_UNSUPPORTED;
    if (tp->precision != FELOG_FP32 && tp->precision != FELOG_BF16_SR) return FELOG_ERR_INVALID_ARG;
    if (!(tp->lr0 >= 0.f)) return FELOG_ERR_INVALID_ARG;
    if (fp->ks < 1 || fp->ks > kMaxKs || fp->max_rounds < 0 || fp->max_rounds >= 65536) return FELOG_ERR_INVALID_ARG;
    const size_t smem = sizeof(int32_t) * kWarps * (wp->length + 2 * tp->window * tp->negatives);
    if (smem > 200 * 1024) return FELOG_ERR_UNSUPPORTED;
    return FELOG_OK;
}

felog_status check_job(int32_t n, int64_t nnz, int32_t dim) {
    if (n < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return FELOG_ERR_BAD_CSR;
    if (dim != 32 && dim != 64 && dim != 128) return FELOG_ERR_UNSUPPORTED;
    return FELOG_OK;
}

}  // namespace felog

using namespace felog;

// ---------------------------------------------------------------------------
// fixed batch (felog_batch_*)
// ---------------------------------------------------------------------------
struct felog_batch {
    int32_t n_jobs = 0;
    BParams p{};
    std::vector<int32_t> position;  // caller index -> plan index
    void *blob = nullptr;           // work memory of all jobs
    size_t blob_bytes = 0;
    BatchPlan plan;
    HostTuning tune;
    cudaGraphExec_t graph = nullptr;
    int graph_rounds = -1;
    double wait_s = kDefaultGridWaitS;  // budget of each grid-barrier wait (persistent form)
};

namespace {

void drop_graph(felog_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_rounds = -1;
}

felog_status batch_reset(felog_batch *b, cudaStream_t s) {
    // clear every job's state (contiguous per job), then initialise
    for (const BJob &jb : b->plan.jobs) {
        felog_status st = job_clear_state(jb, b->p, s);
        if (st) return st;
    }
    return plan_init_jobs(b->plan, b->p, s);
}

}  // namespace

extern "C" felog_status felog_batch_create(const felog_job *jobs, int32_t n_jobs, const felog_walk_params *wp,
                                           const felog_train_params *tp, const felog_feedback_params *fp,
                                           felog_batch **out) {
    if (!out) return FELOG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!jobs || n_jobs < 1) return FELOG_ERR_INVALID_ARG;
    felog_status st = check_params(wp, tp, fp);
    if (st) return st;
    for (int32_t i = 0; i < n_jobs; ++i) {
        if (!csr_shape_ok(&jobs[i].graph)) return FELOG_ERR_BAD_CSR;
        if ((st = check_job(jobs[i].graph.n, jobs[i].graph.nnz, jobs[i].dim))) return st;
        if (jobs[i].graph.n > 0 && (!jobs[i].phi_in || !jobs[i].phi_out)) return FELOG_ERR_INVALID_ARG;
    }
    // every job's graph is checked on the device before any kernel gathers through it
    {
        int32_t *status = nullptr;
        st = record_cuda_error(cudaMalloc(&status, sizeof(int32_t) * n_jobs), "felog_batch_create");
        if (st) return st;
        for (int32_t i = 0; i < n_jobs && !st; ++i)
            st = validate_csr_async(&jobs[i].graph, nullptr, 0, status + i, nullptr);
        std::vector<int32_t> host(n_jobs, 0);
        if (!st)
            st = record_cuda_error(cudaMemcpy(host.data(), status, sizeof(int32_t) * n_jobs, cudaMemcpyDeviceToHost),
                                   "felog_batch_create");
        cudaFree(status);
        if (st) return st;
        for (int32_t i = 0; i < n_jobs; ++i)
            if (host[i]) return FELOG_ERR_BAD_CSR;
    }
    felog_batch *b = new (std::nothrow) felog_batch();
    if (!b) return FELOG_ERR_INVALID_ARG;
    b->n_jobs = n_jobs;
    b->p = make_params(wp, tp, fp);
    b->tune.sgns_form = default_sgns_form(tp);
    // plan order: by dim (stable), so each dim's training items are contiguous
    std::vector<int32_t> order(n_jobs);
    for (int32_t i = 0; i < n_jobs; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return jobs[x].dim < jobs[y].dim; });
    b->position.resize(n_jobs);
    for (int32_t i = 0; i < n_jobs; ++i) b->position[order[i]] = i;
    std::vector<size_t> offs(n_jobs);
    size_t total = 0;
    for (int32_t i = 0; i < n_jobs; ++i) {
        offs[i] = total;
        total += job_work_bytes(jobs[order[i]].graph.n, jobs[order[i]].dim, b->p);
    }
    st = record_cuda_error(cudaMalloc(&b->blob, total), "felog_batch_create");
    if (st) {
        delete b;
        return st;
    }
    b->blob_bytes = total;
    std::vector<BJob> bj(n_jobs);
    for (int32_t i = 0; i < n_jobs; ++i) {
        const felog_job &j = jobs[order[i]];
        BJob &jb = bj[i];
        jb = BJob{};
        jb.offsets = j.graph.offsets;
        jb.cols = j.graph.cols;
        jb.nnz = j.graph.nnz;
        jb.n = j.graph.n;
        jb.dim = j.dim;
        jb.seed = j.seed;
        jb.phi_in = j.phi_in;
        jb.phi_out = j.phi_out;
        job_carve(jb, static_cast<char *>(b->blob) + offs[i], jb.n, b->p);
    }
    st = plan_build(b->plan, bj, b->p, nullptr);
    if (st) {
        cudaFree(b->blob);
        delete b;
        return st;
    }
    *out = b;
    return FELOG_OK;
}

extern "C" felog_status felog_batch_destroy(felog_batch *b) {
    if (!b) return FELOG_OK;
    drop_graph(b);
    plan_release(b->plan, nullptr);
    felog_status st = FELOG_OK;
    if (b->blob) st = record_cuda_error(cudaFree(b->blob), "felog_batch_destroy");
    delete b;
    return st;
}

extern "C" size_t felog_batch_device_bytes(const felog_batch *b) { return b ? b->blob_bytes + b->plan.bytes : 0; }

extern "C" felog_status felog_batch_reset(felog_batch *b, void *stream) {
    if (!b) return FELOG_ERR_INVALID_ARG;
    return batch_reset(b, static_cast<cudaStream_t>(stream));
}

extern "C" felog_status felog_batch_step(felog_batch *b, void *stream) {
    if (!b) return FELOG_ERR_INVALID_ARG;
    return plan_step(b->plan, b->p, b->tune, static_cast<cudaStream_t>(stream), 0x3f);
}

namespace {

// All rounds of every job in one cooperative launch of k_b_persistent (after
// the usual reset).  The grid is as many blocks as can be resident.
unsigned long long wait_budget_ns(double seconds) { return static_cast<unsigned long long>(seconds * 1e9); }

template <class T>
felog_status launch_persistent(felog_batch *b, cudaStream_t s) {
    const BatchPlan &plan = b->plan;
    const BParams &p = b->p;
    GridBarrier *bar = reinterpret_cast<GridBarrier *>(static_cast<char *>(plan.mem) + plan.o_bar);
    felog_status st = record_cuda_error(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s), "persistent");
    if (st) return st;
    const bool mb = p.mode == FELOG_SGNS_MINIBATCH;
    void (*kern)(BArgs, GridBarrier *, unsigned long long) =
        mb ? k_b_persistent<T, 0, true> : (p.K == 5 ? k_b_persistent<T, 5, false> : k_b_persistent<T, 0, false>);
    const size_t smem = sizeof(int32_t) * kWarps * (p.L + 2 * p.window * p.K);
    if (smem > 48 * 1024) {
        st = record_cuda_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(smem)), "persistent");
        if (st) return st;
    }
    int per_sm = 0;
    st = record_cuda_error(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, smem), "persistent");
    if (st) return st;
    if (per_sm < 1) return FELOG_ERR_UNSUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(per_sm * sm_count()));
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return record_cuda_error(cudaLaunchKernelEx(&cfg, kern, plan.args, bar, wait_budget_ns(b->wait_s)),
                             "persistent launch");
}

}  // namespace

extern "C" felog_status felog_batch_run(felog_batch *b, int32_t use_graph, void *stream) {
    if (!b || use_graph < 0 || use_graph > 2) return FELOG_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int R = b->p.max_rounds;
    if (use_graph == 2) {
        felog_status st = batch_reset(b, s);
        if (st) return st;
        return b->p.precision == FELOG_FP32 ? launch_persistent<float>(b, s) : launch_persistent<__nv_bfloat16>(b, s);
    }
    if (!use_graph || s == nullptr) {
        felog_status st = batch_reset(b, s);
        for (int r = 0; !st && r < R; ++r) st = plan_step(b->plan, b->p, b->tune, s, 0x3f);
        return st;
    }
    if (!b->graph || b->graph_rounds != R) {
        drop_graph(b);
        felog_status st = record_cuda_error(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture");
        if (st) return st;
        felog_status st2 = batch_reset(b, s);
        for (int r = 0; !st2 && r < R; ++r) st2 = plan_step(b->plan, b->p, b->tune, s, 0x3f);
        cudaGraph_t g = nullptr;
        st = record_cuda_error(cudaStreamEndCapture(s, &g), "capture");
        if (st2 || st) {
            if (g) cudaGraphDestroy(g);
            return st2 ? st2 : st;
        }
        st = record_cuda_error(cudaGraphInstantiate(&b->graph, g, 0), "graph instantiate");
        cudaGraphDestroy(g);
        if (st) return st;
        b->graph_rounds = R;
    }
    return record_cuda_error(cudaGraphLaunch(b->graph, s), "graph launch");
}

extern "C" felog_status felog_batch_set_wait_limit(felog_batch *b, double seconds) {
    if (!b || !(seconds > 0.0) || seconds > 3600.0) return FELOG_ERR_INVALID_ARG;
    b->wait_s = seconds;
    return FELOG_OK;
}

extern "C" felog_status felog_grid_barrier_check(int32_t phantom, int32_t passes, double seconds,
                                                 int32_t *where, void *stream) {
    if (phantom < 0 || phantom > 1024 || passes < 1 || passes > 1024 || !(seconds > 0.0) || seconds > 60.0)
        return FELOG_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GridBarrier *bar = nullptr;
    felog_status st = record_cuda_error(cudaMallocAsync(&bar, sizeof(GridBarrier), s), "felog_grid_barrier_check");
    if (st) return st;
    st = record_cuda_error(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s), "felog_grid_barrier_check");
    int per_sm = 0;
    if (!st)
        st = record_cuda_error(
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_barrier_check, kBThreads, 0),
            "felog_grid_barrier_check");
    if (!st && per_sm < 1) st = FELOG_ERR_UNSUPPORTED;
    if (!st) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(per_sm * sm_count()));
        cfg.blockDim = dim3(kBThreads);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        st = record_cuda_error(cudaLaunchKernelEx(&cfg, k_grid_barrier_check, bar, static_cast<unsigned>(phantom),
                                                  static_cast<int>(passes), wait_budget_ns(seconds)),
                               "felog_grid_barrier_check");
    }
    GridBarrier h{};
    if (!st)
        st = record_cuda_error(cudaMemcpyAsync(&h, bar, sizeof h, cudaMemcpyDeviceToHost, s),
                               "felog_grid_barrier_check");
    felog_status st2 = record_cuda_error(cudaFreeAsync(bar, s), "felog_grid_barrier_check");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "felog_grid_barrier_check");
    if (st) return st;
    if (st2) return st2;
    if (where) *where = h.error ? h.where : -1;
    return h.error ? FELOG_ERR_TIMEOUT : FELOG_OK;
}

extern "C" felog_status felog_batch_read(felog_batch *b, felog_job_stats *stats, int32_t *rec_n_active,
                                         double *rec_loss, void *stream) {
    if (!b) return FELOG_ERR_INVALID_ARG;
    std::vector<BState> sts;
    std::vector<int32_t> rna, rnn;
    std::vector<double> rl;
    felog_status st = plan_gather(b->plan, b->p, static_cast<cudaStream_t>(stream), sts, rna, rnn, rl);
    if (st) return st;
    // a persistent run whose grid barrier gave up waiting has failed
    GridBarrier bar{};
    st = record_cuda_error(cudaMemcpy(&bar, static_cast<char *>(b->plan.mem) + b->plan.o_bar, sizeof bar,
                                      cudaMemcpyDeviceToHost), "felog_batch_read");
    if (st) return st;
    if (bar.error) return FELOG_ERR_TIMEOUT;
    const int n = b->n_jobs;
    for (int32_t c = 0; c < n; ++c) {
        const int32_t i = b->position[c];
        if (stats) {
            felog_job_stats &o = stats[c];
            o.rounds = sts[i].round;
            o.done = sts[i].done;
            o.tokens = sts[i].clock;
            o.n_live = sts[i].n_live;
            o.loss_last = sts[i].round > 0 ? rl[static_cast<size_t>(sts[i].round - 1) * n + i] : 0.0;
        }
        for (int32_t r = 0; r < b->p.max_rounds; ++r) {
            if (rec_n_active) rec_n_active[static_cast<size_t>(r) * n + c] = rna[static_cast<size_t>(r) * n + i];
            if (rec_loss) rec_loss[static_cast<size_t>(r) * n + c] = rl[static_cast<size_t>(r) * n + i];
        }
    }
    return FELOG_OK;
}

extern "C" felog_status felog_batch_job_buffers(const felog_batch *b, int32_t job, felog_job_buffers *out) {
    if (!b || !out || job < 0 || job >= b->n_jobs) return FELOG_ERR_INVALID_ARG;
    const BJob &jb = b->plan.jobs[b->position[job]];
    out->active[0] = jb.active[0];
    out->active[1] = jb.active[1];
    out->starts = jb.starts;
    out->walks = jb.walks;
    out->counts = jb.counts;
    out->thr = jb.thr;
    out->alias = jb.alias;
    return FELOG_OK;
}

extern "C" felog_status felog_batch_set_tuning(felog_batch *b, const felog_tuning *t) {
    if (!b || !t) return FELOG_ERR_INVALID_ARG;
    if (t->walk_block < 32 || t->walk_block > 1024 || t->walk_block % 32 != 0) return FELOG_ERR_INVALID_ARG;
    if (t->sgns_blocks_per_sm < 1 || t->sgns_blocks_per_sm > 8) return FELOG_ERR_INVALID_ARG;
    if (t->feedback_blocks_per_sm < 1 || t->feedback_blocks_per_sm > 32) return FELOG_ERR_INVALID_ARG;
    if (t->sgns_form != 1 && t->sgns_form != 2 && t->sgns_form != 4) return FELOG_ERR_INVALID_ARG;
    b->tune.walk_block = t->walk_block;
    b->tune.sgns_blocks_per_sm = t->sgns_blocks_per_sm;
    b->tune.feedback_blocks_per_sm = t->feedback_blocks_per_sm;
    b->tune.sgns_form = t->sgns_form;
    drop_graph(b);
    return FELOG_OK;
}

// Autotuner: times the walk launch shape, the trainer's shape (pairs per
// warp, lanes per row, rows prefetched to shared memory or not) with its
// blocks per SM, and the Psi blocks per SM on round 0 of this batch (the
// batch is re-initialised before each probe) and keeps the fastest of each.
// With cache_path, results are looked up and stored in a text file keyed by
// GPU name and batch shape.
extern "C" felog_status felog_batch_autotune(felog_batch *b, const char *cache_path, felog_tuning *out,
                                             void *stream) {
    if (!b) return FELOG_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    int64_t dsum = 0;
    for (int32_t d : b->plan.dims) dsum += d;
    std::string gpu(prop.name);
    std::replace(gpu.begin(), gpu.end(), ' ', '_');  // the cache file is whitespace separated
    const std::string key = gpu + "|tuner=2|n=" + std::to_string(b->plan.args.n_nodes) + "|jobs=" +
                            std::to_string(b->n_jobs) + "|dsum=" + std::to_string(dsum) + "|L=" +
                            std::to_string(b->p.L) + "|w=" + std::to_string(b->p.window) + "|K=" +
                            std::to_string(b->p.K) + "|p=" + std::to_string(b->p.precision);
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string k;
            int wb, sb, fb, form;
            if (!(ls >> k >> wb >> sb >> fb >> form) || k != key) continue;
            b->tune.walk_block = wb;
            b->tune.sgns_blocks_per_sm = sb;
            b->tune.feedback_blocks_per_sm = fb;
            b->tune.sgns_form = form;
            drop_graph(b);
            if (out) *out = felog_tuning{wb, sb, fb, 1, form};
            return FELOG_OK;
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_phase = [&](unsigned before, unsigned phase) -> float {
        batch_reset(b, s);
        plan_step(b->plan, b->p, b->tune, s, before);
        cudaEventRecord(e0, s);
        plan_step(b->plan, b->p, b->tune, s, phase);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    HostTuning best = b->tune;
    float best_ms = 1e30f;
    for (int wb : {128, 256, 512}) {
        b->tune.walk_block = wb;
        const float ms = time_phase(1, 2);
        if (ms < best_ms) { best_ms = ms; best.walk_block = wb; }
    }
    b->tune.walk_block = best.walk_block;
    best_ms = 1e30f;
    if (b->p.mode == FELOG_SGNS_HOGWILD) {
        // trainer shape (form: 2 = two pairs per warp, 16 lanes per row; 1 = one
        // pair per warp, 32 lanes; 4 = form 2 with rows prefetched to shared
        // memory, where the dims allow it), resident blocks per SM
        for (int form : {2, 1, 4}) {
            for (int sb : {1, 2}) {
                b->tune.sgns_form = form;
                b->tune.sgns_blocks_per_sm = sb;
                const float ms = time_phase(1 | 2 | 4, 8);
                if (ms < best_ms) {
                    best_ms = ms;
                    best.sgns_blocks_per_sm = sb;
                    best.sgns_form = form;
                }
            }
        }
    }
    b->tune.sgns_blocks_per_sm = best.sgns_blocks_per_sm;
    b->tune.sgns_form = best.sgns_form;
    best_ms = 1e30f;
    for (int fb : {4, 8, 16}) {
        b->tune.feedback_blocks_per_sm = fb;
        const float ms = time_phase(1 | 2 | 4 | 8, 16);
        if (ms < best_ms) { best_ms = ms; best.feedback_blocks_per_sm = fb; }
    }
    b->tune = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    felog_status st = batch_reset(b, s);
    if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "autotune");
    if (st) return st;
    drop_graph(b);
    if (cache_path) {
        std::ofstream o(cache_path, std::ios::app);
        o << key << " " << best.walk_block << " " << best.sgns_blocks_per_sm << " " << best.feedback_blocks_per_sm
          << " " << best.sgns_form << "\n";
    }
    if (out)
        *out = felog_tuning{best.walk_block, best.sgns_blocks_per_sm, best.feedback_blocks_per_sm, 0, best.sgns_form};
    return FELOG_OK;
}
