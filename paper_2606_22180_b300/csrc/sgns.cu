// Train: skip-gram with negative sampling (Eq. 1, Eq. 2) on one round's corpus.
//
// Work split: one warp per walk (HOGWILD) or per center position (MINIBATCH).
// Lane l owns elements [l*EPL, (l+1)*EPL) of a row (EPL = dim/32), so a row
// is one 128-bit (FP32, dim 128) or 64-bit (BF16, dim 128) load per lane.
// For a center c the warp:
//   1. draws all 2W*K negatives of the center lane-parallel (Philox + alias
//      table) into shared memory;
//   2. keeps phi_out[c] in registers across its 2W pairs;
//   3. per pair, issues the context row and the K negative rows together,
//      forms K+1 partial dot products and reduces them with a transposed
//      reduce-scatter (lane 4t ends with the dot of target t), evaluates the
//      sigmoid of one target per lane and broadcasts the K+1 coefficients;
//   4. updates rows in place (HOGWILD: plain stores, races tolerated as in
//      lock-free SGD) or adds fixed-point increments (MINIBATCH).
// The pair loss -log sigma(s+) - sum log sigma(-s_k) is summed per warp and
// added to a 64-bit fixed-point accumulator (2^-24 resolution), so the
// total does not depend on the order in which warps finish.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "sgns_core.cuh"

namespace felog {

struct SgnsArgs {
    const int32_t *walks;
    int64_t n_walks;
    int32_t L, n, window, K;
    float lr0, inv_T;
    int64_t clock_base;
    const uint64_t *thr;
    const int32_t *alias;
    const uint64_t *S;
    uint64_t seed;
    uint32_t round;
    unsigned long long *loss_acc;
    int32_t stage_flush;
};

// KFIX > 0: the number of negatives is a compile-time constant.
template <int D, class T, int MAXT, int KFIX>
__global__ void __launch_bounds__(kSgnsThreads, 3)
    k_sgns_hogwild(SgnsArgs a, T *__restrict__ phi_in, T *__restrict__ phi_out) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int K = KFIX > 0 ? KFIX : a.K;
    int32_t *wk = smem + wib * (a.L + 2 * a.window * K);
    int32_t *negs = wk + a.L;
    TrainView<T> v{phi_in, phi_out, a.thr, a.alias, static_cast<uint64_t>(a.n), *a.S, a.seed, a.round,
                   a.lr0, a.inv_T, a.clock_base, a.window, a.K, a.L, 0};
    long long loss_fx = 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kWarps;
    for (int64_t wi = static_cast<int64_t>(blockIdx.x) * kWarps + wib; wi < a.n_walks; wi += warps)
        loss_fx += fw_train_walk<D, T, MAXT, KFIX>(v, a.walks + wi * a.L, wi, wk, negs);
    // warp total of the loss, then one integer add per warp
    for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
    if (lane == 0 && loss_fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(loss_fx));
}


// Form 4: the half-warp trainer with each step's rows prefetched to shared
// memory (hw_train_walk_pf; shared-memory layout in pf_bytes_per_warp).

template <int D, class T, int KFIX>
__global__ void __launch_bounds__(kSgnsThreads, 2)
    k_sgns_hogwild_pf(SgnsArgs a, T *__restrict__ phi_in, T *__restrict__ phi_out) {
    extern __shared__ __align__(16) int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int K = KFIX > 0 ? KFIX : a.K;
    const int per_warp = pf_bytes_per_warp(a.L, a.window, K, D, static_cast<int>(sizeof(T)));
    char *base = reinterpret_cast<char *>(smem) + wib * per_warp;
    int32_t *wk = reinterpret_cast<int32_t *>(base);
    int32_t *negs = wk + a.L;
    char *rows = base + 4 * ((a.L + 2 * a.window * K + 3) & ~3);
    TrainView<T> v{phi_in, phi_out, a.thr, a.alias, static_cast<uint64_t>(a.n), *a.S, a.seed, a.round,
                   a.lr0, a.inv_T, a.clock_base, a.window, a.K, a.L, 0};
    long long loss_fx = 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kWarps;
    if constexpr (kPfSupported<D, T>) {
        for (int64_t wi = static_cast<int64_t>(blockIdx.x) * kWarps + wib; wi < a.n_walks; wi += warps)
            loss_fx += hw_train_walk_pf<D, T, KFIX>(v, a.walks + wi * a.L, wi, wk, negs, rows);
    }
    for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
    if (lane == 0 && loss_fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(loss_fx));
}

// Form 5: the half-warp trainer on float tables with each step's row
// increments added by the bulk-copy engine (hw_train_walk<..., BULK>).
template <int D, int KFIX>
__global__ void __launch_bounds__(kSgnsThreads, 2)
    k_sgns_hogwild_bulk(SgnsArgs a, float *__restrict__ phi_in, float *__restrict__ phi_out) {
    extern __shared__ __align__(16) int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int K = KFIX > 0 ? KFIX : a.K;
    char *base = reinterpret_cast<char *>(smem) + wib * bulk_bytes_per_warp(a.L, a.window, K, D);
    int32_t *wk = reinterpret_cast<int32_t *>(base);
    int32_t *negs = wk + a.L;
    float *slots = reinterpret_cast<float *>(base + 4 * ((a.L + 2 * a.window * K + 3) & ~3));
    TrainView<float> v{phi_in, phi_out, a.thr, a.alias, static_cast<uint64_t>(a.n), *a.S, a.seed, a.round,
                       a.lr0, a.inv_T, a.clock_base, a.window, a.K, a.L, 0};
    long long loss_fx = 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kWarps;
    for (int64_t wi = static_cast<int64_t>(blockIdx.x) * kWarps + wib; wi < a.n_walks; wi += warps)
        loss_fx += hw_train_walk<D, float, KFIX, false, true, true>(v, a.walks + wi * a.L, wi, wk, negs, slots);
    for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
    if (lane == 0 && loss_fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(loss_fx));
}

// Shared memory words per warp of the half-warp trainer: walk and negative
// ids (rounded up to 16 bytes), then with STAGE the staged phi_in increments.
inline int hw_words_per_warp(int L, int window, int K, int dim, bool stage) {
    const int ids = (L + 2 * window * K + 3) & ~3;
    return ids + (stage ? static_cast<int>(stage_floats(window, dim)) : 0);
}

template <int D, class T, int KFIX, bool STAGE>
__global__ void __launch_bounds__(kSgnsThreads, 2)
    k_sgns_hogwild_hw(SgnsArgs a, T *__restrict__ phi_in, T *__restrict__ phi_out) {
    extern __shared__ __align__(16) int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int K = KFIX > 0 ? KFIX : a.K;
    const int ids = (a.L + 2 * a.window * K + 3) & ~3;
    const int R = 2 * a.window + 1;
    int32_t *wk = smem + wib * (ids + (STAGE ? R * D : 0));
    int32_t *negs = wk + a.L;
    float *delta = nullptr;
    if constexpr (STAGE) {
        delta = reinterpret_cast<float *>(wk + ids);
        for (int i = lane; i < R * D; i += 32) delta[i] = 0.f;
        __syncwarp();
    }
    TrainView<T> v{phi_in, phi_out, a.thr, a.alias, static_cast<uint64_t>(a.n), *a.S, a.seed, a.round,
                   a.lr0, a.inv_T, a.clock_base, a.window, a.K, a.L, a.stage_flush};
    long long loss_fx = 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kWarps;
    for (int64_t wi = static_cast<int64_t>(blockIdx.x) * kWarps + wib; wi < a.n_walks; wi += warps)
        loss_fx += hw_train_walk<D, T, KFIX, STAGE>(v, a.walks + wi * a.L, wi, wk, negs, delta);
    for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
    if (lane == 0 && loss_fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(loss_fx));
}


// ----------------------------------------------------------------------------
// MINIBATCH: one warp per center position of the batch [b0, b1) (the per-center
// and per-row routines are in sgns_core.cuh, shared with the batched trainer).
// ----------------------------------------------------------------------------
template <int D, class T, int MAXT>
__global__ void __launch_bounds__(kSgnsThreads)
    k_sgns_mb_grad(SgnsArgs a, int64_t b0, int64_t b1, float eta, const T *__restrict__ phi_in,
                   const T *__restrict__ phi_out, MbState st) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t *negs = smem + wib * (2 * a.window * a.K);
    const int64_t tok = b0 + static_cast<int64_t>(blockIdx.x) * kWarps + wib;
    if (tok >= b1) return;
    const int64_t wi = tok / a.L;
    const int p = static_cast<int>(tok - wi * a.L);
    const MbView v{a.thr, a.alias, static_cast<uint64_t>(a.n), *a.S, a.seed, a.round, a.window, a.K, a.L};
    const float closs = mb_grad_center<D, T, MAXT>(v, a.walks + wi * a.L, wi, p, eta, phi_in, phi_out, st, negs);
    long long loss_fx = __float2ll_rn(closs * kLossScaleF);
    for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
    if (lane == 0 && loss_fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(loss_fx));
}

// Apply the accumulated increments of the touched rows and clear them.
// The last block to finish resets the list counters.
template <int D, class T>
__global__ void __launch_bounds__(256)
    k_sgns_mb_apply(T *__restrict__ phi_in, T *__restrict__ phi_out, MbState st, uint64_t seed,
                    uint32_t batch_key) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    const int32_t n_in = st.counters[0], n_out = st.counters[1];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5);
         i < static_cast<int64_t>(n_in) + n_out; i += warps) {
        const bool is_in = i < n_in;
        const int32_t r = is_in ? st.list_in[i] : st.list_out[i - n_in];
        mb_apply_row<D, T>(is_in ? phi_in : phi_out, is_in ? st.acc_in : st.acc_out, is_in ? st.mark_in : st.mark_out,
                           r, is_in, seed, batch_key, lane);
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(st.counters + 2, 1) == static_cast<int>(gridDim.x) - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        st.counters[0] = 0;
        st.counters[1] = 0;
        st.counters[2] = 0;
    }
}

__global__ void k_loss_finish(const unsigned long long *__restrict__ acc, const int32_t *__restrict__ timeout,
                              double *__restrict__ loss) {
    *loss = *timeout ? __longlong_as_double(0x7ff8000000000000LL)
                     : static_cast<double>(static_cast<long long>(*acc)) / kLossScale;
}

// ----------------------------------------------------------------------------
// Table initialisation.
// ----------------------------------------------------------------------------
template <class T>
__global__ void k_init_tables(int32_t n, int32_t dim, uint64_t seed, T *__restrict__ phi_in,
                              T *__restrict__ phi_out) {
    const int64_t groups = static_cast<int64_t>(n) * (dim / 4);
    for (int64_t gidx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; gidx < groups;
         gidx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = static_cast<int32_t>(gidx / (dim / 4));
        const int32_t i4 = static_cast<int32_t>(gidx - static_cast<int64_t>(v) * (dim / 4));
        const u32x4 r = philox(seed, static_cast<uint32_t>(i4), static_cast<uint32_t>(v), 0u, kStreamInit);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
        const float fd = static_cast<float>(dim);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float u = static_cast<float>(w[k] >> 8) * 5.9604644775390625e-08f;  // 2^-24
            const float x = __fdiv_rn(u - 0.5f, fd);
            const int64_t off = static_cast<int64_t>(v) * dim + i4 * 4 + k;
            if constexpr (std::is_same<T, float>::value) {
                phi_in[off] = x;
                phi_out[off] = 0.f;
            } else {
                phi_in[off] = __float2bfloat16_rn(x);
                phi_out[off] = __float2bfloat16_rn(0.f);
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Host side.
// ----------------------------------------------------------------------------
struct TrainWorkspace {
    unsigned long long *loss_acc;
    int32_t *timeout;  // set by a TILE launch whose tensor-core wait gave up
    float *tile_scratch;  // TILE mode, tiles in order: a tile's staged dY rows
    MbState mb;
};

size_t tile_scratch_floats();

felog_status launch_tile(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                         const felog_train_params *tp, const uint64_t *thr, const int32_t *alias,
                         const uint64_t *S, uint64_t seed, int32_t round, int64_t clock_base,
                         void *phi_in, void *phi_out, unsigned long long *loss_acc, int32_t *timeout,
                         float *scratch, cudaStream_t s);

static bool minibatch_mode(const felog_train_params *tp) { return tp->mode == FELOG_SGNS_MINIBATCH; }

static TrainWorkspace carve_train(Carver &c, int32_t n, const felog_train_params *tp) {
    TrainWorkspace w{};
    w.loss_acc = c.take<unsigned long long>(1);
    w.timeout = c.take<int32_t>(1);
    if (tp->mode == FELOG_SGNS_TILE) w.tile_scratch = c.take<float>(tile_scratch_floats());
    if (minibatch_mode(tp)) {
        const size_t nn = n > 0 ? static_cast<size_t>(n) : 1;
        w.mb.acc_in = c.take<long long>(nn * tp->dim);
        w.mb.acc_out = c.take<long long>(nn * tp->dim);
        w.mb.mark_in = c.take<uint32_t>(nn);
        w.mb.mark_out = c.take<uint32_t>(nn);
        w.mb.list_in = c.take<int32_t>(nn);
        w.mb.list_out = c.take<int32_t>(nn);
        w.mb.counters = c.take<int32_t>(4);
    }
    return w;
}

static bool params_ok(const felog_train_params *tp) {
    if (!tp) return false;
    if (tp->dim != 32 && tp->dim != 64 && tp->dim != 128 && tp->dim != 256) return false;
    if (tp->window < 1 || tp->window > 16 || tp->negatives < 1 || tp->negatives > 15) return false;
    if (tp->mode != FELOG_SGNS_HOGWILD && tp->mode != FELOG_SGNS_MINIBATCH && tp->mode != FELOG_SGNS_TILE)
        return false;
    if (tp->mode == FELOG_SGNS_TILE) {
        if (tp->dim > 128) return false;
        if (tp->tile_negatives != 0 && (tp->tile_negatives < 128 || tp->tile_negatives > 512 ||
                                        tp->tile_negatives % 128 != 0))
            return false;
        if (tp->tile_ctas < 0) return false;
    }
    if (tp->precision != FELOG_FP32 && tp->precision != FELOG_BF16_SR) return false;
    if (tp->mode == FELOG_SGNS_MINIBATCH && tp->minibatch < 1) return false;
    if (tp->hogwild_form < 0 || tp->hogwild_form > 5) return false;
    if (tp->hogwild_form >= 2 && (tp->dim > 128 || tp->negatives > 7)) return false;
    if (tp->hogwild_form == 3 && tp->window > kStageMaxWindow) return false;
    if (tp->stage_flush < 0) return false;
    if (!(tp->lr0 >= 0.f) || tp->lr_total_tokens <= 0) return false;
    return true;
}

template <int D, class T, int MAXT, int KFIX>
static felog_status launch_train(const SgnsArgs &a, const felog_train_params *tp, void *phi_in,
                                 void *phi_out, TrainWorkspace &w, cudaStream_t s) {
    T *pin = static_cast<T *>(phi_in);
    T *pout = static_cast<T *>(phi_out);
    if (!minibatch_mode(tp)) {
        // half-warp form for dim <= 128 and K + 1 <= 8, full-warp form otherwise;
        // form 3 stages the window's phi_in increments (window <= 15) when asked
        // for: faster (R-MAT 20, float: 559 vs 613 ms per round), but hub rows
        // then collect many warps' delayed increments and the link AUC of the
        // 10-round run fell from 0.797 to 0.735, so it is not the default
        const bool half_warp = D <= 128 && MAXT == 8 && tp->hogwild_form != 1;
        const bool stage = half_warp && tp->hogwild_form == 3;
        constexpr int DH = D <= 128 ? D : 128;
        // form 4 (rows prefetched with cp.async) for rows of 128 to 512 bytes; the automatic
        // choice for bf16 tables of dim 128 (R-MAT 20: 412 against 423 ms per round for
        // form 2, same link AUC), not for float tables (687 against 608 ms)
        constexpr bool kBf16 = !std::is_same<T, float>::value;
        const bool prefetch = half_warp && kPfSupported<DH, T> &&
                              (tp->hogwild_form == 4 || (tp->hogwild_form == 0 && kBf16 && DH == 128));
        size_t smem = half_warp ? sizeof(int32_t) * kWarps * hw_words_per_warp(a.L, a.window, a.K, DH, stage)
                                : sizeof(int32_t) * kWarps * (a.L + 2 * a.window * a.K);
        if (prefetch)
            smem = static_cast<size_t>(kWarps) * pf_bytes_per_warp(a.L, a.window, a.K, DH, static_cast<int>(sizeof(T)));
        // form 5 (row increments added by the bulk-copy engine): float tables
        const bool bulk = half_warp && !kBf16 && tp->hogwild_form == 5;
        if (bulk) smem = static_cast<size_t>(kWarps) * bulk_bytes_per_warp(a.L, a.window, a.K, DH);
        if (smem > 200 * 1024) return FELOG_ERR_UNSUPPORTED;  // walk too long to stage per warp
        void (*kern)(SgnsArgs, T *, T *) = prefetch ? k_sgns_hogwild_pf<DH, T, KFIX>
                                           : stage ? k_sgns_hogwild_hw<DH, T, KFIX, true>
                                                   : (half_warp ? k_sgns_hogwild_hw<DH, T, KFIX, false>
                                                                : k_sgns_hogwild<D, T, MAXT, KFIX>);
        if constexpr (!kBf16) {
            if (bulk) kern = k_sgns_hogwild_bulk<DH, KFIX>;
        }
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSgnsThreads, smem);
        if (per_sm < 1) per_sm = 1;
        // resident warps <= n / rows_per_warp: on small graphs this bounds how
        // many warps update the same rows at once (staleness of lock-free SGD)
        const int64_t rows_per_warp = tp->hogwild_rows_per_warp > 0 ? tp->hogwild_rows_per_warp : 16;
        const int64_t cap_blocks = std::max<int64_t>(1, a.n / rows_per_warp / kWarps);
        const int64_t want = (a.n_walks + kWarps - 1) / kWarps;
        const int blocks = static_cast<int>(
            std::min<int64_t>({want, static_cast<int64_t>(per_sm) * sm_count(), cap_blocks}));
        kern<<<blocks, kSgnsThreads, smem, s>>>(a, pin, pout);
        return check_launch("felog_train (hogwild)");
    }
    const size_t smem = sizeof(int32_t) * kWarps * (2 * a.window * a.K);
    const int64_t total = a.n_walks * a.L;
    const int64_t B = tp->minibatch;
    felog_status st = record_cuda_error(cudaMemsetAsync(w.mb.counters, 0, 4 * sizeof(int32_t), s), "train");
    if (st) return st;
    int apply_blocks = sm_count() * 4;
    for (int64_t b0 = 0, bi = 0; b0 < total; b0 += B, ++bi) {
        const int64_t b1 = std::min(total, b0 + B);
        const double f = 1.0 - static_cast<double>(a.clock_base + b0) / static_cast<double>(tp->lr_total_tokens);
        const float eta = static_cast<float>(static_cast<double>(tp->lr0) * (f < 1e-4 ? 1e-4 : f));
        const int grid = static_cast<int>((b1 - b0 + kWarps - 1) / kWarps);
        k_sgns_mb_grad<D, T, MAXT><<<grid, kSgnsThreads, smem, s>>>(a, b0, b1, eta, pin, pout, w.mb);
        k_sgns_mb_apply<D, T><<<apply_blocks, 256, 0, s>>>(pin, pout, w.mb, a.seed,
                                                           (a.round << 20) ^ static_cast<uint32_t>(bi));
    }
    return check_launch("felog_train (minibatch)");
}

template <int D, class T>
static felog_status dispatch_maxt(const SgnsArgs &a, const felog_train_params *tp, void *pi,
                                  void *po, TrainWorkspace &w, cudaStream_t s) {
    if (tp->negatives == 5) return launch_train<D, T, 8, 5>(a, tp, pi, po, w, s);
    if (tp->negatives + 1 <= 8) return launch_train<D, T, 8, 0>(a, tp, pi, po, w, s);
    return launch_train<D, T, 16, 0>(a, tp, pi, po, w, s);
}

template <class T>
static felog_status dispatch_dim(const SgnsArgs &a, const felog_train_params *tp, void *pi, void *po,
                                 TrainWorkspace &w, cudaStream_t s) {
    switch (tp->dim) {
        case 32: return dispatch_maxt<32, T>(a, tp, pi, po, w, s);
        case 64: return dispatch_maxt<64, T>(a, tp, pi, po, w, s);
        case 128: return dispatch_maxt<128, T>(a, tp, pi, po, w, s);
        case 256: return dispatch_maxt<256, T>(a, tp, pi, po, w, s);
    }
    return FELOG_ERR_UNSUPPORTED;
}

}  // namespace felog

using namespace felog;

namespace felog {
// element pairs (x[2p], x[2p+1]) per thread; the pair's random word carries
// r16[2p + 1] in its upper half and r16[2p] in its lower half
__global__ void k_sr_bf16(const float *__restrict__ x, const uint16_t *__restrict__ r16, int64_t n,
                          uint16_t *__restrict__ out) {
    const int64_t pairs = (n + 1) / 2;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < pairs;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = 2 * q;
        const bool two = i + 1 < n;
        const float hi = two ? x[i + 1] : 0.f;
        const uint32_t bits = (two ? static_cast<uint32_t>(r16[i + 1]) << 16 : 0u) | r16[i];
        const uint32_t t = sr_pack_bf16x2(hi, x[i], bits);
        out[i] = static_cast<uint16_t>(t & 0xffffu);
        if (two) out[i + 1] = static_cast<uint16_t>(t >> 16);
    }
}
}  // namespace felog

extern "C" felog_status felog_sr_bf16(const float *x, const uint16_t *r16, int64_t n, uint16_t *out,
                                      void *stream) {
    if (n < 0 || (n > 0 && (!x || !r16 || !out))) return FELOG_ERR_INVALID_ARG;
    if (n == 0) return FELOG_OK;
    const int64_t pairs = (n + 1) / 2;
    const int grid = static_cast<int>(std::min<int64_t>((pairs + 255) / 256, static_cast<int64_t>(sm_count()) * 8));
    k_sr_bf16<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, r16, n, out);
    return check_launch("felog_sr_bf16");
}

extern "C" size_t felog_train_workspace_bytes(int64_t n_walks, int32_t L, int32_t n,
                                              const felog_train_params *tp) {
    (void)n_walks;
    (void)L;
    if (!params_ok(tp)) return 0;
    Carver c(nullptr, 0);
    carve_train(c, n, tp);
    return align_up(c.used, 256);
}

extern "C" felog_status felog_train(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                                    const felog_train_params *tp, const uint64_t *thr,
                                    const int32_t *alias, const uint64_t *S, uint64_t seed,
                                    int32_t round, int64_t clock_base, void *phi_in, void *phi_out,
                                    double *loss, void *workspace, size_t workspace_bytes,
                                    void *stream) {
    if (!params_ok(tp)) return FELOG_ERR_INVALID_ARG;
    if (n_walks < 0 || L < 1 || L > 65535 || n < 1 || round < 0 || round >= 65536 || clock_base < 0 ||
        !loss)
        return FELOG_ERR_INVALID_ARG;
    if (n_walks > 0 && (!walks || !thr || !alias || !S || !phi_in || !phi_out)) return FELOG_ERR_INVALID_ARG;
    if (n_walks > 0xffffffffLL) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_train_workspace_bytes(n_walks, L, n, tp))
        return FELOG_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    TrainWorkspace w = carve_train(c, n, tp);
    felog_status st = record_cuda_error(cudaMemsetAsync(w.loss_acc, 0, sizeof(unsigned long long), s), "train");
    if (!st) st = record_cuda_error(cudaMemsetAsync(w.timeout, 0, sizeof(int32_t), s), "train");
    if (st) return st;
    if (minibatch_mode(tp)) {
        st = record_cuda_error(cudaMemsetAsync(w.mb.mark_in, 0, sizeof(uint32_t) * n, s), "train");
        if (!st) st = record_cuda_error(cudaMemsetAsync(w.mb.mark_out, 0, sizeof(uint32_t) * n, s), "train");
        if (!st) st = record_cuda_error(cudaMemsetAsync(w.mb.acc_in, 0, sizeof(long long) * n * tp->dim, s), "train");
        if (!st) st = record_cuda_error(cudaMemsetAsync(w.mb.acc_out, 0, sizeof(long long) * n * tp->dim, s), "train");
        if (st) return st;
    }
    if (n_walks > 0 && tp->mode == FELOG_SGNS_TILE) {
        st = launch_tile(walks, n_walks, L, n, tp, thr, alias, S, seed, round, clock_base, phi_in, phi_out,
                         w.loss_acc, w.timeout, w.tile_scratch, s);
        if (st) return st;
    } else if (n_walks > 0) {
        SgnsArgs a;
        a.walks = walks;
        a.n_walks = n_walks;
        a.L = L;
        a.n = n;
        a.window = tp->window;
        a.K = tp->negatives;
        a.lr0 = tp->lr0;
        a.inv_T = static_cast<float>(1.0 / static_cast<double>(tp->lr_total_tokens));
        a.clock_base = clock_base;
        a.thr = thr;
        a.alias = alias;
        a.S = S;
        a.seed = seed;
        a.round = static_cast<uint32_t>(round);
        a.loss_acc = w.loss_acc;
        a.stage_flush = tp->stage_flush;
        st = tp->precision == FELOG_FP32 ? dispatch_dim<float>(a, tp, phi_in, phi_out, w, s)
                                         : dispatch_dim<__nv_bfloat16>(a, tp, phi_in, phi_out, w, s);
        if (st) return st;
    }
    k_loss_finish<<<1, 1, 0, s>>>(w.loss_acc, w.timeout, loss);
    st = check_launch("felog_train");
    if (st || n_walks == 0 || tp->mode != FELOG_SGNS_TILE) return st;
    // TILE: a launch that gave up waiting for the tensor cores is a failed
    // call.  Outside stream capture the call waits for the launch and reads
    // the flag; during capture the NaN loss is the only report.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    st = record_cuda_error(cudaStreamIsCapturing(s, &cap), "felog_train (tile)");
    if (st || cap != cudaStreamCaptureStatusNone) return st;
    int32_t timed_out = 0;
    st = record_cuda_error(cudaMemcpyAsync(&timed_out, w.timeout, sizeof timed_out, cudaMemcpyDeviceToHost, s),
                           "felog_train (tile)");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "felog_train (tile)");
    if (!st && timed_out) st = FELOG_ERR_TIMEOUT;
    return st;
}

extern "C" felog_status felog_init_tables(int32_t n, int32_t dim, int32_t precision, uint64_t seed,
                                          void *phi_in, void *phi_out, void *stream) {
    if (n < 0 || (dim != 32 && dim != 64 && dim != 128 && dim != 256)) return FELOG_ERR_INVALID_ARG;
    if (precision != FELOG_FP32 && precision != FELOG_BF16_SR) return FELOG_ERR_INVALID_ARG;
    if (n == 0) return FELOG_OK;
    if (!phi_in || !phi_out) return FELOG_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t groups = static_cast<int64_t>(n) * (dim / 4);
    const int grid = static_cast<int>(std::min<int64_t>(ceil_div(groups, 256), sm_count() * 16));
    if (precision == FELOG_FP32)
        k_init_tables<float><<<grid, 256, 0, s>>>(n, dim, seed, static_cast<float *>(phi_in),
                                                  static_cast<float *>(phi_out));
    else
        k_init_tables<__nv_bfloat16><<<grid, 256, 0, s>>>(n, dim, seed, static_cast<__nv_bfloat16 *>(phi_in),
                                                          static_cast<__nv_bfloat16 *>(phi_out));
    return check_launch("felog_init_tables");
}
