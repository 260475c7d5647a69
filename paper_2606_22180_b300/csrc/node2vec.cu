// node2vec second-order walks, a Sample variant the paper names (Section
// 5.4); the transition rule is node2vec's (Grover and Leskovec, KDD 2016).
// Having come from t to v, the next node x (a neighbour of v) has weight
// 1/p if x == t, 1 if x is a neighbour of t, 1/q otherwise.
//
// Sampled by rejection: step 1 is uniform; at a later step, attempt a draws
// Philox(x0 = t | a << 16, x1 = s, x2 = r*wpr + j, stream 8), proposes
// neighbour floor(u64 * deg / 2^64) and accepts iff (hi64 >> 11) * 2^-53 <
// alpha(x) / alpha_max (binary64, evaluated in an exactly equivalent integer
// form); after 64 rejected attempts the last proposal is taken.  "x is a
// neighbour of t" is a binary search in t's sorted CSR row, made only when
// it decides the attempt.  A group of lanes per walker tries consecutive
// attempts side by side.  Rows, -1 padding and counts as in felog_walk.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace felog {

int sm_count();
bool csr_shape_ok(const felog_csr *g);

constexpr uint32_t kStreamN2v = 8;
constexpr int kN2vThreads = 256;
constexpr uint32_t kN2vAttempts = 64;

// x in the sorted row cols[lo, hi)?
__device__ __forceinline__ bool in_row(const int32_t *__restrict__ cols, int32_t lo, int32_t hi, int32_t x) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        const int32_t c = __ldg(cols + mid);
        if (c == x) return true;
        if (c < x) lo = mid + 1;
        else hi = mid;
    }
    return false;
}

// acceptance iff (hi64 >> 11) < K with K = ceil(alpha / alpha_max * 2^53):
// the integer form of (hi64 >> 11) * 2^-53 < alpha / alpha_max in binary64
// (both sides scaled by a power of two, exact; m < T iff m < ceil(T) for an
// integer m), so the kernel needs no FP64
struct N2vThresholds {
    uint64_t back, near, far;  // for x == t, x ~ t, otherwise
};

constexpr int kN2vLanes = 4;  // lanes per walker: attempts tried side by side
constexpr int kN2vWalkersPerWarp = 32 / kN2vLanes;
constexpr int kN2vRounds = static_cast<int>(kN2vAttempts) / kN2vLanes;
constexpr int kN2vGroup = 8;  // steps buffered per walker before they are stored
constexpr int kN2vBlocksPerSm = 6;  // resident blocks at <= 40 registers; the grid is one wave of them
static_assert(kN2vAttempts % kN2vLanes == 0 && 32 % kN2vLanes == 0, "attempt rounds must tile the warp");

// Each walker owns kN2vLanes lanes.  Round k tries attempts k*G .. k*G+G-1
// at once, one per lane, and takes the first that accepts, which is the
// attempt the one-at-a-time loop would stop at (after 64 rejections, the
// 64th proposal).  A non-return proposal is accepted outright below both of
// its possible thresholds and rejected at or above both; only in between,
// and only for lanes ahead of the group's first outright acceptance, is t's
// row searched.  The lanes of a walker keep its state in step; the first
// lane counts and buffers 8 steps in shared memory, which the group then
// stores as whole 32-byte sectors (one id per step per walker, interleaved
// with random reads of the graph, left sectors half-written in L2 and cost
// several DRAM writes each).
template <bool COUNT>
__global__ void __launch_bounds__(kN2vThreads, kN2vBlocksPerSm)
    k_walk_n2v(const int32_t *__restrict__ offsets, const int32_t *__restrict__ cols, int32_t n, int64_t nnz,
               const int32_t *__restrict__ starts, int32_t n_starts, int32_t L, int32_t wpr, N2vThresholds th,
               uint64_t seed, uint32_t round, int32_t *__restrict__ walks, uint32_t *__restrict__ counts) {
    __shared__ int32_t stage[kN2vThreads / kN2vLanes][kN2vGroup];
    const int lane = threadIdx.x & 31;
    const int rank = lane % kN2vLanes;
    const int gbase = lane - rank;
    const uint32_t gmask = ((1u << kN2vLanes) - 1u) << gbase;
    int32_t *buf = stage[threadIdx.x / kN2vLanes];
    const uint64_t lo_thr = th.near < th.far ? th.near : th.far;
    const uint64_t hi_thr = th.near < th.far ? th.far : th.near;
    const bool near_wins = th.near > th.far;  // between the thresholds, accept iff x ~ t does
    const int64_t total = static_cast<int64_t>(n_starts) * wpr;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w0 = warp * kN2vWalkersPerWarp; w0 < total; w0 += n_warps * kN2vWalkersPerWarp) {
        const int64_t w = w0 + lane / kN2vLanes;
        const bool valid = w < total;
        int32_t s = -1;
        uint32_t x2 = 0;
        if (valid) {
            const int32_t j = static_cast<int32_t>(w / n_starts);
            s = __ldg(starts + (w - static_cast<int64_t>(j) * n_starts));
            x2 = round * static_cast<uint32_t>(wpr) + static_cast<uint32_t>(j);
            if (s < 0 || s >= n) s = -1;  // a start outside the graph: a row of -1
        }
        int32_t *row = walks + (valid ? w : 0) * L;
        if (valid && rank == 0) {
            buf[0] = s;
            if (COUNT && s >= 0) atomicAdd(counts + s, 1u);
        }
        int32_t prev = -1, v = s, plo = 0, phi = 0;  // plo, phi: prev's row
        bool alive = valid && s >= 0;
        for (int32_t t = 1; t < L; ++t) {
            int32_t lo = 0, hi = 0;
            if (alive) {
                lo = __ldg(offsets + v);
                hi = __ldg(offsets + v + 1);
                // a row outside [0, nnz] ends the walk like a node without neighbours
                if (hi <= lo || lo < 0 || hi > nnz) {
                    alive = false;
                    lo = hi = 0;
                }
            }
            const uint64_t deg = static_cast<uint64_t>(static_cast<int64_t>(hi) - lo);
            int32_t nxt = -1;
            bool done = !alive;
            for (int k = 0; k < kN2vRounds; ++k) {
                if (__ballot_sync(kFull, !done) == 0) break;
                int32_t prop = -1;
                int state = 0;  // 0 reject, 1 accept, 2 decided by t's row
                if (!done) {
                    const uint32_t a = static_cast<uint32_t>(k * kN2vLanes + rank);
                    const u32x4 r = philox(seed, static_cast<uint32_t>(t) | (a << 16), static_cast<uint32_t>(s), x2,
                                           kStreamN2v);
                    prop = __ldg(cols + lo + static_cast<int64_t>(mulhi64(lo64(r), deg)));
                    if (prev < 0) {
                        state = a == 0;  // first step: uniform, the first proposal
                    } else {
                        const uint64_t m = hi64(r) >> 11;
                        if (prop == prev) state = m < th.back;
                        else if (m < lo_thr) state = 1;
                        else if (m < hi_thr) state = 2;
                    }
                }
                const uint32_t quick = __ballot_sync(kFull, state == 1) & gmask;
                const uint32_t ahead = quick ? (quick & (~quick + 1u)) - 1u : ~0u;  // lanes before it
                if (state == 2) state = ((ahead >> lane) & 1u) && in_row(cols, plo, phi, prop) == near_wins;
                const uint32_t acc = __ballot_sync(kFull, state == 1) & gmask;
                const int src = acc ? __ffs(acc) - 1 : gbase + kN2vLanes - 1;
                const int32_t pick = __shfl_sync(kFull, prop, src);
                if (!done && (acc || k == kN2vRounds - 1)) {
                    nxt = pick;
                    done = true;
                }
            }
            if (alive && (nxt < 0 || nxt >= n)) {  // a column outside the graph ends the walk
                nxt = -1;
                alive = false;
            }
            if (alive) {
                prev = v;
                plo = lo;
                phi = hi;
                v = nxt;
                if (COUNT && rank == 0) atomicAdd(counts + nxt, 1u);
            }
            if (valid && rank == 0) buf[t % kN2vGroup] = nxt;
            if (t % kN2vGroup == kN2vGroup - 1) {
                __syncwarp();
                if (valid)
                    for (int i = rank; i < kN2vGroup; i += kN2vLanes) row[t - (kN2vGroup - 1) + i] = buf[i];
                __syncwarp();
            }
        }
        const int32_t rest = L % kN2vGroup;  // steps still buffered
        __syncwarp();
        if (valid)
            for (int i = rank; i < rest; i += kN2vLanes) row[L - rest + i] = buf[i];
        __syncwarp();
    }
}

}  // namespace felog

using namespace felog;

extern "C" felog_status felog_walk_node2vec(const felog_csr *g, const int32_t *starts, int32_t n_starts,
                                            const felog_walk_params *wp, double p, double q, uint64_t seed,
                                            int32_t round, int32_t *walks, uint32_t *counts, void *stream) {
    if (!csr_shape_ok(g)) return FELOG_ERR_BAD_CSR;
    if (!wp || wp->length < 1 || wp->length > 65535 || wp->walks_per_round < 1 || n_starts < 0 || round < 0 ||
        round >= 65536)
        return FELOG_ERR_INVALID_ARG;
    if (!(p > 0.0) || !(q > 0.0) || !(p < 1e300) || !(q < 1e300)) return FELOG_ERR_INVALID_ARG;
    if (n_starts == 0) return FELOG_OK;
    if (!starts || !walks) return FELOG_ERR_INVALID_ARG;
    const double ap = 1.0 / p, aq = 1.0 / q;
    const double amax = ap > 1.0 ? (ap > aq ? ap : aq) : (1.0 > aq ? 1.0 : aq);
    auto fixed = [](double ratio) { return static_cast<uint64_t>(std::ceil(std::ldexp(ratio, 53))); };
    const N2vThresholds th{fixed(ap / amax), fixed(1.0 / amax), fixed(aq / amax)};
    const int64_t total = static_cast<int64_t>(n_starts) * wp->walks_per_round;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t per_block = kN2vThreads / kN2vLanes;
    const int blocks = static_cast<int>(std::min<int64_t>(ceil_div(total, per_block), static_cast<int64_t>(sm_count()) * kN2vBlocksPerSm));
    if (counts)
        k_walk_n2v<true><<<blocks, kN2vThreads, 0, s>>>(g->offsets, g->cols, g->n, g->nnz, starts, n_starts, wp->length,
                                                        wp->walks_per_round, th, seed, static_cast<uint32_t>(round),
                                                        walks, counts);
    else
        k_walk_n2v<false><<<blocks, kN2vThreads, 0, s>>>(g->offsets, g->cols, g->n, g->nnz, starts, n_starts, wp->length,
                                                         wp->walks_per_round, th, seed, static_cast<uint32_t>(round),
                                                         walks, counts);
    return check_launch("felog_walk_node2vec");
}
