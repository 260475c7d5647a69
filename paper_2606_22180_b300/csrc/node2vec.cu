// node2vec second-order walks, a Sample variant the paper names (Section
// 5.4); the transition rule is node2vec's (Grover and Leskovec, KDD 2016).
// Having come from t to v, the next node x (a neighbour of v) has weight
// 1/p if x == t, 1 if x is a neighbour of t, 1/q otherwise.
//
// One walker per thread, sampled by rejection: step 1 is uniform; at a
// later step, attempt a draws Philox(x0 = t | a << 16, x1 = s, x2 = r*wpr +
// j, stream 8), proposes neighbour floor(u64 * deg / 2^64) and accepts iff
// (hi64 >> 11) * 2^-53 < alpha(x) / alpha_max (binary64), after 64 rejected
// attempts the last proposal.  "x is a neighbour of t" is a binary search
// in t's sorted CSR row, made only when it decides the attempt.  Rows, -1
// padding and counts as in felog_walk.
#include <algorithm>

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

struct N2vThresholds {
    double back, near, far;  // alpha / alpha_max for x == t, x ~ t, otherwise
};

constexpr int kN2vGroup = 8;  // steps buffered per walker before they are stored

// the buffered steps t0 .. t0 + n - 1 of one walker to its row: 32 bytes in
// two 16-byte stores when whole and aligned, else one by one
__device__ __forceinline__ void n2v_flush(int32_t *__restrict__ dst, const int32_t *__restrict__ buf, int n) {
    if (n == kN2vGroup && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        reinterpret_cast<int4 *>(dst)[0] = make_int4(buf[0], buf[kN2vThreads], buf[2 * kN2vThreads], buf[3 * kN2vThreads]);
        reinterpret_cast<int4 *>(dst)[1] =
            make_int4(buf[4 * kN2vThreads], buf[5 * kN2vThreads], buf[6 * kN2vThreads], buf[7 * kN2vThreads]);
    } else {
        for (int i = 0; i < n; ++i) dst[i] = buf[i * kN2vThreads];
    }
}

// Each walker buffers its steps in shared memory and stores them 8 at a time,
// so that a row's 32-byte sectors are written whole: one at a time, the
// stores of 600k walkers interleaved with random reads of the graph were
// evicted from L2 half-written and cost several DRAM writes each.  The
// acceptance test only searches t's row when the draw u falls between the
// two thresholds that x != t can have (below both: accept; at or above
// both: reject), which takes the same decision the full test would.
template <bool COUNT>
__global__ void __launch_bounds__(kN2vThreads)
    k_walk_n2v(const int32_t *__restrict__ offsets, const int32_t *__restrict__ cols,
               const int32_t *__restrict__ starts, int32_t n_starts, int32_t L, int32_t wpr, N2vThresholds th,
               uint64_t seed, uint32_t round, int32_t *__restrict__ walks, uint32_t *__restrict__ counts) {
    __shared__ int32_t stage[kN2vGroup * kN2vThreads];
    int32_t *buf = stage + threadIdx.x;  // step t0 + i at buf[i * kN2vThreads]
    const double lo_thr = th.near < th.far ? th.near : th.far;
    const double hi_thr = th.near < th.far ? th.far : th.near;
    const bool near_wins = th.near > th.far;  // between the thresholds, accept iff x ~ t does
    const int64_t total = static_cast<int64_t>(n_starts) * wpr;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; w < total; w += stride) {
        const int32_t j = static_cast<int32_t>(w / n_starts);
        const int32_t i = static_cast<int32_t>(w - static_cast<int64_t>(j) * n_starts);
        const int32_t s = __ldg(starts + i);
        const uint32_t x2 = round * static_cast<uint32_t>(wpr) + static_cast<uint32_t>(j);
        int32_t *row = walks + w * L;
        buf[0] = s;
        if (COUNT) atomicAdd(counts + s, 1u);
        int32_t prev = -1, v = s, plo = 0, phi = 0;  // plo, phi: prev's row
        bool alive = true;
        for (int32_t t = 1; t < L; ++t) {
            int32_t nxt = -1;
            if (alive) {
                const int32_t lo = __ldg(offsets + v), hi = __ldg(offsets + v + 1);
                const int64_t deg = static_cast<int64_t>(hi) - lo;
                if (deg == 0) {
                    alive = false;
                } else {
                    for (uint32_t a = 0; a < kN2vAttempts; ++a) {
                        const u32x4 r = philox(seed, static_cast<uint32_t>(t) | (a << 16), static_cast<uint32_t>(s),
                                               x2, kStreamN2v);
                        nxt = __ldg(cols + lo + static_cast<int64_t>(mulhi64(lo64(r), static_cast<uint64_t>(deg))));
                        if (prev < 0) break;  // first step: uniform
                        const double u = static_cast<double>(hi64(r) >> 11) * 0x1p-53;
                        if (nxt == prev) {
                            if (u < th.back) break;
                        } else if (u < lo_thr) {
                            break;
                        } else if (u < hi_thr && in_row(cols, plo, phi, nxt) == near_wins) {
                            break;
                        }
                    }
                    prev = v;
                    plo = lo;
                    phi = hi;
                    v = nxt;
                    if (COUNT) atomicAdd(counts + nxt, 1u);
                }
            }
            buf[(t % kN2vGroup) * kN2vThreads] = nxt;
            if (t % kN2vGroup == kN2vGroup - 1) n2v_flush(row + t - (kN2vGroup - 1), buf, kN2vGroup);
        }
        const int32_t rest = L % kN2vGroup;  // steps still buffered
        if (rest) n2v_flush(row + L - rest, buf, rest);
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
    const N2vThresholds th{ap / amax, 1.0 / amax, aq / amax};
    const int64_t total = static_cast<int64_t>(n_starts) * wp->walks_per_round;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = static_cast<int>(std::min<int64_t>(ceil_div(total, kN2vThreads), static_cast<int64_t>(sm_count()) * 8));
    if (counts)
        k_walk_n2v<true><<<blocks, kN2vThreads, 0, s>>>(g->offsets, g->cols, starts, n_starts, wp->length,
                                                        wp->walks_per_round, th, seed, static_cast<uint32_t>(round),
                                                        walks, counts);
    else
        k_walk_n2v<false><<<blocks, kN2vThreads, 0, s>>>(g->offsets, g->cols, starts, n_starts, wp->length,
                                                         wp->walks_per_round, th, seed, static_cast<uint32_t>(round),
                                                         walks, counts);
    return check_launch("felog_walk_node2vec");
}
