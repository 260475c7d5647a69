// Integer pieces of the unigram^0.75 alias table (Eq. 2's Pn(u)), shared by
// the single-graph builder (noise.cu) and the multi-graph one (batch.cu).
#pragma once

#include "common.cuh"

namespace felog {

typedef unsigned __int128 u128;

constexpr int kNoiseThreads = 256;
constexpr int kNoiseItems = 16;
constexpr int kNoiseTile = kNoiseThreads * kNoiseItems;

struct NoiseAgg {
    u128 D, E;
    int32_t nL, nH;
};

__device__ __forceinline__ double three_quarter_power(uint32_t c) {
    const double x = static_cast<double>(c);
    return __dmul_rn(__dsqrt_rn(x), __dsqrt_rn(__dsqrt_rn(x)));
}

// Per-item classification given S.
__device__ __forceinline__ void classify(uint64_t Wv, uint64_t n, uint64_t S, bool &light,
                                         uint64_t &amount) {
    const uint64_t m = n * Wv;
    light = m < S;
    amount = light ? S - m : m - S;
}

// Table entry of item v from the prefix sums (see noise.cu): a light item
// keeps its mass and points at the first heavy item whose cumulative surplus
// reaches its cumulative deficit; a heavy item that runs dry holds its
// remainder and points at the next heavy item; the rest are full buckets.
__device__ __forceinline__ void alias_entry(int32_t v, uint64_t Wv, uint64_t n, uint64_t S, u128 k,
                                            int32_t rank, const u128 *__restrict__ light_D, int32_t nL,
                                            const int32_t *__restrict__ heavy_idx,
                                            const u128 *__restrict__ heavy_E, int32_t nH, u128 Dtot,
                                            uint64_t *thr, int32_t *alias) {
    const uint64_t m = n * Wv;
    if (m < S) {
        // first heavy with E >= D(i)
        int32_t lo = 0, hi = nH;  // answer in [0, nH)
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (heavy_E[mid] >= k) hi = mid;
            else lo = mid + 1;
        }
        *thr = m;
        *alias = heavy_idx[lo < nH ? lo : nH - 1];
    } else if (k >= Dtot) {
        *thr = S;
        *alias = v;
    } else {
        // first light with D > E(j)
        int32_t lo = 0, hi = nL;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (light_D[mid] > k) hi = mid;
            else lo = mid + 1;
        }
        const u128 Dc = lo < nL ? light_D[lo] : Dtot;
        *thr = S - static_cast<uint64_t>(Dc - k);
        const int32_t r = rank + 1;
        *alias = heavy_idx[r < nH ? r : nH - 1];
    }
}

}  // namespace felog
