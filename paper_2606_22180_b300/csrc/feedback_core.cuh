// Neighbourhood-consistency score Psi of one node (Eq. 4), shared by the
// single-graph and multi-graph feedback kernels.  See feedback.cu for the
// subset and summation-order rules.
#pragma once

#include "common.cuh"

namespace felog {

constexpr int kMaxKs = 32;

__device__ __forceinline__ double elem(const float *p, int64_t i) { return static_cast<double>(p[i]); }
__device__ __forceinline__ double elem(const __nv_bfloat16 *p, int64_t i) {
    return static_cast<double>(__bfloat162float(p[i]));
}

__device__ __forceinline__ double butterfly(double s) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kFull, s, o));
    return s;
}

// Reduce-scatter of 16 per-lane partial sums over the warp: each total is
// formed from the same pairs of partials as butterfly() (xor distance 16,
// 8, 4, 2, 1), so it is bit-identical to the butterfly's; afterwards lanes
// 2t and 2t + 1 hold total t.
__device__ __forceinline__ double reduce_scatter16_f64(double (&v)[16], int lane) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int dist = 16 >> s;
        const int half = 8 >> s;
        const bool upper = (lane & dist) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double send = upper ? v[i] : v[i + half];
            const double keep = upper ? v[i + half] : v[i];
            v[i] = __dadd_rn(keep, __shfl_xor_sync(kFull, send, dist));
        }
    }
    return __dadd_rn(v[0], __shfl_xor_sync(kFull, v[0], 1));
}

// Psi of node v (deg > 0) on a warp; sub / sorted are this warp's kMaxKs-int
// shared buffers.  Every lane returns the same value.  A neighbour id outside
// [0, n) (a malformed graph) counts as a zero row, so nothing is read out of
// range; on a well-formed graph it never occurs.
template <class T>
__device__ __forceinline__ double psi_node(const int32_t *__restrict__ cols, const T *__restrict__ phi,
                                           int64_t n, int32_t dim, int32_t ks, uint64_t seed, uint32_t round,
                                           int64_t v, int32_t lo, int64_t deg, int32_t *sub, int32_t *sorted) {
    const int lane = threadIdx.x & 31;
    int32_t m;
    if (deg <= ks) {
        m = static_cast<int32_t>(deg);
        if (lane < m) sorted[lane] = lane;
    } else {
        m = ks;
        int64_t t_mine = 0;
        if (lane < ks) {
            const int64_t j = deg - ks + lane;
            const u32x4 r = philox(seed, static_cast<uint32_t>(lane), static_cast<uint32_t>(v), round,
                                   kStreamPsi);
            t_mine = static_cast<int64_t>(mulhi64(lo64(r), static_cast<uint64_t>(j + 1)));
        }
        // Floyd's sequential resolution, on lane 0
        for (int s = 0; s < ks; ++s) {
            const int64_t t = __shfl_sync(kFull, t_mine, s);
            if (lane == 0) {
                bool present = false;
                for (int a = 0; a < s; ++a) present |= sub[a] == t;
                sub[s] = static_cast<int32_t>(present ? deg - ks + s : t);
            }
        }
        __syncwarp();
        if (lane < m) {
            const int32_t x = sub[lane];
            int rank = 0;
            for (int a = 0; a < m; ++a) rank += sub[a] < x;
            sorted[rank] = x;
        }
    }
    __syncwarp();
    // elements l, l+32, ... of phi[v] (dim <= 256, so at most 8 per lane).
    // Products of two float values are exact in binary64, so fma(x, y, s)
    // rounds exactly as s + x * y does: one FP64 instruction per term.
    const T *pv = phi + v * dim;
    const int per_lane = dim >> 5;
    double xv[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xv[c] = c < per_lane ? elem(pv, lane + 32 * c) : 0.0;
    double nv = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < per_lane) nv = __fma_rn(xv[c], xv[c], nv);
    nv = butterfly(nv);
    const double sq_nv = __dsqrt_rn(nv);
    // neighbours in chunks of 8: their row loads overlap, and the 16 partial
    // sums of a chunk (|u|^2 and x.u per neighbour) are reduced together by a
    // reduce-scatter that adds the same pairs as the xor butterfly (so each
    // total is bit-identical to it) with 16 instead of 80 additions per lane;
    // lane 4b then forms the cosine of neighbour b, and the cosines are added
    // in ascending subset order
    constexpr int G = 8;
    double sum = 0.0;
    for (int a0 = 0; a0 < m; a0 += G) {
        const T *pu[G];
        bool inside[G];
#pragma unroll
        for (int b = 0; b < G; ++b) {
            const int32_t u = a0 + b < m ? cols[lo + sorted[a0 + b]] : -1;
            inside[b] = u >= 0 && u < n;
            pu[b] = phi + static_cast<int64_t>(inside[b] ? u : v) * dim;
        }
        double part[2 * G];  // part[2b] = |u_b|^2, part[2b + 1] = x . u_b
#pragma unroll
        for (int i = 0; i < 2 * G; ++i) part[i] = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c >= per_lane) break;
            double y[G];
#pragma unroll
            for (int b = 0; b < G; ++b) y[b] = inside[b] ? elem(pu[b], lane + 32 * c) : 0.0;
#pragma unroll
            for (int b = 0; b < G; ++b) {
                part[2 * b] = __fma_rn(y[b], y[b], part[2 * b]);
                part[2 * b + 1] = __fma_rn(xv[c], y[b], part[2 * b + 1]);
            }
        }
        const double tot = reduce_scatter16_f64(part, lane);  // lanes 2t, 2t+1: total t
        const double d2 = __shfl_down_sync(kFull, tot, 2);    // at lane 4b: x . u_b
        double cs = 0.0;
        const int b_mine = lane >> 2;
        if ((lane & 3) == 0 && a0 + b_mine < m && nv > 0.0 && tot > 0.0)
            cs = __ddiv_rn(d2, __dmul_rn(sq_nv, __dsqrt_rn(tot)));
#pragma unroll
        for (int b = 0; b < G; ++b) {
            const double cb = __shfl_sync(kFull, cs, 4 * b);
            if (a0 + b < m) sum = __dadd_rn(sum, cb);
        }
    }
    const double psi = __ddiv_rn(sum, static_cast<double>(m));
    __syncwarp();
    return psi;
}

}  // namespace felog
