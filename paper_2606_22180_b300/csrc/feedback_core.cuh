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

// Psi of node v (deg > 0) on a warp; sub / sorted are this warp's kMaxKs-int
// shared buffers.  Every lane returns the same value.
template <class T>
__device__ __forceinline__ double psi_node(const int32_t *__restrict__ cols, const T *__restrict__ phi,
                                           int32_t dim, int32_t ks, uint64_t seed, uint32_t round, int64_t v,
                                           int32_t lo, int64_t deg, int32_t *sub, int32_t *sorted) {
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
    // elements l, l+32, ... of phi[v] (dim <= 256, so at most 8 per lane)
    const T *pv = phi + v * dim;
    const int per_lane = dim >> 5;
    double xv[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xv[c] = c < per_lane ? elem(pv, lane + 32 * c) : 0.0;
    double nv = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < per_lane) nv = __dadd_rn(nv, __dmul_rn(xv[c], xv[c]));
    nv = butterfly(nv);
    // neighbours in groups of 4 so that their row loads overlap; each dot
    // product keeps the fixed per-lane order and butterfly, and the cosines
    // are added in ascending subset order
    constexpr int G = 4;
    double sum = 0.0;
    for (int a0 = 0; a0 < m; a0 += G) {
        const T *pu[G];
#pragma unroll
        for (int b = 0; b < G; ++b) {
            const int32_t u = a0 + b < m ? cols[lo + sorted[a0 + b]] : 0;
            pu[b] = phi + static_cast<int64_t>(u) * dim;
        }
        double nu[G], dt[G];
#pragma unroll
        for (int b = 0; b < G; ++b) nu[b] = dt[b] = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c >= per_lane) break;
            double y[G];
#pragma unroll
            for (int b = 0; b < G; ++b) y[b] = elem(pu[b], lane + 32 * c);
#pragma unroll
            for (int b = 0; b < G; ++b) {
                nu[b] = __dadd_rn(nu[b], __dmul_rn(y[b], y[b]));
                dt[b] = __dadd_rn(dt[b], __dmul_rn(xv[c], y[b]));
            }
        }
#pragma unroll
        for (int b = 0; b < G; ++b) {
            if (a0 + b >= m) break;
            const double n2 = butterfly(nu[b]);
            const double d2 = butterfly(dt[b]);
            double cs = 0.0;
            if (nv > 0.0 && n2 > 0.0) cs = __ddiv_rn(d2, __dmul_rn(__dsqrt_rn(nv), __dsqrt_rn(n2)));
            sum = __dadd_rn(sum, cs);
        }
    }
    const double psi = __ddiv_rn(sum, static_cast<double>(m));
    __syncwarp();
    return psi;
}

}  // namespace felog
