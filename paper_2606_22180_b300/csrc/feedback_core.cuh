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
    const T *pv = phi + v * dim;
    double nv = 0.0;
    for (int i = lane; i < dim; i += 32) {
        const double x = elem(pv, i);
        nv = __dadd_rn(nv, __dmul_rn(x, x));
    }
    nv = butterfly(nv);
    double sum = 0.0;
    for (int a = 0; a < m; ++a) {
        const int32_t u = cols[lo + sorted[a]];
        const T *pu = phi + static_cast<int64_t>(u) * dim;
        double nu = 0.0, dt = 0.0;
        for (int i = lane; i < dim; i += 32) {
            const double y = elem(pu, i);
            nu = __dadd_rn(nu, __dmul_rn(y, y));
            dt = __dadd_rn(dt, __dmul_rn(elem(pv, i), y));
        }
        nu = butterfly(nu);
        dt = butterfly(dt);
        double cs = 0.0;
        if (nv > 0.0 && nu > 0.0) cs = __ddiv_rn(dt, __dmul_rn(__dsqrt_rn(nv), __dsqrt_rn(nu)));
        sum = __dadd_rn(sum, cs);
    }
    const double psi = __ddiv_rn(sum, static_cast<double>(m));
    __syncwarp();
    return psi;
}

}  // namespace felog
