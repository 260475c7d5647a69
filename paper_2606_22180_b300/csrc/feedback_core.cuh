// Neighbourhood-consistency score Psi of one node (Eq. 4), shared by the
// single-graph and multi-graph feedback kernels.  See feedback.cu for the
// subset and summation-order rules.
#pragma once

#include "common.cuh"

namespace felog {

constexpr int kMaxKs = 32;

// binary32 -> binary64, exactly, by moving the fields of a normal number:
// the sign stays, the 8-bit exponent is rebiased by 1023 - 127 = 896 into
// 11 bits, and the 23 fraction bits become the top of the 52.  This keeps the
// conversions (one per row element) off the FP64 pipe, which on this GPU
// issues two instructions per clock per SM and is what bounds Psi.  Zeros,
// subnormals, infinities and NaNs take the ordinary conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e - 1u >= 254u) return static_cast<double>(f);
    const uint32_t hi = (b & 0x80000000u) | (((b >> 3) & 0x0fffffffu) + (896u << 20));
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(b << 29));
}

__device__ __forceinline__ double elem(const float *p, int64_t i) { return f32_to_f64(p[i]); }
__device__ __forceinline__ double elem(const __nv_bfloat16 *p, int64_t i) {
    return f32_to_f64(__bfloat162float(p[i]));
}

__device__ __forceinline__ double butterfly(double s) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kFull, s, o));
    return s;
}

// Reduce-scatter of the first NP (2, 4, 8 or 16) per-lane partial sums over
// the warp: each total is formed from the same pairs of partials as
// butterfly() (xor distance 16, 8, 4, 2, 1), so it is bit-identical to the
// butterfly's.  The first log2(NP) levels halve the partials a lane carries,
// the remaining levels add the one it keeps; afterwards the 32 / NP lanes
// lane / (32 / NP) == t hold total t.
template <int NP>
__device__ __forceinline__ double reduce_scatter_f64(double (&v)[16], int lane) {
    constexpr int S = NP == 16 ? 4 : NP == 8 ? 3 : NP == 4 ? 2 : 1;
    static_assert(NP == 2 << (S - 1), "NP: 2, 4, 8 or 16");
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int dist = 16 >> s;
        const int half = (NP / 2) >> s;
        const bool upper = (lane & dist) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double send = upper ? v[i] : v[i + half];
            const double keep = upper ? v[i + half] : v[i];
            v[i] = __dadd_rn(keep, __shfl_xor_sync(kFull, send, dist));
        }
    }
    double t = v[0];
#pragma unroll
    for (int d = 16 >> S; d >= 1; d >>= 1) t = __dadd_rn(t, __shfl_xor_sync(kFull, t, d));
    return t;
}

// Psi is computed for a group of nodes on one warp in two parts.
//
// psi_node_totals (per node, all lanes): the neighbour subset, |x|^2 and,
// for each subset neighbour u_a, |u_a|^2 and x . u_a, each a binary64 sum in
// the fixed order; they are left in the warp's scratch.
//
// psi_group_finish (per group): the cosines of every (node, neighbour) slot,
// one slot per lane, then on lane i the mean of node i's cosines in
// ascending subset order.  The square roots and divisions of a node thus run
// on one lane instead of the whole warp, with the same operations in the
// same order, so the values are those of the one-node-per-warp form bit for
// bit.
//
// Scratch of one warp (shared memory): nv[kPsiGroup] = |x|^2 per node,
// m[kPsiGroup] = subset size (0: not evaluated), and u2 / xu
// [kPsiGroup * ks <= kPsiSlots]: the totals of slot i * ks + a.
constexpr int kPsiGroup = 32;
constexpr int kPsiSlots = 256;

__host__ __device__ inline int psi_group_size(int ks) { return ks * kPsiGroup <= kPsiSlots ? kPsiGroup : kPsiSlots / ks; }

struct PsiScratch {
    double nv[kPsiGroup];
    double u2[kPsiSlots];
    double xu[kPsiSlots];
    int32_t m[kPsiGroup];
    int32_t sub[kMaxKs];
    int32_t sorted[kMaxKs];
};

// Totals of node v (deg > 0) into slot row `row` of the scratch; returns the
// subset size.  A neighbour id outside [0, n) (a malformed graph) counts as a
// zero row, so nothing is read out of range; on a well-formed graph it never
// occurs.
template <class T>
__device__ __forceinline__ int32_t psi_node_totals(const int32_t *__restrict__ cols, const T *__restrict__ phi,
                                                   int64_t n, int32_t dim, int32_t ks, uint64_t seed, uint32_t round,
                                                   int64_t v, int32_t lo, int64_t deg, PsiScratch &w, int row) {
    const int lane = threadIdx.x & 31;
    int32_t *sub = w.sub, *sorted = w.sorted;
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
    if (lane == 0) w.nv[row] = nv;
    // neighbours in chunks of 8: their row loads overlap, and the partial
    // sums of a chunk (|u|^2 and x.u per neighbour) are reduced together by a
    // reduce-scatter that adds the same pairs as the xor butterfly (so each
    // total is bit-identical to it) with 16 instead of 80 additions per lane
    // for a full chunk
    constexpr int G = 8;
    double *u2 = w.u2 + row * ks;
    double *xu = w.xu + row * ks;
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
        // slots past the subset (m - a0 < G, warp-uniform) keep their zero
        // partials: the FMAs they would run add +0 exactly, so they are skipped
        const int live = min(G, m - a0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c >= per_lane) break;
            double y[G];
#pragma unroll
            for (int b = 0; b < G; ++b) y[b] = b < live && inside[b] ? elem(pu[b], lane + 32 * c) : 0.0;
#pragma unroll
            for (int b = 0; b < G; ++b) {
                if (b >= live) break;
                part[2 * b] = __fma_rn(y[b], y[b], part[2 * b]);
                part[2 * b + 1] = __fma_rn(xv[c], y[b], part[2 * b + 1]);
            }
        }
        // only the 2 * live partials of the live slots are reduced (fewer
        // halving levels for a short chunk; the same tree for each total)
        double tot;
        int grp;  // lanes per total: total t sits in lanes [t * grp, t * grp + grp)
        if (live > 4) {
            tot = reduce_scatter_f64<16>(part, lane);
            grp = 2;
        } else if (live > 2) {
            tot = reduce_scatter_f64<8>(part, lane);
            grp = 4;
        } else if (live > 1) {
            tot = reduce_scatter_f64<4>(part, lane);
            grp = 8;
        } else {
            tot = reduce_scatter_f64<2>(part, lane);
            grp = 16;
        }
        // total 2b is |u_b|^2, total 2b + 1 is x . u_b
        const int t_mine = lane / grp;
        const int b_mine = t_mine >> 1;
        if (lane % grp == 0 && b_mine < live) ((t_mine & 1) ? xu : u2)[a0 + b_mine] = tot;
    }
    if (lane == 0) w.m[row] = m;
    __syncwarp();
    return m;
}

// Cosines and means of rows 0..count-1 (count <= psi_group_size(ks)); lane i
// < count returns Psi of row i (NaN where m[i] == 0, a node not evaluated).
__device__ __forceinline__ double psi_group_finish(PsiScratch &w, int count, int32_t ks) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    // cos = x.u / (sqrt(|x|^2) * sqrt(|u|^2)), 0 for a zero row; written over xu
    for (int s = lane; s < count * ks; s += 32) {
        const int i = s / ks, a = s - i * ks;
        if (a < w.m[i]) {
            const double nv = w.nv[i], tot = w.u2[s];
            double cs = 0.0;
            if (nv > 0.0 && tot > 0.0) cs = __ddiv_rn(w.xu[s], __dmul_rn(__dsqrt_rn(nv), __dsqrt_rn(tot)));
            w.xu[s] = cs;
        }
    }
    __syncwarp();
    double psi = __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
    if (lane < count) {
        const int32_t m = w.m[lane];
        if (m > 0) {
            const double *cs = w.xu + lane * ks;
            double sum = 0.0;
            for (int a = 0; a < m; ++a) sum = __dadd_rn(sum, cs[a]);
            psi = __ddiv_rn(sum, static_cast<double>(m));
        }
    }
    __syncwarp();
    return psi;
}

}  // namespace felog
