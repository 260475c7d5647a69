// One uniform truncated walk (Section 2; Algorithm 1, Sampling), shared by
// the single-graph and multi-graph walk kernels.
#pragma once

#include "common.cuh"

namespace felog {

// Fills row[0..L) with the walk from local node s keyed by x2 (= round * wpr
// + rep): step t >= 1 draws Philox(x0=t, x1=s, x2, stream 0) and moves to
// neighbour floor(u64 * deg / 2^64).  A node without neighbours ends the walk
// and the rest of the row is -1.  COUNT adds every written node to counts[];
// VEC stores 4 steps at a time (L % 4 == 0, row 16-byte aligned).
// Guards (a graph of n nodes and nnz columns): a start outside [0, n) gives a
// row of -1; a row whose offsets leave [0, nnz] ends the walk like a node
// without neighbours; a column outside [0, n) ends it before it is written.
// On a well-formed graph none of them changes a walk.
template <bool COUNT, bool VEC>
__device__ __forceinline__ void walk_fill_row(const int32_t *__restrict__ offsets,
                                              const int32_t *__restrict__ cols, int32_t n, int64_t nnz,
                                              int32_t s, int32_t L, uint64_t seed, uint32_t x2,
                                              int32_t *__restrict__ row, uint32_t *__restrict__ counts) {
    int32_t v = s;
    bool alive = s >= 0 && s < n;
    if (!alive) s = -1;
    if (COUNT && alive) atomicAdd(counts + s, 1u);
    if (VEC) {
        int4 buf;
        buf.x = s;
        for (int32_t t0 = 0; t0 < L; t0 += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t t = t0 + u;
                if (t == 0) continue;
                int32_t nxt = -1;
                if (alive) {
                    const int32_t lo = __ldg(offsets + v), hi = __ldg(offsets + v + 1);
                    const int64_t deg = static_cast<int64_t>(hi) - lo;
                    if (deg <= 0 || lo < 0 || hi > nnz) {
                        alive = false;
                    } else {
                        const u32x4 r = philox(seed, static_cast<uint32_t>(t),
                                               static_cast<uint32_t>(s), x2, kStreamWalk);
                        const uint64_t idx = mulhi64(lo64(r), static_cast<uint64_t>(deg));
                        nxt = __ldg(cols + lo + static_cast<int64_t>(idx));
                        if (nxt < 0 || nxt >= n) {
                            nxt = -1;
                            alive = false;
                        } else {
                            v = nxt;
                            if (COUNT) atomicAdd(counts + nxt, 1u);
                        }
                    }
                }
                if (u == 0) buf.x = nxt;
                if (u == 1) buf.y = nxt;
                if (u == 2) buf.z = nxt;
                if (u == 3) buf.w = nxt;
            }
            *reinterpret_cast<int4 *>(row + t0) = buf;
        }
    } else {
        row[0] = s;
        for (int32_t t = 1; t < L; ++t) {
            int32_t nxt = -1;
            if (alive) {
                const int32_t lo = __ldg(offsets + v), hi = __ldg(offsets + v + 1);
                const int64_t deg = static_cast<int64_t>(hi) - lo;
                if (deg <= 0 || lo < 0 || hi > nnz) {
                    alive = false;
                } else {
                    const u32x4 r = philox(seed, static_cast<uint32_t>(t),
                                           static_cast<uint32_t>(s), x2, kStreamWalk);
                    const uint64_t idx = mulhi64(lo64(r), static_cast<uint64_t>(deg));
                    nxt = __ldg(cols + lo + static_cast<int64_t>(idx));
                    if (nxt < 0 || nxt >= n) {
                        nxt = -1;
                        alive = false;
                    } else {
                        v = nxt;
                        if (COUNT) atomicAdd(counts + nxt, 1u);
                    }
                }
            }
            row[t] = nxt;
        }
    }
}

// M walks of one thread in lockstep (walk m from local node s[m], keyed by
// x2[m], into rows[m]; only the first nm are real): the same steps as
// walk_fill_row for each, with the M walks' dependent loads in flight
// together, so a thread hides M times the memory latency of one walk.
template <bool COUNT, int M>
__device__ __forceinline__ void walk_fill_rows_vec(const int32_t *__restrict__ offsets,
                                                   const int32_t *__restrict__ cols, int32_t n, int64_t nnz,
                                                   const int32_t (&s_in)[M], int nm, int32_t L, uint64_t seed,
                                                   const uint32_t (&x2)[M], int32_t *const (&rows)[M],
                                                   uint32_t *__restrict__ counts) {
    int32_t s[M], v[M];
    bool alive[M];
    int4 buf[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        s[m] = s_in[m];
        alive[m] = m < nm && s[m] >= 0 && s[m] < n;
        if (!alive[m]) s[m] = -1;
        v[m] = s[m];
        if (COUNT && alive[m]) atomicAdd(counts + s[m], 1u);
        buf[m].x = s[m];
    }
    for (int32_t t0 = 0; t0 < L; t0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int32_t t = t0 + u;
            if (t == 0) continue;
            int32_t lo[M], hi[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                lo[m] = 0;
                hi[m] = 0;
                if (alive[m]) {
                    lo[m] = __ldg(offsets + v[m]);
                    hi[m] = __ldg(offsets + v[m] + 1);
                }
            }
            int32_t nxt[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                nxt[m] = -1;
                if (alive[m]) {
                    const int64_t deg = static_cast<int64_t>(hi[m]) - lo[m];
                    if (deg <= 0 || lo[m] < 0 || hi[m] > nnz) {
                        alive[m] = false;
                    } else {
                        const u32x4 r = philox(seed, static_cast<uint32_t>(t), static_cast<uint32_t>(s[m]), x2[m],
                                               kStreamWalk);
                        const uint64_t idx = mulhi64(lo64(r), static_cast<uint64_t>(deg));
                        nxt[m] = __ldg(cols + lo[m] + static_cast<int64_t>(idx));
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (alive[m]) {
                    if (nxt[m] < 0 || nxt[m] >= n) {
                        nxt[m] = -1;
                        alive[m] = false;
                    } else {
                        v[m] = nxt[m];
                        if (COUNT) atomicAdd(counts + nxt[m], 1u);
                    }
                }
                if (u == 0) buf[m].x = nxt[m];
                if (u == 1) buf[m].y = nxt[m];
                if (u == 2) buf[m].z = nxt[m];
                if (u == 3) buf[m].w = nxt[m];
            }
        }
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m < nm) *reinterpret_cast<int4 *>(rows[m] + t0) = buf[m];
    }
}

}  // namespace felog
