// Noise distribution Pn(u) of Eq. 2 as an exact integer alias table.
//
// Weights: W_v = c_v ? max(1, floor(c_v^0.75 / cmax^0.75 * 2^32)) : 0 with
// c^0.75 = sqrt(c) * sqrt(sqrt(c)) in binary64 (each operation correctly
// rounded); S = sum W.  With masses m_v = n W_v, item v is light if m_v < S
// and heavy otherwise; light deficit d_v = S - m_v, heavy surplus
// e_v = m_v - S.
//
// The table is the one produced by the sequential sweep (a light cursor and
// a heavy cursor moving up in index order; the current heavy item fills light
// buckets until its remaining mass drops below S, then fills its own bucket
// with that remainder and hands its deficit to the next heavy item).  That
// sweep is a merge of two prefix sums, which is what makes it parallel
// (Huebschle-Schneider and Sanders, "Parallel Weighted Random Sampling",
// ESA 2019).  With D(i) = sum of deficits of lights before i and
// E(j) = sum of surpluses of heavies up to and including j:
//   light i : thr = m_i, alias = first heavy j with E(j) >= D(i)
//   heavy j : if E(j) >= D_total : thr = S, alias = j
//             else thr = S - (D(i*) - E(j)), alias = next heavy after j,
//                  i* = first light with D(i*) > E(j) (D_total if none).
// Prefix sums can exceed 2^64, so they are carried in unsigned __int128.
// Everything is integer, so the table is identical to the sequential one.
#include "noise_core.cuh"

namespace felog {

__global__ void k_noise_max(const uint32_t *__restrict__ counts, int32_t n, uint32_t *__restrict__ cmax) {
    uint32_t m = 0;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x)
        m = max(m, counts[v]);
    m = __reduce_max_sync(kFull, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(cmax, m);
}

__global__ void k_noise_weights(const uint32_t *__restrict__ counts, int32_t n,
                                const uint32_t *__restrict__ cmax, uint64_t *__restrict__ W,
                                unsigned long long *__restrict__ S) {
    const uint32_t cm = *cmax;
    const double wmax = cm ? three_quarter_power(cm) : 1.0;
    unsigned long long local = 0;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t c = counts[v];
        uint64_t w = 0;
        if (c) {
            const double q = floor(__dmul_rn(__ddiv_rn(three_quarter_power(c), wmax), 4294967296.0));
            w = static_cast<uint64_t>(q);
            if (w < 1) w = 1;
        }
        W[v] = w;
        local += w;
    }
    // warp sum of 64-bit values
    for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(S, local);
}

__global__ void __launch_bounds__(kNoiseThreads)
    k_noise_tile_agg(const uint64_t *__restrict__ W, int32_t n, const unsigned long long *__restrict__ Sp,
                     NoiseAgg *__restrict__ tile_agg) {
    __shared__ NoiseAgg part[kNoiseThreads];
    const uint64_t S = *Sp;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kNoiseTile;
    NoiseAgg a{0, 0, 0, 0};
    for (int k = 0; k < kNoiseItems; ++k) {
        const int64_t v = base + static_cast<int64_t>(k) * kNoiseThreads + threadIdx.x;
        if (v >= n) break;
        bool light;
        uint64_t amt;
        classify(W[v], static_cast<uint64_t>(n), S, light, amt);
        if (light) { a.D += amt; a.nL += 1; }
        else { a.E += amt; a.nH += 1; }
    }
    part[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        NoiseAgg t{0, 0, 0, 0};
        for (int i = 0; i < kNoiseThreads; ++i) {
            t.D += part[i].D; t.E += part[i].E; t.nL += part[i].nL; t.nH += part[i].nH;
        }
        tile_agg[blockIdx.x] = t;
    }
}

// exclusive scan of tile aggregates (serial; a few thousand tiles at most)
__global__ void k_noise_tile_scan(NoiseAgg *__restrict__ tile_agg, int32_t n_tiles,
                                  NoiseAgg *__restrict__ total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    NoiseAgg run{0, 0, 0, 0};
    for (int32_t t = 0; t < n_tiles; ++t) {
        const NoiseAgg x = tile_agg[t];
        tile_agg[t] = run;
        run.D += x.D; run.E += x.E; run.nL += x.nL; run.nH += x.nH;
    }
    *total = run;
}

// Per item: D(i) (lights, exclusive) or E(j) (heavies, inclusive), the
// compacted light-D list and heavy (index, E) lists, heavy ranks.
__global__ void __launch_bounds__(kNoiseThreads)
    k_noise_scatter(const uint64_t *__restrict__ W, int32_t n, const unsigned long long *__restrict__ Sp,
                    const NoiseAgg *__restrict__ tile_off, u128 *__restrict__ key,
                    int32_t *__restrict__ rank, u128 *__restrict__ light_D,
                    int32_t *__restrict__ heavy_idx, u128 *__restrict__ heavy_E) {
    __shared__ NoiseAgg part[kNoiseThreads];
    const uint64_t S = *Sp;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kNoiseTile +
                         static_cast<int64_t>(threadIdx.x) * kNoiseItems;  // contiguous items
    NoiseAgg a{0, 0, 0, 0};
    for (int k = 0; k < kNoiseItems; ++k) {
        const int64_t v = base + k;
        if (v >= n) break;
        bool light;
        uint64_t amt;
        classify(W[v], static_cast<uint64_t>(n), S, light, amt);
        if (light) { a.D += amt; a.nL += 1; }
        else { a.E += amt; a.nH += 1; }
    }
    part[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        NoiseAgg run = tile_off[blockIdx.x];
        for (int i = 0; i < kNoiseThreads; ++i) {
            const NoiseAgg x = part[i];
            part[i] = run;
            run.D += x.D; run.E += x.E; run.nL += x.nL; run.nH += x.nH;
        }
    }
    __syncthreads();
    NoiseAgg run = part[threadIdx.x];
    for (int k = 0; k < kNoiseItems; ++k) {
        const int64_t v = base + k;
        if (v >= n) break;
        bool light;
        uint64_t amt;
        classify(W[v], static_cast<uint64_t>(n), S, light, amt);
        if (light) {
            key[v] = run.D;  // exclusive
            light_D[run.nL] = run.D;
            rank[v] = run.nL;
            run.D += amt;
            run.nL += 1;
        } else {
            run.E += amt;
            key[v] = run.E;  // inclusive
            heavy_idx[run.nH] = static_cast<int32_t>(v);
            heavy_E[run.nH] = run.E;
            rank[v] = run.nH;
            run.nH += 1;
        }
    }
}

__global__ void k_noise_finish(const uint64_t *__restrict__ W, int32_t n,
                               const unsigned long long *__restrict__ Sp,
                               const NoiseAgg *__restrict__ total, const u128 *__restrict__ key,
                               const int32_t *__restrict__ rank, const u128 *__restrict__ light_D,
                               const int32_t *__restrict__ heavy_idx,
                               const u128 *__restrict__ heavy_E, uint64_t *__restrict__ thr,
                               int32_t *__restrict__ alias) {
    const uint64_t S = *Sp;
    const int32_t nL = total->nL, nH = total->nH;
    const u128 Dtot = total->D;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (S == 0) {
            thr[v] = 0;
            alias[v] = static_cast<int32_t>(v);
            continue;
        }
        alias_entry(static_cast<int32_t>(v), W[v], static_cast<uint64_t>(n), S, key[v], rank[v], light_D, nL,
                    heavy_idx, heavy_E, nH, Dtot, thr + v, alias + v);
    }
}

struct NoiseWorkspace {
    uint32_t *cmax;
    NoiseAgg *total;
    NoiseAgg *tile;
    uint64_t *W;
    u128 *key;
    int32_t *rank;
    u128 *light_D;
    int32_t *heavy_idx;
    u128 *heavy_E;
};

static NoiseWorkspace carve_noise(Carver &c, int32_t n) {
    NoiseWorkspace w;
    const int tiles = n > 0 ? ceil_div(n, kNoiseTile) : 1;
    const size_t nn = n > 0 ? static_cast<size_t>(n) : 1;
    w.cmax = c.take<uint32_t>(1);
    w.total = c.take<NoiseAgg>(1);
    w.tile = c.take<NoiseAgg>(tiles);
    w.W = c.take<uint64_t>(nn);
    w.key = c.take<u128>(nn);
    w.rank = c.take<int32_t>(nn);
    w.light_D = c.take<u128>(nn);
    w.heavy_idx = c.take<int32_t>(nn);
    w.heavy_E = c.take<u128>(nn);
    return w;
}

int sm_count();

}  // namespace felog

using namespace felog;

extern "C" size_t felog_noise_workspace_bytes(int32_t n) {
    Carver c(nullptr, 0);
    carve_noise(c, n);
    return align_up(c.used, 256);
}

extern "C" felog_status felog_noise_table(const uint32_t *counts, int32_t n, uint64_t *thr,
                                          int32_t *alias, uint64_t *S, void *workspace,
                                          size_t workspace_bytes, void *stream) {
    if (n < 0 || !S || (n > 0 && (!counts || !thr || !alias))) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_noise_workspace_bytes(n)) return FELOG_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    NoiseWorkspace w = carve_noise(c, n);
    unsigned long long *Sd = reinterpret_cast<unsigned long long *>(S);
    felog_status st = record_cuda_error(cudaMemsetAsync(w.cmax, 0, sizeof(uint32_t), s), "noise");
    if (st) return st;
    st = record_cuda_error(cudaMemsetAsync(Sd, 0, sizeof(uint64_t), s), "noise");
    if (st || n == 0) return st;
    const int grid = std::min(ceil_div(n, 256), sm_count() * 8);
    const int tiles = ceil_div(n, kNoiseTile);
    k_noise_max<<<grid, 256, 0, s>>>(counts, n, w.cmax);
    k_noise_weights<<<grid, 256, 0, s>>>(counts, n, w.cmax, w.W, Sd);
    k_noise_tile_agg<<<tiles, kNoiseThreads, 0, s>>>(w.W, n, Sd, w.tile);
    k_noise_tile_scan<<<1, 32, 0, s>>>(w.tile, tiles, w.total);
    k_noise_scatter<<<tiles, kNoiseThreads, 0, s>>>(w.W, n, Sd, w.tile, w.key, w.rank, w.light_D,
                                                     w.heavy_idx, w.heavy_E);
    k_noise_finish<<<grid, 256, 0, s>>>(w.W, n, Sd, w.total, w.key, w.rank, w.light_D, w.heavy_idx,
                                         w.heavy_E, thr, alias);
    return check_launch("felog_noise_table");
}
