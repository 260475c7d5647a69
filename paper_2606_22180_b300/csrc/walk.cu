// Sample: active-set compaction and uniform truncated random walks.
//
// Section 2 ("Sampling process") and Algorithm 1 (Sampling over V_a).  One
// thread runs one walker; a warp owns 32 consecutive walkers, so the start
// list is read coalesced and the warp's output rows are contiguous.  Each
// step is two dependent gathers (offsets[v], offsets[v+1] then cols[...]),
// the latency chain that bounds the kernel; the Philox block of the step is
// computed while the previous gather is in flight.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "walk_core.cuh"

namespace felog {

static thread_local char g_last_error[256] = "";

felog_status record_cuda_error(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return FELOG_OK;
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", where, cudaGetErrorString(e));
    return FELOG_ERR_CUDA;
}

felog_status check_launch(const char *where) { return record_cuda_error(cudaGetLastError(), where); }

// ---------------------------------------------------------------------------
// Stable compaction of active flags (three phases: tile counts, scan of tile
// counts in one block, local scan + scatter).
// ---------------------------------------------------------------------------
constexpr int kCompactThreads = 256;
constexpr int kCompactItems = 16;
constexpr int kCompactTile = kCompactThreads * kCompactItems;

__global__ void __launch_bounds__(kCompactThreads)
    k_compact_count(const uint8_t *__restrict__ active, int32_t n, int32_t *__restrict__ tile_count) {
    __shared__ int32_t warp_sum[kCompactThreads / 32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kCompactTile;
    int32_t c = 0;
    for (int i = threadIdx.x; i < kCompactTile; i += kCompactThreads) {
        const int64_t v = base + i;
        if (v < n) c += active[v] != 0;
    }
    c = __reduce_add_sync(kFull, c);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t s = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) s += warp_sum[w];
        tile_count[blockIdx.x] = s;
    }
}

// exclusive scan of tile counts in place; total to *n_active
__global__ void __launch_bounds__(1024)
    k_compact_scan(int32_t *__restrict__ tile_count, int32_t n_tiles, int32_t *__restrict__ n_active) {
    __shared__ int32_t carry_s;
    __shared__ int32_t warp_tot[32];
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int32_t base = 0; base < n_tiles; base += 1024) {
        const int32_t i = base + threadIdx.x;
        const int32_t x = i < n_tiles ? tile_count[i] : 0;
        int32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if ((threadIdx.x & 31) >= o) incl += y;
        }
        if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            int32_t t = warp_tot[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, t, o);
                if (threadIdx.x >= o) t += y;
            }
            warp_tot[threadIdx.x] = t;  // inclusive
        }
        __syncthreads();
        const int32_t warp_excl = (threadIdx.x >> 5) ? warp_tot[(threadIdx.x >> 5) - 1] : 0;
        const int32_t carry = carry_s;
        if (i < n_tiles) tile_count[i] = carry + warp_excl + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + warp_tot[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_active = carry_s;
}

__global__ void __launch_bounds__(kCompactThreads)
    k_compact_scatter(const uint8_t *__restrict__ active, int32_t n,
                      const int32_t *__restrict__ tile_offset, int32_t *__restrict__ starts) {
    __shared__ int32_t warp_tot[kCompactThreads / 32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kCompactTile;
    // thread t owns items [t*kCompactItems, (t+1)*kCompactItems) of the tile
    const int64_t my = base + static_cast<int64_t>(threadIdx.x) * kCompactItems;
    uint32_t bits = 0;
#pragma unroll
    for (int k = 0; k < kCompactItems; ++k) {
        const int64_t v = my + k;
        if (v < n && active[v]) bits |= 1u << k;
    }
    const int32_t c = __popc(bits);
    int32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, incl, o);
        if ((threadIdx.x & 31) >= o) incl += y;
    }
    if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = incl;
    __syncthreads();
    int32_t warp_excl = 0;
    for (int w = 0; w < (threadIdx.x >> 5); ++w) warp_excl += warp_tot[w];
    int32_t pos = tile_offset[blockIdx.x] + warp_excl + incl - c;
    while (bits) {
        const int k = __ffs(bits) - 1;
        bits &= bits - 1;
        starts[pos++] = static_cast<int32_t>(my + k);
    }
}

}  // namespace felog

using namespace felog;

extern "C" size_t felog_compact_workspace_bytes(int32_t n) {
    const int tiles = n > 0 ? ceil_div(n, kCompactTile) : 1;
    return align_up(sizeof(int32_t) * static_cast<size_t>(tiles), 256);
}

extern "C" felog_status felog_compact_active(const uint8_t *active, int32_t n, int32_t *starts,
                                             int32_t *n_active, void *workspace,
                                             size_t workspace_bytes, void *stream) {
    if (n < 0 || !n_active || (n > 0 && (!active || !starts))) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_compact_workspace_bytes(n)) return FELOG_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        return record_cuda_error(cudaMemsetAsync(n_active, 0, sizeof(int32_t), s), "compact");
    }
    const int tiles = ceil_div(n, kCompactTile);
    int32_t *tile = static_cast<int32_t *>(workspace);
    k_compact_count<<<tiles, kCompactThreads, 0, s>>>(active, n, tile);
    k_compact_scan<<<1, 1024, 0, s>>>(tile, tiles, n_active);
    k_compact_scatter<<<tiles, kCompactThreads, 0, s>>>(active, n, tile, starts);
    return check_launch("felog_compact_active");
}

// ---------------------------------------------------------------------------
// Allocation-free compaction.  Same kernels as felog_compact_active; the
// per-tile counts live in a file-scope device array instead of a caller
// workspace, so a caller that may not allocate device memory can still run
// the compaction.  Every tile slot a call uses is written by k_compact_count
// before it is read, so nothing needs clearing between calls.
// ---------------------------------------------------------------------------
namespace felog {

constexpr int kNoAllocMaxTiles = 4096;  // 4096 tiles x 4096 flags = 2^24 nodes
static __device__ __align__(256) int32_t g_compact_tiles[kNoAllocMaxTiles];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static int32_t *g_noalloc_tiles[kMaxDevices] = {};

// Device address of g_compact_tiles for the current device (host code can
// only name the symbol, not its device address).
static felog_status noalloc_tiles(int32_t **out) {
    int dev = 0;
    felog_status st = record_cuda_error(cudaGetDevice(&dev), "compact_noalloc");
    if (st) return st;
    if (dev < 0 || dev >= kMaxDevices) return FELOG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_tiles[dev]) {
        void *p = nullptr;
        st = record_cuda_error(cudaGetSymbolAddress(&p, g_compact_tiles), "cudaGetSymbolAddress");
        if (st) return st;
        g_noalloc_tiles[dev] = static_cast<int32_t *>(p);
    }
    *out = g_noalloc_tiles[dev];
    return FELOG_OK;
}

}  // namespace felog

extern "C" int32_t felog_compact_active_noalloc_max_n(void) {
    return static_cast<int32_t>(kNoAllocMaxTiles) * kCompactTile;
}

extern "C" felog_status felog_compact_active_noalloc(const uint8_t *active, int32_t n, int32_t *starts,
                                                     int32_t *n_active, void *stream) {
    if (n < 0 || !n_active || (n > 0 && (!active || !starts))) return FELOG_ERR_INVALID_ARG;
    if (n > felog_compact_active_noalloc_max_n()) return FELOG_ERR_INVALID_ARG;
    int32_t *tile = nullptr;
    felog_status st = noalloc_tiles(&tile);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) return record_cuda_error(cudaMemsetAsync(n_active, 0, sizeof(int32_t), s), "compact");
    const int tiles = ceil_div(n, kCompactTile);
    k_compact_count<<<tiles, kCompactThreads, 0, s>>>(active, n, tile);
    k_compact_scan<<<1, 1024, 0, s>>>(tile, tiles, n_active);
    k_compact_scatter<<<tiles, kCompactThreads, 0, s>>>(active, n, tile, starts);
    return check_launch("felog_compact_active_noalloc");
}

// ---------------------------------------------------------------------------
// Walk kernel.
// ---------------------------------------------------------------------------
namespace felog {

constexpr int kWalkThreads = 256;

// One walker per thread.  VEC: row length is a multiple of 4, rows 16-byte
// aligned, output buffered 4 steps at a time and stored as one int4.
template <bool COUNT, bool VEC>
__global__ void __launch_bounds__(kWalkThreads)
    k_walk(const int32_t *__restrict__ offsets, const int32_t *__restrict__ cols, int32_t n, int64_t nnz,
           const int32_t *__restrict__ starts, int32_t n_starts, int32_t L, int32_t wpr,
           uint64_t seed, uint32_t round, int32_t *__restrict__ walks,
           uint32_t *__restrict__ counts) {
    const int64_t total = static_cast<int64_t>(n_starts) * wpr;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; w < total;
         w += stride) {
        const int32_t j = static_cast<int32_t>(w / n_starts);
        const int32_t i = static_cast<int32_t>(w - static_cast<int64_t>(j) * n_starts);
        const int32_t s = __ldg(starts + i);
        const uint32_t x2 = round * static_cast<uint32_t>(wpr) + static_cast<uint32_t>(j);
        walk_fill_row<COUNT, VEC>(offsets, cols, n, nnz, s, L, seed, x2, walks + w * L, counts);
    }
}

// kWalkPerThread walks per thread in lockstep (walk_fill_rows_vec), walks
// g * M .. g * M + M - 1 for thread-group index g; 4-step int4 stores.
constexpr int kWalkPerThread = 2;

template <bool COUNT, int M>
__global__ void __launch_bounds__(kWalkThreads)
    k_walk_m(const int32_t *__restrict__ offsets, const int32_t *__restrict__ cols, int32_t n, int64_t nnz,
             const int32_t *__restrict__ starts, int32_t n_starts, int32_t L, int32_t wpr, uint64_t seed,
             uint32_t round, int32_t *__restrict__ walks, uint32_t *__restrict__ counts) {
    const int64_t total = static_cast<int64_t>(n_starts) * wpr;
    const int64_t groups = (total + M - 1) / M;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < groups; g += stride) {
        int32_t s[M];
        uint32_t x2[M];
        int32_t *rows[M];
        const int nm = static_cast<int>(total - g * M < M ? total - g * M : M);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int64_t w = g * M + (m < nm ? m : 0);
            const int32_t j = static_cast<int32_t>(w / n_starts);
            const int32_t i = static_cast<int32_t>(w - static_cast<int64_t>(j) * n_starts);
            s[m] = __ldg(starts + i);
            x2[m] = round * static_cast<uint32_t>(wpr) + static_cast<uint32_t>(j);
            rows[m] = walks + w * L;
        }
        walk_fill_rows_vec<COUNT, M>(offsets, cols, n, nnz, s, nm, L, seed, x2, rows, counts);
    }
}

__global__ void k_count(const int32_t *__restrict__ tokens, int64_t n_tokens,
                        uint32_t *__restrict__ counts) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_tokens;
         p += stride) {
        const int32_t v = tokens[p];
        if (v >= 0) atomicAdd(counts + v, 1u);
    }
}

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

bool csr_shape_ok(const felog_csr *g) {
    return g && g->n >= 0 && g->nnz >= 0 && g->nnz < (int64_t(1) << 31) && g->offsets &&
           (g->nnz == 0 || g->cols);
}

// ---------------------------------------------------------------------------
// Device-side validation of a CSR (and optionally a start list).  One warp
// per row: lane 0 checks the row's offsets, the lanes stride its columns.
// Columns are read only where 0 <= offsets[v] <= offsets[v+1] <= nnz, so a
// malformed graph is reported without any out-of-range read.  Problems are
// OR-ed into *status as FELOG_CSR_* bits.
// ---------------------------------------------------------------------------
constexpr int kValidateThreads = 256;

__global__ void __launch_bounds__(kValidateThreads)
    k_validate_csr(const int32_t *__restrict__ offsets, const int32_t *__restrict__ cols, int32_t n, int64_t nnz,
                   const int32_t *__restrict__ starts, int32_t n_starts, int32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    int32_t bad = 0;
    if (warp == 0 && lane == 0 && (offsets[0] != 0 || offsets[n] != nnz)) bad |= FELOG_CSR_ENDS;
    for (int64_t v = warp; v < n; v += warps) {
        const int32_t lo = offsets[v], hi = offsets[v + 1];
        if (hi < lo) {
            bad |= FELOG_CSR_DECREASING;
            continue;
        }
        if (lo < 0 || hi > nnz) {
            bad |= FELOG_CSR_ENDS;
            continue;
        }
        for (int64_t e = lo + lane; e < hi; e += 32) {
            const int32_t c = cols[e];
            if (c < 0 || c >= n) bad |= FELOG_CSR_COL_RANGE;
            if (c == v) bad |= FELOG_CSR_SELF_LOOP;
            if (e + 1 < hi && cols[e + 1] <= c) bad |= FELOG_CSR_ORDER;
        }
    }
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t i = tid; i < n_starts; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t s = starts[i];
        if (s < 0 || s >= n) bad |= FELOG_CSR_START_RANGE;
    }
    const unsigned any = __reduce_or_sync(kFull, static_cast<unsigned>(bad));
    if (lane == 0 && any) atomicOr(status, static_cast<int32_t>(any));
}

felog_status validate_csr_async(const felog_csr *g, const int32_t *starts, int32_t n_starts, int32_t *status,
                                cudaStream_t s) {
    felog_status st = record_cuda_error(cudaMemsetAsync(status, 0, sizeof(int32_t), s), "felog_validate_csr");
    if (st) return st;
    const int64_t warps = std::max<int64_t>(g->n, (n_starts + 31) / 32);
    const int blocks = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(warps, kValidateThreads / 32), static_cast<int64_t>(sm_count()) * 16)));
    k_validate_csr<<<blocks, kValidateThreads, 0, s>>>(g->offsets, g->cols, g->n, g->nnz, starts, n_starts, status);
    return check_launch("felog_validate_csr");
}

}  // namespace felog

extern "C" felog_status felog_validate_csr(const felog_csr *g, const int32_t *starts, int32_t n_starts,
                                           int32_t *status, void *stream) {
    if (!csr_shape_ok(g)) return FELOG_ERR_BAD_CSR;
    if (!status || n_starts < 0 || (n_starts > 0 && !starts)) return FELOG_ERR_INVALID_ARG;
    return validate_csr_async(g, starts, n_starts, status, static_cast<cudaStream_t>(stream));
}

extern "C" felog_status felog_walk(const felog_csr *g, const int32_t *starts, int32_t n_starts,
                                   const felog_walk_params *wp, uint64_t seed, int32_t round,
                                   int32_t *walks, uint32_t *counts, void *stream) {
    if (!csr_shape_ok(g)) return FELOG_ERR_BAD_CSR;
    if (!wp || wp->length < 1 || wp->walks_per_round < 1 || n_starts < 0 || round < 0 ||
        round >= 65536)
        return FELOG_ERR_INVALID_ARG;
    if (n_starts == 0) return FELOG_OK;
    if (!starts || !walks) return FELOG_ERR_INVALID_ARG;
    const int64_t total = static_cast<int64_t>(n_starts) * wp->walks_per_round;
    const int L = wp->length;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool vec = (L % 4 == 0) && (reinterpret_cast<uintptr_t>(walks) % 16 == 0);
    if (vec) {
        constexpr int M = kWalkPerThread;
        const int blocks = static_cast<int>(std::min<int64_t>(ceil_div((total + M - 1) / M, kWalkThreads),
                                                              static_cast<int64_t>(sm_count()) * 8));
        if (counts)
            k_walk_m<true, M><<<blocks, kWalkThreads, 0, s>>>(g->offsets, g->cols, g->n, g->nnz, starts, n_starts, L,
                                                              wp->walks_per_round, seed, static_cast<uint32_t>(round),
                                                              walks, counts);
        else
            k_walk_m<false, M><<<blocks, kWalkThreads, 0, s>>>(g->offsets, g->cols, g->n, g->nnz, starts, n_starts,
                                                               L, wp->walks_per_round, seed,
                                                               static_cast<uint32_t>(round), walks, counts);
        return check_launch("felog_walk");
    }
    const int blocks = static_cast<int>(
        std::min<int64_t>(ceil_div(total, kWalkThreads), static_cast<int64_t>(sm_count()) * 8));
#define FELOG_WALK_LAUNCH(C, V)                                                                   \
    k_walk<C, V><<<blocks, kWalkThreads, 0, s>>>(g->offsets, g->cols, g->n, g->nnz, starts, n_starts, L, \
                                                 wp->walks_per_round, seed,                        \
                                                 static_cast<uint32_t>(round), walks, counts)
    if (counts) {
        if (vec) FELOG_WALK_LAUNCH(true, true);
        else FELOG_WALK_LAUNCH(true, false);
    } else {
        if (vec) FELOG_WALK_LAUNCH(false, true);
        else FELOG_WALK_LAUNCH(false, false);
    }
#undef FELOG_WALK_LAUNCH
    return check_launch("felog_walk");
}

extern "C" felog_status felog_count(const int32_t *tokens, int64_t n_tokens, int32_t n,
                                    uint32_t *counts, void *stream) {
    if (n_tokens < 0 || n < 0 || (n_tokens > 0 && (!tokens || !counts))) return FELOG_ERR_INVALID_ARG;
    if (n_tokens == 0) return FELOG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = static_cast<int>(std::min<int64_t>(ceil_div(n_tokens, 256), sm_count() * 16));
    k_count<<<blocks, 256, 0, s>>>(tokens, n_tokens, counts);
    return check_launch("felog_count");
}

extern "C" const char *felog_status_string(felog_status st) {
    switch (st) {
        case FELOG_OK: return "ok";
        case FELOG_ERR_INVALID_ARG: return "invalid argument";
        case FELOG_ERR_BAD_CSR: return "malformed CSR";
        case FELOG_ERR_WORKSPACE: return "workspace missing or too small";
        case FELOG_ERR_CUDA: return "CUDA error";
        case FELOG_ERR_UNSUPPORTED: return "unsupported parameter combination";
        case FELOG_ERR_TIMEOUT: return "timed out";
    }
    return "unknown status";
}

extern "C" const char *felog_last_cuda_error(void) { return felog::g_last_error; }
