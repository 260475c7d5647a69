// FaBC: frequency-aware bitmap compression of walk sequences (Section
// 5.2.2, Eq. 7, Eq. 8), for persisting or moving a round's corpus.
//
// Selection: nodes ordered by corpus frequency p (count / total, ties to
// the smaller id); with c = 1/L + 1/32 and g(k) = 1 - F_k + k c, k grows
// from 0 while p(k+1) >= c + 0.1 g(k).  The candidates come from k_max
// rounds of a device-wide argmax over (count, -id); the rule itself runs on
// the host in binary64.
//
// Format, for N sequences of L ids and B = ceil(L / 8):
//   N*k int32    the selected ids, stored with every sequence
//   N*k*B bytes  bitmap (s, j) at (s*k + j)*B, bit i = walks[s][i] == ids[j]
//   int32 tail   the ids no bitmap covers, in sequence and position order
// Encode and decode work one warp per sequence: the bitmaps are ballots over
// 32 positions at a time, and the tail positions are ranked within the
// sequence by ballot prefix counts; a scan of the per-sequence tail lengths
// gives each sequence's place in the tail.
#include <algorithm>

#include "common.cuh"

namespace felog {

int sm_count();

constexpr int kFabcMaxK = 32;
constexpr int kFabcThreads = 256;
constexpr int kFabcWarps = kFabcThreads / 32;
constexpr int kScanItems = 16;
constexpr int kScanTile = kFabcThreads * kScanItems;

// ---------------------------------------------------------------------------
// selection
// ---------------------------------------------------------------------------
__global__ void k_fabc_total(const uint32_t *__restrict__ counts, int32_t n, unsigned long long *__restrict__ total) {
    unsigned long long s = 0;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x)
        s += counts[v];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

// keys[r] = max over nodes not among keys[0..r) of (count << 32 | ~id): the
// most frequent remaining node, the smaller id on ties
__global__ void k_fabc_argmax(const uint32_t *__restrict__ counts, int32_t n, int32_t r,
                              unsigned long long *__restrict__ keys) {
    __shared__ int32_t taken[kFabcMaxK];
    if (threadIdx.x < r) taken[threadIdx.x] = static_cast<int32_t>(~static_cast<uint32_t>(keys[threadIdx.x]));
    __syncthreads();
    unsigned long long best = 0;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        bool skip = false;
        for (int j = 0; j < r; ++j) skip |= taken[j] == v;
        const unsigned long long key =
            (static_cast<unsigned long long>(counts[v]) << 32) | (~static_cast<uint32_t>(v));
        if (!skip && key > best) best = key;
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(kFull, best, o);
        best = other > best ? other : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&keys[r], best);
}

// ---------------------------------------------------------------------------
// tail lengths and their exclusive scan
// ---------------------------------------------------------------------------
// coverage of 32 positions of a sequence by the k ids held in lanes 0..k-1
__device__ __forceinline__ uint32_t covered_ids(int32_t v, bool in, int32_t my_id, int k, int lane, uint32_t *per_id) {
    uint32_t any = 0;
    for (int j = 0; j < k; ++j) {
        const int32_t idj = __shfl_sync(kFull, my_id, j);
        const uint32_t m = __ballot_sync(kFull, in && v == idj);
        if (lane == j) *per_id = m;
        any |= m;
    }
    return any;
}

__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_tail_len(const int32_t *__restrict__ walks, int64_t n_seq, int32_t L, const int32_t *__restrict__ ids,
                    int32_t k, int64_t *__restrict__ len) {
    const int lane = threadIdx.x & 31;
    const int32_t my_id = lane < k ? ids[lane] : 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kFabcWarps;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * kFabcWarps + (threadIdx.x >> 5); s < n_seq; s += warps) {
        const int32_t *row = walks + s * L;
        int64_t t = 0;
        for (int c = 0; c < L; c += 32) {
            const bool in = c + lane < L;
            const int32_t v = in ? row[c + lane] : 0;
            uint32_t mine = 0;
            const uint32_t cov = covered_ids(v, in, my_id, k, lane, &mine);
            const uint32_t valid = __ballot_sync(kFull, in);
            t += __popc(valid & ~cov);
        }
        if (lane == 0) len[s] = t;
    }
}

__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_tail_len_dec(const uint8_t *__restrict__ bm, int64_t n_seq, int32_t L, int32_t k, int64_t *__restrict__ len) {
    const int lane = threadIdx.x & 31;
    const int B = (L + 7) / 8;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kFabcWarps;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * kFabcWarps + (threadIdx.x >> 5); s < n_seq; s += warps) {
        int64_t t = 0;
        for (int c = 0; c < L; c += 32) {
            const int i = c + lane;
            bool cov = false;
            for (int j = 0; j < k && i < L; ++j) cov |= (bm[(s * k + j) * B + (i >> 3)] >> (i & 7)) & 1u;
            t += __popc(__ballot_sync(kFull, i < L && !cov));
        }
        if (lane == 0) len[s] = t;
    }
}

// exclusive scan of len[n] into off[n] (in place allowed), total into *total
__global__ void __launch_bounds__(kFabcThreads)
    k_scan_tiles(const int64_t *__restrict__ len, int64_t n, int64_t *__restrict__ tile_sum) {
    __shared__ int64_t part[kFabcWarps];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + static_cast<int64_t>(k) * kFabcThreads + threadIdx.x;
        if (i < n) s += len[i];
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kFabcWarps; ++w) t += part[w];
        tile_sum[blockIdx.x] = t;
    }
}

__global__ void k_scan_top(int64_t *__restrict__ tile_sum, int64_t tiles, int64_t *__restrict__ total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t run = 0;
    for (int64_t t = 0; t < tiles; ++t) {
        const int64_t x = tile_sum[t];
        tile_sum[t] = run;
        run += x;
    }
    *total = run;
}

__global__ void __launch_bounds__(kFabcThreads)
    k_scan_apply(int64_t *__restrict__ len, int64_t n, const int64_t *__restrict__ tile_off) {
    __shared__ int64_t part[kFabcThreads];
    // each thread owns kScanItems consecutive items of the tile
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? len[base + k] : 0;
        s += v[k];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = tile_off[blockIdx.x];
        for (int i = 0; i < kFabcThreads; ++i) {
            const int64_t x = part[i];
            part[i] = run;
            run += x;
        }
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) len[base + k] = run;
        run += v[k];
    }
}

// ---------------------------------------------------------------------------
// encode / decode.  The tail starts 4Nk + NkB bytes into the buffer, which is
// a multiple of 4 only when NkB is; otherwise its entries are moved byte by
// byte (the layout has no padding, so its size is exactly Eq. 7's count).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void put32(uint8_t *p, int64_t i, int32_t v, bool aligned) {
    if (aligned) {
        reinterpret_cast<int32_t *>(p)[i] = v;
    } else {
        const uint32_t u = static_cast<uint32_t>(v);
        for (int b = 0; b < 4; ++b) p[4 * i + b] = static_cast<uint8_t>(u >> (8 * b));
    }
}
__device__ __forceinline__ int32_t get32(const uint8_t *p, int64_t i, bool aligned) {
    if (aligned) return reinterpret_cast<const int32_t *>(p)[i];
    uint32_t u = 0;
    for (int b = 0; b < 4; ++b) u |= static_cast<uint32_t>(p[4 * i + b]) << (8 * b);
    return static_cast<int32_t>(u);
}
__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_encode(const int32_t *__restrict__ walks, int64_t n_seq, int32_t L, const int32_t *__restrict__ ids,
                  int32_t k, const int64_t *__restrict__ off, uint8_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int B = (L + 7) / 8;
    const int32_t my_id = lane < k ? ids[lane] : 0;
    int32_t *idreg = reinterpret_cast<int32_t *>(out);
    uint8_t *bm = out + 4 * n_seq * k, *tail = bm + n_seq * k * B;
    const bool aligned = ((n_seq * k * B) & 3) == 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kFabcWarps;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * kFabcWarps + (threadIdx.x >> 5); s < n_seq; s += warps) {
        const int32_t *row = walks + s * L;
        if (lane < k) idreg[s * k + lane] = my_id;
        int64_t t = off[s];
        for (int c = 0; c < L; c += 32) {
            const bool in = c + lane < L;
            const int32_t v = in ? row[c + lane] : 0;
            uint32_t mine = 0;  // lane j: the bits of id j in these 32 positions
            const uint32_t cov = covered_ids(v, in, my_id, k, lane, &mine);
            // lane j < k writes bytes c/8 .. c/8 + 3 of bitmap j (those below B)
            if (lane < k)
                for (int b = 0; b < 4 && c / 8 + b < B; ++b) bm[(s * k + lane) * B + c / 8 + b] = static_cast<uint8_t>(mine >> (8 * b));
            const uint32_t keep = __ballot_sync(kFull, in) & ~cov;
            if (keep >> lane & 1u) put32(tail, t + __popc(keep & ((1u << lane) - 1u)), v, aligned);
            t += __popc(keep);
        }
    }
}

__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_decode(const uint8_t *__restrict__ in, int64_t n_seq, int32_t L, int32_t k, const int64_t *__restrict__ off,
                  int64_t tail_cap, int32_t *__restrict__ walks) {
    const int lane = threadIdx.x & 31;
    const int B = (L + 7) / 8;
    const int32_t *idreg = reinterpret_cast<const int32_t *>(in);
    const uint8_t *bm = in + 4 * n_seq * k, *tail = bm + n_seq * k * B;
    const bool aligned = ((n_seq * k * B) & 3) == 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kFabcWarps;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * kFabcWarps + (threadIdx.x >> 5); s < n_seq; s += warps) {
        int32_t my_id = 0;
        if (lane < k) my_id = idreg[s * k + lane];
        int64_t t = off[s];
        for (int c = 0; c < L; c += 32) {
            const int i = c + lane;
            int found = -1;
            for (int j = 0; j < k && i < L; ++j)
                if (found < 0 && ((bm[(s * k + j) * B + (i >> 3)] >> (i & 7)) & 1u)) found = j;
            int32_t v = 0;
            for (int j = 0; j < k; ++j) {  // every lane joins the shuffles
                const int32_t idj = __shfl_sync(kFull, my_id, j);
                if (found == j) v = idj;
            }
            const uint32_t fromtail = __ballot_sync(kFull, i < L && found < 0);
            if (fromtail >> lane & 1u) {
                const int64_t ti = t + __popc(fromtail & ((1u << lane) - 1u));
                v = ti < tail_cap ? get32(tail, ti, aligned) : -1;  // past the buffer: -1
            }
            if (i < L) walks[s * L + i] = v;
            t += __popc(fromtail);
        }
    }
}

struct FabcWorkspace {
    unsigned long long *total;
    unsigned long long *keys;
    int64_t *off;
    int64_t *tile;
};

static FabcWorkspace carve_fabc(Carver &c, int64_t n_seq) {
    FabcWorkspace w;
    w.total = c.take<unsigned long long>(1);
    w.keys = c.take<unsigned long long>(kFabcMaxK);
    w.off = c.take<int64_t>(n_seq > 0 ? static_cast<size_t>(n_seq) : 1);
    w.tile = c.take<int64_t>(n_seq > 0 ? static_cast<size_t>((n_seq + kScanTile - 1) / kScanTile) : 1);
    return w;
}

static int seq_grid(int64_t n_seq) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n_seq + kFabcWarps - 1) / kFabcWarps, sm_count() * 8)));
}

static felog_status scan_offsets(FabcWorkspace &w, int64_t n_seq, int64_t *total, cudaStream_t s) {
    const int64_t tiles = (n_seq + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<static_cast<int>(tiles), kFabcThreads, 0, s>>>(w.off, n_seq, w.tile);
    k_scan_top<<<1, 32, 0, s>>>(w.tile, tiles, total);
    k_scan_apply<<<static_cast<int>(tiles), kFabcThreads, 0, s>>>(w.off, n_seq, w.tile);
    return check_launch("fabc scan");
}

}  // namespace felog

using namespace felog;

extern "C" int32_t felog_fabc_max_k(void) { return kFabcMaxK; }

extern "C" size_t felog_fabc_workspace_bytes(int64_t n_seq) {
    if (n_seq < 0) return 0;
    Carver c(nullptr, 0);
    carve_fabc(c, n_seq);
    return align_up(c.used, 256);
}

extern "C" size_t felog_fabc_max_bytes(int64_t n_seq, int32_t L, int32_t k) {
    if (n_seq < 0 || L < 1 || k < 0 || k > kFabcMaxK) return 0;
    const int64_t B = (L + 7) / 8;
    return static_cast<size_t>(4 * n_seq * k + n_seq * k * B + 4 * n_seq * static_cast<int64_t>(L));
}

extern "C" felog_status felog_fabc_select(const uint32_t *counts, int32_t n, int32_t L, int32_t k_max, int32_t *ids,
                                          int32_t *k, double *F, void *workspace, size_t workspace_bytes,
                                          void *stream) {
    if (n < 0 || L < 1 || k_max < 0 || k_max > kFabcMaxK || !ids || !k || (n > 0 && !counts))
        return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_fabc_workspace_bytes(0)) return FELOG_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    FabcWorkspace w = carve_fabc(c, 0);
    *k = 0;
    if (F) *F = 0.0;
    if (n == 0 || k_max == 0) return FELOG_OK;
    felog_status st = record_cuda_error(cudaMemsetAsync(w.total, 0, sizeof(unsigned long long), s), "fabc");
    if (!st) st = record_cuda_error(cudaMemsetAsync(w.keys, 0, sizeof(unsigned long long) * kFabcMaxK, s), "fabc");
    if (st) return st;
    const int grid = std::max(1, std::min((n + 255) / 256, sm_count() * 4));
    k_fabc_total<<<grid, 256, 0, s>>>(counts, n, w.total);
    for (int r = 0; r < k_max; ++r) k_fabc_argmax<<<grid, 256, 0, s>>>(counts, n, r, w.keys);
    st = check_launch("felog_fabc_select");
    if (st) return st;
    unsigned long long h[1 + kFabcMaxK];
    st = record_cuda_error(cudaMemcpyAsync(h, w.total, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s), "fabc");
    if (!st) st = record_cuda_error(cudaMemcpyAsync(h + 1, w.keys, sizeof(unsigned long long) * k_max, cudaMemcpyDeviceToHost, s), "fabc");
    if (!st) st = record_cuda_error(cudaStreamSynchronize(s), "fabc");
    if (st) return st;
    const unsigned long long total = h[0];
    const double cc = 1.0 / static_cast<double>(L) + 1.0 / 32.0;
    double Fk = 0.0, g = 1.0;
    int32_t kk = 0;
    while (kk < k_max && total > 0) {
        const unsigned long long key = h[1 + kk];
        const double p = static_cast<double>(static_cast<uint32_t>(key >> 32)) / static_cast<double>(total);
        if (!(p >= cc + 0.1 * g)) break;
        ids[kk] = static_cast<int32_t>(~static_cast<uint32_t>(key));
        kk += 1;
        Fk += p;
        g = 1.0 - Fk + static_cast<double>(kk) * cc;
    }
    *k = kk;
    if (F) *F = Fk;
    return FELOG_OK;
}

extern "C" felog_status felog_fabc_encode(const int32_t *walks, int64_t n_seq, int32_t L, const int32_t *ids, int32_t k,
                                          uint8_t *out, size_t out_bytes, int64_t *tail, void *workspace,
                                          size_t workspace_bytes, void *stream) {
    if (n_seq < 0 || L < 1 || k < 0 || k > kFabcMaxK || !tail) return FELOG_ERR_INVALID_ARG;
    if (n_seq > 0 && (!walks || !out || (k > 0 && !ids))) return FELOG_ERR_INVALID_ARG;
    if (out_bytes < felog_fabc_max_bytes(n_seq, L, k)) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_fabc_workspace_bytes(n_seq)) return FELOG_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    FabcWorkspace w = carve_fabc(c, n_seq);
    if (n_seq == 0) return record_cuda_error(cudaMemsetAsync(tail, 0, sizeof(int64_t), s), "fabc");
    const int grid = seq_grid(n_seq);
    k_fabc_tail_len<<<grid, kFabcThreads, 0, s>>>(walks, n_seq, L, ids, k, w.off);
    felog_status st = scan_offsets(w, n_seq, tail, s);
    if (st) return st;
    k_fabc_encode<<<grid, kFabcThreads, 0, s>>>(walks, n_seq, L, ids, k, w.off, out);
    return check_launch("felog_fabc_encode");
}

extern "C" felog_status felog_fabc_decode(const uint8_t *in, size_t in_bytes, int64_t n_seq, int32_t L, int32_t k,
                                          int32_t *walks, void *workspace, size_t workspace_bytes, void *stream) {
    if (n_seq < 0 || L < 1 || k < 0 || k > kFabcMaxK) return FELOG_ERR_INVALID_ARG;
    const int64_t head = 4 * n_seq * k + n_seq * k * ((L + 7) / 8);
    if (static_cast<int64_t>(in_bytes) < head) return FELOG_ERR_INVALID_ARG;
    if (n_seq > 0 && (!in || !walks)) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_fabc_workspace_bytes(n_seq)) return FELOG_ERR_WORKSPACE;
    if (n_seq == 0) return FELOG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    FabcWorkspace w = carve_fabc(c, n_seq);
    const int grid = seq_grid(n_seq);
    k_fabc_tail_len_dec<<<grid, kFabcThreads, 0, s>>>(in + 4 * n_seq * k, n_seq, L, k, w.off);
    felog_status st = scan_offsets(w, n_seq, reinterpret_cast<int64_t *>(w.total), s);
    if (st) return st;
    k_fabc_decode<<<grid, kFabcThreads, 0, s>>>(in, n_seq, L, k, w.off, (static_cast<int64_t>(in_bytes) - head) / 4,
                                                 walks);
    return check_launch("felog_fabc_decode");
}
