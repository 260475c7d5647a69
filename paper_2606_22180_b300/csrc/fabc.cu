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
// For k >= 1, encode and decode work one warp per sequence: the bitmaps are
// ballots over 32 positions at a time, and the tail positions are ranked
// within the sequence by ballot prefix counts; a scan of the per-sequence
// tail lengths gives each sequence's place in the tail.  A block first copies
// a tile of up to 64 whole sequences (their walks, or their ids, bitmaps and
// stretch of tail) to shared memory with independent coalesced loads; only
// sequences too long for 24 KB are read in place.  For k = 0 the encoding is
// the walks verbatim and both directions are one streaming copy.
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
// per-sequence work, shared by the staged kernels (a tile of whole sequences
// copied to shared memory first) and the unstaged ones (long sequences,
// read straight from global memory)
// ---------------------------------------------------------------------------
// The selected ids as the warp holds them.  K > 0: k == K and every lane
// keeps all K ids in registers (the loops over ids unroll); K == 0: any
// k <= 32, id j in lane j, fetched by shuffle.
template <int K>
struct IdSet {
    int32_t r[K > 0 ? K : 1];
    int32_t mine;
    int k;
};
template <int K>
__device__ __forceinline__ IdSet<K> load_ids(const int32_t *__restrict__ ids, int k, int lane) {
    IdSet<K> s;
    s.k = k;
    s.mine = K == 0 && lane < k ? __ldg(ids + lane) : 0;
#pragma unroll
    for (int j = 0; j < (K > 0 ? K : 1); ++j) s.r[j] = K > 0 ? __ldg(ids + j) : 0;
    return s;
}

// coverage of 32 positions by the ids: the OR of the per-id ballots, and
// in lane j the ballot of id j
template <int K>
__device__ __forceinline__ uint32_t covered_ids(int32_t v, bool in, const IdSet<K> &ids, int lane, uint32_t *per_id) {
    uint32_t any = 0;
    if constexpr (K > 0) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t m = __ballot_sync(kFull, in && v == ids.r[j]);
            if (lane == j) *per_id = m;
            any |= m;
        }
    } else {
        for (int j = 0; j < ids.k; ++j) {
            const int32_t idj = __shfl_sync(kFull, ids.mine, j);  // every lane, before any short-circuit
            const uint32_t m = __ballot_sync(kFull, in && v == idj);
            if (lane == j) *per_id = m;
            any |= m;
        }
    }
    return any;
}

// number of positions of row[0..L) that no id covers (the whole warp)
template <int K>
__device__ __forceinline__ int64_t tail_len_seq(const int32_t *row, int32_t L, const IdSet<K> &ids, int lane) {
    int t = 0;
    for (int c = 0; c < L; c += 32) {
        const bool in = c + lane < L;
        const int32_t v = in ? row[c + lane] : 0;
        if constexpr (K > 0) {
            bool cov = false;
#pragma unroll
            for (int j = 0; j < K; ++j) cov |= v == ids.r[j];
            t += __popc(__ballot_sync(kFull, in && !cov));
        } else {
            uint32_t mine = 0;
            const uint32_t cov = covered_ids<K>(v, in, ids, lane, &mine);
            t += __popc(__ballot_sync(kFull, in) & ~cov);
        }
    }
    return t;
}

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

// encodes one sequence from row[0..L): its k bitmaps into bms[0..k*B), its
// tail from index t on
template <int K>
__device__ __forceinline__ void encode_seq(const int32_t *row, int32_t L, int B, const IdSet<K> &ids, int lane,
                                           int64_t t, uint8_t *bms, uint8_t *tail, bool aligned) {
    const int k = K > 0 ? K : ids.k;
    for (int c = 0; c < L; c += 32) {
        const bool in = c + lane < L;
        const int32_t v = in ? row[c + lane] : 0;
        uint32_t mine = 0;  // lane j: the bits of id j in these 32 positions
        const uint32_t cov = covered_ids<K>(v, in, ids, lane, &mine);
        // lane j < k writes bytes c/8 .. c/8 + 3 of bitmap j (those below B)
        if (lane < k)
            for (int b = 0; b < 4 && c / 8 + b < B; ++b)
                bms[lane * B + c / 8 + b] = static_cast<uint8_t>(mine >> (8 * b));
        const uint32_t keep = __ballot_sync(kFull, in) & ~cov;
        if (keep >> lane & 1u) put32(tail, t + __popc(keep & ((1u << lane) - 1u)), v, aligned);
        t += __popc(keep);
    }
}

// decodes one sequence: bms = its k*B bitmap bytes, id j in lane j, tail
// entry t of the sequence at tailp + 4t (entries at or past cap decode as -1)
template <int K>
__device__ __forceinline__ void decode_seq(const uint8_t *bms, int32_t my_id, int32_t L, int B, int k, int lane,
                                           int64_t t, const uint8_t *tailp, int64_t cap, bool aligned,
                                           int32_t *out) {
    for (int c = 0; c < L; c += 32) {
        const int i = c + lane;
        int found = -1;  // the first id whose bit is set
        if (i < L) {
            const uint8_t *by = bms + (i >> 3);
            const int sh = i & 7;
            if constexpr (K > 0) {
#pragma unroll
                for (int j = K - 1; j >= 0; --j)
                    if ((by[j * B] >> sh) & 1u) found = j;
            } else {
                for (int j = k - 1; j >= 0; --j)
                    if ((by[j * B] >> sh) & 1u) found = j;
            }
        }
        int32_t v = __shfl_sync(kFull, my_id, found < 0 ? 0 : found);
        const uint32_t fromtail = __ballot_sync(kFull, i < L && found < 0);
        if (fromtail >> lane & 1u) {
            const int64_t ti = t + __popc(fromtail & ((1u << lane) - 1u));
            v = ti < cap ? get32(tailp, ti, aligned) : -1;
        }
        if (i < L) out[i] = v;
        t += __popc(fromtail);
    }
}

// ---------------------------------------------------------------------------
// staging: a block copies its tile to shared memory and works from there.
// Decode moves bytes with independent word loads issued back to back (4 per
// thread in flight); encode uses cp.async, two tiles deep.
// ---------------------------------------------------------------------------
constexpr int kStageBytes = 24576;  // shared memory per block
constexpr int kStageMaxSeq = 64;    // sequences per tile
constexpr int kStageUnroll = 4;

// n bytes from global src (any alignment) to shared dst (4-byte aligned,
// n + 4 bytes of room): the bytes land at dst + o, o = src mod 4, so that
// the aligned middle moves as 4-byte words; returns o
__device__ __forceinline__ int stage_bytes(uint8_t *dst, const uint8_t *__restrict__ src, int n) {
    const int o = static_cast<int>(reinterpret_cast<uintptr_t>(src) & 3u);
    const int head = min(n, (4 - o) & 3);
    if (static_cast<int>(threadIdx.x) < head) dst[o + threadIdx.x] = src[threadIdx.x];
    const int nw = (n - head) >> 2;
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(src + head);
    uint32_t *dw = reinterpret_cast<uint32_t *>(dst + o + head);
    for (int base = threadIdx.x; base < nw; base += kStageUnroll * blockDim.x) {
        uint32_t r[kStageUnroll];
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            const int i = base + u * static_cast<int>(blockDim.x);
            if (i < nw) r[u] = __ldg(sw + i);
        }
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            const int i = base + u * static_cast<int>(blockDim.x);
            if (i < nw) dw[i] = r[u];
        }
    }
    const int done = head + 4 * nw;
    if (static_cast<int>(threadIdx.x) < n - done) dst[o + done + threadIdx.x] = src[done + threadIdx.x];
    return o;
}

// asynchronous global -> shared copies (cp.async), waited on per commit group
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

// encode tiles: TS sequences, a multiple of 4 so that every tile starts on a
// 16-byte boundary of the walks; 0 = sequences too long to stage.  Two
// buffers of offsets and walks (the next tile arrives while this one is
// encoded) and the tile's bitmaps, written out whole afterwards.
constexpr int kEncodeStageBytes = 40960;
static_assert(kEncodeStageBytes <= 48 * 1024, "dynamic shared memory above 48 KB needs an opt-in");
static int encode_buffer_bytes(int ts, int32_t L) { return align16(ts * 8) + align16(4 * ts * L); }
static int encode_stage_bytes(int ts, int32_t L, int32_t k) {
    return 2 * encode_buffer_bytes(ts, L) + align16(ts * k * ((L + 7) / 8));
}
static int encode_tile_seqs(int32_t L, int32_t k) {
    if (L > kEncodeStageBytes / 32) return 0;
    int ts = kStageMaxSeq;
    while (ts > 0 && encode_stage_bytes(ts, L, k) > kEncodeStageBytes) ts -= 4;
    return ts;
}

// decode tiles stage per sequence: its offset, k ids, k*B bitmap bytes and
// at most L tail entries
static int decode_stage_bytes(int ts, int32_t L, int32_t k) {
    const int B = (L + 7) / 8;
    return align16(ts * 8) + align16(4 * ts * k + 4) + align16(ts * k * B + 4) + align16(4 * ts * L + 4);
}
static int decode_tile_seqs(int32_t L, int32_t k) {
    int ts = kStageMaxSeq;
    while (ts > 0 && decode_stage_bytes(ts, L, k) > kStageBytes) --ts;
    return ts;
}

// ---------------------------------------------------------------------------
// encode, k >= 1.  COUNT: the tail length of every sequence into len; else
// the encoding, the tail of sequence s starting at off[s].  The tail starts 4Nk + NkB
// bytes into the buffer, a multiple of 4 only when NkB is; otherwise its
// entries move byte by byte (the layout has no padding: its size is exactly
// Eq. 7's count).  K > 0: compiled for k == K (see IdSet).
// ---------------------------------------------------------------------------
template <bool COUNT, int K>
__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_encode_st(const int32_t *__restrict__ walks, int64_t n_seq, int32_t L, int32_t ts,
                     const int32_t *__restrict__ ids, int32_t k, const int64_t *__restrict__ off,
                     int64_t *__restrict__ len, uint8_t *__restrict__ out) {
    extern __shared__ int4 fabc_smem[];
    const int B = (L + 7) / 8;
    const int buf_bytes = align16(ts * 8) + align16(4 * ts * L);
    uint8_t *sbm = reinterpret_cast<uint8_t *>(fabc_smem) + 2 * buf_bytes;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const IdSet<K> idset = load_ids<K>(ids, k, lane);
    int32_t *idreg = reinterpret_cast<int32_t *>(out);
    uint8_t *bm = out + 4 * n_seq * k, *tail = bm + n_seq * k * B;
    const bool aligned = ((n_seq * k * B) & 3) == 0;
    const bool vec = (reinterpret_cast<uintptr_t>(walks) & 15u) == 0;  // then every tile start is (ts % 4 == 0)
    const int64_t n_tiles = (n_seq + ts - 1) / ts;
    // copies tile ti into buffer b: its offsets (encode) and walks
    auto issue = [&](int64_t ti, int b) {
        uint8_t *base = reinterpret_cast<uint8_t *>(fabc_smem) + b * buf_bytes;
        int64_t *so = reinterpret_cast<int64_t *>(base);
        int32_t *tl = reinterpret_cast<int32_t *>(base + align16(ts * 8));
        const int64_t s0 = ti * ts;
        const int ns = static_cast<int>(n_seq - s0 < ts ? n_seq - s0 : ts);
        const int n = ns * L;
        const int32_t *src = walks + s0 * L;
        int i0 = 0;
        if (vec) {
            const int n4 = n >> 2;
            for (int i = threadIdx.x; i < n4; i += blockDim.x) cp_async16(tl + 4 * i, src + 4 * i);
            i0 = 4 * n4;
        }
        for (int i = i0 + static_cast<int>(threadIdx.x); i < n; i += blockDim.x) cp_async4(tl + i, src + i);
        if (!COUNT && static_cast<int>(threadIdx.x) < ns) cp_async8(so + threadIdx.x, off + s0 + threadIdx.x);
    };
    int64_t ti = blockIdx.x;
    if (ti < n_tiles) issue(ti, 0);
    cp_async_commit();
    for (int b = 0; ti < n_tiles; ti += gridDim.x, b ^= 1) {
        if (ti + gridDim.x < n_tiles) issue(ti + gridDim.x, b ^ 1);
        cp_async_commit();
        cp_async_wait<1>();  // this thread's copies of tile ti
        __syncthreads();     // and everyone's
        uint8_t *base = reinterpret_cast<uint8_t *>(fabc_smem) + b * buf_bytes;
        const int64_t *soff = reinterpret_cast<const int64_t *>(base);
        const int32_t *tile = reinterpret_cast<const int32_t *>(base + align16(ts * 8));
        const int64_t s0 = ti * ts;
        const int ns = static_cast<int>(n_seq - s0 < ts ? n_seq - s0 : ts);
        for (int si = warp; si < ns; si += kFabcWarps) {
            const int32_t *row = tile + si * L;
            if (COUNT) {
                const int64_t t = tail_len_seq<K>(row, L, idset, lane);
                if (lane == 0) len[s0 + si] = t;
            } else {
                encode_seq<K>(row, L, B, idset, lane, soff[si], sbm + si * k * B, tail, aligned);
            }
        }
        __syncthreads();
        if (!COUNT) {  // the tile's ids and bitmaps, contiguous in the output (4-byte aligned: ts % 4 == 0)
            for (int i = threadIdx.x; i < ns * k; i += blockDim.x) idreg[s0 * k + i] = __ldg(ids + i % k);
            const int nb = ns * k * B, nw = nb >> 2;
            uint32_t *dw = reinterpret_cast<uint32_t *>(bm + s0 * k * B);
            const uint32_t *sw = reinterpret_cast<const uint32_t *>(sbm);
            for (int i = threadIdx.x; i < nw; i += blockDim.x) dw[i] = sw[i];
            if (static_cast<int>(threadIdx.x) < nb - 4 * nw) bm[s0 * k * B + 4 * nw + threadIdx.x] = sbm[4 * nw + threadIdx.x];
        }
    }
    cp_async_wait<0>();
}

// the same, one warp per sequence straight from global memory (long L)
template <bool COUNT>
__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_encode_g(const int32_t *__restrict__ walks, int64_t n_seq, int32_t L, const int32_t *__restrict__ ids,
                    int32_t k, const int64_t *__restrict__ off, int64_t *__restrict__ len, uint8_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int B = (L + 7) / 8;
    const IdSet<0> idset = load_ids<0>(ids, k, lane);
    int32_t *idreg = reinterpret_cast<int32_t *>(out);
    uint8_t *bm = out + 4 * n_seq * k, *tail = bm + n_seq * k * B;
    const bool aligned = ((n_seq * k * B) & 3) == 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kFabcWarps;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * kFabcWarps + (threadIdx.x >> 5); s < n_seq; s += warps) {
        const int32_t *row = walks + s * L;
        if (COUNT) {
            const int64_t t = tail_len_seq<0>(row, L, idset, lane);
            if (lane == 0) len[s] = t;
        } else {
            if (lane < k) idreg[s * k + lane] = idset.mine;
            encode_seq<0>(row, L, B, idset, lane, off[s], bm + s * k * B, tail, aligned);
        }
    }
}

// ---------------------------------------------------------------------------
// decode, k >= 1.  Tail lengths first, one thread per sequence: L minus the set bits
// of the OR of its k bitmaps (bits at or past L ignored).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_tail_len_dec(const uint8_t *__restrict__ bm, int64_t n_seq, int32_t L, int32_t k, int64_t *__restrict__ len) {
    const int B = (L + 7) / 8;
    const int last_bits = L - 8 * (B - 1);
    const uint32_t last_mask = (1u << last_bits) - 1u;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < n_seq;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint8_t *b = bm + s * k * B;
        int32_t cov = 0;
        for (int i = 0; i < B; ++i) {
            uint32_t x = 0;
            for (int j = 0; j < k; ++j) x |= __ldg(b + j * B + i);
            if (i == B - 1) x &= last_mask;
            cov += __popc(x);
        }
        len[s] = L - cov;
    }
}

// staged: per tile, the offsets, ids, bitmaps and the tile's stretch of the
// tail [off[s0], off[s0 + ns]) go to shared memory (tail entries at or past
// cap, the end of the buffer, decode as -1).  K > 0: compiled for k == K.
template <int K>
__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_decode_st(const uint8_t *__restrict__ in, int64_t n_seq, int32_t L, int32_t k, int32_t ts,
                     const int64_t *__restrict__ off, const int64_t *__restrict__ total, int64_t cap,
                     int32_t *__restrict__ walks) {
    extern __shared__ int4 fabc_smem[];
    const int B = (L + 7) / 8;
    uint8_t *base = reinterpret_cast<uint8_t *>(fabc_smem);
    int64_t *soff = reinterpret_cast<int64_t *>(base);
    uint8_t *sids = base + align16(ts * 8);
    uint8_t *sbm = sids + align16(4 * ts * k + 4);
    uint8_t *stl = sbm + align16(ts * k * B + 4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t *bm = in + 4 * n_seq * k, *tail = bm + n_seq * k * B;
    const int64_t n_tiles = (n_seq + ts - 1) / ts;
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const int64_t s0 = ti * ts;
        const int ns = static_cast<int>(n_seq - s0 < ts ? n_seq - s0 : ts);
        const int64_t t0 = off[s0];
        const int64_t t1 = s0 + ns < n_seq ? off[s0 + ns] : *total;
        const int64_t hi = t1 < cap ? t1 : cap, lo = t0 < hi ? t0 : hi;
        if (static_cast<int>(threadIdx.x) < ns) soff[threadIdx.x] = off[s0 + threadIdx.x] - t0;
        const int oid = stage_bytes(sids, in + 4 * s0 * k, 4 * ns * k);
        const int obm = stage_bytes(sbm, bm + s0 * k * B, ns * k * B);
        const int otl = stage_bytes(stl, tail + 4 * lo, static_cast<int>(4 * (hi - lo)));
        __syncthreads();
        for (int si = warp; si < ns; si += kFabcWarps) {
            const int32_t my_id = lane < k ? get32(sids + oid, static_cast<int64_t>(si) * k + lane, oid == 0) : 0;
            decode_seq<K>(sbm + obm + si * k * B, my_id, L, B, k, lane, soff[si], stl + otl, hi - t0, otl == 0,
                          walks + (s0 + si) * L);
        }
        __syncthreads();
    }
}

// unstaged, one warp per sequence (long L)
__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_decode_g(const uint8_t *__restrict__ in, int64_t n_seq, int32_t L, int32_t k,
                    const int64_t *__restrict__ off, int64_t cap, int32_t *__restrict__ walks) {
    const int lane = threadIdx.x & 31;
    const int B = (L + 7) / 8;
    const int32_t *idreg = reinterpret_cast<const int32_t *>(in);
    const uint8_t *bm = in + 4 * n_seq * k, *tail = bm + n_seq * k * B;
    const bool aligned = ((n_seq * k * B) & 3) == 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kFabcWarps;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * kFabcWarps + (threadIdx.x >> 5); s < n_seq; s += warps) {
        const int32_t my_id = lane < k ? idreg[s * k + lane] : 0;
        decode_seq<0>(bm + s * k * B, my_id, L, B, k, lane, off[s], tail, cap, aligned, walks + s * L);
    }
}

// ---------------------------------------------------------------------------
// k = 0: the encoding is the walks themselves (no ids, no bitmaps, every
// position in the tail), so encode and decode are a copy: dst[i] = src[i]
// for i < n_src, -1 up to n (a tail cut short); block 0 writes *total = n.
// ---------------------------------------------------------------------------
constexpr int kCopyUnroll = 4;

__global__ void __launch_bounds__(kFabcThreads)
    k_fabc_copy(const int32_t *__restrict__ src, int64_t n_src, int64_t n, int32_t *__restrict__ dst,
                int64_t *__restrict__ total) {
    if (total && blockIdx.x == 0 && threadIdx.x == 0) *total = n;
    const int64_t m = n_src < n ? n_src : n;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t done = 0;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
        const int64_t m4 = m >> 2;
        const int4 *s4 = reinterpret_cast<const int4 *>(src);
        int4 *d4 = reinterpret_cast<int4 *>(dst);
        for (int64_t base = tid; base < m4; base += kCopyUnroll * nthreads) {
            int4 r[kCopyUnroll];
#pragma unroll
            for (int u = 0; u < kCopyUnroll; ++u)
                if (base + u * nthreads < m4) r[u] = __ldcs(s4 + base + u * nthreads);
#pragma unroll
            for (int u = 0; u < kCopyUnroll; ++u)
                if (base + u * nthreads < m4) __stcs(d4 + base + u * nthreads, r[u]);
        }
        done = 4 * m4;
    }
    for (int64_t i = done + tid; i < m; i += nthreads) dst[i] = src[i];
    for (int64_t i = m + tid; i < n; i += nthreads) dst[i] = -1;
}

// ---------------------------------------------------------------------------
// exclusive scan of len[n] into itself, the total into *total
// ---------------------------------------------------------------------------
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

__device__ __forceinline__ int64_t warp_inclusive_scan(int64_t x, int lane) {
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// one warp: the tile sums into their exclusive prefix, 32 at a time
__global__ void k_scan_top(int64_t *__restrict__ tile_sum, int64_t tiles, int64_t *__restrict__ total) {
    const int lane = threadIdx.x;
    int64_t run = 0;
    for (int64_t b = 0; b < tiles; b += 32) {
        const int64_t i = b + lane;
        const int64_t x = i < tiles ? tile_sum[i] : 0;
        const int64_t inc = warp_inclusive_scan(x, lane);
        if (i < tiles) tile_sum[i] = run + inc - x;
        run += __shfl_sync(kFull, inc, 31);
    }
    if (lane == 0) *total = run;
}

__global__ void __launch_bounds__(kFabcThreads)
    k_scan_apply(int64_t *__restrict__ len, int64_t n, const int64_t *__restrict__ tile_off) {
    __shared__ int64_t wsum[kFabcWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // each thread owns kScanItems consecutive items of the tile
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? len[base + k] : 0;
        s += v[k];
    }
    const int64_t inc = warp_inclusive_scan(s, lane);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int64_t run = tile_off[blockIdx.x] + inc - s;
    for (int w = 0; w < warp; ++w) run += wsum[w];
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) len[base + k] = run;
        run += v[k];
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
static int copy_grid(int64_t n) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n / 4 + kFabcThreads - 1) / kFabcThreads, sm_count() * 8)));
}
static int tile_grid(int64_t n_seq, int ts) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n_seq + ts - 1) / ts, sm_count() * 8)));
}
// one wave of resident blocks of a persistent kernel (each block walks its
// tiles in a pipeline, so blocks beyond one wave would only wait)
template <class Kernel>
static int resident_grid(Kernel kernel, int smem, int64_t n_tiles) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kFabcThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(n_tiles, static_cast<int64_t>(sm_count()) * per_sm)));
}

// the staged kernels compiled for k = 1..4, the generic loop above that
template <bool COUNT, int K>
static void launch_encode_k(int k, int64_t n_tiles, int smem, cudaStream_t s, const int32_t *walks, int64_t n_seq,
                            int32_t L, int ts, const int32_t *ids, int64_t *off, uint8_t *out) {
    k_fabc_encode_st<COUNT, K><<<resident_grid(k_fabc_encode_st<COUNT, K>, smem, n_tiles), kFabcThreads, smem, s>>>(
        walks, n_seq, L, ts, ids, k, COUNT ? nullptr : off, COUNT ? off : nullptr, out);
}
template <bool COUNT>
static void launch_encode_st(int k, int64_t n_tiles, int smem, cudaStream_t s, const int32_t *walks, int64_t n_seq,
                             int32_t L, int ts, const int32_t *ids, int64_t *off, uint8_t *out) {
    switch (k) {
    case 1: launch_encode_k<COUNT, 1>(k, n_tiles, smem, s, walks, n_seq, L, ts, ids, off, out); break;
    case 2: launch_encode_k<COUNT, 2>(k, n_tiles, smem, s, walks, n_seq, L, ts, ids, off, out); break;
    case 3: launch_encode_k<COUNT, 3>(k, n_tiles, smem, s, walks, n_seq, L, ts, ids, off, out); break;
    case 4: launch_encode_k<COUNT, 4>(k, n_tiles, smem, s, walks, n_seq, L, ts, ids, off, out); break;
    default: launch_encode_k<COUNT, 0>(k, n_tiles, smem, s, walks, n_seq, L, ts, ids, off, out); break;
    }
}
template <int K>
static void launch_decode_k(int grid, int smem, cudaStream_t s, const uint8_t *in, int64_t n_seq, int32_t L, int32_t k,
                            int ts, const int64_t *off, const int64_t *total, int64_t cap, int32_t *walks) {
    k_fabc_decode_st<K><<<grid, kFabcThreads, smem, s>>>(in, n_seq, L, k, ts, off, total, cap, walks);
}
static void launch_decode_st(int grid, int smem, cudaStream_t s, const uint8_t *in, int64_t n_seq, int32_t L,
                             int32_t k, int ts, const int64_t *off, const int64_t *total, int64_t cap, int32_t *walks) {
    switch (k) {
    case 1: launch_decode_k<1>(grid, smem, s, in, n_seq, L, k, ts, off, total, cap, walks); break;
    case 2: launch_decode_k<2>(grid, smem, s, in, n_seq, L, k, ts, off, total, cap, walks); break;
    case 3: launch_decode_k<3>(grid, smem, s, in, n_seq, L, k, ts, off, total, cap, walks); break;
    case 4: launch_decode_k<4>(grid, smem, s, in, n_seq, L, k, ts, off, total, cap, walks); break;
    default: launch_decode_k<0>(grid, smem, s, in, n_seq, L, k, ts, off, total, cap, walks); break;
    }
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
    if ((reinterpret_cast<uintptr_t>(out) & 3u) || (reinterpret_cast<uintptr_t>(walks) & 3u)) return FELOG_ERR_INVALID_ARG;
    if (out_bytes < felog_fabc_max_bytes(n_seq, L, k)) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_fabc_workspace_bytes(n_seq)) return FELOG_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    FabcWorkspace w = carve_fabc(c, n_seq);
    if (n_seq == 0) return record_cuda_error(cudaMemsetAsync(tail, 0, sizeof(int64_t), s), "fabc");
    if (k == 0) {
        k_fabc_copy<<<copy_grid(n_seq * L), kFabcThreads, 0, s>>>(walks, n_seq * L, n_seq * L,
                                                                  reinterpret_cast<int32_t *>(out), tail);
        return check_launch("felog_fabc_encode");
    }
    const int ts = encode_tile_seqs(L, k);
    const int smem = ts ? encode_stage_bytes(ts, L, k) : 0;
    // tail lengths, then their offsets
    const int64_t n_tiles = ts ? (n_seq + ts - 1) / ts : 0;
    if (ts)
        launch_encode_st<true>(k, n_tiles, smem, s, walks, n_seq, L, ts, ids, w.off, out);
    else
        k_fabc_encode_g<true><<<seq_grid(n_seq), kFabcThreads, 0, s>>>(walks, n_seq, L, ids, k, nullptr, w.off, out);
    felog_status st = scan_offsets(w, n_seq, tail, s);
    if (st) return st;
    if (ts)
        launch_encode_st<false>(k, n_tiles, smem, s, walks, n_seq, L, ts, ids, w.off, out);
    else
        k_fabc_encode_g<false><<<seq_grid(n_seq), kFabcThreads, 0, s>>>(walks, n_seq, L, ids, k, w.off, nullptr, out);
    return check_launch("felog_fabc_encode");
}

extern "C" felog_status felog_fabc_decode(const uint8_t *in, size_t in_bytes, int64_t n_seq, int32_t L, int32_t k,
                                          int32_t *walks, void *workspace, size_t workspace_bytes, void *stream) {
    if (n_seq < 0 || L < 1 || k < 0 || k > kFabcMaxK) return FELOG_ERR_INVALID_ARG;
    const int64_t head = 4 * n_seq * k + n_seq * k * ((L + 7) / 8);
    if (static_cast<int64_t>(in_bytes) < head) return FELOG_ERR_INVALID_ARG;
    if (n_seq > 0 && (!in || !walks)) return FELOG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in) & 3u) || (reinterpret_cast<uintptr_t>(walks) & 3u)) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_fabc_workspace_bytes(n_seq)) return FELOG_ERR_WORKSPACE;
    if (n_seq == 0) return FELOG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    FabcWorkspace w = carve_fabc(c, n_seq);
    int64_t *total = reinterpret_cast<int64_t *>(w.total);
    const int64_t cap = (static_cast<int64_t>(in_bytes) - head) / 4;
    if (k == 0) {
        k_fabc_copy<<<copy_grid(n_seq * L), kFabcThreads, 0, s>>>(reinterpret_cast<const int32_t *>(in), cap,
                                                                  n_seq * L, walks, nullptr);
        return check_launch("felog_fabc_decode");
    }
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n_seq + kFabcThreads - 1) / kFabcThreads, sm_count() * 8)));
    k_fabc_tail_len_dec<<<grid, kFabcThreads, 0, s>>>(in + 4 * n_seq * k, n_seq, L, k, w.off);
    felog_status st = scan_offsets(w, n_seq, total, s);
    if (st) return st;
    const int ts = decode_tile_seqs(L, k);
    if (ts)
        launch_decode_st(tile_grid(n_seq, ts), decode_stage_bytes(ts, L, k), s, in, n_seq, L, k, ts, w.off, total, cap,
                         walks);
    else
        k_fabc_decode_g<<<seq_grid(n_seq), kFabcThreads, 0, s>>>(in, n_seq, L, k, w.off, cap, walks);
    return check_launch("felog_fabc_decode");
}
