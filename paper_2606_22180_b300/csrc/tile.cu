// Shared-negatives tile form of Eq. 2 on the tensor cores (tcgen05).
//
// Estimator (a variant of the per-pair draws of Eq. 2): tile t holds the
// centers at corpus positions [t*Tc, t*Tc + Tc) (position = walk*L + pos,
// Tc = 128 - 2w); the tile draws Ns negatives once, draw j from
// Philox(x0 = j, x1 = t, x2 = round, stream 7) and the alias table; every
// pair (context x, center c) of the tile uses all Ns of them with weight
// K / Ns, skipping a negative equal to c.  eta is the rate of the tile's
// first center.  Scores read the tables as they stood when the tile's rows
// were gathered; the summed increments are added when the tile ends.
//
// One CTA of 8 warps per SM works through tiles (warps g and g + 4 share
// the tensor-memory lanes of rows 32g .. 32g + 31 and split each epilogue's
// columns between them).  A tile's 128 rows are the
// positions [t*Tc - w, t*Tc - w + 128): every context of the tile's centers
// lies among them.  With X = phi_in of those positions (128 x d) and
// Y = [phi_out of the positions; phi_out of the Ns negatives] (128 + Ns
// rows), three bf16 contractions with f32 accumulation in tensor memory do
// the dense work:
//   S  = X Y^T        scores of every (position, target) pair
//   G  = grad(S)      epilogue on CUDA cores: positives on the band
//                     |p - q| <= w of the same walk, negatives weighted by
//                     K/Ns times the row's pair count (minus pairs whose
//                     center equals the negative)
//   dX = G Y          increments of phi_in rows
//   dY = G^T X        increments of phi_out rows
// The increments are added to the tables with vector reductions (bf16
// tables: stochastically rounded increments against the gathered values).
//
// Shared memory (no-swizzle core-matrix layout, see tc_core.cuh): X
// 128 x d, Y (128 + Ns) x d, G 128 x (128 + Ns), all bf16; with bf16 tables
// and tiles allowed to overlap, a second X/Y stage receives the next tile's
// rows (cp.async) while this tile computes.  Tensor memory: 512 columns; S
// in columns [0, 128 + Ns), dX in [256, 256 + d), dY reuses [0, 2d) once S
// has been read (positions 0..127, then rows NY - 128 .. NY - 1 of G^T X,
// whose last Ns are the negatives).
#include <algorithm>
#include <type_traits>

#include "sgns_core.cuh"
#include "tc_core.cuh"

namespace felog {

constexpr uint32_t kStreamTile = 7;
constexpr int kTileThreads = 256;  // 8 warps; warps g and g + 4 share TMEM lanes 32g ..
constexpr int kTileRows = 128;
constexpr uint32_t kTileWaitLimit = 1u << 26;  // polls of an mbarrier before reporting a timeout

struct TileArgs {
    const int32_t *walks;
    int64_t total;  // n_walks * L
    int64_t n_tiles;
    int32_t L, n, window, K, Ns, Tc;
    float lr0;
    double inv_total;  // 1 / lr_total_tokens
    int64_t clock_base;
    const uint64_t *thr;
    const int32_t *alias;
    const uint64_t *S;
    uint64_t seed;
    uint32_t round;
    unsigned long long *loss_acc;
    int32_t *timeout;
    float *scratch;  // in-order form: dY rows of a tile, added when the tile ends (else null)
};

// 8 floats -> 8 bf16 (round to nearest) packed in 4 words
__device__ __forceinline__ uint4 pack8(const float4 &a, const float4 &b) {
    uint4 r;
    __nv_bfloat162 h;
    h = __floats2bfloat162_rn(a.x, a.y); r.x = *reinterpret_cast<uint32_t *>(&h);
    h = __floats2bfloat162_rn(a.z, a.w); r.y = *reinterpret_cast<uint32_t *>(&h);
    h = __floats2bfloat162_rn(b.x, b.y); r.z = *reinterpret_cast<uint32_t *>(&h);
    h = __floats2bfloat162_rn(b.z, b.w); r.w = *reinterpret_cast<uint32_t *>(&h);
    return r;
}

__device__ __forceinline__ uint4 ld_row8(const float *p) {
    float4 a, b;
    asm volatile("ld.global.cg.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w) : "l"(p));
    asm volatile("ld.global.cg.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w) : "l"(p + 4));
    return pack8(a, b);
}
__device__ __forceinline__ uint4 ld_row8(const __nv_bfloat16 *p) {
    uint4 r;
    asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

// current packed bf16 values of p[0..8) (the rounding reference of add8);
// float tables need none
__device__ __forceinline__ uint4 ld_row8_raw(const __nv_bfloat16 *p) { return ld_row8(p); }
__device__ __forceinline__ uint4 ld_row8_raw(const float *) { return make_uint4(0, 0, 0, 0); }

// 16-byte asynchronous copy global -> shared (L2 only); src_bytes = 0
// writes zeros without reading.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// number of set bits of the 128-bit mask m[0..4) at positions lo..hi
__device__ __forceinline__ int popc_range(const uint32_t *m, int lo, int hi) {
    int c = 0;
#pragma unroll
    for (int wd = 0; wd < 4; ++wd) {
        const int a = max(lo - 32 * wd, 0), b = min(hi - 32 * wd, 31);
        if (a <= b) {
            const uint32_t sel = (b - a == 31) ? 0xffffffffu : (((1u << (b - a + 1)) - 1u) << a);
            c += __popc(m[wd] & sel);
        }
    }
    return c;
}

// Adds 8 increments (f32) to table elements p[0..8); `snap` holds the 8
// gathered values as packed bf16 (used by bf16 tables for stochastic
// rounding of gathered value + increment).
__device__ __forceinline__ void add8(float *p, const float *d, uint4, uint32_t) {
    red_add_v4(p, d[0], d[1], d[2], d[3]);
    red_add_v4(p + 4, d[4], d[5], d[6], d[7]);
}
__device__ __forceinline__ void add8(__nv_bfloat16 *p, const float *d, uint4 snap, uint32_t w) {
    const uint32_t raw[4] = {snap.x, snap.y, snap.z, snap.w};
    float dd[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) dd[i] = d[i];
    add_delta_raw<8>(p, raw, dd, w);
}

// sigma(s) and log(1 + exp(-|s|)) from one exponential
__device__ __forceinline__ void sigmoid_softplus(float s, float &sig, float &l1p) {
    const float e = __expf(-fabsf(s));
    const float r = __fdividef(1.f, 1.f + e);
    sig = s >= 0.f ? r : e * r;
    l1p = __logf(1.f + e);
}

constexpr int kMaxNegBlocks = 4;                   // Ns <= 512
constexpr int kMaxNs = 128 * kMaxNegBlocks;

// Per-tile bookkeeping in shared memory (two, for the current and the next
// tile).
struct TileStage {
    int32_t node[kTileRows];                 // node of each row position (-1: none)
    int16_t lo[kTileRows], hi[kTileRows];    // rows of the same walk as row q
    int32_t neg[kMaxNs];                     // shared negatives
    uint32_t negm[kTileRows][kMaxNs / 32];   // center p: bit j set where negative j equals it
    uint32_t valid[4];                       // bit p: row p is a center with a node
    uint32_t hitm[4];                        // bit p: that center equals a shared negative
    uint32_t nodem[4];                       // bit p: row p holds a node
    uint32_t bloom[128];                     // 4096-bit filter of the negatives
    uint16_t rows_x[kTileRows];              // rows of node[q] among contexts in a pair (phi_in)
    uint16_t rows_c[kTileRows];              // rows of node[p] among centers in a pair and negatives (phi_out)
    uint16_t rows_n[kMaxNs];                 // the same count for negative j
};

// Pairs of row q: centers p in [plo, phi] \ {q} with a node (phi < plo: none).
__device__ __forceinline__ int row_pairs(const TileStage &S, int q, int w, int Tc, int &plo, int &phi) {
    plo = max(max(q - w, w), static_cast<int>(S.lo[q]));
    phi = min(min(q + w, w + Tc - 1), static_cast<int>(S.hi[q]));
    if (S.node[q] < 0) phi = plo - 1;
    uint32_t vm[4];
#pragma unroll
    for (int wd = 0; wd < 4; ++wd) vm[wd] = S.valid[wd];
    const bool q_in = q >= plo && q <= phi;
    return popc_range(vm, plo, phi) - (q_in ? static_cast<int>(S.valid[q >> 5] >> (q & 31) & 1u) : 0);
}
// Center p takes part in a pair: a valid center with another node of its walk within w.
__device__ __forceinline__ bool center_used(const TileStage &S, int p, int w) {
    if (!(S.valid[p >> 5] >> (p & 31) & 1u)) return false;
    uint32_t nm[4];
#pragma unroll
    for (int wd = 0; wd < 4; ++wd) nm[wd] = S.nodem[wd];
    return popc_range(nm, max(p - w, static_cast<int>(S.lo[p])), min(p + w, static_cast<int>(S.hi[p]))) > 1;
}

// Open-addressing table node -> (rows in phi_in, rows in phi_out), 1024
// slots, in shared memory; a tile holds at most 128 + 128 + 512 distinct
// nodes, so every probe sequence ends.
constexpr uint32_t kRowHashSlots = 1024;
__device__ __forceinline__ uint32_t row_hash_slot(uint32_t *keys, int32_t v, bool insert) {
    uint32_t h = (static_cast<uint32_t>(v) * 0x9E3779B1u) >> 22;
    for (uint32_t probe = 0; probe < kRowHashSlots; ++probe) {
        const uint32_t k = insert ? atomicCAS(&keys[h], 0xffffffffu, static_cast<uint32_t>(v)) : keys[h];
        if (k == static_cast<uint32_t>(v) || (insert && k == 0xffffffffu)) return h;
        h = (h + 1) & (kRowHashSlots - 1);
    }
    return 0;  // not reached
}

// Dynamic shared memory: two X buffers, a ring of three Y blocks, one G;
// each 128 x 128 (G) or 128 x d bf16 in the core-matrix layout.
__host__ __device__ inline uint32_t tile_smem_bytes(int D) { return (2 + 3) * kTileRows * D * 2 + kTileRows * 128 * 2; }

template <int D, class T>
__global__ void __launch_bounds__(kTileThreads, 1)
    k_sgns_tile(TileArgs a, T *__restrict__ phi_in, T *__restrict__ phi_out) {
    constexpr bool kAsync = std::is_same<T, __nv_bfloat16>::value;
    constexpr uint32_t kBuf = kTileRows * D * 2;  // one X or Y buffer
    constexpr uint32_t kXo = 0, kYo = 2 * kBuf, kGo = 5 * kBuf;
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ TileStage st_s[2];
    __shared__ __align__(8) uint64_t bar_s[3];  // [0]: S ready, [1]: dX/dY ready, [2]: drain after a timeout
    __shared__ uint32_t tmem_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = smem_addr(sm);
    const uint32_t bar_S = smem_addr(&bar_s[0]), bar_D = smem_addr(&bar_s[1]), bar_Z = smem_addr(&bar_s[2]);
    const int w = a.window, Ns = a.Ns, P = Ns / 128, NB = P + 1;  // column blocks per tile
    const uint64_t nn = static_cast<uint64_t>(a.n), Ssum = *a.S;
    const float omega = static_cast<float>(a.K) / static_cast<float>(Ns);
    const bool inorder = a.scratch != nullptr;  // tiles strictly in order, dY staged until the tile ends
    // epilogue roles: warps g and g + 4 share TMEM lanes 32g .. 32g + 31
    const int quarter = warp & 3, half = warp >> 2;
    const int q = quarter * 32 + lane;  // row of this thread in the epilogues

    auto tile_of = [&](int64_t B) { return blockIdx.x + (B / NB) * static_cast<int64_t>(gridDim.x); };

    // Rows, shared negatives, masks and row counts of tile t into stage `sg`;
    // hash_off: a free 8 KB of dynamic shared memory (the Y slot filled next).
    auto setup = [&](int sg, int64_t t, uint32_t hash_off) {
        TileStage &S = st_s[sg];
        const int64_t pos0 = t * a.Tc - w;  // corpus position of row 0
        if (tid < kTileRows) {
            const int64_t pos = pos0 + tid;
            int32_t v = -1;
            int lo = 1, hi = 0;
            if (pos >= 0 && pos < a.total) {
                v = walk_id(__ldg(a.walks + pos), static_cast<uint64_t>(a.n));
                const int64_t wstart = pos - pos % a.L;  // first position of this walk
                const int64_t wend = (wstart + a.L < a.total ? wstart + a.L : a.total) - 1;  // last position
                lo = wstart > pos0 ? static_cast<int>(wstart - pos0) : 0;
                hi = wend - pos0 < kTileRows - 1 ? static_cast<int>(wend - pos0) : kTileRows - 1;
            }
            S.node[tid] = v;
            S.lo[tid] = static_cast<int16_t>(lo);
            S.hi[tid] = static_cast<int16_t>(hi);
            S.bloom[tid] = 0;
        }
        __syncthreads();
        for (int j = tid; j < Ns; j += kTileThreads) {
            const u32x4 r = philox(a.seed, static_cast<uint32_t>(j), static_cast<uint32_t>(t), a.round, kStreamTile);
            const uint64_t b = mulhi64(lo64(r), nn);
            const uint64_t coin = mulhi64(hi64(r), Ssum);
            const uint64_t th = __ldg(reinterpret_cast<const unsigned long long *>(a.thr) + b);
            const int32_t v = coin < th ? static_cast<int32_t>(b) : __ldg(a.alias + b);
            S.neg[j] = v;
            atomicOr(&S.bloom[(static_cast<uint32_t>(v) * 0x9E3779B1u) >> 25], 1u << (v & 31));
        }
        __syncthreads();
        // valid centers, row nodes, and centers equal to a negative (exact
        // check behind the bloom filter), as 128-bit masks
        if (tid < kTileRows) {
            const int32_t v = S.node[tid];
            const bool valid = v >= 0 && tid >= w && tid < w + a.Tc;
            bool hit = false;
            if (valid && (S.bloom[(static_cast<uint32_t>(v) * 0x9E3779B1u) >> 25] >> (v & 31) & 1u)) {
                uint32_t any = 0;
                for (int wd = 0; wd < Ns / 32; ++wd) {
                    uint32_t mw = 0;
                    for (int b = 0; b < 32; ++b) mw |= (S.neg[32 * wd + b] == v ? 1u : 0u) << b;
                    S.negm[tid][wd] = mw;
                    any |= mw;
                }
                hit = any != 0;
            }
            const uint32_t vb = __ballot_sync(kFull, valid), hb = __ballot_sync(kFull, hit);
            const uint32_t nb = __ballot_sync(kFull, v >= 0);
            if (lane == 0) {
                S.valid[warp] = vb;
                S.hitm[warp] = hb;
                S.nodem[warp] = nb;
            }
        }
        // rows per node: the averaging of a node's increments over its rows
        uint32_t *hkey = reinterpret_cast<uint32_t *>(sm + hash_off);
        uint32_t *hcnt = hkey + kRowHashSlots;  // rows in phi_in (low 16 bits), phi_out (high 16)
        for (uint32_t e = tid; e < kRowHashSlots; e += kTileThreads) {
            hkey[e] = 0xffffffffu;
            hcnt[e] = 0;
        }
        __syncthreads();
        bool ctx = false, ctr = false;
        if (tid < kTileRows) {
            int plo_, phi_;
            ctx = row_pairs(S, tid, w, a.Tc, plo_, phi_) > 0;
            ctr = center_used(S, tid, w);
            if (ctx) atomicAdd(&hcnt[row_hash_slot(hkey, S.node[tid], true)], 1u);
            if (ctr) atomicAdd(&hcnt[row_hash_slot(hkey, S.node[tid], true)], 1u << 16);
        }
        for (int j = tid; j < Ns; j += kTileThreads)
            atomicAdd(&hcnt[row_hash_slot(hkey, S.neg[j], true)], 1u << 16);
        __syncthreads();
        if (tid < kTileRows) {
            const uint32_t c = (ctx || ctr) ? hcnt[row_hash_slot(hkey, S.node[tid], false)] : 0u;
            S.rows_x[tid] = ctx ? static_cast<uint16_t>(c & 0xffffu) : 1;
            S.rows_c[tid] = ctr ? static_cast<uint16_t>(c >> 16) : 1;
        }
        for (int j = tid; j < Ns; j += kTileThreads)
            S.rows_n[j] = static_cast<uint16_t>(hcnt[row_hash_slot(hkey, S.neg[j], false)] >> 16);
        __syncthreads();  // before the gather reuses the table's memory
    };

    // 128 rows into a buffer, as bf16 in the core-matrix layout: kind 0 =
    // phi_in of the positions (X), 1 = phi_out of the centers (Y, block 0),
    // 2 = phi_out of negatives 128 (b - 1) .. (Y, block b >= 1).  bf16
    // tables: asynchronous copies (finished by cp.async waits); float
    // tables: converting loads.
    auto gather = [&](uint32_t off, const TileStage &S, int kind, int b) {
        const int r8 = lane & 7, cq = lane >> 3;  // row within group, chunk within 4
        constexpr int kUnitsPerGroup = D / 32;    // 4 chunks of 8 per unit
#pragma unroll 4
        for (int u = warp; u < 16 * kUnitsPerGroup; u += kTileThreads / 32) {
            const int r = (u / kUnitsPerGroup) * 8 + r8, c = ((u % kUnitsPerGroup) * 4 + cq) * 8;
            int32_t v;
            if (kind == 0) v = S.node[r];
            else if (kind == 1) v = (r >= w && r < w + a.Tc) ? S.node[r] : -1;  // centers only
            else v = S.neg[128 * (b - 1) + r];
            const T *src = (kind == 0 ? phi_in : phi_out) + static_cast<int64_t>(max(v, 0)) * D + c;
            const uint32_t o = off + core_offset(r, c, kTileRows);
            if constexpr (kAsync) {
                cp_async16(base + o, src, v >= 0 ? 16u : 0u);
            } else {
                uint4 val = make_uint4(0, 0, 0, 0);
                if (v >= 0) val = ld_row8(src);
                *reinterpret_cast<uint4 *>(sm + o) = val;
            }
        }
    };
    // data of block B: stage, X buffer, Y ring slot
    auto fetch_block = [&](int64_t B) {
        const int64_t k = B / NB;
        const int b = static_cast<int>(B % NB);
        const TileStage &S = st_s[k & 1];
        if (b == 0) gather(kXo + (k & 1) * kBuf, S, 0, 0);
        gather(kYo + (B % 3) * kBuf, S, b == 0 ? 1 : 2, b);
    };
    auto issue_s = [&](int64_t B) {  // S_B = X Y_B^T into TMEM region B % 2
        const uint32_t xs = base + kXo + ((B / NB) & 1) * kBuf, ys = base + kYo + (B % 3) * kBuf;
#pragma unroll
        for (int s = 0; s < D / 16; ++s)
            mma_bf16(tmem_s + (B & 1) * 128, smem_desc(xs + 2 * s * 2048, 2048, 128), smem_desc(ys + 2 * s * 2048, 2048, 128),
                     mma_idesc_bf16(128, 128, 0, 0), s > 0);
    };

    if (tid == 0) {
        mbar_init(bar_S, 1);
        mbar_init(bar_D, 1);
        mbar_init(bar_Z, 1);
    }
    if (warp == 0) tmem_alloc(smem_addr(&tmem_s), 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tmem_s;
    const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
    const uint32_t tdx = tm + lane_off + 256;  // dX of this thread's row
    uint32_t ph_S = 0, ph_D = 0;
    double loss = 0.0;
    bool failed = false;
    const int64_t n_blocks = ((a.n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x) * NB;  // this CTA's blocks

    // per-row state of the current tile (set by block 0)
    int32_t vq = -1;
    int plo = 0, phi = -1, cnt = 0;
    bool any_hit = false;
    uint32_t sr = 1;
    float eta = 0.f;

    if (n_blocks > 0) {
        setup(0, tile_of(0), kYo);
        fetch_block(0);
        if (!inorder && n_blocks > 1) fetch_block(1);
        if constexpr (kAsync) cp_async_wait_all();
        fence_async_smem();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            issue_s(0);
            mma_commit(bar_S);
        }
    }
    for (int64_t B = 0; B < n_blocks; ++B) {
        const int64_t k = B / NB, t = tile_of(B);
        const int b = static_cast<int>(B % NB);
        const TileStage &S = st_s[k & 1];
        const uint32_t xo = kXo + (k & 1) * kBuf, yo = kYo + (B % 3) * kBuf;
        const uint32_t treg = tm + lane_off + (B & 1) * 128;  // S_B, then dY_B
        failed = !mbar_wait(bar_S, ph_S, kTileWaitLimit);
        ph_S ^= 1;
        tc_fence_after();
        if (__syncthreads_or(failed)) break;
        // ---- epilogue 1: G = gradient of block b's scores (bf16) --------------
        if (b == 0) {
            vq = S.node[q];
            eta = static_cast<float>(static_cast<double>(a.lr0) *
                                     fmax(1e-4, 1.0 - static_cast<double>(a.clock_base + t * a.Tc) * a.inv_total));
            cnt = row_pairs(S, q, w, a.Tc, plo, phi);
            uint32_t hm[4];
#pragma unroll
            for (int wd = 0; wd < 4; ++wd) hm[wd] = S.hitm[wd];
            const bool q_in = q >= plo && q <= phi;
            any_hit = popc_range(hm, plo, phi) - (q_in ? static_cast<int>(S.hitm[q >> 5] >> (q & 31) & 1u) : 0) > 0;
            const u32x4 rw = philox(a.seed, static_cast<uint32_t>(t), static_cast<uint32_t>(q | (half << 8)), a.round, kStreamSR);
            sr = rw.x | 1u;
        }
        float row_loss = 0.f;
        if (b == 0) {
            // positive band, columns 32c .. 32c+31: half 0 takes the warp's own
            // chunk, half 1 the other three (two band edges and a zero chunk).
            // Scores outside a row's pairs get coefficient 0 (no branches).
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                if ((c == quarter) != (half == 0)) continue;  // warp-uniform
                uint32_t packed[16];
                if (c >= quarter - 1 && c <= quarter + 1) {
                    uint32_t r[32];
                    tmem_ld32(treg + 32 * c, r);
                    uint32_t pm = S.valid[c];  // pairs of row q among columns 32c .. 32c+31
                    const int a0 = plo - 32 * c, b0 = phi - 32 * c;
                    pm &= (a0 <= 0 ? 0xffffffffu : (a0 >= 32 ? 0u : (0xffffffffu << a0)));
                    pm &= (b0 >= 31 ? 0xffffffffu : (b0 < 0 ? 0u : (0xffffffffu >> (31 - b0))));
                    if (q >= 32 * c && q < 32 * c + 32) pm &= ~(1u << (q - 32 * c));
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        float g2[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float on = static_cast<float>(pm >> (i + h) & 1u);
                            const float s = __uint_as_float(r[i + h]);
                            float sig, l1p;
                            sigmoid_softplus(s, sig, l1p);
                            g2[h] = on * eta * (1.f - sig);
                            row_loss += on * (fmaxf(-s, 0.f) + l1p);  // -log sigma(s)
                        }
                        __nv_bfloat162 hv = __floats2bfloat162_rn(g2[0], g2[1]);
                        packed[i / 2] = *reinterpret_cast<uint32_t *>(&hv);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) packed[i] = 0;
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    *reinterpret_cast<uint4 *>(sm + kGo + core_offset(q, 32 * c + 8 * kk, kTileRows)) =
                        make_uint4(packed[4 * kk], packed[4 * kk + 1], packed[4 * kk + 2], packed[4 * kk + 3]);
            }
        } else {
            // shared negatives 128 (b - 1) + 32c + i: half 0 chunks 0 and 2, half 1 chunks 1 and 3
#pragma unroll 1
            for (int c = half; c < 4; c += 2) {
                uint32_t r[32];
                tmem_ld32(treg + 32 * c, r);
                float mk[32];  // pairs of row q that count this negative
#pragma unroll
                for (int i = 0; i < 32; ++i) mk[i] = static_cast<float>(cnt);
                if (any_hit) {  // pairs whose center is this negative do not count
                    const int word = 4 * (b - 1) + c;
#pragma unroll
                    for (int wd = 0; wd < 4; ++wd) {
                        const int a0 = plo - 32 * wd, b0 = phi - 32 * wd;
                        uint32_t hb = S.hitm[wd];
                        hb &= (a0 <= 0 ? 0xffffffffu : (a0 >= 32 ? 0u : (0xffffffffu << a0)));
                        hb &= (b0 >= 31 ? 0xffffffffu : (b0 < 0 ? 0u : (0xffffffffu >> (31 - b0))));
                        if ((q >> 5) == wd) hb &= ~(1u << (q & 31));
                        while (hb) {
                            const int p = 32 * wd + __ffs(hb) - 1;
                            hb &= hb - 1;
                            const uint32_t mw = S.negm[p][word];
#pragma unroll
                            for (int i = 0; i < 32; ++i) mk[i] -= static_cast<float>(mw >> i & 1u);
                        }
                    }
                }
                tmem_wait_ld();
                uint32_t packed[16];
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    float g2[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float s = __uint_as_float(r[i + h]);
                        float sig, l1p;
                        sigmoid_softplus(s, sig, l1p);
                        g2[h] = -eta * omega * mk[i + h] * sig;
                        row_loss += omega * mk[i + h] * (fmaxf(s, 0.f) + l1p);  // -log sigma(-s)
                    }
                    __nv_bfloat162 hv = __floats2bfloat162_rn(g2[0], g2[1]);
                    packed[i / 2] = *reinterpret_cast<uint32_t *>(&hv);
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    *reinterpret_cast<uint4 *>(sm + kGo + core_offset(q, 32 * c + 8 * kk, kTileRows)) =
                        make_uint4(packed[4 * kk], packed[4 * kk + 1], packed[4 * kk + 2], packed[4 * kk + 3]);
            }
        }
        loss += static_cast<double>(row_loss);
        // the next block's rows must have landed before its S is issued
        if constexpr (kAsync) cp_async_wait_all();
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- dX (+)= G Y_b; dY_b = G^T X; then S of the next block -----------
        const bool has_next = B + 1 < n_blocks;
        const bool next_is_new_tile = (B + 1) % NB == 0;
        if (tid == 0) {
            const uint32_t gs = base + kGo, xs = base + xo, ys = base + yo;  // G, X, Y_b
#pragma unroll
            for (int s = 0; s < 8; ++s)
                mma_bf16(tm + 256, smem_desc(gs + 2 * s * 2048, 2048, 128), smem_desc(ys + 2 * s * 128, 128, 2048),
                         mma_idesc_bf16(128, D, 0, 1), b > 0 || s > 0);
#pragma unroll
            for (int s = 0; s < 8; ++s)
                mma_bf16(tm + (B & 1) * 128, smem_desc(gs + 2 * s * 128, 128, 2048), smem_desc(xs + 2 * s * 128, 128, 2048),
                         mma_idesc_bf16(128, D, 1, 1), s > 0);
            mma_commit(bar_D);
            if (has_next && !inorder) {  // its rows landed before the barrier above
                issue_s(B + 1);
                mma_commit(bar_S);
            }
        }
        // ---- meanwhile: rows of block B + 2 (a new tile's setup first) -------
        if (!inorder && B + 2 < n_blocks) {
            if ((B + 2) % NB == 0) setup(((B + 2) / NB) & 1, tile_of(B + 2), kYo + ((B + 2) % 3) * kBuf);
            fetch_block(B + 2);
        } else if (inorder && has_next && !next_is_new_tile) {
            fetch_block(B + 1);  // in order: the next block of this tile; its S is issued after epilogue 2
        }
        failed = !mbar_wait(bar_D, ph_D, kTileWaitLimit);
        ph_D ^= 1;
        tc_fence_after();
        if (__syncthreads_or(failed)) break;
        // ---- epilogue 2: add dY_b (and dX at the tile's last block) ------------
        {
            const int c0 = half == 0 ? 0 : (D / 32 + 1) / 2, c1 = half == 0 ? (D / 32 + 1) / 2 : D / 32;
            bool use;
            T *prow;
            float scale;  // 1 / rows of this node in phi_out in this tile
            if (b == 0) {  // center q: used iff it takes part in a pair
                use = center_used(S, q, w);
                prow = phi_out + static_cast<int64_t>(max(S.node[q], 0)) * D;
                scale = 1.f / static_cast<float>(S.rows_c[q]);
            } else {  // a negative row is always added (a zero increment changes nothing)
                use = true;
                prow = phi_out + static_cast<int64_t>(S.neg[128 * (b - 1) + q]) * D;
                scale = 1.f / static_cast<float>(S.rows_n[128 * (b - 1) + q]);
            }
            float *scr = inorder ? a.scratch + (static_cast<int64_t>(b) * kTileRows + q) * D : nullptr;
#pragma unroll 1
            for (int c = c0; c < c1; ++c) {
                uint32_t r[32];
                tmem_ld32(treg + 32 * c, r);
                tmem_wait_ld();
                if (!use) continue;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int col = 32 * c + 8 * kk;
                    float d8[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) d8[i] = scale * __uint_as_float(r[8 * kk + i]);
                    if (inorder) {
                        *reinterpret_cast<float4 *>(scr + col) = make_float4(d8[0], d8[1], d8[2], d8[3]);
                        *reinterpret_cast<float4 *>(scr + col + 4) = make_float4(d8[4], d8[5], d8[6], d8[7]);
                    } else {
                        const uint4 snap = *reinterpret_cast<const uint4 *>(sm + yo + core_offset(q, col, kTileRows));
                        add8(prow + col, d8, snap, xorshift32(sr));
                    }
                }
            }
            if (inorder && !use) {
                for (int c = c0; c < c1; ++c)
                    for (int col = 32 * c; col < 32 * c + 32; col += 4)
                        *reinterpret_cast<float4 *>(scr + col) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (b == NB - 1) {  // dX of row q
                const bool ux = vq >= 0 && cnt > 0;
                T *px = phi_in + static_cast<int64_t>(max(vq, 0)) * D;
                const float sx = 1.f / static_cast<float>(S.rows_x[q]);
#pragma unroll 1
                for (int c = c0; c < c1; ++c) {
                    uint32_t r[32];
                    tmem_ld32(tdx + 32 * c, r);
                    tmem_wait_ld();
                    if (!ux) continue;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int col = 32 * c + 8 * kk;
                        float d8[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) d8[i] = sx * __uint_as_float(r[8 * kk + i]);
                        const uint4 snap = *reinterpret_cast<const uint4 *>(sm + xo + core_offset(q, col, kTileRows));
                        add8(px + col, d8, snap, xorshift32(sr));
                    }
                }
            }
        }
        // ---- in order: at the tile's end add the staged dY rows, then read
        //      the next tile (which sees every update of this one) -------------
        if (inorder && b == NB - 1) {
            __syncthreads();
            for (int e = tid; e < NB * kTileRows * (D / 8); e += kTileThreads) {
                const int bb = e / (kTileRows * (D / 8)), row = (e / (D / 8)) % kTileRows, col = (e % (D / 8)) * 8;
                int32_t v;
                if (bb == 0) v = (row >= w && row < w + a.Tc) ? S.node[row] : -1;
                else v = S.neg[128 * (bb - 1) + row];
                if (v < 0) continue;
                const float *src = a.scratch + (static_cast<int64_t>(bb) * kTileRows + row) * D + col;
                float d8[8];
                bool nz = false;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    d8[i] = src[i];
                    nz |= d8[i] != 0.f;
                }
                if (!nz) continue;
                T *p = phi_out + static_cast<int64_t>(v) * D + col;
                add8(p, d8, ld_row8_raw(p), xorshift32(sr));
            }
            __threadfence();
            __syncthreads();
            if (has_next) {
                setup((k + 1) & 1, tile_of(B + 1), kYo + ((B + 1) % 3) * kBuf);
                fetch_block(B + 1);
                if constexpr (kAsync) cp_async_wait_all();
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
                tc_fence_after();
                if (tid == 0) {
                    issue_s(B + 1);
                    mma_commit(bar_S);
                }
            }
        } else if (inorder && has_next) {
            // the next block of this tile was fetched above; issue its S now
            if constexpr (kAsync) cp_async_wait_all();
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                issue_s(B + 1);
                mma_commit(bar_S);
            }
        }
        tc_fence_before();
    }
    if constexpr (kAsync) cp_async_wait_all();  // none left in flight, also after a timeout
    // After a timeout the tables are in an undefined state and the launch has
    // failed (the host reports FELOG_ERR_TIMEOUT).  MMAs committed before the
    // failed wait may still run: one more commit by the issuing thread tracks
    // all of them, and a bounded wait on it lets them finish before the
    // tensor memory they write is freed.
    if (__syncthreads_or(failed)) {
        if (tid == 0) {
            atomicExch(a.timeout, 1);
            mma_commit(bar_Z);
        }
        mbar_wait(bar_Z, 0, kTileWaitLimit);
    }
    long long fx = __double2ll_rn(loss * kLossScale);
    for (int o = 16; o; o >>= 1) fx += __shfl_xor_sync(kFull, fx, o);
    if (lane == 0 && fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(fx));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tm, 512);
}

template <int D, class T>
static felog_status launch_tile_dim(TileArgs a, int ctas, void *pi, void *po, cudaStream_t s) {
    auto kern = k_sgns_tile<D, T>;
    const int bytes = static_cast<int>(std::max<uint32_t>(tile_smem_bytes(D), 122880));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return record_cuda_error(e, "felog_train (tile)");
    kern<<<ctas, kTileThreads, bytes, s>>>(a, static_cast<T *>(pi), static_cast<T *>(po));
    return check_launch("felog_train (tile)");
}

// Rows per concurrent tile under the automatic cap.  A tile adds its summed
// increments to ~750 rows at once, computed from values gathered when it
// began.  With many tiles in flight, those stale steps pile up on shared
// rows (hubs above all).  On 1,000 nodes with one tile per SM training
// diverged; on R-MAT 20 (2^20 nodes, 10 rounds) link AUC fell from 0.832 (8
// tiles) through 0.809 (37) to 0.709 (148).  At most n / kTileRowsPerCta
// tiles run at once: 37 on 2^20 nodes, one on graphs below 56,000 nodes.
constexpr int64_t kTileRowsPerCta = 28000;

// Floats of the in-order form's staging buffer (dY of one tile's blocks).
size_t tile_scratch_floats() { return static_cast<size_t>(kMaxNegBlocks + 1) * kTileRows * 128; }

// Launches the tile trainer over walks[n_walks][L]; called by felog_train
// after argument checks.  tile_ctas <= 0: min(SMs, max(1, n / 28000)) tiles
// at once; 1 runs the tiles in order (the reproducible form, which stages
// each tile's dY rows in `scratch`, tile_scratch_floats() floats).
felog_status launch_tile(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                         const felog_train_params *tp, const uint64_t *thr, const int32_t *alias,
                         const uint64_t *S, uint64_t seed, int32_t round, int64_t clock_base,
                         void *phi_in, void *phi_out, unsigned long long *loss_acc, int32_t *timeout,
                         float *scratch, cudaStream_t s) {
    TileArgs a;
    a.walks = walks;
    a.total = n_walks * L;
    a.L = L;
    a.n = n;
    a.window = tp->window;
    a.K = tp->negatives;
    a.Ns = tp->tile_negatives > 0 ? tp->tile_negatives : kMaxNs;
    a.Tc = kTileRows - 2 * tp->window;
    a.n_tiles = (a.total + a.Tc - 1) / a.Tc;
    a.lr0 = tp->lr0;
    a.inv_total = 1.0 / static_cast<double>(tp->lr_total_tokens);
    a.clock_base = clock_base;
    a.thr = thr;
    a.alias = alias;
    a.S = S;
    a.seed = seed;
    a.round = static_cast<uint32_t>(round);
    a.loss_acc = loss_acc;
    a.timeout = timeout;
    if (a.n_tiles == 0) return FELOG_OK;
    if (a.n_tiles > 0xffffffffLL) return FELOG_ERR_INVALID_ARG;
    int ctas = tp->tile_ctas > 0
                   ? std::min(tp->tile_ctas, sm_count())
                   : static_cast<int>(std::min<int64_t>(sm_count(), std::max<int64_t>(1, n / kTileRowsPerCta)));
    ctas = static_cast<int>(std::min<int64_t>(ctas, a.n_tiles));
    a.scratch = ctas == 1 ? scratch : nullptr;  // one CTA: tiles strictly in order
    const bool f32 = tp->precision == FELOG_FP32;
    switch (tp->dim) {
        case 32: return f32 ? launch_tile_dim<32, float>(a, ctas, phi_in, phi_out, s)
                            : launch_tile_dim<32, __nv_bfloat16>(a, ctas, phi_in, phi_out, s);
        case 64: return f32 ? launch_tile_dim<64, float>(a, ctas, phi_in, phi_out, s)
                            : launch_tile_dim<64, __nv_bfloat16>(a, ctas, phi_in, phi_out, s);
        case 128: return f32 ? launch_tile_dim<128, float>(a, ctas, phi_in, phi_out, s)
                             : launch_tile_dim<128, __nv_bfloat16>(a, ctas, phi_in, phi_out, s);
    }
    return FELOG_ERR_UNSUPPORTED;
}

}  // namespace felog
