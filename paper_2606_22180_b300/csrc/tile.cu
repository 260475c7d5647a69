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
    int32_t prefetch;  // gather the next tile while this one computes (2 stages)
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

// Per-stage tile bookkeeping (shared memory).
struct TileStage {
    int32_t node[kTileRows];       // node of each row position (-1: none)
    int16_t lo[kTileRows], hi[kTileRows];  // rows of the same walk as row q
    int32_t neg[kTileRows];        // shared negatives (Ns used)
    uint32_t negm[kTileRows][4];   // center p: bit j set where negative j equals it
    uint32_t valid[4];             // bit p: row p is a center with a node
    uint32_t hitm[4];              // bit p: that center equals a shared negative
    uint32_t nodem[4];             // bit p: row p holds a node
    uint32_t bloom[32];
};

// Dynamic shared memory: `stages` copies of [X (128 x d) | Y (128 + Ns rows
// x d)], then G (128 x (128 + Ns)), all bf16 in the core-matrix layout.
__host__ __device__ inline uint32_t tile_stage_bytes(int D, int NY) { return (kTileRows + NY) * D * 2; }
__host__ __device__ inline uint32_t tile_smem_bytes(int D, int NY, int stages) {
    const uint32_t b = stages * tile_stage_bytes(D, NY) + kTileRows * NY * 2;
    return b > 122880 ? b : 122880;  // at least 120 KB: one CTA (and its 512 TMEM columns) per SM
}

template <int D, class T>
__global__ void __launch_bounds__(kTileThreads, 1)
    k_sgns_tile(TileArgs a, T *__restrict__ phi_in, T *__restrict__ phi_out) {
    constexpr bool kAsync = std::is_same<T, __nv_bfloat16>::value;
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ TileStage st_s[2];
    __shared__ __align__(8) uint64_t bar_s;
    __shared__ uint32_t tmem_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = smem_addr(sm);
    const uint32_t bar = smem_addr(&bar_s);
    const int w = a.window, Ns = a.Ns, NY = kTileRows + Ns;
    const int stages = a.prefetch ? 2 : 1;
    const uint32_t xbytes = kTileRows * D * 2, sbytes = tile_stage_bytes(D, NY);
    const uint32_t goff = stages * sbytes;  // G
    const uint64_t nn = static_cast<uint64_t>(a.n), Ssum = *a.S;
    const float omega = static_cast<float>(a.K) / static_cast<float>(Ns);
    // epilogue roles: warps g and g + 4 share TMEM lanes 32g .. 32g + 31
    const int quarter = warp & 3, half = warp >> 2;
    const int q = quarter * 32 + lane;  // row of this thread in the epilogues
    const int neg_lane0 = 256 - NY;     // dY lane of the first negative (second half of G^T X)

    // Rows, shared negatives and masks of tile t into stage `sg`.
    auto setup = [&](int sg, int64_t t) {
        TileStage &S = st_s[sg];
        const int64_t pos0 = t * a.Tc - w;  // corpus position of row 0
        if (tid < kTileRows) {
            const int64_t pos = pos0 + tid;
            int32_t v = -1;
            int lo = 1, hi = 0;
            if (pos >= 0 && pos < a.total) {
                v = __ldg(a.walks + pos);
                const int64_t wstart = pos - pos % a.L;  // first position of this walk
                const int64_t wend = (wstart + a.L < a.total ? wstart + a.L : a.total) - 1;  // last position
                lo = wstart > pos0 ? static_cast<int>(wstart - pos0) : 0;
                hi = wend - pos0 < kTileRows - 1 ? static_cast<int>(wend - pos0) : kTileRows - 1;
            }
            S.node[tid] = v;
            S.lo[tid] = static_cast<int16_t>(lo);
            S.hi[tid] = static_cast<int16_t>(hi);
            if (tid < 32) S.bloom[tid] = 0;
        }
        __syncthreads();
        if (tid >= kTileRows && tid < kTileRows + Ns) {
            const int j = tid - kTileRows;
            const u32x4 r = philox(a.seed, static_cast<uint32_t>(j), static_cast<uint32_t>(t), a.round, kStreamTile);
            const uint64_t b = mulhi64(lo64(r), nn);
            const uint64_t coin = mulhi64(hi64(r), Ssum);
            const uint64_t th = __ldg(reinterpret_cast<const unsigned long long *>(a.thr) + b);
            const int32_t v = coin < th ? static_cast<int32_t>(b) : __ldg(a.alias + b);
            S.neg[j] = v;
            atomicOr(&S.bloom[(static_cast<uint32_t>(v) * 0x9E3779B1u) >> 27], 1u << (v & 31));
        }
        __syncthreads();
        // valid centers, row nodes, and centers equal to a negative (exact
        // check behind a bloom filter), as 128-bit masks
        if (tid < kTileRows) {
            const int32_t v = S.node[tid];
            const bool valid = v >= 0 && tid >= w && tid < w + a.Tc;
            bool hit = false;
            if (valid && (S.bloom[(static_cast<uint32_t>(v) * 0x9E3779B1u) >> 27] >> (v & 31) & 1u)) {
                uint32_t mw[4] = {0, 0, 0, 0};
#pragma unroll
                for (int wd = 0; wd < 4; ++wd)
                    for (int b = 0; b < 32 && 32 * wd + b < Ns; ++b) mw[wd] |= (S.neg[32 * wd + b] == v ? 1u : 0u) << b;
                hit = (mw[0] | mw[1] | mw[2] | mw[3]) != 0;
#pragma unroll
                for (int wd = 0; wd < 4; ++wd) S.negm[tid][wd] = mw[wd];
            }
            const uint32_t vb = __ballot_sync(kFull, valid), hb = __ballot_sync(kFull, hit);
            const uint32_t nb = __ballot_sync(kFull, v >= 0);
            if (lane == 0) {
                S.valid[warp] = vb;
                S.hitm[warp] = hb;
                S.nodem[warp] = nb;
            }
        }
    };

    // X (phi_in of positions) and Y (phi_out of centers and negatives) of the
    // tile in stage `sg` into the core-matrix layout, as bf16: asynchronous
    // copies for bf16 tables (completed by cp_async_wait_all), converting
    // loads for float tables.
    auto gather = [&](int sg) {
        const TileStage &S = st_s[sg];
        const uint32_t xo = sg * sbytes, yo = xo + xbytes;
        const int r8 = lane & 7, cq = lane >> 3;  // row within group, chunk within 4
        constexpr int kUnitsPerGroup = D / 32;    // 4 chunks of 8 per unit
        const int units = (kTileRows / 8 + NY / 8) * kUnitsPerGroup;
#pragma unroll 4
        for (int u = warp; u < units; u += kTileThreads / 32) {
            const int gi = u / kUnitsPerGroup, c = ((u % kUnitsPerGroup) * 4 + cq) * 8;
            const bool isx = gi < kTileRows / 8;
            const int r = (isx ? gi : gi - kTileRows / 8) * 8 + r8;
            int32_t v;
            if (isx) v = S.node[r];
            else if (r < kTileRows) v = (r >= w && r < w + a.Tc) ? S.node[r] : -1;  // centers only
            else v = S.neg[r - kTileRows];
            const uint32_t off = isx ? xo + core_offset(r, c, kTileRows) : yo + core_offset(r, c, NY);
            const T *src = (isx ? phi_in : phi_out) + static_cast<int64_t>(max(v, 0)) * D + c;
            if constexpr (kAsync) {
                cp_async16(base + off, src, v >= 0 ? 16u : 0u);
            } else {
                uint4 val = make_uint4(0, 0, 0, 0);
                if (v >= 0) val = ld_row8(src);
                *reinterpret_cast<uint4 *>(sm + off) = val;
            }
        }
    };

    if (tid == 0) mbar_init(bar, 1);
    if (warp == 0) tmem_alloc(smem_addr(&tmem_s), 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tmem_s;
    const uint32_t lane_base = tm + (static_cast<uint32_t>(quarter * 32) << 16);
    uint32_t phase = 0;
    double loss = 0.0;
    bool failed = false;

    int64_t t = blockIdx.x;
    if (t < a.n_tiles) {
        setup(0, t);
        gather(0);
        if constexpr (kAsync) cp_async_wait_all();
        fence_async_smem();
        __syncthreads();
    }
    for (int sg = 0; t < a.n_tiles; t += gridDim.x, sg ^= (stages - 1)) {
        const TileStage &S = st_s[sg];
        const uint32_t xs = base + sg * sbytes, ys = xs + xbytes, gs = base + goff;
        const int64_t tn = t + gridDim.x;  // this CTA's next tile
        // ---- S = X Y^T ---------------------------------------------------------
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < D / 16; ++s)
                mma_bf16(tm, smem_desc(xs + 2 * s * (kTileRows * 16), kTileRows * 16, 128),
                         smem_desc(ys + 2 * s * (NY * 16), NY * 16, 128), mma_idesc_bf16(128, NY, 0, 0), s > 0);
            mma_commit(bar);
        }
        // ---- meanwhile: the next tile's rows into the other stage --------------
        if (stages == 2 && tn < a.n_tiles) {
            setup(sg ^ 1, tn);
            gather(sg ^ 1);
        }
        failed = !mbar_wait(bar, phase, kTileWaitLimit);
        phase ^= 1;
        tc_fence_after();
        if (__syncthreads_or(failed)) break;
        // ---- epilogue: gradient G (bf16).  Row q pairs with the centers
        //      p in [plo, phi] \ {q} whose node is >= 0 ----------------------------
        const int32_t vq = S.node[q];
        const float eta = static_cast<float>(
            static_cast<double>(a.lr0) *
            fmax(1e-4, 1.0 - static_cast<double>(a.clock_base + t * a.Tc) * a.inv_total));
        int plo = max(max(q - w, w), static_cast<int>(S.lo[q]));
        int phi = min(min(q + w, w + a.Tc - 1), static_cast<int>(S.hi[q]));
        if (vq < 0) phi = plo - 1;
        uint32_t vm[4], hm[4], nm[4];
#pragma unroll
        for (int wd = 0; wd < 4; ++wd) {
            vm[wd] = S.valid[wd];
            hm[wd] = S.hitm[wd];
            nm[wd] = S.nodem[wd];
        }
        const bool q_in = q >= plo && q <= phi;
        const int cnt = popc_range(vm, plo, phi) - (q_in ? static_cast<int>(S.valid[q >> 5] >> (q & 31) & 1u) : 0);
        const bool any_hit = popc_range(hm, plo, phi) - (q_in ? static_cast<int>(S.hitm[q >> 5] >> (q & 31) & 1u) : 0) > 0;
        float row_loss = 0.f;
        // positive band, columns 32c .. 32c+31: half 0 takes the warp's own
        // chunk, half 1 the other three (two band edges and a zero chunk).
        // Scores outside a row's pairs get coefficient 0 (no branches).
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            if ((c == quarter) != (half == 0)) continue;  // warp-uniform
            uint32_t packed[16];
            if (c >= quarter - 1 && c <= quarter + 1) {
                uint32_t r[32];
                tmem_ld32(lane_base + 32 * c, r);
                // pairs of row q among columns 32c .. 32c+31
                uint32_t pm = S.valid[c];
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
            for (int k = 0; k < 4; ++k)
                *reinterpret_cast<uint4 *>(sm + goff + core_offset(q, 32 * c + 8 * k, kTileRows)) =
                    make_uint4(packed[4 * k], packed[4 * k + 1], packed[4 * k + 2], packed[4 * k + 3]);
        }
#pragma unroll 1
        for (int c = half; c < Ns / 32; c += 2) {  // shared negatives, columns 128 + 32c ..
            uint32_t r[32];
            tmem_ld32(lane_base + kTileRows + 32 * c, r);
            float mk[32];  // pair count of row q that counts negative 32c + i
#pragma unroll
            for (int i = 0; i < 32; ++i) mk[i] = static_cast<float>(cnt);
            if (any_hit) {  // pairs whose center is this negative do not count
#pragma unroll
                for (int wd = 0; wd < 4; ++wd) {
                    const int a0 = plo - 32 * wd, b0 = phi - 32 * wd;
                    uint32_t hb = hm[wd];
                    hb &= (a0 <= 0 ? 0xffffffffu : (a0 >= 32 ? 0u : (0xffffffffu << a0)));
                    hb &= (b0 >= 31 ? 0xffffffffu : (b0 < 0 ? 0u : (0xffffffffu >> (31 - b0))));
                    if ((q >> 5) == wd) hb &= ~(1u << (q & 31));
                    while (hb) {
                        const int p = 32 * wd + __ffs(hb) - 1;
                        hb &= hb - 1;
                        const uint32_t mw = S.negm[p][c];
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
            for (int k = 0; k < 4; ++k)
                *reinterpret_cast<uint4 *>(sm + goff + core_offset(q, kTileRows + 32 * c + 8 * k, kTileRows)) =
                    make_uint4(packed[4 * k], packed[4 * k + 1], packed[4 * k + 2], packed[4 * k + 3]);
        }
        loss += static_cast<double>(row_loss);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- dX = G Y, dY = G^T X (second half: j in [NY - 128, NY)) --------
        if (tid == 0) {
            for (int s = 0; s < NY / 16; ++s)
                mma_bf16(tm + 256, smem_desc(gs + 2 * s * (kTileRows * 16), kTileRows * 16, 128),
                         smem_desc(ys + 2 * s * 128, 128, NY * 16), mma_idesc_bf16(128, D, 0, 1), s > 0);
            for (int h = 0; h < 2; ++h) {
                const uint32_t g0 = gs + (h ? (NY - kTileRows) / 8 : 0) * (kTileRows * 16);
#pragma unroll
                for (int s = 0; s < kTileRows / 16; ++s)
                    mma_bf16(tm + h * D, smem_desc(g0 + 2 * s * 128, 128, kTileRows * 16),
                             smem_desc(xs + 2 * s * 128, 128, kTileRows * 16), mma_idesc_bf16(128, D, 1, 1), s > 0);
            }
            mma_commit(bar);
        }
        failed = !mbar_wait(bar, phase, kTileWaitLimit);
        phase ^= 1;
        tc_fence_after();
        if (__syncthreads_or(failed)) break;
        // ---- add the increments to the tables: half 0 adds dX of row q and dY
        //      of negative q - (256 - NY), half 1 dY of position q -------------
        {
            const u32x4 rw = philox(a.seed, static_cast<uint32_t>(t), static_cast<uint32_t>(q), a.round, kStreamSR);
            uint32_t sr0 = (half ? rw.z : rw.x) | 1u, sr1 = rw.y | 1u;
            // position q is a center of some pair iff it is a valid center with
            // another node of its walk within w; a negative row is always added
            // (a zero increment leaves a table unchanged)
            bool first;
            if (half == 0) {
                first = vq >= 0 && cnt > 0;
            } else {
                const bool vc = S.valid[q >> 5] >> (q & 31) & 1u;
                const int clo = max(q - w, static_cast<int>(S.lo[q])), chi = min(q + w, static_cast<int>(S.hi[q]));
                first = vc && popc_range(nm, clo, chi) > 1;
            }
            const int jn = q - neg_lane0;  // negative held by this TMEM lane
            const bool second = half == 0 && jn >= 0;
            T *p1 = (half == 0 ? phi_in : phi_out) + static_cast<int64_t>(max(vq, 0)) * D;
            T *p2 = phi_out + static_cast<int64_t>(jn >= 0 ? S.neg[jn] : 0) * D;
            const uint32_t t1 = half == 0 ? lane_base + 256 : lane_base;  // dX or dY(positions)
            const uint32_t s1 = half == 0 ? xs - base : ys - base;
            const int R1 = half == 0 ? kTileRows : NY;
#pragma unroll 1
            for (int c = 0; c < D / 32; ++c) {
                uint32_t r1[32], r2[32];
                tmem_ld32(t1 + 32 * c, r1);
                if (half == 0) tmem_ld32(lane_base + D + 32 * c, r2);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int col = 32 * c + 8 * k;
                    float d8[8];
                    if (first) {
                        const uint4 snap = *reinterpret_cast<const uint4 *>(sm + s1 + core_offset(q, col, R1));
#pragma unroll
                        for (int i = 0; i < 8; ++i) d8[i] = __uint_as_float(r1[8 * k + i]);
                        add8(p1 + col, d8, snap, xorshift32(sr0));
                    }
                    if (second) {
                        const uint4 snap =
                            *reinterpret_cast<const uint4 *>(sm + (ys - base) + core_offset(kTileRows + jn, col, NY));
#pragma unroll
                        for (int i = 0; i < 8; ++i) d8[i] = __uint_as_float(r2[8 * k + i]);
                        add8(p2 + col, d8, snap, xorshift32(sr1));
                    }
                }
            }
        }
        // ---- the next tile: with one stage its rows are read only now, after
        //      these reductions (tiles strictly in order) ------------------------
        if (stages == 1 && tn < a.n_tiles) {
            __threadfence();
            __syncthreads();
            setup(0, tn);
            gather(0);
        }
        if constexpr (kAsync) cp_async_wait_all();
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    }
    if constexpr (kAsync) cp_async_wait_all();  // none left in flight, also after a timeout
    if (failed && tid == 0) atomicExch(a.timeout, 1);
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
    const int NY = kTileRows + a.Ns;
    // two stages (next tile gathered during this one) for bf16 tables when
    // tiles may overlap and the buffers fit; one stage keeps tiles in order
    a.prefetch = std::is_same<T, __nv_bfloat16>::value && ctas > 1 &&
                 tile_smem_bytes(D, NY, 2) + sizeof(TileStage) * 2 + 1024 <= 227 * 1024;
    const int bytes = static_cast<int>(tile_smem_bytes(D, NY, a.prefetch ? 2 : 1));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return record_cuda_error(e, "felog_train (tile)");
    kern<<<ctas, kTileThreads, bytes, s>>>(a, static_cast<T *>(pi), static_cast<T *>(po));
    return check_launch("felog_train (tile)");
}

// Rows per concurrent tile under the automatic cap: a tile adds its summed
// increments to ~300 rows at once, computed from values gathered when it
// began, so too many tiles in flight on a small graph pile stale steps onto
// the same rows and training diverges (1,000 nodes with one tile per SM
// does); at most n / kTileRowsPerCta tiles run at once.
constexpr int64_t kTileRowsPerCta = 2048;

// Launches the tile trainer over walks[n_walks][L]; called by felog_train
// after argument checks.  tile_ctas <= 0: min(SMs, max(1, n / 2048)) tiles
// at once; 1 runs the tiles in order (the reproducible form).
felog_status launch_tile(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                         const felog_train_params *tp, const uint64_t *thr, const int32_t *alias,
                         const uint64_t *S, uint64_t seed, int32_t round, int64_t clock_base,
                         void *phi_in, void *phi_out, unsigned long long *loss_acc, int32_t *timeout,
                         cudaStream_t s) {
    TileArgs a;
    a.walks = walks;
    a.total = n_walks * L;
    a.L = L;
    a.n = n;
    a.window = tp->window;
    a.K = tp->negatives;
    a.Ns = tp->tile_negatives > 0 ? tp->tile_negatives : 64;
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
