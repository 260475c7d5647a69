// Train: skip-gram with negative sampling (Eq. 1, Eq. 2) on one round's corpus.
//
// Work split: one warp per walk (HOGWILD) or per center position (MINIBATCH).
// Lane l owns elements [l*EPL, (l+1)*EPL) of a row (EPL = dim/32), so a row
// is one 128-bit (FP32, dim 128) or 64-bit (BF16, dim 128) load per lane.
// For a center c the warp:
//   1. draws all 2W*K negatives of the center lane-parallel (Philox + alias
//      table) into shared memory;
//   2. keeps phi_out[c] in registers across its 2W pairs;
//   3. per pair, issues the context row and the K negative rows together,
//      forms K+1 partial dot products and reduces them with a transposed
//      reduce-scatter (lane 4t ends with the dot of target t), evaluates the
//      sigmoid of one target per lane and broadcasts the K+1 coefficients;
//   4. updates rows in place (HOGWILD: plain stores, races tolerated as in
//      lock-free SGD) or adds fixed-point increments (MINIBATCH).
// The pair loss -log sigma(s+) - sum log sigma(-s_k) is summed per warp and
// added to a 64-bit fixed-point accumulator (2^-24 resolution), so the
// total does not depend on the order in which warps finish.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace felog {

int sm_count();

constexpr int kSgnsThreads = 256;
constexpr int kWarps = kSgnsThreads / 32;
constexpr double kLossScale = 16777216.0;            // 2^24
constexpr float kLossScaleF = 16777216.0f;
constexpr float kDeltaScale = 1099511627776.0f;      // 2^40
constexpr float kDeltaUnscale = 9.094947017729282e-13f;  // 2^-40

// ----------------------------------------------------------------------------
// Row access: EPL contiguous elements per lane, float math.
// ----------------------------------------------------------------------------
template <int EPL>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&x)[EPL]) {
    if constexpr (EPL == 1) {
        x[0] = p[0];
    } else if constexpr (EPL == 2) {
        const float2 a = *reinterpret_cast<const float2 *>(p);
        x[0] = a.x; x[1] = a.y;
    } else {
#pragma unroll
        for (int i = 0; i < EPL; i += 4) {
            const float4 a = *reinterpret_cast<const float4 *>(p + i);
            x[i] = a.x; x[i + 1] = a.y; x[i + 2] = a.z; x[i + 3] = a.w;
        }
    }
}

template <int EPL>
__device__ __forceinline__ void store_row(float *__restrict__ p, const float (&x)[EPL], uint32_t) {
    if constexpr (EPL == 1) {
        p[0] = x[0];
    } else if constexpr (EPL == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    } else {
#pragma unroll
        for (int i = 0; i < EPL; i += 4)
            *reinterpret_cast<float4 *>(p + i) = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
    }
}

__device__ __forceinline__ float bf16_bits_to_float(uint32_t h) { return __uint_as_float(h << 16); }

template <int EPL>
__device__ __forceinline__ void load_row(const __nv_bfloat16 *__restrict__ p, float (&x)[EPL]) {
    if constexpr (EPL == 1) {
        x[0] = bf16_bits_to_float(*reinterpret_cast<const uint16_t *>(p));
    } else if constexpr (EPL == 2) {
        const uint32_t a = *reinterpret_cast<const uint32_t *>(p);
        x[0] = bf16_bits_to_float(a & 0xffffu); x[1] = bf16_bits_to_float(a >> 16);
    } else if constexpr (EPL == 4) {
        const uint2 a = *reinterpret_cast<const uint2 *>(p);
        x[0] = bf16_bits_to_float(a.x & 0xffffu); x[1] = bf16_bits_to_float(a.x >> 16);
        x[2] = bf16_bits_to_float(a.y & 0xffffu); x[3] = bf16_bits_to_float(a.y >> 16);
    } else {
#pragma unroll
        for (int i = 0; i < EPL; i += 8) {
            const uint4 a = *reinterpret_cast<const uint4 *>(p + i);
            x[i + 0] = bf16_bits_to_float(a.x & 0xffffu); x[i + 1] = bf16_bits_to_float(a.x >> 16);
            x[i + 2] = bf16_bits_to_float(a.y & 0xffffu); x[i + 3] = bf16_bits_to_float(a.y >> 16);
            x[i + 4] = bf16_bits_to_float(a.z & 0xffffu); x[i + 5] = bf16_bits_to_float(a.z >> 16);
            x[i + 6] = bf16_bits_to_float(a.w & 0xffffu); x[i + 7] = bf16_bits_to_float(a.w >> 16);
        }
    }
}

// 32-bit integer mixer (a bijection with full avalanche; "lowbias32",
// C. Wellons' hash-prospector).  Spreads one random word over several
// rounding decisions.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Stochastic rounding to bfloat16: add 16 uniform random bits below the
// kept mantissa, then truncate.  NaN stays a quiet NaN; infinities stay.
__device__ __forceinline__ uint32_t sr_bf16(float x, uint32_t r16) {
    const uint32_t b = __float_as_uint(x);
    if ((b & 0x7f800000u) == 0x7f800000u) return (b & 0x007fffffu) ? 0x7fc0u : (b >> 16);
    return (b + (r16 & 0xffffu)) >> 16;
}

// r: one uniform 32-bit word for this row store on this lane
template <int EPL>
__device__ __forceinline__ void store_row(__nv_bfloat16 *__restrict__ p, const float (&x)[EPL],
                                         uint32_t r) {
    uint32_t h[EPL];
#pragma unroll
    for (int i = 0; i < EPL; i += 2) {
        h[i] = sr_bf16(x[i], r);
        if (i + 1 < EPL) h[i + 1] = sr_bf16(x[i + 1], r >> 16);
        r = mix32(r + 0x9E3779B9u);
    }
    if constexpr (EPL == 1) {
        *reinterpret_cast<uint16_t *>(p) = static_cast<uint16_t>(h[0]);
    } else if constexpr (EPL == 2) {
        *reinterpret_cast<uint32_t *>(p) = h[0] | (h[1] << 16);
    } else if constexpr (EPL == 4) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    } else {
#pragma unroll
        for (int i = 0; i < EPL; i += 8)
            *reinterpret_cast<uint4 *>(p + i) =
                make_uint4(h[i] | (h[i + 1] << 16), h[i + 2] | (h[i + 3] << 16),
                           h[i + 4] | (h[i + 5] << 16), h[i + 6] | (h[i + 7] << 16));
    }
}

// ----------------------------------------------------------------------------
// Transposed reduction of MAXT per-lane partial sums (MAXT = 2^m, m <= 5):
// after it, lane (t << (5 - m)) .. holds the warp-wide total of value t.
// ----------------------------------------------------------------------------
template <int MAXT>
__device__ __forceinline__ float reduce_scatter(float (&v)[MAXT], int lane) {
    static_assert(MAXT == 8 || MAXT == 16, "MAXT");
    constexpr int M = MAXT == 8 ? 3 : 4;
    // stage with xor distance 16 >> s halves the number of live values
#pragma unroll
    for (int s = 0; s < M; ++s) {
        const int dist = 16 >> s;
        const int half = MAXT >> (s + 1);
        const bool upper = (lane & dist) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, dist);
        }
    }
    float r = v[0];
#pragma unroll
    for (int dist = 16 >> M; dist >= 1; dist >>= 1) r += __shfl_xor_sync(kFull, r, dist);
    return r;
}

template <int MAXT>
__device__ __forceinline__ int target_of_lane(int lane) {
    // inverse of src(t) = t << (5 - M) restricted to the bit positions used
    constexpr int M = MAXT == 8 ? 3 : 4;
    return lane >> (5 - M);
}

__device__ __forceinline__ float softplus_neg(float s) {
    // -log sigma(s) = log(1 + exp(-s))
    return s >= 0.f ? log1pf(__expf(-s)) : -s + log1pf(__expf(s));
}

__device__ __forceinline__ int32_t draw_negative(const uint64_t *__restrict__ thr,
                                                 const int32_t *__restrict__ alias, uint64_t n,
                                                 uint64_t S, uint64_t seed, uint32_t round,
                                                 uint32_t walk, uint32_t pos, uint32_t q,
                                                 uint32_t k) {
    const u32x4 r = philox(seed, (q << 8) | k, walk, (round << 16) | pos, kStreamNeg);
    const uint64_t b = mulhi64(lo64(r), n);
    const uint64_t coin = mulhi64(hi64(r), S);
    const uint64_t t = __ldg(reinterpret_cast<const unsigned long long *>(thr) + b);
    const int32_t a = __ldg(alias + b);
    return coin < t ? static_cast<int32_t>(b) : a;
}

struct SgnsArgs {
    const int32_t *walks;
    int64_t n_walks;
    int32_t L, n, window, K;
    float lr0, inv_T;
    int64_t clock_base;
    const uint64_t *thr;
    const int32_t *alias;
    const uint64_t *S;
    uint64_t seed;
    uint32_t round;
    unsigned long long *loss_acc;
};

// ----------------------------------------------------------------------------
// HOGWILD: one warp per walk; every increment is applied at once as an
// atomic delta, so concurrent updates of a hot row commute instead of
// overwriting each other (a lost-update race would drop most negative-sample
// updates when many warps share few rows).  Rows are read through L2
// (ld.global.cg) so a warp sees its own earlier deltas.
//   float tables : vector red.global.add (one 16-byte reduction per lane);
//   bf16 tables  : the lane rounds value-read + delta stochastically and adds
//                  the resulting bf16 increment with a vector bf16 reduction
//                  (see sr_increment).
// ----------------------------------------------------------------------------

template <int EPL>
__device__ __forceinline__ void load_row_cg(const float *__restrict__ p, float (&x)[EPL]) {
    if constexpr (EPL == 1) {
        x[0] = __ldcg(p);
    } else if constexpr (EPL == 2) {
        const float2 a = __ldcg(reinterpret_cast<const float2 *>(p));
        x[0] = a.x; x[1] = a.y;
    } else {
#pragma unroll
        for (int i = 0; i < EPL; i += 4) {
            const float4 a = __ldcg(reinterpret_cast<const float4 *>(p + i));
            x[i] = a.x; x[i + 1] = a.y; x[i + 2] = a.z; x[i + 3] = a.w;
        }
    }
}

template <int EPL>
__device__ __forceinline__ void load_row_cg(const __nv_bfloat16 *__restrict__ p, float (&x)[EPL]) {
    if constexpr (EPL == 1) {
        x[0] = bf16_bits_to_float(__ldcg(reinterpret_cast<const unsigned short *>(p)));
    } else if constexpr (EPL == 2) {
        const uint32_t a = __ldcg(reinterpret_cast<const unsigned int *>(p));
        x[0] = bf16_bits_to_float(a & 0xffffu); x[1] = bf16_bits_to_float(a >> 16);
    } else if constexpr (EPL == 4) {
        const uint2 a = __ldcg(reinterpret_cast<const uint2 *>(p));
        x[0] = bf16_bits_to_float(a.x & 0xffffu); x[1] = bf16_bits_to_float(a.x >> 16);
        x[2] = bf16_bits_to_float(a.y & 0xffffu); x[3] = bf16_bits_to_float(a.y >> 16);
    } else {
#pragma unroll
        for (int i = 0; i < EPL; i += 8) {
            const uint4 a = __ldcg(reinterpret_cast<const uint4 *>(p + i));
            x[i + 0] = bf16_bits_to_float(a.x & 0xffffu); x[i + 1] = bf16_bits_to_float(a.x >> 16);
            x[i + 2] = bf16_bits_to_float(a.y & 0xffffu); x[i + 3] = bf16_bits_to_float(a.y >> 16);
            x[i + 4] = bf16_bits_to_float(a.z & 0xffffu); x[i + 5] = bf16_bits_to_float(a.z >> 16);
            x[i + 6] = bf16_bits_to_float(a.w & 0xffffu); x[i + 7] = bf16_bits_to_float(a.w >> 16);
        }
    }
}

__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}
__device__ __forceinline__ void red_add_v2(float *p, float a, float b) {
    asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// float table: add delta; `cur` (the value last read) is not needed
template <int EPL>
__device__ __forceinline__ void add_delta(float *__restrict__ p, const float (&cur)[EPL],
                                          const float (&delta)[EPL], uint32_t) {
    (void)cur;
    if constexpr (EPL == 1) {
        atomicAdd(p, delta[0]);
    } else if constexpr (EPL == 2) {
        red_add_v2(p, delta[0], delta[1]);
    } else {
#pragma unroll
        for (int i = 0; i < EPL; i += 4) red_add_v4(p + i, delta[i], delta[i + 1], delta[i + 2], delta[i + 3]);
    }
}

__device__ __forceinline__ uint32_t bf16_bits(float x) { return __float_as_uint(x) >> 16; }


// xorshift32 (Marsaglia, "Xorshift RNGs", 2003): per-lane stream of words
// for stochastic rounding, seeded once per center from Philox.
__device__ __forceinline__ uint32_t xorshift32(uint32_t &s) {
    s ^= s << 13;
    s ^= s >> 17;
    s ^= s << 5;
    return s;
}

__device__ __forceinline__ uint32_t sub_bf16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ void red_add_bf16x2_v2(__nv_bfloat16 *p, uint32_t a, uint32_t b) {
    asm volatile("red.relaxed.gpu.global.add.noftz.v2.bf16x2 [%0], {%1, %2};" ::"l"(p), "r"(a), "r"(b)
                 : "memory");
}
__device__ __forceinline__ void red_add_bf16x2_v1(__nv_bfloat16 *p, uint32_t a) {
    asm volatile("red.relaxed.gpu.global.add.noftz.bf16x2 [%0], %1;" ::"l"(p), "r"(a) : "memory");
}

// Two elements: stochastically rounded targets t = SR(cur + delta) (16
// random bits each, added below the kept mantissa, then truncated), packed
// with the current values, and the bf16x2 increment t - cur (exact when cur
// and t share a binade, rounded to nearest otherwise).  Added atomically to
// memory, the increment reproduces SR(cur + delta) exactly when no other
// update intervened, and loses no concurrent update when one did.
__device__ __forceinline__ uint32_t sr_increment2(float c0, float c1, float d0, float d1, uint32_t r0,
                                                  uint32_t r1) {
    const uint32_t b0 = __float_as_uint(c0 + d0) + (r0 & 0xffffu);
    const uint32_t b1 = __float_as_uint(c1 + d1) + (r1 & 0xffffu);
    const uint32_t t = __byte_perm(b0, b1, 0x7632);
    const uint32_t c = __byte_perm(__float_as_uint(c0), __float_as_uint(c1), 0x7632);
    return sub_bf16x2(t, c);
}

// bf16 table: `cur` holds the values last read (exact bf16); one random word
// w serves four elements (its two halves and the high halves of two odd
// multiples of it).
template <int EPL>
__device__ __forceinline__ void add_delta(__nv_bfloat16 *__restrict__ p, const float (&cur)[EPL],
                                          const float (&delta)[EPL], uint32_t w) {
    if constexpr (EPL == 1) {
        const float t = bf16_bits_to_float(sr_bf16(cur[0] + delta[0], w));
        const __nv_bfloat16 inc = __float2bfloat16_rn(t - cur[0]);
        if (__bfloat16_as_ushort(inc) & 0x7fffu) atomicAdd(p, inc);
    } else if constexpr (EPL == 2) {
        const uint32_t inc = sr_increment2(cur[0], cur[1], delta[0], delta[1], w, w >> 16);
        if (inc & 0x7fff7fffu) red_add_bf16x2_v1(p, inc);
    } else {
#pragma unroll
        for (int i = 0; i < EPL; i += 4) {
            const uint32_t w2 = w * 0x9E3779B9u, w3 = w * 0x85EBCA6Bu;
            const uint32_t i01 = sr_increment2(cur[i], cur[i + 1], delta[i], delta[i + 1], w, w >> 16);
            const uint32_t i23 = sr_increment2(cur[i + 2], cur[i + 3], delta[i + 2], delta[i + 3], w2 >> 16,
                                               w3 >> 16);
            if ((i01 | i23) & 0x7fff7fffu) red_add_bf16x2_v2(p + i, i01, i23);
            w = xorshift32(w);
        }
    }
}

// KFIX > 0: the number of negatives is a compile-time constant.
template <int D, class T, int MAXT, int KFIX>
__global__ void __launch_bounds__(kSgnsThreads, 3)
    k_sgns_hogwild(SgnsArgs a, T *__restrict__ phi_in, T *__restrict__ phi_out) {
    constexpr int EPL = D / 32;
    constexpr int SRC_SHIFT = 5 - (MAXT == 8 ? 3 : 4);
    constexpr bool kBf16 = !std::is_same<T, float>::value;
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = a.window, L = a.L;
    const int K = KFIX > 0 ? KFIX : a.K;
    const int per_warp = L + 2 * W * K;
    int32_t *wk = smem + wib * per_warp;
    int32_t *negs = wk + L;
    const uint64_t S = *a.S;
    const uint64_t n = static_cast<uint64_t>(a.n);
    const int my_t = target_of_lane<MAXT>(lane);
    const bool loss_lane = (lane & ((32 / MAXT) - 1)) == 0;
    long long loss_fx = 0;  // this lane's loss terms, 2^-24 units
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kWarps;
    for (int64_t wi = static_cast<int64_t>(blockIdx.x) * kWarps + wib; wi < a.n_walks; wi += warps) {
        const int32_t *row = a.walks + wi * L;
        for (int p = lane; p < L; p += 32) wk[p] = row[p];
        __syncwarp();
        for (int p = 0; p < L; ++p) {
            const int32_t c = wk[p];
            if (c < 0) continue;
            // all negatives of this center, lane-parallel
            for (int idx = lane; idx < 2 * W * K; idx += 32) {
                const int q = idx / K, k = idx - q * K;
                negs[idx] = draw_negative(a.thr, a.alias, n, S, a.seed, a.round,
                                          static_cast<uint32_t>(wi), static_cast<uint32_t>(p),
                                          static_cast<uint32_t>(q), static_cast<uint32_t>(k));
            }
            __syncwarp();
            const float tclock = static_cast<float>(a.clock_base + wi * L + p);
            const float eta = a.lr0 * fmaxf(1e-4f, 1.0f - tclock * a.inv_T);
            float oc[EPL], oc0[EPL], doc[EPL];
            float closs = 0.f;
            // stochastic-rounding stream of this lane for this center (bf16 only)
            uint32_t srs = 0;
            if constexpr (kBf16)
                srs = philox(a.seed, static_cast<uint32_t>(lane), static_cast<uint32_t>(wi),
                             (a.round << 16) | static_cast<uint32_t>(p), kStreamSR).x | 1u;
            T *oc_ptr = phi_out + static_cast<int64_t>(c) * D + lane * EPL;
            load_row_cg<EPL>(oc_ptr, oc);
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                oc0[e] = oc[e];
                doc[e] = 0.f;
            }
            for (int o = -W; o <= W; ++o) {
                if (o == 0) continue;
                const int pp = p + o;
                if (pp < 0 || pp >= L) continue;
                const int32_t x = wk[pp];
                if (x < 0) continue;
                const int q = o < 0 ? o + W : o + W - 1;
                int32_t nid[MAXT];
                nid[0] = c;
#pragma unroll
                for (int t = 1; t < MAXT; ++t) {
                    int32_t v = -1;
                    if (t <= K) {
                        v = negs[q * K + t - 1];
                        if (v == c) v = -1;  // a negative equal to the center is skipped
                    }
                    nid[t] = v;
                }
                float ix[EPL];
                T *ix_ptr = phi_in + static_cast<int64_t>(x) * D + lane * EPL;
                load_row_cg<EPL>(ix_ptr, ix);
                float nr[MAXT][EPL];
#pragma unroll
                for (int t = 1; t < MAXT; ++t) {
                    if (nid[t] >= 0) {
                        load_row_cg<EPL>(phi_out + static_cast<int64_t>(nid[t]) * D + lane * EPL, nr[t]);
                    } else {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) nr[t][e] = 0.f;
                    }
                }
#pragma unroll
                for (int e = 0; e < EPL; ++e) nr[0][e] = oc[e];
                float pd[MAXT];
#pragma unroll
                for (int t = 0; t < MAXT; ++t) {
                    float s = 0.f;
#pragma unroll
                    for (int e = 0; e < EPL; ++e) s = fmaf(ix[e], nr[t][e], s);
                    pd[t] = s;
                }
                const float dot = reduce_scatter<MAXT>(pd, lane);
                int32_t my_id = nid[0];
#pragma unroll
                for (int t = 1; t < MAXT; ++t)
                    if (t == my_t) my_id = nid[t];
                float g = 0.f;
                if (my_id >= 0) {
                    const bool pos = my_t == 0;
                    const float sig = __frcp_rn(1.f + __expf(-dot));
                    g = eta * ((pos ? 1.f : 0.f) - sig);
                    // -log sigma(s) for the center, -log sigma(-s) = -log(1 - sigma(s)) for a negative
                    if (loss_lane) closs -= __logf(fmaxf(pos ? sig : 1.f - sig, 1e-30f));
                }
                float gt[MAXT];
#pragma unroll
                for (int t = 0; t < MAXT; ++t) gt[t] = __shfl_sync(kFull, g, t << SRC_SHIFT);
                float din[EPL];
#pragma unroll
                for (int e = 0; e < EPL; ++e) din[e] = gt[0] * oc[e];
#pragma unroll
                for (int t = 1; t < MAXT; ++t) {
                    if (nid[t] < 0) continue;
                    float dn[EPL];
#pragma unroll
                    for (int e = 0; e < EPL; ++e) {
                        din[e] = fmaf(gt[t], nr[t][e], din[e]);
                        dn[e] = gt[t] * ix[e];
                    }
                    add_delta<EPL>(phi_out + static_cast<int64_t>(nid[t]) * D + lane * EPL, nr[t], dn,
                                   kBf16 ? xorshift32(srs) : 0u);
                }
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    const float u = gt[0] * ix[e];
                    oc[e] += u;
                    doc[e] += u;
                }
                add_delta<EPL>(ix_ptr, ix, din, kBf16 ? xorshift32(srs) : 0u);
            }
            add_delta<EPL>(oc_ptr, oc0, doc, kBf16 ? xorshift32(srs) : 0u);
            loss_fx += __float2ll_rn(closs * kLossScaleF);
            __syncwarp();
        }
    }
    // warp total of the loss, then one integer add per warp
    for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
    if (lane == 0 && loss_fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(loss_fx));
}

// ----------------------------------------------------------------------------
// HOGWILD, half-warp form (dim <= 128, K + 1 <= 8): the two 16-lane halves of
// a warp train two pairs of the same center at once; lane l of half h owns
// elements [(l & 15) * EPL, (l & 15 + 1) * EPL) of a row (EPL = dim / 16), so
// a bf16 row of 128 is one 128-bit access per lane.  Per pair this halves
// the reduction, sigmoid, broadcast and loop overhead of the full-warp form.
// Both halves hold phi_out[c] for the whole center; its increment is added
// to memory once, at the end of the center.  The two halves exchange their increments of
// phi_out[c] after every step, so each pair sees the updates of all earlier
// steps of its center.  Updates are atomic deltas, as in the full-warp form.
// ----------------------------------------------------------------------------
template <int EPL>
__device__ __forceinline__ void load_raw(const __nv_bfloat16 *__restrict__ p, uint32_t (&w)[EPL / 2]) {
    if constexpr (EPL == 2) {
        w[0] = __ldcg(reinterpret_cast<const unsigned int *>(p));
    } else if constexpr (EPL == 4) {
        const uint2 a = __ldcg(reinterpret_cast<const uint2 *>(p));
        w[0] = a.x; w[1] = a.y;
    } else {
        const uint4 a = __ldcg(reinterpret_cast<const uint4 *>(p));
        w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    }
}

template <int EPL>
__device__ __forceinline__ void unpack_bf16(const uint32_t (&w)[EPL / 2], float (&x)[EPL]) {
#pragma unroll
    for (int i = 0; i < EPL / 2; ++i) {
        x[2 * i] = __uint_as_float(w[i] << 16);
        x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

// hi16(w * C) + b: one 16-bit random value for one rounding, added below the
// kept mantissa of float bits b (multiply-high mixing of one random word by
// distinct odd constants gives each element its own value).
__device__ __forceinline__ uint32_t add_rand16(uint32_t b, uint32_t w, uint32_t C) {
    return __umulhi(w * C, 0x10000u) + b;
}

__device__ __forceinline__ void red_add_bf16x2_v4(__nv_bfloat16 *p, uint32_t a, uint32_t b, uint32_t c,
                                                  uint32_t d) {
    asm volatile("red.relaxed.gpu.global.add.noftz.v4.bf16x2 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a),
                 "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// bf16 row slice: raw = packed bf16 values last read, delta in float; one
// random word w covers the slice.
template <int EPL>
__device__ __forceinline__ void add_delta_raw(__nv_bfloat16 *__restrict__ p, const uint32_t (&raw)[EPL / 2],
                                              const float (&delta)[EPL], uint32_t w) {
    constexpr uint32_t C[8] = {0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu,
                               0x165667B1u, 0xD3A2646Cu | 1u, 0xFD7046C5u, 0xB55A4F09u};
    uint32_t inc[EPL / 2];
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < EPL / 2; ++i) {
        const float c0 = __uint_as_float(raw[i] << 16), c1 = __uint_as_float(raw[i] & 0xffff0000u);
        const uint32_t b0 = add_rand16(__float_as_uint(c0 + delta[2 * i]), w, C[(2 * i) & 7]);
        const uint32_t b1 = add_rand16(__float_as_uint(c1 + delta[2 * i + 1]), w, C[(2 * i + 1) & 7]);
        inc[i] = sub_bf16x2(__byte_perm(b0, b1, 0x7632), raw[i]);
        any |= inc[i];
    }
    if (!(any & 0x7fff7fffu)) return;  // every element rounded back to its current value
    if constexpr (EPL == 2) {
        red_add_bf16x2_v1(p, inc[0]);
    } else if constexpr (EPL == 4) {
        red_add_bf16x2_v2(p, inc[0], inc[1]);
    } else {
        red_add_bf16x2_v4(p, inc[0], inc[1], inc[2], inc[3]);
    }
}

// Transposed reduction of 8 partial sums over the 16 lanes of a half warp:
// afterwards lanes 2t and 2t+1 of the half hold the total of value t.
__device__ __forceinline__ float reduce_scatter16(float (&v)[8], int hl) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int dist = 8 >> s;
        const int half = 4 >> s;
        const bool upper = (hl & dist) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, dist);
        }
    }
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

// fp32 rows in the half-warp form: lane hl owns float4 chunks hl and hl + 16
// (EPL = 8) so that every 128-bit access of a half warp covers 256
// contiguous bytes; EPL <= 4 is one contiguous chunk.
template <int EPL>
__device__ __forceinline__ const float *hw_chunk(const float *row, int hl, int c) {
    return EPL == 8 ? row + (hl + 16 * c) * 4 : row + hl * EPL;
}
template <int EPL>
__device__ __forceinline__ void hw_load(const float *__restrict__ row, int hl, float (&x)[EPL]) {
    if constexpr (EPL == 8) {
        const float4 a = __ldcg(reinterpret_cast<const float4 *>(row + hl * 4));
        const float4 b = __ldcg(reinterpret_cast<const float4 *>(row + 64 + hl * 4));
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
        load_row_cg<EPL>(row + hl * EPL, x);
    }
}
template <int EPL>
__device__ __forceinline__ void hw_add(float *__restrict__ row, int hl, const float (&d)[EPL]) {
    if constexpr (EPL == 8) {
        red_add_v4(row + hl * 4, d[0], d[1], d[2], d[3]);
        red_add_v4(row + 64 + hl * 4, d[4], d[5], d[6], d[7]);
    } else {
        const float unused[EPL] = {};
        add_delta<EPL>(row + hl * EPL, unused, d, 0u);
    }
}

template <int D, class T, int KFIX>
__global__ void __launch_bounds__(kSgnsThreads, 2)
    k_sgns_hogwild_hw(SgnsArgs a, T *__restrict__ phi_in, T *__restrict__ phi_out) {
    constexpr int EPL = D / 16;
    constexpr int MAXT = 8;
    constexpr bool kBf16 = !std::is_same<T, float>::value;
    static_assert(EPL == 2 || EPL == 4 || EPL == 8, "dim");
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int h = lane >> 4, hl = lane & 15;
    const int W = a.window, L = a.L;
    const int K = KFIX > 0 ? KFIX : a.K;
    const int per_warp = L + 2 * W * K;
    int32_t *wk = smem + wib * per_warp;
    int32_t *negs = wk + L;
    const uint64_t S = *a.S;
    const uint64_t n = static_cast<uint64_t>(a.n);
    const int my_t = hl >> 1;
    const bool loss_lane = (hl & 1) == 0;
    long long loss_fx = 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kWarps;
    for (int64_t wi = static_cast<int64_t>(blockIdx.x) * kWarps + wib; wi < a.n_walks; wi += warps) {
        const int32_t *row = a.walks + wi * L;
        for (int p = lane; p < L; p += 32) wk[p] = row[p];
        __syncwarp();
        for (int p = 0; p < L; ++p) {
            const int32_t c = wk[p];
            if (c < 0) continue;
            for (int idx = lane; idx < 2 * W * K; idx += 32) {
                const int q = idx / K, k = idx - q * K;
                negs[idx] = draw_negative(a.thr, a.alias, n, S, a.seed, a.round,
                                          static_cast<uint32_t>(wi), static_cast<uint32_t>(p),
                                          static_cast<uint32_t>(q), static_cast<uint32_t>(k));
            }
            __syncwarp();
            const float tclock = static_cast<float>(a.clock_base + wi * L + p);
            const float eta = a.lr0 * fmaxf(1e-4f, 1.0f - tclock * a.inv_T);
            T *oc_row = phi_out + static_cast<int64_t>(c) * D;
            float oc[EPL], doc[EPL];
            uint32_t oc_raw[kBf16 ? EPL / 2 : 1];
            if constexpr (kBf16) {
                load_raw<EPL>(oc_row + hl * EPL, oc_raw);
                unpack_bf16<EPL>(oc_raw, oc);
            } else {
                hw_load<EPL>(reinterpret_cast<const float *>(oc_row), hl, oc);
            }
#pragma unroll
            for (int e = 0; e < EPL; ++e) doc[e] = 0.f;
            float closs = 0.f;
            uint32_t srs = 0;
            if constexpr (kBf16)
                srs = philox(a.seed, static_cast<uint32_t>(lane), static_cast<uint32_t>(wi),
                             (a.round << 16) | static_cast<uint32_t>(p), kStreamSR).x | 1u;
            // window offsets o in [lo, hi] \ {0}; lo <= 0 <= hi
            const int lo = max(-W, -p), hi = min(W, L - 1 - p);
            const int npairs = hi - lo;
            for (int j0 = 0; j0 < npairs; j0 += 2) {
                const int j = j0 + h;
                int o = lo + j;
                if (o >= 0) ++o;
                bool valid = j < npairs;
                const int32_t x = valid ? wk[p + o] : -1;
                valid = valid && x >= 0;
                const int q = o < 0 ? o + W : o + W - 1;
                int32_t nid[MAXT];
                nid[0] = valid ? c : -1;
#pragma unroll
                for (int t = 1; t < MAXT; ++t) {
                    int32_t v = -1;
                    if (t <= K && valid) {
                        v = negs[q * K + t - 1];
                        if (v == c) v = -1;
                    }
                    nid[t] = v;
                }
                T *ix_row = phi_in + static_cast<int64_t>(valid ? x : 0) * D;
                float ix[EPL];
                uint32_t ix_raw[kBf16 ? EPL / 2 : 1];
                float nr[MAXT][EPL];
                uint32_t nr_raw[MAXT][kBf16 ? EPL / 2 : 1];
                if constexpr (kBf16) {
                    if (valid) load_raw<EPL>(ix_row + hl * EPL, ix_raw);
                    else {
#pragma unroll
                        for (int i = 0; i < EPL / 2; ++i) ix_raw[i] = 0u;
                    }
#pragma unroll
                    for (int t = 1; t < MAXT; ++t) {
                        if (nid[t] >= 0) load_raw<EPL>(phi_out + static_cast<int64_t>(nid[t]) * D + hl * EPL, nr_raw[t]);
                        else {
#pragma unroll
                            for (int i = 0; i < EPL / 2; ++i) nr_raw[t][i] = 0u;
                        }
                    }
                    unpack_bf16<EPL>(ix_raw, ix);
#pragma unroll
                    for (int t = 1; t < MAXT; ++t) unpack_bf16<EPL>(nr_raw[t], nr[t]);
                } else {
                    if (valid) hw_load<EPL>(reinterpret_cast<const float *>(ix_row), hl, ix);
                    else {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) ix[e] = 0.f;
                    }
#pragma unroll
                    for (int t = 1; t < MAXT; ++t) {
                        if (nid[t] >= 0)
                            hw_load<EPL>(reinterpret_cast<const float *>(phi_out + static_cast<int64_t>(nid[t]) * D), hl, nr[t]);
                        else {
#pragma unroll
                            for (int e = 0; e < EPL; ++e) nr[t][e] = 0.f;
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < EPL; ++e) nr[0][e] = oc[e];
                float pd[MAXT];
#pragma unroll
                for (int t = 0; t < MAXT; ++t) {
                    float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int e = 0; e < EPL; e += 2)
                        s2 = __ffma2_rn(make_float2(ix[e], ix[e + 1]), make_float2(nr[t][e], nr[t][e + 1]), s2);
                    pd[t] = s2.x + s2.y;
                }
                const float dot = reduce_scatter16(pd, hl);
                int32_t my_id = nid[0];
#pragma unroll
                for (int t = 1; t < MAXT; ++t)
                    if (t == my_t) my_id = nid[t];
                float g = 0.f;
                if (my_id >= 0) {
                    const bool pos = my_t == 0;
                    const float sig = __frcp_rn(1.f + __expf(-dot));
                    g = eta * ((pos ? 1.f : 0.f) - sig);
                    if (loss_lane) closs -= __logf(fmaxf(pos ? sig : 1.f - sig, 1e-30f));
                }
                float gt[MAXT];
#pragma unroll
                for (int t = 0; t < MAXT; ++t) {
                    gt[t] = 0.f;
                    if (t <= K) gt[t] = __shfl_sync(kFull, g, (h << 4) | (t << 1));
                }
                float din[EPL];
#pragma unroll
                for (int e = 0; e < EPL; e += 2) {
                    const float2 r = __fmul2_rn(make_float2(gt[0], gt[0]), make_float2(oc[e], oc[e + 1]));
                    din[e] = r.x;
                    din[e + 1] = r.y;
                }
#pragma unroll
                for (int t = 1; t < MAXT; ++t) {
                    if (nid[t] < 0) continue;
                    float dn[EPL];
#pragma unroll
                    for (int e = 0; e < EPL; e += 2) {
                        const float2 gg = make_float2(gt[t], gt[t]);
                        const float2 r = __ffma2_rn(gg, make_float2(nr[t][e], nr[t][e + 1]), make_float2(din[e], din[e + 1]));
                        din[e] = r.x;
                        din[e + 1] = r.y;
                        const float2 u = __fmul2_rn(gg, make_float2(ix[e], ix[e + 1]));
                        dn[e] = u.x;
                        dn[e + 1] = u.y;
                    }
                    T *nrow = phi_out + static_cast<int64_t>(nid[t]) * D;
                    if constexpr (kBf16) {
                        srs = srs * 1664525u + 1013904223u;
                        add_delta_raw<EPL>(nrow + hl * EPL, nr_raw[t], dn, srs);
                    } else {
                        hw_add<EPL>(reinterpret_cast<float *>(nrow), hl, dn);
                    }
                }
                // both pairs of this step update phi_out[c]: each half adds its own
                // increment and the other half's, so the next step sees both
#pragma unroll
                for (int e = 0; e < EPL; e += 2) {
                    const float2 gg = make_float2(gt[0], gt[0]);
                    const float2 u = __fmul2_rn(gg, make_float2(ix[e], ix[e + 1]));
                    const float v0 = __shfl_xor_sync(kFull, u.x, 16), v1 = __shfl_xor_sync(kFull, u.y, 16);
                    oc[e] += u.x + v0;
                    oc[e + 1] += u.y + v1;
                    doc[e] += u.x + v0;
                    doc[e + 1] += u.y + v1;
                }
                if (valid) {
                    if constexpr (kBf16) {
                        srs = srs * 1664525u + 1013904223u;
                        add_delta_raw<EPL>(ix_row + hl * EPL, ix_raw, din, srs);
                    } else {
                        hw_add<EPL>(reinterpret_cast<float *>(ix_row), hl, din);
                    }
                }
            }
            // the summed increment of phi_out[c] (identical in both halves), added by half 0
            if (h == 0) {
                if constexpr (kBf16) {
                    srs = srs * 1664525u + 1013904223u;
                    add_delta_raw<EPL>(oc_row + hl * EPL, oc_raw, doc, srs);
                } else {
                    hw_add<EPL>(reinterpret_cast<float *>(oc_row), hl, doc);
                }
            }
            loss_fx += __float2ll_rn(closs * kLossScaleF);
            __syncwarp();
        }
    }
    for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
    if (lane == 0 && loss_fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(loss_fx));
}

// ----------------------------------------------------------------------------
// MINIBATCH: one warp per center position of the batch [b0, b1).  Tables are
// read only; increments go to 64-bit fixed-point accumulators (2^-40 units),
// which makes the per-row sums exact and order independent.
// ----------------------------------------------------------------------------
struct MbState {
    long long *acc_in, *acc_out;  // [n][D]
    uint32_t *mark_in, *mark_out; // [n]
    int32_t *list_in, *list_out;  // [n]
    int32_t *counters;            // [0] = |list_in|, [1] = |list_out|, [2] = apply ticket
};

template <int EPL>
__device__ __forceinline__ void add_fixed(long long *__restrict__ p, const float (&x)[EPL]) {
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        const long long q = __float2ll_rn(x[e] * kDeltaScale);
        if (q) atomicAdd(reinterpret_cast<unsigned long long *>(p + e), static_cast<unsigned long long>(q));
    }
}

__device__ __forceinline__ void mark_row(uint32_t *mark, int32_t *list, int32_t *counter, int32_t r) {
    if (atomicExch(mark + r, 1u) == 0u) list[atomicAdd(counter, 1)] = r;
}

template <int D, class T, int MAXT>
__global__ void __launch_bounds__(kSgnsThreads)
    k_sgns_mb_grad(SgnsArgs a, int64_t b0, int64_t b1, float eta, const T *__restrict__ phi_in,
                   const T *__restrict__ phi_out, MbState st) {
    constexpr int EPL = D / 32;
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = a.window, K = a.K, L = a.L;
    int32_t *negs = smem + wib * (2 * W * K);
    const uint64_t S = *a.S;
    const uint64_t n = static_cast<uint64_t>(a.n);
    const int my_t = target_of_lane<MAXT>(lane);
    const bool loss_lane = (lane & ((32 / MAXT) - 1)) == 0;
    const int64_t tok = b0 + static_cast<int64_t>(blockIdx.x) * kWarps + wib;
    if (tok >= b1) return;
    const int64_t wi = tok / L;
    const int p = static_cast<int>(tok - wi * L);
    const int32_t *row = a.walks + wi * L;
    const int32_t c = row[p];
    if (c < 0) return;
    for (int idx = lane; idx < 2 * W * K; idx += 32) {
        const int q = idx / K, k = idx - q * K;
        negs[idx] = draw_negative(a.thr, a.alias, n, S, a.seed, a.round, static_cast<uint32_t>(wi),
                                  static_cast<uint32_t>(p), static_cast<uint32_t>(q),
                                  static_cast<uint32_t>(k));
    }
    __syncwarp();
    float oc[EPL], doc[EPL];
    load_row<EPL>(phi_out + static_cast<int64_t>(c) * D + lane * EPL, oc);
#pragma unroll
    for (int e = 0; e < EPL; ++e) doc[e] = 0.f;
    float closs = 0.f;
    bool any = false;
    for (int o = -W; o <= W; ++o) {
        if (o == 0) continue;
        const int pp = p + o;
        if (pp < 0 || pp >= L) continue;
        const int32_t x = row[pp];
        if (x < 0) continue;
        any = true;
        const int q = o < 0 ? o + W : o + W - 1;
        int32_t nid[MAXT];
        nid[0] = c;
#pragma unroll
        for (int t = 1; t < MAXT; ++t) {
            int32_t v = -1;
            if (t <= K) {
                v = negs[q * K + t - 1];
                if (v == c) v = -1;
            }
            nid[t] = v;
        }
        float ix[EPL];
        load_row<EPL>(phi_in + static_cast<int64_t>(x) * D + lane * EPL, ix);
        float nr[MAXT][EPL];
#pragma unroll
        for (int t = 1; t < MAXT; ++t) {
            if (nid[t] >= 0) load_row<EPL>(phi_out + static_cast<int64_t>(nid[t]) * D + lane * EPL, nr[t]);
            else {
#pragma unroll
                for (int e = 0; e < EPL; ++e) nr[t][e] = 0.f;
            }
        }
#pragma unroll
        for (int e = 0; e < EPL; ++e) nr[0][e] = oc[e];
        float pd[MAXT];
#pragma unroll
        for (int t = 0; t < MAXT; ++t) {
            float s = 0.f;
#pragma unroll
            for (int e = 0; e < EPL; ++e) s = fmaf(ix[e], nr[t][e], s);
            pd[t] = s;
        }
        const float dot = reduce_scatter<MAXT>(pd, lane);
        int32_t my_id = nid[0];
#pragma unroll
        for (int t = 1; t < MAXT; ++t)
            if (t == my_t) my_id = nid[t];
        float g = 0.f;
        if (my_id >= 0) {
            const float label = my_t == 0 ? 1.f : 0.f;
            const float sig = 1.f / (1.f + expf(-dot));
            g = eta * (label - sig);
            if (loss_lane) closs += my_t == 0 ? softplus_neg(dot) : softplus_neg(-dot);
        }
        float gt[MAXT];
#pragma unroll
        for (int t = 0; t < MAXT; ++t) gt[t] = __shfl_sync(kFull, g, t << (5 - (MAXT == 8 ? 3 : 4)));
        float din[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            din[e] = gt[0] * oc[e];
            doc[e] = fmaf(gt[0], ix[e], doc[e]);
        }
#pragma unroll
        for (int t = 1; t < MAXT; ++t) {
            if (nid[t] < 0) continue;
            float dn[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                din[e] = fmaf(gt[t], nr[t][e], din[e]);
                dn[e] = gt[t] * ix[e];
            }
            add_fixed<EPL>(st.acc_out + static_cast<int64_t>(nid[t]) * D + lane * EPL, dn);
            if (lane == 0) mark_row(st.mark_out, st.list_out, st.counters + 1, nid[t]);
        }
        add_fixed<EPL>(st.acc_in + static_cast<int64_t>(x) * D + lane * EPL, din);
        if (lane == 0) mark_row(st.mark_in, st.list_in, st.counters + 0, x);
    }
    if (any) {
        add_fixed<EPL>(st.acc_out + static_cast<int64_t>(c) * D + lane * EPL, doc);
        if (lane == 0) mark_row(st.mark_out, st.list_out, st.counters + 1, c);
    }
    long long loss_fx = __float2ll_rn(closs * kLossScaleF);
    for (int o = 16; o; o >>= 1) loss_fx += __shfl_xor_sync(kFull, loss_fx, o);
    if (lane == 0 && loss_fx != 0) atomicAdd(a.loss_acc, static_cast<unsigned long long>(loss_fx));
}

// Apply the accumulated increments of the touched rows and clear them.
// The last block to finish resets the list counters.
template <int D, class T>
__global__ void __launch_bounds__(256)
    k_sgns_mb_apply(T *__restrict__ phi_in, T *__restrict__ phi_out, MbState st, uint64_t seed,
                    uint32_t batch_key) {
    constexpr int EPL = D / 32;
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    const int32_t n_in = st.counters[0], n_out = st.counters[1];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5);
         i < static_cast<int64_t>(n_in) + n_out; i += warps) {
        const bool is_in = i < n_in;
        const int32_t r = is_in ? st.list_in[i] : st.list_out[i - n_in];
        T *tab = is_in ? phi_in : phi_out;
        long long *acc = (is_in ? st.acc_in : st.acc_out) + static_cast<int64_t>(r) * D + lane * EPL;
        float v[EPL];
        load_row<EPL>(tab + static_cast<int64_t>(r) * D + lane * EPL, v);
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            const long long q = acc[e];
            acc[e] = 0;
            v[e] += __ll2float_rn(q) * kDeltaUnscale;
        }
        uint32_t rr = 0;
        if constexpr (!std::is_same<T, float>::value)
            rr = philox(seed, static_cast<uint32_t>(lane) | (is_in ? 0u : 0x100u),
                        static_cast<uint32_t>(r), batch_key, kStreamSR).x;
        store_row<EPL>(tab + static_cast<int64_t>(r) * D + lane * EPL, v, rr);
        if (lane == 0) (is_in ? st.mark_in : st.mark_out)[r] = 0u;
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(st.counters + 2, 1) == static_cast<int>(gridDim.x) - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        st.counters[0] = 0;
        st.counters[1] = 0;
        st.counters[2] = 0;
    }
}

__global__ void k_loss_finish(const unsigned long long *__restrict__ acc, double *__restrict__ loss) {
    *loss = static_cast<double>(static_cast<long long>(*acc)) / kLossScale;
}

// ----------------------------------------------------------------------------
// Table initialisation.
// ----------------------------------------------------------------------------
template <class T>
__global__ void k_init_tables(int32_t n, int32_t dim, uint64_t seed, T *__restrict__ phi_in,
                              T *__restrict__ phi_out) {
    const int64_t groups = static_cast<int64_t>(n) * (dim / 4);
    for (int64_t gidx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; gidx < groups;
         gidx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = static_cast<int32_t>(gidx / (dim / 4));
        const int32_t i4 = static_cast<int32_t>(gidx - static_cast<int64_t>(v) * (dim / 4));
        const u32x4 r = philox(seed, static_cast<uint32_t>(i4), static_cast<uint32_t>(v), 0u, kStreamInit);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
        const float fd = static_cast<float>(dim);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float u = static_cast<float>(w[k] >> 8) * 5.9604644775390625e-08f;  // 2^-24
            const float x = __fdiv_rn(u - 0.5f, fd);
            const int64_t off = static_cast<int64_t>(v) * dim + i4 * 4 + k;
            if constexpr (std::is_same<T, float>::value) {
                phi_in[off] = x;
                phi_out[off] = 0.f;
            } else {
                phi_in[off] = __float2bfloat16_rn(x);
                phi_out[off] = __float2bfloat16_rn(0.f);
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Host side.
// ----------------------------------------------------------------------------
struct TrainWorkspace {
    unsigned long long *loss_acc;
    MbState mb;
};

static bool minibatch_mode(const felog_train_params *tp) { return tp->mode == FELOG_SGNS_MINIBATCH; }

static TrainWorkspace carve_train(Carver &c, int32_t n, const felog_train_params *tp) {
    TrainWorkspace w{};
    w.loss_acc = c.take<unsigned long long>(1);
    if (minibatch_mode(tp)) {
        const size_t nn = n > 0 ? static_cast<size_t>(n) : 1;
        w.mb.acc_in = c.take<long long>(nn * tp->dim);
        w.mb.acc_out = c.take<long long>(nn * tp->dim);
        w.mb.mark_in = c.take<uint32_t>(nn);
        w.mb.mark_out = c.take<uint32_t>(nn);
        w.mb.list_in = c.take<int32_t>(nn);
        w.mb.list_out = c.take<int32_t>(nn);
        w.mb.counters = c.take<int32_t>(4);
    }
    return w;
}

static bool params_ok(const felog_train_params *tp) {
    if (!tp) return false;
    if (tp->dim != 32 && tp->dim != 64 && tp->dim != 128 && tp->dim != 256) return false;
    if (tp->window < 1 || tp->window > 16 || tp->negatives < 1 || tp->negatives > 15) return false;
    if (tp->mode != FELOG_SGNS_HOGWILD && tp->mode != FELOG_SGNS_MINIBATCH) return false;
    if (tp->precision != FELOG_FP32 && tp->precision != FELOG_BF16_SR) return false;
    if (tp->mode == FELOG_SGNS_MINIBATCH && tp->minibatch < 1) return false;
    if (tp->hogwild_form < 0 || tp->hogwild_form > 2) return false;
    if (tp->hogwild_form == 2 && (tp->dim > 128 || tp->negatives > 7)) return false;
    if (!(tp->lr0 >= 0.f) || tp->lr_total_tokens <= 0) return false;
    return true;
}

template <int D, class T, int MAXT, int KFIX>
static felog_status launch_train(const SgnsArgs &a, const felog_train_params *tp, void *phi_in,
                                 void *phi_out, TrainWorkspace &w, cudaStream_t s) {
    T *pin = static_cast<T *>(phi_in);
    T *pout = static_cast<T *>(phi_out);
    if (!minibatch_mode(tp)) {
        const size_t smem = sizeof(int32_t) * kWarps * (a.L + 2 * a.window * a.K);
        if (smem > 200 * 1024) return FELOG_ERR_UNSUPPORTED;  // walk too long to stage per warp
        // half-warp form for dim <= 128 and K + 1 <= 8, full-warp form otherwise
        const bool half_warp = D <= 128 && MAXT == 8 && tp->hogwild_form != 1;
        auto kern = half_warp ? k_sgns_hogwild_hw<(D <= 128 ? D : 128), T, KFIX> : k_sgns_hogwild<D, T, MAXT, KFIX>;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSgnsThreads, smem);
        if (per_sm < 1) per_sm = 1;
        // resident warps <= n / rows_per_warp: on small graphs this bounds how
        // many warps update the same rows at once (staleness of lock-free SGD)
        const int64_t rows_per_warp = tp->hogwild_rows_per_warp > 0 ? tp->hogwild_rows_per_warp : 16;
        const int64_t cap_blocks = std::max<int64_t>(1, a.n / rows_per_warp / kWarps);
        const int64_t want = (a.n_walks + kWarps - 1) / kWarps;
        const int blocks = static_cast<int>(
            std::min<int64_t>({want, static_cast<int64_t>(per_sm) * sm_count(), cap_blocks}));
        kern<<<blocks, kSgnsThreads, smem, s>>>(a, pin, pout);
        return check_launch("felog_train (hogwild)");
    }
    const size_t smem = sizeof(int32_t) * kWarps * (2 * a.window * a.K);
    const int64_t total = a.n_walks * a.L;
    const int64_t B = tp->minibatch;
    felog_status st = record_cuda_error(cudaMemsetAsync(w.mb.counters, 0, 4 * sizeof(int32_t), s), "train");
    if (st) return st;
    int apply_blocks = sm_count() * 4;
    for (int64_t b0 = 0, bi = 0; b0 < total; b0 += B, ++bi) {
        const int64_t b1 = std::min(total, b0 + B);
        const double f = 1.0 - static_cast<double>(a.clock_base + b0) / static_cast<double>(tp->lr_total_tokens);
        const float eta = static_cast<float>(static_cast<double>(tp->lr0) * (f < 1e-4 ? 1e-4 : f));
        const int grid = static_cast<int>((b1 - b0 + kWarps - 1) / kWarps);
        k_sgns_mb_grad<D, T, MAXT><<<grid, kSgnsThreads, smem, s>>>(a, b0, b1, eta, pin, pout, w.mb);
        k_sgns_mb_apply<D, T><<<apply_blocks, 256, 0, s>>>(pin, pout, w.mb, a.seed,
                                                           (a.round << 20) ^ static_cast<uint32_t>(bi));
    }
    return check_launch("felog_train (minibatch)");
}

template <int D, class T>
static felog_status dispatch_maxt(const SgnsArgs &a, const felog_train_params *tp, void *pi,
                                  void *po, TrainWorkspace &w, cudaStream_t s) {
    if (tp->negatives == 5) return launch_train<D, T, 8, 5>(a, tp, pi, po, w, s);
    if (tp->negatives + 1 <= 8) return launch_train<D, T, 8, 0>(a, tp, pi, po, w, s);
    return launch_train<D, T, 16, 0>(a, tp, pi, po, w, s);
}

template <class T>
static felog_status dispatch_dim(const SgnsArgs &a, const felog_train_params *tp, void *pi, void *po,
                                 TrainWorkspace &w, cudaStream_t s) {
    switch (tp->dim) {
        case 32: return dispatch_maxt<32, T>(a, tp, pi, po, w, s);
        case 64: return dispatch_maxt<64, T>(a, tp, pi, po, w, s);
        case 128: return dispatch_maxt<128, T>(a, tp, pi, po, w, s);
        case 256: return dispatch_maxt<256, T>(a, tp, pi, po, w, s);
    }
    return FELOG_ERR_UNSUPPORTED;
}

}  // namespace felog

using namespace felog;

extern "C" size_t felog_train_workspace_bytes(int64_t n_walks, int32_t L, int32_t n,
                                              const felog_train_params *tp) {
    (void)n_walks;
    (void)L;
    if (!params_ok(tp)) return 0;
    Carver c(nullptr, 0);
    carve_train(c, n, tp);
    return align_up(c.used, 256);
}

extern "C" felog_status felog_train(const int32_t *walks, int64_t n_walks, int32_t L, int32_t n,
                                    const felog_train_params *tp, const uint64_t *thr,
                                    const int32_t *alias, const uint64_t *S, uint64_t seed,
                                    int32_t round, int64_t clock_base, void *phi_in, void *phi_out,
                                    double *loss, void *workspace, size_t workspace_bytes,
                                    void *stream) {
    if (!params_ok(tp)) return FELOG_ERR_INVALID_ARG;
    if (n_walks < 0 || L < 1 || L > 65535 || n < 1 || round < 0 || round >= 65536 || clock_base < 0 ||
        !loss)
        return FELOG_ERR_INVALID_ARG;
    if (n_walks > 0 && (!walks || !thr || !alias || !S || !phi_in || !phi_out)) return FELOG_ERR_INVALID_ARG;
    if (n_walks > 0xffffffffLL) return FELOG_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < felog_train_workspace_bytes(n_walks, L, n, tp))
        return FELOG_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(workspace, workspace_bytes);
    TrainWorkspace w = carve_train(c, n, tp);
    felog_status st = record_cuda_error(cudaMemsetAsync(w.loss_acc, 0, sizeof(unsigned long long), s), "train");
    if (st) return st;
    if (minibatch_mode(tp)) {
        st = record_cuda_error(cudaMemsetAsync(w.mb.mark_in, 0, sizeof(uint32_t) * n, s), "train");
        if (!st) st = record_cuda_error(cudaMemsetAsync(w.mb.mark_out, 0, sizeof(uint32_t) * n, s), "train");
        if (!st) st = record_cuda_error(cudaMemsetAsync(w.mb.acc_in, 0, sizeof(long long) * n * tp->dim, s), "train");
        if (!st) st = record_cuda_error(cudaMemsetAsync(w.mb.acc_out, 0, sizeof(long long) * n * tp->dim, s), "train");
        if (st) return st;
    }
    if (n_walks > 0) {
        SgnsArgs a;
        a.walks = walks;
        a.n_walks = n_walks;
        a.L = L;
        a.n = n;
        a.window = tp->window;
        a.K = tp->negatives;
        a.lr0 = tp->lr0;
        a.inv_T = static_cast<float>(1.0 / static_cast<double>(tp->lr_total_tokens));
        a.clock_base = clock_base;
        a.thr = thr;
        a.alias = alias;
        a.S = S;
        a.seed = seed;
        a.round = static_cast<uint32_t>(round);
        a.loss_acc = w.loss_acc;
        st = tp->precision == FELOG_FP32 ? dispatch_dim<float>(a, tp, phi_in, phi_out, w, s)
                                         : dispatch_dim<__nv_bfloat16>(a, tp, phi_in, phi_out, w, s);
        if (st) return st;
    }
    k_loss_finish<<<1, 1, 0, s>>>(w.loss_acc, loss);
    return check_launch("felog_train");
}

extern "C" felog_status felog_init_tables(int32_t n, int32_t dim, int32_t precision, uint64_t seed,
                                          void *phi_in, void *phi_out, void *stream) {
    if (n < 0 || (dim != 32 && dim != 64 && dim != 128 && dim != 256)) return FELOG_ERR_INVALID_ARG;
    if (precision != FELOG_FP32 && precision != FELOG_BF16_SR) return FELOG_ERR_INVALID_ARG;
    if (n == 0) return FELOG_OK;
    if (!phi_in || !phi_out) return FELOG_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t groups = static_cast<int64_t>(n) * (dim / 4);
    const int grid = static_cast<int>(std::min<int64_t>(ceil_div(groups, 256), sm_count() * 16));
    if (precision == FELOG_FP32)
        k_init_tables<float><<<grid, 256, 0, s>>>(n, dim, seed, static_cast<float *>(phi_in),
                                                  static_cast<float *>(phi_out));
    else
        k_init_tables<__nv_bfloat16><<<grid, 256, 0, s>>>(n, dim, seed, static_cast<__nv_bfloat16 *>(phi_in),
                                                          static_cast<__nv_bfloat16 *>(phi_out));
    return check_launch("felog_init_tables");
}
