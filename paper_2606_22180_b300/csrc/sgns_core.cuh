// Device building blocks of the SGNS kernels (Eq. 2 updates, row access,
// stochastic rounding, reductions, negative draws), shared by the single-graph
// kernels in sgns.cu and the multi-graph kernels in batch.cu.
#pragma once

#include <math.h>

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

// NC: read the alias table through the read-only data cache (right for a
// kernel that does not write the table; a persistent kernel that rebuilds it
// every round passes false and reads it through L2).
template <bool NC = true>
__device__ __forceinline__ int32_t draw_negative(const uint64_t *__restrict__ thr,
                                                 const int32_t *__restrict__ alias, uint64_t n,
                                                 uint64_t S, uint64_t seed, uint32_t round,
                                                 uint32_t walk, uint32_t pos, uint32_t q,
                                                 uint32_t k) {
    const u32x4 r = philox(seed, (q << 8) | k, walk, (round << 16) | pos, kStreamNeg);
    const uint64_t b = mulhi64(lo64(r), n);
    const uint64_t coin = mulhi64(hi64(r), S);
    const uint64_t t = NC ? __ldg(reinterpret_cast<const unsigned long long *>(thr) + b)
                          : __ldcg(reinterpret_cast<const unsigned long long *>(thr) + b);
    const int32_t a = NC ? __ldg(alias + b) : __ldcg(alias + b);
    // b < n always; an alias outside [0, n) (a damaged table) falls back to b
    return coin < t || static_cast<uint64_t>(static_cast<uint32_t>(a)) >= n ? static_cast<int32_t>(b) : a;
}

// A walk entry as the trainers read it: ids outside [0, n) count as padding,
// so a damaged corpus cannot index the tables out of range.
__device__ __forceinline__ int32_t walk_id(int32_t x, uint64_t n) {
    return static_cast<uint64_t>(static_cast<uint32_t>(x)) < n ? x : -1;
}

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

__device__ __forceinline__ void red_add_bf16x2_v4(__nv_bfloat16 *p, uint32_t a, uint32_t b, uint32_t c,
                                                  uint32_t d) {
    asm volatile("red.relaxed.gpu.global.add.noftz.v4.bf16x2 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a),
                 "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Two stochastically rounded bf16 values packed in one word: hi = SR(x_hi)
// with the random word's upper 16 bits, lo = SR(x_lo) with its lower 16.  The
// conversion instruction with the .rs rounding mode adds the random bits
// below the kept bits of each float and truncates, which is the rounding the
// oracle defines (checked bit for bit on a B300 over 2^20 random pairs,
// both halves); one instruction replaces the two additions and the pack.
__device__ __forceinline__ uint32_t sr_pack_bf16x2(float x_hi, float x_lo, uint32_t rbits) {
    uint32_t t;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(t) : "f"(x_hi), "f"(x_lo), "r"(rbits));
    return t;
}

// bf16 row slice: raw = packed bf16 values last read, delta in float; one
// random word w (a step of the lane's LCG) covers the slice.  Element pair i
// rounds with w * C_i for an odd constant C_i: its upper half, the product's
// well-mixed high bits, serves the upper element; its lower half, whose bits
// only depend on w's low bits (short periods in an LCG), is xored with w's
// high half before it serves the lower element.
template <int EPL>
__device__ __forceinline__ void add_delta_raw(__nv_bfloat16 *__restrict__ p, const uint32_t (&raw)[EPL / 2],
                                              const float (&delta)[EPL], uint32_t w) {
    constexpr uint32_t C[4] = {0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu};
    const uint32_t whi = w >> 16;
    uint32_t inc[EPL / 2];
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < EPL / 2; ++i) {
        const float c0 = __uint_as_float(raw[i] << 16), c1 = __uint_as_float(raw[i] & 0xffff0000u);
        const uint32_t t = sr_pack_bf16x2(c1 + delta[2 * i + 1], c0 + delta[2 * i], (w * C[i & 3]) ^ whi);
        inc[i] = sub_bf16x2(t, raw[i]);
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

// As add_delta_raw, with the row's current values also given as floats
// (cur[e] = the bf16 value in raw, already unpacked by the caller), and the
// sums cur + delta formed two at a time.
template <int EPL>
__device__ __forceinline__ void add_delta_vals(__nv_bfloat16 *__restrict__ p, const float (&cur)[EPL],
                                               const uint32_t (&raw)[EPL / 2], const float (&delta)[EPL],
                                               uint32_t w) {
    constexpr uint32_t C[4] = {0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu};
    const uint32_t whi = w >> 16;
    uint32_t inc[EPL / 2];
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < EPL / 2; ++i) {
        const float2 x = __fadd2_rn(make_float2(cur[2 * i], cur[2 * i + 1]),
                                    make_float2(delta[2 * i], delta[2 * i + 1]));
        const uint32_t t = sr_pack_bf16x2(x.y, x.x, (w * C[i & 3]) ^ whi);
        inc[i] = sub_bf16x2(t, raw[i]);
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


// One graph's training state as seen by a warp (the half-warp form below
// trains one walk of it at a time).
template <class T>
struct TrainView {
    T *phi_in, *phi_out;
    const uint64_t *thr;
    const int32_t *alias;
    uint64_t n, S, seed;
    uint32_t round;
    float lr0, inv_T;
    int64_t clock_base;  // token clock at the start of this graph's round
    int W, K, L;
    int stage_flush;     // STAGE: flush every staged increment every stage_flush centers (0: on leaving)
};

// The full-warp Hogwild trainer of one walk (any dim, K + 1 <= MAXT): one
// pair at a time, lane l owns elements [l * EPL, (l + 1) * EPL) of a row
// (EPL = dim / 32), the K + 1 dots are reduced by a transposed reduce-scatter
// (lane t << (5 - log2 MAXT) ends with the dot of target t), one sigmoid per
// lane, coefficients broadcast; updates as atomic deltas (see add_delta).
// wk (L ints) and negs (2 W K ints) are this warp's shared memory.  Returns
// this lane's loss in 2^-24 units.
template <int D, class T, int MAXT, int KFIX, bool NC = true>
__device__ __forceinline__ long long fw_train_walk(const TrainView<T> &a, const int32_t *__restrict__ row,
                                                   int64_t wi, int32_t *wk, int32_t *negs) {
    constexpr int EPL = D / 32;
    constexpr int SRC_SHIFT = 5 - (MAXT == 8 ? 3 : 4);
    constexpr bool kBf16 = !std::is_same<T, float>::value;
    const int lane = threadIdx.x & 31;
    const int W = a.W, L = a.L;
    const int K = KFIX > 0 ? KFIX : a.K;
    const uint64_t S = a.S, n = a.n;
    T *const phi_in = a.phi_in;
    T *const phi_out = a.phi_out;
    const int my_t = target_of_lane<MAXT>(lane);
    const bool loss_lane = (lane & ((32 / MAXT) - 1)) == 0;
    long long loss_fx = 0;  // this lane's loss terms, 2^-24 units
    for (int p = lane; p < L; p += 32) wk[p] = walk_id(row[p], n);
    __syncwarp();
    for (int p = 0; p < L; ++p) {
        const int32_t c = wk[p];
        if (c < 0) continue;
        // all negatives of this center, lane-parallel
        for (int idx = lane; idx < 2 * W * K; idx += 32) {
            const int q = idx / K, k = idx - q * K;
            negs[idx] = draw_negative<NC>(a.thr, a.alias, n, S, a.seed, a.round,
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

    return loss_fx;
}

// Staged phi_in increments (STAGE): a warp keeps, for each of the 2W + 1
// positions of its current window, the summed increment of that position's
// phi_in row in shared memory (fp32, `delta`: (2W + 1) rows of D floats, slot
// = position mod (2W + 1)).  A pair reads phi_in[x] from memory plus every
// pending increment this warp holds for node x (all window positions whose
// node is x), so the warp sees all of its own updates as before; the pair's
// increment is added to the slot of its context position; when a position
// leaves the window its summed increment is added to memory once (fp32:
// vector reduction; bf16: stochastically rounded against the row read at
// that moment).  Other warps see a position's phi_in updates when it leaves
// the window instead of after each pair.  Layout of a slot row: lane l of a
// half owns floats [l * EPL, (l + 1) * EPL) for EPL <= 4, and for EPL = 8
// the two 4-float chunks at l * 4 and 64 + l * 4 (conflict-free 16-byte
// accesses by the 16 lanes).
template <int EPL>
__device__ __forceinline__ float *delta_chunk(float *slot_row, int hl, int c) {
    return EPL == 8 ? slot_row + c * 64 + hl * 4 : slot_row + hl * EPL;
}

template <int EPL>
__device__ __forceinline__ void delta_load(float *slot_row, int hl, float (&d)[EPL]) {
    if constexpr (EPL == 8) {
        const float4 a = *reinterpret_cast<const float4 *>(delta_chunk<EPL>(slot_row, hl, 0));
        const float4 b = *reinterpret_cast<const float4 *>(delta_chunk<EPL>(slot_row, hl, 1));
        d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
        d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
    } else if constexpr (EPL == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(slot_row + hl * 4);
        d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
    } else {
        const float2 a = *reinterpret_cast<const float2 *>(slot_row + hl * 2);
        d[0] = a.x; d[1] = a.y;
    }
}

template <int EPL>
__device__ __forceinline__ void delta_store(float *slot_row, int hl, const float (&d)[EPL]) {
    if constexpr (EPL == 8) {
        *reinterpret_cast<float4 *>(delta_chunk<EPL>(slot_row, hl, 0)) = make_float4(d[0], d[1], d[2], d[3]);
        *reinterpret_cast<float4 *>(delta_chunk<EPL>(slot_row, hl, 1)) = make_float4(d[4], d[5], d[6], d[7]);
    } else if constexpr (EPL == 4) {
        *reinterpret_cast<float4 *>(slot_row + hl * 4) = make_float4(d[0], d[1], d[2], d[3]);
    } else {
        *reinterpret_cast<float2 *>(slot_row + hl * 2) = make_float2(d[0], d[1]);
    }
}

// Largest window (2W + 1 positions, one per lane) the staged form handles.
constexpr int kStageMaxWindow = 15;

// Floats of staged increments per warp.
inline size_t stage_floats(int window, int dim) { return static_cast<size_t>(2 * window + 1) * dim; }

// Bulk reductions (form 5, float tables): a step's row increments are
// written to shared memory in the row's own layout and added to the table
// by the bulk-copy engine, one cp.reduce.async.bulk of the whole row each,
// instead of two vector reductions per lane.  A half's K + 1 slots (K
// negatives, then the context) are reused every step once the engine has
// read them (wait_group.read by the issuing lane).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_reduce_add_f32(float *gdst, const float *ssrc, uint32_t bytes) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(ssrc));
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(gdst), "r"(s),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// writes lane hl's elements of a float row increment into a shared-memory
// slot laid out as the row itself (the layout of hw_load / hw_add)
template <int EPL>
__device__ __forceinline__ void slot_store(float *slot, int hl, const float (&d)[EPL]) {
    if constexpr (EPL == 8) {
        *reinterpret_cast<float4 *>(slot + hl * 4) = make_float4(d[0], d[1], d[2], d[3]);
        *reinterpret_cast<float4 *>(slot + 64 + hl * 4) = make_float4(d[4], d[5], d[6], d[7]);
    } else if constexpr (EPL == 4) {
        *reinterpret_cast<float4 *>(slot + hl * 4) = make_float4(d[0], d[1], d[2], d[3]);
    } else {
        *reinterpret_cast<float2 *>(slot + hl * 2) = make_float2(d[0], d[1]);
    }
}

// Shared memory of one warp of the bulk-reduction form: the walk and
// negative ids (rounded up to 16 bytes), then 2 halves x (K + 1) row slots.
__host__ __device__ inline int bulk_bytes_per_warp(int L, int window, int K, int dim) {
    return 4 * ((L + 2 * window * K + 3) & ~3) + 2 * (K + 1) * dim * 4;
}

// Trains all pairs of one walk (row: L node ids local to the graph; wi: the
// walk's index in the graph's round, which keys its negatives and its
// token clock).  wk (L ints) and negs (2 W K ints) are this warp's shared
// memory, and with STAGE delta ((2W + 1) * D floats, all zero on entry and
// on return); with BULK (float tables, not STAGE) `delta` is the warp's
// 2 (K + 1) row slots instead.  Returns this lane's loss in 2^-24 units.
template <int D, class T, int KFIX, bool STAGE = false, bool NC = true, bool BULK = false>
__device__ __forceinline__ long long hw_train_walk(const TrainView<T> &a, const int32_t *__restrict__ row,
                                                   int64_t wi, int32_t *wk, int32_t *negs,
                                                   float *delta = nullptr) {
    constexpr int EPL = D / 16;
    constexpr int MAXT = 8;
    constexpr bool kBf16 = !std::is_same<T, float>::value;
    static_assert(EPL == 2 || EPL == 4 || EPL == 8, "dim");
    static_assert(!BULK || (!kBf16 && !STAGE), "bulk reductions: float tables, not staged");
    const int lane = threadIdx.x & 31;
    const int h = lane >> 4, hl = lane & 15;
    const int W = a.W, L = a.L;
    const int K = KFIX > 0 ? KFIX : a.K;
    float *const slots = BULK ? delta + h * (K + 1) * D : nullptr;  // this half's K + 1 row slots
    const uint64_t S = a.S, n = a.n;
    T *const phi_in = a.phi_in;
    T *const phi_out = a.phi_out;
    const int my_t = hl >> 1;
    const bool loss_lane = (hl & 1) == 0;
    long long loss_fx = 0;
    const int R = 2 * W + 1;
    int sbase = W + 1;  // slot of position p - W, i.e. (p - W) mod R, at p = 0

    // adds the staged increment of position q (slot sq) to memory and clears
    // the slot; half 0 of the warp does it
    auto flush = [&](int q, int sq, uint32_t rw) {
        const int32_t y = wk[q];
        if (h == 0 && y >= 0) {
            float *srow = delta + sq * D;
            float d[EPL];
            delta_load<EPL>(srow, hl, d);
            bool nz = false;
#pragma unroll
            for (int e = 0; e < EPL; ++e) nz |= d[e] != 0.f;
            if (!__any_sync(0x0000ffffu, nz)) return;  // nothing staged for this position
            const float zero[EPL] = {};
            delta_store<EPL>(srow, hl, zero);
            T *grow = phi_in + static_cast<int64_t>(y) * D;
            if constexpr (kBf16) {
                uint32_t raw[EPL / 2];
                load_raw<EPL>(grow + hl * EPL, raw);
                add_delta_raw<EPL>(grow + hl * EPL, raw, d, rw);
            } else {
                hw_add<EPL>(reinterpret_cast<float *>(grow), hl, d);
            }
        }
    };

    for (int p = lane; p < L; p += 32) wk[p] = walk_id(row[p], n);
    __syncwarp();
    for (int p = 0; p < L; ++p) {
        uint32_t srs = 0;
        if constexpr (kBf16)
            srs = philox(a.seed, static_cast<uint32_t>(lane), static_cast<uint32_t>(wi),
                         (a.round << 16) | static_cast<uint32_t>(p), kStreamSR).x | 1u;
        if constexpr (STAGE) {
            // position p - W - 1 leaves the window (its slot is the one before sbase)
            if (p > 0) sbase = sbase + 1 == R ? 0 : sbase + 1;
            if (a.stage_flush > 0 && p > 0 && p % a.stage_flush == 0) {
                // every position of the previous window, p - 1 - W .. p - 1 + W
                int sq = sbase == 0 ? R - 1 : sbase - 1;
                for (int q = p - 1 - W; q <= p - 1 + W; ++q) {
                    if (q >= 0 && q < L) {
                        srs = srs * 1664525u + 1013904223u;
                        flush(q, sq, srs);
                    }
                    sq = sq + 1 == R ? 0 : sq + 1;
                }
                __syncwarp();
            } else {
                const int q = p - W - 1;
                if (q >= 0) {
                    srs = srs * 1664525u + 1013904223u;
                    flush(q, sbase == 0 ? R - 1 : sbase - 1, srs);
                    __syncwarp();
                }
            }
        }
        const int32_t c = wk[p];
        if (c < 0) continue;
        for (int idx = lane; idx < 2 * W * K; idx += 32) {
            const int q = idx / K, k = idx - q * K;
            negs[idx] = draw_negative<NC>(a.thr, a.alias, n, S, a.seed, a.round,
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
        // window offsets o in [lo, hi] \ {0}; lo <= 0 <= hi
        const int lo = max(-W, -p), hi = min(W, L - 1 - p);
        const int npairs = hi - lo;
        // STAGE: lane i stands for window position p - W + i (i < R)
        int32_t win_id = -1;
        if constexpr (STAGE) {
            const int pos = p - W + lane;
            if (lane < R && pos >= 0 && pos < L) win_id = wk[pos];
        }
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
            if constexpr (STAGE) {
                // add this warp's pending increments of node x (every window
                // position holding x, its own position included)
                const int32_t x0 = __shfl_sync(kFull, x, 0), x1 = __shfl_sync(kFull, x, 16);
                const uint32_t m0 = __ballot_sync(kFull, win_id >= 0 && win_id == x0);
                const uint32_t m1 = __ballot_sync(kFull, win_id >= 0 && win_id == x1);
                uint32_t mine = valid ? (h ? m1 : m0) : 0u;
                while (__any_sync(kFull, mine != 0)) {
                    if (mine) {
                        const int b = __ffs(mine) - 1;
                        mine &= mine - 1;
                        const int sl = sbase + b >= R ? sbase + b - R : sbase + b;
                        float d[EPL];
                        delta_load<EPL>(delta + sl * D, hl, d);
#pragma unroll
                        for (int e = 0; e < EPL; ++e) ix[e] += d[e];
                    }
                }
                __syncwarp();
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
            if constexpr (BULK) {
                // the engine has read the previous step's slots before they are rewritten
                if (hl == 0) bulk_wait_read_all();
                __syncwarp();
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
                    add_delta_vals<EPL>(nrow + hl * EPL, nr[t], nr_raw[t], dn, srs);
                } else if constexpr (BULK) {
                    slot_store<EPL>(slots + (t - 1) * D, hl, dn);
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
            if constexpr (STAGE) {
                if (valid) {  // the context position's slot takes the increment
                    const int i = o + W;
                    float *srow = delta + (sbase + i >= R ? sbase + i - R : sbase + i) * D;
                    float d[EPL];
                    delta_load<EPL>(srow, hl, d);
#pragma unroll
                    for (int e = 0; e < EPL; ++e) d[e] += din[e];
                    delta_store<EPL>(srow, hl, d);
                }
                __syncwarp();
            } else if (valid) {
                if constexpr (kBf16) {
                    srs = srs * 1664525u + 1013904223u;
                    add_delta_vals<EPL>(ix_row + hl * EPL, ix, ix_raw, din, srs);
                } else if constexpr (BULK) {
                    slot_store<EPL>(slots + K * D, hl, din);
                } else {
                    hw_add<EPL>(reinterpret_cast<float *>(ix_row), hl, din);
                }
            }
            if constexpr (BULK) {
                // the slots' writes reach the async proxy, then one lane per
                // half hands every written row to the bulk-copy engine
                fence_proxy_async_smem();
                __syncwarp();
                if (hl == 0) {
#pragma unroll
                    for (int t = 1; t < MAXT; ++t)
                        if (t <= K && nid[t] >= 0)
                            bulk_reduce_add_f32(reinterpret_cast<float *>(phi_out + static_cast<int64_t>(nid[t]) * D),
                                                slots + (t - 1) * D, D * 4);
                    if (valid) bulk_reduce_add_f32(reinterpret_cast<float *>(ix_row), slots + K * D, D * 4);
                    bulk_commit();
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
    if constexpr (BULK) {
        // every reduction of this walk has completed (the slots are free and
        // nothing is in flight when the warp moves on or exits)
        if (hl == 0) bulk_wait_all();
        __syncwarp();
    }
    if constexpr (STAGE) {
        // the last window: positions max(0, L - W - 1) .. L - 1 are still staged
        uint32_t rw = 0;
        if constexpr (kBf16)
            rw = philox(a.seed, static_cast<uint32_t>(lane), static_cast<uint32_t>(wi),
                        (a.round << 16) | static_cast<uint32_t>(L), kStreamSR).x | 1u;
        int sq = sbase;  // slot of position L - 1 - W
        for (int q = L - 1 - W; q < L; ++q) {
            if (q >= 0) {
                rw = rw * 1664525u + 1013904223u;
                flush(q, sq, rw);
            }
            sq = sq + 1 == R ? 0 : sq + 1;
        }
        __syncwarp();
    }
    return loss_fx;
}

// ----------------------------------------------------------------------------
// HOGWILD, half-warp form with the next step's rows prefetched (form 4): the
// context row and the K negative rows of step j + 1 are copied to shared
// memory with cp.async (16-byte chunks, bypassing L1; invalid rows zero-filled)
// while step j computes, so the L2 latency of a step's rows overlaps the
// previous step's dots, sigmoid and reductions.  Rows live in a per-warp
// double buffer: [2 stages][2 halves][K + 1 rows][D values of T]; lane l of a
// half copies and later reads the same 16-byte chunks of each row (chunks l
// and l + 16 for a 512-byte row, chunk l for a 256-byte row), so a lane
// needs only its own copies to complete; a 128-byte row is copied by the
// half's first 8 lanes, 16 bytes each, and read 8 bytes per lane, so every
// lane waits for the whole half's copies (cp.async.wait_group, then the
// warp's __syncwarp).  The arithmetic is form 2's; a step's rows are read one
// step earlier than form 2 reads them (before the previous step's updates of
// the same rows, if any, reach memory).  Rows of 128, 256 or 512 bytes: float
// dim 32, 64 or 128, bf16 dim 64 or 128.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_none() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// rows of 128, 256 or 512 bytes: float dim 32/64/128, bf16 dim 64/128
template <int D, class T>
constexpr bool kPfSupported = (std::is_same<T, float>::value && (D == 32 || D == 64 || D == 128)) ||
                              (!std::is_same<T, float>::value && (D == 64 || D == 128));

// Shared memory of one warp of the prefetching form: the walk and negative
// ids (rounded up to 16 bytes), then the double buffer of rows.
__host__ __device__ inline int pf_bytes_per_warp(int L, int window, int K, int dim, int elem) {
    const int ids = 4 * ((L + 2 * window * K + 3) & ~3);
    return ids + 2 * 2 * (K + 1) * dim * elem;
}

template <int D, class T, int KFIX>
__device__ __forceinline__ long long hw_train_walk_pf(const TrainView<T> &a, const int32_t *__restrict__ row,
                                                      int64_t wi, int32_t *wk, int32_t *negs, char *rowbuf) {
    constexpr int EPL = D / 16;
    constexpr int MAXT = 8;
    constexpr bool kBf16 = !std::is_same<T, float>::value;
    constexpr int ROWB = D * static_cast<int>(sizeof(T));  // bytes of a row
    constexpr int CHUNKS = ROWB / 256;  // 16-byte copies per lane: 2 (512 B), 1 (256 B); 0: 128-byte rows,
                                        // copied by the half's first 8 lanes, 16 bytes each
    static_assert(kPfSupported<D, T>, "rows of 128, 256 or 512 bytes");
    const int lane = threadIdx.x & 31;
    const int h = lane >> 4, hl = lane & 15;
    const int W = a.W, L = a.L;
    const int K = KFIX > 0 ? KFIX : a.K;
    const uint64_t S = a.S, n = a.n;
    T *const phi_in = a.phi_in;
    T *const phi_out = a.phi_out;
    const int my_t = hl >> 1;
    const bool loss_lane = (hl & 1) == 0;
    long long loss_fx = 0;
    const uint32_t buf0 = static_cast<uint32_t>(__cvta_generic_to_shared(rowbuf));
    // shared-memory address of row t of half h in stage s
    auto slot = [&](int s, int t) -> uint32_t {
        return buf0 + static_cast<uint32_t>(((s * 2 + h) * (K + 1) + t) * ROWB);
    };
    auto slot_ptr = [&](int s, int t) -> const char * {
        return rowbuf + ((s * 2 + h) * (K + 1) + t) * ROWB;
    };

    for (int p = lane; p < L; p += 32) wk[p] = walk_id(row[p], n);
    __syncwarp();
    for (int p = 0; p < L; ++p) {
        uint32_t srs = 0;
        if constexpr (kBf16)
            srs = philox(a.seed, static_cast<uint32_t>(lane), static_cast<uint32_t>(wi),
                         (a.round << 16) | static_cast<uint32_t>(p), kStreamSR).x | 1u;
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
        const int lo = max(-W, -p), hi = min(W, L - 1 - p);
        const int npairs = hi - lo;
        const int steps = (npairs + 1) >> 1;
        // the pair of this half in step j: offset o, context x, negatives nid[1..K]
        auto pair_of = [&](int j, int &o, int32_t &x, int32_t (&nid)[MAXT]) -> bool {
            const int jj = 2 * j + h;
            o = lo + jj;
            if (o >= 0) ++o;
            bool valid = jj < npairs;
            x = valid ? wk[p + o] : -1;
            valid = valid && x >= 0;
            const int q = o < 0 ? o + W : o + W - 1;
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
            return valid;
        };
        // copies of step j's rows (context, then negatives) into stage j & 1
        auto issue = [&](int j) {
            int o;
            int32_t x, nid[MAXT];
            const bool valid = pair_of(j, o, x, nid);
            const int s = j & 1;
            const char *ix_src = reinterpret_cast<const char *>(phi_in + static_cast<int64_t>(valid ? x : 0) * D);
            if constexpr (CHUNKS == 0) {
                if (hl < 8) cp_async16_zfill(slot(s, 0) + hl * 16, ix_src + hl * 16, valid);
            }
#pragma unroll
            for (int ch = 0; ch < CHUNKS; ++ch)
                cp_async16_zfill(slot(s, 0) + (ch * 16 + hl) * 16, ix_src + (ch * 16 + hl) * 16, valid);
#pragma unroll
            for (int t = 1; t < MAXT; ++t) {
                if (t > K) break;
                const bool ok = nid[t] >= 0;
                const char *src = reinterpret_cast<const char *>(phi_out + static_cast<int64_t>(ok ? nid[t] : 0) * D);
                if constexpr (CHUNKS == 0) {
                    if (hl < 8) cp_async16_zfill(slot(s, t) + hl * 16, src + hl * 16, ok);
                }
#pragma unroll
                for (int ch = 0; ch < CHUNKS; ++ch)
                    cp_async16_zfill(slot(s, t) + (ch * 16 + hl) * 16, src + (ch * 16 + hl) * 16, ok);
            }
            cp_async_commit_group();
        };
        // this lane's values of row t of stage s (the chunks it copied), as floats and raw bf16 words
        auto read_row = [&](int s, int t, float (&v)[EPL], uint32_t (&raw)[kBf16 ? EPL / 2 : 1]) {
            const char *base = slot_ptr(s, t);
            if constexpr (kBf16 && EPL == 4) {
                const uint2 w = *reinterpret_cast<const uint2 *>(base + hl * 8);
                raw[0] = w.x; raw[1] = w.y;
                unpack_bf16<EPL>(raw, v);
            } else if constexpr (kBf16) {
                const uint4 w = *reinterpret_cast<const uint4 *>(base + hl * 16);
                raw[0] = w.x; raw[1] = w.y; raw[2] = w.z; raw[3] = w.w;
                unpack_bf16<EPL>(raw, v);
            } else if constexpr (EPL == 2) {
                const float2 u = *reinterpret_cast<const float2 *>(base + hl * 8);
                v[0] = u.x; v[1] = u.y;
            } else if constexpr (EPL == 8) {
                const float4 u = *reinterpret_cast<const float4 *>(base + hl * 16);
                const float4 w = *reinterpret_cast<const float4 *>(base + 256 + hl * 16);
                v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
                v[4] = w.x; v[5] = w.y; v[6] = w.z; v[7] = w.w;
            } else {
                const float4 u = *reinterpret_cast<const float4 *>(base + hl * 16);
                v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
            }
        };

        if (steps > 0) issue(0);
        for (int j = 0; j < steps; ++j) {
            if (j + 1 < steps) issue(j + 1);
            else cp_async_commit_group();  // an empty group: wait_group 1 below then means step j
            cp_async_wait_prev();
            // a 128-byte row is read by lanes other than the 8 that copied it: every
            // lane's copies of step j have landed before any lane reads
            if constexpr (CHUNKS == 0) __syncwarp();
            const int s = j & 1;
            int o;
            int32_t x, nid[MAXT];
            const bool valid = pair_of(j, o, x, nid);
            float ix[EPL];
            uint32_t ix_raw[kBf16 ? EPL / 2 : 1];
            read_row(s, 0, ix, ix_raw);
            float pd[MAXT];
#pragma unroll
            for (int t = 0; t < MAXT; ++t) {
                float r[EPL];
                uint32_t rr[kBf16 ? EPL / 2 : 1];
                if (t == 0) {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) r[e] = oc[e];
                } else if (t <= K) {
                    read_row(s, t, r, rr);
                } else {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) r[e] = 0.f;
                }
                float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int e = 0; e < EPL; e += 2)
                    s2 = __ffma2_rn(make_float2(ix[e], ix[e + 1]), make_float2(r[e], r[e + 1]), s2);
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
                const float2 r2 = __fmul2_rn(make_float2(gt[0], gt[0]), make_float2(oc[e], oc[e + 1]));
                din[e] = r2.x;
                din[e + 1] = r2.y;
            }
#pragma unroll
            for (int t = 1; t < MAXT; ++t) {
                if (t > K || nid[t] < 0) continue;
                float nr[EPL];
                uint32_t nr_raw[kBf16 ? EPL / 2 : 1];
                read_row(s, t, nr, nr_raw);
                float dn[EPL];
#pragma unroll
                for (int e = 0; e < EPL; e += 2) {
                    const float2 gg = make_float2(gt[t], gt[t]);
                    const float2 r2 = __ffma2_rn(gg, make_float2(nr[e], nr[e + 1]), make_float2(din[e], din[e + 1]));
                    din[e] = r2.x;
                    din[e + 1] = r2.y;
                    const float2 u = __fmul2_rn(gg, make_float2(ix[e], ix[e + 1]));
                    dn[e] = u.x;
                    dn[e + 1] = u.y;
                }
                T *nrow = phi_out + static_cast<int64_t>(nid[t]) * D;
                if constexpr (kBf16) {
                    srs = srs * 1664525u + 1013904223u;
                    add_delta_vals<EPL>(nrow + hl * EPL, nr, nr_raw, dn, srs);
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
                T *ix_row = phi_in + static_cast<int64_t>(x) * D;
                if constexpr (kBf16) {
                    srs = srs * 1664525u + 1013904223u;
                    add_delta_vals<EPL>(ix_row + hl * EPL, ix, ix_raw, din, srs);
                } else {
                    hw_add<EPL>(reinterpret_cast<float *>(ix_row), hl, din);
                }
            }
            __syncwarp();  // stage s is refilled by the issue of step j + 2
        }
        cp_async_wait_none();
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
    return loss_fx;
}

// ----------------------------------------------------------------------------
// Synchronous minibatch (the deterministic form), shared by the single-graph
// kernels (sgns.cu) and the batched ones (batch.cu): one warp per center
// position; the tables are read only; increments go to 64-bit fixed-point
// accumulators (2^-40 units), which makes the per-row sums exact and order
// independent; touched rows are marked (and, when lists are given, listed).
// ----------------------------------------------------------------------------
struct MbState {
    long long *acc_in, *acc_out;  // [n][D]
    uint32_t *mark_in, *mark_out; // [n]
    int32_t *list_in, *list_out;  // [n], or null: rows are only marked
    int32_t *counters;            // [0] = |list_in|, [1] = |list_out|, [2] = apply ticket
};

struct MbView {
    const uint64_t *thr;
    const int32_t *alias;
    uint64_t n, S, seed;
    uint32_t round;
    int W, K, L;
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
    if (!list) {
        mark[r] = 1u;
        return;
    }
    if (atomicExch(mark + r, 1u) == 0u) list[atomicAdd(counter, 1)] = r;
}

// All pairs of center position p of walk wi (row = its L ids); eta is the
// batch's rate; negs: this warp's 2 W K ints of shared memory.  Returns this
// lane's share of the loss.
template <int D, class T, int MAXT, bool NC = true>
__device__ __forceinline__ float mb_grad_center(const MbView &a, const int32_t *__restrict__ row, int64_t wi, int p,
                                                float eta, const T *__restrict__ phi_in,
                                                const T *__restrict__ phi_out, const MbState &st, int32_t *negs) {
    constexpr int EPL = D / 32;
    const int lane = threadIdx.x & 31;
    const int W = a.W, K = a.K, L = a.L;
    const uint64_t n = a.n;
    const int my_t = target_of_lane<MAXT>(lane);
    const bool loss_lane = (lane & ((32 / MAXT) - 1)) == 0;
    const int32_t c = walk_id(row[p], n);
    if (c < 0) return 0.f;
    for (int idx = lane; idx < 2 * W * K; idx += 32) {
        const int q = idx / K, k = idx - q * K;
        negs[idx] = draw_negative<NC>(a.thr, a.alias, n, a.S, a.seed, a.round, static_cast<uint32_t>(wi),
                                  static_cast<uint32_t>(p), static_cast<uint32_t>(q), static_cast<uint32_t>(k));
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
        const int32_t x = walk_id(row[pp], n);
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
    return closs;
}

// Adds row r's accumulated increment to table `tab` (stochastically rounded
// for bf16, bits from Philox(seed; lane | table << 8, r, batch_key, stream 4)),
// then clears the accumulator and the mark; one warp per row.
template <int D, class T>
__device__ __forceinline__ void mb_apply_row(T *__restrict__ tab, long long *__restrict__ acc_tab,
                                             uint32_t *__restrict__ mark, int32_t r, bool is_in, uint64_t seed,
                                             uint32_t batch_key, int lane) {
    constexpr int EPL = D / 32;
    long long *acc = acc_tab + static_cast<int64_t>(r) * D + lane * EPL;
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
        rr = philox(seed, static_cast<uint32_t>(lane) | (is_in ? 0u : 0x100u), static_cast<uint32_t>(r), batch_key,
                    kStreamSR).x;
    store_row<EPL>(tab + static_cast<int64_t>(r) * D + lane * EPL, v, rr);
    if (lane == 0) mark[r] = 0u;
}

}  // namespace felog
