// Shared device helpers of the CUDA path: Philox4x32-10, 64-bit multiply-high,
// status plumbing.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "felog.h"

namespace felog {

constexpr uint32_t kStreamWalk = 0;
constexpr uint32_t kStreamPsi = 1;
constexpr uint32_t kStreamNeg = 2;
constexpr uint32_t kStreamInit = 3;
constexpr uint32_t kStreamSR = 4;

struct u32x4 {
    uint32_t x, y, z, w;
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds, each two
// 32x32->64 products; the key advances by the Weyl constants between rounds.
__device__ __forceinline__ u32x4 philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                        uint32_t c3) {
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ uint64_t lo64(const u32x4 &w) {
    return (static_cast<uint64_t>(w.y) << 32) | w.x;
}
__device__ __forceinline__ uint64_t hi64(const u32x4 &w) {
    return (static_cast<uint64_t>(w.w) << 32) | w.z;
}
// floor(u * m / 2^64)
__device__ __forceinline__ uint64_t mulhi64(uint64_t u, uint64_t m) { return __umul64hi(u, m); }

constexpr unsigned kFull = 0xffffffffu;

inline int ceil_div(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

// Records the CUDA error (if any) and maps it to a status.
felog_status check_launch(const char *where);
felog_status record_cuda_error(cudaError_t e, const char *where);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-provided workspace.
struct Carver {
    char *base;
    size_t size, used = 0;
    Carver(void *b, size_t s) : base(static_cast<char *>(b)), size(s) {}
    template <class T>
    T *take(size_t count, size_t align = 256) {
        used = align_up(used, align);
        T *p = reinterpret_cast<T *>(base ? base + used : nullptr);
        used += count * sizeof(T);
        return p;
    }
    bool ok() const { return base != nullptr && used <= size; }
};

}  // namespace felog
