// Feedback: neighbourhood-consistency score Psi (Eq. 4) and next active set
// (Eq. 5), one warp per evaluated node.
//
// The neighbour subset is all neighbours when deg <= ks, else ks distinct
// CSR positions chosen by Floyd's algorithm (Bentley and Floyd, CACM 1987)
// with step s drawing uniformly from [0, deg - ks + s] via Philox(x0=s,
// x1=v, x2=round, stream 1); positions are sorted ascending.
//
// All arithmetic is binary64 with explicit round-to-nearest intrinsics (no
// FMA contraction) in one fixed order, so Psi and the decision Psi < mu are
// reproducible bit for bit: lane l sums elements l, l+32, l+64, ...; the 32
// partials are combined by a xor butterfly over distances 16, 8, 4, 2, 1;
// cos = dot / (sqrt(|v|^2) * sqrt(|u|^2)) (0 for a zero row); Psi is the sum
// of the cosines in ascending subset order divided by the subset size.
// Rows are converted exactly from float or bfloat16.
#include <math.h>

#include "common.cuh"

namespace felog {

int sm_count();
bool csr_shape_ok(const felog_csr *g);

constexpr int kPsiThreads = 256;
constexpr int kPsiWarps = kPsiThreads / 32;
constexpr int kMaxKs = 32;

__device__ __forceinline__ double elem(const float *p, int64_t i) { return static_cast<double>(p[i]); }
__device__ __forceinline__ double elem(const __nv_bfloat16 *p, int64_t i) {
    return static_cast<double>(__bfloat162float(p[i]));
}

__device__ __forceinline__ double butterfly(double s) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kFull, s, o));
    return s;
}

template <class T>
__global__ void __launch_bounds__(kPsiThreads)
    k_feedback(const int32_t *__restrict__ offsets, const int32_t *__restrict__ cols, int32_t n,
               const T *__restrict__ phi, int32_t dim, int32_t enabled, double mu, int32_t ks,
               int32_t reactivate, uint64_t seed, uint32_t round, const uint8_t *__restrict__ active_in,
               uint8_t *__restrict__ active_out, double *__restrict__ psi_out,
               int32_t *__restrict__ n_next) {
    __shared__ int32_t sub_s[kPsiWarps][kMaxKs];
    __shared__ int32_t sorted_s[kPsiWarps][kMaxKs];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t *sub = sub_s[wib];
    int32_t *sorted = sorted_s[wib];
    int32_t count = 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kPsiWarps;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kPsiWarps + wib; v < n; v += warps) {
        const int32_t lo = offsets[v];
        const int64_t deg = static_cast<int64_t>(offsets[v + 1]) - lo;
        const bool evaluate = deg > 0 && (reactivate || active_in[v]);
        double psi = __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
        if (evaluate) {
            int32_t m;
            if (deg <= ks) {
                m = static_cast<int32_t>(deg);
                if (lane < m) sorted[lane] = lane;
            } else {
                m = ks;
                int64_t t_mine = 0;
                if (lane < ks) {
                    const int64_t j = deg - ks + lane;
                    const u32x4 r = philox(seed, static_cast<uint32_t>(lane), static_cast<uint32_t>(v), round,
                                           kStreamPsi);
                    t_mine = static_cast<int64_t>(mulhi64(lo64(r), static_cast<uint64_t>(j + 1)));
                }
                // Floyd's sequential resolution, on lane 0
                for (int s = 0; s < ks; ++s) {
                    const int64_t t = __shfl_sync(kFull, t_mine, s);
                    if (lane == 0) {
                        bool present = false;
                        for (int a = 0; a < s; ++a) present |= sub[a] == t;
                        sub[s] = static_cast<int32_t>(present ? deg - ks + s : t);
                    }
                }
                __syncwarp();
                if (lane < m) {
                    const int32_t x = sub[lane];
                    int rank = 0;
                    for (int a = 0; a < m; ++a) rank += sub[a] < x;
                    sorted[rank] = x;
                }
            }
            __syncwarp();
            const T *pv = phi + v * dim;
            double nv = 0.0;
            for (int i = lane; i < dim; i += 32) {
                const double x = elem(pv, i);
                nv = __dadd_rn(nv, __dmul_rn(x, x));
            }
            nv = butterfly(nv);
            double sum = 0.0;
            for (int a = 0; a < m; ++a) {
                const int32_t u = cols[lo + sorted[a]];
                const T *pu = phi + static_cast<int64_t>(u) * dim;
                double nu = 0.0, dt = 0.0;
                for (int i = lane; i < dim; i += 32) {
                    const double y = elem(pu, i);
                    nu = __dadd_rn(nu, __dmul_rn(y, y));
                    dt = __dadd_rn(dt, __dmul_rn(elem(pv, i), y));
                }
                nu = butterfly(nu);
                dt = butterfly(dt);
                double cs = 0.0;
                if (nv > 0.0 && nu > 0.0) cs = __ddiv_rn(dt, __dmul_rn(__dsqrt_rn(nv), __dsqrt_rn(nu)));
                sum = __dadd_rn(sum, cs);
            }
            psi = __ddiv_rn(sum, static_cast<double>(m));
            __syncwarp();
        }
        uint8_t next;
        if (!enabled) next = deg > 0;
        else next = evaluate && psi < mu;
        if (lane == 0) {
            active_out[v] = next;
            if (psi_out) psi_out[v] = psi;
        }
        count += next;
    }
    if (lane == 0 && count) atomicAdd(n_next, count);
}

}  // namespace felog

using namespace felog;

extern "C" felog_status felog_feedback(const felog_csr *g, const void *phi_in, int32_t dim,
                                       int32_t precision, const felog_feedback_params *fp,
                                       uint64_t seed, int32_t round, const uint8_t *active_in,
                                       uint8_t *active_out, double *psi, int32_t *n_next,
                                       void *stream) {
    if (!csr_shape_ok(g)) return FELOG_ERR_BAD_CSR;
    if (!fp || fp->ks < 1 || fp->ks > kMaxKs || round < 0 || !n_next) return FELOG_ERR_INVALID_ARG;
    if (dim != 32 && dim != 64 && dim != 128 && dim != 256) return FELOG_ERR_INVALID_ARG;
    if (precision != FELOG_FP32 && precision != FELOG_BF16_SR) return FELOG_ERR_INVALID_ARG;
    if (g->n > 0 && (!phi_in || !active_in || !active_out)) return FELOG_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    felog_status st = record_cuda_error(cudaMemsetAsync(n_next, 0, sizeof(int32_t), s), "feedback");
    if (st || g->n == 0) return st;
    const int grid = std::min(ceil_div(g->n, kPsiWarps), sm_count() * 16);
    if (precision == FELOG_FP32)
        k_feedback<float><<<grid, kPsiThreads, 0, s>>>(
            g->offsets, g->cols, g->n, static_cast<const float *>(phi_in), dim, fp->enabled, fp->mu,
            fp->ks, fp->reactivate, seed, static_cast<uint32_t>(round), active_in, active_out, psi, n_next);
    else
        k_feedback<__nv_bfloat16><<<grid, kPsiThreads, 0, s>>>(
            g->offsets, g->cols, g->n, static_cast<const __nv_bfloat16 *>(phi_in), dim, fp->enabled,
            fp->mu, fp->ks, fp->reactivate, seed, static_cast<uint32_t>(round), active_in, active_out,
            psi, n_next);
    return check_launch("felog_feedback");
}
