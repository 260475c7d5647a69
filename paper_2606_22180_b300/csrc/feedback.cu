// Feedback: neighbourhood-consistency score Psi (Eq. 4) and next active set
// (Eq. 5); a warp takes groups of consecutive nodes (feedback_core.cuh).
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

#include "feedback_core.cuh"

namespace felog {

int sm_count();
bool csr_shape_ok(const felog_csr *g);

constexpr int kPsiThreads = 256;
constexpr int kPsiWarps = kPsiThreads / 32;

template <class T>
__global__ void __launch_bounds__(kPsiThreads)
    k_feedback(const int32_t *__restrict__ offsets, const int32_t *__restrict__ cols, int32_t n, int64_t nnz,
               const T *__restrict__ phi, int32_t dim, int32_t enabled, double mu, int32_t ks,
               int32_t reactivate, uint64_t seed, uint32_t round, const uint8_t *__restrict__ active_in,
               uint8_t *__restrict__ active_out, double *__restrict__ psi_out,
               int32_t *__restrict__ n_next) {
    __shared__ PsiScratch scratch[kPsiWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    PsiScratch &w = scratch[wib];
    const int GN = psi_group_size(ks);
    int32_t count = 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * kPsiWarps;
    // a warp takes GN consecutive nodes at a time: their totals one node after
    // the other, then their cosines and means lane-parallel
    for (int64_t base = (static_cast<int64_t>(blockIdx.x) * kPsiWarps + wib) * GN; base < n; base += warps * GN) {
        const int cnt = static_cast<int>(n - base < GN ? n - base : GN);
        for (int i = 0; i < cnt; ++i) {
            const int64_t v = base + i;
            const int32_t lo = offsets[v], hi = offsets[v + 1];
            // a row outside [0, nnz] (a malformed graph) is treated as isolated
            const int64_t deg = lo >= 0 && hi <= nnz ? static_cast<int64_t>(hi) - lo : 0;
            const bool evaluate = deg > 0 && (reactivate || active_in[v]);
            if (evaluate) psi_node_totals<T>(cols, phi, n, dim, ks, seed, round, v, lo, deg, w, i);
            else if (lane == 0) w.m[i] = 0;
        }
        const double psi = psi_group_finish(w, cnt, ks);  // NaN for nodes not evaluated
        if (lane < cnt) {
            const int64_t v = base + lane;
            const int32_t lo = offsets[v], hi = offsets[v + 1];
            const bool live = lo >= 0 && hi <= nnz && hi > lo;
            const bool evaluated = w.m[lane] > 0;  // m, not Psi, marks an evaluated node
            const uint8_t next = enabled ? static_cast<uint8_t>(evaluated && psi < mu) : static_cast<uint8_t>(live);
            active_out[v] = next;
            if (psi_out) psi_out[v] = psi;
            count += next;
        }
        __syncwarp();
    }
    for (int o = 16; o; o >>= 1) count += __shfl_xor_sync(kFull, count, o);
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
    const int grid = std::min(ceil_div(g->n, kPsiWarps * psi_group_size(fp->ks)), sm_count() * 16);
    if (precision == FELOG_FP32)
        k_feedback<float><<<grid, kPsiThreads, 0, s>>>(
            g->offsets, g->cols, g->n, g->nnz, static_cast<const float *>(phi_in), dim, fp->enabled, fp->mu,
            fp->ks, fp->reactivate, seed, static_cast<uint32_t>(round), active_in, active_out, psi, n_next);
    else
        k_feedback<__nv_bfloat16><<<grid, kPsiThreads, 0, s>>>(
            g->offsets, g->cols, g->n, g->nnz, static_cast<const __nv_bfloat16 *>(phi_in), dim, fp->enabled,
            fp->mu, fp->ks, fp->reactivate, seed, static_cast<uint32_t>(round), active_in, active_out,
            psi, n_next);
    return check_launch("felog_feedback");
}
