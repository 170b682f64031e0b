// ssa_warp.cu -- warp-per-trajectory forward and adjoint for networks with many reactions
// (arXiv 2602.19775, Section 2, Section 3.2, Eqs. 3, 5, 6, 7, Section 3.1).
//
// One warp simulates one trajectory. Lane l owns the Philox blocks b = l, l + 32, ... of each step,
// i.e. the words q = 4b..4b+3 and the reactions j = q - 1 they drive, so no Philox word is computed
// twice. Per step:
//   - each lane evaluates its reactions' propensities, its partial sum of a0 (fixed order) and its
//     local exponential race;
//   - a0 is a butterfly sum over the lanes (every lane obtains the same bits);
//   - the Gumbel-max choice is a butterfly argmax of (a_j, E_j, j) with the comparison a_i E_b > a_b E_i
//     and ties to the lowest j;
//   - the clock, the sample writes and the state update are warp-uniform (lanes share the stoichiometry
//     and observable loops).
// The network tables and the per-reaction values are stored lane-major (jpos in ssa_internal.cuh), so
// the lanes' table reads are free of shared-memory bank conflicts.
// The adjoint keeps per-reaction values in per-warp shared memory and accumulates the state adjoint
// through a species -> reactant-slot incidence table in a fixed order (no atomics, deterministic).
// A run recorded by the warp forward is differentiated by the warp adjoint, which repeats the same
// binary32 operations in the same order.
#include <cstdint>

#include "ssa_warp_body.cuh"

namespace ssa {

template <int READOUT, bool RECORD>
__global__ void __launch_bounds__(256) fwd_warp_kernel(const FwdParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int N = p.N, M = p.M;
    const int Npad = (N + 3) & ~3;
    int4 *s_rx = reinterpret_cast<int4 *>(smem);
    int *s_st = reinterpret_cast<int *>(smem + 16 * p.Mp);
    float *s_k = reinterpret_cast<float *>(smem + p.tab_bytes);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + p.tab_bytes + p.k_bytes);
    int *s_ok = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 8);
    int *X = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 16) + wib * Npad;

    if (!stage_tables(smem, p.rx, p.tab_bytes, s_k, p.k_rates, p.k_bytes, s_bar, s_ok, p.err)) return;
    const int64_t i = (int64_t)blockIdx.x * W + wib;
    if (i >= p.n_traj) return;  // whole warp
    warp_fwd_body<READOUT, RECORD>(p, s_rx, s_st, s_k, X, i);
}

// The soft forward (Eq. 4) on the warp layout: the staged tables and rates, then the species-major update
// list; per warp X [Npad], dX [Npad] (floats) and the keys / weights y [Mp].
template <int READOUT, bool RECORD>
__global__ void __launch_bounds__(256) fwd_warp_soft_kernel(const FwdParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int wib = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int Npad = (p.N + 3) & ~3;
    int4 *s_rx = reinterpret_cast<int4 *>(smem);
    float *s_k = reinterpret_cast<float *>(smem + p.tab_bytes);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + p.tab_bytes + p.k_bytes);
    int *s_ok = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 8);
    int *s_upd = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 16);
    float *wbase = reinterpret_cast<float *>(s_upd + p.upd_words) + wib * (2 * Npad + p.Mp);

    if (!stage_tables(smem, p.rx, p.tab_bytes, s_k, p.k_rates, p.k_bytes, s_bar, s_ok, p.err)) return;
    for (uint32_t q = threadIdx.x; q < p.upd_words; q += blockDim.x) s_upd[q] = p.upd[q];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * W + wib;
    if (i >= p.n_traj) return;  // whole warp
    warp_soft_fwd_body<READOUT, RECORD>(p, s_rx, s_k, s_upd, wbase, wbase + Npad, wbase + 2 * Npad, i);
}

// Gradient of the soft forward on the warp layout: tables, rates, the update list, then per warp
// Xs [kSoftK][Npad], lam [Npad], dX [Npad], a, h, y, c1, c2, dA [Mp]; dA reduced over the block in a fixed order.
template <int READOUT>
__global__ void __launch_bounds__(256) adj_warp_soft_kernel(const AdjParams p, const int *upd, uint32_t upd_words)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int N = p.N, M = p.M, Mp = p.Mp;
    const int Npad = (N + 3) & ~3;
    int4 *s_rx = reinterpret_cast<int4 *>(smem);
    int *s_st = reinterpret_cast<int *>(smem + 16 * Mp);
    const int *s_inc_ptr = reinterpret_cast<const int *>(smem + p.inc_off);
    const int *s_inc = reinterpret_cast<const int *>(smem + p.inc_list_off);
    float *s_k = reinterpret_cast<float *>(smem + p.tab_bytes);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + p.tab_bytes + p.k_bytes);
    int *s_ok = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 8);
    int *s_upd = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 16);
    const size_t per_warp = (size_t)(kSoftK + 2) * Npad + 6 * (size_t)Mp;
    float *base0 = reinterpret_cast<float *>(s_upd + upd_words);
    float *wbase = base0 + wib * per_warp;
    float *Xs = wbase;
    float *lam = Xs + kSoftK * Npad;
    float *dX = lam + Npad;
    float *aj = dX + Npad;
    float *hj = aj + Mp;
    float *y = hj + Mp;
    float *c1 = y + Mp;
    float *c2 = c1 + Mp;
    float *dA = c2 + Mp;

    if (!stage_tables(smem, p.rx, p.tab_bytes, s_k, p.k_rates, p.k_bytes, s_bar, s_ok, p.err)) {
        for (int j = threadIdx.x; j < M; j += blockDim.x) p.partial[(int64_t)blockIdx.x * M + j] = 0.0f;
        return;
    }
    for (uint32_t q = threadIdx.x; q < upd_words; q += blockDim.x) s_upd[q] = upd[q];
    for (int j = lane; j < Mp; j += 32) dA[j] = 0.0f;
    __syncthreads();

    const int64_t n = p.n_traj;
    const int64_t i = (int64_t)blockIdx.x * W + wib;
    int st = -1;
    if (i < n) st = p.status[i];
    const bool active = st == SSA_TRAJ_OK || st == SSA_TRAJ_ABSORBED || st == SSA_TRAJ_STEP_CAP;
    if (active)
        warp_soft_adj_body<READOUT>(p, s_rx, s_st, s_inc_ptr, s_inc, s_k, s_upd, Xs, lam, dX, aj, hj, y, c1, c2, dA, i,
                                    st);
    __syncthreads();
    const int nb = (M + 4) >> 2;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        float acc = 0.0f;
        for (int w = 0; w < W; ++w) acc += base0[w * per_warp + (kSoftK + 2) * Npad + 5 * Mp + jpos(j, nb)];
        p.partial[(int64_t)blockIdx.x * M + j] = acc;
    }
}

template <int READOUT>
__global__ void __launch_bounds__(256) adj_warp_kernel(const AdjParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int N = p.N, M = p.M, Mp = p.Mp;
    const int Npad = (N + 3) & ~3;
    int4 *s_rx = reinterpret_cast<int4 *>(smem);
    int *s_st = reinterpret_cast<int *>(smem + 16 * Mp);
    const int *s_inc_ptr = reinterpret_cast<const int *>(smem + p.inc_off);
    const int *s_inc = reinterpret_cast<const int *>(smem + p.inc_list_off);
    float *s_k = reinterpret_cast<float *>(smem + p.tab_bytes);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + p.tab_bytes + p.k_bytes);
    int *s_ok = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 8);
    // per warp: X [Npad] int, lambda [Npad], a_j [Mp], log keys / weights, then slot-0 contributions [Mp],
    // w_j, then slot-1 contributions [Mp], dA [Mp]
    const size_t per_warp = (size_t)2 * Npad + 4 * (size_t)Mp;
    float *wbase = reinterpret_cast<float *>(smem + p.tab_bytes + p.k_bytes + 16) + wib * per_warp;
    int *X = reinterpret_cast<int *>(wbase);
    float *lam = wbase + Npad;
    float *aj = lam + Npad;
    float *lj = aj + Mp;
    float *ct = lj + Mp;
    float *dA = ct + Mp;

    if (!stage_tables(smem, p.rx, p.tab_bytes, s_k, p.k_rates, p.k_bytes, s_bar, s_ok, p.err)) {
        for (int j = threadIdx.x; j < M; j += blockDim.x) p.partial[(int64_t)blockIdx.x * M + j] = 0.0f;
        return;
    }
    for (int j = lane; j < Mp; j += 32) dA[j] = 0.0f;

    const int64_t n = p.n_traj;
    const int64_t i = (int64_t)blockIdx.x * W + wib;
    int st = -1;
    if (i < n) st = p.status[i];
    const bool active = st == SSA_TRAJ_OK || st == SSA_TRAJ_ABSORBED || st == SSA_TRAJ_STEP_CAP;
    if (active) warp_adj_body<READOUT>(p, s_rx, s_st, s_inc_ptr, s_inc, s_k, X, lam, aj, lj, ct, dA, i, st);
    __syncthreads();
    // fixed-order reduction over the block's warps
    float *base0 = reinterpret_cast<float *>(smem + p.tab_bytes + p.k_bytes + 16);
    const int nb = (M + 4) >> 2;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        float acc = 0.0f;
        for (int w = 0; w < W; ++w) acc += base0[w * per_warp + 2 * Npad + 3 * Mp + jpos(j, nb)];
        p.partial[(int64_t)blockIdx.x * M + j] = acc;
    }
}

// ---------------------------------------------------------------------------------------------
template <int R, bool REC>
static cudaError_t launch_fwd_w(const FwdParams &p, int warps, size_t smem, cudaStream_t st)
{
    auto kern = fwd_warp_kernel<R, REC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (p.n_traj + warps - 1) / warps;
    kern<<<(unsigned)grid, warps * 32, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_forward_warp(const FwdParams &p, int readout, bool record, int warps, size_t smem, cudaStream_t st)
{
    if (p.n_traj == 0) return cudaSuccess;
    if (readout == SSA_READOUT_HOLD)
        return record ? launch_fwd_w<0, true>(p, warps, smem, st) : launch_fwd_w<0, false>(p, warps, smem, st);
    if (readout == SSA_READOUT_BIN)
        return record ? launch_fwd_w<2, true>(p, warps, smem, st) : launch_fwd_w<2, false>(p, warps, smem, st);
    return record ? launch_fwd_w<1, true>(p, warps, smem, st) : launch_fwd_w<1, false>(p, warps, smem, st);
}

template <int R, bool REC>
static cudaError_t launch_fwd_soft_w(const FwdParams &p, int warps, size_t smem, cudaStream_t st)
{
    auto kern = fwd_warp_soft_kernel<R, REC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (p.n_traj + warps - 1) / warps;
    kern<<<(unsigned)grid, warps * 32, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_forward_warp_soft(const FwdParams &p, int readout, bool record, int warps, size_t smem,
                                     cudaStream_t st)
{
    if (p.n_traj == 0) return cudaSuccess;
    if (readout == SSA_READOUT_HOLD)
        return record ? launch_fwd_soft_w<0, true>(p, warps, smem, st) : launch_fwd_soft_w<0, false>(p, warps, smem, st);
    if (readout == SSA_READOUT_BIN)
        return record ? launch_fwd_soft_w<2, true>(p, warps, smem, st) : launch_fwd_soft_w<2, false>(p, warps, smem, st);
    return record ? launch_fwd_soft_w<1, true>(p, warps, smem, st) : launch_fwd_soft_w<1, false>(p, warps, smem, st);
}

template <int R>
static cudaError_t launch_adj_soft_w(const AdjParams &p, const int *upd, uint32_t upd_words, int warps, size_t smem,
                                     int64_t grid, cudaStream_t st)
{
    auto kern = adj_warp_soft_kernel<R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, warps * 32, smem, st>>>(p, upd, upd_words);
    return cudaGetLastError();
}

cudaError_t launch_backward_warp_soft(const AdjParams &p, const int *upd, uint32_t upd_words, int readout, int warps,
                                      size_t smem, int64_t grid, cudaStream_t st)
{
    if (grid == 0) return cudaSuccess;
    if (readout == SSA_READOUT_HOLD) return launch_adj_soft_w<0>(p, upd, upd_words, warps, smem, grid, st);
    if (readout == SSA_READOUT_BIN) return launch_adj_soft_w<2>(p, upd, upd_words, warps, smem, grid, st);
    return launch_adj_soft_w<1>(p, upd, upd_words, warps, smem, grid, st);
}

template <int R>
static cudaError_t launch_adj_w(const AdjParams &p, int warps, size_t smem, int64_t grid, cudaStream_t st)
{
    auto kern = adj_warp_kernel<R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, warps * 32, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_backward_warp(const AdjParams &p, int readout, int warps, size_t smem, int64_t grid,
                                 cudaStream_t st)
{
    if (grid == 0) return cudaSuccess;
    switch (readout) {
    case SSA_READOUT_HOLD: return launch_adj_w<0>(p, warps, smem, grid, st);
    case SSA_READOUT_LINEAR: return launch_adj_w<1>(p, warps, smem, grid, st);
    default: return launch_adj_w<2>(p, warps, smem, grid, st);
    }
}

}  // namespace ssa
