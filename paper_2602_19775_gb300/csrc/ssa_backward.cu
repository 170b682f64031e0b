// ssa_backward.cu -- straight-through adjoint kernels (arXiv 2602.19775, Eqs. 3, 5, 7; the
// reparametrised waiting time of Section 3.1; the adjoint recursion in the Figure 1 caption).
//
// One thread walks one recorded trajectory backwards. The state is reconstructed exactly from
// the final counts and the event log (X_k = X_{k+1} - v_{j_k}; integers are reversible) and is
// verified against the forward's checkpoints every K steps. At every step the thread regenerates
// the step's Philox words, recomputes the forward's propensities and keys bit for bit (the same
// binary32 operations; the recomputed Gumbel-max choice is checked against the logged one), and
// applies the adjoint of the surrogate graph
//     X_{k+1} = X_k + sum_j y~_j v_j,  y~ = softmax((log a_j + G_j)/T),
//     tau_k = E_0/a0,  t_{k+1} = t_k + tau_k,
// with lambda = dL/dX_{k+1} and mu = dL/dt_{k+1}:
//     w_j = v_j . lambda,  g_j = y~_j (w_j - sum_i y~_i w_i),  psi_j = g_j / T  (a_j > 0 only)
//     dL/da0 = -(mu + dL/dtau_k|readout) tau_k / a0
//     dL/dlog k_{r(j)} += psi_j + dL/da0 a_j
//     dL/dX_k = lambda + sum_j psi_j dlog a_j/dX + dL/da0 sum_j da_j/dX + (readout terms)
// The softmax is formed as y~_j ~ exp2((log2 r_j - log2 r_max)/T) with r_j = a_j/E_j.
// Per-reaction sums dL/dlog a_j are kept per thread in shared memory, reduced over the block in
// a fixed order, then over blocks in a fixed order, and mapped to parameters (deterministic).
#include <cstdint>

#include "ssa_adj_body.cuh"

namespace ssa {

template <int READOUT, int MC>
__global__ void __launch_bounds__(256) adj_thread_kernel(const AdjParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int N = p.N, M = p.M;
    int4 *s_rx = reinterpret_cast<int4 *>(smem);
    int *s_st = reinterpret_cast<int *>(smem + 16 * p.Mp);
    float *s_k = reinterpret_cast<float *>(smem + p.tab_bytes);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + p.tab_bytes + p.k_bytes);
    int *s_ok = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 8);
    unsigned char *dyn = smem + p.tab_bytes + p.k_bytes + 16;
    int *s_X = reinterpret_cast<int *>(dyn);
    float *s_lam = reinterpret_cast<float *>(dyn) + (size_t)N * B;
    float *s_dlam = s_lam + (size_t)N * B;
    float *s_dA = s_dlam + (size_t)N * B;  // [M][B]
    float *s_q = s_dA + (size_t)M * B;     // [M][B], runtime-size variant only

    if (!stage_tables(smem, p.rx, p.tab_bytes, s_k, p.k_rates, p.k_bytes, s_bar, s_ok, p.err)) {
        for (int j = tid; j < M; j += B) p.partial[(int64_t)blockIdx.x * M + j] = 0.0f;
        return;
    }

    const int64_t n = p.n_traj;
    const int64_t i = (int64_t)blockIdx.x * B + tid;
    int st = -1;
    if (i < n) st = p.status[i];
    const bool active = st == SSA_TRAJ_OK || st == SSA_TRAJ_ABSORBED || st == SSA_TRAJ_STEP_CAP;
    float dAr[MC > 0 ? MC : 1];
#pragma unroll
    for (int j = 0; j < (MC > 0 ? MC : 1); ++j) dAr[j] = 0.0f;
    if (MC == 0)
        for (int j = 0; j < M; ++j) s_dA[j * B + tid] = 0.0f;

    if (active)
        thread_adj_body<READOUT, MC>(p, s_rx, s_st, s_k, s_X + tid, s_lam + tid, s_dlam + tid, s_q + tid, s_dA + tid, B, i,
                                     st, dAr);
    if (MC > 0) {
#pragma unroll
        for (int j = 0; j < (MC > 0 ? MC : 1); ++j)
            if (j < M) s_dA[j * B + tid] = dAr[j];
    }
    __syncthreads();
    // fixed-order block reduction of the per-reaction adjoints
    const int warp = tid >> 5, lane = tid & 31, nwarps = B >> 5;
    for (int j = warp; j < M; j += nwarps) {
        float acc = 0.0f;
        for (int u = lane; u < B; u += 32) acc += s_dA[j * B + u];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) p.partial[(int64_t)blockIdx.x * M + j] = acc;
    }
}

// dA[j] = sum over blocks of partial[b][j]: one block per reaction, a fixed strided assignment of the
// partial rows to threads and a fixed shared-memory tree, so the result does not depend on timing.
__global__ void reduce_partials_kernel(const float *partial, int64_t nblk, int M, float *dA)
{
    __shared__ float red[256];
    const int j = blockIdx.x;
    float acc = 0.0f;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) acc += partial[b * M + j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) dA[j] = red[0];
}

// dtheta[r] = sum_{j: r(j) = r} dA[j], summed in increasing j.
__global__ void map_params_kernel(const float *dA, int M, const int *rate_index, int P, float *dtheta)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int j = 0; j < M; ++j)
            if (rate_index[j] == r) acc += dA[j];
        dtheta[r] = acc;
    }
}

// The wide-range adjoint's reductions: as above, in binary64 (values beyond the binary32 range).
__global__ void reduce_partials64_kernel(const double *partial, int64_t nblk, int M, double *dA)
{
    __shared__ double red[256];
    const int j = blockIdx.x;
    double acc = 0.0;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) acc += partial[b * M + j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) dA[j] = red[0];
}

__global__ void map_params64_kernel(const double *dA, int M, const int *rate_index, int P, double *dtheta)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < M; ++j)
            if (rate_index[j] == r) acc += dA[j];
        dtheta[r] = acc;
    }
}

template <int R, int MC>
static cudaError_t launch_adj_t(const AdjParams &p, int block, size_t smem, int64_t grid, cudaStream_t st)
{
    auto kern = adj_thread_kernel<R, MC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

int thread_kernel_mc(int M);

template <int R>
static cudaError_t launch_adj_mc(const AdjParams &p, int block, size_t smem, int64_t grid, cudaStream_t st)
{
    switch (thread_kernel_mc(p.M)) {
    case 2: return launch_adj_t<R, 2>(p, block, smem, grid, st);
    case 4: return launch_adj_t<R, 4>(p, block, smem, grid, st);
    case 8: return launch_adj_t<R, 8>(p, block, smem, grid, st);
    case 16: return launch_adj_t<R, 16>(p, block, smem, grid, st);
    default: return launch_adj_t<R, 0>(p, block, smem, grid, st);
    }
}

cudaError_t launch_backward_thread(const AdjParams &p, int readout, int block, size_t smem, int64_t grid,
                                   cudaStream_t st)
{
    if (grid == 0) return cudaSuccess;
    switch (readout) {
    case SSA_READOUT_HOLD: return launch_adj_mc<SSA_READOUT_HOLD>(p, block, smem, grid, st);
    case SSA_READOUT_LINEAR: return launch_adj_mc<SSA_READOUT_LINEAR>(p, block, smem, grid, st);
    default: return launch_adj_mc<SSA_READOUT_BIN>(p, block, smem, grid, st);
    }
}

cudaError_t launch_reduce_partials(const float *partial, int64_t nblk, int M, const int *rate_index, int P,
                                   float *dA_tmp, float *dtheta, cudaStream_t st)
{
    if (M > 0) reduce_partials_kernel<<<M, 256, 0, st>>>(partial, nblk, M, dA_tmp);
    if (P > 0) map_params_kernel<<<(P + 255) / 256, 256, 0, st>>>(dA_tmp, M, rate_index, P, dtheta);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials64(const double *partial, int64_t nblk, int M, const int *rate_index, int P,
                                     double *dA_tmp, double *dtheta, cudaStream_t st)
{
    if (M > 0) reduce_partials64_kernel<<<M, 256, 0, st>>>(partial, nblk, M, dA_tmp);
    if (P > 0) map_params64_kernel<<<(P + 255) / 256, 256, 0, st>>>(dA_tmp, M, rate_index, P, dtheta);
    return cudaGetLastError();
}

}  // namespace ssa
