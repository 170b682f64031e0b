// ssa_forward.cu -- forward kernels: exact direct-method SSA with the Gumbel-max choice.
//
// One thread simulates one trajectory (arXiv 2602.19775, Section 2 and Section 3.2):
//   a_j = k_j h_j(X)            mass-action propensity, binary32, h formed exactly in int64
//   a0  = sum_j a_j             fixed order j = 0..M-1
//   tau = E_0 / a0, E_0 = -ln u_0                      (inverse transform, Section 2)
//   j*  = argmax_j a_j / E_j,  E_j = -ln u_{1+j}       (= argmax log a_j + G_j, G_j = -ln E_j)
//   t  += (double) tau                                  (FP64 clock)
//   X  += v_{j*}                                        (Eq. 6, exact int32, range-checked)
// Counts live in shared memory as [species][thread] (bank-conflict free); the network tables are
// staged into shared memory by one bulk TMA copy per block. With `record`, each draw's reaction
// index is packed 8-per-uint4 into an event log laid out [step/8][trajectory] (coalesced: the
// threads of a warp advance their step counters together), the state is checkpointed every K
// steps, and each sample records its bracketing step and interpolation weight.
#include <algorithm>
#include <cstdint>

#include "ssa_fwd_body.cuh"

namespace ssa {

// Thread-per-trajectory forward. MC > 0: the network has at most MC reactions (tables padded with
// zero-rate, order-0 entries), per-reaction loops are unrolled and the step's variates live in
// registers. MC == 0: runtime loops for any size.
template <int READOUT, bool RECORD, bool REPLAY, int MC>
__global__ void __launch_bounds__(256) fwd_thread_kernel(const FwdParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    int4 *s_rx = reinterpret_cast<int4 *>(smem);
    int *s_st = reinterpret_cast<int *>(smem + 16 * p.Mp);
    float *s_k = reinterpret_cast<float *>(smem + p.tab_bytes);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + p.tab_bytes + p.k_bytes);
    int *s_ok = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 8);
    int *s_X = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 16);

    if (!stage_tables(smem, p.rx, p.tab_bytes, s_k, p.k_rates, p.k_bytes, s_bar, s_ok, p.err)) return;

    const int64_t i = (int64_t)blockIdx.x * B + tid;
    if (i >= p.n_traj) return;
    thread_fwd_body<READOUT, RECORD, REPLAY, MC>(p, s_rx, s_st, s_k, s_X + tid, B, i);
}

// Validate the per-call inputs once: sample times ascending within [0, t_end] (strictly, from above 0,
// for the bin readout, whose bins (t_{s-1}, t_s] must not be empty), observed species within [0, N).
// A failure marks every trajectory SSA_TRAJ_BAD_INPUT.
__global__ void validate_inputs_kernel(const double *ts, int S, double t_end, const int *obs_sp, int n_obs, int N,
                                       int strict, int *flag)
{
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double lo = s > 0 ? ts[s - 1] : 0.0;
        const bool ok = ts[s] >= 0.0 && ts[s] <= t_end && (s == 0 || ts[s] >= ts[s - 1]) && (!strict || ts[s] > lo);
        if (!ok) atomicOr(flag, kErrBadSamples);
    }
    for (int c = threadIdx.x; c < n_obs; c += blockDim.x)
        if (obs_sp[c] < 0 || obs_sp[c] >= N) atomicOr(flag, kErrBadObs);
}

// k_j = exp(theta_{r(j)}) rounded once to binary32 (computed in binary64); lane_major stores reaction j
// at jpos(j) for the warp kernels (position q nb + b holds reaction 4 b + q - 1).
__global__ void rates_kernel(const float *log_rates, const int *rate_index, int M, int M_pad, int lane_major,
                             float *k_out)
{
    const int nb = (M + 4) >> 2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M_pad; e += gridDim.x * blockDim.x) {
        const int j = !lane_major ? e : (e < 4 * nb ? 4 * (e % nb) + e / nb - 1 : -1);
        k_out[e] = (j >= 0 && j < M) ? (float)exp((double)log_rates[rate_index[j]]) : 0.0f;
    }
}

// Deterministic ensemble mean: per-chunk column sums (fixed order), then a fixed-order sum.
// Deterministic ensemble mean in two passes, both over tiles of 64 columns with 4 row groups per block
// (256 threads): a warp reads 32 consecutive columns of one row (coalesced), each thread sums every 4th row
// of its group, and the 4 group sums are added in a fixed order.
// Pass 1: chunk b (rows b*chunk .. b*chunk + chunk - 1) -> partial[b][c]; the chunks are strided over
// gridDim.y, so any number of chunks fits the 65,535 limit; each chunk's sum is the same whatever the grid.
constexpr int kColTile = 64, kColGroups = 4;
template <typename T>
__global__ void __launch_bounds__(kColTile * kColGroups) colsum_chunks_kernel(const T *obs, int64_t n_traj,
                                                                              int64_t row_len, int64_t chunk,
                                                                              float *partial)
{
    __shared__ float part[kColGroups][kColTile];
    const int g = threadIdx.x / kColTile, cl = threadIdx.x % kColTile;
    const int64_t n_chunks = (n_traj + chunk - 1) / chunk;
    for (int64_t ct = blockIdx.x; ct * kColTile < row_len; ct += gridDim.x) {
        const int64_t c = ct * kColTile + cl;
        for (int64_t b = blockIdx.y; b < n_chunks; b += gridDim.y) {
            const int64_t t0 = b * chunk;
            const int64_t t1 = min(n_traj, t0 + chunk);
            float acc = 0.0f;
            if (c < row_len)
                for (int64_t t = t0 + g; t < t1; t += kColGroups) acc += (float)obs[t * row_len + c];
            part[g][cl] = acc;
            __syncthreads();
            if (g == 0 && c < row_len)
                partial[b * row_len + c] = ((part[0][cl] + part[1][cl]) + part[2][cl]) + part[3][cl];
            __syncthreads();
        }
    }
}

// Pass 2: out[c] = (sum over chunks of partial[b][c]) inv_n, the chunks split over the 4 row groups.
__global__ void __launch_bounds__(kColTile * kColGroups) colsum_final_kernel(const float *partial, int64_t n_chunks,
                                                                             int64_t row_len, float inv_n, float *out)
{
    __shared__ float part[kColGroups][kColTile];
    const int g = threadIdx.x / kColTile, cl = threadIdx.x % kColTile;
    for (int64_t ct = blockIdx.x; ct * kColTile < row_len; ct += gridDim.x) {
        const int64_t c = ct * kColTile + cl;
        float acc = 0.0f;
        if (c < row_len)
            for (int64_t b = g; b < n_chunks; b += kColGroups) acc += partial[b * row_len + c];
        part[g][cl] = acc;
        __syncthreads();
        if (g == 0 && c < row_len) out[c] = (((part[0][cl] + part[1][cl]) + part[2][cl]) + part[3][cl]) * inv_n;
        __syncthreads();
    }
}

// Test hook: the exponential variates -ln u of given Philox words.
__global__ void exp_variates_kernel(const uint32_t *words, int64_t n, float *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = neg_log_unit(u01(words[i]));
}

// Test hook: uniforms of arbitrary (trajectory, step) pairs.
__global__ void philox_uniforms_kernel(uint64_t seed, const uint64_t *traj, const uint64_t *step, int64_t n,
                                       int n_words, float *out)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint64_t g = traj[r];
    for (int b = 0; 4 * b < n_words; ++b) {
        const uint4 x = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)step[r], (uint32_t)g, (uint32_t)(g >> 32)),
                                      (uint32_t)seed, (uint32_t)(seed >> 32));
        for (int q = 0; q < 4 && 4 * b + q < n_words; ++q) out[r * n_words + 4 * b + q] = u01(word_of(x, q));
    }
}

// Test hook: unpack the event log.
__global__ void unpack_events_kernel(const uint4 *ev, const int *draws, int64_t n_traj, int64_t stride, int *out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_traj * stride) return;
    const int64_t i = idx / stride, k = idx % stride;
    int v = -1;
    if (k < draws[i]) {
        const uint4 row = ev[(k >> 3) * n_traj + i];
        const int slot = (int)(k & 7);
        const uint32_t w = word_of(row, slot >> 1);
        v = (slot & 1) ? (int)(w >> 16) : (int)(w & 0xffff);
    }
    out[idx] = v;
}

// Bin readout with a shared upstream gradient: its binary64 prefix sums over bins (bin_prefix_block)
__global__ void __launch_bounds__(kPrefixThreads) bin_prefix_kernel(const float *g, int S, int n_obs, double *prefix)
{
    bin_prefix_block(g, S, n_obs, prefix);
}

// Test hook: brackets [S][n] -> [n][S].
__global__ void transpose_brackets_kernel(const int *brk, int64_t n_traj, int S, int *out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_traj * S) return;
    const int64_t i = idx / S;
    const int s = (int)(idx % S);
    out[idx] = brk[(int64_t)s * n_traj + i];
}

// Test hook, bin readout: the per-edge brackets from the slots (slot q of trajectory i: state brk[q],
// edges from first[q] up to the next slot's first edge; nslots[i] slots).
__global__ void bin_brackets_kernel(const int *brk, const int *first, const int *nslots, int64_t n_traj, int S, int *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_traj) return;
    const int nq = min(nslots[i], S);
    for (int q = 0; q < nq; ++q) {
        const int lo = max(first[(int64_t)q * n_traj + i], 0);
        const int hi = q + 1 < nq ? min(first[(int64_t)(q + 1) * n_traj + i], S) : S;
        for (int s = lo; s < hi; ++s) out[i * S + s] = brk[(int64_t)q * n_traj + i];
    }
}

// Status histogram for ssa_run_status.
__global__ void status_count_kernel(const int *status, int64_t n, unsigned long long *counts)
{
    __shared__ unsigned long long c[SSA_TRAJ_N_CODES];
    if (threadIdx.x < SSA_TRAJ_N_CODES) c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = status[i];
        if (s >= 0 && s < SSA_TRAJ_N_CODES) atomicAdd(&c[s], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < SSA_TRAJ_N_CODES) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
}

// ---------------------------------------------------------------------------------------------
// Launch helpers used by the API layer
// ---------------------------------------------------------------------------------------------
template <int R, bool REC, bool REP, int MC>
static cudaError_t launch_fwd_t(const FwdParams &p, int block, size_t smem, cudaStream_t st)
{
    auto kern = fwd_thread_kernel<R, REC, REP, MC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (p.n_traj + block - 1) / block;
    kern<<<(unsigned)grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

// compile-time reaction bound used for a network of M reactions (0 = runtime loops)
int thread_kernel_mc(int M) { return M <= 2 ? 2 : M <= 4 ? 4 : M <= 8 ? 8 : M <= 16 ? 16 : 0; }

template <int R, bool REC>
static cudaError_t launch_fwd_mc(const FwdParams &p, int mc, int block, size_t smem, cudaStream_t st)
{
    switch (mc) {
    case 2: return launch_fwd_t<R, REC, false, 2>(p, block, smem, st);
    case 4: return launch_fwd_t<R, REC, false, 4>(p, block, smem, st);
    case 8: return launch_fwd_t<R, REC, false, 8>(p, block, smem, st);
    case 16: return launch_fwd_t<R, REC, false, 16>(p, block, smem, st);
    default: return launch_fwd_t<R, REC, false, 0>(p, block, smem, st);
    }
}

cudaError_t launch_forward_thread(const FwdParams &p, int readout, bool record, bool replay, int block,
                                  size_t smem, cudaStream_t st)
{
    if (p.n_traj == 0) return cudaSuccess;
    if (replay) {  // test hook: runtime loops, always recorded
        switch (readout) {
        case SSA_READOUT_HOLD: return launch_fwd_t<SSA_READOUT_HOLD, true, true, 0>(p, block, smem, st);
        case SSA_READOUT_LINEAR: return launch_fwd_t<SSA_READOUT_LINEAR, true, true, 0>(p, block, smem, st);
        default: return launch_fwd_t<SSA_READOUT_BIN, true, true, 0>(p, block, smem, st);
        }
    }
    const int mc = thread_kernel_mc(p.M);
    switch (readout) {
    case SSA_READOUT_HOLD:
        return record ? launch_fwd_mc<SSA_READOUT_HOLD, true>(p, mc, block, smem, st)
                      : launch_fwd_mc<SSA_READOUT_HOLD, false>(p, mc, block, smem, st);
    case SSA_READOUT_LINEAR:
        return record ? launch_fwd_mc<SSA_READOUT_LINEAR, true>(p, mc, block, smem, st)
                      : launch_fwd_mc<SSA_READOUT_LINEAR, false>(p, mc, block, smem, st);
    default:
        return record ? launch_fwd_mc<SSA_READOUT_BIN, true>(p, mc, block, smem, st)
                      : launch_fwd_mc<SSA_READOUT_BIN, false>(p, mc, block, smem, st);
    }
}

cudaError_t launch_validate_inputs(const double *ts, int S, double t_end, const int *obs_sp, int n_obs, int N,
                                  int strict, int *flag, cudaStream_t st)
{
    if (S > 0 || n_obs > 0) validate_inputs_kernel<<<1, 256, 0, st>>>(ts, S, t_end, obs_sp, n_obs, N, strict, flag);
    return cudaGetLastError();
}

cudaError_t launch_rates(const float *log_rates, const int *rate_index, int M, int M_pad, int lane_major, float *k_out,
                         cudaStream_t st)
{
    rates_kernel<<<(M_pad + 255) / 256, 256, 0, st>>>(log_rates, rate_index, M, M_pad, lane_major, k_out);
    return cudaGetLastError();
}

cudaError_t launch_ensemble_mean(const void *obs, bool is_int, int64_t n_traj, int64_t row_len, float *partial,
                                 int64_t chunk, float *out, cudaStream_t st)
{
    if (row_len == 0) return cudaSuccess;
    const int64_t n_chunks = (n_traj + chunk - 1) / chunk;
    const float inv_n = n_traj > 0 ? 1.0f / (float)n_traj : 0.0f;
    const unsigned tiles = (unsigned)std::min<int64_t>((row_len + kColTile - 1) / kColTile, 65535);
    if (n_chunks > 0) {
        dim3 g(tiles, (unsigned)std::min<int64_t>(n_chunks, 65535));
        if (is_int)
            colsum_chunks_kernel<int><<<g, kColTile * kColGroups, 0, st>>>(static_cast<const int *>(obs), n_traj, row_len,
                                                                           chunk, partial);
        else
            colsum_chunks_kernel<float><<<g, kColTile * kColGroups, 0, st>>>(static_cast<const float *>(obs), n_traj,
                                                                             row_len, chunk, partial);
    }
    colsum_final_kernel<<<tiles, kColTile * kColGroups, 0, st>>>(partial, n_chunks, row_len, inv_n, out);
    return cudaGetLastError();
}

// out[c] = sum over rows of x[row][c], in fixed chunks of rows and then over chunks (deterministic)
cudaError_t launch_column_sums(const float *x, int64_t n_rows, int64_t row_len, float *partial, int64_t chunk, float *out,
                               cudaStream_t st)
{
    if (row_len == 0) return cudaSuccess;
    const int64_t n_chunks = (n_rows + chunk - 1) / chunk;
    const unsigned tiles = (unsigned)std::min<int64_t>((row_len + kColTile - 1) / kColTile, 65535);
    if (n_chunks > 0) {
        dim3 g(tiles, (unsigned)std::min<int64_t>(n_chunks, 65535));
        colsum_chunks_kernel<float><<<g, kColTile * kColGroups, 0, st>>>(x, n_rows, row_len, chunk, partial);
    }
    colsum_final_kernel<<<tiles, kColTile * kColGroups, 0, st>>>(partial, n_chunks, row_len, 1.0f, out);
    return cudaGetLastError();
}

cudaError_t launch_exp_variates(const uint32_t *words, int64_t n, float *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    exp_variates_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(words, n, out);
    return cudaGetLastError();
}

cudaError_t launch_philox_uniforms(uint64_t seed, const uint64_t *traj, const uint64_t *step, int64_t n, int n_words,
                                   float *out, cudaStream_t st)
{
    if (n == 0 || n_words == 0) return cudaSuccess;
    philox_uniforms_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(seed, traj, step, n, n_words, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack_events(const uint4 *ev, const int *draws, int64_t n_traj, int64_t stride, int *out,
                                 cudaStream_t st)
{
    const int64_t total = n_traj * stride;
    if (total == 0) return cudaSuccess;
    unpack_events_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(ev, draws, n_traj, stride, out);
    return cudaGetLastError();
}

cudaError_t launch_transpose_brackets(const int *brk, int64_t n_traj, int S, const int *first, const int *nslots,
                                      int *out, cudaStream_t st)
{
    const int64_t total = n_traj * S;
    if (total == 0) return cudaSuccess;
    if (first)
        bin_brackets_kernel<<<(unsigned)((n_traj + 255) / 256), 256, 0, st>>>(brk, first, nslots, n_traj, S, out);
    else
        transpose_brackets_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(brk, n_traj, S, out);
    return cudaGetLastError();
}

cudaError_t launch_bin_prefix(const float *g, int S, int n_obs, double *prefix, cudaStream_t st)
{
    bin_prefix_kernel<<<1, kPrefixThreads, 0, st>>>(g, S, n_obs, prefix);
    return cudaGetLastError();
}

cudaError_t launch_status_count(const int *status, int64_t n, unsigned long long *counts, cudaStream_t st)
{
    status_count_kernel<<<152, 256, 0, st>>>(status, n, counts);
    return cudaGetLastError();
}

}  // namespace ssa
