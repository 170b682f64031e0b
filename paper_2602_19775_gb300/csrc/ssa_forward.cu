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
#include <cstdint>

#include "ssa_internal.cuh"

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
    const int N = p.N, M = p.M;
    int4 *s_rx = reinterpret_cast<int4 *>(smem);
    int *s_st = reinterpret_cast<int *>(smem + 16 * p.Mp);
    float *s_k = reinterpret_cast<float *>(smem + p.tab_bytes);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + p.tab_bytes + p.k_bytes);
    int *s_ok = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 8);
    int *s_X = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 16);

    if (!stage_tables(smem, p.rx, p.tab_bytes, s_k, p.k_rates, p.k_bytes, s_bar, s_ok, p.err)) return;

    const int64_t i = (int64_t)blockIdx.x * B + tid;
    if (i >= p.n_traj) return;
    const int64_t n = p.n_traj;
    int *X = s_X + tid;  // X[s * B]

    const int *x0 = p.x0 + (p.x0_per_traj ? i * N : 0);
    const bool bad_obs = (*p.flag & kErrBadObs) != 0;
    bool bad_input = (*p.flag & (kErrBadSamples | kErrBadObs)) != 0;
    for (int s = 0; s < N; ++s) {
        const int v = x0[s];
        X[s * B] = v;
        bad_input |= v < 0;
    }
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32);
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);

    double t = 0.0;
    int s = 0;
    // next clock threshold: the next sample time, or t_end once every sample is written
    double thr = p.S > 0 ? p.ts[0] : p.t_end;
    int status = bad_input ? SSA_TRAJ_BAD_INPUT : SSA_TRAJ_OK;
    int k = 0;        // index of the current state X_k
    int draws = 0;
    int ck_left = p.K, ck_row = 0;
    uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0;  // event pack (8 x uint16)
    int n_ev = 0;
    const uint16_t *ev_in = nullptr;
    if (REPLAY) {
        ev_in = p.ev_in + i * p.ev_in_stride;
        n_ev = (int)min((int64_t)p.n_ev_in[i], p.ev_in_stride);  // never read past the caller's row
    }
    constexpr int NQ = MC > 0 ? MC + 1 : 1;
    float E[NQ], En[NQ];
    if (MC > 0) step_noise<NQ>(E, 0u, c2, c3, key0, key1);

    while (!bad_input) {
        if (k >= p.max_steps) { status = SSA_TRAJ_STEP_CAP; break; }
        float a0 = 0.0f, ab = 0.0f, Eb = 1.0f, E0;
        int jb = -1;
        if constexpr (MC > 0) {
            step_noise<NQ>(En, (uint32_t)(k + 1), c2, c3, key0, key1);  // next step, state-independent
            E0 = E[0];
#pragma unroll
            for (int j = 0; j < MC; ++j) {
                const float a = __fmul_rn(s_k[j], mass_action_h(s_rx[j], X, B));
                a0 = __fadd_rn(a0, a);
                if (!REPLAY) race(a, E[j + 1], j, ab, Eb, jb);
            }
        } else {
            uint4 cache;
            int cb = -1;
            E0 = exp_variate((uint32_t)k, 0, c2, c3, key0, key1, cache, cb);
            for (int j = 0; j < M; ++j) {
                const float a = __fmul_rn(s_k[j], mass_action_h(s_rx[j], X, B));
                a0 = __fadd_rn(a0, a);
                if (!REPLAY && a > 0.0f) race(a, exp_variate((uint32_t)k, j + 1, c2, c3, key0, key1, cache, cb), j, ab, Eb, jb);
            }
        }
        if (!(a0 < CUDART_INF_F)) { status = SSA_TRAJ_BAD_RATE; break; }
        if (a0 == 0.0f) { status = SSA_TRAJ_ABSORBED; break; }
        if (REPLAY) {
            if (k >= n_ev) { status = SSA_TRAJ_REPLAY_MISMATCH; break; }
            jb = ev_in[k];
            if (jb >= M || !(__fmul_rn(s_k[jb], mass_action_h(s_rx[jb], X, B)) > 0.0f)) {
                status = SSA_TRAJ_REPLAY_MISMATCH;
                break;
            }
        }
        if (jb < 0) { status = SSA_TRAJ_BAD_RATE; break; }  // no positive key (NaN rates)
        const float tau = __fdividef(E0, a0);
        const double t_next = t + f2d_pos(tau);
        const int4 rj = s_rx[jb];
        // a sample falls in [t_k, t_{k+1}) or the horizon ends (both clocks are non-negative)
        const bool slow = gt_nonneg(t_next, thr);
        const bool cross = slow && gt_nonneg(t_next, p.t_end);
        if (!cross) {
            // range check of X + v_j before anything is written for this draw
            for (int e = rj.z; e < rj.w; ++e) {
                const int st = s_st[e];
                const int x = X[stoich_species(st) * B], d = stoich_delta(st);
                if (d < 0 && x + d < 0) status = SSA_TRAJ_NEG_COUNT;
                else if (d > 0 && x > 2147483647 - d) status = SSA_TRAJ_OVERFLOW;
            }
        }
        if (RECORD) {
            e0 = __funnelshift_r(e0, e1, 16);
            e1 = __funnelshift_r(e1, e2, 16);
            e2 = __funnelshift_r(e2, e3, 16);
            e3 = (e3 >> 16) | ((uint32_t)jb << 16);
            if ((k & 7) == 7) p.ev[(int64_t)(k >> 3) * n + i] = make_uint4(e0, e1, e2, e3);
        }
        draws = k + 1;
        if (status != SSA_TRAJ_OK) break;  // rejected update: samples hold X_k below
        if (slow) {
            // samples with t_k <= t_s < t_{k+1}
            while (s < p.S && gt_nonneg(t_next, p.ts[s])) {
                if (READOUT == SSA_READOUT_HOLD) {
                    int *o = static_cast<int *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                    for (int c = 0; c < p.n_obs; ++c) o[c] = X[p.obs_sp[c] * B];
                } else {
                    const float alpha = __fdiv_rn(d2f_nonneg(p.ts[s] - t), tau);
                    float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                    for (int c = 0; c < p.n_obs; ++c) {
                        const int sp = p.obs_sp[c];
                        int dv = 0;
                        for (int e = rj.z; e < rj.w; ++e)
                            if (stoich_species(s_st[e]) == sp) dv += stoich_delta(s_st[e]);
                        o[c] = __fmaf_rn(alpha, (float)dv, (float)X[sp * B]);
                    }
                    if (RECORD) p.brk_a[(int64_t)s * n + i] = alpha;
                }
                if (RECORD) p.brk_k[(int64_t)s * n + i] = k;
                ++s;
            }
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;  // the crossing draw is made but not applied
        }
        for (int e = rj.z; e < rj.w; ++e) {
            const int st = s_st[e];
            X[stoich_species(st) * B] += stoich_delta(st);
        }
        t = t_next;
        ++k;
        if (RECORD && --ck_left == 0) {
            ck_left = p.K;
            ++ck_row;
            int *ck = p.ckpt + (int64_t)ck_row * N * n + i;
            for (int sp = 0; sp < N; ++sp) ck[(int64_t)sp * n] = X[sp * B];
        }
        if constexpr (MC > 0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) E[q] = En[q];
        }
    }
    if (REPLAY && status == SSA_TRAJ_OK && draws != n_ev) status = SSA_TRAJ_REPLAY_MISMATCH;
    // samples after the last state hold it (absorbed, capped, rejected or bad input)
    for (; s < p.S; ++s) {
        if (READOUT == SSA_READOUT_HOLD) {
            int *o = static_cast<int *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
            for (int c = 0; c < p.n_obs; ++c) o[c] = bad_obs ? 0 : X[p.obs_sp[c] * B];
        } else {
            float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
            for (int c = 0; c < p.n_obs; ++c) o[c] = bad_obs ? 0.0f : (float)X[p.obs_sp[c] * B];
            if (RECORD) p.brk_a[(int64_t)s * n + i] = -1.0f;
        }
        if (RECORD) p.brk_k[(int64_t)s * n + i] = k;
    }
    p.draws[i] = draws;
    p.status[i] = status;
    if (RECORD) {
        if (draws & 7) {
            for (int pad = draws & 7; pad < 8; ++pad) {
                e0 = __funnelshift_r(e0, e1, 16);
                e1 = __funnelshift_r(e1, e2, 16);
                e2 = __funnelshift_r(e2, e3, 16);
                e3 = e3 >> 16;
            }
            p.ev[(int64_t)((draws - 1) >> 3) * n + i] = make_uint4(e0, e1, e2, e3);
        }
        for (int sp = 0; sp < N; ++sp) {
            p.xfinal[(int64_t)sp * n + i] = X[sp * B];
            p.ckpt[(int64_t)sp * n + i] = x0[sp];  // checkpoint 0 = X_0
        }
    }
}

// Validate the per-call inputs once: sample times ascending within [0, t_end], observed species
// within [0, N). A failure marks every trajectory SSA_TRAJ_BAD_INPUT.
__global__ void validate_inputs_kernel(const double *ts, int S, double t_end, const int *obs_sp, int n_obs, int N,
                                       int *flag)
{
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const bool ok = ts[s] >= 0.0 && ts[s] <= t_end && (s == 0 || ts[s] >= ts[s - 1]);
        if (!ok) atomicOr(flag, kErrBadSamples);
    }
    for (int c = threadIdx.x; c < n_obs; c += blockDim.x)
        if (obs_sp[c] < 0 || obs_sp[c] >= N) atomicOr(flag, kErrBadObs);
}

// k_j = exp(theta_{r(j)}) rounded once to binary32 (computed in binary64).
__global__ void rates_kernel(const float *log_rates, const int *rate_index, int M, int M_pad, float *k_out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M_pad; j += gridDim.x * blockDim.x)
        k_out[j] = j < M ? (float)exp((double)log_rates[rate_index[j]]) : 0.0f;
}

// Deterministic ensemble mean: per-chunk column sums (fixed order), then a fixed-order sum.
template <typename T>
__global__ void colsum_chunks_kernel(const T *obs, int64_t n_traj, int64_t row_len, int64_t chunk, float *partial)
{
    const int64_t t0 = (int64_t)blockIdx.y * chunk;
    const int64_t t1 = min(n_traj, t0 + chunk);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < row_len; c += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int64_t t = t0; t < t1; ++t) acc += (float)obs[t * row_len + c];
        partial[(int64_t)blockIdx.y * row_len + c] = acc;
    }
}

__global__ void colsum_final_kernel(const float *partial, int64_t n_chunks, int64_t row_len, float inv_n, float *out)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < row_len; c += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int64_t b = 0; b < n_chunks; ++b) acc += partial[b * row_len + c];
        out[c] = acc * inv_n;
    }
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

// Test hook: brackets [S][n] -> [n][S].
__global__ void transpose_brackets_kernel(const int *brk, int64_t n_traj, int S, int *out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_traj * S) return;
    const int64_t i = idx / S;
    const int s = (int)(idx % S);
    out[idx] = brk[(int64_t)s * n_traj + i];
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
        return readout == SSA_READOUT_HOLD ? launch_fwd_t<0, true, true, 0>(p, block, smem, st)
                                           : launch_fwd_t<1, true, true, 0>(p, block, smem, st);
    }
    const int mc = thread_kernel_mc(p.M);
    if (readout == SSA_READOUT_HOLD)
        return record ? launch_fwd_mc<0, true>(p, mc, block, smem, st) : launch_fwd_mc<0, false>(p, mc, block, smem, st);
    return record ? launch_fwd_mc<1, true>(p, mc, block, smem, st) : launch_fwd_mc<1, false>(p, mc, block, smem, st);
}

cudaError_t launch_validate_inputs(const double *ts, int S, double t_end, const int *obs_sp, int n_obs, int N, int *flag,
                                  cudaStream_t st)
{
    if (S > 0 || n_obs > 0) validate_inputs_kernel<<<1, 256, 0, st>>>(ts, S, t_end, obs_sp, n_obs, N, flag);
    return cudaGetLastError();
}

cudaError_t launch_rates(const float *log_rates, const int *rate_index, int M, int M_pad, float *k_out, cudaStream_t st)
{
    rates_kernel<<<(M_pad + 255) / 256, 256, 0, st>>>(log_rates, rate_index, M, M_pad, k_out);
    return cudaGetLastError();
}

cudaError_t launch_ensemble_mean(const void *obs, bool is_int, int64_t n_traj, int64_t row_len, float *partial,
                                 int64_t chunk, float *out, cudaStream_t st)
{
    if (row_len == 0) return cudaSuccess;
    const int64_t n_chunks = (n_traj + chunk - 1) / chunk;
    const float inv_n = n_traj > 0 ? 1.0f / (float)n_traj : 0.0f;
    if (n_chunks > 0) {
        dim3 g((unsigned)((row_len + 127) / 128), (unsigned)n_chunks);
        if (is_int) colsum_chunks_kernel<int><<<g, 128, 0, st>>>(static_cast<const int *>(obs), n_traj, row_len, chunk, partial);
        else colsum_chunks_kernel<float><<<g, 128, 0, st>>>(static_cast<const float *>(obs), n_traj, row_len, chunk, partial);
    }
    colsum_final_kernel<<<(unsigned)((row_len + 127) / 128), 128, 0, st>>>(partial, n_chunks, row_len, inv_n, out);
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

cudaError_t launch_transpose_brackets(const int *brk, int64_t n_traj, int S, int *out, cudaStream_t st)
{
    const int64_t total = n_traj * S;
    if (total == 0) return cudaSuccess;
    transpose_brackets_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(brk, n_traj, S, out);
    return cudaGetLastError();
}

cudaError_t launch_status_count(const int *status, int64_t n, unsigned long long *counts, cudaStream_t st)
{
    status_count_kernel<<<152, 256, 0, st>>>(status, n, counts);
    return cudaGetLastError();
}

}  // namespace ssa
