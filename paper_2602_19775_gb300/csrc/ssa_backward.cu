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

#include "ssa_internal.cuh"

namespace ssa {

template <int READOUT>
__global__ void __launch_bounds__(256) adj_thread_kernel(const AdjParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int N = p.N, M = p.M;
    int4 *s_rx = reinterpret_cast<int4 *>(smem);
    int *s_st = reinterpret_cast<int *>(smem + 16 * M);
    float *s_k = reinterpret_cast<float *>(smem + p.tab_bytes);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + p.tab_bytes + p.k_bytes);
    int *s_ok = reinterpret_cast<int *>(smem + p.tab_bytes + p.k_bytes + 8);
    unsigned char *dyn = smem + p.tab_bytes + p.k_bytes + 16;
    int *s_X = reinterpret_cast<int *>(dyn);
    float *s_lam = reinterpret_cast<float *>(dyn) + (size_t)N * B;
    float *s_dlam = s_lam + (size_t)N * B;
    float *s_q = s_dlam + (size_t)N * B;
    float *s_dA = s_q + (size_t)M * B;

    if (!stage_tables(smem, p.rx, p.tab_bytes, s_k, p.k_rates, p.k_bytes, s_bar, s_ok, p.err)) {
        for (int j = tid; j < M; j += B) p.partial[(int64_t)blockIdx.x * M + j] = 0.0f;
        return;
    }
    for (int j = 0; j < M; ++j) s_dA[j * B + tid] = 0.0f;

    const int64_t n = p.n_traj;
    const int64_t i = (int64_t)blockIdx.x * B + tid;
    int st = -1;
    if (i < n) st = p.status[i];
    const bool active = st == SSA_TRAJ_OK || st == SSA_TRAJ_ABSORBED || st == SSA_TRAJ_STEP_CAP;

    if (active) {
        int *X = s_X + tid;
        float *lam = s_lam + tid;
        float *dlam = s_dlam + tid;
        float *qb = s_q + tid;
        float *dA = s_dA + tid;
        const int64_t d = p.draws[i];
        const int64_t L = (st == SSA_TRAJ_OK) ? d - 1 : d;  // index of the last visited state
        for (int s = 0; s < N; ++s) {
            X[s * B] = p.xfinal[(int64_t)s * n + i];
            lam[s * B] = 0.0f;
            dlam[s * B] = 0.0f;
        }
        const uint64_t gid = p.traj_offset + (uint64_t)i;
        const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32);
        const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
        const int nb = (M + 4) >> 2;
        const float invT = p.invT;
        const float *gl = p.dl_dobs + i * p.dl_stride;

        int64_t row_cached = -1;
        uint4 row = make_uint4(0, 0, 0, 0);
        auto event_at = [&](int64_t kk) -> int {
            const int64_t r = kk >> 3;
            if (r != row_cached) { row = p.ev[r * n + i]; row_cached = r; }
            const int slot = (int)(kk & 7);
            const uint32_t w = word_of(row, slot >> 1);
            return (slot & 1) ? (int)(w >> 16) : (int)(w & 0xffff);
        };

        int s_hi = p.S - 1;
        int brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
        float mu = 0.0f;
        int mism = 0;

        for (int64_t k = L; k >= 0; --k) {
            const bool draw = (k < L) || (st == SSA_TRAJ_OK);
            const int s_top = s_hi;
            while (s_hi >= 0 && brk_next == (int)k) {
                --s_hi;
                brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
            }
            // samples s_hi+1 .. s_top are bracketed by state k
            if (draw) {
                const int jk = event_at(k);
                // pass 1: the forward's propensities, a0 and keys, bit for bit
                float a0 = 0.0f, E0 = 1.0f, best = 0.0f, lmax = -CUDART_INF_F;
                int jb = -1;
                for (int b = 0; b < nb; ++b) {
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)k, c2, c3), key0, key1);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = 4 * b + q - 1;
                        if (j < 0) { E0 = -logf(u01(r.x)); continue; }
                        if (j >= M) break;
                        const float a = __fmul_rn(s_k[j], mass_action_h(s_rx[j], X, B));
                        a0 = __fadd_rn(a0, a);
                        float l = -CUDART_INF_F;
                        if (a > 0.0f) {
                            const float E = -logf(u01(word_of(r, q)));
                            const float key = __fdiv_rn(a, E);
                            if (key > best) { best = key; jb = j; }
                            l = __log2f(key);
                            lmax = fmaxf(lmax, l);
                        }
                        qb[j * B] = l;
                    }
                }
                mism += (jb != jk);
                const float tau = __fdiv_rn(E0, a0);
                const int4 rk = s_rx[jk];
                // readout terms that involve X_{k+1} and the clock (LINEAR interpolation)
                float dt_dir = 0.0f, dtau_dir = 0.0f;
                if (READOUT == SSA_READOUT_LINEAR) {
                    for (int s = s_hi + 1; s <= s_top; ++s) {
                        const float alpha = p.brk_a[(int64_t)s * n + i];
                        if (alpha < 0.0f) continue;
                        float c = 0.0f;
                        for (int o = 0; o < p.n_obs; ++o) {
                            const float g = gl[(int64_t)s * p.n_obs + o];
                            const int sp = p.obs_sp[o];
                            lam[sp * B] += alpha * g;
                            int dv = 0;
                            for (int e = rk.z; e < rk.w; ++e)
                                if (stoich_species(s_st[e]) == sp) dv += stoich_delta(s_st[e]);
                            c += g * (float)dv;
                        }
                        dt_dir -= c / tau;
                        dtau_dir -= alpha * c / tau;
                    }
                }
                const float dtau = mu + dtau_dir;
                // pass 2: soft sample weights and w_j = v_j . lambda
                float Z = 0.0f, Wq = 0.0f;
                for (int j = 0; j < M; ++j) {
                    const float l = qb[j * B];
                    const float q = (l == -CUDART_INF_F) ? 0.0f : exp2f((l - lmax) * invT);
                    qb[j * B] = q;
                    if (q > 0.0f) {
                        const int4 rx = s_rx[j];
                        float w = 0.0f;
                        for (int e = rx.z; e < rx.w; ++e) w += (float)stoich_delta(s_st[e]) * lam[stoich_species(s_st[e]) * B];
                        Z += q;
                        Wq += q * w;
                    }
                }
                const float invZ = 1.0f / Z;
                const float Wbar = Wq * invZ;
                const float dLda0 = -dtau * tau / a0;
                // pass 3: per-reaction adjoints and the state adjoint
                for (int j = 0; j < M; ++j) {
                    const int4 rx = s_rx[j];
                    const float kj = s_k[j];
                    const float h = mass_action_h(rx, X, B);
                    const float a = __fmul_rn(kj, h);
                    const float q = qb[j * B];
                    float psi = 0.0f;
                    if (q > 0.0f) {
                        float w = 0.0f;
                        for (int e = rx.z; e < rx.w; ++e) w += (float)stoich_delta(s_st[e]) * lam[stoich_species(s_st[e]) * B];
                        psi = q * invZ * (w - Wbar) * invT;
                    }
                    dA[j * B] += psi + dLda0 * a;
                    if (rx.x >= 0) {
                        const float x1 = (float)X[rx.x * B];
                        const float c_tau = dLda0 * kj;
                        if (rx.y < 0) {
                            dlam[rx.x * B] += (a > 0.0f ? psi / x1 : 0.0f) + c_tau;
                        } else if (rx.y == rx.x) {
                            const float dh = x1 - 0.5f;  // d/dX [X (X - 1)/2]
                            dlam[rx.x * B] += (a > 0.0f ? psi * dh / h : 0.0f) + c_tau * dh;
                        } else {
                            const float x2 = (float)X[rx.y * B];
                            dlam[rx.x * B] += (a > 0.0f ? psi / x1 : 0.0f) + c_tau * x2;
                            dlam[rx.y * B] += (a > 0.0f ? psi / x2 : 0.0f) + c_tau * x1;
                        }
                    }
                }
                mu += dt_dir;  // t_{k+1} = t_k + tau_k
            }
            // lambda_k = lambda_{k+1} + (choice and waiting-time terms) + direct readout terms
            for (int s = 0; s < N; ++s) {
                lam[s * B] += dlam[s * B];
                dlam[s * B] = 0.0f;
            }
            for (int s = s_hi + 1; s <= s_top; ++s) {
                float coef = 1.0f;
                if (READOUT == SSA_READOUT_LINEAR && draw) {
                    const float alpha = p.brk_a[(int64_t)s * n + i];
                    if (alpha >= 0.0f) coef = 1.0f - alpha;
                }
                for (int o = 0; o < p.n_obs; ++o)
                    lam[p.obs_sp[o] * B] += coef * gl[(int64_t)s * p.n_obs + o];
            }
            if ((k % p.K) == 0) {
                const int *ck = p.ckpt + (k / p.K) * (int64_t)N * n + i;
                for (int s = 0; s < N; ++s) mism += (ck[s * n] != X[s * B]);
            }
            if (k > 0) {
                const int4 rp = s_rx[event_at(k - 1)];
                for (int e = rp.z; e < rp.w; ++e) X[stoich_species(s_st[e]) * B] -= stoich_delta(s_st[e]);
            }
        }
        if (mism) atomicAdd(p.mismatch, mism);
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

// dA[j] = sum over blocks (fixed order); dtheta[r] = sum_{j: r(j) = r} dA[j] (fixed order).
// Launched with one block so that the block barrier orders both phases.
__global__ void reduce_partials_kernel(const float *partial, int64_t nblk, int M, const int *rate_index, int P,
                                       float *dA_tmp, float *dtheta)
{
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        float acc = 0.0f;
        for (int64_t b = 0; b < nblk; ++b) acc += partial[b * M + j];
        dA_tmp[j] = acc;
    }
    __threadfence_block();
    __syncthreads();
    for (int r = threadIdx.x; r < P; r += blockDim.x) {
        float acc = 0.0f;
        for (int j = 0; j < M; ++j)
            if (rate_index[j] == r) acc += dA_tmp[j];
        dtheta[r] = acc;
    }
}

template <int R>
static cudaError_t launch_adj_t(const AdjParams &p, int block, size_t smem, int64_t grid, cudaStream_t st)
{
    auto kern = adj_thread_kernel<R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_backward_thread(const AdjParams &p, int readout, int block, size_t smem, int64_t grid,
                                   cudaStream_t st)
{
    if (grid == 0) return cudaSuccess;
    return readout == SSA_READOUT_HOLD ? launch_adj_t<0>(p, block, smem, grid, st)
                                       : launch_adj_t<1>(p, block, smem, grid, st);
}

cudaError_t launch_reduce_partials(const float *partial, int64_t nblk, int M, const int *rate_index, int P,
                                   float *dA_tmp, float *dtheta, cudaStream_t st)
{
    reduce_partials_kernel<<<1, 512, 0, st>>>(partial, nblk, M, rate_index, P, dA_tmp, dtheta);
    return cudaGetLastError();
}

}  // namespace ssa
