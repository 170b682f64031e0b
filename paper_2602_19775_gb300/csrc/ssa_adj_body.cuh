// ssa_adj_body.cuh -- per-trajectory body of the thread-per-trajectory straight-through adjoint
// (arXiv 2602.19775, Eqs. 3, 5, 7; Section 3.1; Figure 1), shared by the single-network kernel and the
// batch kernel.
#pragma once

#include "ssa_internal.cuh"

namespace ssa {

// State adjoint of reaction j: choice path psi * dlog a/dX (a > 0) and waiting-time path
// c_tau * da/dX with c_tau = dL/da0 * k_j (polynomial derivative, also where a_j = 0).
__device__ __forceinline__ void reaction_state_adjoint(const int4 rx, const int *X, int B, float a, float h, float psi,
                                                       float c_tau, float *dlam)
{
    if (rx.x < 0) return;
    const float x1 = int2f(X[rx.x * B]);
    if (rx.y < 0) {
        dlam[rx.x * B] += sadj_first(x1, a, psi, c_tau);
    } else if (rx.y == rx.x) {
        dlam[rx.x * B] += sadj_homodimer(x1, a, h, psi, c_tau);
    } else {
        const float x2 = int2f(X[rx.y * B]);
        dlam[rx.x * B] += sadj_hetero(x1, x2, a, psi, c_tau);
        dlam[rx.y * B] += sadj_hetero(x2, x1, a, psi, c_tau);
    }
}

__device__ __forceinline__ float stoich_dot(const int4 rx, const int *s_st, const float *lam, int B)
{
    float w = 0.0f;
    for (int e = rx.z; e < rx.w; ++e) w += (float)stoich_delta(s_st[e]) * lam[stoich_species(s_st[e]) * B];
    return w;
}

// Per-trajectory body of the thread adjoint. X, lam, dlam point at this trajectory's column (stride B);
// q and dA at its column of the runtime-size buffers [M][B] (MC == 0); dAr holds the per-reaction
// adjoints in registers when MC > 0.
template <int READOUT, int MC>
__device__ __forceinline__ void thread_adj_body(const AdjParams &p, const int4 *s_rx, const int *s_st,
                                                const float *s_k, int *X, float *lam, float *dlam, float *qbuf,
                                                float *dA, const int B, const int64_t i, const int st,
                                                float (&dAr)[MC > 0 ? MC : 1])
{
    const int N = p.N, M = p.M;
    const int64_t n = p.n_traj;
    const int d = p.draws[i];
    const int L = (st == SSA_TRAJ_OK) ? d - 1 : d;  // index of the last visited state
    for (int s = 0; s < N; ++s) {
        X[s * B] = p.xfinal[(int64_t)s * n + i];
        lam[s * B] = 0.0f;
        dlam[s * B] = 0.0f;
    }
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32);
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    const float invT = p.invT;
    const float *gl = p.dl_dobs + i * p.dl_stride;

    int row_cached = -1;
    uint4 row = make_uint4(0, 0, 0, 0);
    auto event_at = [&](int kk) -> int {
        const int r = kk >> 3;
        if (r != row_cached) { row = p.ev[(int64_t)r * n + i]; row_cached = r; }
        const int slot = kk & 7;
        const uint32_t w = word_of(row, slot >> 1);
        return (slot & 1) ? (int)(w >> 16) : (int)(w & 0xffff);
    };

    int s_hi = p.S - 1;
    int brk_next = (READOUT != SSA_READOUT_BIN && s_hi >= 0) ? p.brk_k[(int64_t)s_hi * n + i] : -1;
    // BIN: one recorded slot per state interval that holds edges
    BinSlots bslots{-1, -1};
    float d_first = 0.0f, d_last = 0.0f;
    if (READOUT == SSA_READOUT_BIN) bin_slots_init(bslots, p.brk_k, p.brk_tail, n, i);
    float mu = 0.0f;
    int mism = 0;
    int ck_row = L / p.K, ck_off = L - ck_row * p.K;  // checkpoint c holds X_{cK}

    constexpr int NQ = MC > 0 ? MC + 1 : 1;
    float E[NQ], En[NQ];
    const bool draw_last = st == SSA_TRAJ_OK;
    if (MC > 0) step_noise<NQ>(E, (uint32_t)(draw_last ? L : (L > 0 ? L - 1 : 0)), c2, c3, key0, key1);

    // BIN readout: gq = g of the bin that contains t_{k+1} (none past the last edge), xo = X_{k+1}
    // at the observables
    constexpr bool kBin = READOUT == SSA_READOUT_BIN;
    float gq[kBinMaxObs], gk[kBinMaxObs];
    int osp[kBinMaxObs], xo[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) osp[c] = (kBin && c < p.n_obs) ? p.obs_sp[c] : 0;
    auto xobs = [&](int c) { return X[osp[c] * B]; };
    auto addx = [&](int c, float v) { lam[osp[c] * B] += v; };
    if (kBin) {
        bin_grad(gq, gl, p.n_obs, p.ts, p.S, p.S);
#pragma unroll
        for (int c = 0; c < kBinMaxObs; ++c) xo[c] = c < p.n_obs ? xobs(c) : 0;
    }

    for (int k = L; k >= 0; --k) {
        const bool draw = (k < L) || draw_last;
        const int s_top = s_hi;
        if (READOUT == SSA_READOUT_BIN) {
            bin_slots_step(bslots, p.brk_k, p.brk_s, p.brk_a, p.ts, n, i, k, s_hi, d_first, d_last);
        } else {
            while (s_hi >= 0 && brk_next == k) {
                --s_hi;
                brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
            }
        }
        // samples s_hi+1 .. s_top are bracketed by state k
        if (kBin) {
            if (s_hi < s_top) bin_grad(gk, gl, p.n_obs, p.ts, p.S, s_hi + 1);
            else {
#pragma unroll
                for (int c = 0; c < kBinMaxObs; ++c) gk[c] = gq[c];
            }
        }
        float tau_k = 0.0f;
        if (draw) {
            const int jk = event_at(k);
            float a0 = 0.0f, ab = 0.0f, Eb = 1.0f, E0, lmax = -CUDART_INF_F;
            int jb = -1;
            float ar[MC > 0 ? MC : 1], lr[MC > 0 ? MC : 1];
            // pass 1: the forward's propensities, a0 and race, bit for bit; log2 keys
            if constexpr (MC > 0) {
                if (k > 0) step_noise<NQ>(En, (uint32_t)(k - 1), c2, c3, key0, key1);  // prefetch
                E0 = E[0];
#pragma unroll
                for (int j = 0; j < MC; ++j) {
                    const float a = __fmul_rn(s_k[j], mass_action_h(s_rx[j], X, B));
                    a0 = __fadd_rn(a0, a);
                    race(a, E[j + 1], j, ab, Eb, jb);
                    ar[j] = a;
                    lr[j] = a > 0.0f ? __log2f(a) - __log2f(E[j + 1]) : -CUDART_INF_F;
                    lmax = fmaxf(lmax, lr[j]);
                }
            } else {
                uint4 cache;
                int cb = -1;
                E0 = exp_variate((uint32_t)k, 0, c2, c3, key0, key1, cache, cb);
                for (int j = 0; j < M; ++j) {
                    const float a = __fmul_rn(s_k[j], mass_action_h(s_rx[j], X, B));
                    a0 = __fadd_rn(a0, a);
                    float l = -CUDART_INF_F;
                    if (a > 0.0f) {
                        const float Ej = exp_variate((uint32_t)k, j + 1, c2, c3, key0, key1, cache, cb);
                        race(a, Ej, j, ab, Eb, jb);
                        l = __log2f(a) - __log2f(Ej);
                        lmax = fmaxf(lmax, l);
                    }
                    qbuf[j * B] = l;
                }
            }
            mism += (jb != jk);
            const float tau = waiting_time(E0, a0);
            tau_k = tau;
            const int4 rk = s_rx[jk];
            // BIN: t_{k+1} ends this interval and starts the next, in the bin of gq
            if (kBin) mu -= bin_transition(xobs, xo, gq, p.n_obs);
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
                    const float c_tau = __fdividef(c, tau);
                    dt_dir -= c_tau;
                    dtau_dir -= alpha * c_tau;
                }
            }
            const float dtau = mu + dtau_dir;
            const float dLda0 = -dtau * tau / a0;
            // pass 2: soft-sample weights y~_j ~ exp2((l_j - l_max)/T) and W = sum y~ w
            float Z = 0.0f, Wq = 0.0f;
            if constexpr (MC > 0) {
                float wr[MC];
#pragma unroll
                for (int j = 0; j < MC; ++j) {
                    const float q = lr[j] == -CUDART_INF_F ? 0.0f : exp2f((lr[j] - lmax) * invT);
                    lr[j] = q;
                    wr[j] = stoich_dot(s_rx[j], s_st, lam, B);
                    Z += q;
                    Wq += q * wr[j];
                }
                const float invZ = __fdividef(1.0f, Z), Wbar = Wq * invZ;
                // pass 3: per-reaction adjoints and the state adjoint
                // every w_j is already read, so the state adjoint accumulates into lambda
#pragma unroll
                for (int j = 0; j < MC; ++j) {
                    const float psi = lr[j] > 0.0f ? lr[j] * invZ * (wr[j] - Wbar) * invT : 0.0f;
                    dAr[j] += psi + dLda0 * ar[j];
                    const int4 rx = s_rx[j];
                    reaction_state_adjoint(rx, X, B, ar[j], mass_action_h(rx, X, B), psi, dLda0 * s_k[j], lam);
                }
            } else {
                for (int j = 0; j < M; ++j) {
                    const float l = qbuf[j * B];
                    const float q = (l == -CUDART_INF_F) ? 0.0f : exp2f((l - lmax) * invT);
                    qbuf[j * B] = q;
                    if (q > 0.0f) {
                        Z += q;
                        Wq += q * stoich_dot(s_rx[j], s_st, lam, B);
                    }
                }
                const float invZ = __fdividef(1.0f, Z), Wbar = Wq * invZ;
                for (int j = 0; j < M; ++j) {
                    const int4 rx = s_rx[j];
                    const float h = mass_action_h(rx, X, B);
                    const float a = __fmul_rn(s_k[j], h);
                    const float q = qbuf[j * B];
                    const float psi = q > 0.0f ? q * invZ * (stoich_dot(rx, s_st, lam, B) - Wbar) * invT : 0.0f;
                    dA[j * B] += psi + dLda0 * a;
                    reaction_state_adjoint(rx, X, B, a, h, psi, dLda0 * s_k[j], dlam);
                }
            }
            mu += dt_dir;  // t_{k+1} = t_k + tau_k
        }
        // lambda_k = lambda_{k+1} + (choice and waiting-time terms) + direct readout terms
        if (MC == 0) {
            for (int s = 0; s < N; ++s) {
                lam[s * B] += dlam[s * B];
                dlam[s * B] = 0.0f;
            }
        }
        if (kBin) {
            bin_state_terms(addx, d_first, d_last, gl, p.bin_prefix, p.n_obs, s_hi + 1, s_top, draw, tau_k, gq, gk);
#pragma unroll
            for (int c = 0; c < kBinMaxObs; ++c) {
                gq[c] = gk[c];
                if (c < p.n_obs) xo[c] = xobs(c);
            }
        } else {
            for (int s = s_hi + 1; s <= s_top; ++s) {
                float coef = 1.0f;
                if (READOUT == SSA_READOUT_LINEAR && draw) {
                    const float alpha = p.brk_a[(int64_t)s * n + i];
                    if (alpha >= 0.0f) coef = 1.0f - alpha;
                }
                for (int o = 0; o < p.n_obs; ++o) lam[p.obs_sp[o] * B] += coef * gl[(int64_t)s * p.n_obs + o];
            }
        }
        if (ck_off == 0) {
            const int *ck = p.ckpt + (int64_t)ck_row * N * n + i;
            for (int s = 0; s < N; ++s) mism += (ck[(int64_t)s * n] != X[s * B]);
            --ck_row;
            ck_off = p.K;
        }
        --ck_off;
        if (k > 0) {
            const int4 rp = s_rx[event_at(k - 1)];
            for (int e = rp.z; e < rp.w; ++e) X[stoich_species(s_st[e]) * B] -= stoich_delta(s_st[e]);
        }
        if constexpr (MC > 0) {
            if (draw) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) E[q] = En[q];
            }
        }
    }
    if (mism) atomicAdd(p.mismatch, mism);
}

}  // namespace ssa
