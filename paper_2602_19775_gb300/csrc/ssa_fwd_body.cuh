// ssa_fwd_body.cuh -- per-trajectory body of the thread-per-trajectory forward (arXiv 2602.19775,
// Section 2, Section 3.2, Eq. 6), shared by the single-network kernel and the batch kernel.
#pragma once

#include "ssa_internal.cuh"

namespace ssa {

// Per-trajectory body of the thread-per-trajectory forward: X points at this trajectory's counts,
// species s at X[s * B]; the tables may live in shared or global memory.
template <int READOUT, bool RECORD, bool REPLAY, int MC>
__device__ __forceinline__ void thread_fwd_body(const FwdParams &p, const int4 *s_rx, const int *s_st,
                                                const float *s_k, int *X, const int B, const int64_t i)
{
    const int N = p.N, M = p.M;
    const int64_t n = p.n_traj;

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
    // BIN readout: integral of the open bin up to t_k per observable (species clamped when invalid)
    float bacc[kBinMaxObs];
    BinRuns bruns;
    bin_runs_init(bruns);
    int osp[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) {
        bacc[c] = 0.0f;
        osp[c] = (READOUT == SSA_READOUT_BIN && c < p.n_obs && !bad_obs) ? p.obs_sp[c] : 0;
    }
    auto xobs = [&](int c) { return X[osp[c] * B]; };

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
        const float tau = waiting_time(E0, a0);
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
            const int s_first = s;
            if constexpr (READOUT == SSA_READOUT_BIN) {
                s = bin_edges<RECORD>(p, i, s, t, t_next, k, bacc, xobs, bruns);
            } else {
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
            }
            // BIN: the rest of [t_k, t_{k+1}) after the last edge opens the next bin
            if (READOUT == SSA_READOUT_BIN && !cross && s > s_first)
                bin_accumulate(bacc, xobs, p.n_obs, d2f_nonneg(t_next - p.ts[s - 1]));
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;  // the crossing draw is made but not applied
        } else if (READOUT == SSA_READOUT_BIN) {
            bin_accumulate(bacc, xobs, p.n_obs, tau);
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
    if constexpr (READOUT == SSA_READOUT_BIN) bin_tail<RECORD>(p, i, s, t, k, bacc, xobs, bad_obs, bruns);
    for (; READOUT != SSA_READOUT_BIN && s < p.S; ++s) {
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

}  // namespace ssa
