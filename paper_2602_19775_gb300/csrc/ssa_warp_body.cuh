// ssa_warp_body.cuh -- per-trajectory bodies of the warp-per-trajectory forward and adjoint, shared by
// the single-network kernels and the batch kernel.
#pragma once

#include "ssa_adj_body.cuh"

// Philox blocks a lane draws together in the adjoint's first pass (the forward draws four); a tuning
// constant: more blocks give the scheduler more independent work but keep more registers live.
#ifndef SSA_WARP_ADJ_CHUNK
#define SSA_WARP_ADJ_CHUNK 1
#endif

namespace ssa {

// One step's propensities, a0 and race over this lane's Philox blocks b = lane, lane + 32, ...
// Returns E_0 on lane 0. If aj / lj are given, stores a_j and log2(a_j / E_j) (or -inf) for this
// lane's reactions. The forward takes the lane's blocks four at a time: their Philox words and
// variates are drawn first (four independent dependency chains for the scheduler to interleave), then
// the reactions are evaluated in increasing j, so the sums and the race see the same values in the
// same order as the adjoint's one-block-at-a-time loop (which keeps fewer values live).
template <bool STORE>
__device__ __forceinline__ void warp_step_eval(const FwdParamsView &v, int k, const int *X, float &a0, float &E0,
                                               float &ab, float &Eb, int &jb, float *aj, float *lj, float &lmax)
{
    constexpr int CH = STORE ? SSA_WARP_ADJ_CHUNK : 4;
    const int lane = threadIdx.x & 31;
    float a0p = 0.0f;
    E0 = 0.0f;
    ab = 0.0f;
    Eb = 1.0f;
    jb = -1;
    lmax = -CUDART_INF_F;
    const int n_rounds = (v.nb + 31) >> 5;  // blocks per lane, rounded up
    for (int t0 = 0; t0 < n_rounds; t0 += CH) {
        float E[CH][4];
#pragma unroll
        for (int t = 0; t < CH; ++t) {
            const int b = lane + 32 * (t0 + t);
            if (b < v.nb) {
                const uint4 r = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)k, v.c2, v.c3), v.key0, v.key1);
                E[t][0] = neg_log_unit(u01(r.x));
                E[t][1] = neg_log_unit(u01(r.y));
                E[t][2] = neg_log_unit(u01(r.z));
                E[t][3] = neg_log_unit(u01(r.w));
            }
        }
#pragma unroll
        for (int t = 0; t < CH; ++t) {
            const int b = lane + 32 * (t0 + t);
            if (b >= v.nb) break;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // predicated rather than branched: word 0 of lane 0's first block (j = -1) drives the waiting
                // time, and its table slot, like the padded ones (j >= M), has rate 0, so it adds 0 to a0, never
                // wins the race (a_j E_b > a_b E_j fails for a_j = 0) and its key is -inf (log2 0)
                const int j = 4 * b + q - 1;
                if (q == 0 && j < 0) E0 = E[t][0];
                const int pos = q * v.nb + b;
                const float a = __fmul_rn(v.s_k[pos], mass_action_h_sel(v.s_rx[pos], X));
                a0p = __fadd_rn(a0p, a);
                race(a, E[t][q], j, ab, Eb, jb);
                if (STORE) {
                    const float l = __log2f(a) - __log2f(E[t][q]);
                    lmax = fmaxf(lmax, l);
                    if (j >= 0 && j < v.M) {
                        aj[pos] = a;
                        lj[pos] = l;
                    }
                }
            }
        }
    }
    a0 = warp_sum(a0p);
    warp_race_combine(ab, Eb, jb);
    E0 = __shfl_sync(0xffffffffu, E0, 0);
    if (STORE) lmax = warp_max(lmax);
}

// Bin readout (Section 4.4) on a warp-per-trajectory forward. Every lane runs the same bookkeeping on the
// same values (the running integrals, the edges found by bisection, the slot count); lane 0 stores the bin an
// interval's first edge closes and the slot record, and whole bins held at one state are written by the
// warp along the trajectory's own row (consecutive lanes on consecutive floats). The values are those of
// the thread kernels' bin readout.
template <class XF>
__device__ __forceinline__ void warp_bin_held(const FwdParams &p, int64_t i, int lo, int hi, const XF &xobs, bool zero)
{
    if (lo > hi) return;
    const int lane = threadIdx.x & 31, no = p.n_obs;
    float xv[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) xv[c] = (c < no && !zero) ? obs_f(xobs(c)) : 0.0f;
    float *row = static_cast<float *>(p.obs_out) + i * (int64_t)p.S * no;
    for (int64_t e = (int64_t)lo * no + lane; e < (int64_t)(hi + 1) * no; e += 32) {
        const int c = no == 1 ? 0 : (int)(e % no);
        float v = xv[0];
#pragma unroll
        for (int c2 = 1; c2 < kBinMaxObs; ++c2) v = c == c2 ? xv[c2] : v;
        row[e] = v;
    }
}

template <bool RECORD, class XF>
__device__ __forceinline__ void warp_bin_first_edge(const FwdParams &p, int64_t i, int s, double t_k, int k,
                                                    float (&acc)[kBinMaxObs], const XF &xobs, int &slots, bool zero)
{
    float o[kBinMaxObs];
    const float d = bin_close(acc, xobs, p.n_obs, p.ts, s, t_k, true, o);
    if ((threadIdx.x & 31) == 0) {
        float *dst = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
        for (int c = 0; c < p.n_obs; ++c) dst[c] = zero ? 0.0f : o[c];
        if (RECORD) {
            const int64_t at = (int64_t)slots * p.n_traj + i;
            p.brk_k[at] = k;
            p.brk_s[at] = s;
            p.brk_a[at] = d;
        }
    }
    if (RECORD) ++slots;
}

// the edges in the state interval [t_k, t_next) from s on; returns the first edge at or after t_next
template <bool RECORD, class XF>
__device__ __forceinline__ int warp_bin_edges(const FwdParams &p, int64_t i, int s, double t_k, double t_next, int k,
                                              float (&acc)[kBinMaxObs], const XF &xobs, int &slots)
{
    int lo = s, hi = p.S;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (gt_nonneg(t_next, p.ts[mid])) lo = mid + 1;
        else hi = mid;
    }
    if (lo > s) {
        warp_bin_first_edge<RECORD>(p, i, s, t_k, k, acc, xobs, slots, false);
        warp_bin_held(p, i, s + 1, lo - 1, xobs, false);
    }
    return lo;
}

// after the last state (held from t_k on): close the first remaining bin, hold the rest, record the slot count
template <bool RECORD, class XF>
__device__ __forceinline__ void warp_bin_tail(const FwdParams &p, int64_t i, int s, double t_k, int k,
                                              float (&acc)[kBinMaxObs], const XF &xobs, bool bad_obs, int &slots)
{
    if (s < p.S) {
        warp_bin_first_edge<RECORD>(p, i, s, t_k, k, acc, xobs, slots, bad_obs);
        warp_bin_held(p, i, s + 1, p.S - 1, xobs, bad_obs);
    }
    if (RECORD && (threadIdx.x & 31) == 0) p.brk_tail[i] = slots;
}

// Per-trajectory body of the warp forward (all 32 lanes of one warp); X = this warp's counts.
template <int READOUT, bool RECORD>
__device__ __forceinline__ void warp_fwd_body(const FwdParams &p, const int4 *s_rx, const int *s_st, const float *s_k,
                                              int *X, const int64_t i)
{
    const int lane = threadIdx.x & 31;
    const int N = p.N, M = p.M;
    const int64_t n = p.n_traj;

    const int *x0 = p.x0 + (p.x0_per_traj ? i * N : 0);
    const bool bad_obs = (*p.flag & kErrBadObs) != 0;
    bool neg = false;
    for (int s = lane; s < N; s += 32) {
        X[s] = x0[s];
        neg |= x0[s] < 0;
    }
    const bool bad_input = __any_sync(0xffffffffu, neg) || (*p.flag & (kErrBadSamples | kErrBadObs)) != 0;
    __syncwarp();
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    FwdParamsView v{s_rx, s_k, M, (M + 4) >> 2, (uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)p.seed,
                    (uint32_t)(p.seed >> 32)};

    double t = 0.0;
    int s = 0;
    double thr = p.S > 0 ? p.ts[0] : p.t_end;
    int status = bad_input ? SSA_TRAJ_BAD_INPUT : SSA_TRAJ_OK;
    int k = 0, draws = 0, ck_left = p.K, ck_row = 0;
    uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    constexpr bool kBin = READOUT == SSA_READOUT_BIN;
    float bacc[kBinMaxObs];
    int osp[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) {
        bacc[c] = 0.0f;
        osp[c] = (kBin && c < p.n_obs && !bad_obs) ? p.obs_sp[c] : 0;
    }
    auto xobs = [&](int c) { return X[osp[c]]; };
    int slots = 0;

    while (!bad_input) {
        if (k >= p.max_steps) { status = SSA_TRAJ_STEP_CAP; break; }
        float a0, E0, ab, Eb, lmax;
        int jb;
        warp_step_eval<false>(v, k, X, a0, E0, ab, Eb, jb, nullptr, nullptr, lmax);
        if (!(a0 < CUDART_INF_F)) { status = SSA_TRAJ_BAD_RATE; break; }
        if (a0 == 0.0f) { status = SSA_TRAJ_ABSORBED; break; }
        if (jb < 0) { status = SSA_TRAJ_BAD_RATE; break; }
        const float tau = waiting_time(E0, a0);
        const double t_next = t + f2d_pos(tau);
        const int4 rj = s_rx[jpos(jb, v.nb)];
        const bool slow = gt_nonneg(t_next, thr);
        const bool cross = slow && gt_nonneg(t_next, p.t_end);
        if (!cross) {
            bool bad_neg = false, bad_ovf = false;
            for (int e = rj.z + lane; e < rj.w; e += 32) {
                const int st = s_st[e];
                const int x = X[stoich_species(st)], d = stoich_delta(st);
                bad_neg |= d < 0 && x + d < 0;
                bad_ovf |= d > 0 && x > 2147483647 - d;
            }
            if (__any_sync(0xffffffffu, bad_neg)) status = SSA_TRAJ_NEG_COUNT;
            else if (__any_sync(0xffffffffu, bad_ovf)) status = SSA_TRAJ_OVERFLOW;
        }
        if (RECORD) {
            e0 = __funnelshift_r(e0, e1, 16);
            e1 = __funnelshift_r(e1, e2, 16);
            e2 = __funnelshift_r(e2, e3, 16);
            e3 = (e3 >> 16) | ((uint32_t)jb << 16);
            if (lane == 0 && (k & 7) == 7) p.ev[(int64_t)(k >> 3) * n + i] = make_uint4(e0, e1, e2, e3);
        }
        draws = k + 1;
        if (status != SSA_TRAJ_OK) break;
        if (slow && kBin) {
            const int s_first = s;
            s = warp_bin_edges<RECORD>(p, i, s, t, t_next, k, bacc, xobs, slots);
            if (!cross && s > s_first) bin_accumulate(bacc, xobs, p.n_obs, d2f_nonneg(t_next - p.ts[s - 1]));
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;
        } else if (kBin) {
            bin_accumulate(bacc, xobs, p.n_obs, tau);
        }
        if (slow && !kBin) {
            while (s < p.S && gt_nonneg(t_next, p.ts[s])) {
                if (READOUT == SSA_READOUT_HOLD) {
                    int *o = static_cast<int *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                    for (int c = lane; c < p.n_obs; c += 32) o[c] = X[p.obs_sp[c]];
                } else {
                    const float alpha = __fdiv_rn(d2f_nonneg(p.ts[s] - t), tau);
                    float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                    for (int c = lane; c < p.n_obs; c += 32) {
                        const int sp = p.obs_sp[c];
                        int dv = 0;
                        for (int e = rj.z; e < rj.w; ++e)
                            if (stoich_species(s_st[e]) == sp) dv += stoich_delta(s_st[e]);
                        o[c] = __fmaf_rn(alpha, (float)dv, (float)X[sp]);
                    }
                    if (RECORD && lane == 0) p.brk_a[(int64_t)s * n + i] = alpha;
                }
                if (RECORD && lane == 0) p.brk_k[(int64_t)s * n + i] = k;
                ++s;
            }
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;
        }
        __syncwarp();
        for (int e = rj.z + lane; e < rj.w; e += 32) {
            const int st = s_st[e];
            X[stoich_species(st)] += stoich_delta(st);  // the entries of one reaction name distinct species
        }
        __syncwarp();
        t = t_next;
        ++k;
        if (RECORD && --ck_left == 0) {
            ck_left = p.K;
            ++ck_row;
            int *ck = p.ckpt + (int64_t)ck_row * N * n + i;
            for (int sp = lane; sp < N; sp += 32) ck[(int64_t)sp * n] = X[sp];
        }
    }
    __syncwarp();
    if constexpr (kBin) warp_bin_tail<RECORD>(p, i, s, t, k, bacc, xobs, bad_obs, slots);
    for (; !kBin && s < p.S; ++s) {
        if (READOUT == SSA_READOUT_HOLD) {
            int *o = static_cast<int *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
            for (int c = lane; c < p.n_obs; c += 32) o[c] = bad_obs ? 0 : X[p.obs_sp[c]];
        } else {
            float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
            for (int c = lane; c < p.n_obs; c += 32) o[c] = bad_obs ? 0.0f : (float)X[p.obs_sp[c]];
            if (RECORD && lane == 0) p.brk_a[(int64_t)s * n + i] = -1.0f;
        }
        if (RECORD && lane == 0) p.brk_k[(int64_t)s * n + i] = k;
    }
    if (lane == 0) {
        p.draws[i] = draws;
        p.status[i] = status;
    }
    if (RECORD) {
        if ((draws & 7) && lane == 0) {
            for (int pad = draws & 7; pad < 8; ++pad) {
                e0 = __funnelshift_r(e0, e1, 16);
                e1 = __funnelshift_r(e1, e2, 16);
                e2 = __funnelshift_r(e2, e3, 16);
                e3 = e3 >> 16;
            }
            p.ev[(int64_t)((draws - 1) >> 3) * n + i] = make_uint4(e0, e1, e2, e3);
        }
        for (int sp = lane; sp < N; sp += 32) {
            p.xfinal[(int64_t)sp * n + i] = X[sp];
            p.ckpt[(int64_t)sp * n + i] = x0[sp];
        }
    }
}

// One step of the soft forward (Section 3.3, Eq. 4) at the real state X, all 32 lanes: lane l evaluates the
// reactions of its Philox blocks (relaxed propensities with negative factors clipped at 0, keys
// l_j = log2 a_j - log2 E_j), the warp reduces a0 and the largest key, the lanes turn their keys into
// unnormalised weights w_j = exp2((l_j - l_max)/T) (kept in y by lane-major position), and each species sums
// its own change dX_s = sum_j (w_j / Z) v_js through the species-major update list in increasing j (no atomics:
// the specialised thread kernels' order of the update). With AH, a_j and h_j are kept too (the adjoint's
// re-evaluation). Returns a0; sets E0, invZ = 1/Z and whether X + dX is finite. The forward and the adjoint's
// segment re-runs call this one function, so the regenerated states are the forward's bit for bit.
template <bool AH>
__device__ __forceinline__ float warp_soft_step(const int4 *s_rx, const float *s_k, const int *s_upd, int N, int M,
                                                float invT, int k, uint32_t c2, uint32_t c3, uint32_t key0,
                                                uint32_t key1, const float *X, float *a_out, float *h_out, float *y,
                                                float *dX, float &E0, float &invZ, bool &finite)
{
    const int lane = threadIdx.x & 31, nb = (M + 4) >> 2;
    const int upd_base = (N + 1 + 3) & ~3;  // the list follows the padded pointer array
    float a0p = 0.0f, lmaxp = -CUDART_INF_F;
    E0 = 0.0f;
    for (int b = lane; b < nb; b += 32) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)k, c2, c3), key0, key1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // predicated: the waiting-time word's slot (j = -1) and the padded ones have rate 0 (they add 0 to
            // a0 and have key -inf), and the factor is chosen by selects rather than by branches on the order
            const int j = 4 * b + q - 1;
            const float E = neg_log_unit(u01(word_of(r, q)));
            if (q == 0 && j < 0) E0 = E;
            const int pos = q * nb + b;
            const int4 rx = s_rx[pos];
            const float x1 = X[rx.x >= 0 ? rx.x : 0], x2 = X[rx.y >= 0 ? rx.y : 0];
            const float h = rx.x < 0 ? 1.0f : rx.y < 0 ? hs_first(x1) : rx.y == rx.x ? hs_homodimer(x1) : hs_hetero(x1, x2);
            const float a = __fmul_rn(s_k[pos], h);
            a0p = __fadd_rn(a0p, a);
            const float l = a > 0.0f ? log2f(a) - log2f(E) : -CUDART_INF_F;
            if (j >= 0 && j < M) {
                y[pos] = l;
                if (AH) {
                    a_out[pos] = a;
                    h_out[pos] = h;
                }
            }
            lmaxp = fmaxf(lmaxp, l);
        }
    }
    const float a0 = warp_sum(a0p), lmax = warp_max(lmaxp);
    E0 = __shfl_sync(0xffffffffu, E0, 0);
    float Zp = 0.0f;
    for (int b = lane; b < nb; b += 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = 4 * b + q - 1;
            const bool live = j >= 0 && j < M;
            const int pos = q * nb + b;
            const float l = live ? y[pos] : -CUDART_INF_F;
            const float w = l == -CUDART_INF_F ? 0.0f : exp2f((l - lmax) * invT);
            if (live) y[pos] = w;
            Zp += w;  // + 0 outside the live slots: the same bits
        }
    }
    invZ = __fdividef(1.0f, warp_sum(Zp));
    __syncwarp();
    bool fin = true;
    for (int sp = lane; sp < N; sp += 32) {
        float d = 0.0f;
        for (int e = s_upd[sp]; e < s_upd[sp + 1]; ++e) {
            const int ent = s_upd[upd_base + e];
            d = __fmaf_rn(y[ent >> 8] * invZ, (float)(int)(signed char)(ent & 0xff), d);
        }
        dX[sp] = d;
        fin &= fabsf(__fadd_rn(X[sp], d)) < CUDART_INF_F;
    }
    finite = __all_sync(0xffffffffu, fin);
    __syncwarp();
    return a0;
}

// Per-trajectory body of the warp soft forward (Eq. 4). Clock, samples and readouts are the forward's;
// recorded, the float state is checkpointed every kSoftK steps ([n_ckpt][N][n_traj], checkpoint 0 = X_0) with
// the sample brackets, for the adjoint's segment re-runs.
template <int READOUT, bool RECORD>
__device__ __forceinline__ void warp_soft_fwd_body(const FwdParams &p, const int4 *s_rx, const float *s_k,
                                                   const int *s_upd, float *X, float *dX, float *y, const int64_t i)
{
    const int lane = threadIdx.x & 31;
    const int N = p.N, M = p.M;
    const int64_t n = p.n_traj;
    const int *x0 = p.x0 + (p.x0_per_traj ? i * N : 0);
    const bool bad_obs = (*p.flag & kErrBadObs) != 0;
    bool neg = false;
    for (int sp = lane; sp < N; sp += 32) {
        X[sp] = int2f(x0[sp]);
        neg |= x0[sp] < 0;
    }
    const bool bad_input = __any_sync(0xffffffffu, neg) || (*p.flag & (kErrBadSamples | kErrBadObs)) != 0;
    __syncwarp();
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32), key0 = (uint32_t)p.seed,
                   key1 = (uint32_t)(p.seed >> 32);
    double t = 0.0;
    int s = 0;
    double thr = p.S > 0 ? p.ts[0] : p.t_end;
    int status = bad_input ? SSA_TRAJ_BAD_INPUT : SSA_TRAJ_OK;
    int k = 0, draws = 0, ck_left = p.K, ck_row = 0;
    constexpr bool kBin = READOUT == SSA_READOUT_BIN;
    float bacc[kBinMaxObs];
    int osp[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) {
        bacc[c] = 0.0f;
        osp[c] = (kBin && c < p.n_obs && !bad_obs) ? p.obs_sp[c] : 0;
    }
    auto xobs = [&](int c) { return X[osp[c]]; };
    int slots = 0;
    float *obs = static_cast<float *>(p.obs_out);
    float *ckf = reinterpret_cast<float *>(p.ckpt);

    while (!bad_input) {
        if (k >= p.max_steps) { status = SSA_TRAJ_STEP_CAP; break; }
        float E0, invZ;
        bool finite;
        const float a0 = warp_soft_step<false>(s_rx, s_k, s_upd, N, M, p.invT, k, c2, c3, key0, key1, X, nullptr,
                                               nullptr, y, dX, E0, invZ, finite);
        if (!(a0 < CUDART_INF_F)) { status = SSA_TRAJ_BAD_RATE; break; }
        if (a0 == 0.0f) { status = SSA_TRAJ_ABSORBED; break; }
        const float tau = waiting_time(E0, a0);
        const double t_next = t + f2d_pos(tau);
        const bool slow = gt_nonneg(t_next, thr);
        const bool cross = slow && gt_nonneg(t_next, p.t_end);
        draws = k + 1;
        if (!cross && !finite) { status = SSA_TRAJ_BAD_RATE; break; }
        if (slow && kBin) {
            const int s_first = s;
            s = warp_bin_edges<RECORD>(p, i, s, t, t_next, k, bacc, xobs, slots);
            if (!cross && s > s_first) bin_accumulate(bacc, xobs, p.n_obs, d2f_nonneg(t_next - p.ts[s - 1]));
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;
        } else if (kBin) {
            bin_accumulate(bacc, xobs, p.n_obs, tau);
        }
        if (slow && !kBin) {
            while (s < p.S && gt_nonneg(t_next, p.ts[s])) {
                float *o = obs + ((int64_t)i * p.S + s) * p.n_obs;
                if (READOUT == SSA_READOUT_HOLD) {
                    for (int c = lane; c < p.n_obs; c += 32) o[c] = X[p.obs_sp[c]];
                } else {
                    const float alpha = __fdiv_rn(d2f_nonneg(p.ts[s] - t), tau);
                    for (int c = lane; c < p.n_obs; c += 32) {
                        const int sp = p.obs_sp[c];
                        o[c] = __fmaf_rn(alpha, dX[sp], X[sp]);
                    }
                    if (RECORD && lane == 0) p.brk_a[(int64_t)s * n + i] = alpha;
                }
                if (RECORD && lane == 0) p.brk_k[(int64_t)s * n + i] = k;
                ++s;
            }
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;
        }
        __syncwarp();
        for (int sp = lane; sp < N; sp += 32) X[sp] = __fadd_rn(X[sp], dX[sp]);
        __syncwarp();
        t = t_next;
        ++k;
        if (RECORD && --ck_left == 0) {
            ck_left = p.K;
            ++ck_row;
            for (int sp = lane; sp < N; sp += 32) ckf[((int64_t)ck_row * N + sp) * n + i] = X[sp];
        }
    }
    __syncwarp();
    if constexpr (kBin) warp_bin_tail<RECORD>(p, i, s, t, k, bacc, xobs, bad_obs, slots);
    for (; !kBin && s < p.S; ++s) {
        float *o = obs + ((int64_t)i * p.S + s) * p.n_obs;
        for (int c = lane; c < p.n_obs; c += 32) o[c] = bad_obs ? 0.0f : X[p.obs_sp[c]];
        if (RECORD && lane == 0) {
            if (READOUT == SSA_READOUT_LINEAR) p.brk_a[(int64_t)s * n + i] = -1.0f;
            p.brk_k[(int64_t)s * n + i] = k;
        }
    }
    if (lane == 0) {
        p.draws[i] = draws;
        p.status[i] = status;
    }
    if (RECORD)
        for (int sp = lane; sp < N; sp += 32) ckf[(int64_t)sp * n + i] = int2f(x0[sp]);  // checkpoint 0 = X_0
}

// Exact gradient of the soft forward on the warp layout, one trajectory (all 32 lanes): the specialised thread
// kernels' soft adjoint in the warp's arrays. Segment by segment from the end, the kSoftK states are
// regenerated from the float checkpoint with the forward's own step (the state after a segment must equal the
// next checkpoint bit for bit), then walked back: the step is evaluated again at X_k, the readout terms give
// the waiting-time adjoint, w_j = v_j . lambda, psi_j = y~_j (w_j - sum y~ w) / T, dA_j += psi_j + dL/da0 a_j,
// and every reactant slot's contribution (choice path and waiting-time path, clipped where a factor is) is
// gathered per species through the reactant-slot incidence list in increasing j, added to lambda in that
// order. Per-warp arrays: Xs [kSoftK][Npad], lam, dX [Npad]; a, h, y, c1, c2 [Mp]; dA [Mp] accumulates.
template <int READOUT>
__device__ __forceinline__ void warp_soft_adj_body(const AdjParams &p, const int4 *s_rx, const int *s_st,
                                                   const int *s_inc_ptr, const int *s_inc, const float *s_k,
                                                   const int *s_upd, float *Xs, float *lam, float *dX, float *aj,
                                                   float *hj, float *y, float *c1, float *c2, float *dA,
                                                   const int64_t i, const int st)
{
    const int lane = threadIdx.x & 31;
    const int N = p.N, M = p.M, nb = (M + 4) >> 2, Npad = (N + 3) & ~3;
    const int64_t n = p.n_traj;
    const int d = p.draws[i];
    const int L = (st == SSA_TRAJ_OK) ? d - 1 : d;  // index of the last visited state
    const bool draw_last = st == SSA_TRAJ_OK;
    const int K = p.K;  // kSoftK
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2w = (uint32_t)gid, c3w = (uint32_t)(gid >> 32), key0 = (uint32_t)p.seed,
                   key1 = (uint32_t)(p.seed >> 32);
    const float invT = p.invT;
    const float *gl = p.dl_dobs + i * p.dl_stride;
    const float *ckf = reinterpret_cast<const float *>(p.ckpt);
    for (int sp = lane; sp < N; sp += 32) lam[sp] = 0.0f;
    int s_hi = p.S - 1;
    int brk_next = (READOUT != SSA_READOUT_BIN && s_hi >= 0) ? p.brk_k[(int64_t)s_hi * n + i] : -1;
    constexpr bool kBin = READOUT == SSA_READOUT_BIN;
    BinSlots bslots{-1, -1};
    float d_first = 0.0f, d_last = 0.0f;
    if (kBin) bin_slots_init(bslots, p.brk_k, p.brk_tail, n, i);
    float mu = 0.0f;
    int mism = 0;
    float gq[kBinMaxObs], gk[kBinMaxObs];
    int osp[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) osp[c] = (kBin && c < p.n_obs) ? p.obs_sp[c] : 0;
    auto addx = [&](int c, float v) { lam[osp[c]] += v; };
    if (kBin) bin_grad(gq, gl, p.n_obs, p.ts, p.S, p.S);
    __syncwarp();

    for (int c = L / K; c >= 0; --c) {
        const int k0 = c * K, k1 = min(k0 + K - 1, L);
        // regenerate the segment's states: Xs[kk - k0] = X_kk
        for (int sp = lane; sp < N; sp += 32) Xs[sp] = ckf[((int64_t)c * N + sp) * n + i];
        __syncwarp();
        for (int kk = k0; kk < k1 || (kk == k1 && k1 < L); ++kk) {
            const float *Xc = Xs + (size_t)(kk - k0) * Npad;
            float E0, invZ;
            bool finite;
            warp_soft_step<false>(s_rx, s_k, s_upd, N, M, invT, kk, c2w, c3w, key0, key1, Xc, nullptr, nullptr, y, dX,
                                  E0, invZ, finite);
            if (kk < k1) {
                float *Xn = Xs + (size_t)(kk + 1 - k0) * Npad;
                for (int sp = lane; sp < N; sp += 32) Xn[sp] = __fadd_rn(Xc[sp], dX[sp]);
            } else {  // the state after the segment: the next checkpoint
                int bad = 0;
                for (int sp = lane; sp < N; sp += 32)
                    bad += __fadd_rn(Xc[sp], dX[sp]) != ckf[((int64_t)(c + 1) * N + sp) * n + i];
                mism += __reduce_add_sync(0xffffffffu, bad);
            }
            __syncwarp();
        }
        for (int k = k1; k >= k0; --k) {
            const float *Xk = Xs + (size_t)(k - k0) * Npad;
            const bool draw = (k < L) || draw_last;
            const int s_top = s_hi;
            if (kBin) {
                bin_slots_step(bslots, p.brk_k, p.brk_s, p.brk_a, p.ts, n, i, k, s_hi, d_first, d_last);
                if (s_hi < s_top) bin_grad(gk, gl, p.n_obs, p.ts, p.S, s_hi + 1);
                else {
#pragma unroll
                    for (int q = 0; q < kBinMaxObs; ++q) gk[q] = gq[q];
                }
            } else {
                while (s_hi >= 0 && brk_next == k) {
                    --s_hi;
                    brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
                }
            }
            float tau_k = 0.0f;
            if (draw) {
                float E0, invZ;
                bool finite;
                const float a0 = warp_soft_step<true>(s_rx, s_k, s_upd, N, M, invT, k, c2w, c3w, key0, key1, Xk, aj,
                                                      hj, y, dX, E0, invZ, finite);
                const float tau = waiting_time(E0, a0);
                tau_k = tau;
                float dt_dir = 0.0f, dtau_dir = 0.0f;
                if (kBin) {  // t_{k+1} ends this interval and starts the next, in the bin of gq
                    float cb = 0.0f;
#pragma unroll
                    for (int q = 0; q < kBinMaxObs; ++q)
                        if (q < p.n_obs) cb = __fmaf_rn(gq[q], dX[osp[q]], cb);
                    mu -= cb;
                }
                if (READOUT == SSA_READOUT_LINEAR) {
                    // serial on lane 0 (observed species may repeat), broadcast afterwards
                    if (lane == 0) {
                        for (int s = s_hi + 1; s <= s_top; ++s) {
                            const float alpha = p.brk_a[(int64_t)s * n + i];
                            if (alpha < 0.0f) continue;
                            float cl = 0.0f;
                            for (int o = 0; o < p.n_obs; ++o) {
                                const float g = gl[(int64_t)s * p.n_obs + o];
                                const int sp = p.obs_sp[o];
                                lam[sp] += alpha * g;
                                cl += g * dX[sp];
                            }
                            const float c_tau = __fdividef(cl, tau);
                            dt_dir -= c_tau;
                            dtau_dir -= alpha * c_tau;
                        }
                    }
                    dt_dir = __shfl_sync(0xffffffffu, dt_dir, 0);
                    dtau_dir = __shfl_sync(0xffffffffu, dtau_dir, 0);
                }
                __syncwarp();
                const float dtau = mu + dtau_dir;
                const float dLda0 = -dtau * tau / a0;
                // w_j = v_j . lambda (kept in c1 until the slots take it) and sum_j y~_j w_j
                float Wp = 0.0f;
                for (int b = lane; b < nb; b += 32) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = 4 * b + q - 1;
                        if (j < 0 || j >= M) continue;
                        const int pos = q * nb + b;
                        const int4 rx = s_rx[pos];
                        float w = 0.0f;
                        for (int e = rx.z; e < rx.w; ++e) w += (float)stoich_delta(s_st[e]) * lam[stoich_species(s_st[e])];
                        c1[pos] = w;
                        Wp += (y[pos] * invZ) * w;
                    }
                }
                const float Wbar = warp_sum(Wp);
                __syncwarp();
                // psi, dA and the reactant-slot contributions (choice path where a > 0, waiting-time path where
                // the factor is not clipped)
                for (int b = lane; b < nb; b += 32) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = 4 * b + q - 1;
                        if (j < 0 || j >= M) continue;
                        const int pos = q * nb + b;
                        const float yj = y[pos] * invZ, a = aj[pos];
                        const float psi = yj > 0.0f ? yj * (c1[pos] - Wbar) * invT : 0.0f;
                        dA[pos] += psi + dLda0 * a;
                        const float ctau = dLda0 * s_k[pos];
                        const int4 rx = s_rx[pos];
                        float v1 = 0.0f, v2 = 0.0f;
                        if (rx.x >= 0) {
                            const float x1 = Xk[rx.x];
                            if (rx.y < 0) {
                                v1 = sadj_first(x1, a, psi, x1 < 0.0f ? 0.0f : ctau);
                            } else if (rx.y == rx.x) {
                                v1 = sadj_homodimer(x1, a, hj[pos], psi, __fmul_rn(x1, x1 - 1.0f) < 0.0f ? 0.0f : ctau);
                            } else {
                                const float x2 = Xk[rx.y];
                                const float cc = __fmul_rn(x1, x2) < 0.0f ? 0.0f : ctau;
                                v1 = sadj_hetero(x1, x2, a, psi, cc);
                                v2 = sadj_hetero(x2, x1, a, psi, cc);
                            }
                        }
                        c1[pos] = v1;
                        c2[pos] = v2;
                    }
                }
                __syncwarp();
                // lambda_s += the contributions of its reactant slots, one at a time in increasing j
                for (int sp = lane; sp < N; sp += 32) {
                    float acc = lam[sp];
                    for (int e = s_inc_ptr[sp]; e < s_inc_ptr[sp + 1]; ++e) {
                        const int slot = s_inc[e];  // 2 j + reactant slot
                        acc += ((slot & 1) ? c2 : c1)[jpos(slot >> 1, nb)];
                    }
                    lam[sp] = acc;
                }
                mu += dt_dir;
            }
            __syncwarp();
            if (kBin) {
                if (lane == 0)
                    bin_state_terms(addx, d_first, d_last, gl, p.bin_prefix, p.n_obs, s_hi + 1, s_top, draw, tau_k, gq,
                                    gk);
#pragma unroll
                for (int q = 0; q < kBinMaxObs; ++q) gq[q] = gk[q];
            } else if (lane == 0) {
                for (int s = s_hi + 1; s <= s_top; ++s) {
                    float coef = 1.0f;
                    if (READOUT == SSA_READOUT_LINEAR && draw) {
                        const float alpha = p.brk_a[(int64_t)s * n + i];
                        if (alpha >= 0.0f) coef = 1.0f - alpha;
                    }
                    for (int o = 0; o < p.n_obs; ++o) lam[p.obs_sp[o]] += coef * gl[(int64_t)s * p.n_obs + o];
                }
            }
            __syncwarp();
        }
    }
    if (lane == 0 && mism) atomicAdd(p.mismatch, mism);
}

// Per-trajectory body of the warp adjoint (all 32 lanes). X, lam, aj, lj, ct, dA are this warp's buffers;
// dA accumulates over every trajectory the warp processes.
template <int READOUT>
__device__ __forceinline__ void warp_adj_body(const AdjParams &p, const int4 *s_rx, const int *s_st,
                                              const int *s_inc_ptr, const int *s_inc, const float *s_k, int *X,
                                              float *lam, float *aj, float *lj, float *ct, float *dA, const int64_t i,
                                              const int st)
{
    const int lane = threadIdx.x & 31;
    const int N = p.N, M = p.M;
    const int64_t n = p.n_traj;
    const int d = p.draws[i];
    const int L = (st == SSA_TRAJ_OK) ? d - 1 : d;
    for (int s = lane; s < N; s += 32) {
        X[s] = p.xfinal[(int64_t)s * n + i];
        lam[s] = 0.0f;
    }
    __syncwarp();
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    FwdParamsView v{s_rx, s_k, M, (M + 4) >> 2, (uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)p.seed,
                    (uint32_t)(p.seed >> 32)};
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
    constexpr bool kBin = READOUT == SSA_READOUT_BIN;
    int s_hi = p.S - 1;
    int brk_next = (!kBin && s_hi >= 0) ? p.brk_k[(int64_t)s_hi * n + i] : -1;
    // BIN readout: the recorded slots (one per state interval with edges), gq = g of the bin that contains
    // t_{k+1}, xo = X_{k+1} at the observables; every lane keeps the same copies
    BinSlots bslots{-1, -1};
    float d_first = 0.0f, d_last = 0.0f;
    float gq[kBinMaxObs], gk[kBinMaxObs];
    int osp[kBinMaxObs], xo[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) osp[c] = (kBin && c < p.n_obs) ? p.obs_sp[c] : 0;
    auto xobs = [&](int c) { return X[osp[c]]; };
    auto addx = [&](int c, float v) { lam[osp[c]] += v; };
    if (kBin) {
        bin_slots_init(bslots, p.brk_k, p.brk_tail, n, i);
        bin_grad(gq, gl, p.n_obs, p.ts, p.S, p.S);
#pragma unroll
        for (int c = 0; c < kBinMaxObs; ++c) xo[c] = c < p.n_obs ? xobs(c) : 0;
    }
    float mu = 0.0f;
    int mism = 0;
    int ck_row = L / p.K, ck_off = L - ck_row * p.K;
    // passes 2 and 3 read only shared memory, so the lanes take the 4 nb slots one at a time, 32 per round
    // (slot pos = q nb + b holds reaction 4 b + q - 1): ceil(4 nb / 32) rounds instead of ceil(nb / 32)
    // rounds of four slots (at nb = 76, 95% of the lanes busy instead of 79%; below nb = 32, up to four times
    // fewer rounds). A lane's first slot, as (q, b); it then advances by 32 slots.
    const int q_first = lane / v.nb, b_first = lane - q_first * v.nb;
    auto next_slot = [&](int &q, int &b) {
        b += 32;
        while (b >= v.nb) {
            b -= v.nb;
            ++q;
        }
    };

    for (int k = L; k >= 0; --k) {
        const bool draw = (k < L) || (st == SSA_TRAJ_OK);
        const int s_top = s_hi;
        if (kBin) {
            bin_slots_step(bslots, p.brk_k, p.brk_s, p.brk_a, p.ts, n, i, k, s_hi, d_first, d_last);
            if (s_hi < s_top) bin_grad(gk, gl, p.n_obs, p.ts, p.S, s_hi + 1);
            else {
#pragma unroll
                for (int c = 0; c < kBinMaxObs; ++c) gk[c] = gq[c];
            }
        } else {
            while (s_hi >= 0 && brk_next == k) {
                --s_hi;
                brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
            }
        }
        float tau_k = 0.0f;
        if (draw) {
            const int jk = event_at(k);
            float a0, E0, ab, Eb, lmax;
            int jb;
            warp_step_eval<true>(v, k, X, a0, E0, ab, Eb, jb, aj, lj, lmax);
            mism += (jb != jk);
            const float tau = waiting_time(E0, a0);
            tau_k = tau;
            const int4 rk = s_rx[jpos(jk, v.nb)];
            // BIN: t_{k+1} ends this interval and starts the next, in the bin of gq
            if (kBin) mu -= bin_transition(xobs, xo, gq, p.n_obs);
            float dt_dir = 0.0f, dtau_dir = 0.0f;
            if (READOUT == SSA_READOUT_LINEAR) {
                // serial on lane 0 (observed species may repeat), broadcast afterwards
                if (lane == 0) {
                    for (int s = s_hi + 1; s <= s_top; ++s) {
                        const float alpha = p.brk_a[(int64_t)s * n + i];
                        if (alpha < 0.0f) continue;
                        float c = 0.0f;
                        for (int o = 0; o < p.n_obs; ++o) {
                            const float g = gl[(int64_t)s * p.n_obs + o];
                            const int sp = p.obs_sp[o];
                            lam[sp] += alpha * g;
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
                dt_dir = __shfl_sync(0xffffffffu, dt_dir, 0);
                dtau_dir = __shfl_sync(0xffffffffu, dtau_dir, 0);
            }
            __syncwarp();
            const float dtau = mu + dtau_dir;
            const float dLda0 = -dtau * tau / a0;
            // pass 2: weights and w_j over this lane's reactions
            float Zp = 0.0f, Wp = 0.0f;
            for (int pos = lane, q = q_first, b = b_first; pos < 4 * v.nb; pos += 32, next_slot(q, b)) {
                {
                    // predicated rather than branched (the lanes hold reactions with 1 to 4 stoichiometric
                    // entries); the slots of j = -1 and j >= M hold no entries, and their weight is 0
                    const int j = 4 * b + q - 1;
                    const bool live = j >= 0 && j < M;
                    const float l = live ? lj[pos] : -CUDART_INF_F;
                    const float qv = l == -CUDART_INF_F ? 0.0f : exp2f((l - lmax) * invT);
                    const int4 rx = s_rx[pos];
                    float w = 0.0f;
                    if (rx.w - rx.z <= 4) {
#pragma unroll
                        for (int t = 0; t < 4; ++t)
                            if (rx.z + t < rx.w) {
                                const int se = s_st[rx.z + t];
                                w += (float)stoich_delta(se) * lam[stoich_species(se)];
                            }
                    } else {
                        for (int e = rx.z; e < rx.w; ++e) w += (float)stoich_delta(s_st[e]) * lam[stoich_species(s_st[e])];
                    }
                    if (live) {
                        lj[pos] = qv;
                        ct[pos] = w;  // kept for pass 3, which overwrites the slot afterwards
                    }
                    Zp += qv;  // + 0 where qv = 0: the same bits
                    Wp += qv > 0.0f ? qv * w : 0.0f;
                }
            }
            const float Z = warp_sum(Zp), Wq = warp_sum(Wp);
            const float invZ = __fdividef(1.0f, Z), Wbar = Wq * invZ;
            // pass 3: per-reaction adjoints and reactant-slot contributions to the state adjoint
            for (int pos = lane, q = q_first, b = b_first; pos < 4 * v.nb; pos += 32, next_slot(q, b)) {
                {
                    const int j = 4 * b + q - 1;
                    const bool live = j >= 0 && j < M;  // predicated: the other slots write zero contributions
                    const int4 rx = s_rx[pos];
                    const float qv = live ? lj[pos] : 0.0f, a = live ? aj[pos] : 0.0f;
                    float psi = 0.0f;
                    if (qv > 0.0f) psi = qv * invZ * (ct[pos] - Wbar) * invT;  // w_j from pass 2
                    if (live) dA[pos] += psi + dLda0 * a;
                    // d log a_j / dX and d a_j / dX of each reactant slot, formed with selects (the lanes hold
                    // reactions of different orders): first order is the hetero form with x2 = 1
                    const bool has1 = rx.x >= 0, has2 = rx.y >= 0, homo = has2 && rx.y == rx.x;
                    const float c_tau = dLda0 * s_k[pos];
                    const float x1 = int2f(X[has1 ? rx.x : 0]);
                    const float xr2 = int2f(X[has2 ? rx.y : 0]);
                    const float x2 = (has2 && !homo) ? xr2 : 1.0f;
                    const float dh = x1 - 0.5f;
                    const float num = homo ? psi * dh : psi;
                    const float den = homo ? mass_action_h_sel(rx, X) : x1;
                    const float t1 = a > 0.0f ? __fdividef(num, den) : 0.0f;
                    const float c1 = has1 ? t1 + c_tau * (homo ? dh : x2) : 0.0f;
                    const float c2 = (has2 && !homo) ? (a > 0.0f ? __fdividef(psi, xr2) : 0.0f) + c_tau * x1 : 0.0f;
                    // the soft weight and w_j of this reaction are spent: its slots take the contributions
                    lj[pos] = c1;  // reactant slot 0
                    ct[pos] = c2;  // reactant slot 1
                }
            }
            __syncwarp();
            // lambda_s += sum of the reactant-slot contributions of species s. With N <= 32 each species
            // gets g = 32 / 2^ceil(log2 N) lanes that stride over its incidence list with four
            // accumulators and combine by a butterfly inside the group; with more species each lane takes
            // whole species. The order is fixed, so the result is the same on every run.
            int pow2 = 1;
            while (pow2 < N && pow2 < 32) pow2 <<= 1;
            const int gsz = N <= 32 ? 32 / pow2 : 1;
            for (int base = 0; base < N; base += 32 / gsz) {
                const int sp = base + lane / gsz, r = lane % gsz;
                float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, c3 = 0.0f;
                if (sp < N) {
                    const int e1 = s_inc_ptr[sp + 1];
                    int e = s_inc_ptr[sp] + r;
                    auto slot_val = [&](int ee) {
                        const int slot = s_inc[ee];  // 2 j + reactant slot
                        return ((slot & 1) ? ct : lj)[jpos(slot >> 1, v.nb)];
                    };
                    for (; e + 3 * gsz < e1; e += 4 * gsz) {
                        c0 += slot_val(e);
                        c1 += slot_val(e + gsz);
                        c2 += slot_val(e + 2 * gsz);
                        c3 += slot_val(e + 3 * gsz);
                    }
                    for (; e < e1; e += gsz) c0 += slot_val(e);
                }
                float acc = (c0 + c1) + (c2 + c3);
                for (int off = gsz >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if (r == 0 && sp < N) lam[sp] += acc;
            }
            mu += dt_dir;
        }
        __syncwarp();
        if (kBin) {
            if (lane == 0)
                bin_state_terms(addx, d_first, d_last, gl, p.bin_prefix, p.n_obs, s_hi + 1, s_top, draw, tau_k, gq, gk);
#pragma unroll
            for (int c = 0; c < kBinMaxObs; ++c) {
                gq[c] = gk[c];
                if (c < p.n_obs) xo[c] = xobs(c);
            }
        } else if (lane == 0) {
            for (int s = s_hi + 1; s <= s_top; ++s) {
                float coef = 1.0f;
                if (READOUT == SSA_READOUT_LINEAR && draw) {
                    const float alpha = p.brk_a[(int64_t)s * n + i];
                    if (alpha >= 0.0f) coef = 1.0f - alpha;
                }
                for (int o = 0; o < p.n_obs; ++o) lam[p.obs_sp[o]] += coef * gl[(int64_t)s * p.n_obs + o];
            }
        }
        if (ck_off == 0) {
            const int *ck = p.ckpt + (int64_t)ck_row * N * n + i;
            int bad = 0;
            for (int s = lane; s < N; s += 32) bad += (ck[(int64_t)s * n] != X[s]);
            mism += __reduce_add_sync(0xffffffffu, bad);
            --ck_row;
            ck_off = p.K;
        }
        --ck_off;
        __syncwarp();
        if (k > 0) {
            const int4 rp = s_rx[jpos(event_at(k - 1), v.nb)];
            for (int e = rp.z + lane; e < rp.w; e += 32) X[stoich_species(s_st[e])] -= stoich_delta(s_st[e]);
        }
        __syncwarp();
    }
    if (lane == 0 && mism) atomicAdd(p.mismatch, mism);
}

}  // namespace ssa
