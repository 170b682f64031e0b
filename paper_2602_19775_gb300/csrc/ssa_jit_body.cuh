// ssa_jit_body.cuh -- thread-per-trajectory forward and straight-through adjoint specialised to one
// network at run time (arXiv 2602.19775, Section 2, Section 3.2, Eqs. 3, 5, 6, 7, Section 3.1).
//
// This file is compiled by NVRTC, not by nvcc: the library prepends a generated prologue that
// defines JN (species), JM (reactions) and the network hooks
//     jit_props(X, k, a, h)       h_j(X) and a_j = k_j h_j for every reaction, in reaction order
//     jit_check(X, jb)            status of applying v_jb to X (negative count / overflow)
//     jit_apply(X, jb), jit_unapply(X, jb)
//     jit_dv(jb, sp)              component sp of v_jb
//     jit_w(lam, w)               w_j = v_j . lambda for every reaction
//     jit_state_adj(X, a, h, psi, ctau, lam)   the state adjoint of every reaction, in order
// with the reactant indices and stoichiometry written into the code as constants. Counts and the
// state adjoint then live in registers and every table lookup disappears. The arithmetic is the
// generic thread kernels' (same helpers from ssa_device.cuh, same order), so a specialised run
// reproduces the generic run's trajectories bit for bit. A third forward runs the plain direct method
// (Section 2) for comparison. Compiled with SSA_JIT_SOFT defined, the same text yields the soft-forward
// kernels (Eq. 4) and their adjoint instead.

namespace ssa {

__device__ __forceinline__ int jit_xsel(const int (&X)[JN], int sp)
{
    int v = 0;
#pragma unroll
    for (int s = 0; s < JN; ++s) v = (s == sp) ? X[s] : v;
    return v;
}

__device__ __forceinline__ void jit_lam_add(float (&lam)[JN], int sp, float v)
{
#pragma unroll
    for (int s = 0; s < JN; ++s)
        if (s == sp) lam[s] += v;
}

// Compensated accumulation for walks of ~1e6 steps (the wide-range adjoint): hi + lo carries the running sum
// to about twice binary32's precision. Each step adds a small increment to a state adjoint that it changes by
// ~1e-4 of its size, so a binary32 sum would drop most of the increment's bits every step; emulating that
// rounding in the FP64 oracle moves its full-horizon gradient by ~1e-3. (Knuth's two-sum: the rounding error
// of hi + v is exact in binary32.)
__device__ __forceinline__ void acc2(float &hi, float &lo, float v)
{
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// hi <- the binary32 sum of hi + lo, lo <- its remainder (fast two-sum; |lo| is far below |hi|)
__device__ __forceinline__ void fold2(float &hi, float &lo)
{
    const float s = __fadd_rn(hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
}

__device__ __forceinline__ void jit_lam_add2(float (&lam)[JN], float (&lo)[JN], int sp, float v)
{
#pragma unroll
    for (int s = 0; s < JN; ++s)
        if (s == sp) acc2(lam[s], lo[s], v);
}

// BIN readout state of a forward: cleared integrals, observed species (0 where the list is invalid)
__device__ __forceinline__ void jit_bin_init(const FwdParams &p, bool bad_obs, float (&bacc)[kBinMaxObs],
                                             int (&osp)[kBinMaxObs])
{
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) {
        bacc[c] = 0.0f;
        osp[c] = (c < p.n_obs && !bad_obs) ? p.obs_sp[c] : 0;
    }
}

// Coalesced sample stores. A trajectory's samples are one row of obs [n_traj][S][n_obs], written one at a
// time as its clock passes them, so a warp's per-thread stores land in 32 different rows. Instead each
// thread collects a window of W = 16 / n_obs consecutive samples (n_obs <= 4) in its row of a per-block
// shared buffer; at the top of every step the warp's active lanes copy the completed windows together, two
// windows per store instruction (consecutive words of two rows). A lane whose window fills
// while it still has samples to write in the same step, and every lane after its last step, writes its own
// window. The values and their places are those of direct stores.
constexpr int kJitFwdBlock = 64;    // threads per block of the specialised forwards
constexpr int kStageWords = 16;     // words of a thread's sample window

struct SampleStage {
    uint32_t *row;   // this thread's window in shared memory
    uint32_t *out;   // obs_out as 32-bit words
    int64_t base;    // first word of this trajectory's row
    int n_obs, W, S;
    int lo, cnt;     // the window holds samples lo .. lo + cnt - 1
    bool ready;      // complete and not yet copied
};

__device__ __forceinline__ void stage_own_flush(SampleStage &g)
{
    const int words = g.cnt * g.n_obs;
    const int64_t w0 = g.base + (int64_t)g.lo * g.n_obs;
    uint32_t *dst = g.out + w0;
    if (((reinterpret_cast<uintptr_t>(dst) & 7) | (words & 1)) == 0) {  // 8-byte stores when aligned
        for (int q = 0; q < words; q += 2)
            *reinterpret_cast<uint2 *>(dst + q) = *reinterpret_cast<const uint2 *>(g.row + q);
    } else {
        for (int q = 0; q < words; ++q) dst[q] = g.row[q];
    }
    g.lo += g.cnt;
    g.cnt = 0;
    g.ready = false;
}

// one sample s (the next in order) of n_obs values
template <class VAL>
__device__ __forceinline__ void stage_put(SampleStage &g, int s, const VAL &val)
{
    if (g.ready) stage_own_flush(g);  // a second window completes within one step
    uint32_t *w = g.row + g.cnt * g.n_obs;
    for (int c = 0; c < g.n_obs; ++c) w[c] = val(c);
    ++g.cnt;
    if (g.cnt == g.W || s + 1 == g.S) g.ready = true;
}

// the warp's active lanes copy every completed window, two at a time
__device__ __forceinline__ void stage_warp_flush(SampleStage &g, const uint32_t *s_stage)
{
    const unsigned m = __activemask();
    unsigned rd = __ballot_sync(m, g.ready);
    if (!rd) return;
    const int lane = threadIdx.x & 31;
    const int first = threadIdx.x & ~31;
    const int rank = __popc(m & ((1u << lane) - 1u)), nm = __popc(m);
    const int64_t dst = g.base + (int64_t)g.lo * g.n_obs;
    const int words = g.cnt * g.n_obs;
    __syncwarp(m);
    while (rd) {
        const int a = __ffs(rd) - 1;
        rd &= rd - 1;
        int b = -1;
        if (rd) {
            b = __ffs(rd) - 1;
            rd &= rd - 1;
        }
        const long long da = __shfl_sync(m, (long long)dst, a);
        const int wa = __shfl_sync(m, words, a);
        long long db = 0;
        int wb = 0;
        if (b >= 0) {
            db = __shfl_sync(m, (long long)dst, b);
            wb = __shfl_sync(m, words, b);
        }
        // the words of window a, then of window b, shared out over the participating lanes in the order of
        // their lane numbers (lanes that have left the step loop take no part): one store instruction when all
        // 32 lanes take part, a few otherwise
        for (int pw = rank; pw < wa + wb; pw += nm) {
            const bool in_a = pw < wa;
            const int q = in_a ? pw : pw - wa;
            g.out[(in_a ? da : db) + q] = s_stage[(first + (in_a ? a : b)) * kStageWords + q];
        }
    }
    __syncwarp(m);
    if (g.ready) {
        g.lo += g.cnt;
        g.cnt = 0;
        g.ready = false;
    }
}

template <int READOUT, bool RECORD>
__device__ __forceinline__ void jit_fwd(const FwdParams &p)
{
    __shared__ __align__(16) uint32_t s_stage[kJitFwdBlock * kStageWords];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_traj) return;
    const int64_t n = p.n_traj;
    float kr[JM];
#pragma unroll
    for (int j = 0; j < JM; ++j) kr[j] = p.k_rates[j];

    const int *x0 = p.x0 + (p.x0_per_traj ? i * JN : 0);
    const bool bad_obs = (*p.flag & kErrBadObs) != 0;
    bool bad_input = (*p.flag & (kErrBadSamples | kErrBadObs)) != 0;
    int X[JN];
#pragma unroll
    for (int s = 0; s < JN; ++s) {
        X[s] = x0[s];
        bad_input |= X[s] < 0;
    }
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32);
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);

    double t = 0.0;
    int s = 0;
    double thr = p.S > 0 ? p.ts[0] : p.t_end;
    int status = bad_input ? SSA_TRAJ_BAD_INPUT : SSA_TRAJ_OK;
    int k = 0, draws = 0;
    int ck_left = p.K, ck_row = 0;
    uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    constexpr int NQ = JM + 1;
    float E[NQ], En[NQ];
    step_noise<NQ>(E, 0u, c2, c3, key0, key1);
    float bacc[kBinMaxObs];
    BinRuns bruns;
    bin_runs_init(bruns);
    int osp[kBinMaxObs];
    jit_bin_init(p, bad_obs, bacc, osp);
    auto xobs = [&](int c) { return jit_xsel(X, osp[c]); };
    const bool staged = READOUT != SSA_READOUT_BIN && p.n_obs >= 1 && p.n_obs <= 4 && blockDim.x <= kJitFwdBlock;
    SampleStage stg{s_stage + threadIdx.x * kStageWords, static_cast<uint32_t *>(p.obs_out), i * p.S * p.n_obs,
                    p.n_obs, staged ? kStageWords / p.n_obs : 1, p.S, 0, 0, false};

    while (!bad_input) {
        if (staged) stage_warp_flush(stg, s_stage);
        if (k >= p.max_steps) { status = SSA_TRAJ_STEP_CAP; break; }
        step_noise<NQ>(En, (uint32_t)(k + 1), c2, c3, key0, key1);  // next step, state-independent
        float a[JM], h[JM];
        jit_props(X, kr, a, h);
        float a0 = 0.0f, ab = 0.0f, Eb = 1.0f;
        int jb = -1;
        const float E0 = E[0];
#pragma unroll
        for (int j = 0; j < JM; ++j) {
            a0 = __fadd_rn(a0, a[j]);
            race(a[j], E[j + 1], j, ab, Eb, jb);
        }
        if (!(a0 < CUDART_INF_F)) { status = SSA_TRAJ_BAD_RATE; break; }
        if (a0 == 0.0f) { status = SSA_TRAJ_ABSORBED; break; }
        if (jb < 0) { status = SSA_TRAJ_BAD_RATE; break; }
        const float tau = waiting_time(E0, a0);
        const double t_next = t + f2d_pos(tau);
        const bool slow = gt_nonneg(t_next, thr);
        const bool cross = slow && gt_nonneg(t_next, p.t_end);
        if (!cross) status = jit_check(X, jb);
        if (RECORD) {
            e0 = __funnelshift_r(e0, e1, 16);
            e1 = __funnelshift_r(e1, e2, 16);
            e2 = __funnelshift_r(e2, e3, 16);
            e3 = (e3 >> 16) | ((uint32_t)jb << 16);
            if ((k & 7) == 7) p.ev[(int64_t)(k >> 3) * n + i] = make_uint4(e0, e1, e2, e3);
        }
        draws = k + 1;
        if (status != SSA_TRAJ_OK) break;
        if (slow) {
            const int s_first = s;
            if constexpr (READOUT == SSA_READOUT_BIN) {
                s = bin_edges<RECORD>(p, i, s, t, t_next, k, bacc, xobs, bruns);
            } else {
                while (s < p.S && gt_nonneg(t_next, p.ts[s])) {
                    if (READOUT == SSA_READOUT_HOLD) {
                        if (staged) {
                            stage_put(stg, s, [&](int c) { return (uint32_t)jit_xsel(X, p.obs_sp[c]); });
                        } else {
                            int *o = static_cast<int *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                            for (int c = 0; c < p.n_obs; ++c) o[c] = jit_xsel(X, p.obs_sp[c]);
                        }
                    } else {
                        const float alpha = __fdiv_rn(d2f_nonneg(p.ts[s] - t), tau);
                        auto lin = [&](int c) {
                            const int sp = p.obs_sp[c];
                            return __fmaf_rn(alpha, (float)jit_dv(jb, sp), (float)jit_xsel(X, sp));
                        };
                        if (staged) {
                            stage_put(stg, s, [&](int c) { return __float_as_uint(lin(c)); });
                        } else {
                            float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                            for (int c = 0; c < p.n_obs; ++c) o[c] = lin(c);
                        }
                        if (RECORD) p.brk_a[(int64_t)s * n + i] = alpha;
                    }
                    if (RECORD) p.brk_k[(int64_t)s * n + i] = k;
                    ++s;
                }
            }
            if (READOUT == SSA_READOUT_BIN && !cross && s > s_first)
                bin_accumulate(bacc, xobs, p.n_obs, d2f_nonneg(t_next - p.ts[s - 1]));
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;  // the crossing draw is made but not applied
        } else if (READOUT == SSA_READOUT_BIN) {
            bin_accumulate(bacc, xobs, p.n_obs, tau);
        }
        jit_apply(X, jb);
        t = t_next;
        ++k;
        if (RECORD && --ck_left == 0) {
            ck_left = p.K;
            ++ck_row;
            int *ck = p.ckpt + (int64_t)ck_row * JN * n + i;
#pragma unroll
            for (int sp = 0; sp < JN; ++sp) ck[(int64_t)sp * n] = X[sp];
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) E[q] = En[q];
    }
    if constexpr (READOUT == SSA_READOUT_BIN) bin_tail<RECORD>(p, i, s, t, k, bacc, xobs, bad_obs, bruns);
    for (; READOUT != SSA_READOUT_BIN && s < p.S; ++s) {
        if (READOUT == SSA_READOUT_HOLD) {
            if (staged) {
                stage_put(stg, s, [&](int c) { return (uint32_t)(bad_obs ? 0 : jit_xsel(X, p.obs_sp[c])); });
            } else {
                int *o = static_cast<int *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                for (int c = 0; c < p.n_obs; ++c) o[c] = bad_obs ? 0 : jit_xsel(X, p.obs_sp[c]);
            }
        } else {
            if (staged) {
                stage_put(stg, s, [&](int c) { return __float_as_uint(bad_obs ? 0.0f : (float)jit_xsel(X, p.obs_sp[c])); });
            } else {
                float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                for (int c = 0; c < p.n_obs; ++c) o[c] = bad_obs ? 0.0f : (float)jit_xsel(X, p.obs_sp[c]);
            }
            if (RECORD) p.brk_a[(int64_t)s * n + i] = -1.0f;
        }
        if (RECORD) p.brk_k[(int64_t)s * n + i] = k;
    }
    if (staged && stg.cnt > 0) stage_own_flush(stg);  // the last window, by the thread itself
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
#pragma unroll
        for (int sp = 0; sp < JN; ++sp) {
            p.xfinal[(int64_t)sp * n + i] = X[sp];
            p.ckpt[(int64_t)sp * n + i] = x0[sp];  // checkpoint 0 = X_0
        }
    }
}

// The plain direct method (Section 2), forward only: per step one Philox block gives E_0 = -ln u_0
// for the waiting time and u_1 for the choice, the first reaction j (in reaction order) whose
// cumulative propensity exceeds u_1 a0 (all in binary32, the cumulative sum in the order of a0).
// Everything else -- clock, samples, range checks, update -- is the Gumbel-max forward's.
template <int READOUT>
__device__ __forceinline__ void jit_fwd_direct(const FwdParams &p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_traj) return;
    float kr[JM];
#pragma unroll
    for (int j = 0; j < JM; ++j) kr[j] = p.k_rates[j];
    const int *x0 = p.x0 + (p.x0_per_traj ? i * JN : 0);
    const bool bad_obs = (*p.flag & kErrBadObs) != 0;
    bool bad_input = (*p.flag & (kErrBadSamples | kErrBadObs)) != 0;
    int X[JN];
#pragma unroll
    for (int s = 0; s < JN; ++s) {
        X[s] = x0[s];
        bad_input |= X[s] < 0;
    }
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32);
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    double t = 0.0;
    int s = 0;
    double thr = p.S > 0 ? p.ts[0] : p.t_end;
    int status = bad_input ? SSA_TRAJ_BAD_INPUT : SSA_TRAJ_OK;
    int k = 0, draws = 0;
    uint4 r = philox4x32_10(make_uint4(0u, 0u, c2, c3), key0, key1);
    float E0 = neg_log_unit(u01(r.x)), U1 = u01(r.y);
    float bacc[kBinMaxObs];
    BinRuns bruns;
    bin_runs_init(bruns);
    int osp[kBinMaxObs];
    jit_bin_init(p, bad_obs, bacc, osp);
    auto xobs = [&](int c) { return jit_xsel(X, osp[c]); };
    while (!bad_input) {
        if (k >= p.max_steps) { status = SSA_TRAJ_STEP_CAP; break; }
        r = philox4x32_10(make_uint4(0u, (uint32_t)(k + 1), c2, c3), key0, key1);  // next step
        float a[JM], h[JM];
        jit_props(X, kr, a, h);
        float a0 = 0.0f;
#pragma unroll
        for (int j = 0; j < JM; ++j) a0 = __fadd_rn(a0, a[j]);
        if (!(a0 < CUDART_INF_F)) { status = SSA_TRAJ_BAD_RATE; break; }
        if (a0 == 0.0f) { status = SSA_TRAJ_ABSORBED; break; }
        const float target = __fmul_rn(U1, a0);
        float cum = 0.0f;
        int jb = -1, last = -1;
#pragma unroll
        for (int j = 0; j < JM; ++j) {
            if (a[j] > 0.0f) {
                last = j;
                cum = __fadd_rn(cum, a[j]);
                if (jb < 0 && cum > target) jb = j;
            }
        }
        if (jb < 0) jb = last;  // u_1 a0 rounded up to a0: the last active reaction
        if (jb < 0) { status = SSA_TRAJ_BAD_RATE; break; }
        const float tau = waiting_time(E0, a0);
        const double t_next = t + f2d_pos(tau);
        const bool slow = gt_nonneg(t_next, thr);
        const bool cross = slow && gt_nonneg(t_next, p.t_end);
        if (!cross) status = jit_check(X, jb);
        draws = k + 1;
        if (status != SSA_TRAJ_OK) break;
        if (slow) {
            const int s_first = s;
            if constexpr (READOUT == SSA_READOUT_BIN) {
                s = bin_edges<false>(p, i, s, t, t_next, k, bacc, xobs, bruns);
            } else {
                while (s < p.S && gt_nonneg(t_next, p.ts[s])) {
                    if (READOUT == SSA_READOUT_HOLD) {
                        int *o = static_cast<int *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                        for (int c = 0; c < p.n_obs; ++c) o[c] = jit_xsel(X, p.obs_sp[c]);
                    } else {
                        const float alpha = __fdiv_rn(d2f_nonneg(p.ts[s] - t), tau);
                        float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
                        for (int c = 0; c < p.n_obs; ++c) {
                            const int sp = p.obs_sp[c];
                            o[c] = __fmaf_rn(alpha, (float)jit_dv(jb, sp), (float)jit_xsel(X, sp));
                        }
                    }
                    ++s;
                }
            }
            if (READOUT == SSA_READOUT_BIN && !cross && s > s_first)
                bin_accumulate(bacc, xobs, p.n_obs, d2f_nonneg(t_next - p.ts[s - 1]));
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;
        } else if (READOUT == SSA_READOUT_BIN) {
            bin_accumulate(bacc, xobs, p.n_obs, tau);
        }
        jit_apply(X, jb);
        t = t_next;
        ++k;
        E0 = neg_log_unit(u01(r.x));
        U1 = u01(r.y);
    }
    if constexpr (READOUT == SSA_READOUT_BIN) bin_tail<false>(p, i, s, t, k, bacc, xobs, bad_obs, bruns);
    for (; READOUT != SSA_READOUT_BIN && s < p.S; ++s) {
        if (READOUT == SSA_READOUT_HOLD) {
            int *o = static_cast<int *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
            for (int c = 0; c < p.n_obs; ++c) o[c] = bad_obs ? 0 : jit_xsel(X, p.obs_sp[c]);
        } else {
            float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
            for (int c = 0; c < p.n_obs; ++c) o[c] = bad_obs ? 0.0f : (float)jit_xsel(X, p.obs_sp[c]);
        }
    }
    p.draws[i] = draws;
    p.status[i] = status;
}

// Per-trajectory adjoint; returns the trajectory's per-reaction adjoints in dAr.
//
// NT temperatures at once (NT > 1): the walk, the regenerated noise, the propensities, the race check and
// the log keys do not depend on T, so they are computed once per step; each temperature t keeps its own
// lambda, mu and dAr[t] and runs the T-dependent part (soft weights, psi, the state adjoint) with invT_t,
// in the same operation order as a single-temperature walk, so every dAr[t] equals that walk's to binary32
// rounding (the two kernels may contract products into fused multiply-adds differently).
//
// WIDE (long trajectories, NT = 1): the adjoint is linear in the upstream gradient, and over ~1e6 draws the
// straight-through recursion can grow it far beyond the binary32 range (on the oscillator to ~1e73 at
// t = 400 in binary64). The walk then keeps lambda, mu and dAr as binary32 values times 2^sc, one
// exponent per trajectory: at every checkpoint boundary, when the largest magnitude exceeds 2^32, all of
// them are multiplied by 2^-e (exact) and sc grows by e; each upstream-gradient term enters multiplied by
// 2^-sc. The trajectory's result is dAr 2^sc. With sc = 0 the arithmetic is the plain walk's bit for bit.
template <int READOUT, bool WIDE = false, int NT = 1>
__device__ __forceinline__ void jit_adj_traj(const AdjParams &p, const float (&kr)[JM], const int64_t i, const int st,
                                             float (&dAr)[NT][JM], int &sc)
{
    static_assert(!WIDE || NT == 1, "the wide-range walk takes one temperature");
    sc = 0;
    float inj = 1.0f;  // 2^-sc: the factor of every upstream-gradient term
    const int64_t n = p.n_traj;
    const int d = p.draws[i];
    const int L = (st == SSA_TRAJ_OK) ? d - 1 : d;  // index of the last visited state
    int X[JN];
    float lam[NT][JN];
    float lam_lo[JN], mu_lo = 0.0f;  // WIDE: compensation terms of lam[0] and mu[0]
#pragma unroll
    for (int s = 0; s < JN; ++s) {
        X[s] = p.xfinal[(int64_t)s * n + i];
        lam_lo[s] = 0.0f;
#pragma unroll
        for (int t = 0; t < NT; ++t) lam[t][s] = 0.0f;
    }
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32);
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    float invT[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) invT[t] = NT == 1 ? p.invT : p.invT_multi[t];
    const float *gl = p.dl_dobs + i * p.dl_stride;

    // The walk's loads are issued well before their use (a load consumed where it is issued stalls the
    // trajectory for the memory latency): the log row below the current one, the brackets of the next two
    // samples and the weight of the next, the next checkpoint.
    int row_cached = -1;
    uint4 row = make_uint4(0, 0, 0, 0), row_below = row;
    auto event_at = [&](int kk) -> int {
        const int r = kk >> 3;
        if (r != row_cached) {
            row = (r == row_cached - 1) ? row_below : p.ev[(int64_t)r * n + i];
            row_cached = r;
            if (r > 0) row_below = p.ev[(int64_t)(r - 1) * n + i];
        }
        const int slot = kk & 7;
        const uint32_t w = word_of(row, slot >> 1);
        return (slot & 1) ? (int)(w >> 16) : (int)(w & 0xffff);
    };

    int s_hi = p.S - 1;
    auto brk_k_at = [&](int s) { return (READOUT != SSA_READOUT_BIN && s >= 0) ? p.brk_k[(int64_t)s * n + i] : -1; };
    auto brk_a_at = [&](int s) { return (READOUT == SSA_READOUT_LINEAR && s >= 0) ? p.brk_a[(int64_t)s * n + i] : 0.0f; };
    int brk_next = brk_k_at(s_hi), brk_next2 = brk_k_at(s_hi - 1);
    float a_next = brk_a_at(s_hi), a_top = 0.0f;  // the weights of samples s_hi and s_top
    // BIN: one recorded slot per state interval that holds edges
    BinSlots bslots{-1, -1};
    float d_first = 0.0f, d_last = 0.0f;
    if (READOUT == SSA_READOUT_BIN) bin_slots_init(bslots, p.brk_k, p.brk_tail, n, i);
    float mu[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) mu[t] = 0.0f;
    int mism = 0;
    int ck_row = L / p.K, ck_off = L - ck_row * p.K;  // checkpoint c holds X_{cK}
    int ckv[JN];
#pragma unroll
    for (int s = 0; s < JN; ++s) ckv[s] = p.ckpt[((int64_t)ck_row * JN + s) * n + i];

    constexpr int NQ = JM + 1;
    float E[NQ], En[NQ];
    const bool draw_last = st == SSA_TRAJ_OK;
    step_noise<NQ>(E, (uint32_t)(draw_last ? L : (L > 0 ? L - 1 : 0)), c2, c3, key0, key1);

    // BIN readout (NT = 1): gq = g of the bin that contains t_{k+1}, xo = X_{k+1} at the observables
    constexpr bool kBin = READOUT == SSA_READOUT_BIN;
    static_assert(!kBin || NT == 1, "the bin readout's adjoint takes one temperature");
    float gq[kBinMaxObs], gk[kBinMaxObs];
    int osp[kBinMaxObs], xo[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) osp[c] = (kBin && c < p.n_obs) ? p.obs_sp[c] : 0;
    auto xobs = [&](int c) { return jit_xsel(X, osp[c]); };
    auto addx = [&](int c, float v) { jit_lam_add(lam[0], osp[c], v); };
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
        } else if (s_hi >= 0 && brk_next == k) {
            a_top = a_next;
            do {
                --s_hi;
                brk_next = brk_next2;
                brk_next2 = brk_k_at(s_hi - 1);
            } while (s_hi >= 0 && brk_next == k);
            a_next = brk_a_at(s_hi);
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
            if (k > 0) step_noise<NQ>(En, (uint32_t)(k - 1), c2, c3, key0, key1);  // prefetch
            float a[JM], h[JM], lr[JM];
            jit_props(X, kr, a, h);
            float a0 = 0.0f, ab = 0.0f, Eb = 1.0f, lmax = -CUDART_INF_F;
            int jb = -1;
            const float E0 = E[0];
            // pass 1: the forward's a0 and race, bit for bit; log2 keys
#pragma unroll
            for (int j = 0; j < JM; ++j) {
                a0 = __fadd_rn(a0, a[j]);
                race(a[j], E[j + 1], j, ab, Eb, jb);
                lr[j] = a[j] > 0.0f ? __log2f(a[j]) - __log2f(E[j + 1]) : -CUDART_INF_F;
                lmax = fmaxf(lmax, lr[j]);
            }
            mism += (jb != jk);
            // The walk's divisions by a0 (tau = E0/a0 and d tau/d a0 = -tau/a0) take one approximate
            // reciprocal per step, accurate to 2 ulp where a0 s lies in [2^-126, 2^126]: the power of two s
            // puts it there. They only enter the gradient (the clock is the forward's), and without the IEEE
            // division's slow-path branches the step is one block of straight-line code.
            const float sc_a0 = a0 < 0x1p-126f ? 0x1p24f : (a0 > 0x1p126f ? 0x1p-24f : 1.0f);
            const float ra0 = __fdividef(1.0f, a0 * sc_a0);
            const float tau = (E0 * sc_a0) * ra0;
            tau_k = tau;
            // BIN: t_{k+1} ends this interval and starts the next, in the bin of gq
            if (kBin) mu[0] -= bin_transition(xobs, xo, gq, p.n_obs);
            // readout terms that involve X_{k+1} and the clock (LINEAR interpolation)
            float dt_dir = 0.0f, dtau_dir = 0.0f;
            if (READOUT == SSA_READOUT_LINEAR) {
                for (int s = s_hi + 1; s <= s_top; ++s) {
                    const float alpha = s == s_top ? a_top : p.brk_a[(int64_t)s * n + i];
                    if (alpha < 0.0f) continue;
                    float c = 0.0f;
                    for (int o = 0; o < p.n_obs; ++o) {
                        const float g = WIDE ? gl[(int64_t)s * p.n_obs + o] * inj : gl[(int64_t)s * p.n_obs + o];
                        const int sp = p.obs_sp[o];
                        if (WIDE) jit_lam_add2(lam[0], lam_lo, sp, alpha * g);
                        else {
#pragma unroll
                            for (int t = 0; t < NT; ++t) jit_lam_add(lam[t], sp, alpha * g);
                        }
                        c += g * (float)jit_dv(jk, sp);
                    }
                    const float c_tau = __fdividef(c, tau);
                    dt_dir -= c_tau;
                    dtau_dir -= alpha * c_tau;
                }
            }
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const float dtau = WIDE ? (mu[t] + dtau_dir) + mu_lo : mu[t] + dtau_dir;
                const float dLda0 = ((-dtau * tau) * sc_a0) * ra0;
                // pass 2: soft-sample weights y~_j ~ exp2((l_j - l_max)/T) and W = sum y~ w
                float wr[JM], qr[JM];
                jit_w(lam[t], wr);
                float Z = 0.0f, Wq = 0.0f;
#pragma unroll
                for (int j = 0; j < JM; ++j) {
                    const float q = lr[j] == -CUDART_INF_F ? 0.0f : exp2f((lr[j] - lmax) * invT[t]);
                    qr[j] = q;
                    Z += q;
                    Wq += q * wr[j];
                }
                const float invZ = __fdividef(1.0f, Z), Wbar = Wq * invZ;
                // pass 3: per-reaction adjoints, then the state adjoint of every reaction in order
                float psi[JM], ctau[JM];
#pragma unroll
                for (int j = 0; j < JM; ++j) {
                    psi[j] = qr[j] > 0.0f ? qr[j] * invZ * (wr[j] - Wbar) * invT[t] : 0.0f;
                    dAr[t][j] += psi[j] + dLda0 * a[j];
                    ctau[j] = dLda0 * kr[j];
                }
                if (WIDE) {
                    // this step's state-adjoint increment in binary32, then added to the compensated sum
                    float dl[JN];
#pragma unroll
                    for (int s = 0; s < JN; ++s) dl[s] = 0.0f;
                    jit_state_adj(X, a, h, psi, ctau, dl);
#pragma unroll
                    for (int s = 0; s < JN; ++s) acc2(lam[0][s], lam_lo[s], dl[s]);
                    acc2(mu[0], mu_lo, dt_dir);  // t_{k+1} = t_k + tau_k
                } else {
                    jit_state_adj(X, a, h, psi, ctau, lam[t]);
                    mu[t] += dt_dir;  // t_{k+1} = t_k + tau_k
                }
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
                    const float alpha = s == s_top ? a_top : p.brk_a[(int64_t)s * n + i];
                    if (alpha >= 0.0f) coef = 1.0f - alpha;
                }
                for (int o = 0; o < p.n_obs; ++o) {
                    const float g = WIDE ? gl[(int64_t)s * p.n_obs + o] * inj : gl[(int64_t)s * p.n_obs + o];
                    if (WIDE) jit_lam_add2(lam[0], lam_lo, p.obs_sp[o], coef * g);
                    else {
#pragma unroll
                        for (int t = 0; t < NT; ++t) jit_lam_add(lam[t], p.obs_sp[o], coef * g);
                    }
                }
            }
        }
        if (WIDE) {  // keep the binary32 parts the rounded sums, which the next step's w_j and dtau read
#pragma unroll
            for (int s = 0; s < JN; ++s) fold2(lam[0][s], lam_lo[s]);
            fold2(mu[0], mu_lo);
        }
        if (ck_off == 0) {
#pragma unroll
            for (int s = 0; s < JN; ++s) mism += (ckv[s] != X[s]);
            --ck_row;
            ck_off = p.K;
            if (ck_row >= 0) {
#pragma unroll
                for (int s = 0; s < JN; ++s) ckv[s] = p.ckpt[((int64_t)ck_row * JN + s) * n + i];
            }
            if constexpr (WIDE) {
                float m = fabsf(mu[0]);
#pragma unroll
                for (int s = 0; s < JN; ++s) m = fmaxf(m, fabsf(lam[0][s]));
#pragma unroll
                for (int j = 0; j < JM; ++j) m = fmaxf(m, fabsf(dAr[0][j]));
                if (m > 0x1p32f && m <= 3.4028235e38f) {
                    const int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;  // 32 <= e <= 127
                    const float f = ldexpf(1.0f, -e);
                    mu[0] *= f;
                    mu_lo *= f;
#pragma unroll
                    for (int s = 0; s < JN; ++s) {
                        lam[0][s] *= f;
                        lam_lo[s] *= f;
                    }
#pragma unroll
                    for (int j = 0; j < JM; ++j) dAr[0][j] *= f;
                    sc += e;
                    inj = ldexpf(1.0f, -sc);
                }
            }
        }
        --ck_off;
        if (k > 0) jit_unapply(X, event_at(k - 1));
        if (draw) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) E[q] = En[q];
        }
    }
    if (mism) atomicAdd(p.mismatch, mism);
}

// ---------------------------------------------------------------------------------------------
// Soft forward (Section 3.3, Eq. 4): the state is real and moves every step by the expected
// stoichiometry sum_j y~_j v_j of the soft sample y~ = softmax((log a + G)/T), drawn from the same
// variates as the Gumbel-max forward. Clock, samples and readouts are the forward's; there are no range
// checks. Its gradient is the exact gradient of this relaxed model: the straight-through adjoint's
// arithmetic along the soft path, whose states the adjoint regenerates segment by segment from float
// checkpoints taken every kSoftK steps.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float jit_fsel(const float (&X)[JN], int sp)
{
    float v = 0.0f;
#pragma unroll
    for (int s = 0; s < JN; ++s) v = (s == sp) ? X[s] : v;
    return v;
}

// Propensities, soft sample and relaxed update of the state X with the step variates E (E[0] for the
// waiting time, E[1 + j] for reaction j): keys l_j = log2 a_j - log2 E_{1+j} = (ln a_j + G_j)/ln 2, so
// y~_j = exp2((l_j - l_max)/T) / Z. Returns a0.
__device__ __forceinline__ float jit_soft_step(const float (&X)[JN], const float (&kr)[JM], const float (&E)[JM + 1],
                                               float invT, float (&a)[JM], float (&h)[JM], float (&y)[JM],
                                               float (&dX)[JN])
{
    jit_props_soft(X, kr, a, h);
    float a0 = 0.0f, lmax = -CUDART_INF_F;
#pragma unroll
    for (int j = 0; j < JM; ++j) {
        a0 = __fadd_rn(a0, a[j]);
        y[j] = a[j] > 0.0f ? log2f(a[j]) - log2f(E[j + 1]) : -CUDART_INF_F;
        lmax = fmaxf(lmax, y[j]);
    }
    float Z = 0.0f;
#pragma unroll
    for (int j = 0; j < JM; ++j) {
        y[j] = y[j] == -CUDART_INF_F ? 0.0f : exp2f((y[j] - lmax) * invT);
        Z += y[j];
    }
    const float invZ = __fdividef(1.0f, Z);
#pragma unroll
    for (int j = 0; j < JM; ++j) y[j] *= invZ;
    jit_dx_soft(y, dX);
    return a0;
}

template <int READOUT, bool RECORD>
__device__ __forceinline__ void jit_fwd_soft(const FwdParams &p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_traj) return;
    const int64_t n = p.n_traj;
    float kr[JM];
#pragma unroll
    for (int j = 0; j < JM; ++j) kr[j] = p.k_rates[j];
    const int *x0 = p.x0 + (p.x0_per_traj ? i * JN : 0);
    const bool bad_obs = (*p.flag & kErrBadObs) != 0;
    bool bad_input = (*p.flag & (kErrBadSamples | kErrBadObs)) != 0;
    float X[JN];
#pragma unroll
    for (int s = 0; s < JN; ++s) {
        const int v = x0[s];
        X[s] = int2f(v);
        bad_input |= v < 0;
    }
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32);
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    double t = 0.0;
    int s = 0;
    double thr = p.S > 0 ? p.ts[0] : p.t_end;
    int status = bad_input ? SSA_TRAJ_BAD_INPUT : SSA_TRAJ_OK;
    int k = 0, draws = 0;
    int ck_left = p.K, ck_row = 0;
    constexpr int NQ = JM + 1;
    float E[NQ], En[NQ];
    step_noise<NQ>(E, 0u, c2, c3, key0, key1);
    float bacc[kBinMaxObs];
    BinRuns bruns;
    bin_runs_init(bruns);
    int osp[kBinMaxObs];
    jit_bin_init(p, bad_obs, bacc, osp);
    auto xobs = [&](int c) { return jit_fsel(X, osp[c]); };
    float *obs = static_cast<float *>(p.obs_out);
    float *ckf = reinterpret_cast<float *>(p.ckpt);

    while (!bad_input) {
        if (k >= p.max_steps) { status = SSA_TRAJ_STEP_CAP; break; }
        step_noise<NQ>(En, (uint32_t)(k + 1), c2, c3, key0, key1);
        float a[JM], h[JM], y[JM], dX[JN];
        const float a0 = jit_soft_step(X, kr, E, p.invT, a, h, y, dX);
        if (!(a0 < CUDART_INF_F)) { status = SSA_TRAJ_BAD_RATE; break; }
        if (a0 == 0.0f) { status = SSA_TRAJ_ABSORBED; break; }
        const float tau = waiting_time(E[0], a0);
        const double t_next = t + f2d_pos(tau);
        const bool slow = gt_nonneg(t_next, thr);
        const bool cross = slow && gt_nonneg(t_next, p.t_end);
        bool finite = true;
#pragma unroll
        for (int q = 0; q < JN; ++q) finite &= fabsf(__fadd_rn(X[q], dX[q])) < CUDART_INF_F;
        draws = k + 1;
        if (!cross && !finite) { status = SSA_TRAJ_BAD_RATE; break; }
        if (slow) {
            const int s_first = s;
            if constexpr (READOUT == SSA_READOUT_BIN) {
                s = bin_edges<RECORD>(p, i, s, t, t_next, k, bacc, xobs, bruns);
            } else {
                while (s < p.S && gt_nonneg(t_next, p.ts[s])) {
                    float *o = obs + ((int64_t)i * p.S + s) * p.n_obs;
                    if (READOUT == SSA_READOUT_HOLD) {
                        for (int c = 0; c < p.n_obs; ++c) o[c] = jit_fsel(X, p.obs_sp[c]);
                    } else {
                        const float alpha = __fdiv_rn(d2f_nonneg(p.ts[s] - t), tau);
                        for (int c = 0; c < p.n_obs; ++c) {
                            const int sp = p.obs_sp[c];
                            o[c] = __fmaf_rn(alpha, jit_fsel(dX, sp), jit_fsel(X, sp));
                        }
                        if (RECORD) p.brk_a[(int64_t)s * n + i] = alpha;
                    }
                    if (RECORD) p.brk_k[(int64_t)s * n + i] = k;
                    ++s;
                }
            }
            if (READOUT == SSA_READOUT_BIN && !cross && s > s_first)
                bin_accumulate(bacc, xobs, p.n_obs, d2f_nonneg(t_next - p.ts[s - 1]));
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;
        } else if (READOUT == SSA_READOUT_BIN) {
            bin_accumulate(bacc, xobs, p.n_obs, tau);
        }
#pragma unroll
        for (int q = 0; q < JN; ++q) X[q] = __fadd_rn(X[q], dX[q]);
        t = t_next;
        ++k;
        if (RECORD && --ck_left == 0) {
            ck_left = p.K;
            ++ck_row;
#pragma unroll
            for (int q = 0; q < JN; ++q) ckf[((int64_t)ck_row * JN + q) * n + i] = X[q];
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) E[q] = En[q];
    }
    if constexpr (READOUT == SSA_READOUT_BIN) bin_tail<RECORD>(p, i, s, t, k, bacc, xobs, bad_obs, bruns);
    for (; READOUT != SSA_READOUT_BIN && s < p.S; ++s) {
        float *o = obs + ((int64_t)i * p.S + s) * p.n_obs;
        for (int c = 0; c < p.n_obs; ++c) o[c] = bad_obs ? 0.0f : jit_fsel(X, p.obs_sp[c]);
        if (RECORD && READOUT == SSA_READOUT_LINEAR) p.brk_a[(int64_t)s * n + i] = -1.0f;
        if (RECORD) p.brk_k[(int64_t)s * n + i] = k;
    }
    p.draws[i] = draws;
    p.status[i] = status;
    if (RECORD) {
#pragma unroll
        for (int q = 0; q < JN; ++q) ckf[(int64_t)q * n + i] = int2f(x0[q]);  // checkpoint 0 = X_0
    }
}

// Exact gradient of the soft forward, one trajectory; per-reaction adjoints into dAr.
template <int READOUT>
__device__ __forceinline__ void jit_adj_soft_traj(const AdjParams &p, const float (&kr)[JM], const int64_t i,
                                                  const int st, float (&dAr)[JM])
{
    const int64_t n = p.n_traj;
    const int d = p.draws[i];
    const int L = (st == SSA_TRAJ_OK) ? d - 1 : d;  // index of the last visited state
    const bool draw_last = st == SSA_TRAJ_OK;
    const int K = p.K;  // == kSoftK
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32);
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    const float invT = p.invT;
    const float *gl = p.dl_dobs + i * p.dl_stride;
    const float *ckf = reinterpret_cast<const float *>(p.ckpt);
    constexpr int NQ = JM + 1;
    float lam[JN];
#pragma unroll
    for (int q = 0; q < JN; ++q) lam[q] = 0.0f;

    int s_hi = p.S - 1;
    int brk_next = (READOUT != SSA_READOUT_BIN && s_hi >= 0) ? p.brk_k[(int64_t)s_hi * n + i] : -1;
    // BIN: one recorded slot per state interval that holds edges
    BinSlots bslots{-1, -1};
    float d_first = 0.0f, d_last = 0.0f;
    if (READOUT == SSA_READOUT_BIN) bin_slots_init(bslots, p.brk_k, p.brk_tail, n, i);
    float mu = 0.0f;
    int mism = 0;
    constexpr bool kBin = READOUT == SSA_READOUT_BIN;
    float gq[kBinMaxObs], gk[kBinMaxObs];
    int osp[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) osp[c] = (kBin && c < p.n_obs) ? p.obs_sp[c] : 0;
    auto addx = [&](int c, float v) { jit_lam_add(lam, osp[c], v); };
    if (kBin) bin_grad(gq, gl, p.n_obs, p.ts, p.S, p.S);

    float Xs[kSoftK][JN];  // states k0 .. k1 of the segment being walked
    for (int c = L / K; c >= 0; --c) {
        const int k0 = c * K, k1 = min(k0 + K - 1, L);
        float X[JN];
#pragma unroll
        for (int q = 0; q < JN; ++q) X[q] = ckf[((int64_t)c * JN + q) * n + i];
        // regenerate the segment's states with the forward's arithmetic
        for (int kk = k0; kk <= k1; ++kk) {
#pragma unroll
            for (int q = 0; q < JN; ++q) Xs[kk - k0][q] = X[q];
            if (kk < L) {
                float E[NQ], a[JM], h[JM], y[JM], dX[JN];
                step_noise<NQ>(E, (uint32_t)kk, c2, c3, key0, key1);
                jit_soft_step(X, kr, E, invT, a, h, y, dX);
#pragma unroll
                for (int q = 0; q < JN; ++q) X[q] = __fadd_rn(X[q], dX[q]);
            }
        }
        if (k1 < L) {  // the state after the segment is the next checkpoint, bit for bit
#pragma unroll
            for (int q = 0; q < JN; ++q) mism += X[q] != ckf[((int64_t)(c + 1) * JN + q) * n + i];
        }
        for (int k = k1; k >= k0; --k) {
            float Xk[JN];
#pragma unroll
            for (int q = 0; q < JN; ++q) Xk[q] = Xs[k - k0][q];
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
            if (kBin) {
                if (s_hi < s_top) bin_grad(gk, gl, p.n_obs, p.ts, p.S, s_hi + 1);
                else {
#pragma unroll
                    for (int c2b = 0; c2b < kBinMaxObs; ++c2b) gk[c2b] = gq[c2b];
                }
            }
            float tau_k = 0.0f;
            if (draw) {
                float E[NQ], a[JM], h[JM], y[JM], dX[JN];
                step_noise<NQ>(E, (uint32_t)k, c2, c3, key0, key1);
                const float a0 = jit_soft_step(Xk, kr, E, invT, a, h, y, dX);
                const float tau = waiting_time(E[0], a0);
                tau_k = tau;
                float dt_dir = 0.0f, dtau_dir = 0.0f;
                if (kBin) {  // t_{k+1} ends this interval and starts the next, in the bin of gq
                    float cb = 0.0f;
#pragma unroll
                    for (int q = 0; q < kBinMaxObs; ++q)
                        if (q < p.n_obs) cb = __fmaf_rn(gq[q], jit_fsel(dX, osp[q]), cb);
                    mu -= cb;
                }
                if (READOUT == SSA_READOUT_LINEAR) {
                    for (int s = s_hi + 1; s <= s_top; ++s) {
                        const float alpha = p.brk_a[(int64_t)s * n + i];
                        if (alpha < 0.0f) continue;
                        float cl = 0.0f;
                        for (int o = 0; o < p.n_obs; ++o) {
                            const float g = gl[(int64_t)s * p.n_obs + o];
                            const int sp = p.obs_sp[o];
                            jit_lam_add(lam, sp, alpha * g);
                            cl += g * jit_fsel(dX, sp);
                        }
                        const float c_tau = __fdividef(cl, tau);
                        dt_dir -= c_tau;
                        dtau_dir -= alpha * c_tau;
                    }
                }
                const float dtau = mu + dtau_dir;
                const float dLda0 = -dtau * tau / a0;
                float wr[JM];
                jit_w(lam, wr);
                float Wbar = 0.0f;
#pragma unroll
                for (int j = 0; j < JM; ++j) Wbar += y[j] * wr[j];
                float psi[JM], ctau[JM];
#pragma unroll
                for (int j = 0; j < JM; ++j) {
                    psi[j] = y[j] > 0.0f ? y[j] * (wr[j] - Wbar) * invT : 0.0f;
                    dAr[j] += psi[j] + dLda0 * a[j];
                    ctau[j] = dLda0 * kr[j];
                }
                jit_state_adj_soft(Xk, a, h, psi, ctau, lam);
                mu += dt_dir;
            }
            if (kBin) {
                bin_state_terms(addx, d_first, d_last, gl, p.bin_prefix, p.n_obs, s_hi + 1, s_top, draw, tau_k, gq, gk);
#pragma unroll
                for (int q = 0; q < kBinMaxObs; ++q) gq[q] = gk[q];
            } else {
                for (int s = s_hi + 1; s <= s_top; ++s) {
                    float coef = 1.0f;
                    if (READOUT == SSA_READOUT_LINEAR && draw) {
                        const float alpha = p.brk_a[(int64_t)s * n + i];
                        if (alpha >= 0.0f) coef = 1.0f - alpha;
                    }
                    for (int o = 0; o < p.n_obs; ++o)
                        jit_lam_add(lam, p.obs_sp[o], coef * gl[(int64_t)s * p.n_obs + o]);
                }
            }
        }
    }
    if (mism) atomicAdd(p.mismatch, mism);
}

template <int READOUT, bool SOFT, bool WIDE = false, int NT = 1>
__device__ __forceinline__ void jit_adj(const AdjParams &p)
{
    extern __shared__ float s_dA[];  // [NT][JM][blockDim.x] (WIDE: binary64)
    __shared__ int s_len[256], s_perm[256];
    const int B = blockDim.x, tid = threadIdx.x;
    const int64_t n = p.n_traj;
    // the threads of the block take its trajectories longest first, so that each warp walks trajectories
    // of similar length (a warp's reverse walk lasts as long as its longest lane)
    const int64_t i0 = (int64_t)blockIdx.x * B;
    s_len[tid] = i0 + tid < n ? p.draws[i0 + tid] : -1;
    __syncthreads();
    const int key = s_len[tid];
    int rank = 0;
    for (int u = 0; u < B; ++u) {
        const int ku = s_len[u];
        rank += (ku > key) || (ku == key && u < tid);
    }
    s_perm[rank] = tid;
    __syncthreads();
    const int64_t i = i0 + s_perm[tid];
    float kr[JM], dAr[NT][JM];
#pragma unroll
    for (int j = 0; j < JM; ++j) {
        kr[j] = p.k_rates[j];
#pragma unroll
        for (int t = 0; t < NT; ++t) dAr[t][j] = 0.0f;
    }
    int st = -1;
    if (i < n) st = p.status[i];
    const bool active = st == SSA_TRAJ_OK || st == SSA_TRAJ_ABSORBED || st == SSA_TRAJ_STEP_CAP;
    int sc = 0;
    if (active) {
        if constexpr (SOFT) jit_adj_soft_traj<READOUT>(p, kr, i, st, dAr[0]);
        else jit_adj_traj<READOUT, WIDE, NT>(p, kr, i, st, dAr, sc);
    }
    const int warp = tid >> 5, lane = tid & 31, nwarps = B >> 5;
    if constexpr (WIDE) {
        // binary64 values dAr 2^sc, reduced over the block in a fixed order
        // (a trajectory whose accumulators overflowed within one segment contributes inf or NaN, which
        // reaches the result)
        double *s_dA64 = reinterpret_cast<double *>(s_dA);
#pragma unroll
        for (int j = 0; j < JM; ++j) s_dA64[j * B + tid] = ldexp((double)dAr[0][j], sc);
        __syncthreads();
        for (int j = warp; j < JM; j += nwarps) {
            double acc = 0.0;
            for (int u = lane; u < B; u += 32) acc += s_dA64[j * B + u];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) p.partial64[(int64_t)blockIdx.x * JM + j] = acc;
        }
        return;
    }
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int j = 0; j < JM; ++j) s_dA[(t * JM + j) * B + tid] = dAr[t][j];
    __syncthreads();
    // fixed-order block reduction of the per-reaction adjoints (the generic kernels' order); temperature t
    // writes its block sums to partial + t gridDim.x JM
    for (int tj = warp; tj < NT * JM; tj += nwarps) {
        float acc = 0.0f;
        for (int u = lane; u < B; u += 32) acc += s_dA[tj * B + u];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        const int t = tj / JM, j = tj - t * JM;
        if (lane == 0) p.partial[((int64_t)t * gridDim.x + blockIdx.x) * JM + j] = acc;
    }
}

}  // namespace ssa

#ifndef SSA_JIT_SOFT
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_hold(const ssa::FwdParams p)
{
    ssa::jit_fwd<SSA_READOUT_HOLD, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_hold_rec(const ssa::FwdParams p)
{
    ssa::jit_fwd<SSA_READOUT_HOLD, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_linear(const ssa::FwdParams p)
{
    ssa::jit_fwd<SSA_READOUT_LINEAR, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_linear_rec(const ssa::FwdParams p)
{
    ssa::jit_fwd<SSA_READOUT_LINEAR, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_bin(const ssa::FwdParams p)
{
    ssa::jit_fwd<SSA_READOUT_BIN, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_bin_rec(const ssa::FwdParams p)
{
    ssa::jit_fwd<SSA_READOUT_BIN, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_bin_direct(const ssa::FwdParams p)
{
    ssa::jit_fwd_direct<SSA_READOUT_BIN>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_hold_direct(const ssa::FwdParams p)
{
    ssa::jit_fwd_direct<SSA_READOUT_HOLD>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_linear_direct(const ssa::FwdParams p)
{
    ssa::jit_fwd_direct<SSA_READOUT_LINEAR>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_hold(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_HOLD, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_linear(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_LINEAR, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_bin(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_BIN, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_hold_t2(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_HOLD, false, false, 2>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_hold_t3(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_HOLD, false, false, 3>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_linear_t2(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_LINEAR, false, false, 2>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_linear_t3(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_LINEAR, false, false, 3>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_hold_wide(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_HOLD, false, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_linear_wide(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_LINEAR, false, true>(p);
}
#else  // the soft-forward program of the same network
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_hold_soft(const ssa::FwdParams p)
{
    ssa::jit_fwd_soft<SSA_READOUT_HOLD, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_hold_soft_rec(const ssa::FwdParams p)
{
    ssa::jit_fwd_soft<SSA_READOUT_HOLD, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_hold_soft(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_HOLD, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_linear_soft(const ssa::FwdParams p)
{
    ssa::jit_fwd_soft<SSA_READOUT_LINEAR, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_linear_soft_rec(const ssa::FwdParams p)
{
    ssa::jit_fwd_soft<SSA_READOUT_LINEAR, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_linear_soft(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_LINEAR, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_bin_soft(const ssa::FwdParams p)
{
    ssa::jit_fwd_soft<SSA_READOUT_BIN, false>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_fwd_bin_soft_rec(const ssa::FwdParams p)
{
    ssa::jit_fwd_soft<SSA_READOUT_BIN, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) ssa_jit_adj_bin_soft(const ssa::AdjParams p)
{
    ssa::jit_adj<SSA_READOUT_BIN, true>(p);
}
#endif
