// ssa_device.cuh -- device arithmetic and kernel parameter blocks shared by the library's kernels
// and by the network-specialised kernels compiled at run time (NVRTC), so both evaluate every step with
// the same instructions in the same order.
#pragma once

#ifdef __CUDACC_RTC__
#define CUDART_INF_F __int_as_float(0x7f800000)
#else
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>
#endif

#include "../../include/ssa.h"

namespace ssa {

// per-step uniform mapping: u = ((x >> 9) + 1/2) 2^-23, exact in binary32. Built from the bits:
// 1 + m 2^-23 (m = x >> 9 placed in the mantissa of 1.0) minus (1 - 2^-24) is exactly
// m 2^-23 + 2^-24, so no integer-to-float conversion is needed.
__device__ __forceinline__ float u01(uint32_t x)
{
    return __fsub_rn(__uint_as_float(0x3F800000u | (x >> 9)), 0x1.fffffep-1f);
}

// Exact int -> binary32 for 0 <= x < 2^23 through the bits of 2^23 + x (the integer pipe), with the
// plain conversion for other values.
__device__ __forceinline__ float int2f(int x)
{
    if ((unsigned)x < (1u << 23)) return __fsub_rn(__uint_as_float(0x4B000000u | (unsigned)x), 8388608.0f);
    return __int2float_rn(x);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, two 32x32->64 products each,
// round keys bumped by the two Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &r, int q)
{
    return q == 0 ? r.x : q == 1 ? r.y : q == 2 ? r.z : r.w;
}

// Mass-action combinatorial factor h_j(X) (Section 2): 1, X_i, X_i X_l or X_i (X_i - 1)/2, equal
// to the exact integer rounded once to binary32. Counts below 2^24 are exact in binary32, so one
// correctly rounded binary32 product gives the same value as the exact 64-bit product rounded
// once; larger counts take the 64-bit route.
__device__ __forceinline__ float h_first(int x1) { return int2f(x1); }

__device__ __forceinline__ float h_homodimer(int x1)
{
    if (x1 < 2) return 0.0f;
    if (x1 < (1 << 23)) return __fmul_rn(int2f(x1), int2f(x1 - 1)) * 0.5f;
    return __ll2float_rn(((long long)x1 * (x1 - 1)) >> 1);
}

__device__ __forceinline__ float h_hetero(int x1, int x2)
{
    if ((x1 | x2) < (1 << 23)) return __fmul_rn(int2f(x1), int2f(x2));
    return __ll2float_rn((long long)x1 * x2);
}

// Mass-action factors of the real-valued state of the soft forward (Eq. 4); a relaxed state can leave the
// integers, and a factor that comes out negative there is taken as 0 (a propensity cannot be negative).
__device__ __forceinline__ float hs_first(float x1) { return fmaxf(x1, 0.0f); }
__device__ __forceinline__ float hs_homodimer(float x1) { return fmaxf(__fmul_rn(x1, x1 - 1.0f) * 0.5f, 0.0f); }
__device__ __forceinline__ float hs_hetero(float x1, float x2) { return fmaxf(__fmul_rn(x1, x2), 0.0f); }

__device__ __forceinline__ float mass_action_h(const int4 rx, const int *X, int stride)
{
    if (rx.x < 0) return 1.0f;
    const int x1 = X[rx.x * stride];
    if (rx.y < 0) return h_first(x1);
    if (rx.y == rx.x) return h_homodimer(x1);
    return h_hetero(x1, X[rx.y * stride]);
}

// The same value as mass_action_h from selects instead of branches: the lanes of a warp-per-trajectory kernel
// evaluate reactions of different orders side by side, and branches on the order would run one after another.
// An absent reactant counts as 1 (order 0: 1 x 1; order 1: x1 x 1, exact); a homodimer multiplies x1 by
// max(x1 - 1, 0) and halves (0 for x1 < 2). Counts of 2^23 and more take the exact 64-bit path.
__device__ __forceinline__ float mass_action_h_sel(const int4 rx, const int *X)
{
    const bool homo = rx.y >= 0 && rx.y == rx.x;
    const int x1 = rx.x >= 0 ? X[rx.x >= 0 ? rx.x : 0] : 1;
    const int xr2 = X[rx.y >= 0 ? rx.y : 0];
    const int x2 = homo ? max(x1 - 1, 0) : (rx.y >= 0 ? xr2 : 1);
    if ((unsigned)(x1 | x2) >= (1u << 23)) return mass_action_h(rx, X, 1);
    const float h = __fmul_rn(int2f(x1), int2f(x2));
    return homo ? h * 0.5f : h;
}

// a > b for non-negative, non-NaN binary64 values: IEEE 754 orders them like their bit patterns
// read as unsigned integers, so the comparison runs on the integer pipe instead of the FP64 pipe.
__device__ __forceinline__ bool gt_nonneg(double a, double b)
{
    return (unsigned long long)__double_as_longlong(a) > (unsigned long long)__double_as_longlong(b);
}

// binary64 -> binary32, round to nearest even, for a non-negative value in the binary32 normal
// range, from the IEEE 754 fields on the integer pipe (other values take the plain conversion):
// the 52-bit fraction is cut to 23 bits and rounded on the 29 dropped bits; a carry out of the
// fraction increments the exponent field, as it should.
__device__ __forceinline__ float d2f_nonneg(double d)
{
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const int e = (int)(hi >> 20) - 896;  // binary32 exponent field
    if (e >= 1 && e <= 254 && (hi >> 31) == 0) {
        uint32_t f = ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t r = lo & 0x1fffffffu;
        f += (r > 0x10000000u) || (r == 0x10000000u && (f & 1u));
        return __uint_as_float(f);
    }
    return __double2float_rn(d);
}

// binary32 -> binary64 for a positive normal value by re-biasing the exponent field (IEEE 754
// layouts), which keeps the conversion off the FP64 pipe; other values take the plain conversion.
__device__ __forceinline__ double f2d_pos(float x)
{
    const uint32_t b = __float_as_uint(x);
    if (b - 0x00800000u < 0x7f000000u) return __hiloint2double((int)((b >> 3) + 0x38000000u), (int)(b << 29));
    return (double)x;
}

__device__ __forceinline__ int stoich_species(int e) { return e >> 8; }
__device__ __forceinline__ int stoich_delta(int e) { return (int)(signed char)(e & 0xff); }

// Exponential variate E = -ln u of a uniform u in (0, 1), the one function every kernel draws its
// waiting times and race variates with (CUDA's logf, within one unit in the last place).
__device__ __forceinline__ float neg_log_unit(float u) { return -logf(u); }

// Exponential variates of one step, E[q] = -ln u_q for the first NQ words of the step's Philox
// stream (q = 0 drives the waiting time, q = 1 + j reaction j). They do not depend on the state,
// so the kernels draw the next step's variates while the current step's state-dependent chain
// runs (instruction-level parallelism at low occupancy).
template <int NQ>
__device__ __forceinline__ void step_noise(float (&E)[NQ], uint32_t k, uint32_t c2, uint32_t c3, uint32_t key0,
                                           uint32_t key1)
{
#pragma unroll
    for (int b = 0; b < (NQ + 3) / 4; ++b) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)b, k, c2, c3), key0, key1);
        if (4 * b + 0 < NQ) E[4 * b + 0] = neg_log_unit(u01(r.x));
        if (4 * b + 1 < NQ) E[4 * b + 1] = neg_log_unit(u01(r.y));
        if (4 * b + 2 < NQ) E[4 * b + 2] = neg_log_unit(u01(r.z));
        if (4 * b + 3 < NQ) E[4 * b + 3] = neg_log_unit(u01(r.w));
    }
}

// -ln u_q of one word (runtime-indexed variant for networks without a compile-time size).
__device__ __forceinline__ float exp_variate(uint32_t k, int q, uint32_t c2, uint32_t c3, uint32_t key0, uint32_t key1,
                                             uint4 &cache, int &cached_b)
{
    const int b = q >> 2;
    if (b != cached_b) {
        cache = philox4x32_10(make_uint4((uint32_t)b, k, c2, c3), key0, key1);
        cached_b = b;
    }
    return neg_log_unit(u01(word_of(cache, q & 3)));
}

// The waiting time tau = E_0 / a0 (Section 2), rounded once (IEEE division). The clock adds ~1e6 of these
// over a long trajectory; an approximate division's error is not centred on zero, and its bias would move
// the clock systematically (by ~1e-5 over 1e6 draws of the oscillator), flipping sample brackets and the
// LINEAR readout's interpolation weights.
__device__ __forceinline__ float waiting_time(float E0, float a0) { return __fdiv_rn(E0, a0); }

// The Gumbel-max choice as an exponential race: argmax_j a_j/E_j, compared as a_j E_b > a_b E_j
// (binary32 products); ties keep the lowest j. The adjoint repeats the identical comparisons.
__device__ __forceinline__ void race(float a, float E, int j, float &ab, float &Eb, int &jb)
{
    if (__fmul_rn(a, Eb) > __fmul_rn(ab, E)) {
        ab = a;
        Eb = E;
        jb = j;
    }
}

// Increments of the state adjoint dL/dX from one reaction (mass action): the choice path
// psi * dlog a/dX (only where a > 0) and the waiting-time path c_tau * dh/dX with c_tau = dL/da0 * k
// (polynomial derivative, also where a = 0). xs is the species' own count, xo the other reactant's.
__device__ __forceinline__ float sadj_first(float xs, float a, float psi, float c_tau)
{
    return (a > 0.0f ? __fdividef(psi, xs) : 0.0f) + c_tau;
}

__device__ __forceinline__ float sadj_homodimer(float xs, float a, float h, float psi, float c_tau)
{
    const float dh = xs - 0.5f;  // d/dX [X (X - 1)/2]
    return (a > 0.0f ? __fdividef(psi * dh, h) : 0.0f) + c_tau * dh;
}

__device__ __forceinline__ float sadj_hetero(float xs, float xo, float a, float psi, float c_tau)
{
    return (a > 0.0f ? __fdividef(psi, xs) : 0.0f) + c_tau * xo;
}

// ------------------------------------------------------------------------------------------
// Exact bin-averaged readout (Section 4.4): obs_s = (1/D_s) * integral over (t_{s-1}, t_s] of the
// piecewise-constant path, t_{-1} = 0, D_s = t_s - t_{s-1}. The forward keeps, per observable, the
// integral acc of the open bin from its left edge up to t_k, adding X_k tau_k for every step that stays
// inside the bin. An edge t_s in [t_k, t_{k+1}), at offset d = t_s - t_k, closes a bin: the first edge
// of a step closes the bin that began before t_k, obs = (acc + X_k d) / D_s; a later edge closes a bin
// that lies inside the step, where the path is X_k, obs = X_k. The rest of the step, t_{k+1} minus the
// last edge, opens the next bin. A stopped path holds its last state. The bins held at X_k inside a step
// are buffered as runs and written by the warp when the trajectories stop (coalesced), and recording keeps
// one slot per state interval that holds edges -- its state k, first edge and that edge's offset d -- not
// one bracket per edge.
//
// The adjoint walks the same pieces backwards. With g_b = dL/dobs_b / D_b, the state X_k receives the
// overlap of its interval with every bin times that bin's g; the event time t_{k+1} (the end of one
// interval and the start of the next) receives g_b (X_k - X_{k+1}) for the bin b that contains it,
// which enters dL/dtau_k with the later times.
// ------------------------------------------------------------------------------------------
constexpr int kBinMaxObs = SSA_BIN_MAX_OBS;

// an observed count as binary32: integer states (exact below 2^23) and the real states of the soft forward
__device__ __forceinline__ float obs_f(int x) { return int2f(x); }
__device__ __forceinline__ float obs_f(float x) { return x; }

// acc[c] += X_c len for the observables (xobs(c) = count of observable c)
template <class XF>
__device__ __forceinline__ void bin_accumulate(float (&acc)[kBinMaxObs], const XF &xobs, int n_obs, float len)
{
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c)
        if (c < n_obs) acc[c] = __fmaf_rn(obs_f(xobs(c)), len, acc[c]);
}

// Close bin s at its right edge ts[s] >= t_k and write its averages to o; first: the bin began before
// t_k (acc holds its integral up to t_k). Clears acc and returns d = ts[s] - t_k.
template <class XF>
__device__ __forceinline__ float bin_close(float (&acc)[kBinMaxObs], const XF &xobs, int n_obs, const double *ts, int s,
                                           double t_k, bool first, float *o)
{
    const float d = d2f_nonneg(ts[s] - t_k);
    const float D = d2f_nonneg(ts[s] - (s > 0 ? ts[s - 1] : 0.0));
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) {
        if (c < n_obs) {
            const float x = obs_f(xobs(c));
            o[c] = first ? __fdiv_rn(__fmaf_rn(x, d, acc[c]), D) : x;
            acc[c] = 0.0f;
        }
    }
    return d;
}

// g[c] = dL/dobs_b[c] / D_b for bin b, 0 past the last bin
__device__ __forceinline__ void bin_grad(float (&g)[kBinMaxObs], const float *gl, int n_obs, const double *ts, int S,
                                         int b)
{
    const bool in = b < S;
    const float D = in ? d2f_nonneg(ts[b] - (b > 0 ? ts[b - 1] : 0.0)) : 1.0f;
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) g[c] = (in && c < n_obs) ? __fdiv_rn(gl[(int64_t)b * n_obs + c], D) : 0.0f;
}

// sum_c g_c (X_{k+1} - X_k)_c at the observables (xo: X_{k+1}); dL/dt_{k+1} receives minus this
template <class XF>
__device__ __forceinline__ float bin_transition(const XF &xobs, const int (&xo)[kBinMaxObs], const float (&g)[kBinMaxObs],
                                                int n_obs)
{
    float c = 0.0f;
#pragma unroll
    for (int q = 0; q < kBinMaxObs; ++q)
        if (q < n_obs) c = __fmaf_rn(g[q], (float)(xo[q] - xobs(q)), c);
    return c;
}

// dL/dX_k from the bins that the interval of state k overlaps. Edges s_first..s_last (none if
// s_first > s_last) lie in it, at offsets d_first and d_last from t_k; gq: g of the bin that contains
// t_{k+1}, gk: of the bin that contains t_k; draw: the interval ends at t_{k+1} = t_k + tau (else the path
// holds X_k to the end); addx(c, v) adds v to the adjoint of observable c.
// prefix: when every trajectory has the same upstream gradient, prefix[s][c] = sum over bins below s of
// dL/dobs (binary64, [S + 1][kBinMaxObs]), so a run of whole bins costs one difference; else nullptr.
template <class AF>
__device__ __forceinline__ void bin_state_terms(const AF &addx, float d_first, float d_last, const float *gl,
                                                const double *prefix, int n_obs, int s_first, int s_last, bool draw,
                                                float tau, const float (&gq)[kBinMaxObs],
                                                const float (&gk)[kBinMaxObs])
{
    if (s_first > s_last) {  // the interval lies inside one bin
        if (draw) {
#pragma unroll
            for (int c = 0; c < kBinMaxObs; ++c)
                if (c < n_obs) addx(c, gq[c] * tau);
        }
        return;
    }
    if (draw) {  // t_{k+1} - t_{s_last} in the bin after the last edge
        const float r = tau - d_last;
#pragma unroll
        for (int c = 0; c < kBinMaxObs; ++c)
            if (c < n_obs) addx(c, gq[c] * r);
    }
    // whole bins: overlap D_s, so g_s D_s = dL/dobs_s
    if (prefix) {
        if (s_last > s_first) {
#pragma unroll
            for (int c = 0; c < kBinMaxObs; ++c)
                if (c < n_obs)
                    addx(c, (float)(prefix[(int64_t)(s_last + 1) * kBinMaxObs + c] -
                                    prefix[(int64_t)(s_first + 1) * kBinMaxObs + c]));
        }
    } else {
        for (int s = s_first + 1; s <= s_last; ++s) {
#pragma unroll
            for (int c = 0; c < kBinMaxObs; ++c)
                if (c < n_obs) addx(c, gl[(int64_t)s * n_obs + c]);
        }
    }
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c)  // t_{s_first} - t_k in the bin that contains t_k
        if (c < n_obs) addx(c, gk[c] * d_first);
}

// Bin readout with a shared upstream gradient g [S][n_obs]: prefix[s][c] = sum_{b < s} g[b][c] in binary64,
// for s = 0..S ([S + 1][kBinMaxObs]), computed by one block of kPrefixThreads threads: each thread sums a
// contiguous chunk of bins, the chunk totals are scanned in shared memory (fixed order), and each thread writes
// its chunk's prefixes. Every block that runs it gets the same bits.
constexpr int kPrefixThreads = 256;
__device__ __forceinline__ void bin_prefix_block(const float *g, int S, int n_obs, double *prefix)
{
    __shared__ double part[kPrefixThreads];
    const int tid = threadIdx.x;
    const int chunk = (S + kPrefixThreads - 1) / kPrefixThreads;
    const int lo = min(tid * chunk, S), hi = min(lo + chunk, S);
    for (int c = 0; c < kBinMaxObs; ++c) {
        double acc = 0.0;
        if (c < n_obs)
            for (int b = lo; b < hi; ++b) acc += (double)g[(int64_t)b * n_obs + c];
        part[tid] = acc;
        __syncthreads();
        for (int off = 1; off < kPrefixThreads; off <<= 1) {  // inclusive scan of the chunk totals
            const double v = tid >= off ? part[tid - off] : 0.0;
            __syncthreads();
            part[tid] += v;
            __syncthreads();
        }
        double run = tid > 0 ? part[tid - 1] : 0.0;  // sum of the bins below this chunk
        if (tid == 0) prefix[c] = 0.0;
        for (int b = lo; b < hi; ++b) {
            if (c < n_obs) run += (double)g[(int64_t)b * n_obs + c];
            prefix[(int64_t)(b + 1) * kBinMaxObs + c] = run;
        }
        __syncthreads();
    }
}

// The adjoint's walk over the recorded slots of the bin readout (from the last): at state k, if the
// slot below is k's, its edges are first..s_top, and s_hi drops below them. Returns whether state k holds
// edges; d_first/d_last are the offsets of its first and last edge from t_k.
struct BinSlots {
    int q;     // next slot to read, from the last
    int kq;    // its state (-1: none left)
};
__device__ __forceinline__ void bin_slots_init(BinSlots &w, const int *brk_k, const int *brk_tail, int64_t n, int64_t i)
{
    w.q = brk_tail[i] - 1;
    w.kq = w.q >= 0 ? brk_k[(int64_t)w.q * n + i] : -1;
}
__device__ __forceinline__ void bin_slots_step(BinSlots &w, const int *brk_k, const int *brk_s, const float *brk_a,
                                               const double *ts, int64_t n, int64_t i, int k, int &s_hi,
                                               float &d_first, float &d_last)
{
    if (w.kq != k) return;
    const int64_t at = (int64_t)w.q * n + i;
    const int first = brk_s[at];
    d_first = brk_a[at];
    d_last = s_hi > first ? d_first + d2f_nonneg(ts[s_hi] - ts[first]) : d_first;
    s_hi = first - 1;
    --w.q;
    w.kq = w.q >= 0 ? brk_k[(int64_t)w.q * n + i] : -1;
}

// Soft forward: the float state is checkpointed every kSoftK steps; the adjoint re-runs each segment.
constexpr int kSoftK = 8;

// Error bits written to the workspace flag word by kernels.
constexpr int kErrStageTimeout = 1;
constexpr int kErrBadSamples = 2;
constexpr int kErrBadObs = 4;


// ------------------------------------------------------------------------------------------
// Kernel parameter blocks
// ------------------------------------------------------------------------------------------
struct FwdParams {
    const int4 *rx;
    const float *k_rates;  // [M padded to 4]
    uint32_t tab_bytes, k_bytes;
    int N, M, Mp, nnz;  // Mp: padded reaction count, >= M + 1, multiple of 4, >= the unrolled width
    uint32_t inc_off, inc_list_off;  // byte offsets of the species -> reactant-slot incidence in the tables
    int64_t n_traj;
    uint64_t traj_offset, seed;
    const int *x0;
    int x0_per_traj;
    double t_end;
    const double *ts;
    int S;
    const int *obs_sp;
    int n_obs;
    int64_t max_steps;
    float invT;       // soft forward (Eq. 4): 1/T of its soft sample
    const int *upd;   // warp soft forward: species-major update list (ssa_network::d_upd), upd_words ints
    uint32_t upd_words;
    void *obs_out;
    int *draws, *status;
    const int *flag;  // workspace error flags (bad sample times -> every trajectory BAD_INPUT)
    int *err;
    // record
    int K;
    uint4 *ev;        // [ev_rows][n_traj], 8 uint16 events per uint4
    int *ckpt;        // [n_ckpt][N][n_traj]
    int *brk_k;       // [S][n_traj]
    float *brk_a;     // [S][n_traj]
    int *brk_s;       // [S][n_traj], BIN readout: first edge of slot q (brk_k, brk_a: its state, offset)
    int *brk_tail;    // [n_traj], BIN readout: number of slots
    int *xfinal;      // [N][n_traj]
    // replay
    const uint16_t *ev_in;
    const int *n_ev_in;
    int64_t ev_in_stride;
};

struct AdjParams {
    const int4 *rx;
    const float *k_rates;
    uint32_t tab_bytes, k_bytes;
    int N, M, Mp, nnz;  // Mp: padded reaction count, >= M + 1, multiple of 4, >= the unrolled width
    uint32_t inc_off, inc_list_off;  // byte offsets of the species -> reactant-slot incidence in the tables
    int64_t n_traj;
    uint64_t traj_offset, seed;
    const double *ts;
    int S;
    const int *obs_sp;
    int n_obs;
    int K;
    const int *draws, *status;
    const uint4 *ev;
    const int *ckpt;
    const int *brk_k;
    const float *brk_a;
    const int *brk_s;
    const int *brk_tail;
    const int *xfinal;
    const float *dl_dobs;
    int64_t dl_stride;  // elements between trajectories (0 = shared)
    const double *bin_prefix;  // BIN readout with a shared dl_dobs: its prefix sums over bins, else nullptr
    float invT;
    float *partial;   // [gridDim.x][M]
    int *mismatch;    // backward consistency failures
    int *err;
    // wide-range adjoint (long trajectories): per-block binary64 sums of the per-reaction adjoints, each
    // trajectory's binary32 accumulators scaled back by its power-of-two exponent
    double *partial64;  // [gridDim.x][M]
    // several temperatures in one walk (network-specialised kernels): 1/T_t, t < the kernel's count; the
    // block sums of temperature t go to partial + t gridDim.x M
    float invT_multi[4];
};


// Bin readout, forward: the held runs of bins buffered for the warp-wide write, and the slot count.
constexpr int kBinRuns = 8;
struct BinRuns {
    int n;                           // buffered runs
    int slots;                       // recorded slots
    int lo[kBinRuns], hi[kBinRuns];  // bins lo..hi hold v
    float v[kBinRuns][kBinMaxObs];
};
__device__ __forceinline__ void bin_runs_init(BinRuns &r)
{
    r.n = 0;
    r.slots = 0;
#pragma unroll
    for (int q = 0; q < kBinRuns; ++q) {
        r.lo[q] = r.hi[q] = 0;
#pragma unroll
        for (int c = 0; c < kBinMaxObs; ++c) r.v[q][c] = 0.0f;
    }
}

// The first edge s of a state interval (t_k <= t_s): close its bin, and record the interval's slot.
template <bool RECORD, class XF>
__device__ __forceinline__ void bin_first_edge(const FwdParams &p, int64_t i, int s, double t_k, int k,
                                               float (&acc)[kBinMaxObs], const XF &xobs, BinRuns &r)
{
    float *o = static_cast<float *>(p.obs_out) + ((int64_t)i * p.S + s) * p.n_obs;
    const float d = bin_close(acc, xobs, p.n_obs, p.ts, s, t_k, true, o);
    if (RECORD) {
        const int64_t at = (int64_t)r.slots * p.n_traj + i;
        p.brk_k[at] = k;
        p.brk_s[at] = s;
        p.brk_a[at] = d;
        ++r.slots;
    }
}

// Bins lo..hi lie inside the interval of X_k: buffer the run (the thread writes it itself when the buffer
// is full).
template <class XF>
__device__ __forceinline__ void bin_held_run(const FwdParams &p, int64_t i, int lo, int hi, const XF &xobs, BinRuns &r)
{
    if (lo > hi) return;
    const int no = p.n_obs;
    if (r.n < kBinRuns) {
        r.lo[r.n] = lo;
        r.hi[r.n] = hi;
#pragma unroll
        for (int c = 0; c < kBinMaxObs; ++c) r.v[r.n][c] = c < no ? obs_f(xobs(c)) : 0.0f;
        ++r.n;
        return;
    }
    float *row = static_cast<float *>(p.obs_out) + (int64_t)i * p.S * no;
    for (int s = lo; s <= hi; ++s)
        for (int c = 0; c < no; ++c) row[(int64_t)s * no + c] = obs_f(xobs(c));
}

// Bin readout, one state interval [t_k, t_next): the edges in it from s on are found by bisection (the
// edges increase strictly); the first closes its bin, the others are whole bins held at X_k. Returns the
// index of the first edge at or after t_next.
template <bool RECORD, class XF>
__device__ __forceinline__ int bin_edges(const FwdParams &p, int64_t i, int s, double t_k, double t_next, int k,
                                         float (&acc)[kBinMaxObs], const XF &xobs, BinRuns &r)
{
    int lo = s, hi = p.S;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (gt_nonneg(t_next, p.ts[mid])) lo = mid + 1;
        else hi = mid;
    }
    if (lo > s) {
        bin_first_edge<RECORD>(p, i, s, t_k, k, acc, xobs, r);
        bin_held_run(p, i, s + 1, lo - 1, xobs, r);
    }
    return lo;
}

// Bin readout, after the last state X_k (held from t_k on): the first remaining bin s may have begun
// before t_k, the later ones hold X_k exactly. Each thread closes its first remaining bin (and records its
// slot); then the warp writes the buffered runs and the held tails of its trajectories together, one run
// at a time with consecutive lanes on consecutive floats, so these stores are coalesced. Recording stores
// the number of slots in brk_tail[i]. Every lane of the warp whose trajectory index is below n_traj must
// call this.
template <bool RECORD, class XF>
__device__ __forceinline__ void bin_tail(const FwdParams &p, int64_t i, int s, double t_k, int k,
                                         float (&acc)[kBinMaxObs], const XF &xobs, bool bad_obs, BinRuns &r)
{
    const int64_t n = p.n_traj;
    const int S = p.S, no = p.n_obs;
    float *obs = static_cast<float *>(p.obs_out);
    if (s < S) {
        float *o = obs + ((int64_t)i * S + s) * no;
        bin_first_edge<RECORD>(p, i, s, t_k, k, acc, xobs, r);
        if (bad_obs)
            for (int c = 0; c < no; ++c) o[c] = 0.0f;
    }
    if (RECORD) p.brk_tail[i] = r.slots;
    float xv[kBinMaxObs];
#pragma unroll
    for (int c = 0; c < kBinMaxObs; ++c) xv[c] = (c < no && !bad_obs) ? obs_f(xobs(c)) : 0.0f;
    const int lane = (int)(threadIdx.x & 31);
    const int64_t base = i - lane;
    const unsigned mask = base + 32 <= n ? 0xffffffffu : ((1u << (unsigned)(n - base)) - 1u);
    const int writers = __popc(mask);  // the live lanes 0 .. writers-1 of the (last, partial) warp
    const int first = s + 1;  // first held row
    for (int j = 0; j < 32 && ((mask >> j) & 1u); ++j) {
        const int nj = __shfl_sync(mask, r.n, j);
        for (int q = 0; q < nj; ++q) {  // lane j's buffered runs
            const int lo = __shfl_sync(mask, r.lo[q], j), hi = __shfl_sync(mask, r.hi[q], j);
            float vq[kBinMaxObs];
#pragma unroll
            for (int c = 0; c < kBinMaxObs; ++c) vq[c] = __shfl_sync(mask, r.v[q][c], j);
            float *row = obs + (base + j) * (int64_t)S * no;
            for (int64_t e = (int64_t)lo * no + lane; e < (int64_t)(hi + 1) * no; e += writers) {
                const int c = no == 1 ? 0 : (int)(e % no);
                float v = vq[0];
#pragma unroll
                for (int c2 = 1; c2 < kBinMaxObs; ++c2) v = c == c2 ? vq[c2] : v;
                row[e] = v;
            }
        }
        const int fj = __shfl_sync(mask, first, j);
        float vj[kBinMaxObs];
#pragma unroll
        for (int c = 0; c < kBinMaxObs; ++c) vj[c] = __shfl_sync(mask, xv[c], j);
        if (fj >= S) continue;  // the same for every lane
        float *row = obs + (base + j) * (int64_t)S * no;
        for (int64_t e = (int64_t)fj * no + lane; e < (int64_t)S * no; e += writers) {
            const int c = no == 1 ? 0 : (int)(e % no);
            float v = vj[0];
#pragma unroll
            for (int q = 1; q < kBinMaxObs; ++q) v = c == q ? vj[q] : v;
            row[e] = v;
        }
    }
}

}  // namespace ssa
