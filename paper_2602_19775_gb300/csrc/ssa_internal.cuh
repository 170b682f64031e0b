// ssa_internal.cuh -- internal structures and device helpers of the GB300 SSA library.
//
// Everything here is private to libssa; the public ABI is include/ssa.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "../../include/ssa.h"

namespace ssa {

// ------------------------------------------------------------------------------------------
// Device-side network tables (built once by ssa_create_network)
//   rx[j]     = {r1, r2, s_begin, s_end}: reactant slots (canonical: r1 = -1 means order 0,
//               r2 = -1 means first order, r1 == r2 a homodimer) and the CSR range of v_j
//   stoich[e] = (species << 8) | (uint8)delta
// The two arrays are contiguous (rx first) so one bulk copy stages both into shared memory.
// ------------------------------------------------------------------------------------------
struct NetTables {
    const int4 *rx;
    const int *stoich;
    const int *rate_index;
    int N, M, P, nnz;
    uint32_t tab_bytes;  // 16 * M + 4 * nnz_pad, a multiple of 16
};

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
__device__ __forceinline__ float mass_action_h(const int4 rx, const int *X, int stride)
{
    if (rx.x < 0) return 1.0f;
    const int x1 = X[rx.x * stride];
    if (rx.y < 0) return int2f(x1);
    if (rx.y == rx.x) {
        if (x1 < 2) return 0.0f;
        if (x1 < (1 << 23)) return __fmul_rn(int2f(x1), int2f(x1 - 1)) * 0.5f;
        return __ll2float_rn(((long long)x1 * (x1 - 1)) >> 1);
    }
    const int x2 = X[rx.y * stride];
    if ((x1 | x2) < (1 << 23)) return __fmul_rn(int2f(x1), int2f(x2));
    return __ll2float_rn((long long)x1 * x2);
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
        if (4 * b + 0 < NQ) E[4 * b + 0] = -logf(u01(r.x));
        if (4 * b + 1 < NQ) E[4 * b + 1] = -logf(u01(r.y));
        if (4 * b + 2 < NQ) E[4 * b + 2] = -logf(u01(r.z));
        if (4 * b + 3 < NQ) E[4 * b + 3] = -logf(u01(r.w));
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
    return -logf(u01(word_of(cache, q & 3)));
}

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

// Per-warp view of a step's inputs (warp-per-trajectory kernels).
struct FwdParamsView {
    const int4 *s_rx;
    const float *s_k;
    int M, nb;
    uint32_t c2, c3, key0, key1;
};

// Warp reductions shared by the warp-per-trajectory kernels (butterfly: every lane gets the same
// bits; the race keeps the lowest j on equal products).
__device__ __forceinline__ void warp_race_combine(float &ab, float &Eb, int &jb)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ao = __shfl_xor_sync(0xffffffffu, ab, off);
        const float Eo = __shfl_xor_sync(0xffffffffu, Eb, off);
        const int jo = __shfl_xor_sync(0xffffffffu, jb, off);
        if (jo >= 0) {
            const float lhs = __fmul_rn(ao, Eb), rhs = __fmul_rn(ab, Eo);
            if (jb < 0 || lhs > rhs || (lhs == rhs && jo < jb)) {
                ab = ao;
                Eb = Eo;
                jb = jo;
            }
        }
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// ------------------------------------------------------------------------------------------
// Shared-memory staging of the network tables and the per-call rate constants with the bulk
// (non-tensor) TMA copy engine: cp.async.bulk global -> shared, completion on an mbarrier.
// The wait is bounded; on timeout the block records an error and skips its work.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait: at most `limit` polls (each try_wait may suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

constexpr uint32_t kWaitLimit = 1u << 24;

// Error bits written to the workspace flag word by kernels.
constexpr int kErrStageTimeout = 1;
constexpr int kErrBadSamples = 2;
constexpr int kErrBadObs = 4;

// Stage `tab_bytes` of tables and `k_bytes` of rate constants (both multiples of 16, both
// 16-byte aligned) into s_tab / s_k. Every thread of the block must call this. Returns false
// (and sets err_flag) if the copy did not complete within the bound.
__device__ __forceinline__ bool stage_tables(void *s_tab, const void *g_tab, uint32_t tab_bytes, void *s_k,
                                             const void *g_k, uint32_t k_bytes, uint64_t *bar,
                                             int *s_ok, int *err_flag)
{
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, tab_bytes + k_bytes);
        bulk_copy_g2s(s_tab, g_tab, tab_bytes, bar);
        bulk_copy_g2s(s_k, g_k, k_bytes, bar);
        bool ok = mbar_wait_bounded(bar, 0, kWaitLimit);
        if (!ok) {
            atomicOr(err_flag, kErrStageTimeout);
            // give the copies in flight a second bounded chance to land before the block exits
            mbar_wait_bounded(bar, 0, kWaitLimit);
        }
        *s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

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
    const int *xfinal;
    const float *dl_dobs;
    int64_t dl_stride;  // elements between trajectories (0 = shared)
    float invT;
    float *partial;   // [gridDim.x][M]
    int *mismatch;    // backward consistency failures
    int *err;
};

}  // namespace ssa
