// ssa_internal.cuh -- internal structures and device helpers of the GB300 SSA library.
//
// Everything here is private to libssa; the public ABI is include/ssa.h.
#pragma once

#include "ssa_device.cuh"

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

// Per-warp view of a step's inputs (warp-per-trajectory kernels).
struct FwdParamsView {
    const int4 *s_rx;
    const float *s_k;
    int M, nb;
    uint32_t c2, c3, key0, key1;
};

// Lane-major position of reaction j in the tables of the warp-per-trajectory kernels. Reaction j is
// driven by word q = (j + 1) % 4 of Philox block b = (j + 1) / 4, which lane b % 32 draws; storing it
// at q * nb + b (nb = number of blocks) puts the entries the 32 lanes read for one word q side by
// side, so those shared-memory accesses are free of bank conflicts.
__device__ __forceinline__ int jpos(int j, int nb) { return ((j + 1) & 3) * nb + ((j + 1) >> 2); }

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

}  // namespace ssa
