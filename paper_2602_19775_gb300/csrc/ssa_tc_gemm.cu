// ssa_tc_gemm.cu -- bf16 GEMM on the fifth-generation tensor cores (tcgen05) with TMA loads and
// TMEM accumulators:  D[m][n] = sum_t sum_k A_t[m][k] B_t[n][k]  (+ bias[n]).
//
// It serves the one dense contraction of the gene-regulatory network (arXiv 2602.19775,
// Section 4.3): the hidden-gene activation energies E1 = W1 x + b1 of every input image, and the
// weight gradient dW1 = G^T x of the backward pass.
//
// Layout. Operands are K-major bf16 rows in global memory (row stride a multiple of 16 bytes).
// For each 64-wide K chunk a CTA loads, per operand, eight TMA boxes of 8 elements x `rows`;
// each box lands as `rows` x 16 bytes, so eight consecutive rows of one box form one 8 x 8
// "core matrix" of 128 contiguous bytes -- the tcgen05 K-major layout without swizzle, with
// core matrices 128 B apart along M/N (stride byte offset) and rows*16 B apart along K (leading
// byte offset). Out-of-range boxes are zero-filled by TMA.
//
// Pipeline. One CTA of 128 threads computes a 128 x NT tile. Thread 0 issues the TMA loads of a
// two-stage ring and the tcgen05.mma instructions (M = 128, N = NT, K = 16 per instruction), and
// commits each stage to an mbarrier that frees it; warp 0 allocates the TMEM columns; after the
// last commit every warp reads its 32 TMEM lanes (tcgen05.ld 32x32b) for the epilogue.
// Terms either share one accumulator or keep one each (`separate`); separate accumulators are
// summed in binary64 in the epilogue. Every wait is bounded and reports a timeout in `err`.
#include <algorithm>
#include <atomic>
#include <cstring>

#include <cuda.h>

#include "ssa_tc.cuh"

namespace ssa {

namespace {

constexpr int kErrTcTimeout = 8;

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// shared-memory matrix descriptor, K-major without swizzle (version 1 for this architecture)
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr(p) >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N >> 3, M >> 4
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 2^e as a binary64 power of two for |e| <= 1022 (its exponent field): an exact scale
__device__ __forceinline__ double pow2_d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

}  // namespace

template <int NT>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ TcMaps maps, const TcArgs args)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kTileA = 128 * 64 * 2;  // bytes of one A tile (128 rows x 64 K)
    constexpr int kTileB = NT * 64 * 2;
    const int stage_bytes = args.n_a * kTileA + args.n_b * kTileB;
    unsigned char *stage0 = tc_smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tc_smem + 2 * stage_bytes);  // full[2], empty[2]
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 4);
    int *s_ok = reinterpret_cast<int *>(bars + 5);

    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
    const int n_acc = args.separate ? args.n_terms : 1;
    // this CTA's K chunks (all of them without a split)
    const int total_chunks = (args.K + 63) / 64;
    const int c0 = args.k_split > 1 ? (int)blockIdx.z * args.chunks_per : 0;
    const int my_chunks = args.k_split > 1 ? min(args.chunks_per, total_chunks - c0) : total_chunks;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(n_acc * NT)) ncols <<= 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) mbar_init(&bars[b], 1);
        *s_ok = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (tid == 0) {
        const int n_chunks = my_chunks;  // local chunk ch loads global chunk c0 + ch
        const uint32_t idesc = tc_idesc(128, NT);
        auto issue = [&](int ch) {
            unsigned char *st = stage0 + (ch & 1) * stage_bytes;
            uint64_t *full = &bars[ch & 1];
            mbar_arrive_expect_tx(full, (uint32_t)stage_bytes);
            for (int a = 0; a < args.n_a; ++a)
                for (int c = 0; c < 8; ++c)
                    tma_load_2d(st + a * kTileA + c * (128 * 16), &maps.a[a], (c0 + ch) * 64 + 8 * c, m0, full);
            for (int b = 0; b < args.n_b; ++b)
                for (int c = 0; c < 8; ++c)
                    tma_load_2d(st + args.n_a * kTileA + b * kTileB + c * (NT * 16), &maps.b[b], (c0 + ch) * 64 + 8 * c,
                                n0, full);
        };
        bool ok = true;
        issue(0);
        for (int ch = 0; ch < n_chunks && ok; ++ch) {
            if (ch + 1 < n_chunks) {
                if (ch + 1 >= 2) ok = mbar_wait_bounded(&bars[2 + ((ch + 1) & 1)], ((ch - 1) >> 1) & 1, kWaitLimit);
                if (!ok) break;
                issue(ch + 1);
            }
            ok = mbar_wait_bounded(&bars[ch & 1], (ch >> 1) & 1, kWaitLimit);
            if (!ok) break;
            tc_fence_after();
            unsigned char *st = stage0 + (ch & 1) * stage_bytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                for (int t = 0; t < args.n_terms; ++t) {
                    const int ai = t < args.n_a ? t : args.n_a - 1;
                    const int bi = t < args.n_b ? t : args.n_b - 1;
                    const uint64_t ad = smem_desc(st + ai * kTileA + kk * 2 * (128 * 16), 128 * 16, 128);
                    const uint64_t bd = smem_desc(st + args.n_a * kTileA + bi * kTileB + kk * 2 * (NT * 16), NT * 16, 128);
                    const uint32_t col = args.separate ? (uint32_t)(t * NT) : 0u;
                    const uint32_t accum = (ch > 0 || kk > 0 || (!args.separate && t > 0)) ? 1u : 0u;
                    tc_mma(tmem + col, ad, bd, idesc, accum);
                }
            }
            tc_commit(&bars[2 + (ch & 1)]);
        }
        if (ok) ok = mbar_wait_bounded(&bars[2 + ((n_chunks - 1) & 1)], ((n_chunks - 1) >> 1) & 1, kWaitLimit);
        if (!ok) {
            atomicOr(args.err, kErrTcTimeout);
            // let anything still in flight land before the CTA releases its TMEM and exits
            mbar_wait_bounded(&bars[2 + ((n_chunks - 1) & 1)], ((n_chunks - 1) >> 1) & 1, kWaitLimit);
            *s_ok = 0;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*s_ok && args.limb_grid) {
        // exact limb sum: each accumulator to its integer T_t (a power-of-two scale, then an exact conversion),
        // combined in int64; the split slabs keep the (lo, hi) pairs, otherwise one rounding to binary64.
        // Sixteen columns per tensor-memory load, so a warp waits on 8 terms x NT/16 loads.
        const int row = m0 + 32 * warp + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        const int g = *args.limb_grid, lb = args.limb_bits;
        for (int c16 = 0; c16 < NT / 16; ++c16) {
            long long lo[16], hi[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) lo[i] = hi[i] = 0;
            for (int t = 0; t < args.n_terms; ++t) {
                float v[16];
                tmem_ld16(lane_base + (uint32_t)(t * NT + 16 * c16), v);
                // 2^-(g + lb t) as two binary32 powers of two (exponent fields), each inside the normal range for
                // any grid a bf16 limb can sit on; both products are exact
                const int e = -(g + lb * t), e1 = e >> 1, e2 = e - e1;
                const float q1 = __int_as_float((127 + e1) << 23), q2 = __int_as_float((127 + e2) << 23);
                const long long w = 1ll << (lb * (t & 3));
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const long long T = (long long)__float2int_rn((v[i] * q1) * q2);
                    if (t < 4) lo[i] += T * w;
                    else hi[i] += T * w;
                }
            }
            if (row < args.M) {
                // (hi 2^(4 lb) + lo) 2^g: both terms exact in binary64 (below 2^43 in magnitude), one rounding
                const double sh = pow2_d(4 * lb + g), sl = pow2_d(g);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = n0 + 16 * c16 + i;
                    if (col < args.N) {
                        if (args.k_split > 1) {
                            longlong2 *dp = reinterpret_cast<longlong2 *>(args.Dpart) +
                                            ((int64_t)blockIdx.z * args.M + row) * args.N + col;
                            *dp = make_longlong2(lo[i], hi[i]);
                        } else {
                            const double x = fma((double)hi[i], sh, (double)lo[i] * sl);
                            const double b = args.bias ? (double)args.bias[col] : 0.0;
                            args.D[(int64_t)row * args.ldd + col] = (float)(x + b);
                        }
                    }
                }
            }
        }
    } else if (*s_ok) {
        const int row = m0 + 32 * warp + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c8 = 0; c8 < NT / 8; ++c8) {
            float v[8];
            double acc[8];
            if (args.separate) {
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = 0.0;
                for (int t = 0; t < args.n_terms; ++t) {
                    tmem_ld8(lane_base + (uint32_t)(t * NT + 8 * c8), v);
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[i] += (double)v[i];
                }
            } else {
                tmem_ld8(lane_base + (uint32_t)(8 * c8), v);
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = (double)v[i];
            }
            if (row < args.M) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int col = n0 + 8 * c8 + i;
                    if (col < args.N) {
                        if (args.k_split > 1) {
                            args.Dpart[((int64_t)blockIdx.z * args.M + row) * args.N + col] = acc[i];
                        } else {
                            const double b = args.bias ? (double)args.bias[col] : 0.0;
                            args.D[(int64_t)row * args.ldd + col] = (float)(acc[i] + b);
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// ---------------------------------------------------------------------------------------------
// Plain GEMM kernel (one A, one B, one accumulator), built for throughput: 128 x 256 tiles, 64-wide
// K blocks loaded by one TMA box per operand into the 128-byte-swizzled K-major layout (each row of a
// block is 128 bytes, eight rows form a 1,024-byte swizzle atom), a four-stage mbarrier ring, one
// thread issuing the TMA loads and another issuing tcgen05.mma, so loads run ahead of the tensor
// cores; the accumulator is 256 TMEM columns read back by all four warps.
// ---------------------------------------------------------------------------------------------
constexpr int kSwBN = 256;
constexpr int kSwStages = 4;
constexpr int kSwTileA = 128 * 128;    // bytes: 128 rows x 64 bf16
constexpr int kSwTileB = kSwBN * 128;  // bytes: 256 rows x 64 bf16
constexpr int kSwStage = kSwTileA + kSwTileB;

// shared-memory matrix descriptor, K-major, 128-byte swizzle: stride between 8-row groups 1,024 B
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *p)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr(p) >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)2 << 61;               // 128-byte swizzle
    return d;
}


// split K: with Dpart given, the CTAs of blockIdx.z = s take the 64-wide K blocks [s per, (s + 1) per) and
// write their sums in binary64 to Dpart [gridDim.z][M][N] (no bias); tc_splitk_reduce_kernel adds them
__global__ void __launch_bounds__(128, 1) tc_gemm_sw128_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                const __grid_constant__ CUtensorMap mapB, int M,
                                                                int N, int K, const float *bias, float *D, int ldd,
                                                                double *Dpart, int chunks_per, int *err)
{
    extern __shared__ __align__(1024) unsigned char sw_raw[];
    // the swizzled tiles need 1,024-byte alignment
    unsigned char *sw = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(sw_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t *full = reinterpret_cast<uint64_t *>(sw + kSwStages * kSwStage);
    uint64_t *empty = full + kSwStages;
    uint64_t *done = empty + kSwStages;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(done + 1);
    int *s_ok = reinterpret_cast<int *>(s_tmem + 1);
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * kSwBN;
    const int total_kb = (K + 63) / 64;
    const int kb0 = Dpart ? (int)blockIdx.z * chunks_per : 0;
    const int nkb = Dpart ? max(0, min(chunks_per, total_kb - kb0)) : total_kb;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"(kSwBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int b = 0; b < kSwStages; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        mbar_init(done, 1);
        *s_ok = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (tid == 0) {
        // TMA producer: wait for the stage to be free, then load both operands of k block kb
        for (int kb = 0; kb < nkb; ++kb) {
            const int st = kb % kSwStages, round = kb / kSwStages;
            if (round > 0 && !mbar_wait_bounded(&empty[st], (round - 1) & 1, kWaitLimit)) {
                atomicOr(err, kErrTcTimeout);
                *s_ok = 0;
                break;
            }
            if (!*(volatile int *)s_ok) break;
            unsigned char *stage = sw + st * kSwStage;
            mbar_arrive_expect_tx(&full[st], (uint32_t)kSwStage);
            tma_load_2d(stage, &mapA, (kb0 + kb) * 64, m0, &full[st]);
            tma_load_2d(stage + kSwTileA, &mapB, (kb0 + kb) * 64, n0, &full[st]);
        }
    } else if (tid == 32) {
        // MMA issuer: four K = 16 steps per block, advancing the descriptors by 32 bytes inside the atom
        const uint32_t idesc = tc_idesc(128, kSwBN);
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int st = kb % kSwStages, round = kb / kSwStages;
            ok = mbar_wait_bounded(&full[st], round & 1, kWaitLimit) && *(volatile int *)s_ok;
            if (!ok) break;
            tc_fence_after();
            const unsigned char *stage = sw + st * kSwStage;
            const uint64_t ad = smem_desc_sw128(stage), bd = smem_desc_sw128(stage + kSwTileA);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc_mma(tmem, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            tc_commit(&empty[st]);  // the stage is free once these MMAs have read it
        }
        if (ok) tc_commit(done);
        else {
            atomicOr(err, kErrTcTimeout);
            *(volatile int *)s_ok = 0;
        }
    }
    __syncwarp();
    // epilogue: wait for the last MMA, then every warp reads its 32 TMEM lanes
    bool have = mbar_wait_bounded(done, 0, kWaitLimit);
    if (!have && tid == 0) atomicOr(err, kErrTcTimeout);
    tc_fence_after();
    if (have && *(volatile int *)s_ok) {
        const int row = m0 + 32 * warp + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c16 = 0; c16 < kSwBN / 16; ++c16) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)(16 * c16), v);
            const int col0 = n0 + 16 * c16;
            if (Dpart) {
                if (row < M) {
                    double *dp = Dpart + ((int64_t)blockIdx.z * M + row) * N + col0;
                    if (col0 + 16 <= N && (N % 2) == 0) {
#pragma unroll
                        for (int i = 0; i < 16; i += 2)
                            *reinterpret_cast<double2 *>(dp + i) = make_double2((double)v[i], (double)v[i + 1]);
                    } else {
                        for (int i = 0; i < 16 && col0 + i < N; ++i) dp[i] = (double)v[i];
                    }
                }
            } else if (row < M) {
                float *dst = D + (int64_t)row * ldd + col0;
                if (col0 + 16 <= N && (ldd % 4) == 0 && (reinterpret_cast<uintptr_t>(D) & 15) == 0) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        float4 o = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                        if (bias) {
                            o.x += bias[col0 + i];
                            o.y += bias[col0 + i + 1];
                            o.z += bias[col0 + i + 2];
                            o.w += bias[col0 + i + 3];
                        }
                        *reinterpret_cast<float4 *>(dst + i) = o;
                    }
                } else {
                    for (int i = 0; i < 16 && col0 + i < N; ++i) dst[i] = v[i] + (bias ? bias[col0 + i] : 0.0f);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSwBN) : "memory");
    }
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2D bf16 K-major operand: rows x K (elements), row stride ld elements (multiple of 8), box 8 x box_rows
bool tc_make_map(CUtensorMap *map, const void *base, int rows, int K, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld % 8) || K > ld) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the same operand with one 64-element x box_rows box per K block, 128-byte swizzled in shared memory
static bool tc_make_map_sw128(CUtensorMap *map, const void *base, int rows, int K, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld % 8) || K > ld) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


// D[m][n] = (sum over splits s in order of Dpart[s][m][n]) + bias[n], rounded once to binary32
__global__ void tc_splitk_reduce_kernel(const double *Dpart, int k_split, int M, int N, const float *bias, float *D,
                                        int ldd)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    const int m = (int)(e / N), n = (int)(e % N);
    double acc = 0.0;
    for (int s = 0; s < k_split; ++s) acc += Dpart[(int64_t)s * M * N + e];
    D[(int64_t)m * ldd + n] = (float)(acc + (bias ? (double)bias[n] : 0.0));
}

// the same for the exact limb sum: int64 (lo, hi) pairs of every split, added exactly in split order
__global__ void tc_splitk_reduce_limbs_kernel(const longlong2 *Dpart, int k_split, int M, int N, const int *limb_grid,
                                             int limb_bits, const float *bias, float *D, int ldd)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    const int m = (int)(e / N), n = (int)(e % N);
    long long lo = 0, hi = 0;
    for (int s = 0; s < k_split; ++s) {
        const longlong2 v = Dpart[(int64_t)s * M * N + e];
        lo += v.x;
        hi += v.y;
    }
    const int g = *limb_grid;
    const double x = fma((double)hi, pow2_d(4 * limb_bits + g), (double)lo * pow2_d(g));
    D[(int64_t)m * ldd + n] = (float)(x + (bias ? (double)bias[n] : 0.0));
}

int tc_split_count(int M, int N, int K, int nt)
{
    const int64_t tiles = (int64_t)((M + 127) / 128) * ((N + nt - 1) / nt);
    const int total = (K + 63) / 64;
    constexpr int kTargetCtas = 152;  // one CTA per SM of this part
    if (tiles >= kTargetCtas || total <= 1) return 1;
    int k = (int)std::min<int64_t>(total, kTargetCtas / tiles);
    if (k <= 1) return 1;
    const int per = (total + k - 1) / k;
    return (total + per - 1) / per;  // every split non-empty
}

size_t tc_split_words(int M, int N, int K, int nt)
{
    const int k = tc_split_count(M, N, K, nt);
    return k > 1 ? (size_t)k * M * N : 0;
}

// K splits of the plain GEMM (1: none) and the K blocks of each: the output tiles times the splits come up
// to one CTA per SM, and every split keeps at least four K blocks so that each CTA still fills its ring
static int sw_split(int M, int N, int K, int *per)
{
    const int64_t tiles = (int64_t)((M + 127) / 128) * ((N + kSwBN - 1) / kSwBN);
    const int total = (K + 63) / 64;
    constexpr int kTargetCtas = 152;
    *per = total;
    const int k = (int)std::min<int64_t>(total / 4, tiles >= kTargetCtas ? 1 : kTargetCtas / tiles);
    if (k <= 1) return 1;
    *per = (total + k - 1) / k;
    return (total + *per - 1) / *per;  // every split non-empty
}

static cudaError_t tc_gemm_sw128_launch(const CUtensorMap &ma, const CUtensorMap &mb, int M, int N, int K,
                                        const float *bias, float *D, int ldd, double *work, int *err, cudaStream_t st)
{
    const size_t smem = (size_t)kSwStages * kSwStage + 128 + 1024;  // ring, barriers, alignment slack
    // the attribute is set once per device and kept by the context, so calls inside a graph capture make no
    // further runtime calls (after cudaDeviceReset the launch fails with an error instead)
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !(attr_set.load() & (1ull << dev))) {
        e = cudaFuncSetAttribute(tc_gemm_sw128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) attr_set.fetch_or(1ull << dev);
    }
    int per = (K + 63) / 64;
    const int k_split = work ? sw_split(M, N, K, &per) : 1;
    dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + kSwBN - 1) / kSwBN), (unsigned)k_split);
    tc_gemm_sw128_kernel<<<grid, 128, smem, st>>>(ma, mb, M, N, K, bias, D, ldd, k_split > 1 ? work : nullptr, per,
                                                  err);
    if (k_split > 1) {
        const int64_t n = (int64_t)M * N;
        tc_splitk_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(work, k_split, M, N, bias, D, ldd);
    }
    return cudaGetLastError();
}

int64_t sw_gemm_work_words(int M, int N, int K)
{
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    int per;
    const int k_split = sw_split(M, N, K, &per);
    return k_split > 1 ? (int64_t)k_split * M * N : 0;
}

template <int NT>
static cudaError_t tc_launch_t(const TcMaps &maps, const TcArgs &args_in, cudaStream_t st)
{
    TcArgs args = args_in;
    args.k_split = 1;
    args.chunks_per = 0;
    if (args.Dpart) {
        args.k_split = tc_split_count(args.M, args.N, args.K, NT);
        const int total = (args.K + 63) / 64;
        args.chunks_per = (total + args.k_split - 1) / args.k_split;
    }
    const size_t stage = (size_t)args.n_a * 128 * 128 + (size_t)args.n_b * NT * 128;
    // 64 KB of slack past the ring: every core-matrix address a descriptor can form from these
    // tiles stays inside the CTA's shared-memory allocation
    const size_t smem = 2 * stage + 64 + 65536;
    if (smem > 232448) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((args.M + 127) / 128), (unsigned)((args.N + NT - 1) / NT), (unsigned)args.k_split);
    tc_gemm_kernel<NT><<<grid, 128, smem, st>>>(maps, args);
    if (args.k_split > 1) {
        const int64_t total = (int64_t)args.M * args.N;
        if (args.limb_grid)
            tc_splitk_reduce_limbs_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
                reinterpret_cast<const longlong2 *>(args.Dpart), args.k_split, args.M, args.N, args.limb_grid,
                args.limb_bits, args.bias, args.D, args.ldd);
        else
            tc_splitk_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(args.Dpart, args.k_split, args.M,
                                                                                     args.N, args.bias, args.D, args.ldd);
    }
    return cudaGetLastError();
}

cudaError_t tc_gemm_launch(const TcMaps &maps, const TcArgs &args, int nt, cudaStream_t st)
{
    if (args.M == 0 || args.N == 0) return cudaSuccess;
    switch (nt) {
    case 64: return tc_launch_t<64>(maps, args, st);
    case 112: return tc_launch_t<112>(maps, args, st);
    case 128: return tc_launch_t<128>(maps, args, st);
    default: return cudaErrorInvalidValue;
    }
}

ssa_status set_error(ssa_status code, const char *text);

}  // namespace ssa

extern "C" int64_t ssa_bf16_gemm_work_words(int32_t M, int32_t N, int32_t K)
{
    return ssa::sw_gemm_work_words(M, N, K);
}

extern "C" ssa_status ssa_bf16_gemm(const uint16_t *A, const uint16_t *B, int32_t M, int32_t N, int32_t K,
                                    int32_t lda, int32_t ldb, const float *bias, float *D, int32_t ldd, double *work,
                                    int64_t work_words, int32_t *err_flag, void *stream)
{
    using namespace ssa;
    if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldd < N) return set_error(SSA_ERR_INVALID_ARG, "bad GEMM sizes");
    if ((M > 0 && N > 0) && (!D || !err_flag || (K > 0 && (!A || !B))))
        return set_error(SSA_ERR_INVALID_ARG, "NULL GEMM operand");
    if ((lda % 8) || (ldb % 8)) return set_error(SSA_ERR_INVALID_ARG, "lda and ldb must be multiples of 8 (16-byte rows)");
    if (work && (reinterpret_cast<uintptr_t>(work) & 15))
        return set_error(SSA_ERR_INVALID_ARG, "the GEMM work buffer must be 16-byte aligned");
    if (work && work_words < sw_gemm_work_words(M, N, K))
        return set_error(SSA_ERR_WORKSPACE, "GEMM work buffer smaller than ssa_bf16_gemm_work_words");
    if (M == 0 || N == 0) return SSA_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (K == 0) {  // an empty sum: D = bias (or 0)
        const int64_t n = (int64_t)M * N;
        tc_splitk_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nullptr, 0, M, N, bias, D, ldd);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? SSA_OK : set_error(SSA_ERR_CUDA, cudaGetErrorString(e));
    }
    CUtensorMap ma, mb;
    if (!tc_make_map_sw128(&ma, A, M, K, lda, 128) || !tc_make_map_sw128(&mb, B, N, K, ldb, kSwBN))
        return set_error(SSA_ERR_INVALID_ARG, "tensor map encoding failed (alignment or driver entry point)");
    cudaError_t e = tc_gemm_sw128_launch(ma, mb, M, N, K, bias, D, ldd, work_words > 0 ? work : nullptr, err_flag, st);
    return e == cudaSuccess ? SSA_OK : set_error(SSA_ERR_CUDA, cudaGetErrorString(e));
}
