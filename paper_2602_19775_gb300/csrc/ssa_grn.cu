// ssa_grn.cu -- the gene-regulatory-network classifier of arXiv 2602.19775, Section 4.3 (Figure 4A):
// n_in clamped input transcription factors x (counts round(255 p)), n_hid hidden gene products h and
// n_out output gene products y. Reactions (j < n_dyn: production of dynamic species j; j >= n_dyn:
// degradation of species j - n_dyn, with n_dyn = n_hid + n_out):
//     production of h_i:  k_max sigma(E1_i),  E1 = W1 x + b1
//     production of y_o:  k_max sigma(E2_o),  E2 = W2 h + b2
//     degradation of s:   d_s X_s,            d = exp(log_d)
// Parameters W1, b1, W2, b2, log_d (203,796 for 784 -> 256 -> 10).
//
// The dense contraction E1 = W1 x runs on the tcgen05 tensor cores, once per image. W1 (bf16) is
// split into 6-bit limbs on a common power-of-two grid; with integer counts x <= 255 every partial
// sum of one limb is an integer multiple of the limb's quantum below 2^24 quanta, so the binary32
// accumulation in TMEM is exact; the epilogue turns each accumulator into that integer and adds the limbs
// in int64 (two 42-bit halves), which is W1 x exactly, rounded once to binary64 before b1 is added. E2 = W2 h is kept exactly as an int64 fixed-point sum (bf16 W2 on its own
// grid times integer counts), updated by +-W2[:, i] when h_i changes.
//
// The SSA and the straight-through adjoint run one warp per trajectory (lanes own Philox blocks as
// in the mass-action warp kernels). With the HOLD readout the loss does not depend on event times,
// so the waiting-time path contributes nothing and the adjoint is the choice path of Eqs. 3, 5, 7.
// The backward accumulates dL/dE1 per trajectory (dW1 = G^T x follows on the tensor cores with bf16
// hi/lo limbs of G), and dW2 = sum_k G2_k h_k^T by summation by parts: with R = sum_{m >= k} G2_m
// accumulated backwards, undoing an event that changed h_i by delta adds delta R to dW2[:, i]
// (h starts at zero), so each step costs O(n_out) instead of O(n_out n_hid).
#include <algorithm>
#include <cstring>
#include <new>

#include <cuda.h>

#include "ssa_host.h"
#include "ssa_tc.cuh"

namespace ssa {

cudaError_t launch_reduce_partials(const float *partial, int64_t nblk, int M, const int *rate_index, int P,
                                   float *dA_tmp, float *dtheta, cudaStream_t st);
cudaError_t launch_validate_inputs(const double *ts, int S, double t_end, const int *obs_sp, int n_obs, int N,
                                  int strict, int *flag, cudaStream_t st);
cudaError_t launch_column_sums(const float *x, int64_t n_rows, int64_t row_len, float *partial, int64_t chunk, float *out,
                               cudaStream_t st);

constexpr int kGrnLimbs = 8;       // 6-bit limbs of W1 on one grid: 48 bits of dynamic range
constexpr int kGrnLimbBits = 6;
constexpr int kGrnOutBatch = 12;   // output counts up to this take the adjoint's batched W2 column loads
constexpr int kGrnWarps = 4;

struct GrnParams {
    int n_in, n_hid, n_out, n_dyn, M, Mp, nb;
    float k_max;
    int64_t n_traj, tpi;
    uint64_t traj_offset, seed;
    const float *E1;      // [n_img][n_hid]
    const int *W2fix;     // [n_out][n_hid]: W2 = W2fix * 2^g2
    const float *W2f;     // [n_out][n_hid]
    const float *b2;      // [n_out]
    const float *dvec;    // [n_dyn]: d = exp(log_d)
    const int *grid;      // [0] = g2
    double t_end;
    const double *ts;
    int S;
    int64_t max_steps;
    int *obs_out;         // [n_traj][S][n_out]
    int *draws, *status;
    const int *flag;
    int *err;
    int K;
    uint4 *ev;
    int *ckpt;            // hard path: [n_ckpt][n_dyn][n_traj]
    int *brk_k;           // [S][n_traj]
    int *xfinal;          // [n_dyn][n_traj]
    // backward
    const float *dl_dobs;
    int64_t dl_stride;
    float invT;
    float *G1;            // [n_traj][n_hid]
    float *dW2t;          // [n_traj][n_out n_hid]: per-trajectory dL/dW2
    float *partial;       // [blocks][n_out + n_dyn]
    int *mismatch;
    // soft path: float checkpoints [n_traj][n_ckpt][n_dyn] (trajectory-major, one warp writes a row) and the
    // adjoint's scratch [n_traj][8][grn_soft_row]: per step of the segment being walked, its state, output
    // propensities, unnormalised soft weights and 1/Z
    int64_t n_ckpt;
    float *seg;
};

namespace {

// logistic sigma(e) in binary32 from expf and correctly rounded divisions (a few ulp)
__device__ __forceinline__ float sigmoid_f(float e)
{
    if (e >= 0.0f) return __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-e)));
    const float z = expf(e);
    return __fdiv_rn(z, __fadd_rn(1.0f, z));
}

__device__ __forceinline__ float e2_value(long long acc, float scale, float b2)
{
    return __fadd_rn(b2, __fmul_rn(__ll2float_rn(acc), scale));
}

// propensity of reaction j (one lane's view); padded j >= M give 0
__device__ __forceinline__ float grn_prop(const GrnParams &p, int j, const float *aH, const float *aO, const int *X,
                                          const float *s_d)
{
    if (j < p.n_hid) return aH[j];
    if (j < p.n_dyn) return aO[j - p.n_hid];
    if (j < p.M) return __fmul_rn(s_d[j - p.n_dyn], int2f(X[j - p.n_dyn]));
    return 0.0f;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// preparation: exponent range of the weights, W1 limbs, fixed-point W2, inputs in bf16
// ---------------------------------------------------------------------------------------------
__global__ void grn_exponents_kernel(const uint16_t *W1, int64_t n1, const uint16_t *W2, int64_t n2, int *grid)
{
    // grid[0]: max exponent field of W1, grid[1]: min exponent field of nonzero W2 (bf16 fields)
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n1 + n2; q += (int64_t)gridDim.x * blockDim.x) {
        const uint16_t v = q < n1 ? W1[q] : W2[q - n1];
        const int e = (v >> 7) & 0xff;
        if (e == 0) continue;  // zero (or subnormal, treated on the slow path below)
        if (q < n1) atomicMax(&grid[0], e);
        else atomicMin(&grid[1], e);
    }
}

__device__ __forceinline__ float bf16_to_float(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }

__device__ __forceinline__ uint16_t float_to_bf16_exact(float f) { return (uint16_t)(__float_as_uint(f) >> 16); }

// bf16 -> bf16 with round to nearest even (the hi/lo split of the backward)
__device__ __forceinline__ uint16_t float_to_bf16_rn(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

__global__ void grn_prepare_kernel(const uint16_t *W1, const uint16_t *W2, const int32_t *x_img, const float *log_d,
                                   int n_in, int n_hid, int n_out, int64_t n_img, int n_in_pad, uint16_t *W1L,
                                   int *W2fix, float *W2f, uint16_t *xb, float *dvec, int *grid)
{
    // W1 on the grid 2^g1, g1 = (max exponent + 1) - 48: |W1| = n 2^g1, n < 2^48, limbs of 6 bits
    const int g1 = (grid[0] - 127 + 1) - kGrnLimbBits * kGrnLimbs;
    // W2 on the grid 2^g2, g2 = (min exponent) - 7: every nonzero bf16 value is an integer multiple
    const int g2 = grid[1] - 127 - 7;
    const int64_t nW1 = (int64_t)n_hid * n_in_pad;
    const int64_t total = kGrnLimbs * nW1 + (int64_t)n_out * n_hid + n_img * n_in_pad + n_hid + n_out;
    for (int64_t qq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; qq < total; qq += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = qq;
        if (q < kGrnLimbs * nW1) {
            const int t = (int)(q / nW1);
            const int64_t r = q % nW1;
            const int h = (int)(r / n_in_pad), p = (int)(r % n_in_pad);
            float limb = 0.0f;
            if (p < n_in) {
                const float w = bf16_to_float(W1[(int64_t)h * n_in + p]);
                if (w != 0.0f) {
                    const double nd = fabs((double)w) * exp2(-(double)g1);
                    const unsigned long long nn = (unsigned long long)nd;
                    if ((double)nn != nd && t == 0) atomicOr(&grid[2], 1);  // below the grid: inexact
                    const unsigned digit = (unsigned)((nn >> (kGrnLimbBits * t)) & ((1u << kGrnLimbBits) - 1));
                    limb = (float)ldexp((double)digit, g1 + kGrnLimbBits * t) * (w < 0.0f ? -1.0f : 1.0f);
                }
            }
            W1L[q] = float_to_bf16_exact(limb);  // at most 6 significant bits: exact in bf16
            continue;
        }
        q -= kGrnLimbs * nW1;
        if (q < (int64_t)n_out * n_hid) {
            const float w = bf16_to_float(W2[q]);
            W2f[q] = w;
            const double nd = (double)w * exp2(-(double)g2);
            if (fabs(nd) >= 1073741824.0 || (double)(long long)nd != nd) atomicOr(&grid[2], 2);
            W2fix[q] = (int)fmax(-1073741823.0, fmin(1073741823.0, nd));
            continue;
        }
        q -= (int64_t)n_out * n_hid;
        if (q < n_img * n_in_pad) {
            const int64_t img = q / n_in_pad;
            const int p = (int)(q % n_in_pad);
            const int xv = p < n_in ? x_img[img * n_in + p] : 0;
            if (xv < 0 || xv > 256) atomicOr(&grid[2], 4);  // counts above 256 are not exact in bf16
            xb[q] = float_to_bf16_exact((float)xv);
            continue;
        }
        q -= n_img * n_in_pad;
        dvec[q] = (float)exp((double)log_d[q]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        grid[3] = g2;
        grid[4] = g1;  // the limb grid of the tensor-core contraction's exact sum
    }
}

// ---------------------------------------------------------------------------------------------
// forward: one warp per trajectory
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) grn_fwd_kernel(const GrnParams p, int record)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int nh = p.n_hid, no = p.n_out, nd = p.n_dyn;
    int *s_W2fix = reinterpret_cast<int *>(smem);
    float *s_d = reinterpret_cast<float *>(s_W2fix + no * nh);
    float *s_b2 = s_d + nd;
    const int ndp = (nd + 3) & ~3, nhp = (nh + 3) & ~3;
    const int nop = (no + 3) & ~3;
    const size_t per_warp = (size_t)ndp + nhp + 3 * (size_t)nop;  // X, aH, E2acc (2 words each), aO
    // offsets from the shared array itself (not through an integer round trip), so that every access below
    // compiles to a shared-memory load or store with 32-bit addressing
    unsigned char *wb = smem + ((4 * ((size_t)no * nh + nd + ((no + 3) & ~3)) + 15) & ~(size_t)15);
    int *X = reinterpret_cast<int *>(wb) + wib * per_warp;
    float *aH = reinterpret_cast<float *>(X + ndp);
    long long *E2acc = reinterpret_cast<long long *>(aH + nhp);
    float *aO = reinterpret_cast<float *>(E2acc + no);

    for (int q = threadIdx.x; q < no * nh; q += blockDim.x) s_W2fix[q] = p.W2fix[q];
    for (int q = threadIdx.x; q < nd; q += blockDim.x) s_d[q] = p.dvec[q];
    for (int q = threadIdx.x; q < no; q += blockDim.x) s_b2[q] = p.b2[q];
    __syncthreads();

    const int64_t i = (int64_t)blockIdx.x * W + wib;
    if (i >= p.n_traj) return;
    const int64_t n = p.n_traj;
    const float scale = exp2f((float)p.grid[0]);
    const float *E1 = p.E1 + (i / p.tpi) * nh;
    for (int s = lane; s < nd; s += 32) X[s] = 0;
    for (int h = lane; h < nh; h += 32) aH[h] = p.k_max * sigmoid_f(E1[h]);
    for (int o = lane; o < no; o += 32) {
        E2acc[o] = 0;
        aO[o] = p.k_max * sigmoid_f(s_b2[o]);
    }
    __syncwarp();
    const bool bad_input = (*p.flag & kErrBadSamples) != 0;
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32), key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);

    double t = 0.0;
    int s = 0;
    double thr = p.S > 0 ? p.ts[0] : p.t_end;
    int status = bad_input ? SSA_TRAJ_BAD_INPUT : SSA_TRAJ_OK;
    int k = 0, draws = 0, ck_left = p.K, ck_row = 0;
    uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    while (!bad_input) {
        if (k >= p.max_steps) { status = SSA_TRAJ_STEP_CAP; break; }
        float a0p = 0.0f, ab = 0.0f, Eb = 1.0f, E0 = 0.0f;
        int jb = -1;
        for (int b = lane; b < p.nb; b += 32) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)k, c2, c3), key0, key1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // predicated: every word's variate is formed (the warp forms it whenever one lane needs it), word
                // 0 of lane 0's first block is E0, and j = -1 takes part with rate 0 (adds 0, never wins)
                const int j = 4 * b + q - 1;
                const float E = neg_log_unit(u01(word_of(r, q)));
                if (q == 0 && j < 0) E0 = E;
                const float a = j < 0 ? 0.0f : grn_prop(p, max(j, 0), aH, aO, X, s_d);
                a0p = __fadd_rn(a0p, a);
                race(a, E, j, ab, Eb, jb);
            }
        }
        const float a0 = warp_sum(a0p);
        warp_race_combine(ab, Eb, jb);
        E0 = __shfl_sync(0xffffffffu, E0, 0);
        if (!(a0 < CUDART_INF_F)) { status = SSA_TRAJ_BAD_RATE; break; }
        if (a0 == 0.0f) { status = SSA_TRAJ_ABSORBED; break; }
        if (jb < 0) { status = SSA_TRAJ_BAD_RATE; break; }
        const float tau = waiting_time(E0, a0);
        const double t_next = t + f2d_pos(tau);
        const bool slow = gt_nonneg(t_next, thr);
        const bool cross = slow && gt_nonneg(t_next, p.t_end);
        const int sp = jb < nd ? jb : jb - nd;
        const int delta = jb < nd ? 1 : -1;
        if (!cross && delta > 0 && X[sp] == 2147483647) status = SSA_TRAJ_OVERFLOW;
        if (record) {
            e0 = __funnelshift_r(e0, e1, 16);
            e1 = __funnelshift_r(e1, e2, 16);
            e2 = __funnelshift_r(e2, e3, 16);
            e3 = (e3 >> 16) | ((uint32_t)jb << 16);
            if (lane == 0 && (k & 7) == 7) p.ev[(int64_t)(k >> 3) * n + i] = make_uint4(e0, e1, e2, e3);
        }
        draws = k + 1;
        if (status != SSA_TRAJ_OK) break;
        if (slow) {
            while (s < p.S && gt_nonneg(t_next, p.ts[s])) {
                int *o = p.obs_out + ((int64_t)i * p.S + s) * no;
                for (int c = lane; c < no; c += 32) o[c] = X[nh + c];
                if (record && lane == 0) p.brk_k[(int64_t)s * n + i] = k;
                ++s;
            }
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;
        }
        __syncwarp();
        if (lane == 0) X[sp] += delta;
        if (sp < nh) {
            for (int o = lane; o < no; o += 32) {
                E2acc[o] += (long long)delta * s_W2fix[o * nh + sp];
                aO[o] = p.k_max * sigmoid_f(e2_value(E2acc[o], scale, s_b2[o]));
            }
        }
        __syncwarp();
        t = t_next;
        ++k;
        if (record && --ck_left == 0) {
            ck_left = p.K;
            ++ck_row;
            int *ck = p.ckpt + (int64_t)ck_row * nd * n + i;
            for (int q = lane; q < nd; q += 32) ck[(int64_t)q * n] = X[q];
        }
    }
    __syncwarp();
    for (; s < p.S; ++s) {
        int *o = p.obs_out + ((int64_t)i * p.S + s) * no;
        for (int c = lane; c < no; c += 32) o[c] = X[nh + c];
        if (record && lane == 0) p.brk_k[(int64_t)s * n + i] = k;
    }
    if (lane == 0) {
        p.draws[i] = draws;
        p.status[i] = status;
    }
    if (record) {
        if ((draws & 7) && lane == 0) {
            for (int pad = draws & 7; pad < 8; ++pad) {
                e0 = __funnelshift_r(e0, e1, 16);
                e1 = __funnelshift_r(e1, e2, 16);
                e2 = __funnelshift_r(e2, e3, 16);
                e3 = e3 >> 16;
            }
            p.ev[(int64_t)((draws - 1) >> 3) * n + i] = make_uint4(e0, e1, e2, e3);
        }
        for (int q = lane; q < nd; q += 32) {
            p.xfinal[(int64_t)q * n + i] = X[q];
            p.ckpt[(int64_t)q * n + i] = 0;  // checkpoint 0: every gene starts at zero
        }
    }
}

// ---------------------------------------------------------------------------------------------
// soft forward (Section 3.3, Eq. 4; the first training phase of Section 3.5): one warp per trajectory and
// real-valued counts. Every step all reactions enter the soft sample y~ = softmax((log a + G)/T) of the same
// Gumbel noise, and every count moves by its expected change y~_prod - y~_deg; a negative count degrades at
// rate 0. E2 = W2 h + b2 is recomputed from the relaxed hidden counts (binary32 W2). The step is one shared
// routine, so the adjoint's re-runs from the float checkpoints reproduce the forward's states bit for bit.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int kGrnSoftK = 8;  // float checkpoints of the soft forward every 8 steps

// output propensities k_max sigma(W2 h + b2) of the relaxed state X (the warp's lanes cooperate)
__device__ __forceinline__ void grn_soft_outputs(const GrnParams &p, const float *s_W2, const float *s_b2,
                                                 const float *X, float *aO, int lane)
{
    const int nh = p.n_hid, no = p.n_out;
    for (int o = 0; o < no; ++o) {
        float part = 0.0f;
        for (int h = lane; h < nh; h += 32) part = __fmaf_rn(s_W2[(size_t)o * nh + h], X[h], part);
        const float e2 = __fadd_rn(warp_sum(part), s_b2[o]);
        if (lane == (o & 31)) aO[o] = p.k_max * sigmoid_f(e2);
    }
    __syncwarp();
}

// one soft step from state X at step k: propensities, keys, then the unnormalised
// weights q_j = exp2((l_j - l_max)/T); returns a0 and sets E0 and invZ = 1/sum q
__device__ __forceinline__ float grn_soft_weights(const GrnParams &p, const float *s_d, const float *X, const float *aH,
                                                  const float *aO, float *q, int k, uint32_t c2,
                                                  uint32_t c3, uint32_t key0, uint32_t key1, int lane, float &E0,
                                                  float &invZ)
{
    const int nh = p.n_hid, nd = p.n_dyn, M = p.M;
    float a0p = 0.0f, lmaxp = -CUDART_INF_F, e0 = 0.0f;
    for (int b = lane; b < p.nb; b += 32) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)k, c2, c3), key0, key1);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int j = 4 * b + w - 1;
            if (j < 0) { e0 = neg_log_unit(u01(r.x)); continue; }
            if (j >= M) continue;
            const float a = j < nh ? aH[j] : j < nd ? aO[j - nh] : __fmul_rn(s_d[j - nd], fmaxf(X[j - nd], 0.0f));
            a0p = __fadd_rn(a0p, a);
            const float l = a > 0.0f ? log2f(a) - log2f(neg_log_unit(u01(word_of(r, w)))) : -CUDART_INF_F;
            q[j] = l;
            lmaxp = fmaxf(lmaxp, l);
        }
    }
    const float a0 = warp_sum(a0p), lmax = warp_max(lmaxp);
    E0 = __shfl_sync(0xffffffffu, e0, 0);
    __syncwarp();
    float Zp = 0.0f;
    for (int j = lane; j < M; j += 32) {
        const float wgt = q[j] == -CUDART_INF_F ? 0.0f : exp2f((q[j] - lmax) * p.invT);
        q[j] = wgt;
        Zp += wgt;
    }
    invZ = __fdividef(1.0f, warp_sum(Zp));
    __syncwarp();
    return a0;
}

// the relaxed update X += (y~_prod - y~_deg) for every dynamic species
__device__ __forceinline__ void grn_soft_update(const GrnParams &p, float *X, const float *q, float invZ, int lane)
{
    const int nd = p.n_dyn;
    for (int u = lane; u < nd; u += 32) X[u] = __fadd_rn(X[u], (q[u] - q[nd + u]) * invZ);
    __syncwarp();
}

}  // namespace

__global__ void __launch_bounds__(128) grn_soft_fwd_kernel(const GrnParams p, float *obs, int record)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int nh = p.n_hid, no = p.n_out, nd = p.n_dyn, M = p.M;
    const int ndp = (nd + 3) & ~3, nhp = (nh + 3) & ~3, nop = (no + 3) & ~3, Mq = (M + 3) & ~3;
    float *s_W2 = reinterpret_cast<float *>(smem);  // [no][nh]
    float *s_d = s_W2 + (size_t)no * nh;            // [nd]
    float *s_b2 = s_d + nd;                         // [no]
    float *X = s_b2 + nop + (size_t)wib * (ndp + nhp + nop + Mq);
    float *aH = X + ndp;   // production of the hidden genes: constant per image
    float *aO = aH + nhp;  // production of the outputs
    float *q = aO + nop;   // per reaction: key, then unnormalised soft weight
    for (int u = threadIdx.x; u < no * nh; u += blockDim.x) s_W2[u] = p.W2f[u];
    for (int u = threadIdx.x; u < nd; u += blockDim.x) s_d[u] = p.dvec[u];
    for (int u = threadIdx.x; u < no; u += blockDim.x) s_b2[u] = p.b2[u];
    __syncthreads();

    const int64_t i = (int64_t)blockIdx.x * W + wib;
    if (i >= p.n_traj) return;
    const int64_t n = p.n_traj;
    float *ckf = reinterpret_cast<float *>(p.ckpt);
    const float *E1 = p.E1 + (i / p.tpi) * nh;
    for (int u = lane; u < nd; u += 32) X[u] = 0.0f;
    for (int h = lane; h < nh; h += 32) aH[h] = p.k_max * sigmoid_f(E1[h]);
    __syncwarp();
    grn_soft_outputs(p, s_W2, s_b2, X, aO, lane);
    const bool bad_input = (*p.flag & kErrBadSamples) != 0;
    const uint64_t gid = p.traj_offset + (uint64_t)i;
    const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32), key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);

    double t = 0.0;
    int s = 0;
    double thr = p.S > 0 ? p.ts[0] : p.t_end;
    int status = bad_input ? SSA_TRAJ_BAD_INPUT : SSA_TRAJ_OK;
    int k = 0, draws = 0, ck_left = kGrnSoftK, ck_row = 0;
    while (!bad_input) {
        if (k >= p.max_steps) { status = SSA_TRAJ_STEP_CAP; break; }
        float E0, invZ;
        const float a0 = grn_soft_weights(p, s_d, X, aH, aO, q, k, c2, c3, key0, key1, lane, E0, invZ);
        if (!(a0 < CUDART_INF_F)) { status = SSA_TRAJ_BAD_RATE; break; }
        if (a0 == 0.0f) { status = SSA_TRAJ_ABSORBED; break; }
        const float tau = waiting_time(E0, a0);
        const double t_next = t + f2d_pos(tau);
        const bool slow = gt_nonneg(t_next, thr);
        const bool cross = slow && gt_nonneg(t_next, p.t_end);
        draws = k + 1;
        if (slow) {
            while (s < p.S && gt_nonneg(t_next, p.ts[s])) {
                float *o = obs + ((int64_t)i * p.S + s) * no;
                for (int c = lane; c < no; c += 32) o[c] = X[nh + c];
                if (record && lane == 0) p.brk_k[(int64_t)s * n + i] = k;
                ++s;
            }
            thr = s < p.S ? p.ts[s] : p.t_end;
            if (cross) break;
        }
        grn_soft_update(p, X, q, invZ, lane);
        grn_soft_outputs(p, s_W2, s_b2, X, aO, lane);
        t = t_next;
        ++k;
        if (record && --ck_left == 0) {
            ck_left = kGrnSoftK;
            ++ck_row;
            for (int u = lane; u < nd; u += 32) ckf[((int64_t)i * p.n_ckpt + ck_row) * nd + u] = X[u];
        }
    }
    __syncwarp();
    for (; s < p.S; ++s) {
        float *o = obs + ((int64_t)i * p.S + s) * no;
        for (int c = lane; c < no; c += 32) o[c] = X[nh + c];
        if (record && lane == 0) p.brk_k[(int64_t)s * n + i] = k;
    }
    if (lane == 0) {
        p.draws[i] = draws;
        p.status[i] = status;
    }
    if (record)
        for (int u = lane; u < nd; u += 32) ckf[(int64_t)i * p.n_ckpt * nd + u] = 0.0f;  // checkpoint 0: all at zero
}

// ---------------------------------------------------------------------------------------------
// soft adjoint: the exact gradient of the relaxed model (the straight-through adjoint's arithmetic along
// the soft path). Per 8-step segment the forward's own step routines re-run the states from their float
// checkpoint (the end must equal the next checkpoint bit for bit) and leave, per step, the state, the output
// propensities, the unnormalised soft weights and 1/Z in the trajectory's row of a global scratch; the walk
// back reads them instead of drawing the step again. In the relaxed model every hidden count changes every
// step, so dL/dW2 = sum_k G2_k h_k^T takes a rank-8 update of the trajectory's dW2 row once per segment.
// Shared memory holds W2 per block and ~8 KB per warp.
// ---------------------------------------------------------------------------------------------
namespace {

// one step's row of the soft adjoint's segment scratch: X [ndp] | aO [nop] | q [Mq] | 1/Z and padding [4]
__host__ __device__ inline int grn_soft_row(int nd, int no, int M)
{
    return ((nd + 3) & ~3) + ((no + 3) & ~3) + ((M + 3) & ~3) + 4;
}

}  // namespace

__global__ void __launch_bounds__(128, 5) grn_soft_adj_kernel(const GrnParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int nh = p.n_hid, no = p.n_out, nd = p.n_dyn, M = p.M;
    const int ndp = (nd + 3) & ~3, nhp = (nh + 3) & ~3, nop = (no + 3) & ~3, Mq = (M + 3) & ~3;
    const int RS = grn_soft_row(nd, no, M);
    float *s_W2 = reinterpret_cast<float *>(smem);
    float *s_d = s_W2 + (size_t)no * nh;
    float *s_b2 = s_d + nd;
    const size_t per_warp = 3 * (size_t)ndp + 2 * (size_t)nhp + (2 + kGrnSoftK) * (size_t)nop + (size_t)Mq;
    float *X = s_b2 + nop + (size_t)wib * per_warp;  // the state being stepped or differentiated
    float *lam = X + ndp;                             // dL/dX of the state after the step
    float *dlogd = lam + ndp;
    float *aH = dlogd + ndp;
    float *G1 = aH + nhp;
    float *aO = G1 + nhp;
    float *db2 = aO + nop;
    float *G2h = db2 + nop;                           // [kGrnSoftK][nop]: dL/dE2 of the segment's steps
    float *q = G2h + kGrnSoftK * nop;
    for (int u = threadIdx.x; u < no * nh; u += blockDim.x) s_W2[u] = p.W2f[u];
    for (int u = threadIdx.x; u < nd; u += blockDim.x) s_d[u] = p.dvec[u];
    for (int u = threadIdx.x; u < no; u += blockDim.x) s_b2[u] = p.b2[u];
    for (int u = lane; u < nd; u += 32) dlogd[u] = 0.0f;
    for (int u = lane; u < no; u += 32) db2[u] = 0.0f;
    __syncthreads();

    const int64_t n = p.n_traj;
    const int64_t i = (int64_t)blockIdx.x * W + wib;
    int st = -1;
    if (i < n) st = p.status[i];
    const bool active = st == SSA_TRAJ_OK || st == SSA_TRAJ_ABSORBED || st == SSA_TRAJ_STEP_CAP;
    if (i < n) {  // zeroed with the lane mapping of the per-segment updates
        float *dW2 = p.dW2t + i * (int64_t)no * nh;
        for (int h = lane; h < nh; h += 32)
            for (int o = 0; o < no; ++o) dW2[(size_t)o * nh + h] = 0.0f;
        if (!active)
            for (int h = lane; h < nh; h += 32) p.G1[i * nh + h] = 0.0f;
    }
    if (active) {
        const float *ckf = reinterpret_cast<const float *>(p.ckpt) + i * p.n_ckpt * nd;
        float *seg = p.seg + i * (int64_t)kGrnSoftK * RS;
        float *dW2 = p.dW2t + i * (int64_t)no * nh;
        const float *E1 = p.E1 + (i / p.tpi) * nh;
        const int d = p.draws[i];
        // a finished run's last draw is the crossing one, which moves no observed state
        const int L = (st == SSA_TRAJ_OK) ? d - 1 : d;
        for (int u = lane; u < nd; u += 32) lam[u] = 0.0f;
        for (int h = lane; h < nh; h += 32) {
            aH[h] = p.k_max * sigmoid_f(E1[h]);
            G1[h] = 0.0f;
        }
        __syncwarp();
        const uint64_t gid = p.traj_offset + (uint64_t)i;
        const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32), key0 = (uint32_t)p.seed,
                       key1 = (uint32_t)(p.seed >> 32);
        const float invT = p.invT;
        const float *gl = p.dl_dobs + i * p.dl_stride;
        int s_hi = p.S - 1;
        int brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
        int mism = 0;
        for (int c = L / kGrnSoftK; c >= 0; --c) {
            const int k0 = c * kGrnSoftK, k1 = min(k0 + kGrnSoftK - 1, L);
            for (int u = lane; u < nd; u += 32) X[u] = ckf[(int64_t)c * nd + u];
            __syncwarp();
            for (int kk = k0; kk <= k1; ++kk) {  // re-run the segment with the forward's routines
                float *row = seg + (kk - k0) * RS;
                for (int u = lane; u < nd; u += 32) row[u] = X[u];
                if (kk < L) {
                    grn_soft_outputs(p, s_W2, s_b2, X, aO, lane);
                    float E0, invZ;
                    grn_soft_weights(p, s_d, X, aH, aO, q, kk, c2, c3, key0, key1, lane, E0, invZ);
                    for (int o = lane; o < no; o += 32) row[ndp + o] = aO[o];
                    for (int j = lane; j < M; j += 32) row[ndp + nop + j] = q[j];
                    if (lane == 0) row[ndp + nop + Mq] = invZ;
                    grn_soft_update(p, X, q, invZ, lane);
                }
            }
            if (k1 < L) {
                int bad = 0;
                for (int u = lane; u < nd; u += 32) bad += X[u] != ckf[(int64_t)(c + 1) * nd + u];
                mism += __reduce_add_sync(0xffffffffu, bad);
            }
            __syncwarp();  // the scratch rows were written lane-strided; the walk reads them across lanes
            for (int k = k1; k >= k0; --k) {
                const float *row = seg + (k - k0) * RS;
                float *G2 = G2h + (k - k0) * nop;
                for (int o = lane; o < no; o += 32) G2[o] = 0.0f;
                const int s_top = s_hi;
                while (s_hi >= 0 && brk_next == k) {
                    --s_hi;
                    brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
                }
                if (k < L) {
                    for (int u = lane; u < nd; u += 32) X[u] = row[u];
                    for (int o = lane; o < no; o += 32) aO[o] = row[ndp + o];
                    const float invZ = row[ndp + nop + Mq];
                    // W = sum_j q_j w_j / Z with w_j = +lam_s (production) or -lam_s (degradation)
                    float Wp = 0.0f;
                    for (int j = lane; j < M; j += 32) {
                        const float qj = row[ndp + nop + j];
                        q[j] = qj;
                        Wp += qj * (j < nd ? lam[j] : -lam[j - nd]);
                    }
                    const float Wbar = warp_sum(Wp) * invZ;
                    __syncwarp();
                    // choice-path adjoints psi_j = dL/dlog a_j of the productions (HOLD readout: no waiting-time path)
                    for (int j = lane; j < nd; j += 32) {
                        const float psi = q[j] > 0.0f ? q[j] * invZ * (lam[j] - Wbar) * invT : 0.0f;
                        if (j < nh)
                            G1[j] += psi * (1.0f - __fdividef(aH[j], p.k_max));
                        else
                            G2[j - nh] = psi * (1.0f - __fdividef(aO[j - nh], p.k_max));
                    }
                    __syncwarp();
                    // the degradations: psi of d_u max(X_u, 0); a weight q > 0 implies a > 0, so X_u > 0 there
                    for (int u = lane; u < nd; u += 32) {
                        const float qd = q[nd + u];
                        const float psi = qd > 0.0f ? qd * invZ * (-lam[u] - Wbar) * invT : 0.0f;
                        dlogd[u] += psi;
                        float acc = qd > 0.0f ? __fdividef(psi, X[u]) : 0.0f;
                        if (u < nh)
                            for (int o = 0; o < no; ++o) acc += s_W2[(size_t)o * nh + u] * G2[o];
                        lam[u] += acc;
                    }
                }
                __syncwarp();
                // HOLD samples of the outputs at state k
                for (int s = s_hi + 1; s <= s_top; ++s)
                    for (int o = lane; o < no; o += 32) lam[nh + o] += gl[(int64_t)s * no + o];
                __syncwarp();
            }
            // the segment's rank-(k1 - k0 + 1) update of dL/dW2 and dL/db2
            const int len = k1 - k0 + 1;
            for (int h = lane; h < nh; h += 32) {
                float xs[kGrnSoftK];
#pragma unroll
                for (int r = 0; r < kGrnSoftK; ++r) xs[r] = r < len ? seg[r * RS + h] : 0.0f;
                for (int o = 0; o < no; ++o) {
                    float acc = dW2[(size_t)o * nh + h];
#pragma unroll
                    for (int r = 0; r < kGrnSoftK; ++r)
                        if (r < len) acc = __fmaf_rn(G2h[r * nop + o], xs[r], acc);
                    dW2[(size_t)o * nh + h] = acc;
                }
            }
            for (int o = lane; o < no; o += 32)
                for (int r = 0; r < len; ++r) db2[o] += G2h[r * nop + o];
            __syncwarp();
        }
        for (int h = lane; h < nh; h += 32) p.G1[i * nh + h] = G1[h];
        if (lane == 0 && mism) atomicAdd(p.mismatch, mism);
    }
    __syncthreads();
    // fixed-order sum over the block's warps: [db2 | dlogd]
    const int red = no + nd;
    const float *base0 = s_b2 + nop;
    for (int u = threadIdx.x; u < red; u += blockDim.x) {
        float acc = 0.0f;
        for (int w = 0; w < W; ++w) {
            const float *wp = base0 + w * per_warp;
            acc += u < no ? wp[3 * ndp + 2 * nhp + nop + u] : wp[2 * ndp + (u - no)];
        }
        p.partial[(int64_t)blockIdx.x * red + u] = acc;
    }
}

// ---------------------------------------------------------------------------------------------
// backward: one warp per trajectory, reverse walk
// ---------------------------------------------------------------------------------------------
#ifndef SSA_GRN_ADJ_BLOCKS
#define SSA_GRN_ADJ_BLOCKS 6  // resident blocks per SM the adjoint is compiled for (36 KB of shared memory each)
#endif
__global__ void __launch_bounds__(128, SSA_GRN_ADJ_BLOCKS) grn_adj_kernel(const GrnParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int nh = p.n_hid, no = p.n_out, nd = p.n_dyn, Mp = p.Mp;
    float *s_d = reinterpret_cast<float *>(smem);
    float *s_b2 = s_d + nd;
    const int ndp = (nd + 3) & ~3, nhp = (nh + 3) & ~3, nop = (no + 3) & ~3;
    // per warp (words): X, lam, ctd [ndp each], aH, G1 [nhp each], E2acc [2 nop], aO, G2, R, db2 [nop each],
    // lj [Mp], dlogd [ndp]. dL/dW2 goes to the trajectory's own row of p.dW2t (global, L2-resident while the
    // warp works on it), which keeps the per-warp shared memory independent of n_out x n_hid.
    const size_t per_warp = 4 * (size_t)ndp + 2 * (size_t)nhp + 6 * (size_t)nop + (size_t)Mp;
    unsigned char *wb = smem + ((4 * ((size_t)nd + nop) + 15) & ~(size_t)15);  // shared-space offsets (see the forward)
    float *wbase = reinterpret_cast<float *>(wb) + wib * per_warp;
    int *X = reinterpret_cast<int *>(wbase);
    float *lam = wbase + ndp;
    float *ctd = lam + ndp;
    float *aH = ctd + ndp;
    float *G1 = aH + nhp;
    long long *E2acc = reinterpret_cast<long long *>(G1 + nhp);
    float *aO = reinterpret_cast<float *>(E2acc + nop);
    float *G2 = aO + nop;
    float *R = G2 + nop;
    float *db2 = R + nop;
    float *lj = db2 + nop;
    float *dlogd = lj + Mp;
    const int *__restrict__ W2fix = p.W2fix;
    const float *__restrict__ W2f = p.W2f;

    for (int q = threadIdx.x; q < nd; q += blockDim.x) s_d[q] = p.dvec[q];
    for (int q = threadIdx.x; q < no; q += blockDim.x) s_b2[q] = p.b2[q];
    for (int q = lane; q < nd; q += 32) dlogd[q] = 0.0f;
    for (int q = lane; q < no; q += 32) db2[q] = 0.0f;
    __syncthreads();

    const int64_t n = p.n_traj;
    const int64_t i = (int64_t)blockIdx.x * W + wib;
    int st = -1;
    if (i < n) st = p.status[i];
    const bool active = st == SSA_TRAJ_OK || st == SSA_TRAJ_ABSORBED || st == SSA_TRAJ_STEP_CAP;
    float *dW2 = p.dW2t + (i < n ? i : 0) * (int64_t)no * nh;
    if (i < n)
        for (int q = lane; q < no * nh; q += 32) dW2[q] = 0.0f;
    if (active) {
        const float scale = exp2f((float)p.grid[0]);
        const float inv_kmax = 1.0f / p.k_max;
        const float *E1 = p.E1 + (i / p.tpi) * nh;
        const int d = p.draws[i];
        const int L = (st == SSA_TRAJ_OK) ? d - 1 : d;
        for (int s = lane; s < nd; s += 32) {
            X[s] = p.xfinal[(int64_t)s * n + i];
            lam[s] = 0.0f;
        }
        for (int h = lane; h < nh; h += 32) {
            aH[h] = p.k_max * sigmoid_f(E1[h]);
            G1[h] = 0.0f;
        }
        __syncwarp();
        // E2 at the final state, exactly (integer fixed point)
        for (int o = lane; o < no; o += 32) {
            long long acc = 0;
            for (int h = 0; h < nh; ++h) acc += (long long)__ldg(W2fix + o * nh + h) * X[h];
            E2acc[o] = acc;
            aO[o] = p.k_max * sigmoid_f(e2_value(acc, scale, s_b2[o]));
            R[o] = 0.0f;
        }
        __syncwarp();
        const uint64_t gid = p.traj_offset + (uint64_t)i;
        const uint32_t c2 = (uint32_t)gid, c3 = (uint32_t)(gid >> 32), key0 = (uint32_t)p.seed,
                       key1 = (uint32_t)(p.seed >> 32);
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
        int brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
        int mism = 0;
        int ck_row = L / p.K, ck_off = L - ck_row * p.K;
        for (int k = L; k >= 0; --k) {
            const bool draw = (k < L) || (st == SSA_TRAJ_OK);
            const int s_top = s_hi;
            while (s_hi >= 0 && brk_next == k) {
                --s_hi;
                brk_next = s_hi >= 0 ? p.brk_k[(int64_t)s_hi * n + i] : -1;
            }
            if (draw) {
                const int jk = event_at(k);
                // pass 1: the forward's propensities and race, log2 keys
                float ab = 0.0f, Eb = 1.0f, lmaxp = -CUDART_INF_F;
                int jb = -1;
                for (int b = lane; b < p.nb; b += 32) {
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)k, c2, c3), key0, key1);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        // predicated as in the forward (j = -1 and a = 0 add nothing and have key -inf)
                        const int j = 4 * b + q - 1;
                        const float E = neg_log_unit(u01(word_of(r, q)));
                        const float a = j < 0 ? 0.0f : grn_prop(p, max(j, 0), aH, aO, X, s_d);
                        race(a, E, j, ab, Eb, jb);
                        const float l = a > 0.0f ? __log2f(a) - __log2f(E) : -CUDART_INF_F;
                        lmaxp = fmaxf(lmaxp, l);
                        if (j >= 0 && j < p.M) lj[j] = l;
                    }
                }
                warp_race_combine(ab, Eb, jb);
                const float lmax = warp_max(lmaxp);
                mism += (jb != jk);
                __syncwarp();
                // pass 2: soft-sample weights q_j = exp2((l_j - l_max)/T), Z = sum q, W = sum q w with
                // w_j = +lam_s (production of s) or -lam_s (degradation of s); one loop per reaction range, so
                // neither pass branches on the kind of reaction
                float Zp = 0.0f, Wp = 0.0f;
                for (int j = lane; j < nd; j += 32) {
                    const float l = lj[j];
                    const float qv = l > -CUDART_INF_F ? exp2f((l - lmax) * invT) : 0.0f;
                    lj[j] = qv;
                    Zp += qv;
                    Wp = fmaf(qv, lam[j], Wp);
                }
                for (int s2 = lane; s2 < nd; s2 += 32) {
                    const float l = lj[nd + s2];
                    const float qv = l > -CUDART_INF_F ? exp2f((l - lmax) * invT) : 0.0f;
                    lj[nd + s2] = qv;
                    Zp += qv;
                    Wp = fmaf(-qv, lam[s2], Wp);
                }
                const float Z = warp_sum(Zp), Wq = warp_sum(Wp);
                const float invZ = __fdividef(1.0f, Z), Wbar = Wq * invZ;
                const float cz = invZ * invT;
                // pass 3: choice-path adjoints psi_j = q_j / Z (w_j - W/Z) / T per reaction (HOLD readout: no
                // waiting-time path); d log(k_max sigma(E)) / dE = 1 - sigma(E)
                for (int h = lane; h < nh; h += 32) {
                    const float psi = lj[h] * cz * (lam[h] - Wbar);
                    G1[h] = fmaf(psi, 1.0f - aH[h] * inv_kmax, G1[h]);
                }
                for (int o = lane; o < no; o += 32) {
                    const float psi = lj[nh + o] * cz * (lam[nh + o] - Wbar);
                    G2[o] = psi * (1.0f - aO[o] * inv_kmax);
                }
                for (int s2 = lane; s2 < nd; s2 += 32) {
                    const float psi = lj[nd + s2] * cz * (-lam[s2] - Wbar);
                    dlogd[s2] += psi;
                    ctd[s2] = X[s2] > 0 ? __fdividef(psi, int2f(X[s2])) : 0.0f;  // a = d X > 0 where X > 0
                }
                __syncwarp();
                for (int o = lane; o < no; o += 32) {
                    db2[o] += G2[o];
                    R[o] += G2[o];
                }
                // lam_h += (W2^T G2)_h for the hidden genes; every species adds its degradation term
                if (no <= kGrnOutBatch) {
                    // up to kGrnOutBatch outputs: the column's loads are issued together (one L1 latency per
                    // hidden gene instead of one per output), then summed in output order
                    for (int h = lane; h < nh; h += 32) {
                        float w[kGrnOutBatch];
#pragma unroll
                        for (int o = 0; o < kGrnOutBatch; ++o) w[o] = o < no ? __ldg(W2f + o * nh + h) : 0.0f;
                        float acc = ctd[h];
#pragma unroll
                        for (int o = 0; o < kGrnOutBatch; ++o)
                            if (o < no) acc = fmaf(w[o], G2[o], acc);
                        lam[h] += acc;
                    }
                } else {
                    for (int h = lane; h < nh; h += 32) {
                        float acc = ctd[h];
                        for (int o = 0; o < no; ++o) acc = fmaf(__ldg(W2f + o * nh + h), G2[o], acc);
                        lam[h] += acc;
                    }
                }
                for (int s2 = nh + lane; s2 < nd; s2 += 32) lam[s2] += ctd[s2];
            }
            __syncwarp();
            // HOLD samples of the outputs at state k
            for (int s = s_hi + 1; s <= s_top; ++s)
                for (int o = lane; o < no; o += 32) lam[nh + o] += gl[(int64_t)s * no + o];
            if (ck_off == 0) {
                const int *ck = p.ckpt + (int64_t)ck_row * nd * n + i;
                int bad = 0;
                for (int q = lane; q < nd; q += 32) bad += (ck[(int64_t)q * n] != X[q]);
                mism += __reduce_add_sync(0xffffffffu, bad);
                --ck_row;
                ck_off = p.K;
            }
            --ck_off;
            __syncwarp();
            if (k > 0) {
                // undo event k-1 (state k -> k-1); a hidden change adds delta R to dW2[:, i]
                const int jp = event_at(k - 1);
                const int sp = jp < nd ? jp : jp - nd;
                const int delta = jp < nd ? 1 : -1;
                if (lane == 0) X[sp] -= delta;
                if (sp < nh) {
                    for (int o = lane; o < no; o += 32) {
                        dW2[o * nh + sp] += (float)delta * R[o];
                        E2acc[o] -= (long long)delta * __ldg(W2fix + o * nh + sp);
                        aO[o] = p.k_max * sigmoid_f(e2_value(E2acc[o], scale, s_b2[o]));
                    }
                }
            }
            __syncwarp();
        }
        for (int h = lane; h < nh; h += 32) p.G1[i * nh + h] = G1[h];
        if (lane == 0 && mism) atomicAdd(p.mismatch, mism);
    } else if (i < n) {
        for (int h = lane; h < nh; h += 32) p.G1[i * nh + h] = 0.0f;
    }
    __syncthreads();
    // fixed-order sum over the block's warps: [db2 | dlogd]
    const int red = no + nd;
    float *base0 = reinterpret_cast<float *>(wb);
    for (int q = threadIdx.x; q < red; q += blockDim.x) {
        float acc = 0.0f;
        for (int w = 0; w < W; ++w) {
            const float *wp = base0 + w * per_warp;
            acc += q < no ? wp[3 * ndp + 2 * nhp + 5 * nop + q] : wp[3 * ndp + 2 * nhp + 6 * nop + Mp + (q - no)];
        }
        p.partial[(int64_t)blockIdx.x * red + q] = acc;
    }
}

// per-image sums of dL/dE1 (fixed order over the image's trajectories), db1, and the transposed
// hi/lo bf16 limbs G^T for the tensor-core dW1 = G^T x
__global__ void grn_image_grad_kernel(const float *G1, int64_t n_img, int64_t tpi, int nh, int n_img_pad, float *Gimg,
                                      uint16_t *Gt_hi, uint16_t *Gt_lo)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)nh * n_img_pad;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int h = (int)(q / n_img_pad);
        const int64_t img = q % n_img_pad;
        float acc = 0.0f;
        if (img < n_img)
            for (int64_t t = 0; t < tpi; ++t) acc += G1[(img * tpi + t) * nh + h];
        if (img < n_img) Gimg[img * nh + h] = acc;
        const uint16_t hi = float_to_bf16_rn(acc);
        Gt_hi[q] = hi;
        Gt_lo[q] = float_to_bf16_rn(acc - bf16_to_float(hi));
    }
}

__global__ void grn_db1_kernel(const float *Gimg, int64_t n_img, int nh, float *db1)
{
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int64_t img = 0; img < n_img; ++img) acc += Gimg[img * nh + h];
        db1[h] = acc;
    }
}

__global__ void grn_transpose_x_kernel(const int32_t *x_img, int64_t n_img, int n_in, int n_img_pad, uint16_t *xT)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n_in * n_img_pad;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(q / n_img_pad);
        const int64_t img = q % n_img_pad;
        xT[q] = float_to_bf16_exact(img < n_img ? (float)x_img[img * n_in + p] : 0.0f);
    }
}

__global__ void grn_split_partials_kernel(const float *red, int no, int nd, float *db2, float *dlogd)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < no + nd; q += gridDim.x * blockDim.x) {
        if (q < no) db2[q] = red[q];
        else dlogd[q - no] = red[q];
    }
}

}  // namespace ssa

// =============================================================================================
// C ABI
// =============================================================================================
using namespace ssa;

namespace {

// N-tile of the tensor-core dW1 = G^T x (n_in columns)
int grn_dw1_nt(const ssa_grn *g) { return (g->n_in % 112 == 0) ? 112 : 64; }

WsLayout grn_layout(const ssa_grn *g, int64_t n_img, int64_t tpi, int32_t S, const ssa_fwd_opts *o)
{
    WsLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = (off + bytes + 255) / 256 * 256;
        return at;
    };
    const int64_t n = n_img * tpi;
    L.n_in_pad = (g->n_in + 7) / 8 * 8;
    L.n_img_pad = (int)((n_img + 7) / 8 * 8);
    L.limbs = kGrnLimbs;
    L.red_len = g->n_out + g->n_dyn;
    L.M_pad = g->Mp;
    L.flag = take(16 * sizeof(int));
    L.counts = take(SSA_TRAJ_N_CODES * sizeof(unsigned long long));
    L.k_rates = take(16);
    L.ts = take((size_t)(S > 0 ? S : 1) * sizeof(double));
    L.obs_sp = take(16);
    L.draws = take((size_t)(n > 0 ? n : 1) * sizeof(int));
    L.status = take((size_t)(n > 0 ? n : 1) * sizeof(int));
    L.E1 = take((size_t)(n_img > 0 ? n_img : 1) * g->n_hid * sizeof(float));
    L.W1L = take((size_t)kGrnLimbs * g->n_hid * L.n_in_pad * 2);
    L.xb = take((size_t)(n_img > 0 ? n_img : 1) * L.n_in_pad * 2);
    L.W2fix = take((size_t)g->n_out * g->n_hid * 4);
    L.W2f = take((size_t)g->n_out * g->n_hid * 4);
    L.dvec = take((size_t)g->n_dyn * 4);
    L.grid = take(16 * sizeof(int));
    // split-K partial sums of E1 (forward) and of dW1 (backward), when the product fills too few SMs
    size_t tc_words = n_img > 0 ? 2 * tc_split_words((int)n_img, g->n_hid, g->n_in, 64) : 0;  // (lo, hi) pairs
    if (o->record && n_img > 0)
        tc_words = std::max(tc_words, tc_split_words(g->n_hid, g->n_in, (int)n_img, grn_dw1_nt(g)));
    L.tcpart = take(std::max<size_t>(tc_words, 1) * sizeof(double));
    if (o->record) {
        // the soft forward keeps float checkpoints every 8 steps; the hard one int counts every K
        const int K = o->selector == SSA_SELECT_SOFT ? kGrnSoftK : o->ckpt_interval > 0 ? o->ckpt_interval : 64;
        L.ev_rows = (o->max_steps + 7) / 8;
        L.n_ckpt = o->max_steps / K + 1;
        L.max_blocks = (n + kGrnWarps - 1) / kGrnWarps;
        L.xfinal = take((size_t)g->n_dyn * n * 4);
        L.ev = take((size_t)L.ev_rows * n * sizeof(uint4));
        L.ckpt = take((size_t)L.n_ckpt * g->n_dyn * n * 4);
        L.brk_k = take((size_t)S * n * 4);
        L.brk_a = take(16);
        L.partial = take((size_t)(L.max_blocks > 0 ? L.max_blocks : 1) * L.red_len * 4);
        L.dA = take(16);
        L.G1 = take((size_t)(n > 0 ? n : 1) * g->n_hid * 4);
        L.Gimg = take((size_t)(n_img > 0 ? n_img : 1) * g->n_hid * 4);
        L.Gt = take((size_t)2 * g->n_hid * L.n_img_pad * 2);
        L.xT = take((size_t)g->n_in * L.n_img_pad * 2);
        L.red = take((size_t)L.red_len * 4);
        L.dW2t = take((size_t)(n > 0 ? n : 1) * g->n_out * g->n_hid * 4);
        L.dW2_chunk = std::max<int64_t>(256, (n + 65534) / 65535);
        L.dW2p = take((size_t)((n + L.dW2_chunk - 1) / L.dW2_chunk + 1) * g->n_out * g->n_hid * 4);
        if (o->selector == SSA_SELECT_SOFT)
            L.soft_seg = take((size_t)(n > 0 ? n : 1) * kGrnSoftK * grn_soft_row(g->n_dyn, g->n_out, g->M) * 4);
    }
    L.total = off;
    return L;
}

size_t grn_fwd_smem(const ssa_grn *g)
{
    const int ndp = (g->n_dyn + 3) & ~3, nhp = (g->n_hid + 3) & ~3, nop = (g->n_out + 3) & ~3;
    return 4 * ((size_t)g->n_out * g->n_hid + g->n_dyn + nop) + 16 + 4 * (size_t)kGrnWarps * (ndp + nhp + 3 * (size_t)nop);
}

size_t grn_soft_fwd_smem(const ssa_grn *g)
{
    const int ndp = (g->n_dyn + 3) & ~3, nhp = (g->n_hid + 3) & ~3, nop = (g->n_out + 3) & ~3, Mq = (g->M + 3) & ~3;
    return 4 * ((size_t)g->n_out * g->n_hid + g->n_dyn + nop) + 4 * (size_t)kGrnWarps * (ndp + nhp + nop + Mq);
}

size_t grn_soft_adj_smem(const ssa_grn *g)
{
    const int ndp = (g->n_dyn + 3) & ~3, nhp = (g->n_hid + 3) & ~3, nop = (g->n_out + 3) & ~3, Mq = (g->M + 3) & ~3;
    const size_t per_warp = 3 * (size_t)ndp + 2 * (size_t)nhp + (2 + kGrnSoftK) * (size_t)nop + (size_t)Mq;
    return 4 * ((size_t)g->n_out * g->n_hid + g->n_dyn + nop + (size_t)kGrnWarps * per_warp);
}

// shared memory one CTA may hold on sm_103a
constexpr size_t kGrnMaxSmem = 227 * 1024;

size_t grn_adj_smem(const ssa_grn *g)
{
    const int ndp = (g->n_dyn + 3) & ~3, nhp = (g->n_hid + 3) & ~3, nop = (g->n_out + 3) & ~3;
    const size_t per_warp = 4 * (size_t)ndp + 2 * (size_t)nhp + 6 * (size_t)nop + (size_t)g->Mp;
    return 4 * ((size_t)g->n_dyn + nop) + 16 + 4 * (size_t)kGrnWarps * per_warp;
}

#define GRN_CUDA_TRY(expr)                                                                              \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess) return set_error(SSA_ERR_CUDA, cudaGetErrorString(e_));                   \
    } while (0)

}  // namespace

extern "C" ssa_status ssa_grn_create(int32_t n_in, int32_t n_hid, int32_t n_out, float k_max, ssa_grn **out)
{
    if (!out) return set_error(SSA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_hid < 1 || n_out < 1 || n_in > (1 << 16) || n_hid > 4096 || n_out > 1024)
        return set_error(SSA_ERR_INVALID_ARG, "GRN sizes out of range");
    if (2 * (n_hid + n_out) > 65535) return set_error(SSA_ERR_UNSUPPORTED, "too many reactions for the uint16 log");
    // exactness of the tensor-core contraction: one 6-bit limb times 8-bit counts, summed over n_in,
    // stays below 2^24 quanta
    if ((int64_t)n_in * 63 * 256 >= (int64_t)1 << 24) return set_error(SSA_ERR_UNSUPPORTED, "n_in above 1040");
    if (!(k_max > 0.0f)) return set_error(SSA_ERR_INVALID_ARG, "k_max must be positive");
    ssa_grn *g = new (std::nothrow) ssa_grn();
    if (!g) return set_error(SSA_ERR_CUDA, "host allocation failed");
    g->n_in = n_in;
    g->n_hid = n_hid;
    g->n_out = n_out;
    g->n_dyn = n_hid + n_out;
    g->M = 2 * g->n_dyn;
    g->Mp = (g->M + 4) / 4 * 4;
    g->k_max = k_max;
    *out = g;
    return SSA_OK;
}

extern "C" void ssa_grn_destroy(ssa_grn *g) { delete g; }

extern "C" size_t ssa_grn_workspace_bytes(const ssa_grn *g, int64_t n_img, int64_t traj_per_img, int32_t n_samples,
                                          const ssa_fwd_opts *opts)
{
    if (!g || n_img < 0 || traj_per_img < 1 || n_samples < 0 || !opts || opts->max_steps < 1) return 0;
    return grn_layout(g, n_img, traj_per_img, n_samples, opts).total;
}

extern "C" ssa_status ssa_grn_forward(const ssa_grn *g, const uint16_t *W1, const float *b1, const uint16_t *W2,
                                      const float *b2, const float *log_d, int64_t n_img, int64_t traj_per_img,
                                      int64_t traj_offset, const int32_t *x_img, double t_end,
                                      const double *sample_times, int32_t S, uint64_t seed, const ssa_fwd_opts *opts,
                                      void *workspace, size_t workspace_bytes, int32_t *obs_out, int32_t *draws_out,
                                      int32_t *status_out, void *stream, ssa_run **run_out)
{
    if (run_out) *run_out = nullptr;
    if (!g || !opts) return set_error(SSA_ERR_INVALID_ARG, "NULL network or options");
    if (opts->readout != SSA_READOUT_HOLD) return set_error(SSA_ERR_UNSUPPORTED, "the GRN reads out with HOLD only");
    const bool soft = opts->selector == SSA_SELECT_SOFT;
    if (!soft && (opts->selector != SSA_SELECT_GUMBEL || opts->temperature != 0.0f))
        return set_error(SSA_ERR_UNSUPPORTED, "the GRN runs the Gumbel-max selector or the soft forward");
    if (soft && (!(opts->temperature > 0.0f) || !(opts->temperature < 3.0e38f)))
        return set_error(SSA_ERR_UNSUPPORTED, "the GRN's soft forward needs T > 0");
    if (soft && (grn_soft_fwd_smem(g) > kGrnMaxSmem || (opts->record && grn_soft_adj_smem(g) > kGrnMaxSmem)))
        return set_error(SSA_ERR_UNSUPPORTED, "the GRN's soft path keeps W2 (and a recorded run dL/dW2) in shared memory: "
                                              "n_out * n_hid too large");
    if (opts->max_steps < 1 || opts->max_steps > 0x7fffffffLL || (opts->ckpt_interval % 8) || opts->ckpt_interval < 0)
        return set_error(SSA_ERR_INVALID_ARG, "invalid options");
    if (n_img < 0 || traj_per_img < 1 || traj_offset < 0 || S < 0 || !(t_end >= 0.0) || !(t_end < 1e300))
        return set_error(SSA_ERR_INVALID_ARG, "bad sizes or horizon");
    if (!W1 || !b1 || !W2 || !b2 || !log_d || (n_img > 0 && !x_img) || (S > 0 && !sample_times))
        return set_error(SSA_ERR_INVALID_ARG, "NULL input pointer");
    const int64_t n = n_img * traj_per_img;
    if (n > 0 && S > 0 && !obs_out) return set_error(SSA_ERR_INVALID_ARG, "obs_out is NULL");
    const WsLayout L = grn_layout(g, n_img, traj_per_img, S, opts);
    if (!workspace || workspace_bytes < L.total) return set_error(SSA_ERR_WORKSPACE, "workspace too small");
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return set_error(SSA_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if ((reinterpret_cast<uintptr_t>(W1) | reinterpret_cast<uintptr_t>(W2)) & 1)
        return set_error(SSA_ERR_INVALID_ARG, "weights must be 2-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    int *flag = reinterpret_cast<int *>(ws + L.flag);
    int *grid = reinterpret_cast<int *>(ws + L.grid);
    GRN_CUDA_TRY(cudaMemsetAsync(flag, 0, 16 * sizeof(int), st));
    const int init_grid[4] = {0, 255, 0, 0};
    GRN_CUDA_TRY(cudaMemcpyAsync(grid, init_grid, sizeof(init_grid), cudaMemcpyHostToDevice, st));
    if (S > 0) GRN_CUDA_TRY(cudaMemcpyAsync(ws + L.ts, sample_times, (size_t)S * 8, cudaMemcpyDeviceToDevice, st));
    GRN_CUDA_TRY(launch_validate_inputs(reinterpret_cast<const double *>(ws + L.ts), S, t_end, nullptr, 0, g->n_dyn,
                                        0, flag, st));
    grn_exponents_kernel<<<64, 256, 0, st>>>(W1, (int64_t)g->n_hid * g->n_in, W2, (int64_t)g->n_out * g->n_hid, grid);
    grn_prepare_kernel<<<256, 256, 0, st>>>(W1, W2, x_img, log_d, g->n_in, g->n_hid, g->n_out, n_img, L.n_in_pad,
                                            reinterpret_cast<uint16_t *>(ws + L.W1L), reinterpret_cast<int *>(ws + L.W2fix),
                                            reinterpret_cast<float *>(ws + L.W2f), reinterpret_cast<uint16_t *>(ws + L.xb),
                                            reinterpret_cast<float *>(ws + L.dvec), grid);
    GRN_CUDA_TRY(cudaGetLastError());
    // E1 = W1 x + b1 on the tensor cores: one accumulator per limb, summed in binary64
    if (n_img > 0) {
        TcMaps maps;
        memset(&maps, 0, sizeof(maps));
        if (!tc_make_map(&maps.a[0], ws + L.xb, (int)n_img, g->n_in, L.n_in_pad, 128))
            return set_error(SSA_ERR_CUDA, "tensor map encoding failed");
        for (int t = 0; t < kGrnLimbs; ++t)
            if (!tc_make_map(&maps.b[t], ws + L.W1L + (size_t)t * g->n_hid * L.n_in_pad * 2, g->n_hid, g->n_in,
                             L.n_in_pad, 64))
                return set_error(SSA_ERR_CUDA, "tensor map encoding failed");
        TcArgs args{(int)n_img, g->n_hid, g->n_in, 1, kGrnLimbs, kGrnLimbs, 1, b1,
                    reinterpret_cast<float *>(ws + L.E1), g->n_hid, flag + 4};
        args.Dpart = reinterpret_cast<double *>(ws + L.tcpart);  // split K when the tiles underfill the SMs
        args.limb_grid = grid + 4;  // limb t is an integer multiple of 2^(g1 + 6 t): summed exactly in int64
        args.limb_bits = kGrnLimbBits;
        GRN_CUDA_TRY(tc_gemm_launch(maps, args, 64, st));
    }
    GrnParams p{};
    p.n_in = g->n_in;
    p.n_hid = g->n_hid;
    p.n_out = g->n_out;
    p.n_dyn = g->n_dyn;
    p.M = g->M;
    p.Mp = g->Mp;
    p.nb = (g->M + 4) >> 2;
    p.k_max = g->k_max;
    p.n_traj = n;
    p.tpi = traj_per_img;
    p.traj_offset = (uint64_t)traj_offset;
    p.seed = seed;
    p.E1 = reinterpret_cast<const float *>(ws + L.E1);
    p.W2fix = reinterpret_cast<const int *>(ws + L.W2fix);
    p.W2f = reinterpret_cast<const float *>(ws + L.W2f);
    p.b2 = b2;
    p.dvec = reinterpret_cast<const float *>(ws + L.dvec);
    p.grid = grid + 3;
    p.t_end = t_end;
    p.ts = reinterpret_cast<const double *>(ws + L.ts);
    p.S = S;
    p.max_steps = opts->max_steps;
    p.obs_out = obs_out;
    p.draws = reinterpret_cast<int *>(ws + L.draws);
    p.status = reinterpret_cast<int *>(ws + L.status);
    p.flag = flag;
    p.err = flag + 1;
    p.K = opts->ckpt_interval > 0 ? opts->ckpt_interval : 64;
    if (opts->record) {
        p.ev = reinterpret_cast<uint4 *>(ws + L.ev);
        p.ckpt = reinterpret_cast<int *>(ws + L.ckpt);
        p.brk_k = reinterpret_cast<int *>(ws + L.brk_k);
        p.xfinal = reinterpret_cast<int *>(ws + L.xfinal);
        p.n_ckpt = L.n_ckpt;
    }
    if (n > 0 && soft) {
        p.invT = 1.0f / opts->temperature;
        const size_t smem = grn_soft_fwd_smem(g);
        GRN_CUDA_TRY(cudaFuncSetAttribute(grn_soft_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        grn_soft_fwd_kernel<<<(unsigned)((n + kGrnWarps - 1) / kGrnWarps), 32 * kGrnWarps, smem, st>>>(
            p, reinterpret_cast<float *>(obs_out), opts->record);
        GRN_CUDA_TRY(cudaGetLastError());
    } else if (n > 0) {
        const size_t smem = grn_fwd_smem(g);
        GRN_CUDA_TRY(cudaFuncSetAttribute(grn_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        grn_fwd_kernel<<<(unsigned)((n + kGrnWarps - 1) / kGrnWarps), 32 * kGrnWarps, smem, st>>>(p, opts->record);
        GRN_CUDA_TRY(cudaGetLastError());
    }
    if (n > 0 && draws_out) GRN_CUDA_TRY(cudaMemcpyAsync(draws_out, p.draws, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    if (n > 0 && status_out) GRN_CUDA_TRY(cudaMemcpyAsync(status_out, p.status, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    if (run_out) {
        ssa_run *run = new (std::nothrow) ssa_run();
        if (!run) return set_error(SSA_ERR_CUDA, "host allocation failed");
        run->net = nullptr;
        run->variant = 32;
        run->grn = g;
        run->n_img = n_img;
        run->traj_per_img = traj_per_img;
        run->n_traj = n;
        run->traj_offset = (uint64_t)traj_offset;
        run->seed = seed;
        run->S = S;
        run->n_obs = g->n_out;
        run->opts = *opts;
        run->t_end = t_end;
        run->ws = ws;
        run->L = L;
        run->x_img = x_img;
        run->b2 = b2;
        *run_out = run;
    }
    return SSA_OK;
}

extern "C" ssa_status ssa_grn_backward(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride, float temperature,
                                       float *dW1, float *db1, float *dW2, float *db2, float *dlog_d, void *stream)
{
    if (!run || !run->grn) return set_error(SSA_ERR_INVALID_ARG, "not a GRN run");
    if (!run->opts.record) return set_error(SSA_ERR_STATE, "the forward was not recorded");
    if (!(temperature > 0.0f)) return set_error(SSA_ERR_INVALID_ARG, "temperature must be > 0");
    const bool soft = run->opts.selector == SSA_SELECT_SOFT;
    if (soft && temperature != run->opts.temperature)
        return set_error(SSA_ERR_INVALID_ARG, "the gradient of the soft forward is taken at the forward's temperature");
    if (!dW1 || !db1 || !dW2 || !db2 || !dlog_d) return set_error(SSA_ERR_INVALID_ARG, "NULL gradient output");
    if (dl_traj_stride != 0 && dl_traj_stride < (int64_t)run->S * run->n_obs)
        return set_error(SSA_ERR_INVALID_ARG, "dl_traj_stride must be 0 or >= n_samples * n_out");
    if (!dl_dobs && run->n_traj > 0 && run->S > 0) return set_error(SSA_ERR_INVALID_ARG, "dl_dobs is NULL");
    const ssa_grn *g = run->grn;
    const WsLayout &L = run->L;
    unsigned char *ws = run->ws;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *flag = reinterpret_cast<int *>(ws + L.flag);
    GRN_CUDA_TRY(cudaMemsetAsync(flag + 2, 0, sizeof(int), st));
    const int64_t n = run->n_traj;
    GrnParams p{};
    p.n_in = g->n_in;
    p.n_hid = g->n_hid;
    p.n_out = g->n_out;
    p.n_dyn = g->n_dyn;
    p.M = g->M;
    p.Mp = g->Mp;
    p.nb = (g->M + 4) >> 2;
    p.k_max = g->k_max;
    p.n_traj = n;
    p.tpi = run->traj_per_img;
    p.traj_offset = run->traj_offset;
    p.seed = run->seed;
    p.E1 = reinterpret_cast<const float *>(ws + L.E1);
    p.W2fix = reinterpret_cast<const int *>(ws + L.W2fix);
    p.W2f = reinterpret_cast<const float *>(ws + L.W2f);
    p.b2 = run->b2;
    p.dvec = reinterpret_cast<const float *>(ws + L.dvec);
    p.grid = reinterpret_cast<const int *>(ws + L.grid) + 3;
    p.S = run->S;
    p.K = run->opts.ckpt_interval > 0 ? run->opts.ckpt_interval : 64;
    p.draws = reinterpret_cast<int *>(ws + L.draws);
    p.status = reinterpret_cast<int *>(ws + L.status);
    p.ev = reinterpret_cast<uint4 *>(ws + L.ev);
    p.ckpt = reinterpret_cast<int *>(ws + L.ckpt);
    p.brk_k = reinterpret_cast<int *>(ws + L.brk_k);
    p.xfinal = reinterpret_cast<int *>(ws + L.xfinal);
    p.dl_dobs = dl_dobs;
    p.dl_stride = dl_traj_stride;
    p.invT = 1.0f / temperature;
    p.G1 = reinterpret_cast<float *>(ws + L.G1);
    p.dW2t = reinterpret_cast<float *>(ws + L.dW2t);
    p.partial = reinterpret_cast<float *>(ws + L.partial);
    p.mismatch = flag + 2;
    p.err = flag + 1;
    p.n_ckpt = L.n_ckpt;
    p.seg = soft ? reinterpret_cast<float *>(ws + L.soft_seg) : nullptr;
    const int64_t nblk = (n + kGrnWarps - 1) / kGrnWarps;
    float *red = reinterpret_cast<float *>(ws + L.red);
    if (n > 0 && soft) {
        const size_t smem = grn_soft_adj_smem(g);
        GRN_CUDA_TRY(cudaFuncSetAttribute(grn_soft_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        grn_soft_adj_kernel<<<(unsigned)nblk, 32 * kGrnWarps, smem, st>>>(p);
        GRN_CUDA_TRY(cudaGetLastError());
    } else if (n > 0) {
        const size_t smem = grn_adj_smem(g);
        GRN_CUDA_TRY(cudaFuncSetAttribute(grn_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        grn_adj_kernel<<<(unsigned)nblk, 32 * kGrnWarps, smem, st>>>(p);
        GRN_CUDA_TRY(cudaGetLastError());
    }
    GRN_CUDA_TRY(launch_reduce_partials(p.partial, nblk, L.red_len, nullptr, 0, red, nullptr, st));
    grn_split_partials_kernel<<<(L.red_len + 255) / 256, 256, 0, st>>>(red, g->n_out, g->n_dyn, db2, dlog_d);
    GRN_CUDA_TRY(launch_column_sums(p.dW2t, n, (int64_t)g->n_out * g->n_hid, reinterpret_cast<float *>(ws + L.dW2p),
                                    L.dW2_chunk, dW2, st));
    uint16_t *Gt = reinterpret_cast<uint16_t *>(ws + L.Gt);
    uint16_t *xT = reinterpret_cast<uint16_t *>(ws + L.xT);
    const size_t gt_len = (size_t)g->n_hid * L.n_img_pad;
    grn_image_grad_kernel<<<256, 256, 0, st>>>(p.G1, run->n_img, run->traj_per_img, g->n_hid, L.n_img_pad,
                                               reinterpret_cast<float *>(ws + L.Gimg), Gt, Gt + gt_len);
    grn_db1_kernel<<<(g->n_hid + 127) / 128, 128, 0, st>>>(reinterpret_cast<const float *>(ws + L.Gimg), run->n_img,
                                                           g->n_hid, db1);
    grn_transpose_x_kernel<<<256, 256, 0, st>>>(run->x_img, run->n_img, g->n_in, L.n_img_pad, xT);
    GRN_CUDA_TRY(cudaGetLastError());
    if (run->n_img == 0) {  // no images: dL/dW1 is an empty sum (and a zero-length K has no tensor map)
        GRN_CUDA_TRY(cudaMemsetAsync(dW1, 0, (size_t)g->n_hid * g->n_in * sizeof(float), st));
        return SSA_OK;
    }
    // dW1[h][p] = sum_img G[img][h] x[img][p] on the tensor cores (hi + lo bf16 limbs of G)
    TcMaps maps;
    memset(&maps, 0, sizeof(maps));
    const int nt = grn_dw1_nt(g);
    if (!tc_make_map(&maps.a[0], Gt, g->n_hid, (int)run->n_img, L.n_img_pad, 128) ||
        !tc_make_map(&maps.a[1], Gt + gt_len, g->n_hid, (int)run->n_img, L.n_img_pad, 128) ||
        !tc_make_map(&maps.b[0], xT, g->n_in, (int)run->n_img, L.n_img_pad, nt))
        return set_error(SSA_ERR_CUDA, "tensor map encoding failed");
    TcArgs args{g->n_hid, g->n_in, (int)run->n_img, 2, 1, 2, 0, nullptr, dW1, g->n_in, flag + 4};
    args.Dpart = reinterpret_cast<double *>(ws + L.tcpart);
    GRN_CUDA_TRY(tc_gemm_launch(maps, args, nt, st));
    return SSA_OK;
}

extern "C" ssa_status ssa_grn_activations(const ssa_run *run, float *E1_out, int32_t *host_flags, void *stream)
{
    if (!run || !run->grn || !E1_out) return set_error(SSA_ERR_INVALID_ARG, "not a GRN run");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GRN_CUDA_TRY(cudaMemcpyAsync(E1_out, run->ws + run->L.E1, (size_t)run->n_img * run->grn->n_hid * 4,
                                 cudaMemcpyDeviceToDevice, st));
    if (host_flags) {
        int f[4];
        GRN_CUDA_TRY(cudaMemcpyAsync(f, run->ws + run->L.grid, sizeof(f), cudaMemcpyDeviceToHost, st));
        int e[8];
        GRN_CUDA_TRY(cudaMemcpyAsync(e, run->ws + run->L.flag, sizeof(e), cudaMemcpyDeviceToHost, st));
        GRN_CUDA_TRY(cudaStreamSynchronize(st));
        host_flags[0] = f[2];  // inexact limbs / fixed point / counts
        host_flags[1] = e[4];  // tensor-core wait timeout
    }
    return SSA_OK;
}
