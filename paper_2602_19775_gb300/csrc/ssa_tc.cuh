// ssa_tc.cuh -- interface of the tcgen05 GEMM (ssa_tc_gemm.cu) to the other translation units.
#pragma once

#include <cuda.h>

#include "ssa_internal.cuh"

namespace ssa {

constexpr int kTcMaxA = 2;
constexpr int kTcMaxB = 8;

// TMA descriptors of the A_t and B_t operands (bf16, K-major rows)
struct TcMaps {
    CUtensorMap a[kTcMaxA];
    CUtensorMap b[kTcMaxB];
};

struct TcArgs {
    int M, N, K;
    int n_a, n_b, n_terms;  // term t multiplies A[min(t, n_a - 1)] by B[min(t, n_b - 1)]
    int separate;           // 1: one TMEM accumulator per term, summed in binary64
    const float *bias;      // [N] or nullptr
    float *D;               // [M][ldd]
    int ldd;
    int *err;
    // split K (filled by tc_gemm_launch when Dpart is given): the CTAs of blockIdx.z = s take K chunks
    // [s per, (s + 1) per) and write their binary64 sums to Dpart [k_split][M][N]; a second kernel adds the
    // splits in order and the bias
    double *Dpart;          // nullptr: one pass over K per tile
    int k_split, chunks_per;
    // exact limb sum (separate accumulators, n_terms = 8): term t is T_t 2^(g + limb_bits t) with T_t an
    // integer below 2^24 in magnitude and g = *limb_grid. The epilogue converts each term to T_t and adds
    // lo = sum_{t<4} T_t 2^(limb_bits t) and hi = sum_{t>=4} T_t 2^(limb_bits (t-4)) in int64 (exact), and
    // D = (hi 2^(4 limb_bits) + lo) 2^g + bias, rounded once to binary64 and then to binary32. With a split,
    // Dpart holds the (lo, hi) pairs of each split as int64 [k_split][M][N][2], added exactly.
    const int *limb_grid;   // nullptr: binary64 sum of the accumulators
    int limb_bits;
};

bool tc_make_map(CUtensorMap *map, const void *base, int rows, int K, int ld, int box_rows);
cudaError_t tc_gemm_launch(const TcMaps &maps, const TcArgs &args, int nt, cudaStream_t st);
// K splits tc_gemm_launch uses for an M x N x K product with N-tiles of nt (1: no split), and the binary64
// words of its Dpart buffer
int tc_split_count(int M, int N, int K, int nt);
size_t tc_split_words(int M, int N, int K, int nt);  // the exact limb sum takes twice as many

}  // namespace ssa
