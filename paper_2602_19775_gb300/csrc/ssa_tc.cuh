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
};

bool tc_make_map(CUtensorMap *map, const void *base, int rows, int K, int ld, int box_rows);
cudaError_t tc_gemm_launch(const TcMaps &maps, const TcArgs &args, int nt, cudaStream_t st);
// K splits tc_gemm_launch uses for an M x N x K product with N-tiles of nt (1: no split), and the binary64
// words of its Dpart buffer
int tc_split_count(int M, int N, int K, int nt);
size_t tc_split_words(int M, int N, int K, int nt);

}  // namespace ssa
