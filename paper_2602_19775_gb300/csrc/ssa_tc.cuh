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
};

bool tc_make_map(CUtensorMap *map, const void *base, int rows, int K, int ld, int box_rows);
cudaError_t tc_gemm_launch(const TcMaps &maps, const TcArgs &args, int nt, cudaStream_t st);

}  // namespace ssa
