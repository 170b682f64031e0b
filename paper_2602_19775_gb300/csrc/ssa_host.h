// ssa_host.h -- host-side definitions shared by the C-ABI translation units (private).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "ssa_internal.cuh"

struct ssa_network {
    int32_t N, M, Mp, P, nnz, nnz_pad;  // Mp = 4 * ceil((M + 1)/4): padded reaction count
    // d_blob = [rx: int4 Mp][stoich: int nnz_pad][inc_ptr: int N+1, padded][inc_list: int 2M, padded]
    //          [rate_index: int Mp][the four table parts again, rx lane-major]; a table region is what
    //          the kernels stage into shared memory
    void *d_blob;
    uint32_t inc_off, inc_list_off;
    int4 *d_rx;
    int4 *d_rx_warp;  // the same tables with rx in lane-major order (jpos), for the warp kernels
    // species -> the stoichiometric changes it receives, for the relaxed update of the warp soft forward:
    // [upd_ptr: int N+1, padded to 4][upd_list: (jpos(j) << 8) | (delta & 0xff), reactions in increasing j]
    int *d_upd;
    uint32_t upd_words;
    int *d_stoich;
    int *d_rate_index;
    uint32_t tab_bytes;
    // host copies of the reaction table and stoichiometry (canonical slot order), from which the
    // network-specialised kernels are generated
    std::vector<int4> h_rx;
    std::vector<int> h_st;
};

struct ssa_grn {
    int32_t n_in, n_hid, n_out, n_dyn, M, Mp;
    float k_max;
};

namespace ssa {
struct WsLayout {
    size_t flag, counts, k_rates, ts, obs_sp, draws, status;
    size_t xfinal, ev, ckpt, brk_k, brk_a, brk_s, brk_tail, bin_prefix, partial, dA;
    size_t partial64, dA64;  // wide-range adjoint: binary64 block sums [ceil(n/128)][M] and [M]
    size_t tcpart;           // GRN: binary64 split-K partial sums of the tensor-core contractions
    size_t total;
    int64_t ev_rows, n_ckpt, max_blocks;
    int M_pad;
    // gene-regulatory-network runs
    size_t E1, W1L, xb, W2fix, W2f, dvec, grid, G1, Gimg, Gt, xT, red, dW2t, dW2p;
    size_t soft_seg;  // soft adjoint: per step of the segment being walked, state, aO, weights, 1/Z
    int n_in_pad, n_img_pad, limbs, red_len;
    int64_t dW2_chunk;
};
ssa_status set_error(ssa_status code, const char *text);
}  // namespace ssa

struct ssa_run {
    const ssa_network *net;
    int variant;  // 1: thread per trajectory, 2: thread per trajectory, network-specialised, 32: warp
    const ssa_grn *grn;  // non-null for a gene-regulatory-network run
    int64_t n_img, traj_per_img;
    const int32_t *x_img;  // caller's inputs, kept alive by the caller until the backward
    const float *b2;
    int64_t n_traj;
    uint64_t traj_offset, seed;
    int32_t S, n_obs;
    ssa_fwd_opts opts;
    double t_end;
    unsigned char *ws;
    ssa::WsLayout L;
};
