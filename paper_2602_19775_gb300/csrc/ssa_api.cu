// ssa_api.cu -- host side of the C ABI declared in include/ssa.h.
//
// Validates arguments, lays out the caller's workspace, stages per-call inputs (rate constants,
// sample grid, observed species) into it, picks the kernel variant and launch shape, and keeps
// the small run handle that lets ssa_backward revisit a recorded forward.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ssa_host.h"

namespace ssa {
cudaError_t launch_forward_thread(const FwdParams &p, int readout, bool record, bool replay, int block, size_t smem,
                                  cudaStream_t st);
cudaError_t launch_validate_inputs(const double *ts, int S, double t_end, const int *obs_sp, int n_obs, int N,
                                  int strict, int *flag, cudaStream_t st);
cudaError_t launch_rates(const float *log_rates, const int *rate_index, int M, int M_pad, int lane_major, float *k_out,
                         cudaStream_t st);
cudaError_t launch_ensemble_mean(const void *obs, bool is_int, int64_t n_traj, int64_t row_len, float *partial,
                                 int64_t chunk, float *out, cudaStream_t st);
cudaError_t launch_philox_uniforms(uint64_t seed, const uint64_t *traj, const uint64_t *step, int64_t n,
                                   int n_words, float *out, cudaStream_t st);
cudaError_t launch_unpack_events(const uint4 *ev, const int *draws, int64_t n_traj, int64_t stride, int *out,
                                 cudaStream_t st);
cudaError_t launch_status_count(const int *status, int64_t n, unsigned long long *counts, cudaStream_t st);
cudaError_t launch_bin_prefix(const float *g, int S, int n_obs, double *prefix, cudaStream_t st);
cudaError_t launch_transpose_brackets(const int *brk, int64_t n_traj, int S, const int *first, const int *nslots,
                                      int *out, cudaStream_t st);
cudaError_t launch_backward_thread(const AdjParams &p, int readout, int block, size_t smem, int64_t grid,
                                   cudaStream_t st);
cudaError_t launch_reduce_partials(const float *partial, int64_t nblk, int M, const int *rate_index, int P,
                                   float *dA_tmp, float *dtheta, cudaStream_t st);
cudaError_t launch_forward_warp(const FwdParams &p, int readout, bool record, int warps, size_t smem, cudaStream_t st);
cudaError_t launch_forward_warp_soft(const FwdParams &p, int readout, bool record, int warps, size_t smem,
                                     cudaStream_t st);
cudaError_t launch_backward_warp_soft(const AdjParams &p, const int *upd, uint32_t upd_words, int readout, int warps,
                                      size_t smem, int64_t grid, cudaStream_t st);
cudaError_t launch_backward_warp(const AdjParams &p, int readout, int warps, size_t smem, int64_t grid,
                                 cudaStream_t st);
int thread_kernel_mc(int M);
cudaError_t launch_exp_variates(const uint32_t *words, int64_t n, float *out, cudaStream_t st);
struct JitKernels;
bool jit_eligible(const ssa_network *net);
const JitKernels *jit_kernels(const ssa_network *net, std::string &why);
const JitKernels *jit_soft_kernels(const ssa_network *net, std::string &why);
cudaError_t jit_launch_forward(const JitKernels *k, const FwdParams &p, int readout, bool record, int selector,
                               int block, cudaStream_t st);
cudaError_t jit_launch_backward(const JitKernels *k, const AdjParams &p, int readout, int block, int64_t grid,
                                cudaStream_t st);
cudaError_t jit_launch_backward_wide(const JitKernels *k, const AdjParams &p, int readout, int block, int64_t grid,
                                     cudaStream_t st);
cudaError_t jit_launch_backward_multi(const JitKernels *k, const AdjParams &p, int readout, int n_temps, int block,
                                      int64_t grid, cudaStream_t st);
constexpr int kMaxFusedTemps = 3;  // temperatures one specialised walk takes at once
cudaError_t launch_reduce_partials64(const double *partial, int64_t nblk, int M, const int *rate_index, int P,
                                     double *dA_tmp, double *dtheta, cudaStream_t st);
constexpr int kJitBlock = 64;
constexpr int kJitAdjBlock = 128;  // the specialised adjoint orders a block's trajectories by length over its 4 warps
}  // namespace ssa

using namespace ssa;

// ---------------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static ssa_status fail(ssa_status code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(expr)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess) return fail(SSA_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));       \
    } while (0)

extern "C" const char *ssa_last_error(void) { return g_err; }

namespace ssa {
// record an error text for ssa_last_error from another translation unit
ssa_status set_error(ssa_status code, const char *text) { return fail(code, "%s", text); }
}  // namespace ssa

// ---------------------------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------------------------


namespace {
constexpr size_t kAlign = 256;
constexpr int kWarpsPerBlock = 4;  // warp-per-trajectory kernels
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }



int effective_K(const ssa_fwd_opts *o)
{
    if (o->selector == SSA_SELECT_SOFT) return kSoftK;  // float checkpoints; the adjoint re-runs each segment
    return o->ckpt_interval > 0 ? o->ckpt_interval : 64;
}

WsLayout layout(const ssa_network *net, int64_t n, int32_t S, const ssa_fwd_opts *o)
{
    WsLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, kAlign);
        return at;
    };
    L.M_pad = net->Mp;
    L.flag = take(16 * sizeof(int));
    L.counts = take(SSA_TRAJ_N_CODES * sizeof(unsigned long long));
    L.k_rates = take((size_t)L.M_pad * sizeof(float));
    L.ts = take((size_t)(S > 0 ? S : 1) * sizeof(double));
    L.obs_sp = take((size_t)64 * sizeof(int));  // n_obs <= 64
    L.draws = take((size_t)(n > 0 ? n : 1) * sizeof(int));
    L.status = take((size_t)(n > 0 ? n : 1) * sizeof(int));
    if (o->record) {
        const int K = effective_K(o);
        L.ev_rows = (o->max_steps + 7) / 8;
        L.n_ckpt = o->max_steps / K + 1;
        L.max_blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;  // the warp kernels launch the most blocks
        L.xfinal = take((size_t)net->N * n * sizeof(int));
        L.ev = take((size_t)L.ev_rows * n * sizeof(uint4));
        L.ckpt = take((size_t)L.n_ckpt * net->N * n * sizeof(int));
        L.brk_k = take((size_t)S * n * sizeof(int));
        L.brk_a = take((size_t)S * n * sizeof(float));
        L.brk_s = take((size_t)S * n * sizeof(int));
        L.brk_tail = take((size_t)(n > 0 ? n : 1) * sizeof(int));
        L.bin_prefix = take((size_t)(S + 1) * SSA_BIN_MAX_OBS * sizeof(double));
        // block sums of one backward: the warp kernels launch the most blocks; a specialised walk over
        // several temperatures writes one set of block sums per temperature
        const int64_t fused_blocks = kMaxFusedTemps * ((n + kJitAdjBlock - 1) / kJitAdjBlock);
        const int64_t part_rows = std::max<int64_t>(std::max<int64_t>(L.max_blocks, fused_blocks), 1);
        L.partial = take((size_t)part_rows * net->M * sizeof(float));
        L.dA = take((size_t)net->M * sizeof(float));
        const int64_t wide_blocks = (n + kJitAdjBlock - 1) / kJitAdjBlock;
        L.partial64 = take((size_t)(wide_blocks > 0 ? wide_blocks : 1) * net->M * sizeof(double));
        L.dA64 = take((size_t)net->M * sizeof(double));
    }
    L.total = off;
    return L;
}

bool opts_valid(const ssa_fwd_opts *o)
{
    if (!o) return false;
    if (o->readout != SSA_READOUT_HOLD && o->readout != SSA_READOUT_LINEAR && o->readout != SSA_READOUT_BIN) return false;
    if (o->max_steps < 1 || o->max_steps > 0x7fffffffLL) return false;
    if (o->ckpt_interval < 0 || (o->ckpt_interval % 8) != 0) return false;
    if (o->threads_per_traj != 0 && o->threads_per_traj != 1 && o->threads_per_traj != 32) return false;
    if (o->block_threads != 0 && (o->block_threads % 32 != 0 || o->block_threads < 32 || o->block_threads > 256))
        return false;
    if (o->no_specialize != 0 && o->no_specialize != 1) return false;
    if (o->selector != SSA_SELECT_GUMBEL && o->selector != SSA_SELECT_DIRECT && o->selector != SSA_SELECT_SOFT)
        return false;
    if (o->selector == SSA_SELECT_DIRECT && o->record) return false;  // the gradient is of the Gumbel-max choice
    if (o->selector == SSA_SELECT_SOFT) {
        if (!(o->temperature > 0.0f) || !(o->temperature < 3.0e38f)) return false;
    } else if (o->temperature != 0.0f) {
        return false;
    }
    return true;
}

size_t smem_limit()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 48 * 1024;
    return (size_t)v;
}

size_t fwd_smem(const ssa_network *net, int block) { return net->tab_bytes + (size_t)net->Mp * 4 + 16 + (size_t)net->N * block * 4; }
size_t adj_smem(const ssa_network *net, int block)
{
    return net->tab_bytes + (size_t)net->Mp * 4 + 16 + (size_t)(3 * net->N + 2 * net->M) * block * 4;
}

size_t fwd_warp_smem(const ssa_network *net)
{
    return net->tab_bytes + (size_t)net->Mp * 4 + 16 + (size_t)kWarpsPerBlock * ((net->N + 3) & ~3) * 4;
}
// the soft forward on the warp layout: tables, rates, the update list, and per warp X, dX [Npad] and y [Mp]
size_t fwd_warp_soft_smem(const ssa_network *net)
{
    return net->tab_bytes + (size_t)net->Mp * 4 + 16 + (size_t)net->upd_words * 4 +
           (size_t)kWarpsPerBlock * (2 * ((net->N + 3) & ~3) + (size_t)net->Mp) * 4;
}

// its gradient: tables, rates, the update list, and per warp Xs [kSoftK][Npad], lam, dX [Npad], a, h, y, c1, c2, dA [Mp]
size_t adj_warp_soft_smem(const ssa_network *net)
{
    return net->tab_bytes + (size_t)net->Mp * 4 + 16 + (size_t)net->upd_words * 4 +
           (size_t)kWarpsPerBlock * ((kSoftK + 2) * (size_t)((net->N + 3) & ~3) + 6 * (size_t)net->Mp) * 4;
}

size_t adj_warp_smem(const ssa_network *net)
{
    return net->tab_bytes + (size_t)net->Mp * 4 + 16 +
           (size_t)kWarpsPerBlock * (2 * ((net->N + 3) & ~3) + 4 * (size_t)net->Mp) * 4;
}

// one thread per trajectory up to 16 reactions (unrolled, register-resident), one warp above
int pick_variant(const ssa_network *net, const ssa_fwd_opts *o)
{
    if (o->threads_per_traj) return o->threads_per_traj;
    if (!o->no_specialize && jit_eligible(net)) return 1;
    return net->M <= 16 ? 1 : 32;
}

int pick_block(size_t (*need)(const ssa_network *, int), const ssa_network *net, int requested, size_t limit)
{
    if (requested) return need(net, requested) <= limit ? requested : 0;
    // small blocks spread an uneven trajectory count evenly over the 152 SMs
    for (int b : {64, 32})
        if (need(net, b) <= limit) return b;
    return 0;
}
}  // namespace



extern "C" ssa_status ssa_create_network(int32_t n_species, int32_t n_reactions, const int32_t *reactants,
                                         const int32_t *stoich_ptr, const int32_t *stoich_species,
                                         const int32_t *stoich_delta, int32_t n_params, const int32_t *rate_index,
                                         ssa_network **out)
{
    if (!out) return fail(SSA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_species < 1 || n_species > (1 << 22)) return fail(SSA_ERR_INVALID_ARG, "n_species %d out of range", n_species);
    if (n_reactions < 1) return fail(SSA_ERR_INVALID_ARG, "n_reactions %d < 1", n_reactions);
    if (n_reactions > 65535) return fail(SSA_ERR_UNSUPPORTED, "n_reactions %d > 65535 (uint16 event log)", n_reactions);
    if (n_params < 1) return fail(SSA_ERR_INVALID_ARG, "n_params %d < 1", n_params);
    if (!reactants || !stoich_ptr || !rate_index) return fail(SSA_ERR_INVALID_ARG, "NULL table");
    if (stoich_ptr[0] != 0) return fail(SSA_ERR_INVALID_ARG, "stoich_ptr[0] != 0");
    for (int j = 0; j < n_reactions; ++j)
        if (stoich_ptr[j + 1] < stoich_ptr[j]) return fail(SSA_ERR_INVALID_ARG, "stoich_ptr not monotone at %d", j);
    const int nnz = stoich_ptr[n_reactions];
    if (nnz > 0 && (!stoich_species || !stoich_delta)) return fail(SSA_ERR_INVALID_ARG, "NULL stoichiometry");
    // at least M + 1 rounded up to 4, and at least the unrolled reaction count of the
    // thread-per-trajectory kernels (2, 4, 8 or 16 for M <= 16), which read every padded entry
    int Mp = (n_reactions + 4) / 4 * 4;
    if (n_reactions <= 16) Mp = std::max(Mp, thread_kernel_mc(n_reactions));
    std::vector<int4> rx(Mp, make_int4(-1, -1, 0, 0));  // padding: order 0, no change, rate 0
    for (int j = 0; j < n_reactions; ++j) {
        int r1 = reactants[2 * j], r2 = reactants[2 * j + 1];
        if (r1 < -1 || r1 >= n_species || r2 < -1 || r2 >= n_species)
            return fail(SSA_ERR_INVALID_ARG, "reactant of reaction %d out of range", j);
        if (r1 < 0) { r1 = r2; r2 = -1; }
        if (rate_index[j] < 0 || rate_index[j] >= n_params)
            return fail(SSA_ERR_INVALID_ARG, "rate_index[%d] = %d out of range", j, rate_index[j]);
        rx[j] = make_int4(r1, r2, stoich_ptr[j], stoich_ptr[j + 1]);
    }
    for (int j = 0; j < n_reactions; ++j)  // one entry per species in a reaction's net change
        for (int e = stoich_ptr[j]; e < stoich_ptr[j + 1]; ++e)
            for (int f = stoich_ptr[j]; f < e; ++f)
                if (stoich_species[e] == stoich_species[f])
                    return fail(SSA_ERR_INVALID_ARG, "reaction %d lists species %d twice in its net change", j,
                                stoich_species[e]);
    const int nnz_pad = (nnz + 3) / 4 * 4;
    std::vector<int> st(nnz_pad > 0 ? nnz_pad : 4, 0);
    for (int e = 0; e < nnz; ++e) {
        if (stoich_species[e] < 0 || stoich_species[e] >= n_species)
            return fail(SSA_ERR_INVALID_ARG, "stoich_species[%d] out of range", e);
        if (stoich_delta[e] < -127 || stoich_delta[e] > 127)
            return fail(SSA_ERR_INVALID_ARG, "stoich_delta[%d] = %d outside [-127, 127]", e, stoich_delta[e]);
        st[e] = (stoich_species[e] << 8) | (stoich_delta[e] & 0xff);
    }
    std::vector<int> ri(Mp, 0);
    for (int j = 0; j < n_reactions; ++j) ri[j] = rate_index[j];
    // species -> reactant slots (2j + slot) in increasing order; a homodimer lists slot 0 only
    std::vector<int> inc_ptr(n_species + 1, 0), inc_list;
    for (int sp = 0; sp < n_species; ++sp) {
        for (int j = 0; j < n_reactions; ++j) {
            if (rx[j].x == sp) inc_list.push_back(2 * j);
            if (rx[j].y == sp && rx[j].y != rx[j].x) inc_list.push_back(2 * j + 1);
        }
        inc_ptr[sp + 1] = (int)inc_list.size();
    }
    // species -> (lane-major position of j, delta) over the reactions that change it, in increasing j
    const int nb_warp = (n_reactions + 4) >> 2;
    std::vector<std::vector<int>> upd_by_species(n_species);
    for (int j = 0; j < n_reactions; ++j)
        for (int e = stoich_ptr[j]; e < stoich_ptr[j + 1]; ++e)
            upd_by_species[stoich_species[e]].push_back((((j + 1) & 3) * nb_warp + ((j + 1) >> 2)) << 8 |
                                                        (stoich_delta[e] & 0xff));
    const int upd_ptr_pad = (n_species + 1 + 3) / 4 * 4;
    std::vector<int> upd(upd_ptr_pad, 0);
    for (int sp = 0; sp < n_species; ++sp) {
        upd.insert(upd.end(), upd_by_species[sp].begin(), upd_by_species[sp].end());
        upd[sp + 1] = (int)upd.size() - upd_ptr_pad;
    }
    for (int sp = n_species + 1; sp < upd_ptr_pad; ++sp) upd[sp] = upd[n_species];
    upd.resize((upd.size() + 3) / 4 * 4, 0);
    const int inc_ptr_pad = (n_species + 1 + 3) / 4 * 4;
    const int inc_list_pad = ((int)inc_list.size() + 3) / 4 * 4;
    inc_ptr.resize(inc_ptr_pad, inc_ptr[n_species]);
    inc_list.resize(inc_list_pad > 0 ? inc_list_pad : 4, 0);

    ssa_network *net = new (std::nothrow) ssa_network();
    if (!net) return fail(SSA_ERR_CUDA, "host allocation failed");
    net->N = n_species;
    net->M = n_reactions;
    net->P = n_params;
    net->Mp = Mp;
    net->nnz = nnz;
    net->nnz_pad = nnz_pad;
    net->inc_off = (uint32_t)(16 * Mp + 4 * nnz_pad);
    net->inc_list_off = net->inc_off + (uint32_t)(4 * inc_ptr_pad);
    net->tab_bytes = net->inc_list_off + (uint32_t)(4 * inc_list_pad);
    // blob = [tables][rate_index: int Mp][tables again, with rx in the warp kernels' lane-major order]
    //        [species-major update list of the warp soft forward]
    net->upd_words = (uint32_t)upd.size();
    const size_t bytes = 2 * (size_t)net->tab_bytes + (size_t)Mp * 4 + 4 * (size_t)net->upd_words;
    cudaError_t e = cudaMalloc(&net->d_blob, bytes);
    if (e != cudaSuccess) {
        delete net;
        return fail(SSA_ERR_CUDA, "cudaMalloc(network tables): %s", cudaGetErrorString(e));
    }
    unsigned char *b = static_cast<unsigned char *>(net->d_blob);
    net->h_rx.assign(rx.begin(), rx.begin() + n_reactions);
    net->h_st.assign(st.begin(), st.begin() + nnz);
    net->d_rx = reinterpret_cast<int4 *>(b);
    net->d_stoich = reinterpret_cast<int *>(b + 16 * Mp);
    net->d_rate_index = reinterpret_cast<int *>(b + net->tab_bytes);
    e = cudaMemcpy(net->d_rx, rx.data(), 16 * (size_t)Mp, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(net->d_stoich, st.data(), 4 * (size_t)nnz_pad, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(net->d_rate_index, ri.data(), 4 * (size_t)Mp, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && inc_ptr_pad > 0)
        e = cudaMemcpy(b + net->inc_off, inc_ptr.data(), 4 * (size_t)inc_ptr_pad, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && inc_list_pad > 0)
        e = cudaMemcpy(b + net->inc_list_off, inc_list.data(), 4 * (size_t)inc_list_pad, cudaMemcpyHostToDevice);
    net->d_rx_warp = reinterpret_cast<int4 *>(b + net->tab_bytes + (size_t)Mp * 4);
    if (e == cudaSuccess) e = cudaMemcpy(net->d_rx_warp, net->d_rx, net->tab_bytes, cudaMemcpyDeviceToDevice);
    net->d_upd = reinterpret_cast<int *>(b + 2 * (size_t)net->tab_bytes + (size_t)Mp * 4);
    if (e == cudaSuccess) e = cudaMemcpy(net->d_upd, upd.data(), 4 * (size_t)net->upd_words, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int nb = (n_reactions + 4) >> 2;
        std::vector<int4> rxp(Mp, make_int4(-1, -1, 0, 0));
        for (int j = 0; j < n_reactions; ++j) rxp[((j + 1) & 3) * nb + ((j + 1) >> 2)] = rx[j];
        e = cudaMemcpy(net->d_rx_warp, rxp.data(), 16 * (size_t)Mp, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(net->d_blob);
        delete net;
        return fail(SSA_ERR_CUDA, "cudaMemcpy(network tables): %s", cudaGetErrorString(e));
    }
    *out = net;
    return SSA_OK;
}

extern "C" void ssa_destroy_network(ssa_network *net)
{
    if (!net) return;
    cudaFree(net->d_blob);
    delete net;
}

extern "C" size_t ssa_forward_workspace_bytes(const ssa_network *net, int64_t n_traj, int32_t n_samples,
                                              const ssa_fwd_opts *opts)
{
    if (!net || n_traj < 0 || n_samples < 0 || !opts_valid(opts)) return 0;
    return layout(net, n_traj, n_samples, opts).total;
}

static ssa_status forward_impl(const ssa_network *net, const float *log_rates, int64_t n_traj, int64_t traj_offset,
                               const int32_t *x0, int32_t x0_per_traj, double t_end, const double *sample_times,
                               int32_t S, const int32_t *obs_species, int32_t n_obs, uint64_t seed,
                               const ssa_fwd_opts *opts, const uint16_t *ev_in, const int32_t *n_ev_in,
                               int64_t ev_stride, void *workspace, size_t ws_bytes, void *obs_out,
                               int32_t *draws_out, int32_t *status_out, void *stream, ssa_run **run_out)
{
    if (run_out) *run_out = nullptr;
    if (!net) return fail(SSA_ERR_INVALID_ARG, "network is NULL");
    if (!opts_valid(opts)) return fail(SSA_ERR_INVALID_ARG, "invalid ssa_fwd_opts");
    if (n_traj < 0 || n_traj > (1LL << 40)) return fail(SSA_ERR_INVALID_ARG, "n_traj %lld out of range", (long long)n_traj);
    if (traj_offset < 0) return fail(SSA_ERR_INVALID_ARG, "traj_offset < 0");
    if (S < 0 || n_obs < 0 || n_obs > 64) return fail(SSA_ERR_INVALID_ARG, "n_samples/n_obs out of range (n_obs <= 64)");
    if (!(t_end >= 0.0) || !(t_end < 1e300)) return fail(SSA_ERR_INVALID_ARG, "t_end must be finite and >= 0");
    if (!log_rates || (!x0 && n_traj > 0) || (S > 0 && !sample_times) || (n_obs > 0 && !obs_species))
        return fail(SSA_ERR_INVALID_ARG, "NULL input pointer");
    if (S > 0 && n_obs > 0 && n_traj > 0 && !obs_out) return fail(SSA_ERR_INVALID_ARG, "obs_out is NULL");
    if (ev_in && (ev_stride < 1 || !n_ev_in)) return fail(SSA_ERR_INVALID_ARG, "bad replay arguments");
    if (opts->record && opts->max_steps > 0x7fffffffLL) return fail(SSA_ERR_INVALID_ARG, "max_steps too large");
    const WsLayout L = layout(net, n_traj, S, opts);
    if (!workspace || ws_bytes < L.total) return fail(SSA_ERR_WORKSPACE, "workspace %zu bytes < required %zu", ws_bytes, L.total);
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return fail(SSA_ERR_WORKSPACE, "workspace not 256-byte aligned");
    const size_t limit = smem_limit();
    int variant = ev_in ? 1 : pick_variant(net, opts);  // replay is a thread-per-trajectory test hook
    // the thread variant runs as network-specialised kernels when the network qualifies (variant 2)
    const JitKernels *jit = nullptr;
    if (opts->selector == SSA_SELECT_SOFT) {
        // the network-specialised thread kernels (forward and gradient) where the network qualifies, else the
        // warp kernels (forward only)
        if (ev_in) return fail(SSA_ERR_UNSUPPORTED, "the soft forward has no replay mode");
        std::string why = "the network is not eligible (N, M <= 24, at most 96 stoichiometric entries)";
        if (variant == 1 && !opts->no_specialize && jit_eligible(net)) {
            jit = jit_soft_kernels(net, why);
            if (jit) variant = 2;
        }
        if (variant == 1 && opts->threads_per_traj == 1)
            return fail(SSA_ERR_UNSUPPORTED, "the soft forward with one thread per trajectory needs the "
                        "network-specialised kernels: %s", why.c_str());
        if (variant == 1) variant = 32;
    } else if (variant == 1 && !ev_in && !opts->no_specialize && jit_eligible(net)) {
        std::string why;
        jit = jit_kernels(net, why);
        if (jit) variant = 2;
    }
    if (opts->readout == SSA_READOUT_BIN && n_obs > SSA_BIN_MAX_OBS)
        return fail(SSA_ERR_UNSUPPORTED, "the bin readout takes at most %d observables per call", SSA_BIN_MAX_OBS);
    if (opts->selector == SSA_SELECT_DIRECT && (variant != 2 || ev_in))
        return fail(SSA_ERR_UNSUPPORTED, "the direct method runs on the network-specialised kernels (N and M <= 24)");
    int block = 0;
    if (variant == 2) {
        block = kJitBlock;
    } else if (variant == 1) {
        block = pick_block(fwd_smem, net, opts->block_threads, limit);
        if (!block) return fail(SSA_ERR_UNSUPPORTED, "network too large for the thread-per-trajectory forward");
        if (opts->record && !pick_block(adj_smem, net, 0, limit))
            return fail(SSA_ERR_UNSUPPORTED, "network too large for the thread-per-trajectory adjoint");
    } else if (opts->selector == SSA_SELECT_SOFT) {
        if (fwd_warp_soft_smem(net) > limit || (opts->record && adj_warp_soft_smem(net) > limit))
            return fail(SSA_ERR_UNSUPPORTED, "network too large for the warp-per-trajectory soft forward");
    } else {
        if (fwd_warp_smem(net) > limit || (opts->record && adj_warp_smem(net) > limit))
            return fail(SSA_ERR_UNSUPPORTED, "network too large for the warp-per-trajectory kernels");
    }

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    int *flag = reinterpret_cast<int *>(ws + L.flag);
    CUDA_TRY(cudaMemsetAsync(flag, 0, 16 * sizeof(int), st));
    if (S > 0) CUDA_TRY(cudaMemcpyAsync(ws + L.ts, sample_times, (size_t)S * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (n_obs > 0) CUDA_TRY(cudaMemcpyAsync(ws + L.obs_sp, obs_species, (size_t)n_obs * sizeof(int), cudaMemcpyDeviceToDevice, st));
    // the warp kernels read their tables and rates lane-major
    CUDA_TRY(launch_rates(log_rates, net->d_rate_index, net->M, L.M_pad, variant == 32 ? 1 : 0,
                          reinterpret_cast<float *>(ws + L.k_rates), st));
    CUDA_TRY(launch_validate_inputs(reinterpret_cast<const double *>(ws + L.ts), S, t_end,
                                    reinterpret_cast<const int *>(ws + L.obs_sp), n_obs, net->N,
                                    opts->readout == SSA_READOUT_BIN ? 1 : 0, flag, st));
    FwdParams p{};
    p.rx = variant == 32 ? net->d_rx_warp : net->d_rx;
    p.k_rates = reinterpret_cast<const float *>(ws + L.k_rates);
    p.tab_bytes = net->tab_bytes;
    p.k_bytes = (uint32_t)(L.M_pad * 4);
    p.N = net->N;
    p.M = net->M;
    p.Mp = net->Mp;
    p.inc_off = net->inc_off;
    p.inc_list_off = net->inc_list_off;
    p.nnz = net->nnz;
    p.n_traj = n_traj;
    p.traj_offset = (uint64_t)traj_offset;
    p.seed = seed;
    p.x0 = x0;
    p.x0_per_traj = x0_per_traj ? 1 : 0;
    p.t_end = t_end;
    p.ts = reinterpret_cast<const double *>(ws + L.ts);
    p.S = S;
    p.obs_sp = reinterpret_cast<const int *>(ws + L.obs_sp);
    p.n_obs = n_obs;
    p.max_steps = opts->max_steps;
    p.invT = opts->selector == SSA_SELECT_SOFT ? 1.0f / opts->temperature : 0.0f;
    p.upd = net->d_upd;
    p.upd_words = net->upd_words;
    p.obs_out = obs_out;
    p.draws = reinterpret_cast<int *>(ws + L.draws);
    p.status = reinterpret_cast<int *>(ws + L.status);
    p.flag = flag;
    p.err = flag + 1;
    p.K = effective_K(opts);
    if (opts->record) {
        p.ev = reinterpret_cast<uint4 *>(ws + L.ev);
        p.ckpt = reinterpret_cast<int *>(ws + L.ckpt);
        p.brk_k = reinterpret_cast<int *>(ws + L.brk_k);
        p.brk_a = reinterpret_cast<float *>(ws + L.brk_a);
        p.brk_s = reinterpret_cast<int *>(ws + L.brk_s);
        p.brk_tail = reinterpret_cast<int *>(ws + L.brk_tail);
        p.xfinal = reinterpret_cast<int *>(ws + L.xfinal);
    }
    p.ev_in = ev_in;
    p.n_ev_in = n_ev_in;
    p.ev_in_stride = ev_stride;
    if (variant == 2)
        CUDA_TRY(jit_launch_forward(jit, p, opts->readout, opts->record != 0, opts->selector, block, st));
    else if (variant == 1)
        CUDA_TRY(launch_forward_thread(p, opts->readout, opts->record != 0, ev_in != nullptr, block, fwd_smem(net, block), st));
    else if (opts->selector == SSA_SELECT_SOFT)
        CUDA_TRY(launch_forward_warp_soft(p, opts->readout, opts->record != 0, kWarpsPerBlock, fwd_warp_soft_smem(net),
                                          st));
    else
        CUDA_TRY(launch_forward_warp(p, opts->readout, opts->record != 0, kWarpsPerBlock, fwd_warp_smem(net), st));
    if (n_traj > 0 && draws_out) CUDA_TRY(cudaMemcpyAsync(draws_out, p.draws, (size_t)n_traj * 4, cudaMemcpyDeviceToDevice, st));
    if (n_traj > 0 && status_out) CUDA_TRY(cudaMemcpyAsync(status_out, p.status, (size_t)n_traj * 4, cudaMemcpyDeviceToDevice, st));
    if (run_out) {
        ssa_run *run = new (std::nothrow) ssa_run();
        if (!run) return fail(SSA_ERR_CUDA, "host allocation failed");
        run->net = net;
        run->variant = variant;
        run->n_traj = n_traj;
        run->traj_offset = (uint64_t)traj_offset;
        run->seed = seed;
        run->S = S;
        run->n_obs = n_obs;
        run->opts = *opts;
        run->t_end = t_end;
        run->ws = ws;
        run->L = L;
        *run_out = run;
    }
    return SSA_OK;
}

extern "C" ssa_status ssa_forward(const ssa_network *net, const float *log_rates, int64_t n_traj, int64_t traj_offset,
                                  const int32_t *x0, int32_t x0_per_traj, double t_end, const double *sample_times,
                                  int32_t n_samples, const int32_t *obs_species, int32_t n_obs, uint64_t seed,
                                  const ssa_fwd_opts *opts, void *workspace, size_t workspace_bytes, void *obs_out,
                                  int32_t *draws_out, int32_t *status_out, void *stream, ssa_run **run_out)
{
    return forward_impl(net, log_rates, n_traj, traj_offset, x0, x0_per_traj, t_end, sample_times, n_samples,
                        obs_species, n_obs, seed, opts, nullptr, nullptr, 0, workspace, workspace_bytes, obs_out,
                        draws_out, status_out, stream, run_out);
}

extern "C" ssa_status ssa_forward_replay(const ssa_network *net, const float *log_rates, int64_t n_traj,
                                         int64_t traj_offset, const int32_t *x0, int32_t x0_per_traj, double t_end,
                                         const double *sample_times, int32_t n_samples, const int32_t *obs_species,
                                         int32_t n_obs, uint64_t seed, const ssa_fwd_opts *opts,
                                         const uint16_t *events, const int32_t *n_events, int64_t events_stride,
                                         void *workspace, size_t workspace_bytes, void *obs_out, int32_t *draws_out,
                                         int32_t *status_out, void *stream, ssa_run **run_out)
{
    if (!events || !n_events) return fail(SSA_ERR_INVALID_ARG, "replay needs events and n_events");
    return forward_impl(net, log_rates, n_traj, traj_offset, x0, x0_per_traj, t_end, sample_times, n_samples,
                        obs_species, n_obs, seed, opts, events, n_events, events_stride, workspace, workspace_bytes,
                        obs_out, draws_out, status_out, stream, run_out);
}

// Everything ssa_backward and ssa_backward_wide share: argument checks, the kernel variant and launch
// shape, and the adjoint parameters (the per-block sums are left unset).
static ssa_status backward_setup(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride, float temperature,
                                 const void *dl_dlog_rates, cudaStream_t st, AdjParams &p, const JitKernels *&jit,
                                 int &block, int64_t &grid)
{
    if (run && dl_traj_stride != 0 && dl_traj_stride < (int64_t)run->S * run->n_obs)
        return fail(SSA_ERR_INVALID_ARG, "dl_traj_stride must be 0 or >= n_samples * n_obs");
    if (!run) return fail(SSA_ERR_INVALID_ARG, "run is NULL");
    if (!run->net) return fail(SSA_ERR_STATE, "a gene-regulatory-network run is differentiated by ssa_grn_backward");
    if (!run->opts.record) return fail(SSA_ERR_STATE, "the forward was not recorded (opts.record = 0)");
    if (!(temperature > 0.0f) || !(temperature < 3.0e38f)) return fail(SSA_ERR_INVALID_ARG, "temperature must be > 0");
    if (!dl_dlog_rates) return fail(SSA_ERR_INVALID_ARG, "dl_dlog_rates is NULL");
    if (!dl_dobs && run->n_traj > 0 && run->S > 0 && run->n_obs > 0) return fail(SSA_ERR_INVALID_ARG, "dl_dobs is NULL");
    const ssa_network *net = run->net;
    const WsLayout &L = run->L;
    unsigned char *ws = run->ws;
    const size_t limit = smem_limit();
    block = 0;
    grid = 0;
    jit = nullptr;
    const bool soft = run->opts.selector == SSA_SELECT_SOFT;
    if (soft && temperature != run->opts.temperature)
        return fail(SSA_ERR_INVALID_ARG, "the gradient of a soft forward is taken at the forward's temperature");
    if (run->variant == 2) {
        std::string why;
        jit = soft ? jit_soft_kernels(net, why) : jit_kernels(net, why);
        if (!jit) return fail(SSA_ERR_STATE, "specialised kernels unavailable: %s", why.c_str());
        block = kJitAdjBlock;
        grid = (run->n_traj + block - 1) / block;
    } else if (run->variant == 1) {
        block = pick_block(adj_smem, net, 0, limit);
        if (!block) return fail(SSA_ERR_UNSUPPORTED, "network too large for the thread-per-trajectory adjoint");
        grid = (run->n_traj + block - 1) / block;
    } else {
        grid = (run->n_traj + kWarpsPerBlock - 1) / kWarpsPerBlock;
    }
    int *flag = reinterpret_cast<int *>(ws + L.flag);
    CUDA_TRY(cudaMemsetAsync(flag + 2, 0, sizeof(int), st));  // mismatch counter
    p = AdjParams{};
    p.rx = run->variant == 32 ? net->d_rx_warp : net->d_rx;
    p.k_rates = reinterpret_cast<const float *>(ws + L.k_rates);
    p.tab_bytes = net->tab_bytes;
    p.k_bytes = (uint32_t)(L.M_pad * 4);
    p.N = net->N;
    p.M = net->M;
    p.Mp = net->Mp;
    p.inc_off = net->inc_off;
    p.inc_list_off = net->inc_list_off;
    p.nnz = net->nnz;
    p.n_traj = run->n_traj;
    p.traj_offset = run->traj_offset;
    p.seed = run->seed;
    p.ts = reinterpret_cast<const double *>(ws + L.ts);
    p.S = run->S;
    p.obs_sp = reinterpret_cast<const int *>(ws + L.obs_sp);
    p.n_obs = run->n_obs;
    p.K = effective_K(&run->opts);
    p.draws = reinterpret_cast<const int *>(ws + L.draws);
    p.status = reinterpret_cast<const int *>(ws + L.status);
    p.ev = reinterpret_cast<const uint4 *>(ws + L.ev);
    p.ckpt = reinterpret_cast<const int *>(ws + L.ckpt);
    p.brk_k = reinterpret_cast<const int *>(ws + L.brk_k);
    p.brk_a = reinterpret_cast<const float *>(ws + L.brk_a);
    p.brk_s = reinterpret_cast<const int *>(ws + L.brk_s);
    p.brk_tail = reinterpret_cast<const int *>(ws + L.brk_tail);
    p.xfinal = reinterpret_cast<const int *>(ws + L.xfinal);
    p.dl_dobs = dl_dobs;
    p.dl_stride = dl_traj_stride;
    p.bin_prefix = nullptr;
    if (run->opts.readout == SSA_READOUT_BIN && dl_traj_stride == 0 && run->S > 0 && run->n_obs > 0) {
        double *pre = reinterpret_cast<double *>(ws + L.bin_prefix);
        CUDA_TRY(launch_bin_prefix(dl_dobs, run->S, run->n_obs, pre, st));
        p.bin_prefix = pre;
    }
    p.invT = 1.0f / temperature;
    p.mismatch = flag + 2;
    p.err = flag + 1;
    return SSA_OK;
}

extern "C" ssa_status ssa_backward(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride, float temperature,
                                   float *dl_dlog_rates, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AdjParams p;
    const JitKernels *jit = nullptr;
    int block = 0;
    int64_t grid = 0;
    const ssa_status s = backward_setup(run, dl_dobs, dl_traj_stride, temperature, dl_dlog_rates, st, p, jit, block, grid);
    if (s != SSA_OK) return s;
    const ssa_network *net = run->net;
    unsigned char *ws = run->ws;
    p.partial = reinterpret_cast<float *>(ws + run->L.partial);
    if (run->variant == 2)
        CUDA_TRY(jit_launch_backward(jit, p, run->opts.readout, block, grid, st));
    else if (run->variant == 1)
        CUDA_TRY(launch_backward_thread(p, run->opts.readout, block, adj_smem(net, block), grid, st));
    else if (run->opts.selector == SSA_SELECT_SOFT)
        CUDA_TRY(launch_backward_warp_soft(p, net->d_upd, net->upd_words, run->opts.readout, kWarpsPerBlock,
                                           adj_warp_soft_smem(net), grid, st));
    else
        CUDA_TRY(launch_backward_warp(p, run->opts.readout, kWarpsPerBlock, adj_warp_smem(net), grid, st));
    CUDA_TRY(launch_reduce_partials(p.partial, grid, net->M, net->d_rate_index, net->P,
                                    reinterpret_cast<float *>(ws + run->L.dA), dl_dlog_rates, st));
    return SSA_OK;
}

extern "C" ssa_status ssa_backward_multi(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride,
                                         const float *temperatures, int32_t n_temps, float *dl_dlog_rates, void *stream)
{
    if (!run) return fail(SSA_ERR_INVALID_ARG, "run is NULL");
    if (!run->net) return fail(SSA_ERR_STATE, "a gene-regulatory-network run is differentiated by ssa_grn_backward");
    if (!dl_dlog_rates) return fail(SSA_ERR_INVALID_ARG, "dl_dlog_rates is NULL");
    if (n_temps < 1 || !temperatures) return fail(SSA_ERR_INVALID_ARG, "n_temps must be >= 1 with a host temperature list");
    for (int t = 0; t < n_temps; ++t)
        if (!(temperatures[t] > 0.0f) || !(temperatures[t] < 3.0e38f))
            return fail(SSA_ERR_INVALID_ARG, "temperature %d must be > 0", t);
    const bool fused = run->variant == 2 && run->opts.selector == SSA_SELECT_GUMBEL &&
                       (run->opts.readout == SSA_READOUT_HOLD || run->opts.readout == SSA_READOUT_LINEAR) &&
                       n_temps >= 2;
    if (!fused) {  // one walk per temperature
        for (int t = 0; t < n_temps; ++t) {
            const ssa_status s = ssa_backward(run, dl_dobs, dl_traj_stride, temperatures[t],
                                              dl_dlog_rates + (size_t)t * run->net->P, stream);
            if (s != SSA_OK) return s;
        }
        return SSA_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ssa_network *net = run->net;
    unsigned char *ws = run->ws;
    for (int t0 = 0; t0 < n_temps; t0 += kMaxFusedTemps) {
        const int nt = std::min(kMaxFusedTemps, n_temps - t0);
        float *out = dl_dlog_rates + (size_t)t0 * net->P;
        if (nt == 1) {
            const ssa_status s = ssa_backward(run, dl_dobs, dl_traj_stride, temperatures[t0], out, stream);
            if (s != SSA_OK) return s;
            continue;
        }
        AdjParams p;
        const JitKernels *jit = nullptr;
        int block = 0;
        int64_t grid = 0;
        const ssa_status s = backward_setup(run, dl_dobs, dl_traj_stride, temperatures[t0], out, st, p, jit, block, grid);
        if (s != SSA_OK) return s;
        for (int t = 0; t < nt; ++t) p.invT_multi[t] = 1.0f / temperatures[t0 + t];
        p.partial = reinterpret_cast<float *>(ws + run->L.partial);
        CUDA_TRY(jit_launch_backward_multi(jit, p, run->opts.readout, nt, block, grid, st));
        for (int t = 0; t < nt; ++t)
            CUDA_TRY(launch_reduce_partials(p.partial + (size_t)t * grid * net->M, grid, net->M, net->d_rate_index,
                                            net->P, reinterpret_cast<float *>(ws + run->L.dA), out + (size_t)t * net->P,
                                            st));
    }
    return SSA_OK;
}

extern "C" ssa_status ssa_backward_wide(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride, float temperature,
                                        double *dl_dlog_rates, void *stream)
{
    if (run && (run->variant != 2 || run->opts.selector != SSA_SELECT_GUMBEL ||
                (run->opts.readout != SSA_READOUT_HOLD && run->opts.readout != SSA_READOUT_LINEAR)))
        return fail(SSA_ERR_UNSUPPORTED, "the wide-range adjoint runs on a Gumbel-max forward with the HOLD or LINEAR "
                                         "readout on the network-specialised kernels");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AdjParams p;
    const JitKernels *jit = nullptr;
    int block = 0;
    int64_t grid = 0;
    const ssa_status s = backward_setup(run, dl_dobs, dl_traj_stride, temperature, dl_dlog_rates, st, p, jit, block, grid);
    if (s != SSA_OK) return s;
    const ssa_network *net = run->net;
    unsigned char *ws = run->ws;
    p.partial64 = reinterpret_cast<double *>(ws + run->L.partial64);
    CUDA_TRY(jit_launch_backward_wide(jit, p, run->opts.readout, block, grid, st));
    CUDA_TRY(launch_reduce_partials64(p.partial64, grid, net->M, net->d_rate_index, net->P,
                                      reinterpret_cast<double *>(ws + run->L.dA64), dl_dlog_rates, st));
    return SSA_OK;
}

extern "C" ssa_status ssa_run_status(const ssa_run *run, int64_t *host_counts, int64_t *host_bwd_mismatch, void *stream)
{
    if (!run || !host_counts) return fail(SSA_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *ws = run->ws;
    unsigned long long *counts = reinterpret_cast<unsigned long long *>(ws + run->L.counts);
    CUDA_TRY(cudaMemsetAsync(counts, 0, SSA_TRAJ_N_CODES * sizeof(unsigned long long), st));
    if (run->n_traj > 0)
        CUDA_TRY(launch_status_count(reinterpret_cast<const int *>(ws + run->L.status), run->n_traj, counts, st));
    unsigned long long hc[SSA_TRAJ_N_CODES];
    int flags[4];
    CUDA_TRY(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(flags, ws + run->L.flag, sizeof(flags), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int c = 0; c < SSA_TRAJ_N_CODES; ++c) host_counts[c] = (int64_t)hc[c];
    if (host_bwd_mismatch) *host_bwd_mismatch = flags[2];
    if (flags[1] & kErrStageTimeout) return fail(SSA_ERR_CUDA, "a kernel timed out staging its tables");
    return SSA_OK;
}

extern "C" ssa_status ssa_run_events(const ssa_run *run, int32_t *events_out, int64_t stride, void *stream)
{
    if (!run || !events_out || stride < 1) return fail(SSA_ERR_INVALID_ARG, "bad arguments");
    if (!run->opts.record) return fail(SSA_ERR_STATE, "the forward was not recorded");
    if (run->opts.selector == SSA_SELECT_SOFT) return fail(SSA_ERR_STATE, "a soft forward keeps no event log");
    unsigned char *ws = run->ws;
    CUDA_TRY(launch_unpack_events(reinterpret_cast<const uint4 *>(ws + run->L.ev),
                                  reinterpret_cast<const int *>(ws + run->L.draws), run->n_traj, stride, events_out,
                                  static_cast<cudaStream_t>(stream)));
    return SSA_OK;
}

extern "C" ssa_status ssa_run_brackets(const ssa_run *run, int32_t *brackets_out, void *stream)
{
    if (!run || (!brackets_out && run->n_traj > 0 && run->S > 0)) return fail(SSA_ERR_INVALID_ARG, "bad arguments");
    if (!run->opts.record) return fail(SSA_ERR_STATE, "the forward was not recorded");
    const bool bin = run->opts.readout == SSA_READOUT_BIN;
    CUDA_TRY(launch_transpose_brackets(reinterpret_cast<const int *>(run->ws + run->L.brk_k), run->n_traj, run->S,
                                       bin ? reinterpret_cast<const int *>(run->ws + run->L.brk_s) : nullptr,
                                       reinterpret_cast<const int *>(run->ws + run->L.brk_tail), brackets_out,
                                       static_cast<cudaStream_t>(stream)));
    return SSA_OK;
}

extern "C" void ssa_destroy_run(ssa_run *run) { delete run; }

extern "C" int32_t ssa_run_variant(const ssa_run *run) { return run ? run->variant : 0; }

extern "C" ssa_status ssa_exp_variates(const uint32_t *words, int64_t n, float *out, void *stream)
{
    if (n < 0 || (n > 0 && (!words || !out))) return fail(SSA_ERR_INVALID_ARG, "bad arguments");
    CUDA_TRY(launch_exp_variates(words, n, out, static_cast<cudaStream_t>(stream)));
    return SSA_OK;
}

extern "C" size_t ssa_ensemble_mean_workspace_bytes(int64_t n_traj, int64_t row_len)
{
    if (n_traj < 0 || row_len < 0) return 0;
    const int64_t chunk = 256;
    const int64_t n_chunks = (n_traj + chunk - 1) / chunk;
    return (size_t)((n_chunks > 0 ? n_chunks : 1) * (row_len > 0 ? row_len : 1)) * sizeof(float);
}

extern "C" ssa_status ssa_ensemble_mean(const void *obs, int32_t obs_is_int, int64_t n_traj, int64_t row_len,
                                        void *workspace, size_t workspace_bytes, float *mean_out, void *stream)
{
    if (n_traj < 0 || row_len < 0) return fail(SSA_ERR_INVALID_ARG, "negative size");
    if ((n_traj > 0 && row_len > 0 && !obs) || (row_len > 0 && !mean_out)) return fail(SSA_ERR_INVALID_ARG, "NULL pointer");
    if (!workspace || workspace_bytes < ssa_ensemble_mean_workspace_bytes(n_traj, row_len))
        return fail(SSA_ERR_WORKSPACE, "workspace too small");
    CUDA_TRY(launch_ensemble_mean(obs, obs_is_int != 0, n_traj, row_len, static_cast<float *>(workspace), 256, mean_out,
                                  static_cast<cudaStream_t>(stream)));
    return SSA_OK;
}

extern "C" ssa_status ssa_philox_uniforms(uint64_t seed, const uint64_t *traj, const uint64_t *step, int64_t n,
                                          int32_t n_words, float *out, void *stream)
{
    if (n < 0 || n_words < 0) return fail(SSA_ERR_INVALID_ARG, "negative size");
    if (n > 0 && n_words > 0 && (!traj || !step || !out)) return fail(SSA_ERR_INVALID_ARG, "NULL pointer");
    CUDA_TRY(launch_philox_uniforms(seed, traj, step, n, n_words, out, static_cast<cudaStream_t>(stream)));
    return SSA_OK;
}
