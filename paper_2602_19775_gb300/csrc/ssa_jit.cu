// ssa_jit.cu -- network-specialised kernels compiled at run time with NVRTC.
//
// For a network with few species and reactions, the thread-per-trajectory forward and adjoint are
// generated with the network written into the code: the reactant indices, orders and stoichiometric
// changes become constants, so the counts X and the state adjoint lambda live in registers, every
// propensity is a fixed expression, and the update X += v_j is a switch over j with immediate
// increments. The per-step arithmetic is the generic kernels' (the shared helpers of ssa_device.cuh
// in the same order), so both give the same trajectories bit for bit; only the table lookups and
// the shared-memory traffic go away. The generated source is compiled once per distinct network and
// process (cached for its lifetime) for sm_103a and loaded as a context-independent CUDA library.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvrtc.h>

#include "ssa_host.h"
#include "ssa_jit_text.h"  // generated by build.py: the texts of ssa_device.cuh, ssa_jit_body.cuh, ssa.h

namespace ssa {

constexpr int kJitMaxSpecies = 24;
constexpr int kJitMaxReactions = 24;
constexpr int kJitMaxNnz = 96;

struct JitKernels {
    cudaKernel_t fwd[3][2];     // [readout][record], Gumbel-max choice (soft set: the soft forward)
    cudaKernel_t fwd_direct[3]; // [readout], direct method, forward only (not in the soft set)
    cudaKernel_t adj[3];        // [readout]
    cudaKernel_t adj_wide[2];   // [HOLD, LINEAR], wide-range adjoint (not in the soft set)
    cudaKernel_t adj_multi[2][2];  // [HOLD, LINEAR][2 or 3 temperatures] in one walk (not in the soft set)
};

namespace {

std::mutex g_jit_mu;
// source text -> kernels; libraries stay loaded until the process exits
std::map<std::string, JitKernels> g_jit_cache;
std::map<std::string, std::string> g_jit_failed;  // source text -> reason

void emit(std::string &out, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
void emit(std::string &out, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    out += buf;
}

// The event hooks written as selects (bit 1: X -= v_jb, 2: a component of v_jb, 4: X += v_jb, 8: the range
// check) for networks with up to kJitSelectNnz stoichiometric entries; the others switch on jb. Timed on one
// box (C2 step: adjoint 0.745 ms with switches, 0.716 with the component as selects, 0.739 with X -= v_jb as
// selects, 0.713 with both; the oscillator's forward + adjoint 4.75e9 steps/s with switches and with the
// component as selects, 4.62e9 once X -= v_jb is selects): the component only.
#ifndef SSA_JIT_SELECT
#define SSA_JIT_SELECT 2
#endif
constexpr int kJitSelectNnz = 48;

int st_species(int e) { return e >> 8; }
int st_delta(int e) { return (int)(signed char)(e & 0xff); }

// The network hooks that ssa_jit_body.cuh calls, written out for one network.
std::string jit_source(const ssa_network *net)
{
    const int N = net->N, M = net->M;
    std::string s;
    s += "#include \"ssa_device.cuh\"\n";
    emit(s, "#define JN %d\n#define JM %d\nnamespace ssa {\n", N, M);
    // propensities, in reaction order
    s += "__device__ __forceinline__ void jit_props(const int (&X)[JN], const float (&k)[JM], float (&a)[JM], "
         "float (&h)[JM])\n{\n";
    for (int j = 0; j < M; ++j) {
        const int4 r = net->h_rx[j];
        if (r.x < 0) emit(s, "    h[%d] = 1.0f;\n", j);
        else if (r.y < 0) emit(s, "    h[%d] = h_first(X[%d]);\n", j, r.x);
        else if (r.y == r.x) emit(s, "    h[%d] = h_homodimer(X[%d]);\n", j, r.x);
        else emit(s, "    h[%d] = h_hetero(X[%d], X[%d]);\n", j, r.x, r.y);
        emit(s, "    a[%d] = __fmul_rn(k[%d], h[%d]);\n", j, j, j);
    }
    s += "}\n";
    // The event-dependent hooks (range check, X += v_jb, X -= v_jb, a component of v_jb) switch on jb, whose
    // cases the lanes of a warp run one after another when their events differ; up to kJitSelectNnz
    // stoichiometric entries, the hooks named in SSA_JIT_SELECT are written instead as selects over every entry
    // (the same results, no divergence; a tuning choice, set by timing both forms).
    const bool small = net->nnz <= kJitSelectNnz;
    const bool sel_check = small && (SSA_JIT_SELECT & 8), sel_apply = small && (SSA_JIT_SELECT & 4);
    const bool sel_unapply = small && (SSA_JIT_SELECT & 1), sel_dv = small && (SSA_JIT_SELECT & 2);
    // range check of X + v_jb (entries in table order; the last failing entry decides)
    s += "__device__ __forceinline__ int jit_check(const int (&X)[JN], int jb)\n{\n    int st = SSA_TRAJ_OK;\n";
    if (sel_check) {
        for (int j = 0; j < M; ++j)
            for (int e = net->h_rx[j].z; e < net->h_rx[j].w; ++e) {
                const int sp = st_species(net->h_st[e]), d = st_delta(net->h_st[e]);
                if (d < 0) emit(s, "    st = (jb == %d && X[%d] + (%d) < 0) ? SSA_TRAJ_NEG_COUNT : st;\n", j, sp, d);
                else if (d > 0) emit(s, "    st = (jb == %d && X[%d] > 2147483647 - %d) ? SSA_TRAJ_OVERFLOW : st;\n", j, sp, d);
            }
    } else {
        s += "    switch (jb) {\n";
        for (int j = 0; j < M; ++j) {
            emit(s, "    case %d:\n", j);
            for (int e = net->h_rx[j].z; e < net->h_rx[j].w; ++e) {
                const int sp = st_species(net->h_st[e]), d = st_delta(net->h_st[e]);
                if (d < 0) emit(s, "        if (X[%d] + (%d) < 0) st = SSA_TRAJ_NEG_COUNT;\n", sp, d);
                else if (d > 0) emit(s, "        if (X[%d] > 2147483647 - %d) st = SSA_TRAJ_OVERFLOW;\n", sp, d);
            }
            s += "        break;\n";
        }
        s += "    default: break;\n    }\n";
    }
    s += "    return st;\n}\n";
    // X += v_jb and X -= v_jb
    for (int dir = 0; dir < 2; ++dir) {
        emit(s, "__device__ __forceinline__ void %s(int (&X)[JN], int jb)\n{\n", dir == 0 ? "jit_apply" : "jit_unapply");
        if (dir == 0 ? sel_apply : sel_unapply) {
            // per species, the change of the reaction that fired (a chain of selects over its entries)
            for (int sp = 0; sp < N; ++sp) {
                std::string expr = "0";
                for (int j = M - 1; j >= 0; --j)
                    for (int e = net->h_rx[j].z; e < net->h_rx[j].w; ++e)
                        if (st_species(net->h_st[e]) == sp) {
                            char buf[64];
                            snprintf(buf, sizeof(buf), "(jb == %d ? %d : ", j, st_delta(net->h_st[e]));
                            expr = buf + expr + ")";
                        }
                // appended directly: the expression may exceed emit's buffer
                if (expr != "0") s += "    X[" + std::to_string(sp) + "] " + (dir == 0 ? "+=" : "-=") + " " + expr + ";\n";
            }
        } else {
            s += "    switch (jb) {\n";
            for (int j = 0; j < M; ++j) {
                emit(s, "    case %d:\n", j);
                for (int e = net->h_rx[j].z; e < net->h_rx[j].w; ++e)
                    emit(s, "        X[%d] %s %d;\n", st_species(net->h_st[e]), dir == 0 ? "+=" : "-=",
                         st_delta(net->h_st[e]));
                s += "        break;\n";
            }
            s += "    default: break;\n    }\n";
        }
        s += "}\n";
    }
    // component sp of v_jb
    s += "__device__ __forceinline__ int jit_dv(int jb, int sp)\n{\n    int v = 0;\n";
    if (sel_dv) {
        for (int j = 0; j < M; ++j)
            for (int e = net->h_rx[j].z; e < net->h_rx[j].w; ++e)
                emit(s, "    v += (jb == %d && sp == %d) ? %d : 0;\n", j, st_species(net->h_st[e]), st_delta(net->h_st[e]));
    } else {
        s += "    switch (jb) {\n";
        for (int j = 0; j < M; ++j) {
            emit(s, "    case %d:\n", j);
            for (int e = net->h_rx[j].z; e < net->h_rx[j].w; ++e)
                emit(s, "        if (sp == %d) v += %d;\n", st_species(net->h_st[e]), st_delta(net->h_st[e]));
            s += "        break;\n";
        }
        s += "    default: break;\n    }\n";
    }
    s += "    return v;\n}\n";
    // w_j = v_j . lambda, summed over the entries in table order from zero
    s += "__device__ __forceinline__ void jit_w(const float (&lam)[JN], float (&w)[JM])\n{\n";
    for (int j = 0; j < M; ++j) {
        s += "    {\n        float v = 0.0f;\n";
        for (int e = net->h_rx[j].z; e < net->h_rx[j].w; ++e)
            emit(s, "        v += (float)(%d) * lam[%d];\n", st_delta(net->h_st[e]), st_species(net->h_st[e]));
        emit(s, "        w[%d] = v;\n    }\n", j);
    }
    s += "}\n";
    // state adjoint of every reaction, in order
    s += "__device__ __forceinline__ void jit_state_adj(const int (&X)[JN], const float (&a)[JM], const float (&h)[JM], "
         "const float (&psi)[JM], const float (&ctau)[JM], float (&lam)[JN])\n{\n";
    for (int j = 0; j < M; ++j) {
        const int4 r = net->h_rx[j];
        if (r.x < 0) continue;
        if (r.y < 0) {
            emit(s, "    lam[%d] += sadj_first(int2f(X[%d]), a[%d], psi[%d], ctau[%d]);\n", r.x, r.x, j, j, j);
        } else if (r.y == r.x) {
            emit(s, "    lam[%d] += sadj_homodimer(int2f(X[%d]), a[%d], h[%d], psi[%d], ctau[%d]);\n", r.x, r.x, j, j,
                 j, j);
        } else {
            emit(s, "    {\n        const float x1 = int2f(X[%d]), x2 = int2f(X[%d]);\n", r.x, r.y);
            emit(s, "        lam[%d] += sadj_hetero(x1, x2, a[%d], psi[%d], ctau[%d]);\n", r.x, j, j, j);
            emit(s, "        lam[%d] += sadj_hetero(x2, x1, a[%d], psi[%d], ctau[%d]);\n    }\n", r.y, j, j, j);
        }
    }
    s += "}\n";
    // soft forward (Eq. 4): propensities of the real-valued state (negative factors clipped to 0), the
    // relaxed update dX = sum_j y_j v_j (entries in table order), and the state adjoint with the
    // waiting-time derivative of a clipped factor removed
    s += "__device__ __forceinline__ void jit_props_soft(const float (&X)[JN], const float (&k)[JM], float (&a)[JM], "
         "float (&h)[JM])\n{\n";
    for (int j = 0; j < M; ++j) {
        const int4 r = net->h_rx[j];
        if (r.x < 0) emit(s, "    h[%d] = 1.0f;\n", j);
        else if (r.y < 0) emit(s, "    h[%d] = hs_first(X[%d]);\n", j, r.x);
        else if (r.y == r.x) emit(s, "    h[%d] = hs_homodimer(X[%d]);\n", j, r.x);
        else emit(s, "    h[%d] = hs_hetero(X[%d], X[%d]);\n", j, r.x, r.y);
        emit(s, "    a[%d] = __fmul_rn(k[%d], h[%d]);\n", j, j, j);
    }
    s += "}\n";
    s += "__device__ __forceinline__ void jit_dx_soft(const float (&y)[JM], float (&dX)[JN])\n{\n";
    s += "#pragma unroll\n    for (int q = 0; q < JN; ++q) dX[q] = 0.0f;\n";
    for (int j = 0; j < M; ++j)
        for (int e = net->h_rx[j].z; e < net->h_rx[j].w; ++e)
            emit(s, "    dX[%d] = __fmaf_rn(y[%d], %d.0f, dX[%d]);\n", st_species(net->h_st[e]), j, st_delta(net->h_st[e]),
                 st_species(net->h_st[e]));
    s += "}\n";
    s += "__device__ __forceinline__ void jit_state_adj_soft(const float (&X)[JN], const float (&a)[JM], "
         "const float (&h)[JM], const float (&psi)[JM], const float (&ctau)[JM], float (&lam)[JN])\n{\n";
    for (int j = 0; j < M; ++j) {
        const int4 r = net->h_rx[j];
        if (r.x < 0) continue;
        if (r.y < 0) {
            emit(s, "    lam[%d] += sadj_first(X[%d], a[%d], psi[%d], X[%d] < 0.0f ? 0.0f : ctau[%d]);\n", r.x, r.x, j, j,
                 r.x, j);
        } else if (r.y == r.x) {
            emit(s, "    lam[%d] += sadj_homodimer(X[%d], a[%d], h[%d], psi[%d], __fmul_rn(X[%d], X[%d] - 1.0f) < 0.0f ? "
                    "0.0f : ctau[%d]);\n", r.x, r.x, j, j, j, r.x, r.x, j);
        } else {
            emit(s, "    {\n        const float x1 = X[%d], x2 = X[%d];\n", r.x, r.y);
            emit(s, "        const float c = __fmul_rn(x1, x2) < 0.0f ? 0.0f : ctau[%d];\n", j);
            emit(s, "        lam[%d] += sadj_hetero(x1, x2, a[%d], psi[%d], c);\n", r.x, j, j);
            emit(s, "        lam[%d] += sadj_hetero(x2, x1, a[%d], psi[%d], c);\n    }\n", r.y, j, j);
        }
    }
    s += "}\n}  // namespace ssa\n#include \"ssa_jit_body.cuh\"\n";
    return s;
}

const char *kStddef = "#pragma once\ntypedef unsigned long size_t;\n";
const char *kStdint =
    "#pragma once\ntypedef signed char int8_t;\ntypedef short int16_t;\ntypedef int int32_t;\ntypedef long int64_t;\n"
    "typedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\ntypedef unsigned int uint32_t;\n"
    "typedef unsigned long uint64_t;\ntypedef unsigned long uintptr_t;\n";

bool compile(const std::string &src, std::vector<char> &cubin, std::string &why)
{
    const char *hdr_text[] = {kJitTextDevice, kJitTextBody, kJitTextApi, kStddef, kStdint};
    const char *hdr_name[] = {"ssa_device.cuh", "ssa_jit_body.cuh", "../../include/ssa.h", "stddef.h", "stdint.h"};
    nvrtcProgram prog;
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "ssa_network.cu", 5, hdr_text, hdr_name);
    if (r != NVRTC_SUCCESS) {
        why = nvrtcGetErrorString(r);
        return false;
    }
    // -default-device: the C declarations of ssa.h (for its constants) are read as device declarations
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "--fmad=true", "-default-device"};
    r = nvrtcCompileProgram(prog, 4, opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        if (n) nvrtcGetProgramLog(prog, &log[0]);
        why = std::string(nvrtcGetErrorString(r)) + ": " + log.substr(0, 400);
        nvrtcDestroyProgram(&prog);
        return false;
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin.resize(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    return n > 0;
}

}  // namespace

bool jit_eligible(const ssa_network *net)
{
    return net->N <= kJitMaxSpecies && net->M <= kJitMaxReactions && net->nnz <= kJitMaxNnz;
}

namespace {
// Kernels of `net` (soft: the soft-forward program of the same text), compiling and loading them on
// first use. Returns nullptr (with the reason in `why`) if the network is not eligible or compilation
// failed.
const JitKernels *jit_load(const ssa_network *net, bool soft, std::string &why)
{
    if (!jit_eligible(net)) {
        why = "network above the specialisation limits (24 species, 24 reactions, 96 stoichiometric entries)";
        return nullptr;
    }
    const std::string src = (soft ? std::string("#define SSA_JIT_SOFT 1\n") : std::string()) + jit_source(net);
    std::lock_guard<std::mutex> lock(g_jit_mu);
    auto f = g_jit_failed.find(src);
    if (f != g_jit_failed.end()) {
        why = f->second;
        return nullptr;
    }
    auto it = g_jit_cache.find(src);
    if (it != g_jit_cache.end()) return &it->second;
    std::vector<char> cubin;
    if (!compile(src, cubin, why)) {
        g_jit_failed[src] = why;
        return nullptr;
    }
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        why = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
        g_jit_failed[src] = why;
        return nullptr;
    }
    JitKernels k{};
    const char *rname[3] = {"hold", "linear", "bin"};
    bool ok = true;
    for (int r = 0; r < 3; ++r) {
        const std::string base = std::string(rname[r]) + (soft ? "_soft" : "");
        for (int rec = 0; rec < 2; ++rec) {
            const std::string nm = "ssa_jit_fwd_" + base + (rec ? "_rec" : "");
            ok &= cudaLibraryGetKernel(&k.fwd[r][rec], lib, nm.c_str()) == cudaSuccess;
        }
        ok &= cudaLibraryGetKernel(&k.adj[r], lib, ("ssa_jit_adj_" + base).c_str()) == cudaSuccess;
        if (!soft)
            ok &= cudaLibraryGetKernel(&k.fwd_direct[r], lib, ("ssa_jit_fwd_" + base + "_direct").c_str()) == cudaSuccess;
        if (!soft && r < 2) {
            ok &= cudaLibraryGetKernel(&k.adj_wide[r], lib, ("ssa_jit_adj_" + base + "_wide").c_str()) == cudaSuccess;
            for (int nt = 2; nt <= 3; ++nt)
                ok &= cudaLibraryGetKernel(&k.adj_multi[r][nt - 2], lib,
                                           ("ssa_jit_adj_" + base + "_t" + std::to_string(nt)).c_str()) == cudaSuccess;
        }
    }
    if (!ok) {
        why = "a specialised kernel is missing from the library";
        g_jit_failed[src] = why;
        cudaLibraryUnload(lib);
        return nullptr;
    }
    return &(g_jit_cache[src] = k);
}
}  // namespace

const JitKernels *jit_kernels(const ssa_network *net, std::string &why) { return jit_load(net, false, why); }
const JitKernels *jit_soft_kernels(const ssa_network *net, std::string &why) { return jit_load(net, true, why); }

cudaError_t jit_launch_forward(const JitKernels *k, const FwdParams &p, int readout, bool record, int selector,
                               int block, cudaStream_t st)
{
    if (p.n_traj == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((p.n_traj + block - 1) / block);
    void *args[] = {const_cast<FwdParams *>(&p)};
    const int r = readout;  // SSA_READOUT_HOLD, _LINEAR, _BIN index the tables
    const cudaKernel_t f = selector == SSA_SELECT_DIRECT ? k->fwd_direct[r] : k->fwd[r][record ? 1 : 0];
    return cudaLaunchKernel(reinterpret_cast<const void *>(f), dim3(grid), dim3((unsigned)block), args, 0, st);
}

cudaError_t jit_launch_backward(const JitKernels *k, const AdjParams &p, int readout, int block, int64_t grid,
                                cudaStream_t st)
{
    if (grid == 0) return cudaSuccess;
    void *args[] = {const_cast<AdjParams *>(&p)};
    const size_t smem = (size_t)4 * p.M * block;
    return cudaLaunchKernel(reinterpret_cast<const void *>(k->adj[readout]),
                            dim3((unsigned)grid), dim3((unsigned)block), args, smem, st);
}

cudaError_t jit_launch_backward_wide(const JitKernels *k, const AdjParams &p, int readout, int block, int64_t grid,
                                     cudaStream_t st)
{
    if (grid == 0) return cudaSuccess;
    if (readout != SSA_READOUT_HOLD && readout != SSA_READOUT_LINEAR) return cudaErrorInvalidValue;
    void *args[] = {const_cast<AdjParams *>(&p)};
    const size_t smem = (size_t)8 * p.M * block;  // binary64 block reduction
    return cudaLaunchKernel(reinterpret_cast<const void *>(k->adj_wide[readout]),
                            dim3((unsigned)grid), dim3((unsigned)block), args, smem, st);
}

cudaError_t jit_launch_backward_multi(const JitKernels *k, const AdjParams &p, int readout, int n_temps, int block,
                                      int64_t grid, cudaStream_t st)
{
    if (grid == 0) return cudaSuccess;
    if ((readout != SSA_READOUT_HOLD && readout != SSA_READOUT_LINEAR) || n_temps < 2 || n_temps > 3)
        return cudaErrorInvalidValue;
    void *args[] = {const_cast<AdjParams *>(&p)};
    const size_t smem = (size_t)4 * n_temps * p.M * block;
    return cudaLaunchKernel(reinterpret_cast<const void *>(k->adj_multi[readout][n_temps - 2]),
                            dim3((unsigned)grid), dim3((unsigned)block), args, smem, st);
}

}  // namespace ssa

using namespace ssa;

extern "C" ssa_status ssa_network_specialize(ssa_network *net, int32_t *host_ok)
{
    if (!net || !host_ok) return set_error(SSA_ERR_INVALID_ARG, "NULL argument");
    std::string why;
    *host_ok = jit_kernels(net, why) ? 1 : 0;
    if (!*host_ok) set_error(SSA_OK, why.c_str());
    return SSA_OK;
}
