/*
 * ssa.h -- C ABI of the GB300 (sm_103a) library for exact stochastic simulation with a
 * Gumbel-max reaction choice and a Gumbel-Softmax straight-through adjoint
 * (arXiv 2602.19775, "Exact Discrete Stochastic Simulation with Deep-Learning-Scale Gradient
 * Optimization").
 *
 * Conventions for every entry point
 *   - Plain C types only. `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Pointers documented as "device" must be device (or managed) memory on the current device;
 *     "host" pointers are read before the call returns.
 *   - The caller owns every buffer it passes, including the workspace; the library owns only the
 *     opaque handles and the small constant tables they hold.
 *   - Every call except ssa_create_*, ssa_destroy_*, ssa_run_status and ssa_last_error is
 *     asynchronous on `stream`.
 *   - Return value: SSA_OK (0) or a negative error code; ssa_last_error() gives a text for the
 *     most recent failure on the calling thread. No C++ exception crosses this boundary.
 *   - Per-trajectory outcomes are written as SSA_TRAJ_* codes to a device status array.
 *
 * Noise: Philox4x32-10 (Salmon et al., SC'11), key = (seed_lo, seed_hi), counter =
 * (b, k, i_lo, i_hi) for global trajectory id i (= traj_offset + local index), step k and block b;
 * word q = 4b + w of the step's stream gives u_q = ((x >> 9) + 1/2) 2^-23 in (0,1); u_0 drives the
 * waiting time and u_{1+j} reaction j. Results depend only on (network, parameters, x0, seed,
 * global trajectory id), never on launch shape, chunking or batching.
 */
#ifndef SSA_H
#define SSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ssa_status;

#define SSA_OK 0
#define SSA_ERR_INVALID_ARG (-1) /* an argument is out of range or inconsistent */
#define SSA_ERR_CUDA (-2)        /* a CUDA runtime call failed (text in ssa_last_error) */
#define SSA_ERR_WORKSPACE (-3)   /* workspace too small or misaligned (need 256-byte alignment) */
#define SSA_ERR_UNSUPPORTED (-4) /* valid but outside the library's limits (e.g. M > 65535) */
#define SSA_ERR_STATE (-5)       /* the run handle cannot serve this call (e.g. not recorded) */

/* per-trajectory status codes */
#define SSA_TRAJ_OK 0             /* reached t_end; the crossing draw was made, not applied */
#define SSA_TRAJ_ABSORBED 1       /* a0 == 0 before t_end; the state holds to t_end          */
#define SSA_TRAJ_STEP_CAP 2       /* max_steps draws made and applied before t_end           */
#define SSA_TRAJ_NEG_COUNT 3      /* the chosen update would make a count negative           */
#define SSA_TRAJ_OVERFLOW 4       /* the chosen update would leave the int32 range           */
#define SSA_TRAJ_BAD_RATE 5       /* a propensity or a0 was not finite                       */
#define SSA_TRAJ_BAD_INPUT 6      /* sample times not ascending within [0, t_end]           */
#define SSA_TRAJ_REPLAY_MISMATCH 7/* replay: the given events do not fit the trajectory     */
#define SSA_TRAJ_N_CODES 8

#define SSA_READOUT_HOLD 0   /* obs = X(t_s), right-continuous; int32 output              */
#define SSA_READOUT_LINEAR 1 /* obs = X_k + (t_s - t_k)/tau_k (X_{k+1} - X_k); float output */
/* Exact bin average (Section 4.4): obs_s = the integral of the piecewise-constant path over the
 * bin (t_{s-1}, t_s], t_{-1} = 0, divided by its width; float output. The sample times are the
 * bins' right edges and must be strictly increasing with t_0 > 0 (else every trajectory reports
 * SSA_TRAJ_BAD_INPUT); a stopped path holds its last state. At most SSA_BIN_MAX_OBS observables
 * per call (call again with other species: the paths depend only on the seed). Runs on the
 * thread-per-trajectory kernels (generic and network-specialised), on the warp-per-trajectory
 * kernels and in the batch; the GRN calls return SSA_ERR_UNSUPPORTED for it. */
#define SSA_READOUT_BIN 2
#define SSA_BIN_MAX_OBS 4

typedef struct ssa_network ssa_network;
typedef struct ssa_run ssa_run;

typedef struct ssa_fwd_opts {
    int32_t readout;          /* SSA_READOUT_HOLD, SSA_READOUT_LINEAR or SSA_READOUT_BIN          */
    int32_t record;           /* nonzero: keep event log, checkpoints and sample brackets so that
                                 ssa_backward can run on this forward                            */
    int32_t ckpt_interval;    /* K: checkpoint the state every K steps (multiple of 8; 0 -> 64)   */
    int32_t threads_per_traj; /* 0: choose; 1: one thread per trajectory; 32: one warp per
                                 trajectory (networks with hundreds of reactions)               */
    int64_t max_steps;        /* cap on reaction draws per trajectory (>= 1); sizes the log       */
    int32_t block_threads;    /* 0: choose; else a multiple of 32 in [32, 1024]                  */
    int32_t no_specialize;    /* 0: run the thread variant as kernels compiled for this network
                                 (NVRTC, at most 24 species, 24 reactions, 96 stoichiometric
                                 entries; the same results bit for bit) when it qualifies;
                                 1: always the generic kernels                                  */
    int32_t selector;         /* SSA_SELECT_GUMBEL (the method), SSA_SELECT_DIRECT (the plain
                                 direct method, forward only: record must be 0) or
                                 SSA_SELECT_SOFT (the relaxed forward of Eq. 4). The direct
                                 method runs on the network-specialised kernels only; the soft
                                 forward on them where the network qualifies, otherwise on the
                                 warp-per-trajectory kernels                                    */
    float temperature;        /* SSA_SELECT_SOFT: T > 0 of its soft sample; else must be 0       */
} ssa_fwd_opts;

#define SSA_SELECT_GUMBEL 0 /* j* = argmax_j a_j / E_{1+j}, the Gumbel-max choice (Section 3.2)    */
#define SSA_SELECT_DIRECT 1 /* the first j with a_1 + ... + a_j > u_1 a0 in reaction order: the
                               standard direct method (Section 2), the plain-SSA comparator       */
/* The soft forward (Section 3.3, Eq. 4): the state is real-valued and moves every step by the
 * expected stoichiometry sum_j y~_j v_j of the soft sample y~ = softmax((log a + G)/T) of the same
 * Gumbel noise; a mass-action factor that comes out negative on a relaxed state is taken as 0. The
 * clock, the samples and the three readouts are the forward's; observables are float for every
 * readout. Recorded, it checkpoints the float state every 8 steps (ckpt_interval is ignored), and
 * ssa_backward then gives the exact gradient of this relaxed model (it re-runs each 8-step segment,
 * so its temperature argument must equal opts.temperature). No event log is kept. Networks beyond the
 * specialised kernels' limits (or threads_per_traj = 32, or no_specialize) run the soft forward one warp
 * per trajectory: every species sums its changes in increasing reaction order as the specialised kernels
 * do, a0 and the normaliser are warp sums (so the results agree with the specialised kernels to binary32
 * rounding, not bit for bit), and ssa_backward there re-runs each 8-step segment the same way. */
#define SSA_SELECT_SOFT 2

/*
 * ssa_create_network -- a mass-action reaction network (Section 2).
 *   n_species N >= 1, n_reactions M in [1, 65535].
 *   reactants      host int32 [M][2]: reactant species of reaction j or -1 for an empty slot.
 *                  Order = number of non-negative slots; equal slots = homodimer.
 *                  Propensity (Section 2): a_j = k_j h_j(X) with h = 1, X_i, X_i X_l or
 *                  X_i (X_i - 1)/2.
 *   stoich_ptr     host int32 [M+1], CSR row pointer of the net change v_j (Eq. 6).
 *   stoich_species host int32 [nnz] in [0, N); stoich_delta host int32 [nnz] in [-127, 127].
 *   n_params P >= 1; rate_index host int32 [M] in [0, P): k_j = exp(theta[rate_index[j]]).
 *   out            receives the handle (device tables are allocated here).
 * Errors: SSA_ERR_INVALID_ARG for any out-of-range entry, SSA_ERR_CUDA on allocation failure.
 */
ssa_status ssa_create_network(int32_t n_species, int32_t n_reactions, const int32_t *reactants,
                              const int32_t *stoich_ptr, const int32_t *stoich_species,
                              const int32_t *stoich_delta, int32_t n_params,
                              const int32_t *rate_index, ssa_network **out);
void ssa_destroy_network(ssa_network *net);

/*
 * ssa_forward_workspace_bytes -- bytes of device workspace ssa_forward needs for this
 * (network, n_traj, n_samples, opts). With opts->record the size includes the event log
 * (2 bytes per step up to max_steps), checkpoints every K steps, the sample brackets and the
 * per-block partial sums of the backward. Returns 0 for invalid arguments.
 */
size_t ssa_forward_workspace_bytes(const ssa_network *net, int64_t n_traj, int32_t n_samples,
                                   const ssa_fwd_opts *opts);

/*
 * ssa_forward -- simulate n_traj independent trajectories with the exact direct method
 * (Section 2: propensities, a0, tau = -ln(u_0)/a0) and the Gumbel-max choice
 * j* = argmax_j [log a_j + G_j] of Section 3.2 (computed as argmax a_j/E_j, E_j = -ln u_{1+j},
 * the same choice), applying X <- X + v_{j*} (Eq. 6) until the clock passes t_end.
 *   log_rates     device float [P]: theta = log k.
 *   n_traj >= 0; traj_offset: global id of the first trajectory (Philox counter).
 *   x0            device int32 [N] (x0_per_traj = 0) or [n_traj][N] (x0_per_traj = 1).
 *   t_end >= 0.   sample_times device double [n_samples], ascending, each in [0, t_end]
 *                 (BIN: strictly increasing, the first > 0).
 *   obs_species   device int32 [n_obs] in [0, N) (BIN: n_obs <= SSA_BIN_MAX_OBS).
 *   workspace     device, >= ssa_forward_workspace_bytes(...), 256-byte aligned, caller-owned;
 *                 it must stay alive and untouched until ssa_destroy_run(*run_out).
 *   obs_out       device [n_traj][n_samples][n_obs]: int32 (HOLD) or float (LINEAR, Section 4.1;
 *                 BIN, Section 4.4).
 *   draws_out     device int32 [n_traj] or NULL: reaction draws including the crossing draw.
 *   status_out    device int32 [n_traj] or NULL: SSA_TRAJ_* per trajectory.
 *   run_out       receives a handle for ssa_backward / ssa_run_status (may be NULL).
 * Precision: FP32 propensities, keys and waiting times; FP64 clock and sample comparisons;
 * exact int32 counts.
 */
ssa_status ssa_forward(const ssa_network *net, const float *log_rates, int64_t n_traj,
                       int64_t traj_offset, const int32_t *x0, int32_t x0_per_traj, double t_end,
                       const double *sample_times, int32_t n_samples, const int32_t *obs_species,
                       int32_t n_obs, uint64_t seed, const ssa_fwd_opts *opts, void *workspace,
                       size_t workspace_bytes, void *obs_out, int32_t *draws_out,
                       int32_t *status_out, void *stream, ssa_run **run_out);

/*
 * ssa_forward_replay -- as ssa_forward, but reaction k of trajectory i is events[i][k] (given,
 * e.g. by an independent implementation) instead of the Gumbel-max choice; waiting times still
 * come from the trajectory's own noise. Trajectories whose clock and given events disagree
 * (a given event with a_j = 0, too few or too many events for t_end) get
 * SSA_TRAJ_REPLAY_MISMATCH.
 *   events    device uint16 [n_traj][events_stride]; n_events device int32 [n_traj].
 */
ssa_status ssa_forward_replay(const ssa_network *net, const float *log_rates, int64_t n_traj,
                              int64_t traj_offset, const int32_t *x0, int32_t x0_per_traj,
                              double t_end, const double *sample_times, int32_t n_samples,
                              const int32_t *obs_species, int32_t n_obs, uint64_t seed,
                              const ssa_fwd_opts *opts, const uint16_t *events,
                              const int32_t *n_events, int64_t events_stride, void *workspace,
                              size_t workspace_bytes, void *obs_out, int32_t *draws_out,
                              int32_t *status_out, void *stream, ssa_run **run_out);

/*
 * ssa_backward -- straight-through gradient of a recorded forward (Eqs. 3, 5, 7; the
 * reparametrised waiting time of Section 3.1; the adjoint recursion of Figure 1), walking each
 * trajectory backwards and regenerating the same Gumbel noise from Philox.
 *   dl_dobs        device float, dL/dobs of trajectory i at dl_dobs + i * dl_traj_stride, laid
 *                  out [n_samples][n_obs]. dl_traj_stride = n_samples * n_obs for a full
 *                  [n_traj][n_samples][n_obs] array, or 0 when every trajectory has the same
 *                  upstream gradient (a loss on ensemble means, Section 3.5).
 *   temperature    T > 0 (Eq. 3); for a soft forward (SSA_SELECT_SOFT) the forward's T.
 *   dl_dlog_rates  device float [P], overwritten with dL/dtheta summed over trajectories
 *                  (deterministic reduction order).
 * Trajectories whose status is not OK/ABSORBED/STEP_CAP contribute nothing. Callable any number
 * of times on one run (e.g. several temperatures). SSA_ERR_STATE if the run was not recorded.
 */
ssa_status ssa_backward(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride,
                        float temperature, float *dl_dlog_rates, void *stream);

/*
 * ssa_backward_multi -- the straight-through gradient of one recorded forward at several temperatures
 * (Eq. 3's T; e.g. T in {0.1, 0.5, 1.0}), each what ssa_backward gives at that T (to binary32 rounding
 * where one walk serves several temperatures). The reverse
 * walk, the regenerated noise, the propensities and the keys do not depend on T: on the
 * network-specialised kernels (ssa_run_variant = 2, Gumbel-max forward, HOLD or LINEAR readout) one walk
 * serves up to three temperatures at once, each with its own lambda, mu and partial sums; otherwise,
 * and for the remainder, one walk per temperature.
 *   temperatures   host float [n_temps], each > 0; n_temps >= 1.
 *   dl_dlog_rates  device float [n_temps][P], overwritten; row t for temperatures[t].
 *   Other arguments and errors as ssa_backward.
 */
ssa_status ssa_backward_multi(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride,
                              const float *temperatures, int32_t n_temps, float *dl_dlog_rates,
                              void *stream);

/*
 * ssa_backward_wide -- the same straight-through gradient as ssa_backward (same equations, same walk,
 * same noise) for trajectories whose adjoint leaves the binary32 range: over ~1e6 draws the
 * recursion of Figure 1 can grow dL/dX geometrically (on the activator-repressor oscillator of
 * Section 4.2 the binary64 gradient of one trajectory reaches ~1e73 at t = 400). Each trajectory
 * carries its binary32 accumulators (lambda, mu, dL/dlog a_j) times 2^sc with its own integer
 * exponent sc, renormalised by a power of two at every checkpoint once they exceed 2^32 (exact), and
 * the per-trajectory results are summed in binary64.
 *   dl_dlog_rates  device double [P], overwritten (deterministic reduction order).
 *   Other arguments as ssa_backward. A trajectory whose accumulators overflow within one checkpoint
 *   interval makes the result inf or NaN.
 * Runs on recorded Gumbel-max forwards with the HOLD or LINEAR readout on the network-specialised
 * kernels (ssa_run_variant = 2); SSA_ERR_UNSUPPORTED otherwise.
 */
ssa_status ssa_backward_wide(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride,
                             float temperature, double *dl_dlog_rates, void *stream);

/*
 * ssa_run_status -- synchronises `stream`, counts the per-trajectory status codes of the run into
 * host counts[SSA_TRAJ_N_CODES] and returns the number of backward consistency failures (the
 * recomputed Gumbel-max choice or a checkpoint disagreeing with the log) in *host_bwd_mismatch
 * (may be NULL; counted by the last ssa_backward).
 */
ssa_status ssa_run_status(const ssa_run *run, int64_t *host_counts, int64_t *host_bwd_mismatch,
                          void *stream);

/*
 * ssa_run_events -- test hook: unpack the recorded event log into device int32
 * [n_traj][stride], -1 after each trajectory's last draw (stride >= the longest trajectory).
 */
ssa_status ssa_run_events(const ssa_run *run, int32_t *events_out, int64_t stride, void *stream);

/*
 * ssa_run_brackets -- test hook: the recorded sample brackets of a recorded forward, as device
 * int32 [n_traj][n_samples]: the index k of the state X_k with t_k <= t_s < t_{k+1}.
 */
ssa_status ssa_run_brackets(const ssa_run *run, int32_t *brackets_out, void *stream);

void ssa_destroy_run(ssa_run *run);

/* ssa_run_variant -- the kernels a run used: 1 generic thread per trajectory, 2 thread per trajectory
 * compiled for the network, 32 warp per trajectory (0 for NULL). */
int32_t ssa_run_variant(const ssa_run *run);

/*
 * ssa_network_specialize -- compile (once per process and network) and load the kernels specialised
 * to this network, so that the first forward does not pay for it; *host_ok = 1 if they are
 * available, else 0 with the reason in ssa_last_error() (network above the limits, or the run-time
 * compiler failed). Returns SSA_OK unless an argument is NULL. No counterpart in the paper.
 */
ssa_status ssa_network_specialize(ssa_network *net, int32_t *host_ok);

/*
 * Gene-regulatory-network classifier (Section 4.3, Figure 4A): n_in clamped input counts x (the
 * pixels, round(255 p)), n_hid hidden and n_out output gene products starting from zero. Reaction
 * j < n_dyn = n_hid + n_out produces dynamic species j, reaction n_dyn + s degrades species s:
 *   production of hidden i: k_max sigma(E1_i), E1 = W1 x + b1   (one tensor-core contraction per image)
 *   production of output o: k_max sigma(E2_o), E2 = W2 h + b2   (kept exactly in integer fixed point)
 *   degradation of s:       exp(log_d_s) X_s
 * Trajectory i belongs to image i / traj_per_img. Readout: HOLD of the n_out outputs.
 * Limits: n_in <= 1040 (exact tensor-core accumulation of 6-bit limbs times 8-bit counts), counts
 * x in [0, 256], 2 (n_hid + n_out) <= 65535.
 */
typedef struct ssa_grn ssa_grn;
ssa_status ssa_grn_create(int32_t n_in, int32_t n_hid, int32_t n_out, float k_max, ssa_grn **out);
void ssa_grn_destroy(ssa_grn *g);
size_t ssa_grn_workspace_bytes(const ssa_grn *g, int64_t n_img, int64_t traj_per_img, int32_t n_samples,
                               const ssa_fwd_opts *opts);
/*
 * ssa_grn_forward -- E1 for every image on the tcgen05 tensor cores, then the exact SSA with the
 * Gumbel-max choice, one warp per trajectory.
 *   W1 device bf16 [n_hid][n_in], b1 device float [n_hid], W2 device bf16 [n_out][n_hid],
 *   b2 device float [n_out], log_d device float [n_hid + n_out]; x_img device int32 [n_img][n_in].
 *   opts->readout must be SSA_READOUT_HOLD. obs_out device int32 [n_img * traj_per_img][S][n_out].
 *   The weights, b2 and x_img must stay alive until the backward.
 *   opts->selector SSA_SELECT_SOFT (temperature > 0): the soft forward of Eq. 4 (the first training
 *   phase of Section 3.5), relaxed counts; obs_out then holds float values. Recorded, it keeps every
 *   count every 8 steps (opts->ckpt_interval, still checked to be 0 or a positive multiple of 8, does
 *   not apply) and ssa_grn_backward returns the exact gradient of that relaxed model. The soft path
 *   holds W2 (n_out * n_hid floats) in shared memory: SSA_ERR_UNSUPPORTED when it does not fit.
 */
ssa_status ssa_grn_forward(const ssa_grn *g, const uint16_t *W1, const float *b1, const uint16_t *W2,
                           const float *b2, const float *log_d, int64_t n_img, int64_t traj_per_img,
                           int64_t traj_offset, const int32_t *x_img, double t_end,
                           const double *sample_times, int32_t n_samples, uint64_t seed,
                           const ssa_fwd_opts *opts, void *workspace, size_t workspace_bytes,
                           int32_t *obs_out, int32_t *draws_out, int32_t *status_out, void *stream,
                           ssa_run **run_out);
/*
 * ssa_grn_backward -- the straight-through gradient (Eqs. 3, 5, 7) of a recorded GRN forward:
 * dW1 [n_hid][n_in] (tensor cores), db1 [n_hid], dW2 [n_out][n_hid], db2 [n_out],
 * dlog_d [n_hid + n_out], all device float, overwritten; dl_dobs as in ssa_backward. For a soft
 * forward, temperature must equal the forward's (SSA_ERR_INVALID_ARG otherwise).
 */
ssa_status ssa_grn_backward(ssa_run *run, const float *dl_dobs, int64_t dl_traj_stride,
                            float temperature, float *dW1, float *db1, float *dW2, float *db2,
                            float *dlog_d, void *stream);
/*
 * ssa_grn_activations -- test hook: E1 [n_img][n_hid] (device float) of a GRN run, and, if
 * host_flags is given (synchronising), host_flags[0] = inexact-input bits (1: a W1 value below the
 * 48-bit limb grid, 2: W2 outside the fixed-point range, 4: a count outside [0, 256]) and
 * host_flags[1] = tensor-core timeout.
 */
ssa_status ssa_grn_activations(const ssa_run *run, float *E1_out, int32_t *host_flags, void *stream);

/*
 * ssa_ensemble_mean -- the ensemble average that the paper's losses compare (Sections 3.5 and
 * 4.1: MSE between simulated and target ensemble-averaged trajectories): the mean over
 * trajectories of obs [n_traj][row_len] (device; int32 when obs_is_int, else float) into device
 * float [row_len]. Column sums run over fixed chunks of 256 trajectories, then over chunks, in a
 * fixed order, so the result is bitwise reproducible.
 *   workspace: device, >= ssa_ensemble_mean_workspace_bytes(n_traj, row_len).
 *   Any n_traj: the chunks are spread over at most 65,535 blocks in y.
 */
size_t ssa_ensemble_mean_workspace_bytes(int64_t n_traj, int64_t row_len);
ssa_status ssa_ensemble_mean(const void *obs, int32_t obs_is_int, int64_t n_traj, int64_t row_len,
                             void *workspace, size_t workspace_bytes, float *mean_out, void *stream);

/*
 * ssa_ensemble_mean_static -- the same mean as ssa_ensemble_mean, for callers that cannot allocate
 * device memory when they call (recording into a CUDA graph, where cudaMalloc is not allowed during
 * stream capture; real-time loops that forbid allocator calls; libraries with no access to the
 * application's allocator). The paper has no counterpart: this is an interface convenience.
 *   It allocates nothing: the column partial sums live in a fixed device array of 1,048,576 floats
 *   (4 MiB) that the library defines and every GPU that loads the library keeps until the process
 *   exits. ceil(n_traj / 256) * row_len must not exceed 1,048,576; larger inputs are rejected with
 *   SSA_ERR_UNSUPPORTED (use ssa_ensemble_mean with a workspace instead).
 *   The first call on a device looks up that device's address of the array
 *   (cudaGetSymbolAddress); make that first call before any stream capture on the device (a first
 *   call on a capturing stream returns SSA_ERR_UNSUPPORTED). The address is kept per device index
 *   for the life of the process: do not use this entry point across a cudaDeviceReset.
 *   All calls share the one array: calls that may run at the same time on the GPU (different
 *   streams without ordering between them) race and corrupt each other's result. Each call writes
 *   every scratch entry it reads, so no clearing is needed between calls.
 *   obs device [n_traj][row_len] (int32 when obs_is_int, else float); mean_out device float
 *   [row_len].
 */
ssa_status ssa_ensemble_mean_static(const void *obs, int32_t obs_is_int, int64_t n_traj,
                                    int64_t row_len, float *mean_out, void *stream);

/*
 * ssa_philox_uniforms -- test hook: out[r][q] = u_q of step step[r] of trajectory traj[r]
 * (device uint64 arrays [n], device float out [n][n_words]).
 */
ssa_status ssa_philox_uniforms(uint64_t seed, const uint64_t *traj, const uint64_t *step,
                               int64_t n, int32_t n_words, float *out, void *stream);

/*
 * ssa_bf16_gemm -- D[m][n] = sum_k A[m][k] B[n][k] (+ bias[n]) on the tcgen05 tensor cores, binary32
 * accumulation in tensor memory. The GRN classifier's dense contraction (Section 4.3, Figure 4A:
 * activation energy E = b + sum w x) is this product; the entry point exposes it for tests and users.
 *   A device bf16 [M][lda], B device bf16 [N][ldb] (K-major rows; lda, ldb multiples of 8 and
 *   16-byte aligned bases), D device float [M][ldd], bias device float [N] or NULL.
 *   work, work_words: device binary64 scratch (16-byte aligned) of at least
 *   ssa_bf16_gemm_work_words(M, N, K) words, owned by the caller, or NULL / 0. With it, a product
 *   whose 128 x 256 output tiles fill few of the SMs splits K across CTAs: each split's binary32
 *   tensor-memory sum is stored in binary64, a second kernel adds the splits in a fixed order and the
 *   bias and rounds once to binary32 (deterministic). Without it, one CTA per tile takes all of K.
 *   K = 0 writes D = bias (or 0).
 *   err_flag device int32, set nonzero by the kernel if a bounded wait timed out.
 * Errors: SSA_ERR_INVALID_ARG (sizes, NULL operands, alignment), SSA_ERR_WORKSPACE (work too small).
 */
ssa_status ssa_bf16_gemm(const uint16_t *A, const uint16_t *B, int32_t M, int32_t N, int32_t K,
                         int32_t lda, int32_t ldb, const float *bias, float *D, int32_t ldd,
                         double *work, int64_t work_words, int32_t *err_flag, void *stream);

/* ssa_bf16_gemm_work_words -- binary64 words of the work buffer ssa_bf16_gemm splits K into for this
 * shape (0: it would not split). Host only. */
int64_t ssa_bf16_gemm_work_words(int32_t M, int32_t N, int32_t K);

/*
 * ssa_exp_variates -- test hook: out[i] = -ln u(words[i]) with u(x) = ((x >> 9) + 1/2) 2^-23, the
 * exponential variate every kernel draws from a Philox word (device uint32 words [n], device float
 * out [n]), with the logarithm the kernels use (within one unit in the last place).
 */
ssa_status ssa_exp_variates(const uint32_t *words, int64_t n, float *out, void *stream);

/*
 * ssa_pipe_rates -- measurement support (no counterpart in the paper): throughput of the
 * instruction classes an SSA step is made of on the current GPU, as operations per SM per clock at
 * the device's maximum SM clock, written to host_rates[5] = {binary32 FMA, binary64 add, the
 * exponential variate -ln u the kernels use (an accurate binary32 logarithm), 32-bit integer multiply
 * (high and low), lg2.approx}. Also returns that clock (MHz) and the SM
 * count. Synchronous; allocates and frees a small device buffer.
 */
ssa_status ssa_pipe_rates(double *host_rates, double *host_sm_clock_mhz, int32_t *host_sm_count);

/*
 * Batch of networks -- many reaction networks of different sizes, each with its own parameters,
 * initial state, sample grid, observables and trajectory count, simulated and differentiated
 * together: one persistent forward launch and one persistent adjoint launch for the whole batch
 * (Sections 2-3: each network runs exactly the computation of ssa_forward(record) followed by
 * ssa_backward). No counterpart in the paper, which trains one network at a time; it exists for
 * workloads of many small networks that would each underfill the GPU.
 *
 * ssa_batch_item fields (all device pointers stay owned by the caller and must outlive the batch):
 *   net              network handle from ssa_create_network.
 *   log_rates        device float [net P]: theta, k_j = exp(theta[rate_index[j]]).
 *   x0               device int32 [net N], shared by the item's trajectories.
 *   n_traj >= 0, seed, traj_offset >= 0: trajectory i of the item draws the Philox stream of global
 *                    trajectory traj_offset + i under seed, as in ssa_forward.
 *   t_end, sample_times device double [n_samples], obs_species device int32 [n_obs] (n_obs <= 64),
 *   max_steps, ckpt_interval (0: choose; else a multiple of 8), threads_per_traj (0: choose, 1, 32;
 *                    1 needs N <= 16 and M <= 16): as ssa_fwd_opts.
 *   obs_out          device [n_traj][n_samples][n_obs], int32 (HOLD) or float (LINEAR, BIN; BIN:
 *                    n_obs <= SSA_BIN_MAX_OBS and the bin-edge rule of SSA_READOUT_BIN).
 *   dl_dobs, dl_traj_stride: upstream gradient as in ssa_backward.
 *   dl_dlog_rates    device float [net P], overwritten with the item's dL/dtheta.
 */
typedef struct ssa_batch ssa_batch;

typedef struct ssa_batch_item {
    const ssa_network *net;
    const float *log_rates;
    const int32_t *x0;
    int64_t n_traj;
    uint64_t seed;
    int64_t traj_offset;
    double t_end;
    const double *sample_times;
    int32_t n_samples;
    int32_t n_obs;
    const int32_t *obs_species;
    int64_t max_steps;
    int32_t ckpt_interval;
    int32_t threads_per_traj;
    void *obs_out;
    const float *dl_dobs;
    int64_t dl_traj_stride;
    float *dl_dlog_rates;
} ssa_batch_item;

/*
 * ssa_batch_create -- validate and copy the item descriptors (host array [n_items]); readout and
 * temperature T > 0 apply to every item (readout SSA_READOUT_HOLD, _LINEAR or _BIN). Allocates host
 * memory only. Errors: SSA_ERR_INVALID_ARG, SSA_ERR_UNSUPPORTED (thread variant requested for a network
 * with N > 16 or M > 16; the bin readout with more than SSA_BIN_MAX_OBS observables in an item).
 */
ssa_status ssa_batch_create(const ssa_batch_item *items, int32_t n_items, int32_t readout,
                            float temperature, ssa_batch **out);
void ssa_batch_destroy(ssa_batch *batch);

/*
 * ssa_batch_set_plan -- override the variant (1 or 32), the checkpoint interval (multiple of 8) and
 * the expected draws per trajectory (> 0; used to order work longest first; <= 0 keeps the current
 * estimate) of one item. Invalidates the captured graph and the workspace layout.
 */
ssa_status ssa_batch_set_plan(ssa_batch *batch, int32_t item, int32_t threads_per_traj,
                              int32_t ckpt_interval, double est_draws);

/* ssa_batch_workspace_bytes -- device workspace ssa_batch_run needs under the current plan. */
/*
 * ssa_batch_set_soft -- soft = 1: every item runs the soft forward of Eq. 4 (Section 3.3, as
 * SSA_SELECT_SOFT) at the batch temperature, recorded, and the adjoint gives the exact gradient of that
 * relaxed model at the same temperature (the per-item dL/dlog k). Every item runs as warp units with a
 * float checkpoint every 8 steps (ckpt_interval and the autotuner's choices do not apply; the autotuner
 * returns without work); observables are float for every readout; there is no event log
 * (ssa_batch_item_events returns SSA_ERR_STATE). soft = 0 restores the Gumbel-max batch. Call before a
 * run: the next run rebuilds the plan and the workspace size changes (ssa_batch_workspace_bytes).
 * Errors: SSA_ERR_INVALID_ARG, SSA_ERR_UNSUPPORTED (an item asks for threads_per_traj = 1).
 */
ssa_status ssa_batch_set_soft(ssa_batch *batch, int32_t soft);

size_t ssa_batch_workspace_bytes(const ssa_batch *batch);

/*
 * ssa_batch_run -- rates, input checks, persistent forward, persistent adjoint, fixed-order
 * reduction of every item's partial sums and the map to dl_dlog_rates, enqueued on `stream`.
 * workspace: device, 256-byte aligned, >= ssa_batch_workspace_bytes; the first call with a given
 * workspace lays it out (copies the descriptors, synchronises the stream); later calls with the
 * same workspace only launch. use_graph != 0 captures the launch sequence into a CUDA graph on the
 * first call (stream must not be the legacy default stream) and replays it afterwards; the device
 * pointers named in the items are baked in, so their contents may change between calls but not
 * their addresses. Calls on one batch must not overlap. Results are identical with and without the
 * graph and do not depend on the order in which the GPU runs the work units.
 */
ssa_status ssa_batch_run(ssa_batch *batch, void *workspace, size_t workspace_bytes, int32_t use_graph,
                         void *stream);

/*
 * ssa_batch_item_outputs -- after ssa_batch_run: copy one item's draws and trajectory status codes
 * (device int32 [n_traj] each, either may be NULL) and, if host_bwd_mismatch is not NULL,
 * synchronise and return the item's count of adjoint replay disagreements (0 on a sound run).
 */
ssa_status ssa_batch_item_outputs(const ssa_batch *batch, int32_t item, int32_t *draws_out,
                                  int32_t *status_out, int64_t *host_bwd_mismatch, void *stream);

/*
 * ssa_batch_item_events, ssa_batch_item_brackets -- test hooks after ssa_batch_run, as
 * ssa_run_events and ssa_run_brackets for one item: device int32 [n_traj][stride] events (-1 after
 * the last draw) and device int32 [n_traj][n_samples] sample brackets.
 */
ssa_status ssa_batch_item_events(const ssa_batch *batch, int32_t item, int32_t *events_out,
                                 int64_t stride, void *stream);
ssa_status ssa_batch_item_brackets(const ssa_batch *batch, int32_t item, int32_t *brackets_out,
                                   void *stream);

/*
 * ssa_batch_autotune -- pilot-based plan (no counterpart in the paper). Items that may run either
 * variant (threads_per_traj = 0 and N, M <= 16) time min(pilot_traj, n_traj) trajectories through
 * ssa_forward(record) + ssa_backward under both and keep the faster. Then all items' pilots run
 * together as one pilot batch, and each item's cost estimate (used to order the work longest first)
 * becomes its pilot's mean draws (host_draws_out [n_items] receives them, may be NULL). Last, the
 * checkpoint interval of every item that did not fix one: the pilot batch is timed with K = c x
 * 16 N (rounded to a multiple of 8 in [8, 4096]) for c in {1/4, 1, 4} and the fastest c is kept (the
 * reverse walk rebuilds states exactly from the event log, so K sets only how often the state is
 * stored and checked). Allocates and
 * frees pilot buffers with cudaMalloc, synchronises `stream`, writes nothing the caller owns.
 * Invalidates the captured graph and the workspace layout; the workspace size may change (more units
 * for the warp variant).
 */
ssa_status ssa_batch_autotune(ssa_batch *batch, int64_t pilot_traj, void *stream,
                              double *host_draws_out);

/* ssa_batch_item_variant -- the item's planned variant: 1 (thread) or 32 (warp); 0 if invalid. */
int32_t ssa_batch_item_variant(const ssa_batch *batch, int32_t item);

/* ssa_batch_item_ckpt_interval -- the item's planned checkpoint interval K; 0 if invalid. */
int32_t ssa_batch_item_ckpt_interval(const ssa_batch *batch, int32_t item);

const char *ssa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SSA_H */
