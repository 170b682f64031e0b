/*
 * ssa_oracle.c -- plain, slow, FP64 CPU oracle of the exact Gillespie simulation with a
 * Gumbel-max reaction choice and of its Gumbel-Softmax straight-through gradient.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this file:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it. It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it follows (arXiv 2602.19775):
 *   - Section 2: mass-action propensities a_j(X; theta) (first order k X_i, hetero second
 *     order k X_i X_l, homodimer k X_i (X_i - 1)/2, zeroth order k), total rate a0 = sum_j a_j,
 *     waiting time tau = -ln(u)/a0, update X <- X + v_j.
 *   - Section 3.2 (the unnumbered Gumbel-max equation): j* = argmax_j [log a_j + G_j],
 *     G_j = -ln(-ln u_j).
 *   - Section 3.3, Eq. 3: soft sample y~_j = softmax_j((log a_j + G_j)/T) with the same G.
 *   - Section 3.4, Eqs. 5-7: y_ST = stopgrad(y - y~) + y~; forward applies v_{j*} (Eq. 6);
 *     the backward differentiates X_{k+1} = X_k + sum_j y~_j v_j (Eq. 7).
 *   - Section 3.1: the reparametrised waiting time, d tau/d theta = -(tau/a0) d a0/d theta.
 *   - Figure 1 caption: the adjoint recursion dL/dX_k = dL/dX_k|direct +
 *     (dX_ST(k+1)/dX_k)^T dL/dX_{k+1}, with the Gumbel draws held fixed.
 *   - Section 4.1: each trajectory is linearly interpolated onto a uniform time grid
 *     (LINEAR readout); the HOLD readout is the right-continuous path value X(t_s).
 *   - Section 3.3, Eq. 4 (the soft forward, selector 2): the state is real-valued and moves by the
 *     expected stoichiometry sum_j y~_j v_j of the soft sample, every step; its gradient is the exact
 *     gradient of that relaxed model, which the same adjoint computes along the soft path.
 *   - Section 4.4: the BIN readout averages the piecewise-constant path exactly over each bin,
 *     through its cumulative integral C(b) = int_0^b X(t) dt: obs_s = (C(b_s) - C(b_{s-1}))/
 *     (b_s - b_{s-1}). Reading: the bins are (b_{s-1}, b_s] with b_s = t_s and b_{-1} = 0 (the
 *     sample times are the bins' right edges), strictly increasing with t_0 > 0; the path holds
 *     its last state after it stops.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - Noise: counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). Key =
 *     (seed_lo, seed_hi); counter = (b, k, i_lo, i_hi) for trajectory i, step k and block b.
 *     Word q of the step's stream is q = 4b + w; u_0 drives tau and u_{1+j} drives reaction j.
 *     u = ((x >> 9) + 0.5) * 2^-23, which lies strictly inside (0,1) and is exact in binary32.
 *   - A reaction with a_j = 0 is masked out of the argmax and of the softmax (y~_j = 0 and no
 *     choice-path gradient); it still enters a0 and therefore the waiting-time gradient through
 *     the polynomial derivative d a_j/dX.
 *   - The draw that crosses t_end is made but not applied; with LINEAR readout it supplies
 *     X_{n+1} for samples after the last event.
 *   - a0 == 0: the state is absorbing; no further draw.
 *   - Parameters are log rates: k_j = exp(theta_{r(j)}), several reactions may share one.
 *   - Soft forward: a relaxed state can leave the integers; a mass-action factor h_j(X) that comes out
 *     negative there (X_i < 0, or 0 < X_i < 1 in a homodimer) is taken as 0, and so is its derivative.
 *     No range checks apply; the draw that crosses t_end still supplies the soft target X_{k+1} for the
 *     LINEAR readout.
 *
 * Everything is double precision; event counts are exact integers.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------------------- */
/* Network description (all host pointers, owned by the caller).                             */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    int32_t n_species;             /* N */
    int32_t n_reactions;           /* M */
    const int32_t *reactants;      /* [M][2]; species index or -1 for an empty slot */
    const int32_t *stoich_ptr;     /* [M+1]; CSR row pointer of the net change v_j */
    const int32_t *stoich_species; /* [nnz] */
    const int32_t *stoich_delta;   /* [nnz] */
    int32_t n_params;              /* P */
    const double *log_rates;       /* [P]: theta = log k */
    const int32_t *rate_index;     /* [M]: reaction j uses theta[rate_index[j]] */
} orc_network;

enum { ORC_HOLD = 0, ORC_LINEAR = 1, ORC_BIN = 2 };

/* per-trajectory status codes */
enum {
    ORC_OK = 0,           /* reached t_end (the crossing draw was made, not applied) */
    ORC_ABSORBED = 1,     /* a0 == 0 before t_end: the state holds to t_end           */
    ORC_STEP_CAP = 2,     /* max_steps draws were made and applied before t_end        */
    ORC_NEG_COUNT = 3,    /* an update would make a count negative; stopped before it  */
    ORC_OVERFLOW = 4,     /* an update would leave int32 range; stopped before it      */
    ORC_BAD_RATE = 5      /* a propensity was not finite                               */
};

/* ---------------------------------------------------------------------------------------- */
/* Philox4x32-10, from the published definition (Salmon et al., SC'11, Section 4):           */
/* ten rounds of two 32x32->64 multiplications with round keys bumped by the Weyl constants.  */
/* ---------------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* u = ((x >> 9) + 1/2) * 2^-23, strictly inside (0,1). */
static double orc_u01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Uniform number q of step k of trajectory i (q = 0 drives tau, q = 1 + j drives reaction j). */
static double orc_uniform(uint64_t seed, uint64_t traj, uint64_t step, int64_t q)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)(q / 4), (uint32_t)step, (uint32_t)traj, (uint32_t)(traj >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return orc_u01(out[q % 4]);
}

/* Exported for tests: n words of block b of step k of trajectory i, flattened. */
void orc_uniforms(uint64_t seed, uint64_t traj, uint64_t step, int64_t n_words, double *out)
{
    for (int64_t q = 0; q < n_words; ++q) out[q] = orc_uniform(seed, traj, step, q);
}

void orc_philox_blocks(uint64_t seed, const uint32_t *ctrs /*[n][4]*/, int64_t n, uint32_t *out /*[n][4]*/)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctrs + 4 * i, key, out + 4 * i);
}

/* ---------------------------------------------------------------------------------------- */
/* Mass-action propensities (Section 2) and their derivatives with respect to the state.     */
/* ---------------------------------------------------------------------------------------- */

/* combinatorial factor h_j(X): 1, X_i, X_i X_l, or X_i (X_i - 1) / 2 */
static double orc_h(const orc_network *net, int j, const double *X)
{
    int r1 = net->reactants[2 * j], r2 = net->reactants[2 * j + 1];
    if (r1 < 0 && r2 < 0) return 1.0;
    if (r1 < 0) { r1 = r2; r2 = -1; }
    if (r2 < 0) return X[r1];
    if (r1 == r2) return X[r1] * (X[r1] - 1.0) / 2.0;
    return X[r1] * X[r2];
}

/* add c * d h_j / d X to grad[N] */
static void orc_add_dh(const orc_network *net, int j, const double *X, double c, double *grad)
{
    int r1 = net->reactants[2 * j], r2 = net->reactants[2 * j + 1];
    if (r1 < 0 && r2 < 0) return;
    if (r1 < 0) { r1 = r2; r2 = -1; }
    if (r2 < 0) { grad[r1] += c; return; }
    if (r1 == r2) { grad[r1] += c * (2.0 * X[r1] - 1.0) / 2.0; return; }
    grad[r1] += c * X[r2];
    grad[r2] += c * X[r1];
}

/* ---------------------------------------------------------------------------------------- */
/* One trajectory: the stored path.                                                           */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    int64_t n_draws;   /* number of reaction draws, including a crossing draw */
    int64_t n_states;  /* number of states X_0..X_{n_states-1} visited */
    int32_t status;
    int32_t crossed;   /* 1 if the last draw crossed t_end (made, not applied) */
    /* growable arrays */
    int64_t cap;
    double *X;         /* [cap+1][N] state before draw k (X_0 ... ) */
    double *t;         /* [cap+1] t_k */
    double *tau;       /* [cap] tau_k */
    int32_t *j;        /* [cap] j_k */
    double *margin;    /* [cap] (s1 - s2)/s1 in the a/E form; 1 if one reaction is active */
} orc_path;

static int orc_path_grow(orc_path *p, int N, int64_t need)
{
    if (need <= p->cap) return 0;
    int64_t nc = p->cap ? p->cap : 64;
    while (nc < need) nc *= 2;
    double *X = (double *)realloc(p->X, (size_t)(nc + 1) * N * sizeof(double));
    double *t = (double *)realloc(p->t, (size_t)(nc + 1) * sizeof(double));
    double *tau = (double *)realloc(p->tau, (size_t)nc * sizeof(double));
    int32_t *jj = (int32_t *)realloc(p->j, (size_t)nc * sizeof(int32_t));
    double *mg = (double *)realloc(p->margin, (size_t)nc * sizeof(double));
    if (X) p->X = X;
    if (t) p->t = t;
    if (tau) p->tau = tau;
    if (jj) p->j = jj;
    if (mg) p->margin = mg;
    if (!X || !t || !tau || !jj || !mg) return -1;
    p->cap = nc;
    return 0;
}

static void orc_path_free(orc_path *p)
{
    free(p->X); free(p->t); free(p->tau); free(p->j); free(p->margin);
    memset(p, 0, sizeof(*p));
}

typedef struct {
    const orc_network *net;
    double t_end;
    int64_t max_steps;
    uint64_t seed;
    int32_t selector; /* 0: Gumbel-max (Section 3.2); 1: the standard direct method (Section 2);
                         2: the soft forward (Eq. 4) */
    double temperature; /* T of the soft forward */
} orc_sim_cfg;

/* h_j on the state of the path: the relaxed state of the soft forward clips a negative factor to 0 */
static double orc_h_path(const orc_network *net, int j, const double *X, int soft)
{
    const double h = orc_h(net, j, X);
    return (soft && h < 0.0) ? 0.0 : h;
}

/*
 * Simulate trajectory `traj` from x0 (Section 2 + the Gumbel-max choice of Section 3.2).
 * Returns 0, or -1 on allocation failure.
 */
static int orc_simulate_one(const orc_sim_cfg *cfg, uint64_t traj, const int32_t *x0, orc_path *p)
{
    const orc_network *net = cfg->net;
    const int N = net->n_species, M = net->n_reactions;
    double *a = (double *)malloc((size_t)(M > 0 ? M : 1) * sizeof(double));
    double *ys = (double *)malloc((size_t)(M > 0 ? M : 1) * sizeof(double)); /* soft sample */
    if (!a || !ys) { free(a); free(ys); return -1; }
    p->n_draws = 0;
    p->crossed = 0;
    p->status = ORC_OK;
    if (orc_path_grow(p, N, 1)) { free(a); free(ys); return -1; }
    for (int i = 0; i < N; ++i) p->X[i] = (double)x0[i];
    p->t[0] = 0.0;
    int64_t k = 0;
    for (;;) {
        double *X = p->X + (size_t)k * N;
        if (k >= cfg->max_steps) { p->status = ORC_STEP_CAP; break; }
        /* propensities, total rate (Section 2) */
        double a0 = 0.0;
        int bad = 0;
        for (int j = 0; j < M; ++j) {
            double kj = exp(net->log_rates[net->rate_index[j]]);
            a[j] = kj * orc_h_path(net, j, X, cfg->selector == 2);
            if (!isfinite(a[j]) || a[j] < 0.0) bad = 1;
            a0 += a[j];
        }
        if (bad) { p->status = ORC_BAD_RATE; break; }
        if (a0 == 0.0) { p->status = ORC_ABSORBED; break; }
        if (orc_path_grow(p, N, k + 2)) { free(a); free(ys); return -1; }
        X = p->X + (size_t)k * N;
        /* waiting time by inverse transform (Section 2) */
        double u0 = orc_uniform(cfg->seed, traj, (uint64_t)k, 0);
        double tau = -log(u0) / a0;
        int best = -1;
        if (cfg->selector == 2) {
            /* soft sample (Eq. 3) over the active reactions; best = its largest weight (the hard choice) */
            double zmax = -INFINITY, s2 = -INFINITY, Z = 0.0;
            for (int j = 0; j < M; ++j) {
                ys[j] = -INFINITY;
                if (!(a[j] > 0.0)) continue;
                double u = orc_uniform(cfg->seed, traj, (uint64_t)k, 1 + j);
                double z = (log(a[j]) - log(-log(u))) / cfg->temperature;
                ys[j] = z;
                if (z > zmax) { s2 = zmax; zmax = z; best = j; }
                else if (z > s2) { s2 = z; }
            }
            for (int j = 0; j < M; ++j) {
                ys[j] = ys[j] == -INFINITY ? 0.0 : exp(ys[j] - zmax);
                Z += ys[j];
            }
            for (int j = 0; j < M; ++j) ys[j] /= Z;
            p->margin[k] = (s2 == -INFINITY) ? 1.0 : -expm1((s2 - zmax) * cfg->temperature);
        } else if (cfg->selector == 0) {
            /* Gumbel-max choice over the active reactions (Section 3.2); ties to the lowest j */
            double s1 = -INFINITY, s2 = -INFINITY;
            for (int j = 0; j < M; ++j) {
                if (!(a[j] > 0.0)) continue;
                double u = orc_uniform(cfg->seed, traj, (uint64_t)k, 1 + j);
                double G = -log(-log(u));
                double key = log(a[j]) + G;
                if (key > s1) { s2 = s1; s1 = key; best = j; }
                else if (key > s2) { s2 = key; }
            }
            p->margin[k] = (s2 == -INFINITY) ? 1.0 : -expm1(s2 - s1);
        } else {
            /* direct method (Section 2): the first reaction whose cumulative propensity exceeds u_1 a0;
               the margin is the distance of u_1 a0 to the nearest cumulative boundary, relative to a0 */
            double r = orc_uniform(cfg->seed, traj, (uint64_t)k, 1) * a0, cum = 0.0, lo = 0.0;
            for (int j = 0; j < M; ++j) {
                if (!(a[j] > 0.0)) continue;
                best = j;
                lo = cum;
                cum += a[j];
                if (cum > r) break;
            }
            const double d_lo = best >= 0 && lo > 0.0 ? r - lo : INFINITY;
            const double d_hi = cum > r && cum < a0 ? cum - r : INFINITY;
            const double d = d_lo < d_hi ? d_lo : d_hi;
            p->margin[k] = isfinite(d) ? d / a0 : 1.0;
        }
        p->j[k] = best;
        p->tau[k] = tau;
        double t_next = p->t[k] + tau;
        p->t[k + 1] = t_next;
        p->n_draws = k + 1;
        double *Xn = p->X + (size_t)(k + 1) * N;
        if (cfg->selector == 2) {
            /* relaxed update (Eq. 4): X_{k+1} = X_k + sum_j y~_j v_j; also written for the crossing draw,
               whose X_{k+1} is not a visited state but is what LINEAR interpolates towards */
            for (int i = 0; i < N; ++i) Xn[i] = X[i];
            for (int j = 0; j < M; ++j)
                for (int e = net->stoich_ptr[j]; e < net->stoich_ptr[j + 1]; ++e)
                    Xn[net->stoich_species[e]] += ys[j] * (double)net->stoich_delta[e];
            if (t_next > cfg->t_end) { p->crossed = 1; p->status = ORC_OK; break; }
            int bad_x = 0;
            for (int i = 0; i < N; ++i) bad_x |= !isfinite(Xn[i]);
            if (bad_x) { p->status = ORC_BAD_RATE; break; }
            ++k;
            continue;
        }
        if (t_next > cfg->t_end) { p->crossed = 1; p->status = ORC_OK; break; }
        /* integer update (Eq. 6), with range checks */
        int stop = 0;
        for (int i = 0; i < N; ++i) Xn[i] = X[i];
        for (int e = net->stoich_ptr[best]; e < net->stoich_ptr[best + 1]; ++e) {
            int s = net->stoich_species[e];
            Xn[s] += (double)net->stoich_delta[e];
        }
        for (int i = 0; i < N; ++i) {
            if (Xn[i] < 0.0) { p->status = ORC_NEG_COUNT; stop = 1; }
            else if (Xn[i] > 2147483647.0) { p->status = ORC_OVERFLOW; stop = 1; }
        }
        if (stop) {
            /* the draw was made but not applied: the trajectory stops at X_k */
            break;
        }
        ++k;
    }
    p->n_states = k + 1;
    free(a);
    free(ys);
    return 0;
}

/* Bracket of sample time ts: the largest k with t_k <= ts (right-continuous path). */
static int64_t orc_bracket(const orc_path *p, double ts)
{
    int64_t k = 0;
    while (k + 1 < p->n_states && p->t[k + 1] <= ts) ++k;
    return k;
}

/* Does state k have a draw that the LINEAR readout may interpolate towards? */
static int orc_has_next(const orc_path *p, int64_t k)
{
    /* a draw exists at k if k < n_draws; it was applied if k + 1 < n_states, or it is the
       crossing draw; a draw rejected by a range check is not interpolated */
    if (k >= p->n_draws) return 0;
    if (k + 1 < p->n_states) return 1;
    return p->crossed;
}

/* Cumulative integral C(b) = int_0^b X_sp(t) dt of the right-continuous step path (Section 4.4):
   the whole intervals [t_i, t_{i+1}) before the bracket of b, then the part [t_k, b]. */
static double orc_cumulative(const orc_path *p, int N, int sp, double b)
{
    const int64_t kb = orc_bracket(p, b);
    double c = 0.0;
    for (int64_t i = 0; i < kb; ++i) c += p->X[(size_t)i * N + sp] * (p->t[i + 1] - p->t[i]);
    return c + p->X[(size_t)kb * N + sp] * (b - p->t[kb]);
}

/* Readout (Section 4.1): HOLD = X(t_s); LINEAR = linear interpolation on the event grid;
   (Section 4.4) BIN = exact average over the bin (t_{s-1}, t_s], t_{-1} = 0. */
static void orc_readout(const orc_network *net, const orc_path *p, const double *ts, int S,
                        const int32_t *obs_species, int n_obs, int readout, int soft, double *obs /*[S][n_obs]*/)
{
    const int N = net->n_species;
    if (readout == ORC_BIN) {
        for (int s = 0; s < S; ++s) {
            const double lo = s > 0 ? ts[s - 1] : 0.0;
            for (int o = 0; o < n_obs; ++o) {
                const int sp = obs_species[o];
                obs[(size_t)s * n_obs + o] =
                    (orc_cumulative(p, N, sp, ts[s]) - orc_cumulative(p, N, sp, lo)) / (ts[s] - lo);
            }
        }
        return;
    }
    for (int s = 0; s < S; ++s) {
        int64_t k = orc_bracket(p, ts[s]);
        const double *X = p->X + (size_t)k * N;
        for (int o = 0; o < n_obs; ++o) {
            int sp = obs_species[o];
            double v = X[sp];
            if (readout == ORC_LINEAR && orc_has_next(p, k)) {
                double alpha = (ts[s] - p->t[k]) / p->tau[k];
                double dv = 0.0;
                int j = p->j[k];
                if (soft) dv = p->X[(size_t)(k + 1) * N + sp] - X[sp]; /* the soft step (Eq. 4) */
                else
                    for (int e = net->stoich_ptr[j]; e < net->stoich_ptr[j + 1]; ++e)
                        if (net->stoich_species[e] == sp) dv += (double)net->stoich_delta[e];
                v = X[sp] + alpha * dv;
            }
            obs[(size_t)s * n_obs + o] = v;
        }
    }
}

/*
 * Straight-through adjoint of one trajectory (Eqs. 3, 5, 7; Section 3.1; Figure 1 recursion).
 * dL_dobs: [S][n_obs] for this trajectory. Adds dL/dtheta into dtheta[P].
 */
static int orc_adjoint_one(const orc_sim_cfg *cfg, uint64_t traj, const orc_path *p,
                           const double *ts, int S, const int32_t *obs_species, int n_obs,
                           int readout, const double *dL_dobs, double T, double *dtheta)
{
    const orc_network *net = cfg->net;
    const int N = net->n_species, M = net->n_reactions;
    const int soft = cfg->selector == 2;
    double *lam = (double *)calloc((size_t)N, sizeof(double));     /* dL/dX_{k+1} */
    double *lam_new = (double *)calloc((size_t)N, sizeof(double));
    double *dXdir = (double *)calloc((size_t)N, sizeof(double));
    double *gbar = (double *)calloc((size_t)N, sizeof(double));
    double *a = (double *)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
    double *z = (double *)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
    double *y = (double *)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
    double *w = (double *)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
    int64_t *kb = (int64_t *)calloc((size_t)(S > 0 ? S : 1), sizeof(int64_t));
    if (!lam || !lam_new || !dXdir || !gbar || !a || !z || !y || !w || !kb) {
        free(lam); free(lam_new); free(dXdir); free(gbar); free(a); free(z); free(y); free(w); free(kb);
        return -1;
    }
    for (int s = 0; s < S; ++s) kb[s] = orc_bracket(p, ts[s]);

    double mu = 0.0; /* dL/dt_{k+1} */
    for (int64_t k = p->n_states - 1; k >= 0; --k) {
        const double *X = p->X + (size_t)k * N;
        const int draw = orc_has_next(p, k);
        double dt_dir = 0.0, dtau_dir = 0.0;
        for (int i = 0; i < N; ++i) dXdir[i] = 0.0;
        /* BIN: obs_e = (C(b_e) - C(b_{e-1}))/D_e, so dL/dC(b_e) = g_e - g_{e+1} with g_e = dL/dobs_e / D_e.
           C(b) = sum_{i<kb} X_i (t_{i+1} - t_i) + X_kb (b - t_kb) gives dC/dX_k = t_{k+1} - t_k (k < kb) or
           b - t_k (k = kb), and dC/dt_k = X_{k-1} - X_k for 1 <= k <= kb (t_k ends the previous interval
           and starts this one); b_{-1} = 0 is fixed. */
        if (readout == ORC_BIN) {
            for (int e = 0; e < S; ++e) {
                if (kb[e] < k) continue;
                const double lo = e > 0 ? ts[e - 1] : 0.0;
                for (int o = 0; o < n_obs; ++o) {
                    const int sp = obs_species[o];
                    const double g_e = dL_dobs[(size_t)e * n_obs + o] / (ts[e] - lo);
                    const double g_n = e + 1 < S ? dL_dobs[(size_t)(e + 1) * n_obs + o] / (ts[e + 1] - ts[e]) : 0.0;
                    const double gC = g_e - g_n;
                    dXdir[sp] += gC * (kb[e] > k ? p->t[k + 1] - p->t[k] : ts[e] - p->t[k]);
                    if (k >= 1) dt_dir += gC * (p->X[(size_t)(k - 1) * N + sp] - X[sp]);
                }
            }
        }
        /* direct readout terms of the samples bracketed by state k (HOLD, LINEAR) */
        for (int s = 0; s < S && readout != ORC_BIN; ++s) {
            if (kb[s] != k) continue;
            for (int i = 0; i < N; ++i) gbar[i] = 0.0;
            for (int o = 0; o < n_obs; ++o) gbar[obs_species[o]] += dL_dobs[(size_t)s * n_obs + o];
            if (readout == ORC_LINEAR && draw) {
                /* obs = X_k + alpha (X_{k+1} - X_k), alpha = (t_s - t_k)/tau_k */
                double alpha = (ts[s] - p->t[k]) / p->tau[k];
                double c = 0.0; /* gbar . (X_{k+1} - X_k): gbar . v_{j_k}, or the soft step */
                int j = p->j[k];
                if (soft)
                    for (int i = 0; i < N; ++i) c += gbar[i] * (p->X[(size_t)(k + 1) * N + i] - X[i]);
                else
                    for (int e = net->stoich_ptr[j]; e < net->stoich_ptr[j + 1]; ++e)
                        c += gbar[net->stoich_species[e]] * (double)net->stoich_delta[e];
                for (int i = 0; i < N; ++i) {
                    lam[i] += alpha * gbar[i];          /* into X_{k+1} */
                    dXdir[i] += (1.0 - alpha) * gbar[i];
                }
                dt_dir += -c / p->tau[k];               /* d alpha/d t_k = -1/tau_k */
                dtau_dir += -alpha * c / p->tau[k];     /* d alpha/d tau_k = -alpha/tau_k */
            } else {
                for (int i = 0; i < N; ++i) dXdir[i] += gbar[i];
            }
        }
        for (int i = 0; i < N; ++i) lam_new[i] = lam[i] + dXdir[i];
        if (draw) {
            /* recompute the step's propensities and Gumbel perturbations (same noise) */
            double a0 = 0.0;
            for (int j = 0; j < M; ++j) {
                a[j] = exp(net->log_rates[net->rate_index[j]]) * orc_h_path(net, j, X, soft);
                a0 += a[j];
            }
            double tau = p->tau[k];
            double dtau = mu + dtau_dir;
            /* Eq. 3: soft sample over the active reactions */
            double zmax = -INFINITY;
            for (int j = 0; j < M; ++j) {
                if (a[j] > 0.0) {
                    double u = orc_uniform(cfg->seed, traj, (uint64_t)k, 1 + j);
                    z[j] = (log(a[j]) - log(-log(u))) / T;
                    if (z[j] > zmax) zmax = z[j];
                }
            }
            double Z = 0.0;
            for (int j = 0; j < M; ++j) { y[j] = (a[j] > 0.0) ? exp(z[j] - zmax) : 0.0; Z += y[j]; }
            for (int j = 0; j < M; ++j) y[j] /= Z;
            /* Eq. 7: dL/dy~_j = v_j . dL/dX_{k+1} */
            double wbar = 0.0;
            for (int j = 0; j < M; ++j) {
                w[j] = 0.0;
                for (int e = net->stoich_ptr[j]; e < net->stoich_ptr[j + 1]; ++e)
                    w[j] += (double)net->stoich_delta[e] * lam[net->stoich_species[e]];
                wbar += y[j] * w[j];
            }
            /* softmax backward: dL/dz_j = y_j (w_j - sum_i y_i w_i); dL/dlog a_j = that / T */
            /* waiting time: tau = E0/a0, so dL/da0 = -dtau * tau / a0 (Section 3.1) */
            double dLda0 = -dtau * tau / a0;
            for (int j = 0; j < M; ++j) {
                double choice = (a[j] > 0.0) ? y[j] * (w[j] - wbar) / T : 0.0;
                /* theta = log k: d log a_j / d theta = 1, d a_j / d theta = a_j */
                dtheta[net->rate_index[j]] += choice + dLda0 * a[j];
                /* state path: choice through d log a_j/dX = (dh/dX)/h; tau through d a_j/dX */
                if (a[j] > 0.0) {
                    double h = orc_h(net, j, X);
                    orc_add_dh(net, j, X, choice / h, lam_new);
                }
                double kj = exp(net->log_rates[net->rate_index[j]]);
                if (!soft || orc_h(net, j, X) >= 0.0) orc_add_dh(net, j, X, dLda0 * kj, lam_new);
            }
        }
        mu = mu + dt_dir; /* t_{k+1} = t_k + tau_k: mu becomes dL/dt_k */
        for (int i = 0; i < N; ++i) lam[i] = lam_new[i];
    }
    free(lam); free(lam_new); free(dXdir); free(gbar); free(a); free(z); free(y); free(w); free(kb);
    return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Batched driver with a thread pool over trajectories.                                       */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    const orc_network *net;
    int64_t n_traj;
    int64_t traj_offset;
    const int32_t *x0;
    int32_t x0_per_traj;
    double t_end;
    const double *ts;
    int32_t S;
    const int32_t *obs_species;
    int32_t n_obs;
    uint64_t seed;
    int32_t readout;
    int64_t max_steps;
    const double *dL_dobs;     /* [n_traj][S][n_obs] or NULL */
    double temperature;
    double *obs_out;           /* [n_traj][S][n_obs] or NULL */
    int64_t *draws_out;        /* [n_traj] or NULL */
    int32_t *status_out;       /* [n_traj] or NULL */
    double *dtheta_traj_out;   /* [n_traj][P] or NULL */
    int32_t *events_out;       /* [n_traj][ev_cap] or NULL (-1 padded) */
    double *margins_out;       /* [n_traj][ev_cap] or NULL */
    double *times_out;         /* [n_traj][ev_cap] t_{k+1} per draw, or NULL */
    int64_t ev_cap;
    int32_t *final_x_out;      /* [n_traj][N] or NULL: last visited state */
    int32_t selector;          /* 0: Gumbel-max, 1: direct method */
    /* work distribution */
    int32_t n_threads;
    int64_t next;              /* guarded by lock */
    pthread_mutex_t lock;
    int error;
} orc_job;

static void *orc_worker(void *arg)
{
    orc_job *job = (orc_job *)arg;
    const orc_network *net = job->net;
    const int N = net->n_species, P = net->n_params;
    orc_sim_cfg cfg = {net, job->t_end, job->max_steps, job->seed, job->selector, job->temperature};
    orc_path path;
    memset(&path, 0, sizeof(path));
    double *dth = (double *)calloc((size_t)(P > 0 ? P : 1), sizeof(double));
    double *obs = (double *)calloc((size_t)(job->S * job->n_obs > 0 ? job->S * job->n_obs : 1), sizeof(double));
    if (!dth || !obs) { free(dth); free(obs); pthread_mutex_lock(&job->lock); job->error = 1; pthread_mutex_unlock(&job->lock); return NULL; }
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t i = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (i >= job->n_traj) break;
        uint64_t traj = (uint64_t)(job->traj_offset + i);
        const int32_t *x0 = job->x0 + (job->x0_per_traj ? (size_t)i * N : 0);
        if (orc_simulate_one(&cfg, traj, x0, &path)) { job->error = 1; break; }
        orc_readout(net, &path, job->ts, job->S, job->obs_species, job->n_obs, job->readout, job->selector == 2, obs);
        if (job->obs_out)
            memcpy(job->obs_out + (size_t)i * job->S * job->n_obs, obs, (size_t)job->S * job->n_obs * sizeof(double));
        if (job->draws_out) job->draws_out[i] = path.n_draws;
        if (job->status_out) job->status_out[i] = path.status;
        if (job->final_x_out)
            for (int s = 0; s < N; ++s)
                job->final_x_out[(size_t)i * N + s] = (int32_t)path.X[(size_t)(path.n_states - 1) * N + s];
        if (job->events_out || job->margins_out || job->times_out) {
            for (int64_t q = 0; q < job->ev_cap; ++q) {
                int have = q < path.n_draws;
                if (job->events_out) job->events_out[(size_t)i * job->ev_cap + q] = have ? path.j[q] : -1;
                if (job->margins_out) job->margins_out[(size_t)i * job->ev_cap + q] = have ? path.margin[q] : NAN;
                if (job->times_out) job->times_out[(size_t)i * job->ev_cap + q] = have ? path.t[q + 1] : NAN;
            }
        }
        if (job->dL_dobs && job->dtheta_traj_out) {
            for (int r = 0; r < P; ++r) dth[r] = 0.0;
            if (orc_adjoint_one(&cfg, traj, &path, job->ts, job->S, job->obs_species, job->n_obs,
                                job->readout, job->dL_dobs + (size_t)i * job->S * job->n_obs,
                                job->temperature, dth)) { job->error = 1; break; }
            memcpy(job->dtheta_traj_out + (size_t)i * P, dth, (size_t)P * sizeof(double));
        }
    }
    orc_path_free(&path);
    free(dth);
    free(obs);
    return NULL;
}

/*
 * Simulate n_traj trajectories (global ids traj_offset + i) and, if dL_dobs is given, the
 * straight-through gradient of each one. Returns 0 on success, -1 on bad input or allocation
 * failure.
 */
int orc_run_sel(int32_t selector, const orc_network *net, int64_t n_traj, int64_t traj_offset,
                const int32_t *x0, int32_t x0_per_traj, double t_end,
                const double *ts, int32_t S, const int32_t *obs_species, int32_t n_obs,
                uint64_t seed, int32_t readout, int64_t max_steps,
                const double *dL_dobs, double temperature,
                double *obs_out, int64_t *draws_out, int32_t *status_out,
                double *dtheta_traj_out,
                int32_t *events_out, double *margins_out, double *times_out, int64_t ev_cap,
                int32_t *final_x_out, int32_t n_threads)
{
    if (!net || n_traj < 0 || S < 0 || n_obs < 0 || max_steps < 0) return -1;
    if (selector != 0 && selector != 1 && selector != 2) return -1;
    if (selector == 1 && dL_dobs) return -1;  /* the straight-through gradient is of the Gumbel-max choice */
    if (selector == 2 && !(temperature > 0.0)) return -1; /* the soft forward needs its T */
    if (net->n_species <= 0 || net->n_reactions < 0) return -1;
    if (readout != ORC_HOLD && readout != ORC_LINEAR && readout != ORC_BIN) return -1;
    for (int s = 0; s < S; ++s) {
        if (!(ts[s] >= 0.0 && ts[s] <= t_end)) return -1;
        if (s > 0 && ts[s] < ts[s - 1]) return -1;
        /* BIN: bins (t_{s-1}, t_s] of positive width, t_{-1} = 0 */
        if (readout == ORC_BIN && !(ts[s] > (s > 0 ? ts[s - 1] : 0.0))) return -1;
    }
    for (int o = 0; o < n_obs; ++o)
        if (obs_species[o] < 0 || obs_species[o] >= net->n_species) return -1;
    if (dL_dobs && !(temperature > 0.0)) return -1;
    orc_job job;
    memset(&job, 0, sizeof(job));
    job.net = net; job.n_traj = n_traj; job.traj_offset = traj_offset; job.x0 = x0;
    job.x0_per_traj = x0_per_traj; job.t_end = t_end; job.ts = ts; job.S = S;
    job.obs_species = obs_species; job.n_obs = n_obs; job.seed = seed; job.readout = readout;
    job.max_steps = max_steps; job.dL_dobs = dL_dobs; job.temperature = temperature;
    job.obs_out = obs_out; job.draws_out = draws_out; job.status_out = status_out;
    job.dtheta_traj_out = dtheta_traj_out; job.events_out = events_out;
    job.margins_out = margins_out; job.times_out = times_out; job.ev_cap = ev_cap;
    job.final_x_out = final_x_out;
    job.selector = selector;
    job.n_threads = n_threads > 0 ? n_threads : 1;
    pthread_mutex_init(&job.lock, NULL);
    if (job.n_threads == 1) {
        orc_worker(&job);
    } else {
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)job.n_threads);
        if (!th) { pthread_mutex_destroy(&job.lock); return -1; }
        for (int t = 0; t < job.n_threads; ++t) pthread_create(&th[t], NULL, orc_worker, &job);
        for (int t = 0; t < job.n_threads; ++t) pthread_join(th[t], NULL);
        free(th);
    }
    pthread_mutex_destroy(&job.lock);
    return job.error ? -1 : 0;
}

int orc_run(const orc_network *net, int64_t n_traj, int64_t traj_offset,
            const int32_t *x0, int32_t x0_per_traj, double t_end,
            const double *ts, int32_t S, const int32_t *obs_species, int32_t n_obs,
            uint64_t seed, int32_t readout, int64_t max_steps,
            const double *dL_dobs, double temperature,
            double *obs_out, int64_t *draws_out, int32_t *status_out,
            double *dtheta_traj_out,
            int32_t *events_out, double *margins_out, double *times_out, int64_t ev_cap,
            int32_t *final_x_out, int32_t n_threads)
{
    return orc_run_sel(0, net, n_traj, traj_offset, x0, x0_per_traj, t_end, ts, S, obs_species, n_obs, seed,
                       readout, max_steps, dL_dobs, temperature, obs_out, draws_out, status_out,
                       dtheta_traj_out, events_out, margins_out, times_out, ev_cap, final_x_out, n_threads);
}

/* ======================================================================================== */
/* Gene-regulatory-network classifier (Section 4.3, Figure 4A).                               */
/*                                                                                            */
/* Species: n_in clamped input transcription factors x_p (constant counts), n_hid hidden gene  */
/* products h_i and n_out output gene products y_o; the dynamic species are s = 0..n_dyn-1     */
/* with n_dyn = n_hid + n_out (hidden first). Reactions: j < n_dyn is the production of       */
/* species j, j >= n_dyn the degradation of species j - n_dyn. Propensities:                  */
/*   production of h_i:  k_max sigma(E1_i),  E1 = W1 x + b1   (the promoter's ON probability    */
/*                                                            is a logistic in an affine      */
/*                                                            function of the regulators)     */
/*   production of y_o:  k_max sigma(E2_o),  E2 = W2 h + b2                                     */
/*   degradation of s:   d_s X_s,            d_s = exp(log_d_s)                                 */
/* The simulation, the Gumbel-max choice and the straight-through adjoint follow the same      */
/* definitions as the mass-action oracle above; parameters are W1, b1, W2, b2 and log_d.      */
/* With soft = 1 the forward is the relaxed one of Eq. 4 (the first training phase of Section  */
/* 3.5): real-valued counts moved every step by the soft sample, a degradation propensity of a */
/* negative count taken as 0, and the gradient is the exact gradient of that relaxed model.   */
/* ======================================================================================== */
typedef struct {
    int32_t n_in, n_hid, n_out;
    const double *W1;    /* [n_hid][n_in] */
    const double *b1;    /* [n_hid] */
    const double *W2;    /* [n_out][n_hid] */
    const double *b2;    /* [n_out] */
    const double *log_d; /* [n_hid + n_out] */
    double k_max;
} orc_grn;

static double orc_sigmoid(double e) { return e >= 0.0 ? 1.0 / (1.0 + exp(-e)) : exp(e) / (1.0 + exp(e)); }

typedef struct {
    const orc_grn *g;
    int64_t n_img, traj_per_img, traj_offset;
    const int32_t *x_img; /* [n_img][n_in] */
    double t_end;
    const double *ts;
    int32_t S;
    uint64_t seed;
    int64_t max_steps;
    const double *dL_dobs; /* [n_traj][S][n_out] or NULL */
    double T;
    double *obs_out;       /* [n_traj][S][n_out] */
    int64_t *draws_out;
    int32_t *status_out;
    double *dE1_out;       /* [n_traj][n_hid]: dL/dE1 per trajectory (or NULL) */
    double *dW2_out;       /* [n_traj][n_out][n_hid] (or NULL) */
    double *db2_out;       /* [n_traj][n_out] */
    double *dlogd_out;     /* [n_traj][n_dyn] */
    int32_t *events_out;   /* [n_traj][ev_cap] or NULL */
    double *margins_out;
    int64_t ev_cap;
    int32_t soft;          /* 1: the relaxed forward of Eq. 4 at temperature T */
    int64_t next;
    pthread_mutex_t lock;
    int error;
} orc_grn_job;

/* propensities of all M = 2 n_dyn reactions at state X (double counts; soft: a negative count degrades at 0) */
static void orc_grn_prop(const orc_grn *g, const double *E1, const double *X, double *a, double *E2, int soft)
{
    const int nh = g->n_hid, no = g->n_out, nd = nh + no;
    for (int o = 0; o < no; ++o) {
        double e = g->b2[o];
        for (int i = 0; i < nh; ++i) e += g->W2[(size_t)o * nh + i] * X[i];
        E2[o] = e;
    }
    for (int i = 0; i < nh; ++i) a[i] = g->k_max * orc_sigmoid(E1[i]);
    for (int o = 0; o < no; ++o) a[nh + o] = g->k_max * orc_sigmoid(E2[o]);
    for (int s = 0; s < nd; ++s) a[nd + s] = exp(g->log_d[s]) * (soft && X[s] < 0.0 ? 0.0 : X[s]);
}

static void *orc_grn_worker(void *arg)
{
    orc_grn_job *job = (orc_grn_job *)arg;
    const orc_grn *g = job->g;
    const int nh = g->n_hid, no = g->n_out, nd = nh + no, M = 2 * nd, ni = g->n_in;
    const int S = job->S;
    double *E1 = (double *)malloc(sizeof(double) * nh);
    double *E2 = (double *)malloc(sizeof(double) * no);
    double *a = (double *)malloc(sizeof(double) * M);
    double *y = (double *)malloc(sizeof(double) * M);
    double *lam = (double *)malloc(sizeof(double) * nd);
    double *lam_new = (double *)malloc(sizeof(double) * nd);
    double *G2 = (double *)malloc(sizeof(double) * no);
    if (!E1 || !E2 || !a || !y || !lam || !lam_new || !G2) { job->error = 1; goto done; }
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t i = job->next++;
        pthread_mutex_unlock(&job->lock);
        const int64_t n_traj = job->n_img * job->traj_per_img;
        if (i >= n_traj) break;
        const uint64_t traj = (uint64_t)(job->traj_offset + i);
        const int32_t *x = job->x_img + (size_t)(i / job->traj_per_img) * ni;
        for (int h = 0; h < nh; ++h) {
            double e = g->b1[h];
            for (int p = 0; p < ni; ++p) e += g->W1[(size_t)h * ni + p] * (double)x[p];
            E1[h] = e;
        }
        /* forward with the full path kept */
        int64_t cap = 256, n_states = 0, n_draws = 0;
        double *Xh = (double *)malloc(sizeof(double) * (cap + 1) * nd);
        double *th = (double *)malloc(sizeof(double) * (cap + 1));
        double *tauh = (double *)malloc(sizeof(double) * cap);
        int32_t *jh = (int32_t *)malloc(sizeof(int32_t) * cap);
        double *mh = (double *)malloc(sizeof(double) * cap);
        if (!Xh || !th || !tauh || !jh || !mh) { job->error = 1; free(Xh); free(th); free(tauh); free(jh); free(mh); break; }
        for (int s = 0; s < nd; ++s) Xh[s] = 0.0;
        th[0] = 0.0;
        int32_t status = ORC_OK, crossed = 0;
        int64_t k = 0;
        for (;;) {
            if (k >= job->max_steps) { status = ORC_STEP_CAP; break; }
            if (k + 2 > cap) {
                cap *= 2;
                Xh = (double *)realloc(Xh, sizeof(double) * (cap + 1) * nd);
                th = (double *)realloc(th, sizeof(double) * (cap + 1));
                tauh = (double *)realloc(tauh, sizeof(double) * cap);
                jh = (int32_t *)realloc(jh, sizeof(int32_t) * cap);
                mh = (double *)realloc(mh, sizeof(double) * cap);
                if (!Xh || !th || !tauh || !jh || !mh) { job->error = 1; break; }
            }
            const double *X = Xh + (size_t)k * nd;
            orc_grn_prop(g, E1, X, a, E2, job->soft);
            double a0 = 0.0;
            for (int j = 0; j < M; ++j) a0 += a[j];
            if (a0 == 0.0) { status = ORC_ABSORBED; break; }
            const double tau = -log(orc_uniform(job->seed, traj, (uint64_t)k, 0)) / a0;
            int best = -1;
            double s1 = -INFINITY, s2 = -INFINITY;
            for (int j = 0; j < M; ++j) {
                if (!(a[j] > 0.0)) continue;
                const double key = log(a[j]) - log(-log(orc_uniform(job->seed, traj, (uint64_t)k, 1 + j)));
                if (key > s1) { s2 = s1; s1 = key; best = j; }
                else if (key > s2) s2 = key;
            }
            jh[k] = best;
            tauh[k] = tau;
            mh[k] = (s2 == -INFINITY) ? 1.0 : -expm1(s2 - s1);
            th[k + 1] = th[k] + tau;
            n_draws = k + 1;
            if (th[k + 1] > job->t_end) { crossed = 1; break; }
            double *Xn = Xh + (size_t)(k + 1) * nd;
            for (int s = 0; s < nd; ++s) Xn[s] = X[s];
            if (job->soft) {
                /* relaxed update (Eq. 4): production j adds y~_j to species j, degradation removes it */
                double zmax = -INFINITY, Z = 0.0;
                for (int j = 0; j < M; ++j) {
                    y[j] = -INFINITY;
                    if (a[j] > 0.0)
                        y[j] = (log(a[j]) - log(-log(orc_uniform(job->seed, traj, (uint64_t)k, 1 + j)))) / job->T;
                    if (y[j] > zmax) zmax = y[j];
                }
                for (int j = 0; j < M; ++j) { y[j] = y[j] == -INFINITY ? 0.0 : exp(y[j] - zmax); Z += y[j]; }
                for (int j = 0; j < M; ++j) {
                    if (j < nd) Xn[j] += y[j] / Z;
                    else Xn[j - nd] -= y[j] / Z;
                }
            } else if (best < nd) {
                Xn[best] += 1.0;
            } else {
                Xn[best - nd] -= 1.0;
            }
            ++k;
        }
        if (job->error) break;
        n_states = k + 1;
        /* readout: HOLD of the outputs at each sample time */
        double *obs = job->obs_out + (size_t)i * S * no;
        for (int s = 0; s < S; ++s) {
            int64_t kb = 0;
            while (kb + 1 < n_states && th[kb + 1] <= job->ts[s]) ++kb;
            for (int o = 0; o < no; ++o) obs[(size_t)s * no + o] = Xh[(size_t)kb * nd + nh + o];
        }
        if (job->draws_out) job->draws_out[i] = n_draws;
        if (job->status_out) job->status_out[i] = status;
        if (job->events_out)
            for (int64_t q = 0; q < job->ev_cap; ++q) {
                job->events_out[(size_t)i * job->ev_cap + q] = q < n_draws ? jh[q] : -1;
                if (job->margins_out) job->margins_out[(size_t)i * job->ev_cap + q] = q < n_draws ? mh[q] : NAN;
            }
        /* straight-through adjoint (HOLD readout: no time terms) */
        if (job->dL_dobs) {
            double *dE1 = job->dE1_out + (size_t)i * nh;
            double *dW2 = job->dW2_out + (size_t)i * no * nh;
            double *db2 = job->db2_out + (size_t)i * no;
            double *dld = job->dlogd_out + (size_t)i * nd;
            for (int h = 0; h < nh; ++h) dE1[h] = 0.0;
            for (int q = 0; q < no * nh; ++q) dW2[q] = 0.0;
            for (int o = 0; o < no; ++o) db2[o] = 0.0;
            for (int s = 0; s < nd; ++s) { dld[s] = 0.0; lam[s] = 0.0; }
            const double *gl = job->dL_dobs + (size_t)i * S * no;
            double mu = 0.0;
            for (int64_t kk = n_states - 1; kk >= 0; --kk) {
                const double *X = Xh + (size_t)kk * nd;
                const int draw = kk < n_draws && (kk + 1 < n_states || crossed);
                for (int s = 0; s < nd; ++s) lam_new[s] = lam[s];
                if (draw) {
                    orc_grn_prop(g, E1, X, a, E2, job->soft);
                    double a0 = 0.0;
                    for (int j = 0; j < M; ++j) a0 += a[j];
                    const double tau = tauh[kk];
                    const double dtau = mu; /* HOLD readout: no direct time terms */
                    double zmax = -INFINITY;
                    for (int j = 0; j < M; ++j) {
                        if (a[j] > 0.0) {
                            y[j] = (log(a[j]) - log(-log(orc_uniform(job->seed, traj, (uint64_t)kk, 1 + j)))) / job->T;
                            if (y[j] > zmax) zmax = y[j];
                        }
                    }
                    double Z = 0.0;
                    for (int j = 0; j < M; ++j) { y[j] = a[j] > 0.0 ? exp(y[j] - zmax) : 0.0; Z += y[j]; }
                    double wbar = 0.0;
                    for (int j = 0; j < M; ++j) {
                        y[j] /= Z;
                        const double w = j < nd ? lam[j] : -lam[j - nd]; /* v_j = +e_s or -e_s */
                        wbar += y[j] * w;
                    }
                    const double dLda0 = -dtau * tau / a0;
                    for (int o = 0; o < no; ++o) G2[o] = 0.0;
                    for (int j = 0; j < M; ++j) {
                        const double w = j < nd ? lam[j] : -lam[j - nd];
                        const double psi = a[j] > 0.0 ? y[j] * (w - wbar) / job->T : 0.0;
                        const double tot = psi + dLda0 * a[j]; /* dL/dlog a_j */
                        if (j < nh) {
                            dE1[j] += tot * (1.0 - orc_sigmoid(E1[j]));
                        } else if (j < nd) {
                            const int o = j - nh;
                            G2[o] = tot * (1.0 - orc_sigmoid(E2[o]));
                        } else {
                            const int s = j - nd;
                            dld[s] += tot;
                            const double d = exp(g->log_d[s]);
                            lam_new[s] += (a[j] > 0.0 ? psi / X[s] : 0.0) +
                                          (job->soft && X[s] < 0.0 ? 0.0 : dLda0 * d);
                        }
                    }
                    for (int o = 0; o < no; ++o) {
                        db2[o] += G2[o];
                        for (int h = 0; h < nh; ++h) {
                            dW2[(size_t)o * nh + h] += G2[o] * X[h];
                            lam_new[h] += g->W2[(size_t)o * nh + h] * G2[o];
                        }
                    }
                }
                for (int s = 0; s < S; ++s) {
                    int64_t kb = 0;
                    while (kb + 1 < n_states && th[kb + 1] <= job->ts[s]) ++kb;
                    if (kb != kk) continue;
                    for (int o = 0; o < no; ++o) lam_new[nh + o] += gl[(size_t)s * no + o];
                }
                for (int s = 0; s < nd; ++s) lam[s] = lam_new[s];
            }
        }
        free(Xh); free(th); free(tauh); free(jh); free(mh);
    }
done:
    free(E1); free(E2); free(a); free(y); free(lam); free(lam_new); free(G2);
    return NULL;
}

/* soft = 1: the relaxed forward of Eq. 4 at temperature T (T > 0 required) and its exact gradient. */
int orc_grn_run_sel(int32_t soft, const orc_grn *g, int64_t n_img, int64_t traj_per_img, int64_t traj_offset,
                    const int32_t *x_img, double t_end, const double *ts, int32_t S, uint64_t seed, int64_t max_steps,
                    const double *dL_dobs, double T, double *obs_out, int64_t *draws_out, int32_t *status_out,
                    double *dE1_out, double *dW2_out, double *db2_out, double *dlogd_out,
                    int32_t *events_out, double *margins_out, int64_t ev_cap, int32_t n_threads)
{
    if (!g || g->n_in < 0 || g->n_hid < 1 || g->n_out < 1 || n_img < 0 || traj_per_img < 1 || S < 0) return -1;
    if (soft != 0 && soft != 1) return -1;
    if (soft && !(T > 0.0)) return -1;
    for (int s = 0; s < S; ++s)
        if (!(ts[s] >= 0.0 && ts[s] <= t_end) || (s > 0 && ts[s] < ts[s - 1])) return -1;
    if (dL_dobs && (!(T > 0.0) || !dE1_out || !dW2_out || !db2_out || !dlogd_out)) return -1;
    orc_grn_job job;
    memset(&job, 0, sizeof(job));
    job.g = g; job.n_img = n_img; job.traj_per_img = traj_per_img; job.traj_offset = traj_offset;
    job.x_img = x_img; job.t_end = t_end; job.ts = ts; job.S = S; job.seed = seed; job.max_steps = max_steps;
    job.dL_dobs = dL_dobs; job.T = T; job.obs_out = obs_out; job.draws_out = draws_out;
    job.status_out = status_out; job.dE1_out = dE1_out; job.dW2_out = dW2_out; job.db2_out = db2_out;
    job.dlogd_out = dlogd_out; job.events_out = events_out; job.margins_out = margins_out; job.ev_cap = ev_cap;
    job.soft = soft;
    pthread_mutex_init(&job.lock, NULL);
    const int nt = n_threads > 0 ? n_threads : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
    if (!th) return -1;
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, orc_grn_worker, &job);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&job.lock);
    return job.error ? -1 : 0;
}

int orc_grn_run(const orc_grn *g, int64_t n_img, int64_t traj_per_img, int64_t traj_offset, const int32_t *x_img,
                double t_end, const double *ts, int32_t S, uint64_t seed, int64_t max_steps,
                const double *dL_dobs, double T, double *obs_out, int64_t *draws_out, int32_t *status_out,
                double *dE1_out, double *dW2_out, double *db2_out, double *dlogd_out,
                int32_t *events_out, double *margins_out, int64_t ev_cap, int32_t n_threads)
{
    return orc_grn_run_sel(0, g, n_img, traj_per_img, traj_offset, x_img, t_end, ts, S, seed, max_steps, dL_dobs, T,
                           obs_out, draws_out, status_out, dE1_out, dW2_out, db2_out, dlogd_out, events_out,
                           margins_out, ev_cap, n_threads);
}
