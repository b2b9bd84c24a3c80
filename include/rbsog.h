/*
 * rbsog.h -- C ABI of the GB300 (sm_103a) random batch sum-of-Gaussians
 * (RBSOG) force evaluation and velocity-Verlet integrator.
 *
 * Method: Liang, Xu, Xu, Zhao, "Random batch sum-of-Gaussians method for
 * molecular dynamics simulations of particle systems" (arXiv:2205.13824).
 * Section and equation numbers below refer to that paper.
 *
 * Conventions shared by every entry point
 *   - Every call returns an rbsog_status; nothing throws or aborts across the
 *     ABI.  On failure rbsog_last_error() describes the cause.
 *   - Arrays of particle vectors are row-major [n][3] doubles in the caller's
 *     particle order.  Pointers may be host memory (pageable or pinned) or
 *     device memory of the context's device: copies use cudaMemcpyDefault.
 *   - The caller owns every buffer it passes; the library copies what it
 *     needs and never frees or retains caller memory after the call returns.
 *   - Work is enqueued on the CUDA stream given to rbsog_create (0 = the
 *     legacy default stream).  Internally the context runs on its own stream
 *     and orders itself after / before the caller's stream with events.
 *     Calls that return host values (energies, state into host memory,
 *     statuses of device checks) synchronise with that work.
 *   - Units are the caller's; all Coulomb terms are multiplied by
 *     coulomb_prefactor (Bjerrum length x kT in reduced units).
 */
#ifndef RBSOG_H
#define RBSOG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbsog_ctx rbsog_ctx; /* opaque, owned by the library */

typedef enum {
    RBSOG_OK = 0,
    RBSOG_EINVAL = 1,   /* invalid argument or parameter set                 */
    RBSOG_ENOMEM = 2,   /* device or host allocation failed                  */
    RBSOG_ECUDA = 3,    /* a CUDA runtime call failed                        */
    RBSOG_ESTATE = 4,   /* call out of order (e.g. step before set_state)    */
    RBSOG_ENUMERIC = 5, /* non-finite force found on the device, or a
                           neighbour list exceeded its capacity              */
    RBSOG_ETIMEOUT = 6  /* a bounded device wait gave up                     */
} rbsog_status;

typedef enum {
    RBSOG_FP64 = 0,  /* plain FP64 everywhere: the comparator path           */
    RBSOG_FP32C = 1  /* 32-bit fixed-point positions, FP32 pair and sincos
                        arithmetic, compensated FP32 rho(k) partials; FP64
                        for the cross-block rho combine, energies and the
                        integrator's state.  Near field on neighbour lists
                        with a skin of r_c / 10, rebuilt on the device when a
                        particle has moved more than half the skin (boxes with
                        fewer than 3 cells of side 1.1 r_c per side: the cell
                        stencil every step)                                 */
} rbsog_precision;

/* Parameters of one system (Sec. 2 and 3; Algorithm 1). */
typedef struct {
    double L[3];              /* periodic cuboid edges L_x, L_y, L_z (Sec. 2)                */
    double b;                 /* SOG base b > 1 (Eq. 2.5)                                     */
    double sigma;             /* SOG width sigma; <= 0: solve sigma and omega0 jointly from
                                 the C0/C1 conditions at r_c (Eqs. 2.10-2.11)                 */
    double omega0;            /* narrowest weight; <= 0 with sigma > 0: C0 value of Eq. 2.11   */
    int32_t M;                /* last Gaussian index, M+1 terms (Eq. 2.8), 0 <= M < 128       */
    double r_c;               /* near cutoff (Eq. 2.7); floor(L_d / r_c) >= 3, r_c < L_d / 2 */
    int32_t P;                /* frequencies per step, the batch size of Eq. 3.24, >= 1      */
    double coulomb_prefactor; /* multiplies every Coulomb term                                */
    double wca_sigma;         /* soft repulsion 4e[(s/r)^12-(s/r)^6]+e for r < 2^(1/6) s;
                                 0 disables it                                               */
    double wca_eps;
    double dt;                /* velocity-Verlet step                                         */
    double mass;              /* particle mass (all particles)                                */
    double T_target;          /* Berendsen target temperature (k_B = 1)                        */
    double tau_T;             /* Berendsen time constant; <= 0: NVE                            */
    uint64_t seed;            /* key of the counter-based generator of the sampler            */
    int64_t n_ksets;          /* k-sets to pre-sample (Algorithm 1 line 2); one is consumed
                                 per force evaluation; >= 1                                   */
    int32_t chain_len;        /* samples per Metropolis-Hastings chain; 0: 256                  */
    int32_t precision;        /* rbsog_precision                                               */
    int32_t boundary;         /* zero-frequency term (Sec. 3.2): 0 tinfoil (no term);
                                 1 spherical infinite boundary, U0 = (2 pi / 3V) |M|^2
                                 (Eq. 3.14); 2 planar infinite boundary along z,
                                 U0 = (2 pi / V) M_z^2 (Eq. 3.15); M = sum_i q_i r_i over the
                                 positions folded into [0, L); times coulomb_prefactor       */
    int32_t near_kernel;      /* FP32C neighbour-list path only: 0 the combined G/F table
                                 (default); 1 the paper's core-shell kernel (Sec. 3.4):
                                 pairs with r < r_in from a 10-term Taylor series of the
                                 Gaussian sums in r^2 (Eqs. 3.25-3.26), the others from a
                                 table indexed by the low exponent bits and 8 high mantissa
                                 bits of the FP32 r^2, linearly interpolated.  RBSOG_EINVAL
                                 when the system does not run on neighbour lists.            */
    double r_in;              /* core radius of near_kernel 1; <= 0: r_c / 3; the table covers
                                 at most 8 octaves of r^2 from r_in^2 up to r_c^2           */
    int32_t thermostat;       /* with tau_T > 0: 0 Berendsen rescale after the second half
                                 kick; 1 Langevin dynamics with friction 1/tau_T and bath
                                 temperature T_target in the BAOAB splitting (v += dt/2 F/m;
                                 x += dt/2 v; v = c1 v + c2 z, c1 = e^{-dt/tau_T},
                                 c2 = sqrt((1 - c1^2) T_target/m); x += dt/2 v; forces;
                                 v += dt/2 F/m).  The noise z of particle i in the step with
                                 step counter t is Philox4x64-10 (key (seed, 2^63 + 1),
                                 counter (t, i, 0, 0)) through Box-Muller;
                                 2 Nose-Hoover with thermostat mass Q = g T_target tau_T^2
                                 (g = 3N - 3) in the symmetric Trotter splitting: each step
                                 is velocity Verlet followed by the end half of its
                                 thermostat update and the start half of the next, each
                                 xi += dt/4 G; v *= e^{-xi dt/2}; eta += dt/2 xi;
                                 xi += dt/4 G with G = (2K - g T_target)/Q; set_state
                                 starts xi = eta = 0; U + K + U_th is conserved            */
    int32_t sampler;          /* frequency sampler (Sec. 3.3): 0 the mixture distribution by
                                 Metropolis-Hastings chains (default); 1 per-Gaussian
                                 independent sampling: Gaussian l, normalised over k != 0, is
                                 sampled exactly P_l = ceil(P S_l / S) times per set, S_l =
                                 w_l s_l^3 (prod_d H_l^d - 1) its share of S (Gaussians with
                                 S_l <= 1e-16 S dropped), each frequency weighted by S_l/P_l;
                                 a set then holds P_eff = sum_l P_l frequencies (the largest
                                 over a batch, shorter sets padded with weight-0 entries;
                                 rbsog_info.P_set).  The same for every system of a batch;
                                 chain_len is unused.  Frequency eta of set t draws the
                                 Philox4x64-10 blocks A, B with key (seed, 2^63 + 2) and
                                 counters (t, eta, 0, 0), (t, eta, 1, 0); its first non-zero
                                 coordinate is x if u(A0) < P(m_x != 0 | m != 0), else y if
                                 u(A1) < P(m_y != 0 | m_x = 0, m != 0), else z; earlier
                                 coordinates are 0, that one is drawn given |m_d| >= 1 and
                                 later ones unconditioned, |m_d| by inverting with u(B_d) the
                                 sums 1 + sum_{i=1..j} 2 e^{-x i^2}, x = (pi s_l / L_d)^2,
                                 j <= ceil(sqrt(50 / x)), the sign from bit d of A2
                                 (u(r) = (r >> 11) 2^-53).
                                 With sampler 0 each set of the sequence is folded on the
                                 device after sampling: a Metropolis-Hastings chain repeats
                                 its state on every rejection (about half of the draws), and
                                 each run of equal consecutive frequencies is evaluated once
                                 and weighted by its length in rho(k), the far force and the
                                 energy -- the same sums up to rounding.  An explicit k-set
                                 (rbsog_compute_forces) is evaluated entry by entry.         */
} rbsog_params;

/* Energies of the last force evaluation (Eqs. 3.1, 3.6-3.8) and kinetic state. */
typedef struct {
    double U_near; /* (1/2) sum q_i q_j N(r_ij) over pairs within r_c                   */
    double U_far;  /* random-batch estimate (pi^{3/2} S / (2 P V)) sum_eta |rho(k_eta)|^2 */
    double U_self; /* (1/2) F_M(0) sum q_i^2                                              */
    double U_wca;  /* soft repulsion                                                      */
    double K;      /* kinetic energy after the last completed step                        */
    double T;      /* 2K / (3N - 3)                                                       */
    double U_bound; /* zero-frequency (boundary) term; 0 for tinfoil                      */
    double U_th;   /* Nose-Hoover thermostat energy (1/2) Q xi^2 + g T_target eta; 0 otherwise */
} rbsog_energies;

/* Solved SOG decomposition (Eqs. 2.8-2.11) and the normaliser S (Eq. 3.16). */
typedef struct {
    double sigma, omega0, S;
    int32_t M;
    int32_t ncell[3];         /* cell grid of the near-field cell list                      */
    int64_t n_chains;         /* sampler chains; chain c fills sequence entries
                                 [c * chain_len, (c + 1) * chain_len)                       */
    int32_t chain_len;
    int32_t P_set;            /* frequencies per k-set: P, or P_eff with sampler 1          */
    int64_t list_builds;      /* FP32C neighbour-list path: builds run since set_params (any
                                 system of the context); 0 off that path.  Reading it waits
                                 for the context's queued work                              */
} rbsog_info;

/* Create a context for n >= 2 particles on CUDA device `device`; `stream`
 * is a cudaStream_t (or NULL for the legacy default stream).  *out is set
 * to NULL on failure. */
rbsog_status rbsog_create(rbsog_ctx **out, int64_t n, int device, void *stream);

/* Validate p, solve the SOG parameters if asked (Eqs. 2.10-2.11, host FP64),
 * compute S (Eq. 3.16), and pre-sample the frequency sequence of
 * Algorithm 1 on the device (independent Metropolis-Hastings chains,
 * Sec. 3.3).  Rejects (RBSOG_EINVAL): b <= 1, sigma/omega0 invalid, M outside
 * [0, 127], P < 1, n_ksets < 1, r_c <= 0, r_c >= L_d / 2, fewer than 3 cells
 * per side, mass <= 0, an unknown precision.  Resets the k-set cursor. */
rbsog_status rbsog_set_params(rbsog_ctx *ctx, const rbsog_params *p);

/* Parameters as solved by the last rbsog_set_params.  omega and s (length
 * M+1, host) may be NULL. */
rbsog_status rbsog_get_info(const rbsog_ctx *ctx, rbsog_info *info, double *omega, double *s);

/* Load charges q[n], positions x[n][3] (folded into the box) and
 * velocities v[n][3] (NULL: zero), host or device.  Rejects a non-neutral
 * charge vector, |sum q| > 1e-12 sum |q| (the method assumes neutrality,
 * Sec. 2).  Invalidates the stored forces: the next step first evaluates
 * them.  FP32C neighbour lists are kept: the next force evaluation's
 * displacement test rebuilds them if any particle moved more than half the
 * skin since they were built.  Synchronises. */
rbsog_status rbsog_set_state(rbsog_ctx *ctx, const double *q, const double *x, const double *v);

/* One force evaluation F = F_N + F*_F (+ WCA) at the current positions
 * (Eq. 3.9 first line, Eq. 3.24).  m_kset: P integer frequency vectors
 * m[P][3] (k = 2 pi m / L; P_set of rbsog_info with the per-Gaussian
 * sampler) in host or device memory, each weighted S / P as mixture samples,
 * or NULL to take the next k-set of the pre-sampled sequence with its own
 * weights (advancing the cursor).  f_out
 * ([n][3], host or device) and e_out (host) may be NULL.  The forces are
 * also kept as the context's current forces. */
rbsog_status rbsog_compute_forces(rbsog_ctx *ctx, const int32_t *m_kset, double *f_out,
                                  rbsog_energies *e_out);

/* Advance nsteps velocity-Verlet steps of Algorithm 1, each consuming the
 * next k-set (RBSOG_ENUMERIC at the next synchronising call if a force was
 * non-finite or a neighbour list overflowed); with tau_T > 0 velocities are
 * rescaled by
 * sqrt(1 + dt/tau_T (T_target/T - 1)) after the second half kick.  Enqueued
 * asynchronously (replayed from a CUDA graph of one step when profiling is
 * off).  The energies rbsog_get_energies reads afterwards are those of the
 * last step; the steps before it may leave the pair energies out.  Returns
 * RBSOG_EINVAL if the sequence would run out of k-sets. */
rbsog_status rbsog_step(rbsog_ctx *ctx, int64_t nsteps);

/* Copy the current state out (any pointer may be NULL; host or device):
 * x[n][3] folded positions, v[n][3], f[n][3] current forces, *step the
 * number of completed steps.  Synchronises and reports RBSOG_ENUMERIC if a
 * non-finite force was produced since the last check. */
rbsog_status rbsog_get_state(rbsog_ctx *ctx, double *x, double *v, double *f, int64_t *step);

/* Number of k-sets consumed so far (the cursor into the pre-sampled
 * sequence; host value, no synchronisation). */
rbsog_status rbsog_get_cursor(const rbsog_ctx *ctx, int64_t *kset_cursor);

/* Resume from a checkpoint: after rbsog_set_state, load the forces f[n][3]
 * (host or device) that belong to those positions, the k-set cursor and
 * the step counter, so that the next step continues the run exactly (the
 * stored forces are used instead of a new force evaluation).  Rejects a
 * cursor outside [0, n_ksets]. */
rbsog_status rbsog_restore(rbsog_ctx *ctx, const double *f, int64_t kset_cursor, int64_t step);

/* Steps for a caller that keeps the state in its own memory: the same
 * result, bit for bit, as rbsog_set_state(q, x, v), rbsog_restore(f,
 * kset_cursor, step) (or no restore when f is NULL: the forces of x are then
 * computed first, consuming one k-set), rbsog_step(nsteps) and
 * rbsog_get_state(x_out, v_out, f_out), i.e. nsteps velocity-Verlet steps of
 * Algorithm 1 from the given state.  One call, one synchronisation at the
 * end; the last step's new positions are copied out while the rest of that
 * step (forces, second half kick) runs.  q[n], x, v, f, x_out, v_out,
 * f_out ([n][3] FP64) may be host or device memory; outputs may be NULL and
 * may alias the inputs.  Single-system contexts only (RBSOG_EINVAL for a
 * batch of several systems or a serving batch); RBSOG_EINVAL for
 * non-neutral charges, nsteps < 1, a negative cursor or step, or a
 * k-sequence too short for the steps; RBSOG_ENUMERIC as rbsog_get_state.
 * On return the outputs are written. */
rbsog_status rbsog_step_io(rbsog_ctx *ctx, const double *q, const double *x, const double *v, const double *f,
                           int64_t kset_cursor, int64_t step, int64_t nsteps, double *x_out, double *v_out,
                           double *f_out);

/* Energies of the last force evaluation and the kinetic energy (host). */
rbsog_status rbsog_get_energies(rbsog_ctx *ctx, rbsog_energies *e);

/* Copy k-sets [set0, set0 + nsets) of the pre-sampled sequence as
 * m[nsets * P][3] int32 (host or device). */
rbsog_status rbsog_get_kseq(rbsog_ctx *ctx, int64_t set0, int64_t nsets, int32_t *m_out);

/* Structure factors rho(k) = sum_j q_j e^{i k . r_j} (Eq. 3.4) at the current
 * positions for P integer vectors m[P][3] (host or device); rho_out is
 * [P][2] (Re, Im) doubles, host or device.  Uses the same sweep and combine
 * kernels as the force path. */
rbsog_status rbsog_rho(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *rho_out);

/* Cell list of the current positions (the near-field traversal structure):
 * cell_start[ncell + 1] offsets, perm[n] particle index in cell order
 * (within a cell by increasing fixed-point x = trunc(x (2^32 / L_x)), then
 * index), nbr[n] number of partners within r_c per particle (caller order).
 * Cells have side >= r_c (FP64) or >= 1.1 r_c (FP32C with neighbour lists).
 * Any pointer may be NULL. */
rbsog_status rbsog_get_cells(rbsog_ctx *ctx, int32_t *cell_start, int32_t *perm, int32_t *nbr);

/* Kernel-level timing: when on, launches run eagerly with a CUDA event pair
 * around each kernel; rbsog_get_profile returns, per kernel name, the launch
 * count and the summed device time in ms since profiling was switched on.
 * names: array of `cap` char[32] slots. Returns the number of kernels. */
rbsog_status rbsog_set_profiling(rbsog_ctx *ctx, int on);
rbsog_status rbsog_get_profile(rbsog_ctx *ctx, int32_t cap, char (*names)[32], int64_t *launches,
                               double *ms, int32_t *count);

/* Allocation-free structure factors.  The paper has no counterpart to this
 * entry point; it serves callers that cannot allocate device memory where
 * they need rho(k) -- code inside a region that forbids allocation (for
 * example work being recorded into a stream capture) or an embedding host
 * whose allocator must not be re-entered or has a fixed budget.
 *
 * Computes the same structure factors as rbsog_rho, in FP64, but without a
 * context: q[n], x[n][3] (any real positions), m[P][3] and rho_out[P][2]
 * (Re, Im) are caller-owned DEVICE buffers on the current device; L[3] is
 * host memory.  Work is enqueued on `stream` (cudaStream_t, NULL = legacy
 * default stream); the call does not synchronise.
 *
 * It allocates nothing: its partial sums live in a file-scope device array
 * of RBSOG_NOALLOC_MAX_P * 64 complex FP64 values (2 MiB) that every GPU
 * which loads the library holds until the process exits.  The first call in
 * a CUDA context (per device; again after that device's context was reset)
 * looks up the array's device address with cudaGetSymbolAddress, with the
 * device current; make that first call before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU (different
 * streams, or host threads) race and must be ordered by the caller.  Each
 * call overwrites every partial it reads, so no clearing is needed.
 *
 * Returns RBSOG_EINVAL for n < 1, P < 1, P > RBSOG_NOALLOC_MAX_P, a
 * non-positive box edge or a NULL pointer; RBSOG_ECUDA if a CUDA call fails. */
#define RBSOG_NOALLOC_MAX_P 2048
rbsog_status rbsog_rho_noalloc(int64_t n, const double *q, const double *x, const double *L,
                               const int32_t *m, int32_t P, double *rho_out, void *stream);

/* Configurational virial tensor W_ab = -dU/d eps_ab of the current
 * positions under the affine map r -> (1 + eps) r of positions and box (r_c
 * and the SOG fixed): the near field (+ WCA) sum over pairs r_ij,a F_ij,b
 * in FP64, plus the random-batch estimate of the far field on the k-set
 * m[P][3] (host or device): each sampled k weighted as in the energy (Eq.
 * 3.24), pi^{3/2} S / (2 P V) |rho(k)|^2, times
 * delta_ab + 2 k_a k_b dF~/d(k^2) / F~ (Eq. 3.5), which is unbiased for the
 * exact far virial.  W_out[9] (host or device) row-major and symmetric; the
 * pressure is (2K + trace W) / (3V).  Single system; rebuilds the cell list;
 * synchronises.  The boundary term is not included. */
rbsog_status rbsog_compute_virial(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *W_out);

/* Pressure tensor of Appendix A, P_ab = (1/V) sum_i (m v_ia v_ib + r_ia f_ib),
 * the second sum read as the configurational virial W_ab of
 * rbsog_compute_virial on the k-set m[P][3] (host or device), the first from
 * the current velocities; FP64 fixed-order sums.  P_out[9] (host or device)
 * row-major.  Single system; synchronises.  RBSOG_EINVAL for a NULL pointer,
 * P < 1 or a batch of several systems; RBSOG_ESTATE before set_state. */
rbsog_status rbsog_compute_pressure(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *P_out);

/* Time-correlation observables of Appendix A on the device (single system):
 * the mean-squared displacement eta_msd(t) = <|r(t0 + t) - r(t0)|^2> and the
 * velocity autocorrelation <v(t0) . v(t0 + t)>, averaged over the particles
 * and the time origins t0.  Time is counted in samples: each
 * rbsog_observe_sample takes the current positions and velocities as the
 * next frame (enqueued on the context's stream, no synchronisation), so call
 * it after every rbsog_step(ctx, s) to sample every s steps.  Positions are
 * unwrapped by adding the minimum-image displacement since the previous
 * sample (a particle must move less than half a box edge between samples).
 * Frames 0, origin_every, 2 origin_every, ... are time origins; each sample
 * adds, for every origin less than n_lags frames back, one FP64 particle sum
 * (fixed order) to the accumulator of its lag.
 *
 * rbsog_observe_start allocates 2 ceil(n_lags / origin_every) origin slots
 * of 32 bytes per particle plus per-particle unwrapping state, clears the
 * accumulators and makes the current state the next sample's frame 0; call
 * it again after rbsog_set_state.  RBSOG_EINVAL for n_lags < 1,
 * origin_every < 1 or more than 64 origins kept (ceil(n_lags /
 * origin_every) > 64), or a batch of several systems.
 * rbsog_observe_result writes msd[n_lags], vacf[n_lags] and count[n_lags]
 * (origins that reached each lag; 0 gives msd = vacf = 0), each host or
 * device, any of them NULL to skip; synchronises.  Sample and result return
 * RBSOG_ESTATE before rbsog_observe_start. */
rbsog_status rbsog_observe_start(rbsog_ctx *ctx, int32_t n_lags, int32_t origin_every);
rbsog_status rbsog_observe_sample(rbsog_ctx *ctx);
rbsog_status rbsog_observe_result(rbsog_ctx *ctx, double *msd, double *vacf, int64_t *count);

/* Green-Kubo shear viscosity of Appendix A from a pressure-tensor series
 * P_series[n_samples][9] (row-major tensors spaced dt apart, host or
 * device; e.g. from rbsog_compute_pressure):
 * C = V / (6 k_B T) sum_{a <= b} of the integral over t of
 * <dP_ab(t0 + t) dP_ab(t0)>, where dP_ab is the component's fluctuation
 * about its mean over the series, each autocorrelation averaged over all
 * origins t0 with t0 + t < n_samples and integrated by the trapezoid rule
 * over the lags 0 .. max_lag - 1.  acf_out[max_lag] (host or device, NULL to
 * skip) receives the summed autocorrelation per lag, *C_out (host) the
 * integral.  Context-free; work on `stream` (cudaStream_t, NULL = legacy
 * default stream), which the call synchronises.  RBSOG_EINVAL for
 * n_samples < 2, max_lag outside [2, n_samples], non-positive dt, V or T,
 * or a NULL P_series or C_out; RBSOG_ECUDA if a CUDA call fails. */
rbsog_status rbsog_green_kubo(const double *P_series, int64_t n_samples, double dt, double V, double T,
                              int32_t max_lag, double *acf_out, double *C_out, void *stream);

/* Heat flux J (Appendix A) of the current state of a single tinfoil system:
 *   J = (1/V) [ sum_i e_i v_i + (1/2) sum_{i<j} (f_ij . (v_i + v_j)) r_ij ],
 * e_i the per-atom energy: m |v_i|^2 / 2, half of each near-field (Coulomb
 * near part, Eq. 2.7, and WCA) pair energy, minus lB F_M(0) q_i^2 / 2, plus
 * the random-batch far energy split over atoms,
 * (c/2) q_i sum_eta Re(e^{-i k_eta . r_i} rho(k_eta)), c = lB pi^{3/2} S/(P V)
 * (Eq. 3.24), whose sum is the far energy.  The far field has no pair
 * forces; its share of the pair term is the random-batch far virial of
 * rbsog_compute_virial split over atoms the same way and contracted with
 * v_i.  k-set m[P][3] (host or device); P = 0 (m may be NULL): no far term.
 * FP64 for both precisions, from the FP64 state.  J_out[3] host or device.
 * RBSOG_EINVAL for a batch of several systems or a non-tinfoil boundary. */
rbsog_status rbsog_compute_heat_flux(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *J_out);

/* Heat conductivity by the Green-Kubo relation of Appendix A from a series
 * J_series[n_samples][3] (spaced dt apart, host or device; e.g. from
 * rbsog_compute_heat_flux): C = V / (3 k_B T^2) times the integral over t of
 * <J(t0) . J(t0 + t)>, the flux as sampled (no mean removed), averaged over
 * all origins t0 with t0 + t < n_samples and integrated by the trapezoid rule
 * over the lags 0 .. max_lag - 1.  acf_out[max_lag] (host or device, NULL to
 * skip), *C_out (host).  Context-free; work on `stream`, which the call
 * synchronises.  RBSOG_EINVAL for n_samples < 2, max_lag outside
 * [2, n_samples], non-positive dt, V or T, or a NULL J_series or C_out. */
rbsog_status rbsog_green_kubo_heat(const double *J_series, int64_t n_samples, double dt, double V, double T,
                                   int32_t max_lag, double *acf_out, double *C_out, void *stream);

/* Roofline denominators measured on `device` by short microbenchmarks (not
 * part of the method): out[0] MUFU sin/cos results per second (each of sin
 * and cos counts one), out[1] FP32 FMA per second, out[2] FP64 FMA per
 * second, out[3] SM clock in MHz while they ran, out[4] SM count.  Allocates
 * 128 bytes of device memory; synchronises. */
rbsog_status rbsog_measure_peaks(int device, double *out);

/* ---- Batched replicas -----------------------------------------------------
 * A batch holds n_sys independent systems of uneven size that advance
 * together: one rbsog_batch_step launches one CUDA graph per step whose
 * kernels cover every system (work tables map blocks to systems), so small
 * systems do not each pay for their own launches.  Every system's work is
 * decomposed exactly as it would be alone, so a system's trajectory is
 * bit-identical alone and in any batch.  Systems of one batch share b,
 * sigma, omega0, M, r_c, P and precision; box, charges, Coulomb prefactor,
 * WCA, dt, mass, thermostat, seed and sequence length are per system.  The
 * rbsog_ctx functions above operate on system 0 of a batch; a context made
 * by rbsog_create is a batch of one.  Destroy a batch with rbsog_destroy. */
typedef struct rbsog_ctx rbsog_batch;
/* n_per[n_sys] particles per system (each >= 2). */
rbsog_status rbsog_batch_create(rbsog_batch **out, int32_t n_sys, const int64_t *n_per, int device,
                                void *stream);
/* p[n_sys]; the same validation as rbsog_set_params for each system. */
rbsog_status rbsog_batch_set_params(rbsog_batch *b, const rbsog_params *p);
/* As rbsog_set_state / rbsog_restore / rbsog_get_state / rbsog_get_energies /
 * rbsog_get_kseq for system `sys` of the batch.  A system loaded with
 * set_state receives its initial force evaluation at the next step; the
 * other systems keep their forces and cursors. */
rbsog_status rbsog_batch_set_state(rbsog_batch *b, int32_t sys, const double *q, const double *x,
                                   const double *v);
rbsog_status rbsog_batch_restore(rbsog_batch *b, int32_t sys, const double *f, int64_t kset_cursor,
                                 int64_t step);
rbsog_status rbsog_batch_get_state(rbsog_batch *b, int32_t sys, double *x, double *v, double *f,
                                   int64_t *step);
rbsog_status rbsog_batch_get_energies(rbsog_batch *b, int32_t sys, rbsog_energies *e);
rbsog_status rbsog_batch_get_kseq(rbsog_batch *b, int32_t sys, int64_t set0, int64_t nsets,
                                  int32_t *m_out);
/* Advance every system of the batch by nsteps velocity-Verlet steps. */
rbsog_status rbsog_batch_step(rbsog_batch *b, int64_t nsteps);

/* Autotuner for launch shapes: times `reps` force evaluations of the whole
 * batch (into scratch forces; state, cursors and energies are untouched)
 * for candidate near-field block sizes (home particles per block) and
 * rho-sweep tiles (particles per tile), keeps the fastest, applies it and
 * remembers it for the systems' size classes (floor(log2 n), P, precision)
 * for every later context of the process.  chosen[2] (host, may be NULL)
 * receives (home, tile; 0 = default rule).  Needs params and state.  The
 * launch shape changes the order of floating-point sums, so results after
 * tuning may differ from untuned ones in the last bits. */
rbsog_status rbsog_batch_autotune(rbsog_batch *b, int32_t reps, int32_t *chosen);

/* Radial distribution functions (Appendix A) of the current positions of
 * system `sys` (rbsog_rdf: of the single system), cubic box only.  Pairs at
 * minimum-image distance r < L/2 are counted once per unordered pair in
 * counts[3][nbins] by charge-sign pair (row 0: ++, 1: +-, 2: --; neutral
 * sites are skipped), bin k holding k dr <= r < (k+1) dr, dr = L/(2 nbins).
 * g[3][nbins] receives the estimate of g(r) = (1/(N_a rho_b)) sum_{i in a}
 * sum_{j in b, j != i} delta(r_ij - r)/(4 pi r^2), rho_b = N_b / V.
 * Distances are measured on positions quantised to L 2^-32 per axis, so the
 * counts are exact integers independent of rounding.  nbins: a power of two
 * in [16, 4096].  counts and g may be host or device pointers or NULL.
 * Synchronises.  Cost O(N^2 / 2) pair visits. */
rbsog_status rbsog_batch_rdf(rbsog_batch *ctx, int32_t sys, int32_t nbins, uint64_t *counts, double *g);
rbsog_status rbsog_rdf(rbsog_ctx *ctx, int32_t nbins, uint64_t *counts, double *g);

/* ---- Serving engine ---------------------------------------------------------
 * Continuous batching of MD jobs (each: n particles, parameters, initial
 * state, a step count).  Jobs wait in a FIFO queue and are admitted while a
 * job slot is free and their estimated device-memory footprint fits the
 * budget; admitted jobs advance together as one batch (one graph launch per
 * step).  A job that has done its steps is frozen on the device and retired
 * (state copied to host) at the end of the quantum; admissions and
 * retirements rebuild the batch at the next quantum, moving the running
 * jobs' state device to device.  Each job's trajectory is the one it would
 * follow alone (same parameters and seed).  All jobs of a server share b,
 * sigma, omega0, M, r_c, P, precision, sampler, near_kernel and r_in (those
 * of the first job submitted).  Host memory for inputs is copied
 * at submit; results stay on the host until released. */
typedef struct rbsog_server rbsog_server;
/* max_jobs >= 1 slots, mem_budget_bytes > 0, quantum >= 1 steps per advance. */
rbsog_status rbsog_server_create(rbsog_server **out, int32_t max_jobs, int64_t mem_budget_bytes,
                                 int32_t quantum, int device, void *stream);
/* Queue a job: q[n], x[n][3], v[n][3] (NULL: zero) in host memory; the
 * sequence length is set to nsteps + 1.  RBSOG_ENOMEM if the job alone
 * exceeds the budget; RBSOG_EINVAL if a shared parameter differs from the
 * first job's. */
rbsog_status rbsog_server_submit(rbsog_server *s, int64_t n, const rbsog_params *p, const double *q,
                                 const double *x, const double *v, int64_t nsteps, int64_t *job_id);
/* Admit what fits, rebuild the batch if its membership changed, advance it
 * by up to `quantum` steps and retire finished jobs (synchronises). */
rbsog_status rbsog_server_advance(rbsog_server *s, int32_t *n_active, int32_t *n_waiting,
                                  int32_t *n_retired);
/* status: 0 waiting, 1 running, 2 done (then x, v, f [n][3], energies and the
 * steps done are copied out to host pointers, any of which may be NULL),
 * 3 cancelled. */
rbsog_status rbsog_server_result(rbsog_server *s, int64_t job_id, int32_t *status, double *x, double *v,
                                 double *f, rbsog_energies *e, int64_t *steps_done);
/* Cancel a job: a waiting job leaves the queue; a running job is frozen at
 * once (no further steps) and leaves the batch at the next rebuild.  Its
 * status becomes 3; it frees its slot and memory budget.  RBSOG_EINVAL for
 * an unknown, finished or already cancelled job. */
rbsog_status rbsog_server_cancel(rbsog_server *s, int64_t job_id);
/* Free a finished or cancelled job's host data. */
rbsog_status rbsog_server_release(rbsog_server *s, int64_t job_id);
const char *rbsog_server_last_error(const rbsog_server *s);
rbsog_status rbsog_server_destroy(rbsog_server *s);

/* Description of the last error on this context (never NULL). */
const char *rbsog_last_error(const rbsog_ctx *ctx);

/* Release all device and host resources of the context (NULL is a no-op). */
rbsog_status rbsog_destroy(rbsog_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RBSOG_H */
