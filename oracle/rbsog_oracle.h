/*
 * FP64 CPU oracle for the random batch sum-of-Gaussians (RBSOG) force
 * evaluation and velocity-Verlet step.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the reference the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it; the product library never links, calls or
 * includes anything here, and nothing here includes the product's headers.
 *
 * Every function follows the paper's formulas in their plain form (no
 * blocking, no fused kernels, no precision tricks).  Where the printed
 * formula is wrong or ambiguous, the reading taken is stated at the
 * function.  Parity status per function:
 *   - all functions declared here are pinned by tests under -m "not gpu"
 *     (closed forms, Table 1, Ewald, Madelung, finite differences,
 *     invariants, brute force, chi-square).
 */
#ifndef RBSOG_ORACLE_H
#define RBSOG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* System description shared by the force routines of the oracle. */
typedef struct {
    double L[3];          /* periodic box edges                               */
    int32_t M;            /* last Gaussian index; the SOG has M+1 terms       */
    const double *omega;  /* [M+1] Gaussian weights omega_l                   */
    const double *s;      /* [M+1] Gaussian widths s_l                        */
    double rc;            /* near-field cutoff r_c                            */
    double lB;            /* Coulomb prefactor (Bjerrum length x kT)          */
    double wca_sigma;     /* WCA sigma; 0 disables the soft repulsion         */
    double wca_eps;       /* WCA epsilon                                      */
} orc_sys;

/* Core-shell approximation of the near-field kernel (Sec. 3.4): pairs with
 * r < r_in take the Gaussian sums from a Q-term Taylor series in r^2 (Eqs.
 * 3.25-3.26, with 1/r and 1/r^3 exact); pairs with r_in <= r < r_c take
 * the whole kernel from a table indexed by the b_exp low exponent bits and
 * the b_man high mantissa bits of the FP32 value of r^2, with linear
 * interpolation inside each bin. */
typedef struct {
    double r_in;          /* core radius                                      */
    int32_t Q;            /* Taylor terms of the core                         */
    int32_t b_exp;        /* exponent bits of the shell-table index           */
    int32_t b_man;        /* mantissa bits of the shell-table index           */
} orc_coreshell;

/* Energies of one force evaluation; every Coulomb term already carries lB. */
typedef struct {
    double U_near;   /* (1/2) sum_ij q_i q_j N(r_ij), r_ij < r_c              */
    double U_far;    /* U*_F: exact Fourier sum or its random-batch estimate  */
    double U_self;   /* (1/2) F_M(0) sum_i q_i^2                              */
    double U_wca;    /* soft-repulsion energy                                 */
    double K;        /* kinetic energy (only filled by the MD driver)         */
    double T;        /* instantaneous temperature 2K/(3N-3)                   */
    double U_th;     /* Nose-Hoover thermostat energy (1/2) Q xi^2 + g T0 eta  */
} orc_energies;

/* ---- sum-of-Gaussians decomposition (Sec. 2, Eqs. 2.5-2.11) ------------- */
void   orc_sog_coeffs(double b, double sigma, int32_t M, double *omega, double *s);
double orc_sog_F(const double *omega, const double *s, int32_t M, double r);
double orc_sog_dF(const double *omega, const double *s, int32_t M, double r);
double orc_sog_omega0(double b, double sigma, int32_t M, double rc);
int    orc_sog_solve(double b, double rc, int32_t M, double *sigma, double *omega0);
double orc_bsa(double b, double sigma, double r);

/* ---- Fourier side (Eqs. 3.4-3.5, 3.16-3.22) ----------------------------- */
double orc_ftilde(const double *omega, const double *s, int32_t M, double k2);
double orc_H(double s, double L, int dual);
double orc_S(const double *omega, const double *s, int32_t M, const double L[3]);
double orc_proposal_q1(int32_t m, double s0, double Ld);

/* ---- counter-based generator and the Metropolis-Hastings sampler -------- */
void    orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
int64_t orc_mh_chain(const double *omega, const double *s, int32_t M, const double L[3],
                     uint64_t seed, uint64_t chain, int64_t len, int32_t *m_out);
int64_t orc_kseq(const double *omega, const double *s, int32_t M, const double L[3],
                 uint64_t seed, int64_t n_chains, int64_t chain_len, int32_t *m_out);

/* ---- per-Gaussian independent sampling (Sec. 3.3, closing remark) ------- */
/* Gaussian l alone, normalised over k != 0, is the distribution
 * p_l(k) = e^{-s_l^2 k^2 / 4} / (prod_d H_l^d - 1); its share of the far sum
 * is S_l = w_l s_l^3 (prod_d H_l^d - 1) (S = sum_l S_l, Eq. 3.16).  Batch
 * sizes adapt to the shares: P_l = ceil(P S_l / S) for S_l > 1e-16 S, else 0
 * (that Gaussian is dropped).  Each set holds the strata in order of l, P_l
 * frequencies each, P_eff = sum_l P_l in all; the estimator weighs a
 * frequency of stratum l by S_l / P_l where the mixture sampler uses S / P.
 * orc_pg_plan fills P_l[M + 1] and S_l[M + 1] and returns P_eff (-1 on a
 * table longer than 2^20 entries).
 *
 * Frequency eta of set t: the coordinates are independent discrete Gaussians
 * p(m_d) proportional to e^{-x_d m_d^2}, x_d = (pi s_l / L_d)^2, conditioned
 * on m != 0 by choosing the first non-zero coordinate d* with its exact
 * conditional probability; coordinates before d* are 0, d* is drawn given
 * m_d* != 0, the ones after it unconditioned.  Each coordinate is drawn by
 * inverting the cumulative table T_d[j] = 1 + sum_{i=1..j} 2 e^{-x_d i^2}
 * (|m| = j, j <= jmax = ceil(sqrt(50 / x_d))), its sign from a random bit.
 * Random numbers: Philox4x64-10, key (seed, 2^63 + 2), counters (t, eta, 0, 0)
 * (two decision uniforms, the sign bits in the third word) and
 * (t, eta, 1, 0) (one uniform per coordinate).  m_out[n_sets][P_eff][3],
 * stratum_out[n_sets][P_eff] (may be NULL). */
int32_t orc_pg_plan(const double *omega, const double *s, int32_t M, const double L[3], int32_t P,
                    int32_t *P_l, double *S_l);
int orc_pg_kseq(const double *omega, const double *s, int32_t M, const double L[3], int32_t P, uint64_t seed,
                int64_t set0, int64_t n_sets, int32_t *m_out, int32_t *stratum_out);
/* Eq. 3.24 with a weight per frequency: U = (lB pi^{3/2} / (2V)) sum_eta
 * c_eta |rho(k_eta)|^2 and its force (c_eta = S / P for every eta is
 * orc_far_rb). */
void orc_far_rb_w(int64_t n, const double *q, const double *x, const orc_sys *sys, int32_t P, const int32_t *m,
                  const double *c, double *f, double *U_rb);

/* ---- cell list and near field (Sec. 3.1, Eq. 3.9 first line) ------------ */
void orc_wrap(int64_t n, double *x, const double L[3]);
int  orc_cell_list(int64_t n, const double *x, const double L[3], double rc,
                   int32_t *ncell, int32_t *cell_of, int32_t *cell_start, int32_t *perm);
void orc_near_direct(int64_t n, const double *q, const double *x, const orc_sys *sys,
                     double *f, double *U_near, double *U_wca, int32_t *nbr);
int  orc_near_cells(int64_t n, const double *q, const double *x, const orc_sys *sys,
                    double *f, double *U_near, double *U_wca, int32_t *nbr);

/* ---- far field (Eq. 3.9 second line; Eq. 3.24) ------------------------- */
int64_t orc_far_exact(int64_t n, const double *q, const double *x, const orc_sys *sys,
                      double tol, double *f, double *U_star);
void orc_rho(int64_t n, const double *q, const double *x, const double L[3],
             int32_t P, const int32_t *m, double *rho);
void orc_far_rb(int64_t n, const double *q, const double *x, const orc_sys *sys,
                double S, int32_t P, const int32_t *m, double *f, double *U_rb, double *rho);
double orc_self_energy(int64_t n, const double *q, const orc_sys *sys);
/* The core-shell kernel at one squared distance: g = force factor
 * 1/r^3 - 2 sum_l w_l/s_l^2 e^{-r^2/s_l^2} and n = 1/r - F_M(r) as the
 * scheme approximates them.  Returns -1 when r2 is outside [0, r_c^2) or the
 * 2^b_exp octaves of the table, starting at the octave of r_in^2, do not
 * reach r_c^2. */
int orc_coreshell_eval(const orc_sys *sys, const orc_coreshell *cs, double r2, double *g, double *n);
/* Configurational virial tensor W_ab = -dU/d eps_ab (row-major W[9]) of the
 * near field (+ WCA) and the far field: the random-batch estimator on the
 * k-set m (P > 0, weights of Eq. 3.24) or the exact Fourier sum (P == 0). */
int orc_virial(int64_t n, const double *q, const double *x, const orc_sys *sys, double S, int32_t P,
               const int32_t *m, double W[9]);
/* Near field (+ WCA, exact) with the core-shell kernel; O(N^2) pair scan.
 * Returns -1 as orc_coreshell_eval for an uncovered table. */
int orc_near_coreshell(int64_t n, const double *q, const double *x, const orc_sys *sys, const orc_coreshell *cs,
                       double *f, double *U_near, double *U_wca);
/* Zero-frequency (boundary) term of the far field (Sec. 3.2, "Analysis of
 * the zero-frequency mode"): kind 0 tinfoil (nothing), 1 spherical infinite
 * boundary U0 = (2 pi / 3V) |M|^2 (Eq. 3.14), 2 planar infinite boundary
 * along z U0 = (2 pi / V) M_z^2 (Eq. 3.15), with M = sum_i q_i r_i over the given positions,
 * times lB.  Adds -dU0/dr_i to f when f is not NULL; returns U0. */
double orc_boundary(int64_t n, const double *q, const double *x, const double L[3], double lB, int32_t kind,
                    double *f);
int orc_forces_sample(int64_t n, const double *q, const double *x, const orc_sys *sys, double S,
                      int32_t P, const int32_t *m, int64_t ns, const int64_t *idx, double *f);

/* ---- total force and the MD driver (Algorithm 1) ------------------------ */
int  orc_forces(int64_t n, const double *q, const double *x, const orc_sys *sys,
                double S, int32_t P, const int32_t *m, double *f, orc_energies *e);
int  orc_md(int64_t n, const double *q, double *x, double *v, double *f,
            const orc_sys *sys, double S, int32_t P, const int32_t *kseq,
            int64_t nsteps, double dt, double mass, double T0, double tau,
            int have_force, orc_energies *e_steps);
/* As orc_md with a thermostat choice: 0 Berendsen rescale (tau > 0), 1
 * Langevin dynamics with friction 1/tau in the BAOAB splitting; the noise of
 * particle i in the step with step counter step0 + t is
 * orc_langevin_noise(seed, step0 + t, i). */
int orc_md_thermo(int64_t n, const double *q, double *x, double *v, double *f,
                  const orc_sys *sys, double S, int32_t P, const int32_t *kseq,
                  int64_t nsteps, double dt, double mass, double T0, double tau,
                  int have_force, orc_energies *e_steps, int32_t thermostat, uint64_t seed, int64_t step0);
/* Three standard normals for the Langevin noise: Philox4x64-10 with key
 * (seed, 2^63 + 1), counter (t, i, 0, 0), Box-Muller. */
void orc_langevin_noise(uint64_t seed, int64_t t, int64_t i, double z[3]);

/* ---- radial distribution functions (Appendix A) ----------------------- */
int  orc_rdf_counts(int64_t n, const double *q, const double *x, double L, int32_t nbins, uint64_t *counts);
void orc_rdf_g(const uint64_t *counts, int32_t nbins, double L, int64_t n_pos, int64_t n_neg, double *g);

/* ---- time-correlation observables (Appendix A) ------------------------- */
/* MSD eta(t) = <|r(t0 + t) - r(t0)|^2> and VACF <v(t0) . v(t0 + t)> over the
 * frames x[f][n][3] (positions folded into [0, L)) and v[f][n][3], f <
 * n_frames, averaged over the particles and the time origins t0 = 0,
 * origin_every, 2 origin_every, ... with t0 + t < n_frames; lags t < n_lags in
 * frames.  Positions are unwrapped by adding the minimum-image displacement
 * between consecutive frames.  count[t] = origins that reached lag t;
 * msd[t] = vacf[t] = 0 where count[t] = 0.  Returns -1 on bad sizes. */
int orc_msd_vacf(int64_t n, int64_t n_frames, const double *x, const double *v, const double *L,
                 int32_t n_lags, int32_t origin_every, double *msd, double *vacf, int64_t *count);

/* Pressure tensor of Appendix A, P_ab = (1/V) sum_i (m v_ia v_ib + r_ia f_ib),
 * the second sum read as the configurational virial W_ab of orc_virial. */
int orc_pressure(int64_t n, const double *q, const double *x, const double *v, double mass,
                 const orc_sys *sys, double S, int32_t P, const int32_t *kset, double *Pt);

/* Green-Kubo shear viscosity of Appendix A: C = V/(6 T) sum_{a<=b} of the
 * integral of <dP_ab(t) dP_ab(0)>, dP the fluctuation of the series
 * Pt[s][9] (row-major tensors, s < n_samples, spacing dt) about its mean,
 * each autocorrelation averaged over all origins, acf[t] = the sum over the
 * six components at lag t < max_lag, the integral by the trapezoid rule up
 * to lag max_lag - 1.  Returns -1 on bad sizes. */
int orc_green_kubo(int64_t n_samples, const double *Pt, double dt, double V, double T, int32_t max_lag,
                   double *acf, double *C);

/* Heat flux J[3] of Appendix A for the current state: per-atom energies
 * (kinetic, half of each near and WCA pair energy, minus the self term, the
 * far energy split over atoms) times velocities plus the per-atom virials
 * (half of r_ij f_ij per ordered pair; the random-batch far virial split over
 * atoms) contracted with the velocities, over V.  P = 0: no far term.
 * e_atom[n], W_atom[n][9] returned when non-NULL.  -1 if fewer than 3 cells
 * per side. */
int orc_heat_flux(int64_t n, const double *q, const double *x, const double *v, double mass,
                  const orc_sys *sys, double S, int32_t P, const int32_t *m, double J[3], double *e_atom,
                  double *W_atom);
/* Green-Kubo heat conductivity V/(3 k_B T^2) * integral <J(0).J(t)> dt. */
int orc_green_kubo_heat(int64_t n_samples, const double *J, double dt, double V, double T, int32_t max_lag,
                        double *acf, double *C);

int  orc_num_threads(void);
int  orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
