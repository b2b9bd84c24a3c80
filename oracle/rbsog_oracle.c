/*
 * FP64 CPU oracle for the random batch sum-of-Gaussians (RBSOG) method of
 * Liang, Xu, Xu and Zhao (arXiv:2205.13824).
 *
 * TEST INFRASTRUCTURE ONLY: the reference that the CUDA path is checked against.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg load this
 * library.  It shares no code with the product library (no headers, no
 * helpers, no generated tables).
 *
 * Style: every routine is the plain definition or the paper's algorithm in
 * the paper's order, in double precision, with loops a reader can check
 * against the formulas.  OpenMP only splits independent outer loops; every
 * sum over particles or frequencies is taken sequentially in index order, so
 * results do not depend on the thread count.  Build with -ffp-contract=off
 * so that x86 and Arm hosts give the same bits.
 *
 * Readings of the paper taken here (each is justified where it is used):
 *   near force   -grad of N(r) = 1/r - F_M(r): (1/r^3 - 2 sum w_l/s_l^2 e^{-r^2/s_l^2}) r_ij
 *                (Eq. 3.9 prints half of this bracket);
 *   far force    F_i = -sum_k (q_i k/V) F~(k) Im(e^{-ik.r_i} rho(k)) (Eq. 3.9 and
 *                Eq. 3.24 print the opposite sign; -grad of U*_F fixes it);
 *   C1 condition 1/r_c^2 + F'(r_c) = 0 (Eq. 2.10 prints a minus);
 *   omega_0      Eq. 2.11 with F restricted to l = 1..M;
 *   H_l^d dual   sqrt(L^2/(pi s^2)) sum_m e^{-m^2 L^2/s^2} (Eq. 3.17 prints pi^2 in the exponent);
 *   proposal     q(m) = (1/2)[erf((m+1/2) pi s_0/L) - erf((m-1/2) pi s_0/L)] (Sec. 3.3
 *                prints an extra factor 1/2 inside erf for m != 0);
 *   self energy  (1/2) F_M(0) sum q^2 with the modified omega_0;
 *   m = 0        a zero proposal is a rejection (the chain repeats its state);
 *   RDF          Appendix A per sign pair, rho = number density of the second
 *                species (N^2, not N(N-1), normalisation), distances measured on
 *                positions quantised to L 2^-32 per axis (cubic box).
 */
#include "rbsog_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the later parallel loops (n >= 1); the previous count is returned. */
int orc_set_num_threads(int n) {
    const int old = orc_num_threads();
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return old;
}

/* ------------------------------------------------------------------------
 * Sum-of-Gaussians decomposition (Sec. 2, Eqs. 2.5-2.11).
 * ------------------------------------------------------------------------ */

/* Eq. 2.9: w_l = (pi/2)^{-1/2} b^{-l} ln(b) / sigma,  s_l = sqrt(2) b^l sigma,
 * for l = 0..M.  omega[0] is the unmodified bilateral-series weight; the
 * caller replaces it by the C0/C1 value of Eq. 2.11. */
void orc_sog_coeffs(double b, double sigma, int32_t M, double *omega, double *s) {
    for (int32_t l = 0; l <= M; ++l) {
        omega[l] = sqrt(2.0 / M_PI) * pow(b, -(double)l) * log(b) / sigma;
        s[l] = sqrt(2.0) * pow(b, (double)l) * sigma;
    }
}

/* Eq. 2.8: F_M(r) = sum_{l=0}^{M} w_l exp(-r^2 / s_l^2). */
double orc_sog_F(const double *omega, const double *s, int32_t M, double r) {
    double acc = 0.0;
    for (int32_t l = 0; l <= M; ++l) acc += omega[l] * exp(-r * r / (s[l] * s[l]));
    return acc;
}

/* d/dr of Eq. 2.8. */
double orc_sog_dF(const double *omega, const double *s, int32_t M, double r) {
    double acc = 0.0;
    for (int32_t l = 0; l <= M; ++l)
        acc += omega[l] * (-2.0 * r / (s[l] * s[l])) * exp(-r * r / (s[l] * s[l]));
    return acc;
}

/* Eq. 2.11, read with F restricted to the Gaussians l = 1..M (the l = 0 term
 * is the unknown): w_0 = e^{r_c^2/s_0^2} [1/r_c - sum_{l>=1} w_l e^{-r_c^2/s_l^2}].
 * This makes r_c F_M(r_c) = 1 exactly (the C0 condition). */
double orc_sog_omega0(double b, double sigma, int32_t M, double rc) {
    double *om = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    double *s = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    orc_sog_coeffs(b, sigma, M, om, s);
    double tail = 0.0;
    for (int32_t l = 1; l <= M; ++l) tail += om[l] * exp(-rc * rc / (s[l] * s[l]));
    double w0 = exp(rc * rc / (s[0] * s[0])) * (1.0 / rc - tail);
    free(om);
    free(s);
    return w0;
}

/* C1 residual g(sigma) = 1 + r_c^2 F_M'(r_c) with w_0 = w_0(sigma) from Eq. 2.11.
 * The C1 condition of Eq. 2.10 is read as 1/r_c^2 + F'(r_c) = 0, i.e. the
 * derivative of N = 1/r - F vanishes at r_c (the printed sign admits no root
 * for decreasing Gaussians). */
static double c1_residual(double b, double sigma, int32_t M, double rc, double *w0_out) {
    double *om = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    double *s = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    orc_sog_coeffs(b, sigma, M, om, s);
    om[0] = orc_sog_omega0(b, sigma, M, rc);
    double g = 1.0 + rc * rc * orc_sog_dF(om, s, M, rc);
    if (w0_out) *w0_out = om[0];
    free(om);
    free(s);
    return g;
}

/* Joint C0/C1 solve (Sec. 2 and the parameter procedure of Sec. 4.1): for
 * given b, r_c and M find sigma such that C1 holds once w_0 satisfies C0.
 * Roots are bracketed on a log grid sigma in [0.05 r_c, 2 r_c] and bisected;
 * of the roots found, the one whose w_0 is closest to the bilateral-series
 * weight (the paper tunes w_0, it does not replace it) is returned.
 * Returns 0 on success, -1 if no root exists in the range. */
int orc_sog_solve(double b, double rc, int32_t M, double *sigma_out, double *omega0_out) {
    const int NG = 3000;
    double lo = 0.05 * rc, hi = 2.0 * rc;
    double best_sig = -1.0, best_w0 = 0.0, best_dev = 1e300;
    double s_prev = lo, g_prev = c1_residual(b, lo, M, rc, NULL);
    for (int i = 1; i <= NG; ++i) {
        double sg = lo * pow(hi / lo, (double)i / NG);
        double g = c1_residual(b, sg, M, rc, NULL);
        if ((g_prev < 0.0) != (g < 0.0)) {
            double a = s_prev, c = sg, ga = g_prev;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (a + c);
                double gm = c1_residual(b, mid, M, rc, NULL);
                if ((gm < 0.0) == (ga < 0.0)) { a = mid; ga = gm; } else { c = mid; }
                if (c - a <= 1e-16 * c) break;
            }
            double root = 0.5 * (a + c), w0;
            c1_residual(b, root, M, rc, &w0);
            double bsa_w0 = sqrt(2.0 / M_PI) * log(b) / root;
            double dev = fabs(w0 / bsa_w0 - 1.0);
            if (dev < best_dev) { best_dev = dev; best_sig = root; best_w0 = w0; }
        }
        s_prev = sg;
        g_prev = g;
    }
    if (best_sig < 0.0) return -1;
    *sigma_out = best_sig;
    *omega0_out = best_w0;
    return 0;
}

/* Eq. 2.5: bilateral series (2 ln b / sqrt(2 pi sigma^2)) sum_{l in Z} b^{-l}
 * exp(-(r/(b^l sigma))^2 / 2), summed over every l whose term is not
 * negligible. */
double orc_bsa(double b, double sigma, double r) {
    double acc = 0.0;
    for (int l = -2000; l <= 20000; ++l) {
        double w = pow(b, (double)l) * sigma;
        double arg = 0.5 * (r / w) * (r / w);
        if (arg > 745.0) continue;
        double t = pow(b, -(double)l) * exp(-arg);
        acc += t;
        if (l > 0 && t < 1e-22 * acc) break;
    }
    return 2.0 * log(b) / sqrt(2.0 * M_PI * sigma * sigma) * acc;
}

/* ------------------------------------------------------------------------
 * Fourier side (Sec. 3.1, Eq. 3.5; Sec. 3.3, Eqs. 3.16-3.17).
 * ------------------------------------------------------------------------ */

/* Eq. 3.5: F~(k) = pi^{3/2} sum_l w_l s_l^3 exp(-s_l^2 k^2 / 4), as a function of k^2. */
double orc_ftilde(const double *omega, const double *s, int32_t M, double k2) {
    double acc = 0.0;
    for (int32_t l = 0; l <= M; ++l)
        acc += omega[l] * s[l] * s[l] * s[l] * exp(-s[l] * s[l] * k2 / 4.0);
    return pow(M_PI, 1.5) * acc;
}

/* Eq. 3.17: H_l^d = sum_{m in Z} exp(-s^2 pi^2 m^2 / L^2).
 * dual = 0: that direct sum.  dual = 1: its Poisson dual
 * sqrt(L^2/(pi s^2)) sum_m exp(-m^2 L^2 / s^2) (the printed dual carries a
 * spurious pi^2 in the exponent).  dual < 0: whichever converges faster. */
double orc_H(double s, double L, int dual) {
    if (dual < 0) dual = (s < L) ? 1 : 0;
    double acc = 1.0;
    if (!dual) {
        double a = s * s * M_PI * M_PI / (L * L);
        for (long m = 1; m < 100000000L; ++m) {
            double t = exp(-a * (double)m * (double)m);
            acc += 2.0 * t;
            if (t < 1e-300 || t < 1e-22 * acc) break;
        }
        return acc;
    }
    double a = L * L / (s * s);
    for (long m = 1; m < 100000000L; ++m) {
        double t = exp(-a * (double)m * (double)m);
        acc += 2.0 * t;
        if (t < 1e-300 || t < 1e-22 * acc) break;
    }
    return sqrt(L * L / (M_PI * s * s)) * acc;
}

/* Eq. 3.16: S = pi^{-3/2} sum_{k != 0} F~(k) = sum_l w_l s_l^3 (prod_d H_l^d - 1). */
double orc_S(const double *omega, const double *s, int32_t M, const double L[3]) {
    double acc = 0.0;
    for (int32_t l = 0; l <= M; ++l) {
        double prod = orc_H(s[l], L[0], -1) * orc_H(s[l], L[1], -1) * orc_H(s[l], L[2], -1);
        acc += omega[l] * s[l] * s[l] * s[l] * (prod - 1.0);
    }
    return acc;
}

/* Proposal mass of one coordinate (Sec. 3.3, Eqs. 3.19-3.22): the normal N(0, (L_d/(s_0 pi))^2/2)
 * integrated over [m - 1/2, m + 1/2]:
 * q(m) = (1/2)[erf((m + 1/2) pi s_0 / L_d) - erf((m - 1/2) pi s_0 / L_d)];
 * for m = 0 this is erf(pi s_0 / (2 L_d)), as printed. */
double orc_proposal_q1(int32_t m, double s0, double Ld) {
    double a = M_PI * s0 / Ld;
    if (m == 0) return erf(0.5 * a);
    return 0.5 * (erf(((double)m + 0.5) * a) - erf(((double)m - 0.5) * a));
}

/* ------------------------------------------------------------------------
 * Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies with the
 * published multipliers and Weyl key increments.
 * ------------------------------------------------------------------------ */
void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform on [0, 1). */
static double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Unnormalised target mass p(m) proportional to F~(k(m)), k = 2 pi m / L (Eq. 3.18). */
static double target_p(const double *omega, const double *s, int32_t M, const double L[3],
                       const int32_t m[3]) {
    double k2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double kd = 2.0 * M_PI * (double)m[d] / L[d];
        k2 += kd * kd;
    }
    double acc = 0.0;
    for (int32_t l = 0; l <= M; ++l)
        acc += omega[l] * s[l] * s[l] * s[l] * exp(-s[l] * s[l] * k2 / 4.0);
    return acc;
}

/* One independence Metropolis-Hastings chain over m in Z^3 \ {0} (Sec. 3.3).
 *
 * Iteration j draws two Philox blocks with key (seed, chain): counter
 * (j, 0, 0, 0) gives four uniforms, turned by Box-Muller into the proposal
 * normals (u0,u1) -> (z_x, z_y), (u2,u3) -> z_z; counter (j, 1, 0, 0) gives
 * the acceptance uniform from its first word.  The proposal is
 * m*_d = round(z_d L_d / (sqrt(2) pi s_0)), rounding half away from zero.
 * The first non-zero proposal starts the chain and is emitted; afterwards
 * every iteration emits the chain state after the accept/reject decision,
 * accepting when u < p(m*) q(m) / (p(m) q(m*)).  A zero proposal has p = 0 and
 * is rejected.  Returns the number of iterations used, or -1 if the chain
 * could not be started within the iteration cap. */
int64_t orc_mh_chain(const double *omega, const double *s, int32_t M, const double L[3],
                     uint64_t seed, uint64_t chain, int64_t len, int32_t *m_out) {
    const double s0 = s[0];
    double sd[3];
    for (int d = 0; d < 3; ++d) sd[d] = L[d] / (sqrt(2.0) * M_PI * s0);
    uint64_t key[2] = {seed, chain};
    int32_t cur[3] = {0, 0, 0};
    double p_cur = 0.0, q_cur = 0.0;
    int have = 0;
    int64_t emitted = 0, j = 0;
    const int64_t cap = 64 * len + 4096;
    while (emitted < len) {
        if (j >= cap) return -1;
        uint64_t ca[4] = {(uint64_t)j, 0, 0, 0}, cb[4] = {(uint64_t)j, 1, 0, 0}, ra[4], rb[4];
        orc_philox4x64_10(ca, key, ra);
        orc_philox4x64_10(cb, key, rb);
        double r01 = sqrt(-2.0 * log(1.0 - u01(ra[0])));
        double r23 = sqrt(-2.0 * log(1.0 - u01(ra[2])));
        double z[3];
        z[0] = r01 * cos(2.0 * M_PI * u01(ra[1]));
        z[1] = r01 * sin(2.0 * M_PI * u01(ra[1]));
        z[2] = r23 * cos(2.0 * M_PI * u01(ra[3]));
        int32_t mp[3];
        for (int d = 0; d < 3; ++d) mp[d] = (int32_t)round(z[d] * sd[d]);
        int zero = (mp[0] == 0 && mp[1] == 0 && mp[2] == 0);
        ++j;
        if (!have) {
            if (zero) continue;
            memcpy(cur, mp, sizeof cur);
            p_cur = target_p(omega, s, M, L, cur);
            q_cur = orc_proposal_q1(cur[0], s0, L[0]) * orc_proposal_q1(cur[1], s0, L[1]) *
                    orc_proposal_q1(cur[2], s0, L[2]);
            have = 1;
        } else if (!zero) {
            double p_new = target_p(omega, s, M, L, mp);
            double q_new = orc_proposal_q1(mp[0], s0, L[0]) * orc_proposal_q1(mp[1], s0, L[1]) *
                           orc_proposal_q1(mp[2], s0, L[2]);
            double ratio = (p_new * q_cur) / (p_cur * q_new);
            if (u01(rb[0]) < ratio) {
                memcpy(cur, mp, sizeof cur);
                p_cur = p_new;
                q_cur = q_new;
            }
        }
        m_out[3 * emitted + 0] = cur[0];
        m_out[3 * emitted + 1] = cur[1];
        m_out[3 * emitted + 2] = cur[2];
        ++emitted;
    }
    return j;
}

/* Algorithm 1 (pre-sampled frequency sequence), with the sampling split over
 * independent chains as in the paper's parallel sampling (Sec. 3.4): chain c
 * fills entries [c * chain_len, (c + 1) * chain_len) of the sequence.
 * Returns the total iteration count, or -1 if a chain failed to start. */
int64_t orc_kseq(const double *omega, const double *s, int32_t M, const double L[3],
                 uint64_t seed, int64_t n_chains, int64_t chain_len, int32_t *m_out) {
    int64_t total = 0;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total) reduction(| : failed)
    for (int64_t c = 0; c < n_chains; ++c) {
        int64_t it = orc_mh_chain(omega, s, M, L, seed, (uint64_t)c, chain_len,
                                  m_out + 3 * c * chain_len);
        if (it < 0) failed = 1; else total += it;
    }
    return failed ? -1 : total;
}

/* ------------------------------------------------------------------------
 * Cell list and near field.
 * ------------------------------------------------------------------------ */

/* Fold coordinates into [0, L_d): x - L floor(x / L), with a result equal to
 * L (possible after rounding) mapped to 0. */
void orc_wrap(int64_t n, double *x, const double L[3]) {
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            double v = x[3 * i + d];
            v = v - L[d] * floor(v / L[d]);
            if (v >= L[d]) v = 0.0;
            x[3 * i + d] = v;
        }
}

/* Cells of side h_d = L_d / n_d with n_d = floor(L_d / r_c) >= 3 (the cell
 * list that makes the near-field sum of Eq. 3.9 O(N), Sec. 3.4).  A particle
 * at wrapped x goes to c_d = floor(x_d / h_d) (clamped to [0, n_d - 1]), cell
 * id (c_z n_y + c_y) n_x + c_x.  Members of a cell are listed in increasing
 * particle index.  Returns -1 if some n_d < 3. */
int orc_cell_list(int64_t n, const double *x, const double L[3], double rc,
                  int32_t *ncell, int32_t *cell_of, int32_t *cell_start, int32_t *perm) {
    double h[3];
    for (int d = 0; d < 3; ++d) {
        ncell[d] = (int32_t)floor(L[d] / rc);
        if (ncell[d] < 3) return -1;
        h[d] = L[d] / (double)ncell[d];
    }
    int64_t nc = (int64_t)ncell[0] * ncell[1] * ncell[2];
    for (int64_t c = 0; c <= nc; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t c3[3];
        for (int d = 0; d < 3; ++d) {
            int32_t c = (int32_t)floor(x[3 * i + d] / h[d]);
            if (c >= ncell[d]) c = ncell[d] - 1;
            if (c < 0) c = 0;
            c3[d] = c;
        }
        cell_of[i] = (c3[2] * ncell[1] + c3[1]) * ncell[0] + c3[0];
        cell_start[cell_of[i] + 1] += 1;
    }
    for (int64_t c = 0; c < nc; ++c) cell_start[c + 1] += cell_start[c];
    int32_t *fill = (int32_t *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = cell_of[i];
        perm[cell_start[c] + fill[c]] = (int32_t)i;
        fill[c] += 1;
    }
    free(fill);
    return 0;
}

/* One ordered pair (i <- j) of the near field with separation d = r_i - r_j
 * (minimum image) and r2 = |d|^2 < r_c^2.
 * Coulomb part: N(r) = 1/r - F_M(r) (Eq. 2.7); its force on i is
 * -dN/dr d/r = (1/r^3 - 2 sum_l w_l / s_l^2 e^{-r^2/s_l^2}) d, times q_i q_j lB.
 * WCA: 4 eps [(sig/r)^12 - (sig/r)^6] + eps for r < 2^{1/6} sig.
 * Energies are halved because every pair is visited from both ends. */
static void near_pair(const orc_sys *sys, double qi, double qj, const double d[3], double r2,
                      double fi[3], double *un, double *uw) {
    double r = sqrt(r2);
    double gsum = 0.0, fsum = 0.0;
    for (int32_t l = 0; l <= sys->M; ++l) {
        double e = exp(-r2 / (sys->s[l] * sys->s[l]));
        fsum += sys->omega[l] * e;
        gsum += sys->omega[l] / (sys->s[l] * sys->s[l]) * e;
    }
    double qq = sys->lB * qi * qj;
    double g = qq * (1.0 / (r2 * r) - 2.0 * gsum);
    fi[0] += g * d[0];
    fi[1] += g * d[1];
    fi[2] += g * d[2];
    *un += 0.5 * qq * (1.0 / r - fsum);
    if (sys->wca_sigma > 0.0) {
        double rcut2 = pow(2.0, 1.0 / 3.0) * sys->wca_sigma * sys->wca_sigma;
        if (r2 < rcut2) {
            double sr2 = sys->wca_sigma * sys->wca_sigma / r2;
            double sr6 = sr2 * sr2 * sr2;
            double gw = 24.0 * sys->wca_eps * (2.0 * sr6 * sr6 - sr6) / r2;
            fi[0] += gw * d[0];
            fi[1] += gw * d[1];
            fi[2] += gw * d[2];
            *uw += 0.5 * (4.0 * sys->wca_eps * (sr6 * sr6 - sr6) + sys->wca_eps);
        }
    }
}

/* Minimum-image separation r_i - r_j: d = x_i - x_j, then d - L rint(d / L). */
static double min_image(const double *xi, const double *xj, const double L[3], double d[3]) {
    for (int k = 0; k < 3; ++k) {
        double t = xi[k] - xj[k];
        t = t - L[k] * rint(t / L[k]);
        d[k] = t;
    }
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* Near field by the O(N^2) minimum-image scan over all pairs (r_c < L/2).
 * f is overwritten; nbr[i] counts the j with |r_ij| < r_c. */
void orc_near_direct(int64_t n, const double *q, const double *x, const orc_sys *sys,
                     double *f, double *U_near, double *U_wca, int32_t *nbr) {
    double *un = (double *)calloc((size_t)n, sizeof(double));
    double *uw = (double *)calloc((size_t)n, sizeof(double));
    const double rc2 = sys->rc * sys->rc;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            double r2 = min_image(x + 3 * i, x + 3 * j, sys->L, d);
            if (r2 < rc2) {
                near_pair(sys, q[i], q[j], d, r2, fi, &un[i], &uw[i]);
                ++cnt;
            }
        }
        f[3 * i + 0] = fi[0];
        f[3 * i + 1] = fi[1];
        f[3 * i + 2] = fi[2];
        if (nbr) nbr[i] = cnt;
    }
    double a = 0.0, b = 0.0;
    for (int64_t i = 0; i < n; ++i) { a += un[i]; b += uw[i]; }
    *U_near = a;
    *U_wca = b;
    free(un);
    free(uw);
}

/* Same near field, visiting only the 27 cells around each particle's cell
 * (cell side >= r_c, at least 3 cells per side so the 27 are distinct).
 * Returns -1 if the box has fewer than 3 cells per side. */
int orc_near_cells(int64_t n, const double *q, const double *x, const orc_sys *sys,
                   double *f, double *U_near, double *U_wca, int32_t *nbr) {
    int32_t nc3[3];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t ncmax = 1;
    for (int d = 0; d < 3; ++d) ncmax *= (int64_t)floor(sys->L[d] / sys->rc) > 0 ? (int64_t)floor(sys->L[d] / sys->rc) : 1;
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncmax + 1));
    if (orc_cell_list(n, x, sys->L, sys->rc, nc3, cell_of, start, perm) != 0) {
        free(cell_of); free(perm); free(start);
        return -1;
    }
    double *un = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *uw = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    const double rc2 = sys->rc * sys->rc;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = cell_of[i];
        int32_t cx = c % nc3[0], cy = (c / nc3[0]) % nc3[1], cz = c / (nc3[0] * nc3[1]);
        double fi[3] = {0.0, 0.0, 0.0};
        int32_t cnt = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int32_t ox = (cx + dx + nc3[0]) % nc3[0];
                    int32_t oy = (cy + dy + nc3[1]) % nc3[1];
                    int32_t oz = (cz + dz + nc3[2]) % nc3[2];
                    int32_t o = (oz * nc3[1] + oy) * nc3[0] + ox;
                    for (int32_t t = start[o]; t < start[o + 1]; ++t) {
                        int32_t j = perm[t];
                        if (j == i) continue;
                        double d[3];
                        double r2 = min_image(x + 3 * i, x + 3 * j, sys->L, d);
                        if (r2 < rc2) {
                            near_pair(sys, q[i], q[j], d, r2, fi, &un[i], &uw[i]);
                            ++cnt;
                        }
                    }
                }
        f[3 * i + 0] = fi[0];
        f[3 * i + 1] = fi[1];
        f[3 * i + 2] = fi[2];
        if (nbr) nbr[i] = cnt;
    }
    double a = 0.0, b = 0.0;
    for (int64_t i = 0; i < n; ++i) { a += un[i]; b += uw[i]; }
    *U_near = a;
    *U_wca = b;
    free(un); free(uw); free(cell_of); free(perm); free(start);
    return 0;
}

/* ------------------------------------------------------------------------
 * Far field.
 * ------------------------------------------------------------------------ */

/* rho(k_eta) = sum_j q_j e^{i k_eta . r_j} (Eq. 3.4), k = 2 pi m / L, for
 * the P integer vectors m; output interleaved (Re, Im). */
void orc_rho(int64_t n, const double *q, const double *x, const double L[3],
             int32_t P, const int32_t *m, double *rho) {
#pragma omp parallel for schedule(static)
    for (int32_t e = 0; e < P; ++e) {
        double k[3];
        for (int d = 0; d < 3; ++d) k[d] = 2.0 * M_PI * (double)m[3 * e + d] / L[d];
        double re = 0.0, im = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double th = k[0] * x[3 * j] + k[1] * x[3 * j + 1] + k[2] * x[3 * j + 2];
            re += q[j] * cos(th);
            im += q[j] * sin(th);
        }
        rho[2 * e] = re;
        rho[2 * e + 1] = im;
    }
}

/* Exact far field with tinfoil boundary (k = 0 dropped, Sec. 3.2):
 *   U*_F = sum_{k != 0} F~(k) |rho(k)|^2 / (2V)                  (Eq. 3.7)
 *   F_i  = -sum_{k != 0} (q_i k / V) F~(k) Im(e^{-i k.r_i} rho(k))
 * (the sign is that of -grad U*_F).  Terms with exp(-s_0^2 k^2/4) < tol are
 * dropped.  k and -k give equal terms, so the sum runs over the half space
 * (m_x > 0, or m_x = 0 and m_y > 0, or m_x = m_y = 0 and m_z > 0) and is
 * doubled.  f is overwritten.  Returns the number of half-space vectors. */
int64_t orc_far_exact(int64_t n, const double *q, const double *x, const orc_sys *sys,
                      double tol, double *f, double *U_star) {
    const double V = sys->L[0] * sys->L[1] * sys->L[2];
    double kcut = 2.0 * sqrt(log(1.0 / tol)) / sys->s[0];
    int32_t mm[3];
    for (int d = 0; d < 3; ++d) mm[d] = (int32_t)ceil(kcut * sys->L[d] / (2.0 * M_PI));
    int64_t cap = (int64_t)(2 * mm[0] + 1) * (2 * mm[1] + 1) * (2 * mm[2] + 1);
    int32_t *mlist = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)cap);
    int64_t nk = 0;
    for (int32_t a = 0; a <= mm[0]; ++a)
        for (int32_t b = -mm[1]; b <= mm[1]; ++b)
            for (int32_t c = -mm[2]; c <= mm[2]; ++c) {
                int half = (a > 0) || (a == 0 && b > 0) || (a == 0 && b == 0 && c > 0);
                if (!half) continue;
                double kx = 2.0 * M_PI * a / sys->L[0], ky = 2.0 * M_PI * b / sys->L[1],
                       kz = 2.0 * M_PI * c / sys->L[2];
                if (kx * kx + ky * ky + kz * kz > kcut * kcut) continue;
                mlist[3 * nk] = a;
                mlist[3 * nk + 1] = b;
                mlist[3 * nk + 2] = c;
                ++nk;
            }
    double *rho = (double *)malloc(sizeof(double) * 2 * (size_t)(nk > 0 ? nk : 1));
    double *ft = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    orc_rho(n, q, x, sys->L, (int32_t)nk, mlist, rho);
    double U = 0.0;
    for (int64_t e = 0; e < nk; ++e) {
        double k2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double kd = 2.0 * M_PI * mlist[3 * e + d] / sys->L[d];
            k2 += kd * kd;
        }
        ft[e] = orc_ftilde(sys->omega, sys->s, sys->M, k2);
        U += 2.0 * ft[e] * (rho[2 * e] * rho[2 * e] + rho[2 * e + 1] * rho[2 * e + 1]) / (2.0 * V);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int64_t e = 0; e < nk; ++e) {
            double k[3];
            for (int d = 0; d < 3; ++d) k[d] = 2.0 * M_PI * mlist[3 * e + d] / sys->L[d];
            double th = k[0] * x[3 * i] + k[1] * x[3 * i + 1] + k[2] * x[3 * i + 2];
            /* Im(e^{-i th} (A + iB)) = cos(th) B - sin(th) A */
            double im = cos(th) * rho[2 * e + 1] - sin(th) * rho[2 * e];
            double g = -2.0 * q[i] / V * ft[e] * im;
            fi[0] += g * k[0];
            fi[1] += g * k[1];
            fi[2] += g * k[2];
        }
        f[3 * i + 0] = sys->lB * fi[0];
        f[3 * i + 1] = sys->lB * fi[1];
        f[3 * i + 2] = sys->lB * fi[2];
    }
    *U_star = sys->lB * U;
    free(mlist); free(rho); free(ft);
    return nk;
}

/* Random-batch far field (Sec. 3.3, Eq. 3.24), for the P sampled vectors m:
 *   F*_i = -(S / P) sum_eta (pi^{3/2} q_i k_eta / V) Im(e^{-i k_eta.r_i} rho(k_eta))
 * (sign of -grad U*_F, as in the exact sum), and the matching unbiased energy
 *   U*_RB = (pi^{3/2} S / (2 P V)) sum_eta |rho(k_eta)|^2
 * (E over k ~ F~(k)/(pi^{3/2} S) of pi^{3/2} S |rho|^2/(2V) is U*_F).
 * f is overwritten; rho (2P values) is returned when non-NULL. */
void orc_far_rb(int64_t n, const double *q, const double *x, const orc_sys *sys,
                double S, int32_t P, const int32_t *m, double *f, double *U_rb, double *rho_out) {
    const double V = sys->L[0] * sys->L[1] * sys->L[2];
    const double c = pow(M_PI, 1.5) * S / ((double)P * V);
    double *rho = (double *)malloc(sizeof(double) * 2 * (size_t)(P > 0 ? P : 1));
    orc_rho(n, q, x, sys->L, P, m, rho);
    double U = 0.0;
    for (int32_t e = 0; e < P; ++e) U += rho[2 * e] * rho[2 * e] + rho[2 * e + 1] * rho[2 * e + 1];
    *U_rb = sys->lB * 0.5 * c * U;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int32_t e = 0; e < P; ++e) {
            double k[3];
            for (int d = 0; d < 3; ++d) k[d] = 2.0 * M_PI * (double)m[3 * e + d] / sys->L[d];
            double th = k[0] * x[3 * i] + k[1] * x[3 * i + 1] + k[2] * x[3 * i + 2];
            double im = cos(th) * rho[2 * e + 1] - sin(th) * rho[2 * e];
            fi[0] += k[0] * im;
            fi[1] += k[1] * im;
            fi[2] += k[2] * im;
        }
        double g = -sys->lB * q[i] * c;
        f[3 * i + 0] = g * fi[0];
        f[3 * i + 1] = g * fi[1];
        f[3 * i + 2] = g * fi[2];
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * 2 * (size_t)P);
    free(rho);
}

/* Total force on a subset of particles only (idx[0..ns)), for checks at sizes
 * where the O(N) sweep over all particles is affordable but N per-particle
 * force sums are not.  Near field: minimum-image scan over the 27 cells
 * around each sampled particle; far field: Eq. 3.24 with rho from all
 * particles.  f is [ns][3]. */
int orc_forces_sample(int64_t n, const double *q, const double *x, const orc_sys *sys, double S,
                      int32_t P, const int32_t *m, int64_t ns, const int64_t *idx, double *f) {
    int32_t nc3[3];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t ncmax = 1;
    for (int d = 0; d < 3; ++d) {
        int64_t c = (int64_t)floor(sys->L[d] / sys->rc);
        ncmax *= c > 0 ? c : 1;
    }
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncmax + 1));
    if (orc_cell_list(n, x, sys->L, sys->rc, nc3, cell_of, start, perm) != 0) {
        free(cell_of); free(perm); free(start);
        return -1;
    }
    const double V = sys->L[0] * sys->L[1] * sys->L[2];
    const double c = pow(M_PI, 1.5) * S / ((double)P * V);
    double *rho = (double *)malloc(sizeof(double) * 2 * (size_t)(P > 0 ? P : 1));
    orc_rho(n, q, x, sys->L, P, m, rho);
    const double rc2 = sys->rc * sys->rc;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < ns; ++t) {
        const int64_t i = idx[t];
        int32_t ci = cell_of[i];
        int32_t cx = ci % nc3[0], cy = (ci / nc3[0]) % nc3[1], cz = ci / (nc3[0] * nc3[1]);
        double fi[3] = {0.0, 0.0, 0.0}, un = 0.0, uw = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int32_t o = (((cz + dz + nc3[2]) % nc3[2]) * nc3[1] + (cy + dy + nc3[1]) % nc3[1]) * nc3[0] +
                                (cx + dx + nc3[0]) % nc3[0];
                    for (int32_t u = start[o]; u < start[o + 1]; ++u) {
                        int32_t j = perm[u];
                        if (j == i) continue;
                        double d[3];
                        double r2 = min_image(x + 3 * i, x + 3 * j, sys->L, d);
                        if (r2 < rc2) near_pair(sys, q[i], q[j], d, r2, fi, &un, &uw);
                    }
                }
        double ff[3] = {0.0, 0.0, 0.0};
        for (int32_t e = 0; e < P; ++e) {
            double k[3];
            for (int d = 0; d < 3; ++d) k[d] = 2.0 * M_PI * (double)m[3 * e + d] / sys->L[d];
            double th = k[0] * x[3 * i] + k[1] * x[3 * i + 1] + k[2] * x[3 * i + 2];
            double im = cos(th) * rho[2 * e + 1] - sin(th) * rho[2 * e];
            ff[0] += k[0] * im;
            ff[1] += k[1] * im;
            ff[2] += k[2] * im;
        }
        double g = -sys->lB * q[i] * c;
        for (int d = 0; d < 3; ++d) f[3 * t + d] = fi[d] + g * ff[d];
    }
    free(rho); free(cell_of); free(perm); free(start);
    return 0;
}

/* Gaussian self energy, (1/2) F_M(0) sum_i q_i^2 = (1/2)(sum_l w_l) sum_i q_i^2
 * (Eq. 3.8; the closed form printed there holds for the unmodified w_0). */
double orc_self_energy(int64_t n, const double *q, const orc_sys *sys) {
    double w = 0.0, q2 = 0.0;
    for (int32_t l = 0; l <= sys->M; ++l) w += sys->omega[l];
    for (int64_t i = 0; i < n; ++i) q2 += q[i] * q[i];
    return sys->lB * 0.5 * w * q2;
}

/* ---- virial ----------------------------------------------------------------
 * Configurational virial tensor W_ab = -dU/d eps_ab under the affine map
 * r -> (1 + eps) r of positions and box (r_c and the SOG fixed): the near
 * field (+ WCA) gives sum over pairs of r_ij,a F_ij,b; the far energy
 * (1/2V) sum_k F~(k) |rho(k)|^2, with V -> V (1 + tr eps) and
 * k -> (1 - eps^T) k at fixed rho, gives
 * (1/2V) sum_k |rho(k)|^2 [F~(k) delta_ab + 2 k_a k_b dF~/d(k^2)], and
 * F~ = pi^{3/2} sum_l w_l s_l^3 e^{-s_l^2 k^2/4} so that
 * 2 dF~/d(k^2) / F~ = -(1/2) T1/T0, T0 = sum_l w_l s_l^3 e^{..}, T1 = sum_l
 * w_l s_l^5 e^{..}.  The random-batch estimator weights each sampled k by
 * pi^{3/2} S / (2 P V) |rho|^2 as the energy's (Eq. 3.24), which makes it
 * unbiased for the exact far virial.  The k-independent self energy adds
 * nothing.  Row-major W[9], times lB for the Coulomb terms. */
static void far_virial_add(const orc_sys *sys, const int32_t m[3], double w, double W[9]) {
    double k[3], k2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        k[d] = 2.0 * M_PI * m[d] / sys->L[d];
        k2 += k[d] * k[d];
    }
    double T0 = 0.0, T1 = 0.0;
    for (int32_t l = 0; l <= sys->M; ++l) {
        const double s2 = sys->s[l] * sys->s[l];
        const double e = sys->omega[l] * s2 * sys->s[l] * exp(-s2 * k2 / 4.0);
        T0 += e;
        T1 += e * s2;
    }
    const double r = T0 > 0.0 ? T1 / T0 : 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) W[3 * a + b] += w * ((a == b ? 1.0 : 0.0) - 0.5 * r * k[a] * k[b]);
}

int orc_virial(int64_t n, const double *q, const double *x, const orc_sys *sys, double S, int32_t P,
               const int32_t *m, double W[9]) {
    for (int c = 0; c < 9; ++c) W[c] = 0.0;
    const double rc2 = sys->rc * sys->rc;
    const double V = sys->L[0] * sys->L[1] * sys->L[2];
    /* near field and WCA: pairs i < j */
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double d[3];
            const double r2 = min_image(x + 3 * i, x + 3 * j, sys->L, d);
            if (!(r2 < rc2)) continue;
            double fi[3] = {0.0, 0.0, 0.0}, un = 0.0, uw = 0.0;
            near_pair(sys, q[i], q[j], d, r2, fi, &un, &uw);   /* force on i from j */
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) W[3 * a + b] += d[a] * fi[b];
        }
    double Wf[9] = {0};
    if (P > 0) {
        double *rho = (double *)malloc(sizeof(double) * 2 * (size_t)P);
        orc_rho(n, q, x, sys->L, P, m, rho);
        const double c = pow(M_PI, 1.5) * S / (2.0 * P * V);
        for (int32_t e = 0; e < P; ++e)
            far_virial_add(sys, m + 3 * e, c * (rho[2 * e] * rho[2 * e] + rho[2 * e + 1] * rho[2 * e + 1]), Wf);
        free(rho);
    } else {
        /* exact sum over the half space (each k with -k, as orc_far_exact) */
        const double kcut = 2.0 * sqrt(log(1e16)) / sys->s[0];
        int32_t mm[3];
        for (int d = 0; d < 3; ++d) mm[d] = (int32_t)ceil(kcut * sys->L[d] / (2.0 * M_PI));
        for (int32_t a = 0; a <= mm[0]; ++a)
            for (int32_t b = -mm[1]; b <= mm[1]; ++b)
                for (int32_t c = -mm[2]; c <= mm[2]; ++c) {
                    const int half = (a > 0) || (a == 0 && b > 0) || (a == 0 && b == 0 && c > 0);
                    if (!half) continue;
                    const int32_t mk[3] = {a, b, c};
                    double k2 = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const double kd = 2.0 * M_PI * mk[d] / sys->L[d];
                        k2 += kd * kd;
                    }
                    if (k2 > kcut * kcut) continue;
                    double rho[2];
                    orc_rho(n, q, x, sys->L, 1, mk, rho);
                    const double ft = orc_ftilde(sys->omega, sys->s, sys->M, k2);
                    far_virial_add(sys, mk, 2.0 * ft * (rho[0] * rho[0] + rho[1] * rho[1]) / (2.0 * V), Wf);
                }
    }
    for (int c = 0; c < 9; ++c) W[c] += sys->lB * Wf[c];
    return 0;
}

/* ---- core-shell near-field kernel (Sec. 3.4) ------------------------------
 * Core, r < r_in (Eqs. 3.25-3.26): with u = r^2,
 *   sum_l w_l/s_l^2 e^{-u/s_l^2} = sum_{i=1}^{Q} (-1)^{i-1} A_i u^{i-1},
 *   A_i = sum_l w_l / ((i-1)! s_l^{2i}),
 * and F_M(u) = sum_{i=0}^{Q} (-1)^i B_i u^i, B_i = sum_l w_l / (i! s_l^{2i})
 * (the energy's series, the same expansion).  Eq. 3.26 prints A_i without
 * the alternating sign of the exponential's series; the series needs it.
 * Shell, r_in <= r < r_c: the FP32 bits of u give the bin (b_exp low
 * exponent bits, b_man high mantissa bits); each bin holds the exact kernel
 * at its lower end and the change to its upper end, and the remaining
 * mantissa bits give the interpolation fraction. */
static double cs_G(const orc_sys *sys, double u) {
    double v = 0.0;
    for (int32_t l = 0; l <= sys->M; ++l) v += sys->omega[l] / (sys->s[l] * sys->s[l]) * exp(-u / (sys->s[l] * sys->s[l]));
    return v;
}

static double cs_F(const orc_sys *sys, double u) {
    double v = 0.0;
    for (int32_t l = 0; l <= sys->M; ++l) v += sys->omega[l] * exp(-u / (sys->s[l] * sys->s[l]));
    return v;
}

static uint32_t f32_bits(float v) {
    uint32_t b;
    memcpy(&b, &v, sizeof b);
    return b;
}

/* first octave (biased FP32 exponent) of the shell table, or -1 if the
 * table's octaves do not reach r_c^2 */
static int cs_first_octave(const orc_sys *sys, const orc_coreshell *cs) {
    if (cs->r_in <= 0.0 || cs->r_in >= sys->rc || cs->b_exp < 0 || cs->b_exp > 4 || cs->b_man < 0 ||
        cs->b_man > 20 || cs->Q < 1)
        return -1;
    const int e0 = (int)((f32_bits((float)(cs->r_in * cs->r_in)) >> 23) & 0xffu);
    const int e1 = (int)((f32_bits((float)(sys->rc * sys->rc)) >> 23) & 0xffu);
    return e1 - e0 < (1 << cs->b_exp) ? e0 : -1;
}

static void cs_exact(const orc_sys *sys, double u, double *g, double *n) {
    const double r = sqrt(u);
    *g = 1.0 / (u * r) - 2.0 * cs_G(sys, u);
    *n = 1.0 / r - cs_F(sys, u);
}

int orc_coreshell_eval(const orc_sys *sys, const orc_coreshell *cs, double r2, double *g, double *n) {
    const int e0 = cs_first_octave(sys, cs);
    if (e0 < 0 || !(r2 >= 0.0) || r2 >= sys->rc * sys->rc) return -1;
    if (r2 < cs->r_in * cs->r_in) {
        const double r = sqrt(r2);
        double gs = 0.0, fs = 0.0, fact = 1.0;
        for (int32_t i = 0; i <= cs->Q; ++i) {
            if (i > 0) fact *= i;                       /* i! */
            double Bi = 0.0, Ai1 = 0.0;                 /* B_i and A_{i+1} */
            for (int32_t l = 0; l <= sys->M; ++l) {
                const double t = pow(sys->s[l] * sys->s[l], -(double)i);
                Bi += sys->omega[l] * t / fact;
                Ai1 += sys->omega[l] * t / (sys->s[l] * sys->s[l]) / fact;
            }
            const double sg = (i % 2) ? -1.0 : 1.0;
            const double ui = pow(r2, (double)i);
            fs += sg * Bi * ui;
            if (i < cs->Q) gs += sg * Ai1 * ui;         /* A_1 .. A_Q */
        }
        *g = 1.0 / (r2 * r) - 2.0 * gs;
        *n = 1.0 / r - fs;
        return 0;
    }
    /* shell: the bin from the FP32 bits of r^2 */
    const uint32_t bits = f32_bits((float)r2);
    const int E = (int)((bits >> 23) & 0xffu);
    const uint32_t mb = (uint32_t)cs->b_man;
    const uint32_t mant = bits & 0x7fffffu;
    const uint32_t m = mant >> (23u - mb);
    const uint32_t rest = mant & ((1u << (23u - mb)) - 1u);
    const double frac = (double)rest / (double)(1u << (23u - mb));
    const double u0 = ldexp(1.0 + (double)m / (double)(1u << mb), E - 127);
    const double u1 = ldexp(1.0 + (double)(m + 1) / (double)(1u << mb), E - 127);
    double g0, n0, g1, n1;
    cs_exact(sys, u0, &g0, &n0);
    cs_exact(sys, u1, &g1, &n1);
    *g = g0 + frac * (g1 - g0);
    *n = n0 + frac * (n1 - n0);
    (void)e0;
    return 0;
}

int orc_near_coreshell(int64_t n, const double *q, const double *x, const orc_sys *sys, const orc_coreshell *cs,
                       double *f, double *U_near, double *U_wca) {
    if (cs_first_octave(sys, cs) < 0) return -1;
    double *un = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *uw = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    const double rc2 = sys->rc * sys->rc;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            const double r2 = min_image(x + 3 * i, x + 3 * j, sys->L, d);
            if (!(r2 < rc2)) continue;
            double g, nn;
            orc_coreshell_eval(sys, cs, r2, &g, &nn);
            const double qq = sys->lB * q[i] * q[j];
            for (int c = 0; c < 3; ++c) fi[c] += qq * g * d[c];
            un[i] += 0.5 * qq * nn;
            if (sys->wca_sigma > 0.0) {
                const double rcut2 = pow(2.0, 1.0 / 3.0) * sys->wca_sigma * sys->wca_sigma;
                if (r2 < rcut2) {
                    const double sr2 = sys->wca_sigma * sys->wca_sigma / r2;
                    const double sr6 = sr2 * sr2 * sr2;
                    const double gw = 24.0 * sys->wca_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                    for (int c = 0; c < 3; ++c) fi[c] += gw * d[c];
                    uw[i] += 0.5 * (4.0 * sys->wca_eps * (sr6 * sr6 - sr6) + sys->wca_eps);
                }
            }
        }
        for (int c = 0; c < 3; ++c) f[3 * i + c] = fi[c];
    }
    double a = 0.0, b = 0.0;
    for (int64_t i = 0; i < n; ++i) { a += un[i]; b += uw[i]; }
    *U_near = a;
    *U_wca = b;
    free(un);
    free(uw);
    return 0;
}

/* Zero-frequency term: the k -> 0 limit of the far field for a neutral
 * system, U0 = -(pi/V) sum_{i,j} q_i q_j lim (k.r_ij)^2 / k^2 (Eq. 3.13),
 * averaged over directions (spherical boundary, Eq. 3.14) or taken along z
 * (planar boundary, Eq. 3.15); both reduce to the dipole moment
 * M = sum_i q_i r_i.  The force is -grad U0: -(4 pi / 3V) q_i M and
 * -(4 pi / V) q_i M_z e_z. */
double orc_boundary(int64_t n, const double *q, const double *x, const double L[3], double lB, int32_t kind,
                    double *f) {
    if (kind != 1 && kind != 2) return 0.0;
    const double V = L[0] * L[1] * L[2];
    double M[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) M[d] += q[i] * x[3 * i + d];
    double U, c[3];
    if (kind == 1) {
        U = 2.0 * M_PI / (3.0 * V) * (M[0] * M[0] + M[1] * M[1] + M[2] * M[2]);
        for (int d = 0; d < 3; ++d) c[d] = -4.0 * M_PI / (3.0 * V) * M[d];
    } else {
        U = 2.0 * M_PI / V * M[2] * M[2];
        c[0] = c[1] = 0.0;
        c[2] = -4.0 * M_PI / V * M[2];
    }
    if (f)
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) f[3 * i + d] += lB * q[i] * c[d];
    return lB * U;
}

/* Total force F = F_N + F_F (+ WCA) at wrapped positions x.  P > 0: the
 * random-batch far field on the P vectors m; P == 0: the exact far sum.
 * Total potential energy U_near + U_far - U_self + U_wca. */
int orc_forces(int64_t n, const double *q, const double *x, const orc_sys *sys,
               double S, int32_t P, const int32_t *m, double *f, orc_energies *e) {
    double *fn = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *ff = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_energies en;
    memset(&en, 0, sizeof en);
    int rc = orc_near_cells(n, q, x, sys, fn, &en.U_near, &en.U_wca, NULL);
    if (rc != 0) { free(fn); free(ff); return rc; }
    if (P > 0) orc_far_rb(n, q, x, sys, S, P, m, ff, &en.U_far, NULL);
    else orc_far_exact(n, q, x, sys, 1e-16, ff, &en.U_far);
    en.U_self = orc_self_energy(n, q, sys);
    for (int64_t i = 0; i < 3 * n; ++i) f[i] = fn[i] + ff[i];
    if (e) *e = en;
    free(fn);
    free(ff);
    return 0;
}

/* Velocity Verlet (Algorithm 1) with an optional Berendsen rescale
 * v <- v sqrt(1 + dt/tau (T0/T - 1)) after the second half kick (tau <= 0:
 * NVE).  Each force evaluation takes the next P vectors of kseq in order;
 * when have_force == 0 the forces at the initial positions are computed
 * first (consuming the first k-set).  x is wrapped after every drift.
 * T = 2K / (3N - 3).  e_steps[t] receives the energies at the end of step t. */
int orc_md_thermo(int64_t n, const double *q, double *x, double *v, double *f,
                  const orc_sys *sys, double S, int32_t P, const int32_t *kseq,
                  int64_t nsteps, double dt, double mass, double T0, double tau,
                  int have_force, orc_energies *e_steps, int32_t thermostat, uint64_t seed, int64_t step0);

/* Langevin noise of particle i in the step that starts with step counter t:
 * Philox4x64-10 with key (seed, 2^63 + 1) (the sampler's chain keys are
 * below 2^63) and counter (t, i, 0, 0); Box-Muller as in the sampler:
 * (u0, u1) -> (z_x, z_y), (u2, u3) -> z_z. */
void orc_langevin_noise(uint64_t seed, int64_t t, int64_t i, double z[3]) {
    const uint64_t key[2] = {seed, 0x8000000000000001ull};
    const uint64_t ctr[4] = {(uint64_t)t, (uint64_t)i, 0, 0};
    uint64_t r[4];
    orc_philox4x64_10(ctr, key, r);
    const double r01 = sqrt(-2.0 * log(1.0 - u01(r[0])));
    const double r23 = sqrt(-2.0 * log(1.0 - u01(r[2])));
    z[0] = r01 * cos(2.0 * M_PI * u01(r[1]));
    z[1] = r01 * sin(2.0 * M_PI * u01(r[1]));
    z[2] = r23 * cos(2.0 * M_PI * u01(r[3]));
}

int orc_md(int64_t n, const double *q, double *x, double *v, double *f,
           const orc_sys *sys, double S, int32_t P, const int32_t *kseq,
           int64_t nsteps, double dt, double mass, double T0, double tau,
           int have_force, orc_energies *e_steps) {
    return orc_md_thermo(n, q, x, v, f, sys, S, P, kseq, nsteps, dt, mass, T0, tau, have_force, e_steps, 0, 0, 0);
}

/* As orc_md, with thermostat 2 (tau > 0): Nose-Hoover, thermostat mass
 * Q = g T0 tau^2 (g = 3N - 3), propagated by the symmetric Trotter
 * splitting; each step is velocity Verlet followed by two thermostat
 * half-steps (its own end and the next step's start), each: xi += dt/4 G;
 * v *= e^{-xi dt/2}; eta += dt/2 xi; xi += dt/4 G, with G = (2K - g T0)/Q
 * at the current K.  U + K + (1/2) Q xi^2 + g T0 eta is conserved.
 * With thermostat 1 (tau > 0): Langevin dynamics with friction
 * 1/tau in the BAOAB splitting, per step: v += dt/2 F/m; x += dt/2 v;
 * v = c1 v + c2 z with c1 = e^{-dt/tau}, c2 = sqrt((1 - c1^2) T0/m) and z the
 * noise of orc_langevin_noise for the step counter step0 + t; x += dt/2 v;
 * forces; v += dt/2 F/m.  The Berendsen rescale is thermostat 0. */
int orc_md_thermo(int64_t n, const double *q, double *x, double *v, double *f,
                  const orc_sys *sys, double S, int32_t P, const int32_t *kseq,
                  int64_t nsteps, double dt, double mass, double T0, double tau,
                  int have_force, orc_energies *e_steps, int32_t thermostat, uint64_t seed, int64_t step0) {
    const int langevin = thermostat == 1 && tau > 0.0;
    const int nh = thermostat == 2 && tau > 0.0;
    const double g_dof = 3.0 * (double)n - 3.0;
    const double Qnh = g_dof * T0 * tau * tau;
    double xi = 0.0, eta = 0.0;
    const double c1 = langevin ? exp(-dt / tau) : 1.0;
    const double c2 = langevin ? sqrt((1.0 - c1 * c1) * T0 / mass) : 0.0;
    int64_t used = 0;
    orc_energies e;
    orc_wrap(n, x, sys->L);
    if (!have_force) {
        int rc = orc_forces(n, q, x, sys, S, P, P > 0 ? kseq : NULL, f, &e);
        if (rc) return rc;
        ++used;
    }
    for (int64_t t = 0; t < nsteps; ++t) {
        for (int64_t i = 0; i < 3 * n; ++i) v[i] += 0.5 * dt * f[i] / mass;
        if (langevin) {
            for (int64_t i = 0; i < 3 * n; ++i) x[i] += 0.5 * dt * v[i];
            for (int64_t i = 0; i < n; ++i) {
                double z[3];
                orc_langevin_noise(seed, step0 + t, i, z);
                for (int d = 0; d < 3; ++d) v[3 * i + d] = c1 * v[3 * i + d] + c2 * z[d];
            }
            for (int64_t i = 0; i < 3 * n; ++i) x[i] += 0.5 * dt * v[i];
        } else {
            for (int64_t i = 0; i < 3 * n; ++i) x[i] += dt * v[i];
        }
        orc_wrap(n, x, sys->L);
        int rc = orc_forces(n, q, x, sys, S, P, P > 0 ? kseq + 3 * (int64_t)P * used : NULL, f, &e);
        if (rc) return rc;
        ++used;
        for (int64_t i = 0; i < 3 * n; ++i) v[i] += 0.5 * dt * f[i] / mass;
        double K = 0.0;
        for (int64_t i = 0; i < 3 * n; ++i) K += 0.5 * mass * v[i] * v[i];
        double T = 2.0 * K / (3.0 * (double)n - 3.0);
        if (nh) {
            /* two consecutive half-steps of the thermostat (the end of this
             * step and the start of the next in the symmetric splitting) */
            for (int h = 0; h < 2; ++h) {
                xi += 0.25 * dt * (2.0 * K - g_dof * T0) / Qnh;
                const double sc = exp(-0.5 * dt * xi);
                for (int64_t i = 0; i < 3 * n; ++i) v[i] *= sc;
                K *= sc * sc;
                eta += 0.5 * dt * xi;
                xi += 0.25 * dt * (2.0 * K - g_dof * T0) / Qnh;
            }
            K = 0.0;
            for (int64_t i = 0; i < 3 * n; ++i) K += 0.5 * mass * v[i] * v[i];
            T = 2.0 * K / (3.0 * (double)n - 3.0);
        }
        e.U_th = nh ? 0.5 * Qnh * xi * xi + g_dof * T0 * eta : 0.0;
        if (!langevin && !nh && tau > 0.0 && T > 0.0) {
            double lam = sqrt(1.0 + dt / tau * (T0 / T - 1.0));
            for (int64_t i = 0; i < 3 * n; ++i) v[i] *= lam;
            K = 0.0;
            for (int64_t i = 0; i < 3 * n; ++i) K += 0.5 * mass * v[i] * v[i];
            T = 2.0 * K / (3.0 * (double)n - 3.0);
        }
        e.K = K;
        e.T = T;
        if (e_steps) e_steps[t] = e;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Radial distribution functions (Appendix A).
 *
 * g(r) = (1/(N rho)) sum_i sum_{j != i} <delta(r_ij - r)> / (4 pi r^2), taken
 * per pair of charge signs (++, +-, --) with rho the number density of the
 * second species, and estimated by a histogram of the minimum-image pair
 * distances on [0, L/2) in nbins equal bins (cubic box of edge L).
 *
 * Distances are measured on positions quantised to L 2^-32 per axis:
 * X = floor(frac(x / L) 2^32) mod 2^32.  On that lattice the minimum-image
 * difference is an exact integer d in [-2^31, 2^31), the squared distance an
 * exact integer R = dx^2 + dy^2 + dz^2 (units (L 2^-32)^2), r < L/2 means
 * R < 2^62, and the bin of width 2^31/nbins lattice units is
 * floor(isqrt(R) / (2^31/nbins)): every bin decision is exact integer
 * arithmetic, so any correct implementation gives the same counts.
 * ------------------------------------------------------------------------ */
static uint32_t rdf_quantise(double x, double L) {
    double t = x / L;
    t = t - floor(t);
    const double v = floor(t * 4294967296.0);
    return (uint32_t)((uint64_t)v & 0xffffffffu);
}

/* floor(sqrt(R)) for R < 2^62, exact */
static uint64_t rdf_isqrt(uint64_t R) {
    uint64_t s = (uint64_t)sqrt((double)R);
    while (s * s > R) --s;
    while ((s + 1) * (s + 1) <= R) ++s;
    return s;
}

int orc_rdf_counts(int64_t n, const double *q, const double *x, double L, int32_t nbins, uint64_t *counts) {
    if (nbins < 16 || nbins > 4096 || (nbins & (nbins - 1)) || !(L > 0.0)) return -1;
    const uint64_t width = (uint64_t)2147483648u / (uint64_t)nbins;   /* lattice units per bin */
    uint32_t *X = malloc(sizeof(uint32_t) * 3 * (size_t)(n > 0 ? n : 1));
    int *sp = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) X[3 * i + d] = rdf_quantise(x[3 * i + d], L);
        sp[i] = q[i] > 0.0 ? 0 : (q[i] < 0.0 ? 1 : -1);   /* sign species; neutral sites are skipped */
    }
    memset(counts, 0, sizeof(uint64_t) * 3 * (size_t)nbins);
    int nt = orc_num_threads();
    uint64_t *part = calloc((size_t)nt * 3 * (size_t)nbins, sizeof(uint64_t));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
#ifdef _OPENMP
        uint64_t *h = part + (size_t)omp_get_thread_num() * 3 * (size_t)nbins;
#else
        uint64_t *h = part;
#endif
        if (sp[i] < 0) continue;
        for (int64_t j = i + 1; j < n; ++j) {
            if (sp[j] < 0) continue;
            uint64_t R = 0;
            for (int d = 0; d < 3; ++d) {
                int64_t dd = (int64_t)X[3 * i + d] - (int64_t)X[3 * j + d];
                if (dd >= 2147483648LL) dd -= 4294967296LL;
                if (dd < -2147483648LL) dd += 4294967296LL;
                R += (uint64_t)(dd * dd);
            }
            if (R >= ((uint64_t)1 << 62)) continue;              /* r >= L/2 */
            const int64_t bin = (int64_t)(rdf_isqrt(R) / width);
            h[(sp[i] + sp[j]) * nbins + bin] += 1;               /* 0: ++, 1: +-, 2: -- */
        }
    }
    for (int t = 0; t < nt; ++t)
        for (int64_t k = 0; k < 3 * (int64_t)nbins; ++k) counts[k] += part[(size_t)t * 3 * nbins + k];
    free(part);
    free(sp);
    free(X);
    return 0;
}

/* Histogram estimate of Appendix A's g(r) for bin k (r in [k dr, (k+1) dr),
 * dr = L / (2 nbins)): the expected number of ordered pairs in the shell is
 * N_a (N_b / V) * shell volume, with shell volume (4 pi / 3)((k+1)^3 - k^3) dr^3;
 * like pairs are counted once per unordered pair, so twice as ordered pairs. */
void orc_rdf_g(const uint64_t *counts, int32_t nbins, double L, int64_t n_pos, int64_t n_neg, double *g) {
    const double V = L * L * L;
    const double dr = L / (2.0 * nbins);
    const double na[3] = {(double)n_pos, (double)n_pos, (double)n_neg};
    const double nb[3] = {(double)n_pos, (double)n_neg, (double)n_neg};
    const double mult[3] = {2.0, 1.0, 2.0};
    for (int t = 0; t < 3; ++t)
        for (int32_t k = 0; k < nbins; ++k) {
            const double shell = 4.0 * M_PI / 3.0 * (pow(k + 1.0, 3) - pow((double)k, 3)) * dr * dr * dr;
            const double expect = na[t] * nb[t] / V * shell;
            g[t * nbins + k] = expect > 0.0 ? mult[t] * (double)counts[t * nbins + k] / expect : 0.0;
        }
}

/* ---- time-correlation observables (Appendix A) ------------------------- */

static double min_image1(double d, double L) { return d - L * nearbyint(d / L); }

/* Appendix A's MSD and VACF, each origin and lag summed over the particles in
 * index order; the frames are unwrapped first. */
int orc_msd_vacf(int64_t n, int64_t n_frames, const double *x, const double *v, const double *L,
                 int32_t n_lags, int32_t origin_every, double *msd, double *vacf, int64_t *count) {
    if (n < 1 || n_frames < 1 || n_lags < 1 || origin_every < 1) return -1;
    double *u = (double *)malloc(sizeof(double) * 3 * n * n_frames);
    if (!u) return -1;
    for (int64_t k = 0; k < 3 * n; ++k) u[k] = x[k];
    for (int64_t f = 1; f < n_frames; ++f)
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                const int64_t a = (f * n + i) * 3 + d, b = ((f - 1) * n + i) * 3 + d;
                u[a] = u[b] + min_image1(x[a] - x[b], L[d]);
            }
    for (int32_t t = 0; t < n_lags; ++t) {
        msd[t] = vacf[t] = 0.0;
        count[t] = 0;
    }
    for (int64_t o = 0; o < n_frames; o += origin_every)
        for (int32_t t = 0; t < n_lags && o + t < n_frames; ++t) {
            double sm = 0.0, sv = 0.0;
            for (int64_t i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d) {
                    const int64_t a = ((o + t) * n + i) * 3 + d, b = (o * n + i) * 3 + d;
                    const double dr = u[a] - u[b];
                    sm += dr * dr;
                    sv += v[b] * v[a];
                }
            msd[t] += sm;
            vacf[t] += sv;
            count[t] += 1;
        }
    for (int32_t t = 0; t < n_lags; ++t)
        if (count[t] > 0) {
            msd[t] /= (double)count[t] * (double)n;
            vacf[t] /= (double)count[t] * (double)n;
        }
    free(u);
    return 0;
}

int orc_pressure(int64_t n, const double *q, const double *x, const double *v, double mass,
                 const orc_sys *sys, double S, int32_t P, const int32_t *kset, double *Pt) {
    double W[9];
    const int rc = orc_virial(n, q, x, sys, S, P, kset, W);
    if (rc) return rc;
    const double V = sys->L[0] * sys->L[1] * sys->L[2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double k = 0.0;
            for (int64_t i = 0; i < n; ++i) k += mass * v[3 * i + a] * v[3 * i + b];
            Pt[3 * a + b] = (k + W[3 * a + b]) / V;
        }
    return 0;
}

int orc_green_kubo(int64_t n_samples, const double *Pt, double dt, double V, double T, int32_t max_lag,
                   double *acf, double *C) {
    if (n_samples < 2 || max_lag < 2 || max_lag > n_samples || T <= 0.0) return -1;
    static const int comp[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int32_t t = 0; t < max_lag; ++t) acf[t] = 0.0;
    for (int c = 0; c < 6; ++c) {
        const int e = 3 * comp[c][0] + comp[c][1];
        double mean = 0.0;
        for (int64_t s = 0; s < n_samples; ++s) mean += Pt[9 * s + e];
        mean /= (double)n_samples;
        for (int32_t t = 0; t < max_lag; ++t) {
            double a = 0.0;
            for (int64_t o = 0; o + t < n_samples; ++o) a += (Pt[9 * o + e] - mean) * (Pt[9 * (o + t) + e] - mean);
            acf[t] += a / (double)(n_samples - t);
        }
    }
    double integral = 0.0;
    for (int32_t t = 0; t + 1 < max_lag; ++t) integral += 0.5 * dt * (acf[t] + acf[t + 1]);
    *C = V / (6.0 * T) * integral;
    return 0;
}

/* ---- heat flux and heat conductivity (Appendix A) ------------------------
 * J = (1/V) [ sum_i e_i v_i + (1/2) sum_{i<j} (f_ij . (v_i + v_j)) r_ij ],
 * e_i the per-atom energy (kinetic and potential).  The pair sum equals
 * sum_i W_i v_i with the per-atom virial W_i,ab = (1/2) sum_{j != i} r_ij,a
 * f_ij,b (r_ij = r_i - r_j minimum image, f_ij the force on i from j): each
 * ordered pair gives r_ij (f_ij . v_i) / 2 and the two orders of a pair give
 * the printed term.  Per-atom energies: (1/2) m |v_i|^2, half of every pair
 * energy (Coulomb near part and WCA), minus the self term (1/2) F_M(0) q_i^2,
 * and the far part.  The random-batch far energy pi^{3/2} S/(2PV) sum_eta
 * |rho(k_eta)|^2 splits over atoms as e_i = (c/2) q_i sum_eta
 * Re(e^{-i k_eta . r_i} rho(k_eta)), c = pi^{3/2} S/(P V), since
 * sum_i q_i e^{-i k . r_i} = conj(rho(k)); the far virial of orc_virial
 * splits the same way, W_i,ab = (c/2) q_i sum_eta Re(e^{-i k.r_i} rho)
 * (delta_ab - (1/2) k_a k_b T1/T0).  Summed over atoms these give U*_RB and
 * the random-batch far virial exactly.  P = 0: no far term.  Coulomb terms
 * times lB.  e_atom[n] and W_atom[n][9] are returned when non-NULL. */
int orc_heat_flux(int64_t n, const double *q, const double *x, const double *v, double mass,
                  const orc_sys *sys, double S, int32_t P, const int32_t *m, double J[3], double *e_atom,
                  double *W_atom) {
    int32_t nc3[3];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t ncmax = 1;
    for (int d = 0; d < 3; ++d) ncmax *= (int64_t)floor(sys->L[d] / sys->rc) > 0 ? (int64_t)floor(sys->L[d] / sys->rc) : 1;
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncmax + 1));
    if (orc_cell_list(n, x, sys->L, sys->rc, nc3, cell_of, start, perm) != 0) {
        free(cell_of); free(perm); free(start);
        return -1;
    }
    double *e = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *W = (double *)calloc(9 * (size_t)(n > 0 ? n : 1), sizeof(double));
    const double rc2 = sys->rc * sys->rc;
    const double V = sys->L[0] * sys->L[1] * sys->L[2];
    double FM0 = 0.0;
    for (int32_t l = 0; l <= sys->M; ++l) FM0 += sys->omega[l];
    /* near field and WCA: every ordered pair from its first atom */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = cell_of[i];
        int32_t cx = c % nc3[0], cy = (c / nc3[0]) % nc3[1], cz = c / (nc3[0] * nc3[1]);
        double ei = 0.0, Wi[9] = {0};
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int32_t ox = (cx + dx + nc3[0]) % nc3[0];
                    int32_t oy = (cy + dy + nc3[1]) % nc3[1];
                    int32_t oz = (cz + dz + nc3[2]) % nc3[2];
                    int32_t o = (oz * nc3[1] + oy) * nc3[0] + ox;
                    for (int32_t t = start[o]; t < start[o + 1]; ++t) {
                        int32_t j = perm[t];
                        if (j == i) continue;
                        double d[3];
                        double r2 = min_image(x + 3 * i, x + 3 * j, sys->L, d);
                        if (!(r2 < rc2)) continue;
                        double fij[3] = {0.0, 0.0, 0.0}, un = 0.0, uw = 0.0;
                        near_pair(sys, q[i], q[j], d, r2, fij, &un, &uw);   /* halves of the pair energy */
                        ei += un + uw;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) Wi[3 * a + b] += 0.5 * d[a] * fij[b];
                    }
                }
        const double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        e[i] = ei + 0.5 * mass * v2 - sys->lB * 0.5 * FM0 * q[i] * q[i];
        for (int c9 = 0; c9 < 9; ++c9) W[9 * i + c9] = Wi[c9];
    }
    if (P > 0) {
        const double c = sys->lB * pow(M_PI, 1.5) * S / ((double)P * V);
        double *rho = (double *)malloc(sizeof(double) * 2 * (size_t)P);
        double *kv = (double *)malloc(sizeof(double) * 4 * (size_t)P);   /* k, T1/T0 */
        orc_rho(n, q, x, sys->L, P, m, rho);
        for (int32_t h = 0; h < P; ++h) {
            double k2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                kv[4 * h + d] = 2.0 * M_PI * (double)m[3 * h + d] / sys->L[d];
                k2 += kv[4 * h + d] * kv[4 * h + d];
            }
            double T0 = 0.0, T1 = 0.0;
            for (int32_t l = 0; l <= sys->M; ++l) {
                const double s2 = sys->s[l] * sys->s[l];
                const double t = sys->omega[l] * s2 * sys->s[l] * exp(-s2 * k2 / 4.0);
                T0 += t;
                T1 += t * s2;
            }
            kv[4 * h + 3] = T0 > 0.0 ? T1 / T0 : 0.0;
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double ei = 0.0, Wi[9] = {0};
            for (int32_t h = 0; h < P; ++h) {
                const double *k = kv + 4 * h;
                const double th = k[0] * x[3 * i] + k[1] * x[3 * i + 1] + k[2] * x[3 * i + 2];
                /* Re(e^{-i th} (A + iB)) = cos(th) A + sin(th) B */
                const double re = cos(th) * rho[2 * h] + sin(th) * rho[2 * h + 1];
                const double w = 0.5 * c * q[i] * re;
                ei += w;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) Wi[3 * a + b] += w * ((a == b ? 1.0 : 0.0) - 0.5 * k[3] * k[a] * k[b]);
            }
            e[i] += ei;
            for (int c9 = 0; c9 < 9; ++c9) W[9 * i + c9] += Wi[c9];
        }
        free(rho);
        free(kv);
    }
    double Js[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double t = e[i] * v[3 * i + a];
            for (int b = 0; b < 3; ++b) t += W[9 * i + 3 * a + b] * v[3 * i + b];
            Js[a] += t;
        }
    for (int a = 0; a < 3; ++a) J[a] = Js[a] / V;
    if (e_atom) memcpy(e_atom, e, sizeof(double) * (size_t)n);
    if (W_atom) memcpy(W_atom, W, sizeof(double) * 9 * (size_t)n);
    free(e); free(W); free(cell_of); free(perm); free(start);
    return 0;
}

/* Heat conductivity by the Green-Kubo relation of Appendix A:
 * C = V / (3 k_B T^2) * integral over t of <J(0) . J(t)>, the average over
 * all origins t0 with t0 + t < n_samples of J(t0) . J(t0 + t) (the flux as
 * sampled, no mean removed: its equilibrium mean is zero), integrated by the
 * trapezoid rule over the lags 0 .. max_lag - 1 spaced dt.  J[n_samples][3];
 * acf[max_lag] receives the autocorrelation per lag. */
int orc_green_kubo_heat(int64_t n_samples, const double *J, double dt, double V, double T, int32_t max_lag,
                        double *acf, double *C) {
    if (n_samples < 2 || max_lag < 2 || max_lag > n_samples || T <= 0.0) return -1;
    for (int32_t t = 0; t < max_lag; ++t) {
        double a = 0.0;
        for (int64_t o = 0; o + t < n_samples; ++o)
            for (int c = 0; c < 3; ++c) a += J[3 * o + c] * J[3 * (o + t) + c];
        acf[t] = a / (double)(n_samples - t);
    }
    double integral = 0.0;
    for (int32_t t = 0; t + 1 < max_lag; ++t) integral += 0.5 * dt * (acf[t] + acf[t + 1]);
    *C = V / (3.0 * T * T) * integral;
    return 0;
}

/* ---- per-Gaussian independent sampling (Sec. 3.3, closing remark) ------- */

#define PG_MAX_JMAX (1 << 20)

/* Cumulative table of one coordinate: T[0] = 1, T[j] = T[j-1] + 2 e^{-x j^2};
 * z = sum_{j>=1} 2 e^{-x j^2} summed on its own (no cancellation when tiny). */
static int pg_table(double s, double L, double **T_out, int32_t *jmax_out, double *z_out) {
    const double a = M_PI * s / L;
    const double x = a * a;
    const double jm = ceil(sqrt(50.0 / x));
    if (!(jm <= (double)PG_MAX_JMAX)) return -1;
    const int32_t jmax = jm < 1.0 ? 1 : (int32_t)jm;
    double *T = (double *)malloc(sizeof(double) * ((size_t)jmax + 1));
    if (!T) return -1;
    T[0] = 1.0;
    double z = 0.0;
    for (int32_t j = 1; j <= jmax; ++j) {
        const double w = 2.0 * exp(-x * (double)j * (double)j);
        T[j] = T[j - 1] + w;
        z = z + w;
    }
    *T_out = T;
    *jmax_out = jmax;
    *z_out = z;
    return 0;
}

/* prod_d (1 + z_d) - 1 expanded, so that tiny z keep their digits. */
static double pg_G(const double z[3]) {
    return (((((z[0] + z[1]) + z[2]) + z[0] * z[1]) + z[0] * z[2]) + z[1] * z[2]) + (z[0] * z[1]) * z[2];
}

int32_t orc_pg_plan(const double *omega, const double *s, int32_t M, const double L[3], int32_t P,
                    int32_t *P_l, double *S_l) {
    double tot = 0.0;
    for (int32_t l = 0; l <= M; ++l) {
        double z[3];
        for (int d = 0; d < 3; ++d) {
            double *T;
            int32_t jm;
            if (pg_table(s[l], L[d], &T, &jm, &z[d])) return -1;
            free(T);
        }
        S_l[l] = omega[l] * s[l] * s[l] * s[l] * pg_G(z);
        tot += S_l[l];
    }
    int32_t P_eff = 0;
    for (int32_t l = 0; l <= M; ++l) {
        P_l[l] = S_l[l] > 1e-16 * tot ? (int32_t)ceil((double)P * S_l[l] / tot) : 0;
        P_eff += P_l[l];
    }
    return P_eff;
}

/* Smallest j in [j0, jmax] with t < T[j]; jmax when rounding put t at the end. */
static int32_t pg_search(const double *T, int32_t j0, int32_t jmax, double t) {
    for (int32_t j = j0; j <= jmax; ++j)
        if (t < T[j]) return j;
    return jmax;
}

int orc_pg_kseq(const double *omega, const double *s, int32_t M, const double L[3], int32_t P, uint64_t seed,
                int64_t set0, int64_t n_sets, int32_t *m_out, int32_t *stratum_out) {
    int32_t P_l[256];
    double S_l[256];
    if (M < 0 || M > 255) return -1;
    const int32_t P_eff = orc_pg_plan(omega, s, M, L, P, P_l, S_l);
    if (P_eff < 0) return -1;
    const uint64_t key[2] = {seed, 0x8000000000000002ull};
    for (int32_t l = 0, eta0 = 0; l <= M; eta0 += P_l[l], ++l) {
        if (P_l[l] == 0) continue;
        double *T[3], z[3];
        int32_t jmax[3];
        for (int d = 0; d < 3; ++d)
            if (pg_table(s[l], L[d], &T[d], &jmax[d], &z[d])) return -1;
        /* P(first non-zero coordinate is x | m != 0), and y given m_x = 0 */
        const double thr1 = ((z[0] * (1.0 + z[1])) * (1.0 + z[2])) / pg_G(z);
        const double den2 = (z[1] + z[2]) + z[1] * z[2];
        const double thr2 = den2 > 0.0 ? (z[1] * (1.0 + z[2])) / den2 : 1.0;
        for (int64_t t = 0; t < n_sets; ++t)
            for (int32_t e = 0; e < P_l[l]; ++e) {
                const int64_t eta = eta0 + e;
                const uint64_t ca[4] = {(uint64_t)(set0 + t), (uint64_t)eta, 0, 0};
                const uint64_t cb[4] = {(uint64_t)(set0 + t), (uint64_t)eta, 1, 0};
                uint64_t ra[4], rb[4];
                orc_philox4x64_10(ca, key, ra);
                orc_philox4x64_10(cb, key, rb);
                const int first = u01(ra[0]) < thr1 ? 0 : (u01(ra[1]) < thr2 ? 1 : 2);
                int32_t *m = m_out + 3 * (t * P_eff + eta);
                for (int d = 0; d < 3; ++d) {
                    const double u = u01(rb[d]);
                    const double Tn = T[d][jmax[d]];
                    int32_t j;
                    if (d < first) j = 0;
                    else if (d == first) j = pg_search(T[d], 1, jmax[d], T[d][0] + u * (Tn - T[d][0]));
                    else j = pg_search(T[d], 0, jmax[d], u * Tn);
                    m[d] = ((ra[2] >> d) & 1u) ? -j : j;
                }
                if (stratum_out) stratum_out[t * P_eff + eta] = l;
            }
        for (int d = 0; d < 3; ++d) free(T[d]);
    }
    return 0;
}

void orc_far_rb_w(int64_t n, const double *q, const double *x, const orc_sys *sys, int32_t P, const int32_t *m,
                  const double *c, double *f, double *U_rb) {
    const double V = sys->L[0] * sys->L[1] * sys->L[2];
    const double pre = pow(M_PI, 1.5) / V;
    double *rho = (double *)malloc(sizeof(double) * 2 * (size_t)(P > 0 ? P : 1));
    orc_rho(n, q, x, sys->L, P, m, rho);
    double U = 0.0;
    for (int32_t e = 0; e < P; ++e) U += c[e] * (rho[2 * e] * rho[2 * e] + rho[2 * e + 1] * rho[2 * e + 1]);
    *U_rb = sys->lB * 0.5 * pre * U;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int32_t e = 0; e < P; ++e) {
            double k[3];
            for (int d = 0; d < 3; ++d) k[d] = 2.0 * M_PI * (double)m[3 * e + d] / sys->L[d];
            const double th = k[0] * x[3 * i] + k[1] * x[3 * i + 1] + k[2] * x[3 * i + 2];
            const double im = c[e] * (cos(th) * rho[2 * e + 1] - sin(th) * rho[2 * e]);
            fi[0] += k[0] * im;
            fi[1] += k[1] * im;
            fi[2] += k[2] * im;
        }
        const double g = -sys->lB * q[i] * pre;
        f[3 * i + 0] = g * fi[0];
        f[3 * i + 1] = g * fi[1];
        f[3 * i + 2] = g * fi[2];
    }
    free(rho);
}
