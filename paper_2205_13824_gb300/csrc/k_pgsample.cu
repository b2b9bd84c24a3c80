// Per-Gaussian independent sampling, the variant the paper describes after
// the mixture sampler (Sec. 3.3): each Gaussian of the far kernel, normalised
// over k != 0, p_l(k) = e^{-s_l^2 k^2 / 4} / (prod_d H_l^d - 1) with
// H_l^d = sum_m e^{-x m^2}, x = (pi s_l / L_d)^2 (Eq. 3.17), is sampled on its
// own with a batch size adapted to its share S_l = w_l s_l^3 (prod_d H_l^d - 1)
// of the normaliser S (Eq. 3.16).
//
// A frequency is drawn exactly: the first non-zero coordinate d* is chosen
// with its conditional probability given m != 0; coordinates before d* are
// 0, d* is drawn given m_d* != 0 and the later ones unconditioned, each by
// inverting the cumulative table T[j] = 1 + sum_{i=1..j} 2 e^{-x i^2} of |m|
// (j <= jmax = ceil(sqrt(50 / x)): the tail beyond is below e^{-50}), its
// sign from a random bit.  Random numbers: Philox4x64-10 with key
// (seed, 2^63 + 2), counters (set, eta, 0, 0) -> decision uniforms and sign
// bits, (set, eta, 1, 0) -> one uniform per coordinate.
//
// The tables and the decision thresholds are built here on the host, and
// the host part of this file is compiled without floating-point
// contraction; the kernel is compiled with -fmad=false.  So every value that
// decides an integer is the IEEE evaluation of the expressions written below.
#include "rbsog_kernels.cuh"

#include <cmath>

namespace rbsog {
namespace {

constexpr double kPiPg = 3.14159265358979323846;
constexpr int32_t kPgMaxJ = 1 << 20;
constexpr int kThreads = 256;

// Cumulative table of |m| for one coordinate and z = sum_{j >= 1} 2 e^{-x j^2}
// summed on its own (it keeps its digits when tiny).
bool coord_table(double s, double L, std::vector<double> &T, int32_t &jmax, double &z) {
    const double a = kPiPg * s / L;
    const double x = a * a;
    const double jm = std::ceil(std::sqrt(50.0 / x));
    if (!(jm <= (double)kPgMaxJ)) return false;
    jmax = jm < 1.0 ? 1 : (int32_t)jm;
    T.assign((size_t)jmax + 1, 0.0);
    T[0] = 1.0;
    z = 0.0;
    for (int32_t j = 1; j <= jmax; ++j) {
        const double w = 2.0 * std::exp(-x * (double)j * (double)j);
        T[j] = T[j - 1] + w;
        z = z + w;
    }
    return true;
}

// prod_d (1 + z_d) - 1, expanded.
double nonzero_mass(const double z[3]) {
    return (((((z[0] + z[1]) + z[2]) + z[0] * z[1]) + z[0] * z[2]) + z[1] * z[2]) + (z[0] * z[1]) * z[2];
}

// Smallest j in [j0, jmax] with t < T[j] (T non-decreasing); jmax if none.
__device__ __forceinline__ int32_t upper_index(const double *__restrict__ T, int32_t j0, int32_t jmax, double t) {
    if (!(t < T[jmax])) return jmax;
    int32_t lo = j0, hi = jmax;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (t < T[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) k_pg_kseq(const PgStratum *__restrict__ strata,
                                                      const int32_t *__restrict__ slot_stratum, int32_t P_eff,
                                                      int32_t P_batch, const double *__restrict__ tab,
                                                      uint64_t seed, int64_t n_sets, int4 *__restrict__ kseq) {
    const int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (g >= n_sets * P_batch) return;
    const int64_t t = g / P_batch;
    const int32_t eta = (int32_t)(g % P_batch);
    if (eta >= P_eff) {
        kseq[g] = make_int4(1, 0, 0, kPgPad);
        return;
    }
    const PgStratum st = strata[slot_stratum[eta]];
    uint64_t ra[4] = {(uint64_t)t, (uint64_t)eta, 0, 0}, rb[4] = {(uint64_t)t, (uint64_t)eta, 1, 0};
    philox4x64_10(ra, seed, 0x8000000000000002ull);
    philox4x64_10(rb, seed, 0x8000000000000002ull);
    const int first = unit53(ra[0]) < st.thr1 ? 0 : (unit53(ra[1]) < st.thr2 ? 1 : 2);
    int m[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double *T = tab + st.tab_off[d];
        const int32_t jm = st.jmax[d];
        const double u = unit53(rb[d]);
        const double Tn = T[jm];
        int32_t j;
        if (d < first) j = 0;
        else if (d == first) j = upper_index(T, 1, jm, T[0] + u * (Tn - T[0]));
        else j = upper_index(T, 0, jm, u * Tn);
        m[d] = ((ra[2] >> d) & 1u) ? -j : j;
    }
    kseq[g] = make_int4(m[0], m[1], m[2], st.l);
}

}  // namespace

bool pg_plan(const double *omega, const double *s, int M, const double L[3], int P, PgPlan &plan) {
    plan = PgPlan{};
    plan.P_l.assign((size_t)M + 1, 0);
    plan.S_l.assign((size_t)M + 1, 0.0);
    std::vector<double> T[3];
    double tot = 0.0;
    for (int l = 0; l <= M; ++l) {
        double z[3];
        int32_t jm;
        for (int d = 0; d < 3; ++d)
            if (!coord_table(s[l], L[d], T[d], jm, z[d])) return false;
        plan.S_l[l] = omega[l] * s[l] * s[l] * s[l] * nonzero_mass(z);
        tot += plan.S_l[l];
    }
    for (int l = 0; l <= M; ++l) {
        if (!(plan.S_l[l] > 1e-16 * tot)) continue;
        plan.P_l[l] = (int32_t)std::ceil((double)P * plan.S_l[l] / tot);
        PgStratum st{};
        st.l = l;
        double z[3];
        for (int d = 0; d < 3; ++d) {
            coord_table(s[l], L[d], T[d], st.jmax[d], z[d]);
            st.tab_off[d] = (int64_t)plan.tables.size();
            plan.tables.insert(plan.tables.end(), T[d].begin(), T[d].end());
        }
        st.thr1 = ((z[0] * (1.0 + z[1])) * (1.0 + z[2])) / nonzero_mass(z);
        const double den2 = (z[1] + z[2]) + z[1] * z[2];
        st.thr2 = den2 > 0.0 ? (z[1] * (1.0 + z[2])) / den2 : 1.0;
        plan.slot_stratum.insert(plan.slot_stratum.end(), (size_t)plan.P_l[l], (int32_t)plan.strata.size());
        plan.strata.push_back(st);
        plan.P_eff += plan.P_l[l];
    }
    return true;
}

cudaError_t launch_pg_sampler(const PgStratum *strata, const int32_t *slot_stratum, int32_t P_eff, int32_t P_batch,
                              const double *tables, uint64_t seed, int64_t n_sets, int4 *kseq, cudaStream_t st,
                              const Prof *prof) {
    ProfScope ps(prof, "pg_sampler");
    const int64_t total = n_sets * P_batch;
    if (total == 0) return cudaSuccess;
    k_pg_kseq<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(strata, slot_stratum, P_eff,
                                                                                   P_batch, tables, seed, n_sets,
                                                                                   kseq);
    return cudaGetLastError();
}

}  // namespace rbsog
