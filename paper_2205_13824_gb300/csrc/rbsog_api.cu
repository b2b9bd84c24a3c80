// C ABI of librbsog (declared in include/rbsog.h).  The engine advances a
// batch of independent systems laid out back to back in device memory; a
// single-system context is a batch of one.  Host code here sets up the
// parameters (SOG solve, S, cell grids, launch layouts, work tables) and
// sequences the device kernels of one force evaluation and one
// velocity-Verlet step, which is captured once into a CUDA graph and
// replayed: one graph launch advances every system of the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "../../include/rbsog.h"
#include "rbsog_kernels.cuh"

using namespace rbsog;

namespace {

constexpr double kPi = 3.14159265358979323846;
// resident rho-sweep blocks per SM when the sweep runs beside the list force
// (measured at N = 1,048,576, P = 500: 3 beats 2, 4 and 6)
constexpr int kSweepBesideNear = 3;

struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};

// Launch-shape tunables chosen by rbsog_batch_autotune, remembered per size
// class (floor(log2 n)), P and precision for every later context in the
// process.  home: near-field home particles per block; tile: rho-sweep
// particles per tile (0 = default rule).
struct Tune {
    int home = 120;
    int tile = 0;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, Tune> g_tune;

std::tuple<int, int, int> tune_key(int64_t n, int P, int prec) {
    int c = 0;
    while ((int64_t(1) << (c + 1)) <= n) ++c;
    return std::make_tuple(c, P, prec);
}

Tune tune_for(int64_t n, int P, int prec) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(n, P, prec));
    if (it != g_tune.end()) return it->second;
    Tune t;
    // FP64 systems whose stencil rows are split over the warps: about one
    // run of 32 home particles per block keeps the four warps' shares even
    if (prec == RBSOG_FP64 && n < kNearSplitMaxN) t.home = 32;
    return t;
}

}  // namespace

struct rbsog_ctx {
    int32_t n_sys = 0;
    std::vector<int64_t> n_per, p_off;
    int64_t n_total = 0;
    int device = 0;
    cudaStream_t user = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_q = nullptr, ev_x = nullptr, ev_io = nullptr;   // rbsog_step_io
    cudaStream_t io = nullptr;                                     // rbsog_step_io downloads
    cudaGraphExec_t graph_tail = nullptr;   // a step without its kick-drift (rbsog_step_io)
    cudaGraphExec_t graph_e = nullptr;      // a whole step with energies (the last of a call)
    cudaGraphExec_t graph_fused = nullptr;  // a step without its kick-drift whose scatter runs
                                            // the next step's kick-drift (rbsog_batch_step)
    std::string err;

    bool have_params = false;
    std::vector<char> have_state, force_valid;
    std::vector<rbsog_params> p;
    // shared SOG (every system of a batch uses the same b, sigma, omega0, M, r_c)
    std::vector<double> omega, s;
    double sigma = 0, omega0 = 0;
    NearSog nsog{};
    int32_t P = 0, precision = 0;
    std::vector<SysDesc> desc;
    std::vector<double> S, sum_q2;
    std::vector<int64_t> n_chains, host_cursor;
    std::vector<int> chain_len;
    std::vector<Tune> tune;            // per-system launch-shape tunables
    int64_t ncell_total = 0;
    int max_cap = 256, max_tile_p = 128;
    std::vector<int2> pblk, nblk, sblk;

    // device buffers
    double4_32a *posq = nullptr, *vel = nullptr, *force = nullptr, *fnear = nullptr, *sp64 = nullptr;
    uint4 *sp32 = nullptr;
    double *staging = nullptr;        // [10 n_total]: three [n][3] regions and one [n]
    double *qpart = nullptr;          // [3 ceil(n_total / 256)] charge sums per block
    double *h_qpart = nullptr;        // pinned mirror of qpart
    int32_t *nbr_sorted = nullptr, *i32_tmp = nullptr;
    CellBuffers cb{};
    double *kpart = nullptr;
    int4 *kseq = nullptr;
    int4 *kfold = nullptr;       // folded k-sets (mixture sampler); see FoldSys
    int32_t *kcount = nullptr;   // distinct runs per k-set
    int64_t *cursor = nullptr, *step_ctr = nullptr;
    double2 *rho_part = nullptr, *rho = nullptr, *epart = nullptr;
    void *ktab = nullptr;
    double *energy = nullptr;
    int32_t *err_flag = nullptr;
    int4 *m_tmp = nullptr;
    int32_t *m3_tmp = nullptr;
    SysDesc *d_desc = nullptr;
    int2 *d_pblk = nullptr, *d_nblk = nullptr, *d_sblk = nullptr;
    int32_t *d_cell_sys = nullptr;
    int32_t *d_mask = nullptr;        // [n_sys] systems that need a force evaluation
    double4_32a *fin_part = nullptr;  // [n_sys * kFinChunks] finalize chunk sums
    double4_32a *dpart = nullptr;     // [particle blocks] dipole-moment partials (boundary terms)
    double4_32a *dip = nullptr;       // [n_sys] boundary force factor per unit charge
    bool any_boundary = false;        // some system has a non-tinfoil boundary
    unsigned int *fin_count = nullptr;   // [n_sys] finalize chunks done
    // per-system step budgets (used by the serving engine): a system whose
    // budget reaches 0 is frozen by every step kernel
    bool use_budget = false;
    int64_t *d_remaining = nullptr;
    std::vector<int64_t> remaining_host;
    // FP32C neighbour lists (Verlet lists with a skin): on when every system's
    // box holds at least 3 cells of side r_c + skin per side
    bool use_list = false;
    double skin = 0.0;
    int32_t list_cap = 0;
    uint4 *sp32c = nullptr, *xref = nullptr, *lpos = nullptr;
    int32_t *linv = nullptr;
    float4 *d_ltab = nullptr;            // combined G/F table of the list path [kLTabN]
    bool use_cs = false;                 // the list path runs the core-shell kernel
    CoreShellDev cs{};
    float4 *d_cstab = nullptr;           // its shell table [cs.n_tab]
    std::vector<float4> h_ltab;
    int32_t *nbr_list = nullptr, *nbr_cnt = nullptr, *list_perm = nullptr, *d_rebuild = nullptr;
    // per-Gaussian independent sampling (rbsog_params.sampler = 1)
    bool pg_sampler = false;
    double *d_kw = nullptr;           // [n_sys * kKwStride] per-stratum estimator weights
    // observables of Appendix A (rbsog_observe_*), single system
    int32_t obs_lags = 0, obs_every = 0, obs_slots = 0;
    int64_t obs_frame = 0;
    double4_32a *obs_xprev = nullptr, *obs_u = nullptr, *obs_ring_u = nullptr, *obs_ring_v = nullptr;
    double2 *obs_part = nullptr;
    double *obs_acc = nullptr;        // [4 n_lags]: MSD sums, VACF sums, then the result
    int64_t *obs_count = nullptr;     // [n_lags]
    // pinned host mirrors
    double *h_energy = nullptr;
    int32_t *h_err = nullptr;
    int64_t *h_i64 = nullptr;

    cudaGraphExec_t graph = nullptr;  // a whole step without energies
    bool capturing = false;           // enqueue_step is being captured into the step graph
    cudaStream_t side = nullptr;      // captures the bodies of conditional graph nodes
    cudaStream_t far = nullptr;       // the rho(k) sweep and combine, beside the near field
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    bool profiling = false;
    std::vector<ProfRec> prof_open, prof_done;
    std::vector<cudaEvent_t> ev_pool;
    std::map<std::string, std::pair<int64_t, double>> prof_acc;
    Prof prof_hook{};
};

namespace {

rbsog_status fail(rbsog_ctx *c, rbsog_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, RBSOG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t dalloc(T **ptr, size_t count) {
    if (*ptr) {
        cudaFree(*ptr);
        *ptr = nullptr;
    }
    if (count == 0) count = 1;
    return cudaMalloc((void **)ptr, sizeof(T) * count);
}

template <class T>
void dfree(T **ptr) {
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
}

void prof_mark(void *self, const char *name, int begin) {
    rbsog_ctx *c = static_cast<rbsog_ctx *>(self);
    auto get = [c]() {
        cudaEvent_t e;
        if (!c->ev_pool.empty()) {
            e = c->ev_pool.back();
            c->ev_pool.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    };
    if (begin) {
        ProfRec r{name, get(), nullptr};
        cudaEventRecord(r.a, c->st);
        c->prof_open.push_back(r);
    } else if (!c->prof_open.empty()) {
        ProfRec r = c->prof_open.back();
        c->prof_open.pop_back();
        r.b = get();
        cudaEventRecord(r.b, c->st);
        c->prof_done.push_back(r);
    }
}

const Prof *prof_of(rbsog_ctx *c) { return c->profiling ? &c->prof_hook : nullptr; }

// ---- SOG set-up on the host (Eqs. 2.9-2.11, 3.16-3.17) ---------------------------

void bsa_coeffs(double b, double sigma, int M, std::vector<double> &w, std::vector<double> &s) {
    w.assign(M + 1, 0.0);
    s.assign(M + 1, 0.0);
    const double w1 = std::sqrt(2.0 / kPi) * std::log(b) / sigma;
    for (int l = 0; l <= M; ++l) {
        w[l] = w1 * std::pow(b, -(double)l);
        s[l] = std::sqrt(2.0) * sigma * std::pow(b, (double)l);
    }
}

int untruncated_terms(double b) { return (int)std::ceil(40.0 * std::log(10.0) / std::log(b)); }

// C0 weight of the narrowest Gaussian: F_M(r_c) = 1/r_c with l >= 1 fixed.
double c0_weight(double b, double sigma, double rc) {
    std::vector<double> w, s;
    const int Mu = untruncated_terms(b);
    bsa_coeffs(b, sigma, Mu, w, s);
    double tail = 0.0;
    for (int l = Mu; l >= 1; --l) tail += w[l] * std::exp(-(rc * rc) / (s[l] * s[l]));
    return (1.0 / rc - tail) * std::exp((rc * rc) / (s[0] * s[0]));
}

// r_c^2 N'(r_c) with N = 1/r - F (zero at the C1 solution).
double c1_defect(double b, double sigma, double rc) {
    std::vector<double> w, s;
    const int Mu = untruncated_terms(b);
    bsa_coeffs(b, sigma, Mu, w, s);
    w[0] = c0_weight(b, sigma, rc);
    double d = 0.0;
    for (int l = Mu; l >= 0; --l) d += w[l] * (2.0 * rc / (s[l] * s[l])) * std::exp(-(rc * rc) / (s[l] * s[l]));
    return rc * rc * d - 1.0;
}

// Solve sigma on a log grid + bisection; choose the root whose w_0 is
// closest to the bilateral-series weight.
bool solve_sigma_uncached(double b, double rc, double &sigma, double &w0) {
    const int ngrid = 2400;
    const double lo = 0.04 * rc, hi = 2.5 * rc;
    double best = -1.0, best_dev = 1e300;
    double sa = lo, fa = c1_defect(b, lo, rc);
    for (int i = 1; i <= ngrid; ++i) {
        const double sb = lo * std::exp(std::log(hi / lo) * i / ngrid);
        const double fb = c1_defect(b, sb, rc);
        if ((fa > 0) != (fb > 0)) {
            double a = sa, c = sb, fla = fa;
            for (int it = 0; it < 300 && (c - a) > 4e-16 * c; ++it) {
                const double m = 0.5 * (a + c);
                const double fm = c1_defect(b, m, rc);
                if ((fm > 0) == (fla > 0)) {
                    a = m;
                    fla = fm;
                } else {
                    c = m;
                }
            }
            const double root = 0.5 * (a + c);
            const double dev = std::fabs(c0_weight(b, root, rc) / (std::sqrt(2.0 / kPi) * std::log(b) / root) - 1.0);
            if (dev < best_dev) {
                best_dev = dev;
                best = root;
            }
        }
        sa = sb;
        fa = fb;
    }
    if (best < 0) return false;
    sigma = best;
    w0 = c0_weight(b, best, rc);
    return true;
}

// The solve costs a few tens of milliseconds (thousands of untruncated series
// evaluations); its result depends on (b, r_c) only and is remembered for the
// process, so contexts that are rebuilt often (the serving engine) pay once.
std::mutex g_sigma_mu;
std::map<std::pair<double, double>, std::pair<double, double>> g_sigma;

bool solve_sigma(double b, double rc, double &sigma, double &w0) {
    {
        std::lock_guard<std::mutex> lk(g_sigma_mu);
        auto it = g_sigma.find({b, rc});
        if (it != g_sigma.end()) {
            sigma = it->second.first;
            w0 = it->second.second;
            return true;
        }
    }
    if (!solve_sigma_uncached(b, rc, sigma, w0)) return false;
    std::lock_guard<std::mutex> lk(g_sigma_mu);
    g_sigma[{b, rc}] = {sigma, w0};
    return true;
}

// theta sum H(s, L) = sum_m exp(-(pi s m / L)^2), evaluated in whichever of
// its two Poisson-dual forms converges faster.
double theta_sum(double s, double L) {
    if (s >= L) {
        const double a = (kPi * s / L) * (kPi * s / L);
        double h = 1.0;
        for (int m = 1; m < 1000000; ++m) {
            const double t = std::exp(-a * m * m);
            h += 2.0 * t;
            if (t < 1e-24 * h) break;
        }
        return h;
    }
    const double a = (L / s) * (L / s);
    double h = 1.0;
    for (int m = 1; m < 1000000; ++m) {
        const double t = std::exp(-a * m * m);
        h += 2.0 * t;
        if (t < 1e-24 * h) break;
    }
    return h * L / (std::sqrt(kPi) * s);
}

void build_near_sog(NearSog &ns, const std::vector<double> &omega, const std::vector<double> &s, int M,
                    double rc) {
    std::memset(&ns, 0, sizeof ns);
    int nd = 0;
    while (nd <= M && s[nd] < 2.0 * rc) ++nd;
    ns.n_direct = nd;
    for (int l = 0; l < nd; ++l) {
        ns.omega[l] = omega[l];
        ns.inv_s2[l] = 1.0 / (s[l] * s[l]);
        ns.omega_f[l] = (float)ns.omega[l];
        ns.omega_s2_f[l] = (float)(ns.omega[l] * ns.inv_s2[l]);
        ns.inv_s2_log2e_f[l] = (float)(ns.inv_s2[l] * 1.4426950408889634);
    }
    ns.n_taylor = 0;
    if (nd <= M) {
        // A[n] = sum_{l >= nd} w_l s_l^{-2n}
        double A[kMaxTaylor + 2];
        for (int n = 0; n < kMaxTaylor + 2; ++n) {
            A[n] = 0.0;
            for (int l = M; l >= nd; --l) A[n] += omega[l] * std::pow(s[l], -2.0 * n);
        }
        const double xmax = rc * rc / (s[nd] * s[nd]);
        // smallest number of terms whose first omitted term x^n / n! is below tol
        auto terms = [xmax](double tol) {
            int nt = 1;
            double fact = 1.0, xp = 1.0;
            while (nt < kMaxTaylor) {
                xp *= xmax;
                fact *= nt;
                if (xp / fact < tol) break;
                ++nt;
            }
            return nt;
        };
        const int nt = terms(1e-19);
        ns.n_taylor = nt;
        ns.n_taylor_f = terms(1e-10);
        double f = 1.0;
        for (int n = 0; n < nt; ++n) {
            if (n > 0) f *= n;
            const double sg = (n % 2) ? -1.0 : 1.0;
            ns.tay_f[n] = sg * A[n] / f;
            ns.tay_g[n] = sg * A[n + 1] / f;
            ns.tay_f_f[n] = (float)ns.tay_f[n];
            ns.tay_g_f[n] = (float)ns.tay_g[n];
        }
    }
}

// Interpolating cubic through Chebyshev nodes of each table interval, in
// monomial form in the interval's local coordinate s in [0, 1).  For the
// production set the largest error (relative to G(0) and F(0)) is at FP32
// rounding level; it is recorded in tab_err.
void build_sog_tables(NearSog &ns, const std::vector<double> &omega, const std::vector<double> &s, int M,
                      double rc) {
    const double du = rc * rc / kTabN;
    auto G = [&](double uu) {
        double v = 0.0;
        for (int l = M; l >= 0; --l) v += omega[l] / (s[l] * s[l]) * std::exp(-uu / (s[l] * s[l]));
        return v;
    };
    auto F = [&](double uu) {
        double v = 0.0;
        for (int l = M; l >= 0; --l) v += omega[l] * std::exp(-uu / (s[l] * s[l]));
        return v;
    };
    double sn[4];
    for (int j = 0; j < 4; ++j) sn[j] = 0.5 - 0.5 * std::cos((2 * j + 1) * kPi / 8.0);
    auto fit = [&](auto fn, int k, double c[4]) {
        // Vandermonde solve with partial pivoting (4 x 4)
        double A[4][5];
        for (int j = 0; j < 4; ++j) {
            double p = 1.0;
            for (int m = 0; m < 4; ++m) {
                A[j][m] = p;
                p *= sn[j];
            }
            A[j][4] = fn((k + sn[j]) * du);
        }
        for (int col = 0; col < 4; ++col) {
            int piv = col;
            for (int r = col + 1; r < 4; ++r)
                if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
            for (int m = 0; m < 5; ++m) std::swap(A[col][m], A[piv][m]);
            for (int r = 0; r < 4; ++r) {
                if (r == col) continue;
                const double f = A[r][col] / A[col][col];
                for (int m = col; m < 5; ++m) A[r][m] -= f * A[col][m];
            }
        }
        for (int m = 0; m < 4; ++m) c[m] = A[m][4] / A[m][m];
    };
    const double g0 = G(0.0), f0 = F(0.0);
    double err = 0.0;
    for (int k = 0; k < kTabN; ++k) {
        double cg[4], cf[4];
        fit(G, k, cg);
        fit(F, k, cf);
        ns.tab_g[k] = make_float4((float)cg[0], (float)cg[1], (float)cg[2], (float)cg[3]);
        ns.tab_f[k] = make_float4((float)cf[0], (float)cf[1], (float)cf[2], (float)cf[3]);
        for (int q = 0; q <= 16; ++q) {
            const double x = q / 16.0;
            const float4 a = ns.tab_g[k], b = ns.tab_f[k];
            const double pg = ((double)a.w * x + a.z) * x * x + (double)a.y * x + a.x;
            const double pf = ((double)b.w * x + b.z) * x * x + (double)b.y * x + b.x;
            err = std::max(err, std::fabs(pg - G((k + x) * du)) / g0);
            err = std::max(err, std::fabs(pf - F((k + x) * du)) / f0);
        }
    }
    ns.tab_scale = (float)(kTabN / (rc * rc));
    ns.tab_err = (float)err;
}

constexpr double kListTabTol = 2e-6;   // largest accepted error of the list path's table

// Combined table of the neighbour-list path: G interpolated by a quadratic
// through the 3 Chebyshev nodes of each interval, F at each interval start
// (F between starts follows from dF/du = -G).  Returns the largest error of
// the FP32 entries for G and F over 33 points per interval, relative to
// G(0) and F(0).
double build_list_table(NearSog &ns, std::vector<float4> &tab, const std::vector<double> &omega,
                        const std::vector<double> &s, int M, double rc) {
    const double h = rc * rc / kLTabN;
    auto G = [&](double uu) {
        double v = 0.0;
        for (int l = M; l >= 0; --l) v += omega[l] / (s[l] * s[l]) * std::exp(-uu / (s[l] * s[l]));
        return v;
    };
    auto F = [&](double uu) {
        double v = 0.0;
        for (int l = M; l >= 0; --l) v += omega[l] * std::exp(-uu / (s[l] * s[l]));
        return v;
    };
    double sn[3];
    for (int j = 0; j < 3; ++j) sn[j] = 0.5 - 0.5 * std::cos((2 * j + 1) * kPi / 6.0);
    const double g0 = G(0.0), f0 = F(0.0);
    double err = 0.0;
    tab.assign(kLTabN, float4{});
    for (int k = 0; k < kLTabN; ++k) {
        // Lagrange form through the nodes, expanded to monomials in s
        double c[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < 3; ++j) {
            const double a = sn[(j + 1) % 3], b = sn[(j + 2) % 3];
            const double wgt = G((k + sn[j]) * h) / ((sn[j] - a) * (sn[j] - b));
            c[0] += wgt * a * b;
            c[1] -= wgt * (a + b);
            c[2] += wgt;
        }
        const float4 e = make_float4((float)c[0], (float)c[1], (float)c[2], (float)F(k * h));
        tab[k] = e;
        for (int q = 0; q <= 32; ++q) {
            const double x = q / 32.0;
            const double pg = ((double)e.z * x + e.y) * x + e.x;
            const double pf = (double)e.w - h * x * (((double)e.z / 3.0 * x + 0.5 * e.y) * x + e.x);
            err = std::max(err, std::fabs(pg - G((k + x) * h)) / g0);
            err = std::max(err, std::fabs(pf - F((k + x) * h)) / f0);
        }
    }
    ns.ltab_scale = (float)(kLTabN / (rc * rc));
    ns.ltab_h = (float)h;
    ns.ltab_err = (float)err;
    return err;
}

// Core-shell kernel of the list path (Sec. 3.4): Taylor coefficients of the
// core (signs of the series folded in) and the shell table over the 2^b_exp
// octaves of r^2 from the octave of r_in^2 (b_exp the smallest of 1..3 that
// reaches r_c^2).  Each bin holds the exact kernel (force factor
// u^{-3/2} - 2 G(u), pair energy u^{-1/2} - F_M(u)) at its lower end and the
// change to its upper end.  False when 8 octaves do not reach r_c^2.
bool build_coreshell(CoreShellDev &cs, std::vector<float4> &tab, const std::vector<double> &omega,
                     const std::vector<double> &s, int M, double rc, double r_in) {
    auto fbits = [](float v) {
        uint32_t b;
        std::memcpy(&b, &v, sizeof b);
        return b;
    };
    const int e0 = (int)((fbits((float)(r_in * r_in)) >> 23) & 0xffu);
    const int e1 = (int)((fbits((float)(rc * rc)) >> 23) & 0xffu);
    int be = 1;
    while (be <= 3 && e1 - e0 >= (1 << be)) ++be;
    if (be > 3) return false;
    std::memset(&cs, 0, sizeof cs);
    double fact = 1.0;
    for (int i = 0; i <= kCsQ; ++i) {
        if (i > 0) fact *= i;
        double A = 0.0, Bc = 0.0;          // A_{i+1} and B_i
        for (int l = 0; l <= M; ++l) {
            const double t = std::pow(s[l] * s[l], -(double)i) / fact;
            Bc += omega[l] * t;
            A += omega[l] * t / (s[l] * s[l]);
        }
        const double sg = (i % 2) ? -1.0 : 1.0;
        if (i < kCsQ) cs.a[i] = (float)(sg * A);
        cs.b[i] = (float)(sg * Bc);
    }
    cs.rin2 = (float)(r_in * r_in);
    cs.emask = (1u << be) - 1u;
    cs.n_tab = 1 << (be + kCsManBits);
    tab.assign((size_t)cs.n_tab, float4{});
    auto kern = [&](double u, double &g, double &n) {
        double G = 0.0, F = 0.0;
        for (int l = M; l >= 0; --l) {
            const double e = std::exp(-u / (s[l] * s[l]));
            G += omega[l] / (s[l] * s[l]) * e;
            F += omega[l] * e;
        }
        g = std::pow(u, -1.5) - 2.0 * G;
        n = 1.0 / std::sqrt(u) - F;
    };
    const int nm = 1 << kCsManBits;
    for (int E = e0; E < e0 + (1 << be); ++E)
        for (int m = 0; m < nm; ++m) {
            const double u0 = std::ldexp(1.0 + (double)m / nm, E - 127);
            const double u1 = std::ldexp(1.0 + (double)(m + 1) / nm, E - 127);
            double g0, n0, g1, n1;
            kern(u0, g0, n0);
            kern(u1, g1, n1);
            tab[(size_t)(((uint32_t)E & cs.emask) << kCsManBits) | (size_t)m] =
                make_float4((float)g0, (float)(g1 - g0), (float)n0, (float)(n1 - n0));
        }
    return true;
}

rbsog_status enter(rbsog_ctx *ctx) {
    CK(cudaSetDevice(ctx->device));
    CK(cudaEventRecord(ctx->ev_in, ctx->user));
    CK(cudaStreamWaitEvent(ctx->st, ctx->ev_in, 0));
    return RBSOG_OK;
}

rbsog_status leave(rbsog_ctx *ctx) {
    CK(cudaEventRecord(ctx->ev_out, ctx->st));
    CK(cudaStreamWaitEvent(ctx->user, ctx->ev_out, 0));
    return RBSOG_OK;
}

BatchView view(rbsog_ctx *c, const int4 *m_explicit = nullptr, int32_t P = -1) {
    BatchView v{};
    v.sys = c->d_desc;
    v.n_sys = c->n_sys;
    v.P = P > 0 ? P : c->P;
    v.n_total = c->n_total;
    v.ncell_total = c->ncell_total;
    v.pblk = c->d_pblk;
    v.n_pblk = (int32_t)c->pblk.size();
    v.nblk = c->d_nblk;
    v.n_nblk = (int32_t)c->nblk.size();
    v.sblk = c->d_sblk;
    v.n_sblk = (int32_t)c->sblk.size();
    v.cell_sys = c->d_cell_sys;
    v.cursor = c->cursor;
    v.step = c->step_ctr;
    v.kseq = c->kseq;
    v.kfold = m_explicit ? nullptr : c->kfold;
    v.kcount = m_explicit ? nullptr : c->kcount;
    v.m_explicit = m_explicit;
    v.max_cap = c->max_cap;
    v.max_tile_p = c->max_tile_p;
    v.force_mask = nullptr;
    v.remaining = c->use_budget ? c->d_remaining : nullptr;
    v.list_cap = c->use_list ? c->list_cap : 0;
    v.precision = c->precision;
    v.fin_part = c->fin_part;
    v.fin_count = c->fin_count;
    v.kw = (c->pg_sampler && !m_explicit) ? c->d_kw : nullptr;
    v.lpos = c->use_list ? c->lpos : nullptr;
    v.linv = c->use_list ? c->linv : nullptr;
    return v;
}

// Cell list + near field + far field for the current positions; total force
// into c->force (caller order).  With a mask, only masked systems take the
// new forces, energies and k-set.
// fuse_kick: the FP32C scatter also runs the step's second half kick (the
// caller then launches no kick); valid only without a boundary term, which
// adds to the force after the scatter.
// fuse_drift (with fuse_kick, neighbour lists): the scatter also runs the
// next step's half kick and drift.
// energy = false (neighbour lists): the list force leaves the pair energies
// out, for steps whose energies nobody reads (not the last step of a call;
// a system on its last budgeted step still gets them).
rbsog_status enqueue_forces(rbsog_ctx *ctx, const BatchView &bv, int32_t *nbr_sorted,
                            double4_32a *force_out = nullptr, bool packed = false, bool fuse_kick = false,
                            bool fuse_drift = false, bool energy = true) {
    const Prof *pf = prof_of(ctx);
    const int prec = ctx->precision;
    double4_32a *kv = fuse_kick ? ctx->vel : nullptr;
    double *kp = fuse_kick ? ctx->kpart : nullptr;
    if (ctx->use_list && !nbr_sorted) {
        // neighbour lists: caller-order fixed-point positions (written by the
        // kick-drift in a step), cell list and lists of the flagged systems,
        // listed pairs, far field in caller order
        if (!packed) CK(launch_fix_pack(bv, ctx->posq, ctx->sp32c, ctx->xref, ctx->d_rebuild, ctx->st, pf));
        // The rho(k) sweep and combine need only the caller-order positions:
        // they run on a second stream beside the list rebuild and the list
        // force (MUFU-bound next to an L1-bound kernel), joined before the
        // scatter.  Profiled launches stay on one stream, so that each
        // kernel's event pair times that kernel alone.
        const bool fork = pf == nullptr;
        if (fork) {
            CK(cudaEventRecord(ctx->ev_fork, ctx->st));
            CK(cudaStreamWaitEvent(ctx->far, ctx->ev_fork, 0));
            CK(launch_rho_sweep(prec, bv, ctx->sp64, ctx->sp32c, ctx->rho_part, ctx->far, pf, kSweepBesideNear));
            CK(launch_rho_combine(prec, bv, ctx->rho_part, ctx->rho, ctx->ktab, ctx->far, pf));
            CK(cudaEventRecord(ctx->ev_join, ctx->far));
        }
        auto rebuild = [&](cudaStream_t s2) -> rbsog_status {
            CK(launch_build_cells(bv, ctx->posq, ctx->cb, prec, ctx->sp64, ctx->sp32, s2, pf,
                                  ctx->d_rebuild + ctx->n_sys));
            CK(launch_list_build(bv, ctx->cb.start, ctx->sp32, ctx->cb.perm, ctx->d_rebuild, ctx->nbr_list,
                                 ctx->nbr_cnt, ctx->list_perm, ctx->xref, ctx->err_flag, s2, pf));
            return RBSOG_OK;
        };
        if (ctx->capturing) {
            // captured step: the rebuild kernels form the body of a
            // conditional node, so steps without a rebuild launch none of them
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            CK(cudaStreamGetCaptureInfo(ctx->st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
            cudaGraphConditionalHandle h;
            CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
            CK(launch_rebuild_condition(h, ctx->d_rebuild + ctx->n_sys, ctx->st));
            CK(cudaStreamGetCaptureInfo(ctx->st, &cs, nullptr, &g, &deps, nullptr, &nd));
            cudaGraphNodeParams np{};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeIf;
            np.conditional.size = 1;
            cudaGraphNode_t cn;
            CK(cudaGraphAddNode(&cn, g, deps, nullptr, nd, &np));
            CK(cudaStreamBeginCaptureToGraph(ctx->side, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
            rbsog_status rs = rebuild(ctx->side);
            cudaGraph_t body = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(ctx->side, &body);
            if (rs != RBSOG_OK) return rs;
            CK(ce);
            CK(cudaStreamUpdateCaptureDependencies(ctx->st, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
        } else {
            // eager launches: the rebuild kernels are gated on the device;
            // profiled steps read the flag first and launch them only on a
            // rebuild, so that their timings are those of real rebuilds
            bool run = true;
            if (pf) {
                int32_t *hf = reinterpret_cast<int32_t *>(ctx->h_i64 + 3);
                CK(cudaMemcpyAsync(hf, ctx->d_rebuild + ctx->n_sys, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
                CK(cudaStreamSynchronize(ctx->st));
                run = *hf != 0;
            }
            if (run) {
                rbsog_status rs = rebuild(ctx->st);
                if (rs != RBSOG_OK) return rs;
            }
        }
        CK(launch_near_list(bv, ctx->nsog, ctx->d_ltab, ctx->nbr_list, ctx->nbr_cnt, ctx->list_perm, ctx->fnear,
                            ctx->st, pf, ctx->use_cs ? &ctx->cs : nullptr, ctx->d_cstab, energy));
        if (fork) {
            CK(cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0));
        } else {
            CK(launch_rho_sweep(prec, bv, ctx->sp64, ctx->sp32c, ctx->rho_part, ctx->st, pf));
            CK(launch_rho_combine(prec, bv, ctx->rho_part, ctx->rho, ctx->ktab, ctx->st, pf));
        }
        const DriftOut dr{ctx->posq, ctx->sp32c, ctx->xref, ctx->d_rebuild};
        CK(launch_far_scatter(prec, bv, ctx->sp64, ctx->sp32c, ctx->ktab, ctx->fnear, nullptr,
                              force_out ? force_out : ctx->force, ctx->err_flag, ctx->st, pf, ctx->epart, kv, kp,
                              fuse_kick && fuse_drift ? &dr : nullptr));
        if (ctx->any_boundary)
            CK(launch_boundary(bv, ctx->posq, ctx->dpart, ctx->dip, ctx->energy, force_out ? force_out : ctx->force,
                               ctx->st, pf));
        return RBSOG_OK;
    }
    CK(launch_build_cells(bv, ctx->posq, ctx->cb, prec, ctx->sp64, ctx->sp32, ctx->st, pf));
    CK(launch_near(prec, bv, ctx->nsog, ctx->cb.start, ctx->sp64, ctx->sp32, ctx->fnear, ctx->epart, nbr_sorted,
                   ctx->st, pf));
    CK(launch_rho_sweep(prec, bv, ctx->sp64, ctx->sp32, ctx->rho_part, ctx->st, pf));
    CK(launch_rho_combine(prec, bv, ctx->rho_part, ctx->rho, ctx->ktab, ctx->st, pf));
    CK(launch_far_scatter(prec, bv, ctx->sp64, ctx->sp32, ctx->ktab, ctx->fnear, ctx->cb.perm,
                          force_out ? force_out : ctx->force, ctx->err_flag, ctx->st, pf, nullptr, kv, kp));
    if (ctx->any_boundary)
        CK(launch_boundary(bv, ctx->posq, ctx->dpart, ctx->dip, ctx->energy, force_out ? force_out : ctx->force,
                           ctx->st, pf));
    return RBSOG_OK;
}

// A step is the kick-drift followed by the tail (forces, second kick,
// energies, thermostat, step counters); rbsog_step_io launches the two parts
// separately for its last step so that the positions can be copied out while
// the tail runs.
rbsog_status enqueue_kick_drift(rbsog_ctx *ctx) {
    const Prof *pf = prof_of(ctx);
    const BatchView bv = view(ctx);
    if (ctx->use_list)
        CK(launch_kick_drift(bv, ctx->posq, ctx->vel, ctx->force, ctx->st, pf, ctx->sp32c, ctx->xref, ctx->d_rebuild));
    else
        CK(launch_kick_drift(bv, ctx->posq, ctx->vel, ctx->force, ctx->st, pf));
    return RBSOG_OK;
}

// drift_next: the step's scatter also runs the next step's kick-drift
// (drift_fusable only).  energy: the step's energies are computed (the last
// step of a call); other steps may leave the pair energies out.
rbsog_status enqueue_step_tail(rbsog_ctx *ctx, bool drift_next = false, bool energy = true) {
    const Prof *pf = prof_of(ctx);
    const BatchView bv = view(ctx);
    const bool fused = ctx->precision == RBSOG_FP32C && !ctx->any_boundary;
    rbsog_status s = enqueue_forces(ctx, bv, nullptr, nullptr, ctx->use_list, fused, drift_next && fused, energy);
    if (s != RBSOG_OK) return s;
    if (!fused) CK(launch_kick(bv, ctx->vel, ctx->force, ctx->kpart, ctx->st, pf));
    bool thermo = false;
    for (auto &pp : ctx->p) thermo = thermo || (pp.tau_T > 0.0 && pp.thermostat != 1);
    // the sums of finalize feed the thermostats and the reported energies;
    // a step with neither only advances the counters
    if (energy || thermo || ctx->use_budget)
        CK(launch_finalize(bv, ctx->epart, ctx->rho, ctx->kpart, 1, ctx->energy, 1, ctx->st, pf));
    else
        CK(launch_finalize_counters(bv, 1, ctx->st, pf));
    if (thermo) CK(launch_rescale(bv, ctx->vel, ctx->energy, ctx->st, pf));
    CK(launch_step_done(bv, ctx->st, pf));
    return RBSOG_OK;
}

rbsog_status enqueue_step(rbsog_ctx *ctx, bool energy = true) {
    rbsog_status s = enqueue_kick_drift(ctx);
    if (s != RBSOG_OK) return s;
    return enqueue_step_tail(ctx, false, energy);
}

// The scatter can run the next step's kick-drift when nothing happens to the
// velocities between this step's second half kick and the next step's first
// one: FP32C on neighbour lists (the scatter writes the total force in
// caller order), no boundary term after the scatter, no thermostat, no step
// budgets (a system could stop after this step).
bool drift_fusable(const rbsog_ctx *ctx) {
    if (ctx->precision != RBSOG_FP32C || !ctx->use_list || ctx->any_boundary || ctx->use_budget) return false;
    for (const auto &pp : ctx->p)
        if (pp.tau_T > 0.0) return false;
    return true;
}

void drop_graph(rbsog_ctx *c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph_e) cudaGraphExecDestroy(c->graph_e);
    if (c->graph_tail) cudaGraphExecDestroy(c->graph_tail);
    if (c->graph_fused) cudaGraphExecDestroy(c->graph_fused);
    c->graph = nullptr;
    c->graph_e = nullptr;
    c->graph_tail = nullptr;
    c->graph_fused = nullptr;
}

// whole: a step without energies; whole_e: a step with them; tail: a step
// without its kick-drift, with energies; tail_drift: a step without its
// kick-drift whose scatter runs the next one's, without energies.
enum class StepPart { whole, whole_e, tail, tail_drift };

// Captures a whole step, its tail, or its tail with the next step's
// kick-drift into *out (once).
rbsog_status capture_step(rbsog_ctx *ctx, StepPart part, cudaGraphExec_t *out) {
    if (*out) return RBSOG_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    rbsog_status es = part == StepPart::whole     ? enqueue_step(ctx, false)
                      : part == StepPart::whole_e ? enqueue_step(ctx, true)
                                                  : enqueue_step_tail(ctx, part == StepPart::tail_drift,
                                                                      part == StepPart::tail);
    ctx->capturing = false;
    cudaError_t ce = cudaStreamEndCapture(ctx->st, &g);
    if (es != RBSOG_OK) {
        if (g) cudaGraphDestroy(g);
        return es;
    }
    if (ce != cudaSuccess) return fail(ctx, RBSOG_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(ctx, RBSOG_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    return RBSOG_OK;
}

rbsog_status check_flags(rbsog_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->h_err, ctx->err_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const int32_t f = *ctx->h_err;
    if (f) {
        CK(cudaMemsetAsync(ctx->err_flag, 0, sizeof(int32_t), ctx->st));
        if (f & 1) return fail(ctx, RBSOG_ENUMERIC, "non-finite force produced on the device");
        if (f & 2) return fail(ctx, RBSOG_ETIMEOUT, "a sampler chain hit its iteration cap");
        if (f & 4)
            return fail(ctx, RBSOG_ENUMERIC, "a neighbour list exceeded its capacity (local density far above the "
                                             "system's mean)");
        return fail(ctx, RBSOG_ECUDA, "device error flag %d", f);
    }
    return RBSOG_OK;
}

rbsog_status upload_desc(rbsog_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->d_desc, ctx->desc.data(), sizeof(SysDesc) * ctx->n_sys, cudaMemcpyHostToDevice,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return RBSOG_OK;
}

// A caller buffer that kernels can read or write in place: device or
// managed memory.  Host memory (pinned or not) goes through the staging
// buffer with a bulk copy: measured faster than kernels reading pinned host
// memory over the host link.
template <class T>
T *kernel_view(T *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error of an unknown pointer
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
    return nullptr;
}

double self_energy(const rbsog_ctx *c, int s) {
    double wsum = 0.0;
    for (size_t l = 0; l < c->omega.size(); ++l) wsum += c->omega[l];
    return 0.5 * wsum * c->sum_q2[s] * c->p[s].coulomb_prefactor;
}

// Systems without valid forces get an initial force evaluation (and consume
// one k-set); the others keep theirs.
rbsog_status initial_forces(rbsog_ctx *ctx) {
    std::vector<int32_t> mask(ctx->n_sys, 0);
    bool any = false;
    for (int s = 0; s < ctx->n_sys; ++s)
        if (!ctx->force_valid[s]) {
            mask[s] = 1;
            any = true;
        }
    if (!any) return RBSOG_OK;
    CK(cudaMemcpyAsync(ctx->d_mask, mask.data(), sizeof(int32_t) * ctx->n_sys, cudaMemcpyHostToDevice, ctx->st));
    BatchView bv = view(ctx);
    bv.force_mask = ctx->d_mask;
    rbsog_status es = enqueue_forces(ctx, bv, nullptr);
    if (es != RBSOG_OK) return es;
    CK(launch_finalize(bv, ctx->epart, ctx->rho, ctx->kpart, 0, ctx->energy, 1, ctx->st, prof_of(ctx)));
    CK(cudaStreamSynchronize(ctx->st));   // the host mask buffer is reused
    for (int s = 0; s < ctx->n_sys; ++s)
        if (mask[s]) {
            ctx->host_cursor[s] += 1;
            ctx->force_valid[s] = 1;
        }
    return RBSOG_OK;
}

// Near-field and rho-sweep launch shapes from the per-system tunables:
// segment grouping, staging chunk, sweep tiles, partial-sum offsets, work
// tables and the buffers whose size depends on them.
rbsog_status apply_layout(rbsog_ctx *ctx) {
    drop_graph(ctx);
    ctx->nblk.clear();
    ctx->sblk.clear();
    ctx->max_cap = 256;
    ctx->max_tile_p = 128;
    int64_t e_off = 0, rp_off = 0;
    for (int s = 0; s < ctx->n_sys; ++s) {
        SysDesc &d = ctx->desc[s];
        int nblocks = 0, npart = 0;
        // with neighbour lists the cell-row blocks only build lists: about
        // 112 home particles fill the builder's 128 threads in one round
        const int home = ctx->use_list ? 112 : ctx->tune[s].home;
        near_layout(d.box, d.n, ctx->precision, home, d.group, d.nseg_x, d.near_cap, nblocks, npart);
        d.near_split = ctx->precision == RBSOG_FP64 && d.n < kNearSplitMaxN ? 1 : 0;
        d.e_off = (int32_t)e_off;
        d.n_epart = npart;
        if (ctx->use_list) {
            // energies come per particle block (the cell-stencil kernel, which
            // rbsog_get_cells still runs, writes one per near block: room for both)
            d.n_epart = d.n_kpart;
            npart = std::max(npart, d.n_kpart);
        }
        far_layout(d.n, ctx->P, ctx->precision, ctx->tune[s].tile, d.tile_p, d.n_ptiles);
        d.rp_off = rp_off;
        for (int b = 0; b < nblocks; ++b) ctx->nblk.push_back(make_int2(s, b));
        for (int b = 0; b < d.n_ptiles; ++b) ctx->sblk.push_back(make_int2(s, b));
        ctx->max_cap = std::max(ctx->max_cap, d.near_cap);
        ctx->max_tile_p = std::max(ctx->max_tile_p, d.tile_p);
        e_off += npart;
        rp_off += (int64_t)ctx->P * d.n_ptiles;
    }
    CK(cudaStreamSynchronize(ctx->st));
    CK(dalloc(&ctx->rho_part, (size_t)rp_off));
    CK(dalloc(&ctx->epart, (size_t)e_off));
    CK(dalloc(&ctx->d_nblk, ctx->nblk.size()));
    CK(dalloc(&ctx->d_sblk, ctx->sblk.size()));
    CK(cudaMemcpyAsync(ctx->d_nblk, ctx->nblk.data(), sizeof(int2) * ctx->nblk.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->d_sblk, ctx->sblk.data(), sizeof(int2) * ctx->sblk.size(), cudaMemcpyHostToDevice, ctx->st));
    return upload_desc(ctx);
}

bool all_state(const rbsog_ctx *ctx) {
    for (char c : ctx->have_state)
        if (!c) return false;
    return true;
}

rbsog_status check_sys(rbsog_ctx *ctx, int32_t sys) {
    if (sys < 0 || sys >= ctx->n_sys) return fail(ctx, RBSOG_EINVAL, "system %d outside [0, %d)", sys, ctx->n_sys);
    return RBSOG_OK;
}

}  // namespace

extern "C" {

rbsog_status rbsog_batch_create(rbsog_batch **out, int32_t n_sys, const int64_t *n_per, int device, void *stream) {
    if (!out || !n_per || n_sys < 1) return RBSOG_EINVAL;
    *out = nullptr;
    int64_t total = 0;
    for (int s = 0; s < n_sys; ++s) {
        if (n_per[s] < 2) return RBSOG_EINVAL;
        total += n_per[s];
    }
    if (total > (int64_t)INT32_MAX / 2) return RBSOG_EINVAL;
    rbsog_ctx *ctx = new (std::nothrow) rbsog_ctx();
    if (!ctx) return RBSOG_ENOMEM;
    ctx->n_sys = n_sys;
    ctx->n_per.assign(n_per, n_per + n_sys);
    ctx->p_off.resize(n_sys);
    for (int s = 0; s < n_sys; ++s) {
        ctx->p_off[s] = ctx->n_total;
        ctx->n_total += n_per[s];
    }
    ctx->have_state.assign(n_sys, 0);
    ctx->force_valid.assign(n_sys, 0);
    ctx->sum_q2.assign(n_sys, 0.0);
    ctx->host_cursor.assign(n_sys, 0);
    ctx->device = device;
    ctx->user = (cudaStream_t)stream;
    ctx->prof_hook.mark = prof_mark;
    ctx->prof_hook.self = ctx;
    auto bail = [&](rbsog_status s) {
        rbsog_destroy(ctx);
        return s;
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(RBSOG_ECUDA);
    if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) != cudaSuccess) return bail(RBSOG_ECUDA);
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess) return bail(RBSOG_ECUDA);
    if (cudaStreamCreateWithFlags(&ctx->far, cudaStreamNonBlocking) != cudaSuccess) return bail(RBSOG_ECUDA);
    if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(RBSOG_ECUDA);
    if (cudaStreamCreateWithFlags(&ctx->io, cudaStreamNonBlocking) != cudaSuccess) return bail(RBSOG_ECUDA);
    if (cudaEventCreateWithFlags(&ctx->ev_q, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_x, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_io, cudaEventDisableTiming) != cudaSuccess)
        return bail(RBSOG_ECUDA);
    if (cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return bail(RBSOG_ECUDA);
    const int64_t n = ctx->n_total;
    bool ok = dalloc(&ctx->posq, n) == cudaSuccess && dalloc(&ctx->vel, n) == cudaSuccess &&
              dalloc(&ctx->force, n) == cudaSuccess && dalloc(&ctx->fnear, n) == cudaSuccess &&
              dalloc(&ctx->sp64, n) == cudaSuccess && dalloc(&ctx->sp32, n) == cudaSuccess &&
              dalloc(&ctx->staging, 10 * n) == cudaSuccess &&
              dalloc(&ctx->qpart, 3 * ((n + 255) / 256)) == cudaSuccess && dalloc(&ctx->nbr_sorted, n) == cudaSuccess &&
              dalloc(&ctx->i32_tmp, n) == cudaSuccess && dalloc(&ctx->cb.cell_of, n) == cudaSuccess &&
              dalloc(&ctx->cb.slot, n) == cudaSuccess && dalloc(&ctx->cb.perm_raw, n) == cudaSuccess &&
              dalloc(&ctx->cb.perm, n) == cudaSuccess && dalloc(&ctx->cb.key, n) == cudaSuccess &&
              dalloc(&ctx->cb.pack, n) == cudaSuccess && dalloc(&ctx->cursor, n_sys) == cudaSuccess &&
              dalloc(&ctx->step_ctr, n_sys) == cudaSuccess &&
              dalloc(&ctx->energy, (size_t)kNumEnergy * n_sys) == cudaSuccess &&
              dalloc(&ctx->err_flag, 1) == cudaSuccess && dalloc(&ctx->d_desc, n_sys) == cudaSuccess &&
              dalloc(&ctx->d_mask, n_sys) == cudaSuccess &&
              dalloc(&ctx->fin_part, (size_t)n_sys * kFinChunks) == cudaSuccess &&
              dalloc(&ctx->dip, n_sys) == cudaSuccess &&
              dalloc(&ctx->fin_count, n_sys) == cudaSuccess &&
              cudaMemset(ctx->fin_count, 0, sizeof(unsigned int) * n_sys) == cudaSuccess;
    if (!ok) return bail(RBSOG_ENOMEM);
    if (cudaMallocHost((void **)&ctx->h_energy, sizeof(double) * kNumEnergy) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_err, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_i64, 4 * sizeof(int64_t)) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_qpart, sizeof(double) * 3 * ((n + 255) / 256)) != cudaSuccess)
        return bail(RBSOG_ENOMEM);
    cudaMemsetAsync(ctx->vel, 0, sizeof(double4_32a) * n, ctx->st);
    cudaMemsetAsync(ctx->force, 0, sizeof(double4_32a) * n, ctx->st);
    cudaMemsetAsync(ctx->posq, 0, sizeof(double4_32a) * n, ctx->st);
    cudaMemsetAsync(ctx->energy, 0, sizeof(double) * kNumEnergy * n_sys, ctx->st);
    cudaMemsetAsync(ctx->err_flag, 0, sizeof(int32_t), ctx->st);
    cudaMemsetAsync(ctx->cursor, 0, sizeof(int64_t) * n_sys, ctx->st);
    cudaMemsetAsync(ctx->step_ctr, 0, sizeof(int64_t) * n_sys, ctx->st);
    if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return bail(RBSOG_ECUDA);
    *out = ctx;
    return RBSOG_OK;
}

rbsog_status rbsog_create(rbsog_ctx **out, int64_t n, int device, void *stream) {
    if (n < 2 || n > (int64_t)INT32_MAX / 2) {
        if (out) *out = nullptr;
        return RBSOG_EINVAL;
    }
    return rbsog_batch_create(out, 1, &n, device, stream);
}

}  // extern "C"

namespace {
// sample_mask (may be null): systems whose k-sequence is sampled here; the
// others receive theirs by copy (serving engine rebuilds).
rbsog_status set_params_impl(rbsog_ctx *ctx, const rbsog_params *pp, const std::vector<char> *sample_mask) {
    if (!ctx || !pp) return RBSOG_EINVAL;
    const int ns = ctx->n_sys;
    std::vector<rbsog_params> p(pp, pp + ns);
    std::vector<BoxDev> box(ns);
    // FP32C uses neighbour lists with a skin of r_c / 10 when every box holds
    // at least 3 cells of side r_c + skin per side (else the cell stencil)
    const double skin = 0.1 * p[0].r_c;
    bool lists = p[0].precision == RBSOG_FP32C && p[0].r_c > 0.0;
    for (int s = 0; s < ns && lists; ++s)
        for (int d = 0; d < 3; ++d)
            if (!(p[s].L[d] > 0.0) || std::floor(p[s].L[d] / (p[s].r_c + skin)) < 3.0) lists = false;
    // slots per particle: 1.5 x the mean count within r_c + skin at the
    // densest system of the batch, plus 48; the builder keeps them per
    // thread in shared memory, which bounds them (denser: cell stencil)
    int32_t list_cap = 0;
    if (lists) {
        double rho_max = 0.0;
        for (int s = 0; s < ns; ++s)
            rho_max = std::max(rho_max, (double)ctx->n_per[s] / (p[s].L[0] * p[s].L[1] * p[s].L[2]));
        const double rl = p[0].r_c + skin;
        const double mean = 4.0 / 3.0 * kPi * rl * rl * rl * rho_max;
        list_cap = (((int)(1.5 * mean) + 48) + 7) / 8 * 8;
        if (list_cap > 280) lists = false;
    }
    // the list path takes G and F from its combined table only: it needs
    // that table at FP32 rounding level (else the cell stencil, which falls
    // back to exp + Taylor sums when its own tables are not accurate enough)
    if (lists) {
        double sg = p[0].sigma, ww0 = p[0].omega0;
        bool ok = p[0].b > 1.0 && p[0].M >= 0 && p[0].M < kMaxGauss && p[0].r_c > 0.0;
        if (ok && !(sg > 0.0)) ok = solve_sigma(p[0].b, p[0].r_c, sg, ww0);
        else if (ok && !(ww0 > 0.0)) ww0 = c0_weight(p[0].b, sg, p[0].r_c);
        if (ok && ww0 > 0.0 && std::isfinite(ww0)) {
            std::vector<double> w, sv;
            bsa_coeffs(p[0].b, sg, p[0].M, w, sv);
            w[0] = ww0;
            NearSog tmp{};
            std::vector<float4> t;
            ok = build_list_table(tmp, t, w, sv, p[0].M, p[0].r_c) < kListTabTol;
        } else {
            ok = false;
        }
        if (!ok) lists = false;
    }
    for (int s = 0; s < ns; ++s) {
        const rbsog_params &q = p[s];
        if (!(q.b > 1.0)) return fail(ctx, RBSOG_EINVAL, "system %d: b must be > 1", s);
        if (q.M < 0 || q.M >= kMaxGauss) return fail(ctx, RBSOG_EINVAL, "system %d: M must be in [0, %d]", s, kMaxGauss - 1);
        if (q.P < 1) return fail(ctx, RBSOG_EINVAL, "system %d: P must be >= 1", s);
        if (q.n_ksets < 1) return fail(ctx, RBSOG_EINVAL, "system %d: n_ksets must be >= 1", s);
        if (!(q.r_c > 0.0)) return fail(ctx, RBSOG_EINVAL, "system %d: r_c must be > 0", s);
        if (!(q.mass > 0.0)) return fail(ctx, RBSOG_EINVAL, "system %d: mass must be > 0", s);
        if (q.thermostat < 0 || q.thermostat > 2)
            return fail(ctx, RBSOG_EINVAL,
                        "system %d: thermostat must be 0 (Berendsen), 1 (Langevin) or 2 (Nose-Hoover)", s);
        if (q.sampler < 0 || q.sampler > 1)
            return fail(ctx, RBSOG_EINVAL, "system %d: sampler must be 0 (mixture) or 1 (per-Gaussian)", s);
        if (s > 0 && q.sampler != p[0].sampler)
            return fail(ctx, RBSOG_EINVAL, "system %d: sampler must be the same for every system", s);
        if (q.near_kernel < 0 || q.near_kernel > 1)
            return fail(ctx, RBSOG_EINVAL, "system %d: near_kernel must be 0 (table) or 1 (core-shell)", s);
        if (s > 0 && (q.near_kernel != p[0].near_kernel || q.r_in != p[0].r_in))
            return fail(ctx, RBSOG_EINVAL, "system %d: near_kernel and r_in must be the same for every system", s);
        if (q.boundary < 0 || q.boundary > 2)
            return fail(ctx, RBSOG_EINVAL, "system %d: boundary must be 0 (tinfoil), 1 (spherical) or 2 (planar)", s);
        if (q.precision != RBSOG_FP64 && q.precision != RBSOG_FP32C)
            return fail(ctx, RBSOG_EINVAL, "system %d: unknown precision %d", s, q.precision);
        if (q.chain_len < 0) return fail(ctx, RBSOG_EINVAL, "system %d: chain_len must be >= 0", s);
        if (q.wca_sigma < 0.0) return fail(ctx, RBSOG_EINVAL, "system %d: wca_sigma must be >= 0", s);
        if (s > 0 && (q.b != p[0].b || q.sigma != p[0].sigma || q.omega0 != p[0].omega0 || q.M != p[0].M ||
                      q.r_c != p[0].r_c || q.P != p[0].P || q.precision != p[0].precision))
            return fail(ctx, RBSOG_EINVAL, "system %d: b, sigma, omega0, M, r_c, P and precision must be the same "
                                           "for every system of a batch", s);
        BoxDev &b = box[s];
        std::memset(&b, 0, sizeof b);
        int64_t ncell = 1;
        for (int d = 0; d < 3; ++d) {
            if (!(q.L[d] > 0.0)) return fail(ctx, RBSOG_EINVAL, "system %d: box edges must be > 0", s);
            if (!(q.r_c < 0.5 * q.L[d])) return fail(ctx, RBSOG_EINVAL, "system %d: r_c must be < L/2", s);
            if (std::floor(q.L[d] / q.r_c) < 3.0)
                return fail(ctx, RBSOG_EINVAL, "system %d: need at least 3 cells per side (L/r_c >= 3)", s);
            b.nc[d] = (int)std::floor(q.L[d] / (lists ? q.r_c + skin : q.r_c));
            ncell *= b.nc[d];
            b.L[d] = q.L[d];
            b.h[d] = q.L[d] / (double)b.nc[d];
            b.L_f[d] = (float)q.L[d];
            b.fix_scale[d] = (float)(q.L[d] / 4294967296.0);
            b.fix_inv[d] = 4294967296.0 / q.L[d];
            b.cell_fix[d] = (float)(4294967296.0 / (double)b.nc[d]);
            b.inv_h[d] = (double)b.nc[d] / q.L[d];
            b.kfac[d] = 2.0 * kPi / q.L[d];
            b.h_f[d] = (float)b.h[d];
        }
        if (ncell > (int64_t)INT32_MAX / 4) return fail(ctx, RBSOG_EINVAL, "system %d: cell grid too large", s);
        b.ncell = (int32_t)ncell;
        b.rc2 = q.r_c * q.r_c;
        b.lB = q.coulomb_prefactor;
        b.wca_s2 = q.wca_sigma * q.wca_sigma;
        b.wca_rc2 = q.wca_sigma > 0.0 ? std::pow(2.0, 1.0 / 3.0) * b.wca_s2 : 0.0;
        b.wca_eps = q.wca_eps;
        b.rc2_f = (float)b.rc2;
        b.lB_f = (float)b.lB;
        b.wca_s2_f = (float)b.wca_s2;
        b.wca_rc2_f = (float)b.wca_rc2;
        b.wca_eps_f = (float)b.wca_eps;
        const double rl = q.r_c + skin;
        b.rl2_f = (float)(rl * rl * (1.0 + 1e-5));
        b.disp2_f = (float)(0.25 * skin * skin * (1.0 - 1e-4));
    }

    // --- SOG (Eqs. 2.9-2.11), shared by the batch
    double sigma = p[0].sigma, w0 = p[0].omega0;
    if (!(sigma > 0.0)) {
        if (!solve_sigma(p[0].b, p[0].r_c, sigma, w0))
            return fail(ctx, RBSOG_EINVAL, "no C0/C1 root for b=%g r_c=%g", p[0].b, p[0].r_c);
    } else if (!(w0 > 0.0)) {
        w0 = c0_weight(p[0].b, sigma, p[0].r_c);
    }
    if (!(w0 > 0.0) || !std::isfinite(w0)) return fail(ctx, RBSOG_EINVAL, "invalid omega0");
    std::vector<double> w, sv;
    bsa_coeffs(p[0].b, sigma, p[0].M, w, sv);
    w[0] = w0;
    std::vector<float4> cstab;
    CoreShellDev cs_new{};
    if (p[0].near_kernel == 1) {
        if (!lists) return fail(ctx, RBSOG_EINVAL, "the core-shell kernel runs on the FP32C neighbour-list path only");
        const double rin = p[0].r_in > 0.0 ? p[0].r_in : p[0].r_c / 3.0;
        if (!(rin < p[0].r_c)) return fail(ctx, RBSOG_EINVAL, "r_in must be below r_c");
        if (!build_coreshell(cs_new, cstab, w, sv, p[0].M, p[0].r_c, rin))
            return fail(ctx, RBSOG_EINVAL, "the core-shell table cannot reach r_c^2 from r_in^2 in 8 octaves");
    }

    // per-Gaussian sampling: plans per system (box-dependent); every set of the
    // batch holds the largest P_eff frequencies, shorter ones padded
    std::vector<PgPlan> plans;
    int32_t P_batch = p[0].P;
    if (p[0].sampler == 1) {
        plans.resize(ns);
        P_batch = 0;
        for (int s = 0; s < ns; ++s) {
            if (!pg_plan(w.data(), sv.data(), p[0].M, p[s].L, p[0].P, plans[s]))
                return fail(ctx, RBSOG_EINVAL, "system %d: per-Gaussian sampling table longer than 2^20", s);
            P_batch = std::max(P_batch, plans[s].P_eff);
        }
    }

    drop_graph(ctx);
    ctx->p = p;
    ctx->any_boundary = false;
    for (auto &pp : p) ctx->any_boundary = ctx->any_boundary || pp.boundary != 0;
    ctx->omega = w;
    ctx->s = sv;
    ctx->sigma = sigma;
    ctx->omega0 = w0;
    ctx->P = P_batch;
    ctx->pg_sampler = p[0].sampler == 1;
    ctx->precision = p[0].precision;
    build_near_sog(ctx->nsog, w, sv, p[0].M, p[0].r_c);
    build_sog_tables(ctx->nsog, w, sv, p[0].M, p[0].r_c);
    build_list_table(ctx->nsog, ctx->h_ltab, w, sv, p[0].M, p[0].r_c);
    ctx->cs = cs_new;
    ctx->use_cs = p[0].near_kernel == 1;

    // --- per-system layout
    ctx->desc.assign(ns, SysDesc{});
    ctx->S.assign(ns, 0.0);
    ctx->n_chains.assign(ns, 0);
    ctx->chain_len.assign(ns, 256);
    ctx->pblk.clear();
    ctx->nblk.clear();
    ctx->sblk.clear();
    std::vector<int32_t> cell_sys;
    int64_t c_off = 0, k_off = 0, kp_off = 0, kc_off = 0;
    ctx->tune.assign(ns, Tune{});
    for (int s = 0; s < ns; ++s) {
        const rbsog_params &q = p[s];
        SysDesc &d = ctx->desc[s];
        d.box = box[s];
        d.p_off = ctx->p_off[s];
        d.n = ctx->n_per[s];
        d.c_off = c_off;
        d.k_off = k_off;
        d.n_sets = q.n_ksets;
        d.kc_off = kc_off;
        kc_off += q.n_ksets;
        d.n_kpart = (int32_t)((d.n + kParticleBlock - 1) / kParticleBlock);
        d.kp_off = (int32_t)kp_off;
        double Ssum = 0.0;
        for (int l = q.M; l >= 0; --l) {
            const double prod = theta_sum(sv[l], q.L[0]) * theta_sum(sv[l], q.L[1]) * theta_sum(sv[l], q.L[2]);
            Ssum += w[l] * sv[l] * sv[l] * sv[l] * (prod - 1.0);
        }
        ctx->S[s] = Ssum;
        ctx->tune[s] = tune_for(d.n, ctx->P, ctx->precision);
        const double V = q.L[0] * q.L[1] * q.L[2];
        d.coef = -q.coulomb_prefactor * std::pow(kPi, 1.5) * Ssum / ((double)ctx->P * V);
        d.half_coef_U = q.coulomb_prefactor * std::pow(kPi, 1.5) * Ssum / (2.0 * ctx->P * V);
        d.dt = q.dt;
        d.mass = q.mass;
        d.inv_mass = 1.0 / q.mass;
        d.half_dt_inv_mass = 0.5 * q.dt * d.inv_mass;
        d.boundary = q.boundary;
        d.thermostat = q.tau_T > 0.0 ? q.thermostat : 0;
        d.half_dt = 0.5 * q.dt;
        d.lv_c1 = d.thermostat == 1 ? std::exp(-q.dt / q.tau_T) : 1.0;
        d.lv_c2 = d.thermostat == 1 ? std::sqrt((1.0 - d.lv_c1 * d.lv_c1) * q.T_target / q.mass) : 0.0;
        d.lv_seed = q.seed;
        d.half_mass_f = (float)(0.5 * q.mass);
        d.nh_Q = d.thermostat == 2 ? (3.0 * (double)d.n - 3.0) * q.T_target * q.tau_T * q.tau_T : 0.0;
        d.T0 = q.T_target;
        d.tau = q.tau_T;
        // per-Gaussian sampling writes one set per "chain"
        ctx->chain_len[s] = ctx->pg_sampler ? ctx->P : (q.chain_len > 0 ? q.chain_len : 256);
        const int64_t total = q.n_ksets * (int64_t)ctx->P;
        ctx->n_chains[s] = (total + ctx->chain_len[s] - 1) / ctx->chain_len[s];
        for (int64_t b = 0; b < d.n_kpart; ++b) ctx->pblk.push_back(make_int2(s, (int)b));
        cell_sys.insert(cell_sys.end(), (size_t)d.box.ncell, s);
        c_off += d.box.ncell;
        k_off += ctx->n_chains[s] * ctx->chain_len[s];
        kp_off += d.n_kpart;
    }
    for (int s = 0; s < ns; ++s) ctx->desc[s].U_self = self_energy(ctx, s);
    ctx->ncell_total = c_off;
    if (c_off > (int64_t)INT32_MAX / 2) return fail(ctx, RBSOG_EINVAL, "cell grids of the batch too large");

    CK(cudaSetDevice(ctx->device));
    CK(dalloc(&ctx->kseq, (size_t)k_off));
    if (!ctx->pg_sampler) {
        CK(dalloc(&ctx->kfold, (size_t)k_off));
        CK(dalloc(&ctx->kcount, (size_t)kc_off));
    } else {   // per-Gaussian draws are independent: no runs to fold
        dfree(&ctx->kfold);
        dfree(&ctx->kcount);
    }
    CK(dalloc(&ctx->rho, (size_t)ns * ctx->P));
    CK(dalloc((unsigned char **)&ctx->ktab, ktab_bytes(ctx->precision, (int64_t)ns * ctx->P)));
    CK(dalloc(&ctx->kpart, (size_t)kp_off));
    CK(dalloc(&ctx->dpart, (size_t)kp_off));
    CK(dalloc(&ctx->cb.count, (size_t)c_off));
    CK(dalloc(&ctx->cb.start, (size_t)c_off + 1));
    CK(dalloc(&ctx->cb.tile_sum, (size_t)cell_scan_tiles(c_off)));
    CK(dalloc(&ctx->m_tmp, (size_t)ctx->P));
    if (ctx->pg_sampler) {
        std::vector<double> kw((size_t)ns * kKwStride, 0.0);
        for (int s = 0; s < ns; ++s)
            for (const PgStratum &st : plans[s].strata)
                kw[(size_t)s * kKwStride + st.l] =
                    (plans[s].S_l[st.l] / plans[s].P_l[st.l]) / (ctx->S[s] / (double)ctx->P);
        CK(dalloc(&ctx->d_kw, kw.size()));
        CK(cudaMemcpy(ctx->d_kw, kw.data(), sizeof(double) * kw.size(), cudaMemcpyHostToDevice));
    } else {
        dfree(&ctx->d_kw);
    }
    CK(dalloc(&ctx->m3_tmp, (size_t)ctx->P * 3));
    CK(dalloc(&ctx->d_pblk, ctx->pblk.size()));
    CK(dalloc(&ctx->d_cell_sys, cell_sys.size()));
    ctx->use_list = lists;
    ctx->skin = lists ? skin : 0.0;
    ctx->list_cap = lists ? list_cap : 0;
    if (lists) {
        const size_t n = (size_t)ctx->n_total;
        CK(dalloc(&ctx->sp32c, n));
        CK(dalloc(&ctx->xref, n));
        CK(dalloc(&ctx->nbr_cnt, n));
        CK(dalloc(&ctx->list_perm, n));
        CK(dalloc(&ctx->lpos, n));
        CK(dalloc(&ctx->linv, n));
        CK(dalloc(&ctx->d_ltab, (size_t)kLTabN));
        CK(cudaMemcpy(ctx->d_ltab, ctx->h_ltab.data(), sizeof(float4) * kLTabN, cudaMemcpyHostToDevice));
        if (ctx->use_cs) {
            CK(dalloc(&ctx->d_cstab, cstab.size()));
            CK(cudaMemcpy(ctx->d_cstab, cstab.data(), sizeof(float4) * cstab.size(), cudaMemcpyHostToDevice));
        }
        CK(dalloc(&ctx->nbr_list, (n + 31) / 32 * 32 * (size_t)ctx->list_cap));
        // flags of the ns systems, the 'any system' flag, and a count of the
        // list builds run since set_params (read by rbsog_get_info)
        CK(dalloc(&ctx->d_rebuild, (size_t)ns + 2));
        CK(cudaMemset(ctx->xref, 0, sizeof(uint4) * n));
        CK(cudaMemset(ctx->nbr_cnt, 0, sizeof(int32_t) * n));
        CK(cudaMemset(ctx->list_perm, 0, sizeof(int32_t) * n));
        // every position write before the first build goes through linv:
        // start from the identity so that it stays inside the array
        std::vector<int32_t> ident(n);
        for (size_t q = 0; q < n; ++q) ident[q] = (int32_t)q;
        CK(cudaMemcpy(ctx->linv, ident.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
        std::vector<int32_t> ones((size_t)ns + 2, 1);
        ones[(size_t)ns + 1] = 0;
        CK(cudaMemcpy(ctx->d_rebuild, ones.data(), sizeof(int32_t) * (ns + 2), cudaMemcpyHostToDevice));
    }
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    es = apply_layout(ctx);
    if (es != RBSOG_OK) return es;
    CK(cudaMemcpyAsync(ctx->d_pblk, ctx->pblk.data(), sizeof(int2) * ctx->pblk.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->d_cell_sys, cell_sys.data(), sizeof(int32_t) * cell_sys.size(), cudaMemcpyHostToDevice,
                       ctx->st));
    CK(cudaMemsetAsync(ctx->cb.count, 0, sizeof(int32_t) * c_off, ctx->st));
    CK(cudaMemsetAsync(ctx->cursor, 0, sizeof(int64_t) * ns, ctx->st));
    CK(cudaMemsetAsync(ctx->step_ctr, 0, sizeof(int64_t) * ns, ctx->st));
    CK(cudaMemsetAsync(ctx->err_flag, 0, sizeof(int32_t), ctx->st));
    es = upload_desc(ctx);
    if (es != RBSOG_OK) return es;
    std::fill(ctx->host_cursor.begin(), ctx->host_cursor.end(), 0);
    std::fill(ctx->force_valid.begin(), ctx->force_valid.end(), 0);

    {
        SamplerDev sp{};
        sp.M = p[0].M;
        for (int l = 0; l <= p[0].M; ++l) {
            sp.omega[l] = w[l];
            sp.s[l] = sv[l];
        }
        std::vector<SamplerSys> ss;
        int64_t coff = 0;
        for (int s = 0; s < ns; ++s) {
            if (sample_mask && !(*sample_mask)[s]) continue;
            SamplerSys y{};
            for (int d = 0; d < 3; ++d) y.L[d] = p[s].L[d];
            y.seed = p[s].seed;
            y.chain_off = coff;
            y.k_off = ctx->desc[s].k_off;
            y.chain_len = ctx->chain_len[s];
            coff += ctx->n_chains[s];
            ss.push_back(y);
        }
        if (ctx->pg_sampler) {
            for (int s = 0; s < ns; ++s) {
                if (sample_mask && !(*sample_mask)[s]) continue;
                const PgPlan &pl = plans[s];
                PgStratum *d_st = nullptr;
                int32_t *d_slot = nullptr;
                double *d_tab = nullptr;
                CK(cudaMallocAsync((void **)&d_st, sizeof(PgStratum) * std::max<size_t>(pl.strata.size(), 1), ctx->st));
                CK(cudaMallocAsync((void **)&d_slot, sizeof(int32_t) * std::max<size_t>(pl.slot_stratum.size(), 1),
                                   ctx->st));
                CK(cudaMallocAsync((void **)&d_tab, sizeof(double) * std::max<size_t>(pl.tables.size(), 1), ctx->st));
                CK(cudaMemcpyAsync(d_st, pl.strata.data(), sizeof(PgStratum) * pl.strata.size(), cudaMemcpyHostToDevice,
                                   ctx->st));
                CK(cudaMemcpyAsync(d_slot, pl.slot_stratum.data(), sizeof(int32_t) * pl.slot_stratum.size(),
                                   cudaMemcpyHostToDevice, ctx->st));
                CK(cudaMemcpyAsync(d_tab, pl.tables.data(), sizeof(double) * pl.tables.size(), cudaMemcpyHostToDevice,
                                   ctx->st));
                CK(launch_pg_sampler(d_st, d_slot, pl.P_eff, ctx->P, d_tab, p[s].seed, p[s].n_ksets,
                                     ctx->kseq + ctx->desc[s].k_off, ctx->st, prof_of(ctx)));
                // the host vectors stay alive until the copies have run
                CK(cudaStreamSynchronize(ctx->st));
                for (void *ptr : {(void *)d_st, (void *)d_slot, (void *)d_tab}) CK(cudaFreeAsync(ptr, ctx->st));
            }
        } else if (!ss.empty()) {
            SamplerSys *d_ss = nullptr;
            CK(cudaMallocAsync((void **)&d_ss, sizeof(SamplerSys) * ss.size(), ctx->st));
            CK(cudaMemcpyAsync(d_ss, ss.data(), sizeof(SamplerSys) * ss.size(), cudaMemcpyHostToDevice, ctx->st));
            CK(launch_mh_sampler(sp, d_ss, (int)ss.size(), coff, ctx->kseq, ctx->err_flag, ctx->st, prof_of(ctx)));
            CK(cudaFreeAsync(d_ss, ctx->st));
            // fold each sampled set's runs of repeated frequencies
            std::vector<FoldSys> fs;
            int64_t set_off = 0;
            for (int s = 0; s < ns; ++s) {
                if (sample_mask && !(*sample_mask)[s]) continue;
                fs.push_back(FoldSys{ctx->desc[s].k_off, ctx->desc[s].kc_off, set_off});
                set_off += ctx->desc[s].n_sets;
            }
            FoldSys *d_fs = nullptr;
            CK(cudaMallocAsync((void **)&d_fs, sizeof(FoldSys) * fs.size(), ctx->st));
            CK(cudaMemcpyAsync(d_fs, fs.data(), sizeof(FoldSys) * fs.size(), cudaMemcpyHostToDevice, ctx->st));
            CK(launch_fold_kseq(d_fs, (int)fs.size(), set_off, ctx->P, ctx->kseq, ctx->kfold, ctx->kcount, ctx->st));
            // the host vector stays alive until the copy has run
            CK(cudaStreamSynchronize(ctx->st));
            CK(cudaFreeAsync(d_fs, ctx->st));
        }
    }
    rbsog_status fs = check_flags(ctx);
    if (fs != RBSOG_OK) return fs;
    ctx->have_params = true;
    return leave(ctx);
}
}  // namespace

extern "C" {

rbsog_status rbsog_batch_set_params(rbsog_batch *ctx, const rbsog_params *pp) {
    return set_params_impl(ctx, pp, nullptr);
}

rbsog_status rbsog_set_params(rbsog_ctx *ctx, const rbsog_params *p) { return rbsog_batch_set_params(ctx, p); }

rbsog_status rbsog_batch_autotune(rbsog_batch *ctx, int32_t reps, int32_t *chosen) {
    if (!ctx || reps < 1) return RBSOG_EINVAL;
    if (!ctx->have_params || !all_state(ctx)) return fail(ctx, RBSOG_ESTATE, "params and state required");
    const bool prof = ctx->profiling;
    ctx->profiling = false;
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    double4_32a *scratch = nullptr;
    CK(cudaMallocAsync((void **)&scratch, sizeof(double4_32a) * ctx->n_total, ctx->st));
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    // time `reps` force evaluations of the whole batch into scratch forces
    // (the simulation state, cursors and energies are not touched)
    auto measure = [&](const Tune &t, float &best) -> rbsog_status {
        for (auto &x : ctx->tune) x = t;
        rbsog_status s2 = apply_layout(ctx);
        if (s2 != RBSOG_OK) return s2;
        const BatchView bv = view(ctx);
        s2 = enqueue_forces(ctx, bv, nullptr, scratch);   // warm-up
        if (s2 != RBSOG_OK) return s2;
        best = 1e30f;
        for (int r = 0; r < reps; ++r) {
            CK(cudaEventRecord(a, ctx->st));
            s2 = enqueue_forces(ctx, bv, nullptr, scratch);
            if (s2 != RBSOG_OK) return s2;
            CK(cudaEventRecord(b, ctx->st));
            CK(cudaEventSynchronize(b));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a, b));
            best = std::min(best, ms);
        }
        return RBSOG_OK;
    };
    const int homes[] = {64, 16, 32, 96, 120, 160, 224};
    const int tiles[] = {0, 256, 512, 1024, 2048};
    Tune best_t;
    float best_ms = 1e30f;
    for (int h : homes) {
        if (ctx->use_list && h != homes[0]) break;   // the block size only shapes the list builder
        Tune t;
        t.home = h;
        float ms = 0.f;
        es = measure(t, ms);
        if (es != RBSOG_OK) return es;
        if (ms < best_ms) {
            best_ms = ms;
            best_t = t;
        }
    }
    for (int tl : tiles) {
        if (tl == 0) continue;   // the default rule was measured with the homes
        Tune t = best_t;
        t.tile = tl;
        float ms = 0.f;
        es = measure(t, ms);
        if (es != RBSOG_OK) return es;
        if (ms < best_ms) {
            best_ms = ms;
            best_t = t;
        }
    }
    for (auto &x : ctx->tune) x = best_t;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (int s = 0; s < ctx->n_sys; ++s) g_tune[tune_key(ctx->desc[s].n, ctx->P, ctx->precision)] = best_t;
    }
    es = apply_layout(ctx);
    if (es != RBSOG_OK) return es;
    CK(cudaFreeAsync(scratch, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->profiling = prof;
    if (chosen) {
        chosen[0] = best_t.home;
        chosen[1] = best_t.tile;
    }
    return leave(ctx);
}

rbsog_status rbsog_get_info(const rbsog_ctx *ctx, rbsog_info *info, double *omega, double *s) {
    if (!ctx || !info) return RBSOG_EINVAL;
    if (!ctx->have_params) return RBSOG_ESTATE;
    info->sigma = ctx->sigma;
    info->omega0 = ctx->omega0;
    info->S = ctx->S[0];
    info->M = ctx->p[0].M;
    for (int d = 0; d < 3; ++d) info->ncell[d] = ctx->desc[0].box.nc[d];
    info->n_chains = ctx->n_chains[0];
    info->chain_len = ctx->chain_len[0];
    info->P_set = ctx->P;
    info->list_builds = 0;
    if (ctx->use_list && ctx->d_rebuild) {
        int32_t nb = 0;
        if (cudaSetDevice(ctx->device) != cudaSuccess ||
            cudaMemcpyAsync(&nb, ctx->d_rebuild + ctx->n_sys + 1, sizeof(int32_t), cudaMemcpyDeviceToHost,
                            ctx->st) != cudaSuccess ||
            cudaStreamSynchronize(ctx->st) != cudaSuccess)
            return RBSOG_ECUDA;
        info->list_builds = nb;
    }
    if (omega) std::memcpy(omega, ctx->omega.data(), sizeof(double) * (ctx->p[0].M + 1));
    if (s) std::memcpy(s, ctx->s.data(), sizeof(double) * (ctx->p[0].M + 1));
    return RBSOG_OK;
}

rbsog_status rbsog_batch_set_state(rbsog_batch *ctx, int32_t sys, const double *q, const double *x,
                                   const double *v) {
    if (!ctx || !q || !x) return RBSOG_EINVAL;
    if (!ctx->have_params) return fail(ctx, RBSOG_ESTATE, "set_params must come first");
    rbsog_status es = check_sys(ctx, sys);
    if (es != RBSOG_OK) return es;
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int64_t n = ctx->n_per[sys], off = ctx->p_off[sys];
    // inputs (host or device) land in the staging regions; the charge sums
    // for the neutrality check and the self energy are block sums on the
    // device, added on the host in block order
    // (read in place when the caller's memory is device-accessible)
    const double *sx = kernel_view(x), *sv = v ? kernel_view(v) : nullptr, *sq = kernel_view(q);
    if (!sq) {
        CK(cudaMemcpyAsync(ctx->staging + 9 * n, q, sizeof(double) * n, cudaMemcpyDefault, ctx->st));
        sq = ctx->staging + 9 * n;
    }
    if (!sx) {
        CK(cudaMemcpyAsync(ctx->staging, x, sizeof(double) * 3 * n, cudaMemcpyDefault, ctx->st));
        sx = ctx->staging;
    }
    if (v && !sv) {
        CK(cudaMemcpyAsync(ctx->staging + 3 * n, v, sizeof(double) * 3 * n, cudaMemcpyDefault, ctx->st));
        sv = ctx->staging + 3 * n;
    }
    const int64_t nb = (n + 255) / 256;
    CK(launch_charge_sums(n, sq, ctx->qpart, ctx->st));
    CK(cudaMemcpyAsync(ctx->h_qpart, ctx->qpart, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    double qs = 0.0, qa = 0.0, q2 = 0.0;
    for (int64_t b = 0; b < nb; ++b) {
        qs += ctx->h_qpart[3 * b];
        qa += ctx->h_qpart[3 * b + 1];
        q2 += ctx->h_qpart[3 * b + 2];
    }
    if (!std::isfinite(qa)) return fail(ctx, RBSOG_EINVAL, "non-finite charge");
    if (std::fabs(qs) > 1e-12 * qa) return fail(ctx, RBSOG_EINVAL, "charges are not neutral (sum %.3e)", qs);
    ctx->sum_q2[sys] = q2;
    ctx->desc[sys].U_self = self_energy(ctx, sys);
    CK(cudaMemcpyAsync(&ctx->d_desc[sys].U_self, &ctx->desc[sys].U_self, sizeof(double), cudaMemcpyHostToDevice,
                       ctx->st));
    CK(launch_pack(n, sx, sq, ctx->posq + off, 1, ctx->p[sys].L, ctx->st));
    if (v) CK(launch_pack(n, sv, nullptr, ctx->vel + off, 0, ctx->p[sys].L, ctx->st));
    else CK(cudaMemsetAsync(ctx->vel + off, 0, sizeof(double4_32a) * n, ctx->st));
    CK(cudaMemsetAsync(ctx->step_ctr + sys, 0, sizeof(int64_t), ctx->st));
    // a new state starts the Nose-Hoover variables xi, eta and their energy at zero
    CK(cudaMemsetAsync(ctx->energy + (int64_t)sys * kNumEnergy + 8, 0, sizeof(double) * 3, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));   // the caller may reuse its buffers
    // neighbour lists stay valid while every particle is within skin/2 of
    // its position at the last build: the displacement test of the next
    // force evaluation decides, for new positions as for integrated ones
    ctx->have_state[sys] = 1;
    ctx->force_valid[sys] = 0;
    return leave(ctx);
}

rbsog_status rbsog_set_state(rbsog_ctx *ctx, const double *q, const double *x, const double *v) {
    return rbsog_batch_set_state(ctx, 0, q, x, v);
}

rbsog_status rbsog_compute_forces(rbsog_ctx *ctx, const int32_t *m_kset, double *f_out, rbsog_energies *e_out) {
    if (!ctx) return RBSOG_EINVAL;
    if (!ctx->have_params || !all_state(ctx)) return fail(ctx, RBSOG_ESTATE, "params and state required");
    if (m_kset && ctx->n_sys != 1) return fail(ctx, RBSOG_EINVAL, "an explicit k-set needs a single system");
    if (!m_kset)
        for (int s = 0; s < ctx->n_sys; ++s)
            if (ctx->host_cursor[s] >= ctx->desc[s].n_sets)
                return fail(ctx, RBSOG_EINVAL, "pre-sampled k-sequence exhausted");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int4 *mex = nullptr;
    if (m_kset) {
        CK(cudaMemcpyAsync(ctx->m3_tmp, m_kset, sizeof(int32_t) * 3 * ctx->P, cudaMemcpyDefault, ctx->st));
        CK(launch_m_to_int4(ctx->P, ctx->m3_tmp, ctx->m_tmp, ctx->st));
        mex = ctx->m_tmp;
    }
    const BatchView bv = view(ctx, mex);
    es = enqueue_forces(ctx, bv, nullptr);
    if (es != RBSOG_OK) return es;
    CK(launch_finalize(bv, ctx->epart, ctx->rho, ctx->kpart, 0, ctx->energy, m_kset ? 0 : 1, ctx->st,
                       prof_of(ctx)));
    if (!m_kset)
        for (auto &c : ctx->host_cursor) c += 1;
    std::fill(ctx->force_valid.begin(), ctx->force_valid.end(), 1);
    if (f_out) {
        CK(launch_unpack(ctx->n_per[0], ctx->force, ctx->staging, ctx->st));
        CK(cudaMemcpyAsync(f_out, ctx->staging, sizeof(double) * 3 * ctx->n_per[0], cudaMemcpyDefault, ctx->st));
    }
    if (e_out || f_out) {
        es = check_flags(ctx);
        if (es != RBSOG_OK) return es;
    }
    if (e_out) {
        CK(cudaMemcpyAsync(ctx->h_energy, ctx->energy, sizeof(double) * kNumEnergy, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        e_out->U_near = ctx->h_energy[0];
        e_out->U_far = ctx->h_energy[1];
        e_out->U_self = ctx->h_energy[2];
        e_out->U_wca = ctx->h_energy[3];
        e_out->K = ctx->h_energy[4];
        e_out->T = ctx->h_energy[5];
        e_out->U_bound = ctx->h_energy[7];
        e_out->U_th = ctx->h_energy[10];
    }
    return leave(ctx);
}

rbsog_status rbsog_batch_step(rbsog_batch *ctx, int64_t nsteps) {
    if (!ctx) return RBSOG_EINVAL;
    if (nsteps < 0) return fail(ctx, RBSOG_EINVAL, "nsteps must be >= 0");
    if (!ctx->have_params || !all_state(ctx)) return fail(ctx, RBSOG_ESTATE, "params and state required");
    bool all_valid = true;
    for (int s = 0; s < ctx->n_sys; ++s) {
        const int64_t run = ctx->use_budget ? std::min(nsteps, ctx->remaining_host[s]) : nsteps;
        const int64_t need = run + (ctx->force_valid[s] ? 0 : 1);
        all_valid = all_valid && ctx->force_valid[s];
        if (ctx->host_cursor[s] + need > ctx->desc[s].n_sets)
            return fail(ctx, RBSOG_EINVAL, "system %d: pre-sampled k-sequence too short (%lld sets left, %lld needed)",
                        s, (long long)(ctx->desc[s].n_sets - ctx->host_cursor[s]), (long long)need);
    }
    if (nsteps == 0 && all_valid) return RBSOG_OK;
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    es = initial_forces(ctx);
    if (es != RBSOG_OK) return es;
    if (ctx->profiling) {
        for (int64_t t = 0; t < nsteps; ++t) {
            es = enqueue_step(ctx, t + 1 == nsteps);
            if (es != RBSOG_OK) return es;
        }
    } else if (nsteps >= 2 && drift_fusable(ctx)) {
        // one kick-drift, then steps whose scatter runs the next step's
        // kick-drift, then a last step that leaves the state at its end
        es = enqueue_kick_drift(ctx);
        if (es != RBSOG_OK) return es;
        es = capture_step(ctx, StepPart::tail_drift, &ctx->graph_fused);
        if (es != RBSOG_OK) return es;
        es = capture_step(ctx, StepPart::tail, &ctx->graph_tail);
        if (es != RBSOG_OK) return es;
        for (int64_t t = 0; t + 1 < nsteps; ++t) CK(cudaGraphLaunch(ctx->graph_fused, ctx->st));
        CK(cudaGraphLaunch(ctx->graph_tail, ctx->st));
    } else if (nsteps > 0) {
        // steps without energies, then the last one with them
        if (nsteps > 1) {
            es = capture_step(ctx, StepPart::whole, &ctx->graph);
            if (es != RBSOG_OK) return es;
        }
        es = capture_step(ctx, StepPart::whole_e, &ctx->graph_e);
        if (es != RBSOG_OK) return es;
        for (int64_t t = 0; t + 1 < nsteps; ++t) CK(cudaGraphLaunch(ctx->graph, ctx->st));
        CK(cudaGraphLaunch(ctx->graph_e, ctx->st));
    }
    for (int s = 0; s < ctx->n_sys; ++s) {
        const int64_t run = ctx->use_budget ? std::min(nsteps, ctx->remaining_host[s]) : nsteps;
        ctx->host_cursor[s] += run;
        if (ctx->use_budget) ctx->remaining_host[s] -= run;
    }
    return leave(ctx);
}

rbsog_status rbsog_step(rbsog_ctx *ctx, int64_t nsteps) { return rbsog_batch_step(ctx, nsteps); }

rbsog_status rbsog_step_io(rbsog_ctx *ctx, const double *q, const double *x, const double *v, const double *f,
                           int64_t kset_cursor, int64_t step, int64_t nsteps, double *x_out, double *v_out,
                           double *f_out) {
    if (!ctx || !q || !x || !v) return RBSOG_EINVAL;
    if (ctx->n_sys != 1) return fail(ctx, RBSOG_EINVAL, "rbsog_step_io needs a single system");
    if (!ctx->have_params) return fail(ctx, RBSOG_ESTATE, "set_params must come first");
    if (ctx->use_budget) return fail(ctx, RBSOG_EINVAL, "rbsog_step_io does not run step budgets");
    if (nsteps < 1 || step < 0 || kset_cursor < 0) return fail(ctx, RBSOG_EINVAL, "need nsteps >= 1, step >= 0, "
                                                                                  "cursor >= 0");
    const int64_t need = nsteps + (f ? 0 : 1);
    if (kset_cursor + need > ctx->desc[0].n_sets)
        return fail(ctx, RBSOG_EINVAL, "pre-sampled k-sequence too short (%lld sets from the cursor, %lld needed)",
                    (long long)(ctx->desc[0].n_sets - std::min(kset_cursor, ctx->desc[0].n_sets)), (long long)need);
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int64_t n = ctx->n_per[0];
    const size_t bytes3 = sizeof(double) * 3 * n;
    // the charges first: their sums (neutrality check, self energy) are
    // added on the host while the other inputs are still being copied
    const double *sq = kernel_view(q);
    if (!sq) {
        CK(cudaMemcpyAsync(ctx->staging + 9 * n, q, sizeof(double) * n, cudaMemcpyDefault, ctx->st));
        sq = ctx->staging + 9 * n;
    }
    const int64_t nb = (n + 255) / 256;
    CK(launch_charge_sums(n, sq, ctx->qpart, ctx->st));
    CK(cudaMemcpyAsync(ctx->h_qpart, ctx->qpart, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaEventRecord(ctx->ev_q, ctx->st));
    const double *in[3] = {x, v, f};
    const double *sin[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) {
        if (!in[k]) continue;
        sin[k] = kernel_view(in[k]);
        if (!sin[k]) {
            CK(cudaMemcpyAsync(ctx->staging + 3 * n * k, in[k], bytes3, cudaMemcpyDefault, ctx->st));
            sin[k] = ctx->staging + 3 * n * k;
        }
    }
    CK(cudaEventSynchronize(ctx->ev_q));
    double qs = 0.0, qa = 0.0, q2 = 0.0;
    for (int64_t b = 0; b < nb; ++b) {
        qs += ctx->h_qpart[3 * b];
        qa += ctx->h_qpart[3 * b + 1];
        q2 += ctx->h_qpart[3 * b + 2];
    }
    if (!std::isfinite(qa) || std::fabs(qs) > 1e-12 * qa) {
        CK(cudaStreamSynchronize(ctx->st));   // the caller may reuse its buffers
        if (!std::isfinite(qa)) return fail(ctx, RBSOG_EINVAL, "non-finite charge");
        return fail(ctx, RBSOG_EINVAL, "charges are not neutral (sum %.3e)", qs);
    }
    ctx->sum_q2[0] = q2;
    ctx->desc[0].U_self = self_energy(ctx, 0);
    std::memcpy(&ctx->h_i64[2], &ctx->desc[0].U_self, sizeof(double));
    ctx->h_i64[0] = kset_cursor;
    ctx->h_i64[1] = step;
    CK(cudaMemcpyAsync(&ctx->d_desc[0].U_self, &ctx->h_i64[2], sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->cursor, ctx->h_i64, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->step_ctr, ctx->h_i64 + 1, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->st));
    CK(launch_pack(n, sin[0], sq, ctx->posq, 1, ctx->p[0].L, ctx->st));
    CK(launch_pack(n, sin[1], nullptr, ctx->vel, 0, ctx->p[0].L, ctx->st));
    if (f) CK(launch_pack(n, sin[2], nullptr, ctx->force, 0, ctx->p[0].L, ctx->st));
    ctx->have_state[0] = 1;
    ctx->host_cursor[0] = kset_cursor;
    ctx->force_valid[0] = f ? 1 : 0;
    es = initial_forces(ctx);
    if (es != RBSOG_OK) return es;
    // all steps but the last one whole; the last one as kick-drift, then its
    // tail while the new positions are copied out on the io stream
    if (ctx->profiling) {
        for (int64_t t = 0; t + 1 < nsteps; ++t) {
            es = enqueue_step(ctx, false);
            if (es != RBSOG_OK) return es;
        }
    } else if (nsteps > 1) {
        es = capture_step(ctx, StepPart::whole, &ctx->graph);
        if (es != RBSOG_OK) return es;
        for (int64_t t = 0; t + 1 < nsteps; ++t) CK(cudaGraphLaunch(ctx->graph, ctx->st));
    }
    es = enqueue_kick_drift(ctx);
    if (es != RBSOG_OK) return es;
    double *out[3] = {x_out, v_out, f_out};
    const double4_32a *src[3] = {ctx->posq, ctx->vel, ctx->force};
    CK(cudaEventRecord(ctx->ev_x, ctx->st));
    CK(cudaStreamWaitEvent(ctx->io, ctx->ev_x, 0));
    if (x_out) {
        double *direct = kernel_view(x_out);
        CK(launch_unpack(n, src[0], direct ? direct : ctx->staging, ctx->io));
        if (!direct) CK(cudaMemcpyAsync(x_out, ctx->staging, bytes3, cudaMemcpyDefault, ctx->io));
    }
    CK(cudaEventRecord(ctx->ev_io, ctx->io));
    if (ctx->profiling) {
        es = enqueue_step_tail(ctx);
        if (es != RBSOG_OK) return es;
    } else {
        es = capture_step(ctx, StepPart::tail, &ctx->graph_tail);
        if (es != RBSOG_OK) return es;
        CK(cudaGraphLaunch(ctx->graph_tail, ctx->st));
    }
    for (int k = 1; k < 3; ++k) {
        if (!out[k]) continue;
        double *direct = kernel_view(out[k]);
        double *reg = ctx->staging + 3 * n * k;
        CK(launch_unpack(n, src[k], direct ? direct : reg, ctx->st));
        if (!direct) CK(cudaMemcpyAsync(out[k], reg, bytes3, cudaMemcpyDefault, ctx->st));
    }
    CK(cudaStreamWaitEvent(ctx->st, ctx->ev_io, 0));
    ctx->host_cursor[0] += nsteps;
    es = check_flags(ctx);   // synchronises: the outputs are in place on return
    if (es != RBSOG_OK) return es;
    return leave(ctx);
}

rbsog_status rbsog_batch_get_state(rbsog_batch *ctx, int32_t sys, double *x, double *v, double *f, int64_t *step) {
    if (!ctx) return RBSOG_EINVAL;
    rbsog_status es = check_sys(ctx, sys);
    if (es != RBSOG_OK) return es;
    if (!ctx->have_state[sys]) return fail(ctx, RBSOG_ESTATE, "no state");
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int64_t n = ctx->n_per[sys], off = ctx->p_off[sys];
    const size_t bytes = sizeof(double) * 3 * n;
    const double4_32a *src[3] = {ctx->posq + off, ctx->vel + off, ctx->force + off};
    double *dst[3] = {x, v, f};
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        double *direct = kernel_view(dst[k]);
        if (direct) {   // written in place (device or managed memory)
            CK(launch_unpack(n, src[k], direct, ctx->st));
            continue;
        }
        double *reg = ctx->staging + 3 * n * k;
        CK(launch_unpack(n, src[k], reg, ctx->st));
        CK(cudaMemcpyAsync(dst[k], reg, bytes, cudaMemcpyDefault, ctx->st));
    }
    if (step) {
        CK(cudaMemcpyAsync(ctx->h_i64, ctx->step_ctr + sys, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        *step = *ctx->h_i64;
    }
    es = check_flags(ctx);
    if (es != RBSOG_OK) return es;
    return leave(ctx);
}

rbsog_status rbsog_get_state(rbsog_ctx *ctx, double *x, double *v, double *f, int64_t *step) {
    return rbsog_batch_get_state(ctx, 0, x, v, f, step);
}

rbsog_status rbsog_get_cursor(const rbsog_ctx *ctx, int64_t *kset_cursor) {
    if (!ctx || !kset_cursor) return RBSOG_EINVAL;
    *kset_cursor = ctx->host_cursor[0];
    return RBSOG_OK;
}

rbsog_status rbsog_batch_restore(rbsog_batch *ctx, int32_t sys, const double *f, int64_t kset_cursor, int64_t step) {
    if (!ctx || !f) return RBSOG_EINVAL;
    rbsog_status es = check_sys(ctx, sys);
    if (es != RBSOG_OK) return es;
    if (!ctx->have_state[sys]) return fail(ctx, RBSOG_ESTATE, "set_state must come first");
    if (kset_cursor < 0 || kset_cursor > ctx->desc[sys].n_sets || step < 0)
        return fail(ctx, RBSOG_EINVAL, "cursor %lld outside [0, %lld]", (long long)kset_cursor,
                    (long long)ctx->desc[sys].n_sets);
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int64_t n = ctx->n_per[sys], off = ctx->p_off[sys];
    const double *sf = kernel_view(f);
    if (!sf) {
        CK(cudaMemcpyAsync(ctx->staging, f, sizeof(double) * 3 * n, cudaMemcpyDefault, ctx->st));
        sf = ctx->staging;
    }
    CK(launch_pack(n, sf, nullptr, ctx->force + off, 0, ctx->p[sys].L, ctx->st));
    ctx->h_i64[0] = kset_cursor;
    ctx->h_i64[1] = step;
    CK(cudaMemcpyAsync(ctx->cursor + sys, ctx->h_i64, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->step_ctr + sys, ctx->h_i64 + 1, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->host_cursor[sys] = kset_cursor;
    ctx->force_valid[sys] = 1;
    return leave(ctx);
}

rbsog_status rbsog_restore(rbsog_ctx *ctx, const double *f, int64_t kset_cursor, int64_t step) {
    return rbsog_batch_restore(ctx, 0, f, kset_cursor, step);
}

rbsog_status rbsog_batch_get_energies(rbsog_batch *ctx, int32_t sys, rbsog_energies *e) {
    if (!ctx || !e) return RBSOG_EINVAL;
    rbsog_status es = check_sys(ctx, sys);
    if (es != RBSOG_OK) return es;
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    CK(cudaMemcpyAsync(ctx->h_energy, ctx->energy + (int64_t)sys * kNumEnergy, sizeof(double) * kNumEnergy,
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    e->U_near = ctx->h_energy[0];
    e->U_far = ctx->h_energy[1];
    e->U_self = ctx->h_energy[2];
    e->U_wca = ctx->h_energy[3];
    e->U_bound = ctx->h_energy[7];
    e->U_th = ctx->h_energy[10];
    e->K = ctx->h_energy[4];
    e->T = ctx->h_energy[5];
    return leave(ctx);
}

rbsog_status rbsog_get_energies(rbsog_ctx *ctx, rbsog_energies *e) { return rbsog_batch_get_energies(ctx, 0, e); }

rbsog_status rbsog_batch_get_kseq(rbsog_batch *ctx, int32_t sys, int64_t set0, int64_t nsets, int32_t *m_out) {
    if (!ctx || !m_out || set0 < 0 || nsets < 0) return RBSOG_EINVAL;
    if (!ctx->have_params) return fail(ctx, RBSOG_ESTATE, "no params");
    rbsog_status es = check_sys(ctx, sys);
    if (es != RBSOG_OK) return es;
    if (set0 + nsets > ctx->desc[sys].n_sets) return fail(ctx, RBSOG_EINVAL, "k-set range beyond the sequence");
    const int64_t cnt = nsets * ctx->P;
    std::vector<int4> tmp((size_t)cnt);
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    CK(cudaMemcpyAsync(tmp.data(), ctx->kseq + ctx->desc[sys].k_off + set0 * ctx->P, sizeof(int4) * cnt,
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<int32_t> m3((size_t)cnt * 3);
    for (int64_t i = 0; i < cnt; ++i) {
        m3[3 * i] = tmp[i].x;
        m3[3 * i + 1] = tmp[i].y;
        m3[3 * i + 2] = tmp[i].z;
    }
    CK(cudaMemcpyAsync(m_out, m3.data(), sizeof(int32_t) * 3 * cnt, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

rbsog_status rbsog_get_kseq(rbsog_ctx *ctx, int64_t set0, int64_t nsets, int32_t *m_out) {
    return rbsog_batch_get_kseq(ctx, 0, set0, nsets, m_out);
}

rbsog_status rbsog_rho(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *rho_out) {
    if (!ctx || !m || !rho_out || P < 1) return RBSOG_EINVAL;
    if (ctx->n_sys != 1) return fail(ctx, RBSOG_EINVAL, "rbsog_rho needs a single system");
    if (!ctx->have_params || !all_state(ctx)) return fail(ctx, RBSOG_ESTATE, "params and state required");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    int32_t *m3 = nullptr;
    int4 *m4 = nullptr;
    double2 *part = nullptr, *rho = nullptr;
    void *kt = nullptr;
    CK(cudaMallocAsync((void **)&m3, sizeof(int32_t) * 3 * P, ctx->st));
    CK(cudaMallocAsync((void **)&m4, sizeof(int4) * P, ctx->st));
    CK(cudaMallocAsync((void **)&part, sizeof(double2) * (size_t)P * ctx->desc[0].n_ptiles, ctx->st));
    CK(cudaMallocAsync((void **)&rho, sizeof(double2) * P, ctx->st));
    CK(cudaMallocAsync(&kt, ktab_bytes(ctx->precision, P), ctx->st));
    CK(cudaMemcpyAsync(m3, m, sizeof(int32_t) * 3 * P, cudaMemcpyDefault, ctx->st));
    CK(launch_m_to_int4(P, m3, m4, ctx->st));
    const BatchView bv = view(ctx, m4, P);
    CK(launch_build_cells(bv, ctx->posq, ctx->cb, ctx->precision, ctx->sp64, ctx->sp32, ctx->st, prof_of(ctx)));
    CK(launch_rho_sweep(ctx->precision, bv, ctx->sp64, ctx->sp32, part, ctx->st, prof_of(ctx)));
    CK(launch_rho_combine(ctx->precision, bv, part, rho, kt, ctx->st, prof_of(ctx)));
    CK(cudaMemcpyAsync(rho_out, rho, sizeof(double2) * P, cudaMemcpyDefault, ctx->st));
    CK(cudaFreeAsync(m3, ctx->st));
    CK(cudaFreeAsync(m4, ctx->st));
    CK(cudaFreeAsync(part, ctx->st));
    CK(cudaFreeAsync(rho, ctx->st));
    CK(cudaFreeAsync(kt, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

namespace {

// Enqueues the virial of system 0 on the k-set m[P][3] (host or device)
// into the device array dW[9]; its scratch is stream-ordered.
rbsog_status virial_device(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *dW) {
    const int64_t n = ctx->n_per[0];
    const int M = ctx->p[0].M;
    int32_t *m3 = nullptr;
    int4 *m4 = nullptr;
    double2 *part = nullptr, *rho = nullptr;
    void *kt = nullptr;
    double *vpart = nullptr, *dom = nullptr, *dsl = nullptr;
    CK(cudaMallocAsync((void **)&m3, sizeof(int32_t) * 3 * P, ctx->st));
    CK(cudaMallocAsync((void **)&m4, sizeof(int4) * P, ctx->st));
    CK(cudaMallocAsync((void **)&part, sizeof(double2) * (size_t)P * ctx->desc[0].n_ptiles, ctx->st));
    CK(cudaMallocAsync((void **)&rho, sizeof(double2) * P, ctx->st));
    CK(cudaMallocAsync(&kt, ktab_bytes(ctx->precision, P), ctx->st));
    CK(cudaMallocAsync((void **)&vpart, sizeof(double) * 6 * (size_t)virial_blocks(n), ctx->st));
    CK(cudaMallocAsync((void **)&dom, sizeof(double) * (M + 1), ctx->st));
    CK(cudaMallocAsync((void **)&dsl, sizeof(double) * (M + 1), ctx->st));
    CK(cudaMemcpyAsync(m3, m, sizeof(int32_t) * 3 * P, cudaMemcpyDefault, ctx->st));
    CK(cudaMemcpyAsync(dom, ctx->omega.data(), sizeof(double) * (M + 1), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(dsl, ctx->s.data(), sizeof(double) * (M + 1), cudaMemcpyHostToDevice, ctx->st));
    CK(launch_m_to_int4(P, m3, m4, ctx->st));
    const BatchView bv = view(ctx, m4, P);
    CK(launch_build_cells(bv, ctx->posq, ctx->cb, ctx->precision, ctx->sp64, ctx->sp32, ctx->st, prof_of(ctx)));
    CK(launch_rho_sweep(ctx->precision, bv, ctx->sp64, ctx->sp32, part, ctx->st, prof_of(ctx)));
    CK(launch_rho_combine(ctx->precision, bv, part, rho, kt, ctx->st, prof_of(ctx)));
    CK(launch_virial(ctx->d_desc, n, ctx->nsog, ctx->cb.start, ctx->cb.perm, ctx->cb.cell_of, ctx->posq, vpart, rho,
                     m3, P, dom, dsl, M, ctx->S[0], dW, ctx->st));
    for (void *ptr : {(void *)m3, (void *)m4, (void *)part, (void *)rho, kt, (void *)vpart, (void *)dom,
                      (void *)dsl})
        CK(cudaFreeAsync(ptr, ctx->st));
    return RBSOG_OK;
}

// Heat flux J[3] of system 0 (Appendix A) into device memory dJ; the far
// term on the k-set m (host or device, P >= 1), none for P == 0.
rbsog_status heat_flux_device(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *dJ) {
    const int64_t n = ctx->n_per[0];
    const int M = ctx->p[0].M;
    const int32_t nb = heat_blocks(n);
    const int32_t Pa = P > 0 ? P : 1;
    int32_t *m3 = nullptr;
    double2 *rpart = nullptr, *rho = nullptr;
    double4_32a *ktab = nullptr;
    double *part = nullptr, *dom = nullptr, *dsl = nullptr;
    CK(cudaMallocAsync((void **)&m3, sizeof(int32_t) * 3 * Pa, ctx->st));
    CK(cudaMallocAsync((void **)&rpart, sizeof(double2) * heat_rho_partials(Pa), ctx->st));
    CK(cudaMallocAsync((void **)&rho, sizeof(double2) * Pa, ctx->st));
    CK(cudaMallocAsync((void **)&ktab, sizeof(double4_32a) * 2 * Pa, ctx->st));
    CK(cudaMallocAsync((void **)&part, sizeof(double) * 6 * (size_t)nb, ctx->st));
    CK(cudaMallocAsync((void **)&dom, sizeof(double) * (M + 1), ctx->st));
    CK(cudaMallocAsync((void **)&dsl, sizeof(double) * (M + 1), ctx->st));
    if (P > 0) CK(cudaMemcpyAsync(m3, m, sizeof(int32_t) * 3 * P, cudaMemcpyDefault, ctx->st));
    CK(cudaMemcpyAsync(dom, ctx->omega.data(), sizeof(double) * (M + 1), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(dsl, ctx->s.data(), sizeof(double) * (M + 1), cudaMemcpyHostToDevice, ctx->st));
    const BatchView bv = view(ctx);
    CK(launch_build_cells(bv, ctx->posq, ctx->cb, ctx->precision, ctx->sp64, ctx->sp32, ctx->st, prof_of(ctx)));
    double FM0 = 0.0;
    for (int l = 0; l <= M; ++l) FM0 += ctx->omega[l];
    const BoxDev &box = ctx->desc[0].box;
    const double lB = ctx->p[0].coulomb_prefactor;
    const double V = box.L[0] * box.L[1] * box.L[2];
    const double half_c = P > 0 ? lB * std::pow(kPi, 1.5) * ctx->S[0] / (2.0 * P * V) : 0.0;
    CK(launch_heat_flux(ctx->d_desc, box, n, ctx->nsog, ctx->cb.start, ctx->cb.perm, ctx->cb.cell_of, ctx->posq,
                        ctx->vel, ctx->p[0].mass, 0.5 * lB * FM0, m3, P, dom, dsl, M, half_c, rpart, rho, ktab, part,
                        part + 3 * (size_t)nb, dJ, ctx->st));
    for (void *ptr : {(void *)m3, (void *)rpart, (void *)rho, (void *)ktab, (void *)part, (void *)dom, (void *)dsl})
        CK(cudaFreeAsync(ptr, ctx->st));
    return RBSOG_OK;
}

rbsog_status single_system_ready(rbsog_ctx *ctx, const char *what) {
    if (ctx->n_sys != 1) return fail(ctx, RBSOG_EINVAL, "%s needs a single system", what);
    if (!ctx->have_params || !all_state(ctx)) return fail(ctx, RBSOG_ESTATE, "params and state required");
    return RBSOG_OK;
}

}  // namespace

rbsog_status rbsog_compute_virial(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *W_out) {
    if (!ctx || !m || !W_out || P < 1) return RBSOG_EINVAL;
    rbsog_status es = single_system_ready(ctx, "rbsog_compute_virial");
    if (es != RBSOG_OK) return es;
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    double *dW = nullptr;
    CK(cudaMallocAsync((void **)&dW, sizeof(double) * 9, ctx->st));
    es = virial_device(ctx, m, P, dW);
    if (es != RBSOG_OK) return es;
    CK(cudaMemcpyAsync(W_out, dW, sizeof(double) * 9, cudaMemcpyDefault, ctx->st));
    CK(cudaFreeAsync(dW, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

rbsog_status rbsog_compute_heat_flux(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *J_out) {
    if (!ctx || !J_out || P < 0 || (P > 0 && !m)) return RBSOG_EINVAL;
    rbsog_status es = single_system_ready(ctx, "rbsog_compute_heat_flux");
    if (es != RBSOG_OK) return es;
    if (ctx->p[0].boundary != 0)
        return fail(ctx, RBSOG_EINVAL, "rbsog_compute_heat_flux covers tinfoil systems (boundary 0)");
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    double *dJ = nullptr;
    CK(cudaMallocAsync((void **)&dJ, sizeof(double) * 3, ctx->st));
    es = heat_flux_device(ctx, m, P, dJ);
    if (es != RBSOG_OK) return es;
    CK(cudaMemcpyAsync(J_out, dJ, sizeof(double) * 3, cudaMemcpyDefault, ctx->st));
    CK(cudaFreeAsync(dJ, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

rbsog_status rbsog_compute_pressure(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *P_out) {
    if (!ctx || !m || !P_out || P < 1) return RBSOG_EINVAL;
    rbsog_status es = single_system_ready(ctx, "rbsog_compute_pressure");
    if (es != RBSOG_OK) return es;
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int64_t n = ctx->n_per[0];
    double *dW = nullptr, *kpart = nullptr, *dP = nullptr;
    CK(cudaMallocAsync((void **)&dW, sizeof(double) * 9, ctx->st));
    CK(cudaMallocAsync((void **)&dP, sizeof(double) * 9, ctx->st));
    CK(cudaMallocAsync((void **)&kpart, sizeof(double) * 6 * (size_t)obs_blocks(n), ctx->st));
    es = virial_device(ctx, m, P, dW);
    if (es != RBSOG_OK) return es;
    const double V = ctx->p[0].L[0] * ctx->p[0].L[1] * ctx->p[0].L[2];
    CK(launch_pressure(n, ctx->vel, ctx->p[0].mass, dW, V, kpart, dP, ctx->st));
    CK(cudaMemcpyAsync(P_out, dP, sizeof(double) * 9, cudaMemcpyDefault, ctx->st));
    for (void *ptr : {(void *)dW, (void *)dP, (void *)kpart}) CK(cudaFreeAsync(ptr, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

rbsog_status rbsog_observe_start(rbsog_ctx *ctx, int32_t n_lags, int32_t origin_every) {
    if (!ctx) return RBSOG_EINVAL;
    if (n_lags < 1 || origin_every < 1)
        return fail(ctx, RBSOG_EINVAL, "n_lags and origin_every must be >= 1");
    const int64_t slots = ((int64_t)n_lags + origin_every - 1) / origin_every;
    if (slots > kObsMaxPairs)
        return fail(ctx, RBSOG_EINVAL, "n_lags / origin_every may keep at most %d origins (asked %lld)", kObsMaxPairs,
                    (long long)slots);
    rbsog_status es = single_system_ready(ctx, "rbsog_observe_start");
    if (es != RBSOG_OK) return es;
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int64_t n = ctx->n_per[0];
    CK(cudaStreamSynchronize(ctx->st));   // earlier samples may still read the buffers being replaced
    CK(dalloc(&ctx->obs_xprev, n));
    CK(dalloc(&ctx->obs_u, n));
    CK(dalloc(&ctx->obs_ring_u, (size_t)slots * n));
    CK(dalloc(&ctx->obs_ring_v, (size_t)slots * n));
    CK(dalloc(&ctx->obs_part, (size_t)obs_blocks(n) * kObsMaxPairs));
    CK(dalloc(&ctx->obs_acc, 4 * (size_t)n_lags));
    CK(dalloc(&ctx->obs_count, n_lags));
    CK(cudaMemsetAsync(ctx->obs_acc, 0, sizeof(double) * 4 * n_lags, ctx->st));
    CK(cudaMemsetAsync(ctx->obs_count, 0, sizeof(int64_t) * n_lags, ctx->st));
    ctx->obs_lags = n_lags;
    ctx->obs_every = origin_every;
    ctx->obs_slots = (int32_t)slots;
    ctx->obs_frame = 0;
    return leave(ctx);
}

rbsog_status rbsog_observe_sample(rbsog_ctx *ctx) {
    if (!ctx) return RBSOG_EINVAL;
    if (ctx->obs_lags == 0) return fail(ctx, RBSOG_ESTATE, "rbsog_observe_start must come first");
    rbsog_status es = single_system_ready(ctx, "rbsog_observe_sample");
    if (es != RBSOG_OK) return es;
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int64_t j = ctx->obs_frame, every = ctx->obs_every;
    const int store = j % every == 0 ? (int)((j / every) % ctx->obs_slots) : -1;
    // the origins c * every <= j still within n_lags of frame j, newest first
    ObsPairs pr{};
    for (int64_t c = j / every; c >= 0 && j - c * every < ctx->obs_lags; --c) {
        pr.slot[pr.n] = (int32_t)(c % ctx->obs_slots);
        pr.lag[pr.n] = (int32_t)(j - c * every);
        ++pr.n;
    }
    CK(launch_obs_sample(ctx->n_per[0], ctx->posq, ctx->vel, ctx->obs_xprev, ctx->obs_u, ctx->obs_ring_u,
                         ctx->obs_ring_v, ctx->p[0].L, j == 0, store, pr, ctx->obs_part, ctx->obs_acc,
                         ctx->obs_acc + ctx->obs_lags, ctx->obs_count, ctx->st));
    ctx->obs_frame = j + 1;
    return leave(ctx);
}

rbsog_status rbsog_observe_result(rbsog_ctx *ctx, double *msd, double *vacf, int64_t *count) {
    if (!ctx) return RBSOG_EINVAL;
    if (ctx->obs_lags == 0) return fail(ctx, RBSOG_ESTATE, "rbsog_observe_start must come first");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int32_t L = ctx->obs_lags;
    double *res = ctx->obs_acc + 2 * L;
    CK(launch_obs_result(L, ctx->n_per[0], ctx->obs_acc, ctx->obs_acc + L, ctx->obs_count, res, ctx->st));
    if (msd) CK(cudaMemcpyAsync(msd, res, sizeof(double) * L, cudaMemcpyDefault, ctx->st));
    if (vacf) CK(cudaMemcpyAsync(vacf, res + L, sizeof(double) * L, cudaMemcpyDefault, ctx->st));
    if (count) CK(cudaMemcpyAsync(count, ctx->obs_count, sizeof(int64_t) * L, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

rbsog_status rbsog_green_kubo(const double *P_series, int64_t n_samples, double dt, double V, double T,
                              int32_t max_lag, double *acf_out, double *C_out, void *stream) {
    rbsog_ctx *ctx = nullptr;   // context-free: CK reports the status only
    if (!P_series || !C_out || n_samples < 2 || max_lag < 2 || max_lag > n_samples || !(T > 0.0) || !(V > 0.0) ||
        !(dt > 0.0))
        return RBSOG_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *ser = nullptr, *scr = nullptr;
    CK(cudaMallocAsync((void **)&ser, sizeof(double) * 9 * (size_t)n_samples, st));
    CK(cudaMallocAsync((void **)&scr, sizeof(double) * (7 + (size_t)max_lag), st));
    CK(cudaMemcpyAsync(ser, P_series, sizeof(double) * 9 * (size_t)n_samples, cudaMemcpyDefault, st));
    CK(launch_green_kubo(ser, n_samples, max_lag, V * dt / (6.0 * T), scr, scr + 7, scr + 6, st));
    if (acf_out) CK(cudaMemcpyAsync(acf_out, scr + 7, sizeof(double) * max_lag, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(C_out, scr + 6, sizeof(double), cudaMemcpyDefault, st));
    CK(cudaFreeAsync(ser, st));
    CK(cudaFreeAsync(scr, st));
    CK(cudaStreamSynchronize(st));
    return RBSOG_OK;
}

rbsog_status rbsog_green_kubo_heat(const double *J_series, int64_t n_samples, double dt, double V, double T,
                                   int32_t max_lag, double *acf_out, double *C_out, void *stream) {
    rbsog_ctx *ctx = nullptr;   // context-free: CK reports the status only
    if (!J_series || !C_out || n_samples < 2 || max_lag < 2 || max_lag > n_samples || !(T > 0.0) || !(V > 0.0) ||
        !(dt > 0.0))
        return RBSOG_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *ser = nullptr, *scr = nullptr;
    CK(cudaMallocAsync((void **)&ser, sizeof(double) * 3 * (size_t)n_samples, st));
    CK(cudaMallocAsync((void **)&scr, sizeof(double) * (1 + (size_t)max_lag), st));
    CK(cudaMemcpyAsync(ser, J_series, sizeof(double) * 3 * (size_t)n_samples, cudaMemcpyDefault, st));
    CK(launch_green_kubo_heat(ser, n_samples, max_lag, V * dt / (3.0 * T * T), scr + 1, scr, st));
    if (acf_out) CK(cudaMemcpyAsync(acf_out, scr + 1, sizeof(double) * max_lag, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(C_out, scr, sizeof(double), cudaMemcpyDefault, st));
    CK(cudaFreeAsync(ser, st));
    CK(cudaFreeAsync(scr, st));
    CK(cudaStreamSynchronize(st));
    return RBSOG_OK;
}

rbsog_status rbsog_get_cells(rbsog_ctx *ctx, int32_t *cell_start, int32_t *perm, int32_t *nbr) {
    if (!ctx) return RBSOG_EINVAL;
    if (ctx->n_sys != 1) return fail(ctx, RBSOG_EINVAL, "rbsog_get_cells needs a single system");
    if (!ctx->have_params || !all_state(ctx)) return fail(ctx, RBSOG_ESTATE, "params and state required");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const Prof *pf = prof_of(ctx);
    const BatchView bv = view(ctx);
    CK(launch_build_cells(bv, ctx->posq, ctx->cb, ctx->precision, ctx->sp64, ctx->sp32, ctx->st, pf));
    if (nbr) {
        CK(launch_near(ctx->precision, bv, ctx->nsog, ctx->cb.start, ctx->sp64, ctx->sp32, ctx->fnear, ctx->epart,
                       ctx->nbr_sorted, ctx->st, pf));
        CK(launch_unsort_i32(ctx->n_total, 0, ctx->cb.perm, ctx->nbr_sorted, ctx->i32_tmp, ctx->st));
        CK(cudaMemcpyAsync(nbr, ctx->i32_tmp, sizeof(int32_t) * ctx->n_total, cudaMemcpyDefault, ctx->st));
    }
    if (cell_start)
        CK(cudaMemcpyAsync(cell_start, ctx->cb.start, sizeof(int32_t) * (ctx->ncell_total + 1), cudaMemcpyDefault,
                           ctx->st));
    if (perm) CK(cudaMemcpyAsync(perm, ctx->cb.perm, sizeof(int32_t) * ctx->n_total, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

rbsog_status rbsog_batch_rdf(rbsog_batch *ctx, int32_t sys, int32_t nbins, uint64_t *counts, double *g) {
    if (!ctx) return RBSOG_EINVAL;
    rbsog_status es = check_sys(ctx, sys);
    if (es != RBSOG_OK) return es;
    if (!ctx->have_params || !ctx->have_state[sys]) return fail(ctx, RBSOG_ESTATE, "params and state required");
    if (nbins < 16 || nbins > 4096 || (nbins & (nbins - 1)))
        return fail(ctx, RBSOG_EINVAL, "nbins must be a power of two in [16, 4096]");
    const double *L = ctx->p[sys].L;
    if (L[0] != L[1] || L[0] != L[2]) return fail(ctx, RBSOG_EINVAL, "the RDF needs a cubic box");
    es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int64_t n = ctx->n_per[sys];
    unsigned long long *d_counts = nullptr;
    double *d_g = nullptr;
    const size_t nc = 3 * (size_t)nbins;
    CK(cudaMallocAsync((void **)&d_counts, sizeof(unsigned long long) * (nc + 2), ctx->st));
    CK(cudaMallocAsync((void **)&d_g, sizeof(double) * nc, ctx->st));
    // the staging buffer (24 bytes per particle) holds the packed uint4 sites
    CK(launch_rdf(n, ctx->posq + ctx->p_off[sys], L[0], nbins, reinterpret_cast<uint4 *>(ctx->staging), d_counts,
                  d_counts + nc, d_g, ctx->st, prof_of(ctx)));
    if (counts) CK(cudaMemcpyAsync(counts, d_counts, sizeof(uint64_t) * nc, cudaMemcpyDefault, ctx->st));
    if (g) CK(cudaMemcpyAsync(g, d_g, sizeof(double) * nc, cudaMemcpyDefault, ctx->st));
    CK(cudaFreeAsync(d_counts, ctx->st));
    CK(cudaFreeAsync(d_g, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

rbsog_status rbsog_rdf(rbsog_ctx *ctx, int32_t nbins, uint64_t *counts, double *g) {
    return rbsog_batch_rdf(ctx, 0, nbins, counts, g);
}

rbsog_status rbsog_set_profiling(rbsog_ctx *ctx, int on) {
    if (!ctx) return RBSOG_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->st));
    for (auto &r : ctx->prof_done) {
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof_done.clear();
    ctx->prof_acc.clear();
    ctx->profiling = on != 0;
    return RBSOG_OK;
}

rbsog_status rbsog_get_profile(rbsog_ctx *ctx, int32_t cap, char (*names)[32], int64_t *launches, double *ms,
                               int32_t *count) {
    if (!ctx || !count) return RBSOG_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->st));
    for (auto &r : ctx->prof_done) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        auto &acc = ctx->prof_acc[r.name];
        acc.first += 1;
        acc.second += t;
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof_done.clear();
    int32_t i = 0;
    for (auto &kv : ctx->prof_acc) {
        if (i < cap) {
            if (names) {
                std::strncpy(names[i], kv.first.c_str(), 31);
                names[i][31] = 0;
            }
            if (launches) launches[i] = kv.second.first;
            if (ms) ms[i] = kv.second.second;
        }
        ++i;
    }
    *count = i;
    return RBSOG_OK;
}

const char *rbsog_last_error(const rbsog_ctx *ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

rbsog_status rbsog_destroy(rbsog_ctx *ctx) {
    if (!ctx) return RBSOG_OK;
    cudaSetDevice(ctx->device);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    drop_graph(ctx);
    for (auto &r : ctx->prof_done) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto &r : ctx->prof_open) cudaEventDestroy(r.a);
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    dfree(&ctx->posq);
    dfree(&ctx->vel);
    dfree(&ctx->force);
    dfree(&ctx->fnear);
    dfree(&ctx->sp64);
    dfree(&ctx->sp32);
    dfree(&ctx->staging);
    dfree(&ctx->qpart);
    if (ctx->h_qpart) cudaFreeHost(ctx->h_qpart);
    ctx->h_qpart = nullptr;
    dfree(&ctx->nbr_sorted);
    dfree(&ctx->i32_tmp);
    dfree(&ctx->cb.cell_of);
    dfree(&ctx->cb.slot);
    dfree(&ctx->cb.count);
    dfree(&ctx->cb.start);
    dfree(&ctx->cb.tile_sum);
    dfree(&ctx->cb.perm_raw);
    dfree(&ctx->cb.perm);
    dfree(&ctx->cb.key);
    dfree(&ctx->sp32c);
    dfree(&ctx->xref);
    dfree(&ctx->nbr_cnt);
    dfree(&ctx->list_perm);
    dfree(&ctx->lpos);
    dfree(&ctx->linv);
    dfree(&ctx->d_ltab);
    dfree(&ctx->d_cstab);
    dfree(&ctx->nbr_list);
    dfree(&ctx->d_rebuild);
    dfree(&ctx->cb.pack);
    dfree(&ctx->kpart);
    dfree(&ctx->kseq);
    dfree(&ctx->kfold);
    dfree(&ctx->kcount);
    dfree(&ctx->cursor);
    dfree(&ctx->step_ctr);
    dfree(&ctx->rho_part);
    dfree(&ctx->rho);
    dfree(&ctx->epart);
    if (ctx->ktab) cudaFree(ctx->ktab);
    dfree(&ctx->energy);
    dfree(&ctx->err_flag);
    dfree(&ctx->m_tmp);
    dfree(&ctx->m3_tmp);
    dfree(&ctx->d_desc);
    dfree(&ctx->d_pblk);
    dfree(&ctx->d_nblk);
    dfree(&ctx->d_sblk);
    dfree(&ctx->d_cell_sys);
    dfree(&ctx->d_mask);
    dfree(&ctx->fin_part);
    dfree(&ctx->dpart);
    dfree(&ctx->dip);
    dfree(&ctx->fin_count);
    dfree(&ctx->d_kw);
    dfree(&ctx->obs_xprev);
    dfree(&ctx->obs_u);
    dfree(&ctx->obs_ring_u);
    dfree(&ctx->obs_ring_v);
    dfree(&ctx->obs_part);
    dfree(&ctx->obs_acc);
    dfree(&ctx->obs_count);
    dfree(&ctx->d_remaining);
    if (ctx->h_energy) cudaFreeHost(ctx->h_energy);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->h_i64) cudaFreeHost(ctx->h_i64);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->ev_q) cudaEventDestroy(ctx->ev_q);
    if (ctx->ev_x) cudaEventDestroy(ctx->ev_x);
    if (ctx->ev_io) cudaEventDestroy(ctx->ev_io);
    if (ctx->st) cudaStreamDestroy(ctx->st);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->far) cudaStreamDestroy(ctx->far);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->io) cudaStreamDestroy(ctx->io);
    delete ctx;
    return RBSOG_OK;
}

}  // extern "C"

// ---- serving engine -------------------------------------------------------------
// Continuous batching of MD jobs: jobs wait in a FIFO queue, are admitted
// while a job slot is free and their device-memory footprint fits the budget,
// and advance together as one batch (one graph launch per step).  A job whose
// step budget is used up is frozen on the device and retired at the end of
// the quantum; admissions and retirements rebuild the batch at the next
// quantum, moving running jobs' state, forces, cursors and k-sequences
// device-to-device so that no running job is re-sampled or perturbed.
namespace {

struct Job {
    int64_t id = 0, n = 0, nsteps = 0, footprint = 0;
    rbsog_params p{};
    std::vector<double> q, x, v;           // inputs until admission
    std::vector<double> xo, vo, fo;        // results after retirement
    rbsog_energies e{};
    int32_t status = 0;                    // 0 waiting, 1 running, 2 done
    int64_t steps_done = 0;
};

}  // namespace

struct rbsog_server {
    int device = 0;
    cudaStream_t user = nullptr;
    int32_t max_jobs = 64, quantum = 50;
    int64_t budget = 0, used = 0;
    std::map<int64_t, Job> jobs;
    std::vector<int64_t> waiting;     // FIFO
    std::vector<int64_t> active;      // system order of the current batch
    rbsog_ctx *batch = nullptr;
    int64_t frozen_n = 0;             // particles of retired jobs still in the batch
    int64_t next_id = 1;
    bool have_shape = false;          // the parameters every job must share (set by the first submit)
    rbsog_params shape{};
    std::string err;
};

namespace {

int64_t footprint_bytes(const Job &j) {
    // state, cell-ordered copies, cell arrays and staging per particle; the
    // k-sequence and its folded copy; cells and partial sums
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) ncell *= (int64_t)std::floor(j.p.L[d] / j.p.r_c);
    return j.n * 256 + (j.nsteps + 1) * ((int64_t)j.p.P * 32 + 4) + ncell * 16 + (int64_t)j.p.P * 4096;
}

rbsog_status srv_fail(rbsog_server *s, rbsog_status st, const std::string &m) {
    s->err = m;
    return st;
}

#define CK_S(srv, call)                                                                 \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return srv_fail(srv, RBSOG_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

// Build a batch of `keep` (running, state moved from the old batch) followed
// by `add` (new, loaded from host); destroy the old batch.
rbsog_status rebuild(rbsog_server *sv, const std::vector<int64_t> &keep, const std::vector<int64_t> &add) {
    std::vector<int64_t> order(keep);
    order.insert(order.end(), add.begin(), add.end());
    rbsog_ctx *old = sv->batch;
    if (order.empty()) {
        if (old) rbsog_destroy(old);
        sv->batch = nullptr;
        sv->active.clear();
        return RBSOG_OK;
    }
    std::vector<int64_t> n_per;
    std::vector<rbsog_params> ps;
    std::vector<char> sample;
    for (size_t k = 0; k < order.size(); ++k) {
        const Job &j = sv->jobs[order[k]];
        n_per.push_back(j.n);
        ps.push_back(j.p);
        sample.push_back(k < keep.size() ? 0 : 1);
    }
    rbsog_ctx *nb = nullptr;
    rbsog_status st = rbsog_batch_create(&nb, (int32_t)order.size(), n_per.data(), sv->device, sv->user);
    if (st != RBSOG_OK) return srv_fail(sv, st, "batch create failed");
    rbsog_ctx *ctx = nb;
    st = set_params_impl(nb, ps.data(), &sample);
    if (st != RBSOG_OK) {
        std::string m = nb->err;
        rbsog_destroy(nb);
        return srv_fail(sv, st, "set_params: " + m);
    }
    nb->use_budget = true;
    nb->remaining_host.assign(order.size(), 0);
    CK(dalloc(&nb->d_remaining, order.size()));
    st = enter(nb);
    if (st != RBSOG_OK) return st;
    // running jobs: everything moves device to device
    std::map<int64_t, int> old_index;
    for (size_t k = 0; k < sv->active.size(); ++k) old_index[sv->active[k]] = (int)k;
    if (old) CK(cudaStreamSynchronize(old->st));
    for (size_t k = 0; k < keep.size(); ++k) {
        const int o = old_index.at(keep[k]);
        const SysDesc &od = old->desc[o];
        const SysDesc &ndsc = nb->desc[k];
        const int64_t n = od.n;
        CK(cudaMemcpyAsync(nb->kseq + ndsc.k_off, old->kseq + od.k_off,
                           sizeof(int4) * old->n_chains[o] * old->chain_len[o], cudaMemcpyDeviceToDevice, nb->st));
        if (nb->kfold && old->kfold) {
            CK(cudaMemcpyAsync(nb->kfold + ndsc.k_off, old->kfold + od.k_off,
                               sizeof(int4) * old->n_chains[o] * old->chain_len[o], cudaMemcpyDeviceToDevice, nb->st));
            CK(cudaMemcpyAsync(nb->kcount + ndsc.kc_off, old->kcount + od.kc_off, sizeof(int32_t) * od.n_sets,
                               cudaMemcpyDeviceToDevice, nb->st));
        }
        CK(cudaMemcpyAsync(nb->posq + ndsc.p_off, old->posq + od.p_off, sizeof(double4_32a) * n,
                           cudaMemcpyDeviceToDevice, nb->st));
        CK(cudaMemcpyAsync(nb->vel + ndsc.p_off, old->vel + od.p_off, sizeof(double4_32a) * n,
                           cudaMemcpyDeviceToDevice, nb->st));
        CK(cudaMemcpyAsync(nb->force + ndsc.p_off, old->force + od.p_off, sizeof(double4_32a) * n,
                           cudaMemcpyDeviceToDevice, nb->st));
        CK(cudaMemcpyAsync(nb->cursor + k, old->cursor + o, sizeof(int64_t), cudaMemcpyDeviceToDevice, nb->st));
        CK(cudaMemcpyAsync(nb->step_ctr + k, old->step_ctr + o, sizeof(int64_t), cudaMemcpyDeviceToDevice, nb->st));
        CK(cudaMemcpyAsync(nb->energy + k * kNumEnergy, old->energy + (int64_t)o * kNumEnergy,
                           sizeof(double) * kNumEnergy, cudaMemcpyDeviceToDevice, nb->st));
        if (nb->use_list && old->use_list) {
            // the running system keeps its neighbour lists, reference
            // positions and rebuild flag: its trajectory is the one it
            // follows alone
            CK(cudaMemcpyAsync(nb->d_rebuild + k, old->d_rebuild + o, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                               nb->st));
            CK(launch_list_move(n, od.p_off, ndsc.p_off, old->list_cap, nb->list_cap, old->nbr_list,
                                old->nbr_cnt, old->list_perm, old->xref, old->linv, nb->nbr_list, nb->nbr_cnt,
                                nb->list_perm, nb->xref, nb->linv, nb->d_rebuild + k, nb->st));
        }
        nb->have_state[k] = 1;
        nb->force_valid[k] = old->force_valid[o];
        nb->host_cursor[k] = old->host_cursor[o];
        nb->sum_q2[k] = old->sum_q2[o];
        nb->desc[k].U_self = self_energy(nb, (int)k);
        nb->remaining_host[k] = old->remaining_host[o];
    }
    st = upload_desc(nb);
    if (st != RBSOG_OK) return st;
    CK(cudaMemcpyAsync(nb->d_remaining, nb->remaining_host.data(), sizeof(int64_t) * keep.size(),
                       cudaMemcpyHostToDevice, nb->st));
    CK(cudaStreamSynchronize(nb->st));
    st = leave(nb);
    if (st != RBSOG_OK) return st;
    // new jobs: loaded from host; their first step starts with a force evaluation
    for (size_t k = keep.size(); k < order.size(); ++k) {
        Job &j = sv->jobs[order[k]];
        st = rbsog_batch_set_state(nb, (int32_t)k, j.q.data(), j.x.data(), j.v.data());
        if (st != RBSOG_OK) {
            std::string m = nb->err;
            rbsog_destroy(nb);
            return srv_fail(sv, st, "set_state: " + m);
        }
        nb->remaining_host[k] = j.nsteps;
        *nb->h_i64 = j.nsteps;
        CK(cudaMemcpyAsync(nb->d_remaining + k, nb->h_i64, sizeof(int64_t), cudaMemcpyHostToDevice, nb->st));
        CK(cudaStreamSynchronize(nb->st));
        j.status = 1;
        std::vector<double>().swap(j.q);
        std::vector<double>().swap(j.x);
        std::vector<double>().swap(j.v);
    }
    if (old) rbsog_destroy(old);
    sv->batch = nb;
    sv->active = order;
    return RBSOG_OK;
}

}  // namespace

extern "C" {

rbsog_status rbsog_server_create(rbsog_server **out, int32_t max_jobs, int64_t mem_budget_bytes, int32_t quantum,
                                 int device, void *stream) {
    if (!out || max_jobs < 1 || mem_budget_bytes <= 0 || quantum < 1) return RBSOG_EINVAL;
    rbsog_server *s = new (std::nothrow) rbsog_server();
    if (!s) return RBSOG_ENOMEM;
    s->max_jobs = max_jobs;
    s->budget = mem_budget_bytes;
    s->quantum = quantum;
    s->device = device;
    s->user = (cudaStream_t)stream;
    *out = s;
    return RBSOG_OK;
}

rbsog_status rbsog_server_submit(rbsog_server *s, int64_t n, const rbsog_params *p, const double *q,
                                 const double *x, const double *v, int64_t nsteps, int64_t *job_id) {
    if (!s || !p || !q || !x || n < 2 || nsteps < 1) return RBSOG_EINVAL;
    Job j;
    j.id = s->next_id++;
    j.n = n;
    j.nsteps = nsteps;
    j.p = *p;
    j.p.n_ksets = nsteps + 1;
    j.q.assign(q, q + n);
    j.x.assign(x, x + 3 * n);
    if (v) j.v.assign(v, v + 3 * n);
    else j.v.assign(3 * n, 0.0);
    j.footprint = footprint_bytes(j);
    if (j.footprint > s->budget) return srv_fail(s, RBSOG_ENOMEM, "job larger than the memory budget");
    // jobs run together in one batch, which shares these parameters
    const rbsog_params &h = s->shape;
    if (s->have_shape && (p->b != h.b || p->sigma != h.sigma || p->omega0 != h.omega0 || p->M != h.M ||
                          p->r_c != h.r_c || p->P != h.P || p->precision != h.precision ||
                          p->sampler != h.sampler || p->near_kernel != h.near_kernel || p->r_in != h.r_in))
        return srv_fail(s, RBSOG_EINVAL, "b, sigma, omega0, M, r_c, P, precision, sampler, near_kernel and r_in "
                                         "must match the server's first job");
    if (!s->have_shape) {
        s->shape = *p;
        s->have_shape = true;
    }
    if (job_id) *job_id = j.id;
    s->waiting.push_back(j.id);
    s->jobs[j.id] = std::move(j);
    return RBSOG_OK;
}

rbsog_status rbsog_server_advance(rbsog_server *s, int32_t *n_active, int32_t *n_waiting, int32_t *n_retired) {
    if (!s) return RBSOG_EINVAL;
    int32_t retired = 0;
    // admission: FIFO, by free slots and memory budget
    std::vector<int64_t> add;
    while (!s->waiting.empty()) {
        const int64_t id = s->waiting.front();
        const Job &j = s->jobs[id];
        if ((int64_t)(s->active.size() + add.size()) >= s->max_jobs || s->used + j.footprint > s->budget) break;
        s->used += j.footprint;
        add.push_back(id);
        s->waiting.erase(s->waiting.begin());
    }
    // Retired jobs stay frozen in the batch (their blocks exit at once) until
    // an admission rebuilds it anyway, or they hold most of its particles.
    int64_t live_n = 0;
    for (int64_t id : s->active)
        if (s->jobs[id].status == 1) live_n += s->jobs[id].n;
    if (!add.empty() || (s->frozen_n > 0 && (live_n == 0 || s->frozen_n > live_n))) {
        std::vector<int64_t> keep;
        for (int64_t id : s->active)
            if (s->jobs[id].status == 1) keep.push_back(id);
        rbsog_status st = rebuild(s, keep, add);
        if (st != RBSOG_OK) return st;
        s->frozen_n = 0;
    }
    rbsog_ctx *b = s->batch;
    if (b) {
        int64_t q = 0;
        for (int64_t r : b->remaining_host) q = std::max(q, r);
        q = std::min<int64_t>(q, s->quantum);
        if (q > 0) {
            rbsog_status st = rbsog_batch_step(b, q);
            if (st != RBSOG_OK) return srv_fail(s, st, "step: " + b->err);
            CK_S(s, cudaStreamSynchronize(b->st));
        }
        // retire finished jobs
        for (size_t k = 0; k < s->active.size(); ++k) {
            Job &j = s->jobs[s->active[k]];
            if (j.status != 1 || b->remaining_host[k] != 0) continue;
            j.xo.resize(3 * j.n);
            j.vo.resize(3 * j.n);
            j.fo.resize(3 * j.n);
            rbsog_status st = rbsog_batch_get_state(b, (int32_t)k, j.xo.data(), j.vo.data(), j.fo.data(),
                                                    &j.steps_done);
            if (st != RBSOG_OK) return srv_fail(s, st, "get_state: " + b->err);
            st = rbsog_batch_get_energies(b, (int32_t)k, &j.e);
            if (st != RBSOG_OK) return srv_fail(s, st, "energies: " + b->err);
            j.status = 2;
            s->used -= j.footprint;
            s->frozen_n += j.n;
            ++retired;
        }
    }
    int32_t act = 0;
    for (int64_t id : s->active)
        if (s->jobs[id].status == 1) ++act;
    if (n_active) *n_active = act;
    if (n_waiting) *n_waiting = (int32_t)s->waiting.size();
    if (n_retired) *n_retired = retired;
    return RBSOG_OK;
}

rbsog_status rbsog_server_result(rbsog_server *s, int64_t job_id, int32_t *status, double *x, double *v,
                                 double *f, rbsog_energies *e, int64_t *steps_done) {
    if (!s) return RBSOG_EINVAL;
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return srv_fail(s, RBSOG_EINVAL, "unknown job");
    const Job &j = it->second;
    if (status) *status = j.status;
    if (j.status != 2) return RBSOG_OK;
    if (x) std::memcpy(x, j.xo.data(), sizeof(double) * 3 * j.n);
    if (v) std::memcpy(v, j.vo.data(), sizeof(double) * 3 * j.n);
    if (f) std::memcpy(f, j.fo.data(), sizeof(double) * 3 * j.n);
    if (e) *e = j.e;
    if (steps_done) *steps_done = j.steps_done;
    return RBSOG_OK;
}

rbsog_status rbsog_server_cancel(rbsog_server *s, int64_t job_id) {
    if (!s) return RBSOG_EINVAL;
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return srv_fail(s, RBSOG_EINVAL, "unknown job");
    Job &j = it->second;
    if (j.status == 0) {
        s->waiting.erase(std::find(s->waiting.begin(), s->waiting.end(), job_id));
    } else if (j.status == 1) {
        // freeze the running system at once (its kernels' blocks leave); it
        // leaves the batch at the next rebuild like a finished job
        rbsog_ctx *b = s->batch;
        const auto pos = std::find(s->active.begin(), s->active.end(), job_id);
        const int k = (int)(pos - s->active.begin());
        CK_S(s, cudaSetDevice(b->device));
        CK_S(s, cudaStreamSynchronize(b->st));
        CK_S(s, cudaMemsetAsync(b->d_remaining + k, 0, sizeof(int64_t), b->st));
        CK_S(s, cudaStreamSynchronize(b->st));
        b->remaining_host[k] = 0;
        s->used -= j.footprint;
        s->frozen_n += j.n;
    } else {
        return srv_fail(s, RBSOG_EINVAL, "job already finished or cancelled");
    }
    j.status = 3;
    std::vector<double>().swap(j.q);
    std::vector<double>().swap(j.x);
    std::vector<double>().swap(j.v);
    return RBSOG_OK;
}

rbsog_status rbsog_server_release(rbsog_server *s, int64_t job_id) {
    if (!s) return RBSOG_EINVAL;
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end() || it->second.status < 2) return srv_fail(s, RBSOG_EINVAL, "job not finished");
    s->jobs.erase(it);
    return RBSOG_OK;
}

const char *rbsog_server_last_error(const rbsog_server *s) { return s ? s->err.c_str() : "null server"; }

rbsog_status rbsog_server_destroy(rbsog_server *s) {
    if (!s) return RBSOG_OK;
    if (s->batch) rbsog_destroy(s->batch);
    delete s;
    return RBSOG_OK;
}

}  // extern "C"
