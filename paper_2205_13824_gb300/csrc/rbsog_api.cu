// C ABI of librbsog (declared in include/rbsog.h): context management,
// parameter set-up on the host (SOG solve, S, cell grid, launch shapes), and
// the sequencing of the device kernels for one force evaluation and one
// velocity-Verlet step, replayed from a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/rbsog.h"
#include "rbsog_kernels.cuh"

using namespace rbsog;

namespace {

constexpr double kPi = 3.14159265358979323846;

struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};

}  // namespace

struct rbsog_ctx {
    int64_t n = 0;
    int device = 0;
    cudaStream_t user = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::string err;

    bool have_params = false, have_state = false, force_valid = false;
    rbsog_params p{};
    // solved parameters
    std::vector<double> omega, s;
    double sigma = 0, omega0 = 0, S = 0, V = 0, coef = 0, half_coef_U = 0, U_self = 0, sum_q2 = 0;
    BoxDev box{};
    NearSog nsog{};
    int group = 1, near_cap = 1024, tile_p = 2048, n_ptiles = 1, n_epart = 1, n_kpart = 1;
    int64_t n_sets = 0, n_chains = 0;
    int chain_len = 256;
    int64_t host_cursor = 0;  // k-sets consumed, mirrored on the host

    // device buffers: per-particle (allocated at create)
    double4_32a *posq = nullptr, *vel = nullptr, *force = nullptr, *fnear = nullptr, *sp64 = nullptr;
    uint4 *sp32 = nullptr;
    double *staging = nullptr;        // [n][3]
    int32_t *nbr_sorted = nullptr, *i32_tmp = nullptr;
    CellBuffers cb{};
    double *kpart = nullptr;
    // per-parameter-set
    int4 *kseq = nullptr;
    int64_t *cursor = nullptr, *step_ctr = nullptr;
    double2 *rho_part = nullptr, *rho = nullptr, *epart = nullptr;
    void *ktab = nullptr;
    int32_t *ncell_alloc = nullptr;  // marker of cell arrays size
    int64_t ncell_cap = 0;
    double *energy = nullptr;
    int32_t *err_flag = nullptr;
    int4 *m_tmp = nullptr;
    int32_t *m3_tmp = nullptr;
    int32_t m_tmp_cap = 0;
    // pinned host mirrors
    double *h_energy = nullptr;
    int32_t *h_err = nullptr;
    int64_t *h_i64 = nullptr;

    // graph of one step
    cudaGraphExec_t graph = nullptr;

    // profiling
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
bool solve_sigma(double b, double rc, double &sigma, double &w0) {
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

void build_near_sog(rbsog_ctx *c) {
    NearSog &ns = c->nsog;
    std::memset(&ns, 0, sizeof ns);
    const int M = c->p.M;
    const double rc = c->p.r_c;
    int nd = 0;
    while (nd <= M && c->s[nd] < 2.0 * rc) ++nd;
    ns.n_direct = nd;
    for (int l = 0; l < nd; ++l) {
        ns.omega[l] = c->omega[l];
        ns.inv_s2[l] = 1.0 / (c->s[l] * c->s[l]);
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
            for (int l = M; l >= nd; --l) A[n] += c->omega[l] * std::pow(c->s[l], -2.0 * n);
        }
        const double xmax = rc * rc / (c->s[nd] * c->s[nd]);
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

FarArgs far_args(rbsog_ctx *c, const int4 *m_explicit, int32_t P) {
    FarArgs a{};
    a.n = c->n;
    a.P = P;
    for (int d = 0; d < 3; ++d) a.L[d] = c->p.L[d];
    a.coef = -c->p.coulomb_prefactor * std::pow(kPi, 1.5) * c->S / ((double)P * c->V);
    a.kseq = c->kseq;
    a.cursor = c->cursor;
    a.m_explicit = m_explicit;
    a.tile_p = c->tile_p;
    a.n_ptiles = c->n_ptiles;
    return a;
}

MdArgs md_args(rbsog_ctx *c) {
    MdArgs a{};
    a.n = c->n;
    a.dt = c->p.dt;
    a.mass = c->p.mass;
    a.inv_mass = 1.0 / c->p.mass;
    for (int d = 0; d < 3; ++d) a.L[d] = c->p.L[d];
    a.T0 = c->p.T_target;
    a.tau = c->p.tau_T;
    a.n_epart = c->n_epart;
    a.n_kpart = c->n_kpart;
    a.P = c->p.P;
    a.half_coef_U = c->p.coulomb_prefactor * std::pow(kPi, 1.5) * c->S / (2.0 * c->p.P * c->V);
    a.U_self = c->U_self;
    return a;
}

// Cell list + near field + far field for the current positions; total force
// into c->force (caller order).  m_explicit: explicit k-set or null.
rbsog_status enqueue_forces(rbsog_ctx *ctx, const int4 *m_explicit, int32_t *nbr_sorted) {
    const Prof *pf = prof_of(ctx);
    const int prec = ctx->p.precision;
    CK(launch_build_cells(ctx->n, ctx->posq, ctx->box, ctx->cb, prec, ctx->sp64, ctx->sp32,
                          ctx->err_flag, ctx->st, pf));
    CK(launch_near(prec, ctx->box, ctx->nsog, ctx->group, ctx->near_cap, ctx->cb.start, ctx->sp64, ctx->sp32,
                   ctx->fnear, ctx->epart, nbr_sorted, ctx->st, pf));
    const FarArgs fa = far_args(ctx, m_explicit, ctx->p.P);
    CK(launch_rho_sweep(prec, fa, ctx->sp64, ctx->sp32, ctx->rho_part, ctx->st, pf));
    CK(launch_rho_combine(prec, fa, ctx->rho_part, ctx->rho, ctx->ktab, ctx->st, pf));
    CK(launch_far_scatter(prec, fa, ctx->sp64, ctx->sp32, ctx->ktab, ctx->fnear, ctx->cb.perm,
                          ctx->force, ctx->err_flag, ctx->st, pf));
    return RBSOG_OK;
}

rbsog_status enqueue_step(rbsog_ctx *ctx) {
    const Prof *pf = prof_of(ctx);
    const MdArgs ma = md_args(ctx);
    CK(launch_kick_drift(ma, ctx->posq, ctx->vel, ctx->force, ctx->st, pf));
    rbsog_status s = enqueue_forces(ctx, nullptr, nullptr);
    if (s != RBSOG_OK) return s;
    CK(launch_kick(ma, ctx->vel, ctx->force, ctx->kpart, ctx->st, pf));
    CK(launch_finalize(ma, ctx->epart, ctx->rho, ctx->kpart, 1, ctx->energy, ctx->cursor, 1,
                       ctx->step_ctr, ctx->st, pf));
    if (ctx->p.tau_T > 0.0) CK(launch_rescale(ma, ctx->vel, ctx->energy, ctx->st, pf));
    return RBSOG_OK;
}

void drop_graph(rbsog_ctx *c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
}

rbsog_status check_flags(rbsog_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->h_err, ctx->err_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const int32_t f = *ctx->h_err;
    if (f) {
        CK(cudaMemsetAsync(ctx->err_flag, 0, sizeof(int32_t), ctx->st));
        if (f & 1) return fail(ctx, RBSOG_ENUMERIC, "non-finite force produced on the device");
        if (f & 2) return fail(ctx, RBSOG_ETIMEOUT, "a sampler chain hit its iteration cap");
        return fail(ctx, RBSOG_ECUDA, "device error flag %d", f);
    }
    return RBSOG_OK;
}

}  // namespace

extern "C" {

rbsog_status rbsog_create(rbsog_ctx **out, int64_t n, int device, void *stream) {
    if (!out) return RBSOG_EINVAL;
    *out = nullptr;
    if (n < 2 || n > (int64_t)INT32_MAX / 2) return RBSOG_EINVAL;
    rbsog_ctx *ctx = new (std::nothrow) rbsog_ctx();
    if (!ctx) return RBSOG_ENOMEM;
    ctx->n = n;
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
    if (cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return bail(RBSOG_ECUDA);
    bool ok = dalloc(&ctx->posq, n) == cudaSuccess && dalloc(&ctx->vel, n) == cudaSuccess &&
              dalloc(&ctx->force, n) == cudaSuccess && dalloc(&ctx->fnear, n) == cudaSuccess &&
              dalloc(&ctx->sp64, n) == cudaSuccess && dalloc(&ctx->sp32, n) == cudaSuccess &&
              dalloc(&ctx->staging, 3 * n) == cudaSuccess && dalloc(&ctx->nbr_sorted, n) == cudaSuccess &&
              dalloc(&ctx->i32_tmp, n) == cudaSuccess && dalloc(&ctx->cb.cell_of, n) == cudaSuccess &&
              dalloc(&ctx->cb.slot, n) == cudaSuccess && dalloc(&ctx->cb.perm_raw, n) == cudaSuccess &&
              dalloc(&ctx->cb.perm, n) == cudaSuccess &&
              dalloc(&ctx->kpart, (size_t)kinetic_num_blocks(n)) == cudaSuccess &&
              dalloc(&ctx->cursor, 1) == cudaSuccess && dalloc(&ctx->step_ctr, 1) == cudaSuccess &&
              dalloc(&ctx->energy, kNumEnergy) == cudaSuccess && dalloc(&ctx->err_flag, 1) == cudaSuccess;
    if (!ok) return bail(RBSOG_ENOMEM);
    if (cudaMallocHost((void **)&ctx->h_energy, sizeof(double) * kNumEnergy) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_err, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_i64, sizeof(int64_t)) != cudaSuccess)
        return bail(RBSOG_ENOMEM);
    cudaMemsetAsync(ctx->vel, 0, sizeof(double4_32a) * n, ctx->st);
    cudaMemsetAsync(ctx->force, 0, sizeof(double4_32a) * n, ctx->st);
    cudaMemsetAsync(ctx->energy, 0, sizeof(double) * kNumEnergy, ctx->st);
    cudaMemsetAsync(ctx->err_flag, 0, sizeof(int32_t), ctx->st);
    cudaMemsetAsync(ctx->cursor, 0, sizeof(int64_t), ctx->st);
    cudaMemsetAsync(ctx->step_ctr, 0, sizeof(int64_t), ctx->st);
    if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return bail(RBSOG_ECUDA);
    ctx->n_kpart = kinetic_num_blocks(n);
    *out = ctx;
    return RBSOG_OK;
}

rbsog_status rbsog_set_params(rbsog_ctx *ctx, const rbsog_params *pp) {
    if (!ctx || !pp) return RBSOG_EINVAL;
    rbsog_params p = *pp;
    if (!(p.b > 1.0)) return fail(ctx, RBSOG_EINVAL, "b must be > 1");
    if (p.M < 0 || p.M >= kMaxGauss) return fail(ctx, RBSOG_EINVAL, "M must be in [0, %d]", kMaxGauss - 1);
    if (p.P < 1) return fail(ctx, RBSOG_EINVAL, "P must be >= 1");
    if (p.n_ksets < 1) return fail(ctx, RBSOG_EINVAL, "n_ksets must be >= 1");
    if (!(p.r_c > 0.0)) return fail(ctx, RBSOG_EINVAL, "r_c must be > 0");
    if (!(p.mass > 0.0)) return fail(ctx, RBSOG_EINVAL, "mass must be > 0");
    if (p.precision != RBSOG_FP64 && p.precision != RBSOG_FP32C)
        return fail(ctx, RBSOG_EINVAL, "unknown precision %d", p.precision);
    if (p.chain_len < 0) return fail(ctx, RBSOG_EINVAL, "chain_len must be >= 0");
    if (p.wca_sigma < 0.0) return fail(ctx, RBSOG_EINVAL, "wca_sigma must be >= 0");
    int nc[3];
    for (int d = 0; d < 3; ++d) {
        if (!(p.L[d] > 0.0)) return fail(ctx, RBSOG_EINVAL, "box edges must be > 0");
        if (!(p.r_c < 0.5 * p.L[d])) return fail(ctx, RBSOG_EINVAL, "r_c must be < L/2");
        nc[d] = (int)std::floor(p.L[d] / p.r_c);
        if (nc[d] < 3) return fail(ctx, RBSOG_EINVAL, "need at least 3 cells per side (L/r_c >= 3)");
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    if (ncell > (int64_t)INT32_MAX / 2) return fail(ctx, RBSOG_EINVAL, "cell grid too large");

    // --- SOG (Eqs. 2.9-2.11)
    double sigma = p.sigma, w0 = p.omega0;
    if (!(sigma > 0.0)) {
        if (!solve_sigma(p.b, p.r_c, sigma, w0))
            return fail(ctx, RBSOG_EINVAL, "no C0/C1 root for b=%g r_c=%g", p.b, p.r_c);
    } else if (!(w0 > 0.0)) {
        w0 = c0_weight(p.b, sigma, p.r_c);
    }
    if (!(w0 > 0.0) || !std::isfinite(w0)) return fail(ctx, RBSOG_EINVAL, "invalid omega0");
    std::vector<double> w, s;
    bsa_coeffs(p.b, sigma, p.M, w, s);
    w[0] = w0;
    double S = 0.0;
    for (int l = p.M; l >= 0; --l) {
        const double prod = theta_sum(s[l], p.L[0]) * theta_sum(s[l], p.L[1]) * theta_sum(s[l], p.L[2]);
        S += w[l] * s[l] * s[l] * s[l] * (prod - 1.0);
    }

    drop_graph(ctx);
    ctx->p = p;
    ctx->omega = w;
    ctx->s = s;
    ctx->sigma = sigma;
    ctx->omega0 = w0;
    ctx->S = S;
    ctx->V = p.L[0] * p.L[1] * p.L[2];
    double wsum = 0.0;
    for (int l = 0; l <= p.M; ++l) wsum += w[l];
    ctx->U_self = 0.5 * wsum * ctx->sum_q2 * p.coulomb_prefactor;

    BoxDev &b = ctx->box;
    std::memset(&b, 0, sizeof b);
    for (int d = 0; d < 3; ++d) {
        b.L[d] = p.L[d];
        b.nc[d] = nc[d];
        b.h[d] = p.L[d] / (double)nc[d];
        b.L_f[d] = (float)p.L[d];
        b.fix_scale[d] = (float)(p.L[d] / 4294967296.0);
    }
    b.ncell = (int32_t)ncell;
    b.rc2 = p.r_c * p.r_c;
    b.lB = p.coulomb_prefactor;
    b.wca_s2 = p.wca_sigma * p.wca_sigma;
    b.wca_rc2 = p.wca_sigma > 0.0 ? std::pow(2.0, 1.0 / 3.0) * b.wca_s2 : 0.0;
    b.wca_eps = p.wca_eps;
    b.rc2_f = (float)b.rc2;
    b.lB_f = (float)b.lB;
    b.wca_s2_f = (float)b.wca_s2;
    b.wca_rc2_f = (float)b.wca_rc2;
    b.wca_eps_f = (float)b.wca_eps;
    build_near_sog(ctx);

    // near field: one thread per home particle, ~110 home particles per block;
    // the staging chunk covers the mean occupancy of the 9 (group + 2) staged
    // cells with 30% head-room (denser regions are processed in chunks)
    const double per_cell = (double)ctx->n / (double)ncell;
    int g = (int)std::lround(120.0 / std::max(per_cell, 1e-3));
    g = std::max(1, std::min(g, std::min(16, nc[0] - 2)));
    ctx->group = g;
    ctx->n_epart = near_num_partials(b, g);
    {
        const double est = 9.0 * (g + 2) * per_cell * 1.15 + 64.0;
        const int cap_max = p.precision == RBSOG_FP64 ? 2048 : 4096;
        ctx->near_cap = std::min(cap_max, std::max(256, ((int)std::ceil(est) + 127) / 128 * 128));
    }

    const int nkt = (p.P + 31) / 32;
    int tp = 2048;
    while (tp > 128 && (double)((ctx->n + tp - 1) / tp) * nkt < 152.0 * 8 * 3) tp /= 2;
    ctx->tile_p = tp;
    ctx->n_ptiles = far_num_ptiles(ctx->n, tp);

    ctx->chain_len = p.chain_len > 0 ? p.chain_len : 256;
    ctx->n_sets = p.n_ksets;
    const int64_t total = p.n_ksets * (int64_t)p.P;
    ctx->n_chains = (total + ctx->chain_len - 1) / ctx->chain_len;

    CK(cudaSetDevice(ctx->device));
    CK(dalloc(&ctx->kseq, (size_t)(ctx->n_chains * ctx->chain_len)));
    CK(dalloc(&ctx->rho_part, (size_t)p.P * ctx->n_ptiles));
    CK(dalloc(&ctx->rho, (size_t)p.P));
    CK(dalloc((unsigned char **)&ctx->ktab, ktab_bytes(p.precision, p.P)));
    CK(dalloc(&ctx->epart, (size_t)ctx->n_epart));
    CK(dalloc(&ctx->cb.count, (size_t)ncell));
    CK(dalloc(&ctx->cb.start, (size_t)ncell + 1));
    CK(dalloc(&ctx->cb.tile_sum, (size_t)cell_scan_tiles((int)ncell)));
    CK(dalloc(&ctx->m_tmp, (size_t)p.P));
    CK(dalloc(&ctx->m3_tmp, (size_t)p.P * 3));
    ctx->m_tmp_cap = p.P;
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    CK(cudaMemsetAsync(ctx->cb.count, 0, sizeof(int32_t) * ncell, ctx->st));
    CK(cudaMemsetAsync(ctx->cursor, 0, sizeof(int64_t), ctx->st));
    CK(cudaMemsetAsync(ctx->step_ctr, 0, sizeof(int64_t), ctx->st));
    CK(cudaMemsetAsync(ctx->err_flag, 0, sizeof(int32_t), ctx->st));
    ctx->host_cursor = 0;

    SamplerDev sp{};
    sp.M = p.M;
    for (int l = 0; l <= p.M; ++l) {
        sp.omega[l] = w[l];
        sp.s[l] = s[l];
    }
    for (int d = 0; d < 3; ++d) sp.L[d] = p.L[d];
    sp.seed = p.seed;
    sp.n_chains = ctx->n_chains;
    sp.chain_len = ctx->chain_len;
    CK(launch_mh_sampler(sp, ctx->kseq, ctx->err_flag, ctx->st, prof_of(ctx)));
    rbsog_status fs = check_flags(ctx);
    if (fs != RBSOG_OK) return fs;
    ctx->have_params = true;
    ctx->force_valid = false;
    return leave(ctx);
}

rbsog_status rbsog_get_info(const rbsog_ctx *ctx, rbsog_info *info, double *omega, double *s) {
    if (!ctx || !info) return RBSOG_EINVAL;
    if (!ctx->have_params) return RBSOG_ESTATE;
    info->sigma = ctx->sigma;
    info->omega0 = ctx->omega0;
    info->S = ctx->S;
    info->M = ctx->p.M;
    for (int d = 0; d < 3; ++d) info->ncell[d] = ctx->box.nc[d];
    info->n_chains = ctx->n_chains;
    info->chain_len = ctx->chain_len;
    if (omega) std::memcpy(omega, ctx->omega.data(), sizeof(double) * (ctx->p.M + 1));
    if (s) std::memcpy(s, ctx->s.data(), sizeof(double) * (ctx->p.M + 1));
    return RBSOG_OK;
}

rbsog_status rbsog_set_state(rbsog_ctx *ctx, const double *q, const double *x, const double *v) {
    if (!ctx || !q || !x) return RBSOG_EINVAL;
    if (!ctx->have_params) return fail(ctx, RBSOG_ESTATE, "set_params must come first");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    std::vector<double> hq((size_t)ctx->n);
    CK(cudaMemcpyAsync(hq.data(), q, sizeof(double) * ctx->n, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    double sq = 0.0, sa = 0.0, s2 = 0.0;
    for (double qi : hq) {
        if (!std::isfinite(qi)) return fail(ctx, RBSOG_EINVAL, "non-finite charge");
        sq += qi;
        sa += std::fabs(qi);
        s2 += qi * qi;
    }
    if (std::fabs(sq) > 1e-12 * sa) return fail(ctx, RBSOG_EINVAL, "charges are not neutral (sum %.3e)", sq);
    ctx->sum_q2 = s2;
    double wsum = 0.0;
    for (int l = 0; l <= ctx->p.M; ++l) wsum += ctx->omega[l];
    ctx->U_self = 0.5 * wsum * s2 * ctx->p.coulomb_prefactor;

    double *qd = nullptr;
    CK(cudaMallocAsync((void **)&qd, sizeof(double) * ctx->n, ctx->st));
    CK(cudaMemcpyAsync(qd, q, sizeof(double) * ctx->n, cudaMemcpyDefault, ctx->st));
    CK(cudaMemcpyAsync(ctx->staging, x, sizeof(double) * 3 * ctx->n, cudaMemcpyDefault, ctx->st));
    CK(launch_pack(ctx->n, ctx->staging, qd, ctx->posq, 1, ctx->p.L, ctx->st));
    if (v) {
        CK(cudaMemcpyAsync(ctx->staging, v, sizeof(double) * 3 * ctx->n, cudaMemcpyDefault, ctx->st));
        CK(launch_pack(ctx->n, ctx->staging, nullptr, ctx->vel, 0, ctx->p.L, ctx->st));
    } else {
        CK(cudaMemsetAsync(ctx->vel, 0, sizeof(double4_32a) * ctx->n, ctx->st));
    }
    CK(cudaFreeAsync(qd, ctx->st));
    CK(cudaMemsetAsync(ctx->step_ctr, 0, sizeof(int64_t), ctx->st));
    drop_graph(ctx);
    ctx->have_state = true;
    ctx->force_valid = false;
    return leave(ctx);
}

rbsog_status rbsog_compute_forces(rbsog_ctx *ctx, const int32_t *m_kset, double *f_out,
                                  rbsog_energies *e_out) {
    if (!ctx) return RBSOG_EINVAL;
    if (!ctx->have_params || !ctx->have_state) return fail(ctx, RBSOG_ESTATE, "params and state required");
    if (!m_kset && ctx->host_cursor >= ctx->n_sets)
        return fail(ctx, RBSOG_EINVAL, "pre-sampled k-sequence exhausted");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const int4 *mex = nullptr;
    if (m_kset) {
        CK(cudaMemcpyAsync(ctx->m3_tmp, m_kset, sizeof(int32_t) * 3 * ctx->p.P, cudaMemcpyDefault, ctx->st));
        CK(launch_m_to_int4(ctx->p.P, ctx->m3_tmp, ctx->m_tmp, ctx->st));
        mex = ctx->m_tmp;
    }
    es = enqueue_forces(ctx, mex, nullptr);
    if (es != RBSOG_OK) return es;
    const MdArgs ma = md_args(ctx);
    CK(launch_finalize(ma, ctx->epart, ctx->rho, ctx->kpart, 0, ctx->energy, ctx->cursor,
                       m_kset ? 0 : 1, nullptr, ctx->st, prof_of(ctx)));
    if (!m_kset) ctx->host_cursor += 1;
    ctx->force_valid = true;
    if (f_out) {
        CK(launch_unpack(ctx->n, ctx->force, ctx->staging, ctx->st));
        CK(cudaMemcpyAsync(f_out, ctx->staging, sizeof(double) * 3 * ctx->n, cudaMemcpyDefault, ctx->st));
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
    }
    return leave(ctx);
}

rbsog_status rbsog_step(rbsog_ctx *ctx, int64_t nsteps) {
    if (!ctx) return RBSOG_EINVAL;
    if (nsteps < 0) return fail(ctx, RBSOG_EINVAL, "nsteps must be >= 0");
    if (!ctx->have_params || !ctx->have_state) return fail(ctx, RBSOG_ESTATE, "params and state required");
    const int64_t need = nsteps + (ctx->force_valid ? 0 : 1);
    if (ctx->host_cursor + need > ctx->n_sets)
        return fail(ctx, RBSOG_EINVAL, "pre-sampled k-sequence too short (%lld sets left, %lld needed)",
                    (long long)(ctx->n_sets - ctx->host_cursor), (long long)need);
    if (nsteps == 0 && ctx->force_valid) return RBSOG_OK;
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    if (!ctx->force_valid) {
        es = enqueue_forces(ctx, nullptr, nullptr);
        if (es != RBSOG_OK) return es;
        const MdArgs ma = md_args(ctx);
        CK(launch_finalize(ma, ctx->epart, ctx->rho, ctx->kpart, 0, ctx->energy, ctx->cursor, 1,
                           nullptr, ctx->st, prof_of(ctx)));
        ctx->host_cursor += 1;
        ctx->force_valid = true;
    }
    if (ctx->profiling) {
        for (int64_t t = 0; t < nsteps; ++t) {
            es = enqueue_step(ctx);
            if (es != RBSOG_OK) return es;
        }
    } else if (nsteps > 0) {
        if (!ctx->graph) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
            es = enqueue_step(ctx);
            cudaError_t ce = cudaStreamEndCapture(ctx->st, &g);
            if (es != RBSOG_OK) {
                if (g) cudaGraphDestroy(g);
                return es;
            }
            if (ce != cudaSuccess) return fail(ctx, RBSOG_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&ctx->graph, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return fail(ctx, RBSOG_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        }
        for (int64_t t = 0; t < nsteps; ++t) CK(cudaGraphLaunch(ctx->graph, ctx->st));
    }
    ctx->host_cursor += nsteps;
    return leave(ctx);
}

rbsog_status rbsog_get_state(rbsog_ctx *ctx, double *x, double *v, double *f, int64_t *step) {
    if (!ctx) return RBSOG_EINVAL;
    if (!ctx->have_state) return fail(ctx, RBSOG_ESTATE, "no state");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const size_t bytes = sizeof(double) * 3 * ctx->n;
    if (x) {
        CK(launch_unpack(ctx->n, ctx->posq, ctx->staging, ctx->st));
        CK(cudaMemcpyAsync(x, ctx->staging, bytes, cudaMemcpyDefault, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    if (v) {
        CK(launch_unpack(ctx->n, ctx->vel, ctx->staging, ctx->st));
        CK(cudaMemcpyAsync(v, ctx->staging, bytes, cudaMemcpyDefault, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    if (f) {
        CK(launch_unpack(ctx->n, ctx->force, ctx->staging, ctx->st));
        CK(cudaMemcpyAsync(f, ctx->staging, bytes, cudaMemcpyDefault, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    if (step) {
        CK(cudaMemcpyAsync(ctx->h_i64, ctx->step_ctr, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        *step = *ctx->h_i64;
    }
    es = check_flags(ctx);
    if (es != RBSOG_OK) return es;
    return leave(ctx);
}

rbsog_status rbsog_get_cursor(const rbsog_ctx *ctx, int64_t *kset_cursor) {
    if (!ctx || !kset_cursor) return RBSOG_EINVAL;
    *kset_cursor = ctx->host_cursor;
    return RBSOG_OK;
}

rbsog_status rbsog_restore(rbsog_ctx *ctx, const double *f, int64_t kset_cursor, int64_t step) {
    if (!ctx || !f) return RBSOG_EINVAL;
    if (!ctx->have_state) return fail(ctx, RBSOG_ESTATE, "set_state must come first");
    if (kset_cursor < 0 || kset_cursor > ctx->n_sets || step < 0)
        return fail(ctx, RBSOG_EINVAL, "cursor %lld outside [0, %lld]", (long long)kset_cursor,
                    (long long)ctx->n_sets);
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    CK(cudaMemcpyAsync(ctx->staging, f, sizeof(double) * 3 * ctx->n, cudaMemcpyDefault, ctx->st));
    CK(launch_pack(ctx->n, ctx->staging, nullptr, ctx->force, 0, ctx->p.L, ctx->st));
    *ctx->h_i64 = kset_cursor;
    CK(cudaMemcpyAsync(ctx->cursor, ctx->h_i64, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *ctx->h_i64 = step;
    CK(cudaMemcpyAsync(ctx->step_ctr, ctx->h_i64, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->host_cursor = kset_cursor;
    ctx->force_valid = true;
    return leave(ctx);
}

rbsog_status rbsog_get_energies(rbsog_ctx *ctx, rbsog_energies *e) {
    if (!ctx || !e) return RBSOG_EINVAL;
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    CK(cudaMemcpyAsync(ctx->h_energy, ctx->energy, sizeof(double) * kNumEnergy, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    e->U_near = ctx->h_energy[0];
    e->U_far = ctx->h_energy[1];
    e->U_self = ctx->h_energy[2];
    e->U_wca = ctx->h_energy[3];
    e->K = ctx->h_energy[4];
    e->T = ctx->h_energy[5];
    return leave(ctx);
}

rbsog_status rbsog_get_kseq(rbsog_ctx *ctx, int64_t set0, int64_t nsets, int32_t *m_out) {
    if (!ctx || !m_out || set0 < 0 || nsets < 0) return RBSOG_EINVAL;
    if (!ctx->have_params) return fail(ctx, RBSOG_ESTATE, "no params");
    if (set0 + nsets > ctx->n_sets) return fail(ctx, RBSOG_EINVAL, "k-set range beyond the sequence");
    const int64_t cnt = nsets * ctx->p.P;
    std::vector<int4> tmp((size_t)cnt);
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    CK(cudaMemcpyAsync(tmp.data(), ctx->kseq + set0 * ctx->p.P, sizeof(int4) * cnt, cudaMemcpyDeviceToHost, ctx->st));
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

rbsog_status rbsog_rho(rbsog_ctx *ctx, const int32_t *m, int32_t P, double *rho_out) {
    if (!ctx || !m || !rho_out || P < 1) return RBSOG_EINVAL;
    if (!ctx->have_params || !ctx->have_state) return fail(ctx, RBSOG_ESTATE, "params and state required");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    int32_t *m3 = nullptr;
    int4 *m4 = nullptr;
    double2 *part = nullptr, *rho = nullptr;
    void *kt = nullptr;
    CK(cudaMallocAsync((void **)&m3, sizeof(int32_t) * 3 * P, ctx->st));
    CK(cudaMallocAsync((void **)&m4, sizeof(int4) * P, ctx->st));
    CK(cudaMallocAsync((void **)&part, sizeof(double2) * (size_t)P * ctx->n_ptiles, ctx->st));
    CK(cudaMallocAsync((void **)&rho, sizeof(double2) * P, ctx->st));
    CK(cudaMallocAsync(&kt, ktab_bytes(ctx->p.precision, P), ctx->st));
    CK(cudaMemcpyAsync(m3, m, sizeof(int32_t) * 3 * P, cudaMemcpyDefault, ctx->st));
    CK(launch_m_to_int4(P, m3, m4, ctx->st));
    CK(launch_build_cells(ctx->n, ctx->posq, ctx->box, ctx->cb, ctx->p.precision, ctx->sp64, ctx->sp32,
                          ctx->err_flag, ctx->st, prof_of(ctx)));
    const FarArgs fa = far_args(ctx, m4, P);
    CK(launch_rho_sweep(ctx->p.precision, fa, ctx->sp64, ctx->sp32, part, ctx->st, prof_of(ctx)));
    CK(launch_rho_combine(ctx->p.precision, fa, part, rho, kt, ctx->st, prof_of(ctx)));
    CK(cudaMemcpyAsync(rho_out, rho, sizeof(double2) * P, cudaMemcpyDefault, ctx->st));
    CK(cudaFreeAsync(m3, ctx->st));
    CK(cudaFreeAsync(m4, ctx->st));
    CK(cudaFreeAsync(part, ctx->st));
    CK(cudaFreeAsync(rho, ctx->st));
    CK(cudaFreeAsync(kt, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
}

rbsog_status rbsog_get_cells(rbsog_ctx *ctx, int32_t *cell_start, int32_t *perm, int32_t *nbr) {
    if (!ctx) return RBSOG_EINVAL;
    if (!ctx->have_params || !ctx->have_state) return fail(ctx, RBSOG_ESTATE, "params and state required");
    rbsog_status es = enter(ctx);
    if (es != RBSOG_OK) return es;
    const Prof *pf = prof_of(ctx);
    CK(launch_build_cells(ctx->n, ctx->posq, ctx->box, ctx->cb, ctx->p.precision, ctx->sp64, ctx->sp32,
                          ctx->err_flag, ctx->st, pf));
    if (nbr) {
        CK(launch_near(ctx->p.precision, ctx->box, ctx->nsog, ctx->group, ctx->near_cap, ctx->cb.start, ctx->sp64,
                       ctx->sp32, ctx->fnear, ctx->epart, ctx->nbr_sorted, ctx->st, pf));
        CK(launch_unsort_i32(ctx->n, ctx->cb.perm, ctx->nbr_sorted, ctx->i32_tmp, ctx->st));
        CK(cudaMemcpyAsync(nbr, ctx->i32_tmp, sizeof(int32_t) * ctx->n, cudaMemcpyDefault, ctx->st));
    }
    if (cell_start)
        CK(cudaMemcpyAsync(cell_start, ctx->cb.start, sizeof(int32_t) * (ctx->box.ncell + 1), cudaMemcpyDefault, ctx->st));
    if (perm) CK(cudaMemcpyAsync(perm, ctx->cb.perm, sizeof(int32_t) * ctx->n, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return leave(ctx);
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

rbsog_status rbsog_get_profile(rbsog_ctx *ctx, int32_t cap, char (*names)[32], int64_t *launches,
                               double *ms, int32_t *count) {
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
    dfree(&ctx->nbr_sorted);
    dfree(&ctx->i32_tmp);
    dfree(&ctx->cb.cell_of);
    dfree(&ctx->cb.slot);
    dfree(&ctx->cb.count);
    dfree(&ctx->cb.start);
    dfree(&ctx->cb.tile_sum);
    dfree(&ctx->cb.perm_raw);
    dfree(&ctx->cb.perm);
    dfree(&ctx->kpart);
    dfree(&ctx->kseq);
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
    if (ctx->h_energy) cudaFreeHost(ctx->h_energy);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->h_i64) cudaFreeHost(ctx->h_i64);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->st) cudaStreamDestroy(ctx->st);
    delete ctx;
    return RBSOG_OK;
}

}  // extern "C"
