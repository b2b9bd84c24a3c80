// Internal declarations shared by the translation units of librbsog: the
// by-value parameter blocks handed to kernels and the host-side launchers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

namespace rbsog {

constexpr int kMaxGauss = 128;   // M + 1 <= kMaxGauss
constexpr int kMaxTaylor = 16;   // terms of the folded wide-Gaussian series
constexpr int kTabN = 64;        // intervals of the FP32 Gaussian-sum tables
constexpr int kLTabN = 128;      // intervals of the neighbour-list path's combined table

// Sum-of-Gaussians near kernel in the form the pair kernels evaluate.
// Gaussians l < n_direct are evaluated with exp; the wide ones (s_l >= 2 r_c)
// are folded into Taylor series in r^2 about 0 with coefficients
//   A[n] = sum_{l >= n_direct} w_l s_l^{-2n},
// so that sum_{wide} w_l e^{-r^2/s_l^2}       = sum_n (-r^2)^n / n! A[n]
// and     sum_{wide} w_l/s_l^2 e^{-r^2/s_l^2} = sum_n (-r^2)^n / n! A[n+1].
struct NearSog {
    int32_t n_direct;
    int32_t n_taylor;              // Taylor terms for FP64 (truncation < 1e-19 relative)
    int32_t n_taylor_f;            // Taylor terms for FP32 (truncation < 1e-10 relative)
    double omega[kMaxGauss];       // w_l, l < n_direct
    double inv_s2[kMaxGauss];      // 1 / s_l^2, l < n_direct
    double tay_f[kMaxTaylor];      // A[n] / n! with sign (-1)^n folded in
    double tay_g[kMaxTaylor];      // A[n+1] / n! with sign (-1)^n folded in
    float omega_f[kMaxGauss];
    float omega_s2_f[kMaxGauss];   // w_l / s_l^2
    float inv_s2_log2e_f[kMaxGauss];  // log2(e) / s_l^2 (argument of ex2)
    float tay_f_f[kMaxTaylor];
    float tay_g_f[kMaxTaylor];
    // FP32 piecewise-cubic tables of the whole Gaussian sums on u = r^2 in
    // [0, r_c^2]: interval k covers u = (k + s) r_c^2 / kTabN, s in [0, 1),
    // and holds the monomial coefficients (c0, c1, c2, c3) in s of
    // G(u) = sum_l w_l / s_l^2 e^{-u/s_l^2} (tab_g) and F_M (tab_f)
    float4 tab_g[kTabN];
    float4 tab_f[kTabN];
    float tab_scale;               // kTabN / r_c^2
    float tab_err;                 // max abs error of the FP32 tables, relative to G(0) / F(0)
    // Combined table of the neighbour-list path (one 16-byte entry per
    // interval, held on the device): interval k of kLTabN covers
    // u = (k + s) h, h = r_c^2 / kLTabN, and holds (g0, g1, g2, F(k h)) with
    // G(u) ~ g0 + g1 s + g2 s^2 and, since dF/du = -G,
    // F(u) ~ F(k h) - h (g0 s + g1 s^2 / 2 + g2 s^3 / 3).
    float ltab_scale;              // kLTabN / r_c^2
    float ltab_h;                  // r_c^2 / kLTabN
    float ltab_err;                // max abs error of G and F from it, relative to G(0) / F(0)
};

// Box, cell grid and pair constants.
struct BoxDev {
    double L[3];
    double h[3];          // cell sides L_d / nc_d
    int32_t nc[3];        // cells per side
    int32_t ncell;
    double rc2;           // r_c * r_c
    double lB;            // Coulomb prefactor
    double wca_s2;        // wca_sigma^2 (0: off)
    double wca_rc2;       // 2^(1/3) wca_sigma^2
    double wca_eps;
    float L_f[3];
    float fix_scale[3];   // L_d / 2^32: fixed-point unit of the FP32C positions
    double fix_inv[3];    // 2^32 / L_d: X_d = trunc(x_d * fix_inv[d]), clamped to [0, 2^32 - 1]
    double kfac[3];       // 2 pi / L_d: k_d = kfac[d] m_d
    float cell_fix[3];    // 2^32 / nc_d: fixed-point length of one cell side
    float rl2_f;          // neighbour lists: (r_c + skin)^2, with a margin above FP32 rounding
    float disp2_f;        // neighbour lists: (skin / 2)^2, with a margin below it
    double inv_h[3];      // nc_d / L_d: cell of x is floor(x_d * inv_h[d]) (clamped)
    float h_f[3];         // h_d in FP32
    // FP32 copies of the pair constants (no double->float conversion in kernels)
    float rc2_f, lB_f, wca_s2_f, wca_rc2_f, wca_eps_f;
};

// Sampler inputs (Sec. 3.3): full SOG (not folded) in FP64, shared by the
// systems of a batch; per system the box, seed and chain layout.
struct SamplerDev {
    int32_t M;
    double omega[kMaxGauss];
    double s[kMaxGauss];
};
struct SamplerSys {
    double L[3];
    uint64_t seed;
    int64_t chain_off;        // first global chain of this system
    int64_t k_off;            // first int4 of this system's sequence
    int32_t chain_len;
};

// Per-kernel timing hook: when non-null the launcher brackets the launch
// with CUDA events through this callback (name, begin/end).
struct Prof {
    void (*mark)(void *self, const char *name, int begin);
    void *self;
};

struct ProfScope {
    const Prof *p;
    const char *name;
    ProfScope(const Prof *p_, const char *n) : p(p_), name(n) {
        if (p && p->mark) p->mark(p->self, name, 1);
    }
    ~ProfScope() {
        if (p && p->mark) p->mark(p->self, name, 0);
    }
};

// ---- sampler (k_sampler.cu) -------------------------------------------------
// One launch, one thread per chain over all systems (sys sorted by chain_off).
cudaError_t launch_mh_sampler(const SamplerDev &sp, const SamplerSys *sys, int n_sys, int64_t total_chains,
                              int4 *kseq, int32_t *err_flag, cudaStream_t st, const Prof *prof);

// Folded k-sets.  A Metropolis-Hastings chain repeats its state on every
// rejected proposal, so about half of a set's P frequencies equal their
// predecessor.  Every term of the random-batch sums (rho(k), the force, the
// energy) depends only on the frequency, so each run of equal consecutive
// frequencies is evaluated once and weighted by its length: the sums are the
// same up to rounding.  Set s of a system becomes kfold[k_off + s P + t] =
// (m, run length) for t < kcount[kc_off + s], zero entries (weight 0) after.
struct FoldSys {
    int64_t k_off;            // first int4 of the system's sequence
    int64_t kc_off;           // first set count of the system
    int64_t set_off;          // first global set (prefix over the listed systems)
};
cudaError_t launch_fold_kseq(const FoldSys *sys, int n_sys, int64_t total_sets, int32_t P, const int4 *kseq,
                             int4 *kfold, int32_t *kcount, cudaStream_t st);

// ---- per-Gaussian independent sampling (k_pgsample.cu) -------------------------
// The variant sampler of Sec. 3.3: Gaussian l alone, normalised over k != 0,
// is sampled P_l = ceil(P S_l / S) times per set (S_l its share of Eq. 3.16;
// Gaussians with S_l <= 1e-16 S are dropped); a set holds the strata in order
// of l, P_eff = sum_l P_l frequencies, padded to the batch's frequencies per
// set with (1, 0, 0) entries of stratum kPgPad and weight 0.  The k-sequence
// entry's w holds the stratum; the estimator weighs it by
// kw[sys * kKwStride + w] = (S_l / P_l) / (S / P_batch).
constexpr int kPgPad = kMaxGauss;
constexpr int kKwStride = kMaxGauss + 1;
struct PgStratum {
    double thr1;          // P(first non-zero coordinate is x | m != 0)
    double thr2;          // P(it is y | m_x = 0, m != 0)
    int64_t tab_off[3];   // cumulative table of each coordinate in the table array
    int32_t jmax[3];      // its last index
    int32_t l;            // Gaussian index
};
struct PgPlan {
    int32_t P_eff = 0;
    std::vector<int32_t> P_l;             // [M + 1]
    std::vector<double> S_l;              // [M + 1]
    std::vector<PgStratum> strata;        // active Gaussians in order of l
    std::vector<int32_t> slot_stratum;    // [P_eff]: index into strata
    std::vector<double> tables;           // cumulative tables, concatenated
};
// false when a coordinate table would exceed 2^20 entries.
bool pg_plan(const double *omega, const double *s, int M, const double L[3], int P, PgPlan &plan);
// Fills kseq[set * P_batch + eta] for sets [0, n_sets) of one system.
cudaError_t launch_pg_sampler(const PgStratum *strata, const int32_t *slot_stratum, int32_t P_eff, int32_t P_batch,
                              const double *tables, uint64_t seed, int64_t n_sets, int4 *kseq, cudaStream_t st,
                              const Prof *prof);

// ---- batch layout -------------------------------------------------------------
// Every kernel works on a batch of independent systems laid out back to back
// (particles, cells, k-sequences, partial sums).  A single system is a batch
// of one.  Each system's work is decomposed exactly as it would be alone, so
// its results do not depend on the other systems in the batch.
struct SysDesc {
    BoxDev box;
    int64_t p_off, n;          // first particle (global index), particle count
    int64_t c_off;             // first cell (global index)
    int32_t group, nseg_x;     // near field: home cells per block, segments per x-row
    int32_t near_cap;          // near field: staged particles per shared-memory chunk
    int32_t near_split;        // near field (FP64 cell stencil): the warps of a block split the rows
    int32_t e_off, n_epart;    // near-energy partials (one per near-field block)
    int32_t tile_p, n_ptiles;  // rho sweep: particles per tile, tiles
    int64_t rp_off;            // first rho partial (double2 units)
    int64_t k_off;             // first int4 of this system's k-sequence
    int64_t n_sets;            // k-sets sampled
    int64_t kc_off;            // first entry of this system's folded-set counts
    int32_t kp_off, n_kpart;   // kinetic partials (one per particle block)
    double coef;               // -lB pi^{3/2} S / (P V): multiplies q_i k Im(...)
    double half_coef_U;        // lB pi^{3/2} S / (2 P V)
    double U_self;
    double dt, inv_mass, mass, T0, tau;
    double half_dt_inv_mass;   // dt / (2 m): the half kick's factor
    int32_t boundary;          // zero-frequency term: 0 tinfoil, 1 spherical, 2 planar (z)
    int32_t thermostat;        // with tau > 0: 0 Berendsen rescale, 1 Langevin (BAOAB), 2 Nose-Hoover
    double half_dt;            // dt / 2
    double lv_c1, lv_c2;       // Langevin: v <- c1 v + c2 z, c1 = e^{-dt/tau}, c2 = sqrt((1 - c1^2) T0 / m)
    uint64_t lv_seed;          // key of the Langevin noise
    float half_mass_f;         // m / 2 (FP32C kinetic-energy terms)
    double nh_Q;               // Nose-Hoover thermostat mass g T0 tau^2, g = 3N - 3
};

// Work tables map a launch's blocks to (system, local block).
struct BatchView {
    const SysDesc *sys;        // [n_sys], device
    int32_t n_sys;
    int32_t P;                 // frequencies per step, the same for every system
    int64_t n_total, ncell_total;
    const int2 *pblk;          // blocks of kParticleBlock particles
    int32_t n_pblk;
    const int2 *nblk;          // near-field blocks
    int32_t n_nblk;
    const int2 *sblk;          // rho-sweep particle tiles
    int32_t n_sblk;
    const int32_t *cell_sys;   // [ncell_total] system of each cell
    int64_t *cursor;           // [n_sys] k-sets consumed
    int64_t *step;             // [n_sys] completed steps
    const int4 *kseq;          // concatenated k-sequences
    const int4 *kfold;         // folded k-sets (same layout; .w = run length), or null:
    const int32_t *kcount;     //   far-field kernels then read kseq and all P entries
    const int4 *m_explicit;    // explicit k-set for a batch of one, or null
    const int32_t *force_mask; // [n_sys]: only systems with a non-zero entry take the new
                               // forces, energies and k-set (null: all systems)
    int64_t *remaining;        // [n_sys] steps left per system; a system at 0 is frozen
                               // (skipped by every step kernel); null: no budgets
    int32_t max_cap;           // largest near staging chunk of the batch
    int32_t max_tile_p;        // largest rho-sweep tile of the batch
    int32_t list_cap;          // neighbour-list slots per particle (0: no lists)
    int32_t precision;         // 0 FP64, 1 FP32C
    uint4 *lpos;               // [n_total] fixed-point positions in the cell order of the
                               // last list build (neighbour-list path; null otherwise)
    int32_t *linv;             // [n_total] cell-order slot of caller particle i at that build
    const double *kw;          // [n_sys * kKwStride] per-stratum weights of per-Gaussian
                               // sampling (null: the mixture sampler, or an explicit k-set)
    double4_32a *fin_part;     // [n_sys * kFinChunks] finalize: per-chunk energy sums
    unsigned int *fin_count;   // [n_sys] finalize: chunks done (reset by the last one)
};
constexpr int kFinChunks = 16;    // blocks per system in the finalize reduction
constexpr int kParticleBlock = 256;
// FP64 systems below this many particles split the cell-stencil rows over
// the warps of a near-field block (their blocks hold few home particles)
constexpr int64_t kNearSplitMaxN = 131072;

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 64x64->128-bit products with the published multipliers, key bumped by the
// published Weyl constants before every round after the first.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// 53 random bits mapped to [0, 1).
__device__ __forceinline__ double unit53(uint64_t x) {
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}


// X = trunc(x * (2^32 / L)) clamped to [0, 2^32 - 1]: the fixed-point
// coordinate of the FP32C path (one FP64 multiply; the scale comes from the
// host).
__device__ __forceinline__ uint32_t fixed32(double x, double inv) {
    // the round-toward-zero conversion to a 32-bit unsigned integer clamps
    // to [0, 2^32 - 1] (PTX cvt semantics), which is the clamp above
    return __double2uint_rz(x * inv);
}

// x folded into [0, L); L mapped to 0.
__device__ __forceinline__ double fold(double x, double L) {
    double v = x - L * floor(x / L);
    return v >= L ? 0.0 : v;
}

// x < 0 or x >= L (L > 0) decided on the bit patterns with integer compares
// (the order of non-negative doubles is that of their bits): the same
// outcome as the FP64 compares, which are scarce on this GPU; -0.0 stays,
// NaN folds to NaN either way.
__device__ __forceinline__ bool outside(double x, long long Lbits) {
    const long long b = __double_as_longlong(x);
    return b >= Lbits || (b < 0 && b != (long long)0x8000000000000000ull);
}

// Folds only the coordinates that left the box (the division is FP64-pipe
// bound).
__device__ __forceinline__ void fold_into_box(double4_32a &p, const BoxDev &box) {
    if (outside(p.x, __double_as_longlong(box.L[0]))) p.x = fold(p.x, box.L[0]);
    if (outside(p.y, __double_as_longlong(box.L[1]))) p.y = fold(p.y, box.L[1]);
    if (outside(p.z, __double_as_longlong(box.L[2]))) p.z = fold(p.z, box.L[2]);
}

// Caller-order fixed-point position (x, y, z, FP32 charge) of particle i for
// the neighbour-list path, and the test of its displacement since the last
// list build: a particle of system `sys` that moved more than skin / 2 sets
// rebuild[sys] and rebuild[n_sys] (any system).
__device__ __forceinline__ void fixed_pack_check(const SysDesc &d, int sys, int n_sys, const double4_32a &p,
                                                 int64_t i, uint4 *__restrict__ sp32c,
                                                 const uint4 *__restrict__ xref, int32_t *__restrict__ rebuild,
                                                 uint4 *__restrict__ lpos, const int32_t *__restrict__ linv) {
    uint4 o;
    o.x = fixed32(p.x, d.box.fix_inv[0]);
    o.y = fixed32(p.y, d.box.fix_inv[1]);
    o.z = fixed32(p.z, d.box.fix_inv[2]);
    o.w = __float_as_uint((float)p.w);
    sp32c[i] = o;
    if (lpos) lpos[linv[i]] = o;
    const uint4 r = xref[i];
    const float dx = (float)(int32_t)(o.x - r.x) * d.box.fix_scale[0];
    const float dy = (float)(int32_t)(o.y - r.y) * d.box.fix_scale[1];
    const float dz = (float)(int32_t)(o.z - r.z) * d.box.fix_scale[2];
    if (fmaf(dz, dz, fmaf(dy, dy, dx * dx)) > d.box.disp2_f && !rebuild[sys]) {
        rebuild[sys] = 1;
        rebuild[n_sys] = 1;
    }
}

// ---- cell list (k_cells.cu) ---------------------------------------------------
struct CellBuffers {
    int32_t *cell_of;     // [n]   cell id of each particle (global)
    int32_t *slot;        // [n]   arrival slot inside its cell (unordered)
    int32_t *count;       // [ncell] zeroed after every scan
    int32_t *start;       // [ncell + 1]
    int32_t *perm_raw;    // [n]   cell order, unordered inside a cell
    int32_t *perm;        // [n]   cell order, increasing index inside a cell
    int32_t *tile_sum;    // [cell_scan_tiles(ncell)] scan tile totals
    unsigned long long *key;   // [n] in perm_raw order: (fixed-point x << 32) | index
    double4_32a *pack;         // [n] in perm_raw order: particle data in the gathered format
};
int cell_scan_tiles(int64_t ncell);
// precision 0: gather FP64 (x, y, z, q) into sp64; 1: 32-bit fixed point
// positions and FP32 charge into sp32.
// gate (device flag, may be null): when non-null and zero, every kernel of
// the build returns at once (the neighbour-list path rebuilds only on demand).
cudaError_t launch_build_cells(const BatchView &bv, const double4_32a *posq, const CellBuffers &cb,
                               int precision, double4_32a *sp64, uint4 *sp32, cudaStream_t st,
                               const Prof *prof, const int32_t *gate = nullptr);

// ---- near field (k_near.cu) ---------------------------------------------------
// Forces (cell order) into fnear; energy partials (U_near, U_wca), one per
// warp, into epart; neighbour counts (cell order) into nbr when non-null.
// home: target home particles per block (tunable, 120 by default)
void near_layout(const BoxDev &box, int64_t n, int precision, int home, int &group, int &nseg_x, int &cap,
                 int &nblocks, int &npartials);
cudaError_t launch_near(int precision, const BatchView &bv, const NearSog &sog, const int32_t *start,
                        const double4_32a *sp64, const uint4 *sp32, double4_32a *fnear, double2 *epart,
                        int32_t *nbr, cudaStream_t st, const Prof *prof);

// ---- neighbour lists (k_verlet.cu), FP32C ------------------------------------
// Lists: sliced by groups of 32 cell-order positions s of the last build
// (list_perm[s] the caller index, linv its inverse): slot k of s at
// ((s / 32) cap + k) 32 + s % 32, nbr_cnt[s] entries, each the cell-order
// position of a partner; lpos[s] the current fixed-point position of the
// particle at s (written by the builder, then by every kick-drift through
// linv); xref[i] the fixed-point position of caller particle i at that
// build; rebuild[n_sys + 1] flags (per system, any).
size_t list_build_smem(int cap, int list_cap);
cudaError_t launch_fix_pack(const BatchView &bv, const double4_32a *posq, uint4 *sp32c, const uint4 *xref,
                            int32_t *rebuild, cudaStream_t st, const Prof *prof);
// Rebuilds the lists of flagged systems from the cell list (cell-order sp32,
// perm) and clears the flags.  err_flag bit 4: a list exceeded list_cap.
cudaError_t launch_list_build(const BatchView &bv, const int32_t *start, const uint4 *sp32, const int32_t *perm,
                              const int32_t *rebuild, int32_t *nbr_list, int32_t *nbr_cnt, int32_t *list_perm,
                              uint4 *xref, int32_t *err_flag, cudaStream_t st, const Prof *prof);
// Sets the condition of a conditional graph node to the 'any system needs a
// rebuild' flag (captured steps).
cudaError_t launch_rebuild_condition(cudaGraphConditionalHandle h, const int32_t *any, cudaStream_t st);
// Moves one running system's lists between batch layouts (serving engine).
cudaError_t launch_list_move(int64_t n, int64_t old_off, int64_t new_off, int old_cap, int new_cap,
                             const int32_t *old_list, const int32_t *old_cnt, const int32_t *old_perm,
                             const uint4 *old_xref, const int32_t *old_linv, int32_t *new_list,
                             int32_t *new_cnt, int32_t *new_perm, uint4 *new_xref, int32_t *new_linv,
                             int32_t *new_flag, cudaStream_t st);
// Near-field force (caller order) with both energies packed in fnear[i].w as
// two floats (U_near high word, U_wca low word).
// Core-shell kernel of the list path (Sec. 3.4): Taylor coefficients of the
// core with the series' signs folded in (a: G, b: F_M, in powers of r^2),
// r_in^2, the shell table's exponent-bit mask and length (entries: kernel
// value at the bin start and its change over the bin, for the force factor
// and the pair energy).
constexpr int kCsQ = 10;         // Taylor terms of the core
constexpr int kCsManBits = 8;    // mantissa bits of the shell-table index
struct CoreShellDev {
    float a[kCsQ];               // G(u)   = sum_{i<Q}  a_i u^i
    float b[kCsQ + 1];           // F_M(u) = sum_{i<=Q} b_i u^i
    float rin2;
    uint32_t emask;              // 2^b_exp - 1
    int32_t n_tab;               // 2^(b_exp + kCsManBits)
};
// cs == nullptr: the combined table (ltab); else the core-shell kernel with
// its table cstab.  energy = false leaves the pair energies out (zero) except
// in systems on their last budgeted step.
cudaError_t launch_near_list(const BatchView &bv, const NearSog &sog, const float4 *ltab, const int32_t *nbr_list,
                             const int32_t *nbr_cnt, const int32_t *list_perm, double4_32a *fnear, cudaStream_t st,
                             const Prof *prof, const CoreShellDev *cs = nullptr, const float4 *cstab = nullptr,
                             bool energy = true);

// ---- far field (k_far.cu) -----------------------------------------------------
// tile_override > 0 replaces the default particles-per-tile rule (tunable)
void far_layout(int64_t n, int32_t P, int precision, int tile_override, int &tile_p, int &n_ptiles);
// blocks_per_sm > 0: a persistent grid of that many blocks per SM, each
// taking several (particle tile, frequency tile) items, which leaves room on
// every SM for a kernel running beside it on another stream.
cudaError_t launch_rho_sweep(int precision, const BatchView &bv, const double4_32a *sp64,
                             const uint4 *sp32, double2 *rho_part, cudaStream_t st, const Prof *prof,
                             int blocks_per_sm = 0);
// Combines partials in FP64 (fixed order) into rho[n_sys * P] and the per-k
// scatter table (k vector, prescaled Re/Im rho, integer m).
cudaError_t launch_rho_combine(int precision, const BatchView &bv, const double2 *rho_part, double2 *rho,
                               void *ktab, cudaStream_t st, const Prof *prof);
// Total force (near + far) written to force[perm[s]] in caller order.  With
// perm null the particles are already in caller order (neighbour-list path):
// force[s] = fnear[s] + far, and the per-particle energies packed in
// fnear[s].w are summed per particle block into epart[e_off + block].
// FP32C with kick_vel non-null: the step's second half kick is fused into
// the kernel (v += dt/2 F/m in caller order and the kinetic-energy partial
// of each particle block into kick_kpart, the bits of launch_kick); only
// when nothing else adds to the force afterwards.
// With drift non-null as well (FP32C, neighbour lists, no thermostat): the
// next step's half kick and drift follow in the same pass, with the
// expressions of launch_kick_drift (drift.posq, and the fixed-point pack and
// displacement test into drift.sp32c / xref / rebuild), so that the next
// step starts at its force evaluation.
struct DriftOut {
    double4_32a *posq;
    uint4 *sp32c;
    const uint4 *xref;
    int32_t *rebuild;
};
cudaError_t launch_far_scatter(int precision, const BatchView &bv, const double4_32a *sp64,
                               const uint4 *sp32, const void *ktab, const double4_32a *fnear,
                               const int32_t *perm, double4_32a *force, int32_t *err_flag, cudaStream_t st,
                               const Prof *prof, double2 *epart = nullptr, double4_32a *kick_vel = nullptr,
                               double *kick_kpart = nullptr, const DriftOut *drift = nullptr);
size_t ktab_bytes(int precision, int64_t nk);

// ---- integrator and reductions (k_md.cu) --------------------------------------
// Device energies per system, 12 doubles: [0] U_near [1] U_far [2] U_self
// [3] U_wca [4] K [5] T [6] lambda (velocity factor of the thermostat)
// [7] U_bound [8] Nose-Hoover xi [9] eta [10] (1/2) Q xi^2 + g T0 eta [11] spare
constexpr int kNumEnergy = 12;
// With sp32c non-null (neighbour-list path) it also writes the fixed-point
// caller-order positions and runs the displacement test (fixed_pack_check).
cudaError_t launch_kick_drift(const BatchView &bv, double4_32a *posq, double4_32a *vel,
                              const double4_32a *force, cudaStream_t st, const Prof *prof,
                              uint4 *sp32c = nullptr, const uint4 *xref = nullptr, int32_t *rebuild = nullptr);
cudaError_t launch_kick(const BatchView &bv, double4_32a *vel, const double4_32a *force, double *kpart,
                        cudaStream_t st, const Prof *prof);
// kFinChunks blocks per system sum chunks of the energy partials, |rho|^2
// and kinetic partials in fixed order; the last block of a system to finish
// adds the chunk sums in chunk order and writes the energies, T and the
// Berendsen factor, and advances the cursor by `advance` and, with kinetic
// terms, the step counter by one.
cudaError_t launch_finalize(const BatchView &bv, const double2 *epart, const double2 *rho, const double *kpart,
                            int with_kinetic, double *energy, int64_t advance, cudaStream_t st,
                            const Prof *prof);
// A step whose energies and temperature nobody reads (no thermostat, no step
// budgets, not the last step of a call): only the cursor advance and the
// step count of finalize, one thread per system.
cudaError_t launch_finalize_counters(const BatchView &bv, int64_t advance, cudaStream_t st, const Prof *prof);
// ---- virial (k_virial.cu) ------------------------------------------------------
// Configurational virial W[9] (row-major, symmetric) of system 0: near field
// (+ WCA) from the cell list (start, perm, cell_of) and the FP64 positions,
// far field from rho[P] of the k-set m3[P][3] and the SOG (omega, sl of
// M + 1 terms, normaliser S).  part: virial_blocks(n) * 6 doubles of scratch.
int32_t virial_blocks(int64_t n);
cudaError_t launch_virial(const SysDesc *sysd, int64_t n, const NearSog &sog, const int32_t *start,
                          const int32_t *perm, const int32_t *cell_of, const double4_32a *posq, double *part,
                          const double2 *rho, const int32_t *m3, int32_t P, const double *omega, const double *sl,
                          int32_t M, double S, double *W, cudaStream_t st);

// ---- heat flux (k_heat.cu) -----------------------------------------------------
// Heat flux J[3] (Appendix A) of system 0 from the FP64 caller-order state:
// near field (+ WCA) over the cell list (start, perm, cell_of), kinetic and
// self terms (half_lB_FM0 = lB F_M(0) / 2), and for P > 0 the random-batch far
// energy and virial split over atoms on the k-set m3[P][3] (half_c = lB
// pi^{3/2} S / (2 P V); SOG omega, sl of M + 1 terms).  Scratch: rpart
// heat_rho_partials(P) double2, rho[P], ktab[2P], part_near and part_far
// 3 * heat_blocks(n) doubles each.
int32_t heat_blocks(int64_t n);
size_t heat_rho_partials(int32_t P);
cudaError_t launch_heat_flux(const SysDesc *sysd, const BoxDev &box, int64_t n, const NearSog &sog,
                             const int32_t *start, const int32_t *perm, const int32_t *cell_of,
                             const double4_32a *posq, const double4_32a *vel, double mass, double half_lB_FM0,
                             const int32_t *m3, int32_t P, const double *omega, const double *sl, int32_t M,
                             double half_c, double2 *rpart, double2 *rho, double4_32a *ktab, double *part_near,
                             double *part_far, double *J, cudaStream_t st);

// ---- observables (k_observe.cu) --------------------------------------------------
// MSD/VACF sampling of system 0 (n particles, caller order): per sample the
// unwrapped positions u (from xprev, the folded positions of the previous
// sample; first != 0 starts them), the origin ring (ring_u, ring_v: slots of
// n entries; store_slot < 0 stores none) and, for each active origin p
// (ring slot pr.slot[p] at lag pr.lag[p]), the sums of |u - u0|^2 and v . v0
// added to msd_sum, vacf_sum and count at that lag.  part: obs_blocks(n) *
// kObsMaxPairs double2 of scratch.
constexpr int kObsMaxPairs = 64;
struct ObsPairs {
    int32_t n;
    int32_t slot[kObsMaxPairs];
    int32_t lag[kObsMaxPairs];
};
int32_t obs_blocks(int64_t n);
cudaError_t launch_obs_sample(int64_t n, const double4_32a *posq, const double4_32a *vel, double4_32a *xprev,
                              double4_32a *u, double4_32a *ring_u, double4_32a *ring_v, const double L[3],
                              int first, int store_slot, const ObsPairs &pr, double2 *part, double *msd_sum,
                              double *vacf_sum, int64_t *count, cudaStream_t st);
// out[0 .. n_lags) = MSD, out[n_lags .. 2 n_lags) = VACF (0 where count = 0).
cudaError_t launch_obs_result(int32_t n_lags, int64_t n, const double *msd_sum, const double *vacf_sum,
                              const int64_t *count, double *out, cudaStream_t st);
// Pt[9] = (sum_i m v_i v_i^T + W) / V; part: obs_blocks(n) * 6 doubles.
cudaError_t launch_pressure(int64_t n, const double4_32a *vel, double mass, const double *W, double V,
                            double *part, double *Pt, cudaStream_t st);
// Green-Kubo: mean[6] scratch, acf[max_lag], *C = scale * trapezoid(acf)
// with scale = V dt / (6 T); series[ns][9] on the device.
cudaError_t launch_green_kubo(const double *series, int64_t ns, int32_t max_lag, double scale, double *mean,
                              double *acf, double *C, cudaStream_t st);
// Green-Kubo heat conductivity: acf[t] = sum over the three components and
// the ns - t origins of J(t0) . J(t0 + t) / (ns - t), *C = scale *
// trapezoid(acf), scale = V dt / (3 T^2); series[ns][3] on the device.
cudaError_t launch_green_kubo_heat(const double *series, int64_t ns, int32_t max_lag, double scale, double *acf,
                                   double *C, cudaStream_t st);

// ---- boundary terms (k_boundary.cu) ---------------------------------------------
// Zero-frequency term of systems with a non-tinfoil boundary: dipole moment
// from the caller-order positions, U0 into energy[sys * kNumEnergy + 7], the
// force term added to the caller-order total force.
cudaError_t launch_boundary(const BatchView &bv, const double4_32a *posq, double4_32a *dpart, double4_32a *dip,
                            double *energy, double4_32a *force, cudaStream_t st, const Prof *prof);
cudaError_t launch_rescale(const BatchView &bv, double4_32a *vel, const double *energy, cudaStream_t st,
                           const Prof *prof);
// With step budgets: one step of every unfrozen system is done.
cudaError_t launch_step_done(const BatchView &bv, cudaStream_t st, const Prof *prof);
// Charge sums per block of 256: part[3 b + (0, 1, 2)] = (sum q, sum |q|, sum q^2).
cudaError_t launch_charge_sums(int64_t n, const double *q, double *part, cudaStream_t st);
// Layout conversions between caller [n][3] arrays and the internal double4_32a.
cudaError_t launch_pack(int64_t n, const double *x3, const double *q, double4_32a *out, int wrap,
                        const double *L, cudaStream_t st);
cudaError_t launch_unpack(int64_t n, const double4_32a *in, double *x3, cudaStream_t st);
cudaError_t launch_unsort_i32(int64_t n, int64_t off, const int32_t *perm, const int32_t *sorted,
                              int32_t *out, cudaStream_t st);
cudaError_t launch_m_to_int4(int32_t P, const int32_t *m3, int4 *out, cudaStream_t st);

// ---- radial distribution functions (k_rdf.cu) --------------------------------
// Sign-pair histograms counts[3][nbins] (++, +-, --) of minimum-image pair
// distances on [0, L/2) for n particles posq[0..n) of a cubic box of edge L,
// nbins a power of two in [16, 4096]; nspec[2] receives the numbers of
// positive and negative sites; g[3][nbins] (optional) the Appendix A estimate.
// pt is scratch of n uint4.
cudaError_t launch_rdf(int64_t n, const double4_32a *posq, double L, int32_t nbins, uint4 *pt,
                       unsigned long long *counts, unsigned long long *nspec, double *g, cudaStream_t st,
                       const Prof *prof);

}  // namespace rbsog

