// Near-field pair force of the SOG split (Eq. 3.9, first line, read as
// -grad of U_N with N(r) = 1/r - F_M(r) of Eq. 2.7), plus the WCA soft
// repulsion, over the device cell list.
//
// Work decomposition.  A block owns `group` consecutive cells of one x-row
// (the home cells; in cell order their particles are contiguous) and one
// thread per home particle.  The block stages the 9 neighbouring row
// segments (x0-1 .. xe, y +-1, z +-1; each is one or two contiguous ranges
// of the cell-ordered arrays) into shared memory with coalesced 16/32-byte
// loads.  Each thread then works in two phases:
//   test     walk the 27-cell candidate ranges of its particle (9 contiguous
//            runs in shared memory) with distance tests only, appending the
//            staged index of every partner within r_c to a private list in
//            shared memory (thread-minor layout, conflict-free);
//   compute  evaluate pair force and energy for the listed partners, so the
//            expensive arithmetic runs without branch divergence.
// Every ordered pair is visited from both ends (no Newton-3 atomics) and each
// particle sums its partners in a fixed order, so forces and energies are
// deterministic.
//
// FP64 path: separations d = (x_i - x_j) - L n with the image shift n of the
// staged cell and r^2 = (dx^2 + dy^2) + dz^2 rounded after every operation,
// the same decisions r^2 < r_c^2 as any IEEE evaluation of the minimum image.
// FP32C path: positions arrive as 32-bit fixed point; staging converts them
// once to FP32 offsets from the block's centre (the int32 wrap of the
// difference is the minimum image), so the per-pair work is pure FP32.
//
// Gaussians with s_l < 2 r_c are evaluated with exp; the wide ones are summed
// as a Taylor series in r^2 (r^2 / s_l^2 <= 1/4 inside the cutoff), which
// removes most transcendental work without changing the kernel beyond
// rounding.
#include <algorithm>
#include <cmath>

#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kThreads = 128;   // one home particle per thread
constexpr int kMaxGroup = 16;
constexpr int kMaxStaged = 9 * (kMaxGroup + 2);
constexpr int kList32 = 32;     // partner-list entries per thread, FP32C (uint16), plus one spare slot
constexpr int kMaxHome = 1024;  // home particles a block can reorder (more: cell order is kept)
constexpr int kList64 = 64;     // partner-list entries per thread, FP64 (int32: index | shift code)

__device__ __forceinline__ int wrap_cell(int c, int n, int &shift) {
    shift = 0;
    if (c < 0) {
        shift = -1;
        return c + n;
    }
    if (c >= n) {
        shift = 1;
        return c - n;
    }
    return c;
}

// Offset of fixed-point coordinate a from origin o as FP32 (minimum image).
__device__ __forceinline__ float fixed_offset(uint32_t a, uint32_t o, float scale) {
    return (float)(int32_t)(a - o) * scale;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int PREC>
struct NearTypes;
template <>
struct NearTypes<0> {
    using real = double;
    using staged = double4_32a;
    using entry = int32_t;
    static constexpr int kList = kList64;
};
template <>
struct NearTypes<1> {
    using real = float;
    using staged = float4;
    using entry = uint16_t;
    static constexpr int kList = kList32;
};

template <int PREC, int ND, int NT>
struct PairMath;

template <int ND, int NT>
struct PairMath<1, ND, NT> {
    // fs = F_M(r) sum, gs = sum w_l/s_l^2 e^{-r^2/s_l^2}; coefficients are
    // read from the grid-constant parameter block (constant-bank operands
    // when the counts are compile-time constants)
    static __device__ __forceinline__ void gauss(const NearSog &s, float r2, float &fs, float &gs) {
        fs = 0.f;
        gs = 0.f;
        const int nd = ND > 0 ? ND : s.n_direct;
#pragma unroll
        for (int l = 0; l < (ND > 0 ? ND : kMaxGauss); ++l) {
            if (l >= nd) break;
            const float e = ex2_approx(-r2 * s.inv_s2_log2e_f[l]);
            fs = fmaf(s.omega_f[l], e, fs);
            gs = fmaf(s.omega_s2_f[l], e, gs);
        }
        const int nt = NT > 0 ? NT : s.n_taylor_f;
        if (nt > 0) {
            float pf = s.tay_f_f[nt - 1], pg = s.tay_g_f[nt - 1];
#pragma unroll
            for (int m = (NT > 0 ? NT : kMaxTaylor) - 2; m >= 0; --m) {
                if (m > nt - 2) continue;
                pf = fmaf(pf, r2, s.tay_f_f[m]);
                pg = fmaf(pg, r2, s.tay_g_f[m]);
            }
            fs += pf;
            gs += pg;
        }
    }
    static __device__ __forceinline__ float inv_sqrt(float r2) { return rsqrtf(r2); }
};

template <int ND, int NT>
struct PairMath<0, ND, NT> {
    static __device__ __forceinline__ void gauss(const NearSog &s, double r2, double &fs, double &gs) {
        fs = 0.0;
        gs = 0.0;
        const int nd = ND > 0 ? ND : s.n_direct;
#pragma unroll
        for (int l = 0; l < (ND > 0 ? ND : kMaxGauss); ++l) {
            if (l >= nd) break;
            const double e = exp(-r2 * s.inv_s2[l]);
            fs += s.omega[l] * e;
            gs += s.omega[l] * s.inv_s2[l] * e;
        }
        const int nt = NT > 0 ? NT : s.n_taylor;
        if (nt > 0) {
            double pf = s.tay_f[nt - 1], pg = s.tay_g[nt - 1];
#pragma unroll
            for (int m = (NT > 0 ? NT : kMaxTaylor) - 2; m >= 0; --m) {
                if (m > nt - 2) continue;
                pf = pf * r2 + s.tay_f[m];
                pg = pg * r2 + s.tay_g[m];
            }
            fs += pf;
            gs += pg;
        }
    }
    static __device__ __forceinline__ double inv_sqrt(double r2) { return 1.0 / sqrt(r2); }
};

template <class real>
struct PairConst {
    real rc2, wrc2, ws2, weps, lB;
};

// FP32C: 6 resident blocks per SM (at most 85 registers), measured faster
// than 4-5 with the shorter partner list; FP64 keeps 4 (no spills)
template <int PREC, int ND, int NT, bool WIN>
__global__ void __launch_bounds__(kThreads, PREC == 1 ? 6 : 4)
    k_near(const BatchView bv, const __grid_constant__ NearSog sog, const int32_t *__restrict__ start,
           const double4_32a *__restrict__ sp64, const uint4 *__restrict__ sp32,
           double4_32a *__restrict__ fnear, double2 *__restrict__ epart, int32_t *__restrict__ nbr) {
    using T = NearTypes<PREC>;
    using real = typename T::real;
    using staged = typename T::staged;
    using entry = typename T::entry;
    using PM = PairMath<PREC, ND, NT>;
    constexpr int kList = T::kList;
    __shared__ int s_off[kMaxStaged + 1];
    __shared__ int s_src[kMaxStaged];
    __shared__ int s_shift[kMaxStaged];
    __shared__ int s_hstart[kMaxGroup + 1];
    __shared__ float4 s_tab[ND < 0 ? 2 * kTabN : 1];   // Gaussian-sum tables (ND < 0)
    __shared__ uint16_t s_hord[WIN && PREC == 1 ? kMaxHome : 1];    // home particles in quadrant order (WIN, FP32C)
    // split (FP64, small systems): the row partials of the four warps
    __shared__ double s_pf[PREC == 0 ? 3 * kThreads : 1];
    __shared__ int s_pc[PREC == 0 ? kThreads : 1];
    extern __shared__ __align__(32) unsigned char smem_raw[];
    // disjoint regions: restrict lets the compiler move staged loads across
    // list stores
    staged *__restrict__ st = reinterpret_cast<staged *>(smem_raw);
    entry *__restrict__ list = reinterpret_cast<entry *>(smem_raw + sizeof(staged) * (size_t)bv.max_cap);   // [kList][kThreads]

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int2 work = bv.nblk[blockIdx.x];
    if (bv.remaining && bv.remaining[work.x] == 0) return;   // frozen system: whole block leaves
    const SysDesc &desc = bv.sys[work.x];
    const BoxDev &box = desc.box;
    const int group = desc.group, nseg_x = desc.nseg_x, cap = desc.near_cap;
    const int64_t coff = desc.c_off;
    const int nx = box.nc[0], ny = box.nc[1], nz = box.nc[2];
    const int sx = work.y % nseg_x, row = work.y / nseg_x;
    const int cy = row % ny, cz = row / ny;
    const int x0 = sx * group, xe = min(x0 + group, nx), nh = xe - x0, w = nh + 2;
    const int ns = 9 * w;

    // staged cell table: (source start, count, packed image shift)
    for (int k = tid; k < ns; k += kThreads) {
        const int r = k / w, xi = k % w;
        int shx, shy, shz;
        const int zz = wrap_cell(cz + r / 3 - 1, nz, shz);
        const int yy = wrap_cell(cy + r % 3 - 1, ny, shy);
        const int xx = wrap_cell(x0 - 1 + xi, nx, shx);
        const int64_t id = coff + (zz * ny + yy) * nx + xx;
        const int b = start[id];
        s_src[k] = b;
        s_off[k + 1] = start[id + 1] - b;   // count for now
        s_shift[k] = (shx + 1) | ((shy + 1) << 2) | ((shz + 1) << 4);
    }
    if (tid <= nh) s_hstart[tid] = start[coff + (cz * ny + cy) * nx + x0 + tid];
    if constexpr (ND < 0)
        for (int k = tid; k < 2 * kTabN; k += kThreads) s_tab[k] = k < kTabN ? sog.tab_g[k] : sog.tab_f[k - kTabN];
    if (tid == 0) s_off[0] = 0;
    __syncthreads();
    if (wid == 0) {  // inclusive scan of counts into offsets, 32 at a time
        int carry = 0;
        for (int base = 0; base < ns; base += 32) {
            const int k = base + lane;
            int v = k < ns ? s_off[k + 1] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            if (k < ns) s_off[k + 1] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    const int total = s_off[ns];
    const int hb = s_hstart[0], he = s_hstart[nh];

    // FP32C origin: centre of the home segment (to FP32 rounding, a few 1e-6
    // of a cell side -- any common origin gives the same offsets' differences)
    uint32_t ox = 0, oy = 0, oz = 0;
    if constexpr (PREC == 1) {
        ox = (uint32_t)__float2ull_rn(((float)x0 + 0.5f * (float)nh) * box.cell_fix[0]);
        oy = (uint32_t)__float2ull_rn(((float)cy + 0.5f) * box.cell_fix[1]);
        oz = (uint32_t)__float2ull_rn(((float)cz + 0.5f) * box.cell_fix[2]);
    }
    const float fsx = box.fix_scale[0], fsy = box.fix_scale[1], fsz = box.fix_scale[2];
    // WIN: the warps take the home particles grouped by the quadrant of their
    // cell's y-z square they sit in (stable within a quadrant, so in x order),
    // so that a warp's lanes see similar row gaps and similar window lengths.
    // The grouping is a deterministic stable counting sort done by warp 0.
    const int nhome = he - hb;
    // (FP32C only: FP64 keeps the cell order, so that its per-block energy
    // sums keep their order)
    const bool reord = WIN && PREC == 1 && nhome <= kMaxHome;
    if constexpr (WIN && PREC == 1) {
        if (reord && wid == 0) {
            auto quad = [&](int p) {
                if (p >= nhome) return 4;
                const uint4 uq = sp32[hb + p];
                return (fixed_offset(uq.y, oy, fsy) > 0.f ? 1 : 0) | (fixed_offset(uq.z, oz, fsz) > 0.f ? 2 : 0);
            };
            int o0 = 0, o1 = 0, o2 = 0, o3 = 0;
            for (int p0 = 0; p0 < nhome; p0 += 32) {
                const int k = quad(p0 + lane);
                o1 += __popc(__ballot_sync(0xffffffffu, k == 0));
                o2 += __popc(__ballot_sync(0xffffffffu, k == 1));
                o3 += __popc(__ballot_sync(0xffffffffu, k == 2));
            }
            o2 += o1;   // exclusive offsets of quadrants 1, 2, 3
            o3 += o2;
            const unsigned lt = (1u << lane) - 1u;
            for (int p0 = 0; p0 < nhome; p0 += 32) {
                const int p = p0 + lane, k = quad(p);
                const unsigned m0 = __ballot_sync(0xffffffffu, k == 0), m1 = __ballot_sync(0xffffffffu, k == 1);
                const unsigned m2 = __ballot_sync(0xffffffffu, k == 2), m3 = __ballot_sync(0xffffffffu, k == 3);
                const unsigned mk = k == 0 ? m0 : k == 1 ? m1 : k == 2 ? m2 : m3;
                const int ok = k == 0 ? o0 : k == 1 ? o1 : k == 2 ? o2 : o3;
                if (p < nhome) s_hord[ok + __popc(mk & lt)] = (uint16_t)p;
                o0 += __popc(m0);
                o1 += __popc(m1);
                o2 += __popc(m2);
                o3 += __popc(m3);
            }
        }
    }
    PairConst<real> pc;
    if constexpr (PREC == 0) {
        pc = PairConst<real>{box.rc2, box.wca_rc2, box.wca_s2, box.wca_eps, box.lB};
    } else {
        pc = PairConst<real>{box.rc2_f, box.wca_rc2_f, box.wca_s2_f, box.wca_eps_f, box.lB_f};
    }

    double e_near = 0.0, e_wca = 0.0;
    // split (FP64 systems below kNearSplitMaxN particles, whose blocks hold
    // too few home particles to keep four warps busy): every warp takes every
    // run of 32 home particles, but only the rows r = wid, wid + 4, ...; the
    // four row partials of a particle are added in warp order.  The order
    // depends on the system alone (not on the block size), so a system's
    // forces are the same bits alone or in a batch.
    const bool split = PREC == 0 && desc.near_split != 0;
    // Staging: one chunk [c0, c1) of the staged region at a time (normally the
    // whole region fits); every warp then works through the home particles in
    // runs of 32 consecutive particles (one per lane).
    for (int c0 = 0; c0 < total; c0 += cap) {
        const int c1 = min(c0 + cap, total);
        if (c0 > 0) __syncthreads();
        for (int r = 0; r < 9; ++r) {
            const int k = r * w;
            const int plo[3] = {s_off[k], s_off[k + 1], s_off[k + w - 1]};
            const int phi[3] = {s_off[k + 1], s_off[k + w - 1], s_off[k + w]};
            const int psrc[3] = {s_src[k], s_src[k + 1], s_src[k + w - 1]};
#pragma unroll
            for (int pp = 0; pp < 3; ++pp) {
                const int a = max(plo[pp], c0), b = min(phi[pp], c1);
                for (int t = a + tid; t < b; t += kThreads) {
                    const int src = psrc[pp] + (t - plo[pp]);
                    if constexpr (PREC == 0) {
                        st[t - c0] = sp64[src];
                    } else {
                        const uint4 u = sp32[src];
                        st[t - c0] = make_float4(fixed_offset(u.x, ox, fsx), fixed_offset(u.y, oy, fsy),
                                                 fixed_offset(u.z, oz, fsz), __uint_as_float(u.w));
                    }
                }
            }
        }
        __syncthreads();
        for (int rb = hb + (split ? 0 : 32 * wid); rb < he; rb += split ? 32 : kThreads) {
            const int pidx = rb - hb + lane;
            const bool active = pidx < nhome;
            const int hi = active ? hb + (reord ? (int)s_hord[pidx] : pidx) : he;
            int cxr = 0;
            while (cxr + 1 < nh && s_hstart[cxr + 1] <= (active ? hi : he - 1)) ++cxr;
            // the warp's lanes cover home cells cx_lo..cx_hi (particles are in
            // cell order); all lanes walk the union of their stencils, so the
            // candidate loops have warp-uniform trip counts and every staged
            // load is a broadcast -- candidates two or more cells away are
            // farther than h >= r_c and fail the distance test
            const int cx_lo = __shfl_sync(0xffffffffu, cxr, 0);
            const int cx_hi = __reduce_max_sync(0xffffffffu, (unsigned)cxr);
            const int t_self = s_off[4 * w + cxr + 1] + (hi - s_hstart[cxr]);
            real ix = 0, iy = 0, iz = 0, qi = 0;
            if (active) {
                if constexpr (PREC == 0) {
                    const double4_32a p = sp64[hi];
                    ix = p.x; iy = p.y; iz = p.z; qi = p.w;
                } else {
                    const uint4 u = sp32[hi];
                    ix = fixed_offset(u.x, ox, fsx);
                    iy = fixed_offset(u.y, oy, fsy);
                    iz = fixed_offset(u.z, oz, fsz);
                    qi = __uint_as_float(u.w);
                }
            } else {
                ix = iy = iz = (real)1e30;   // inactive lanes accept nothing
            }
            real fx = 0, fy = 0, fz = 0, un = 0, uw = 0;
            int cnt = 0, n = 0;
            // pair force and energy for list entries [0, n)
            auto compute = [&]() {
#pragma unroll 2
                for (int e = 0; e < n; ++e) {
                    const entry en = list[e * kThreads + tid];
                    const int t = (int)en & 0xFFFFF;
                    real dx, dy, dz, r2, qj;
                    if constexpr (PREC == 0) {
                        const int code = (int)en >> 20;
                        const double4_32a pj = st[t];
                        const double lx = box.L[0] * (double)((code & 3) - 1);
                        const double ly = box.L[1] * (double)(((code >> 2) & 3) - 1);
                        const double lz = box.L[2] * (double)(((code >> 4) & 3) - 1);
                        dx = __dsub_rn(__dsub_rn(ix, pj.x), lx);
                        dy = __dsub_rn(__dsub_rn(iy, pj.y), ly);
                        dz = __dsub_rn(__dsub_rn(iz, pj.z), lz);
                        r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                        qj = pj.w;
                    } else {
                        const float4 pj = st[t];
                        dx = ix - pj.x;
                        dy = iy - pj.y;
                        dz = iz - pj.z;
                        r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        qj = pj.w;
                    }
                    const real qq = pc.lB * qi * qj;
                    real fs, gs;
                    if constexpr (ND < 0) {
                        // piecewise cubic in r^2 (interval k, local s in [0, 1))
                        const float x = r2 * sog.tab_scale;
                        const int k = min((int)x, kTabN - 1);
                        const float sl = x - (float)k;
                        const float4 cg = s_tab[k], cf = s_tab[kTabN + k];
                        gs = fmaf(fmaf(fmaf(cg.w, sl, cg.z), sl, cg.y), sl, cg.x);
                        fs = fmaf(fmaf(fmaf(cf.w, sl, cf.z), sl, cf.y), sl, cf.x);
                    } else {
                        PM::gauss(sog, r2, fs, gs);
                    }
                    const real inv_r = PM::inv_sqrt(r2);
                    real g = qq * (inv_r * inv_r * inv_r - (real)2 * gs);
                    un += (real)0.5 * qq * (inv_r - fs);
                    if (r2 < pc.wrc2) {
                        const real sr2 = pc.ws2 / r2;
                        const real sr6 = sr2 * sr2 * sr2;
                        g += (real)24 * pc.weps * ((real)2 * sr6 * sr6 - sr6) / r2;
                        uw += (real)0.5 * ((real)4 * pc.weps * (sr6 * sr6 - sr6) + pc.weps);
                    }
                    fx += g * dx;
                    fy += g * dy;
                    fz += g * dz;
                }
                cnt += n;
                n = 0;
            };
            if constexpr (WIN && PREC == 0) {
                // FP64 per-lane windows: the same x-windows as below, found
                // on FP32 offsets from the block centre (a staged particle's
                // offset is its FP64 x plus its cell's image shift, minus the
                // centre), with a margin far above the FP32 rounding; the
                // FP64 distance test decides, with the expressions of the
                // full stencil.  The windows hold every partner in the same
                // staged order, so the lists, and so the forces and energies,
                // are those of the full stencil bit for bit.
                constexpr float kMargin = 1e-3f;
                const float hy = box.h_f[1], hz = box.h_f[2];
                const float inv_hx = 1.0f / box.h_f[0], xbase = 1.0f + 0.5f * (float)nh;
                const double cxa = ((double)x0 + 0.5 * (double)nh) * box.h[0];
                const double cya = ((double)cy + 0.5) * box.h[1], cza = ((double)cz + 0.5) * box.h[2];
                const float fxi = (float)(ix - cxa), fyi = (float)(iy - cya), fzi = (float)(iz - cza);
#pragma unroll 1
                for (int r = split ? wid : 0; r < 9; r += split ? kThreads / 32 : 1) {
                    const int dyr = r % 3 - 1, dzr = r / 3 - 1;
                    const int k0 = r * w;
                    int lo = 0, len = 0, cl = 0;
                    if (active) {
                        const float gy = dyr == 0 ? 0.f
                                                  : fmaxf((dyr < 0 ? fyi + 0.5f * hy : 0.5f * hy - fyi) - kMargin, 0.f);
                        const float gz = dzr == 0 ? 0.f
                                                  : fmaxf((dzr < 0 ? fzi + 0.5f * hz : 0.5f * hz - fzi) - kMargin, 0.f);
                        const float b2 = box.rc2_f - gy * gy - gz * gz;
                        if (b2 > 0.f) {
                            const float bb = sqrtf(b2) + kMargin;
                            const float xl = fxi - bb, xr = fxi + bb;
                            cl = min(max((int)floorf(fmaf(xl, inv_hx, xbase)), 0), w - 1);
                            const int ch = min(max((int)floorf(fmaf(xr, inv_hx, xbase)), 0), w - 1);
                            const double ol = box.L[0] * (double)((s_shift[k0 + cl] & 3) - 1) - cxa;
                            int a = max(s_off[k0 + cl], c0), e = min(s_off[k0 + cl + 1], c1);
                            while (a < e) {   // first x >= xl
                                const int m = (a + e) >> 1;
                                if ((float)(st[m - c0].x + ol) < xl) a = m + 1; else e = m;
                            }
                            lo = a;
                            const double oh = box.L[0] * (double)((s_shift[k0 + ch] & 3) - 1) - cxa;
                            a = max(s_off[k0 + ch], c0);
                            e = min(s_off[k0 + ch + 1], c1);
                            while (a < e) {   // first x > xr
                                const int m = (a + e) >> 1;
                                if ((float)(st[m - c0].x + oh) <= xr) a = m + 1; else e = m;
                            }
                            len = max(min(a, c1) - min(lo, c1), 0);
                        }
                    }
                    const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
                    int kc = k0 + cl;   // staged cell of the next candidate
                    for (int it = 0; it < maxlen; it += kList) {
                        const int m = min(max(len - it, 0), kList);
                        if (__any_sync(0xffffffffu, n + m > kList)) compute();
                        for (int uu = 0; uu < m; ++uu) {
                            const int t = lo + it + uu;
                            while (s_off[kc + 1] <= t) ++kc;
                            const int code = s_shift[kc];
                            const double4_32a pj = st[t - c0];
                            const double dx = __dsub_rn(__dsub_rn(ix, pj.x), box.L[0] * (double)((code & 3) - 1));
                            const double dy = __dsub_rn(__dsub_rn(iy, pj.y), box.L[1] * (double)(((code >> 2) & 3) - 1));
                            const double dz = __dsub_rn(__dsub_rn(iz, pj.z), box.L[2] * (double)(((code >> 4) & 3) - 1));
                            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                            if (r2 < pc.rc2 && t != t_self) {
                                list[n * kThreads + tid] = (entry)((t - c0) | (code << 20));
                                ++n;
                            }
                        }
                    }
                }
            } else if constexpr (WIN) {
                // Per-lane windows.  Every staged row is sorted in x (cells
                // in x order, members by x), so the candidates of lane i in
                // row (dy, dz) are the contiguous run with |x_j - x_i| <= b,
                // b^2 = r_c^2 - (y gap)^2 - (z gap)^2 from the row's y/z
                // extent; it is found by binary search in the two cells that
                // hold its ends.  The margin (far above FP32 rounding of the
                // offsets) keeps the run a superset of the partners; the
                // distance test below decides.
                constexpr float kMargin = 1e-3f;
                constexpr int kChunk = 8;
                const float hx = box.h_f[0], hy = box.h_f[1], hz = box.h_f[2];
                const float inv_hx = 1.0f / hx, xbase = 1.0f + 0.5f * (float)nh;
#pragma unroll 1
                for (int r = 0; r < 9; ++r) {
                    const int dyr = r % 3 - 1, dzr = r / 3 - 1;
                    int lo = 0, len = 0;
                    if (active) {
                        const float gy = dyr == 0 ? 0.f
                                                  : fmaxf((dyr < 0 ? iy + 0.5f * hy : 0.5f * hy - iy) - kMargin, 0.f);
                        const float gz = dzr == 0 ? 0.f
                                                  : fmaxf((dzr < 0 ? iz + 0.5f * hz : 0.5f * hz - iz) - kMargin, 0.f);
                        const float b2 = pc.rc2 - gy * gy - gz * gz;
                        if (b2 > 0.f) {
                            const float bb = sqrtf(b2) + kMargin;
                            const float xl = ix - bb, xr = ix + bb;
                            const int k0 = r * w;
                            const int cl = min(max((int)floorf(fmaf(xl, inv_hx, xbase)), 0), w - 1);
                            const int ch = min(max((int)floorf(fmaf(xr, inv_hx, xbase)), 0), w - 1);
                            int a = max(s_off[k0 + cl], c0), e = min(s_off[k0 + cl + 1], c1);
                            while (a < e) {   // first x >= xl
                                const int m = (a + e) >> 1;
                                if (st[m - c0].x < xl) a = m + 1; else e = m;
                            }
                            lo = a;
                            a = max(s_off[k0 + ch], c0);
                            e = min(s_off[k0 + ch + 1], c1);
                            while (a < e) {   // first x > xr
                                const int m = (a + e) >> 1;
                                if (st[m - c0].x <= xr) a = m + 1; else e = m;
                            }
                            // a cell range that lies wholly after the staged
                            // chunk leaves its bound at or past c1: the run is
                            // clamped to the chunk (and is empty there)
                            len = max(min(a, c1) - min(lo, c1), 0);
                        }
                    }
                    const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
                    for (int it = 0; it < maxlen; it += kChunk) {
                        const int m = len - it;
                        if (__any_sync(0xffffffffu, n + min(max(m, 0), kChunk) > kList)) compute();
                        const int tb = lo + it - c0;
                        // branch-free append: every slot writes list entry n
                        // (one spare slot past kList), only partners advance n;
                        // the particle itself has r^2 = 0 exactly (identical
                        // offsets) and is not counted
#pragma unroll
                        for (int uu = 0; uu < kChunk; ++uu) {
                            const bool in = uu < m;
                            const int t = in ? tb + uu : 0;   // staged slot 0 exists whenever maxlen > 0
                            const float4 pj = st[t];
                            const float dx = ix - pj.x, dy = iy - pj.y, dz = iz - pj.z;
                            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            list[n * kThreads + tid] = (entry)t;
                            n += (in && r2 < pc.rc2 && r2 > 0.f) ? 1 : 0;
                        }
                    }
                }
            } else
            for (int r = split ? wid : 0; r < 9; r += split ? kThreads / 32 : 1) {
                const int kb = r * w + cx_lo, ke = r * w + cx_hi + 3;   // staged cells [kb, ke)
                const int lo = max(s_off[kb], c0), hi3 = min(s_off[ke], c1);
                for (int tb = lo; tb < hi3; tb += kList) {
                    const int te = min(tb + kList, hi3);
                    // the list always has room for a whole run of candidates,
                    // so the test loop never branches into the pair arithmetic
                    if (__any_sync(0xffffffffu, n + (te - tb) > kList)) compute();
                    if constexpr (PREC == 0) {
                        int kc = kb;
                        while (s_off[kc + 1] <= tb) ++kc;
                        for (int t = tb; t < te; ++t) {
                            while (s_off[kc + 1] <= t) ++kc;
                            const int code = s_shift[kc];
                            const double4_32a pj = st[t - c0];
                            const double dx = __dsub_rn(__dsub_rn(ix, pj.x), box.L[0] * (double)((code & 3) - 1));
                            const double dy = __dsub_rn(__dsub_rn(iy, pj.y), box.L[1] * (double)(((code >> 2) & 3) - 1));
                            const double dz = __dsub_rn(__dsub_rn(iz, pj.z), box.L[2] * (double)(((code >> 4) & 3) - 1));
                            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                            if (r2 < pc.rc2 && t != t_self) {
                                list[n * kThreads + tid] = (entry)((t - c0) | (code << 20));
                                ++n;
                            }
                        }
                    } else {
#pragma unroll 4
                        for (int t = tb; t < te; ++t) {
                            const float4 pj = st[t - c0];
                            const float dx = ix - pj.x, dy = iy - pj.y, dz = iz - pj.z;
                            if (fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < pc.rc2 && t != t_self) {
                                list[n * kThreads + tid] = (entry)(t - c0);
                                ++n;
                            }
                        }
                    }
                }
            }
            compute();
            if (split) {
                // the warps' row partials of the run's 32 particles, added in
                // warp order by warp 0
                s_pf[(wid * 3 + 0) * 32 + lane] = fx;
                s_pf[(wid * 3 + 1) * 32 + lane] = fy;
                s_pf[(wid * 3 + 2) * 32 + lane] = fz;
                s_pc[wid * 32 + lane] = cnt;
                __syncthreads();
                if (wid == 0) {
                    for (int w2 = 1; w2 < kThreads / 32; ++w2) {
                        fx += s_pf[(w2 * 3 + 0) * 32 + lane];
                        fy += s_pf[(w2 * 3 + 1) * 32 + lane];
                        fz += s_pf[(w2 * 3 + 2) * 32 + lane];
                        cnt += s_pc[w2 * 32 + lane];
                    }
                }
                __syncthreads();   // the partials are read before the next run writes them
            }
            if (active && (!split || wid == 0)) {
                if (c0 == 0) {
                    fnear[hi] = make_double4_32a((double)fx, (double)fy, (double)fz, 0.0);
                    if (nbr) nbr[hi] = cnt;
                } else {   // later chunks of an oversized region add to the first
                    double4_32a f = fnear[hi];
                    f.x += fx;
                    f.y += fy;
                    f.z += fz;
                    fnear[hi] = f;
                    if (nbr) nbr[hi] += cnt;
                }
            }
            e_near += (double)un;
            e_wca += (double)uw;
        }
    }
    // fixed-order reduction of the energies: warp shuffles, then the warps in
    // order -- one partial per block (the per-system sum of the partials runs
    // on one SM, where FP64 adds are scarce on this GPU)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e_near += __shfl_down_sync(0xffffffffu, e_near, o);
        e_wca += __shfl_down_sync(0xffffffffu, e_wca, o);
    }
    __shared__ double2 s_ew[kThreads / 32];
    if (lane == 0) s_ew[wid] = make_double2(e_near, e_wca);
    __syncthreads();
    if (tid == 0) {
        double2 t = s_ew[0];
#pragma unroll
        for (int w2 = 1; w2 < kThreads / 32; ++w2) {
            t.x += s_ew[w2].x;
            t.y += s_ew[w2].y;
        }
        epart[desc.e_off + work.y] = t;
    }
}

size_t near_smem(int precision, int cap) {
    if (precision == 0) return sizeof(double4_32a) * (size_t)cap + sizeof(int32_t) * kList64 * kThreads;
    return sizeof(float4) * (size_t)cap + sizeof(uint16_t) * (kList32 + 1) * kThreads;
}

}  // namespace

void near_layout(const BoxDev &box, int64_t n, int precision, int home, int &group, int &nseg_x, int &cap,
                 int &nblocks, int &npartials) {
    // one warp per 32 home particles and about `home` home particles per
    // block; the staging chunk covers the mean occupancy of the 9 (group + 2)
    // staged cells with 15% head-room (denser regions are processed in chunks)
    const double per_cell = (double)n / (double)box.ncell;
    int g = (int)std::lround((double)home / std::max(per_cell, 1e-3));
    g = std::max(1, std::min(g, std::min(kMaxGroup, box.nc[0] - 2)));
    group = g;
    nseg_x = (box.nc[0] + g - 1) / g;
    nblocks = nseg_x * box.nc[1] * box.nc[2];
    npartials = nblocks;
    const double est = 9.0 * (g + 2) * per_cell * 1.15 + 64.0;
    const int cap_max = precision == 0 ? 2048 : 4096;
    cap = std::min(cap_max, std::max(256, ((int)std::ceil(est) + 127) / 128 * 128));
}

cudaError_t launch_near(int precision, const BatchView &bv, const NearSog &sog, const int32_t *start,
                        const double4_32a *sp64, const uint4 *sp32, double4_32a *fnear, double2 *epart,
                        int32_t *nbr, cudaStream_t st, const Prof *prof) {
    const size_t sm = near_smem(precision, bv.max_cap);
    // specialised (fully unrolled) variants for the production kernel: b = 1.4878...
    // gives 5 exp Gaussians below 2 r_c and 8 (FP32) / 12 (FP64) Taylor terms
    // for any r_c; other parameter sets take the runtime-count variant
    const bool spec = sog.n_direct == 5 && (precision == 1 ? sog.n_taylor_f == 8 : sog.n_taylor == 12);
    // FP32C evaluates the Gaussian sums from the piecewise-cubic tables when
    // they are accurate to FP32 rounding (any SOG set whose narrowest Gaussian
    // is wide against the table step); otherwise exp + Taylor as FP64 does
    const bool tab = precision == 1 && sog.tab_err < 4e-7f;
    ProfScope ps(prof, precision == 0 ? (spec ? "near_fp64" : "near_fp64_generic")
                                      : (tab ? "near_fp32c" : spec ? "near_fp32c_direct" : "near_fp32c_generic"));
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<bv.n_nblk, kThreads, sm, st>>>(bv, sog, start, sp64, sp32, fnear, epart, nbr);
    };
    if (precision == 1) {
        if (tab) go(k_near<1, -1, 0, true>);
        else if (spec) go(k_near<1, 5, 8, false>);
        else go(k_near<1, 0, 0, false>);
    } else {
        if (spec) go(k_near<0, 5, 12, true>);
        else go(k_near<0, 0, 0, true>);
    }
    return cudaGetLastError();
}

}  // namespace rbsog
