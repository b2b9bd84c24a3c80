// Near field of the FP32C path with neighbour lists (Eq. 3.9, first line,
// read as -grad of U_N with N(r) = 1/r - F_M(r), plus WCA).
//
// Every particle keeps the list of the particles within r_l = r_c + skin of
// it when the list was built.  While no particle of the system has moved by
// more than skin/2 since then, every pair inside r_c is on the lists, so the
// per-step force only has to test the listed candidates (about (r_l/r_c)^3
// times the pairs) instead of a cell stencil.  The displacement test runs in
// the kick-drift kernel on the fixed-point positions; a system whose
// particles moved too far gets its cell list and neighbour lists rebuilt
// inside the same step (the rebuild kernels are gated by a device flag per
// system, so the captured step graph needs no host decision).
//
// Determinism: a system's rebuild decisions depend only on its own
// positions, and a list's order only on the cell list built from them, so a
// system's forces are the same bits alone or in any batch.  Pair terms are
// summed in list order; a run restarted from a checkpoint builds fresh lists
// at the restart step and so agrees with the continuous run to FP32 rounding
// of those sums.  Energies are summed per particle and then over blocks of
// particles in caller order.
//
// Kernels:
//   fix_pack    fixed-point caller-order positions (and the displacement
//               test) for force evaluations that do not follow a kick-drift;
//   list_build  per near-field block (home x-row segment of cells, 9 staged
//               row segments as in the cell-stencil kernel): binary-searched
//               x-windows of r_l in the x-sorted rows, candidates appended
//               to a sliced list (groups of 32 particles, slot-major inside a
//               group);
//   near_list   one thread per particle in the cell order of the last build:
//               listed partners, fixed-point differences (the 32-bit wrap is
//               the minimum image), r^2 < r_c^2, Gaussian sums from one
//               combined FP32 table; force and the two energies per particle;
//   list_clear  resets the rebuild flags after a build.
#include <cmath>
#include <type_traits>

#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kBuildThreads = 128;
constexpr int kMaxGroupB = 16;
constexpr int kMaxStagedB = 9 * (kMaxGroupB + 2);
constexpr int kNearThreads = kParticleBlock;
constexpr int kTabCopies = 8;                  // shared-memory copies of the tables (bank groups)
constexpr int kNearGroup = 4;                  // list candidates whose loads are in flight together
constexpr int kBuildGroup = 4;                 // list build: window candidates tested together

__device__ __forceinline__ int wrap_cell_b(int c, int n) {
    return c < 0 ? c + n : (c >= n ? c - n : c);
}

// Sliced list layout: particles in groups of 32 (cell-order positions s),
// each group's slots contiguous, slot k of the group's 32 particles in one
// 128-byte run: a warp reads one run per slot, and a group's entries stay in
// one compact region for the builder's scattered appends.
__device__ __forceinline__ int64_t slot_index(int64_t s, int k, int cap) {
    return ((s >> 5) * cap + k) * 32 + (s & 31);
}

__device__ __forceinline__ float offset_f(uint32_t a, uint32_t o, float scale) {
    return (float)(int32_t)(a - o) * scale;
}

__global__ void __launch_bounds__(kParticleBlock) k_fix_pack(BatchView bv, const double4_32a *__restrict__ posq,
                                                             uint4 *__restrict__ sp32c,
                                                             const uint4 *__restrict__ xref,
                                                             int32_t *__restrict__ rebuild) {
    const int2 w = bv.pblk[blockIdx.x];
    const SysDesc &d = bv.sys[w.x];
    const int64_t il = (int64_t)w.y * kParticleBlock + threadIdx.x;
    if (il >= d.n) return;
    const int64_t i = d.p_off + il;
    fixed_pack_check(d, w.x, bv.n_sys, posq[i], i, sp32c, xref, rebuild, bv.lpos, bv.linv);
}

// Neighbour lists of the home particles of one near-field block.
__global__ void __launch_bounds__(kBuildThreads) k_list_build(const BatchView bv, const int32_t *__restrict__ start,
                                                              const uint4 *__restrict__ sp32,
                                                              const int32_t *__restrict__ perm,
                                                              const int32_t *__restrict__ rebuild,
                                                              int32_t *__restrict__ nbr_list,
                                                              int32_t *__restrict__ nbr_cnt,
                                                              int32_t *__restrict__ list_perm,
                                                              uint4 *__restrict__ xref,
                                                              int32_t *__restrict__ err_flag) {
    __shared__ int s_off[kMaxStagedB + 1];
    __shared__ int s_src[kMaxStagedB];
    __shared__ int s_hstart[kMaxGroupB + 1];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int2 work = bv.nblk[blockIdx.x];
    if (!rebuild[work.x]) return;                              // this system keeps its lists
    if (bv.remaining && bv.remaining[work.x] == 0) return;
    const SysDesc &desc = bv.sys[work.x];
    const BoxDev &box = desc.box;
    const int group = desc.group, nseg_x = desc.nseg_x, cap = desc.near_cap;
    const int lcap = bv.list_cap;
    // [cap] staged partners: offsets from the block centre and, in w, the
    // particle's cell-order index (as bits)
    float4 *__restrict__ st = reinterpret_cast<float4 *>(smem_raw);
    const int64_t coff = desc.c_off;
    const int nx = box.nc[0], ny = box.nc[1], nz = box.nc[2];
    const int sx = work.y % nseg_x, row = work.y / nseg_x;
    const int cy = row % ny, cz = row / ny;
    const int x0 = sx * group, xe = min(x0 + group, nx), nh = xe - x0, w = nh + 2;
    const int ns = 9 * w;
    for (int k = tid; k < ns; k += kBuildThreads) {
        const int r = k / w, xi = k % w;
        const int zz = wrap_cell_b(cz + r / 3 - 1, nz);
        const int yy = wrap_cell_b(cy + r % 3 - 1, ny);
        const int xx = wrap_cell_b(x0 - 1 + xi, nx);
        const int64_t id = coff + (zz * ny + yy) * nx + xx;
        const int b = start[id];
        s_src[k] = b;
        s_off[k + 1] = start[id + 1] - b;
    }
    if (tid <= nh) s_hstart[tid] = start[coff + (cz * ny + cy) * nx + x0 + tid];
    if (tid == 0) s_off[0] = 0;
    __syncthreads();
    if (wid == 0) {
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
    const uint32_t ox = (uint32_t)__float2ull_rn(((float)x0 + 0.5f * (float)nh) * box.cell_fix[0]);
    const uint32_t oy = (uint32_t)__float2ull_rn(((float)cy + 0.5f) * box.cell_fix[1]);
    const uint32_t oz = (uint32_t)__float2ull_rn(((float)cz + 0.5f) * box.cell_fix[2]);
    const float fsx = box.fix_scale[0], fsy = box.fix_scale[1], fsz = box.fix_scale[2];
    const float hx = box.h_f[0], hy = box.h_f[1], hz = box.h_f[2];
    const float inv_hx = 1.0f / hx, xbase = 1.0f + 0.5f * (float)nh;
    const float rl2 = box.rl2_f;
    constexpr float kMargin = 1e-3f;

    for (int rb = hb; rb < he; rb += kBuildThreads) {   // rounds of home particles
        const int hi = rb + tid;
        const bool active = hi < he;
        float ix = 1e30f, iy = 1e30f, iz = 1e30f;
        if (active) {
            const uint4 u = sp32[hi];
            ix = offset_f(u.x, ox, fsx);
            iy = offset_f(u.y, oy, fsy);
            iz = offset_f(u.z, oz, fsz);
        }
        int cnt = 0;
        bool over = false;
        // slot k of this particle's list is lrow[32 k] (sliced layout)
        int32_t *__restrict__ lrow = nbr_list + slot_index(active ? hi : hb, 0, lcap);
        for (int c0 = 0; c0 < total; c0 += cap) {
            const int c1 = min(c0 + cap, total);
            __syncthreads();
            for (int r = 0; r < 9; ++r) {
                const int k = r * w;
                const int plo[3] = {s_off[k], s_off[k + 1], s_off[k + w - 1]};
                const int phi[3] = {s_off[k + 1], s_off[k + w - 1], s_off[k + w]};
                const int psrc[3] = {s_src[k], s_src[k + 1], s_src[k + w - 1]};
                for (int pp = 0; pp < 3; ++pp) {
                    const int a = max(plo[pp], c0), b = min(phi[pp], c1);
                    for (int t = a + tid; t < b; t += kBuildThreads) {
                        const int src = psrc[pp] + (t - plo[pp]);
                        const uint4 u = sp32[src];
                        st[t - c0] = make_float4(offset_f(u.x, ox, fsx), offset_f(u.y, oy, fsy),
                                                 offset_f(u.z, oz, fsz), __int_as_float(src));
                    }
                }
            }
            __syncthreads();
            if (!active) continue;
            for (int r = 0; r < 9; ++r) {
                const int dyr = r % 3 - 1, dzr = r / 3 - 1;
                const float gy = dyr == 0 ? 0.f : fmaxf((dyr < 0 ? iy + 0.5f * hy : 0.5f * hy - iy) - kMargin, 0.f);
                const float gz = dzr == 0 ? 0.f : fmaxf((dzr < 0 ? iz + 0.5f * hz : 0.5f * hz - iz) - kMargin, 0.f);
                const float b2 = rl2 - gy * gy - gz * gz;
                if (!(b2 > 0.f)) continue;
                const float bb = sqrtf(b2) + kMargin;
                const float xl = ix - bb, xr = ix + bb;
                const int k0 = r * w;
                const int cl = min(max((int)floorf(fmaf(xl, inv_hx, xbase)), 0), w - 1);
                const int ch = min(max((int)floorf(fmaf(xr, inv_hx, xbase)), 0), w - 1);
                int a = max(s_off[k0 + cl], c0), e = min(s_off[k0 + cl + 1], c1);
                while (a < e) {
                    const int m = (a + e) >> 1;
                    if (st[m - c0].x < xl) a = m + 1; else e = m;
                }
                // a cell range that lies wholly after the staged chunk leaves
                // its bound at or past c1: the run is clamped to the chunk
                const int lo = min(a, c1);
                a = max(s_off[k0 + ch], c0);
                e = min(s_off[k0 + ch + 1], c1);
                while (a < e) {
                    const int m = (a + e) >> 1;
                    if (st[m - c0].x <= xr) a = m + 1; else e = m;
                }
                a = min(a, c1);
                // candidates kBuildGroup at a time (independent loads and
                // distance tests in flight), appended in window order
                auto append = [&](const float4 &pj) {
                    const float dx = ix - pj.x, dy = iy - pj.y, dz = iz - pj.z;
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    if (r2 < rl2 && r2 > 0.f) {
                        if (cnt < lcap) lrow[(int64_t)cnt * 32] = __float_as_int(pj.w);
                        else over = true;
                        ++cnt;
                    }
                };
                int t = lo;
                for (; t + kBuildGroup <= a; t += kBuildGroup) {
                    float4 p[kBuildGroup];
#pragma unroll
                    for (int u = 0; u < kBuildGroup; ++u) p[u] = st[t + u - c0];
#pragma unroll
                    for (int u = 0; u < kBuildGroup; ++u) append(p[u]);
                }
                for (; t < a; ++t) append(st[t - c0]);
            }
        }
        if (active) {
            if (over) {
                atomicOr(err_flag, 4);
                cnt = lcap;
            }
            nbr_cnt[hi] = cnt;
            const int ci = perm[hi];
            const uint4 u = sp32[hi];
            list_perm[hi] = ci;
            bv.linv[ci] = hi;
            bv.lpos[hi] = u;
            xref[ci] = u;
        }
    }
}

// Pair force and energies from the neighbour lists, one thread per particle
// (cell order of the last build); results in caller order.  Positions are
// read in that cell order (lpos): the thread's own position is a coalesced
// load and its partners' lie in the few cell rows around it.
// G and F come from one combined table (one 16-byte entry per pair, see
// NearSog), held in shared memory in 8 copies, copy c of entry k at 8 k + c:
// lane l reads copy l % 8, so the 8 lanes of each quarter warp fetch their
// entries from 8 different bank groups whatever the entries are (one
// shared-memory wavefront per quarter warp).
//
// CORESHELL: the paper's core-shell kernel (Sec. 3.4) instead of the combined
// table: pairs with r^2 < r_in^2 take G and F from their Taylor series in r^2
// (Eqs. 3.25-3.26, coefficients with the series' signs in cs), 1/r and
// 1/r^3 exact; the others take the whole kernel (force factor and pair
// energy) from a table indexed by the low exponent bits and 8 high mantissa
// bits of the FP32 r^2, linearly interpolated by the remaining 15 mantissa
// bits (entries: value at the bin start and change over the bin).
//
// energy = 0: the two pair energies are left out (written as zero) except in
// systems taking their last budgeted step; the force arithmetic is the same
// instructions either way, so the forces do not depend on the flag.
template <bool CORESHELL>
__global__ void __launch_bounds__(kNearThreads, 4) k_near_list(const BatchView bv, const float ltab_scale,
                                                            const float ltab_h, const float4 *__restrict__ ltab,
                                                            const __grid_constant__ CoreShellDev cs,
                                                            const int32_t *__restrict__ nbr_list,
                                                            const int32_t *__restrict__ nbr_cnt,
                                                            const int32_t *__restrict__ list_perm,
                                                            double4_32a *__restrict__ fnear, const int energy) {
    extern __shared__ __align__(16) float4 s_tab[];
    const int2 w = bv.pblk[blockIdx.x];
    if (bv.remaining && bv.remaining[w.x] == 0) return;
    const bool want_e = energy != 0 || (bv.remaining && bv.remaining[w.x] == 1);
    // consecutive threads fill consecutive 16-byte slots (no bank conflicts)
    if (CORESHELL) {
        for (int t = threadIdx.x; t < cs.n_tab; t += kNearThreads) s_tab[t] = ltab[t];
    } else {
        for (int t = threadIdx.x; t < kLTabN * kTabCopies; t += kNearThreads) s_tab[t] = ltab[t / kTabCopies];
    }
    __syncthreads();
    const float4 *__restrict__ tab = CORESHELL ? s_tab : s_tab + (threadIdx.x & (kTabCopies - 1));
    const SysDesc &d = bv.sys[w.x];
    const int64_t sl = (int64_t)w.y * kParticleBlock + threadIdx.x;
    if (sl >= d.n) return;
    const BoxDev &box = d.box;
    const int64_t s = d.p_off + sl;
    const uint4 *__restrict__ lpos = bv.lpos;
    const uint4 pi = lpos[s];
    const float qi = box.lB_f * __uint_as_float(pi.w);
    const float fsx = box.fix_scale[0], fsy = box.fix_scale[1], fsz = box.fix_scale[2];
    const float rc2 = box.rc2_f, wrc2 = box.wca_rc2_f, ws2 = box.wca_s2_f, weps = box.wca_eps_f;
    const float tscale = ltab_scale, mh = -ltab_h;
    const int cnt = min(nbr_cnt[s], bv.list_cap);
    constexpr int64_t stride = 32;
    // the step without energies and the step with them: one instantiation of
    // the loop each, chosen per block
    auto run = [&](auto e_tag) {
        constexpr bool E = decltype(e_tag)::value;
        float fx = 0.f, fy = 0.f, fz = 0.f, un = 0.f, uw = 0.f;
        // candidates in groups of kNearGroup: their list words, then their
        // positions, are in flight together (the loads, not the arithmetic,
        // set the pace)
        auto pair = [&](const uint4 &pj) {
            const float dx = offset_f(pi.x, pj.x, fsx), dy = offset_f(pi.y, pj.y, fsy), dz = offset_f(pi.z, pj.z, fsz);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (r2 < rc2) {
                const float qq = qi * __uint_as_float(pj.w);
                float g, inv_r2;
                if (CORESHELL) {
                    if (r2 < cs.rin2) {
                        float gs = cs.a[kCsQ - 1], fs = cs.b[kCsQ];
#pragma unroll
                        for (int i = kCsQ - 2; i >= 0; --i) gs = fmaf(gs, r2, cs.a[i]);
                        if constexpr (E) {
#pragma unroll
                            for (int i = kCsQ - 1; i >= 0; --i) fs = fmaf(fs, r2, cs.b[i]);
                        }
                        const float inv_r = rsqrtf(r2);
                        inv_r2 = inv_r * inv_r;
                        g = qq * (inv_r2 * inv_r - 2.0f * gs);
                        if constexpr (E) un += 0.5f * qq * (inv_r - fs);
                    } else {
                        const uint32_t bits = __float_as_uint(r2);
                        const int idx = (int)((((bits >> 23) & cs.emask) << kCsManBits) |
                                              ((bits >> (23 - kCsManBits)) & ((1u << kCsManBits) - 1u)));
                        const float fr = (float)(bits & ((1u << (23 - kCsManBits)) - 1u)) *
                                         (1.0f / (float)(1u << (23 - kCsManBits)));
                        const float4 e = tab[idx];                 // (g0, dg, n0, dn) of the bin
                        g = qq * fmaf(fr, e.y, e.x);
                        if constexpr (E) un += 0.5f * qq * fmaf(fr, e.w, e.z);
                        inv_r2 = r2 < wrc2 ? __frcp_rn(r2) : 0.f;
                    }
                } else {
                    const float x = r2 * tscale;
                    const int kt = min((int)x, kLTabN - 1);
                    const float sx = x - (float)kt;
                    const float4 e = tab[kt * kTabCopies];      // (g0, g1, g2, F at the interval start)
                    const float gs = fmaf(fmaf(e.z, sx, e.y), sx, e.x);
                    const float inv_r = rsqrtf(r2);
                    inv_r2 = inv_r * inv_r;
                    g = qq * (inv_r2 * inv_r - 2.0f * gs);
                    if constexpr (E) {
                        const float gi = fmaf(fmaf(e.z * (1.0f / 3.0f), sx, 0.5f * e.y), sx, e.x);   // (1/s) int_0^s G
                        const float fs = fmaf(mh * sx, gi, e.w);
                        un += 0.5f * qq * (inv_r - fs);
                    }
                }
                if (r2 < wrc2) {
                    // WCA from 1/r^2 (no divisions: this branch runs for some
                    // lane of most warps, so its length is paid by all lanes)
                    const float sr2 = ws2 * inv_r2;
                    const float sr6 = sr2 * sr2 * sr2;
                    g += 24.0f * weps * (2.0f * sr6 * sr6 - sr6) * inv_r2;
                    if constexpr (E) uw += 0.5f * (4.0f * weps * (sr6 * sr6 - sr6) + weps);
                }
                fx = fmaf(g, dx, fx);
                fy = fmaf(g, dy, fy);
                fz = fmaf(g, dz, fz);
            }
        };
        const int32_t *lp = nbr_list + slot_index(s, 0, bv.list_cap);
        int k = 0;
        if (cnt >= kNearGroup) {
            // the next group's list words (streamed from DRAM) are loaded
            // before this group's pairs are evaluated, so their latency
            // overlaps the arithmetic; only the position gathers (L1/L2) stay
            // exposed
            int j[kNearGroup];
#pragma unroll
            for (int u = 0; u < kNearGroup; ++u) j[u] = lp[u * stride];
            for (; k + kNearGroup <= cnt; k += kNearGroup) {
                uint4 p[kNearGroup];
#pragma unroll
                for (int u = 0; u < kNearGroup; ++u) p[u] = lpos[j[u]];
                if (k + 2 * kNearGroup <= cnt) {
#pragma unroll
                    for (int u = 0; u < kNearGroup; ++u) j[u] = lp[(int64_t)(k + kNearGroup + u) * stride];
                }
#pragma unroll
                for (int u = 0; u < kNearGroup; ++u) pair(p[u]);
            }
        }
        for (; k < cnt; ++k) pair(lpos[lp[(int64_t)k * stride]]);
        // the two energies travel in the w slot as a pair of floats
        fnear[list_perm[s]] = make_double4_32a((double)fx, (double)fy, (double)fz,
                                               __hiloint2double(__float_as_int(un), __float_as_int(uw)));
    };
    if (want_e) run(std::true_type{});
    else run(std::false_type{});
}

// One running system's lists, reference positions and flag moved from one
// batch layout (particles at old_off, lists of old_cap slots) to another; a
// list longer than the new capacity flags the system for a rebuild instead.
__global__ void __launch_bounds__(256) k_list_move(int64_t n, int64_t old_off, int64_t new_off, int old_cap,
                                                   int new_cap, const int32_t *__restrict__ old_list,
                                                   const int32_t *__restrict__ old_cnt,
                                                   const int32_t *__restrict__ old_perm,
                                                   const uint4 *__restrict__ old_xref,
                                                   const int32_t *__restrict__ old_linv, int32_t *__restrict__ new_list,
                                                   int32_t *__restrict__ new_cnt, int32_t *__restrict__ new_perm,
                                                   uint4 *__restrict__ new_xref, int32_t *__restrict__ new_linv,
                                                   int32_t *__restrict__ new_flag) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int cnt = old_cnt[old_off + s];
    const int64_t shift = new_off - old_off;
    new_xref[new_off + s] = old_xref[old_off + s];
    new_linv[new_off + s] = (int32_t)(old_linv[old_off + s] + shift);
    if (cnt > new_cap) {
        new_cnt[new_off + s] = 0;
        new_perm[new_off + s] = (int32_t)(new_off + s);
        *new_flag = 1;
        return;
    }
    new_cnt[new_off + s] = cnt;
    new_perm[new_off + s] = (int32_t)(old_perm[old_off + s] + shift);
    for (int k = 0; k < cnt; ++k)
        new_list[slot_index(new_off + s, k, new_cap)] =
            (int32_t)(old_list[slot_index(old_off + s, k, old_cap)] + shift);
}

// Inside a captured step: the rebuild branch becomes a conditional graph
// node whose condition is the 'any system' flag of the displacement test.
__global__ void k_rebuild_condition(cudaGraphConditionalHandle h, const int32_t *__restrict__ any) {
    cudaGraphSetConditional(h, *any ? 1u : 0u);
}

// Clears the per-system flags and the 'any system' flag after a build and
// counts the builds that ran (rebuild[n_sys + 1]).
__global__ void k_list_clear(int n_sys, int32_t *__restrict__ rebuild) {
    const int any = threadIdx.x == 0 ? rebuild[n_sys] : 0;
    __syncthreads();
    for (int s = threadIdx.x; s <= n_sys; s += blockDim.x) rebuild[s] = 0;
    if (threadIdx.x == 0 && any) rebuild[n_sys + 1] += 1;
}

}  // namespace

cudaError_t launch_rebuild_condition(cudaGraphConditionalHandle h, const int32_t *any, cudaStream_t st) {
    k_rebuild_condition<<<1, 1, 0, st>>>(h, any);
    return cudaGetLastError();
}

size_t list_build_smem(int cap, int list_cap) {
    (void)list_cap;
    return sizeof(float4) * (size_t)cap;
}

cudaError_t launch_fix_pack(const BatchView &bv, const double4_32a *posq, uint4 *sp32c, const uint4 *xref,
                            int32_t *rebuild, cudaStream_t st, const Prof *prof) {
    ProfScope ps(prof, "fix_pack");
    k_fix_pack<<<bv.n_pblk, kParticleBlock, 0, st>>>(bv, posq, sp32c, xref, rebuild);
    return cudaGetLastError();
}

cudaError_t launch_list_build(const BatchView &bv, const int32_t *start, const uint4 *sp32, const int32_t *perm,
                              const int32_t *rebuild, int32_t *nbr_list, int32_t *nbr_cnt, int32_t *list_perm,
                              uint4 *xref, int32_t *err_flag, cudaStream_t st, const Prof *prof) {
    ProfScope ps(prof, "list_build");
    const size_t sm = list_build_smem(bv.max_cap, bv.list_cap);
    cudaError_t e = cudaFuncSetAttribute(k_list_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_list_build<<<bv.n_nblk, kBuildThreads, sm, st>>>(bv, start, sp32, perm, rebuild, nbr_list, nbr_cnt, list_perm,
                                                       xref, err_flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_list_clear<<<1, 64, 0, st>>>(bv.n_sys, const_cast<int32_t *>(rebuild));
    return cudaGetLastError();
}

cudaError_t launch_list_move(int64_t n, int64_t old_off, int64_t new_off, int old_cap, int new_cap,
                             const int32_t *old_list, const int32_t *old_cnt, const int32_t *old_perm,
                             const uint4 *old_xref, const int32_t *old_linv, int32_t *new_list,
                             int32_t *new_cnt, int32_t *new_perm, uint4 *new_xref, int32_t *new_linv,
                             int32_t *new_flag, cudaStream_t st) {
    k_list_move<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, old_off, new_off, old_cap, new_cap,
                                                             old_list, old_cnt, old_perm, old_xref, old_linv,
                                                             new_list, new_cnt, new_perm, new_xref, new_linv,
                                                             new_flag);
    return cudaGetLastError();
}

cudaError_t launch_near_list(const BatchView &bv, const NearSog &sog, const float4 *ltab, const int32_t *nbr_list,
                             const int32_t *nbr_cnt, const int32_t *list_perm, double4_32a *fnear, cudaStream_t st,
                             const Prof *prof, const CoreShellDev *cs, const float4 *cstab, bool energy) {
    if (cs) {
        ProfScope ps(prof, "near_fp32c_coreshell");
        const size_t sm = sizeof(float4) * (size_t)cs->n_tab;
        cudaError_t e = cudaFuncSetAttribute(k_near_list<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_near_list<true><<<bv.n_pblk, kNearThreads, sm, st>>>(bv, 0.f, 0.f, cstab, *cs, nbr_list, nbr_cnt,
                                                               list_perm, fnear, energy ? 1 : 0);
        return cudaGetLastError();
    }
    ProfScope ps(prof, "near_fp32c");
    const CoreShellDev none{};
    k_near_list<false><<<bv.n_pblk, kNearThreads, sizeof(float4) * kLTabN * kTabCopies, st>>>(
        bv, sog.ltab_scale, sog.ltab_h, ltab, none, nbr_list, nbr_cnt, list_perm, fnear, energy ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace rbsog
