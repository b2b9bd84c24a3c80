// Random-batch far field (Sec. 3.3): structure factors of the sampled
// frequencies (Eq. 3.4) and the per-particle force of Eq. 3.24, read with the
// sign of -grad U*_F:
//   F*_i = -(lB pi^{3/2} S / (P V)) q_i sum_eta k_eta Im(e^{-i k_eta . r_i} rho(k_eta)).
//
// rho sweep  grid (particle tiles) x (k tiles: 64 in FP32C, 32 in FP64).  A
//            block stages its particle tile in shared memory with coalesced
//            16/32-byte loads; lane l of every warp owns frequency k_l of the
//            tile (FP32C: k_l and k_{l+32}, whose FP32 work runs as packed
//            f32x2 operations on one broadcast particle load) and each warp
//            sweeps a slice of the tile, reading the particle by a broadcast
//            shared-memory load.  No atomics: each block writes one partial
//            per frequency.
//            FP32C: the phase is m . X over 32-bit fixed-point positions in
//            wrapping integer arithmetic, i.e. reduced exactly modulo 2 pi;
//            cos/sin in FP32 on the reduced angle; runs of 32 terms are
//            summed in FP32 and folded into a two-sum (Knuth) compensated
//            FP32 pair per thread.
//            FP64: phase t = m . (x / L) in FP64, reduced by t - rint(t),
//            cos/sin via sincospi.
// combine    one 128-thread block per frequency sums the block partials in
//            FP64 in a fixed order and writes rho(k) plus the scatter table
//            entry (k vector, coef Re rho, coef Im rho, m).
// scatter    frequencies staged through shared memory in chunks; adds the
//            near-field force and writes the total to the particle's
//            caller-order slot.  FP64: one thread per particle.  FP32C: two
//            particles per thread (l and l + 128 of a 256-particle block), so
//            each staged frequency is read once for both and the FP32 work
//            of the two runs as packed f32x2 operations, which keeps the
//            instruction issue below the sin/cos unit's time per term.
#include <algorithm>

#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kSweepThreads = 256;          // 8 warps
constexpr int kKTile = 32;                  // frequencies per sweep block (FP64)
constexpr int kKTile32 = 64;                // frequencies per sweep block (FP32C), two per lane
constexpr int kCombineThreads = 128;        // one combine block per frequency
constexpr int kScatterThreads = kParticleBlock;
constexpr int kScatter32Threads = kParticleBlock / 2;   // two particles per thread
constexpr int kKChunk32 = 512;              // frequencies per staged chunk (FP32C, 16 KiB)
constexpr int kKChunk64 = 512;              // frequencies per staged chunk (FP64, 32 KiB)
constexpr float kTwoPiF = 6.28318530717958647f;

struct KEntry32 {       // 32 bytes, two 16-byte broadcast loads
    int32_t mx, my, mz;
    float ncre;         // -coef Re rho
    float kx, ky, kz;
    float cim;          // coef Im rho
};
struct KEntry64 {       // 64 bytes
    double kx, ky, kz, cre;
    double cim, mx, my, mz;
};

// Entry k of system s's current k-set (explicit set for a batch of one; the
// folded set, whose .w is the run length, when the sequence was folded).
__device__ __forceinline__ int4 load_m(const BatchView &bv, const SysDesc &d, int s, int k) {
    if (bv.m_explicit) return bv.m_explicit[k];
    const int4 *seq = bv.kfold ? bv.kfold : bv.kseq;
    return seq[d.k_off + bv.cursor[s] * (int64_t)bv.P + k];
}

// Entries of system s's current k-set the far-field kernels evaluate: the
// distinct runs of a folded set, otherwise all P.
__device__ __forceinline__ int set_len(const BatchView &bv, const SysDesc &d, int s) {
    return bv.kcount ? bv.kcount[d.kc_off + bv.cursor[s]] : bv.P;
}

// 1 + t in [1, 2) for a phase given as t = ph 2^-32 turns, t rounded to 23
// bits, built without an int->float conversion instruction; the angle in
// [0, 2 pi) is then (1 + t) 2 pi - 2 pi, one FMA
__device__ __forceinline__ float one_plus_turns(uint32_t ph) {
    const uint32_t r = (ph + 256u) >> 9;                       // 23-bit turns, rounded
    return __uint_as_float(0x3F800000u | r);                   // 1 + turns, exact
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ void two_sum(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

// One sweep item: particle tile sblk[item_x] against frequency tile item_y.
// Every early return is uniform over the block.
template <int PREC>
__device__ __forceinline__ void sweep_item(const BatchView &bv, const double4_32a *__restrict__ sp64,
                                           const uint4 *__restrict__ sp32, double2 *__restrict__ rho_part,
                                           int item_x, int item_y) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ double s_re[kSweepThreads / 32][kKTile32];
    __shared__ double s_im[kSweepThreads / 32][kKTile32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int2 work = bv.sblk[item_x];
    if (bv.remaining && bv.remaining[work.x] == 0) return;   // frozen system: whole item skipped
    const SysDesc &d = bv.sys[work.x];
    const int ptile = work.y;
    const int ktile = PREC == 1 ? kKTile32 : kKTile;
    const int k0 = item_y * ktile;
    const int nk = set_len(bv, d, work.x);
    if (k0 >= nk) return;                                     // beyond the folded set: whole block
    const int64_t p0 = d.p_off + (int64_t)ptile * d.tile_p;
    const int np = (int)min((int64_t)d.tile_p, d.p_off + d.n - p0);

    const int per_warp = (np + 7) / 8;
    const int jb = wid * per_warp, je = min(jb + per_warp, np);
    if (PREC == 1) {
        int4 ma = make_int4(0, 0, 0, 0), mb = ma;
        if (k0 + lane < nk) ma = load_m(bv, d, work.x, k0 + lane);
        if (k0 + lane + 32 < nk) mb = load_m(bv, d, work.x, k0 + lane + 32);
        uint4 *sp = reinterpret_cast<uint4 *>(smem_raw);
        for (int j = tid; j < np; j += kSweepThreads) sp[j] = sp32[p0 + j];
        __syncthreads();
        const float2 two_pi = f2(kTwoPiF, kTwoPiF), m_two_pi = f2(-kTwoPiF, -kTwoPiF);
        float2 re_hi = f2(0.f, 0.f), re_lo = re_hi, im_hi = re_hi, im_lo = re_hi;
        if (k0 + 32 < nk) {
            for (int j0 = jb; j0 < je; j0 += 32) {
                const int j1 = min(j0 + 32, je);
                float2 cr = f2(0.f, 0.f), ci = cr;
#pragma unroll 4
                for (int j = j0; j < j1; ++j) {
                    const uint4 p = sp[j];
                    const uint32_t ph_a = (uint32_t)ma.x * p.x + (uint32_t)ma.y * p.y + (uint32_t)ma.z * p.z;
                    const uint32_t ph_b = (uint32_t)mb.x * p.x + (uint32_t)mb.y * p.y + (uint32_t)mb.z * p.z;
                    const float2 ang = __ffma2_rn(f2(one_plus_turns(ph_a), one_plus_turns(ph_b)), two_pi, m_two_pi);
                    float s_a, c_a, s_b, c_b;
                    __sincosf(ang.x, &s_a, &c_a);
                    __sincosf(ang.y, &s_b, &c_b);
                    const float q = __uint_as_float(p.w);
                    cr = __ffma2_rn(f2(q, q), f2(c_a, c_b), cr);
                    ci = __ffma2_rn(f2(q, q), f2(s_a, s_b), ci);
                }
                two_sum(re_hi.x, re_lo.x, cr.x);
                two_sum(re_hi.y, re_lo.y, cr.y);
                two_sum(im_hi.x, im_lo.x, ci.x);
                two_sum(im_hi.y, im_lo.y, ci.y);
            }
        } else {
            // the set's last tile holds at most 32 frequencies: one per lane
            // (the same expressions, so a frequency's partial is the same bits)
            for (int j0 = jb; j0 < je; j0 += 32) {
                const int j1 = min(j0 + 32, je);
                float cr = 0.f, ci = 0.f;
#pragma unroll 4
                for (int j = j0; j < j1; ++j) {
                    const uint4 p = sp[j];
                    const uint32_t ph_a = (uint32_t)ma.x * p.x + (uint32_t)ma.y * p.y + (uint32_t)ma.z * p.z;
                    const float ang = fmaf(one_plus_turns(ph_a), kTwoPiF, -kTwoPiF);
                    float s_a, c_a;
                    __sincosf(ang, &s_a, &c_a);
                    const float q = __uint_as_float(p.w);
                    cr = fmaf(q, c_a, cr);
                    ci = fmaf(q, s_a, ci);
                }
                two_sum(re_hi.x, re_lo.x, cr);
                two_sum(im_hi.x, im_lo.x, ci);
            }
        }
        s_re[wid][lane] = (double)re_hi.x + (double)re_lo.x;
        s_im[wid][lane] = (double)im_hi.x + (double)im_lo.x;
        s_re[wid][lane + 32] = (double)re_hi.y + (double)re_lo.y;
        s_im[wid][lane + 32] = (double)im_hi.y + (double)im_lo.y;
    } else {
        int4 m = make_int4(0, 0, 0, 0);
        if (k0 + lane < nk) m = load_m(bv, d, work.x, k0 + lane);
        double4_32a *sp = reinterpret_cast<double4_32a *>(smem_raw);
        const double ilx = 1.0 / d.box.L[0], ily = 1.0 / d.box.L[1], ilz = 1.0 / d.box.L[2];
        for (int j = tid; j < np; j += kSweepThreads) {
            const double4_32a p = sp64[p0 + j];
            sp[j] = make_double4_32a(p.x * ilx, p.y * ily, p.z * ilz, p.w);
        }
        __syncthreads();
        const double mx = m.x, my = m.y, mz = m.z;
        double re = 0.0, im = 0.0;
        for (int j = jb; j < je; ++j) {
            const double4_32a p = sp[j];
            double t = fma(mx, p.x, fma(my, p.y, mz * p.z));
            t -= rint(t);
            double s, c;
            sincospi(2.0 * t, &s, &c);
            re = fma(p.w, c, re);
            im = fma(p.w, s, im);
        }
        s_re[wid][lane] = re;
        s_im[wid][lane] = im;
    }
    __syncthreads();
    // warp c sums column c (frequency k0 + c) over the 8 warps, in order
    if (tid < ktile) {
        const int k = k0 + tid;
        if (k < nk) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int w = 0; w < kSweepThreads / 32; ++w) {
                re += s_re[w][tid];
                im += s_im[w][tid];
            }
            rho_part[d.rp_off + (int64_t)k * d.n_ptiles + ptile] = make_double2(re, im);
        }
    }
}

// Full grid: block (x, y) sweeps particle tile sblk[x] against frequency
// tile y.
template <int PREC>
__global__ void __launch_bounds__(kSweepThreads)
    k_rho_sweep(BatchView bv, const double4_32a *__restrict__ sp64, const uint4 *__restrict__ sp32,
                double2 *__restrict__ rho_part) {
    sweep_item<PREC>(bv, sp64, sp32, rho_part, blockIdx.x, blockIdx.y);
}

// Persistent grid: items = (particle tile, frequency tile) pairs, n_x
// particle tiles per frequency tile; a block takes items blockIdx.x,
// blockIdx.x + gridDim.x, ..., which leaves room on each SM for a kernel
// running beside it.
template <int PREC>
__global__ void __launch_bounds__(kSweepThreads)
    k_rho_sweep_resident(BatchView bv, const double4_32a *__restrict__ sp64, const uint4 *__restrict__ sp32,
                         double2 *__restrict__ rho_part, int n_x, int n_items) {
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        sweep_item<PREC>(bv, sp64, sp32, rho_part, it % n_x, it / n_x);
        __syncthreads();   // the next item restages the shared tile
    }
}

template <int PREC>
__global__ void __launch_bounds__(kCombineThreads) k_rho_combine(BatchView bv, const double2 *__restrict__ rho_part,
                                                                 double2 *__restrict__ rho, void *__restrict__ ktab) {
    __shared__ double2 s_w[kCombineThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t gk = blockIdx.x;   // system * P + k: one block per frequency
    const int sy = (int)(gk / bv.P), k = (int)(gk % bv.P);
    if (bv.remaining && bv.remaining[sy] == 0) return;
    const SysDesc &d = bv.sys[sy];
    if (k >= set_len(bv, d, sy)) {   // past the folded set: weight 0 in the energy
        if (threadIdx.x == 0) rho[gk] = make_double2(0.0, 0.0);
        return;
    }
    const double2 *row = rho_part + d.rp_off + (int64_t)k * d.n_ptiles;
    // thread t sums tiles t, t + 128, ... in order; then the warps' trees,
    // then the 4 warps in order
    double re = 0.0, im = 0.0;
    for (int t0 = threadIdx.x; t0 < d.n_ptiles; t0 += 8 * kCombineThreads) {
        double2 v[8];   // eight loads in flight, then the adds in order
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t = t0 + u * kCombineThreads;
            v[u] = t < d.n_ptiles ? row[t] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (t0 + u * kCombineThreads < d.n_ptiles) {
                re += v[u].x;
                im += v[u].y;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) s_w[wid] = make_double2(re, im);
    __syncthreads();
    if (threadIdx.x == 0) {
        re = s_w[0].x;
        im = s_w[0].y;
#pragma unroll
        for (int w2 = 1; w2 < kCombineThreads / 32; ++w2) {
            re += s_w[w2].x;
            im += s_w[w2].y;
        }
        rho[gk] = make_double2(re, im);
        const int4 m = load_m(bv, d, sy, k);
        // 2 pi / L from the host: FP64 divisions are slow on this GPU
        const double kx = d.box.kfac[0] * m.x, ky = d.box.kfac[1] * m.y, kz = d.box.kfac[2] * m.z;
        // per-Gaussian sampling: each frequency weighted by its stratum; a
        // folded set: each distinct frequency by the length of its run
        const double coef = bv.kw ? d.coef * bv.kw[(int64_t)sy * kKwStride + m.w]
                                  : (bv.kfold ? d.coef * (double)m.w : d.coef);
        if (PREC == 1) {
            KEntry32 e;
            e.mx = m.x;
            e.my = m.y;
            e.mz = m.z;
            e.ncre = -(float)(coef * re);
            e.kx = (float)kx;
            e.ky = (float)ky;
            e.kz = (float)kz;
            e.cim = (float)(coef * im);
            reinterpret_cast<KEntry32 *>(ktab)[gk] = e;
        } else {
            KEntry64 e;
            e.kx = kx;
            e.ky = ky;
            e.kz = kz;
            e.cre = coef * re;
            e.cim = coef * im;
            e.mx = m.x;
            e.my = m.y;
            e.mz = m.z;
            reinterpret_cast<KEntry64 *>(ktab)[gk] = e;
        }
    }
}

// Particle l of a scatter block: far force (already multiplied by q) plus the
// near-field force, checked and stored in caller order (returned as well).
__device__ __forceinline__ double4_32a store_total(int64_t s, double fx, double fy, double fz,
                                                   const double4_32a &fn, const int32_t *__restrict__ perm,
                                                   double4_32a *__restrict__ force, int32_t *__restrict__ err_flag) {
    const double tx = fx + fn.x, ty = fy + fn.y, tz = fz + fn.z;
    if (!(isfinite(tx) && isfinite(ty) && isfinite(tz))) atomicOr(err_flag, 1);
    const double4_32a t = make_double4_32a(tx, ty, tz, 0.0);
    force[perm ? perm[s] : s] = t;
    return t;
}

// The step's second half kick of one particle, v += dt/2 F/m, and its FP32C
// kinetic-energy term: the same expressions as the kick kernel, so that the
// fused and the separate kick give the same bits.
__device__ __forceinline__ float kick_one(double4_32a *__restrict__ vel, int64_t i, const double4_32a &f,
                                          const SysDesc &a) {
    double4_32a v = vel[i];
    const double h = a.half_dt_inv_mass;
    v.x += h * f.x;
    v.y += h * f.y;
    v.z += h * f.z;
    vel[i] = v;
    return (float)fma(v.z, v.z, fma(v.y, v.y, v.x * v.x)) * a.half_mass_f;
}

// The second half kick of this step (as kick_one, returning its kinetic
// term), then the next step's half kick and drift with the force just formed
// (the expressions of the kick-drift kernel, so the same bits as launching
// it): positions folded into the box, the fixed-point pack and displacement
// test for the next step's neighbour lists.
__device__ __forceinline__ float kick_drift_one(double4_32a *__restrict__ vel, int64_t i, const double4_32a &f,
                                                const SysDesc &a, int sys, const BatchView &bv,
                                                const DriftOut &dr) {
    double4_32a v = vel[i];
    const double h = a.half_dt_inv_mass;
    v.x += h * f.x;
    v.y += h * f.y;
    v.z += h * f.z;
    const float ke = (float)fma(v.z, v.z, fma(v.y, v.y, v.x * v.x)) * a.half_mass_f;
    v.x += h * f.x;
    v.y += h * f.y;
    v.z += h * f.z;
    double4_32a p = dr.posq[i];
    p.x += a.dt * v.x;
    p.y += a.dt * v.y;
    p.z += a.dt * v.z;
    fold_into_box(p, a.box);
    vel[i] = v;
    dr.posq[i] = p;
    fixed_pack_check(a, sys, bv.n_sys, p, i, dr.sp32c, dr.xref, dr.rebuild, bv.lpos, bv.linv);
    return ke;
}

// The two near energies of a particle packed in fn.w (neighbour-list path),
// summed over a warp's 32 particles by an FP32 tree.
__device__ __forceinline__ float2 warp_energy(bool active, const double4_32a &fn) {
    float en = 0.f, ew = 0.f;
    if (active) {
        en = __int_as_float(__double2hiint(fn.w));
        ew = __int_as_float(__double2loint(fn.w));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        en += __shfl_down_sync(0xffffffffu, en, o);
        ew += __shfl_down_sync(0xffffffffu, ew, o);
    }
    return f2(en, ew);
}

__global__ void __launch_bounds__(kScatterThreads)
    k_far_scatter64(BatchView bv, const double4_32a *__restrict__ sp64, const void *__restrict__ ktab_all,
                    const double4_32a *__restrict__ fnear, const int32_t *__restrict__ perm,
                    double4_32a *__restrict__ force, int32_t *__restrict__ err_flag, double2 *__restrict__ epart) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ double2 s_e[kScatterThreads / 32];
    const int tid = threadIdx.x;
    const int2 work = bv.pblk[blockIdx.x];
    if (bv.remaining && bv.remaining[work.x] == 0) return;   // frozen system: whole block leaves
    const SysDesc &d = bv.sys[work.x];
    const int64_t sl = (int64_t)work.y * kScatterThreads + tid;
    const int64_t s = d.p_off + sl;
    const bool active = sl < d.n;
    const int P = set_len(bv, d, work.x);
    double4_32a *sk = reinterpret_cast<double4_32a *>(smem_raw);
    const double4_32a *kt = reinterpret_cast<const double4_32a *>(ktab_all) + 2 * (int64_t)work.x * bv.P;
    double4_32a p = make_double4_32a(0, 0, 0, 0);
    if (active) p = sp64[s];
    const double ux = p.x / d.box.L[0], uy = p.y / d.box.L[1], uz = p.z / d.box.L[2];
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int c0 = 0; c0 < P; c0 += kKChunk64) {
        const int nk = min(kKChunk64, P - c0);
        __syncthreads();
        for (int t = tid; t < 2 * nk; t += kScatterThreads) sk[t] = kt[2 * c0 + t];
        __syncthreads();
        for (int e = 0; e < nk; ++e) {
            const double4_32a e0 = sk[2 * e], e1 = sk[2 * e + 1];
            double t = fma(e1.y, ux, fma(e1.z, uy, e1.w * uz));
            t -= rint(t);
            double sn, cs;
            sincospi(2.0 * t, &sn, &cs);
            const double im = cs * e1.x - sn * e0.w;
            gx = fma(e0.x, im, gx);
            gy = fma(e0.y, im, gy);
            gz = fma(e0.z, im, gz);
        }
    }
    if (bv.force_mask && !bv.force_mask[work.x]) return;   // whole block
    double4_32a fn = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (active) fn = fnear[s];
    if (!perm) {
        // caller order: one energy partial per particle block (warp trees in
        // FP32, then the warps in FP64, in order)
        const float2 e = warp_energy(active, fn);
        if ((tid & 31) == 0) s_e[tid >> 5] = make_double2((double)e.x, (double)e.y);
        __syncthreads();
        if (tid == 0) {
            double2 t = s_e[0];
            for (int w2 = 1; w2 < kScatterThreads / 32; ++w2) {
                t.x += s_e[w2].x;
                t.y += s_e[w2].y;
            }
            epart[d.e_off + work.y] = t;
        }
    }
    if (active) store_total(s, p.w * gx, p.w * gy, p.w * gz, fn, perm, force, err_flag);
}

// FP32C: thread t of a block owns particles l = t and l = t + 128 of the
// block's 256.  Per frequency both phases are exact 32-bit fixed-point dot
// products; angle, the imaginary part and the three accumulations of the two
// particles run as f32x2 operations (each lane of such an operation rounds
// like the scalar one, so a particle's force is the same as when one thread
// handles it alone).
__global__ void __launch_bounds__(kScatter32Threads, 9)
    k_far_scatter32(BatchView bv, const uint4 *__restrict__ sp32, const float4 *__restrict__ ktab_all,
                    const double4_32a *__restrict__ fnear, const int32_t *__restrict__ perm,
                    double4_32a *__restrict__ force, int32_t *__restrict__ err_flag, double2 *__restrict__ epart,
                    double4_32a *__restrict__ vel, double *__restrict__ kpart, const DriftOut drift) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ double2 s_e[kParticleBlock / 32];
    __shared__ double s_k[kParticleBlock / 32];
    float4 *sk = reinterpret_cast<float4 *>(smem_raw);
    const int tid = threadIdx.x;
    const int2 work = bv.pblk[blockIdx.x];
    if (bv.remaining && bv.remaining[work.x] == 0) return;   // frozen system: whole block leaves
    const SysDesc &d = bv.sys[work.x];
    const int P = set_len(bv, d, work.x);
    const int64_t la = (int64_t)work.y * kParticleBlock + tid, lb = la + kScatter32Threads;
    const bool act_a = la < d.n, act_b = lb < d.n;
    const int64_t sa = d.p_off + la, sb = d.p_off + lb;
    uint4 pa = make_uint4(0, 0, 0, 0), pb = pa;
    if (act_a) pa = sp32[sa];
    if (act_b) pb = sp32[sb];
    const float4 *kt = ktab_all + 2 * (int64_t)work.x * bv.P;
    const float2 two_pi = f2(kTwoPiF, kTwoPiF), m_two_pi = f2(-kTwoPiF, -kTwoPiF);
    float2 gx = f2(0.f, 0.f), gy = gx, gz = gx;
    for (int c0 = 0; c0 < P; c0 += kKChunk32) {
        const int nk = min(kKChunk32, P - c0);
        __syncthreads();
        for (int t = tid; t < 2 * nk; t += kScatter32Threads) sk[t] = kt[2 * c0 + t];
        __syncthreads();
#pragma unroll 4
        for (int e = 0; e < nk; ++e) {
            const float4 e0 = sk[2 * e], e1 = sk[2 * e + 1];
            const uint32_t mx = __float_as_uint(e0.x), my = __float_as_uint(e0.y), mz = __float_as_uint(e0.z);
            const uint32_t ph_a = mx * pa.x + my * pa.y + mz * pa.z;
            const uint32_t ph_b = mx * pb.x + my * pb.y + mz * pb.z;
            const float2 ang = __ffma2_rn(f2(one_plus_turns(ph_a), one_plus_turns(ph_b)), two_pi, m_two_pi);
            float sn_a, cs_a, sn_b, cs_b;
            __sincosf(ang.x, &sn_a, &cs_a);
            __sincosf(ang.y, &sn_b, &cs_b);
            // Im(e^{-i k.r} rho) times coef: cos * coef Im - sin * coef Re
            const float2 im = __ffma2_rn(f2(cs_a, cs_b), f2(e1.w, e1.w), __fmul2_rn(f2(sn_a, sn_b), f2(e0.w, e0.w)));
            gx = __ffma2_rn(f2(e1.x, e1.x), im, gx);
            gy = __ffma2_rn(f2(e1.y, e1.y), im, gy);
            gz = __ffma2_rn(f2(e1.z, e1.z), im, gz);
        }
    }
    if (bv.force_mask && !bv.force_mask[work.x]) return;   // whole block
    double4_32a fa = make_double4_32a(0.0, 0.0, 0.0, 0.0), fb = fa;
    if (act_a) fa = fnear[sa];
    if (act_b) fb = fnear[sb];
    if (!perm) {
        // caller order: one energy partial per 256-particle block, an FP32
        // tree per 32 particles, then the eight trees in FP64 in particle
        // order (warp w holds particles 32w.. and 128 + 32w..)
        const float2 e_a = warp_energy(act_a, fa), e_b = warp_energy(act_b, fb);
        const int w = tid >> 5;
        if ((tid & 31) == 0) {
            s_e[w] = make_double2((double)e_a.x, (double)e_a.y);
            s_e[w + kScatter32Threads / 32] = make_double2((double)e_b.x, (double)e_b.y);
        }
        __syncthreads();
        if (tid == 0) {
            double2 t = s_e[0];
            for (int w2 = 1; w2 < kParticleBlock / 32; ++w2) {
                t.x += s_e[w2].x;
                t.y += s_e[w2].y;
            }
            epart[d.e_off + work.y] = t;
        }
    }
    const float qa = __uint_as_float(pa.w), qb = __uint_as_float(pb.w);
    double4_32a ta = fa, tb = fb;
    if (act_a)
        ta = store_total(sa, (double)(qa * gx.x), (double)(qa * gy.x), (double)(qa * gz.x), fa, perm, force, err_flag);
    if (act_b)
        tb = store_total(sb, (double)(qb * gx.y), (double)(qb * gy.y), (double)(qb * gz.y), fb, perm, force, err_flag);
    if (vel) {
        // the step's second half kick with the force just formed, and the
        // block's kinetic energy summed as the kick kernel sums it: an FP32
        // tree per 32 particles (warp w holds 32w.. and 128 + 32w..), then
        // the eight trees in FP64 in particle order
        float ka = 0.f, kb = 0.f;
        if (drift.posq) {   // caller order (neighbour-list path): perm is null
            if (act_a) ka = kick_drift_one(vel, sa, ta, d, work.x, bv, drift);
            if (act_b) kb = kick_drift_one(vel, sb, tb, d, work.x, bv, drift);
        } else {
            if (act_a) ka = kick_one(vel, perm ? perm[sa] : sa, ta, d);
            if (act_b) kb = kick_one(vel, perm ? perm[sb] : sb, tb, d);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ka += __shfl_down_sync(0xffffffffu, ka, o);
            kb += __shfl_down_sync(0xffffffffu, kb, o);
        }
        const int w = tid >> 5;
        if ((tid & 31) == 0) {
            s_k[w] = (double)ka;
            s_k[w + kScatter32Threads / 32] = (double)kb;
        }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < kParticleBlock / 32; ++q) t += s_k[q];
            kpart[d.kp_off + work.y] = t;
        }
    }
}

}  // namespace

void far_layout(int64_t n, int32_t P, int precision, int tile_override, int &tile_p, int &n_ptiles) {
    // default: at least ~3 waves of sweep blocks (152 SMs x 8 resident blocks)
    const int kt = precision == 1 ? kKTile32 : kKTile;
    const int nkt = (P + kt - 1) / kt;
    int tp = 2048;
    while (tp > 128 && (double)((n + tp - 1) / tp) * nkt < 152.0 * 8 * 3) tp /= 2;
    if (tile_override > 0) tp = std::min(4096, std::max(64, tile_override));
    tile_p = tp;
    n_ptiles = (int)((n + tp - 1) / tp);
}

size_t ktab_bytes(int precision, int64_t nk) {
    return (size_t)nk * (precision == 1 ? sizeof(KEntry32) : sizeof(KEntry64));
}

cudaError_t launch_rho_sweep(int precision, const BatchView &bv, const double4_32a *sp64, const uint4 *sp32,
                             double2 *rho_part, cudaStream_t st, const Prof *prof, int blocks_per_sm) {
    const int kt = precision == 1 ? kKTile32 : kKTile;
    const int nkt = (bv.P + kt - 1) / kt;
    const size_t sm = precision == 1 ? sizeof(uint4) * (size_t)bv.max_tile_p
                                     : sizeof(double4_32a) * (size_t)bv.max_tile_p;
    ProfScope ps(prof, precision == 1 ? "rho_sweep_fp32c" : "rho_sweep_fp64");
    if (blocks_per_sm > 0) {
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const int n_items = bv.n_sblk * nkt;
        const int grid = std::min(n_items, std::max(1, blocks_per_sm * sms));
        if (precision == 1) {
            cudaFuncSetAttribute(k_rho_sweep_resident<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_rho_sweep_resident<1><<<grid, kSweepThreads, sm, st>>>(bv, sp64, sp32, rho_part, bv.n_sblk, n_items);
        } else {
            cudaFuncSetAttribute(k_rho_sweep_resident<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_rho_sweep_resident<0><<<grid, kSweepThreads, sm, st>>>(bv, sp64, sp32, rho_part, bv.n_sblk, n_items);
        }
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)bv.n_sblk, (unsigned)nkt);
    if (precision == 1) {
        cudaFuncSetAttribute(k_rho_sweep<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_rho_sweep<1><<<grid, kSweepThreads, sm, st>>>(bv, sp64, sp32, rho_part);
    } else {
        cudaFuncSetAttribute(k_rho_sweep<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_rho_sweep<0><<<grid, kSweepThreads, sm, st>>>(bv, sp64, sp32, rho_part);
    }
    return cudaGetLastError();
}

cudaError_t launch_rho_combine(int precision, const BatchView &bv, const double2 *rho_part, double2 *rho,
                               void *ktab, cudaStream_t st, const Prof *prof) {
    ProfScope ps(prof, "rho_combine");
    const unsigned blocks = (unsigned)((int64_t)bv.n_sys * bv.P);
    if (precision == 1)
        k_rho_combine<1><<<blocks, kCombineThreads, 0, st>>>(bv, rho_part, rho, ktab);
    else
        k_rho_combine<0><<<blocks, kCombineThreads, 0, st>>>(bv, rho_part, rho, ktab);
    return cudaGetLastError();
}

cudaError_t launch_far_scatter(int precision, const BatchView &bv, const double4_32a *sp64, const uint4 *sp32,
                               const void *ktab, const double4_32a *fnear, const int32_t *perm,
                               double4_32a *force, int32_t *err_flag, cudaStream_t st, const Prof *prof,
                               double2 *epart, double4_32a *kick_vel, double *kick_kpart, const DriftOut *drift) {
    ProfScope ps(prof, precision == 1 ? "far_scatter_fp32c" : "far_scatter_fp64");
    if (precision == 1) {
        const size_t sm = sizeof(KEntry32) * kKChunk32;
        const DriftOut dr = (drift && kick_vel && !perm) ? *drift : DriftOut{nullptr, nullptr, nullptr, nullptr};
        k_far_scatter32<<<bv.n_pblk, kScatter32Threads, sm, st>>>(bv, sp32, static_cast<const float4 *>(ktab),
                                                                   fnear, perm, force, err_flag, epart, kick_vel,
                                                                   kick_kpart, dr);
    } else {
        const size_t sm = sizeof(KEntry64) * kKChunk64;
        k_far_scatter64<<<bv.n_pblk, kScatterThreads, sm, st>>>(bv, sp64, ktab, fnear, perm, force, err_flag,
                                                                 epart);
    }
    return cudaGetLastError();
}

}  // namespace rbsog
