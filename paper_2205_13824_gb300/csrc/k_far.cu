// Random-batch far field (Sec. 3.3): structure factors of the sampled
// frequencies (Eq. 3.4) and the per-particle force of Eq. 3.24, read with the
// sign of -grad U*_F:
//   F*_i = -(lB pi^{3/2} S / (P V)) q_i sum_eta k_eta Im(e^{-i k_eta . r_i} rho(k_eta)).
//
// rho sweep  grid (particle tiles) x (k tiles of 32).  A block stages its
//            particle tile in shared memory with coalesced 16/32-byte loads;
//            lane l of every warp owns frequency k_l of the tile and each warp
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
// combine    one warp per frequency sums the block partials in FP64 in a
//            fixed order and writes rho(k) plus the scatter table entry
//            (k vector, coef Re rho, coef Im rho, m).
// scatter    one thread per particle, frequencies staged through shared
//            memory in chunks; adds the near-field force and writes the total
//            to the particle's caller-order slot.
#include <algorithm>

#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kSweepThreads = 256;          // 8 warps
constexpr int kKTile = 32;                  // frequencies per sweep block
constexpr int kScatterThreads = kParticleBlock;
constexpr int kKChunk32 = 1024;             // frequencies per staged chunk (FP32C, 32 KiB)
constexpr int kKChunk64 = 512;              // frequencies per staged chunk (FP64, 32 KiB)

struct KEntry32 {       // 32 bytes, two 16-byte broadcast loads
    int32_t mx, my, mz;
    float cre;
    float kx, ky, kz;
    float cim;
};
struct KEntry64 {       // 64 bytes
    double kx, ky, kz, cre;
    double cim, mx, my, mz;
};

// Frequency k of system s's current k-set (explicit set for a batch of one).
__device__ __forceinline__ int4 load_m(const BatchView &bv, const SysDesc &d, int s, int k) {
    if (bv.m_explicit) return bv.m_explicit[k];
    return bv.kseq[d.k_off + bv.cursor[s] * (int64_t)bv.P + k];
}

// angle in [0, 2 pi) of a phase given in units of 2^-32 turns, rounded to
// 24 bits of turns without an int->float conversion instruction
__device__ __forceinline__ float turns_to_rad(uint32_t ph) {
    const uint32_t r = (ph + 256u) >> 9;                       // 23-bit turns, rounded
    const float f = __uint_as_float(0x3F800000u | r);          // 1 + turns
    return fmaf(f, 6.28318530717958647f, -6.28318530717958647f);
}

__device__ __forceinline__ void two_sum(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

template <int PREC>
__global__ void __launch_bounds__(kSweepThreads)
    k_rho_sweep(BatchView bv, const double4_32a *__restrict__ sp64, const uint4 *__restrict__ sp32,
                double2 *__restrict__ rho_part) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ double s_re[kSweepThreads / 32][kKTile];
    __shared__ double s_im[kSweepThreads / 32][kKTile];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int2 work = bv.sblk[blockIdx.x];
    if (bv.remaining && bv.remaining[work.x] == 0) return;   // frozen system: whole block leaves
    const SysDesc &d = bv.sys[work.x];
    const int ptile = work.y;
    const int k = blockIdx.y * kKTile + lane;
    const int64_t p0 = d.p_off + (int64_t)ptile * d.tile_p;
    const int np = (int)min((int64_t)d.tile_p, d.p_off + d.n - p0);

    int4 m = make_int4(0, 0, 0, 0);
    if (k < bv.P) m = load_m(bv, d, work.x, k);

    const int per_warp = (np + 7) / 8;
    const int jb = wid * per_warp, je = min(jb + per_warp, np);
    if (PREC == 1) {
        uint4 *sp = reinterpret_cast<uint4 *>(smem_raw);
        for (int j = tid; j < np; j += kSweepThreads) sp[j] = sp32[p0 + j];
        __syncthreads();
        const uint32_t mx = (uint32_t)m.x, my = (uint32_t)m.y, mz = (uint32_t)m.z;
        float re_hi = 0.f, re_lo = 0.f, im_hi = 0.f, im_lo = 0.f;
        for (int j0 = jb; j0 < je; j0 += 32) {
            const int j1 = min(j0 + 32, je);
            float cr = 0.f, ci = 0.f;
#pragma unroll 4
            for (int j = j0; j < j1; ++j) {
                const uint4 p = sp[j];
                const uint32_t ph = mx * p.x + my * p.y + mz * p.z;
                float s, c;
                __sincosf(turns_to_rad(ph), &s, &c);
                const float q = __uint_as_float(p.w);
                cr = fmaf(q, c, cr);
                ci = fmaf(q, s, ci);
            }
            two_sum(re_hi, re_lo, cr);
            two_sum(im_hi, im_lo, ci);
        }
        s_re[wid][lane] = (double)re_hi + (double)re_lo;
        s_im[wid][lane] = (double)im_hi + (double)im_lo;
    } else {
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
    if (wid == 0 && k < bv.P) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int w = 0; w < kSweepThreads / 32; ++w) {
            re += s_re[w][lane];
            im += s_im[w][lane];
        }
        rho_part[d.rp_off + (int64_t)k * d.n_ptiles + ptile] = make_double2(re, im);
    }
}

template <int PREC>
__global__ void __launch_bounds__(256) k_rho_combine(BatchView bv, const double2 *__restrict__ rho_part,
                                                     double2 *__restrict__ rho, void *__restrict__ ktab) {
    const int lane = threadIdx.x & 31;
    const int64_t gk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // system * P + k
    if (gk >= (int64_t)bv.n_sys * bv.P) return;
    const int sy = (int)(gk / bv.P), k = (int)(gk % bv.P);
    if (bv.remaining && bv.remaining[sy] == 0) return;
    const SysDesc &d = bv.sys[sy];
    const double2 *row = rho_part + d.rp_off + (int64_t)k * d.n_ptiles;
    double re = 0.0, im = 0.0;
    for (int t = lane; t < d.n_ptiles; t += 32) {
        const double2 v = row[t];
        re += v.x;
        im += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        rho[gk] = make_double2(re, im);
        const int4 m = load_m(bv, d, sy, k);
        const double kx = 2.0 * kPi * m.x / d.box.L[0], ky = 2.0 * kPi * m.y / d.box.L[1],
                     kz = 2.0 * kPi * m.z / d.box.L[2];
        const double coef = d.coef;
        if (PREC == 1) {
            KEntry32 e;
            e.mx = m.x;
            e.my = m.y;
            e.mz = m.z;
            e.cre = (float)(coef * re);
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

template <int PREC>
__global__ void __launch_bounds__(kScatterThreads)
    k_far_scatter(BatchView bv, const double4_32a *__restrict__ sp64, const uint4 *__restrict__ sp32,
                  const void *__restrict__ ktab_all, const double4_32a *__restrict__ fnear,
                  const int32_t *__restrict__ perm, double4_32a *__restrict__ force,
                  int32_t *__restrict__ err_flag, double2 *__restrict__ epart) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int2 work = bv.pblk[blockIdx.x];
    if (bv.remaining && bv.remaining[work.x] == 0) return;   // frozen system: whole block leaves
    const SysDesc &d = bv.sys[work.x];
    const int64_t sl = (int64_t)work.y * kScatterThreads + tid;
    const int64_t s = d.p_off + sl;
    const bool active = sl < d.n;
    const int P = bv.P;
    double fx, fy, fz;
    if (PREC == 1) {
        float4 *sk = reinterpret_cast<float4 *>(smem_raw);
        const float4 *kt = reinterpret_cast<const float4 *>(ktab_all) + 2 * (int64_t)work.x * P;
        uint4 p = make_uint4(0, 0, 0, 0);
        if (active) p = sp32[s];
        float gx = 0.f, gy = 0.f, gz = 0.f;
        for (int c0 = 0; c0 < P; c0 += kKChunk32) {
            const int nk = min(kKChunk32, P - c0);
            __syncthreads();
            for (int t = tid; t < 2 * nk; t += kScatterThreads) sk[t] = kt[2 * c0 + t];
            __syncthreads();
#pragma unroll 4
            for (int e = 0; e < nk; ++e) {
                const float4 e0 = sk[2 * e], e1 = sk[2 * e + 1];
                const uint32_t ph = (uint32_t)__float_as_int(e0.x) * p.x +
                                    (uint32_t)__float_as_int(e0.y) * p.y +
                                    (uint32_t)__float_as_int(e0.z) * p.z;
                float sn, cs;
                __sincosf(turns_to_rad(ph), &sn, &cs);
                const float im = fmaf(cs, e1.w, -sn * e0.w);
                gx = fmaf(e1.x, im, gx);
                gy = fmaf(e1.y, im, gy);
                gz = fmaf(e1.z, im, gz);
            }
        }
        const float q = __uint_as_float(p.w);
        fx = (double)(q * gx);
        fy = (double)(q * gy);
        fz = (double)(q * gz);
    } else {
        double4_32a *sk = reinterpret_cast<double4_32a *>(smem_raw);
        const double4_32a *kt = reinterpret_cast<const double4_32a *>(ktab_all) + 2 * (int64_t)work.x * P;
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
        fx = p.w * gx;
        fy = p.w * gy;
        fz = p.w * gz;
    }
    if (bv.force_mask && !bv.force_mask[work.x]) return;   // whole block
    double4_32a fn = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (active) fn = fnear[s];
    if (!perm) {
        // caller order (neighbour-list path): the block's near energies, two
        // floats per particle in fn.w, summed in fixed order (an FP32 tree
        // per warp -- FP64 adds are scarce on this GPU -- then the warps in
        // FP64, in order) into one partial per particle block
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
        __shared__ double2 s_e[kScatterThreads / 32];
        if ((tid & 31) == 0) s_e[tid >> 5] = make_double2((double)en, (double)ew);
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
    if (!active) return;
    const double tx = fx + fn.x, ty = fy + fn.y, tz = fz + fn.z;
    if (!(isfinite(tx) && isfinite(ty) && isfinite(tz))) atomicOr(err_flag, 1);
    force[perm ? perm[s] : s] = make_double4_32a(tx, ty, tz, 0.0);
}

}  // namespace

void far_layout(int64_t n, int32_t P, int tile_override, int &tile_p, int &n_ptiles) {
    // default: at least ~3 waves of sweep blocks (152 SMs x 8 resident blocks)
    const int nkt = (P + kKTile - 1) / kKTile;
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
                             double2 *rho_part, cudaStream_t st, const Prof *prof) {
    dim3 grid((unsigned)bv.n_sblk, (unsigned)((bv.P + kKTile - 1) / kKTile));
    ProfScope ps(prof, precision == 1 ? "rho_sweep_fp32c" : "rho_sweep_fp64");
    if (precision == 1) {
        const size_t sm = sizeof(uint4) * (size_t)bv.max_tile_p;
        cudaFuncSetAttribute(k_rho_sweep<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_rho_sweep<1><<<grid, kSweepThreads, sm, st>>>(bv, sp64, sp32, rho_part);
    } else {
        const size_t sm = sizeof(double4_32a) * (size_t)bv.max_tile_p;
        cudaFuncSetAttribute(k_rho_sweep<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_rho_sweep<0><<<grid, kSweepThreads, sm, st>>>(bv, sp64, sp32, rho_part);
    }
    return cudaGetLastError();
}

cudaError_t launch_rho_combine(int precision, const BatchView &bv, const double2 *rho_part, double2 *rho,
                               void *ktab, cudaStream_t st, const Prof *prof) {
    ProfScope ps(prof, "rho_combine");
    const unsigned blocks = (unsigned)(((int64_t)bv.n_sys * bv.P * 32 + 255) / 256);
    if (precision == 1)
        k_rho_combine<1><<<blocks, 256, 0, st>>>(bv, rho_part, rho, ktab);
    else
        k_rho_combine<0><<<blocks, 256, 0, st>>>(bv, rho_part, rho, ktab);
    return cudaGetLastError();
}

cudaError_t launch_far_scatter(int precision, const BatchView &bv, const double4_32a *sp64, const uint4 *sp32,
                               const void *ktab, const double4_32a *fnear, const int32_t *perm,
                               double4_32a *force, int32_t *err_flag, cudaStream_t st, const Prof *prof,
                               double2 *epart) {
    ProfScope ps(prof, precision == 1 ? "far_scatter_fp32c" : "far_scatter_fp64");
    if (precision == 1) {
        const size_t sm = sizeof(KEntry32) * kKChunk32;
        k_far_scatter<1><<<bv.n_pblk, kScatterThreads, sm, st>>>(bv, sp64, sp32, ktab, fnear, perm, force,
                                                                  err_flag, epart);
    } else {
        const size_t sm = sizeof(KEntry64) * kKChunk64;
        k_far_scatter<0><<<bv.n_pblk, kScatterThreads, sm, st>>>(bv, sp64, sp32, ktab, fnear, perm, force,
                                                                  err_flag, epart);
    }
    return cudaGetLastError();
}

}  // namespace rbsog
