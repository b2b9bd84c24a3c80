// Near-field pair force of the SOG split (Eq. 3.9, first line, read as
// -grad of U_N with N(r) = 1/r - F_M(r) of Eq. 2.7), plus the WCA soft
// repulsion, over the device cell list.
//
// Work decomposition: a block owns `group` consecutive cells of one x-row
// (the "home" cells; in cell order their particles are contiguous).  It
// stages the 9 neighbouring row segments (x0-1 .. xe, y +-1, z +-1; every
// segment is one or two contiguous ranges of the cell-ordered arrays) into
// shared memory with coalesced 16/32-byte loads, then each thread walks the
// 27 cells around its home particle in shared memory.  Every ordered pair is
// visited from both ends (no Newton-3 atomics), so forces and the
// fixed-order energy partials are deterministic.
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
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kThreads = 128;
constexpr int kMaxGroup = 16;
constexpr int kMaxStaged = 9 * (kMaxGroup + 2);
constexpr int kCap64 = 2048;   // staged particles per chunk, FP64 (64 KiB)
constexpr int kCap32 = 3072;   // staged particles per chunk, FP32C (48 KiB)

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

template <int PREC>
__global__ void __launch_bounds__(kThreads)
    k_near(BoxDev box, NearSog sog, int group, int nseg_x, const int32_t *__restrict__ start,
           const double4_32a *__restrict__ sp64, const uint4 *__restrict__ sp32,
           double4_32a *__restrict__ fnear, double2 *__restrict__ epart, int32_t *__restrict__ nbr) {
    __shared__ int s_off[kMaxStaged + 1];
    __shared__ int s_src[kMaxStaged];
    __shared__ int s_shift[kMaxStaged];
    __shared__ int s_hstart[kMaxGroup + 1];
    __shared__ double s_red[2][kThreads / 32];
    extern __shared__ __align__(32) unsigned char smem_raw[];
    double4_32a *st64 = reinterpret_cast<double4_32a *>(smem_raw);
    float4 *st32 = reinterpret_cast<float4 *>(smem_raw);
    const int cap = PREC == 0 ? kCap64 : kCap32;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nx = box.nc[0], ny = box.nc[1], nz = box.nc[2];
    const int sx = blockIdx.x % nseg_x, row = blockIdx.x / nseg_x;
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
        const int id = (zz * ny + yy) * nx + xx;
        const int b = start[id];
        s_src[k] = b;
        s_off[k + 1] = start[id + 1] - b;   // count for now
        s_shift[k] = (shx + 1) | ((shy + 1) << 2) | ((shz + 1) << 4);
    }
    if (tid <= nh) s_hstart[tid] = start[(cz * ny + cy) * nx + x0 + tid];
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

    // FP32C origin: centre of the home segment in fixed point
    uint32_t ox = 0, oy = 0, oz = 0;
    if (PREC == 1) {
        const double cxm = ((double)x0 + 0.5 * nh) * box.h[0] / box.L[0];
        const double cym = ((double)cy + 0.5) * box.h[1] / box.L[1];
        const double czm = ((double)cz + 0.5) * box.h[2] / box.L[2];
        ox = (uint32_t)(uint64_t)(cxm * 4294967296.0);
        oy = (uint32_t)(uint64_t)(cym * 4294967296.0);
        oz = (uint32_t)(uint64_t)(czm * 4294967296.0);
    }

    double e_near = 0.0, e_wca = 0.0;
    for (int base = hb; base < he; base += kThreads) {
        const int hi = base + tid;
        const bool active = hi < he;
        int cxr = 0;
        if (active) {
            while (cxr + 1 < nh && s_hstart[cxr + 1] <= hi) ++cxr;
        }
        double4_32a pi64 = make_double4_32a(0, 0, 0, 0);
        float4 pi32 = make_float4(0, 0, 0, 0);
        if (active) {
            if (PREC == 0) {
                pi64 = sp64[hi];
            } else {
                const uint4 u = sp32[hi];
                pi32 = make_float4(fixed_offset(u.x, ox, box.fix_scale[0]),
                                   fixed_offset(u.y, oy, box.fix_scale[1]),
                                   fixed_offset(u.z, oz, box.fix_scale[2]), __uint_as_float(u.w));
            }
        }
        double fx = 0.0, fy = 0.0, fz = 0.0, un = 0.0, uw = 0.0;
        float gx = 0.f, gy = 0.f, gz = 0.f, vn = 0.f, vw = 0.f;
        int cnt = 0;
        for (int c0 = 0; c0 < total; c0 += cap) {
            const int c1 = min(c0 + cap, total);
            __syncthreads();
            for (int t = c0 + tid; t < c1; t += kThreads) {
                int lo = 0, hi2 = ns;   // largest k with s_off[k] <= t
                while (hi2 - lo > 1) {
                    const int mid = (lo + hi2) >> 1;
                    if (s_off[mid] <= t) lo = mid; else hi2 = mid;
                }
                const int src = s_src[lo] + (t - s_off[lo]);
                if (PREC == 0) {
                    st64[t - c0] = sp64[src];
                } else {
                    const uint4 u = sp32[src];
                    st32[t - c0] = make_float4(fixed_offset(u.x, ox, box.fix_scale[0]),
                                               fixed_offset(u.y, oy, box.fix_scale[1]),
                                               fixed_offset(u.z, oz, box.fix_scale[2]),
                                               __uint_as_float(u.w));
                }
            }
            __syncthreads();
            if (!active) continue;
            for (int r = 0; r < 9; ++r) {
                for (int q3 = 0; q3 < 3; ++q3) {
                    const int k = r * w + cxr + q3;
                    const int tb = max(s_off[k], c0), te = min(s_off[k + 1], c1);
                    if (tb >= te) continue;
                    const int srcb = s_src[k] - s_off[k];
                    if (PREC == 0) {
                        const int sh = s_shift[k];
                        const double lx = box.L[0] * (double)((sh & 3) - 1);
                        const double ly = box.L[1] * (double)(((sh >> 2) & 3) - 1);
                        const double lz = box.L[2] * (double)(((sh >> 4) & 3) - 1);
                        for (int t = tb; t < te; ++t) {
                            const double4_32a pj = st64[t - c0];
                            const double dx = __dsub_rn(__dsub_rn(pi64.x, pj.x), lx);
                            const double dy = __dsub_rn(__dsub_rn(pi64.y, pj.y), ly);
                            const double dz = __dsub_rn(__dsub_rn(pi64.z, pj.z), lz);
                            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                                        __dmul_rn(dz, dz));
                            if (!(r2 < box.rc2) || srcb + t == hi) continue;
                            ++cnt;
                            const double inv_r = 1.0 / sqrt(r2);
                            double fs = 0.0, gs = 0.0;
                            for (int l = 0; l < sog.n_direct; ++l) {
                                const double e = exp(-r2 * sog.inv_s2[l]);
                                fs += sog.omega[l] * e;
                                gs += sog.omega[l] * sog.inv_s2[l] * e;
                            }
                            if (sog.n_taylor > 0) {
                                double pf = sog.tay_f[sog.n_taylor - 1], pg = sog.tay_g[sog.n_taylor - 1];
                                for (int m = sog.n_taylor - 2; m >= 0; --m) {
                                    pf = pf * r2 + sog.tay_f[m];
                                    pg = pg * r2 + sog.tay_g[m];
                                }
                                fs += pf;
                                gs += pg;
                            }
                            const double qq = box.lB * pi64.w * pj.w;
                            double g = qq * (inv_r * inv_r * inv_r - 2.0 * gs);
                            un += 0.5 * qq * (inv_r - fs);
                            if (r2 < box.wca_rc2) {
                                const double sr2 = box.wca_s2 / r2;
                                const double sr6 = sr2 * sr2 * sr2;
                                g += 24.0 * box.wca_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                                uw += 0.5 * (4.0 * box.wca_eps * (sr6 * sr6 - sr6) + box.wca_eps);
                            }
                            fx += g * dx;
                            fy += g * dy;
                            fz += g * dz;
                        }
                    } else {
                        const float rc2 = (float)box.rc2;
                        const float wrc2 = (float)box.wca_rc2;
                        for (int t = tb; t < te; ++t) {
                            const float4 pj = st32[t - c0];
                            const float dx = pi32.x - pj.x, dy = pi32.y - pj.y, dz = pi32.z - pj.z;
                            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            if (!(r2 < rc2) || srcb + t == hi) continue;
                            ++cnt;
                            const float inv_r = rsqrtf(r2);
                            float fs = 0.f, gs = 0.f;
                            for (int l = 0; l < sog.n_direct; ++l) {
                                const float e = __expf(-r2 * sog.inv_s2_f[l]);
                                fs = fmaf(sog.omega_f[l], e, fs);
                                gs = fmaf(sog.omega_f[l] * sog.inv_s2_f[l], e, gs);
                            }
                            if (sog.n_taylor > 0) {
                                float pf = sog.tay_f_f[sog.n_taylor - 1], pg = sog.tay_g_f[sog.n_taylor - 1];
                                for (int m = sog.n_taylor - 2; m >= 0; --m) {
                                    pf = fmaf(pf, r2, sog.tay_f_f[m]);
                                    pg = fmaf(pg, r2, sog.tay_g_f[m]);
                                }
                                fs += pf;
                                gs += pg;
                            }
                            const float qq = (float)box.lB * pi32.w * pj.w;
                            float g = qq * (inv_r * inv_r * inv_r - 2.f * gs);
                            vn = fmaf(0.5f * qq, inv_r - fs, vn);
                            if (r2 < wrc2) {
                                const float sr2 = (float)box.wca_s2 / r2;
                                const float sr6 = sr2 * sr2 * sr2;
                                const float we = (float)box.wca_eps;
                                g += 24.f * we * (2.f * sr6 * sr6 - sr6) / r2;
                                vw += 0.5f * (4.f * we * (sr6 * sr6 - sr6) + we);
                            }
                            gx = fmaf(g, dx, gx);
                            gy = fmaf(g, dy, gy);
                            gz = fmaf(g, dz, gz);
                        }
                    }
                }
            }
        }
        if (active) {
            if (PREC == 1) {
                fx = gx;
                fy = gy;
                fz = gz;
                un = vn;
                uw = vw;
            }
            fnear[hi] = make_double4_32a(fx, fy, fz, 0.0);
            if (nbr) nbr[hi] = cnt;
            e_near += un;
            e_wca += uw;
        }
    }
    // fixed-order block reduction of the energies
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e_near += __shfl_down_sync(0xffffffffu, e_near, o);
        e_wca += __shfl_down_sync(0xffffffffu, e_wca, o);
    }
    if (lane == 0) {
        s_red[0][wid] = e_near;
        s_red[1][wid] = e_wca;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) {
            a += s_red[0][i];
            b += s_red[1][i];
        }
        epart[blockIdx.x] = make_double2(a, b);
    }
}

}  // namespace

int near_num_blocks(const BoxDev &box, int group) {
    const int nseg_x = (box.nc[0] + group - 1) / group;
    return nseg_x * box.nc[1] * box.nc[2];
}

cudaError_t launch_near(int precision, const BoxDev &box, const NearSog &sog, int group,
                        const int32_t *start, const double4_32a *sp64, const uint4 *sp32,
                        double4_32a *fnear, double2 *epart, int32_t *nbr, cudaStream_t st,
                        const Prof *prof) {
    if (group < 1 || group > kMaxGroup) return cudaErrorInvalidValue;
    static bool attr_done[2] = {false, false};
    const int nseg_x = (box.nc[0] + group - 1) / group;
    const unsigned blocks = (unsigned)(nseg_x * box.nc[1] * box.nc[2]);
    ProfScope ps(prof, precision == 0 ? "near_fp64" : "near_fp32c");
    if (precision == 0) {
        const size_t sm = sizeof(double4_32a) * kCap64;
        if (!attr_done[0]) {
            cudaFuncSetAttribute(k_near<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            attr_done[0] = true;
        }
        k_near<0><<<blocks, kThreads, sm, st>>>(box, sog, group, nseg_x, start, sp64, sp32, fnear,
                                               epart, nbr);
    } else {
        const size_t sm = sizeof(float4) * kCap32;
        if (!attr_done[1]) {
            cudaFuncSetAttribute(k_near<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            attr_done[1] = true;
        }
        k_near<1><<<blocks, kThreads, sm, st>>>(box, sog, group, nseg_x, start, sp64, sp32, fnear,
                                               epart, nbr);
    }
    return cudaGetLastError();
}

}  // namespace rbsog
