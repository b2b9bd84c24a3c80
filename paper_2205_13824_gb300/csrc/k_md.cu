// Velocity-Verlet integration (Algorithm 1, line 4) with the Berendsen
// rescale, fixed-order energy reductions, and layout conversions between
// the caller's [n][3] arrays and the internal 32-byte particle records.
// All state updates are FP64 and memory-bound: one thread per particle,
// coalesced 32-byte loads and stores.
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kThreads = kParticleBlock;
constexpr int kFinThreads = 256;

// Three standard normals for the Langevin step of particle il in the step
// with step counter t: Philox4x64-10, key (seed, 2^63 + 1) (the sampler's
// chain keys stay below 2^63), counter (t, il, 0, 0); Box-Muller
// (u0, u1) -> (z_x, z_y), (u2, u3) -> z_z.  FP64 arithmetic for the FP64
// path; FP32 for FP32C, where FP64 transcendentals would dominate the step.
__device__ __forceinline__ void langevin_noise(uint64_t seed, int64_t t, int64_t il, int precision, double z[3]) {
    uint64_t c[4] = {(uint64_t)t, (uint64_t)il, 0ull, 0ull};
    philox4x64_10(c, seed, 0x8000000000000001ull);
    if (precision == 1) {
        const float u0 = (float)unit53(c[0]), u1 = (float)unit53(c[1]);
        const float u2 = (float)unit53(c[2]), u3 = (float)unit53(c[3]);
        const float r01 = sqrtf(-2.0f * logf(1.0f - u0)), r23 = sqrtf(-2.0f * logf(1.0f - u2));
        float s1, c1, s3, c3;
        sincospif(2.0f * u1, &s1, &c1);
        sincospif(2.0f * u3, &s3, &c3);
        z[0] = r01 * c1;
        z[1] = r01 * s1;
        z[2] = r23 * c3;
        (void)s3;
    } else {
        const double r01 = sqrt(-2.0 * log(1.0 - unit53(c[0]))), r23 = sqrt(-2.0 * log(1.0 - unit53(c[2])));
        double s1, c1, s3, c3;
        sincospi(2.0 * unit53(c[1]), &s1, &c1);
        sincospi(2.0 * unit53(c[3]), &s3, &c3);
        z[0] = r01 * c1;
        z[1] = r01 * s1;
        z[2] = r23 * c3;
        (void)s3;
    }
}

// v += dt/2 F/m ; x += dt v ; x folded into [0, L).
__global__ void __launch_bounds__(kThreads) k_kick_drift(BatchView bv, double4_32a *__restrict__ posq,
                                                         double4_32a *__restrict__ vel,
                                                         const double4_32a *__restrict__ force,
                                                         uint4 *__restrict__ sp32c, const uint4 *__restrict__ xref,
                                                         int32_t *__restrict__ rebuild) {
    const int2 w = bv.pblk[blockIdx.x];
    if (bv.remaining && bv.remaining[w.x] == 0) return;
    const SysDesc &a = bv.sys[w.x];
    const int64_t il = (int64_t)w.y * kThreads + threadIdx.x;
    if (il >= a.n) return;
    const int64_t i = a.p_off + il;
    const double4_32a f = force[i];
    double4_32a v = vel[i];
    double4_32a p = posq[i];
    const double h = a.half_dt_inv_mass;
    v.x += h * f.x;
    v.y += h * f.y;
    v.z += h * f.z;
    if (a.thermostat == 1) {
        // Langevin, BAOAB: half drift, Ornstein-Uhlenbeck velocity update
        // with this step's noise, half drift
        const double hd = a.half_dt;
        p.x += hd * v.x;
        p.y += hd * v.y;
        p.z += hd * v.z;
        double z[3];
        langevin_noise(a.lv_seed, bv.step[w.x], il, bv.precision, z);
        v.x = a.lv_c1 * v.x + a.lv_c2 * z[0];
        v.y = a.lv_c1 * v.y + a.lv_c2 * z[1];
        v.z = a.lv_c1 * v.z + a.lv_c2 * z[2];
        p.x += hd * v.x;
        p.y += hd * v.y;
        p.z += hd * v.z;
    } else {
        p.x += a.dt * v.x;
        p.y += a.dt * v.y;
        p.z += a.dt * v.z;
    }
    fold_into_box(p, a.box);
    vel[i] = v;
    posq[i] = p;
    if (sp32c) fixed_pack_check(a, w.x, bv.n_sys, p, i, sp32c, xref, rebuild, bv.lpos, bv.linv);
}

// v += dt/2 F/m and the block's kinetic energy sum (fixed order).
__global__ void __launch_bounds__(kThreads) k_kick(BatchView bv, double4_32a *__restrict__ vel,
                                                   const double4_32a *__restrict__ force,
                                                   double *__restrict__ kpart) {
    __shared__ double s_red[kThreads / 32];
    const int2 w = bv.pblk[blockIdx.x];
    if (bv.remaining && bv.remaining[w.x] == 0) return;
    const SysDesc &a = bv.sys[w.x];
    const int64_t il = (int64_t)w.y * kThreads + threadIdx.x;
    const int64_t i = a.p_off + il;
    double ke = 0.0;
    float kf = 0.f;
    if (il < a.n) {
        const double4_32a f = force[i];
        double4_32a v = vel[i];
        const double h = a.half_dt_inv_mass;
        v.x += h * f.x;
        v.y += h * f.y;
        v.z += h * f.z;
        vel[i] = v;
        if (bv.precision == 1)   // FP32C: |v|^2 in FP64, the rest in FP32
            kf = (float)fma(v.z, v.z, fma(v.y, v.y, v.x * v.x)) * a.half_mass_f;
        else
            ke = 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
    }
    if (bv.precision == 1) {
        // FP32C: the warp's terms in an FP32 tree (FP64 adds are scarce on
        // this GPU), the warps in FP64
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kf += __shfl_down_sync(0xffffffffu, kf, o);
        ke = (double)kf;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
    }
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) t += s_red[q];
        kpart[a.kp_off + w.y] = t;
    }
}

// kFinChunks blocks per system, each summing one chunk of the near-energy
// partials, |rho(k)|^2 and kinetic partials in fixed order (thread t takes
// the chunk's entries t, t + 256, ...; then the warps' trees; then the warps
// in order); the last block of the system to finish adds the chunk sums in
// chunk order and writes the energies, T, the Berendsen factor, the cursor
// and the step counter.  No block waits for another.
__global__ void __launch_bounds__(kFinThreads) k_finalize(BatchView bv, const double2 *__restrict__ epart,
                                                          const double2 *__restrict__ rho,
                                                          const double *__restrict__ kpart, int with_kinetic,
                                                          double *__restrict__ energy, int64_t advance) {
    __shared__ double s_red[4][kFinThreads / 32];
    __shared__ bool s_last;
    const int sy = blockIdx.x / kFinChunks, c = blockIdx.x % kFinChunks;
    if (bv.force_mask && !bv.force_mask[sy]) return;
    if (bv.remaining && bv.remaining[sy] == 0) return;
    const SysDesc &a = bv.sys[sy];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    auto chunk = [c](int len, int &lo, int &hi) {
        lo = (int)((int64_t)len * c / kFinChunks);
        hi = (int)((int64_t)len * (c + 1) / kFinChunks);
    };
    double un = 0.0, uw = 0.0, r2 = 0.0, ke = 0.0;
    int lo, hi;
    chunk(a.n_epart, lo, hi);
    for (int j = lo + tid; j < hi; j += kFinThreads) {
        const double2 e = epart[a.e_off + j];
        un += e.x;
        uw += e.y;
    }
    chunk(bv.P, lo, hi);
    if (bv.kw) {   // per-Gaussian sampling: |rho|^2 weighted by the frequency's stratum
        const int4 *ks = bv.kseq + a.k_off + bv.cursor[sy] * (int64_t)bv.P;
        for (int j = lo + tid; j < hi; j += kFinThreads) {
            const double2 r = rho[(int64_t)sy * bv.P + j];
            r2 += bv.kw[(int64_t)sy * kKwStride + ks[j].w] * (r.x * r.x + r.y * r.y);
        }
    } else if (bv.kfold) {   // a folded set: |rho|^2 of each distinct frequency times its run length
        const int4 *ks = bv.kfold + a.k_off + bv.cursor[sy] * (int64_t)bv.P;
        for (int j = lo + tid; j < hi; j += kFinThreads) {
            const double2 r = rho[(int64_t)sy * bv.P + j];
            r2 += (double)ks[j].w * (r.x * r.x + r.y * r.y);
        }
    } else {
        for (int j = lo + tid; j < hi; j += kFinThreads) {
            const double2 r = rho[(int64_t)sy * bv.P + j];
            r2 += r.x * r.x + r.y * r.y;
        }
    }
    if (with_kinetic) {
        chunk(a.n_kpart, lo, hi);
        for (int j = lo + tid; j < hi; j += kFinThreads) ke += kpart[a.kp_off + j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        un += __shfl_down_sync(0xffffffffu, un, o);
        uw += __shfl_down_sync(0xffffffffu, uw, o);
        r2 += __shfl_down_sync(0xffffffffu, r2, o);
        ke += __shfl_down_sync(0xffffffffu, ke, o);
    }
    if (lane == 0) {
        s_red[0][wid] = un;
        s_red[1][wid] = uw;
        s_red[2][wid] = r2;
        s_red[3][wid] = ke;
    }
    __syncthreads();
    if (tid == 0) {
        double t[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
            for (int w = 0; w < kFinThreads / 32; ++w) t[q] += s_red[q][w];
        bv.fin_part[sy * kFinChunks + c] = make_double4_32a(t[0], t[1], t[2], t[3]);
        __threadfence();   // the chunk sum is visible before the count says so
        s_last = atomicAdd(&bv.fin_count[sy], 1u) == kFinChunks - 1;
    }
    __syncthreads();
    if (!s_last || tid != 0) return;
    __threadfence();
    double t[4] = {0, 0, 0, 0};
    for (int q = 0; q < kFinChunks; ++q) {
        const double *v = reinterpret_cast<const double *>(bv.fin_part + sy * kFinChunks + q);
        t[0] += __ldcg(v);        // L2: written by other blocks of this launch
        t[1] += __ldcg(v + 1);
        t[2] += __ldcg(v + 2);
        t[3] += __ldcg(v + 3);
    }
    bv.fin_count[sy] = 0;   // ready for the next launch
    double *en = energy + (int64_t)sy * kNumEnergy;
    if (a.boundary == 0) en[7] = 0.0;   // boundary term: written by its own kernel when on
    en[0] = t[0];
    en[1] = a.half_coef_U * t[2];
    en[2] = a.U_self;
    en[3] = t[1];
    if (with_kinetic) {
        double K = t[3];
        double T = 2.0 * K / (3.0 * (double)a.n - 3.0);
        double lam = 1.0;
        if (a.thermostat == 0 && a.tau > 0.0 && T > 0.0) {
            lam = sqrt(1.0 + a.dt / a.tau * (a.T0 / T - 1.0));
            K *= lam * lam;
            T *= lam * lam;
        } else if (a.thermostat == 2 && a.tau > 0.0) {
            // Nose-Hoover: the end half of this step's thermostat update and
            // the start half of the next one (symmetric Trotter splitting),
            // each xi += dt/4 G; v *= e^{-xi dt/2}; eta += dt/2 xi;
            // xi += dt/4 G with G = (2K - g T0) / Q; the velocity factor is
            // applied by the rescale kernel
            const double g = 3.0 * (double)a.n - 3.0;
            double xi = en[8], eta = en[9];
            for (int h = 0; h < 2; ++h) {
                xi += 0.25 * a.dt * (2.0 * K - g * a.T0) / a.nh_Q;
                const double sc = exp(-0.5 * a.dt * xi);
                lam *= sc;
                K *= sc * sc;
                eta += 0.5 * a.dt * xi;
                xi += 0.25 * a.dt * (2.0 * K - g * a.T0) / a.nh_Q;
            }
            T = 2.0 * K / g;
            en[8] = xi;
            en[9] = eta;
            en[10] = 0.5 * a.nh_Q * xi * xi + g * a.T0 * eta;
        }
        en[4] = K;
        en[5] = T;
        en[6] = lam;
        bv.step[sy] += 1;
    }
    bv.cursor[sy] += advance;
}

__global__ void __launch_bounds__(kThreads) k_rescale(BatchView bv, double4_32a *__restrict__ vel,
                                                      const double *__restrict__ energy) {
    const int2 w = bv.pblk[blockIdx.x];
    if (bv.remaining && bv.remaining[w.x] == 0) return;
    const SysDesc &a = bv.sys[w.x];
    if (a.tau <= 0.0) return;
    const int64_t il = (int64_t)w.y * kThreads + threadIdx.x;
    if (il >= a.n) return;
    const int64_t i = a.p_off + il;
    const double lam = energy[(int64_t)w.x * kNumEnergy + 6];
    double4_32a v = vel[i];
    v.x *= lam;
    v.y *= lam;
    v.z *= lam;
    vel[i] = v;
}

__global__ void __launch_bounds__(kThreads) k_pack(int64_t n, const double *__restrict__ x3,
                                                   const double *__restrict__ q, double4_32a *__restrict__ out,
                                                   int wrap, double Lx, double Ly, double Lz) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    double x = x3 ? x3[3 * i] : 0.0, y = x3 ? x3[3 * i + 1] : 0.0, z = x3 ? x3[3 * i + 2] : 0.0;
    if (wrap) {
        x = fold(x, Lx);
        y = fold(y, Ly);
        z = fold(z, Lz);
    }
    out[i] = make_double4_32a(x, y, z, q ? q[i] : 0.0);
}

__global__ void __launch_bounds__(kThreads) k_unpack(int64_t n, const double4_32a *__restrict__ in,
                                                     double *__restrict__ x3) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const double4_32a p = in[i];
    x3[3 * i] = p.x;
    x3[3 * i + 1] = p.y;
    x3[3 * i + 2] = p.z;
}

// out[perm[off + s] - off] = sorted[off + s] for one system's range.
__global__ void __launch_bounds__(kThreads) k_unsort(int64_t n, int64_t off, const int32_t *__restrict__ perm,
                                                     const int32_t *__restrict__ sorted,
                                                     int32_t *__restrict__ out) {
    const int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (s >= n) return;
    out[perm[off + s] - off] = sorted[off + s];
}

__global__ void k_finalize_counters(BatchView bv, int64_t advance) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= bv.n_sys) return;
    if (bv.force_mask && !bv.force_mask[s]) return;
    if (bv.remaining && bv.remaining[s] == 0) return;
    bv.step[s] += 1;
    bv.cursor[s] += advance;
}

__global__ void k_step_done(int32_t n_sys, int64_t *__restrict__ remaining) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_sys && remaining[s] > 0) remaining[s] -= 1;
}

__global__ void k_m_to_int4(int32_t P, const int32_t *__restrict__ m3, int4 *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    out[k] = make_int4(m3[3 * k], m3[3 * k + 1], m3[3 * k + 2], 0);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_kick_drift(const BatchView &bv, double4_32a *posq, double4_32a *vel, const double4_32a *force,
                              cudaStream_t st, const Prof *prof, uint4 *sp32c, const uint4 *xref, int32_t *rebuild) {
    ProfScope ps(prof, "kick_drift");
    k_kick_drift<<<bv.n_pblk, kThreads, 0, st>>>(bv, posq, vel, force, sp32c, xref, rebuild);
    return cudaGetLastError();
}

cudaError_t launch_kick(const BatchView &bv, double4_32a *vel, const double4_32a *force, double *kpart,
                        cudaStream_t st, const Prof *prof) {
    ProfScope ps(prof, "kick");
    k_kick<<<bv.n_pblk, kThreads, 0, st>>>(bv, vel, force, kpart);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const BatchView &bv, const double2 *epart, const double2 *rho, const double *kpart,
                            int with_kinetic, double *energy, int64_t advance, cudaStream_t st, const Prof *prof) {
    ProfScope ps(prof, "finalize");
    k_finalize<<<bv.n_sys * kFinChunks, kFinThreads, 0, st>>>(bv, epart, rho, kpart, with_kinetic, energy,
                                                               advance);
    return cudaGetLastError();
}

cudaError_t launch_finalize_counters(const BatchView &bv, int64_t advance, cudaStream_t st, const Prof *prof) {
    ProfScope ps(prof, "finalize");
    k_finalize_counters<<<(unsigned)((bv.n_sys + 127) / 128), 128, 0, st>>>(bv, advance);
    return cudaGetLastError();
}

cudaError_t launch_rescale(const BatchView &bv, double4_32a *vel, const double *energy, cudaStream_t st,
                           const Prof *prof) {
    ProfScope ps(prof, "rescale");
    k_rescale<<<bv.n_pblk, kThreads, 0, st>>>(bv, vel, energy);
    return cudaGetLastError();
}

cudaError_t launch_step_done(const BatchView &bv, cudaStream_t st, const Prof *prof) {
    if (!bv.remaining) return cudaSuccess;
    ProfScope ps(prof, "step_done");
    k_step_done<<<(unsigned)((bv.n_sys + 127) / 128), 128, 0, st>>>(bv.n_sys, bv.remaining);
    return cudaGetLastError();
}

// Per block of 256 charges: (sum q, sum |q|, sum q^2) in FP64, the threads'
// terms combined in a fixed tree order.
__global__ void __launch_bounds__(256) k_charge_sums(int64_t n, const double *__restrict__ q,
                                                     double *__restrict__ part) {
    __shared__ double s[3][256];
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * 256 + tid;
    const double v = i < n ? q[i] : 0.0;
    s[0][tid] = v;
    s[1][tid] = fabs(v);
    s[2][tid] = v * v;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h)
            for (int c = 0; c < 3; ++c) s[c][tid] += s[c][tid + h];
        __syncthreads();
    }
    if (tid < 3) part[3 * blockIdx.x + tid] = s[tid][0];
}

cudaError_t launch_charge_sums(int64_t n, const double *q, double *part, cudaStream_t st) {
    k_charge_sums<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, q, part);
    return cudaGetLastError();
}

cudaError_t launch_pack(int64_t n, const double *x3, const double *q, double4_32a *out, int wrap,
                        const double *L, cudaStream_t st) {
    k_pack<<<nblk(n), kThreads, 0, st>>>(n, x3, q, out, wrap, L[0], L[1], L[2]);
    return cudaGetLastError();
}

cudaError_t launch_unpack(int64_t n, const double4_32a *in, double *x3, cudaStream_t st) {
    k_unpack<<<nblk(n), kThreads, 0, st>>>(n, in, x3);
    return cudaGetLastError();
}

cudaError_t launch_unsort_i32(int64_t n, int64_t off, const int32_t *perm, const int32_t *sorted, int32_t *out,
                              cudaStream_t st) {
    k_unsort<<<nblk(n), kThreads, 0, st>>>(n, off, perm, sorted, out);
    return cudaGetLastError();
}

cudaError_t launch_m_to_int4(int32_t P, const int32_t *m3, int4 *out, cudaStream_t st) {
    k_m_to_int4<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(P, m3, out);
    return cudaGetLastError();
}

}  // namespace rbsog
