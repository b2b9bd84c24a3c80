// Heat flux J of Appendix A for system 0, on request (a diagnostic beside
// the step, like the virial), FP64 for both precisions:
//   J = (1/V) sum_i (e_i v_i + W_i v_i),
// e_i the per-atom energy and W_i the per-atom virial:
//   near field (+ WCA), from the cell list (cells of side >= r_c) and the
//     FP64 caller-order state: e_i takes half of each pair energy and W_i v_i
//     half of r_ij (f_ij . v_i) for each ordered pair (i, j) -- the two
//     orders of a pair give the printed (1/2) (f_ij . (v_i + v_j)) r_ij;
//   kinetic m |v_i|^2 / 2 and the self term -lB F_M(0) q_i^2 / 2 per atom;
//   far field, the random-batch energy and virial split over atoms: with
//     R_eta = Re(e^{-i k_eta . r_i} rho(k_eta)) and c = lB pi^{3/2} S / (P V),
//     e_i += (c/2) q_i sum_eta R_eta and
//     W_i v_i += (c/2) q_i sum_eta R_eta (v_i - (1/2) tau_eta (k_eta . v_i) k_eta),
//     tau = T1/T0 of the SOG (the far virial's tensor weight, Eq. 3.5);
//     rho(k) is recomputed here in FP64 from the caller-order positions.
// Every sum runs in a fixed order (per-thread, warp trees, block order).
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRhoGroups = 64;   // particle groups of the FP64 rho(k) sweep
constexpr int kRhoKTile = 32;    // frequencies per rho block, one per lane
constexpr int kRhoTile = 1024;   // particles staged per pass
constexpr int kFarChunk = 128;   // frequencies staged per pass of the far kernel

// Fixed-order block sum of NV values per thread, result in out[] (thread 0).
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV], double out[NV]) {
    __shared__ double s_w[NV][kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        if (lane == 0) s_w[c][wid] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w) t += s_w[c][w];
            out[c] = t;
        }
    __syncthreads();
}

// Both Gaussian sums of the near kernel at r^2: F = sum_l w_l e^{-r^2/s_l^2}
// (F_M) and G = sum_l w_l / s_l^2 e^{-r^2/s_l^2}, the narrow Gaussians
// directly and the wide ones as their Taylor series in r^2.
__device__ __forceinline__ void gauss_fg(const NearSog &s, double r2, double &F, double &G) {
    F = 0.0;
    G = 0.0;
    for (int l = 0; l < s.n_direct; ++l) {
        const double e = exp(-r2 * s.inv_s2[l]);
        F += s.omega[l] * e;
        G += s.omega[l] * s.inv_s2[l] * e;
    }
    if (s.n_taylor > 0) {
        double pf = s.tay_f[s.n_taylor - 1], pg = s.tay_g[s.n_taylor - 1];
        for (int m = s.n_taylor - 2; m >= 0; --m) {
            pf = pf * r2 + s.tay_f[m];
            pg = pg * r2 + s.tay_g[m];
        }
        F += pf;
        G += pg;
    }
}

// One thread per particle (cell order s, particle i = perm[s]): its near
// energy share, kinetic and self terms times v_i, plus its near virial
// times v_i; block sums into part[block][3].
__global__ void __launch_bounds__(kThreads) k_heat_near(const SysDesc *__restrict__ sysd,
                                                        const __grid_constant__ NearSog sog,
                                                        const int32_t *__restrict__ start,
                                                        const int32_t *__restrict__ perm,
                                                        const int32_t *__restrict__ cell_of,
                                                        const double4_32a *__restrict__ posq,
                                                        const double4_32a *__restrict__ vel, double mass,
                                                        double half_lB_FM0, double *__restrict__ part) {
    const SysDesc &d = sysd[0];
    const BoxDev &box = d.box;
    const int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    double out[3] = {0.0, 0.0, 0.0};
    if (s < d.n) {
        const int32_t i = perm[s];
        const double4_32a pi = posq[i];
        const double4_32a vi = vel[i];
        const int nx = box.nc[0], ny = box.nc[1], nz = box.nc[2];
        const int c = cell_of[i] - (int)d.c_off;
        const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
        double e = 0.0, w[3] = {0.0, 0.0, 0.0};
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int ox = (cx + dx + nx) % nx, oy = (cy + dy + ny) % ny, oz = (cz + dz + nz) % nz;
                    const int64_t o = d.c_off + ((int64_t)oz * ny + oy) * nx + ox;
                    for (int32_t t = start[o]; t < start[o + 1]; ++t) {
                        const int32_t j = perm[t];
                        if (j == i) continue;
                        const double4_32a pj = posq[j];
                        double r[3] = {pi.x - pj.x, pi.y - pj.y, pi.z - pj.z};
                        for (int k = 0; k < 3; ++k) r[k] -= box.L[k] * rint(r[k] / box.L[k]);
                        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                        if (!(r2 < box.rc2)) continue;
                        const double inv_r = 1.0 / sqrt(r2);
                        double F, G;
                        gauss_fg(sog, r2, F, G);
                        const double qq = box.lB * pi.w * pj.w;
                        double g = qq * (inv_r * inv_r * inv_r - 2.0 * G);
                        double u = qq * (inv_r - F);
                        if (r2 < box.wca_rc2) {
                            const double sr2 = box.wca_s2 / r2, sr6 = sr2 * sr2 * sr2;
                            g += 24.0 * box.wca_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                            u += 4.0 * box.wca_eps * (sr6 * sr6 - sr6) + box.wca_eps;
                        }
                        e += 0.5 * u;
                        // half of r_ij (f_ij . v_i), f_ij = g r_ij
                        const double h = 0.5 * g * (r[0] * vi.x + r[1] * vi.y + r[2] * vi.z);
                        w[0] += h * r[0];
                        w[1] += h * r[1];
                        w[2] += h * r[2];
                    }
                }
        e += 0.5 * mass * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z) - half_lB_FM0 * pi.w * pi.w;
        out[0] = e * vi.x + w[0];
        out[1] = e * vi.y + w[1];
        out[2] = e * vi.z + w[2];
    }
    double t[3];
    block_sum<3>(out, t);
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) part[(int64_t)blockIdx.x * 3 + c] = t[c];
}

// FP64 rho(k) partials: block (g, kt) sums particle tiles g, g + kRhoGroups,
// ... for the frequencies kt * 32 + lane into rpart[k * kRhoGroups + g].
__global__ void __launch_bounds__(kThreads) k_heat_rho(int64_t n, const double4_32a *__restrict__ posq,
                                                       double ilx, double ily, double ilz,
                                                       const int32_t *__restrict__ m3, int32_t P,
                                                       double2 *__restrict__ rpart) {
    __shared__ double4_32a sp[kRhoTile];
    __shared__ double s_re[kWarps][kRhoKTile], s_im[kWarps][kRhoKTile];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int g = blockIdx.x;
    const int k = blockIdx.y * kRhoKTile + lane;
    double mx = 0.0, my = 0.0, mz = 0.0;
    if (k < P) {
        mx = m3[3 * k];
        my = m3[3 * k + 1];
        mz = m3[3 * k + 2];
    }
    double re = 0.0, im = 0.0;
    for (int64_t p0 = (int64_t)g * kRhoTile; p0 < n; p0 += (int64_t)kRhoGroups * kRhoTile) {
        const int np = (int)(n - p0 < kRhoTile ? n - p0 : kRhoTile);
        __syncthreads();
        for (int j = tid; j < np; j += kThreads) {
            const double4_32a p = posq[p0 + j];
            sp[j] = make_double4_32a(p.x * ilx, p.y * ily, p.z * ilz, p.w);
        }
        __syncthreads();
        const int per = (np + kWarps - 1) / kWarps;
        const int jb = wid * per, je = min(jb + per, np);
        for (int j = jb; j < je; ++j) {
            const double4_32a p = sp[j];
            double t = fma(mx, p.x, fma(my, p.y, mz * p.z));
            t -= rint(t);
            double sn, cs;
            sincospi(2.0 * t, &sn, &cs);
            re = fma(p.w, cs, re);
            im = fma(p.w, sn, im);
        }
    }
    s_re[wid][lane] = re;
    s_im[wid][lane] = im;
    __syncthreads();
    if (wid == 0 && k < P) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kWarps; ++w) {
            a += s_re[w][lane];
            b += s_im[w][lane];
        }
        rpart[(int64_t)k * kRhoGroups + g] = make_double2(a, b);
    }
}

// Per frequency: rho (fixed-order sum of the group partials) and the table
// entry (m, tau = T1/T0, k).
__global__ void __launch_bounds__(128) k_heat_ktab(int32_t P, const double2 *__restrict__ rpart,
                                                    const int32_t *__restrict__ m3, const SysDesc *__restrict__ sysd,
                                                    const double *__restrict__ omega, const double *__restrict__ sl,
                                                    int32_t M, double2 *__restrict__ rho,
                                                    double4_32a *__restrict__ ktab) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P) return;
    double re = 0.0, im = 0.0;
    for (int g = 0; g < kRhoGroups; ++g) {
        const double2 v = rpart[(int64_t)e * kRhoGroups + g];
        re += v.x;
        im += v.y;
    }
    rho[e] = make_double2(re, im);
    const BoxDev &box = sysd[0].box;
    double k[3], k2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        k[a] = box.kfac[a] * m3[3 * e + a];
        k2 += k[a] * k[a];
    }
    double T0 = 0.0, T1 = 0.0;
    for (int l = 0; l <= M; ++l) {
        const double s2 = sl[l] * sl[l];
        const double t = omega[l] * s2 * sl[l] * exp(-s2 * k2 / 4.0);
        T0 += t;
        T1 += t * s2;
    }
    ktab[2 * e] = make_double4_32a(m3[3 * e], m3[3 * e + 1], m3[3 * e + 2], T0 > 0.0 ? T1 / T0 : 0.0);
    ktab[2 * e + 1] = make_double4_32a(k[0], k[1], k[2], 0.0);
}

// One thread per particle (caller order): the far energy and virial shares
// times v_i, frequencies staged in chunks; block sums into part[block][3].
__global__ void __launch_bounds__(kThreads) k_heat_far(int64_t n, const double4_32a *__restrict__ posq,
                                                       const double4_32a *__restrict__ vel,
                                                       const double4_32a *__restrict__ ktab,
                                                       const double2 *__restrict__ rho, int32_t P, double ilx,
                                                       double ily, double ilz, double half_c,
                                                       double *__restrict__ part) {
    __shared__ double4_32a s_k[2 * kFarChunk];
    __shared__ double2 s_rho[kFarChunk];
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    double4_32a p = make_double4_32a(0.0, 0.0, 0.0, 0.0), v = p;
    if (i < n) {
        p = posq[i];
        v = vel[i];
    }
    const double ux = p.x * ilx, uy = p.y * ily, uz = p.z * ilz;
    double A = 0.0, B[3] = {0.0, 0.0, 0.0};
    for (int e0 = 0; e0 < P; e0 += kFarChunk) {
        const int ne = min(kFarChunk, P - e0);
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * ne; t += kThreads) s_k[t] = ktab[2 * e0 + t];
        for (int t = threadIdx.x; t < ne; t += kThreads) s_rho[t] = rho[e0 + t];
        __syncthreads();
        for (int e = 0; e < ne; ++e) {
            const double4_32a mt = s_k[2 * e], kk = s_k[2 * e + 1];
            const double2 r = s_rho[e];
            double t = fma(mt.x, ux, fma(mt.y, uy, mt.z * uz));
            t -= rint(t);
            double sn, cs;
            sincospi(2.0 * t, &sn, &cs);
            const double R = fma(cs, r.x, sn * r.y);   // Re(e^{-i k.r} rho)
            A += R;
            const double h = R * mt.w * (kk.x * v.x + kk.y * v.y + kk.z * v.z);
            B[0] = fma(h, kk.x, B[0]);
            B[1] = fma(h, kk.y, B[1]);
            B[2] = fma(h, kk.z, B[2]);
        }
    }
    double out[3] = {0.0, 0.0, 0.0};
    if (i < n) {
        const double f = half_c * p.w;
        out[0] = f * (2.0 * A * v.x - 0.5 * B[0]);
        out[1] = f * (2.0 * A * v.y - 0.5 * B[1]);
        out[2] = f * (2.0 * A * v.z - 0.5 * B[2]);
    }
    double t[3];
    block_sum<3>(out, t);
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) part[(int64_t)blockIdx.x * 3 + c] = t[c];
}

// J[3] = (sum of the near partials + sum of the far partials) / V, each in
// block order.
__global__ void __launch_bounds__(kThreads) k_heat_total(const double *__restrict__ pn, int32_t nb_near,
                                                         const double *__restrict__ pf, int32_t nb_far, double inv_V,
                                                         double *__restrict__ J) {
    double a[3] = {0.0, 0.0, 0.0}, b[3] = {0.0, 0.0, 0.0}, ta[3], tb[3];
    for (int k = threadIdx.x; k < nb_near; k += kThreads)
        for (int c = 0; c < 3; ++c) a[c] += pn[(int64_t)k * 3 + c];
    if (pf)
        for (int k = threadIdx.x; k < nb_far; k += kThreads)
            for (int c = 0; c < 3; ++c) b[c] += pf[(int64_t)k * 3 + c];
    block_sum<3>(a, ta);
    block_sum<3>(b, tb);
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) J[c] = (ta[c] + tb[c]) * inv_V;
}

}  // namespace

int32_t heat_blocks(int64_t n) { return (int32_t)((n + kThreads - 1) / kThreads); }
size_t heat_rho_partials(int32_t P) { return (size_t)P * kRhoGroups; }

cudaError_t launch_heat_flux(const SysDesc *sysd, const BoxDev &box, int64_t n, const NearSog &sog,
                             const int32_t *start, const int32_t *perm, const int32_t *cell_of,
                             const double4_32a *posq, const double4_32a *vel, double mass, double half_lB_FM0,
                             const int32_t *m3, int32_t P, const double *omega, const double *sl, int32_t M,
                             double half_c, double2 *rpart, double2 *rho, double4_32a *ktab, double *part_near,
                             double *part_far, double *J, cudaStream_t st) {
    const int32_t nb = heat_blocks(n);
    k_heat_near<<<nb, kThreads, 0, st>>>(sysd, sog, start, perm, cell_of, posq, vel, mass, half_lB_FM0, part_near);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double ilx = 1.0 / box.L[0], ily = 1.0 / box.L[1], ilz = 1.0 / box.L[2];
    if (P > 0) {
        const dim3 grid(kRhoGroups, (unsigned)((P + kRhoKTile - 1) / kRhoKTile));
        k_heat_rho<<<grid, kThreads, 0, st>>>(n, posq, ilx, ily, ilz, m3, P, rpart);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_heat_ktab<<<(P + 127) / 128, 128, 0, st>>>(P, rpart, m3, sysd, omega, sl, M, rho, ktab);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_heat_far<<<nb, kThreads, 0, st>>>(n, posq, vel, ktab, rho, P, ilx, ily, ilz, half_c, part_far);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_heat_total<<<1, kThreads, 0, st>>>(part_near, nb, P > 0 ? part_far : nullptr, nb,
                                         1.0 / (box.L[0] * box.L[1] * box.L[2]), J);
    return cudaGetLastError();
}

}  // namespace rbsog
