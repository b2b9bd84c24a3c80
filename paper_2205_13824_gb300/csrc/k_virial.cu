// Configurational virial tensor W_ab = -dU/d eps_ab under the affine map
// r -> (1 + eps) r of positions and box (r_c and the SOG fixed), on request:
//   near field (+ WCA): sum over pairs r_ij,a F_ij,b, each ordered pair
//     taking half, from the cell list (cells of side >= r_c) and the FP64
//     caller-order positions; the Gaussian sum as the FP64 force path takes
//     it (the narrow Gaussians directly, the wide ones as a Taylor series);
//   far field: the random-batch estimator on a given k-set, each sampled k
//     weighted as in the energy (Eq. 3.24), pi^{3/2} S / (2 P V) |rho(k)|^2,
//     times delta_ab + 2 k_a k_b dF~/d(k^2) / F~ = delta_ab - (1/2) k_a k_b
//     T1/T0 with T0 = sum_l w_l s_l^3 e^{-s_l^2 k^2/4}, T1 = sum_l w_l s_l^5
//     e^{-s_l^2 k^2/4} (F~ of Eq. 3.5 up to pi^{3/2}).
// FP64 for both precisions: a diagnostic, not part of the step.
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kThreads = 256;
constexpr int kComp = 6;   // xx, yy, zz, xy, xz, yz

__device__ __forceinline__ double gauss_g(const NearSog &s, double r2) {
    double gs = 0.0;
    for (int l = 0; l < s.n_direct; ++l) gs += s.omega[l] * s.inv_s2[l] * exp(-r2 * s.inv_s2[l]);
    if (s.n_taylor > 0) {
        double pg = s.tay_g[s.n_taylor - 1];
        for (int m = s.n_taylor - 2; m >= 0; --m) pg = pg * r2 + s.tay_g[m];
        gs += pg;
    }
    return gs;
}

// Fixed-order block sum of kComp values per thread (warp trees, then the
// warps in order) into out[kComp] by thread 0.
__device__ __forceinline__ void block_sum6(double v[kComp], double *out) {
    __shared__ double s_w[kComp][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < kComp; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        if (lane == 0) s_w[c][wid] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < kComp; ++c) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += s_w[c][w];
            out[c] = t;
        }
}

__global__ void __launch_bounds__(kThreads) k_virial_near(const SysDesc *__restrict__ sysd,
                                                          const __grid_constant__ NearSog sog,
                                                          const int32_t *__restrict__ start,
                                                          const int32_t *__restrict__ perm,
                                                          const int32_t *__restrict__ cell_of,
                                                          const double4_32a *__restrict__ posq,
                                                          double *__restrict__ part) {
    const SysDesc &d = sysd[0];
    const BoxDev &box = d.box;
    const int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    double v[kComp] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (s < d.n) {
        const int32_t i = perm[s];
        const double4_32a pi = posq[i];
        const int nx = box.nc[0], ny = box.nc[1], nz = box.nc[2];
        const int c = cell_of[i] - (int)d.c_off;
        const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
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
                        double g = box.lB * pi.w * pj.w * (inv_r * inv_r * inv_r - 2.0 * gauss_g(sog, r2));
                        if (r2 < box.wca_rc2) {
                            const double sr2 = box.wca_s2 / r2, sr6 = sr2 * sr2 * sr2;
                            g += 24.0 * box.wca_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                        }
                        const double h = 0.5 * g;   // each ordered pair takes half
                        v[0] += h * r[0] * r[0];
                        v[1] += h * r[1] * r[1];
                        v[2] += h * r[2] * r[2];
                        v[3] += h * r[0] * r[1];
                        v[4] += h * r[0] * r[2];
                        v[5] += h * r[1] * r[2];
                    }
                }
    }
    block_sum6(v, part + (int64_t)blockIdx.x * kComp);
}

// One block: near partials in block order, far terms of the k-set, W[9].
__global__ void __launch_bounds__(kThreads) k_virial_total(const SysDesc *__restrict__ sysd,
                                                           const double *__restrict__ part, int32_t nblocks,
                                                           const double2 *__restrict__ rho,
                                                           const int32_t *__restrict__ m3, int32_t P,
                                                           const double *__restrict__ omega,
                                                           const double *__restrict__ sl, int32_t M, double S,
                                                           double *__restrict__ W) {
    __shared__ double s_near[kComp], s_far[kComp];
    const SysDesc &d = sysd[0];
    double v[kComp] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int c = 0; c < kComp; ++c) v[c] += part[(int64_t)b * kComp + c];
    block_sum6(v, s_near);
    __syncthreads();
    const double V = d.box.L[0] * d.box.L[1] * d.box.L[2];
    const double wfac = d.box.lB * pow(3.14159265358979323846, 1.5) * S / (2.0 * P * V);
    double f[kComp] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int e = threadIdx.x; e < P; e += kThreads) {
        double k[3], k2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            k[a] = d.box.kfac[a] * m3[3 * e + a];
            k2 += k[a] * k[a];
        }
        double T0 = 0.0, T1 = 0.0;
        for (int l = 0; l <= M; ++l) {
            const double s2 = sl[l] * sl[l];
            const double t = omega[l] * s2 * sl[l] * exp(-s2 * k2 / 4.0);
            T0 += t;
            T1 += t * s2;
        }
        const double rr = T0 > 0.0 ? T1 / T0 : 0.0;
        const double w = wfac * (rho[e].x * rho[e].x + rho[e].y * rho[e].y);
        f[0] += w * (1.0 - 0.5 * rr * k[0] * k[0]);
        f[1] += w * (1.0 - 0.5 * rr * k[1] * k[1]);
        f[2] += w * (1.0 - 0.5 * rr * k[2] * k[2]);
        f[3] -= w * 0.5 * rr * k[0] * k[1];
        f[4] -= w * 0.5 * rr * k[0] * k[2];
        f[5] -= w * 0.5 * rr * k[1] * k[2];
    }
    block_sum6(f, s_far);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int ia[kComp] = {0, 4, 8, 1, 2, 5}, ib[kComp] = {0, 4, 8, 3, 6, 7};
        for (int c = 0; c < kComp; ++c) {
            W[ia[c]] = s_near[c] + s_far[c];
            W[ib[c]] = s_near[c] + s_far[c];
        }
    }
}

}  // namespace

int32_t virial_blocks(int64_t n) { return (int32_t)((n + kThreads - 1) / kThreads); }

cudaError_t launch_virial(const SysDesc *sysd, int64_t n, const NearSog &sog, const int32_t *start,
                          const int32_t *perm, const int32_t *cell_of, const double4_32a *posq, double *part,
                          const double2 *rho, const int32_t *m3, int32_t P, const double *omega, const double *sl,
                          int32_t M, double S, double *W, cudaStream_t st) {
    const int32_t nb = virial_blocks(n);
    k_virial_near<<<nb, kThreads, 0, st>>>(sysd, sog, start, perm, cell_of, posq, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_virial_total<<<1, kThreads, 0, st>>>(sysd, part, nb, rho, m3, P, omega, sl, M, S, W);
    return cudaGetLastError();
}

}  // namespace rbsog
