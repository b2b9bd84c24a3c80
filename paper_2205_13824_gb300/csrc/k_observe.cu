// Observables of Appendix A beside the step (single system, FP64, caller
// order):
//   MSD eta(t) = <|r(t0 + t) - r(t0)|^2> and VACF <v(t0) . v(t0 + t)>,
//     averaged over particles and time origins.  Each sample unwraps the
//     folded positions by the minimum-image displacement since the previous
//     sample, stores a new origin (unwrapped r, v) in a ring every
//     origin_every samples, and adds one particle sum per active origin to
//     the accumulator of its lag (fixed-order block sums);
//   pressure tensor P_ab = (1/V) sum_i (m v_ia v_ib + r_ia f_ib), the second
//     sum the configurational virial W_ab;
//   Green-Kubo shear viscosity C = V/(6 T) sum_{a<=b} of the integral of
//     <dP_ab(t) dP_ab(0)> over a pressure-tensor series, each component's
//     fluctuation about its mean, autocorrelations averaged over all
//     origins, trapezoid rule in the lag.
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Fixed-order block sum of NV doubles per thread (warp trees, then the warps
// in order); thread 0 receives the totals.  Ends with the block synchronised
// so that the shared scratch can be reused.
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

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

// One sample: unwrap, store the origin (store_slot >= 0), then for each
// active origin the block's sums of |u - u0|^2 and v . v0 into
// part[block * kObsMaxPairs + p].
__global__ void __launch_bounds__(kThreads) k_obs_sample(int64_t n, const double4_32a *__restrict__ posq,
                                                         const double4_32a *__restrict__ vel,
                                                         double4_32a *__restrict__ xprev,
                                                         double4_32a *__restrict__ u,
                                                         double4_32a *__restrict__ ring_u,
                                                         double4_32a *__restrict__ ring_v, double Lx, double Ly,
                                                         double Lz, int first, int store_slot,
                                                         const __grid_constant__ ObsPairs pr,
                                                         double2 *__restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool ok = i < n;
    double4_32a ui = make_double4_32a(0.0, 0.0, 0.0, 0.0), vi = ui;
    if (ok) {
        const double4_32a x = posq[i];
        if (first) {
            ui = make_double4_32a(x.x, x.y, x.z, 0.0);
        } else {
            const double4_32a p = xprev[i], uo = u[i];
            ui = make_double4_32a(uo.x + min_image(x.x - p.x, Lx), uo.y + min_image(x.y - p.y, Ly),
                                  uo.z + min_image(x.z - p.z, Lz), 0.0);
        }
        xprev[i] = x;
        u[i] = ui;
        vi = vel[i];
        if (store_slot >= 0) {
            ring_u[(int64_t)store_slot * n + i] = ui;
            ring_v[(int64_t)store_slot * n + i] = vi;
        }
    }
    for (int p = 0; p < pr.n; ++p) {
        double s[2] = {0.0, 0.0}, t[2];
        if (ok) {
            const int64_t o = (int64_t)pr.slot[p] * n + i;
            const double4_32a a = ring_u[o], b = ring_v[o];
            const double dx = ui.x - a.x, dy = ui.y - a.y, dz = ui.z - a.z;
            s[0] = dx * dx + dy * dy + dz * dz;
            s[1] = vi.x * b.x + vi.y * b.y + vi.z * b.z;
        }
        block_sum<2>(s, t);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kObsMaxPairs + p] = make_double2(t[0], t[1]);
    }
}

// Block p: the sum over particle blocks (fixed order) of pair p, added to
// the accumulators of its lag; one origin per lag per sample, so no two
// blocks write the same lag.
__global__ void __launch_bounds__(kThreads) k_obs_combine(const double2 *__restrict__ part, int32_t nblocks,
                                                          const __grid_constant__ ObsPairs pr,
                                                          double *__restrict__ msd_sum,
                                                          double *__restrict__ vacf_sum,
                                                          int64_t *__restrict__ count) {
    const int p = blockIdx.x;
    double s[2] = {0.0, 0.0}, t[2];
    for (int b = threadIdx.x; b < nblocks; b += kThreads) {
        const double2 v = part[(int64_t)b * kObsMaxPairs + p];
        s[0] += v.x;
        s[1] += v.y;
    }
    block_sum<2>(s, t);
    if (threadIdx.x == 0) {
        const int lag = pr.lag[p];
        msd_sum[lag] += t[0];
        vacf_sum[lag] += t[1];
        count[lag] += 1;
    }
}

__global__ void k_obs_result(int32_t n_lags, int64_t n, const double *__restrict__ msd_sum,
                             const double *__restrict__ vacf_sum, const int64_t *__restrict__ count,
                             double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_lags) return;
    const double c = (double)count[t] * (double)n;
    out[t] = count[t] > 0 ? msd_sum[t] / c : 0.0;
    out[n_lags + t] = count[t] > 0 ? vacf_sum[t] / c : 0.0;
}

// Kinetic tensor sum_i m v_ia v_ib: block partials (xx, yy, zz, xy, xz, yz).
__global__ void __launch_bounds__(kThreads) k_kin_tensor(int64_t n, const double4_32a *__restrict__ vel,
                                                         double mass, double *__restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, t[6];
    if (i < n) {
        const double4_32a v = vel[i];
        s[0] = mass * v.x * v.x;
        s[1] = mass * v.y * v.y;
        s[2] = mass * v.z * v.z;
        s[3] = mass * v.x * v.y;
        s[4] = mass * v.x * v.z;
        s[5] = mass * v.y * v.z;
    }
    block_sum<6>(s, t);
    if (threadIdx.x == 0)
        for (int c = 0; c < 6; ++c) part[(int64_t)blockIdx.x * 6 + c] = t[c];
}

// P = (kinetic tensor + W) / V, row-major [9].
__global__ void __launch_bounds__(kThreads) k_pressure_total(const double *__restrict__ part, int32_t nblocks,
                                                             const double *__restrict__ W, double inv_V,
                                                             double *__restrict__ Pt) {
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, t[6];
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int c = 0; c < 6; ++c) s[c] += part[(int64_t)b * 6 + c];
    block_sum<6>(s, t);
    if (threadIdx.x == 0) {
        const int ia[6] = {0, 4, 8, 1, 2, 5}, ib[6] = {0, 4, 8, 3, 6, 7};
        for (int c = 0; c < 6; ++c) {
            Pt[ia[c]] = (t[c] + W[ia[c]]) * inv_V;
            Pt[ib[c]] = (t[c] + W[ib[c]]) * inv_V;
        }
    }
}

// The six components a <= b (xx, xy, xz, yy, yz, zz) of a row-major tensor.
__device__ __forceinline__ int gk_comp(int c) { return c < 3 ? c : (c < 5 ? c + 1 : 8); }

__global__ void __launch_bounds__(kThreads) k_gk_mean(const double *__restrict__ series, int64_t ns,
                                                      double *__restrict__ mean) {
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, t[6];
    for (int64_t o = threadIdx.x; o < ns; o += kThreads)
        for (int c = 0; c < 6; ++c) s[c] += series[9 * o + gk_comp(c)];
    block_sum<6>(s, t);
    if (threadIdx.x == 0)
        for (int c = 0; c < 6; ++c) mean[c] = t[c] / (double)ns;
}

// Block t: acf[t] = the products of fluctuations at lag t summed over the
// six components and the origins, divided by the n - t origins.
__global__ void __launch_bounds__(kThreads) k_gk_acf(const double *__restrict__ series, int64_t ns,
                                                     const double *__restrict__ mean, double *__restrict__ acf) {
    const int64_t t = blockIdx.x;
    double m[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) m[c] = mean[c];
    double s[1] = {0.0}, r[1];
    for (int64_t o = threadIdx.x; o + t < ns; o += kThreads) {
        const double *a = series + 9 * o, *b = series + 9 * (o + t);
#pragma unroll
        for (int c = 0; c < 6; ++c) s[0] += (a[gk_comp(c)] - m[c]) * (b[gk_comp(c)] - m[c]);
    }
    block_sum<1>(s, r);
    if (threadIdx.x == 0) acf[t] = r[0] / (double)(ns - t);
}

__global__ void __launch_bounds__(kThreads) k_gk_integral(const double *__restrict__ acf, int32_t max_lag,
                                                          double scale, double *__restrict__ C) {
    double s[1] = {0.0}, t[1];
    for (int k = threadIdx.x; k + 1 < max_lag; k += kThreads) s[0] += acf[k] + acf[k + 1];
    block_sum<1>(s, t);
    if (threadIdx.x == 0) *C = scale * 0.5 * t[0];
}

// Block t: acf[t] = sum over the origins of J(t0) . J(t0 + t) (the flux as
// sampled, no mean removed), divided by the n - t origins.
__global__ void __launch_bounds__(kThreads) k_gkh_acf(const double *__restrict__ series, int64_t ns,
                                                      double *__restrict__ acf) {
    const int64_t t = blockIdx.x;
    double s[1] = {0.0}, r[1];
    for (int64_t o = threadIdx.x; o + t < ns; o += kThreads) {
        const double *a = series + 3 * o, *b = series + 3 * (o + t);
        s[0] += a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    }
    block_sum<1>(s, r);
    if (threadIdx.x == 0) acf[t] = r[0] / (double)(ns - t);
}

}  // namespace

int32_t obs_blocks(int64_t n) { return (int32_t)((n + kThreads - 1) / kThreads); }

cudaError_t launch_obs_sample(int64_t n, const double4_32a *posq, const double4_32a *vel, double4_32a *xprev,
                              double4_32a *u, double4_32a *ring_u, double4_32a *ring_v, const double L[3],
                              int first, int store_slot, const ObsPairs &pr, double2 *part, double *msd_sum,
                              double *vacf_sum, int64_t *count, cudaStream_t st) {
    const int32_t nb = obs_blocks(n);
    k_obs_sample<<<nb, kThreads, 0, st>>>(n, posq, vel, xprev, u, ring_u, ring_v, L[0], L[1], L[2], first,
                                          store_slot, pr, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || pr.n == 0) return e;
    k_obs_combine<<<pr.n, kThreads, 0, st>>>(part, nb, pr, msd_sum, vacf_sum, count);
    return cudaGetLastError();
}

cudaError_t launch_obs_result(int32_t n_lags, int64_t n, const double *msd_sum, const double *vacf_sum,
                              const int64_t *count, double *out, cudaStream_t st) {
    k_obs_result<<<(n_lags + 127) / 128, 128, 0, st>>>(n_lags, n, msd_sum, vacf_sum, count, out);
    return cudaGetLastError();
}

cudaError_t launch_pressure(int64_t n, const double4_32a *vel, double mass, const double *W, double V,
                            double *part, double *Pt, cudaStream_t st) {
    const int32_t nb = obs_blocks(n);
    k_kin_tensor<<<nb, kThreads, 0, st>>>(n, vel, mass, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pressure_total<<<1, kThreads, 0, st>>>(part, nb, W, 1.0 / V, Pt);
    return cudaGetLastError();
}

cudaError_t launch_green_kubo(const double *series, int64_t ns, int32_t max_lag, double scale, double *mean,
                              double *acf, double *C, cudaStream_t st) {
    k_gk_mean<<<1, kThreads, 0, st>>>(series, ns, mean);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gk_acf<<<max_lag, kThreads, 0, st>>>(series, ns, mean, acf);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gk_integral<<<1, kThreads, 0, st>>>(acf, max_lag, scale, C);
    return cudaGetLastError();
}

cudaError_t launch_green_kubo_heat(const double *series, int64_t ns, int32_t max_lag, double scale, double *acf,
                                   double *C, cudaStream_t st) {
    k_gkh_acf<<<max_lag, kThreads, 0, st>>>(series, ns, acf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gk_integral<<<1, kThreads, 0, st>>>(acf, max_lag, scale, C);
    return cudaGetLastError();
}

}  // namespace rbsog
