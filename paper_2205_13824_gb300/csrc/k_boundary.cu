// Zero-frequency (boundary) term of the far field (Sec. 3.2): for a
// periodic system embedded in a medium of finite permittivity the k -> 0
// limit adds, with the dipole moment M = sum_i q_i r_i of the box,
//   spherical boundary (Eq. 3.14): U0 = (2 pi / 3V) |M|^2,
//                                  F_i = -(4 pi / 3V) q_i M;
//   planar boundary along z (Eq. 3.15): U0 = (2 pi / V) M_z^2,
//                                  F_i = -(4 pi / V) q_i M_z e_z;
// times the Coulomb prefactor; tinfoil (the default) adds nothing.  M is
// taken over the positions folded into [0, L), in FP64 for both precisions.
//
// part     one block per particle block: the block's q r sums (fixed order:
//          warp trees, then the warps in order) as one partial;
// combine  one block per system: the partials in fixed order (thread
//          strides, warp trees, the warps in order), U0 into the energy
//          record;
// force    one thread per particle: the term added to its total force.
// Systems with the tinfoil boundary skip all three.
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kThreads = kParticleBlock;

__device__ __forceinline__ bool boundary_on(const BatchView &bv, int sys) {
    if (bv.remaining && bv.remaining[sys] == 0) return false;
    if (bv.force_mask && !bv.force_mask[sys]) return false;
    return bv.sys[sys].boundary != 0;
}

__global__ void __launch_bounds__(kThreads) k_dipole_part(BatchView bv, const double4_32a *__restrict__ posq,
                                                          double4_32a *__restrict__ dpart) {
    __shared__ double s_m[3][kThreads / 32];
    const int2 w = bv.pblk[blockIdx.x];
    if (!boundary_on(bv, w.x)) return;
    const SysDesc &a = bv.sys[w.x];
    const int64_t il = (int64_t)w.y * kThreads + threadIdx.x;
    double mx = 0.0, my = 0.0, mz = 0.0;
    if (il < a.n) {
        const double4_32a p = posq[a.p_off + il];
        mx = p.w * p.x;
        my = p.w * p.y;
        mz = p.w * p.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx += __shfl_down_sync(0xffffffffu, mx, o);
        my += __shfl_down_sync(0xffffffffu, my, o);
        mz += __shfl_down_sync(0xffffffffu, mz, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_m[0][wid] = mx;
        s_m[1][wid] = my;
        s_m[2][wid] = mz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < 3; ++d)
            for (int q = 0; q < kThreads / 32; ++q) t[d] += s_m[d][q];
        dpart[a.kp_off + w.y] = make_double4_32a(t[0], t[1], t[2], 0.0);
    }
}

__global__ void __launch_bounds__(kThreads) k_dipole_combine(BatchView bv, const double4_32a *__restrict__ dpart,
                                                             double4_32a *__restrict__ dip,
                                                             double *__restrict__ energy) {
    __shared__ double s_m[3][kThreads / 32];
    const int sys = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (!boundary_on(bv, sys)) return;
    const SysDesc &a = bv.sys[sys];
    double mx = 0.0, my = 0.0, mz = 0.0;
    for (int b = tid; b < a.n_kpart; b += kThreads) {
        const double4_32a v = dpart[a.kp_off + b];
        mx += v.x;
        my += v.y;
        mz += v.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx += __shfl_down_sync(0xffffffffu, mx, o);
        my += __shfl_down_sync(0xffffffffu, my, o);
        mz += __shfl_down_sync(0xffffffffu, mz, o);
    }
    if (lane == 0) {
        s_m[0][wid] = mx;
        s_m[1][wid] = my;
        s_m[2][wid] = mz;
    }
    __syncthreads();
    if (tid == 0) {
        mx = my = mz = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) {
            mx += s_m[0][q];
            my += s_m[1][q];
            mz += s_m[2][q];
        }
        const double V = a.box.L[0] * a.box.L[1] * a.box.L[2];
        const double pi = 3.14159265358979323846;
        double U, c[3];
        if (a.boundary == 1) {
            U = 2.0 * pi / (3.0 * V) * (mx * mx + my * my + mz * mz);
            c[0] = -4.0 * pi / (3.0 * V) * mx;
            c[1] = -4.0 * pi / (3.0 * V) * my;
            c[2] = -4.0 * pi / (3.0 * V) * mz;
        } else {
            U = 2.0 * pi / V * mz * mz;
            c[0] = c[1] = 0.0;
            c[2] = -4.0 * pi / V * mz;
        }
        const double lB = a.box.lB;
        dip[sys] = make_double4_32a(lB * c[0], lB * c[1], lB * c[2], 0.0);
        energy[(int64_t)sys * kNumEnergy + 7] = lB * U;
    }
}

__global__ void __launch_bounds__(kThreads) k_dipole_force(BatchView bv, const double4_32a *__restrict__ posq,
                                                           const double4_32a *__restrict__ dip,
                                                           double4_32a *__restrict__ force) {
    const int2 w = bv.pblk[blockIdx.x];
    if (!boundary_on(bv, w.x)) return;
    const SysDesc &a = bv.sys[w.x];
    const int64_t il = (int64_t)w.y * kThreads + threadIdx.x;
    if (il >= a.n) return;
    const int64_t i = a.p_off + il;
    const double q = posq[i].w;
    const double4_32a c = dip[w.x];
    double4_32a f = force[i];
    f.x += q * c.x;
    f.y += q * c.y;
    f.z += q * c.z;
    force[i] = f;
}

}  // namespace

cudaError_t launch_boundary(const BatchView &bv, const double4_32a *posq, double4_32a *dpart, double4_32a *dip,
                            double *energy, double4_32a *force, cudaStream_t st, const Prof *prof) {
    ProfScope ps(prof, "boundary");
    k_dipole_part<<<bv.n_pblk, kThreads, 0, st>>>(bv, posq, dpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dipole_combine<<<bv.n_sys, kThreads, 0, st>>>(bv, dpart, dip, energy);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dipole_force<<<bv.n_pblk, kThreads, 0, st>>>(bv, posq, dip, force);
    return cudaGetLastError();
}

}  // namespace rbsog
