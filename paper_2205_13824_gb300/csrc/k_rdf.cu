// Radial distribution functions (Appendix A): histograms of minimum-image
// pair distances on [0, L/2) by charge-sign pair (++, +-, --), and the g(r)
// estimate from them.
//
// Bins are decided in exact integer arithmetic.  Positions are quantised to
// L 2^-32 per axis (X = floor(frac(x/L) 2^32) mod 2^32); the minimum-image
// difference of two quantised coordinates is the 32-bit wrapped difference,
// the squared distance R = dx^2 + dy^2 + dz^2 is an exact 64-bit integer
// (< 3 2^62), r < L/2 is R < 2^62, and with bin width w = 2^31 / nbins
// lattice units the bin is the largest b with (b w)^2 <= R.  An FP32 estimate
// floor(sqrt(R) / w) is within one bin of that (relative error < 2^-22 on a
// value <= 4096) and one integer comparison each way makes it exact, so the
// counts do not depend on rounding and match any exact evaluation.
//
// Layout: one pre-pass packs each particle as uint4 {X, Y, Z, species}; the
// pair kernel is persistent, walks 256 x 256 tile pairs (I <= J) of the
// particle array, stages tile J in shared memory and lets thread i visit
// j = i + t (rotated so that the lanes of a warp read different j and land
// in different bins), with a block histogram in shared memory (32-bit
// counters, flushed to the 64-bit global counts before they can overflow).
#include <cuda_runtime.h>

#include <algorithm>

#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr int kRdfTile = 256;
constexpr uint32_t kSkip = 3;                // neutral or padding site
constexpr uint32_t kFlushEvery = 32768;      // tile pairs between flushes (< 2^32 / 2^16)

__device__ __forceinline__ uint32_t quantise(double x, double L) {
    double t = __ddiv_rn(x, L);
    t = __dsub_rn(t, floor(t));
    const double v = floor(__dmul_rn(t, 4294967296.0));
    return (uint32_t)((unsigned long long)v & 0xffffffffull);
}

__global__ void __launch_bounds__(256) k_rdf_pack(int64_t n, const double4_32a *__restrict__ posq, double L,
                                                  uint4 *__restrict__ pt, unsigned long long *__restrict__ nspec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t s = kSkip;
    if (i < n) {
        const double4_32a p = posq[i];
        s = p.w > 0.0 ? 0u : (p.w < 0.0 ? 1u : kSkip);
        pt[i] = make_uint4(quantise(p.x, L), quantise(p.y, L), quantise(p.z, L), s);
    }
    const unsigned pos = __ballot_sync(0xffffffffu, s == 0u);
    const unsigned neg = __ballot_sync(0xffffffffu, s == 1u);
    if ((threadIdx.x & 31) == 0) {
        if (pos) atomicAdd(&nspec[0], (unsigned long long)__popc(pos));
        if (neg) atomicAdd(&nspec[1], (unsigned long long)__popc(neg));
    }
}

__device__ __forceinline__ void flush(uint32_t *hist, int nh, unsigned long long *__restrict__ counts) {
    for (int k = threadIdx.x; k < nh; k += blockDim.x) {
        const uint32_t v = hist[k];
        if (v) atomicAdd(&counts[k], (unsigned long long)v);
        hist[k] = 0;
    }
}

__global__ void __launch_bounds__(kRdfTile) k_rdf_pairs(int64_t n, const uint4 *__restrict__ pt, int32_t nt,
                                                        int32_t nbins, uint32_t width, float inv_width,
                                                        unsigned long long *__restrict__ counts) {
    extern __shared__ uint32_t hist[];       // [3][nbins]
    __shared__ uint4 tj[kRdfTile];
    const int tid = threadIdx.x;
    const int nh = 3 * nbins;
    for (int k = tid; k < nh; k += kRdfTile) hist[k] = 0;
    const int64_t total = (int64_t)nt * nt;
    uint32_t done = 0;
    for (int64_t p = blockIdx.x; p < total; p += gridDim.x) {
        const int I = (int)(p / nt), J = (int)(p - (int64_t)I * nt);
        if (J < I) continue;                 // block-uniform
        __syncthreads();
        const int64_t jj = (int64_t)J * kRdfTile + tid;
        tj[tid] = jj < n ? pt[jj] : make_uint4(0u, 0u, 0u, kSkip);
        const int64_t ii = (int64_t)I * kRdfTile + tid;
        const uint4 me = ii < n ? pt[ii] : make_uint4(0u, 0u, 0u, kSkip);
        __syncthreads();
        if (me.w != kSkip) {
            // off-diagonal tiles: all 256 j; the diagonal tile: j = tid + t > tid only
            const int t0 = I == J ? 1 : 0;
            const int t1 = I == J ? kRdfTile - tid : kRdfTile;
            uint32_t *h = hist + me.w * nbins;
#pragma unroll 4
            for (int t = t0; t < t1; ++t) {
                const uint4 o = tj[(tid + t) & (kRdfTile - 1)];
                if (o.w == kSkip) continue;
                const int dx = (int)(me.x - o.x), dy = (int)(me.y - o.y), dz = (int)(me.z - o.z);
                const unsigned long long R = (unsigned long long)((long long)dx * dx) +
                                             (unsigned long long)((long long)dy * dy) +
                                             (unsigned long long)((long long)dz * dz);
                if (R >= (1ull << 62)) continue;                         // r >= L/2
                int b = (int)(sqrtf((float)R) * inv_width);
                const unsigned long long lo = (unsigned long long)((uint32_t)b * width);
                if (R < lo * lo) {
                    --b;
                } else {
                    const unsigned long long hi = (unsigned long long)((uint32_t)(b + 1) * width);
                    if (R >= hi * hi) ++b;
                }
                b = min(max(b, 0), nbins - 1);                           // already exact; kept in range
                atomicAdd(&h[o.w * nbins + b], 1u);                      // row me.w + o.w
            }
        }
        if (++done == kFlushEvery) {
            __syncthreads();
            flush(hist, nh, counts);
            __syncthreads();
            done = 0;
        }
    }
    __syncthreads();
    flush(hist, nh, counts);
}

// g for row t (0 ++, 1 +-, 2 --) and bin k: counts scaled by the expected
// number of pairs in the shell, N_a (N_b / V) (4 pi / 3)((k+1)^3 - k^3) dr^3;
// like pairs are counted once per unordered pair (twice as ordered pairs).
__global__ void k_rdf_g(const unsigned long long *__restrict__ counts, int32_t nbins, double L,
                        const unsigned long long *__restrict__ nspec, double *__restrict__ g) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * nbins) return;
    const int t = idx / nbins, k = idx - t * nbins;
    const double np = (double)nspec[0], nn = (double)nspec[1];
    const double na = t == 2 ? nn : np, nb = t == 0 ? np : nn;
    const double mult = t == 1 ? 1.0 : 2.0;
    const double V = L * L * L;
    const double dr = L / (2.0 * nbins);
    const double kk = (double)k;
    const double shell = 4.0 * 3.14159265358979323846 / 3.0 * (3.0 * kk * kk + 3.0 * kk + 1.0) * dr * dr * dr;
    const double expect = na * nb / V * shell;
    g[idx] = expect > 0.0 ? mult * (double)counts[idx] / expect : 0.0;
}

}  // namespace

cudaError_t launch_rdf(int64_t n, const double4_32a *posq, double L, int32_t nbins, uint4 *pt,
                       unsigned long long *counts, unsigned long long *nspec, double *g, cudaStream_t st,
                       const Prof *prof) {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 3 * nbins, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(nspec, 0, sizeof(unsigned long long) * 2, st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        ProfScope ps(prof, "rdf_pack");
        k_rdf_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, posq, L, pt, nspec);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n > 1) {
        ProfScope ps(prof, "rdf_pairs");
        const int nt = (int)((n + kRdfTile - 1) / kRdfTile);
        const size_t smem = sizeof(uint32_t) * 3 * (size_t)nbins;
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_rdf_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rdf_pairs, kRdfTile, smem);
        if (e != cudaSuccess) return e;
        const int64_t tiles = (int64_t)nt * (nt + 1) / 2;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), tiles));
        const uint32_t width = 2147483648u / (uint32_t)nbins;
        k_rdf_pairs<<<(unsigned)grid, kRdfTile, smem, st>>>(n, pt, nt, nbins, width, 1.0f / (float)width, counts);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (g) {
        ProfScope ps(prof, "rdf_g");
        k_rdf_g<<<(unsigned)((3 * nbins + 255) / 256), 256, 0, st>>>(counts, nbins, L, nspec, g);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace rbsog
