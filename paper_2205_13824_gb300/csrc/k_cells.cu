// Device cell list for the near field: a counting sort of particles into
// cells of side >= r_c.  Launches:
//   bin      one thread per particle: cell id (FP64 floor(x * (n / L)), the
//            same decision as any IEEE evaluation of that product; a multiply,
//            not a divide, on GB300's narrow FP64 pipe) and an arrival slot
//            from an integer atomic on the cell's counter;
//   scan     two launches: per-tile warp-shuffle scans, then tile offsets
//            (the counters are cleared for the next build);
//   scatter  one thread per particle: perm_raw[start + slot] = i;
//   order    two passes of one thread per particle: ranks each cell's
//            members by (fixed-point x, particle index), so the order inside
//            a cell -- and everything summed in that order -- is
//            deterministic, and an x-row of cells is sorted in x (the near
//            field searches it); then moves the particle data into cell
//            order -- FP64 (x, y, z, q) or, for the FP32C path, 32-bit
//            fixed-point positions X_d = trunc(x_d * (2^32 / L_d)) with an FP32
//            charge.
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

__global__ void __launch_bounds__(kParticleBlock) k_bin(BatchView bv, const double4_32a *__restrict__ posq,
                                                        int32_t *__restrict__ cell_of, int32_t *__restrict__ slot,
                                                        int32_t *__restrict__ count, const int32_t *__restrict__ gate) {
    if (gate && !*gate) return;
    const int2 w = bv.pblk[blockIdx.x];
    const SysDesc &d = bv.sys[w.x];
    const int64_t il = (int64_t)w.y * kParticleBlock + threadIdx.x;
    if (il >= d.n) return;
    const int64_t i = d.p_off + il;
    const double4_32a p = posq[i];
    const double xs[3] = {p.x, p.y, p.z};
    int c3[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int c = (int)floor(xs[k] * d.box.inv_h[k]);
        c = c >= d.box.nc[k] ? d.box.nc[k] - 1 : c;
        c = c < 0 ? 0 : c;
        c3[k] = c;
    }
    const int cell = (int)d.c_off + (c3[2] * d.box.nc[1] + c3[1]) * d.box.nc[0] + c3[0];
    cell_of[i] = cell;
    slot[i] = atomicAdd(&count[cell], 1);
}

// Exclusive scan of count[0..ncell) into start[0..ncell] in two launches:
//   tile   each block scans a tile of kScanTile counters (8 per thread,
//          warp-shuffle scan of the thread sums) into start[] and writes the
//          tile total;
//   add    each block sums the totals of the tiles before it (fixed order)
//          and adds that offset to its tile; the counters are cleared for the
//          next build and start[ncell] receives the grand total.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) k_scan_tile(int ncell, const int32_t *__restrict__ count,
                                                            int32_t *__restrict__ start,
                                                            int32_t *__restrict__ tile_sum,
                                                            const int32_t *__restrict__ gate) {
    if (gate && !*gate) return;
    __shared__ int warp_tot[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int base = blockIdx.x * kScanTile + tid * kScanPer;
    int v[kScanPer];
    int local = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        v[j] = base + j < ncell ? count[base + j] : 0;
        local += v[j];
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    int woff = 0;
    for (int w = 0; w < wid; ++w) woff += warp_tot[w];
    int run = woff + incl - local;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        if (base + j < ncell) start[base + j] = run;
        run += v[j];
    }
    if (tid == kScanThreads - 1) tile_sum[blockIdx.x] = woff + incl;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int ncell, int ntiles, int32_t *__restrict__ count,
                                                           int32_t *__restrict__ start,
                                                           const int32_t *__restrict__ tile_sum,
                                                           const int32_t *__restrict__ gate) {
    if (gate && !*gate) return;
    __shared__ int s_off;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        int acc = 0;
        for (int t = lane; t < (int)blockIdx.x; t += 32) acc += tile_sum[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) s_off = acc;
    }
    __syncthreads();
    const int off = s_off;
    const int base = blockIdx.x * kScanTile;
    for (int j = tid; j < kScanTile; j += kScanThreads) {
        const int c = base + j;
        if (c < ncell) {
            start[c] += off;
            count[c] = 0;
        }
    }
    if (blockIdx.x == ntiles - 1 && tid == 0) start[ncell] = off + tile_sum[ntiles - 1];
}

__global__ void __launch_bounds__(256) k_scatter(int64_t n, const int32_t *__restrict__ cell_of,
                                                 const int32_t *__restrict__ slot,
                                                 const int32_t *__restrict__ start,
                                                 int32_t *__restrict__ perm_raw, const int32_t *__restrict__ gate) {
    if (gate && !*gate) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm_raw[start[cell_of[i]] + slot[i]] = (int32_t)i;
}

// X = trunc(x * (2^32 / L)) clamped to [0, 2^32 - 1]: one FP64 multiply (the
// scale is computed once on the host), not a division per coordinate.
__device__ __forceinline__ uint32_t to_fixed32(double x, double inv) { return fixed32(x, inv); }

// Order inside a cell, in two passes of one thread per particle:
//   keys    perm_raw slot s holds particle i: key[s] = (X << 32) | i with the
//           fixed-point x coordinate X, and pack[s] = the particle in the
//           gathered format (FP64 (x, y, z, q), or fixed-point X, Y, Z with
//           the FP32 charge);
//   rank    slot s of cell c goes to start[c] + (number of members of c with a
//           smaller key): the members' keys are read from the cached key
//           array (the threads of a cell read the same addresses).
__global__ void __launch_bounds__(256) k_cell_keys(BatchView bv, const int32_t *__restrict__ perm_raw,
                                                   const int32_t *__restrict__ cell_of,
                                                   const double4_32a *__restrict__ posq, int precision,
                                                   unsigned long long *__restrict__ key,
                                                   double4_32a *__restrict__ pack,
                                                   const int32_t *__restrict__ gate) {
    if (gate && !*gate) return;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= bv.n_total) return;
    const int idx = perm_raw[s];
    const BoxDev &box = bv.sys[bv.cell_sys[cell_of[idx]]].box;
    const double4_32a p = posq[idx];
    const uint32_t X = to_fixed32(p.x, box.fix_inv[0]);
    key[s] = ((unsigned long long)X << 32) | (uint32_t)idx;
    if (precision == 0) {
        pack[s] = p;
    } else {
        uint4 o;
        o.x = X;
        o.y = to_fixed32(p.y, box.fix_inv[1]);
        o.z = to_fixed32(p.z, box.fix_inv[2]);
        o.w = __float_as_uint((float)p.w);
        reinterpret_cast<uint4 *>(pack)[s] = o;
    }
}

__global__ void __launch_bounds__(256) k_cell_rank(int64_t n, const int32_t *__restrict__ perm_raw,
                                                   const int32_t *__restrict__ cell_of,
                                                   const int32_t *__restrict__ start,
                                                   const unsigned long long *__restrict__ key,
                                                   const double4_32a *__restrict__ pack, int precision,
                                                   int32_t *__restrict__ perm, double4_32a *__restrict__ sp64,
                                                   uint4 *__restrict__ sp32, const int32_t *__restrict__ gate) {
    if (gate && !*gate) return;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int idx = perm_raw[s];
    const int c = cell_of[idx];
    const int b = start[c], e = start[c + 1];
    const unsigned long long k = key[s];
    int rank = 0;
    for (int u = b; u < e; ++u) rank += key[u] < k ? 1 : 0;
    const int d = b + rank;
    perm[d] = idx;
    if (precision == 0) sp64[d] = pack[s];
    else sp32[d] = reinterpret_cast<const uint4 *>(pack)[s];
}

}  // namespace

int cell_scan_tiles(int64_t ncell) { return (int)((ncell + kScanTile - 1) / kScanTile); }

cudaError_t launch_build_cells(const BatchView &bv, const double4_32a *posq, const CellBuffers &cb,
                               int precision, double4_32a *sp64, uint4 *sp32, cudaStream_t st,
                               const Prof *prof, const int32_t *gate) {
    const int t = 256;
    const int ncell = (int)bv.ncell_total;
    {
        ProfScope ps(prof, "cell_bin");
        k_bin<<<bv.n_pblk, kParticleBlock, 0, st>>>(bv, posq, cb.cell_of, cb.slot, cb.count, gate);
    }
    {
        ProfScope ps(prof, "cell_scan");
        const int ntiles = cell_scan_tiles(ncell);
        k_scan_tile<<<ntiles, kScanThreads, 0, st>>>(ncell, cb.count, cb.start, cb.tile_sum, gate);
        k_scan_add<<<ntiles, kScanThreads, 0, st>>>(ncell, ntiles, cb.count, cb.start, cb.tile_sum, gate);
    }
    {
        ProfScope ps(prof, "cell_scatter");
        const unsigned nb = (unsigned)((bv.n_total + t - 1) / t);
        k_scatter<<<nb, t, 0, st>>>(bv.n_total, cb.cell_of, cb.slot, cb.start, cb.perm_raw, gate);
    }
    {
        ProfScope ps(prof, "cell_order_gather");
        const unsigned nb = (unsigned)((bv.n_total + t - 1) / t);
        k_cell_keys<<<nb, t, 0, st>>>(bv, cb.perm_raw, cb.cell_of, posq, precision, cb.key, cb.pack, gate);
        k_cell_rank<<<nb, t, 0, st>>>(bv.n_total, cb.perm_raw, cb.cell_of, cb.start, cb.key, cb.pack, precision,
                                      cb.perm, sp64, sp32, gate);
    }
    return cudaGetLastError();
}

}  // namespace rbsog
