// Device cell list for the near field: a counting sort of particles into
// cells of side >= r_c.  Four launches:
//   bin      one thread per particle: cell id (FP64 floor(x * (n / L)), the
//            same decision as any IEEE evaluation of that product; a multiply,
//            not a divide, on GB300's narrow FP64 pipe) and an arrival slot
//            from an integer atomic on the cell's counter;
//   scan     two launches: per-tile warp-shuffle scans, then tile offsets
//            (the counters are cleared for the next build);
//   scatter  one thread per particle: perm_raw[start + slot] = i;
//   order    one warp per cell: ranks the cell's members by (fixed-point x,
//            particle index) (keys exchanged by warp shuffles), so the order
//            inside a cell -- and everything summed in that order -- is
//            deterministic, and an x-row of cells is sorted in x (the near
//            field searches it); then gathers the particle data into cell
//            order -- FP64 (x, y, z, q) or, for the FP32C path, 32-bit
//            fixed-point positions X_d = trunc(x_d * (2^32 / L_d)) with an FP32
//            charge.
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

__global__ void __launch_bounds__(kParticleBlock) k_bin(BatchView bv, const double4_32a *__restrict__ posq,
                                                        int32_t *__restrict__ cell_of, int32_t *__restrict__ slot,
                                                        int32_t *__restrict__ count) {
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
                                                            int32_t *__restrict__ tile_sum) {
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
                                                           const int32_t *__restrict__ tile_sum) {
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
                                                 int32_t *__restrict__ perm_raw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm_raw[start[cell_of[i]] + slot[i]] = (int32_t)i;
}

// X = trunc(x * (2^32 / L)) clamped to [0, 2^32 - 1]: one FP64 multiply (the
// scale is computed once on the host), not a division per coordinate.
__device__ __forceinline__ uint32_t to_fixed32(double x, double inv) {
    const double t = x * inv;
    const double c = t < 0.0 ? 0.0 : (t > 4294967295.0 ? 4294967295.0 : t);
    return (uint32_t)__double2ull_rz(c);
}

// One warp per cell: rank = number of members with a smaller key
// (X << 32 | index) (keys exchanged by shuffles for cells of up to 32).
__global__ void __launch_bounds__(256) k_order_gather(BatchView bv, const int32_t *__restrict__ start,
                                                      const int32_t *__restrict__ perm_raw,
                                                      int32_t *__restrict__ perm,
                                                      const double4_32a *__restrict__ posq, int precision,
                                                      double4_32a *__restrict__ sp64, uint4 *__restrict__ sp32) {
    const int lane = threadIdx.x & 31;
    const int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= bv.ncell_total) return;
    const BoxDev &box = bv.sys[bv.cell_sys[cell]].box;
    const int b = start[cell], e = start[cell + 1], cnt = e - b;
    for (int t0 = 0; t0 < cnt; t0 += 32) {
        const int t = t0 + lane;
        const int idx = t < cnt ? perm_raw[b + t] : 0x7fffffff;
        double4_32a p{};
        unsigned long long key = ~0ull;
        if (t < cnt) {
            p = posq[idx];
            key = ((unsigned long long)to_fixed32(p.x, box.fix_inv[0]) << 32) | (uint32_t)idx;
        }
        int rank = 0;
        if (cnt <= 32) {
            for (int u = 0; u < cnt; ++u) rank += (__shfl_sync(0xffffffffu, key, u) < key) ? 1 : 0;
        } else {
            for (int u = 0; u < cnt; ++u) {
                const int j = perm_raw[b + u];
                const unsigned long long kj = ((unsigned long long)to_fixed32(posq[j].x, box.fix_inv[0]) << 32) | (uint32_t)j;
                rank += kj < key ? 1 : 0;
            }
        }
        if (t < cnt) {
            const int s = b + rank;
            perm[s] = idx;
            if (precision == 0) {
                sp64[s] = p;
            } else {
                uint4 o;
                o.x = to_fixed32(p.x, box.fix_inv[0]);
                o.y = to_fixed32(p.y, box.fix_inv[1]);
                o.z = to_fixed32(p.z, box.fix_inv[2]);
                o.w = __float_as_uint((float)p.w);
                sp32[s] = o;
            }
        }
    }
}

}  // namespace

int cell_scan_tiles(int64_t ncell) { return (int)((ncell + kScanTile - 1) / kScanTile); }

cudaError_t launch_build_cells(const BatchView &bv, const double4_32a *posq, const CellBuffers &cb,
                               int precision, double4_32a *sp64, uint4 *sp32, cudaStream_t st,
                               const Prof *prof) {
    const int t = 256;
    const int ncell = (int)bv.ncell_total;
    {
        ProfScope ps(prof, "cell_bin");
        k_bin<<<bv.n_pblk, kParticleBlock, 0, st>>>(bv, posq, cb.cell_of, cb.slot, cb.count);
    }
    {
        ProfScope ps(prof, "cell_scan");
        const int ntiles = cell_scan_tiles(ncell);
        k_scan_tile<<<ntiles, kScanThreads, 0, st>>>(ncell, cb.count, cb.start, cb.tile_sum);
        k_scan_add<<<ntiles, kScanThreads, 0, st>>>(ncell, ntiles, cb.count, cb.start, cb.tile_sum);
    }
    {
        ProfScope ps(prof, "cell_scatter");
        const unsigned nb = (unsigned)((bv.n_total + t - 1) / t);
        k_scatter<<<nb, t, 0, st>>>(bv.n_total, cb.cell_of, cb.slot, cb.start, cb.perm_raw);
    }
    {
        ProfScope ps(prof, "cell_order_gather");
        const unsigned blocks = (unsigned)((bv.ncell_total * 32 + t - 1) / t);
        k_order_gather<<<blocks, t, 0, st>>>(bv, cb.start, cb.perm_raw, cb.perm, posq, precision, sp64, sp32);
    }
    return cudaGetLastError();
}

}  // namespace rbsog
