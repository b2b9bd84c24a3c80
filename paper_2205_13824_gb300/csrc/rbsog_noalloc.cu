// Allocation-free structure factors: rbsog_rho_noalloc.
//
// Some callers cannot allocate device memory at the point where they need
// rho(k): code running inside a region that forbids allocation (a
// stream-ordered pipeline that is being captured, or an embedding host whose
// allocator must not be re-entered), or tools with a fixed memory budget.
// This entry point takes the caller's device buffers only and keeps its
// per-block partial sums in a file-scope device array of fixed size that is
// part of the loaded library.  It computes the same quantity as rbsog_rho
// (FP64), with a sweep kernel whose blocks each loop over a fixed number of
// particle tiles so that the number of partials does not grow with n.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/rbsog.h"

namespace {

constexpr int kGroups = 64;             // particle groups (blocks along the particle axis)
constexpr int kKTile = 32;              // frequencies per block, one per lane
constexpr int kTile = 1024;             // particles staged per pass (32 KiB of double4)
constexpr int kThreads = 256;           // 8 warps
constexpr int kMaxPartials = kGroups * RBSOG_NOALLOC_MAX_P;

// Scratch: one FP64 complex partial per (frequency, group).  Every call
// overwrites all kGroups * P partials it reads, so nothing has to be cleared
// between calls; concurrent calls on the same device share this array.
static __device__ __align__(256) double2 g_rho_scratch[kMaxPartials];

struct alignas(32) PosQ {
    double x, y, z, q;
};

// Block (g, kt): frequencies kt*32 + lane; particle tiles g, g + kGroups, ...
// are staged in shared memory as (x/L, y/L, z/L, q) and swept by the 8 warps;
// the warp sums are combined in a fixed order into one partial per (k, g).
__global__ void __launch_bounds__(kThreads) k_rho_groups(int64_t n, const double *__restrict__ q,
                                                         const double *__restrict__ x, double ilx,
                                                         double ily, double ilz, const int32_t *__restrict__ m,
                                                         int32_t P, double2 *__restrict__ part) {
    __shared__ PosQ sp[kTile];
    __shared__ double s_re[kThreads / 32][kKTile];
    __shared__ double s_im[kThreads / 32][kKTile];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int g = blockIdx.x;
    const int k = blockIdx.y * kKTile + lane;
    double mx = 0.0, my = 0.0, mz = 0.0;
    if (k < P) {
        mx = m[3 * k];
        my = m[3 * k + 1];
        mz = m[3 * k + 2];
    }
    double re = 0.0, im = 0.0;
    for (int64_t p0 = (int64_t)g * kTile; p0 < n; p0 += (int64_t)kGroups * kTile) {
        const int np = (int)(n - p0 < kTile ? n - p0 : kTile);
        __syncthreads();
        for (int j = tid; j < np; j += kThreads) {
            const int64_t i = p0 + j;
            sp[j] = PosQ{x[3 * i] * ilx, x[3 * i + 1] * ily, x[3 * i + 2] * ilz, q[i]};
        }
        __syncthreads();
        const int per = (np + 7) / 8;
        const int jb = wid * per, je = min(jb + per, np);
        for (int j = jb; j < je; ++j) {
            const PosQ p = sp[j];
            double t = fma(mx, p.x, fma(my, p.y, mz * p.z));
            t -= rint(t);
            double s, c;
            sincospi(2.0 * t, &s, &c);
            re = fma(p.q, c, re);
            im = fma(p.q, s, im);
        }
    }
    s_re[wid][lane] = re;
    s_im[wid][lane] = im;
    __syncthreads();
    if (wid == 0 && k < P) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            a += s_re[w][lane];
            b += s_im[w][lane];
        }
        part[(int64_t)k * kGroups + g] = make_double2(a, b);
    }
}

// One warp per frequency: fixed-order FP64 sum of the kGroups partials.
__global__ void __launch_bounds__(256) k_rho_groups_combine(int32_t P, const double2 *__restrict__ part,
                                                            double *__restrict__ rho_out) {
    const int lane = threadIdx.x & 31;
    const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= P) return;
    double re = 0.0, im = 0.0;
    for (int t = lane; t < kGroups; t += 32) {
        const double2 v = part[(int64_t)k * kGroups + t];
        re += v.x;
        im += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        rho_out[2 * k] = re;
        rho_out[2 * k + 1] = im;
    }
}

// Device address of the scratch array, looked up once per CUDA context
// (with that context's device current) the first time the entry point runs
// in it.  The address belongs to the module loaded into that context: after
// a cudaDeviceReset the device gets a new primary context and the array a
// new address, so the cache is keyed on the context's unique id.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
struct ScratchSlot {
    unsigned long long ctx_id;
    double2 *ptr;
};
ScratchSlot g_scratch[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the current context (0 when none is current or on failure),
// through the driver entry points the runtime exposes.
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return 0;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace

extern "C" rbsog_status rbsog_rho_noalloc(int64_t n, const double *q, const double *x, const double *L,
                                          const int32_t *m, int32_t P, double *rho_out, void *stream) {
    if (n < 1 || !q || !x || !L || !m || !rho_out) return RBSOG_EINVAL;
    if (P < 1 || P > RBSOG_NOALLOC_MAX_P) return RBSOG_EINVAL;
    if (!(L[0] > 0.0) || !(L[1] > 0.0) || !(L[2] > 0.0)) return RBSOG_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RBSOG_ECUDA;
    unsigned long long ctx_id = current_ctx_id();
    if (ctx_id == 0) {   // no context current yet: make the device's primary context current
        if (cudaSetDevice(dev) != cudaSuccess) return RBSOG_ECUDA;
        ctx_id = current_ctx_id();
        if (ctx_id == 0) return RBSOG_ECUDA;
    }
    double2 *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        ScratchSlot &sl = g_scratch[dev];
        if (!sl.ptr || sl.ctx_id != ctx_id) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_rho_scratch) != cudaSuccess || !ptr) return RBSOG_ECUDA;
            sl.ptr = static_cast<double2 *>(ptr);
            sl.ctx_id = ctx_id;
        }
        scratch = sl.ptr;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dim3 grid(kGroups, (unsigned)((P + kKTile - 1) / kKTile));
    k_rho_groups<<<grid, kThreads, 0, st>>>(n, q, x, 1.0 / L[0], 1.0 / L[1], 1.0 / L[2], m, P, scratch);
    k_rho_groups_combine<<<(unsigned)(((int64_t)P * 32 + 255) / 256), 256, 0, st>>>(P, scratch, rho_out);
    return cudaGetLastError() == cudaSuccess ? RBSOG_OK : RBSOG_ECUDA;
}
