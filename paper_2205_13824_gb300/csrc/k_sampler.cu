// Frequency sampler of the random batch (Sec. 3.3, Eqs. 3.18-3.22) and the
// pre-sampled sequence of Algorithm 1 (line 2), run as independent
// Metropolis-Hastings chains (the paper's parallel sampling, Sec. 3.4), one
// chain per block.
//
// This translation unit is compiled with -fmad=false: every floating-point
// expression below rounds after each operation, so that the accept/reject
// decisions and the rounded proposals are taken in the same FP64 arithmetic
// as any other IEEE implementation of the same expressions.
#include "rbsog_kernels.cuh"

namespace rbsog {
namespace {

constexpr double kPi = 3.14159265358979323846;

// Unnormalised target mass, proportional to F~(k) of Eq. 3.5 at k = 2 pi m / L.
__device__ double target_mass(const SamplerDev &sp, const double *L, int mx, int my, int mz) {
    const int md[3] = {mx, my, mz};
    double k2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double kd = 2.0 * kPi * (double)md[d] / L[d];
        k2 += kd * kd;
    }
    double acc = 0.0;
    for (int l = 0; l <= sp.M; ++l)
        acc += sp.omega[l] * sp.s[l] * sp.s[l] * sp.s[l] * exp(-sp.s[l] * sp.s[l] * k2 / 4.0);
    return acc;
}

// Proposal mass of one coordinate: the rounded normal of variance
// (L_d / (s_0 pi))^2 / 2, i.e. (1/2)[erf((m+1/2) a) - erf((m-1/2) a)] with
// a = pi s_0 / L_d (Eq. 3.22, without the printed extra 1/2 in the argument).
__device__ double proposal_mass(int m, double s0, double Ld) {
    const double a = kPi * s0 / Ld;
    if (m == 0) return erf(0.5 * a);
    return 0.5 * (erf(((double)m + 0.5) * a) - erf(((double)m - 0.5) * a));
}

// Chain c emits chain_len states into kseq[c * chain_len ...].  Iteration j
// uses the Philox blocks with key (seed, c) and counters (j, 0, 0, 0) (four
// uniforms -> Box-Muller normals for the proposal) and (j, 1, 0, 0) (the
// acceptance uniform).  The first non-zero proposal starts the chain; after
// that each iteration emits the post-decision state.  Zero proposals are
// rejections (p(0) = 0).
//
// The proposals of an independence sampler do not depend on the chain's
// state, so one block runs one chain in rounds of kRound iterations: every
// thread draws one iteration's proposal and evaluates its target and proposal
// masses (the expensive FP64 part) in parallel, then one thread walks the
// round's iterations in order and takes the accept/reject decisions from the
// stored values -- the same values and the same expression as a serial
// chain, so the emitted sequence is identical to it.
constexpr int kRound = 256;

struct Draw {
    int4 m;        // proposal; w = 1 if it is the zero mode
    double p, q;   // target and proposal masses (0 for the zero mode)
    double u;      // acceptance uniform
};

__device__ Draw draw(const SamplerDev &sp, const SamplerSys &y, int64_t c, int64_t j, const double sd[3]) {
    uint64_t ra[4] = {(uint64_t)j, 0, 0, 0};
    uint64_t rb[4] = {(uint64_t)j, 1, 0, 0};
    philox4x64_10(ra, y.seed, (uint64_t)c);
    philox4x64_10(rb, y.seed, (uint64_t)c);
    const double r01 = sqrt(-2.0 * log(1.0 - unit53(ra[0])));
    const double r23 = sqrt(-2.0 * log(1.0 - unit53(ra[2])));
    double z[3];
    z[0] = r01 * cos(2.0 * kPi * unit53(ra[1]));
    z[1] = r01 * sin(2.0 * kPi * unit53(ra[1]));
    z[2] = r23 * cos(2.0 * kPi * unit53(ra[3]));
    int mp[3];
    for (int d = 0; d < 3; ++d) mp[d] = (int)round(z[d] * sd[d]);
    Draw o;
    const bool zero = (mp[0] == 0 && mp[1] == 0 && mp[2] == 0);
    o.m = make_int4(mp[0], mp[1], mp[2], zero ? 1 : 0);
    o.u = unit53(rb[0]);
    if (zero) {
        o.p = o.q = 0.0;
    } else {
        const double s0 = sp.s[0];
        o.p = target_mass(sp, y.L, mp[0], mp[1], mp[2]);
        o.q = proposal_mass(mp[0], s0, y.L[0]) * proposal_mass(mp[1], s0, y.L[1]) *
              proposal_mass(mp[2], s0, y.L[2]);
    }
    return o;
}

__global__ void __launch_bounds__(kRound) k_mh_chain(const __grid_constant__ SamplerDev sp,
                                                     const SamplerSys *__restrict__ sys, int n_sys,
                                                     int64_t total_chains, int4 *__restrict__ kseq,
                                                     int32_t *__restrict__ err_flag) {
    __shared__ Draw s_draw[kRound];
    __shared__ int4 s_out[kRound];
    __shared__ int s_nout, s_done;
    __shared__ int64_t s_base;
    const int tid = threadIdx.x;
    const int64_t g = blockIdx.x;   // global chain
    if (g >= total_chains) return;
    int lo = 0, hi = n_sys;         // system of global chain g: largest lo with chain_off <= g
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sys[mid].chain_off <= g) lo = mid; else hi = mid;
    }
    const SamplerSys &y = sys[lo];
    const int64_t c = g - y.chain_off;           // chain index within its system
    const double s0 = sp.s[0];
    double sd[3];
    for (int d = 0; d < 3; ++d) sd[d] = y.L[d] / (sqrt(2.0) * kPi * s0);
    const int64_t len = y.chain_len;
    const int64_t cap = 64 * len + 4096;
    int4 *out = kseq + y.k_off + c * len;
    // serial state, held by thread 0
    int4 cur = make_int4(0, 0, 0, 0);
    double p_cur = 0.0, q_cur = 0.0;
    bool have = false;
    int64_t emitted = 0;
    for (int64_t j0 = 0;; j0 += kRound) {
        const int64_t j = j0 + tid;
        if (j < cap) s_draw[tid] = draw(sp, y, c, j, sd);
        __syncthreads();
        if (tid == 0) {
            int nout = 0, done = 0;
            for (int k = 0; k < kRound && emitted < len; ++k) {
                if (j0 + k >= cap) {   // bounded: a chain that cannot start reports and stops
                    atomicOr(err_flag, 2);
                    done = 2;
                    break;
                }
                const Draw &dr = s_draw[k];
                const bool zero = dr.m.w != 0;
                if (!have) {
                    if (zero) continue;
                    cur = make_int4(dr.m.x, dr.m.y, dr.m.z, 0);
                    p_cur = dr.p;
                    q_cur = dr.q;
                    have = true;
                } else if (!zero) {
                    const double ratio = (dr.p * q_cur) / (p_cur * dr.q);
                    if (dr.u < ratio) {
                        cur = make_int4(dr.m.x, dr.m.y, dr.m.z, 0);
                        p_cur = dr.p;
                        q_cur = dr.q;
                    }
                }
                s_out[nout++] = cur;
                ++emitted;
            }
            if (emitted >= len && !done) done = 1;
            s_nout = nout;
            s_done = done;
            s_base = emitted - nout;
        }
        __syncthreads();
        const int nout = s_nout, done = s_done;
        const int64_t base = s_base;
        if (tid < nout) out[base + tid] = s_out[tid];
        if (done == 2)   // zero-fill what the stopped chain did not emit
            for (int64_t e = base + nout + tid; e < len; e += kRound) out[e] = make_int4(0, 0, 0, 0);
        if (done) break;
        __syncthreads();   // s_draw / s_out are reused by the next round
    }
}

// One warp per set: the starts of the runs of equal consecutive frequencies
// by ballot (in order), then each run's length from the next start.
__global__ void __launch_bounds__(256) k_fold_sets(const FoldSys *__restrict__ sys, int n_sys, int64_t total_sets,
                                                   int32_t P, const int4 *__restrict__ kseq, int4 *__restrict__ kfold,
                                                   int32_t *__restrict__ kcount) {
    const int lane = threadIdx.x & 31;
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // global set
    if (g >= total_sets) return;
    int lo = 0, hi = n_sys;   // system of set g: largest lo with set_off <= g
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sys[mid].set_off <= g) lo = mid; else hi = mid;
    }
    const FoldSys &y = sys[lo];
    const int64_t s = g - y.set_off;
    const int4 *in = kseq + y.k_off + s * P;
    int4 *out = kfold + y.k_off + s * P;
    int nrun = 0;
    for (int j0 = 0; j0 < P; j0 += 32) {
        const int j = j0 + lane;
        bool start = false;
        int4 m = make_int4(0, 0, 0, 0);
        if (j < P) {
            m = in[j];
            if (j == 0) {
                start = true;
            } else {
                const int4 pr = in[j - 1];
                start = m.x != pr.x || m.y != pr.y || m.z != pr.z;
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, start);
        if (start) out[nrun + __popc(b & ((1u << lane) - 1u))] = make_int4(m.x, m.y, m.z, j);
        nrun += __popc(b);
    }
    __syncwarp();
    for (int t0 = 0; t0 < nrun; t0 += 32) {
        const int t = t0 + lane;
        int len = 0;
        if (t < nrun) len = (t + 1 < nrun ? out[t + 1].w : P) - out[t].w;
        __syncwarp();
        if (t < nrun) out[t].w = len;
        __syncwarp();
    }
    for (int t = nrun + lane; t < P; t += 32) out[t] = make_int4(0, 0, 0, 0);
    if (lane == 0) kcount[y.kc_off + s] = nrun;
}

}  // namespace

cudaError_t launch_fold_kseq(const FoldSys *sys, int n_sys, int64_t total_sets, int32_t P, const int4 *kseq,
                             int4 *kfold, int32_t *kcount, cudaStream_t st) {
    if (total_sets <= 0) return cudaSuccess;
    k_fold_sets<<<(unsigned)((total_sets + 7) / 8), 256, 0, st>>>(sys, n_sys, total_sets, P, kseq, kfold, kcount);
    return cudaGetLastError();
}

cudaError_t launch_mh_sampler(const SamplerDev &sp, const SamplerSys *sys, int n_sys, int64_t total_chains,
                              int4 *kseq, int32_t *err_flag, cudaStream_t st, const Prof *prof) {
    if (total_chains <= 0) return cudaSuccess;
    ProfScope ps(prof, "mh_sampler");
    k_mh_chain<<<(unsigned)total_chains, kRound, 0, st>>>(sp, sys, n_sys, total_chains, kseq, err_flag);
    return cudaGetLastError();
}

}  // namespace rbsog
