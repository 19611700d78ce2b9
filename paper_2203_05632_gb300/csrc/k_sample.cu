// Sampling kernels: Metropolis walk of the electron pairs (Sec. III, Metropolis
// sampling of w(r1,r2)), the per-pair weight factors, and the inverse-CDF
// imaginary times with the per-orbital propagator scales.
#include "internal.cuh"

namespace mcmp2 {

// One Metropolis step for every walker pair: both electrons move by a uniform
// displacement in [-delta, delta]^3; the move is accepted with probability
// min(1, w'/w) with w = g(r1) g(r2) / r12 (the 1/N_g cancels).  FP64 with
// explicit rounding so the same counters give the same walk on the host.
// Four lanes share a pair: lane j evaluates g for electron j&1 at the old (j<2)
// or proposed (j>=2) position (g is FP64-exp bound on GB300).  The pair's
// weight factor a_p = N_g / (g(r1) g(r2)) at the resulting positions is
// written as well (a may be null).
__global__ void metropolis_kernel(DevSystem s, double *__restrict__ r,
                                  const unsigned long long *__restrict__ step_ptr, uint64_t seed,
                                  double delta, unsigned long long *__restrict__ accepted, double *__restrict__ a)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = gid >> 2, j = gid & 3;
    const bool live = p < s.m;
    const int lane = threadIdx.x & 31, g0 = lane & ~3;
    double pos[3] = {0.0, 0.0, 0.0};
    double o1[3] = {0.0, 0.0, 0.0}, o2[3] = {0.0, 0.0, 0.0}, n1[3] = {0.0, 0.0, 0.0}, n2[3] = {0.0, 0.0, 0.0};
    uint32_t u_acc = 0;
    if (live) {
        const uint64_t step = *step_ptr;
        const uint4 A = draw4(seed, step, (uint32_t)p, 0u);
        const uint4 B = draw4(seed, step, (uint32_t)p, 1u);
        const uint32_t u[7] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z};
        const double *r1 = r + 6 * p, *r2 = r1 + 3;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o1[k] = r1[k];
            o2[k] = r2[k];
            n1[k] = __dadd_rn(o1[k], __dmul_rn(delta, __dsub_rn(__dmul_rn(2.0, u32_open(u[k])), 1.0)));
            n2[k] = __dadd_rn(o2[k], __dmul_rn(delta, __dsub_rn(__dmul_rn(2.0, u32_open(u[3 + k])), 1.0)));
        }
        u_acc = u[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) pos[k] = (j == 0) ? o1[k] : (j == 1) ? o2[k] : (j == 2) ? n1[k] : n2[k];
    }
    const double gj = live ? weight_g(s, pos[0], pos[1], pos[2]) : 1.0;
    const double g1o = __shfl_sync(0xffffffffu, gj, g0 + 0), g2o = __shfl_sync(0xffffffffu, gj, g0 + 1);
    const double g1n = __shfl_sync(0xffffffffu, gj, g0 + 2), g2n = __shfl_sync(0xffffffffu, gj, g0 + 3);
    unsigned int acc = 0;
    if (live && j == 0) {
        auto r12 = [](const double *x1, const double *x2) {
            const double dx = __dsub_rn(x1[0], x2[0]), dy = __dsub_rn(x1[1], x2[1]), dz = __dsub_rn(x1[2], x2[2]);
            return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        };
        const double w_old = __ddiv_rn(__dmul_rn(g1o, g2o), r12(o1, o2));
        const double w_new = __ddiv_rn(__dmul_rn(g1n, g2n), r12(n1, n2));
        double *r1 = r + 6 * p, *r2 = r1 + 3;
        double ga = g1o, gb = g2o;
        if (__dmul_rn(u32_open(u_acc), w_old) < w_new) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                r1[k] = n1[k];
                r2[k] = n2[k];
            }
            ga = g1n;
            gb = g2n;
            acc = 1;
        }
        if (a) a[p] = s.Ng / (ga * gb);
    }
    // One atomic per warp.
    const unsigned int total = __reduce_add_sync(0xffffffffu, acc);
    if (lane == 0 && total) atomicAdd(accepted, (unsigned long long)total);
}

// a_p = N_g / (g(r1p) g(r2p)): with 1/(w w) this is the weight factor of a pair of pairs.
__global__ void pair_weights_kernel(DevSystem s, const double *__restrict__ r, double *__restrict__ a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.m) return;
    const double *r1 = r + 6 * p, *r2 = r1 + 3;
    const double g1 = weight_g(s, r1[0], r1[1], r1[2]);
    const double g2 = weight_g(s, r2[0], r2[1], r2[2]);
    a[p] = s.Ng / (g1 * g2);
}

// Imaginary times and propagator scales for one step.  Block t handles time t:
// tau_t = -ln(u)/lambda (analytic inverse CDF of Eq. tauWeight) unless given,
// then scale[t][i] = exp((eps_i - eps_HOMO) tau/2) for occupied and
// scale[t][a] = exp(-(eps_a - eps_LUMO) tau/2) for virtual spinors, so that a
// product X X^dagger of scaled spinor values carries exp(+eps_i tau) or
// exp(-eps_a tau) times exp(-eps_HOMO tau) or exp(+eps_LUMO tau); every factor
// is at most 1 and the four shifts of a pair of pairs multiply to exp(lambda tau).
__global__ void times_kernel(DevSystem s, const unsigned long long *__restrict__ step_ptr, uint64_t seed,
                             const double *__restrict__ tau_given, double *__restrict__ tau,
                             double *__restrict__ scale, float *__restrict__ scale_f)
{
    const int t = blockIdx.x;
    __shared__ double tt;
    if (threadIdx.x == 0) {
        double v;
        if (tau_given) {
            v = tau_given[t];
        } else {
            const uint4 o = draw4(seed, *step_ptr, (uint32_t)t, 2u);
            v = -log(u53_half_open(o.x, o.y)) / s.lambda;
        }
        tt = v;
        tau[t] = v;
    }
    __syncthreads();
    const double x = tt;
    for (int k = threadIdx.x; k < s.n_orb; k += blockDim.x) {
        const double e = s.eps[k];
        const double arg = (k < s.n_occ) ? (e - s.eps_homo) : -(e - s.eps_lumo);
        const double v = exp(0.5 * arg * x);
        scale[(size_t)t * s.n_orb + k] = v;
        if (scale_f) scale_f[(size_t)t * s.n_orb + k] = (float)v;
    }
}

__global__ void advance_step_kernel(unsigned long long *step) { *step += 1ull; }

// Initial positions drawn from g(r1) g(r2): each electron independently from the
// Gaussian mixture g (component k of centre I with probability proportional to
// its mass c_k N(zeta_k) (pi/zeta_k)^{3/2}, given as a cumulative table cdf
// [2 n_centres]), normal deviates of variance 1/(2 zeta) by Box-Muller.
// Counters: {lo, hi} of the reserved step 2^64 - 1, index = pair, tags 3 and 4.
__global__ void initial_walkers_kernel(DevSystem s, double *__restrict__ r, uint64_t seed,
                                       const double *__restrict__ cdf)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.m) return;
    const uint64_t step = ~0ull;
    for (int e = 0; e < 2; ++e) {
        const uint4 a = draw4(seed, step, (uint32_t)p, 3u + 2u * e);
        const uint4 b = draw4(seed, step, (uint32_t)p, 4u + 2u * e);
        const double uc = u32_open(a.x);
        int comp = 2 * s.n_centres - 1;
        for (int i = 0; i < 2 * s.n_centres; ++i)
            if (uc < cdf[i]) {
                comp = i;
                break;
            }
        const int ic = comp >> 1;
        const double zeta = s.wcoef[4 * ic + 1 + 2 * (comp & 1)];
        const double sigma = sqrt(0.5 / zeta);
        const double u1 = u32_open(a.y), u2 = u32_open(a.z), u3 = u32_open(b.x), u4 = u32_open(b.y);
        const double rad1 = sqrt(-2.0 * log(u1)), rad2 = sqrt(-2.0 * log(u3));
        const double z0 = rad1 * cos(6.283185307179586 * u2), z1 = rad1 * sin(6.283185307179586 * u2);
        const double z2 = rad2 * cos(6.283185307179586 * u4);
        double *x = r + 6 * p + 3 * e;
        x[0] = s.centres[3 * ic + 0] + sigma * z0;
        x[1] = s.centres[3 * ic + 1] + sigma * z1;
        x[2] = s.centres[3 * ic + 2] + sigma * z2;
    }
}

cudaError_t launch_initial_walkers(const DevSystem &s, double *r, uint64_t seed, const double *cdf, cudaStream_t st)
{
    initial_walkers_kernel<<<(s.m + 127) / 128, 128, 0, st>>>(s, r, seed, cdf);
    return cudaGetLastError();
}

cudaError_t launch_metropolis(const DevSystem &s, double *r, const unsigned long long *step,
                              uint64_t seed, double delta, unsigned long long *accepted, double *a,
                              cudaStream_t st)
{
    const int threads = 64;  // FP64 exp-bound: spread the 4 m lanes over as many SMs as possible
    const int lanes = 4 * s.m;
    metropolis_kernel<<<(lanes + threads - 1) / threads, threads, 0, st>>>(s, r, step, seed, delta, accepted, a);
    return cudaGetLastError();
}

cudaError_t launch_pair_weights(const DevSystem &s, const double *r, double *a, cudaStream_t st)
{
    const int threads = 32;
    pair_weights_kernel<<<(s.m + threads - 1) / threads, threads, 0, st>>>(s, r, a);
    return cudaGetLastError();
}

cudaError_t launch_times(const DevSystem &s, const unsigned long long *step, uint64_t seed,
                         const double *tau_given, double *tau, double *scale, float *scale_f, cudaStream_t st)
{
    times_kernel<<<s.n_tau, 256, 0, st>>>(s, step, seed, tau_given, tau, scale, scale_f);
    return cudaGetLastError();
}

cudaError_t launch_advance_step(unsigned long long *step, cudaStream_t st)
{
    advance_step_kernel<<<1, 1, 0, st>>>(step);
    return cudaGetLastError();
}

}  // namespace mcmp2
