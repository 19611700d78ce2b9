// Sampling kernels: Metropolis walk of the electron pairs (Sec. III, Metropolis
// sampling of w(r1,r2)), the per-pair weight factors, and the inverse-CDF
// imaginary times with the per-orbital propagator scales.
#include "internal.cuh"

namespace mcmp2 {

// One Metropolis step for every walker pair: both electrons move by a uniform
// displacement in [-delta, delta]^3; the move is accepted with probability
// min(1, w'/w) with w = g(r1) g(r2) / r12 (the 1/N_g cancels).  FP64 with
// explicit rounding so the same counters give the same walk on the host.
// g is FP64-exp bound on GB300, so its terms are spread over the block: one
// thread per (pair, position, centre) evaluates that centre's two Gaussians at
// one of the pair's four positions (old and proposed r1, r2), and one thread per
// pair then adds the centres in index order (every operation rounded as written,
// no contraction, so the same counters give the same walk on the host) and decides the
// move.  The pair's weight factor a_p = N_g / (g(r1) g(r2)) at the resulting
// positions is written as well (a may be null).
constexpr int MET_PAIRS = 4;     // walker pairs per block
constexpr int MET_THREADS = 128;

// Centre i's two Gaussians of the weight function g(r) of Eq. basisSet at (x, y, z),
// with c N(zeta) folded on the host; every operation is rounded as written.
__device__ __forceinline__ double centre_term(const DevSystem &s, int i, double x, double y, double z)
{
    const double dx = __dsub_rn(x, s.centres[3 * i + 0]);
    const double dy = __dsub_rn(y, s.centres[3 * i + 1]);
    const double dz = __dsub_rn(z, s.centres[3 * i + 2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double *w = s.wcoef + 4 * i;
    const double t1 = __dmul_rn(w[0], exp(__dmul_rn(-w[1], d2)));
    const double t2 = __dmul_rn(w[2], exp(__dmul_rn(-w[3], d2)));
    return __dadd_rn(t1, t2);
}

__global__ void __launch_bounds__(MET_THREADS) metropolis_kernel(DevSystem s, double *__restrict__ r,
                                                                 const unsigned long long *__restrict__ step_ptr,
                                                                 uint64_t seed, double delta,
                                                                 unsigned long long *__restrict__ accepted,
                                                                 double *__restrict__ a)
{
    extern __shared__ double terms[];          // [MET_PAIRS][4][n_centres]
    __shared__ double spos[MET_PAIRS][4][3];   // old r1, old r2, proposed r1, proposed r2
    __shared__ uint32_t su[MET_PAIRS];         // the acceptance draw
    __shared__ unsigned int sacc;
    const int nc = s.n_centres;
    const int p0 = blockIdx.x * MET_PAIRS;
    if (threadIdx.x == 0) sacc = 0;
    if (threadIdx.x < MET_PAIRS) {
        const int lp = threadIdx.x, p = p0 + lp;
        if (p < s.m) {
            const uint64_t step = *step_ptr;
            const uint4 A = draw4(seed, step, (uint32_t)p, 0u);
            const uint4 B = draw4(seed, step, (uint32_t)p, 1u);
            const uint32_t u[7] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z};
            const double *r1 = r + 6 * p, *r2 = r1 + 3;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double o1 = r1[k], o2 = r2[k];
                spos[lp][0][k] = o1;
                spos[lp][1][k] = o2;
                spos[lp][2][k] = __dadd_rn(o1, __dmul_rn(delta, __dsub_rn(__dmul_rn(2.0, u32_open(u[k])), 1.0)));
                spos[lp][3][k] = __dadd_rn(o2, __dmul_rn(delta, __dsub_rn(__dmul_rn(2.0, u32_open(u[3 + k])), 1.0)));
            }
            su[lp] = u[6];
        }
    }
    __syncthreads();
    const int per_pair = 4 * nc;
    for (int w = threadIdx.x; w < MET_PAIRS * per_pair; w += MET_THREADS) {
        const int lp = w / per_pair, rem = w - lp * per_pair;
        const int j = rem / nc, i = rem - j * nc;
        if (p0 + lp < s.m) terms[w] = centre_term(s, i, spos[lp][j][0], spos[lp][j][1], spos[lp][j][2]);
    }
    __syncthreads();
    if (threadIdx.x < MET_PAIRS) {
        const int lp = threadIdx.x, p = p0 + lp;
        if (p < s.m) {
            double g[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {  // g = sum over the centres in index order
                double v = 0.0;
                for (int i = 0; i < nc; ++i) v = __dadd_rn(v, terms[lp * per_pair + j * nc + i]);
                g[j] = v;
            }
            auto r12 = [](const double *x1, const double *x2) {
                const double dx = __dsub_rn(x1[0], x2[0]), dy = __dsub_rn(x1[1], x2[1]), dz = __dsub_rn(x1[2], x2[2]);
                return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
            };
            const double w_old = __ddiv_rn(__dmul_rn(g[0], g[1]), r12(spos[lp][0], spos[lp][1]));
            const double w_new = __ddiv_rn(__dmul_rn(g[2], g[3]), r12(spos[lp][2], spos[lp][3]));
            double ga = g[0], gb = g[1];
            if (__dmul_rn(u32_open(su[lp]), w_old) < w_new) {
                double *r1 = r + 6 * p, *r2 = r1 + 3;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    r1[k] = spos[lp][2][k];
                    r2[k] = spos[lp][3][k];
                }
                ga = g[2];
                gb = g[3];
                atomicAdd(&sacc, 1u);
            }
            if (a) a[p] = s.Ng / (ga * gb);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && sacc) atomicAdd(accepted, (unsigned long long)sacc);  // one atomic per block
}

// a_p = N_g / (g(r1p) g(r2p)): with 1/(w w) this is the weight factor of a pair of
// pairs.  As in the Metropolis kernel, one thread per (pair, position, centre)
// evaluates that centre's Gaussians and one thread per pair adds the centres in
// index order, with the Metropolis kernel's rounding.
constexpr int PW_PAIRS = 8;  // walker pairs per block
constexpr int PW_THREADS = 128;
__global__ void __launch_bounds__(PW_THREADS) pair_weights_kernel(DevSystem s, const double *__restrict__ r,
                                                                  double *__restrict__ a)
{
    extern __shared__ double pw_terms[];  // [PW_PAIRS][2][n_centres]
    const int nc = s.n_centres;
    const int p0 = blockIdx.x * PW_PAIRS;
    const int per_pair = 2 * nc;
    for (int w = threadIdx.x; w < PW_PAIRS * per_pair; w += PW_THREADS) {
        const int lp = w / per_pair, rem = w - lp * per_pair;
        const int j = rem / nc, i = rem - j * nc;
        if (p0 + lp < s.m) {
            const double *x = r + 6 * (p0 + lp) + 3 * j;
            pw_terms[w] = centre_term(s, i, x[0], x[1], x[2]);
        }
    }
    __syncthreads();
    if (threadIdx.x < PW_PAIRS && p0 + threadIdx.x < s.m) {
        const double *t = pw_terms + threadIdx.x * per_pair;
        double g1 = 0.0, g2 = 0.0;
        for (int i = 0; i < nc; ++i) g1 = __dadd_rn(g1, t[i]);
        for (int i = 0; i < nc; ++i) g2 = __dadd_rn(g2, t[nc + i]);
        a[p0 + threadIdx.x] = __ddiv_rn(s.Ng, __dmul_rn(g1, g2));
    }
}

// Imaginary times and propagator scales for one step.  Block t handles time t:
// tau_t = -ln(u)/lambda (analytic inverse CDF of Eq. tauWeight) unless given,
// then scale[t][i] = exp((eps_i - eps_HOMO) tau/2) for occupied and
// scale[t][a] = exp(-(eps_a - eps_LUMO) tau/2) for virtual spinors, so that a
// product X X^dagger of scaled spinor values carries exp(+eps_i tau) or
// exp(-eps_a tau) times exp(-eps_HOMO tau) or exp(+eps_LUMO tau); every factor
// is at most 1 and the four shifts of a pair of pairs multiply to exp(lambda tau).
// Block (c, t) handles orbitals 128 c .. 128 c + 127 of time t (each block draws
// the time itself; FP64 exp is slow on GB300, so the orbitals are spread wide).
constexpr int TIMES_THREADS = 128;
__global__ void __launch_bounds__(TIMES_THREADS) times_kernel(DevSystem s,
                                                              const unsigned long long *__restrict__ step_ptr,
                                                              uint64_t seed, const double *__restrict__ tau_given,
                                                              double *__restrict__ tau, double *__restrict__ scale,
                                                              float *__restrict__ scale_f)
{
    const int t = blockIdx.y;
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
        if (blockIdx.x == 0) tau[t] = v;
    }
    __syncthreads();
    const double x = tt;
    for (int k = blockIdx.x * TIMES_THREADS + threadIdx.x; k < s.n_orb; k += gridDim.x * TIMES_THREADS) {
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
    const size_t smem = sizeof(double) * MET_PAIRS * 4 * s.n_centres;  // 256 centres fit the default 48 KB
    metropolis_kernel<<<(s.m + MET_PAIRS - 1) / MET_PAIRS, MET_THREADS, smem, st>>>(s, r, step, seed, delta,
                                                                                    accepted, a);
    return cudaGetLastError();
}

cudaError_t launch_pair_weights(const DevSystem &s, const double *r, double *a, cudaStream_t st)
{
    const size_t smem = sizeof(double) * PW_PAIRS * 2 * s.n_centres;  // 256 centres: 32 KB
    pair_weights_kernel<<<(s.m + PW_PAIRS - 1) / PW_PAIRS, PW_THREADS, smem, st>>>(s, r, a);
    return cudaGetLastError();
}

cudaError_t launch_times(const DevSystem &s, const unsigned long long *step, uint64_t seed,
                         const double *tau_given, double *tau, double *scale, float *scale_f, cudaStream_t st)
{
    const dim3 grid((s.n_orb + TIMES_THREADS - 1) / TIMES_THREADS, s.n_tau);
    times_kernel<<<grid, TIMES_THREADS, 0, st>>>(s, step, seed, tau_given, tau, scale, scale_f);
    return cudaGetLastError();
}

cudaError_t launch_advance_step(unsigned long long *step, cudaStream_t st)
{
    advance_step_kernel<<<1, 1, 0, st>>>(step);
    return cudaGetLastError();
}

}  // namespace mcmp2
