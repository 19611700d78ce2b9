// Step reduction and blocking statistics: I'_n of Eq. redundant from the
// per-tile partial sums, and the Flyvbjerg-Petersen accumulators of
// Eq. uncertainty, in FP64 with compensated sums and a fixed summation order.
#include "internal.cuh"

namespace mcmp2 {

__device__ __forceinline__ void kahan_add(double &s, double &c, double x)
{
    const double y = x - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
}

// One block of 256 threads.  partials: [n_tau][n_tiles].
__global__ void __launch_bounds__(256) reduce_kernel(int n_tau, int m, const double *__restrict__ partials,
                                                     int n_tiles, double *__restrict__ out_slot,
                                                     Stats *__restrict__ st, int update,
                                                     unsigned long long *__restrict__ step)
{
    __shared__ double sv[256], sc[256];
    const int total = n_tau * n_tiles;
    double s = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < total; i += 256) kahan_add(s, c, partials[i]);
    sv[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double S = 0.0, C = 0.0;
    for (int i = 0; i < 256; ++i) {
        kahan_add(S, C, sv[i]);
        kahan_add(S, C, -sc[i]);
    }
    const double npairs = 0.5 * (double)m * (double)(m - 1);
    const double value = S / npairs / (double)n_tau;
    *out_slot = value;
    if (update) {
        st->last = value;
        st->steps += 1;
        kahan_add(st->all_sum, st->all_comp, value);
        kahan_add(st->block_sum, st->block_comp, value);
        st->in_block += 1;
        if (st->in_block == 100) {  // N_b = 100 (Sec. IV)
            const double bm = st->block_sum / 100.0;
            st->n_blocks += 1;
            const double d = bm - st->mean;
            st->mean += d / (double)st->n_blocks;
            st->m2 += d * (bm - st->mean);
            st->block_sum = 0.0;
            st->block_comp = 0.0;
            st->in_block = 0;
        }
    }
    if (step) *step += 1ull;
}

cudaError_t launch_reduce(const DevSystem &s, const double *partials, int n_tiles, double *out_slot,
                          Stats *stats, int update_stats, unsigned long long *step_to_advance,
                          cudaStream_t st)
{
    reduce_kernel<<<1, 256, 0, st>>>(s.n_tau, s.m, partials, n_tiles, out_slot, stats, update_stats,
                                     step_to_advance);
    return cudaGetLastError();
}

}  // namespace mcmp2
