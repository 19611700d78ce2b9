// Step reduction and blocking statistics: I'_n of Eq. redundant from the
// per-tile partial sums, and the Flyvbjerg-Petersen accumulators of
// Eq. uncertainty, in FP64 with compensated sums and a fixed summation order.
#include "../../include/mcmp2.h"
#include "internal.cuh"

namespace mcmp2 {

constexpr int MCMP2_BLOCK = MCMP2_BLOCK_SIZE;

__device__ __forceinline__ void kahan_add(double &s, double &c, double x)
{
    const double y = x - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
}

// Error-free sum of two doubles: s + err == a + b exactly.
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &err)
{
    s = a + b;
    const double bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

constexpr int RED_THREADS = 256;

// Combine (sum, error) pairs held in shared memory by a fixed pairwise tree.
__device__ void tree_reduce(double *sv, double *se, int n_active)
{
    for (int stride = RED_THREADS / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride && threadIdx.x + stride < n_active) {
            double sum, err;
            two_sum(sv[threadIdx.x], sv[threadIdx.x + stride], sum, err);
            sv[threadIdx.x] = sum;
            se[threadIdx.x] += se[threadIdx.x + stride] + err;
        }
        __syncthreads();
    }
}

// RED_BLOCKS blocks each reduce a fixed contiguous slice of partials
// [n_tau][n_tiles] with compensated sums and a pairwise tree of error-free
// additions; the last block to finish combines the slices in block order and
// updates the statistics.  The result does not depend on scheduling.
__global__ void __launch_bounds__(RED_THREADS) reduce_kernel(int n_tau, int m, const double *__restrict__ partials,
                                                             int n_tiles, double *__restrict__ out_slot,
                                                             Stats *__restrict__ st, int update,
                                                             unsigned long long *__restrict__ step,
                                                             ReduceScratch *__restrict__ scratch,
                                                             const int *__restrict__ abort_flag)
{
    __shared__ double sv[RED_THREADS], se[RED_THREADS];
    __shared__ bool last;
    const int total = n_tau * n_tiles;
    const int per = (total + RED_BLOCKS - 1) / RED_BLOCKS;
    const int lo = blockIdx.x * per, hi = min(total, lo + per);
    double s = 0.0, c = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += RED_THREADS) kahan_add(s, c, partials[i]);
    sv[threadIdx.x] = s;
    se[threadIdx.x] = -c;
    __syncthreads();
    tree_reduce(sv, se, RED_THREADS);
    if (threadIdx.x == 0) {
        scratch->sum[blockIdx.x] = sv[0];
        scratch->err[blockIdx.x] = se[0];
        __threadfence();
        last = atomicAdd(&scratch->done, 1u) == RED_BLOCKS - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    sv[threadIdx.x] = threadIdx.x < RED_BLOCKS ? ((volatile double *)scratch->sum)[threadIdx.x] : 0.0;
    se[threadIdx.x] = threadIdx.x < RED_BLOCKS ? ((volatile double *)scratch->err)[threadIdx.x] : 0.0;
    __syncthreads();
    tree_reduce(sv, se, RED_BLOCKS);
    if (threadIdx.x != 0) return;
    scratch->done = 0;
    const double S = sv[0] + se[0];
    const double npairs = 0.5 * (double)m * (double)(m - 1);
    const double value = S / npairs / (double)n_tau;
    // A contraction that gave up on a wait left some partial sums unwritten:
    // report no estimate and leave the statistics untouched.
    const bool aborted = abort_flag && *(volatile const int *)abort_flag;
    *out_slot = aborted ? __longlong_as_double(0x7ff8000000000000ll) : value;
    if (update && !aborted) {
        st->last = value;
        st->steps += 1;
        kahan_add(st->all_sum, st->all_comp, value);
        kahan_add(st->block_sum, st->block_comp, value);
        st->in_block += 1;
        if (st->in_block == MCMP2_BLOCK) {  // N_b = 100 (Sec. IV)
            const double bm = st->block_sum / (double)MCMP2_BLOCK;
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
                          ReduceScratch *scratch, cudaStream_t st, const int *abort_flag)
{
    reduce_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(s.n_tau, s.m, partials, n_tiles, out_slot, stats, update_stats,
                                                       step_to_advance, scratch, abort_flag);
    return cudaGetLastError();
}

}  // namespace mcmp2
