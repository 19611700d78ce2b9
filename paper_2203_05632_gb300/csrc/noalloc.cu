// Allocation-free variant of the FP64 pair-of-pairs contraction.
//
// The regular path keeps the per-tile partial sums in the caller's
// workspace.  This variant keeps them in a fixed-size array that lives in the
// library's own device memory, so a caller needs no device allocation at all:
// it passes its inputs and its output and nothing else.
#include <mutex>

#include "../../include/mcmp2.h"
#include "internal.cuh"

namespace {

// Scratch for the per-tile partial sums of one call: [n_tau][n_tiles] doubles.
// Every GPU that loads the library holds this array until the process exits.
// The reduction's per-block (sum, error) pairs and completion counter follow
// the partial sums in the same array.
constexpr size_t NOALLOC_MAX_PARTIALS = MCMP2_NOALLOC_MAX_PARTIALS;
constexpr size_t REDUCE_DOUBLES = (sizeof(mcmp2::ReduceScratch) + sizeof(double) - 1) / sizeof(double);
static __device__ __align__(256) double g_pair_partials[NOALLOC_MAX_PARTIALS + REDUCE_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double *g_partials_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code only sees a host-side stand-in under the array's name).
// The cached address is not refreshed: a device reset after the first call on
// that device is not supported (the header says so).
int scratch_address(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MCMP2_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_pair_partials) != cudaSuccess || !p) return MCMP2_ECUDA;
        g_partials_addr[dev] = static_cast<double *>(p);
    }
    *out = g_partials_addr[dev];
    return MCMP2_OK;
}

}  // namespace

extern "C" int mcmp2_pair_sum_f64_noalloc(int m, int n_occ, int n_vir, int n_tau, const double *phi,
                                          const double *scale, const double *a, double lambda, double *out,
                                          void *cuda_stream)
{
    if (m < 2 || n_occ < 1 || n_vir < 1 || n_tau < 1 || m > mcmp2::MAX_WALKER_PAIRS || n_tau > mcmp2::MAX_TAU ||
        n_occ + n_vir > 65536 || !phi || !scale || !a || !out || !(lambda > 0.0) || lambda == __builtin_inf())
        return MCMP2_EINVAL;
    // 64-bit count (at most 8.4e6 tiles for the largest m), checked before any narrowing.
    const long long n_tiles = mcmp2::n_tiles_for(m, mcmp2::TILE_PAIRS_F64);
    if ((unsigned long long)n_tiles * (unsigned long long)n_tau > NOALLOC_MAX_PARTIALS) return MCMP2_ENOSPACE;
    double *partials = nullptr;
    const int rc = scratch_address(&partials);
    if (rc != MCMP2_OK) return rc;
    mcmp2::DevSystem s{};
    s.m = m;
    s.n_occ = n_occ;
    s.n_vir = n_vir;
    s.n_orb = n_occ + n_vir;
    s.n_tau = n_tau;
    s.lambda = lambda;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // Every partial is written by its tile before the reduction reads it, so
    // the partials need no clearing; the reduction's completion counter must
    // start at zero and is cleared here (a plain memset, no allocation).
    auto *red = reinterpret_cast<mcmp2::ReduceScratch *>(partials + NOALLOC_MAX_PARTIALS);
    if (cudaMemsetAsync(&red->done, 0, sizeof(red->done), st) != cudaSuccess) return MCMP2_ECUDA;
    if (mcmp2::launch_pairs_f64(s, phi, scale, a, partials, st) != cudaSuccess) return MCMP2_ECUDA;
    if (mcmp2::launch_reduce(s, partials, (int)n_tiles, out, nullptr, 0, nullptr, red, st) != cudaSuccess)
        return MCMP2_ECUDA;
    return MCMP2_OK;
}
