// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mcmp2 {

// Pairs of walker pairs are processed in square tiles of TILE_PAIRS pairs per side.
constexpr int TILE_PAIRS_F64 = 8;     // FP64 form: 64 x 64 complex position-component blocks
constexpr int TILE_PAIRS_MIXED = 16;  // mixed form: 128 operand rows per side (each CTA of a pair, M = N = 256 MMAs)
constexpr int TILE_PAIRS_MIXED_2C = 32;  // mixed form, two-component systems: 4 rows per pair in the same 128 rows

// Running statistics of the production steps (Eq. uncertainty), kept on the device.
struct Stats {
    double block_sum, block_comp;  // Kahan sum of the current block's step estimates
    long long in_block;            // steps in the current block
    long long n_blocks;            // complete blocks
    double mean, m2;               // Welford mean and sum of squared deviations of block means
    long long steps;               // production steps
    double all_sum, all_comp;      // Kahan sum over all production steps
    double last;                   // latest I'_n
    unsigned long long accepted;   // accepted Metropolis moves over production steps
};

// Device view of the loaded system (pointers into the caller's workspace).
struct DevSystem {
    int n_centres, n_shells, n_l, n_occ, n_vir, n_orb, m, n_tau;
    const double *centres;     // [n_centres][3]
    const double *wcoef;       // [n_centres][4]: c1 N(zeta1), zeta1, c2 N(zeta2), zeta2
    const int *shell_centre;   // [n_shells]
    const double *shell_alpha; // [n_shells]
    const double *shell_coef;  // [n_shells]
    const int *fn_shell;       // [n_l] shell of each Cartesian function
    const int *fn_pow;         // [n_l][3] Cartesian powers
    const double *eps;         // [n_orb]
    double eps_homo, eps_lumo, lambda, Ng;
    const double *WL;          // FP64 large operand [n_l][2][n_orb][2] (L-alpha, L-beta; re, im)
    const double *WS;          // FP64 small operand [3 n_l][2][n_orb][2] (S-alpha, S-beta)
    int interaction;           // MCMP2_COULOMB, MCMP2_GAUNT or MCMP2_BREIT (four-component systems)
    int n_comp;                // spinor components: 4, or 2 for two-component systems (FP64 form only)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): a counter-based generator.
// Counter layout: {step_lo, step_hi, index, tag}; key = {seed_lo, seed_hi}.
// tag 0/1: Metropolis move of walker pair `index`; tag 2: imaginary time `index`.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 draw4(uint64_t seed, uint64_t step, uint32_t index, uint32_t tag)
{
    return philox4x32_10(make_uint4((uint32_t)step, (uint32_t)(step >> 32), index, tag),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// (0, 1) from 32 bits: (x + 1/2) 2^-32, exact in double.
__device__ __forceinline__ double u32_open(uint32_t x)
{
    return __dmul_rn(__dadd_rn((double)x, 0.5), 2.3283064365386963e-10);
}

// (0, 1] from 53 bits of two words.
__device__ __forceinline__ double u53_half_open(uint32_t a, uint32_t b)
{
    const double v = __dadd_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0), (double)(b >> 6)), 1.0);
    return __dmul_rn(v, 1.0 / 9007199254740992.0);
}

// Optional record of the per-element values of one tile of the pair-of-pairs sum
// (mcmp2_debug_elements): for the tile (bp, bq) of tp x tp walker pairs,
// out[(t tp + i) tp + j] = Re f/(w w w) of p = bp tp + i, q = bq tp + j at time t
// (0 where p >= q or either index is past m).  out == nullptr: nothing recorded.
struct DebugTile {
    double *out = nullptr;
    int bp = -1, bq = -1;
};

// Records ev on st; while st is being captured into a graph the record becomes
// an external event node, so the event can be read after each replay.
inline cudaError_t record_event(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, st);
}

// ---------------------------------------------------------------------------
// Launch wrappers (defined in the kernel translation units).  All take the
// context's stream and return cudaGetLastError() of the launch.
// ---------------------------------------------------------------------------
cudaError_t launch_metropolis(const DevSystem &s, double *r, const unsigned long long *step,
                              uint64_t seed, double delta, unsigned long long *accepted, double *a,
                              cudaStream_t st);
cudaError_t launch_pair_weights(const DevSystem &s, const double *r, double *a, cudaStream_t st);
cudaError_t launch_times(const DevSystem &s, const unsigned long long *step, uint64_t seed,
                         const double *tau_given, double *tau, double *scale, float *scale_f, cudaStream_t st);
cudaError_t launch_advance_step(unsigned long long *step, cudaStream_t st);
cudaError_t launch_initial_walkers(const DevSystem &s, double *r, uint64_t seed, const double *cdf, cudaStream_t st);

template <typename T>
cudaError_t launch_basis(const DevSystem &s, const double *r, T *B, cudaStream_t st);

cudaError_t launch_spinors_f64(const DevSystem &s, const double *B, double *phi, cudaStream_t st);
cudaError_t prepare_f64();  // sets the FP64 contraction kernel's shared-memory limit
// r (positions [m][2][3]) is read for the Breit gauge term only; it may be null otherwise.
cudaError_t launch_pairs_f64(const DevSystem &s, const double *phi, const double *scale,
                             const double *a, double *partials, cudaStream_t st, const double *r = nullptr,
                             const DebugTile &dbg = DebugTile{});

size_t adjoint_smem_bytes();
cudaError_t launch_adjoint_time(const DevSystem &s, const double *B, const double *phi, const double *scale,
                                const double *tau, const double *a, int t_index, double norm, double *Ybar,
                                double *Ys, double *partials, double *GWL, double *GWS, double *d_eps,
                                cudaStream_t st);

// Reduction scratch: RED_BLOCKS (sum, error) pairs and a completion counter.
constexpr int RED_BLOCKS = 64;
struct ReduceScratch {
    double sum[RED_BLOCKS], err[RED_BLOCKS];
    unsigned int done;
};
cudaError_t launch_reduce(const DevSystem &s, const double *partials, int n_tiles, double *out_slot,
                          Stats *stats, int update_stats, unsigned long long *step_to_advance,
                          ReduceScratch *scratch, cudaStream_t st, const int *abort_flag = nullptr);

__host__ __device__ inline int pair_blocks(int m, int tile_pairs) { return (m + tile_pairs - 1) / tile_pairs; }
// Tiles of the upper triangle, counted in 64 bits: for the largest m the API
// accepts (MAX_WALKER_PAIRS) the count stays far below 2^31.
__host__ __device__ inline long long n_tiles_for(int m, int tile_pairs)
{
    const long long nb = pair_blocks(m, tile_pairs);
    return nb * (nb + 1) / 2;
}
// Largest number of walker pairs any entry point accepts: 8,390,656 FP64 tiles
// of 8 pairs, so every tile count and grid dimension fits an int.
constexpr int MAX_WALKER_PAIRS = 1 << 16;
constexpr int MAX_TAU = 64;  // imaginary times per step
constexpr int MAX_CENTRES = 256;  // atoms (the Metropolis kernel stages 4 x 4 x n_centres doubles per block)

}  // namespace mcmp2
