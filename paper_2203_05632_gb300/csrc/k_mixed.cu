// Mixed-precision integrand engine on the tcgen05 tensor cores (sm_103a).
//
// Per step:
//  1. basis_split_kernel: basis values and gradients at the 2m positions (FP32)
//     as BF16 hi/lo planes (value = hi + lo to ~2^-17).
//  2. spinor_mixed_kernel: spinor formation (Eq. C with kinetic balance) as a
//     real split-BF16 x3 GEMM, phi = [g | grad g] x W (W = C folded with the
//     Pauli matrices), FP32 accumulate in tensor memory.  Its epilogue scales
//     the spinor values by s_k(tau) for every imaginary time and writes the
//     BF16 hi/lo planes of X(x)_ck = phi_k^c(x) s_k(tau): rows 4x + c,
//     occupied and virtual orbitals in separate planes.
//  3. pairs_mixed_kernel: for every (16 x 16 walker-pair tile, tau) the
//     Hermitian products G(x, y)_cd = sum_k X(x)_ck conj(X(y)_dk) over the
//     occupied (G-) and virtual (G+) orbitals,
//       Re G = Xr Yr^T + Xi Yi^T,  Im G = Xi Yr^T - Xr Yi^T,
//     each real product as hi*hi + hi*lo + lo*hi (12 MMAs per 16-deep K step),
//     then the direct and exchange traces of the trace form of Eq. MCMP2 for
//     every pair of pairs, accumulated in FP64 as Re f / (w w w).
// Every wait is bounded in time; on a time-out a kernel records it in a flag,
// stops, drains its own copies, frees tensor memory and returns, and the host
// reports MCMP2_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "../../include/mcmp2.h"
#include "mixed.cuh"
#include "tc_common.cuh"

namespace mcmp2 {

using namespace tc;

namespace {

constexpr unsigned long long TIMEOUT_NS = 2000000000ull;  // 2 s per wait
constexpr int BK = 32;                                    // K elements per stage row (64 B, one swizzle row)
constexpr int TILE_BYTES = 128 * BK * 2;                  // one 128 x 32 BF16 operand tile (8 KB)

__device__ __forceinline__ int n_chunks(int k) { return (k + BK - 1) / BK; }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// ===========================================================================
// 1. Basis values as split BF16 planes
// ===========================================================================
__global__ void basis_split_kernel(DevSystem s, const double *__restrict__ r, __nv_bfloat16 *__restrict__ BLh,
                                   __nv_bfloat16 *__restrict__ BLl, __nv_bfloat16 *__restrict__ BSh,
                                   __nv_bfloat16 *__restrict__ BSl, int nl_pad, int nl3_pad)
{
    const int x = blockIdx.y;
    const int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu >= s.n_l) return;
    const int sh = s.fn_shell[mu];
    const double *A = s.centres + 3 * s.shell_centre[sh];
    const float d[3] = {(float)(r[3 * x + 0] - A[0]), (float)(r[3 * x + 1] - A[1]), (float)(r[3 * x + 2] - A[2])};
    const float al = (float)s.shell_alpha[sh];
    const float e = (float)s.shell_coef[sh] * expf(-al * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
    const int pw[3] = {s.fn_pow[3 * mu], s.fn_pow[3 * mu + 1], s.fn_pow[3 * mu + 2]};
    float pk[3], dk[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float v = 1.f, lower = 0.f;
        for (int i = 0; i < pw[j]; ++i) v *= d[j];
        if (pw[j] > 0) {
            lower = 1.f;
            for (int i = 0; i < pw[j] - 1; ++i) lower *= d[j];
            lower *= (float)pw[j];
        }
        pk[j] = v;
        dk[j] = lower - 2.f * al * v * d[j];
    }
    float vals[4] = {pk[0] * pk[1] * pk[2] * e, dk[0] * pk[1] * pk[2] * e, pk[0] * dk[1] * pk[2] * e,
                     pk[0] * pk[1] * dk[2] * e};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(vals[j]);
        const __nv_bfloat16 lo = __float2bfloat16_rn(vals[j] - __bfloat162float(hi));
        if (j == 0) {
            BLh[(size_t)x * nl_pad + mu] = hi;
            BLl[(size_t)x * nl_pad + mu] = lo;
        } else {
            const size_t o = (size_t)x * nl3_pad + (size_t)(j - 1) * s.n_l + mu;
            BSh[o] = hi;
            BSl[o] = lo;
        }
    }
}

// ===========================================================================
// 2. Spinor formation with fused scale-and-split epilogue
// ===========================================================================
constexpr int SP_STAGES = 4;
constexpr int SP_STAGE_BYTES = 4 * TILE_BYTES;  // A hi, A lo, B hi, B lo
constexpr int SP_THREADS = 192;                 // TMA warp, MMA warp, 4 epilogue warps
constexpr int SP_TMEM_COLS = 256;               // two 128-column accumulators
constexpr int SP_MAX_TAU = 64;                  // scale staging capacity (the API limits n_tau to 64)
constexpr int SP_ROW_BYTES = 144;               // staged row: 64 BF16 (128 B) + 16 B pad against bank conflicts
constexpr int SP_WARP_STAGE = 4 * 32 * SP_ROW_BYTES;  // 4 planes x 32 rows per epilogue warp
constexpr int SP_BARS_OFF = SP_STAGES * SP_STAGE_BYTES;
constexpr int SP_SCALE_OFF = SP_BARS_OFF + (2 * SP_STAGES + 4) * 8 + 16;
constexpr int SP_WSTAGE_OFF = SP_SCALE_OFF + SP_MAX_TAU * 64 * 4;
constexpr int SP_SMEM = SP_WSTAGE_OFF + 4 * SP_WARP_STAGE + 1024;

struct SpinorMaps {
    CUtensorMap m[8];  // 0..3: A_L hi, A_L lo, B_L hi, B_L lo; 4..7: the same for the gradient part
};

struct SpinorArgs {
    const float *scale;   // [n_tau][n_orb]
    __nv_bfloat16 *occ;   // [n_tau][4][rows][k_occ_pad]
    __nv_bfloat16 *vir;   // [n_tau][4][rows][k_vir_pad]
    int *abort_flag;
    int P, nl, n_mt, n_kb, n_kb_occ, n_occ, n_vir, n_orb, n_tau, rows, k_occ_pad, k_vir_pad;
};

__device__ __forceinline__ void sp_tile(int tile, int n_kb, int &mt, int &c4, int &kb)
{
    const int per = 4 * n_kb;
    mt = tile / per;
    const int nt = tile - mt * per;
    c4 = nt / n_kb;
    kb = nt - c4 * n_kb;
}

__global__ void __launch_bounds__(SP_THREADS, 1) spinor_mixed_kernel(const __grid_constant__ SpinorMaps maps,
                                                                     const SpinorArgs args)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + SP_BARS_OFF);
    uint64_t *empty = full + SP_STAGES;
    uint64_t *tfull = empty + SP_STAGES;  // [2]
    uint64_t *tempty = tfull + 2;         // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = args.n_mt * 4 * args.n_kb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SP_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init_fence();
    }
    if (warp == 1) tmem_alloc(tmem_slot, SP_TMEM_COLS);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            for (int i = 0; i < 8; ++i) tma_prefetch(&maps.m[i]);
            int stage = 0;
            uint32_t phase = 0;
            int issued[SP_STAGES] = {};
            uint32_t issued_phase[SP_STAGES] = {};
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                int mt, c4, kb;
                sp_tile(tile, args.n_kb, mt, c4, kb);
                const bool grad = c4 >= 2;
                const CUtensorMap *mp = &maps.m[grad ? 4 : 0];
                const int K = grad ? 3 * args.nl : args.nl;
                const int wt_row = ((c4 & 1) * args.n_kb + kb) * 128;
                for (int c = 0; c < n_chunks(K); ++c) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, args.abort_flag, 11, TIMEOUT_NS)) {
                        ok = false;
                        break;
                    }
                    unsigned char *st = smem + stage * SP_STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[stage], SP_STAGE_BYTES);
                    tma_load_2d(st + 0 * TILE_BYTES, mp + 0, &full[stage], c * BK, mt * 128);
                    tma_load_2d(st + 1 * TILE_BYTES, mp + 1, &full[stage], c * BK, mt * 128);
                    tma_load_2d(st + 2 * TILE_BYTES, mp + 2, &full[stage], c * BK, wt_row);
                    tma_load_2d(st + 3 * TILE_BYTES, mp + 3, &full[stage], c * BK, wt_row);
                    issued[stage] = 1;
                    issued_phase[stage] = phase;
                    if (++stage == SP_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok)
                for (int s = 0; s < SP_STAGES; ++s)
                    if (issued[s]) mbar_drain(&full[s], issued_phase[s], TIMEOUT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0, buf = 0;
            uint32_t phase = 0, tphase[2] = {0, 0};
            bool ok = true;
            const uint32_t id = idesc_bf16(128, false);
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                int mt, c4, kb;
                sp_tile(tile, args.n_kb, mt, c4, kb);
                const int K = c4 >= 2 ? 3 * args.nl : args.nl;
                if (!mbar_wait(&tempty[buf], tphase[buf] ^ 1u, args.abort_flag, 12, TIMEOUT_NS)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + 128u * buf;
                for (int c = 0; c < n_chunks(K); ++c) {
                    if (!mbar_wait(&full[stage], phase, args.abort_flag, 13, TIMEOUT_NS)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const int kvalid = K - c * BK;
                    const int ksteps = kvalid >= BK ? BK / 16 : (kvalid + 15) / 16;
                    const uint32_t base = smem_u32(smem + stage * SP_STAGE_BYTES);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint32_t off = ks * 32;
                        const uint64_t ah = sdesc_sw64(base + 0 * TILE_BYTES + off);
                        const uint64_t al = sdesc_sw64(base + 1 * TILE_BYTES + off);
                        const uint64_t bh = sdesc_sw64(base + 2 * TILE_BYTES + off);
                        const uint64_t bl = sdesc_sw64(base + 3 * TILE_BYTES + off);
                        umma(d, ah, bh, id, (c == 0 && ks == 0) ? 0u : 1u);
                        umma(d, ah, bl, id, 1u);
                        umma(d, al, bh, id, 1u);
                    }
                    umma_commit(&empty[stage]);
                    if (++stage == SP_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                umma_commit(&tfull[buf]);
                tphase[buf] ^= 1u;
                buf ^= 1;
            }
            // Let every MMA this thread issued finish before tensor memory is freed.
            umma_commit(&empty[stage]);
            mbar_drain(&empty[stage], phase, TIMEOUT_NS);
        }
    } else {
        // Epilogue: each lane owns one position row of the tile.  For every time
        // the warp stages its 32 rows x 64 orbitals of the 4 planes in shared
        // memory, then writes them as whole 128-byte row segments (8 lanes per
        // row), so each store instruction touches 4 lines instead of 32.
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
        float *sscale = reinterpret_cast<float *>(smem + SP_SCALE_OFF);  // [n_tau][64]
        unsigned char *wstage = smem + SP_WSTAGE_OFF + ew * SP_WARP_STAGE;
        int buf = 0;
        uint32_t ephase[2] = {0, 0};
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            int mt, c4, kb;
            sp_tile(tile, args.n_kb, mt, c4, kb);
            const bool got = mbar_wait(&tfull[buf], ephase[buf], args.abort_flag, 14, TIMEOUT_NS);
            if (bar_any<1, 128>(!got)) break;  // also: every epilogue warp is done with the previous scales
            ephase[buf] ^= 1u;
            fence_after();
            const bool occ = kb < args.n_kb_occ;
            const int kl = occ ? kb : kb - args.n_kb_occ;
            const int kpad = occ ? args.k_occ_pad : args.k_vir_pad;
            const int k_first = (occ ? 0 : args.n_occ) + kl * 64;  // absolute index of the block's first orbital
            const int k_end = occ ? args.n_occ : args.n_orb;       // one past the region's last orbital
            __nv_bfloat16 *planes = occ ? args.occ : args.vir;
            const size_t plane_elems = (size_t)args.rows * kpad;
            for (int i = threadIdx.x - 64; i < 64 * args.n_tau; i += 128) {
                const int t = i >> 6, k = k_first + (i & 63);
                sscale[i] = k < k_end ? args.scale[(size_t)t * args.n_orb + k] : 0.f;
            }
            bar_sync<1, 128>();
            for (int t = 0; t < args.n_tau; ++t) {
                const float *st_ = sscale + 64 * t;
#pragma unroll 1
                for (int j = 0; j < 4; ++j) {
                    float re[16], im[16];
                    tmem_ld<16>(lane_addr + 128u * buf + 16u * j, re);
                    tmem_ld<16>(lane_addr + 128u * buf + 64u + 16u * j, im);
                    tmem_wait_ld();
                    uint32_t rh[8], rl[8], ih[8], il[8];
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const float s0 = st_[16 * j + i], s1 = st_[16 * j + i + 1];
                        const float xr0 = re[i] * s0, xr1 = re[i + 1] * s1;
                        const float xi0 = im[i] * s0, xi1 = im[i + 1] * s1;
                        const __nv_bfloat162 hr = __floats2bfloat162_rn(xr0, xr1);
                        const __nv_bfloat162 hi = __floats2bfloat162_rn(xi0, xi1);
                        rh[i / 2] = *reinterpret_cast<const uint32_t *>(&hr);
                        ih[i / 2] = *reinterpret_cast<const uint32_t *>(&hi);
                        rl[i / 2] = pack_bf16(xr0 - __low2float(hr), xr1 - __high2float(hr));
                        il[i / 2] = pack_bf16(xi0 - __low2float(hi), xi1 - __high2float(hi));
                    }
                    unsigned char *myrow = wstage + lane * SP_ROW_BYTES + 32 * j;
                    uint4 *d0 = reinterpret_cast<uint4 *>(myrow), *d1 = reinterpret_cast<uint4 *>(myrow + 32 * SP_ROW_BYTES);
                    uint4 *d2 = reinterpret_cast<uint4 *>(myrow + 64 * SP_ROW_BYTES);
                    uint4 *d3 = reinterpret_cast<uint4 *>(myrow + 96 * SP_ROW_BYTES);
                    d0[0] = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                    d0[1] = make_uint4(rh[4], rh[5], rh[6], rh[7]);
                    d1[0] = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                    d1[1] = make_uint4(rl[4], rl[5], rl[6], rl[7]);
                    d2[0] = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                    d2[1] = make_uint4(ih[4], ih[5], ih[6], ih[7]);
                    d3[0] = make_uint4(il[0], il[1], il[2], il[3]);
                    d3[1] = make_uint4(il[4], il[5], il[6], il[7]);
                }
                __syncwarp();
                const int chunk = lane & 7;
#pragma unroll
                for (int pl = 0; pl < 4; ++pl)
#pragma unroll
                    for (int it = 0; it < 8; ++it) {
                        const int r_in = 4 * it + (lane >> 3);
                        const int x = mt * 128 + 32 * quarter + r_in;
                        if (x < args.P) {
                            const uint4 v =
                                *reinterpret_cast<const uint4 *>(wstage + pl * 32 * SP_ROW_BYTES + r_in * SP_ROW_BYTES +
                                                                 16 * chunk);
                            __nv_bfloat16 *dst = planes + ((size_t)t * 4 + pl) * plane_elems + (size_t)(4 * x + c4) * kpad +
                                                 kl * 64 + 8 * chunk;
                            *reinterpret_cast<uint4 *>(dst) = v;
                        }
                    }
                __syncwarp();
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            buf ^= 1;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, SP_TMEM_COLS);
    }
}

// ===========================================================================
// 3. Pair-of-pairs contraction with the trace epilogue
// ===========================================================================
constexpr int PR_STAGES = 3;
constexpr int PR_STAGE_BYTES = 8 * TILE_BYTES;  // A: re_hi, re_lo, im_hi, im_lo; B: the same
constexpr int PR_EPI_WARPS = 8;                 // two per tensor-memory lane quarter
constexpr int PR_THREADS = 64 + 32 * PR_EPI_WARPS;
constexpr int PR_TMEM_COLS = 512;               // G+ re | G+ im | G- re | G- im
constexpr int PR_BARS_OFF = PR_STAGES * PR_STAGE_BYTES;
constexpr int PR_RED_OFF = PR_BARS_OFF + (2 * PR_STAGES + 2) * 8 + 16;
constexpr int PR_SMEM = PR_RED_OFF + 32 * 8 + 1024;

struct PairMaps {
    CUtensorMap occ, vir;  // 3-D: (orbital, row, 4 tau + plane)
};

struct PairArgs {
    const double *a;   // [m] pair weight factors N_g / (g1 g2)
    double *partials;  // [n_tau][n_tiles]
    int *abort_flag;
    int m, n_tiles, nb, n_tau, n_occ, n_vir;
    double inv_lambda;
    unsigned long long timeout_ns;  // limit of every wait
    int withhold_first_copy;        // test hook: never issue the first stage's copy (its wait runs out)
};

__device__ __forceinline__ void pair_tile(int tile, int nb, int &bp, int &bq)
{
    int k = tile, b = 0;
    while (k >= nb - b) {
        k -= nb - b;
        ++b;
    }
    bp = b;
    bq = b + k;
}

__global__ void __launch_bounds__(PR_THREADS, 1) pairs_mixed_kernel(const __grid_constant__ PairMaps maps,
                                                                    const PairArgs args)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + PR_BARS_OFF);
    uint64_t *empty = full + PR_STAGES;
    uint64_t *tmem_full = empty + PR_STAGES;
    uint64_t *tmem_empty = tmem_full + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tmem_empty + 1);
    double *red = reinterpret_cast<double *>(smem + PR_RED_OFF);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_occ_chunks = n_chunks(args.n_occ), n_vir_chunks = n_chunks(args.n_vir);
    const int chunks_per_tile = n_occ_chunks + n_vir_chunks;
    const int n_items = args.n_tiles * args.n_tau;

    if (threadIdx.x == 0) {
        for (int s = 0; s < PR_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tmem_full, 1);
        mbar_init(tmem_empty, PR_EPI_WARPS);
        mbar_init_fence();
    }
    if (warp == 1) tmem_alloc(tmem_slot, PR_TMEM_COLS);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            tma_prefetch(&maps.occ);
            tma_prefetch(&maps.vir);
            int stage = 0;
            uint32_t phase = 0;
            int issued[PR_STAGES] = {};
            uint32_t issued_phase[PR_STAGES] = {};
            bool ok = true;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const int t = item / args.n_tiles, tile = item - t * args.n_tiles;
                int bp, bq;
                pair_tile(tile, args.nb, bp, bq);
                for (int c = 0; c < chunks_per_tile; ++c) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, args.abort_flag, 1, args.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    if (args.withhold_first_copy && item == (int)blockIdx.x && c == 0) {
                        // Test hook: skip this stage entirely; nothing completes its barrier.
                        if (++stage == PR_STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                        continue;
                    }
                    const bool occ = c < n_occ_chunks;
                    const int x = (occ ? c : c - n_occ_chunks) * BK;
                    const CUtensorMap *mp = occ ? &maps.occ : &maps.vir;
                    unsigned char *st = smem + stage * PR_STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[stage], PR_STAGE_BYTES);
#pragma unroll
                    for (int pl = 0; pl < 4; ++pl) {
                        tma_load_3d(st + pl * TILE_BYTES, mp, &full[stage], x, bp * 128, 4 * t + pl);
                        tma_load_3d(st + (4 + pl) * TILE_BYTES, mp, &full[stage], x, bq * 128, 4 * t + pl);
                    }
                    issued[stage] = 1;
                    issued_phase[stage] = phase;
                    if (++stage == PR_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok)
                for (int s = 0; s < PR_STAGES; ++s)
                    if (issued[s]) mbar_drain(&full[s], issued_phase[s], args.timeout_ns);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, tphase = 0;
            bool ok = true;
            const uint32_t id_pos = idesc_bf16(128, false), id_neg = idesc_bf16(128, true);
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                if (!mbar_wait(tmem_empty, tphase ^ 1u, args.abort_flag, 2, args.timeout_ns)) {
                    ok = false;
                    break;
                }
                fence_after();
                for (int c = 0; c < chunks_per_tile; ++c) {
                    if (!mbar_wait(&full[stage], phase, args.abort_flag, 3, args.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const bool occ = c < n_occ_chunks;
                    const int cc = occ ? c : c - n_occ_chunks;
                    const int kvalid = (occ ? args.n_occ : args.n_vir) - cc * BK;
                    const int ksteps = kvalid >= BK ? BK / 16 : (kvalid + 15) / 16;
                    const uint32_t d_re = tmem + (occ ? 256u : 0u), d_im = d_re + 128u;
                    const uint32_t base = smem_u32(smem + stage * PR_STAGE_BYTES);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint32_t off = ks * 32;
                        const uint64_t arh = sdesc_sw64(base + 0 * TILE_BYTES + off);
                        const uint64_t arl = sdesc_sw64(base + 1 * TILE_BYTES + off);
                        const uint64_t aih = sdesc_sw64(base + 2 * TILE_BYTES + off);
                        const uint64_t ail = sdesc_sw64(base + 3 * TILE_BYTES + off);
                        const uint64_t brh = sdesc_sw64(base + 4 * TILE_BYTES + off);
                        const uint64_t brl = sdesc_sw64(base + 5 * TILE_BYTES + off);
                        const uint64_t bih = sdesc_sw64(base + 6 * TILE_BYTES + off);
                        const uint64_t bil = sdesc_sw64(base + 7 * TILE_BYTES + off);
                        const uint32_t acc = (cc == 0 && ks == 0) ? 0u : 1u;
                        // Re G += Xr Yr^T + Xi Yi^T
                        umma(d_re, arh, brh, id_pos, acc);
                        umma(d_re, arh, brl, id_pos, 1u);
                        umma(d_re, arl, brh, id_pos, 1u);
                        umma(d_re, aih, bih, id_pos, 1u);
                        umma(d_re, aih, bil, id_pos, 1u);
                        umma(d_re, ail, bih, id_pos, 1u);
                        // Im G += Xi Yr^T - Xr Yi^T
                        umma(d_im, aih, brh, id_pos, acc);
                        umma(d_im, aih, brl, id_pos, 1u);
                        umma(d_im, ail, brh, id_pos, 1u);
                        umma(d_im, arh, bih, id_neg, 1u);
                        umma(d_im, arh, bil, id_neg, 1u);
                        umma(d_im, arl, bih, id_neg, 1u);
                    }
                    umma_commit(&empty[stage]);
                    if (++stage == PR_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                umma_commit(tmem_full);
                tphase ^= 1u;
            }
            umma_commit(&empty[stage]);
            mbar_drain(&empty[stage], phase, args.timeout_ns);
        }
    } else {
        // ---------------- epilogue (8 warps, two per lane quarter) ----------------
        const int ew = warp - 2;
        const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
        const int qhalf = ew >> 2;     // q-pairs 8*qhalf .. +7 of the tile
        const int row = 32 * quarter + lane;
        const int p_local = row >> 3, e = (row >> 2) & 1, c = lane & 3;
        const int gbase = lane & ~7;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
        uint32_t ephase = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            const int t = item / args.n_tiles, tile = item - t * args.n_tiles;
            int bp, bq;
            pair_tile(tile, args.nb, bp, bq);
            const bool got = mbar_wait(tmem_full, ephase, args.abort_flag, 4, args.timeout_ns);
            if (bar_any<1, 32 * PR_EPI_WARPS>(!got)) break;  // all epilogue warps leave together
            ephase ^= 1u;
            fence_after();
            const int p = bp * 16 + p_local;
            // a_q of the tile's 16 q-pairs, one per lane (lane & 15), fetched by shuffle below.
            const int q_lane = bq * 16 + (lane & 15);
            const double a_lane = q_lane < args.m ? args.a[q_lane] : 0.0;
            double acc = 0.0;  // sum over this warp's q of Re f_pq a_q
            for (int qb = 0; qb < 4; ++qb) {
                const int q0 = 8 * qhalf + 2 * qb;  // two q-pairs per tensor-memory load
                float gpr[16], gpi[16], gmr[16], gmi[16];
                const uint32_t col = 8u * q0;
                tmem_ld<16>(lane_addr + col, gpr);
                tmem_ld<16>(lane_addr + 128u + col, gpi);
                tmem_ld<16>(lane_addr + 256u + col, gmr);
                tmem_ld<16>(lane_addr + 384u + col, gmi);
                tmem_wait_ld();
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) {
                    // This lane holds row c of G-(xe, ye) [own], G+(xe, ye) [dia], G+(xe, y(1-e)) [off].
                    float own_r[4], own_i[4], dia_r[4], dia_i[4], off_r[4], off_i[4];
#pragma unroll
                    for (int d = 0; d < 4; ++d) {  // constant indices keep the arrays in registers
                        const int i0 = 8 * qq + d, i1 = 8 * qq + 4 + d;
                        own_r[d] = e ? gmr[i1] : gmr[i0];
                        own_i[d] = e ? gmi[i1] : gmi[i0];
                        dia_r[d] = e ? gpr[i1] : gpr[i0];
                        dia_i[d] = e ? gpi[i1] : gpi[i0];
                        off_r[d] = e ? gpr[i0] : gpr[i1];
                        off_i[d] = e ? gpi[i0] : gpi[i1];
                    }
                    // Direct: T_e = sum_cd conj(G-_cd) G+_cd over the like-electron block.
                    float tr = 0.f, ti = 0.f;
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        tr += own_r[d] * dia_r[d] + own_i[d] * dia_i[d];
                        ti += own_r[d] * dia_i[d] - own_i[d] * dia_r[d];
                    }
                    tr += __shfl_xor_sync(0xffffffffu, tr, 1);
                    ti += __shfl_xor_sync(0xffffffffu, ti, 1);
                    tr += __shfl_xor_sync(0xffffffffu, tr, 2);
                    ti += __shfl_xor_sync(0xffffffffu, ti, 2);
                    const float ur = __shfl_xor_sync(0xffffffffu, tr, 4);
                    const float ui = __shfl_xor_sync(0xffffffffu, ti, 4);
                    const float direct_re = tr * ur - ti * ui;
                    // Exchange: tr[G-(1q,1p) G+(1p,2q) G-(2q,2p) G+(2p,1q)] = sum_{c,c''} U_{cc''} V_{c''c},
                    // U = G+(1p,2q) G-(2p,2q)^dag, V = G+(2p,1q) G-(1p,1q)^dag.  Lane (e, c) pairs its
                    // rows with lane (1-e, c''): e = 0 takes c'' - c = 0, 1 and e = 1 takes 2, 3 (mod 4).
                    float xr = 0.f;
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const int src = gbase + (e == 0 ? 4 + ((c + s) & 3) : ((c + 2 - s) & 3));
                        float rg_r[4], rg_i[4], ro_r[4], ro_i[4];
#pragma unroll
                        for (int d = 0; d < 4; ++d) {
                            rg_r[d] = __shfl_sync(0xffffffffu, own_r[d], src);
                            rg_i[d] = __shfl_sync(0xffffffffu, own_i[d], src);
                            ro_r[d] = __shfl_sync(0xffffffffu, off_r[d], src);
                            ro_i[d] = __shfl_sync(0xffffffffu, off_i[d], src);
                        }
                        float a1r = 0.f, a1i = 0.f, a2r = 0.f, a2i = 0.f;
#pragma unroll
                        for (int d = 0; d < 4; ++d) {
                            a1r += off_r[d] * rg_r[d] + off_i[d] * rg_i[d];
                            a1i += off_i[d] * rg_r[d] - off_r[d] * rg_i[d];
                            a2r += ro_r[d] * own_r[d] + ro_i[d] * own_i[d];
                            a2i += ro_i[d] * own_r[d] - ro_r[d] * own_i[d];
                        }
                        xr += a1r * a2r - a1i * a2i;
                    }
                    xr += __shfl_xor_sync(0xffffffffu, xr, 1);
                    xr += __shfl_xor_sync(0xffffffffu, xr, 2);
                    xr += __shfl_xor_sync(0xffffffffu, xr, 4);
                    const int ql = q0 + qq;
                    const int q = bq * 16 + ql;
                    const double a_q = __shfl_sync(0xffffffffu, a_lane, ql);
                    const bool valid = p < args.m && q < args.m && (bp < bq || p_local < ql);
                    if (valid) acc += (double)(-0.5f * (direct_re - xr)) * a_q;
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_empty);
            if ((lane & 7) == 0) red[16 * qhalf + 4 * quarter + (lane >> 3)] = (p < args.m) ? acc * args.a[p] : 0.0;
            bar_sync<1, 32 * PR_EPI_WARPS>();
            if (ew == 0 && lane == 0) {
                double sum = 0.0;
                for (int j = 0; j < 32; ++j) sum += red[j];
                args.partials[(size_t)t * args.n_tiles + tile] = sum * args.inv_lambda;
            }
            bar_sync<1, 32 * PR_EPI_WARPS>();
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, PR_TMEM_COLS);
    }
}

// ===========================================================================
// Host side
// ===========================================================================
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
int round8(int x) { return (x + 7) / 8 * 8; }

uint16_t f2bf(float f)  // round to nearest even (finite inputs)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf2f(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// 2-D (or 3-D) BF16 tensor map with 64-byte swizzle and a 32 x 128 box.
int encode(void *out, void *addr, int rank, const cuuint64_t *dims, const cuuint64_t *strides, std::string &err)
{
    auto enc = encode_fn();
    if (!enc) {
        err = "cuTensorMapEncodeTiled is not available from the driver";
        return MCMP2_EUNSUPPORTED;
    }
    const cuuint32_t box[3] = {(cuuint32_t)BK, 128u, 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap map;
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, addr, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return MCMP2_ECUDA;
    }
    std::memcpy(out, &map, sizeof(map));
    return MCMP2_OK;
}

}  // namespace

MixedLayout mixed_layout(int m, int n_l, int n_occ, int n_vir, int n_tau, size_t offset)
{
    MixedLayout L{};
    L.nl = n_l;
    L.nl_pad = round8(n_l);
    L.nl3_pad = round8(3 * n_l);
    L.n_kb_occ = (n_occ + 63) / 64;
    L.n_kb_vir = (n_vir + 63) / 64;
    L.n_kb = L.n_kb_occ + L.n_kb_vir;
    L.wt_rows = 2 * L.n_kb * 128;
    L.P = 2 * m;
    L.rows = 8 * m;
    L.k_occ_pad = (n_occ + 63) / 64 * 64;  // whole 64-orbital blocks: each staged row segment is one 128 B line
    L.k_vir_pad = (n_vir + 63) / 64 * 64;
    L.n_tau = n_tau;
    size_t off = align256(offset);
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.BL_hi = take((size_t)L.P * L.nl_pad * 2);
    L.BL_lo = take((size_t)L.P * L.nl_pad * 2);
    L.BS_hi = take((size_t)L.P * L.nl3_pad * 2);
    L.BS_lo = take((size_t)L.P * L.nl3_pad * 2);
    L.WTL_hi = take((size_t)L.wt_rows * L.nl_pad * 2);
    L.WTL_lo = take((size_t)L.wt_rows * L.nl_pad * 2);
    L.WTS_hi = take((size_t)L.wt_rows * L.nl3_pad * 2);
    L.WTS_lo = take((size_t)L.wt_rows * L.nl3_pad * 2);
    L.occ_planes = take((size_t)n_tau * 4 * L.rows * L.k_occ_pad * 2);
    L.vir_planes = take((size_t)n_tau * 4 * L.rows * L.k_vir_pad * 2);
    L.flag = take(sizeof(int));
    L.end = off;
    return L;
}

int mixed_prepare(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, const double *WL,
                  const double *WS, cudaStream_t st, std::string &err)
{
    plan.ready = false;
    const int nl = s.n_l, no = s.n_orb;
    // Transposed coefficient planes: row (c, kb, ri, kk) of component c, 64-orbital block kb
    // (occupied blocks first), real/imaginary part ri, orbital kk of the block; column = basis index.
    std::vector<uint16_t> lh((size_t)L.wt_rows * L.nl_pad, 0), ll(lh.size(), 0);
    std::vector<uint16_t> sh((size_t)L.wt_rows * L.nl3_pad, 0), sl(sh.size(), 0);
    for (int c = 0; c < 2; ++c)
        for (int kb = 0; kb < L.n_kb; ++kb)
            for (int ri = 0; ri < 2; ++ri)
                for (int kk = 0; kk < 64; ++kk) {
                    int k;
                    if (kb < L.n_kb_occ) {
                        k = kb * 64 + kk;
                        if (k >= s.n_occ) continue;
                    } else {
                        const int kv = (kb - L.n_kb_occ) * 64 + kk;
                        if (kv >= s.n_vir) continue;
                        k = s.n_occ + kv;
                    }
                    const size_t row = ((size_t)(c * L.n_kb + kb) * 2 + ri) * 64 + kk;
                    for (int mu = 0; mu < nl; ++mu) {
                        const float w = (float)WL[(((size_t)mu * 2 + c) * no + k) * 2 + ri];
                        const uint16_t h = f2bf(w);
                        lh[row * L.nl_pad + mu] = h;
                        ll[row * L.nl_pad + mu] = f2bf(w - bf2f(h));
                    }
                    for (int j = 0; j < 3; ++j)
                        for (int mu = 0; mu < nl; ++mu) {
                            const float w = (float)WS[((((size_t)j * nl + mu) * 2 + c) * no + k) * 2 + ri];
                            const uint16_t h = f2bf(w);
                            sh[row * L.nl3_pad + (size_t)j * nl + mu] = h;
                            sl[row * L.nl3_pad + (size_t)j * nl + mu] = f2bf(w - bf2f(h));
                        }
                }
    if (cudaMemcpyAsync(ws + L.WTL_hi, lh.data(), lh.size() * 2, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ws + L.WTL_lo, ll.data(), ll.size() * 2, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ws + L.WTS_hi, sh.data(), sh.size() * 2, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ws + L.WTS_lo, sl.data(), sl.size() * 2, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(ws + L.flag, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        err = "copying the mixed-form operands failed";
        return MCMP2_ECUDA;
    }
    // Tensor maps.  Spinor formation: A = basis planes [P][K], B = transposed coefficients [wt_rows][K].
    int rc;
    {
        const cuuint64_t dl[2] = {(cuuint64_t)nl, (cuuint64_t)L.P}, sl_[1] = {(cuuint64_t)L.nl_pad * 2};
        const cuuint64_t ds[2] = {(cuuint64_t)3 * nl, (cuuint64_t)L.P}, ss_[1] = {(cuuint64_t)L.nl3_pad * 2};
        const cuuint64_t wl[2] = {(cuuint64_t)nl, (cuuint64_t)L.wt_rows};
        const cuuint64_t wsd[2] = {(cuuint64_t)3 * nl, (cuuint64_t)L.wt_rows};
        if ((rc = encode(plan.maps_spinor[0], ws + L.BL_hi, 2, dl, sl_, err)) ||
            (rc = encode(plan.maps_spinor[1], ws + L.BL_lo, 2, dl, sl_, err)) ||
            (rc = encode(plan.maps_spinor[2], ws + L.WTL_hi, 2, wl, sl_, err)) ||
            (rc = encode(plan.maps_spinor[3], ws + L.WTL_lo, 2, wl, sl_, err)) ||
            (rc = encode(plan.maps_spinor[4], ws + L.BS_hi, 2, ds, ss_, err)) ||
            (rc = encode(plan.maps_spinor[5], ws + L.BS_lo, 2, ds, ss_, err)) ||
            (rc = encode(plan.maps_spinor[6], ws + L.WTS_hi, 2, wsd, ss_, err)) ||
            (rc = encode(plan.maps_spinor[7], ws + L.WTS_lo, 2, wsd, ss_, err)))
            return rc;
    }
    // Contraction: planes [4 n_tau][rows][k_pad] as a 3-D tensor (orbital, row, 4 tau + plane).
    {
        const cuuint64_t dO[3] = {(cuuint64_t)s.n_occ, (cuuint64_t)L.rows, (cuuint64_t)4 * L.n_tau};
        const cuuint64_t sO[2] = {(cuuint64_t)L.k_occ_pad * 2, (cuuint64_t)L.rows * L.k_occ_pad * 2};
        const cuuint64_t dV[3] = {(cuuint64_t)s.n_vir, (cuuint64_t)L.rows, (cuuint64_t)4 * L.n_tau};
        const cuuint64_t sV[2] = {(cuuint64_t)L.k_vir_pad * 2, (cuuint64_t)L.rows * L.k_vir_pad * 2};
        if ((rc = encode(plan.maps_pairs[0], ws + L.occ_planes, 3, dO, sO, err)) ||
            (rc = encode(plan.maps_pairs[1], ws + L.vir_planes, 3, dV, sV, err)))
            return rc;
    }
    if (cudaFuncSetAttribute(spinor_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SP_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM) !=
            cudaSuccess) {
        err = "cannot reserve shared memory for the tensor-core kernels";
        return MCMP2_ECUDA;
    }
    plan.ready = true;
    return MCMP2_OK;
}

int mixed_step(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, const double *r,
               const float *scale, const double *a, double *partials, cudaStream_t st, std::string &err,
               cudaEvent_t *ev, int *n_launches, int *n_pair_launches)
{
    if (!plan.ready) {
        err = "mixed path not prepared";
        return MCMP2_ENOTLOADED;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int *flag = reinterpret_cast<int *>(ws + L.flag);
    auto bf = [&](size_t off) { return reinterpret_cast<__nv_bfloat16 *>(ws + off); };

    dim3 gb((s.n_l + 127) / 128, L.P);
    basis_split_kernel<<<gb, 128, 0, st>>>(s, r, bf(L.BL_hi), bf(L.BL_lo), bf(L.BS_hi), bf(L.BS_lo), L.nl_pad,
                                           L.nl3_pad);

    SpinorMaps smaps;
    std::memcpy(&smaps, plan.maps_spinor, sizeof(smaps));
    const int n_mt = (L.P + 127) / 128;
    SpinorArgs sa{scale, bf(L.occ_planes), bf(L.vir_planes), flag, L.P, s.n_l, n_mt, L.n_kb, L.n_kb_occ,
                  s.n_occ, s.n_vir, s.n_orb, s.n_tau, L.rows, L.k_occ_pad, L.k_vir_pad};
    const int sp_tiles = n_mt * 4 * L.n_kb;
    spinor_mixed_kernel<<<sp_tiles < sms ? sp_tiles : sms, SP_THREADS, SP_SMEM, st>>>(smaps, sa);

    PairMaps pmaps;
    std::memcpy(&pmaps.occ, plan.maps_pairs[0], sizeof(CUtensorMap));
    std::memcpy(&pmaps.vir, plan.maps_pairs[1], sizeof(CUtensorMap));
    const int nb = pair_blocks(s.m, 16);
    const int n_tiles = nb * (nb + 1) / 2;
    PairArgs pa{a, partials, flag, s.m, n_tiles, nb, s.n_tau, s.n_occ, s.n_vir, 1.0 / s.lambda, TIMEOUT_NS, 0};
    if (plan.withhold_once_ns) {
        pa.withhold_first_copy = 1;
        pa.timeout_ns = plan.withhold_once_ns;
        plan.withhold_once_ns = 0;
    }
    const int items = n_tiles * s.n_tau;
    if (ev) record_event(ev[0], st);
    pairs_mixed_kernel<<<items < sms ? items : sms, PR_THREADS, PR_SMEM, st>>>(pmaps, pa);
    if (ev) record_event(ev[1], st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("mixed-form launch: ") + cudaGetErrorString(e);
        return MCMP2_ECUDA;
    }
    if (n_launches) *n_launches = 3;
    if (n_pair_launches) *n_pair_launches = 1;
    return MCMP2_OK;
}

int mixed_check_flag(const MixedLayout &L, char *ws, cudaStream_t st, std::string &err)
{
    int h = 0;
    if (cudaMemcpyAsync(&h, ws + L.flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        err = "cannot read the time-out flag";
        return MCMP2_ECUDA;
    }
    if (h != 0) {
        err = "tensor-core kernel timed out waiting (role " + std::to_string(h) + ")";
        cudaMemsetAsync(ws + L.flag, 0, sizeof(int), st);
        return MCMP2_ETIMEOUT;
    }
    return MCMP2_OK;
}

void mixed_release(MixedPlan &plan) { plan.ready = false; }

}  // namespace mcmp2
