// Mixed-precision integrand engine on the tcgen05 tensor cores (sm_103a).
//
// Per step:
//  1. basis_split_kernel: basis values and gradients at the 2m positions (FP32)
//     as BF16 hi/lo planes (value = hi + lo to ~2^-17).
//  2. spinor_mixed_kernel: spinor formation (Eq. C with kinetic balance) as a
//     real split-BF16 x3 GEMM, phi = [g | grad g] x W (W = C folded with the
//     Pauli matrices), FP32 accumulate in tensor memory.  Its epilogue scales
//     the spinor values by s_k(tau) for every imaginary time and writes the
//     BF16 hi/lo planes (or TF32 values) of X(x)_ck = phi_k^c(x) s_k(tau),
//     rows 4x + c (2x + c for two-component systems), occupied and virtual
//     orbitals in separate planes, and the -im planes of the same rows (with
//     X's re planes they are the rows of iX = i X, (-im, re)).
//  3. pairs_mixed_kernel, on CTA pairs: for every (pair tile, tau) the
//     Hermitian products G(x, y)_cd = sum_k X(x)_ck conj(X(y)_dk) over the
//     occupied (G-) and virtual (G+) orbitals as M = N = 256 MMAs whose B
//     operand [Y; iY] yields [Re G | Im G] = [Xr Yr^T + Xi Yi^T | Xi Yr^T - Xr Yi^T]
//     in one accumulator, each real product as hi*hi + hi*lo + lo*hi (6 MMAs
//     per 16-deep K step; 4 in TF32), then the direct and exchange traces of
//     the trace form of Eq. MCMP2 for every pair of pairs, accumulated in FP64
//     as Re f / (w w w); with the Gaunt / Breit terms of Sec. II the epilogue
//     applies the operators to the G- rows (terms_part).
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

// FP32 rounded to the nearest TF32 value (ties away from zero), low 13 bits zero.
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

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
// Runs on CTA pairs (clusters of two CTAs on the two SMs of a TPC).  A work
// unit is (position block pair MT, component pair cp, 64-orbital block kb):
// CTA r owns the 128 positions of block 2 MT + r as its half of the A operand
// of an M = 256 MMA and holds the coefficient rows of component 2 cp + r (64
// orbitals, re and im) as its half of the N = 256 B operand, so each CTA's
// tensor memory collects [re | im] of both components for its own positions,
// and each operand tile read from L2 serves twice the work of a one-CTA
// 128 x 128 tile.
constexpr int SP_STAGES = 4;
constexpr int SP_STAGE_BYTES = 4 * TILE_BYTES;  // A hi, A lo, B hi, B lo (this CTA's halves)
constexpr int SP_EPI_WARPS = 8;                 // two per tensor-memory lane quarter, one per half of 64 orbitals
constexpr int SP_THREADS = 64 + 32 * SP_EPI_WARPS;  // TMA warp, MMA (even CTA) or relay (odd CTA) warp, epilogue warps
constexpr int SP_TMEM_COLS = 512;               // two 256-column accumulators: 2 components x [re | im]
constexpr int SP_MAX_TAU = 64;                  // scale staging capacity (the API limits n_tau to 64)
constexpr int SP_BOX_BYTES = 32 * 128;          // one TMA store box: 32 rows x one 128-byte chunk
constexpr int SP_NBOX_BYTES = 32 * 64;          // one -im box: 32 rows x one 64-byte chunk
constexpr int SP_WARP_STAGE = 2 * SP_BOX_BYTES;  // X and -im boxes of one epilogue warp (1 KB aligned)
static_assert(SP_BOX_BYTES + SP_NBOX_BYTES <= SP_WARP_STAGE, "a warp's X and -im boxes share its stage");
constexpr int SP_BARS_OFF = SP_STAGES * SP_STAGE_BYTES;
constexpr int SP_SCALE_OFF = SP_BARS_OFF + (2 * SP_STAGES + 4) * 8 + 16;
constexpr int SP_WSTAGE_OFF = (SP_SCALE_OFF + SP_MAX_TAU * 64 * 4 + 1023) / 1024 * 1024;  // swizzled boxes: 1 KB aligned
constexpr int SP_SMEM = SP_WSTAGE_OFF + SP_EPI_WARPS * SP_WARP_STAGE + 1024;
static_assert(SP_SMEM <= 232448, "spinor kernel exceeds the shared memory of one CTA");

struct SpinorMaps {
    CUtensorMap m[12];  // 0..3: A_L hi, A_L lo, B_L hi, B_L lo; 4..7: the same for the gradient part;
                        // 8, 9: X occupied / virtual (stores); 10, 11: -im occupied / virtual (stores)
};

// The operand rows X [n_tau][rows][k_pad / 16][128 B] (occupied and virtual) and
// their -im planes [n_tau][rows][k_pad / 16][64 B] are written through the store
// tensor maps of SpinorMaps.
struct SpinorArgs {
    const float *scale;   // [n_tau][n_orb]
    int *abort_flag;
    int P, nl, n_mt, n_kb, n_kb_occ, n_occ, n_vir, n_orb, n_tau;
    int tf32;  // chunk = 16 re (TF32) + 16 im (TF32) instead of re_hi, re_lo, im_hi, im_lo (BF16)
    int ncomp; // spinor components: 4, or 2 (two-component systems: large components only, rows 2x + c)
};

// Unit slot of cluster b on its j-th unit: rounds of G = number of clusters,
// every other round in reverse cluster order.  Slots list the units of the
// small components (K = 3 n_L) before those of the large ones (K = n_L), so
// the snake order gives every cluster a near-equal number of K chunks (39
// against an average of 36.9 at the medium size).
__device__ __forceinline__ int sp_slot(int j, int b, int G) { return j * G + ((j & 1) ? G - 1 - b : b); }

__device__ __forceinline__ void sp_unit(int slot, int n_MT, int n_kb, int ncomp, int &MT, int &cp, int &kb)
{
    const int n_heavy = ncomp == 4 ? n_MT * n_kb : 0;  // units of components 2, 3
    const bool heavy = slot < n_heavy;
    const int u = heavy ? slot : slot - n_heavy;
    MT = u / n_kb;
    kb = u - MT * n_kb;
    cp = heavy ? 1 : 0;
}

__global__ void __launch_bounds__(SP_THREADS, 1) spinor_mixed_kernel(const __grid_constant__ SpinorMaps maps,
                                                                     const SpinorArgs args)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + SP_BARS_OFF);
    uint64_t *empty = full + SP_STAGES;
    uint64_t *tfull = empty + SP_STAGES;  // [2] accumulator complete (both CTAs, multicast)
    uint64_t *tempty = tfull + 2;         // [2] accumulator read out (even CTA: both CTAs' epilogue warps)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int cid = (int)cluster_id(), ncl = (int)cluster_count();
    const int n_MT = (args.n_mt + 1) / 2;
    const int n_units = n_MT * (args.ncomp / 2) * args.n_kb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SP_STAGES; ++s) {
            mbar_init(&full[s], leader ? 2 : 1);  // even CTA: its own copies + the odd CTA's relay
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * SP_EPI_WARPS);
        }
        mbar_init_fence();
    }
    if (warp == 1) tmem_alloc_pair(tmem_slot, SP_TMEM_COLS);
    fence_before();
    __syncthreads();
    cluster_sync();  // barriers of both CTAs initialised before any remote arrive or multicast commit
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        if (lane == 0) {
            for (int i = 0; i < 8; ++i) tma_prefetch(&maps.m[i]);
            int stage = 0;
            uint32_t phase = 0;
            int issued[SP_STAGES] = {};
            uint32_t issued_phase[SP_STAGES] = {};
            bool ok = true;
            for (int jt = 0, slot; ok && (slot = sp_slot(jt, cid, ncl)) < n_units; ++jt) {
                int MT, cp, kb;
                sp_unit(slot, n_MT, args.n_kb, args.ncomp, MT, cp, kb);
                const CUtensorMap *mp = &maps.m[cp ? 4 : 0];
                const int K = cp ? 3 * args.nl : args.nl;
                const int a_row = (2 * MT + (int)rank) * 128;  // past the last block: zero fill, never stored
                const int wt_row = ((int)rank * args.n_kb + kb) * 128;  // component 2 cp + rank
                for (int c = 0; c < n_chunks(K); ++c) {
                    if (!mbar_wait_fast(&empty[stage], phase ^ 1u, args.abort_flag, 11, TIMEOUT_NS)) {
                        ok = false;
                        break;
                    }
                    unsigned char *st = smem + stage * SP_STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[stage], SP_STAGE_BYTES);
                    tma_load_2d(st + 0 * TILE_BYTES, mp + 0, &full[stage], c * BK, a_row);
                    tma_load_2d(st + 1 * TILE_BYTES, mp + 1, &full[stage], c * BK, a_row);
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
    } else if (warp == 1 && !leader) {
        // ---------------- relay (odd CTA): its copies landed -> the even CTA's stage barrier ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int jt = 0, slot; ok && (slot = sp_slot(jt, cid, ncl)) < n_units; ++jt) {
                int MT, cp, kb;
                sp_unit(slot, n_MT, args.n_kb, args.ncomp, MT, cp, kb);
                const int K = cp ? 3 * args.nl : args.nl;
                for (int c = 0; c < n_chunks(K); ++c) {
                    if (!mbar_wait(&full[stage], phase, args.abort_flag, 15, TIMEOUT_NS)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(mapa_shared(&full[stage], 0));
                    if (++stage == SP_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (even CTA) ----------------
        if (lane == 0) {
            int stage = 0, buf = 0;
            uint32_t phase = 0, tphase[2] = {0, 0};
            bool ok = true;
            const uint32_t id = idesc_pair(idesc_bf16(256, false));
            constexpr uint16_t BOTH = 3;
            // Stage-0 descriptors; a stage or K step adds its byte offset / 16 to the address field.
            const uint32_t base0 = smem_u32(smem);
            const uint64_t ah0 = sdesc_sw64(base0 + 0 * TILE_BYTES), al0 = sdesc_sw64(base0 + 1 * TILE_BYTES);
            const uint64_t bh0 = sdesc_sw64(base0 + 2 * TILE_BYTES), bl0 = sdesc_sw64(base0 + 3 * TILE_BYTES);
            for (int jt = 0, slot; ok && (slot = sp_slot(jt, cid, ncl)) < n_units; ++jt) {
                int MT, cp, kb;
                sp_unit(slot, n_MT, args.n_kb, args.ncomp, MT, cp, kb);
                const int K = cp ? 3 * args.nl : args.nl;
                if (!mbar_wait_fast(&tempty[buf], tphase[buf] ^ 1u, args.abort_flag, 12, TIMEOUT_NS)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + 256u * buf;
                for (int c = 0; c < n_chunks(K); ++c) {
                    if (!mbar_wait_fast(&full[stage], phase, args.abort_flag, 13, TIMEOUT_NS)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const int kvalid = K - c * BK;
                    const int ksteps = kvalid >= BK ? BK / 16 : (kvalid + 15) / 16;
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint64_t so = (uint64_t)((stage * SP_STAGE_BYTES + ks * 32) >> 4);
                        const uint64_t ah = ah0 + so, al = al0 + so, bh = bh0 + so, bl = bl0 + so;
                        umma_pair(d, ah, bh, id, (c == 0 && ks == 0) ? 0u : 1u);
                        umma_pair(d, ah, bl, id, 1u);
                        umma_pair(d, al, bh, id, 1u);
                    }
                    umma_pair_commit(&empty[stage], BOTH);
                    if (++stage == SP_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                umma_pair_commit(&tfull[buf], BOTH);
                tphase[buf] ^= 1u;
                buf ^= 1;
            }
            // Let every MMA this thread issued finish before tensor memory is freed.
            umma_pair_commit(&empty[stage], 1);
            mbar_drain(&empty[stage], phase, TIMEOUT_NS);
        }
    } else {
        // Epilogue: each lane owns one position row of its CTA's 128; the two warps of
        // a lane quarter take orbitals 0-31 and 32-63 (chunks 2 jh, 2 jh + 1) of the
        // 64-orbital block, for both components of the unit in turn.  A warp reads a
        // component's accumulator columns (re and im of its 32 orbitals for its 32
        // rows) from tensor memory, and releases the buffer once it holds the second
        // component's.  Then, for every time and chunk, it stages its 32 rows of the
        // chunk in shared memory in the contraction's operand order (re_hi, re_lo,
        // im_hi, im_lo, 32 B each; or re, im as TF32, 64 B each; 128-byte swizzle), and
        // the negated im half of the same rows (64 B per row, 64-byte swizzle), and
        // one lane writes the 4 KB and the 2 KB box with TMA stores.
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int jh = ew >> 2;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
        float *sscale = reinterpret_cast<float *>(smem + SP_SCALE_OFF);  // [n_tau][64]
        unsigned char *sx = smem + SP_WSTAGE_OFF + ew * SP_WARP_STAGE;   // X box: 32 rows x 128 B
        unsigned char *sn = sx + SP_BOX_BYTES;                          // -im box: 32 rows x 64 B
        const uint32_t neg = args.tf32 ? 0x80000000u : 0x80008000u;    // sign bits of the packed values
        const int sw = lane & 7;                                       // 128-byte swizzle of this lane's row
        const int sw64 = (lane >> 1) & 3;                              // 64-byte swizzle of this lane's row
        int buf = 0;
        uint32_t ephase[2] = {0, 0};
        for (int jt = 0, slot; (slot = sp_slot(jt, cid, ncl)) < n_units; ++jt) {
            int MT, cp, kb;
            sp_unit(slot, n_MT, args.n_kb, args.ncomp, MT, cp, kb);
            const int mt = 2 * MT + (int)rank;
            const bool got = mbar_wait(&tfull[buf], ephase[buf], args.abort_flag, 14, TIMEOUT_NS);
            if (bar_any<1, 32 * SP_EPI_WARPS>(!got)) break;  // also: every epilogue warp is done with the previous scales
            ephase[buf] ^= 1u;
            fence_after();
            const bool occ = kb < args.n_kb_occ;
            const int kl = occ ? kb : kb - args.n_kb_occ;
            const int k_first = (occ ? 0 : args.n_occ) + kl * 64;  // absolute index of the block's first orbital
            const int k_end = occ ? args.n_occ : args.n_orb;       // one past the region's last orbital
            const CUtensorMap *mx = &maps.m[occ ? 8 : 9];
            const CUtensorMap *mn = &maps.m[occ ? 10 : 11];
            for (int i = threadIdx.x - 64; i < 64 * args.n_tau; i += 32 * SP_EPI_WARPS) {
                const int t = i >> 6, k = k_first + (i & 63);
                sscale[i] = k < k_end ? args.scale[(size_t)t * args.n_orb + k] : 0.f;
            }
            bar_sync<1, 32 * SP_EPI_WARPS>();
#pragma unroll 1
            for (int cc = 0; cc < 2; ++cc) {
                const int c4 = 2 * cp + cc;
                const uint32_t col = 256u * buf + 128u * cc + 32u * jh;
                float re[2][16], im[2][16];
                tmem_ld<16>(lane_addr + col, re[0]);
                tmem_ld<16>(lane_addr + col + 16u, re[1]);
                tmem_ld<16>(lane_addr + col + 64u, im[0]);
                tmem_ld<16>(lane_addr + col + 80u, im[1]);
                tmem_wait_ld();
                if (cc == 1) {
                    // Both components are in registers: the MMAs may reuse the accumulator.
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_cluster(mapa_shared(&tempty[buf], 0));
                }
#pragma unroll 1
                for (int t = 0; t < args.n_tau; ++t) {
#pragma unroll
                    for (int jj = 0; jj < 2; ++jj) {
                        const int j = 2 * jh + jj;
                        // A chunk past the region's last orbital is never read by the contraction.
                        if (k_first + 16 * j >= k_end) continue;
                        const float *st_ = sscale + 64 * t + 16 * j;
                        uint4 d[8];
                        if (args.tf32) {
                            uint32_t rt[16], it[16];
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const float sc = st_[i];
                                rt[i] = to_tf32(re[jj][i] * sc);
                                it[i] = to_tf32(im[jj][i] * sc);
                            }
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                d[v] = make_uint4(rt[4 * v], rt[4 * v + 1], rt[4 * v + 2], rt[4 * v + 3]);
                                d[4 + v] = make_uint4(it[4 * v], it[4 * v + 1], it[4 * v + 2], it[4 * v + 3]);
                            }
                        } else {
                            uint32_t rh[8], rl[8], ih[8], il[8];
#pragma unroll
                            for (int i = 0; i < 16; i += 2) {
                                const float s0 = st_[i], s1 = st_[i + 1];
                                const float xr0 = re[jj][i] * s0, xr1 = re[jj][i + 1] * s1;
                                const float xi0 = im[jj][i] * s0, xi1 = im[jj][i + 1] * s1;
                                const __nv_bfloat162 hr = __floats2bfloat162_rn(xr0, xr1);
                                const __nv_bfloat162 hi = __floats2bfloat162_rn(xi0, xi1);
                                rh[i / 2] = *reinterpret_cast<const uint32_t *>(&hr);
                                ih[i / 2] = *reinterpret_cast<const uint32_t *>(&hi);
                                rl[i / 2] = pack_bf16(xr0 - __low2float(hr), xr1 - __high2float(hr));
                                il[i / 2] = pack_bf16(xi0 - __low2float(hi), xi1 - __high2float(hi));
                            }
                            d[0] = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                            d[1] = make_uint4(rh[4], rh[5], rh[6], rh[7]);
                            d[2] = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                            d[3] = make_uint4(rl[4], rl[5], rl[6], rl[7]);
                            d[4] = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                            d[5] = make_uint4(ih[4], ih[5], ih[6], ih[7]);
                            d[6] = make_uint4(il[0], il[1], il[2], il[3]);
                            d[7] = make_uint4(il[4], il[5], il[6], il[7]);
                        }
                        // The previous boxes must have been read out before they are overwritten.
                        if (lane == 0) bulk_wait_read_all();
                        __syncwarp();
#pragma unroll
                        for (int v = 0; v < 8; ++v) {
                            // 128-byte swizzle: 16-byte unit v of row `lane`; the im half (v >= 4)
                            // also negated into the -im box (64-byte swizzle)
                            *reinterpret_cast<uint4 *>(sx + lane * 128 + ((v ^ sw) << 4)) = d[v];
                            if (v >= 4) {
                                uint4 w = d[v];
                                w.x ^= neg;
                                w.y ^= neg;
                                w.z ^= neg;
                                w.w ^= neg;
                                *reinterpret_cast<uint4 *>(sn + lane * 64 + (((v - 4) ^ sw64) << 4)) = w;
                            }
                        }
                        fence_proxy_async_smem();
                        __syncwarp();
                        const int x0 = kl * 256 + 64 * j, y0 = mt * 128 + 32 * quarter;
                        if (lane == 0 && y0 < args.P) {
                            // Boxes {64 (X) or 32 (-im) elements, 1 component, 32 positions, 1 time};
                            // positions past P are clipped.
                            tma_store_4d(mx, sx, x0, c4, y0, t);
                            tma_store_4d(mn, sn, x0 / 2, c4, y0, t);
                            bulk_commit();
                        }
                    }
                }
            }
            buf ^= 1;
        }
        if (lane == 0) bulk_wait_all();  // every store of this warp has reached global memory
        __syncwarp();
    }
    fence_before();
    __syncthreads();
    cluster_sync();  // no MMA, copy, store or remote arrive of either CTA is outstanding past this point
    if (warp == 1) {
        fence_after();
        tmem_dealloc_pair(tmem, SP_TMEM_COLS);
    }
}

// ===========================================================================
// 3. Pair-of-pairs contraction with the trace epilogue
// ===========================================================================
// Operand rows: one row per (position x, component c), row NC x + c (NC = 4
// components, or 2 for two-component systems), holding for each 16-orbital
// chunk the four split planes re_hi, re_lo, im_hi, im_lo side by side
// (128 B), so one 128-byte-swizzled TMA box of 128 rows brings all four
// planes of a chunk and the MMA selects a plane by a 32-byte offset.  In the
// TF32 form the 128 B are re and im of the chunk as TF32 (64 B each); the
// same offsets then select (re, K 0-7), (re, K 8-15), (im, K 0-7), (im, K 8-15).
// The negated im planes of the same rows (64 B per chunk) are written beside
// them: with X's re planes they are the rows of iX = i X = (-im, re).
//
// The kernel runs on CTA pairs (clusters of two CTAs on the two SMs of a
// TPC).  Work item = (pair tile, time); a pair tile is two p-blocks x one
// q-block of TP walker pairs (TP = 16, or 32 for two-component systems, so
// that a block is 128 operand rows): CTA r owns p-block bp = 2 BP + r, whose
// 128 rows are its half of the A operand of an M = 256 MMA, and holds the
// q-block's 128 rows as its half of the B operand, CTA 0 from X and CTA 1 from
// iX.  The B half arrives as two 64-byte-swizzled tiles of 128 rows x 64 B: in
// CTA 0 the re and the im half of X's chunk, in CTA 1 the -im planes and X's re
// half, so both CTAs' real-plane B sits in the first tile and the imaginary-plane
// B in the second.  One thread of the even CTA issues cta_group::2 MMAs with M = N = 256:
// with A = X_re planes and B = [Y; iY]_re planes, then A = X_im and B =
// [Y; iY]_im, one accumulator of 256 columns collects
//   [Xr Yr^T + Xi Yi^T | Xi Yr^T - Xr Yi^T] = [Re G | Im G],
// each real product as hi*hi + hi*lo + lo*hi (6 MMAs per 16-orbital chunk;
// 4 TF32 MMAs).  Each CTA's tensor memory thus holds the 128 x 128 complex
// blocks of its own TP x TP tile (rows NC(2p + e) + c, columns NC(2q + e') + d),
// Re in the group's first 128 columns and Im in the next 128.
//
// Per item the tensor cores accumulate G- (K = n_occ) and then G+
// (K = n_vir) in one 256-column half of tensor memory.  Two epilogue groups
// per CTA take alternate items, each with its own half: while one group
// traces item i, the MMAs fill the other half with item i+1.  G- is
// accumulated first in the same columns; its group copies the like-electron
// blocks G-(ep, eq) (the only G- blocks the trace form needs) to shared
// memory as 24-bit floats (FP32 rounded to 15 stored significand bits,
// relative error at most 2^-16, about the error the split BF16 products
// already carry), which frees the columns for G+.
//
// Barriers: each CTA's copies complete on its own stage barrier; a relay
// thread of the odd CTA forwards that completion to the even CTA's stage
// barrier, on which the MMA issuer waits (so each CTA can always drain its
// own copies).  MMA completion is multicast to both CTAs (stage free, G-
// ready, G+ ready); both CTAs' epilogue warps arrive on the even CTA's
// barriers when they have unloaded G- or released the columns.
constexpr int PR_BK = 16;                           // orbitals per chunk (one stage)
constexpr int PR_TILE_BYTES = 128 * 4 * PR_BK * 2;  // 128 rows x (4 planes x 16 BF16) = 16 KB
constexpr int PR_STAGES = 4;
constexpr int PR_BTILE_BYTES = 128 * 2 * PR_BK * 2; // 128 rows x (2 planes x 16 BF16) = 8 KB, 64-byte swizzle
constexpr int PR_STAGE_BYTES = PR_TILE_BYTES + 2 * PR_BTILE_BYTES;  // A chunk, then this CTA's two B tiles
constexpr int PR_GROUPS = 2;
constexpr int PR_GROUP_WARPS = 8;                   // two per tensor-memory lane quarter
constexpr int PR_EPI_WARPS = PR_GROUPS * PR_GROUP_WARPS;
constexpr int PR_QHALVES = PR_GROUP_WARPS / 4;      // warps of a group per tensor-memory lane quarter
constexpr int PR_QW4 = 16 / PR_QHALVES;             // q-pairs per warp and item, four-component tiles
constexpr int PR_QW2 = 32 / PR_QHALVES;             // q-pairs per warp and item, two-component tiles
static_assert(PR_GROUP_WARPS % 4 == 0 && 16 % PR_QHALVES == 0, "a group covers the four lane quarters");
constexpr int PR_THREADS = 64 + 32 * PR_EPI_WARPS;
constexpr int PR_TMEM_COLS = 512;                   // per group: re | im of 128 columns
constexpr int PR_GM_BYTES = 16 * 3 * 128 * 8;       // G- like blocks of one item: 48 KB
constexpr int PR_GM_OFF = PR_STAGES * PR_STAGE_BYTES;
constexpr int PR_BARS_OFF = PR_GM_OFF + PR_GROUPS * PR_GM_BYTES;
constexpr int PR_RED_OFF = PR_BARS_OFF + 192;       // barriers + tensor-memory slot
constexpr int PR_SMEM = PR_RED_OFF + PR_GROUPS * 64 * 8 + 1024;
static_assert(PR_SMEM <= 232448, "contraction kernel exceeds the shared memory of one CTA");
static_assert(PR_STAGE_BYTES % 1024 == 0, "stages must keep the 1024-byte swizzle alignment");
static_assert((2 * PR_STAGES + 4 * PR_GROUPS) * 8 + 4 <= 192, "barrier block too small");

struct PairMaps {
    // 3-D (chunk x plane x orbital, row, tau).  occ, vir: X, 128-byte swizzle, 64 x
    // 128-row boxes (the A operand); hocc, hvir: X, 64-byte swizzle, 32 x 128-row
    // boxes (one half of a chunk); nocc, nvir: the -im planes, 64-byte swizzle, 32 x
    // 128-row boxes.
    CUtensorMap occ, vir, hocc, hvir, nocc, nvir;
};

struct PairArgs {
    const double *a;   // [m] pair weight factors N_g / (g1 g2)
    double *partials;  // [n_tau][n_tiles], one per TP x TP tile (bp <= bq)
    int *abort_flag;
    int m, n_tiles, n_ptiles, nb, n_tau, n_occ, n_vir;
    double inv_lambda;
    unsigned long long timeout_ns;  // limit of every wait
    int withhold_first_copy;        // test hook: never issue the first stage's copy (its wait runs out)
    const double *r = nullptr;      // walker positions [m][2][3] (the Breit terms' unit vectors)
    DebugTile dbg{};                // optional per-element record of one TP x TP tile
};

// Pair tile k -> (BP, bq): row BP of the enumeration holds bq = 2 BP .. nb - 1.
__device__ __forceinline__ void pair_tile(int k, int nb, int &BP, int &bq)
{
    int b = 0;
    while (k >= nb - 2 * b) {
        k -= nb - 2 * b;
        ++b;
    }
    BP = b;
    bq = 2 * b + k;
}

// Index of the TP x TP tile (bp <= bq) in the row-by-row enumeration of the upper triangle.
__device__ __forceinline__ int tile_index(int bp, int bq, int nb) { return bp * nb - bp * (bp - 1) / 2 + (bq - bp); }

__device__ __forceinline__ int pr_chunks(int k) { return (k + PR_BK - 1) / PR_BK; }

// Four floats rounded to 24 bits (sign, exponent, 15 stored significand
// bits; round half away from zero on the magnitude) packed into three words.
__device__ __forceinline__ uint32_t r24(float x) { return (__float_as_uint(x) + 0x80u) >> 8; }
__device__ __forceinline__ uint3 pack24(float a, float b, float c, float d)
{
    const uint32_t A = r24(a), B = r24(b), C = r24(c), D = r24(d);
    return make_uint3(A | (B << 24), (B >> 8) | (C << 16), (C >> 16) | (D << 8));
}
__device__ __forceinline__ void unpack24(uint32_t w0, uint32_t w1, uint32_t w2, float &a, float &b, float &c, float &d)
{
    a = __uint_as_float(w0 << 8);
    b = __uint_as_float(__byte_perm(w0, w1, 0x5433) & 0xFFFFFF00u);
    c = __uint_as_float(__byte_perm(w1, w2, 0x4322) & 0xFFFFFF00u);
    d = __uint_as_float(w2 & 0xFFFFFF00u);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle (8 rows x 128 B
// atoms, 1024 B between 8-row groups), SM100 descriptor version 1.  The
// start address may sit 32, 64 or 96 B into a 1024-byte-aligned tile: the
// swizzle is applied to the absolute address, which selects a 16-element
// slice of every row.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;  // SWIZZLE_128B
    return d;
}

// OR of a predicate over the 256 threads of epilogue group g (named barriers 1 and 2).
__device__ __forceinline__ bool group_any(int g, bool v)
{
    return g == 0 ? bar_any<1, 32 * PR_GROUP_WARPS>(v) : bar_any<2, 32 * PR_GROUP_WARPS>(v);
}

__device__ __forceinline__ void group_sync(int g)
{
    if (g == 0)
        bar_sync<1, 32 * PR_GROUP_WARPS>();
    else
        bar_sync<2, 32 * PR_GROUP_WARPS>();
}


// Where an epilogue group stands: its CTA's rank in the pair, the cluster's item
// sequence, and the even CTA's hand-off barriers (shared::cluster addresses).
struct EpiCtx {
    int rank, cid, ncl, n_items;
    uint32_t munl_even, pfree_even;
};

// ---------------------------------------------------------------------------
// Gaunt and Breit terms (Sec. II: g_ab = (1/r_ab) sum_A c_A O_A(a) O_A(b) with
// O in {1, alpha_x, alpha_y, alpha_z, alpha.n_ab}, c = 1, -1/2, -1/2, -1/2, -1/2).
// With O_A at the points of pair p and O_B at those of pair q, both traces of
// the trace form keep their Coulomb shape once G- is replaced by
// M_AB = O_A G- O_B (the operators are Hermitian):
//   direct   T_AB(x, y) = sum_cd conj(M_AB(x, y)_cd) G+(x, y)_cd, D = sum c_A c_B T_AB(1p,1q) T_AB(2p,2q),
//   exchange tr[M_AB(1p,1q)^dag G+(1p,2q) M_AB(2p,2q)^dag G+(2p,1q)].
// alpha_k has sigma_k in its off-diagonal 2x2 blocks (components L-alpha,
// L-beta, S-alpha, S-beta), so O_A = alpha_k maps row c of G- to row c^3
// (x, y) or c^2 (z) times a phase rho_k(c), and O_B permutes the columns the
// same way; alpha.n is the combination sum_k n_k alpha_k.
// ---------------------------------------------------------------------------

// Row r (of 128) of the parked G- block of q-pair ql: four complex entries.
__device__ __forceinline__ void gm_row(const unsigned char *gm, int ql, int r, float *re, float *im)
{
    const uint2 *gp = reinterpret_cast<const uint2 *>(gm);
    const uint2 w0 = gp[(3 * ql + 0) * 128 + r];
    const uint2 w1 = gp[(3 * ql + 1) * 128 + r];
    const uint2 w2 = gp[(3 * ql + 2) * 128 + r];
    unpack24(w0.x, w0.y, w1.x, re[0], im[0], re[1], im[1]);
    unpack24(w1.y, w2.x, w2.y, re[2], im[2], re[3], im[3]);
}

// h_B = sum_d conj((R O_B)_d) Y_d for O_B = 1, alpha_x, alpha_y, alpha_z, where
// (R alpha_x)_d = R_{d^3}, (R alpha_y)_d = kappa_d R_{d^3} (kappa = i for even d,
// -i for odd d) and (R alpha_z)_d = +-R_{d^2} (+ for even d).  The even- and
// odd-d halves of the two permuted dot products give all four.
__device__ __forceinline__ void row_dots(const float *Rr, const float *Ri, const float *Yr, const float *Yi, float *hr,
                                         float *hi)
{
    float fr = 0.f, fi = 0.f;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        fr += Rr[d] * Yr[d] + Ri[d] * Yi[d];
        fi += Rr[d] * Yi[d] - Ri[d] * Yr[d];
    }
    const float exr = Rr[3] * Yr[0] + Ri[3] * Yi[0] + Rr[1] * Yr[2] + Ri[1] * Yi[2];
    const float exi = Rr[3] * Yi[0] - Ri[3] * Yr[0] + Rr[1] * Yi[2] - Ri[1] * Yr[2];
    const float oxr = Rr[2] * Yr[1] + Ri[2] * Yi[1] + Rr[0] * Yr[3] + Ri[0] * Yi[3];
    const float oxi = Rr[2] * Yi[1] - Ri[2] * Yr[1] + Rr[0] * Yi[3] - Ri[0] * Yr[3];
    const float ezr = Rr[2] * Yr[0] + Ri[2] * Yi[0] + Rr[0] * Yr[2] + Ri[0] * Yi[2];
    const float ezi = Rr[2] * Yi[0] - Ri[2] * Yr[0] + Rr[0] * Yi[2] - Ri[0] * Yr[2];
    const float ozr = Rr[3] * Yr[1] + Ri[3] * Yi[1] + Rr[1] * Yr[3] + Ri[1] * Yi[3];
    const float ozi = Rr[3] * Yi[1] - Ri[3] * Yr[1] + Rr[1] * Yi[3] - Ri[1] * Yr[3];
    hr[0] = fr;
    hi[0] = fi;
    hr[1] = exr + oxr;
    hi[1] = exi + oxi;
    hr[2] = exi - oxi;  // i (ox - ex)
    hi[2] = oxr - exr;
    hr[3] = ezr - ozr;
    hi[3] = ezi - ozi;
}

// sum_B c_B Re(G_B H_B) over B = 0, x, y, z (and n = alpha.n_q with BREIT).
template <bool BREIT>
__device__ __forceinline__ float re_prod_sum(const float *Gr, const float *Gi, const float *Hr, const float *Hi,
                                             float nqx, float nqy, float nqz)
{
    float s = Gr[0] * Hr[0] - Gi[0] * Hi[0];
    float t = 0.f;
#pragma unroll
    for (int B = 1; B < 4; ++B) t += Gr[B] * Hr[B] - Gi[B] * Hi[B];
    if constexpr (BREIT) {
        const float gr = nqx * Gr[1] + nqy * Gr[2] + nqz * Gr[3], gi = nqx * Gi[1] + nqy * Gi[2] + nqz * Gi[3];
        const float hr = nqx * Hr[1] + nqy * Hr[2] + nqz * Hr[3], hi = nqx * Hi[1] + nqy * Hi[2] + nqz * Hi[3];
        t += gr * hr - gi * hi;
    }
    return s - 0.5f * t;
}

// This lane's share of direct - exchange for one pair of pairs with the Gaunt
// (BREIT = false) or Breit terms.  Lane (e, c) holds row c of G+(xe, ye) (dia) and
// G+(xe, y(1-e)) (off); the G- rows come from shared memory (own0: rows of its
// electron's block, par0: the other electron's).  The eight lanes' shares sum
// to D - X.
template <bool BREIT>
__device__ __forceinline__ float terms_part(const unsigned char *gm, int ql, int own0, int par0, int e, int c,
                                            int lane, const float *dia_r, const float *dia_i, const float *off_r,
                                            const float *off_i, float npx, float npy, float npz, float nqx,
                                            float nqy, float nqz)
{
    const float sc = (c & 1) ? -1.f : 1.f;  // rho_y(c) = -i sc, rho_z(c) = sc
    float Rr[4], Ri[4];
    // (a) exchange: as in the Coulomb trace, lane (e, c) pairs its rows with the
    //     other electron's rows c'' (two per lane), now for every (A, B).
    float xl = 0.f;
    const int gbase = lane & ~7;
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        const int cpp = e == 0 ? ((c + s) & 3) : ((c + 2 - s) & 3);
        const int src = gbase + 4 * (1 - e) + cpp;
        const float sp = (cpp & 1) ? -1.f : 1.f;
        float ror[4], roi[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            ror[d] = __shfl_sync(0xffffffffu, off_r[d], src);
            roi[d] = __shfl_sync(0xffffffffu, off_i[d], src);
        }
        float Hr[4], Hi[4], Gr[4], Gi[4];
        // A = 0
        gm_row(gm, ql, own0 + c, Rr, Ri);
        row_dots(Rr, Ri, ror, roi, Hr, Hi);
        gm_row(gm, ql, par0 + cpp, Rr, Ri);
        row_dots(Rr, Ri, off_r, off_i, Gr, Gi);
        xl += re_prod_sum<BREIT>(Gr, Gi, Hr, Hi, nqx, nqy, nqz);
        // A = x, y share rows c^3 and c''^3: products 1 and -sc sp
        float H3r[4], H3i[4], G3r[4], G3i[4];
        gm_row(gm, ql, own0 + (c ^ 3), Rr, Ri);
        row_dots(Rr, Ri, ror, roi, H3r, H3i);
        gm_row(gm, ql, par0 + (cpp ^ 3), Rr, Ri);
        row_dots(Rr, Ri, off_r, off_i, G3r, G3i);
        xl -= 0.5f * (1.f - sc * sp) * re_prod_sum<BREIT>(G3r, G3i, H3r, H3i, nqx, nqy, nqz);
        // A = z: rows c^2 and c''^2, product sc sp
        gm_row(gm, ql, own0 + (c ^ 2), Rr, Ri);
        row_dots(Rr, Ri, ror, roi, Hr, Hi);
        gm_row(gm, ql, par0 + (cpp ^ 2), Rr, Ri);
        row_dots(Rr, Ri, off_r, off_i, Gr, Gi);
        xl -= 0.5f * sc * sp * re_prod_sum<BREIT>(Gr, Gi, Hr, Hi, nqx, nqy, nqz);
        if constexpr (BREIT) {
            // A = alpha.n_p: (nx + i ny sgn) row^3 + nz sgn row^2 on each side, B = 0, x, y, z, n.
            float s0 = 0.f, t = 0.f, anr = 0.f, ani = 0.f, bnr = 0.f, bni = 0.f;
#pragma unroll
            for (int B = 0; B < 4; ++B) {
                const float ar = npx * G3r[B] - npy * sp * G3i[B] + npz * sp * Gr[B];
                const float ai = npx * G3i[B] + npy * sp * G3r[B] + npz * sp * Gi[B];
                const float br = npx * H3r[B] - npy * sc * H3i[B] + npz * sc * Hr[B];
                const float bi = npx * H3i[B] + npy * sc * H3r[B] + npz * sc * Hi[B];
                if (B == 0) {
                    s0 = ar * br - ai * bi;
                } else {
                    const float wq = B == 1 ? nqx : (B == 2 ? nqy : nqz);
                    t += ar * br - ai * bi;
                    anr += wq * ar;
                    ani += wq * ai;
                    bnr += wq * br;
                    bni += wq * bi;
                }
            }
            t += anr * bnr - ani * bni;
            xl -= 0.5f * (s0 - 0.5f * t);
        }
    }
    // (b) direct: lane partials t_AB, slot k = 4A + B (re, im); with BREIT also
    //     t_nB (B = 0, x, y, z, n) for O_A = alpha.n_p.
    float v[32];
    float tn[10];
    {
        float H0r[4], H0i[4], H3r[4], H3i[4], H2r[4], H2i[4];
        gm_row(gm, ql, own0 + c, Rr, Ri);
        row_dots(Rr, Ri, dia_r, dia_i, H0r, H0i);
        gm_row(gm, ql, own0 + (c ^ 3), Rr, Ri);
        row_dots(Rr, Ri, dia_r, dia_i, H3r, H3i);
        gm_row(gm, ql, own0 + (c ^ 2), Rr, Ri);
        row_dots(Rr, Ri, dia_r, dia_i, H2r, H2i);
#pragma unroll
        for (int B = 0; B < 4; ++B) {
            v[2 * B] = H0r[B];
            v[2 * B + 1] = H0i[B];
            v[2 * (4 + B)] = H3r[B];
            v[2 * (4 + B) + 1] = H3i[B];
            v[2 * (8 + B)] = -sc * H3i[B];  // conj(rho_y(c)) = i sc
            v[2 * (8 + B) + 1] = sc * H3r[B];
            v[2 * (12 + B)] = sc * H2r[B];
            v[2 * (12 + B) + 1] = sc * H2i[B];
        }
    }
    if constexpr (BREIT) {
        // t_nB = sum_k n_p,k t_kB (the operator enters linearly), then B = alpha.n_q likewise.
#pragma unroll
        for (int j = 0; j < 8; ++j) tn[j] = npx * v[8 + j] + npy * v[16 + j] + npz * v[24 + j];
        tn[8] = nqx * tn[2] + nqy * tn[4] + nqz * tn[6];
        tn[9] = nqx * tn[3] + nqy * tn[5] + nqz * tn[7];
    }
    // Sum over the four lanes c of the electron by halving exchanges: after them
    // lane c holds T_AB for A = 2 (c & 1) + (c >> 1) and B = 0..3.
    const bool h1 = lane & 1, h2 = lane & 2;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float send = h1 ? v[j] : v[j + 16];
        const float keep = h1 ? v[j + 16] : v[j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float send = h2 ? v[j] : v[j + 8];
        const float keep = h2 ? v[j + 8] : v[j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    float w[8];  // the same T_AB of the other electron
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = __shfl_xor_sync(0xffffffffu, v[j], 4);
    const float cA = ((lane & 3) == 0) ? 1.f : -0.5f;  // A = 0 on lane c = 0 only
    float dl;
    {
        float vr[4], vi[4], wr[4], wi[4];
#pragma unroll
        for (int B = 0; B < 4; ++B) {
            vr[B] = v[2 * B];
            vi[B] = v[2 * B + 1];
            wr[B] = w[2 * B];
            wi[B] = w[2 * B + 1];
        }
        dl = cA * re_prod_sum<BREIT>(vr, vi, wr, wi, nqx, nqy, nqz);
    }
    if constexpr (BREIT) {
        // The alpha.n_p row, summed over all four lanes (each then holds it: count a quarter).
#pragma unroll
        for (int j = 0; j < 10; ++j) tn[j] += __shfl_xor_sync(0xffffffffu, tn[j], 1);
#pragma unroll
        for (int j = 0; j < 10; ++j) tn[j] += __shfl_xor_sync(0xffffffffu, tn[j], 2);
        float nr = 0.f;
#pragma unroll
        for (int B = 0; B < 5; ++B) {
            const float ur = __shfl_xor_sync(0xffffffffu, tn[2 * B], 4);
            const float ui = __shfl_xor_sync(0xffffffffu, tn[2 * B + 1], 4);
            nr += (B == 0 ? 1.f : -0.5f) * (tn[2 * B] * ur - tn[2 * B + 1] * ui);
        }
        dl -= 0.125f * nr;  // c_n = -1/2, a quarter
    }
    dl *= 0.5f;  // both electrons' lanes hold each product
    return dl - xl;
}

__device__ __forceinline__ void unit_pair_vector(const double *r, int p, float &x, float &y, float &z)
{
    const double dx = r[6 * p] - r[6 * p + 3], dy = r[6 * p + 1] - r[6 * p + 4], dz = r[6 * p + 2] - r[6 * p + 5];
    const double inv = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
    x = (float)(dx * inv);
    y = (float)(dy * inv);
    z = (float)(dz * inv);
}

// Trace epilogue of a four-component tile: rows 8p + 4e + c of 16 p-pairs,
// columns 8q + 4e' + d of 16 q-pairs; the eight lanes (e, c) of a pair hold its rows.
// INTER: MCMP2_COULOMB, MCMP2_GAUNT or MCMP2_BREIT.
template <int INTER>
__device__ __forceinline__ void pairs_epilogue_4c(const PairArgs &args, unsigned char *smem, uint32_t tmem,
                                                  int warp, int lane, const EpiCtx &ec, uint64_t *mfull,
                                                  uint64_t *pfull)
{
    const int ew = warp - 2;
    const int g = ew / PR_GROUP_WARPS;
    const int gw = ew - g * PR_GROUP_WARPS;
    const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
    const int qhalf = gw >> 2;     // q-pairs PR_QW4*qhalf .. +PR_QW4-1 of the tile
    const int row = 32 * quarter + lane;
    const int p_local = row >> 3, e = (row >> 2) & 1, c = lane & 3;
    const int gbase = lane & ~7;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16) + 256u * g;
    unsigned char *gm = smem + PR_GM_OFF + g * PR_GM_BYTES;
    double *red = reinterpret_cast<double *>(smem + PR_RED_OFF) + 64 * g;
    uint32_t ph = 0;
    for (int item = ec.cid + g * ec.ncl; item < ec.n_items; item += PR_GROUPS * ec.ncl) {
        const int t = item / args.n_ptiles, pt = item - t * args.n_ptiles;
        int BP, bq;
        pair_tile(pt, args.nb, BP, bq);
        const int bp = 2 * BP + ec.rank;
        // (1) G- like-electron blocks of this lane's row -> shared memory: for q, the
        //     four entries G-(row, 8q + 4e + d) in the order re 0, im 0, re 1, im 1 |
        //     re 2, im 2, re 3, im 3, packed to 24 bits as three uint2.
        const bool got_m = mbar_wait(&mfull[g], ph, args.abort_flag, 4, args.timeout_ns);
        if (group_any(g, !got_m)) break;  // the group leaves together
        fence_after();
#pragma unroll 1
        for (int qb = 0; qb < PR_QW4 / 2; ++qb) {
            const int q0 = PR_QW4 * qhalf + 2 * qb;
            float vr[16], vi[16];
            tmem_ld<16>(lane_addr + 8u * q0, vr);
            tmem_ld<16>(lane_addr + 128u + 8u * q0, vi);
            tmem_wait_ld();
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
                float o_r[4], o_i[4];
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    o_r[d] = e ? vr[8 * qq + 4 + d] : vr[8 * qq + d];
                    o_i[d] = e ? vi[8 * qq + 4 + d] : vi[8 * qq + d];
                }
                const int q = q0 + qq;
                uint2 *gp = reinterpret_cast<uint2 *>(gm);
                const uint3 u = pack24(o_r[0], o_i[0], o_r[1], o_i[1]);
                const uint3 v = pack24(o_r[2], o_i[2], o_r[3], o_i[3]);
                gp[(3 * q + 0) * 128 + row] = make_uint2(u.x, u.y);
                gp[(3 * q + 1) * 128 + row] = make_uint2(u.z, v.x);
                gp[(3 * q + 2) * 128 + row] = make_uint2(v.y, v.z);
            }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(ec.munl_even);
        // (2) traces once G+ is in the same columns.
        const bool got_p = mbar_wait(&pfull[g], ph, args.abort_flag, 6, args.timeout_ns);
        if (group_any(g, !got_p)) break;
        ph ^= 1u;
        fence_after();
        const int p = bp * 16 + p_local;
        // a_q of the tile's 16 q-pairs, one per lane (lane & 15), fetched by shuffle below.
        const int q_lane = bq * 16 + (lane & 15);
        const double a_lane = q_lane < args.m ? args.a[q_lane] : 0.0;
        // Breit: unit vectors n = (r1 - r2) / r12 of this lane's p-pair and of q-pair q_lane.
        float npx = 0.f, npy = 0.f, npz = 0.f, nlx = 0.f, nly = 0.f, nlz = 0.f;
        if constexpr (INTER == MCMP2_BREIT) {
            if (p < args.m) unit_pair_vector(args.r, p, npx, npy, npz);
            if (q_lane < args.m) unit_pair_vector(args.r, q_lane, nlx, nly, nlz);
        }
        double acc = 0.0;  // sum over this warp's q of Re f_pq a_q
        if constexpr (INTER != MCMP2_COULOMB) {
            // One q-pair per tensor-memory load: the operator terms hold more state per q.
#pragma unroll 1
            for (int qi = 0; qi < PR_QW4; ++qi) {
                const int ql = PR_QW4 * qhalf + qi;
                float gpr[8], gpi[8];
                tmem_ld<8>(lane_addr + 8u * ql, gpr);
                tmem_ld<8>(lane_addr + 128u + 8u * ql, gpi);
                tmem_wait_ld();
                float dia_r[4], dia_i[4], off_r[4], off_i[4];
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    dia_r[d] = e ? gpr[4 + d] : gpr[d];
                    dia_i[d] = e ? gpi[4 + d] : gpi[d];
                    off_r[d] = e ? gpr[d] : gpr[4 + d];
                    off_i[d] = e ? gpi[d] : gpi[4 + d];
                }
                const int q = bq * 16 + ql;
                const double a_q = __shfl_sync(0xffffffffu, a_lane, ql);
                const float nqx = __shfl_sync(0xffffffffu, nlx, ql);
                const float nqy = __shfl_sync(0xffffffffu, nly, ql);
                const float nqz = __shfl_sync(0xffffffffu, nlz, ql);
                float part = terms_part<INTER == MCMP2_BREIT>(gm, ql, row & ~3, (row ^ 4) & ~3, e, c, lane, dia_r,
                                                              dia_i, off_r, off_i, npx, npy, npz, nqx, nqy, nqz);
                part += __shfl_xor_sync(0xffffffffu, part, 1);
                part += __shfl_xor_sync(0xffffffffu, part, 2);
                part += __shfl_xor_sync(0xffffffffu, part, 4);
                const bool valid = p < args.m && q < args.m && (bp < bq || (bp == bq && p_local < ql));
                if (valid) acc += (double)(-0.5f * part) * a_q;
                if (args.dbg.out && bp == args.dbg.bp && bq == args.dbg.bq && (lane & 7) == 0)
                    args.dbg.out[((size_t)t * 16 + p_local) * 16 + ql] =
                        valid ? (double)(-0.5f * part) * a_q * args.a[p] * args.inv_lambda : 0.0;
            }
        }
#pragma unroll 1
        for (int qb = 0; qb < (INTER == MCMP2_COULOMB ? PR_QW4 / 2 : 0); ++qb) {
            const int q0 = PR_QW4 * qhalf + 2 * qb;  // two q-pairs per tensor-memory load
            float gpr[16], gpi[16];
            tmem_ld<16>(lane_addr + 8u * q0, gpr);
            tmem_ld<16>(lane_addr + 128u + 8u * q0, gpi);
            tmem_wait_ld();
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
                // This lane holds row c of G-(xe, ye) [own], G+(xe, ye) [dia], G+(xe, y(1-e)) [off].
                const int ql = q0 + qq;
                float dia_r[4], dia_i[4], off_r[4], off_i[4];
#pragma unroll
                for (int d = 0; d < 4; ++d) {  // constant indices keep the arrays in registers
                    const int i0 = 8 * qq + d, i1 = 8 * qq + 4 + d;
                    dia_r[d] = e ? gpr[i1] : gpr[i0];
                    dia_i[d] = e ? gpi[i1] : gpi[i0];
                    off_r[d] = e ? gpr[i0] : gpr[i1];
                    off_i[d] = e ? gpi[i0] : gpi[i1];
                }
                float own_r[4], own_i[4];
                {
                    const uint2 *gp = reinterpret_cast<const uint2 *>(gm);
                    const uint2 w0 = gp[(3 * ql + 0) * 128 + row];
                    const uint2 w1 = gp[(3 * ql + 1) * 128 + row];
                    const uint2 w2 = gp[(3 * ql + 2) * 128 + row];
                    unpack24(w0.x, w0.y, w1.x, own_r[0], own_i[0], own_r[1], own_i[1]);
                    unpack24(w1.y, w2.x, w2.y, own_r[2], own_i[2], own_r[3], own_i[3]);
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
                const int q = bq * 16 + ql;
                const double a_q = __shfl_sync(0xffffffffu, a_lane, ql);
                const bool valid = p < args.m && q < args.m && (bp < bq || (bp == bq && p_local < ql));
                if (valid) acc += (double)(-0.5f * (direct_re - xr)) * a_q;
                if (args.dbg.out && bp == args.dbg.bp && bq == args.dbg.bq && (lane & 7) == 0)
                    args.dbg.out[((size_t)t * 16 + p_local) * 16 + ql] =
                        valid ? (double)(-0.5f * (direct_re - xr)) * a_q * args.a[p] * args.inv_lambda : 0.0;
            }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(ec.pfree_even);
        if ((lane & 7) == 0) red[16 * qhalf + 4 * quarter + (lane >> 3)] = (p < args.m) ? acc * args.a[p] : 0.0;
        group_sync(g);
        if (gw == 0 && lane == 0 && bp <= bq) {
            double sum = 0.0;
            for (int j = 0; j < 16 * PR_QHALVES; ++j) sum += red[j];
            args.partials[(size_t)t * args.n_tiles + tile_index(bp, bq, args.nb)] = sum * args.inv_lambda;
        }
        group_sync(g);
    }
}

// Trace epilogue of a two-component tile (NC = 2): rows 4p + 2e + c of 32
// p-pairs, columns 4q + 2e' + d of 32 q-pairs, so the four lanes (e, c) of a
// pair hold its rows.  Same hand-offs as the four-component epilogue: unload
// the like-electron blocks G-(ep, eq) (2 x 2) to shared memory as 24-bit
// floats, then trace against G+ once it is in the same columns.
__device__ __forceinline__ void pairs_epilogue_2c(const PairArgs &args, unsigned char *smem, uint32_t tmem,
                                                  int warp, int lane, const EpiCtx &ec, uint64_t *mfull,
                                                  uint64_t *pfull)
{
    const int ew = warp - 2;
    const int g = ew / PR_GROUP_WARPS;
    const int gw = ew - g * PR_GROUP_WARPS;
    const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
    const int qhalf = gw >> 2;     // q-pairs PR_QW2*qhalf .. +PR_QW2-1 of the tile
    const int row = 32 * quarter + lane;
    const int p_local = row >> 2, e = (row >> 1) & 1, c = lane & 1;
    const int gbase = lane & ~3;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16) + 256u * g;
    uint32_t *gw32 = reinterpret_cast<uint32_t *>(smem + PR_GM_OFF + g * PR_GM_BYTES);  // [32 q][3][128 rows]
    double *red = reinterpret_cast<double *>(smem + PR_RED_OFF) + 64 * g;
    uint32_t ph = 0;
    for (int item = ec.cid + g * ec.ncl; item < ec.n_items; item += PR_GROUPS * ec.ncl) {
        const int t = item / args.n_ptiles, pt = item - t * args.n_ptiles;
        int BP, bq;
        pair_tile(pt, args.nb, BP, bq);
        const int bp = 2 * BP + ec.rank;
        // (1) G-(xe, ye) row c: entries d = 0, 1 (re, im), packed into three words per q.
        const bool got_m = mbar_wait(&mfull[g], ph, args.abort_flag, 4, args.timeout_ns);
        if (group_any(g, !got_m)) break;
        fence_after();
#pragma unroll 1
        for (int qb = 0; qb < PR_QW2 / 4; ++qb) {
            const int q0 = PR_QW2 * qhalf + 4 * qb;  // four q-pairs per tensor-memory load
            float vr[16], vi[16];
            tmem_ld<16>(lane_addr + 4u * q0, vr);
            tmem_ld<16>(lane_addr + 128u + 4u * q0, vi);
            tmem_wait_ld();
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const float o0r = e ? vr[4 * qq + 2] : vr[4 * qq], o0i = e ? vi[4 * qq + 2] : vi[4 * qq];
                const float o1r = e ? vr[4 * qq + 3] : vr[4 * qq + 1], o1i = e ? vi[4 * qq + 3] : vi[4 * qq + 1];
                const uint3 u = pack24(o0r, o0i, o1r, o1i);
                const int q = q0 + qq;
                gw32[(3 * q + 0) * 128 + row] = u.x;
                gw32[(3 * q + 1) * 128 + row] = u.y;
                gw32[(3 * q + 2) * 128 + row] = u.z;
            }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(ec.munl_even);
        // (2) traces once G+ is in the same columns.
        const bool got_p = mbar_wait(&pfull[g], ph, args.abort_flag, 6, args.timeout_ns);
        if (group_any(g, !got_p)) break;
        ph ^= 1u;
        fence_after();
        const int p = bp * 32 + p_local;
        const int q_lane = bq * 32 + lane;  // a_q of the tile's 32 q-pairs, one per lane
        const double a_lane = q_lane < args.m ? args.a[q_lane] : 0.0;
        double acc = 0.0;
#pragma unroll 1
        for (int qb = 0; qb < PR_QW2 / 4; ++qb) {
            const int q0 = PR_QW2 * qhalf + 4 * qb;
            float gpr[16], gpi[16];
            tmem_ld<16>(lane_addr + 4u * q0, gpr);
            tmem_ld<16>(lane_addr + 128u + 4u * q0, gpi);
            tmem_wait_ld();
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                // Row c of G-(xe, ye) [own], G+(xe, ye) [dia], G+(xe, y(1-e)) [off].
                const int ql = q0 + qq;
                float own_r[2], own_i[2];
                unpack24(gw32[(3 * ql + 0) * 128 + row], gw32[(3 * ql + 1) * 128 + row],
                         gw32[(3 * ql + 2) * 128 + row], own_r[0], own_i[0], own_r[1], own_i[1]);
                float dia_r[2], dia_i[2], off_r[2], off_i[2];
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    const int i0 = 4 * qq + d, i1 = 4 * qq + 2 + d;
                    dia_r[d] = e ? gpr[i1] : gpr[i0];
                    dia_i[d] = e ? gpi[i1] : gpi[i0];
                    off_r[d] = e ? gpr[i0] : gpr[i1];
                    off_i[d] = e ? gpi[i0] : gpi[i1];
                }
                // Direct: T_e = sum_cd conj(G-_cd) G+_cd over the like-electron block.
                float tr = 0.f, ti = 0.f;
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    tr += own_r[d] * dia_r[d] + own_i[d] * dia_i[d];
                    ti += own_r[d] * dia_i[d] - own_i[d] * dia_r[d];
                }
                tr += __shfl_xor_sync(0xffffffffu, tr, 1);
                ti += __shfl_xor_sync(0xffffffffu, ti, 1);
                const float ur = __shfl_xor_sync(0xffffffffu, tr, 2);
                const float ui = __shfl_xor_sync(0xffffffffu, ti, 2);
                const float direct_re = tr * ur - ti * ui;
                // Exchange: sum_{c,c''} U_{cc''} V_{c''c} with U = G+(1p,2q) G-(2p,2q)^dag and
                // V = G+(2p,1q) G-(1p,1q)^dag: lane (0, c) takes c'' = c, lane (1, c'') takes c = 1 - c'',
                // each pairing its rows with those of the other electron's lane.
                const int src = gbase + (e == 0 ? 2 + c : 1 - c);
                float a1r = 0.f, a1i = 0.f, a2r = 0.f, a2i = 0.f;
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    const float rg_r = __shfl_sync(0xffffffffu, own_r[d], src);
                    const float rg_i = __shfl_sync(0xffffffffu, own_i[d], src);
                    const float ro_r = __shfl_sync(0xffffffffu, off_r[d], src);
                    const float ro_i = __shfl_sync(0xffffffffu, off_i[d], src);
                    a1r += off_r[d] * rg_r + off_i[d] * rg_i;
                    a1i += off_i[d] * rg_r - off_r[d] * rg_i;
                    a2r += ro_r * own_r[d] + ro_i * own_i[d];
                    a2i += ro_i * own_r[d] - ro_r * own_i[d];
                }
                float xr = a1r * a2r - a1i * a2i;
                xr += __shfl_xor_sync(0xffffffffu, xr, 1);
                xr += __shfl_xor_sync(0xffffffffu, xr, 2);
                const int q = bq * 32 + ql;
                const double a_q = __shfl_sync(0xffffffffu, a_lane, ql);
                const bool valid = p < args.m && q < args.m && (bp < bq || (bp == bq && p_local < ql));
                if (valid) acc += (double)(-0.5f * (direct_re - xr)) * a_q;
                if (args.dbg.out && bp == args.dbg.bp && bq == args.dbg.bq && (lane & 3) == 0)
                    args.dbg.out[((size_t)t * 32 + p_local) * 32 + ql] =
                        valid ? (double)(-0.5f * (direct_re - xr)) * a_q * args.a[p] * args.inv_lambda : 0.0;
            }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(ec.pfree_even);
        if ((lane & 3) == 0) red[32 * qhalf + 8 * quarter + (lane >> 2)] = (p < args.m) ? acc * args.a[p] : 0.0;
        group_sync(g);
        if (gw == 0 && lane == 0 && bp <= bq) {
            double sum = 0.0;
            for (int j = 0; j < 32 * PR_QHALVES; ++j) sum += red[j];
            args.partials[(size_t)t * args.n_tiles + tile_index(bp, bq, args.nb)] = sum * args.inv_lambda;
        }
        group_sync(g);
    }
}

// Order in which a CTA pair contracts its chunks (producer and MMA issuer alike):
// each item's G+ chunks, with the next item's G- chunks issued PR_TAIL chunks
// before their end, so that the next group unloads its G- while these last G+
// MMAs run instead of leaving the tensor pipe idle.  f(li, item, occ, c) is
// called per chunk (li: the cluster's item counter) and returns false to stop.
constexpr int PR_TAIL = 5;
template <class F>
__device__ __forceinline__ bool for_each_chunk(int cid, int ncl, int n_items, int n_occ_chunks, int n_vir_chunks,
                                               F &&f)
{
    int li = 0;
    for (int item = cid; item < n_items; item += ncl, ++li) {
        const bool has_next = item + ncl < n_items;
        if (li == 0)
            for (int c = 0; c < n_occ_chunks; ++c)
                if (!f(li, item, true, c)) return false;
        const int tail = has_next ? (n_vir_chunks < PR_TAIL ? n_vir_chunks : PR_TAIL) : 0;
        for (int c = 0; c < n_vir_chunks - tail; ++c)
            if (!f(li, item, false, c)) return false;
        if (has_next)
            for (int c = 0; c < n_occ_chunks; ++c)
                if (!f(li + 1, item + ncl, true, c)) return false;
        for (int c = n_vir_chunks - tail; c < n_vir_chunks; ++c)
            if (!f(li, item, false, c)) return false;
    }
    return true;
}

template <bool TF32, int NC, int INTER = MCMP2_COULOMB>
__global__ void __launch_bounds__(PR_THREADS, 1) pairs_mixed_kernel(const __grid_constant__ PairMaps maps,
                                                                    const PairArgs args)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + PR_BARS_OFF);
    uint64_t *empty = full + PR_STAGES;
    uint64_t *mfull = empty + PR_STAGES;  // [group] G- accumulated (both CTAs)
    uint64_t *munl = mfull + PR_GROUPS;   // [group] G- copied out (even CTA: 8 warps x 2 CTAs)
    uint64_t *pfull = munl + PR_GROUPS;   // [group] G+ accumulated (both CTAs)
    uint64_t *pfree = pfull + PR_GROUPS;  // [group] columns free again (even CTA: 8 warps x 2 CTAs)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(pfree + PR_GROUPS);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int cid = (int)cluster_id(), ncl = (int)cluster_count();
    const int n_occ_chunks = pr_chunks(args.n_occ), n_vir_chunks = pr_chunks(args.n_vir);
    const int stages_per_tile = n_occ_chunks + n_vir_chunks;
    const int n_items = args.n_ptiles * args.n_tau;

    if (threadIdx.x == 0) {
        for (int s = 0; s < PR_STAGES; ++s) {
            mbar_init(&full[s], leader ? 2 : 1);  // even CTA: its own copies + the odd CTA's relay
            mbar_init(&empty[s], 1);
        }
        for (int g = 0; g < PR_GROUPS; ++g) {
            mbar_init(&mfull[g], 1);
            mbar_init(&munl[g], 2 * PR_GROUP_WARPS);
            mbar_init(&pfull[g], 1);
            mbar_init(&pfree[g], 2 * PR_GROUP_WARPS);
        }
        mbar_init_fence();
    }
    if (warp == 1) tmem_alloc_pair(tmem_slot, PR_TMEM_COLS);
    fence_before();
    __syncthreads();
    cluster_sync();  // barriers of both CTAs initialised before any remote arrive or multicast commit
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        if (lane == 0) {
            // B half: Y = (re, im) in the even CTA, iY = (-im, re) in the odd one.
            const CUtensorMap *b1_occ = leader ? &maps.hocc : &maps.nocc, *b1_vir = leader ? &maps.hvir : &maps.nvir;
            tma_prefetch(&maps.occ);
            tma_prefetch(&maps.vir);
            tma_prefetch(&maps.hocc);
            tma_prefetch(&maps.hvir);
            tma_prefetch(b1_occ);
            tma_prefetch(b1_vir);
            int stage = 0;
            uint32_t phase = 0;
            int issued[PR_STAGES] = {};
            uint32_t issued_phase[PR_STAGES] = {};
            int cur_item = -1, t = 0, a_row = 0, b_row = 0;
            const bool ok = for_each_chunk(cid, ncl, n_items, n_occ_chunks, n_vir_chunks,
                                           [&](int li, int item, bool occ, int c) {
                if (!mbar_wait_fast(&empty[stage], phase ^ 1u, args.abort_flag, 1, args.timeout_ns)) return false;
                if (args.withhold_first_copy && li == 0 && occ && c == 0) {
                    // Test hook: skip this stage entirely; nothing completes its barrier.
                    if (++stage == PR_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    return true;
                }
                if (item != cur_item) {
                    cur_item = item;
                    t = item / args.n_ptiles;
                    int BP, bq;
                    pair_tile(item - t * args.n_ptiles, args.nb, BP, bq);
                    // A CTA without a p-block (odd block count) loads the last block instead;
                    // its results are discarded.
                    const int bp = 2 * BP + (int)rank;
                    a_row = (bp < args.nb ? bp : args.nb - 1) * 128;
                    b_row = bq * 128;
                }
                const int x = c * 4 * PR_BK;
                unsigned char *st = smem + stage * PR_STAGE_BYTES;
                mbar_arrive_expect_tx(&full[stage], PR_STAGE_BYTES);
                tma_load_3d(st, occ ? &maps.occ : &maps.vir, &full[stage], x, a_row, t);
                // B tile 1 (real planes): X's re half (even CTA) or the -im planes (odd CTA);
                // B tile 2 (imaginary planes): X's im half (even CTA) or X's re half (odd CTA).
                tma_load_3d(st + PR_TILE_BYTES, occ ? b1_occ : b1_vir, &full[stage], leader ? x : x / 2, b_row, t);
                tma_load_3d(st + PR_TILE_BYTES + PR_BTILE_BYTES, occ ? &maps.hocc : &maps.hvir, &full[stage],
                            leader ? x + 2 * PR_BK : x, b_row, t);
                issued[stage] = 1;
                issued_phase[stage] = phase;
                if (++stage == PR_STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
                return true;
            });
            if (!ok)
                for (int s = 0; s < PR_STAGES; ++s)
                    if (issued[s]) mbar_drain(&full[s], issued_phase[s], args.timeout_ns);
        }
    } else if (warp == 1 && !leader) {
        // ---------------- relay (odd CTA): its copies landed -> the even CTA's stage barrier ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int item = cid; item < n_items && ok; item += ncl) {
                for (int c = 0; c < stages_per_tile; ++c) {
                    if (!mbar_wait(&full[stage], phase, args.abort_flag, 7, args.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(mapa_shared(&full[stage], 0));
                    if (++stage == PR_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (even CTA) ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t use[PR_GROUPS] = {0, 0};  // parity of each group's uses so far
            const uint32_t id = idesc_pair(TF32 ? idesc_tf32(256, false) : idesc_bf16(256, false));
            constexpr uint16_t BOTH = 3;
            // Descriptors of stage 0; stage s adds s * PR_STAGE_BYTES to the start-address
            // field (address >> 4 in the low 14 bits, no carry for addresses below 256 KB).
            // Keeping this loop short matters: the tensor pipe drains while it runs.
            const uint32_t base0 = smem_u32(smem);
            const uint64_t arh0 = sdesc_sw128(base0 + 0), arl0 = sdesc_sw128(base0 + 32);
            const uint64_t aih0 = sdesc_sw128(base0 + 64), ail0 = sdesc_sw128(base0 + 96);
            constexpr uint32_t BOFF = PR_TILE_BYTES, BOFF2 = PR_TILE_BYTES + PR_BTILE_BYTES;
            const uint64_t brh0 = sdesc_sw64(base0 + BOFF + 0), brl0 = sdesc_sw64(base0 + BOFF + 32);
            const uint64_t bih0 = sdesc_sw64(base0 + BOFF2 + 0), bil0 = sdesc_sw64(base0 + BOFF2 + 32);
            for_each_chunk(cid, ncl, n_items, n_occ_chunks, n_vir_chunks, [&](int li, int, bool occ, int c) {
                const int g = li & 1;
                const uint32_t d = tmem + 256u * g;  // [Re G | Im G]
                if (c == 0) {
                    // G-: the group has traced its previous item; G+: it has unloaded this item's G-.
                    const bool ready = occ ? mbar_wait_fast(&pfree[g], use[g] ^ 1u, args.abort_flag, 2, args.timeout_ns)
                                           : mbar_wait_fast(&munl[g], use[g], args.abort_flag, 5, args.timeout_ns);
                    if (!ready) return false;
                    fence_after();
                }
                if (!mbar_wait_fast(&full[stage], phase, args.abort_flag, 3, args.timeout_ns)) return false;
                fence_after();
                const uint64_t so = (uint64_t)(stage * (PR_STAGE_BYTES >> 4));
                const uint64_t arh = arh0 + so, arl = arl0 + so, aih = aih0 + so, ail = ail0 + so;
                const uint64_t brh = brh0 + so, brl = brl0 + so, bih = bih0 + so, bil = bil0 + so;
                const uint32_t acc = c == 0 ? 0u : 1u;
                // [Re | Im] += X_re [Y; iY]_re^T + X_im [Y; iY]_im^T (straight-line code:
                // the issue loop must stay short, the tensor pipe drains while it runs).
                if constexpr (TF32) {
                    // descriptors at +0, +32, +64, +96: re K 0-7, re K 8-15, im K 0-7, im K 8-15
                    umma_pair_tf32(d, arh, brh, id, acc);
                    umma_pair_tf32(d, arl, brl, id, 1u);
                    umma_pair_tf32(d, aih, bih, id, 1u);
                    umma_pair_tf32(d, ail, bil, id, 1u);
                } else {
                    umma_pair(d, arh, brh, id, acc);
                    umma_pair(d, arh, brl, id, 1u);
                    umma_pair(d, arl, brh, id, 1u);
                    umma_pair(d, aih, bih, id, 1u);
                    umma_pair(d, aih, bil, id, 1u);
                    umma_pair(d, ail, bih, id, 1u);
                }
                umma_pair_commit(&empty[stage], BOTH);
                if (++stage == PR_STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
                if (occ && c == n_occ_chunks - 1) umma_pair_commit(&mfull[g], BOTH);  // G- to both CTAs' group
                if (!occ && c == n_vir_chunks - 1) {                               // G+ complete
                    umma_pair_commit(&pfull[g], BOTH);
                    use[g] ^= 1u;
                }
                return true;
            });
            // Let every MMA this thread issued finish before tensor memory is freed.
            umma_pair_commit(&empty[stage], 1);
            mbar_drain(&empty[stage], phase, args.timeout_ns);
        }
    } else {
        // ---------------- epilogue: two groups of 8 warps per CTA, alternate items ----------------
        const int g = (warp - 2) / PR_GROUP_WARPS;
        const EpiCtx ec{(int)rank, cid, ncl, n_items, mapa_shared(&munl[g], 0), mapa_shared(&pfree[g], 0)};
        if constexpr (NC == 2)
            pairs_epilogue_2c(args, smem, tmem, warp, lane, ec, mfull, pfull);
        else
            pairs_epilogue_4c<INTER>(args, smem, tmem, warp, lane, ec, mfull, pfull);
    }
    fence_before();
    __syncthreads();
    cluster_sync();  // no MMA, copy or remote arrive of either CTA is outstanding past this point
    if (warp == 1) {
        fence_after();
        tmem_dealloc_pair(tmem, PR_TMEM_COLS);
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

// 2-D (or 3-D) BF16 tensor map with a box_k x 128 box: 32 elements with the 64-byte swizzle
// (spinor formation), or 64 with the 128-byte swizzle (contraction).
int encode(void *out, void *addr, int rank, const cuuint64_t *dims, const cuuint64_t *strides, std::string &err,
           int box_k = BK, CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_64B)
{
    auto enc = encode_fn();
    if (!enc) {
        err = "cuTensorMapEncodeTiled is not available from the driver";
        return MCMP2_EUNSUPPORTED;
    }
    const cuuint32_t box[3] = {(cuuint32_t)box_k, 128u, 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap map;
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, addr, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return MCMP2_ECUDA;
    }
    std::memcpy(out, &map, sizeof(map));
    return MCMP2_OK;
}

// 4-D BF16 tensor map of one operand-row array for the spinor kernel's TMA stores:
// dims (element of a row, component, position, time).  planes = 4 (X: box {64, 1,
// 32, 1} = one 128-byte chunk of 32 positions' rows, 128-byte swizzle) or 2 (the
// -im planes: box {32, 1, 32, 1} = one 64-byte chunk, 64-byte swizzle).
int encode_store(void *out, void *addr, int kpad, int ncomp, int P, int rows, int n_tau, std::string &err,
                 int planes = 4)
{
    auto enc = encode_fn();
    if (!enc) {
        err = "cuTensorMapEncodeTiled is not available from the driver";
        return MCMP2_EUNSUPPORTED;
    }
    const cuuint64_t row_bytes = (cuuint64_t)planes * kpad * 2;
    const cuuint64_t dims[4] = {(cuuint64_t)planes * kpad, (cuuint64_t)ncomp, (cuuint64_t)P, (cuuint64_t)n_tau};
    const cuuint64_t strides[3] = {row_bytes, row_bytes * ncomp, row_bytes * rows};
    const cuuint32_t box[4] = {(cuuint32_t)(16 * planes), 1u, 32u, 1u};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUtensorMap map;
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, addr, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE,
                           planes == 4 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled (store) failed (" + std::to_string((int)r) + ")";
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
    L.k_occ_pad = (n_occ + 63) / 64 * 64;  // whole 64-orbital blocks: the spinor tiles write 512 B row segments
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
    L.occ_nplanes = take((size_t)n_tau * 2 * L.rows * L.k_occ_pad * 2);
    L.vir_nplanes = take((size_t)n_tau * 2 * L.rows * L.k_vir_pad * 2);
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
    // Contraction: operand rows [n_tau][rows][4 k_pad] as a 3-D tensor (chunk x plane x orbital, row, tau);
    // a two-component system fills the first 4m of the 8m rows of each time.
    plan.ncomp = s.n_comp == 2 ? 2 : 4;
    const int rows_used = 2 * plan.ncomp * s.m;
    // The spinor kernel's stores of those rows, row ncomp x + c of position x and component c.
    if ((rc = encode_store(plan.maps_spinor[8], ws + L.occ_planes, L.k_occ_pad, plan.ncomp, L.P, L.rows, L.n_tau,
                           err)) ||
        (rc = encode_store(plan.maps_spinor[9], ws + L.vir_planes, L.k_vir_pad, plan.ncomp, L.P, L.rows, L.n_tau,
                           err)) ||
        (rc = encode_store(plan.maps_spinor[10], ws + L.occ_nplanes, L.k_occ_pad, plan.ncomp, L.P, L.rows, L.n_tau,
                           err, 2)) ||
        (rc = encode_store(plan.maps_spinor[11], ws + L.vir_nplanes, L.k_vir_pad, plan.ncomp, L.P, L.rows, L.n_tau,
                           err, 2)))
        return rc;
    {
        const cuuint64_t dO[3] = {(cuuint64_t)4 * L.k_occ_pad, (cuuint64_t)rows_used, (cuuint64_t)L.n_tau};
        const cuuint64_t sO[2] = {(cuuint64_t)L.k_occ_pad * 8, (cuuint64_t)L.rows * L.k_occ_pad * 8};
        const cuuint64_t dV[3] = {(cuuint64_t)4 * L.k_vir_pad, (cuuint64_t)rows_used, (cuuint64_t)L.n_tau};
        const cuuint64_t sV[2] = {(cuuint64_t)L.k_vir_pad * 8, (cuuint64_t)L.rows * L.k_vir_pad * 8};
        // The -im planes: half the row length.
        const cuuint64_t nO[3] = {(cuuint64_t)2 * L.k_occ_pad, (cuuint64_t)rows_used, (cuuint64_t)L.n_tau};
        const cuuint64_t nsO[2] = {(cuuint64_t)L.k_occ_pad * 4, (cuuint64_t)L.rows * L.k_occ_pad * 4};
        const cuuint64_t nV[3] = {(cuuint64_t)2 * L.k_vir_pad, (cuuint64_t)rows_used, (cuuint64_t)L.n_tau};
        const cuuint64_t nsV[2] = {(cuuint64_t)L.k_vir_pad * 4, (cuuint64_t)L.rows * L.k_vir_pad * 4};
        const auto sw = CU_TENSOR_MAP_SWIZZLE_128B, sw64 = CU_TENSOR_MAP_SWIZZLE_64B;
        if ((rc = encode(plan.maps_pairs[0], ws + L.occ_planes, 3, dO, sO, err, 4 * PR_BK, sw)) ||
            (rc = encode(plan.maps_pairs[1], ws + L.vir_planes, 3, dV, sV, err, 4 * PR_BK, sw)) ||
            (rc = encode(plan.maps_pairs[2], ws + L.occ_planes, 3, dO, sO, err, 2 * PR_BK, sw64)) ||
            (rc = encode(plan.maps_pairs[3], ws + L.vir_planes, 3, dV, sV, err, 2 * PR_BK, sw64)) ||
            (rc = encode(plan.maps_pairs[4], ws + L.occ_nplanes, 3, nO, nsO, err, 2 * PR_BK, sw64)) ||
            (rc = encode(plan.maps_pairs[5], ws + L.vir_nplanes, 3, nV, nsV, err, 2 * PR_BK, sw64)))
            return rc;
    }
    if (cudaFuncSetAttribute(spinor_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SP_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel<false, 4, MCMP2_GAUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PR_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel<true, 4, MCMP2_GAUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PR_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel<false, 4, MCMP2_BREIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PR_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(pairs_mixed_kernel<true, 4, MCMP2_BREIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PR_SMEM) != cudaSuccess) {
        err = "cannot reserve shared memory for the tensor-core kernels";
        return MCMP2_ECUDA;
    }
    // CTA pairs that fit on the device at once (one per TPC): the contraction's persistent grid.
    {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cfg.gridDim = dim3(2 * (sms / 2));
        cfg.blockDim = dim3(PR_THREADS);
        cfg.dynamicSmemBytes = PR_SMEM;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, pairs_mixed_kernel<false, 4>, &cfg) != cudaSuccess || n < 1) {
            err = "the contraction kernel's CTA pairs cannot be resident on this device";
            return MCMP2_EUNSUPPORTED;
        }
        plan.pair_clusters = n;
        cfg.blockDim = dim3(SP_THREADS);
        cfg.dynamicSmemBytes = SP_SMEM;
        n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, spinor_mixed_kernel, &cfg) != cudaSuccess || n < 1) {
            err = "the spinor kernel's CTA pairs cannot be resident on this device";
            return MCMP2_EUNSUPPORTED;
        }
        plan.spinor_clusters = n;
    }
    plan.ready = true;
    return MCMP2_OK;
}

int mixed_step(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, const double *r,
               const float *scale, const double *a, double *partials, cudaStream_t st, std::string &err,
               cudaEvent_t *ev, int *n_launches, int *n_pair_launches, const DebugTile &dbg)
{
    if (!plan.ready) {
        err = "mixed path not prepared";
        return MCMP2_ENOTLOADED;
    }
    int *flag = reinterpret_cast<int *>(ws + L.flag);
    auto bf = [&](size_t off) { return reinterpret_cast<__nv_bfloat16 *>(ws + off); };

    dim3 gb((s.n_l + 127) / 128, L.P);
    basis_split_kernel<<<gb, 128, 0, st>>>(s, r, bf(L.BL_hi), bf(L.BL_lo), bf(L.BS_hi), bf(L.BS_lo), L.nl_pad,
                                           L.nl3_pad);

    SpinorMaps smaps;
    std::memcpy(&smaps, plan.maps_spinor, sizeof(smaps));
    const int n_mt = (L.P + 127) / 128;
    SpinorArgs sa{scale, flag, L.P, s.n_l, n_mt, L.n_kb, L.n_kb_occ, s.n_occ, s.n_vir, s.n_orb, s.n_tau,
                  plan.tf32 ? 1 : 0, plan.ncomp};
    const int sp_units = (n_mt + 1) / 2 * (plan.ncomp / 2) * L.n_kb;  // (position block pair, component pair, kb)
    const int sp_clusters = sp_units < plan.spinor_clusters ? sp_units : plan.spinor_clusters;
    cudaLaunchAttribute sp_attr[1];
    sp_attr[0].id = cudaLaunchAttributeClusterDimension;
    sp_attr[0].val.clusterDim.x = 2;
    sp_attr[0].val.clusterDim.y = 1;
    sp_attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t sp_cfg = {};
    sp_cfg.gridDim = dim3(2 * sp_clusters);
    sp_cfg.blockDim = dim3(SP_THREADS);
    sp_cfg.dynamicSmemBytes = SP_SMEM;
    sp_cfg.stream = st;
    sp_cfg.attrs = sp_attr;
    sp_cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&sp_cfg, spinor_mixed_kernel, smaps, sa) != cudaSuccess) {
        err = "spinor formation launch failed";
        return MCMP2_ECUDA;
    }

    PairMaps pmaps;
    std::memcpy(&pmaps.occ, plan.maps_pairs[0], sizeof(CUtensorMap));
    std::memcpy(&pmaps.vir, plan.maps_pairs[1], sizeof(CUtensorMap));
    std::memcpy(&pmaps.hocc, plan.maps_pairs[2], sizeof(CUtensorMap));
    std::memcpy(&pmaps.hvir, plan.maps_pairs[3], sizeof(CUtensorMap));
    std::memcpy(&pmaps.nocc, plan.maps_pairs[4], sizeof(CUtensorMap));
    std::memcpy(&pmaps.nvir, plan.maps_pairs[5], sizeof(CUtensorMap));
    const int nb = pair_blocks(s.m, plan.ncomp == 2 ? TILE_PAIRS_MIXED_2C : TILE_PAIRS_MIXED);
    const int n_tiles = nb * (nb + 1) / 2;
    int n_ptiles = 0;  // pair tiles: two p-blocks x one q-block, q-block >= the first p-block
    for (int b = 0; 2 * b < nb; ++b) n_ptiles += nb - 2 * b;
    PairArgs pa{a, partials, flag, s.m, n_tiles, n_ptiles, nb, s.n_tau, s.n_occ, s.n_vir, 1.0 / s.lambda,
                TIMEOUT_NS, 0, r};
    pa.dbg = dbg;
    if (plan.withhold_once_ns) {
        pa.withhold_first_copy = 1;
        pa.timeout_ns = plan.withhold_once_ns;
        plan.withhold_once_ns = 0;
    }
    const int items = n_ptiles * s.n_tau;
    const int clusters = items < plan.pair_clusters ? items : plan.pair_clusters;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(PR_THREADS);
    cfg.dynamicSmemBytes = PR_SMEM;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (ev) record_event(ev[0], st);
    cudaError_t e;
    if (plan.ncomp == 2)
        e = plan.tf32 ? cudaLaunchKernelEx(&cfg, pairs_mixed_kernel<true, 2>, pmaps, pa)
                      : cudaLaunchKernelEx(&cfg, pairs_mixed_kernel<false, 2>, pmaps, pa);
    else if (s.interaction == MCMP2_GAUNT)
        e = plan.tf32 ? cudaLaunchKernelEx(&cfg, pairs_mixed_kernel<true, 4, MCMP2_GAUNT>, pmaps, pa)
                      : cudaLaunchKernelEx(&cfg, pairs_mixed_kernel<false, 4, MCMP2_GAUNT>, pmaps, pa);
    else if (s.interaction == MCMP2_BREIT)
        e = plan.tf32 ? cudaLaunchKernelEx(&cfg, pairs_mixed_kernel<true, 4, MCMP2_BREIT>, pmaps, pa)
                      : cudaLaunchKernelEx(&cfg, pairs_mixed_kernel<false, 4, MCMP2_BREIT>, pmaps, pa);
    else
        e = plan.tf32 ? cudaLaunchKernelEx(&cfg, pairs_mixed_kernel<true, 4>, pmaps, pa)
                      : cudaLaunchKernelEx(&cfg, pairs_mixed_kernel<false, 4>, pmaps, pa);
    if (ev) record_event(ev[1], st);
    if (e == cudaSuccess) e = cudaGetLastError();
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
