// Mixed-precision propagator contraction on the tcgen05 tensor cores (sm_103a).
//
// For each imaginary time the scaled spinor values X(x)_ck = phi_k^c(x) s_k(tau)
// (rows x,c = 8p + 4e + c for electron e of walker pair p) are split into
// BF16 hi/lo planes of their real and imaginary parts.  A tile of 16 p-pairs
// x 16 q-pairs computes, for all 128 x 128 (row, column) pairs,
//   G(x, y)_cd = sum_k X(x)_ck conj(X(y)_dk)
//   Re G = Xr Yr^T + Xi Yi^T,   Im G = Xi Yr^T - Xr Yi^T,
// each real product as hi*hi + hi*lo + lo*hi (split BF16 x3, FP32 accumulate
// in tensor memory), over the occupied spinors (G-) and the virtual ones (G+).
// The epilogue forms the direct and exchange traces of the trace form of
// Eq. MCMP2 for every pair of pairs of the tile and accumulates
// Re f / (w w w) in FP64.
//
// Roles (192 threads): warp 0 lane 0 issues TMA loads, warp 1 allocates tensor
// memory and lane 0 issues the MMAs, warps 2..5 run the epilogue (one per
// tensor-memory lane quarter).  Every wait is bounded in time; on a time-out
// the kernel records it in a flag, stops, waits (bounded) for its own copies,
// frees tensor memory and returns, and the host reports MCMP2_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>

#include "../../include/mcmp2.h"
#include "mixed.cuh"

namespace mcmp2 {

namespace {

constexpr int BM = 128;                   // rows per tile side (16 walker pairs x 8)
constexpr int BK = 32;                    // K elements per stage (64 bytes: one 64B swizzle row)
constexpr int STAGES = 3;
constexpr int PLANE_TILE = BM * BK * 2;   // 8 KB
constexpr int STAGE_BYTES = 8 * PLANE_TILE;  // A and B, 4 planes each
constexpr int TMEM_COLS = 512;            // G+ re | G+ im | G- re | G- im, 128 columns each
constexpr int THREADS = 192;
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;  // 2 s per wait

struct MixedMaps {
    CUtensorMap m[8];  // [occ 0..3 | vir 4..7]: re_hi, re_lo, im_hi, im_lo
};

struct MixedArgs {
    const double *a;      // [m] pair weight factors N_g / (g1 g2)
    double *partials;     // [n_tau][n_tiles]
    int *abort_flag;      // set to a nonzero code on a time-out
    int m, n_tiles, nb, t_index, n_occ, n_vir;
    double inv_lambda;
};

struct SmemLayout {
    static constexpr int stages_off = 0;
    static constexpr int bars_off = STAGES * STAGE_BYTES;  // full[S], empty[S], tmem_full, tmem_empty
    static constexpr int tmem_slot_off = bars_off + (2 * STAGES + 2) * 8;
    static constexpr int red_off = tmem_slot_off + 16;     // 16 doubles: per-pair-group partial sums
    static constexpr int total = red_off + 16 * 8;
};
constexpr int SMEM_BYTES = SmemLayout::total + 1024;  // slack for 1024-byte alignment

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a barrier phase.  Returns false (after recording `code`) on a
// time-out, or if another role has already aborted.
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *abort_flag, int code)
{
    const unsigned long long t0 = globaltimer();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63) {
            if (*(volatile int *)abort_flag) return false;
            if (globaltimer() - t0 > TIMEOUT_NS) {
                atomicCAS(abort_flag, 0, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle (8 rows x 64 B atoms,
// stride 512 B between 8-row groups), SM100 descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;   // leading-dimension offset (unused for swizzled K-major)
    d |= (uint64_t)(512u >> 4) << 32;  // stride-dimension offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)4 << 61;            // SWIZZLE_64B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = N = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(bool negate_a)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((negate_a ? 1u : 0u) << 13) | ((uint32_t)(128 >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tile_coords(int tile, int nb, int &bp, int &bq)
{
    int k = tile, b = 0;
    while (k >= nb - b) {
        k -= nb - b;
        ++b;
    }
    bp = b;
    bq = b + k;
}

__device__ __forceinline__ int k_chunks(int n) { return (n + BK - 1) / BK; }

// OR of a predicate over the 128 epilogue threads (named barrier 1).
__device__ __forceinline__ bool epilogue_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(THREADS, 1) pairs_mixed_kernel(const __grid_constant__ MixedMaps maps,
                                                                 const MixedArgs args)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + SmemLayout::bars_off);
    uint64_t *empty = full + STAGES;
    uint64_t *tmem_full = empty + STAGES;
    uint64_t *tmem_empty = tmem_full + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SmemLayout::tmem_slot_off);
    double *red = reinterpret_cast<double *>(smem + SmemLayout::red_off);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_occ_chunks = k_chunks(args.n_occ), n_vir_chunks = k_chunks(args.n_vir);
    const int chunks_per_tile = n_occ_chunks + n_vir_chunks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tmem_full, 1);
        mbar_init(tmem_empty, 4);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            for (int s = 0; s < 8; ++s)
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.m[s])) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            int issued[STAGES] = {};
            uint32_t issued_phase[STAGES] = {};
            bool ok = true;
            for (int tile = blockIdx.x; tile < args.n_tiles && ok; tile += gridDim.x) {
                int bp, bq;
                tile_coords(tile, args.nb, bp, bq);
                for (int c = 0; c < chunks_per_tile; ++c) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, args.abort_flag, 1)) {
                        ok = false;
                        break;
                    }
                    const bool occ = c < n_occ_chunks;
                    const int x = (occ ? c : c - n_occ_chunks) * BK;
                    const CUtensorMap *mp = &maps.m[occ ? 0 : 4];
                    unsigned char *st = smem + stage * STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[stage], STAGE_BYTES);
#pragma unroll
                    for (int pl = 0; pl < 4; ++pl) {
                        tma_load_2d(st + pl * PLANE_TILE, mp + pl, &full[stage], x, bp * BM);
                        tma_load_2d(st + (4 + pl) * PLANE_TILE, mp + pl, &full[stage], x, bq * BM);
                    }
                    issued[stage] = 1;
                    issued_phase[stage] = phase;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Drain: wait (bounded) until the last copies issued into each stage have landed.
                for (int s = 0; s < STAGES; ++s) {
                    if (!issued[s]) continue;
                    const unsigned long long t0 = globaltimer();
                    while (!mbar_try_wait(&full[s], issued_phase[s]) && globaltimer() - t0 < TIMEOUT_NS) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, tphase = 0;
            bool ok = true;
            const uint32_t id_pos = idesc_bf16(false), id_neg = idesc_bf16(true);
            for (int tile = blockIdx.x; tile < args.n_tiles && ok; tile += gridDim.x) {
                if (!mbar_wait(tmem_empty, tphase ^ 1u, args.abort_flag, 2)) {
                    ok = false;
                    break;
                }
                fence_after();
                for (int c = 0; c < chunks_per_tile; ++c) {
                    if (!mbar_wait(&full[stage], phase, args.abort_flag, 3)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const bool occ = c < n_occ_chunks;
                    const int cc = occ ? c : c - n_occ_chunks;
                    const int kvalid = (occ ? args.n_occ : args.n_vir) - cc * BK;
                    const int ksteps = kvalid >= BK ? BK / 16 : (kvalid + 15) / 16;
                    const uint32_t d_re = tmem + (occ ? 256u : 0u), d_im = d_re + 128u;
                    const uint32_t base = smem_u32(smem + stage * STAGE_BYTES);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint32_t off = ks * 32;  // 16 BF16 along K
                        const uint64_t arh = sdesc(base + 0 * PLANE_TILE + off), arl = sdesc(base + 1 * PLANE_TILE + off);
                        const uint64_t aih = sdesc(base + 2 * PLANE_TILE + off), ail = sdesc(base + 3 * PLANE_TILE + off);
                        const uint64_t brh = sdesc(base + 4 * PLANE_TILE + off), brl = sdesc(base + 5 * PLANE_TILE + off);
                        const uint64_t bih = sdesc(base + 6 * PLANE_TILE + off), bil = sdesc(base + 7 * PLANE_TILE + off);
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
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                umma_commit(tmem_full);
                tphase ^= 1u;
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
        const int row = 32 * quarter + lane;
        const int p_local = row >> 3, e = (row >> 2) & 1;
        const int gbase = lane & ~7;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
        uint32_t ephase = 0;
        for (int tile = blockIdx.x; tile < args.n_tiles; tile += gridDim.x) {
            int bp, bq;
            tile_coords(tile, args.nb, bp, bq);
            const bool got = mbar_wait(tmem_full, ephase, args.abort_flag, 4);
            if (epilogue_any(!got)) break;  // all four epilogue warps leave together
            ephase ^= 1u;
            fence_after();
            const int p = bp * 16 + p_local;
            double acc = 0.0;  // sum over q of Re f_pq a_q (valid in every lane of the group)
            for (int ql = 0; ql < 16; ++ql) {
                float gpr[8], gpi[8], gmr[8], gmi[8];
                const uint32_t col = 8u * ql;
                tmem_ld8(lane_addr + col, gpr);
                tmem_ld8(lane_addr + 128u + col, gpi);
                tmem_ld8(lane_addr + 256u + col, gmr);
                tmem_ld8(lane_addr + 384u + col, gmi);
                tmem_wait_ld();
                // This lane holds row c of: G-(xe, ye) [own], G+(xe, ye) [diag], G+(xe, y(1-e)) [off].
                float own_r[4], own_i[4], dia_r[4], dia_i[4], off_r[4], off_i[4];
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    own_r[d] = gmr[4 * e + d];
                    own_i[d] = gmi[4 * e + d];
                    dia_r[d] = gpr[4 * e + d];
                    dia_i[d] = gpi[4 * e + d];
                    off_r[d] = gpr[4 * (1 - e) + d];
                    off_i[d] = gpi[4 * (1 - e) + d];
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
                // Exchange: tr[G-(1q,1p) G+(1p,2q) G-(2q,2p) G+(2p,1q)] = sum_{c,c''} U_{cc''} V_{c''c}
                // with U = G+(1p,2q) G-(2p,2q)^dag and V = G+(2p,1q) G-(1p,1q)^dag.  Lane (e, c)
                // pairs its rows with those of lane (1-e, c'') received by shuffle; e = 0 lanes
                // take c'' - c = 0, 1 and e = 1 lanes c'' - c = 2, 3 (mod 4).
                float xr = 0.f;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int c = lane & 3;
                    const int src = gbase + (e == 0 ? 4 + ((c + s) & 3) : ((c + 2 - s) & 3));
                    float rg_r[4], rg_i[4], ro_r[4], ro_i[4];
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        rg_r[d] = __shfl_sync(0xffffffffu, own_r[d], src);
                        rg_i[d] = __shfl_sync(0xffffffffu, own_i[d], src);
                        ro_r[d] = __shfl_sync(0xffffffffu, off_r[d], src);
                        ro_i[d] = __shfl_sync(0xffffffffu, off_i[d], src);
                    }
                    // A1 = sum_b own_off[b] conj(recv_own[b]); A2 = sum_a recv_off[a] conj(own[a])
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
                const bool valid = p < args.m && q < args.m && (bp < bq || p_local < ql);
                if (valid) acc += (double)(-0.5f * (direct_re - xr)) * args.a[q];
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_empty);
            // Per-pair sums: lane 8j of the warp holds pair p_local = 4 quarter + j.
            if ((lane & 7) == 0) red[4 * quarter + (lane >> 3)] = (p < args.m) ? acc * args.a[p] : 0.0;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (warp == 2 && lane == 0) {
                double sum = 0.0;
                for (int j = 0; j < 16; ++j) sum += red[j];
                args.partials[(size_t)args.t_index * args.n_tiles + tile] = sum * args.inv_lambda;
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Scale and split: plane[pl][row][k] for the occupied (k < n_occ) or virtual block,
// X = phi * s_k(tau) in FP32, hi = bf16(X), lo = bf16(X - hi).
__global__ void scale_split_kernel(const float2 *__restrict__ phi, const double *__restrict__ scale, int rows,
                                   int n_occ, int n_vir, int k_occ_pad, int k_vir_pad, __nv_bfloat16 *occ_planes,
                                   __nv_bfloat16 *vir_planes)
{
    const int n_orb = n_occ + n_vir;
    const int row = blockIdx.y;
    const size_t occ_plane = (size_t)rows * k_occ_pad, vir_plane = (size_t)rows * k_vir_pad;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_orb; k += gridDim.x * blockDim.x) {
        const float2 v = phi[(size_t)row * n_orb + k];
        const float s = (float)scale[k];
        const float xr = v.x * s, xi = v.y * s;
        const __nv_bfloat16 rh = __float2bfloat16_rn(xr), ih = __float2bfloat16_rn(xi);
        const __nv_bfloat16 rl = __float2bfloat16_rn(xr - __bfloat162float(rh));
        const __nv_bfloat16 il = __float2bfloat16_rn(xi - __bfloat162float(ih));
        __nv_bfloat16 *base;
        size_t plane, idx;
        if (k < n_occ) {
            base = occ_planes;
            plane = occ_plane;
            idx = (size_t)row * k_occ_pad + k;
        } else {
            base = vir_planes;
            plane = vir_plane;
            idx = (size_t)row * k_vir_pad + (k - n_occ);
        }
        base[idx] = rh;
        base[plane + idx] = rl;
        base[2 * plane + idx] = ih;
        base[3 * plane + idx] = il;
    }
}

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

}  // namespace

MixedLayout mixed_layout(int m, int n_occ, int n_vir, size_t offset)
{
    MixedLayout L{};
    L.k_occ_pad = (n_occ + 7) / 8 * 8;
    L.k_vir_pad = (n_vir + 7) / 8 * 8;
    L.rows = 8 * m;
    L.rows_pad = L.rows;
    L.planes = align256(offset);
    L.planes_bytes = (size_t)4 * L.rows * (L.k_occ_pad + L.k_vir_pad) * 2;
    L.end = align256(L.planes + L.planes_bytes) + 256;  // + the time-out flag word
    return L;
}

int mixed_prepare(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, std::string &err)
{
    plan.ready = false;
    auto enc = encode_fn();
    if (!enc) {
        err = "cuTensorMapEncodeTiled is not available from the driver";
        return MCMP2_EUNSUPPORTED;
    }
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    char *occ = ws + L.planes;
    char *vir = occ + (size_t)4 * L.rows * L.k_occ_pad * 2;
    for (int blk = 0; blk < 2; ++blk) {
        const int kv = blk == 0 ? s.n_occ : s.n_vir;
        const int kp = blk == 0 ? L.k_occ_pad : L.k_vir_pad;
        char *base = blk == 0 ? occ : vir;
        for (int pl = 0; pl < 4; ++pl) {
            CUtensorMap map;
            const cuuint64_t dims[2] = {(cuuint64_t)kv, (cuuint64_t)L.rows};
            const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
            const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
            const cuuint32_t estr[2] = {1, 1};
            void *addr = base + (size_t)pl * L.rows * kp * 2;
            const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, addr, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
                return MCMP2_ECUDA;
            }
            std::memcpy(plan.tmap[blk * 4 + pl], &map, sizeof(map));
        }
    }
    plan.flag_off = align256(L.planes + L.planes_bytes);
    if (cudaMemset(ws + plan.flag_off, 0, sizeof(int)) != cudaSuccess) {
        err = "cudaMemset of the time-out flag failed";
        return MCMP2_ECUDA;
    }
    if (cudaFuncSetAttribute(pairs_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
        cudaSuccess) {
        err = "cannot reserve shared memory for the tensor-core kernel";
        return MCMP2_ECUDA;
    }
    plan.ready = true;
    return MCMP2_OK;
}

int mixed_pairs(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, const float *phi,
                const double *scale, const double *a, double *partials, cudaStream_t st, std::string &err,
                cudaEvent_t *ev, int *n_launches, int *n_pair_launches)
{
    if (!plan.ready) {
        err = "mixed path not prepared";
        return MCMP2_ENOTLOADED;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = pair_blocks(s.m, 16);
    const int n_tiles = nb * (nb + 1) / 2;
    MixedMaps maps;
    std::memcpy(&maps, plan.tmap, sizeof(maps));
    __nv_bfloat16 *occ = reinterpret_cast<__nv_bfloat16 *>(ws + L.planes);
    __nv_bfloat16 *vir = occ + (size_t)4 * L.rows * L.k_occ_pad;
    int *flag = reinterpret_cast<int *>(ws + plan.flag_off);
    MixedArgs args{a, partials, flag, s.m, n_tiles, nb, 0, s.n_occ, s.n_vir, 1.0 / s.lambda};
    const int grid = n_tiles < sms ? n_tiles : sms;
    int launches = 0, pair_launches = 0;
    for (int t = 0; t < s.n_tau; ++t) {
        dim3 g((s.n_orb + 255) / 256, L.rows);
        scale_split_kernel<<<g, 256, 0, st>>>(reinterpret_cast<const float2 *>(phi), scale + (size_t)t * s.n_orb, L.rows,
                                              s.n_occ, s.n_vir, L.k_occ_pad, L.k_vir_pad, occ, vir);
        ++launches;
        if (ev) cudaEventRecord(ev[2 * t], st);
        args.t_index = t;
        pairs_mixed_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(maps, args);
        if (ev) cudaEventRecord(ev[2 * t + 1], st);
        ++launches;
        ++pair_launches;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("tensor-core contraction launch: ") + cudaGetErrorString(e);
        return MCMP2_ECUDA;
    }
    if (n_launches) *n_launches = launches;
    if (n_pair_launches) *n_pair_launches = pair_launches;
    return MCMP2_OK;
}

int mixed_check_flag(MixedPlan &plan, char *ws, cudaStream_t st, std::string &err)
{
    int h = 0;
    if (cudaMemcpyAsync(&h, ws + plan.flag_off, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        err = "cannot read the time-out flag";
        return MCMP2_ECUDA;
    }
    if (h != 0) {
        err = "tensor-core contraction timed out waiting (role " + std::to_string(h) + ")";
        cudaMemsetAsync(ws + plan.flag_off, 0, sizeof(int), st);
        return MCMP2_ETIMEOUT;
    }
    return MCMP2_OK;
}

void mixed_release(MixedPlan &plan) { plan.ready = false; }

}  // namespace mcmp2
