// FP64 form of the integrand engine: basis values at the walker positions,
// spinor formation (Eq. C with kinetic balance) and the propagator blocks with
// the traced direct and exchange products (trace form of Eq. MCMP2).
// GB300 runs FP64 on CUDA cores only, so these kernels are plain DFMA code;
// the mixed form (k_mixed.cu) is the tensor-core path.
#include "internal.cuh"

namespace mcmp2 {

// ---------------------------------------------------------------------------
// Basis values: B[x][0:n_l] = g_mu(r_x), B[x][(1+j) n_l + mu] = d g_mu / d x_j.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void basis_kernel(DevSystem s, const double *__restrict__ r, T *__restrict__ B, int ldb)
{
    const int x = blockIdx.y;
    const int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu >= s.n_l) return;
    const int sh = s.fn_shell[mu];
    const double *A = s.centres + 3 * s.shell_centre[sh];
    const double d[3] = {r[3 * x + 0] - A[0], r[3 * x + 1] - A[1], r[3 * x + 2] - A[2]};
    const double al = s.shell_alpha[sh];
    const double e = s.shell_coef[sh] * exp(-al * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
    const int pw[3] = {s.fn_pow[3 * mu], s.fn_pow[3 * mu + 1], s.fn_pow[3 * mu + 2]};
    double pk[3], dk[3];  // x_j^a and d/dx_j [x_j^a e^{-al x_j^2}] / e^{-al x_j^2}
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double v = 1.0;
        for (int i = 0; i < pw[j]; ++i) v *= d[j];
        pk[j] = v;
        double lower = 0.0;
        if (pw[j] > 0) {
            lower = 1.0;
            for (int i = 0; i < pw[j] - 1; ++i) lower *= d[j];
            lower *= pw[j];
        }
        dk[j] = lower - 2.0 * al * v * d[j];
    }
    T *row = B + (size_t)x * ldb;
    row[mu] = (T)(pk[0] * pk[1] * pk[2] * e);
    row[s.n_l + mu] = (T)(dk[0] * pk[1] * pk[2] * e);
    row[2 * s.n_l + mu] = (T)(pk[0] * dk[1] * pk[2] * e);
    row[3 * s.n_l + mu] = (T)(pk[0] * pk[1] * dk[2] * e);
}

template <typename T>
cudaError_t launch_basis(const DevSystem &s, const double *r, T *B, cudaStream_t st)
{
    const int threads = 128;
    dim3 grid((s.n_l + threads - 1) / threads, 2 * s.m);
    basis_kernel<T><<<grid, threads, 0, st>>>(s, r, B, 4 * s.n_l);
    return cudaGetLastError();
}
template cudaError_t launch_basis<double>(const DevSystem &, const double *, double *, cudaStream_t);

// ---------------------------------------------------------------------------
// Row-major C[M x N] = A[M x K] B[K x N]: 64 x 64 tiles, 4 x 4 per thread.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) gemm_rm_kernel(int M, int N, int K, const T *__restrict__ A, int lda,
                                                      const T *__restrict__ Bm, int ldb, T *__restrict__ C,
                                                      int ldc)
{
    __shared__ T As[16][64 + 1];
    __shared__ T Bs[16][64 + 1];
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int rr = i >> 4, kk = i & 15;
            const int gr = row0 + rr, gk = k0 + kk;
            As[kk][rr] = (gr < M && gk < K) ? A[(size_t)gr * lda + gk] : T(0);
            const int kb = i >> 6, cc = i & 63;
            const int gkb = k0 + kb, gc = col0 + cc;
            Bs[kb][cc] = (gkb < K && gc < N) ? Bm[(size_t)gkb * ldb + gc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gr = row0 + ty + 16 * i, gc = col0 + tx + 16 * j;
            if (gr < M && gc < N) C[(size_t)gr * ldc + gc] = acc[i][j];
        }
}

template <typename T>
static cudaError_t gemm_rm(int M, int N, int K, const T *A, int lda, const T *B, int ldb, T *C, int ldc,
                           cudaStream_t st)
{
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    gemm_rm_kernel<T><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
    return cudaGetLastError();
}

// Spinor values phi[x][c][k] (complex, c = L-alpha, L-beta, S-alpha, S-beta):
// the large components contract basis values with C^L (Eq. C); the small ones
// contract the gradients with the Pauli-folded C^S (the kinetic-balance condition after Eq. C).  Two-component
// systems (s.n_comp == 2) have the large components only: phi[x][c][k], c =
// alpha, beta.
cudaError_t launch_spinors_f64(const DevSystem &s, const double *B, double *phi, cudaStream_t st)
{
    const int P = 2 * s.m, n4 = 4 * s.n_orb, ld = 2 * s.n_comp * s.n_orb;
    cudaError_t e = gemm_rm<double>(P, n4, s.n_l, B, 4 * s.n_l, s.WL, n4, phi, ld, st);
    if (e != cudaSuccess || s.n_comp == 2) return e;
    return gemm_rm<double>(P, n4, 3 * s.n_l, B + s.n_l, 4 * s.n_l, s.WS, n4, phi + n4, ld, st);
}

// ---------------------------------------------------------------------------
// Pair-of-pairs tiles (FP64 form)
// ---------------------------------------------------------------------------
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

constexpr int F64_TP = TILE_PAIRS_F64;  // 8 pairs = 16 positions = 64 rows per side
constexpr int F64_KC = 16;              // orbitals per staged chunk

// NC = 4 components (L-alpha, L-beta, S-alpha, S-beta) or 2 (alpha, beta: the
// two-component variant); blocks are NC x NC.
template <int NC>
struct F64Smem {
    double2 Gm[2][F64_TP][F64_TP][NC * NC];  // G-(x, y) for same-electron position pairs, [e][xp][yp][c*NC+d]
    union {
        struct {
            double2 A[F64_KC][16 * NC];
            double2 B[F64_KC][16 * NC];
        } ld;
        double2 Gp[16][16][NC * NC];          // G+(x, y) for all position pairs, [xl][yl][c*NC+d]
    } u;
    double part[64];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmulc(double2 a, double2 b)  // conj(a) * b
{
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------------------
// Gaunt and Breit terms of the interaction (Sec. II):
//   g(a,b) = 1/r_ab - alpha(a).alpha(b) / (2 r_ab) - (alpha(a).r_ab)(alpha(b).r_ab) / (2 r_ab^3)
//          = (1/r_ab) sum_A c_A O_A(a) O_A(b),
// O_0 = 1 (c = 1); O_k = alpha_k, k = x, y, z (c = -1/2); O_n = alpha.n with n the
// unit vector from b to a (c = -1/2, Breit only).  alpha.v has sigma.v in its
// off-diagonal 2x2 blocks (components L-alpha, L-beta, S-alpha, S-beta).  The
// operator of each electron pair sits where the two propagators meet at its
// points:  direct  tr[G-(1q,1p) O_A G+(1p,1q) O_B] tr[G-(2q,2p) O_A G+(2p,2q) O_B],
//          exchange tr[G-(1q,1p) O_A G+(1p,2q) O_B G-(2q,2p) O_A G+(2p,1q) O_B],
// summed over the terms A of pair p and B of pair q with c_A c_B.
// ---------------------------------------------------------------------------
struct InteractionTerm {
    bool identity;
    double v[3];  // alpha.v
    double c;
};

// Y = X O for a 4x4 complex X (row-major) and O = 1 or alpha.v.
__device__ __forceinline__ void rmul_op(const double2 *X, const InteractionTerm &o, double2 *Y)
{
    if (o.identity) {
#pragma unroll
        for (int j = 0; j < 16; ++j) Y[j] = X[j];
        return;
    }
    const double2 s00 = make_double2(o.v[2], 0.0), s01 = make_double2(o.v[0], -o.v[1]);
    const double2 s10 = make_double2(o.v[0], o.v[1]), s11 = make_double2(-o.v[2], 0.0);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double2 x0 = X[4 * c], x1 = X[4 * c + 1], x2 = X[4 * c + 2], x3 = X[4 * c + 3];
        const double2 a0 = cmul(x2, s00), a1 = cmul(x3, s10), b0 = cmul(x2, s01), b1 = cmul(x3, s11);
        const double2 c0 = cmul(x0, s00), c1 = cmul(x1, s10), d0 = cmul(x0, s01), d1 = cmul(x1, s11);
        Y[4 * c] = make_double2(a0.x + a1.x, a0.y + a1.y);
        Y[4 * c + 1] = make_double2(b0.x + b1.x, b0.y + b1.y);
        Y[4 * c + 2] = make_double2(c0.x + c1.x, c0.y + c1.y);
        Y[4 * c + 3] = make_double2(d0.x + d1.x, d0.y + d1.y);
    }
}

__device__ __forceinline__ void matmul44(const double2 *A, const double2 *B, double2 *C)
{
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double2 t = cmul(A[4 * i + k], B[4 * k + j]);
                acc.x += t.x;
                acc.y += t.y;
            }
            C[4 * i + j] = acc;
        }
}

// tr[X Y]
__device__ __forceinline__ double2 trace_prod(const double2 *X, const double2 *Y)
{
    double2 t = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double2 u = cmul(X[4 * i + j], Y[4 * j + i]);
            t.x += u.x;
            t.y += u.y;
        }
    return t;
}

__device__ int interaction_terms(int interaction, const double *r, int p, InteractionTerm *t)
{
    t[0].identity = true;
    t[0].c = 1.0;
    for (int k = 0; k < 3; ++k) {
        t[1 + k].identity = false;
        t[1 + k].c = -0.5;
        t[1 + k].v[0] = k == 0;
        t[1 + k].v[1] = k == 1;
        t[1 + k].v[2] = k == 2;
    }
    if (interaction < 2) return 4;
    const double dx = r[6 * p] - r[6 * p + 3], dy = r[6 * p + 1] - r[6 * p + 4], dz = r[6 * p + 2] - r[6 * p + 5];
    const double inv = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
    t[4].identity = false;
    t[4].c = -0.5;
    t[4].v[0] = dx * inv;
    t[4].v[1] = dy * inv;
    t[4].v[2] = dz * inv;
    return 5;
}

// Real part of -1/2 (direct - exchange) with the Gaunt (interaction 1) or Breit (2)
// terms.  M1 = G-(1p,1q), M3 = G-(2p,2q), N11 = G+(1p,1q), N22 = G+(2p,2q),
// M2 = G+(1p,2q), M4 = G+(2p,1q); G-(y,x) = G-(x,y)^dagger.
__device__ __noinline__ double breit_value(int interaction, const double2 *M1, const double2 *M3, const double2 *N11,
                                           const double2 *N22, const double2 *M2, const double2 *M4, const double *r,
                                           int p, int q)
{
    InteractionTerm tp[5], tq[5];
    const int np = interaction_terms(interaction, r, p, tp);
    const int nq = interaction_terms(interaction, r, q, tq);
    double2 M1h[16], M3h[16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            M1h[4 * i + j] = make_double2(M1[4 * j + i].x, -M1[4 * j + i].y);
            M3h[4 * i + j] = make_double2(M3[4 * j + i].x, -M3[4 * j + i].y);
        }
    double2 direct = make_double2(0.0, 0.0), exchange = make_double2(0.0, 0.0);
    double2 QB[16], SB[16], PA[16], RA[16], U[16], W1[16], W2[16];
    for (int B = 0; B < nq; ++B) {
        rmul_op(N11, tq[B], QB);
        rmul_op(N22, tq[B], SB);
        for (int A = 0; A < np; ++A) {
            const double c = tp[A].c * tq[B].c;
            rmul_op(M1h, tp[A], PA);
            rmul_op(M3h, tp[A], RA);
            const double2 d = cmul(trace_prod(PA, QB), trace_prod(RA, SB));
            direct.x += c * d.x;
            direct.y += c * d.y;
            matmul44(PA, M2, U);
            rmul_op(U, tq[B], W1);
            matmul44(RA, M4, U);
            rmul_op(U, tq[B], W2);
            const double2 x = trace_prod(W1, W2);
            exchange.x += c * x.x;
            exchange.y += c * x.y;
        }
    }
    return -0.5 * (direct.x - exchange.x);
}

// One CTA per (tile, tau).  Rows of a tile side are (position, component)
// = NC x_local + c with x_local = 2 p_local + e.  Threads 0..127 own the
// same-electron position blocks (G- and G+), threads 128..255 the cross ones
// (G+ only, since the trace form uses G- only between like electrons).
// WITH_TERMS: the Gaunt / Breit terms (a separate instance keeps the Coulomb
// kernel's registers and stack untouched; four components only).
template <bool WITH_TERMS, int NC>
__global__ void __launch_bounds__(256, 1) pairs_f64_kernel(DevSystem s, const double2 *__restrict__ phi,
                                                           const double *__restrict__ scale,
                                                           const double *__restrict__ a,
                                                           double *__restrict__ partials, int n_tiles,
                                                           const double *__restrict__ r, DebugTile dbg)
{
    static_assert(NC == 4 || (NC == 2 && !WITH_TERMS), "Gaunt / Breit terms need the small components");
    constexpr int NN = NC * NC, ROWS = 16 * NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F64Smem<NC> &sm = *reinterpret_cast<F64Smem<NC> *>(smem_raw);
    const int tile = blockIdx.x, t = blockIdx.y;
    const int nb = pair_blocks(s.m, F64_TP);
    int bp, bq;
    tile_coords(tile, nb, bp, bq);
    const int tid = threadIdx.x;
    const int half = tid >> 7, e = (tid >> 6) & 1, i = tid & 63;
    const int xp = i >> 3, yp = i & 7;
    const int xl = 2 * xp + e, yl = 2 * yp + (half ? 1 - e : e);
    const double *sc = scale + (size_t)t * s.n_orb;
    const int row_base_p = ROWS * bp, row_base_q = ROWS * bq;
    const int rows_valid = 2 * NC * s.m;

    double2 acc[NN];
    for (int pass = 0; pass < 2; ++pass) {  // 0: occupied (G-), 1: virtual (G+)
        const int k_begin = pass == 0 ? 0 : s.n_occ;
        const int k_end = pass == 0 ? s.n_occ : s.n_orb;
        const bool active = (pass == 1) || (half == 0);
#pragma unroll
        for (int j = 0; j < NN; ++j) acc[j] = make_double2(0.0, 0.0);
        for (int k0 = k_begin; k0 < k_end; k0 += F64_KC) {
            for (int idx = tid; idx < F64_KC * ROWS; idx += 256) {
                const int row = idx >> 4, kk = idx & 15, k = k0 + kk;
                double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
                if (k < k_end) {
                    const double f = sc[k];
                    const int ra = row_base_p + row, rb = row_base_q + row;
                    if (ra < rows_valid) {
                        va = phi[(size_t)ra * s.n_orb + k];
                        va.x *= f;
                        va.y *= f;
                    }
                    if (rb < rows_valid) {
                        vb = phi[(size_t)rb * s.n_orb + k];
                        vb.x *= f;
                        vb.y *= f;
                    }
                }
                sm.u.ld.A[kk][row] = va;
                sm.u.ld.B[kk][row] = vb;
            }
            __syncthreads();
            if (active) {
#pragma unroll 4
                for (int kk = 0; kk < F64_KC; ++kk) {
                    double2 xa[NC], yb[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) xa[c] = sm.u.ld.A[kk][NC * xl + c];
#pragma unroll
                    for (int d = 0; d < NC; ++d) yb[d] = sm.u.ld.B[kk][NC * yl + d];
#pragma unroll
                    for (int c = 0; c < NC; ++c)
#pragma unroll
                        for (int d = 0; d < NC; ++d) {
                            // G(x, y)_cd += X(x)_c conj(X(y)_d)
                            double2 &g = acc[NC * c + d];
                            g.x = fma(xa[c].x, yb[d].x, g.x);
                            g.x = fma(xa[c].y, yb[d].y, g.x);
                            g.y = fma(xa[c].y, yb[d].x, g.y);
                            g.y = fma(-xa[c].x, yb[d].y, g.y);
                        }
                }
            }
            __syncthreads();
        }
        if (pass == 0 && half == 0) {
#pragma unroll
            for (int j = 0; j < NN; ++j) sm.Gm[e][xp][yp][j] = acc[j];
        }
    }
#pragma unroll
    for (int j = 0; j < NN; ++j) sm.u.Gp[xl][yl][j] = acc[j];
    __syncthreads();

    // Epilogue: one thread per pair of pairs (p, q) of the tile.
    if (tid < 64) {
        const int px = tid >> 3, qy = tid & 7;
        const int p = F64_TP * bp + px, q = F64_TP * bq + qy;
        double v = 0.0;
        if (p < s.m && q < s.m && (bp < bq || px < qy)) {
            const double2 *M1 = sm.Gm[0][px][qy];          // G-(1p, 1q)
            const double2 *M3 = sm.Gm[1][px][qy];          // G-(2p, 2q)
            const double2 *N11 = sm.u.Gp[2 * px][2 * qy];  // G+(1p, 1q)
            const double2 *N22 = sm.u.Gp[2 * px + 1][2 * qy + 1];  // G+(2p, 2q)
            const double2 *M2 = sm.u.Gp[2 * px][2 * qy + 1];  // G+(1p, 2q)
            const double2 *M4 = sm.u.Gp[2 * px + 1][2 * qy];  // G+(2p, 1q)
            // Direct: tr[G-(1q,1p) G+(1p,1q)] tr[G-(2q,2p) G+(2p,2q)], G-(y,x) = G-(x,y)^dagger.
            double2 t1 = make_double2(0, 0), t2 = make_double2(0, 0);
#pragma unroll
            for (int j = 0; j < NN; ++j) {
                const double2 u1 = cmulc(M1[j], N11[j]), u2 = cmulc(M3[j], N22[j]);
                t1.x += u1.x;
                t1.y += u1.y;
                t2.x += u2.x;
                t2.y += u2.y;
            }
            const double2 direct = cmul(t1, t2);
            // Exchange: tr[G-(1q,1p) G+(1p,2q) G-(2q,2p) G+(2p,1q)] = tr[(M1^dag M2)(M3^dag M4)]
            // = sum_ij (M1^dag M2)_ij (M3^dag M4)_ji.
            double2 ex = make_double2(0, 0);
#pragma unroll
            for (int i2 = 0; i2 < NC; ++i2)
#pragma unroll
                for (int j2 = 0; j2 < NC; ++j2) {
                    double2 s1 = make_double2(0, 0), s2 = make_double2(0, 0);
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
                        const double2 w1 = cmulc(M1[NC * k + i2], M2[NC * k + j2]);
                        const double2 w2 = cmulc(M3[NC * k + j2], M4[NC * k + i2]);
                        s1.x += w1.x;
                        s1.y += w1.y;
                        s2.x += w2.x;
                        s2.y += w2.y;
                    }
                    const double2 w = cmul(s1, s2);
                    ex.x += w.x;
                    ex.y += w.y;
                }
            double F = -0.5 * (direct.x - ex.x);  // real part of -1/2 (direct - exchange)
            if constexpr (WITH_TERMS) F = breit_value(s.interaction, M1, M3, N11, N22, M2, M4, r, p, q);
            v = F * a[p] * a[q] / s.lambda;
        }
        if (dbg.out && bp == dbg.bp && bq == dbg.bq) dbg.out[((size_t)t * F64_TP + px) * F64_TP + qy] = v;
        sm.part[tid] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int j = 0; j < 64; ++j) sum += sm.part[j];
        partials[(size_t)t * n_tiles + tile] = sum;
    }
}

// The shared-memory opt-in is a property of each device's context: remembered per device.
constexpr int F64_MAX_DEVICES = 64;
static bool g_f64_configured[F64_MAX_DEVICES] = {};

static int current_device()
{
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < F64_MAX_DEVICES ? dev : -1;
}

cudaError_t prepare_f64()
{
    const int dev = current_device();
    if (dev < 0) return cudaErrorInvalidDevice;
    cudaError_t e = cudaFuncSetAttribute(pairs_f64_kernel<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(F64Smem<4>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pairs_f64_kernel<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(F64Smem<4>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pairs_f64_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(F64Smem<2>));
    if (e == cudaSuccess) g_f64_configured[dev] = true;
    return e;
}

cudaError_t launch_pairs_f64(const DevSystem &s, const double *phi, const double *scale, const double *a,
                             double *partials, cudaStream_t st, const double *r, const DebugTile &dbg)
{
    if (s.interaction >= 2 && !r) return cudaErrorInvalidValue;
    if (s.n_comp == 2 && s.interaction > 0) return cudaErrorInvalidValue;
    const int dev = current_device();
    if (dev < 0 || !g_f64_configured[dev]) {
        const cudaError_t e = prepare_f64();
        if (e != cudaSuccess) return e;
    }
    const int n_tiles = (int)n_tiles_for(s.m, F64_TP);
    dim3 grid(n_tiles, s.n_tau);
    const double2 *ph = reinterpret_cast<const double2 *>(phi);
    if (s.n_comp == 2)
        pairs_f64_kernel<false, 2><<<grid, 256, sizeof(F64Smem<2>), st>>>(s, ph, scale, a, partials, n_tiles, r, dbg);
    else if (s.interaction > 0)
        pairs_f64_kernel<true, 4><<<grid, 256, sizeof(F64Smem<4>), st>>>(s, ph, scale, a, partials, n_tiles, r, dbg);
    else
        pairs_f64_kernel<false, 4><<<grid, 256, sizeof(F64Smem<4>), st>>>(s, ph, scale, a, partials, n_tiles, r, dbg);
    return cudaGetLastError();
}

}  // namespace mcmp2
