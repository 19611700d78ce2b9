// Adjoint of the FP64 integrand engine: gradient of the replay estimate
// E = (1/n) sum_n I'_n with respect to the orbital energies and the spinor
// coefficients, for fixed samples (common random numbers), with lambda,
// eps_HOMO and eps_LUMO held fixed (the sampling density of tau does not move).
//
// For one pair of pairs, with M1 = G-(1p,1q), M3 = G-(2p,2q), N11 = G+(1p,1q),
// N22 = G+(2p,2q), M2 = G+(1p,2q), M4 = G+(2p,1q), T1 = <M1, N11>,
// T2 = <M3, N22> (Frobenius, first argument conjugated) and
// X = tr[M1^dag M2 M3^dag M4], the real part of F = -1/2 (T1 T2 - X) varies as
// Re dF = Re sum_Z sum_cd W(Z)_cd dZ_cd with
//   W(M1)  = -1/2 conj(T2 N11) + 1/2 conj(M2 M3^dag M4)
//   W(N11) = -1/2 T2 conj(M1)
//   W(M3)  = -1/2 conj(T1 N22) + 1/2 conj(M4 M1^dag M2)
//   W(N22) = -1/2 T1 conj(M3)
//   W(M2)  = 1/2 (M3^dag M4 M1^dag)^T
//   W(M4)  = 1/2 (M1^dag M2 M3^dag)^T.
// Through G(x,y) = X(x) X(y)^dag the scaled spinor values X = phi s receive
//   Ybar(x) += conj(W) X(y),  Ybar(y) += W^T X(x),   dE = Re sum conj(Ybar) dX,
// then dE/d eps_k = (+-tau/2) Re sum conj(Ybar_k) X_k (s_k = exp(+-(eps_k - eps_ref) tau/2))
// and dE/dW^c_jk = sum_x B(x, j) s_k Ybar_ck(x) for the spinor-formation operands.
#include "internal.cuh"

namespace mcmp2 {

namespace {

constexpr int TP = 8;   // pairs per tile side
constexpr int KC = 16;  // orbitals per staged chunk

struct AdjSmem {
    double2 Wm[2][TP][TP][16];  // G- then W for like-electron blocks, [e][xp][yp][c*4+d]
    double2 Wp[16][16][16];     // G+ then W for all position blocks, [xl][yl][c*4+d]
    double2 A[KC][64];          // X of the p-side rows for the current chunk
    double2 B[KC][64];          // X of the q-side rows
    double part[64];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 scale2(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// P = A^dag B for 4x4 row-major blocks.
__device__ __forceinline__ void mm_hn(const double2 *A, const double2 *B, double2 *P)
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double2 s = make_double2(0, 0);
            for (int k = 0; k < 4; ++k) s = add2(s, cmulc(A[4 * k + i], B[4 * k + j]));
            P[4 * i + j] = s;
        }
}

// P = A B^dag.
__device__ __forceinline__ void mm_nh(const double2 *A, const double2 *B, double2 *P)
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double2 s = make_double2(0, 0);
            for (int k = 0; k < 4; ++k) s = add2(s, cmul(A[4 * i + k], conj2(B[4 * j + k])));
            P[4 * i + j] = s;
        }
}

// P = A B.
__device__ __forceinline__ void mm_nn(const double2 *A, const double2 *B, double2 *P)
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double2 s = make_double2(0, 0);
            for (int k = 0; k < 4; ++k) s = add2(s, cmul(A[4 * i + k], B[4 * k + j]));
            P[4 * i + j] = s;
        }
}

__device__ __forceinline__ void tile_of(int tile, int nb, int &bp, int &bq)
{
    int k = tile, b = 0;
    while (k >= nb - b) {
        k -= nb - b;
        ++b;
    }
    bp = b;
    bq = b + k;
}

// One CTA per tile for imaginary time t_index.  norm = 1 / (n_steps n_tau mC2).
__global__ void __launch_bounds__(256, 1) adjoint_tiles_kernel(DevSystem s, const double2 *__restrict__ phi,
                                                               const double *__restrict__ scale,
                                                               const double *__restrict__ a, int t_index,
                                                               double norm, double2 *__restrict__ Ybar,
                                                               double *__restrict__ partials, int n_tiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AdjSmem &sm = *reinterpret_cast<AdjSmem *>(smem_raw);
    const int tile = blockIdx.x;
    const int nb = pair_blocks(s.m, TP);
    int bp, bq;
    tile_of(tile, nb, bp, bq);
    const int tid = threadIdx.x;
    const double *sc = scale + (size_t)t_index * s.n_orb;
    const int row_p0 = 64 * bp, row_q0 = 64 * bq, rows_valid = 8 * s.m;

    auto load_chunk = [&](int k0, int k_end) {
        for (int idx = tid; idx < KC * 64; idx += 256) {
            const int row = idx >> 4, kk = idx & 15, k = k0 + kk;
            double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
            if (k < k_end) {
                const double f = sc[k];
                if (row_p0 + row < rows_valid) va = scale2(phi[(size_t)(row_p0 + row) * s.n_orb + k], f);
                if (row_q0 + row < rows_valid) vb = scale2(phi[(size_t)(row_q0 + row) * s.n_orb + k], f);
            }
            sm.A[kk][row] = va;
            sm.B[kk][row] = vb;
        }
    };

    // ---- forward: propagator blocks (same ownership as the FP64 forward kernel) ----
    {
        const int half = tid >> 7, e = (tid >> 6) & 1, i = tid & 63;
        const int xp = i >> 3, yp = i & 7;
        const int xl = 2 * xp + e, yl = 2 * yp + (half ? 1 - e : e);
        double2 acc[16];
        for (int pass = 0; pass < 2; ++pass) {
            const int k_begin = pass == 0 ? 0 : s.n_occ, k_end = pass == 0 ? s.n_occ : s.n_orb;
            const bool active = (pass == 1) || (half == 0);
            for (int j = 0; j < 16; ++j) acc[j] = make_double2(0.0, 0.0);
            for (int k0 = k_begin; k0 < k_end; k0 += KC) {
                load_chunk(k0, k_end);
                __syncthreads();
                if (active)
                    for (int kk = 0; kk < KC; ++kk) {
                        double2 xa[4], yb[4];
                        for (int c = 0; c < 4; ++c) xa[c] = sm.A[kk][4 * xl + c];
                        for (int d = 0; d < 4; ++d) yb[d] = sm.B[kk][4 * yl + d];
                        for (int c = 0; c < 4; ++c)
                            for (int d = 0; d < 4; ++d) acc[4 * c + d] = add2(acc[4 * c + d], cmul(xa[c], conj2(yb[d])));
                    }
                __syncthreads();
            }
            if (pass == 0 && half == 0)
                for (int j = 0; j < 16; ++j) sm.Wm[e][xp][yp][j] = acc[j];
        }
        for (int j = 0; j < 16; ++j) sm.Wp[xl][yl][j] = acc[j];
    }
    __syncthreads();

    // ---- per pair of pairs: forward value and the W blocks, four threads per pair of pairs ----
    {
        const int role = tid >> 6, pq = tid & 63;
        const int px = pq >> 3, qy = pq & 7;
        const int p = TP * bp + px, q = TP * bq + qy;
        double2 *M1 = sm.Wm[0][px][qy], *M3 = sm.Wm[1][px][qy];
        double2 *N11 = sm.Wp[2 * px][2 * qy], *N22 = sm.Wp[2 * px + 1][2 * qy + 1];
        double2 *M2 = sm.Wp[2 * px][2 * qy + 1], *M4 = sm.Wp[2 * px + 1][2 * qy];
        const bool valid = p < s.m && q < s.m && (bp < bq || px < qy);
        double2 Wa[16], Wb[16];
        double v = 0.0;
        if (valid) {
            const double w = a[p] * a[q] / s.lambda;
            const double g = w * norm;  // weight of this pair of pairs in E
            double2 T1 = make_double2(0, 0), T2 = make_double2(0, 0);
            for (int j = 0; j < 16; ++j) {
                T1 = add2(T1, cmulc(M1[j], N11[j]));
                T2 = add2(T2, cmulc(M3[j], N22[j]));
            }
            double2 R[16];
            if (role == 0) {
                // forward value; W(M1) = -1/2 conj(T2 N11) + 1/2 conj(M2 M3^dag M4); W(N11) = -1/2 T2 conj(M1)
                double2 P[16], Q[16];
                mm_hn(M1, M2, P);
                mm_hn(M3, M4, Q);
                double2 X = make_double2(0, 0);
                for (int i2 = 0; i2 < 4; ++i2)
                    for (int j2 = 0; j2 < 4; ++j2) X = add2(X, cmul(P[4 * i2 + j2], Q[4 * j2 + i2]));
                v = -0.5 * (cmul(T1, T2).x - X.x) * w;
                mm_nh(M2, M3, R);
                mm_nn(R, M4, P);
                for (int j = 0; j < 16; ++j) {
                    Wa[j] = scale2(add2(scale2(conj2(cmul(T2, N11[j])), -0.5), scale2(conj2(P[j]), 0.5)), g);
                    Wb[j] = scale2(cmul(T2, conj2(M1[j])), -0.5 * g);
                }
            } else if (role == 1) {
                // W(M3) = -1/2 conj(T1 N22) + 1/2 conj(M4 M1^dag M2); W(N22) = -1/2 T1 conj(M3)
                double2 P[16];
                mm_nh(M4, M1, R);
                mm_nn(R, M2, P);
                for (int j = 0; j < 16; ++j) {
                    Wa[j] = scale2(add2(scale2(conj2(cmul(T1, N22[j])), -0.5), scale2(conj2(P[j]), 0.5)), g);
                    Wb[j] = scale2(cmul(T1, conj2(M3[j])), -0.5 * g);
                }
            } else if (role == 2) {
                // W(M2) = 1/2 (M3^dag M4 M1^dag)^T
                double2 Q[16];
                mm_hn(M3, M4, Q);
                mm_nh(Q, M1, R);
                for (int i2 = 0; i2 < 4; ++i2)
                    for (int j2 = 0; j2 < 4; ++j2) Wa[4 * i2 + j2] = scale2(R[4 * j2 + i2], 0.5 * g);
            } else {
                // W(M4) = 1/2 (M1^dag M2 M3^dag)^T
                double2 P[16];
                mm_hn(M1, M2, P);
                mm_nh(P, M3, R);
                for (int i2 = 0; i2 < 4; ++i2)
                    for (int j2 = 0; j2 < 4; ++j2) Wa[4 * i2 + j2] = scale2(R[4 * j2 + i2], 0.5 * g);
            }
        } else {
            for (int j = 0; j < 16; ++j) Wa[j] = Wb[j] = make_double2(0.0, 0.0);
        }
        if (role == 0) sm.part[pq] = v;
        __syncthreads();  // every original block has been read
        double2 *dstA = role == 0 ? M1 : role == 1 ? M3 : role == 2 ? M2 : M4;
        for (int j = 0; j < 16; ++j) dstA[j] = Wa[j];
        if (role < 2) {
            double2 *dstB = role == 0 ? N11 : N22;
            for (int j = 0; j < 16; ++j) dstB[j] = Wb[j];
        }
    }
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int j = 0; j < 64; ++j) sum += sm.part[j];
        partials[(size_t)t_index * n_tiles + tile] = sum;
    }

    // ---- adjoint contraction: Ybar_p(x) += conj(W(x, .)) X_q,  Ybar_q(y) += W(., y)^T X_p ----
    const bool pside = tid < 128;
    const int r = (tid & 127) >> 1;      // row of this side: 4 x_local + c
    const int kk0 = (tid & 1) * 8;       // 8 orbitals of the chunk
    const int xl = r >> 2, cc = r & 3;
    for (int pass = 0; pass < 2; ++pass) {
        const int k_begin = pass == 0 ? 0 : s.n_occ, k_end = pass == 0 ? s.n_occ : s.n_orb;
        for (int k0 = k_begin; k0 < k_end; k0 += KC) {
            load_chunk(k0, k_end);
            __syncthreads();
            double2 out[8];
            for (int j = 0; j < 8; ++j) out[j] = make_double2(0.0, 0.0);
            for (int o = 0; o < 16; ++o) {      // positions of the other side
                for (int d = 0; d < 4; ++d) {   // components of the other side
                    double2 w;
                    if (pass == 0) {
                        const bool like = (xl & 1) == (o & 1);
                        if (!like) continue;
                        w = pside ? sm.Wm[xl & 1][xl >> 1][o >> 1][4 * cc + d] : sm.Wm[xl & 1][o >> 1][xl >> 1][4 * d + cc];
                    } else {
                        w = pside ? sm.Wp[xl][o][4 * cc + d] : sm.Wp[o][xl][4 * d + cc];
                    }
                    if (pside) w = conj2(w);
                    for (int j = 0; j < 8; ++j) {
                        const double2 xv = pside ? sm.B[kk0 + j][4 * o + d] : sm.A[kk0 + j][4 * o + d];
                        out[j] = add2(out[j], cmul(w, xv));
                    }
                }
            }
            const int grow = (pside ? row_p0 : row_q0) + r;
            if (grow < rows_valid)
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + kk0 + j;
                    if (k < k_end) {
                        double *dst = reinterpret_cast<double *>(Ybar + (size_t)grow * s.n_orb + k);
                        atomicAdd(dst, out[j].x);
                        atomicAdd(dst + 1, out[j].y);
                    }
                }
            __syncthreads();
        }
    }
}

// d eps_k += (+-tau/2) Re sum_rows conj(Ybar_k) X_k; one block per orbital.
__global__ void adjoint_eps_kernel(DevSystem s, const double2 *__restrict__ phi, const double *__restrict__ scale,
                                   const double *__restrict__ tau, int t_index, const double2 *__restrict__ Ybar,
                                   double *__restrict__ d_eps)
{
    const int k = blockIdx.x;
    const int rows = 8 * s.m;
    const double f = scale[(size_t)t_index * s.n_orb + k];
    double acc = 0.0;
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
        const double2 x = phi[(size_t)row * s.n_orb + k];
        const double2 y = Ybar[(size_t)row * s.n_orb + k];
        acc += (y.x * x.x + y.y * x.y) * f;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sgn = k < s.n_occ ? 0.5 : -0.5;
        d_eps[k] += sgn * tau[t_index] * red[0];
    }
}

// Ys[x][c][k] = Ybar[4x + c][k] s_k (the coefficient adjoint before contraction with B).
__global__ void adjoint_scale_kernel(DevSystem s, const double2 *__restrict__ Ybar, const double *__restrict__ scale,
                                     int t_index, double2 *__restrict__ Ys)
{
    const size_t n = (size_t)8 * s.m * s.n_orb;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % s.n_orb);
        Ys[i] = scale2(Ybar[i], scale[(size_t)t_index * s.n_orb + k]);
    }
}

// C[M x N] += A^T B with A stored [K][lda] (columns m), B [K][ldb]: 64 x 64 tiles.
__global__ void __launch_bounds__(256) gemm_tn_acc_kernel(int M, int N, int K, const double *__restrict__ A, int lda,
                                                          const double *__restrict__ Bm, int ldb,
                                                          double *__restrict__ C, int ldc)
{
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = i >> 6, cc = i & 63;
            const int gk = k0 + kk;
            As[kk][cc] = (gk < K && row0 + cc < M) ? A[(size_t)gk * lda + row0 + cc] : 0.0;
            Bs[kk][cc] = (gk < K && col0 + cc < N) ? Bm[(size_t)gk * ldb + col0 + cc] : 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk < 16; ++kk) {
            double av[4], bv[4];
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const int gr = row0 + ty + 16 * i, gc = col0 + tx + 16 * j;
            if (gr < M && gc < N) C[(size_t)gr * ldc + gc] += acc[i][j];
        }
}

}  // namespace

size_t adjoint_smem_bytes() { return sizeof(AdjSmem); }

// One imaginary time of the adjoint for one step.  Ybar must be zero on entry;
// GWL [n_l][4 n_orb], GWS [3 n_l][4 n_orb] and d_eps [n_orb] accumulate.
cudaError_t launch_adjoint_time(const DevSystem &s, const double *B, const double *phi, const double *scale,
                                const double *tau, const double *a, int t_index, double norm, double *Ybar,
                                double *Ys, double *partials, double *GWL, double *GWS, double *d_eps,
                                cudaStream_t st)
{
    // The shared-memory opt-in belongs to the current device's context: set on every call (cheap).
    const size_t smem = sizeof(AdjSmem);
    {
        const cudaError_t e =
            cudaFuncSetAttribute(adjoint_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int n_tiles = (int)n_tiles_for(s.m, TP);
    adjoint_tiles_kernel<<<n_tiles, 256, smem, st>>>(s, reinterpret_cast<const double2 *>(phi), scale, a, t_index,
                                                     norm, reinterpret_cast<double2 *>(Ybar), partials, n_tiles);
    adjoint_eps_kernel<<<s.n_orb, 256, 0, st>>>(s, reinterpret_cast<const double2 *>(phi), scale, tau, t_index,
                                                reinterpret_cast<const double2 *>(Ybar), d_eps);
    adjoint_scale_kernel<<<1024, 256, 0, st>>>(s, reinterpret_cast<const double2 *>(Ybar), scale, t_index,
                                               reinterpret_cast<double2 *>(Ys));
    // Ys viewed as [P][8 n_orb] doubles: columns (c, k, re/im); L components first.
    const int P = 2 * s.m, n4 = 4 * s.n_orb, ldy = 8 * s.n_orb;
    dim3 gl((n4 + 63) / 64, (s.n_l + 63) / 64), gs((n4 + 63) / 64, (3 * s.n_l + 63) / 64);
    gemm_tn_acc_kernel<<<gl, 256, 0, st>>>(s.n_l, n4, P, B, 4 * s.n_l, Ys, ldy, GWL, n4);
    gemm_tn_acc_kernel<<<gs, 256, 0, st>>>(3 * s.n_l, n4, P, B + s.n_l, 4 * s.n_l, Ys + n4, ldy, GWS, n4);
    return cudaGetLastError();
}

}  // namespace mcmp2
