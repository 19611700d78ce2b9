/*
 * mcmp2_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle), not the product.
 *
 * A plain, slow, FP64 CPU restatement of the Monte Carlo four-component
 * relativistic MP2 method of Cruz, Garza, Yanai and Hirata (J. Chem. Phys.
 * 2022, arXiv 2203.05632), Sec. III.  Only the test suite, the package's
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header or table with the CUDA library; every function below
 * follows the paper's equations in their order and notation, with the
 * readings listed where the text is silent or garbled.
 *
 * Readings of the paper used here:
 *  - Eq. C with its kinetic-balance condition: n_L real Cartesian Gaussians g_mu.
 *    The large 2-spinor basis is {g_mu e_alpha, g_mu e_beta}; the small one
 *    is {i(sigma.p)(g_mu e_s)} = {(sigma.grad)(g_mu e_s)} (restricted kinetic
 *    balance, p = -i grad).  C has 4 n_L rows: L-alpha, L-beta, S-alpha,
 *    S-beta coefficient blocks.
 *  - Eq. MCMP2 is read in its trace form, derived from Eq. FinalMP2 with the
 *    Laplace transform of 1/D:
 *       E2 = -1/2 Int (1/r12 r34) { tr[G-(3,1)G+(1,3)] tr[G-(4,2)G+(2,4)]
 *                                   - tr[G-(3,1)G+(1,4)G-(4,2)G+(2,3)] },
 *    which reduces to the printed -2/+1 scalar form for closed-shell
 *    nonrelativistic spin orbitals.
 *  - The per-sample estimate keeps the real part (the imaginary part of
 *    f(p,q) + f(q,p) cancels).
 *  - N_zeta = (2 zeta/pi)^{3/4} in Eq. basisSet.
 *  - n_tau imaginary times per step share the walkers; their estimates are
 *    averaged.
 *  - Blocking (Eq. uncertainty): incomplete trailing block excluded, I_N is
 *    the mean of the complete block means.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
 * from its published definition, with the counter layout described at
 * or_philox4x32_10.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int n_centres;
    const double *centres;    /* [n_centres][3] bohr */
    const double *weight;     /* [n_centres][4]: c1, zeta1, c2, zeta2 (Table 1) */
    int n_shells;
    const int *shell_centre;
    const int *shell_l;       /* 0, 1, 2 */
    const double *shell_alpha;
    const double *shell_coef;
    int n_occ, n_vir;
    const double *C;          /* complex interleaved, [4 n_L][n_orb] row-major */
    const double *eps;        /* [n_orb], occupied first */
    int interaction;          /* 0: Coulomb 1/r12; 1: + Gaunt; 2: + Gaunt + gauge (full Breit) */
} or_system;

/* ---------------------------------------------------------------------- */
/* Basis functions (Eq. C and its kinetic-balance condition)               */
/* ---------------------------------------------------------------------- */

static const int CART[3][6][3] = {
    {{0, 0, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}},
};
static const int NCART[3] = {1, 3, 6};

int or_n_functions(const or_system *s)
{
    int n = 0;
    for (int k = 0; k < s->n_shells; ++k) n += NCART[s->shell_l[k]];
    return n;
}

static double ipow(double x, int k)
{
    double v = 1.0;
    for (int i = 0; i < k; ++i) v *= x;
    return v;
}

/* g_mu(r) = coef (x-Ax)^a (y-Ay)^b (z-Az)^c exp(-alpha |r-A|^2) and its gradient. */
void or_basis_at(const or_system *s, const double *r, double *val, double *grad)
{
    int mu = 0;
    for (int k = 0; k < s->n_shells; ++k) {
        const double *A = s->centres + 3 * s->shell_centre[k];
        const double d[3] = {r[0] - A[0], r[1] - A[1], r[2] - A[2]};
        const double al = s->shell_alpha[k];
        const double e = s->shell_coef[k] * exp(-al * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
        const int l = s->shell_l[k];
        for (int c = 0; c < NCART[l]; ++c, ++mu) {
            const int *pw = CART[l][c];
            double poly = ipow(d[0], pw[0]) * ipow(d[1], pw[1]) * ipow(d[2], pw[2]);
            val[mu] = poly * e;
            for (int j = 0; j < 3; ++j) {
                /* d/dx_j [x_j^a exp(-al x_j^2)] = (a x_j^{a-1} - 2 al x_j^{a+1}) exp(...) */
                double other = 1.0;
                for (int i = 0; i < 3; ++i)
                    if (i != j) other *= ipow(d[i], pw[i]);
                double dj = -2.0 * al * ipow(d[j], pw[j] + 1);
                if (pw[j] > 0) dj += pw[j] * ipow(d[j], pw[j] - 1);
                grad[3 * mu + j] = other * dj * e;
            }
        }
    }
}

/* Four-component spinor values phi_k^c(r), c = L-alpha, L-beta, S-alpha, S-beta.
 * Large components by Eq. C; small components by applying sigma.grad to the
 * 2-spinor g_mu e_s (kinetic balance with i(sigma.p) = sigma.grad).
 * phi: complex interleaved [n_orb][4]. */
void or_spinors_at(const or_system *s, const double *r, double *phi_out)
{
    const int nL = or_n_functions(s);
    const int n = s->n_occ + s->n_vir;
    double *val = malloc(sizeof(double) * nL);
    double *grad = malloc(sizeof(double) * 3 * nL);
    or_basis_at(s, r, val, grad);
    const cplx *C = (const cplx *)s->C;
    /* Pauli matrices sigma_x, sigma_y, sigma_z. */
    const cplx sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    cplx *phi = (cplx *)phi_out;
    for (int k = 0; k < n; ++k) {
        cplx la = 0, lb = 0, sa = 0, sb = 0;
        for (int mu = 0; mu < nL; ++mu) {
            const cplx cLa = C[(size_t)(0 * nL + mu) * n + k];
            const cplx cLb = C[(size_t)(1 * nL + mu) * n + k];
            const cplx cSa = C[(size_t)(2 * nL + mu) * n + k];
            const cplx cSb = C[(size_t)(3 * nL + mu) * n + k];
            la += cLa * val[mu];
            lb += cLb * val[mu];
            /* (sigma.grad)(g e_s) = sum_j sigma_j e_s d_j g; e_alpha = (1,0), e_beta = (0,1). */
            for (int j = 0; j < 3; ++j) {
                const double dg = grad[3 * mu + j];
                sa += (cSa * sig[j][0][0] + cSb * sig[j][0][1]) * dg;
                sb += (cSa * sig[j][1][0] + cSb * sig[j][1][1]) * dg;
            }
        }
        phi[4 * k + 0] = la;
        phi[4 * k + 1] = lb;
        phi[4 * k + 2] = sa;
        phi[4 * k + 3] = sb;
    }
    free(val);
    free(grad);
}

/* ---------------------------------------------------------------------- */
/* Weight functions (Eq. basisSet, N_g, Eq. tauWeight)                     */
/* ---------------------------------------------------------------------- */

static double n_zeta(double zeta) { return pow(2.0 * zeta / M_PI, 0.75); }

/* g(r) = sum_I sum_{k=1,2} c_k(I) N_zeta exp(-zeta_k(I) |r - R_I|^2). */
double or_g(const or_system *s, const double *r)
{
    double g = 0.0;
    for (int ic = 0; ic < s->n_centres; ++ic) {
        const double *R = s->centres + 3 * ic;
        const double d2 = (r[0] - R[0]) * (r[0] - R[0]) + (r[1] - R[1]) * (r[1] - R[1]) +
                          (r[2] - R[2]) * (r[2] - R[2]);
        const double *w = s->weight + 4 * ic;
        g += w[0] * n_zeta(w[1]) * exp(-w[1] * d2) + w[2] * n_zeta(w[3]) * exp(-w[3] * d2);
    }
    return g;
}

/* N_g = Int Int g(r1) g(r2) / r12, analytically: for unnormalised s Gaussians
 * exp(-a|r-A|^2), exp(-b|r-B|^2) the Coulomb integral is
 * (pi/a)^{3/2} (pi/b)^{3/2} erf(sqrt(ab/(a+b)) R) / R, with the R -> 0 limit
 * 2 sqrt(ab/(pi(a+b))) (pi/a)^{3/2} (pi/b)^{3/2}. */
double or_Ng(const or_system *s)
{
    double total = 0.0;
    for (int ic = 0; ic < s->n_centres; ++ic)
        for (int jc = 0; jc < s->n_centres; ++jc) {
            const double *A = s->centres + 3 * ic, *B = s->centres + 3 * jc;
            const double R = sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) +
                                  (A[2] - B[2]) * (A[2] - B[2]));
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) {
                    const double ca = s->weight[4 * ic + 2 * k], a = s->weight[4 * ic + 2 * k + 1];
                    const double cb = s->weight[4 * jc + 2 * l], b = s->weight[4 * jc + 2 * l + 1];
                    const double rho = a * b / (a + b);
                    const double vol = pow(M_PI / a, 1.5) * pow(M_PI / b, 1.5);
                    const double coul = (R > 0.0) ? erf(sqrt(rho) * R) / R : 2.0 * sqrt(rho / M_PI);
                    total += ca * n_zeta(a) * cb * n_zeta(b) * vol * coul;
                }
        }
    return total;
}

/* lambda = 2 (eps_LUMO - eps_HOMO). */
double or_lambda(const or_system *s)
{
    double homo = -INFINITY, lumo = INFINITY;
    for (int i = 0; i < s->n_occ; ++i) homo = fmax(homo, s->eps[i]);
    for (int a = 0; a < s->n_vir; ++a) lumo = fmin(lumo, s->eps[s->n_occ + a]);
    return 2.0 * (lumo - homo);
}

/* ---------------------------------------------------------------------- */
/* Green's function traces and the MC-MP2 integrand (Sec. III)             */
/* ---------------------------------------------------------------------- */

/* kind = -1: G-(r_d, r_o, -tau) = sum_i phi_i(r_d) phi_i^dag(r_o) exp(+eps_i tau)
 * kind = +1: G+(r_d, r_o,  tau) = sum_a phi_a(r_d) phi_a^dag(r_o) exp(-eps_a tau)
 * phi_d, phi_o: spinor values at the two points, [n_orb][4] complex. */
static void green(const or_system *s, const cplx *phi_d, const cplx *phi_o, double tau, int kind,
                  cplx G[4][4])
{
    const int k0 = (kind < 0) ? 0 : s->n_occ;
    const int k1 = (kind < 0) ? s->n_occ : s->n_occ + s->n_vir;
    for (int c = 0; c < 4; ++c)
        for (int d = 0; d < 4; ++d) G[c][d] = 0;
    for (int k = k0; k < k1; ++k) {
        const double w = exp(-(double)kind * s->eps[k] * tau);
        for (int c = 0; c < 4; ++c)
            for (int d = 0; d < 4; ++d) G[c][d] += phi_d[4 * k + c] * conj(phi_o[4 * k + d]) * w;
    }
}

void or_green(const or_system *s, const double *phi_d, const double *phi_o, double tau, int kind,
              double *G_out)
{
    cplx G[4][4];
    green(s, (const cplx *)phi_d, (const cplx *)phi_o, tau, kind, G);
    memcpy(G_out, G, sizeof(G));
}

static void matmul4(cplx A[4][4], cplx B[4][4], cplx out[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx v = 0;
            for (int k = 0; k < 4; ++k) v += A[i][k] * B[k][j];
            out[i][j] = v;
        }
}

static cplx trace4(cplx A[4][4]) { return A[0][0] + A[1][1] + A[2][2] + A[3][3]; }

/* The interaction between electrons a and b (Sec. II, operator g_ij):
 *   g(a,b) = 1/r_ab - alpha(a).alpha(b) / (2 r_ab) - (alpha(a).r_ab)(alpha(b).r_ab) / (2 r_ab^3)
 *          = (1/r_ab) sum_A c_A O_A(a) O_A(b),
 * with O_0 = 1 (c = 1), O_k = alpha_k (k = x, y, z; c = -1/2) for the Gaunt term and
 * O_n = alpha.n, n = r_ab / r_ab (c = -1/2) for the gauge term.  alpha_k has sigma_k in its
 * off-diagonal 2x2 blocks (components L-alpha, L-beta, S-alpha, S-beta).  Returns the count. */
static int interaction_terms(const or_system *s, const double *ra, const double *rb, cplx O[5][4][4],
                             double c[5])
{
    static const cplx sig[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    memset(O, 0, sizeof(cplx) * 5 * 16);
    for (int d = 0; d < 4; ++d) O[0][d][d] = 1;
    c[0] = 1.0;
    if (s->interaction <= 0) return 1;
    double n[3] = {ra[0] - rb[0], ra[1] - rb[1], ra[2] - rb[2]};
    const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int k = 0; k < 3; ++k) n[k] /= len;
    const int count = s->interaction >= 2 ? 5 : 4;
    for (int A = 1; A < count; ++A) {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v) {
                cplx val = 0;
                if (A <= 3)
                    val = sig[A - 1][u][v];
                else
                    for (int k = 0; k < 3; ++k) val += n[k] * sig[k][u][v];
                O[A][u][2 + v] = val;  /* L rows, S columns */
                O[A][2 + u][v] = val;  /* S rows, L columns */
            }
        c[A] = -0.5;
    }
    return count;
}

static cplx trace_of_product(int n_mat, cplx (*const *mats)[4])
{
    cplx acc[4][4], tmp[4][4];
    memcpy(acc, mats[0], sizeof(acc));
    for (int k = 1; k < n_mat; ++k) {
        matmul4(acc, (cplx(*)[4])mats[k], tmp);
        memcpy(acc, tmp, sizeof(acc));
    }
    return trace4(acc);
}

/* f(r1,r2,r3,r4,tau) * r12 * r34 at one sample, the two integrands of the
 * trace-form Eq. MCMP2:  -1/2 { tr[G-31 G+13] tr[G-42 G+24] - tr[G-31 G+14 G-42 G+23] }.
 * With the Gaunt / Breit terms each point x carries the operator of its electron
 * pair's interaction term where the two propagators meet at x: for terms A of
 * g(1,2) and B of g(3,4),
 *   direct   tr[G-31 O_A G+13 O_B] tr[G-42 O_A G+24 O_B],
 *   exchange tr[G-31 O_A G+14 O_B G-42 O_A G+23 O_B],
 * summed with c_A c_B. */
static cplx integrand(const or_system *s, const cplx *p1, const cplx *p2, const cplx *p3,
                      const cplx *p4, double tau, const double *r1, const double *r2, const double *r3,
                      const double *r4)
{
    if (s->interaction > 0) {
        cplx Gm31[4][4], Gp13[4][4], Gm42[4][4], Gp24[4][4], Gp14[4][4], Gp23[4][4];
        green(s, p3, p1, tau, -1, Gm31);
        green(s, p1, p3, tau, +1, Gp13);
        green(s, p4, p2, tau, -1, Gm42);
        green(s, p2, p4, tau, +1, Gp24);
        green(s, p1, p4, tau, +1, Gp14);
        green(s, p2, p3, tau, +1, Gp23);
        cplx OA[5][4][4], OB[5][4][4];
        double cA[5], cB[5];
        const int nA = interaction_terms(s, r1, r2, OA, cA);
        const int nB = interaction_terms(s, r3, r4, OB, cB);
        cplx direct = 0, exchange = 0;
        for (int A = 0; A < nA; ++A)
            for (int B = 0; B < nB; ++B) {
                cplx (*const d1[4])[4] = {Gm31, OA[A], Gp13, OB[B]};
                cplx (*const d2[4])[4] = {Gm42, OA[A], Gp24, OB[B]};
                cplx (*const x[8])[4] = {Gm31, OA[A], Gp14, OB[B], Gm42, OA[A], Gp23, OB[B]};
                direct += cA[A] * cB[B] * trace_of_product(4, d1) * trace_of_product(4, d2);
                exchange += cA[A] * cB[B] * trace_of_product(8, x);
            }
        return -0.5 * (direct - exchange);
    }
    (void)r1;
    (void)r2;
    (void)r3;
    (void)r4;
    cplx Gm31[4][4], Gp13[4][4], Gm42[4][4], Gp24[4][4], Gp14[4][4], Gp23[4][4];
    green(s, p3, p1, tau, -1, Gm31);
    green(s, p1, p3, tau, +1, Gp13);
    green(s, p4, p2, tau, -1, Gm42);
    green(s, p2, p4, tau, +1, Gp24);
    green(s, p1, p4, tau, +1, Gp14);
    green(s, p2, p3, tau, +1, Gp23);
    cplx a[4][4], b[4][4], c[4][4], d[4][4];
    matmul4(Gm31, Gp13, a);
    matmul4(Gm42, Gp24, b);
    const cplx direct = trace4(a) * trace4(b);
    matmul4(Gm31, Gp14, a);
    matmul4(Gm42, Gp23, c);
    matmul4(a, c, d);
    const cplx exchange = trace4(d);
    return -0.5 * (direct - exchange);
}

/* The quotient of Eq. redundant for one pair of electron pairs and one tau:
 * f / (w(r1,r2) w(r3,r4) w(tau)) with w(r1,r2) = g(r1) g(r2) / (N_g r12) and
 * w(tau) = lambda exp(-lambda tau).  The 1/r12 1/r34 of f cancel against
 * the weights.  out = {Re, Im}. */
static cplx quotient(const or_system *s, const cplx *p1, const cplx *p2, const cplx *p3,
                     const cplx *p4, double g1, double g2, double g3, double g4, double tau,
                     double Ng, double lambda, const double *r1, const double *r2, const double *r3,
                     const double *r4)
{
    const cplx F = integrand(s, p1, p2, p3, p4, tau, r1, r2, r3, r4);
    return F * (Ng / (g1 * g2)) * (Ng / (g3 * g4)) * (exp(lambda * tau) / lambda);
}

void or_pair_value(const or_system *s, const double *r1, const double *r2, const double *r3,
                   const double *r4, double tau, double *out)
{
    const int n = s->n_occ + s->n_vir;
    double *phi = malloc(sizeof(double) * 2 * 4 * n * 4);
    const double *rr[4] = {r1, r2, r3, r4};
    double g[4];
    for (int k = 0; k < 4; ++k) {
        or_spinors_at(s, rr[k], phi + (size_t)k * 8 * n);
        g[k] = or_g(s, rr[k]);
    }
    const cplx *P = (const cplx *)phi;
    const cplx v = quotient(s, P, P + 4 * n, P + 8 * n, P + 12 * n, g[0], g[1], g[2], g[3], tau,
                            or_Ng(s), or_lambda(s), r1, r2, r3, r4);
    out[0] = creal(v);
    out[1] = cimag(v);
    free(phi);
}

/* Kahan-compensated accumulation. */
typedef struct { double s, c; } kahan;
static void kadd(kahan *k, double x)
{
    const double y = x - k->c;
    const double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* Spinor values and g at all 2m walker positions of one step.
 * r: [m][2][3]; position x = 2p + e holds electron e (0: r1, 1: r2) of pair p. */
static void positions_prepare(const or_system *s, int m, const double *r, cplx *phi, double *g,
                              int n_threads)
{
    const int n = s->n_occ + s->n_vir;
#pragma omp parallel for schedule(dynamic) num_threads(n_threads)
    for (int x = 0; x < 2 * m; ++x) {
        or_spinors_at(s, r + 3 * x, (double *)(phi + (size_t)x * 4 * n));
        g[x] = or_g(s, r + 3 * x);
    }
}

/* Replay mode: per-step estimates I'_n of Eq. redundant from given samples.
 * r: [n][m][2][3]; tau: [n][n_tau].  per_step[n] receives
 * (1/n_tau) sum_t (1/mC2) sum_{p<q} Re f/(w w w); abs_per_step (optional)
 * receives the same with |Re| (the scale of the cancellation). */
int or_eval_steps(const or_system *s, long n_steps, int m, int n_tau, const double *r,
                  const double *tau, double *per_step, double *abs_per_step, int n_threads)
{
    if (m < 2 || n_tau < 1) return -1;
    if (n_threads <= 0) n_threads = 1;
    const int n = s->n_occ + s->n_vir;
    const double Ng = or_Ng(s), lambda = or_lambda(s);
    const double npairs = 0.5 * (double)m * (double)(m - 1);
    cplx *phi = malloc(sizeof(cplx) * (size_t)2 * m * 4 * n);
    double *g = malloc(sizeof(double) * 2 * m);
    double *part = malloc(sizeof(double) * m);
    double *apart = malloc(sizeof(double) * m);
    for (long st = 0; st < n_steps; ++st) {
        const double *rs = r + (size_t)st * m * 6;
        positions_prepare(s, m, rs, phi, g, n_threads);
        kahan tot = {0, 0}, atot = {0, 0};
        for (int t = 0; t < n_tau; ++t) {
            const double tt = tau[st * n_tau + t];
#pragma omp parallel for schedule(dynamic) num_threads(n_threads)
            for (int p = 0; p < m - 1; ++p) {
                kahan acc = {0, 0}, aacc = {0, 0};
                const cplx *p1 = phi + (size_t)(2 * p) * 4 * n, *p2 = phi + (size_t)(2 * p + 1) * 4 * n;
                for (int q = p + 1; q < m; ++q) {
                    const cplx *p3 = phi + (size_t)(2 * q) * 4 * n;
                    const cplx *p4 = phi + (size_t)(2 * q + 1) * 4 * n;
                    const double v = creal(quotient(s, p1, p2, p3, p4, g[2 * p], g[2 * p + 1],
                                                    g[2 * q], g[2 * q + 1], tt, Ng, lambda, rs + 6 * p,
                                                    rs + 6 * p + 3, rs + 6 * q, rs + 6 * q + 3));
                    kadd(&acc, v);
                    kadd(&aacc, fabs(v));
                }
                part[p] = acc.s;
                apart[p] = aacc.s;
            }
            kahan st_t = {0, 0}, ast_t = {0, 0};
            for (int p = 0; p < m - 1; ++p) {
                kadd(&st_t, part[p]);
                kadd(&ast_t, apart[p]);
            }
            kadd(&tot, st_t.s / npairs);
            kadd(&atot, ast_t.s / npairs);
        }
        per_step[st] = tot.s / n_tau;
        if (abs_per_step) abs_per_step[st] = atot.s / n_tau;
    }
    free(phi);
    free(g);
    free(part);
    free(apart);
    return 0;
}

/* Re f/(w w w) for selected pairs of walker pairs (p < q) at one step, for
 * each of the n_tau times.  r: [m][2][3]; out: [n_sel][n_tau]. */
int or_eval_pairs(const or_system *s, int m, int n_tau, const double *r, const double *tau,
                  int n_sel, const int *psel, const int *qsel, double *out, int n_threads)
{
    if (n_threads <= 0) n_threads = 1;
    const int n = s->n_occ + s->n_vir;
    const double Ng = or_Ng(s), lambda = or_lambda(s);
    cplx *phi = malloc(sizeof(cplx) * (size_t)2 * m * 4 * n);
    double *g = malloc(sizeof(double) * 2 * m);
    positions_prepare(s, m, r, phi, g, n_threads);
    int bad = 0;
#pragma omp parallel for schedule(dynamic) num_threads(n_threads) reduction(| : bad)
    for (int k = 0; k < n_sel; ++k) {
        const int p = psel[k], q = qsel[k];
        if (p < 0 || q < 0 || p >= m || q >= m || p == q) {
            bad = 1;
            continue;
        }
        for (int t = 0; t < n_tau; ++t)
            out[(size_t)k * n_tau + t] =
                creal(quotient(s, phi + (size_t)(2 * p) * 4 * n, phi + (size_t)(2 * p + 1) * 4 * n,
                               phi + (size_t)(2 * q) * 4 * n, phi + (size_t)(2 * q + 1) * 4 * n,
                               g[2 * p], g[2 * p + 1], g[2 * q], g[2 * q + 1], tau[t], Ng, lambda,
                               r + 6 * p, r + 6 * p + 3, r + 6 * q, r + 6 * q + 3));
    }
    free(phi);
    free(g);
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* Random numbers and sampling                                             */
/* ---------------------------------------------------------------------- */

/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of
 *   (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
 *   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
 * with the key bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Counter layout shared by the sampling steps (a published-definition
 * generator, keyed by the 64-bit seed):
 *   ctr = {step_lo, step_hi, index, tag}, key = {seed_lo, seed_hi}
 *   tag 0, 1: Metropolis move of walker pair `index` at `step`
 *   tag 2:    imaginary time number `index` at `step`. */
static void draw(uint64_t seed, uint64_t step, uint32_t index, uint32_t tag, uint32_t out[4])
{
    const uint32_t ctr[4] = {(uint32_t)step, (uint32_t)(step >> 32), index, tag};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

static double u32_open(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

/* (0, 1] with 53 random bits. */
static double u53_half_open(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 1.0) * (1.0 / 9007199254740992.0);
}

/* tau = -ln(u)/lambda: the analytic inverse CDF of w(tau) = lambda exp(-lambda tau). */
void or_tau_draws(uint64_t seed, uint64_t step, int n_tau, double lambda, double *tau)
{
    for (int t = 0; t < n_tau; ++t) {
        uint32_t o[4];
        draw(seed, step, (uint32_t)t, 2u, o);
        tau[t] = -log(u53_half_open(o[0], o[1])) / lambda;
    }
}

/* Unnormalised pair weight g(r1) g(r2) / r12 (the 1/N_g cancels in ratios). */
static double pair_weight(const or_system *s, const double *r1, const double *r2)
{
    const double dx = r1[0] - r2[0], dy = r1[1] - r2[1], dz = r1[2] - r2[2];
    const double r12 = sqrt(dx * dx + dy * dy + dz * dz);
    return or_g(s, r1) * or_g(s, r2) / r12;
}

/* Metropolis walk of the m electron pairs under w(r1,r2) for n_steps steps
 * numbered step0, step0+1, ...  Each step moves both electrons of every pair
 * by a uniform displacement in [-delta, delta]^3 and accepts with
 * probability min(1, w'/w).  r: [m][2][3], updated in place.
 * Returns the number of accepted moves. */
long or_metropolis(const or_system *s, int m, double *r, uint64_t seed, uint64_t step0,
                   long n_steps, double delta)
{
    long accepted = 0;
    for (long st = 0; st < n_steps; ++st) {
        const uint64_t step = step0 + (uint64_t)st;
        for (int p = 0; p < m; ++p) {
            uint32_t a[4], b[4];
            draw(seed, step, (uint32_t)p, 0u, a);
            draw(seed, step, (uint32_t)p, 1u, b);
            const uint32_t u[7] = {a[0], a[1], a[2], a[3], b[0], b[1], b[2]};
            double *r1 = r + 6 * p, *r2 = r + 6 * p + 3;
            double n1[3], n2[3];
            for (int j = 0; j < 3; ++j) {
                n1[j] = r1[j] + delta * (2.0 * u32_open(u[j]) - 1.0);
                n2[j] = r2[j] + delta * (2.0 * u32_open(u[3 + j]) - 1.0);
            }
            const double w_old = pair_weight(s, r1, r2);
            const double w_new = pair_weight(s, n1, n2);
            if (u32_open(u[6]) * w_old < w_new) {
                memcpy(r1, n1, sizeof(n1));
                memcpy(r2, n2, sizeof(n2));
                ++accepted;
            }
        }
    }
    return accepted;
}

/* Burn-in: n_burn Metropolis steps from step 0.  After every complete window
 * of `window` steps the displacement is rescaled by the window's acceptance
 * fraction a as delta <- delta * min(2, max(0.5, a / 0.5)), steering towards
 * half acceptance; the final delta is returned. */
double or_burn_in(const or_system *s, int m, double *r, uint64_t seed, long n_burn, double delta,
                  int window)
{
    long done = 0;
    while (done < n_burn) {
        const long len = (n_burn - done < window) ? n_burn - done : window;
        const long acc = or_metropolis(s, m, r, seed, (uint64_t)done, len, delta);
        if (len == window) {
            const double a = (double)acc / (double)((long)m * window);
            double f = a / 0.5;
            if (f > 2.0) f = 2.0;
            if (f < 0.5) f = 0.5;
            delta = delta * f;
        }
        done += len;
    }
    return delta;
}

/* ---------------------------------------------------------------------- */
/* Statistics (Eq. uncertainty)                                            */
/* ---------------------------------------------------------------------- */

/* I_N, sigma_N^2, sigma-bar_N and the number of complete blocks from per-step
 * estimates I'_n with block size nb:
 *   sigma_N^2 = (N_b/N) sum_blocks (block mean - I_N)^2,
 *   sigma-bar_N = sigma_N / sqrt(N/N_b). */
void or_blocking(const double *per_step, long n, int nb, double *out)
{
    const long nblk = n / nb;
    out[0] = out[1] = out[2] = 0.0;
    out[3] = (double)nblk;
    if (nblk == 0) return;
    kahan mean = {0, 0};
    for (long b = 0; b < nblk; ++b) {
        kahan bs = {0, 0};
        for (int k = 0; k < nb; ++k) kadd(&bs, per_step[b * nb + k]);
        kadd(&mean, bs.s / nb);
    }
    const double IN = mean.s / (double)nblk;
    kahan v = {0, 0};
    for (long b = 0; b < nblk; ++b) {
        kahan bs = {0, 0};
        for (int k = 0; k < nb; ++k) kadd(&bs, per_step[b * nb + k]);
        const double d = bs.s / nb - IN;
        kadd(&v, d * d);
    }
    const double N = (double)(nblk * nb);
    const double sig2 = ((double)nb / N) * v.s;
    out[0] = IN;
    out[1] = sig2;
    out[2] = sqrt(sig2) / sqrt(N / nb);
}

/* A complete run: burn-in (excluded from statistics), then n_steps steps of
 * Metropolis move, n_tau imaginary-time draws and the estimator of
 * Eq. redundant.  r: [m][2][3] initial positions, updated.  per_step: [n_steps].
 * Returns the final Metropolis displacement. */
double or_run(const or_system *s, int m, double *r, uint64_t seed, long n_burn, double delta0,
              int window, long n_steps, int n_tau, double *per_step, double *taus_out,
              long *accepted, int n_threads)
{
    const double delta = or_burn_in(s, m, r, seed, n_burn, delta0, window);
    const double lambda = or_lambda(s);
    double *tau = malloc(sizeof(double) * n_tau);
    long acc = 0;
    for (long st = 0; st < n_steps; ++st) {
        const uint64_t step = (uint64_t)n_burn + (uint64_t)st;
        acc += or_metropolis(s, m, r, seed, step, 1, delta);
        or_tau_draws(seed, step, n_tau, lambda, tau);
        if (taus_out) memcpy(taus_out + st * n_tau, tau, sizeof(double) * n_tau);
        or_eval_steps(s, 1, m, n_tau, r, tau, per_step + st, NULL, n_threads);
    }
    if (accepted) *accepted = acc;
    free(tau);
    return delta;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
