/*
 * mp2_reference.c -- TEST INFRASTRUCTURE ONLY (the oracle), not the product.
 *
 * Two-electron Coulomb integrals for the deterministic (sum-over-states)
 * relativistic MP2 energy of Eq. FinalMP2, used to check the Monte Carlo
 * estimate on small systems.  The spinor integrals (ia|jb) of the paper's
 * two-electron integral definition are expanded over the real functions
 *   f_{4 mu + 0} = g_mu,  f_{4 mu + j} = d g_mu / d x_j  (j = 1, 2, 3),
 * which span the large (Eq. C) and kinetically balanced small (the kinetic-balance condition after Eq. C)
 * components.  This file computes (PQ|RS) over those real functions with the
 * McMurchie-Davidson scheme (Hermite expansion of Gaussian products and the
 * Boys function), written from the mathematics; the spinor transformation and
 * the energy formula are done by the Python side of the oracle.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n_centres;
    const double *centres;
    const double *weight;
    int n_shells;
    const int *shell_centre;
    const int *shell_l;
    const double *shell_alpha;
    const double *shell_coef;
    int n_occ, n_vir;
    const double *C;
    const double *eps;
} or_system;

#define LMAX_PAIR 8                 /* highest l_a + l_b of a function pair */
#define LMAX_TOT (2 * LMAX_PAIR)
#define ED (LMAX_PAIR + 1)

/* ---------------------------------------------------------------------- */
/* Boys function F_n(T) = Int_0^1 t^{2n} exp(-T t^2) dt                     */
/* ---------------------------------------------------------------------- */
static void boys(int nmax, double T, double *F)
{
    if (T < 35.0) {
        /* F_nmax by its series exp(-T) sum_k (2T)^k / ((2n+1)(2n+3)...(2n+2k+1)),
         * then downward recursion F_{n} = (2T F_{n+1} + exp(-T)) / (2n + 1). */
        const double eT = exp(-T);
        double term = 1.0 / (2 * nmax + 1), sum = term;
        for (int k = 1; k < 400; ++k) {
            term *= 2.0 * T / (2 * nmax + 2 * k + 1);
            sum += term;
            if (term < 1e-17 * sum) break;
        }
        F[nmax] = eT * sum;
        for (int n = nmax - 1; n >= 0; --n) F[n] = (2.0 * T * F[n + 1] + eT) / (2 * n + 1);
    } else {
        /* Large T: F_0 = sqrt(pi/T)/2 erf(sqrt T), upward recursion. */
        const double eT = exp(-T);
        F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
        for (int n = 0; n < nmax; ++n) F[n + 1] = ((2 * n + 1) * F[n] - eT) / (2.0 * T);
    }
}

/* ---------------------------------------------------------------------- */
/* Hermite expansion of a product of two Cartesian Gaussians               */
/* ---------------------------------------------------------------------- */

/* 1-D coefficients E^{ij}_t for x_A^i x_B^j exp(-a x_A^2 - b x_B^2)
 * = sum_t E^{ij}_t Lambda_t(x_P; p):
 *   E^{00}_0 = exp(-mu X_AB^2),
 *   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1},
 *   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}. */
static void hermite_1d(int imax, int jmax, double a, double b, double A, double B,
                       double E[ED][ED][2 * ED])
{
    const double p = a + b, mu = a * b / p, P = (a * A + b * B) / p;
    const double XPA = P - A, XPB = P - B, XAB = A - B;
    memset(E, 0, sizeof(double) * ED * ED * 2 * ED);
    E[0][0][0] = exp(-mu * XAB * XAB);
    for (int i = 0; i <= imax; ++i) {
        for (int j = 0; j <= jmax; ++j) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; ++t) {
                double v;
                if (i > 0) {
                    const double *e = E[i - 1][j];
                    v = (t > 0 ? e[t - 1] / (2 * p) : 0.0) + XPA * e[t] + (t + 1) * e[t + 1];
                } else {
                    const double *e = E[i][j - 1];
                    v = (t > 0 ? e[t - 1] / (2 * p) : 0.0) + XPB * e[t] + (t + 1) * e[t + 1];
                }
                E[i][j][t] = v;
            }
        }
    }
}

/* A Cartesian primitive c x_A^l y_A^m z_A^n exp(-alpha r_A^2). */
typedef struct {
    double c, alpha, A[3];
    int pw[3];
} prim;

/* Hermite expansion of a product of two real functions, each a short sum of
 * primitives on one centre with one exponent:  f_P f_Q = sum_tuv E_tuv Lambda_tuv. */
typedef struct {
    double p, P[3];
    int L;
    double E[ED][ED][ED];
} pair_expansion;

static void expand_pair(const prim *a, int na, const prim *b, int nb, pair_expansion *out)
{
    memset(out, 0, sizeof(*out));
    const double al = a[0].alpha, be = b[0].alpha;
    out->p = al + be;
    int L = 0;
    for (int k = 0; k < 3; ++k) out->P[k] = (al * a[0].A[k] + be * b[0].A[k]) / out->p;
    static double Ex[ED][ED][2 * ED], Ey[ED][ED][2 * ED], Ez[ED][ED][2 * ED];
#pragma omp threadprivate(Ex, Ey, Ez)
    int imax[3] = {0, 0, 0}, jmax[3] = {0, 0, 0};
    for (int u = 0; u < na; ++u)
        for (int k = 0; k < 3; ++k) imax[k] = a[u].pw[k] > imax[k] ? a[u].pw[k] : imax[k];
    for (int v = 0; v < nb; ++v)
        for (int k = 0; k < 3; ++k) jmax[k] = b[v].pw[k] > jmax[k] ? b[v].pw[k] : jmax[k];
    hermite_1d(imax[0], jmax[0], al, be, a[0].A[0], b[0].A[0], Ex);
    hermite_1d(imax[1], jmax[1], al, be, a[0].A[1], b[0].A[1], Ey);
    hermite_1d(imax[2], jmax[2], al, be, a[0].A[2], b[0].A[2], Ez);
    for (int u = 0; u < na; ++u)
        for (int v = 0; v < nb; ++v) {
            const int *i = a[u].pw, *j = b[v].pw;
            const double c = a[u].c * b[v].c;
            for (int t = 0; t <= i[0] + j[0]; ++t)
                for (int s = 0; s <= i[1] + j[1]; ++s)
                    for (int r = 0; r <= i[2] + j[2]; ++r) {
                        out->E[t][s][r] += c * Ex[i[0]][j[0]][t] * Ey[i[1]][j[1]][s] * Ez[i[2]][j[2]][r];
                        if (t + s + r > L) L = t + s + r;
                    }
        }
    out->L = L;
}

/* Hermite Coulomb integrals R^0_{tuv}(alpha, X) for t+u+v <= L:
 *   R^n_{000} = (-2 alpha)^n F_n(alpha |X|^2),
 *   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_x R^{n+1}_{t,u,v}  (likewise u, v). */
#define RD (LMAX_TOT + 1)
static void hermite_coulomb(int L, double alpha, const double X[3], double R[RD][RD][RD])
{
    static double Rn[RD][RD][RD][RD];
#pragma omp threadprivate(Rn)
    double F[RD + 1];
    boys(L, alpha * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]), F);
    double f = 1.0;
    for (int n = 0; n <= L; ++n) {
        Rn[n][0][0][0] = f * F[n];
        f *= -2.0 * alpha;
    }
    for (int N = 1; N <= L; ++N)
        for (int n = 0; n <= L - N; ++n)
            for (int t = 0; t <= N; ++t)
                for (int u = 0; u <= N - t; ++u) {
                    const int v = N - t - u;
                    double val;
                    if (t > 0)
                        val = (t > 1 ? (t - 1) * Rn[n + 1][t - 2][u][v] : 0.0) + X[0] * Rn[n + 1][t - 1][u][v];
                    else if (u > 0)
                        val = (u > 1 ? (u - 1) * Rn[n + 1][t][u - 2][v] : 0.0) + X[1] * Rn[n + 1][t][u - 1][v];
                    else
                        val = (v > 1 ? (v - 1) * Rn[n + 1][t][u][v - 2] : 0.0) + X[2] * Rn[n + 1][t][u][v - 1];
                    Rn[n][t][u][v] = val;
                }
    for (int t = 0; t <= L; ++t)
        for (int u = 0; u <= L - t; ++u)
            for (int v = 0; v <= L - t - u; ++v) R[t][u][v] = Rn[0][t][u][v];
}

/* (ab|cd) = 2 pi^{5/2} / (p q sqrt(p+q)) sum_{tuv} E^{ab}_{tuv}
 *           sum_{t'u'v'} (-1)^{t'+u'+v'} E^{cd}_{t'u'v'} R_{t+t',u+u',v+v'}(pq/(p+q), P-Q). */
static double eri_pairs(const pair_expansion *ab, const pair_expansion *cd)
{
    static double R[RD][RD][RD];
#pragma omp threadprivate(R)
    const double p = ab->p, q = cd->p, alpha = p * q / (p + q);
    const double X[3] = {ab->P[0] - cd->P[0], ab->P[1] - cd->P[1], ab->P[2] - cd->P[2]};
    const int L = ab->L + cd->L;
    hermite_coulomb(L, alpha, X, R);
    double sum = 0.0;
    for (int t = 0; t <= ab->L; ++t)
        for (int u = 0; u <= ab->L - t; ++u)
            for (int v = 0; v <= ab->L - t - u; ++v) {
                const double e1 = ab->E[t][u][v];
                if (e1 == 0.0) continue;
                double inner = 0.0;
                for (int t2 = 0; t2 <= cd->L; ++t2)
                    for (int u2 = 0; u2 <= cd->L - t2; ++u2)
                        for (int v2 = 0; v2 <= cd->L - t2 - u2; ++v2) {
                            const double e2 = cd->E[t2][u2][v2];
                            if (e2 == 0.0) continue;
                            const double sg = ((t2 + u2 + v2) & 1) ? -1.0 : 1.0;
                            inner += sg * e2 * R[t + t2][u + u2][v + v2];
                        }
                sum += e1 * inner;
            }
    return 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * sum;
}

/* Coulomb integral over four single primitives (for the checks):
 * each primitive given as centre[3], alpha, powers[3]. */
double mp2_prim_eri(const double *A, double a, const int *pa, const double *B, double b,
                    const int *pb, const double *Cc, double c, const int *pc, const double *D,
                    double d, const int *pd)
{
    prim pr[4] = {{1.0, a, {A[0], A[1], A[2]}, {pa[0], pa[1], pa[2]}},
                  {1.0, b, {B[0], B[1], B[2]}, {pb[0], pb[1], pb[2]}},
                  {1.0, c, {Cc[0], Cc[1], Cc[2]}, {pc[0], pc[1], pc[2]}},
                  {1.0, d, {D[0], D[1], D[2]}, {pd[0], pd[1], pd[2]}}};
    pair_expansion ab, cd;
    expand_pair(&pr[0], 1, &pr[1], 1, &ab);
    expand_pair(&pr[2], 1, &pr[3], 1, &cd);
    return eri_pairs(&ab, &cd);
}

/* ---------------------------------------------------------------------- */
/* Real functions g_mu and d g_mu / d x_j                                  */
/* ---------------------------------------------------------------------- */

static const int CART[3][6][3] = {
    {{0, 0, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}},
};
static const int NCART[3] = {1, 3, 6};

/* Real function F = 4 mu + j as a sum of at most two primitives. */
static int real_function(const or_system *s, int F, prim out[2])
{
    const int mu = F / 4, j = F % 4;
    int k = 0, m = 0;
    for (k = 0; k < s->n_shells; ++k) {
        if (mu < m + NCART[s->shell_l[k]]) break;
        m += NCART[s->shell_l[k]];
    }
    const int *pw = CART[s->shell_l[k]][mu - m];
    const double *A = s->centres + 3 * s->shell_centre[k];
    const double al = s->shell_alpha[k], c = s->shell_coef[k];
    prim base = {c, al, {A[0], A[1], A[2]}, {pw[0], pw[1], pw[2]}};
    if (j == 0) {
        out[0] = base;
        return 1;
    }
    /* d/dx [x^a e^{-al x^2}] = a x^{a-1} e - 2 al x^{a+1} e */
    const int d = j - 1;
    int n = 0;
    out[n] = base;
    out[n].pw[d] += 1;
    out[n].c = -2.0 * al * c;
    ++n;
    if (pw[d] > 0) {
        out[n] = base;
        out[n].pw[d] -= 1;
        out[n].c = pw[d] * c;
        ++n;
    }
    return n;
}

/* (PQ|RS) over the real functions of one ERI. */
double mp2_ao_eri(const or_system *s, const int *PQ, const int *RS)
{
    prim a[2], b[2], c[2], d[2];
    const int na = real_function(s, PQ[0], a), nb = real_function(s, PQ[1], b);
    const int nc = real_function(s, RS[0], c), nd = real_function(s, RS[1], d);
    pair_expansion ab, cd;
    expand_pair(a, na, b, nb, &ab);
    expand_pair(c, nc, d, nd, &cd);
    return eri_pairs(&ab, &cd);
}

/* Coulomb matrix over a list of real-function pairs:
 * out[u][v] = (P_u Q_u | P_v Q_v), pairs given as flat [n_pairs][2]. */
int mp2_pair_eri_matrix(const or_system *s, int n_pairs, const int *pairs, double *out, int n_threads)
{
    if (n_threads <= 0) n_threads = 1;
    pair_expansion *ex = malloc(sizeof(pair_expansion) * (size_t)n_pairs);
    if (!ex) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic) num_threads(n_threads) reduction(| : bad)
    for (int u = 0; u < n_pairs; ++u) {
        prim a[2], b[2];
        const int na = real_function(s, pairs[2 * u], a), nb = real_function(s, pairs[2 * u + 1], b);
        expand_pair(a, na, b, nb, &ex[u]);
        if (ex[u].L > LMAX_PAIR) bad = 1;
    }
    if (bad) {
        free(ex);
        return -2;
    }
#pragma omp parallel for schedule(dynamic) num_threads(n_threads)
    for (int u = 0; u < n_pairs; ++u)
        for (int v = u; v < n_pairs; ++v) {
            const double val = eri_pairs(&ex[u], &ex[v]);
            out[(size_t)u * n_pairs + v] = val;
            out[(size_t)v * n_pairs + u] = val;
        }
    free(ex);
    return 0;
}
