/*
 * mcmp2.h -- C ABI of the GB300 Monte Carlo four-component relativistic MP2
 * library (Cruz, Garza, Yanai, Hirata, arXiv 2203.05632).
 *
 * The library evaluates, entirely on one GPU, the per-step Monte Carlo
 * estimate of the second-order energy of Eq. FinalMP2 in the 13-dimensional
 * form of Eq. MCMP2 (Sec. III): a Metropolis move of m electron-pair walkers
 * under w(r1,r2) = g(r1) g(r2) / (N_g r12) (Eq. basisSet), large- and
 * kinetically balanced small-component basis values at the 2m positions (Eq. C
 * with the kinetic-balance condition that follows it), four-component spinors,
 * imaginary times tau from the inverse CDF of w(tau) = lambda exp(-lambda tau)
 * (Eq. tauWeight), the 4x4
 * propagator blocks G-(x,y,-tau) and G+(x,y,tau) between all walker pairs,
 * and the traced direct and exchange products summed over all mC2 pairs of
 * pairs (Eq. redundant), with Flyvbjerg-Petersen blocking (Eq. uncertainty).
 *
 * Conventions for every call:
 *  - Units are bohr and hartree.  Complex numbers are (re, im) double pairs.
 *  - Every call returns MCMP2_OK (0) or a negative MCMP2_E* status; no call
 *    aborts or throws.  mcmp2_last_error() gives the message of the last
 *    failure on a context.
 *  - Pointers named *_host are host memory read or written synchronously
 *    with respect to the context's stream (the call returns after the copy).
 *  - The context owns no device memory: the caller allocates one device
 *    workspace of mcmp2_workspace_bytes() bytes, binds it, and keeps it
 *    alive until mcmp2_destroy().  All work is issued on the stream given at
 *    creation.
 *  - A context is not thread-safe; calls on one context must not overlap.
 *
 * Readings of the paper fixed by this interface:
 *  - Basis (Eq. C and the kinetic-balance condition after it, restricted kinetic balance): n_L real Cartesian
 *    Gaussians g_mu (shells of l = 0, 1, 2 expanded in the order s; x, y, z;
 *    xx, xy, xz, yy, yz, zz), g_mu(r) = coef (x-Ax)^a (y-Ay)^b (z-Az)^c
 *    exp(-alpha |r-A|^2).  Large 2-spinor basis {g_mu e_alpha, g_mu e_beta};
 *    small 2-spinor basis {(sigma.grad)(g_mu e_alpha), (sigma.grad)(g_mu e_beta)}
 *    (= i(sigma.p) of the large ones).  Spinor coefficients C have 4 n_L rows:
 *    L-alpha, L-beta, S-alpha, S-beta blocks of n_L rows each.
 *  - The integrand is the trace form of Eq. MCMP2 derived from Eq. FinalMP2:
 *    -1/2 { tr[G-(3,1)G+(1,3)] tr[G-(4,2)G+(2,4)] - tr[G-(3,1)G+(1,4)G-(4,2)G+(2,3)] }
 *    with (r1, r2) = pair p, (r3, r4) = pair q; its real part is summed over p < q.
 *  - n_tau imaginary times per step are shared by all pairs and averaged.
 */
#ifndef MCMP2_H
#define MCMP2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define MCMP2_OK 0
#define MCMP2_EINVAL (-1)      /* bad argument, size or state */
#define MCMP2_ENOTLOADED (-2)  /* system, workspace or walkers missing */
#define MCMP2_ECUDA (-3)       /* a CUDA call failed (message has the CUDA error) */
#define MCMP2_ENONFINITE (-4)  /* an input or a step result is not finite */
#define MCMP2_ETIMEOUT (-5)    /* a bounded device wait ran out */
#define MCMP2_ENOSPACE (-6)    /* workspace or caller buffer too small */
#define MCMP2_EUNSUPPORTED (-7) /* no sm_103 device, or a feature this build lacks */

/* Arithmetic of the propagator and spinor contractions. */
#define MCMP2_FP64 0   /* complex128 throughout (CUDA-core DFMA) */
#define MCMP2_MIXED 1  /* split-BF16 x3 tensor-core products, FP32 accumulate; FP64 sampling and sums */
#define MCMP2_TF32 2   /* as MCMP2_MIXED, but the propagators are single TF32 tensor-core products of
                        * operands rounded to nearest TF32 (10-bit significand): 2/3 of the MMAs,
                        * relative error per operand <= 2^-11, unbiased */

/* Two-electron interaction (Sec. II, operator g_ij).  The paper's runs keep the
 * Coulomb term only; the Gaunt term -alpha(i).alpha(j)/(2 r_ij) and the gauge
 * term -(alpha(i).r_ij)(alpha(j).r_ij)/(2 r_ij^3) (together: Breit) can be added. */
#define MCMP2_COULOMB 0
#define MCMP2_GAUNT 1  /* Coulomb + Gaunt */
#define MCMP2_BREIT 2  /* Coulomb + Gaunt + gauge term */

/* Sampling constants.  Sec. III (after Eq. basisSet) draws the walker pairs from
 * w(r1,r2) by the Metropolis algorithm but leaves the proposal, its step size and
 * the burn-in open.  Reading used here: a move displaces both electrons of a pair by
 * independent uniform offsets in the cube [-delta, delta]^3 and is accepted with
 * probability min(1, w'/w); delta starts at MCMP2_DELTA0 and, during burn-in only,
 * is multiplied after every MCMP2_ADAPT_WINDOW steps by clamp(a / 0.5, 0.5, 2),
 * a being the window's acceptance fraction; production steps keep delta fixed. */
#define MCMP2_DELTA0 0.6        /* initial Metropolis displacement (bohr) */
#define MCMP2_ADAPT_WINDOW 20   /* burn-in steps per displacement adaptation */
#define MCMP2_BLOCK_SIZE 100    /* Flyvbjerg-Petersen block size N_b (Sec. IV) */

typedef struct mcmp2_ctx mcmp2_ctx;

/* Problem sizes that fix the workspace. */
typedef struct {
    int n_centres;    /* atoms (centres of basis shells and of g), 1 .. 256 */
    int n_functions;  /* n_L, scalar Cartesian Gaussians after shell expansion */
    int n_occ;        /* occupied positive-energy spinors (even, >= 2) */
    int n_vir;        /* virtual positive-energy spinors (even, >= 2) */
    int m;            /* electron-pair walkers (2 <= m <= 65536) */
    int n_tau;        /* imaginary times per step (1 <= n_tau <= 64) */
} mcmp2_dims;

/* Basis shells and the weight function g of Eq. basisSet. */
typedef struct {
    int n_centres;
    const double *centres;      /* [n_centres][3] */
    const double *weight;       /* [n_centres][4]: c1, zeta1, c2, zeta2 (Table 1 layout) */
    int n_shells;
    const int *shell_centre;    /* [n_shells] */
    const int *shell_l;         /* [n_shells], 0..2 */
    const double *shell_alpha;  /* [n_shells] exponents > 0 */
    const double *shell_coef;   /* [n_shells] */
} mcmp2_basis;

/* Running statistics of the production steps (burn-in excluded). */
typedef struct {
    double energy;       /* I_N: mean of the complete block means */
    double variance;     /* sigma_N^2 of Eq. uncertainty */
    double error;        /* sigma-bar_N = sigma_N / sqrt(N/N_b) */
    int64_t n_blocks;    /* complete blocks */
    int64_t steps;       /* production steps accumulated */
    double mean_all;     /* mean of all step estimates, incomplete block included */
    double last_step;    /* I'_n of the latest step */
    double accept_rate;  /* Metropolis acceptance over the production steps */
} mcmp2_result;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (plumbing of this library; the paper has no counterpart)
 * (a cudaStream_t; NULL for the legacy default stream) in `precision`
 * (MCMP2_FP64, MCMP2_MIXED or MCMP2_TF32).  Fails with MCMP2_EUNSUPPORTED on
 * devices other than compute capability 10.3. */
int mcmp2_create(mcmp2_ctx **ctx, int device, void *cuda_stream, int precision);

/* Select the two-electron interaction of the integrand (MCMP2_COULOMB, the default,
 * MCMP2_GAUNT or MCMP2_BREIT) for the following steps and replays.  Each electron pair's
 * interaction (1/r_ab) sum_A c_A O_A(a) O_A(b), O_A in {1, alpha_x, alpha_y, alpha_z,
 * alpha.n_ab}, enters the trace form with O_A at the two points of the pair (the
 * weight's 1/r_ab is unchanged).  All three precisions (the tensor-core forms apply
 * the operators to the G- blocks in their trace epilogue); four-component systems
 * only (MCMP2_EUNSUPPORTED after mcmp2_load_system_2c); mcmp2_backward requires
 * MCMP2_COULOMB.  Statistics accumulated so far are kept; checkpoints record the
 * interaction. */
int mcmp2_set_interaction(mcmp2_ctx *ctx, int interaction);

/* Release the context (not the caller's workspace).  NULL is ignored. */
void mcmp2_destroy(mcmp2_ctx *ctx);

/* Message of the last failed call on ctx (never NULL; "" if none). */
const char *mcmp2_last_error(const mcmp2_ctx *ctx);

/* Bytes of device workspace needed for `dims` in `precision` (plumbing of this
 * library; the paper has no counterpart). */
int mcmp2_workspace_bytes(const mcmp2_dims *dims, int precision, size_t *bytes);

/* Bind a device workspace (256-byte aligned, >= mcmp2_workspace_bytes) for `dims`.
 * The caller owns the memory and keeps it alive until mcmp2_destroy(); it is not
 * freed by the library.  Rebinding discards the loaded system, walkers and
 * statistics.  Plumbing of this library; the paper has no counterpart. */
int mcmp2_bind_workspace(mcmp2_ctx *ctx, const mcmp2_dims *dims, void *dptr, size_t bytes);

/* Load the system: the inputs a Dirac-Hartree-Fock calculation furnishes
 * (Sec. IV: MO coefficients and orbital energies) in the basis of Eq. C with
 * kinetic balance, plus the weight-function parameters of Eq. basisSet
 * (Table 1 layout).  n_occ occupied then n_vir virtual spinors with
 * coefficients C_host (complex, [4 n_L][n_occ + n_vir] row-major, rows
 * L-alpha, L-beta, S-alpha, S-beta blocks) and energies eps_host
 * ([n_occ + n_vir]).  Sizes must match the bound dims (MCMP2_EINVAL).
 * Requires max occupied eps < min virtual eps, so that the exponent of
 * Eq. tauWeight, lambda = 2 (eps_LUMO - eps_HOMO), is positive (MCMP2_EINVAL);
 * non-finite entries give MCMP2_ENONFINITE.  Host arrays are copied; N_g (the
 * normalisation after Eq. basisSet) is evaluated in closed form. */
int mcmp2_load_system(mcmp2_ctx *ctx, const mcmp2_basis *basis, int n_occ, int n_vir,
                      const double *C_host, const double *eps_host);

/* Two-component variant (Sec. II: the Monte Carlo algorithm holds unchanged for
 * two-component Hamiltonians such as X2C).  The spinors have the components
 * alpha and beta only, phi_k(r) = sum_mu (C^a_{mu k} g_mu(r), C^b_{mu k} g_mu(r)),
 * so G-(x,y,-tau) and G+(x,y,tau) are 2x2 complex blocks in the same trace form
 * (a quarter of the four-component contraction work).  C2_host: complex
 * [2 n_L][n_occ + n_vir] row-major, rows alpha block then beta block; the other
 * arguments and checks as in mcmp2_load_system.  The result equals
 * mcmp2_load_system with these rows as L-alpha, L-beta and zero small rows.
 * All three precisions; the tensor-core forms contract 32 x 32-pair tiles of
 * 2x2 blocks (mcmp2_debug_partials then reports tile_pairs = 32).  The Coulomb
 * interaction only (MCMP2_EUNSUPPORTED otherwise, also from
 * mcmp2_set_interaction afterwards); mcmp2_backward covers four-component
 * systems only. */
int mcmp2_load_system_2c(mcmp2_ctx *ctx, const mcmp2_basis *basis, int n_occ, int n_vir,
                         const double *C2_host, const double *eps_host);

/* Walker pairs for the Metropolis walk of Sec. III (after Eq. basisSet: the
 * pairs are distributed as w(r1, r2) by the Metropolis algorithm; the burn-in
 * steps are excluded from the statistics of Eq. uncertainty).  Sets the m walker
 * pairs from r_host ([m][2][3], bohr), or, if r_host is NULL, draws them from
 * g(r1) g(r2) (each electron from the Gaussian mixture g; Philox counters of the
 * reserved step 2^64 - 1), and runs `burn_in` Metropolis steps with seed `seed`
 * (steps numbered from 0), adapting the displacement every MCMP2_ADAPT_WINDOW
 * steps by delta <- delta * clamp(a/0.5, 0.5, 2) with a the window's acceptance
 * fraction.  Resets the statistics and the step counter to burn_in.
 * MCMP2_ENONFINITE for a non-finite position, MCMP2_ENOTLOADED before a system. */
int mcmp2_set_walkers(mcmp2_ctx *ctx, const double *r_host, uint64_t seed, int64_t burn_in);

/* Run n production steps with seed `seed`, all on the device: the Metropolis
 * move (Sec. III), n_tau imaginary times by the inverse CDF of Eq. tauWeight,
 * the redundant-walker estimate I'_n of Eq. redundant over all mC2 pairs of
 * walker pairs, and the blocking update of Eq. uncertainty (N_b =
 * MCMP2_BLOCK_SIZE).  Steps continue the context's step counter, so consecutive
 * calls with one seed equal one call.  Writes the running statistics to
 * out_host (may be NULL; then nothing is copied back and the call does not wait
 * for the device).  MCMP2_ENOTLOADED without walkers; MCMP2_ENONFINITE if a step
 * estimate is not finite; MCMP2_ETIMEOUT if a bounded device wait ran out. */
int mcmp2_run_steps(mcmp2_ctx *ctx, int64_t n, uint64_t seed, mcmp2_result *out_host);

/* Replay mode: evaluate I'_n of Eq. redundant for n given samples (positions
 * and imaginary times supplied by the caller instead of drawn), without moving
 * walkers or touching the statistics.  r_host: [n][m][2][3]; tau_host:
 * [n][n_tau] (finite, >= 0, else MCMP2_EINVAL); per_step_host: [n] output. */
int mcmp2_eval_fixed(mcmp2_ctx *ctx, int64_t n, const double *r_host, const double *tau_host,
                     double *per_step_host);

/* Copy the current walker positions ([m][2][3]) and the Metropolis displacement
 * delta to the host (either pointer may be NULL). */
int mcmp2_get_walkers(mcmp2_ctx *ctx, double *r_host, double *delta_host);

/* Per-tile partial sums of the latest step, for sampled checks at full size:
 * out_host[t * n_tiles + k] = sum over the pairs (p < q) of tile k of the
 * summand Re f/(w w w) of Eq. redundant at time t, tiles of `tile_pairs` pairs
 * per side enumerated row by row over the upper triangle (bp <= bq).
 * *n_tiles and *tile_pairs are written; capacity is the length of out_host in
 * doubles (MCMP2_ENOSPACE if short; out_host NULL only reports the sizes). */
int mcmp2_debug_partials(mcmp2_ctx *ctx, double *out_host, size_t capacity, int *n_tiles,
                         int *tile_pairs);

/* Element-by-element record of one tile of the pair-of-pairs sum of Eq. redundant,
 * for checking every summand at full size.  Evaluates one replay step for the
 * positions r_host ([m][2][3]) and times tau_host ([n_tau], finite, >= 0) with the
 * kernels and launch shape of mcmp2_eval_fixed, and records for the tile (bp, bq)
 * of T x T walker pairs (T = tile_pairs: 8 in the FP64 form, 16 in the
 * tensor-core forms, 32 for two-component systems there; 0 <= bp <= bq <
 * ceil(m / T), else MCMP2_EINVAL) every summand
 *   out_host[(t T + i) T + j] = Re f(p, q, tau_t) / (w(r1p, r2p) w(r1q, r2q) w(tau_t)),
 *   p = bp T + i, q = bq T + j,
 * with the loaded interaction, for p < q < m, and 0 for the other entries.
 * capacity >= n_tau T^2 doubles (MCMP2_ENOSPACE).  *step_host (may be NULL)
 * receives that step's I'_n, *tile_pairs (may be NULL) receives T.  The walk
 * and the statistics are untouched. */
int mcmp2_debug_elements(mcmp2_ctx *ctx, const double *r_host, const double *tau_host, int bp, int bq,
                         double *out_host, size_t capacity, double *step_host, int *tile_pairs);

/* Gradient of the replay estimate E = (1/n) sum_n I'_n for the n given samples
 * (common random numbers: r_host [n][m][2][3], tau_host [n][n_tau] as in
 * mcmp2_eval_fixed) with respect to the orbital energies and the spinor
 * coefficients of the loaded system, with lambda, eps_HOMO and eps_LUMO held
 * at their loaded values (the density the times were drawn from does not
 * move).  Hand-written adjoint of the propagator products and traces (the
 * derivative of the trace form of Eq. MCMP2), back through the spinor values
 * to eps and C.  Outputs (host): energy_host (E, may be NULL), d_eps_host
 * [n_orb], d_C_host complex [4 n_L][n_orb] in the layout of C, as
 * dE/dRe C + i dE/dIm C.  FP64 contexts only (MCMP2_EUNSUPPORTED otherwise). */
int mcmp2_backward(mcmp2_ctx *ctx, int64_t n, const double *r_host, const double *tau_host, double *energy_host,
                   double *d_eps_host, double *d_C_host);

/* Launch counters and CUDA-event timing of the pair-of-pairs contraction
 * kernel (the dominant kernel), measured on the context's stream.  Measurement
 * plumbing of this library; the paper has no counterpart. */
typedef struct {
    int64_t launches;       /* kernels this context launched since the last reset */
    int64_t pair_launches;  /* launches of the pair-of-pairs contraction kernel */
    double pair_ms;         /* summed event time of those launches (ms); 0 unless timing is on */
} mcmp2_profile_counters;

/* mode 0: read the counters (synchronises the stream when timing is on);
 * mode 1: reset them and time every later contraction launch with events;
 * mode 2: reset them and stop timing.  out may be NULL for modes 1 and 2. */
int mcmp2_profile(mcmp2_ctx *ctx, int mode, mcmp2_profile_counters *out_host);

/* Test hook for the bounded waits of the tensor-core contraction (mixed form):
 * the next contraction launch withholds its first operand copy, so its
 * consumer's wait (limited to wait_limit_s seconds, at most 10) runs out; the
 * kernel then stops, drains its own copies, frees tensor memory and returns,
 * and the call that issued it reports MCMP2_ETIMEOUT.  The context stays
 * usable.  The paper has no counterpart; this exists to test failure
 * reporting without a device fault. */
int mcmp2_test_stall_next(mcmp2_ctx *ctx, double wait_limit_s);

/* Restartable runs (Sec. III, last paragraph: each processor records its
 * number of steps, I_N and sigma-bar_N, so a run can be resumed, and resumed
 * indefinitely).  Size of a checkpoint (walkers, displacement, step counter,
 * statistics, digest of the system and interaction) and its serialisation into /
 * restoration from a host buffer.  Restoring into a context with the same system,
 * interaction and dims continues bit-identically; anything else gives
 * MCMP2_EINVAL, a short buffer MCMP2_ENOSPACE (checkpoint) or MCMP2_EINVAL
 * (restore). */
int mcmp2_checkpoint_bytes(const mcmp2_ctx *ctx, size_t *bytes);
int mcmp2_checkpoint(mcmp2_ctx *ctx, void *buf_host, size_t capacity);
int mcmp2_restore(mcmp2_ctx *ctx, const void *buf_host, size_t bytes);

/* Allocation-free evaluation of one step estimate from given spinor values.
 *
 * The paper has no counterpart: this call exists for callers that cannot
 * allocate device memory.  Some programs reserve their whole device-memory
 * budget up front and hand it to their own pool, so a later cudaMalloc (or a
 * framework allocator) would fail or is forbidden; others run this work in a
 * section of their program that must never call into an allocator.  Such a
 * caller cannot create the workspace the other entry points need.
 *
 * It computes the same quantity as the contraction and reduction of the FP64
 * form with the Coulomb interaction (there is no context, hence no
 * mcmp2_set_interaction): I'_n = (1/n_tau) sum_t (1/mC2) sum_{p<q} Re f/(w w w),
 * and writes it to out.  Inputs, all device pointers on the current device:
 *   phi   [8m][n_occ + n_vir] complex (re, im doubles): spinor value phi_k^c at
 *         row 4 x + c, position x = 2p + e (electron e of walker pair p),
 *         c = L-alpha, L-beta, S-alpha, S-beta; occupied columns first;
 *   scale [n_tau][n_occ + n_vir]: exp((eps_i - eps_HOMO) tau_t / 2) for
 *         occupied and exp(-(eps_a - eps_LUMO) tau_t / 2) for virtual spinors;
 *   a     [m]: N_g / (g(r1p) g(r2p));
 *   lambda = 2 (eps_LUMO - eps_HOMO) > 0;
 *   out   one double (device), written on cuda_stream.
 * Work is issued on cuda_stream (a cudaStream_t, NULL for the legacy default
 * stream); the call does not wait for it.
 *
 * Scratch: the per-tile partial sums live in a fixed array of
 * MCMP2_NOALLOC_MAX_PARTIALS doubles (512 KiB, plus about 1 KiB for the
 * reduction's per-block sums) inside the library, held on every GPU that
 * loads the library until the process exits.  It needs
 * n_tau * ceil(m/8) (ceil(m/8) + 1) / 2 <= MCMP2_NOALLOC_MAX_PARTIALS (for
 * example m = 1024 with n_tau <= 7); larger sizes return MCMP2_ENOSPACE
 * before any work is issued; m <= 65536 and n_tau <= 64 as for a context
 * (MCMP2_EINVAL otherwise).  The array is shared by all calls and keeps the
 * last call's contents; every entry a call reads is first written by that
 * call, and the reduction's completion counter is cleared at the start of
 * each call.  Calls that overlap on the GPU (on
 * different streams, or from different threads) race on the array and give
 * wrong results: serialise them.  The first call on each device looks up the
 * array's device address (with that device current); make that first call
 * before any stream capture.  The address is kept for the life of the
 * process, so resetting a device (cudaDeviceReset) after the first call on it
 * is not supported.  No cudaMalloc, cudaFree or other allocating routine is
 * called.
 * Returns MCMP2_OK, MCMP2_EINVAL (bad sizes, null pointers, lambda), MCMP2_ENOSPACE
 * (sizes beyond the scratch array) or MCMP2_ECUDA (a launch failed). */
#define MCMP2_NOALLOC_MAX_PARTIALS 65536
int mcmp2_pair_sum_f64_noalloc(int m, int n_occ, int n_vir, int n_tau, const double *phi, const double *scale,
                               const double *a, double lambda, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MCMP2_H */
