// C ABI of the library (include/mcmp2.h): context, caller-owned workspace,
// system loading with the host-side folding of the spinor coefficients, and
// the orchestration of sampling, integrand and statistics on one stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mcmp2.h"

#include <nvtx3/nvToolsExt.h>
#include "internal.cuh"
#include "mixed.cuh"

using namespace mcmp2;

namespace {

constexpr int REPLAY_CHUNK = 16;  // replay-mode steps staged per host->device copy

// A named range around a public call, for profilers that read NVTX ranges
// (header-only NVTX v3: a no-op unless a tool is attached).
struct CallRange {
    explicit CallRange(const char *name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange &) = delete;
    CallRange &operator=(const CallRange &) = delete;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Offsets of every array inside the caller's workspace.
struct Layout {
    size_t centres, wcoef, shell_centre, shell_alpha, shell_coef, fn_shell, fn_pow, eps, WL, WS;
    size_t r, a, tau, scale, scale_f, step, burn_acc, stats, per_step, stage_r, stage_tau, red, cdf;
    size_t elements;  // per-element record of one tile: [n_tau][32][32] doubles (the largest tile)
    size_t B, phi, partials;
    size_t Ybar, Ys, GWL, GWS, d_eps;  // adjoint buffers (FP64 form)
    MixedLayout mixed;
    size_t total;
    int tile_pairs, n_tiles;
};

bool dims_valid(const mcmp2_dims *d)
{
    return d && d->n_centres >= 1 && d->n_centres <= MAX_CENTRES && d->n_functions >= 1 && d->n_occ >= 2 && d->n_vir >= 2 && d->m >= 2 &&
           d->n_tau >= 1 && d->n_occ % 2 == 0 && d->n_vir % 2 == 0 && d->n_functions <= 65536 &&
           d->m <= MAX_WALKER_PAIRS && d->n_tau <= MAX_TAU && d->n_occ + d->n_vir <= 65536;
}

Layout make_layout(const mcmp2_dims &d, int precision)
{
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t nl = d.n_functions, no = d.n_occ + d.n_vir, m = d.m, nc = d.n_centres;
    L.centres = take(nc * 3 * 8);
    L.wcoef = take(nc * 4 * 8);
    L.shell_centre = take(nl * 4);
    L.shell_alpha = take(nl * 8);
    L.shell_coef = take(nl * 8);
    L.fn_shell = take(nl * 4);
    L.fn_pow = take(nl * 3 * 4);
    L.eps = take(no * 8);
    L.WL = take(nl * 4 * no * 8);
    L.WS = take(3 * nl * 4 * no * 8);
    L.r = take(m * 6 * 8);
    L.a = take(m * 8);
    L.tau = take(d.n_tau * 8);
    L.scale = take(d.n_tau * no * 8);
    L.scale_f = take(d.n_tau * no * 4);
    L.red = take(sizeof(ReduceScratch));
    L.cdf = take(2 * nc * 8);
    L.step = take(8);
    L.burn_acc = take(8);
    L.stats = take(sizeof(Stats));
    L.per_step = take(REPLAY_CHUNK * 8);
    L.stage_r = take(REPLAY_CHUNK * m * 6 * 8);
    L.stage_tau = take(REPLAY_CHUNK * d.n_tau * 8);
    L.elements = take((size_t)d.n_tau * TILE_PAIRS_MIXED_2C * TILE_PAIRS_MIXED_2C * 8);
    if (precision == MCMP2_FP64) {
        L.tile_pairs = TILE_PAIRS_F64;
        L.B = take(2 * m * 4 * nl * 8);
        L.phi = take(8 * m * no * 16);
        L.Ybar = take(8 * m * no * 16);
        L.Ys = take(8 * m * no * 16);
        L.GWL = take(nl * 4 * no * 8);
        L.GWS = take(3 * nl * 4 * no * 8);
        L.d_eps = take(no * 8);
    } else {
        L.tile_pairs = TILE_PAIRS_MIXED;
        L.mixed = mixed_layout(d.m, d.n_functions, d.n_occ, d.n_vir, d.n_tau, off);
        off = align256(L.mixed.end);
    }
    L.n_tiles = (int)n_tiles_for(d.m, L.tile_pairs);
    L.partials = take((size_t)d.n_tau * L.n_tiles * 8);
    L.total = off;
    return L;
}

uint64_t fnv1a(uint64_t h, const void *data, size_t n)
{
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}


const int NCART[3] = {1, 3, 6};
const int CART[3][6][3] = {
    {{0, 0, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}},
};

struct Checkpoint {
    uint64_t magic, version;
    mcmp2_dims dims;
    uint64_t digest;
    unsigned long long step;
    double delta;
    Stats stats;
};
constexpr uint64_t CK_MAGIC = 0x324d43504d32434dull;  // "MC2PMC2M"

}  // namespace

struct mcmp2_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int precision = MCMP2_FP64;
    int interaction = MCMP2_COULOMB;
    std::string err;
    bool bound = false, loaded = false, walkers = false;
    mcmp2_dims dims{};
    char *ws = nullptr;
    size_t ws_bytes = 0;
    Layout L{};
    DevSystem sys{};
    double delta = MCMP2_DELTA0;
    uint64_t digest = 0;
    MixedPlan mixed{};
    // profiling
    long long launches = 0, pair_launches = 0;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pair_events;
    double graph_pair_ms = 0.0;
    // CUDA graph of one production step (replayed by run_steps)
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side_stream = nullptr;           // the captured step's branch for the imaginary times
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_seed = 0;
    double graph_delta = 0.0;
    bool graph_timing = false;
    long long graph_launches = 0, graph_pair_launches = 0;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    bool gev_pending = false;  // the last replay's contraction events are not yet accumulated

    // Adds the contraction time of the last replay (waits for it to finish).
    cudaError_t collect_graph_time()
    {
        if (!gev_pending) return cudaSuccess;
        gev_pending = false;
        cudaError_t e = cudaEventSynchronize(gev[1]);
        if (e != cudaSuccess) return e;
        float t = 0.f;
        e = cudaEventElapsedTime(&t, gev[0], gev[1]);
        if (e == cudaSuccess) graph_pair_ms += t;
        return e;
    }

    void drop_graph()
    {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
    }

    int fail(int code, const char *fmt, ...)
    {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int cuda(cudaError_t e, const char *what)
    {
        if (e == cudaSuccess) return MCMP2_OK;
        return fail(MCMP2_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    template <typename T> T *at(size_t off) { return reinterpret_cast<T *>(ws + off); }
};

#define CK(call, what)                                   \
    do {                                                 \
        const int rc_ = ctx->cuda((call), (what));       \
        if (rc_ != MCMP2_OK) return rc_;                 \
    } while (0)

extern "C" {

int mcmp2_create(mcmp2_ctx **out, int device, void *cuda_stream, int precision)
{
    if (!out) return MCMP2_EINVAL;
    *out = nullptr;
    if (precision != MCMP2_FP64 && precision != MCMP2_MIXED && precision != MCMP2_TF32) return MCMP2_EINVAL;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return MCMP2_EUNSUPPORTED;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return MCMP2_ECUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return MCMP2_EUNSUPPORTED;
    auto *ctx = new mcmp2_ctx();
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    ctx->precision = precision;
    *out = ctx;
    return MCMP2_OK;
}

static void drop_events(mcmp2_ctx *ctx)
{
    for (auto &ev : ctx->pair_events) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    ctx->pair_events.clear();
}

void mcmp2_destroy(mcmp2_ctx *ctx)
{
    if (!ctx) return;
    drop_events(ctx);
    ctx->drop_graph();
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    for (auto &e : ctx->gev)
        if (e) cudaEventDestroy(e);
    mixed_release(ctx->mixed);
    delete ctx;
}

const char *mcmp2_last_error(const mcmp2_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int mcmp2_workspace_bytes(const mcmp2_dims *dims, int precision, size_t *bytes)
{
    if (!dims_valid(dims) || !bytes ||
        (precision != MCMP2_FP64 && precision != MCMP2_MIXED && precision != MCMP2_TF32))
        return MCMP2_EINVAL;
    *bytes = make_layout(*dims, precision).total;
    return MCMP2_OK;
}

int mcmp2_bind_workspace(mcmp2_ctx *ctx, const mcmp2_dims *dims, void *dptr, size_t bytes)
{
    if (!ctx) return MCMP2_EINVAL;
    if (!dims_valid(dims)) return ctx->fail(MCMP2_EINVAL, "invalid dims");
    if (!dptr || (reinterpret_cast<uintptr_t>(dptr) & 255)) return ctx->fail(MCMP2_EINVAL, "workspace must be 256-byte aligned");
    const Layout L = make_layout(*dims, ctx->precision);
    if (bytes < L.total) return ctx->fail(MCMP2_ENOSPACE, "workspace %zu bytes < %zu needed", bytes, L.total);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->dims = *dims;
    ctx->L = L;
    ctx->ws = static_cast<char *>(dptr);
    ctx->ws_bytes = bytes;
    CK(cudaMemsetAsync(ctx->ws + L.red, 0, sizeof(ReduceScratch), ctx->stream), "clear reduction scratch");
    CK(cudaStreamSynchronize(ctx->stream), "bind sync");
    ctx->bound = true;
    ctx->loaded = ctx->walkers = false;
    ctx->drop_graph();
    return MCMP2_OK;
}

}  // extern "C"

namespace {

// Loads a system whose coefficients C have 4 n_L rows (L-alpha, L-beta,
// S-alpha, S-beta); n_comp = 2 marks a two-component system (C's small rows
// are zero and the step evaluates 2 x 2 blocks).
int load_system_impl(mcmp2_ctx *ctx, const mcmp2_basis *b, int n_occ, int n_vir, const double *C, const double *eps,
                     int n_comp)
{
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->bound) return ctx->fail(MCMP2_ENOTLOADED, "no workspace bound");
    const mcmp2_dims &d = ctx->dims;
    if (!b || !C || !eps || !b->centres || !b->weight || !b->shell_centre || !b->shell_l || !b->shell_alpha ||
        !b->shell_coef)
        return ctx->fail(MCMP2_EINVAL, "null pointer in system");
    if (b->n_centres != d.n_centres || n_occ != d.n_occ || n_vir != d.n_vir || b->n_shells < 1)
        return ctx->fail(MCMP2_EINVAL, "system sizes do not match the bound dims");
    // Expand shells to Cartesian functions.
    std::vector<int> fn_shell, fn_pow;
    for (int k = 0; k < b->n_shells; ++k) {
        const int l = b->shell_l[k];
        if (l < 0 || l > 2) return ctx->fail(MCMP2_EINVAL, "shell %d: l=%d not in 0..2", k, l);
        if (b->shell_centre[k] < 0 || b->shell_centre[k] >= b->n_centres)
            return ctx->fail(MCMP2_EINVAL, "shell %d: bad centre", k);
        if (!(b->shell_alpha[k] > 0.0) || !std::isfinite(b->shell_alpha[k]) || !std::isfinite(b->shell_coef[k]))
            return ctx->fail(MCMP2_EINVAL, "shell %d: bad exponent or coefficient", k);
        for (int c = 0; c < NCART[l]; ++c) {
            fn_shell.push_back(k);
            for (int j = 0; j < 3; ++j) fn_pow.push_back(CART[l][c][j]);
        }
    }
    const int nl = (int)fn_shell.size();
    if (nl != d.n_functions) return ctx->fail(MCMP2_EINVAL, "basis has %d functions, dims say %d", nl, d.n_functions);
    if (b->n_shells > nl) return ctx->fail(MCMP2_EINVAL, "too many shells");
    const int no = n_occ + n_vir;
    for (size_t i = 0; i < (size_t)4 * nl * no * 2; ++i)
        if (!std::isfinite(C[i])) return ctx->fail(MCMP2_ENONFINITE, "C has a non-finite entry");
    double homo = -INFINITY, lumo = INFINITY;
    for (int k = 0; k < no; ++k) {
        if (!std::isfinite(eps[k])) return ctx->fail(MCMP2_ENONFINITE, "eps has a non-finite entry");
        if (k < n_occ) homo = std::fmax(homo, eps[k]);
        else lumo = std::fmin(lumo, eps[k]);
    }
    if (!(lumo > homo)) return ctx->fail(MCMP2_EINVAL, "need max occupied eps < min virtual eps");
    for (int i = 0; i < b->n_centres; ++i) {
        for (int j = 0; j < 3; ++j)
            if (!std::isfinite(b->centres[3 * i + j])) return ctx->fail(MCMP2_ENONFINITE, "bad centre");
        if (!(b->weight[4 * i + 1] > 0.0) || !(b->weight[4 * i + 3] > 0.0) || !std::isfinite(b->weight[4 * i]) ||
            !std::isfinite(b->weight[4 * i + 2]))
            return ctx->fail(MCMP2_EINVAL, "centre %d: bad weight parameters", i);
    }
    // Weight function: c N(zeta) with N(zeta) = (2 zeta / pi)^{3/4} (Eq. basisSet).
    std::vector<double> wcoef(4 * (size_t)b->n_centres);
    for (int i = 0; i < b->n_centres; ++i) {
        const double *w = b->weight + 4 * i;
        wcoef[4 * i + 0] = w[0] * std::pow(2.0 * w[1] / M_PI, 0.75);
        wcoef[4 * i + 1] = w[1];
        wcoef[4 * i + 2] = w[2] * std::pow(2.0 * w[3] / M_PI, 0.75);
        wcoef[4 * i + 3] = w[3];
    }
    // N_g = Int Int g g / r12 in closed form: each pair of s Gaussians exp(-a r_A^2),
    // exp(-b r_B^2) contributes (pi/a)^{3/2} (pi/b)^{3/2} erf(sqrt(ab/(a+b)) R)/R.
    double Ng = 0.0;
    for (int i = 0; i < b->n_centres; ++i)
        for (int j = 0; j < b->n_centres; ++j) {
            const double *A = b->centres + 3 * i, *B = b->centres + 3 * j;
            const double R = std::sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) +
                                       (A[2] - B[2]) * (A[2] - B[2]));
            for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) {
                    const double ca = wcoef[4 * i + 2 * u], za = wcoef[4 * i + 2 * u + 1];
                    const double cb = wcoef[4 * j + 2 * v], zb = wcoef[4 * j + 2 * v + 1];
                    const double rho = za * zb / (za + zb);
                    const double f = R > 0.0 ? std::erf(std::sqrt(rho) * R) / R : 2.0 * std::sqrt(rho / M_PI);
                    Ng += ca * cb * std::pow(M_PI / za, 1.5) * std::pow(M_PI / zb, 1.5) * f;
                }
        }
    // Spinor-formation operands.  Large: WL[mu][c][k] = C^{L c}_{mu k}.  Small:
    // phi^S = sum_mu sum_s C^{S s}_{mu k} (sigma.grad)(g_mu e_s), so the
    // gradient component j of g_mu enters component c' with sigma_j[c'][s] C^{S s}.
    const double sig_re[3][2][2] = {{{0, 1}, {1, 0}}, {{0, 0}, {0, 0}}, {{1, 0}, {0, -1}}};
    const double sig_im[3][2][2] = {{{0, 0}, {0, 0}}, {{0, -1}, {1, 0}}, {{0, 0}, {0, 0}}};
    std::vector<double> WL((size_t)nl * 4 * no), WS((size_t)3 * nl * 4 * no);
    auto Cre = [&](int row, int k) { return C[((size_t)row * no + k) * 2]; };
    auto Cim = [&](int row, int k) { return C[((size_t)row * no + k) * 2 + 1]; };
    for (int mu = 0; mu < nl; ++mu)
        for (int c = 0; c < 2; ++c)
            for (int k = 0; k < no; ++k) {
                WL[(((size_t)mu * 2 + c) * no + k) * 2 + 0] = Cre(c * nl + mu, k);
                WL[(((size_t)mu * 2 + c) * no + k) * 2 + 1] = Cim(c * nl + mu, k);
            }
    for (int j = 0; j < 3; ++j)
        for (int mu = 0; mu < nl; ++mu)
            for (int cp = 0; cp < 2; ++cp)
                for (int k = 0; k < no; ++k) {
                    double re = 0.0, im = 0.0;
                    for (int s = 0; s < 2; ++s) {
                        const double sr = sig_re[j][cp][s], si = sig_im[j][cp][s];
                        const double cr = Cre((2 + s) * nl + mu, k), ci = Cim((2 + s) * nl + mu, k);
                        re += sr * cr - si * ci;
                        im += sr * ci + si * cr;
                    }
                    const size_t o = ((((size_t)j * nl + mu) * 2 + cp) * no + k) * 2;
                    WS[o] = re;
                    WS[o + 1] = im;
                }
    std::vector<double> shell_alpha(b->shell_alpha, b->shell_alpha + b->n_shells);
    std::vector<double> shell_coef(b->shell_coef, b->shell_coef + b->n_shells);
    std::vector<int> shell_centre(b->shell_centre, b->shell_centre + b->n_shells);

    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const Layout &L = ctx->L;
    cudaStream_t st = ctx->stream;
    auto h2d = [&](size_t off, const void *src, size_t n) {
        return cudaMemcpyAsync(ctx->ws + off, src, n, cudaMemcpyHostToDevice, st);
    };
    CK(h2d(L.centres, b->centres, sizeof(double) * 3 * b->n_centres), "copy centres");
    CK(h2d(L.wcoef, wcoef.data(), sizeof(double) * wcoef.size()), "copy weights");
    CK(h2d(L.shell_centre, shell_centre.data(), sizeof(int) * shell_centre.size()), "copy shells");
    CK(h2d(L.shell_alpha, shell_alpha.data(), sizeof(double) * shell_alpha.size()), "copy shells");
    CK(h2d(L.shell_coef, shell_coef.data(), sizeof(double) * shell_coef.size()), "copy shells");
    CK(h2d(L.fn_shell, fn_shell.data(), sizeof(int) * fn_shell.size()), "copy functions");
    CK(h2d(L.fn_pow, fn_pow.data(), sizeof(int) * fn_pow.size()), "copy functions");
    CK(h2d(L.eps, eps, sizeof(double) * no), "copy eps");
    CK(h2d(L.WL, WL.data(), sizeof(double) * WL.size()), "copy WL");
    CK(h2d(L.WS, WS.data(), sizeof(double) * WS.size()), "copy WS");
    CK(cudaStreamSynchronize(st), "load sync");

    DevSystem &S = ctx->sys;
    S.n_centres = b->n_centres;
    S.n_shells = b->n_shells;
    S.n_l = nl;
    S.n_occ = n_occ;
    S.n_vir = n_vir;
    S.n_orb = no;
    S.m = d.m;
    S.n_tau = d.n_tau;
    S.centres = ctx->at<double>(L.centres);
    S.wcoef = ctx->at<double>(L.wcoef);
    S.shell_centre = ctx->at<int>(L.shell_centre);
    S.shell_alpha = ctx->at<double>(L.shell_alpha);
    S.shell_coef = ctx->at<double>(L.shell_coef);
    S.fn_shell = ctx->at<int>(L.fn_shell);
    S.fn_pow = ctx->at<int>(L.fn_pow);
    S.eps = ctx->at<double>(L.eps);
    S.eps_homo = homo;
    S.eps_lumo = lumo;
    S.lambda = 2.0 * (lumo - homo);
    S.Ng = Ng;
    S.WL = ctx->at<double>(L.WL);
    S.WS = ctx->at<double>(L.WS);
    S.interaction = ctx->interaction;
    S.n_comp = n_comp;
    if (ctx->precision != MCMP2_FP64) {  // a two-component tile holds 32 pairs (4 operand rows each)
        ctx->L.tile_pairs = n_comp == 2 ? TILE_PAIRS_MIXED_2C : TILE_PAIRS_MIXED;
        ctx->L.n_tiles = (int)n_tiles_for(d.m, ctx->L.tile_pairs);
    }

    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, b->centres, sizeof(double) * 3 * b->n_centres);
    h = fnv1a(h, b->weight, sizeof(double) * 4 * b->n_centres);
    h = fnv1a(h, b->shell_centre, sizeof(int) * b->n_shells);
    h = fnv1a(h, b->shell_l, sizeof(int) * b->n_shells);
    h = fnv1a(h, b->shell_alpha, sizeof(double) * b->n_shells);
    h = fnv1a(h, b->shell_coef, sizeof(double) * b->n_shells);
    h = fnv1a(h, C, sizeof(double) * 2 * 4 * (size_t)nl * no);
    h = fnv1a(h, eps, sizeof(double) * no);
    h = fnv1a(h, &n_comp, sizeof(n_comp));
    // Cumulative masses of the weight function's Gaussians, for drawing initial positions.
    {
        std::vector<double> cdf(2 * (size_t)b->n_centres);
        double tot = 0.0;
        for (int i = 0; i < b->n_centres; ++i)
            for (int k = 0; k < 2; ++k) {
                const double c = wcoef[4 * i + 2 * k], z = wcoef[4 * i + 2 * k + 1];
                tot += std::fabs(c) * std::pow(M_PI / z, 1.5);
                cdf[2 * i + k] = tot;
            }
        for (auto &v : cdf) v /= tot;
        cdf.back() = 1.0;
        CK(cudaMemcpyAsync(ctx->ws + L.cdf, cdf.data(), cdf.size() * 8, cudaMemcpyHostToDevice, st), "copy mixture");
        CK(cudaStreamSynchronize(st), "load sync");
    }
    ctx->digest = h;
    ctx->loaded = true;
    ctx->drop_graph();  // kernel arguments captured by value (energies, lambda) change with the system
    if (ctx->precision == MCMP2_FP64) CK(prepare_f64(), "configure FP64 kernels");
    ctx->walkers = false;
    if (ctx->precision != MCMP2_FP64) {
        ctx->mixed.tf32 = ctx->precision == MCMP2_TF32;
        const int rc = mixed_prepare(ctx->mixed, S, L.mixed, ctx->ws, WL.data(), WS.data(), st, ctx->err);
        if (rc != MCMP2_OK) {
            ctx->loaded = false;
            return rc;
        }
    }
    return MCMP2_OK;
}

}  // namespace

extern "C" {

int mcmp2_load_system(mcmp2_ctx *ctx, const mcmp2_basis *b, int n_occ, int n_vir, const double *C,
                      const double *eps)
{
    CallRange range_("mcmp2_load_system");
    return load_system_impl(ctx, b, n_occ, n_vir, C, eps, 4);
}

int mcmp2_load_system_2c(mcmp2_ctx *ctx, const mcmp2_basis *b, int n_occ, int n_vir, const double *C2,
                         const double *eps)
{
    CallRange range_("mcmp2_load_system_2c");
    if (!ctx) return MCMP2_EINVAL;
    if (ctx->interaction != MCMP2_COULOMB)
        return ctx->fail(MCMP2_EUNSUPPORTED, "the Gaunt / Breit terms need the small components");
    if (!ctx->bound) return ctx->fail(MCMP2_ENOTLOADED, "no workspace bound");
    if (!C2) return ctx->fail(MCMP2_EINVAL, "null pointer in system");
    const size_t nl = (size_t)ctx->dims.n_functions, no = (size_t)n_occ + n_vir;
    if (n_occ != ctx->dims.n_occ || n_vir != ctx->dims.n_vir)
        return ctx->fail(MCMP2_EINVAL, "system sizes do not match the bound dims");
    // Rows alpha, beta of the two-component spinors become the large rows of a
    // four-component coefficient matrix whose small rows are zero.
    std::vector<double> C4(4 * nl * no * 2, 0.0);
    std::copy(C2, C2 + 2 * nl * no * 2, C4.begin());
    return load_system_impl(ctx, b, n_occ, n_vir, C4.data(), eps, 2);
}

}  // extern "C"

namespace {

int reset_stats(mcmp2_ctx *ctx)
{
    CK(cudaMemsetAsync(ctx->ws + ctx->L.stats, 0, sizeof(Stats), ctx->stream), "reset stats");
    return MCMP2_OK;
}

// The integrand engine for one step: from positions r and times (drawn or
// given) to I'_n in out_slot.  Optionally updates statistics and advances the step.
int step_integrand(mcmp2_ctx *ctx, const double *r, const double *tau_given, uint64_t seed, double *out_slot,
                   int update, bool advance, bool weights_ready = false, cudaStream_t st_in = nullptr,
                   cudaEvent_t *fixed_ev = nullptr, const DebugTile &dbg = DebugTile{}, bool times_ready = false)
{
    const Layout &L = ctx->L;
    const DevSystem &S = ctx->sys;
    cudaStream_t st = st_in ? st_in : ctx->stream;
    unsigned long long *step = ctx->at<unsigned long long>(L.step);
    double *a = ctx->at<double>(L.a);
    double *tau = ctx->at<double>(L.tau);
    double *scale = ctx->at<double>(L.scale);
    double *partials = ctx->at<double>(L.partials);
    if (!weights_ready) {
        CK(launch_pair_weights(S, r, a, st), "pair weights");
        ctx->launches += 1;
    }
    float *scale_f = ctx->precision != MCMP2_FP64 ? ctx->at<float>(L.scale_f) : nullptr;
    if (!times_ready) {
        CK(launch_times(S, step, seed, tau_given, tau, scale, scale_f, st), "imaginary times");
        ctx->launches += 1;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (fixed_ev) {
        ev[0] = fixed_ev[0];
        ev[1] = fixed_ev[1];
    } else if (ctx->timing) {
        CK(cudaEventCreate(&ev[0]), "event");
        CK(cudaEventCreate(&ev[1]), "event");
        ctx->pair_events.emplace_back(ev[0], ev[1]);
    }
    cudaEvent_t e0 = ev[0], e1 = ev[1];
    if (ctx->precision == MCMP2_FP64) {
        double *B = ctx->at<double>(L.B);
        double *phi = ctx->at<double>(L.phi);
        CK(launch_basis<double>(S, r, B, st), "basis values");
        CK(launch_spinors_f64(S, B, phi, st), "spinor formation");
        if (e0) CK(record_event(e0, st), "event");
        CK(launch_pairs_f64(S, phi, scale, a, partials, st, r, dbg), "pair-of-pairs tiles");
        if (e1) CK(record_event(e1, st), "event");
        ctx->launches += 4;
        ctx->pair_launches += 1;
    } else {
        int n_launch = 0, n_pair = 0;
        const int rc = mixed_step(ctx->mixed, S, L.mixed, ctx->ws, r, scale_f, a, partials, st, ctx->err,
                                  ev[0] ? ev : nullptr, &n_launch, &n_pair, dbg);
        if (rc != MCMP2_OK) return rc;
        ctx->launches += n_launch;
        ctx->pair_launches += n_pair;
    }
    CK(launch_reduce(S, partials, L.n_tiles, out_slot, ctx->at<Stats>(L.stats), update, advance ? step : nullptr,
                     ctx->at<ReduceScratch>(L.red), st,
                     ctx->precision != MCMP2_FP64 ? ctx->at<int>(L.mixed.flag) : nullptr),
       "step reduction");
    ctx->launches += 1;
    return MCMP2_OK;
}

bool all_finite(const double *x, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

}  // namespace

extern "C" {

int mcmp2_set_walkers(mcmp2_ctx *ctx, const double *r_host, uint64_t seed, int64_t burn_in)
{
    CallRange range_("mcmp2_set_walkers");
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->loaded) return ctx->fail(MCMP2_ENOTLOADED, "no system loaded");
    if (burn_in < 0) return ctx->fail(MCMP2_EINVAL, "burn_in < 0");
    const size_t n = (size_t)ctx->dims.m * 6;
    if (r_host && !all_finite(r_host, n)) return ctx->fail(MCMP2_ENONFINITE, "non-finite walker position");
    const Layout &L = ctx->L;
    cudaStream_t st = ctx->stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (r_host)
        CK(cudaMemcpyAsync(ctx->ws + L.r, r_host, n * sizeof(double), cudaMemcpyHostToDevice, st), "copy walkers");
    else
        CK(launch_initial_walkers(ctx->sys, ctx->at<double>(L.r), seed, ctx->at<double>(L.cdf), st), "initial draw");
    CK(cudaMemsetAsync(ctx->ws + L.step, 0, 8, st), "reset step");
    int rc = reset_stats(ctx);
    if (rc) return rc;
    ctx->delta = MCMP2_DELTA0;
    unsigned long long *step = ctx->at<unsigned long long>(L.step);
    unsigned long long *acc = ctx->at<unsigned long long>(L.burn_acc);
    int64_t done = 0;
    while (done < burn_in) {
        const int64_t len = std::min<int64_t>(MCMP2_ADAPT_WINDOW, burn_in - done);
        CK(cudaMemsetAsync(acc, 0, 8, st), "reset acceptance");
        for (int64_t i = 0; i < len; ++i) {
            CK(launch_metropolis(ctx->sys, ctx->at<double>(L.r), step, seed, ctx->delta, acc, nullptr, st),
               "metropolis");
            CK(launch_advance_step(step, st), "advance step");
        }
        if (len == MCMP2_ADAPT_WINDOW) {
            unsigned long long hacc = 0;
            CK(cudaMemcpyAsync(&hacc, acc, 8, cudaMemcpyDeviceToHost, st), "read acceptance");
            CK(cudaStreamSynchronize(st), "burn-in sync");
            const double a = (double)hacc / (double)((long)ctx->dims.m * MCMP2_ADAPT_WINDOW);
            double f = a / 0.5;
            if (f > 2.0) f = 2.0;
            if (f < 0.5) f = 0.5;
            ctx->delta = ctx->delta * f;
        }
        done += len;
    }
    CK(cudaStreamSynchronize(st), "set_walkers sync");
    ctx->walkers = true;
    return MCMP2_OK;
}

int mcmp2_run_steps(mcmp2_ctx *ctx, int64_t n, uint64_t seed, mcmp2_result *out)
{
    CallRange range_("mcmp2_run_steps");
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->walkers) return ctx->fail(MCMP2_ENOTLOADED, "walkers not set");
    if (n < 0) return ctx->fail(MCMP2_EINVAL, "n < 0");
    const Layout &L = ctx->L;
    cudaStream_t st = ctx->stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    Stats *stats = ctx->at<Stats>(L.stats);
    double *r = ctx->at<double>(L.r);
    // One step is captured once into a CUDA graph (its kernels read the step
    // counter from device memory, so the graph is the same for every step)
    // and replayed n times on the caller's stream.
    if (ctx->precision != MCMP2_FP64 && ctx->mixed.withhold_once_ns && n > 0) {
        // A pending test stall applies to one directly issued step.
        CK(launch_metropolis(ctx->sys, r, ctx->at<unsigned long long>(L.step), seed, ctx->delta, &stats->accepted,
                             ctx->at<double>(L.a), st),
           "metropolis");
        const int rc = step_integrand(ctx, r, nullptr, seed, ctx->at<double>(L.per_step), 1, true, true);
        if (rc) return rc;
        --n;
    }
    if (n > 0 && (!ctx->graph || ctx->graph_seed != seed || ctx->graph_delta != ctx->delta ||
                  ctx->graph_timing != ctx->timing)) {
        ctx->drop_graph();
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "capture stream");
        if (!ctx->side_stream) CK(cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking), "side stream");
        if (!ctx->fork_ev) CK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming), "event");
        if (!ctx->join_ev) CK(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming), "event");
        if (ctx->timing && !ctx->gev[0]) {
            CK(cudaEventCreate(&ctx->gev[0]), "event");
            CK(cudaEventCreate(&ctx->gev[1]), "event");
        }
        const long long l0 = ctx->launches, p0 = ctx->pair_launches;
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        // The imaginary times depend only on the step counter: a side branch
        // draws them while the Metropolis move runs.
        int rc = ctx->cuda(cudaEventRecord(ctx->fork_ev, ctx->cap_stream), "fork");
        if (rc == MCMP2_OK) rc = ctx->cuda(cudaStreamWaitEvent(ctx->side_stream, ctx->fork_ev, 0), "fork");
        if (rc == MCMP2_OK)
            rc = ctx->cuda(launch_times(ctx->sys, ctx->at<unsigned long long>(L.step), seed, nullptr,
                                        ctx->at<double>(L.tau), ctx->at<double>(L.scale),
                                        ctx->precision != MCMP2_FP64 ? ctx->at<float>(L.scale_f) : nullptr,
                                        ctx->side_stream),
                           "imaginary times");
        if (rc == MCMP2_OK) rc = ctx->cuda(cudaEventRecord(ctx->join_ev, ctx->side_stream), "join");
        if (rc == MCMP2_OK)
            rc = ctx->cuda(launch_metropolis(ctx->sys, r, ctx->at<unsigned long long>(L.step), seed, ctx->delta,
                                             &stats->accepted, ctx->at<double>(L.a), ctx->cap_stream),
                           "metropolis");
        if (rc == MCMP2_OK) rc = ctx->cuda(cudaStreamWaitEvent(ctx->cap_stream, ctx->join_ev, 0), "join");
        ctx->launches += 2;
        if (rc == MCMP2_OK)
            rc = step_integrand(ctx, r, nullptr, seed, ctx->at<double>(L.per_step), 1, true, true, ctx->cap_stream,
                                ctx->timing ? ctx->gev : nullptr, DebugTile{}, true);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &g);
        ctx->graph_launches = ctx->launches - l0;
        ctx->graph_pair_launches = ctx->pair_launches - p0;
        ctx->launches = l0;
        ctx->pair_launches = p0;
        if (rc != MCMP2_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CK(ec, "end capture");
        const cudaError_t ei = cudaGraphInstantiate(&ctx->graph, g, 0);
        cudaGraphDestroy(g);
        CK(ei, "instantiate step graph");
        ctx->graph_seed = seed;
        ctx->graph_delta = ctx->delta;
        ctx->graph_timing = ctx->timing;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (ctx->timing) CK(ctx->collect_graph_time(), "event time");  // before the events are re-recorded
        CK(cudaGraphLaunch(ctx->graph, st), "launch step graph");
        ctx->launches += ctx->graph_launches;
        ctx->pair_launches += ctx->graph_pair_launches;
        if (ctx->timing) ctx->gev_pending = true;
    }
    if (out) {
        Stats h;
        CK(cudaMemcpyAsync(&h, stats, sizeof(Stats), cudaMemcpyDeviceToHost, st), "read statistics");
        CK(cudaStreamSynchronize(st), "run_steps sync");
        out->steps = h.steps;
        out->n_blocks = h.n_blocks;
        out->energy = h.n_blocks ? h.mean : 0.0;
        out->variance = h.n_blocks ? h.m2 / (double)h.n_blocks : 0.0;
        out->error = h.n_blocks ? std::sqrt(out->variance) / std::sqrt((double)h.n_blocks) : 0.0;
        out->mean_all = h.steps ? h.all_sum / (double)h.steps : 0.0;
        out->last_step = h.last;
        out->accept_rate = h.steps ? (double)h.accepted / ((double)h.steps * ctx->dims.m) : 0.0;
        if (!std::isfinite(h.all_sum) || !std::isfinite(h.mean) || !std::isfinite(h.m2))
            return ctx->fail(MCMP2_ENONFINITE, "a step estimate is not finite");
    }
    if (ctx->precision != MCMP2_FP64 && out) {
        const int rc = mixed_check_flag(ctx->L.mixed, ctx->ws, st, ctx->err);
        if (rc) return rc;
    }
    return MCMP2_OK;
}

int mcmp2_eval_fixed(mcmp2_ctx *ctx, int64_t n, const double *r_host, const double *tau_host, double *out)
{
    CallRange range_("mcmp2_eval_fixed");
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->loaded) return ctx->fail(MCMP2_ENOTLOADED, "no system loaded");
    if (n < 0 || (n > 0 && (!r_host || !tau_host || !out))) return ctx->fail(MCMP2_EINVAL, "bad replay arguments");
    const int m = ctx->dims.m, nt = ctx->dims.n_tau;
    if (!all_finite(r_host, (size_t)n * m * 6)) return ctx->fail(MCMP2_ENONFINITE, "non-finite position");
    for (int64_t i = 0; i < n * nt; ++i)
        if (!(tau_host[i] >= 0.0) || !std::isfinite(tau_host[i]))
            return ctx->fail(MCMP2_EINVAL, "imaginary times must be finite and >= 0");
    const Layout &L = ctx->L;
    cudaStream_t st = ctx->stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    double *sr = ctx->at<double>(L.stage_r), *stau = ctx->at<double>(L.stage_tau);
    double *slots = ctx->at<double>(L.per_step);
    for (int64_t s0 = 0; s0 < n; s0 += REPLAY_CHUNK) {
        const int len = (int)std::min<int64_t>(REPLAY_CHUNK, n - s0);
        CK(cudaMemcpyAsync(sr, r_host + (size_t)s0 * m * 6, sizeof(double) * len * m * 6, cudaMemcpyHostToDevice, st),
           "copy positions");
        CK(cudaMemcpyAsync(stau, tau_host + (size_t)s0 * nt, sizeof(double) * len * nt, cudaMemcpyHostToDevice, st),
           "copy times");
        for (int j = 0; j < len; ++j) {
            const int rc = step_integrand(ctx, sr + (size_t)j * m * 6, stau + (size_t)j * nt, 0, slots + j, 0, false);
            if (rc) return rc;
        }
        CK(cudaMemcpyAsync(out + s0, slots, sizeof(double) * len, cudaMemcpyDeviceToHost, st), "copy results");
        CK(cudaStreamSynchronize(st), "replay sync");
    }
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(out[i])) {
            // A step whose kernels gave up on a wait reports NaN: name the time-out if that is why.
            if (ctx->precision != MCMP2_FP64) {
                const int rc = mixed_check_flag(ctx->L.mixed, ctx->ws, st, ctx->err);
                if (rc) return rc;
            }
            return ctx->fail(MCMP2_ENONFINITE, "step %lld is not finite", (long long)i);
        }
    return MCMP2_OK;
}

int mcmp2_backward(mcmp2_ctx *ctx, int64_t n, const double *r_host, const double *tau_host, double *energy_host,
                   double *d_eps_host, double *d_C_host)
{
    CallRange range_("mcmp2_backward");
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->loaded) return ctx->fail(MCMP2_ENOTLOADED, "no system loaded");
    if (ctx->precision != MCMP2_FP64) return ctx->fail(MCMP2_EUNSUPPORTED, "the adjoint runs in the FP64 form");
    if (ctx->interaction != MCMP2_COULOMB)
        return ctx->fail(MCMP2_EUNSUPPORTED, "the adjoint covers the Coulomb interaction");
    if (ctx->sys.n_comp != 4) return ctx->fail(MCMP2_EUNSUPPORTED, "the adjoint covers four-component systems");
    if (n < 1 || !r_host || !tau_host || !d_eps_host || !d_C_host) return ctx->fail(MCMP2_EINVAL, "bad backward arguments");
    const int m = ctx->dims.m, nt = ctx->dims.n_tau;
    if (!all_finite(r_host, (size_t)n * m * 6)) return ctx->fail(MCMP2_ENONFINITE, "non-finite position");
    for (int64_t i = 0; i < n * nt; ++i)
        if (!(tau_host[i] >= 0.0) || !std::isfinite(tau_host[i]))
            return ctx->fail(MCMP2_EINVAL, "imaginary times must be finite and >= 0");
    const Layout &L = ctx->L;
    const DevSystem &S = ctx->sys;
    cudaStream_t st = ctx->stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int nl = S.n_l, no = S.n_orb;
    CK(cudaMemsetAsync(ctx->ws + L.GWL, 0, (size_t)nl * 4 * no * 8, st), "zero gradients");
    CK(cudaMemsetAsync(ctx->ws + L.GWS, 0, (size_t)3 * nl * 4 * no * 8, st), "zero gradients");
    CK(cudaMemsetAsync(ctx->ws + L.d_eps, 0, (size_t)no * 8, st), "zero gradients");
    const double npairs = 0.5 * (double)m * (double)(m - 1);
    const double norm = 1.0 / ((double)n * nt * npairs);
    double *sr = ctx->at<double>(L.stage_r), *stau = ctx->at<double>(L.stage_tau);
    double *slots = ctx->at<double>(L.per_step);
    double *a = ctx->at<double>(L.a), *tau = ctx->at<double>(L.tau), *scale = ctx->at<double>(L.scale);
    double *B = ctx->at<double>(L.B), *phi = ctx->at<double>(L.phi), *partials = ctx->at<double>(L.partials);
    unsigned long long *step = ctx->at<unsigned long long>(L.step);
    std::vector<double> per(n);
    for (int64_t s0 = 0; s0 < n; s0 += REPLAY_CHUNK) {
        const int len = (int)std::min<int64_t>(REPLAY_CHUNK, n - s0);
        CK(cudaMemcpyAsync(sr, r_host + (size_t)s0 * m * 6, sizeof(double) * len * m * 6, cudaMemcpyHostToDevice, st),
           "copy positions");
        CK(cudaMemcpyAsync(stau, tau_host + (size_t)s0 * nt, sizeof(double) * len * nt, cudaMemcpyHostToDevice, st),
           "copy times");
        for (int j = 0; j < len; ++j) {
            const double *rj = sr + (size_t)j * m * 6;
            CK(launch_pair_weights(S, rj, a, st), "pair weights");
            CK(launch_times(S, step, 0, stau + (size_t)j * nt, tau, scale, nullptr, st), "imaginary times");
            CK(launch_basis<double>(S, rj, B, st), "basis values");
            CK(launch_spinors_f64(S, B, phi, st), "spinor formation");
            for (int t = 0; t < nt; ++t) {
                CK(cudaMemsetAsync(ctx->ws + L.Ybar, 0, (size_t)8 * m * no * 16, st), "zero adjoint");
                CK(launch_adjoint_time(S, B, phi, scale, tau, a, t, norm, ctx->at<double>(L.Ybar), ctx->at<double>(L.Ys),
                                       partials, ctx->at<double>(L.GWL), ctx->at<double>(L.GWS),
                                       ctx->at<double>(L.d_eps), st),
                   "adjoint");
            }
            CK(launch_reduce(S, partials, L.n_tiles, slots + j, ctx->at<Stats>(L.stats), 0, nullptr,
                             ctx->at<ReduceScratch>(L.red), st),
               "reduce");
        }
        CK(cudaMemcpyAsync(per.data() + s0, slots, sizeof(double) * len, cudaMemcpyDeviceToHost, st), "copy results");
        CK(cudaStreamSynchronize(st), "backward sync");
    }
    std::vector<double> gwl((size_t)nl * 4 * no), gws((size_t)3 * nl * 4 * no);
    CK(cudaMemcpyAsync(gwl.data(), ctx->ws + L.GWL, gwl.size() * 8, cudaMemcpyDeviceToHost, st), "copy gradients");
    CK(cudaMemcpyAsync(gws.data(), ctx->ws + L.GWS, gws.size() * 8, cudaMemcpyDeviceToHost, st), "copy gradients");
    CK(cudaMemcpyAsync(d_eps_host, ctx->ws + L.d_eps, (size_t)no * 8, cudaMemcpyDeviceToHost, st), "copy gradients");
    CK(cudaStreamSynchronize(st), "backward sync");
    // Fold dE/dW back to dE/dC: W^{Lc}_{mu k} = C^{Lc}_{mu k}; W^{Sc'}_{(j,mu) k} =
    // sum_s sigma_j[c'][s] C^{Ss}_{mu k}, so dE/dC^{Ss} = sum_{j,c'} conj(sigma_j[c'][s]) dE/dW^{Sc'}.
    const double sig_re[3][2][2] = {{{0, 1}, {1, 0}}, {{0, 0}, {0, 0}}, {{1, 0}, {0, -1}}};
    const double sig_im[3][2][2] = {{{0, 0}, {0, 0}}, {{0, -1}, {1, 0}}, {{0, 0}, {0, 0}}};
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < nl; ++mu)
            for (int k = 0; k < no; ++k) {
                const size_t src = (((size_t)mu * 2 + c) * no + k) * 2, dst = (((size_t)c * nl + mu) * no + k) * 2;
                d_C_host[dst] = gwl[src];
                d_C_host[dst + 1] = gwl[src + 1];
            }
    for (int s_ = 0; s_ < 2; ++s_)
        for (int mu = 0; mu < nl; ++mu)
            for (int k = 0; k < no; ++k) {
                double re = 0.0, im = 0.0;
                for (int j = 0; j < 3; ++j)
                    for (int cp = 0; cp < 2; ++cp) {
                        const size_t src = ((((size_t)j * nl + mu) * 2 + cp) * no + k) * 2;
                        const double gr = gws[src], gi = gws[src + 1];
                        const double sr_ = sig_re[j][cp][s_], si = -sig_im[j][cp][s_];  // conj(sigma)
                        re += sr_ * gr - si * gi;
                        im += sr_ * gi + si * gr;
                    }
                const size_t dst = (((size_t)(2 + s_) * nl + mu) * no + k) * 2;
                d_C_host[dst] = re;
                d_C_host[dst + 1] = im;
            }
    if (energy_host) {
        double e = 0.0, c = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double y = per[i] - c, t = e + y;
            c = (t - e) - y;
            e = t;
        }
        *energy_host = e / (double)n;
    }
    for (int k = 0; k < no; ++k)
        if (!std::isfinite(d_eps_host[k])) return ctx->fail(MCMP2_ENONFINITE, "non-finite gradient");
    return MCMP2_OK;
}

int mcmp2_get_walkers(mcmp2_ctx *ctx, double *r_host, double *delta_host)
{
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->walkers) return ctx->fail(MCMP2_ENOTLOADED, "walkers not set");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (r_host) {
        CK(cudaMemcpyAsync(r_host, ctx->ws + ctx->L.r, sizeof(double) * 6 * ctx->dims.m, cudaMemcpyDeviceToHost,
                           ctx->stream),
           "copy walkers");
        CK(cudaStreamSynchronize(ctx->stream), "sync");
    }
    if (delta_host) *delta_host = ctx->delta;
    return MCMP2_OK;
}

int mcmp2_debug_partials(mcmp2_ctx *ctx, double *out, size_t capacity, int *n_tiles, int *tile_pairs)
{
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->loaded) return ctx->fail(MCMP2_ENOTLOADED, "no system loaded");
    if (n_tiles) *n_tiles = ctx->L.n_tiles;
    if (tile_pairs) *tile_pairs = ctx->L.tile_pairs;
    const size_t need = (size_t)ctx->L.n_tiles * ctx->dims.n_tau;
    if (!out) return MCMP2_OK;
    if (capacity < need) return ctx->fail(MCMP2_ENOSPACE, "need %zu doubles", need);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(out, ctx->ws + ctx->L.partials, need * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
       "copy partials");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    return MCMP2_OK;
}

int mcmp2_debug_elements(mcmp2_ctx *ctx, const double *r_host, const double *tau_host, int bp, int bq,
                         double *out_host, size_t capacity, double *step_host, int *tile_pairs)
{
    CallRange range_("mcmp2_debug_elements");
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->loaded) return ctx->fail(MCMP2_ENOTLOADED, "no system loaded");
    const int m = ctx->dims.m, nt = ctx->dims.n_tau, tp = ctx->L.tile_pairs;
    if (tile_pairs) *tile_pairs = tp;
    if (!r_host || !tau_host || !out_host) return ctx->fail(MCMP2_EINVAL, "bad element-record arguments");
    const int nb = pair_blocks(m, tp);
    if (bp < 0 || bq < bp || bq >= nb) return ctx->fail(MCMP2_EINVAL, "tile (%d, %d) outside 0 <= bp <= bq < %d", bp, bq, nb);
    const size_t need = (size_t)nt * tp * tp;
    if (capacity < need) return ctx->fail(MCMP2_ENOSPACE, "need %zu doubles", need);
    if (!all_finite(r_host, (size_t)m * 6)) return ctx->fail(MCMP2_ENONFINITE, "non-finite position");
    for (int i = 0; i < nt; ++i)
        if (!(tau_host[i] >= 0.0) || !std::isfinite(tau_host[i]))
            return ctx->fail(MCMP2_EINVAL, "imaginary times must be finite and >= 0");
    const Layout &L = ctx->L;
    cudaStream_t st = ctx->stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    double *sr = ctx->at<double>(L.stage_r), *stau = ctx->at<double>(L.stage_tau);
    CK(cudaMemcpyAsync(sr, r_host, sizeof(double) * m * 6, cudaMemcpyHostToDevice, st), "copy positions");
    CK(cudaMemcpyAsync(stau, tau_host, sizeof(double) * nt, cudaMemcpyHostToDevice, st), "copy times");
    CK(cudaMemsetAsync(ctx->ws + L.elements, 0, need * sizeof(double), st), "clear element record");
    DebugTile dbg;
    dbg.out = ctx->at<double>(L.elements);
    dbg.bp = bp;
    dbg.bq = bq;
    double *slot = ctx->at<double>(L.per_step);
    const int rc = step_integrand(ctx, sr, stau, 0, slot, 0, false, false, nullptr, nullptr, dbg);
    if (rc) return rc;
    double step = 0.0;
    CK(cudaMemcpyAsync(out_host, dbg.out, need * sizeof(double), cudaMemcpyDeviceToHost, st), "copy elements");
    CK(cudaMemcpyAsync(&step, slot, sizeof(double), cudaMemcpyDeviceToHost, st), "copy step");
    CK(cudaStreamSynchronize(st), "element record sync");
    if (ctx->precision != MCMP2_FP64) {
        const int rc2 = mixed_check_flag(ctx->L.mixed, ctx->ws, st, ctx->err);
        if (rc2) return rc2;
    }
    if (step_host) *step_host = step;
    return MCMP2_OK;
}

int mcmp2_profile(mcmp2_ctx *ctx, int mode, mcmp2_profile_counters *out)
{
    if (!ctx) return MCMP2_EINVAL;
    if (mode == 1 || mode == 2) {
        drop_events(ctx);
        ctx->launches = ctx->pair_launches = 0;
        CK(ctx->collect_graph_time(), "event time");
        ctx->graph_pair_ms = 0.0;
        ctx->timing = (mode == 1);
        return MCMP2_OK;
    }
    if (mode != 0 || !out) return ctx->fail(MCMP2_EINVAL, "bad profile mode");
    CK(ctx->collect_graph_time(), "event time");
    out->launches = ctx->launches;
    out->pair_launches = ctx->pair_launches;
    double ms = 0.0;
    if (!ctx->pair_events.empty()) {
        CK(cudaStreamSynchronize(ctx->stream), "sync");
        for (auto &ev : ctx->pair_events) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, ev.first, ev.second), "event time");
            ms += t;
        }
    }
    out->pair_ms = ms + ctx->graph_pair_ms;
    return MCMP2_OK;
}

int mcmp2_set_interaction(mcmp2_ctx *ctx, int interaction)
{
    if (!ctx) return MCMP2_EINVAL;
    if (interaction != MCMP2_COULOMB && interaction != MCMP2_GAUNT && interaction != MCMP2_BREIT)
        return ctx->fail(MCMP2_EINVAL, "unknown interaction");
    if (interaction != MCMP2_COULOMB && ctx->loaded && ctx->sys.n_comp == 2)
        return ctx->fail(MCMP2_EUNSUPPORTED, "the Gaunt / Breit terms need the small components");
    ctx->interaction = interaction;
    ctx->sys.interaction = interaction;
    ctx->drop_graph();  // the captured step holds the system by value
    return MCMP2_OK;
}

int mcmp2_test_stall_next(mcmp2_ctx *ctx, double wait_limit_s)
{
    if (!ctx) return MCMP2_EINVAL;
    if (ctx->precision == MCMP2_FP64) return ctx->fail(MCMP2_EUNSUPPORTED, "the hook applies to the tensor-core forms");
    if (!(wait_limit_s > 0.0) || wait_limit_s > 10.0) return ctx->fail(MCMP2_EINVAL, "wait limit must be in (0, 10] s");
    ctx->mixed.withhold_once_ns = (unsigned long long)(wait_limit_s * 1e9);
    ctx->drop_graph();  // the next step is issued directly, not replayed
    return MCMP2_OK;
}

namespace {
// Digest a checkpoint carries: the system's, extended by the interaction, so a
// walk restores only into the same system with the same integrand.
uint64_t run_digest(const mcmp2_ctx *ctx)
{
    if (ctx->interaction == MCMP2_COULOMB) return ctx->digest;  // unchanged for the paper's operator
    return fnv1a(ctx->digest, &ctx->interaction, sizeof(ctx->interaction));
}
}  // namespace

int mcmp2_checkpoint_bytes(const mcmp2_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return MCMP2_EINVAL;
    *bytes = sizeof(Checkpoint) + sizeof(double) * 6 * (size_t)ctx->dims.m;
    return MCMP2_OK;
}

int mcmp2_checkpoint(mcmp2_ctx *ctx, void *buf, size_t capacity)
{
    CallRange range_("mcmp2_checkpoint");
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->walkers) return ctx->fail(MCMP2_ENOTLOADED, "walkers not set");
    size_t need = 0;
    mcmp2_checkpoint_bytes(ctx, &need);
    if (!buf || capacity < need) return ctx->fail(MCMP2_ENOSPACE, "checkpoint needs %zu bytes", need);
    Checkpoint ck{};
    ck.magic = CK_MAGIC;
    ck.version = 1;
    ck.dims = ctx->dims;
    ck.digest = run_digest(ctx);
    ck.delta = ctx->delta;
    cudaStream_t st = ctx->stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(&ck.step, ctx->ws + ctx->L.step, 8, cudaMemcpyDeviceToHost, st), "copy step");
    CK(cudaMemcpyAsync(&ck.stats, ctx->ws + ctx->L.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st), "copy stats");
    CK(cudaMemcpyAsync(static_cast<char *>(buf) + sizeof(Checkpoint), ctx->ws + ctx->L.r,
                       sizeof(double) * 6 * ctx->dims.m, cudaMemcpyDeviceToHost, st),
       "copy walkers");
    CK(cudaStreamSynchronize(st), "sync");
    std::memcpy(buf, &ck, sizeof(ck));
    return MCMP2_OK;
}

int mcmp2_restore(mcmp2_ctx *ctx, const void *buf, size_t bytes)
{
    CallRange range_("mcmp2_restore");
    if (!ctx) return MCMP2_EINVAL;
    if (!ctx->loaded) return ctx->fail(MCMP2_ENOTLOADED, "no system loaded");
    if (!buf || bytes < sizeof(Checkpoint)) return ctx->fail(MCMP2_EINVAL, "checkpoint truncated");
    Checkpoint ck;
    std::memcpy(&ck, buf, sizeof(ck));
    if (ck.magic != CK_MAGIC || ck.version != 1) return ctx->fail(MCMP2_EINVAL, "not a checkpoint");
    if (std::memcmp(&ck.dims, &ctx->dims, sizeof(mcmp2_dims)) != 0) return ctx->fail(MCMP2_EINVAL, "dims differ");
    if (ck.digest != run_digest(ctx))
        return ctx->fail(MCMP2_EINVAL, "checkpoint belongs to another system or interaction");
    const size_t need = sizeof(Checkpoint) + sizeof(double) * 6 * (size_t)ctx->dims.m;
    if (bytes < need) return ctx->fail(MCMP2_EINVAL, "checkpoint truncated");
    const double *r = reinterpret_cast<const double *>(static_cast<const char *>(buf) + sizeof(Checkpoint));
    if (!all_finite(r, 6 * (size_t)ctx->dims.m) || !std::isfinite(ck.delta))
        return ctx->fail(MCMP2_ENONFINITE, "checkpoint holds non-finite values");
    cudaStream_t st = ctx->stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(ctx->ws + ctx->L.step, &ck.step, 8, cudaMemcpyHostToDevice, st), "copy step");
    CK(cudaMemcpyAsync(ctx->ws + ctx->L.stats, &ck.stats, sizeof(Stats), cudaMemcpyHostToDevice, st), "copy stats");
    CK(cudaMemcpyAsync(ctx->ws + ctx->L.r, r, sizeof(double) * 6 * ctx->dims.m, cudaMemcpyHostToDevice, st),
       "copy walkers");
    CK(cudaStreamSynchronize(st), "sync");
    ctx->delta = ck.delta;
    ctx->walkers = true;
    return MCMP2_OK;
}

}  // extern "C"
