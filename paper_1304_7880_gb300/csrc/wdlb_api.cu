// C ABI of the WDLB library (declared in include/wdlb.h): context lifetime,
// workspace layout, host tables, time stepping with CUDA-graph replay, FP64
// reductions and host transfers.  All arithmetic of the method runs in the
// kernels of wdlb_kernels.cuh; this file only validates, lays out memory and
// enqueues work on the context stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/wdlb.h"
#include "wdlb_launch.h"
#include "wdlb_tables.h"

using namespace wdlb;

namespace {

constexpr int kGraphChunk = 50;   // steps per captured graph (even: buffer parity preserved)

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// ---------------------------------------------------------------------------
// Tables (Sec. 3 ball of the smeared density; contact shell of Eq. campoc).
// ---------------------------------------------------------------------------
struct Tables {
    std::vector<int> ball;    // 3 per vector
    std::vector<int> shell;   // 3 per vector, +e and -e adjacent
    double wshell = 0.0;
};

struct Layout {
    size_t f[2], nu, hb, cprev, tprev, nscale, stage, snap, partial, result, status, shell_e, shell_k, ball, total;
};

int storage_bytes(int storage) { return storage == WDLB_STORE_F64 ? 8 : (storage == WDLB_STORE_F32 ? 4 : 2); }
int compute_bytes(int storage) { return storage == WDLB_STORE_F64 ? 8 : 4; }

Layout layout_for(long long N, long long Npad, int storage, int nshell, int nball)
{
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t sS = storage_bytes(storage), sT = compute_bytes(storage);
    L.f[0] = take(NQ * Npad * sS);
    L.f[1] = take(NQ * Npad * sS);
    L.nu = take(Npad * 4 * sT);
    L.hb = take(Npad * sT);
    L.cprev = take(3 * Npad * sT);
    L.tprev = take(Npad * sT);
    L.nscale = take(Npad * sT);
    L.stage = take(4 * N * sizeof(double));
    L.snap = take(N * sizeof(double));
    L.partial = take(kStatBlocks * 6 * sizeof(double));
    L.result = take(16 * sizeof(double));
    L.status = take(16 * sizeof(int));
    L.shell_e = take(std::max(nshell, 1) * sizeof(int4));
    L.shell_k = take(std::max(nshell, 1) * 4 * sT);
    L.ball = take(std::max(nball, 1) * sizeof(int4));
    L.total = off;
    return L;
}

const Launchers &launchers_for(int storage)
{
    if (storage == WDLB_STORE_F64) return launchers_f64();
    if (storage == WDLB_STORE_F32) return launchers_f32();
    return launchers_f16();
}

}  // namespace

struct wdlb_ctx {
    wdlb_lattice lat{};
    int walls = 0;
    double sigma = 0, tau = 0, g[3] = {0, 0, 0};
    wdlb_options opt{};
    long long N = 0, Npad = 0;
    Tables tab;
    KParams kp{};
    DevBufs dev{};
    Layout lay{};
    char *base = nullptr;
    bool owns_base = false;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    int cur = 0;
    bool initialised = false;
    int64_t steps = 0;
    int64_t launches = 0;
    double last_residual = NAN;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> prof_events;   // event pool of wdlb_profile_step
    const Launchers *L = nullptr;
    std::string err;
};

namespace {

std::string g_create_error;

wdlb_status fail(wdlb_ctx *ctx, wdlb_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_create_error = buf;
    return s;
}

wdlb_status cuda_fail(wdlb_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, WDLB_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define WDLB_CUDA(ctx, call)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

wdlb_status validate(wdlb_lattice lat, double sigma, int32_t walls, const wdlb_options *opt)
{
    if (lat.nx < 1 || lat.ny < 1 || lat.nz < 1) return WDLB_ERR_ARG;
    if (walls != WDLB_WALLS_NONE && walls != WDLB_WALLS_Z) return WDLB_ERR_ARG;
    if (walls == WDLB_WALLS_Z && lat.nz < 3) return WDLB_ERR_ARG;
    long long N = (long long)lat.nx * lat.ny * lat.nz;
    if (N >= (1LL << 31) / 32) return WDLB_ERR_ARG;
    if (!(sigma >= 1.0 && sigma <= 8.0)) return WDLB_ERR_ARG;
    if (opt) {
        if (opt->closure < 0 || opt->closure > 2) return WDLB_ERR_ARG;
        if (opt->omega_mode < 0 || opt->omega_mode > 1) return WDLB_ERR_ARG;
        if (opt->storage < 0 || opt->storage > 2) return WDLB_ERR_ARG;
        if (!(opt->n_ref >= 0.0) || !std::isfinite(opt->k_cross)) return WDLB_ERR_ARG;
    }
    return WDLB_OK;
}

wdlb_status check_status_word(wdlb_ctx *ctx)
{
    int h = 0;
    WDLB_CUDA(ctx, cudaMemcpyAsync(&h, ctx->dev.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    WDLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) return fail(ctx, WDLB_ERR_UNSTABLE, "non-physical state: smeared packing fraction >= 1 or density not finite/positive");
    return WDLB_OK;
}

void set_params(wdlb_ctx *ctx)
{
    KParams &p = ctx->kp;
    p.nx = ctx->lat.nx;
    p.ny = ctx->lat.ny;
    p.nz = ctx->lat.nz;
    p.walls = ctx->walls;
    p.N = (int)ctx->N;
    p.Npad = (int)ctx->Npad;
    p.nshell = (int)(ctx->tab.shell.size() / 3);
    p.nball = (int)(ctx->tab.ball.size() / 3);
    p.closure = ctx->opt.closure;
    p.omega_mode = ctx->opt.omega_mode;
    p.interactions = ctx->opt.interactions ? 1 : 0;
    for (int d = 0; d < 3; d++) p.g[d] = ctx->g[d];
    p.tau = ctx->tau;
    p.omega = 1.0 / ctx->tau;
    p.k_cross = ctx->opt.k_cross;
    p.sig2 = ctx->sigma * ctx->sigma;
    p.beta = 2.0 * p.sig2 * std::sqrt(CS2 / M_PI);
    p.wshell = ctx->tab.wshell;
    p.chi_of_n = M_PI * ctx->sigma * ctx->sigma * ctx->sigma / 6.0;
    p.c_half = p.chi_of_n / (2.0 * std::max(p.nball, 1));
    p.h_pred = KAPPA * p.beta / 6.0;
    const double s2 = 2.0 * ctx->sigma;
    p.s2 = (std::fabs(s2 - std::round(s2)) < 1e-12) ? (int)std::lround(s2) : 0;
    p.tiled = 0;
    // n_off / ref_ng are set at init (they may depend on the initial state)
}

void set_reference(wdlb_ctx *ctx, double n_ref)
{
    KParams &p = ctx->kp;
    p.n_off = n_ref;
    p.ref_ng = n_ref * contact_g_host(ctx->opt.closure, p.chi_of_n * n_ref);
    p.h_off = 0.5 * p.chi_of_n * p.n_off;
}

void drop_graphs(wdlb_ctx *ctx)
{
    for (auto &g : ctx->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

wdlb_status init_from_stage(wdlb_ctx *ctx, const double *d_n, const double *d_u)
{
    double n_ref = ctx->opt.n_ref;
    if (n_ref <= 0.0) {
        cudaError_t e = launch_sum_density(ctx->kp, d_n, ctx->dev.partial, ctx->dev.result, ctx->stream,
                                           &ctx->launches);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sum density");
        double sum = 0.0;
        WDLB_CUDA(ctx, cudaMemcpyAsync(&sum, ctx->dev.result, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        WDLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        long long fluid = ctx->walls ? (long long)ctx->lat.nx * ctx->lat.ny * (ctx->lat.nz - 2) : ctx->N;
        n_ref = sum / double(fluid);
        if (!(n_ref > 0.0) || !std::isfinite(n_ref)) return fail(ctx, WDLB_ERR_ARG, "initial density must be positive");
    }
    set_reference(ctx, n_ref);
    drop_graphs(ctx);   // kernel parameters changed
    ctx->cur = 0;
    WDLB_CUDA(ctx, cudaMemsetAsync(ctx->dev.status, 0, sizeof(int), ctx->stream));
    WDLB_CUDA(ctx, cudaMemsetAsync(ctx->dev.snap, 0, ctx->N * sizeof(double), ctx->stream));
    cudaError_t e = ctx->L->init(ctx->kp, ctx->dev, ctx->cur, d_n, d_u, ctx->stream, &ctx->launches);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "init kernel");
    ctx->initialised = true;
    ctx->steps = 0;
    ctx->last_residual = NAN;
    return WDLB_OK;
}

wdlb_status step_direct(wdlb_ctx *ctx, int64_t n)
{
    for (int64_t s = 0; s < n; s++) {
        cudaError_t e = ctx->L->step(ctx->kp, ctx->dev, ctx->cur, ctx->stream, &ctx->launches);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step kernels");
        ctx->cur ^= 1;
    }
    return WDLB_OK;
}

wdlb_status ensure_graph(wdlb_ctx *ctx)
{
    int c = ctx->cur;
    if (ctx->graph[c]) return WDLB_OK;
    cudaGraph_t g = nullptr;
    WDLB_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int64_t dummy = 0;
    int cc = c;
    cudaError_t err = cudaSuccess;
    for (int s = 0; s < kGraphChunk && err == cudaSuccess; s++) {
        err = ctx->L->step(ctx->kp, ctx->dev, cc, ctx->stream, &dummy);
        cc ^= 1;
    }
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "graph capture");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
    cudaError_t e3 = cudaGraphInstantiate(&ctx->graph[c], g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return cuda_fail(ctx, e3, "cudaGraphInstantiate");
    return WDLB_OK;
}

wdlb_status stats(wdlb_ctx *ctx, int update_snap, double r[6])
{
    cudaError_t e = ctx->L->stats(ctx->kp, ctx->dev, ctx->cur, update_snap, ctx->stream, &ctx->launches);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stats kernels");
    WDLB_CUDA(ctx, cudaMemcpyAsync(r, ctx->dev.result, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return check_status_word(ctx);
}

}  // namespace

extern "C" {

void wdlb_default_options(wdlb_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->closure = WDLB_CLOSURE_CS;
    opt->omega_mode = WDLB_OMEGA_CONST;
    opt->storage = WDLB_STORE_F32;
    opt->interactions = 1;
    opt->k_cross = 2.0;
    opt->n_ref = 0.0;
}

wdlb_status wdlb_workspace_size(wdlb_lattice lat, double sigma, int32_t walls, const wdlb_options *opt,
                                uint64_t *bytes)
{
    wdlb_options o;
    if (opt)
        o = *opt;
    else
        wdlb_default_options(&o);
    if (!bytes) return WDLB_ERR_ARG;
    wdlb_status s = validate(lat, sigma, walls, &o);
    if (s != WDLB_OK) return s;
    Tables t;
    build_ball(sigma, t.ball);
    build_shell(sigma, t.shell, &t.wshell);
    long long N = (long long)lat.nx * lat.ny * lat.nz;
    long long Npad = (N + 63) / 64 * 64;
    *bytes = layout_for(N, Npad, o.storage, (int)t.shell.size() / 3, (int)t.ball.size() / 3).total;
    return WDLB_OK;
}

wdlb_status wdlb_create(wdlb_lattice lat, double sigma, int32_t walls, double tau, const double g[3],
                        const wdlb_options *opt, wdlb_ctx **out)
{
    if (!out) return fail(nullptr, WDLB_ERR_ARG, "out is NULL");
    *out = nullptr;
    wdlb_options o;
    if (opt)
        o = *opt;
    else
        wdlb_default_options(&o);
    if (validate(lat, sigma, walls, &o) != WDLB_OK) return fail(nullptr, WDLB_ERR_ARG, "invalid lattice, sigma or options");
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(nullptr, WDLB_ERR_ARG, "tau must be > 0.5");
    if (g && !(std::isfinite(g[0]) && std::isfinite(g[1]) && std::isfinite(g[2])))
        return fail(nullptr, WDLB_ERR_ARG, "g must be finite");

    wdlb_ctx *ctx = new (std::nothrow) wdlb_ctx();
    if (!ctx) return fail(nullptr, WDLB_ERR_OOM, "host allocation failed");
    ctx->lat = lat;
    ctx->walls = walls;
    ctx->sigma = sigma;
    ctx->tau = tau;
    if (g)
        for (int d = 0; d < 3; d++) ctx->g[d] = g[d];
    ctx->opt = o;
    ctx->N = (long long)lat.nx * lat.ny * lat.nz;
    ctx->Npad = (ctx->N + 63) / 64 * 64;
    build_ball(sigma, ctx->tab.ball);
    build_shell(sigma, ctx->tab.shell, &ctx->tab.wshell);
    ctx->L = &launchers_for(o.storage);
    set_params(ctx);
    ctx->kp.tiled = ctx->L->prepare(ctx->kp) ? 1 : 0;
    set_reference(ctx, o.n_ref > 0 ? o.n_ref : 1.0);
    const int nshell = ctx->kp.nshell, nball = ctx->kp.nball;
    ctx->lay = layout_for(ctx->N, ctx->Npad, o.storage, nshell, nball);

    // stream
    if (o.stream) {
        ctx->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            return fail(nullptr, WDLB_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        ctx->owns_stream = true;
    }
    // memory
    if (o.workspace) {
        if (o.workspace_bytes < ctx->lay.total || (reinterpret_cast<uintptr_t>(o.workspace) & 255)) {
            wdlb_destroy(ctx);
            return fail(nullptr, WDLB_ERR_OOM, "workspace too small or not 256-byte aligned (need %zu bytes)",
                        ctx->lay.total);
        }
        ctx->base = static_cast<char *>(o.workspace);
    } else {
        cudaError_t e = cudaMalloc(&ctx->base, ctx->lay.total);
        if (e != cudaSuccess) {
            ctx->base = nullptr;
            wdlb_destroy(ctx);
            return fail(nullptr, WDLB_ERR_OOM, "cudaMalloc(%zu): %s", ctx->lay.total, cudaGetErrorString(e));
        }
        ctx->owns_base = true;
    }
    char *b = ctx->base;
    const Layout &L = ctx->lay;
    ctx->dev.f[0] = b + L.f[0];
    ctx->dev.f[1] = b + L.f[1];
    ctx->dev.nu = b + L.nu;
    ctx->dev.hb = b + L.hb;
    ctx->dev.cprev = b + L.cprev;
    ctx->dev.tprev = b + L.tprev;
    ctx->dev.nscale = b + L.nscale;
    ctx->dev.stage = reinterpret_cast<double *>(b + L.stage);
    ctx->dev.snap = reinterpret_cast<double *>(b + L.snap);
    ctx->dev.partial = reinterpret_cast<double *>(b + L.partial);
    ctx->dev.result = reinterpret_cast<double *>(b + L.result);
    ctx->dev.status = reinterpret_cast<int *>(b + L.status);
    ctx->dev.shell_e = reinterpret_cast<const int4 *>(b + L.shell_e);
    ctx->dev.shell_k = b + L.shell_k;
    ctx->dev.ball = reinterpret_cast<const int4 *>(b + L.ball);

    // tables to the device
    std::vector<int4> se(std::max(nshell, 1)), be(std::max(nball, 1));
    std::vector<double> kd(4 * std::max(nshell, 1));
    std::vector<float> kf(4 * std::max(nshell, 1));
    for (int m = 0; m < nshell; m++) {
        int x = ctx->tab.shell[3 * m], y = ctx->tab.shell[3 * m + 1], z = ctx->tab.shell[3 * m + 2];
        se[m] = make_int4(x, y, z, 0);
        double len = std::sqrt(double(x * x + y * y + z * z));
        double k[4] = {x / len, y / len, z / len, 0.0};
        for (int c = 0; c < 4; c++) {
            kd[4 * m + c] = k[c];
            kf[4 * m + c] = float(k[c]);
        }
    }
    for (int m = 0; m < nball; m++)
        be[m] = make_int4(ctx->tab.ball[3 * m], ctx->tab.ball[3 * m + 1], ctx->tab.ball[3 * m + 2], 0);
    cudaError_t e = cudaMemcpyAsync(b + L.shell_e, se.data(), se.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = o.storage == WDLB_STORE_F64
                ? cudaMemcpyAsync(b + L.shell_k, kd.data(), kd.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)
                : cudaMemcpyAsync(b + L.shell_k, kf.data(), kf.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.ball, be.data(), be.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dev.status, 0, 16 * sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        wdlb_destroy(ctx);
        return fail(nullptr, WDLB_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
    }
    *out = ctx;
    return WDLB_OK;
}

wdlb_status wdlb_init_fields(wdlb_ctx *ctx, const double *n, const double *u)
{
    if (!ctx || !n) return ctx ? fail(ctx, WDLB_ERR_ARG, "n is NULL") : WDLB_ERR_ARG;
    double *sn = ctx->dev.stage, *su = ctx->dev.stage + ctx->N;
    WDLB_CUDA(ctx, cudaMemcpyAsync(sn, n, ctx->N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (u) WDLB_CUDA(ctx, cudaMemcpyAsync(su, u, 3 * ctx->N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    wdlb_status s = init_from_stage(ctx, sn, u ? su : nullptr);
    if (s != WDLB_OK) return s;
    WDLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return WDLB_OK;
}

wdlb_status wdlb_init_fields_device(wdlb_ctx *ctx, const double *d_n, const double *d_u)
{
    if (!ctx || !d_n) return ctx ? fail(ctx, WDLB_ERR_ARG, "d_n is NULL") : WDLB_ERR_ARG;
    return init_from_stage(ctx, d_n, d_u);
}

wdlb_status wdlb_step(wdlb_ctx *ctx, int64_t nsteps)
{
    if (!ctx) return WDLB_ERR_ARG;
    if (nsteps < 0) return fail(ctx, WDLB_ERR_ARG, "nsteps < 0");
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "wdlb_step before wdlb_init_fields");
    int64_t left = nsteps;
    if (left >= kGraphChunk) {
        // graphs for both buffer parities are captured lazily when first needed
        while (left >= kGraphChunk) {
            wdlb_status s = ensure_graph(ctx);
            if (s != WDLB_OK) return s;
            WDLB_CUDA(ctx, cudaGraphLaunch(ctx->graph[ctx->cur], ctx->stream));
            ctx->launches += 3 * kGraphChunk;
            left -= kGraphChunk;   // even chunk: parity unchanged
        }
    }
    wdlb_status s = step_direct(ctx, left);
    if (s != WDLB_OK) return s;
    ctx->steps += nsteps;
    return WDLB_OK;
}

wdlb_status wdlb_moments_device(wdlb_ctx *ctx, double *d_n, double *d_u)
{
    if (!ctx) return WDLB_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "moments before init");
    cudaError_t e = ctx->L->moments(ctx->kp, ctx->dev, ctx->cur, d_n, d_u, ctx->stream, &ctx->launches);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "moments kernels");
    return WDLB_OK;
}

wdlb_status wdlb_moments(wdlb_ctx *ctx, double *n, double *u)
{
    if (!ctx) return WDLB_ERR_ARG;
    double *sn = ctx->dev.stage, *su = ctx->dev.stage + ctx->N;
    wdlb_status s = wdlb_moments_device(ctx, sn, su);
    if (s != WDLB_OK) return s;
    if (n) WDLB_CUDA(ctx, cudaMemcpyAsync(n, sn, ctx->N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (u) WDLB_CUDA(ctx, cudaMemcpyAsync(u, su, 3 * ctx->N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return check_status_word(ctx);
}

wdlb_status wdlb_fields(wdlb_ctx *ctx, double *nbar, double *C, double *A, double *u)
{
    if (!ctx) return WDLB_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "fields before init");
    // temporary FP64 outputs (test and inspection path; the time step never allocates)
    const size_t N = ctx->N;
    double *buf = nullptr;
    const size_t nu_bytes = ctx->lay.hb - ctx->lay.nu;   // the field array is overwritten by the moments pass
    WDLB_CUDA(ctx, cudaMalloc(&buf, 13 * N * sizeof(double) + nu_bytes));
    double *dn = buf, *dC = buf + N, *dA = buf + 4 * N, *du = buf + 10 * N;
    char *save = reinterpret_cast<char *>(buf + 13 * N);
    cudaError_t e = cudaMemcpyAsync(save, ctx->dev.nu, nu_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = ctx->L->fields(ctx->kp, ctx->dev, ctx->cur, dn, dC, dA, du, ctx->stream, &ctx->launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->dev.nu, save, nu_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && nbar) e = cudaMemcpyAsync(nbar, dn, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && C) e = cudaMemcpyAsync(C, dC, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && A) e = cudaMemcpyAsync(A, dA, 6 * N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fields");
    return check_status_word(ctx);
}

wdlb_status wdlb_get_populations(wdlb_ctx *ctx, double *f)
{
    if (!ctx || !f) return ctx ? fail(ctx, WDLB_ERR_ARG, "f is NULL") : WDLB_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "populations before init");
    for (int q = 0; q < NQ; q++) {
        cudaError_t e = ctx->L->population(ctx->kp, ctx->dev, ctx->cur, q, ctx->dev.stage, ctx->stream, &ctx->launches);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "population kernel");
        WDLB_CUDA(ctx, cudaMemcpyAsync(f + (size_t)q * ctx->N, ctx->dev.stage, ctx->N * sizeof(double),
                                       cudaMemcpyDeviceToHost, ctx->stream));
        WDLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return WDLB_OK;
}

wdlb_status wdlb_pore_average(wdlb_ctx *ctx, wdlb_pore_stats *out)
{
    if (!ctx || !out) return ctx ? fail(ctx, WDLB_ERR_ARG, "out is NULL") : WDLB_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "pore average before init");
    double r[6];
    wdlb_status s = stats(ctx, 0, r);
    if (s != WDLB_OK) return s;
    out->mass = r[0];
    out->mean_n = r[5] > 0 ? r[0] / r[5] : NAN;
    out->mean_ux = r[5] > 0 ? r[1] / r[5] : NAN;
    out->flux_x = r[2] / (double(ctx->lat.nx) * ctx->lat.ny);
    if (ctx->walls && out->mean_ux != 0.0) {
        double H = ctx->lat.nz - 2;
        out->eta_eff = out->mean_n * ctx->g[0] * H * H / (12.0 * out->mean_ux);
    } else {
        out->eta_eff = NAN;
    }
    out->residual = ctx->last_residual;
    out->steps = ctx->steps;
    return WDLB_OK;
}

wdlb_status wdlb_run_steady(wdlb_ctx *ctx, double tol, int32_t check_every, int64_t max_steps,
                            int64_t *steps_done, double *residual)
{
    if (!ctx) return WDLB_ERR_ARG;
    if (check_every < 1 || max_steps < 0 || !(tol > 0)) return fail(ctx, WDLB_ERR_ARG, "bad steady-state arguments");
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "run_steady before init");
    double r[6];
    wdlb_status s = stats(ctx, 1, r);
    if (s != WDLB_OK) return s;
    int64_t done = 0;
    double res = NAN;
    while (done < max_steps) {
        int64_t n = std::min<int64_t>(check_every, max_steps - done);
        s = wdlb_step(ctx, n);
        if (s != WDLB_OK) return s;
        done += n;
        s = stats(ctx, 1, r);
        if (s != WDLB_OK) return s;
        res = r[4] > 0 ? r[3] / (double(n) * r[4]) : 0.0;
        ctx->last_residual = res;
        if (res < tol) break;
    }
    if (steps_done) *steps_done = done;
    if (residual) *residual = res;
    return WDLB_OK;
}

wdlb_status wdlb_velocity_set(int32_t *c, double *w)
{
    for (int q = 0; q < NQ; q++) {
        if (c) {
            c[3 * q] = cx_of(q);
            c[3 * q + 1] = cy_of(q);
            c[3 * q + 2] = cz_of(q);
        }
        if (w) w[q] = w_of(q);
    }
    return WDLB_OK;
}

wdlb_status wdlb_stencil(double sigma, int32_t which, int32_t *vecs, int32_t cap, int32_t *count, double *weight)
{
    if (!(sigma >= 1.0 && sigma <= 8.0) || (which != 0 && which != 1) || cap < 0) return WDLB_ERR_ARG;
    std::vector<int> v;
    double w = 0.0;
    if (which == 0)
        build_ball(sigma, v);
    else
        build_shell(sigma, v, &w);
    int m = (int)v.size() / 3;
    if (vecs)
        for (int k = 0; k < std::min(m, (int)cap); k++)
            for (int d = 0; d < 3; d++) vecs[3 * k + d] = v[3 * k + d];
    if (count) *count = m;
    if (weight) *weight = w;
    return WDLB_OK;
}

wdlb_status wdlb_profile_step(wdlb_ctx *ctx, int64_t nsteps, double ms[3])
{
    if (!ctx || !ms) return ctx ? fail(ctx, WDLB_ERR_ARG, "ms is NULL") : WDLB_ERR_ARG;
    if (nsteps < 1) return fail(ctx, WDLB_ERR_ARG, "nsteps < 1");
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "profile before init");
    std::vector<cudaEvent_t> &ev = ctx->prof_events;
    while ((int64_t)ev.size() < 6 * nsteps) {
        cudaEvent_t e = nullptr;
        WDLB_CUDA(ctx, cudaEventCreate(&e));
        ev.push_back(e);
    }
    cudaError_t err = cudaSuccess;
    for (int64_t s = 0; s < nsteps && err == cudaSuccess; s++) {
        for (int part = 0; part < 3 && err == cudaSuccess; part++) {
            err = cudaEventRecord(ev[6 * s + 2 * part], ctx->stream);
            if (err == cudaSuccess) err = ctx->L->step_part(ctx->kp, ctx->dev, ctx->cur, part, ctx->stream, &ctx->launches);
            if (err == cudaSuccess) err = cudaEventRecord(ev[6 * s + 2 * part + 1], ctx->stream);
        }
        ctx->cur ^= 1;
        ctx->steps += 1;
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
    double acc[3] = {0, 0, 0};
    for (int64_t s = 0; s < nsteps && err == cudaSuccess; s++)
        for (int part = 0; part < 3 && err == cudaSuccess; part++) {
            float t = 0.f;
            err = cudaEventElapsedTime(&t, ev[6 * s + 2 * part], ev[6 * s + 2 * part + 1]);
            acc[part] += t;
        }
    if (err != cudaSuccess) return cuda_fail(ctx, err, "profile step");
    for (int k = 0; k < 3; k++) ms[k] = acc[k] / double(nsteps);
    return check_status_word(ctx);
}

int64_t wdlb_launch_count(const wdlb_ctx *ctx) { return ctx ? ctx->launches : 0; }

const char *wdlb_last_error(const wdlb_ctx *ctx)
{
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

void wdlb_destroy(wdlb_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    for (auto &e : ctx->prof_events) cudaEventDestroy(e);
    if (ctx->owns_base && ctx->base) cudaFree(ctx->base);
    if (ctx->owns_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"

