// C ABI of the WDLB library (declared in include/wdlb.h): context lifetime,
// workspace layout, host tables, time stepping with CUDA-graph replay, FP64
// reductions and host transfers.  All arithmetic of the method runs in the
// kernels of wdlb_kernels.cuh; this file only validates, lays out memory and
// enqueues work on the context stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/wdlb.h"
#include "wdlb_dw.cuh"
#include "wdlb_launch.h"
#include "wdlb_tables.h"

namespace {
// NVTX range over a host-side phase of the library (named in Nsight Systems
// timelines and selectable with ncu --nvtx); NVTX is header-only and costs a
// null check when no tool is attached.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace

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
    std::vector<double> wvec; // weight of each shell vector
    double wshell = 0.0;      // uniform weight in the kernels (1 for the compact shell)
};

struct Layout {
    size_t f[2], nu, hb, cprev, tprev, nscale, stage, snap, partial, result, status, shell_e, shell_k, ball;
    size_t params, kbufs, items;   // one-slot step tables (KParams, KBufs of both parities, work items)
    size_t tmaps;                  // tensor maps of the TMA tile (nu, hb), 64-byte aligned
    size_t nitems;
    size_t total;
};

int storage_bytes(int storage) { return storage == WDLB_STORE_F64 ? 8 : (storage == WDLB_STORE_F32 ? 4 : 2); }
int compute_bytes(int storage) { return storage == WDLB_STORE_F64 ? 8 : 4; }

// Work items of a lattice stepped alone: blocks of 256 nodes for the moments,
// and bricks or blocks for the smeared density and the shell sums.
size_t step_items(wdlb_lattice lat, long long N)
{
    const size_t nb = size_t((N + 255) / 256);
    const size_t nt = size_t((lat.nx + 7) / 8) * size_t((lat.ny + 7) / 8) * size_t((lat.nz + 3) / 4);
    return nb + 2 * std::max(nb, nt);
}

Layout layout_for(wdlb_lattice lat, long long N, long long Npad, int storage, int nshell, int nball)
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
    L.params = take(sizeof(KParams));
    L.kbufs = take(2 * kKBufsMaxBytes);
    L.nitems = step_items(lat, N);
    L.items = take(L.nitems * sizeof(BatchItem));
    L.tmaps = take(2 * sizeof(CUtensorMap));
    L.total = off;
    return L;
}

// cuTensorMapEncodeTiled of the driver, through the runtime's entry-point
// query (no link against the driver library); NULL if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor maps of the tiled shell kernel's TMA staging (sigma 4: halo 4, tile
// 16 x 16 x (TZ + 8) nodes): nu as the 4-D tensor (component, x, y, z) of
// floats, hb as the 3-D tensor (x, y, z).  Needs 16-byte row strides for hb
// (nx a multiple of 4).  Returns false where the kernel must stage per node.
bool encode_tile_maps(const KParams &p, const wdlb_options &o, void *nu, void *hb, CUtensorMap maps[2])
{
    if (!p.tiled || p.s2 != 8 || o.storage == WDLB_STORE_F64 || o.staging != WDLB_STAGING_AUTO) return false;
    if (p.nx % 4 != 0 || p.nx < 16 || p.ny < 16) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint32_t SZ = (cuuint32_t)(tile_depth(p.tile) + 8);
    const cuuint64_t nx = p.nx, ny = p.ny, nz = p.nz;
    const cuuint64_t dnu[4] = {4, nx, ny, nz}, snu[3] = {16, 16 * nx, 16 * nx * ny};
    const cuuint32_t bnu[4] = {4, 16, 16, SZ}, es[4] = {1, 1, 1, 1};
    const cuuint64_t dhb[3] = {nx, ny, nz}, shb[2] = {4 * nx, 4 * nx * ny};
    const cuuint32_t bhb[3] = {16, 16, SZ};
    return enc(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nu, dnu, snu, bnu, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
           enc(&maps[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, hb, dhb, shb, bhb, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

const Launchers &launchers_for(int storage, int collision)
{
    if (storage == WDLB_STORE_F64) return launchers_f64();
    if (storage == WDLB_STORE_F32) return collision == WDLB_COLLISION_DW ? launchers_f32dw() : launchers_f32();
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
    double prev_flux = NAN;        // pore flux at the last residual test
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    BatchLaunch launch{};          // one-slot step tables in device memory (bufs[p]: input buffer p)
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
        // FP16 storage is for periodic boxes only: in a driven slit its 10-bit
        // deviations leave u_x errors of 2 to 15 % at steady state
        if (opt->storage == WDLB_STORE_F16 && walls == WDLB_WALLS_Z) return WDLB_ERR_ARG;
        if (!(opt->n_ref >= 0.0) || !std::isfinite(opt->k_cross)) return WDLB_ERR_ARG;
        // the double-word collision: FP32 storage, lattices with walls
        if (opt->collision < 0 || opt->collision > 1) return WDLB_ERR_ARG;
        if (opt->collision == WDLB_COLLISION_DW && (opt->storage != WDLB_STORE_F32 || walls != WDLB_WALLS_Z))
            return WDLB_ERR_ARG;
        if (opt->tile < -1 || opt->tile > 2 || opt->autotune < 0 || opt->autotune > 1) return WDLB_ERR_ARG;
        if (opt->shell_rule < 0 || opt->shell_rule > 1) return WDLB_ERR_ARG;
        if (opt->shell_rule == WDLB_SHELL_COMPACT) {
            std::vector<int> v;
            std::vector<double> w;
            if (!build_shell_compact(sigma, v, w)) return WDLB_ERR_ARG;
        }
    }
    return WDLB_OK;
}

wdlb_status check_status_word(wdlb_ctx *ctx)
{
    int h = 0;
    WDLB_CUDA(ctx, cudaMemcpyAsync(&h, ctx->dev.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    WDLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h & kStatusBounds)
        return fail(ctx, WDLB_ERR_CUDA, "checked build: a kernel index left its array (the access was skipped)");
    if (h & kStatusTimeout)
        return fail(ctx, WDLB_ERR_TIMEOUT, "a bounded wait for the TMA tile ran out (the brick was skipped)");
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
    p.shell_rule = ctx->opt.shell_rule;
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
    for (int d = 0; d < 3; d++) dw_split(p.g[d], p.g_dw[d]);
    dw_split(p.omega, p.omega_dw);
    dw_split(p.interactions ? p.k_cross * 4.5 : 0.0, p.ka_dw);
    set_float_params(p);
    const double s2 = 2.0 * ctx->sigma;
    p.s2 = (std::fabs(s2 - std::round(s2)) < 1e-12) ? (int)std::lround(s2) : 0;
    p.tiled = 0;
    p.ball_r = 0;
    for (size_t m = 0; m < ctx->tab.ball.size(); m++) p.ball_r = std::max(p.ball_r, std::abs(ctx->tab.ball[m]));
    const size_t tsize = ctx->opt.storage == WDLB_STORE_F64 ? sizeof(double) : sizeof(float);
    p.ball_tiled = ball_tile_smem(p.ball_r, p.nball, tsize) <= kBallTileMaxSmem ? 1 : 0;
    // n_off / ref_ng are set at init (they may depend on the initial state)
}

void set_reference(wdlb_ctx *ctx, double n_ref)
{
    KParams &p = ctx->kp;
    p.n_off = n_ref;
    p.ref_ng = n_ref * contact_g_host(ctx->opt.closure, p.chi_of_n * n_ref);
    p.h_off = 0.5 * p.chi_of_n * p.n_off;
    set_float_params(p);
}

void drop_graphs(wdlb_ctx *ctx)
{
    for (auto &g : ctx->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// One-slot step tables of a lattice stepped alone: its parameters, its
// buffers for both input parities and its work items, so that it runs the
// same kernels as a slot of a batch.  Synchronous (host vectors).
cudaError_t upload_step_tables(wdlb_ctx *ctx)
{
    char *b = ctx->base;
    const Layout &L = ctx->lay;
    const KParams &p = ctx->kp;
    std::vector<char> kb(2 * kKBufsMaxBytes, 0);
    ctx->L->kbufs_fill(ctx->dev, 0, kb.data());
    ctx->L->kbufs_fill(ctx->dev, 1, kb.data() + kKBufsMaxBytes);
    std::vector<BatchItem> items;
    const int nb = (int)((ctx->N + 255) / 256);
    const int tx = (p.nx + 7) / 8, ty = (p.ny + 7) / 8, tz = (p.nz + 7) / 8;
    auto bricks = [&](int depth) {
        const int bz = (p.nz + depth - 1) / depth;
        for (int z = 0; z < bz; z++)
            for (int y = 0; y < ty; y++)
                for (int x = 0; x < tx; x++) items.push_back(BatchItem{0, x, y, z});
    };
    auto blocks = [&]() {
        for (int k = 0; k < nb; k++) items.push_back(BatchItem{0, k, 0, 0});
    };
    BatchLaunch &LL = ctx->launch;
    LL = BatchLaunch{};
    LL.params = reinterpret_cast<const KParams *>(b + L.params);
    LL.bufs[0] = b + L.kbufs;
    LL.bufs[1] = b + L.kbufs + kKBufsMaxBytes;
    const BatchItem *dit = reinterpret_cast<const BatchItem *>(b + L.items);
    LL.node_items = dit;
    blocks();
    LL.n_node_items = nb;
    if (p.ball_tiled) {
        LL.ball_items = dit + items.size();
        bricks(kBallTile);
        LL.n_ball_items = tx * ty * tz;
        LL.ball_smem = ball_tile_smem(p.ball_r, p.nball, ctx->opt.storage == WDLB_STORE_F64 ? 8 : 4);
    } else {
        LL.ball_node_items = dit + items.size();
        blocks();
        LL.n_ball_node_items = nb;
    }
    BatchGroup &G = LL.groups[0];
    G.s2 = p.tiled ? p.s2 : 0;
    G.walls = ctx->walls;
    G.tiled = p.tiled;
    G.closure = p.closure;
    G.tile = p.tiled ? p.tile : -1;
    G.rule = p.shell_rule;
    G.items = dit + items.size();
    if (p.tiled)
        bricks(tile_depth(p.tile));
    else
        blocks();
    G.nitems = (int)(items.size() - (G.items - dit));
    LL.ngroups = 1;
    if (items.size() > L.nitems) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(b + L.params, &p, sizeof(KParams), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.kbufs, kb.data(), kb.size(), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + L.items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e;
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
    WDLB_CUDA(ctx, cudaMemcpyAsync(const_cast<KParams *>(ctx->launch.params), &ctx->kp, sizeof(KParams),
                                   cudaMemcpyHostToDevice, ctx->stream));
    ctx->cur = 0;
    WDLB_CUDA(ctx, cudaMemsetAsync(ctx->dev.status, 0, sizeof(int), ctx->stream));
    WDLB_CUDA(ctx, cudaMemsetAsync(ctx->dev.snap, 0, ctx->N * sizeof(double), ctx->stream));
    cudaError_t e = ctx->L->init(ctx->kp, ctx->dev, ctx->cur, d_n, d_u, ctx->stream, &ctx->launches);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "init kernel");
    ctx->initialised = true;
    ctx->steps = 0;
    ctx->last_residual = NAN;
    ctx->prev_flux = NAN;
    return WDLB_OK;
}

wdlb_status step_direct(wdlb_ctx *ctx, int64_t n)
{
    for (int64_t s = 0; s < n; s++) {
        cudaError_t e = ctx->L->batch_step(ctx->launch, ctx->cur, -1, -1, ctx->stream, &ctx->launches);
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
        err = ctx->L->batch_step(ctx->launch, cc, -1, -1, ctx->stream, &dummy);
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

namespace {

// ---------------------------------------------------------------------------
// Tile autotuner: a process-wide table (storage, 2 sigma, walls, nz, shell
// rule, collision arithmetic) -> tile
// shape of the tiled shell kernel, filled on first use by timing every shape
// on a scratch lattice of the key, or from the built-in table.
// ---------------------------------------------------------------------------
struct TuneKey {
    int storage, s2, walls, nz, rule, collision;
    bool operator<(const TuneKey &o) const
    {
        return std::make_tuple(storage, s2, walls, nz, rule, collision) <
               std::make_tuple(o.storage, o.s2, o.walls, o.nz, o.rule, o.collision);
    }
};

std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tune;

int two_sigma(double sigma)
{
    const double s2 = 2.0 * sigma;
    return std::fabs(s2 - std::round(s2)) < 1e-12 ? (int)std::lround(s2) : 0;
}

// Whether the tiled shell kernel serves these arguments (the launchers apply
// the same rule when preparing a context).
bool tiled_applies(wdlb_lattice lat, double sigma, const wdlb_options &o)
{
    const int s2 = two_sigma(sigma);
    return o.storage != WDLB_STORE_F64 && o.closure == WDLB_CLOSURE_CS && (s2 == 6 || s2 == 8 || s2 == 12) &&
           lat.nx >= 8 && lat.ny >= 8;
}

// Built-in choice when no probe runs (the winners of the probe at every nz
// measured): the 512-thread shape for sigma 6 (one 160 KB block per SM),
// 8 x 8 x 4 bricks for sigma 4 (three 61 KB blocks per SM), 8^3 bricks for
// sigma 3 (three 55 KB blocks per SM).
int tile_builtin(int s2, int walls, int nz)
{
    (void)walls;
    (void)nz;
    return s2 == 12 ? WDLB_TILE_8x8x8_WIDE : (s2 == 8 ? WDLB_TILE_8x8x4 : WDLB_TILE_8x8x8);
}

// Time each shape's shell kernel on a scratch lattice of the key: nz as
// given and a square cross-section of about 2^20 / nz nodes, so that the
// kernel fills the GPU as a batch of pores does (a single small pore leaves
// SMs idle and would favour shapes that merely make more blocks).  The
// scratch contexts force their shape, so they do not come back here.
wdlb_status probe_tiles(wdlb_lattice lat, double sigma, int32_t walls, const wdlb_options &o, int *best,
                        double ms[3])
{
    TraceRange tr("autotune_probe");
    int side = (int)std::ceil(std::sqrt(double(1 << 20) / double(lat.nz)) / 8.0) * 8;
    side = std::max(8, std::min(side, 512));
    wdlb_lattice pl{side, side, lat.nz};
    const long long N = (long long)pl.nx * pl.ny * pl.nz;
    std::vector<double> n(N, 0.4 / (sigma * sigma * sigma));
    if (walls)
        for (long long i = 0; i < (long long)pl.nx * pl.ny; i++) n[i] = n[N - 1 - i] = 0.0;
    const double g[3] = {1e-6, 0.0, 0.0};
    *best = -1;
    for (int v = 0; v < 3; v++) {
        ms[v] = NAN;
        wdlb_options po = o;
        po.tile = v;
        po.autotune = 0;
        po.workspace = nullptr;
        po.workspace_bytes = 0;
        po.stream = nullptr;
        po.n_ref = 0.0;
        wdlb_ctx *c = nullptr;
        if (wdlb_create(pl, sigma, walls, 1.0, g, &po, &c) != WDLB_OK) continue;
        double t[3];
        if (c->kp.tiled && c->kp.tile == v && wdlb_init_fields(c, n.data(), nullptr) == WDLB_OK &&
            wdlb_profile_step(c, 2, t) == WDLB_OK && wdlb_profile_step(c, 6, t) == WDLB_OK)
            ms[v] = t[2];
        wdlb_destroy(c);
        if (std::isfinite(ms[v]) && (*best < 0 || ms[v] < ms[*best])) *best = v;
    }
    return *best >= 0 ? WDLB_OK : WDLB_ERR_CUDA;
}

int choose_tile(wdlb_lattice lat, double sigma, int32_t walls, const wdlb_options &o)
{
    if (!tiled_applies(lat, sigma, o)) return WDLB_TILE_8x8x8;
    if (o.tile >= 0) return o.tile;
    const TuneKey key{o.storage, two_sigma(sigma), walls, lat.nz, o.shell_rule, o.collision};
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
    int v = tile_builtin(key.s2, walls, lat.nz);
    if (o.autotune) {
        int b = -1;
        double ms[3];
        if (probe_tiles(lat, sigma, walls, o, &b, ms) == WDLB_OK) v = b;
    }
    g_tune[key] = v;
    return v;
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
    opt->tile = WDLB_TILE_AUTO;
    opt->autotune = 1;
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
    build_shell_rule(sigma, o.shell_rule, t.shell, t.wvec);
    long long N = (long long)lat.nx * lat.ny * lat.nz;
    long long Npad = (N + 63) / 64 * 64;
    *bytes = layout_for(lat, N, Npad, o.storage, (int)t.shell.size() / 3, (int)t.ball.size() / 3).total;
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
    build_shell_rule(sigma, o.shell_rule, ctx->tab.shell, ctx->tab.wvec);
    ctx->tab.wshell = o.shell_rule == WDLB_SHELL_COMPACT ? 1.0 : ctx->tab.wvec[0];
    ctx->L = &launchers_for(o.storage, o.collision);
    set_params(ctx);
    ctx->kp.tile = choose_tile(lat, sigma, walls, o);
    ctx->kp.tiled = ctx->L->prepare(ctx->kp) ? 1 : 0;
    set_reference(ctx, o.n_ref > 0 ? o.n_ref : 1.0);
    const int nshell = ctx->kp.nshell, nball = ctx->kp.nball;
    ctx->lay = layout_for(lat, ctx->N, ctx->Npad, o.storage, nshell, nball);

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
    ctx->kp.wait_limit = o.wait_limit != 0 ? o.wait_limit : kDefaultWaitLimit;
    CUtensorMap maps[2];
    ctx->kp.tma = encode_tile_maps(ctx->kp, o, ctx->dev.nu, ctx->dev.hb, maps) ? 1 : 0;
    ctx->kp.tmaps = ctx->kp.tma ? b + L.tmaps : nullptr;

    // tables to the device
    std::vector<int4> se(std::max(nshell, 1)), be(std::max(nball, 1));
    std::vector<double> kd(4 * std::max(nshell, 1));
    std::vector<float> kf(4 * std::max(nshell, 1));
    for (int m = 0; m < nshell; m++) {
        int x = ctx->tab.shell[3 * m], y = ctx->tab.shell[3 * m + 1], z = ctx->tab.shell[3 * m + 2];
        se[m] = make_int4(x, y, z, 0);
        double len = std::sqrt(double(x * x + y * y + z * z));
        double k[4] = {x / len, y / len, z / len, o.shell_rule == WDLB_SHELL_COMPACT ? ctx->tab.wvec[m] : 0.0};
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
    if (e == cudaSuccess && ctx->kp.tma)
        e = cudaMemcpyAsync(b + L.tmaps, maps, sizeof(maps), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = upload_step_tables(ctx);
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
    TraceRange tr("wdlb_init_fields");
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
    TraceRange tr("wdlb_step");
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
    TraceRange tr("wdlb_moments");
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
    for (int part = 0; part < 2 && e == cudaSuccess; part++)
        e = ctx->L->batch_step(ctx->launch, ctx->cur, part, -1, ctx->stream, &ctx->launches);
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

wdlb_status wdlb_thermal_fields(wdlb_ctx *ctx, const double *T, double *Q, double *B, double *FT)
{
    if (!ctx) return WDLB_ERR_ARG;
    if (!T) return fail(ctx, WDLB_ERR_ARG, "T is NULL");
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "thermal fields before init");
    const size_t N = ctx->N;
    const int nxy = ctx->lat.nx * ctx->lat.ny;
    for (size_t i = 0; i < N; i++) {
        const int z = (int)(i / nxy);
        const bool solid = ctx->walls && (z == 0 || z == ctx->lat.nz - 1);
        if (!solid && !(std::isfinite(T[i]) && T[i] > 0.0))
            return fail(ctx, WDLB_ERR_ARG, "T must be finite and positive on fluid nodes (node %zu)", i);
    }
    // temporary FP64 arrays (an inspection path; the time step never allocates)
    double *buf = nullptr;
    const size_t nu_bytes = ctx->lay.hb - ctx->lay.nu;   // the field array is overwritten by the moments pass
    WDLB_CUDA(ctx, cudaMalloc(&buf, 8 * N * sizeof(double) + nu_bytes));
    double *dT = buf, *dQ = buf + N, *dB = buf + 2 * N, *dF = buf + 5 * N;
    char *save = reinterpret_cast<char *>(buf + 8 * N);
    cudaError_t e = cudaMemcpyAsync(save, ctx->dev.nu, nu_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dT, T, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    for (int part = 0; part < 2 && e == cudaSuccess; part++)
        e = ctx->L->batch_step(ctx->launch, ctx->cur, part, -1, ctx->stream, &ctx->launches);
    if (e == cudaSuccess) e = ctx->L->thermal(ctx->kp, ctx->dev, ctx->cur, dT, dQ, dB, dF, ctx->stream, &ctx->launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->dev.nu, save, nu_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && Q) e = cudaMemcpyAsync(Q, dQ, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && B) e = cudaMemcpyAsync(B, dB, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && FT) e = cudaMemcpyAsync(FT, dF, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "thermal fields");
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

// Steady-state residual: relative change per step of the pore flux sum(n u_x)
// (FP64 reduction) between two tests `interval` steps apart.
static double flux_residual(wdlb_ctx *ctx, const double r[6], int64_t interval)
{
    const double q = r[2];
    double res;
    if (!std::isfinite(ctx->prev_flux))
        res = INFINITY;
    else if (q == 0.0)
        res = q == ctx->prev_flux ? 0.0 : INFINITY;
    else
        res = std::fabs(q - ctx->prev_flux) / (double(interval) * std::fabs(q));
    ctx->prev_flux = q;
    return res;
}

wdlb_status wdlb_run_steady(wdlb_ctx *ctx, double tol, int32_t check_every, int64_t max_steps,
                            int64_t *steps_done, double *residual)
{
    TraceRange tr("wdlb_run_steady");
    if (!ctx) return WDLB_ERR_ARG;
    if (check_every < 1 || max_steps < 0 || !(tol > 0)) return fail(ctx, WDLB_ERR_ARG, "bad steady-state arguments");
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "run_steady before init");
    double r[6];
    wdlb_status s = stats(ctx, 1, r);
    if (s != WDLB_OK) return s;
    ctx->prev_flux = r[2];
    int64_t done = 0;
    double res = NAN;
    while (done < max_steps) {
        int64_t n = std::min<int64_t>(check_every, max_steps - done);
        s = wdlb_step(ctx, n);
        if (s != WDLB_OK) return s;
        done += n;
        s = stats(ctx, 1, r);
        if (s != WDLB_OK) return s;
        res = flux_residual(ctx, r, n);
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

wdlb_status wdlb_shell_table(double sigma, int32_t rule, int32_t *vecs, double *weights, int32_t cap,
                             int32_t *count)
{
    if (!(sigma >= 1.0 && sigma <= 8.0) || (rule != WDLB_SHELL_FULL && rule != WDLB_SHELL_COMPACT) || cap < 0)
        return WDLB_ERR_ARG;
    std::vector<int> v;
    std::vector<double> w;
    if (!build_shell_rule(sigma, rule, v, w)) return WDLB_ERR_ARG;
    const int m = (int)w.size();
    for (int k = 0; k < std::min(m, (int)cap); k++) {
        if (vecs)
            for (int d = 0; d < 3; d++) vecs[3 * k + d] = v[3 * k + d];
        if (weights) weights[k] = w[k];
    }
    if (count) *count = m;
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
            if (err == cudaSuccess)
                err = ctx->L->batch_step(ctx->launch, ctx->cur, part, -1, ctx->stream, &ctx->launches);
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

// ---- checkpoint ------------------------------------------------------------
namespace {

struct StateHeader {
    uint64_t magic;
    int32_t version, storage, nx, ny, nz, walls, shell_rule;
    int64_t N, steps;
    double sigma, tau, n_ref;
};
constexpr uint64_t kStateMagic = 0x3137454b50444c57ull;   // "WLDPKE71"

// Device regions of the state, in blob order: (offset in the context's
// memory, bytes).
std::vector<std::pair<size_t, size_t>> state_regions(const wdlb_ctx *ctx)
{
    const Layout &L = ctx->lay;
    const size_t sS = storage_bytes(ctx->opt.storage), sT = compute_bytes(ctx->opt.storage);
    const size_t P = (size_t)ctx->Npad;
    return {{L.f[ctx->cur], NQ * P * sS}, {L.nu, 4 * P * sT}, {L.cprev, 3 * P * sT}, {L.tprev, P * sT},
            {L.nscale, P * sT}};
}

}  // namespace

wdlb_status wdlb_state_bytes(const wdlb_ctx *ctx, uint64_t *bytes)
{
    if (!ctx || !bytes) return WDLB_ERR_ARG;
    uint64_t b = sizeof(StateHeader);
    for (auto &r : state_regions(ctx)) b += r.second;
    *bytes = b;
    return WDLB_OK;
}

wdlb_status wdlb_save_state(wdlb_ctx *ctx, void *host, uint64_t bytes)
{
    if (!ctx || !host) return ctx ? fail(ctx, WDLB_ERR_ARG, "host is NULL") : WDLB_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, WDLB_ERR_STATE, "save before init");
    uint64_t need = 0;
    wdlb_state_bytes(ctx, &need);
    if (bytes < need) return fail(ctx, WDLB_ERR_ARG, "state buffer too small (%llu < %llu)",
                                  (unsigned long long)bytes, (unsigned long long)need);
    StateHeader h{kStateMagic, 2, ctx->opt.storage, ctx->lat.nx, ctx->lat.ny, ctx->lat.nz, ctx->walls,
                  ctx->opt.shell_rule, ctx->N, ctx->steps, ctx->sigma, ctx->tau, ctx->kp.n_off};
    char *out = static_cast<char *>(host);
    std::memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    for (auto &r : state_regions(ctx)) {
        WDLB_CUDA(ctx, cudaMemcpyAsync(out + off, ctx->base + r.first, r.second, cudaMemcpyDeviceToHost, ctx->stream));
        off += r.second;
    }
    WDLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return WDLB_OK;
}

wdlb_status wdlb_load_state(wdlb_ctx *ctx, const void *host, uint64_t bytes)
{
    if (!ctx || !host) return ctx ? fail(ctx, WDLB_ERR_ARG, "host is NULL") : WDLB_ERR_ARG;
    uint64_t need = 0;
    wdlb_state_bytes(ctx, &need);
    if (bytes < need) return fail(ctx, WDLB_ERR_ARG, "state buffer too small");
    StateHeader h;
    std::memcpy(&h, host, sizeof(h));
    if (h.magic != kStateMagic || h.version != 2) return fail(ctx, WDLB_ERR_ARG, "not a saved state");
    if (h.storage != ctx->opt.storage || h.nx != ctx->lat.nx || h.ny != ctx->lat.ny || h.nz != ctx->lat.nz ||
        h.walls != ctx->walls || h.shell_rule != ctx->opt.shell_rule || h.N != ctx->N || h.sigma != ctx->sigma ||
        h.tau != ctx->tau)
        return fail(ctx, WDLB_ERR_ARG, "saved state belongs to another lattice or configuration");
    set_reference(ctx, h.n_ref);
    drop_graphs(ctx);
    WDLB_CUDA(ctx, cudaMemcpyAsync(const_cast<KParams *>(ctx->launch.params), &ctx->kp, sizeof(KParams),
                                   cudaMemcpyHostToDevice, ctx->stream));
    const char *in = static_cast<const char *>(host);
    size_t off = sizeof(h);
    for (auto &r : state_regions(ctx)) {
        WDLB_CUDA(ctx, cudaMemcpyAsync(ctx->base + r.first, in + off, r.second, cudaMemcpyHostToDevice, ctx->stream));
        off += r.second;
    }
    WDLB_CUDA(ctx, cudaMemsetAsync(ctx->dev.status, 0, sizeof(int), ctx->stream));
    WDLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->initialised = true;
    ctx->steps = h.steps;
    ctx->last_residual = NAN;
    ctx->prev_flux = NAN;
    return WDLB_OK;
}

wdlb_status wdlb_autotune(wdlb_lattice lat, double sigma, int32_t walls, const wdlb_options *opt, int32_t *best,
                          double ms[3])
{
    wdlb_options o;
    if (opt)
        o = *opt;
    else
        wdlb_default_options(&o);
    if (validate(lat, sigma, walls, &o) != WDLB_OK || !tiled_applies(lat, sigma, o)) return WDLB_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    int b = -1;
    double t[3];
    wdlb_status s = probe_tiles(lat, sigma, walls, o, &b, t);
    if (s != WDLB_OK) return s;
    g_tune[TuneKey{o.storage, two_sigma(sigma), walls, lat.nz, o.shell_rule, o.collision}] = b;
    if (best) *best = b;
    if (ms)
        for (int v = 0; v < 3; v++) ms[v] = t[v];
    return WDLB_OK;
}

wdlb_status wdlb_tile_info(const wdlb_ctx *ctx, int32_t *tiled, int32_t *tile)
{
    if (!ctx) return WDLB_ERR_ARG;
    if (tiled) *tiled = ctx->kp.tiled;
    if (tile) *tile = ctx->kp.tiled ? ctx->kp.tile : -1;
    return WDLB_OK;
}

wdlb_status wdlb_staging_info(const wdlb_ctx *ctx, int32_t *tma)
{
    if (!ctx || !tma) return WDLB_ERR_ARG;
    *tma = ctx->kp.tiled ? ctx->kp.tma : 0;
    return WDLB_OK;
}

void wdlb_autotune_reset(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.clear();
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

// ===========================================================================
// Batch of independent lattices stepped together (continuous batching).
// Every slot is an ordinary context whose workspace is carved from the
// batch's pool and whose stream is the batch's stream; a batch step launches,
// for all slots at once, the moments and smeared-density kernels over a table
// of (slot, node block) items and one shell kernel per group of slots with
// the same kernel variant (sigma, walls).  Kernel bodies are those of the
// single-lattice path, so a pore gives the same result alone and in a batch.
// ===========================================================================

struct wdlb_batch {
    wdlb_options opt{};
    const Launchers *L = nullptr;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    char *pool = nullptr;
    size_t pool_bytes = 0;
    bool owns_pool = false;
    std::vector<std::pair<size_t, size_t>> free_list;   // (offset, bytes), sorted by offset
    struct Slot {
        wdlb_ctx *ctx = nullptr;
        size_t off = 0, bytes = 0;
    };
    std::vector<Slot> slots;
    // device tables
    KParams *d_params = nullptr;
    int *d_flow = nullptr;             // persistent step: counts [3P], done [3P], next, abort
    bool flow = false;                 // the persistent kernel serves the current tables
    char *d_bufs[2] = {nullptr, nullptr};
    BatchItem *d_items = nullptr;
    size_t items_cap = 0;
    // residual test in one set of launches: per-slot statistics buffers and
    // the results [6P] and status words [P] of all slots
    StatSlot *d_stat = nullptr;
    double *d_res = nullptr;
    int *d_st = nullptr;
    BatchLaunch launch{};
    bool dirty = true;
    int64_t steps_since_build = 0;
    cudaGraphExec_t graph = nullptr;   // two steps: parity 0 then 1
    cudaStream_t side[kMaxBatchGroups] = {};     // shell groups 1.. during capture
    cudaEvent_t fork[kMaxBatchGroups] = {}, join[kMaxBatchGroups] = {};
    int64_t launches = 0;
    int64_t graph_launches = 0;        // kernels in one graph replay
    std::string err;
};

namespace {

wdlb_status bfail(wdlb_batch *b, wdlb_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_create_error = buf;
    return s;
}

bool pool_alloc(wdlb_batch *b, size_t bytes, size_t *off)
{
    for (size_t k = 0; k < b->free_list.size(); k++) {
        auto &fr = b->free_list[k];
        if (fr.second >= bytes) {
            *off = fr.first;
            fr.first += bytes;
            fr.second -= bytes;
            if (fr.second == 0) b->free_list.erase(b->free_list.begin() + k);
            return true;
        }
    }
    return false;
}

void pool_free(wdlb_batch *b, size_t off, size_t bytes)
{
    auto &fl = b->free_list;
    auto it = std::lower_bound(fl.begin(), fl.end(), std::make_pair(off, size_t(0)));
    it = fl.insert(it, std::make_pair(off, bytes));
    // merge with neighbours
    size_t k = it - fl.begin();
    if (k + 1 < fl.size() && fl[k].first + fl[k].second == fl[k + 1].first) {
        fl[k].second += fl[k + 1].second;
        fl.erase(fl.begin() + k + 1);
    }
    if (k > 0 && fl[k - 1].first + fl[k - 1].second == fl[k].first) {
        fl[k - 1].second += fl[k].second;
        fl.erase(fl.begin() + k);
    }
}

void batch_drop_graph(wdlb_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// Rebuild the device tables after slots changed.
wdlb_status batch_build(wdlb_batch *b)
{
    TraceRange tr("batch_build");
    const int P = (int)b->slots.size();
    std::vector<KParams> params(P);
    std::vector<StatSlot> stat(P, StatSlot{nullptr, nullptr, nullptr, nullptr});
    std::vector<char> bufs0(b->L->kbufs_bytes * P, 0), bufs1(b->L->kbufs_bytes * P, 0);
    std::vector<BatchItem> node_items, ball_items, ball_node_items;
    size_t ball_smem = 0;
    struct Key {
        int s2, walls, tiled, closure, tile, rule;
        bool operator<(const Key &o) const
        {
            return std::make_tuple(s2, walls, tiled, closure, tile, rule) <
                   std::make_tuple(o.s2, o.walls, o.tiled, o.closure, o.tile, o.rule);
        }
    };
    std::map<Key, std::vector<BatchItem>> groups;
    for (int s = 0; s < P; s++) {
        wdlb_ctx *c = b->slots[s].ctx;
        if (!c) continue;
        params[s] = c->kp;
        stat[s] = StatSlot{c->dev.stage, c->dev.snap, c->dev.partial, c->dev.status};
        b->L->kbufs_fill(c->dev, c->cur, bufs0.data() + s * b->L->kbufs_bytes);
        b->L->kbufs_fill(c->dev, c->cur ^ 1, bufs1.data() + s * b->L->kbufs_bytes);
        const int N = (int)c->N;
        for (int k = 0; k < (N + 255) / 256; k++) node_items.push_back(BatchItem{s, k, 0, 0});
        if (c->kp.ball_tiled) {
            const int bt = kBallTile;
            const int tx = (c->lat.nx + bt - 1) / bt, ty = (c->lat.ny + bt - 1) / bt, tz = (c->lat.nz + bt - 1) / bt;
            for (int z = 0; z < tz; z++)
                for (int y = 0; y < ty; y++)
                    for (int x = 0; x < tx; x++) ball_items.push_back(BatchItem{s, x, y, z});
            const size_t tsize = c->opt.storage == WDLB_STORE_F64 ? sizeof(double) : sizeof(float);
            ball_smem = std::max(ball_smem, ball_tile_smem(c->kp.ball_r, c->kp.nball, tsize));
        } else {
            for (int k = 0; k < (N + 255) / 256; k++) ball_node_items.push_back(BatchItem{s, k, 0, 0});
        }
        Key key{c->kp.tiled ? c->kp.s2 : 0, c->walls, c->kp.tiled, c->kp.closure, c->kp.tiled ? c->kp.tile : -1,
                c->kp.shell_rule};
        auto &g = groups[key];
        if (c->kp.tiled) {
            const int depth = tile_depth(c->kp.tile);
            const int tx = (c->lat.nx + 7) / 8, ty = (c->lat.ny + 7) / 8, tz = (c->lat.nz + depth - 1) / depth;
            for (int z = 0; z < tz; z++)
                for (int y = 0; y < ty; y++)
                    for (int x = 0; x < tx; x++) g.push_back(BatchItem{s, x, y, z});
        } else {
            for (int k = 0; k < (N + 255) / 256; k++) g.push_back(BatchItem{s, k, 0, 0});
        }
    }
    if ((int)groups.size() > kMaxBatchGroups) return bfail(b, WDLB_ERR_ARG, "too many kernel variants in one batch");
    size_t total = node_items.size() + ball_items.size() + ball_node_items.size();
    for (auto &g : groups) total += g.second.size();
    if (total > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->items_cap = std::max<size_t>(total, 2 * b->items_cap);
        if (cudaMalloc(&b->d_items, b->items_cap * sizeof(BatchItem)) != cudaSuccess) {
            b->d_items = nullptr;
            b->items_cap = 0;
            return bfail(b, WDLB_ERR_OOM, "batch work table");
        }
    }
    std::vector<BatchItem> all(node_items);
    BatchLaunch &L = b->launch;
    L.params = b->d_params;
    L.bufs[0] = b->d_bufs[0];
    L.bufs[1] = b->d_bufs[1];
    L.node_items = b->d_items;
    L.n_node_items = (int)node_items.size();
    L.ball_items = b->d_items + all.size();
    L.n_ball_items = (int)ball_items.size();
    L.ball_smem = ball_smem;
    all.insert(all.end(), ball_items.begin(), ball_items.end());
    L.ball_node_items = b->d_items + all.size();
    L.n_ball_node_items = (int)ball_node_items.size();
    all.insert(all.end(), ball_node_items.begin(), ball_node_items.end());
    L.ngroups = 0;
    for (auto &g : groups) {
        BatchGroup &G = L.groups[L.ngroups++];
        G.s2 = g.first.s2;
        G.walls = g.first.walls;
        G.tiled = g.first.tiled;
        G.closure = g.first.closure;
        G.tile = g.first.tile;
        G.rule = g.first.rule;
        G.items = b->d_items + all.size();
        G.nitems = (int)g.second.size();
        all.insert(all.end(), g.second.begin(), g.second.end());
    }
    cudaError_t e = cudaSuccess;
    // item counts per slot and phase for the persistent step
    b->flow = b->opt.persistent && b->L->flow_ok(L);
    std::vector<int> counts(3 * size_t(std::max(P, 1)), 0);
    for (const BatchItem &it : node_items) counts[3 * it.slot + 0]++;
    for (const BatchItem &it : ball_items) counts[3 * it.slot + 1]++;
    for (auto &g : groups)
        for (const BatchItem &it : g.second) counts[3 * it.slot + 2]++;
    if (P > 0 && b->flow)
        e = cudaMemcpyAsync(b->d_flow, counts.data(), 3 * P * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && P > 0)
        e = cudaMemcpyAsync(b->d_params, params.data(), P * sizeof(KParams), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && P > 0)
        e = cudaMemcpyAsync(b->d_stat, stat.data(), P * sizeof(StatSlot), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && P > 0)
        e = cudaMemcpyAsync(b->d_bufs[0], bufs0.data(), bufs0.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && P > 0)
        e = cudaMemcpyAsync(b->d_bufs[1], bufs1.data(), bufs1.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !all.empty())
        e = cudaMemcpyAsync(b->d_items, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // host vectors go out of scope
    if (e != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "batch tables: %s", cudaGetErrorString(e));
    batch_drop_graph(b);
    b->dirty = false;
    b->steps_since_build = 0;
    return WDLB_OK;
}

wdlb_status batch_step_direct(wdlb_batch *b, int64_t n)
{
    for (int64_t s = 0; s < n; s++) {
        cudaError_t e = b->L->batch_step(b->launch, (int)(b->steps_since_build & 1), -1, -1, b->stream, &b->launches);
        if (e != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "batch step: %s", cudaGetErrorString(e));
        b->steps_since_build++;
    }
    return WDLB_OK;
}

// One time step inside the batch's graph capture.  The shell groups (pores of
// different sigma, geometry or tile shape) touch disjoint pores, so with more
// than one group their launches fork onto side streams after the smeared
// density and join before the next step: the groups' last waves overlap
// instead of leaving SMs idle between launches.
cudaError_t batch_capture_step(wdlb_batch *b, int parity, int64_t *count)
{
    const BatchLaunch &L = b->launch;
    cudaError_t e = b->L->batch_step(L, parity, 0, -1, b->stream, count);
    if (e == cudaSuccess) e = b->L->batch_step(L, parity, 1, -1, b->stream, count);
    if (e != cudaSuccess || L.ngroups <= 1) {
        if (e == cudaSuccess) e = b->L->batch_step(L, parity, 2, -1, b->stream, count);
        return e;
    }
    e = cudaEventRecord(b->fork[0], b->stream);
    for (int g = 1; g < L.ngroups && e == cudaSuccess; g++) {
        e = cudaStreamWaitEvent(b->side[g], b->fork[0], 0);
        if (e == cudaSuccess) e = b->L->batch_step(L, parity, 2, g, b->side[g], count);
        if (e == cudaSuccess) e = cudaEventRecord(b->join[g], b->side[g]);
    }
    if (e == cudaSuccess) e = b->L->batch_step(L, parity, 2, 0, b->stream, count);
    for (int g = 1; g < L.ngroups && e == cudaSuccess; g++) e = cudaStreamWaitEvent(b->stream, b->join[g], 0);
    return e;
}

// Side streams and events of the fork/join (created outside any capture).
cudaError_t batch_side_streams(wdlb_batch *b)
{
    cudaError_t e = cudaSuccess;
    if (!b->fork[0]) e = cudaEventCreateWithFlags(&b->fork[0], cudaEventDisableTiming);
    for (int g = 1; g < b->launch.ngroups && e == cudaSuccess; g++) {
        if (!b->side[g]) e = cudaStreamCreateWithFlags(&b->side[g], cudaStreamNonBlocking);
        if (e == cudaSuccess && !b->join[g]) e = cudaEventCreateWithFlags(&b->join[g], cudaEventDisableTiming);
    }
    return e;
}

wdlb_status batch_ensure_graph(wdlb_batch *b)
{
    if (b->graph) return WDLB_OK;
    if (b->launch.ngroups > 1 && batch_side_streams(b) != cudaSuccess)
        return bfail(b, WDLB_ERR_CUDA, "batch side streams");
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bfail(b, WDLB_ERR_CUDA, "batch capture");
    int64_t count = 0;
    cudaError_t e = cudaSuccess;
    for (int parity = 0; parity < 2 && e == cudaSuccess; parity++) e = batch_capture_step(b, parity, &count);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, WDLB_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "batch graph: %s", cudaGetErrorString(e));
    b->graph_launches = count;
    return WDLB_OK;
}

}  // namespace

extern "C" {

wdlb_status wdlb_batch_create(const wdlb_options *opt, uint64_t pool_bytes, int32_t max_pores, wdlb_batch **out)
{
    if (!out) return bfail(nullptr, WDLB_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (max_pores < 1 || pool_bytes < 4096) return bfail(nullptr, WDLB_ERR_ARG, "bad batch size");
    wdlb_options o;
    if (opt)
        o = *opt;
    else
        wdlb_default_options(&o);
    if (o.closure < 0 || o.closure > 2 || o.omega_mode < 0 || o.omega_mode > 1 || o.storage < 0 || o.storage > 2 ||
        o.collision < 0 || o.collision > 1 || (o.collision == WDLB_COLLISION_DW && o.storage != WDLB_STORE_F32))
        return bfail(nullptr, WDLB_ERR_ARG, "invalid options");
    wdlb_batch *b = new (std::nothrow) wdlb_batch();
    if (!b) return bfail(nullptr, WDLB_ERR_OOM, "host allocation failed");
    b->opt = o;
    b->L = &launchers_for(o.storage, o.collision);
    b->slots.resize(max_pores);
    if (o.stream) {
        b->stream = static_cast<cudaStream_t>(o.stream);
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return bfail(nullptr, WDLB_ERR_CUDA, "cudaStreamCreate");
    } else {
        b->owns_stream = true;
    }
    if (o.workspace) {
        if ((reinterpret_cast<uintptr_t>(o.workspace) & 255) || o.workspace_bytes < pool_bytes) {
            wdlb_batch_destroy(b);
            return bfail(nullptr, WDLB_ERR_ARG, "pool must be 256-byte aligned and at least pool_bytes long");
        }
        b->pool = static_cast<char *>(o.workspace);
    } else {
        if (cudaMalloc(&b->pool, pool_bytes) != cudaSuccess) {
            b->pool = nullptr;
            wdlb_batch_destroy(b);
            return bfail(nullptr, WDLB_ERR_OOM, "cudaMalloc(%llu) for the batch pool", (unsigned long long)pool_bytes);
        }
        b->owns_pool = true;
    }
    b->pool_bytes = pool_bytes & ~size_t(255);
    b->free_list.push_back(std::make_pair(size_t(0), b->pool_bytes));
    if (cudaMalloc(&b->d_flow, (6 * size_t(max_pores) + 8) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_params, max_pores * sizeof(KParams)) != cudaSuccess ||
        cudaMalloc(&b->d_stat, max_pores * sizeof(StatSlot)) != cudaSuccess ||
        cudaMalloc(&b->d_res, 6 * size_t(max_pores) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_st, max_pores * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_bufs[0], max_pores * b->L->kbufs_bytes) != cudaSuccess ||
        cudaMalloc(&b->d_bufs[1], max_pores * b->L->kbufs_bytes) != cudaSuccess) {
        wdlb_batch_destroy(b);
        return bfail(nullptr, WDLB_ERR_OOM, "batch tables");
    }
    *out = b;
    return WDLB_OK;
}

wdlb_status wdlb_batch_pore_bytes(const wdlb_batch *b, const wdlb_pore_desc *d, uint64_t *bytes)
{
    if (!b || !d || !bytes) return WDLB_ERR_ARG;
    wdlb_options o = b->opt;
    return wdlb_workspace_size(d->lat, d->sigma, d->walls, &o, bytes);
}

wdlb_status wdlb_batch_add(wdlb_batch *b, const wdlb_pore_desc *d, const double *n, const double *u, int32_t *slot)
{
    if (!b || !d || !n || !slot) return b ? bfail(b, WDLB_ERR_ARG, "NULL argument") : WDLB_ERR_ARG;
    *slot = -1;
    int s = -1;
    for (int k = 0; k < (int)b->slots.size(); k++)
        if (!b->slots[k].ctx) {
            s = k;
            break;
        }
    if (s < 0) return bfail(b, WDLB_ERR_OOM, "all %d slots in use", (int)b->slots.size());
    uint64_t need = 0;
    wdlb_status st = wdlb_batch_pore_bytes(b, d, &need);
    if (st != WDLB_OK) return bfail(b, st, "invalid pore description");
    need = align256(need);
    size_t off = 0;
    if (!pool_alloc(b, need, &off)) return bfail(b, WDLB_ERR_OOM, "pool has no room for %llu bytes", (unsigned long long)need);
    wdlb_options o = b->opt;
    o.workspace = b->pool + off;
    o.workspace_bytes = need;
    o.stream = b->stream;
    wdlb_ctx *c = nullptr;
    st = wdlb_create(d->lat, d->sigma, d->walls, d->tau, d->g, &o, &c);
    if (st != WDLB_OK) {
        pool_free(b, off, need);
        return bfail(b, st, "create: %s", wdlb_last_error(nullptr));
    }
    st = wdlb_init_fields(c, n, u);
    if (st != WDLB_OK) {
        bfail(b, st, "init: %s", c->err.c_str());
        wdlb_destroy(c);
        pool_free(b, off, need);
        return st;
    }
    b->slots[s].ctx = c;
    b->slots[s].off = off;
    b->slots[s].bytes = need;
    b->dirty = true;
    *slot = s;
    return WDLB_OK;
}

wdlb_status wdlb_batch_remove(wdlb_batch *b, int32_t slot)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].ctx) return WDLB_ERR_ARG;
    wdlb_destroy(b->slots[slot].ctx);   // synchronises the stream
    pool_free(b, b->slots[slot].off, b->slots[slot].bytes);
    b->slots[slot] = wdlb_batch::Slot{};
    b->dirty = true;
    return WDLB_OK;
}

wdlb_status wdlb_batch_step(wdlb_batch *b, int64_t nsteps)
{
    TraceRange tr("wdlb_batch_step");
    if (!b || nsteps < 0) return WDLB_ERR_ARG;
    if (b->dirty) {
        wdlb_status s = batch_build(b);
        if (s != WDLB_OK) return s;
    }
    if (b->flow && nsteps > 0) {
        // one persistent launch for all nsteps (counters zeroed first)
        const int P = (int)b->slots.size();
        FlowLaunch F;
        F.count = b->d_flow;
        F.done = b->d_flow + 3 * P;
        F.next = reinterpret_cast<unsigned *>(b->d_flow + 6 * P);
        F.abort_flag = b->d_flow + 6 * P + 1;
        F.nsteps = (int)nsteps;
        F.parity0 = (int)(b->steps_since_build & 1);
        F.nslots = P;
        F.wait_limit = b->opt.wait_limit != 0 ? b->opt.wait_limit : kDefaultWaitLimit;
        cudaError_t e = cudaMemsetAsync(F.done, 0, (3 * P + 2) * sizeof(int), b->stream);
        if (e == cudaSuccess) e = b->L->flow_step(b->launch, F, b->stream, &b->launches);
        if (e != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "persistent batch step: %s", cudaGetErrorString(e));
        b->steps_since_build += nsteps;
        for (auto &sl : b->slots)
            if (sl.ctx) {
                sl.ctx->cur ^= (int)(nsteps & 1);
                sl.ctx->steps += nsteps;
            }
        return WDLB_OK;
    }
    int64_t left = nsteps;
    if (b->steps_since_build & 1) {
        if (left > 0) {
            wdlb_status s = batch_step_direct(b, 1);
            if (s != WDLB_OK) return s;
            left--;
        }
    }
    if (left >= 2) {
        wdlb_status s = batch_ensure_graph(b);
        if (s != WDLB_OK) return s;
        while (left >= 2) {
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "batch graph launch");
            b->launches += b->graph_launches;
            b->steps_since_build += 2;
            left -= 2;
        }
    }
    wdlb_status s = batch_step_direct(b, left);
    if (s != WDLB_OK) return s;
    for (auto &sl : b->slots)
        if (sl.ctx) {
            sl.ctx->cur ^= (int)(nsteps & 1);
            sl.ctx->steps += nsteps;
        }
    return WDLB_OK;
}

wdlb_status wdlb_batch_profile_step(wdlb_batch *b, int64_t nsteps, double ms[3])
{
    TraceRange tr("wdlb_batch_profile_step");
    if (!b || !ms || nsteps < 1) return WDLB_ERR_ARG;
    if (b->dirty) {
        wdlb_status s = batch_build(b);
        if (s != WDLB_OK) return s;
    }
    std::vector<cudaEvent_t> ev(6 * nsteps, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    for (int64_t s = 0; s < nsteps && e == cudaSuccess; s++) {
        const int parity = (int)(b->steps_since_build & 1);
        for (int part = 0; part < 3 && e == cudaSuccess; part++) {
            e = cudaEventRecord(ev[6 * s + 2 * part], b->stream);
            if (e == cudaSuccess) e = b->L->batch_step(b->launch, parity, part, -1, b->stream, &b->launches);
            if (e == cudaSuccess) e = cudaEventRecord(ev[6 * s + 2 * part + 1], b->stream);
        }
        if (e == cudaSuccess) b->steps_since_build++;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    double acc[3] = {0, 0, 0};
    for (int64_t s = 0; s < nsteps && e == cudaSuccess; s++)
        for (int part = 0; part < 3 && e == cudaSuccess; part++) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[6 * s + 2 * part], ev[6 * s + 2 * part + 1]);
            acc[part] += t;
        }
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "batch profile step: %s", cudaGetErrorString(e));
    for (auto &sl : b->slots)
        if (sl.ctx) {
            sl.ctx->cur ^= (int)(nsteps & 1);
            sl.ctx->steps += nsteps;
        }
    for (int k = 0; k < 3; k++) ms[k] = acc[k] / double(nsteps);
    return WDLB_OK;
}

wdlb_status wdlb_batch_residuals(wdlb_batch *b, int32_t interval, double *res, int32_t *status)
{
    if (!b || interval < 1) return WDLB_ERR_ARG;
    const int P = (int)b->slots.size();
    std::vector<double> r(6 * P, 0.0);
    std::vector<int> stw(P, 0);
    if (!b->dirty && P > 0) {
        // every slot in three launches and two copies, with the partition and
        // reduction order of the per-slot statistics (the same bits)
        cudaError_t e = b->L->batch_stats(b->launch, (int)(b->steps_since_build & 1), b->d_stat, P, 1, b->d_res,
                                          b->d_st, b->stream, &b->launches);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r.data(), b->d_res, 6 * size_t(P) * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(stw.data(), b->d_st, size_t(P) * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "batch residuals: %s", cudaGetErrorString(e));
    } else {
        for (int s = 0; s < P; s++) {
            wdlb_ctx *c = b->slots[s].ctx;
            if (!c) continue;
            cudaError_t e = c->L->stats(c->kp, c->dev, c->cur, 1, b->stream, &b->launches);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&r[6 * s], c->dev.result, 6 * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&stw[s], c->dev.status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
            if (e != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "batch residuals: %s", cudaGetErrorString(e));
        }
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, WDLB_ERR_CUDA, "batch residuals sync");
    for (int s = 0; s < P; s++) {
        wdlb_ctx *c = b->slots[s].ctx;
        double v = NAN;
        if (c) {
            v = flux_residual(c, &r[6 * s], interval);
            c->last_residual = v;
        }
        if (res) res[s] = v;
        if (status)
            status[s] = c ? ((stw[s] & kStatusBounds)    ? WDLB_ERR_CUDA
                             : (stw[s] & kStatusTimeout) ? WDLB_ERR_TIMEOUT
                             : (stw[s] ? WDLB_ERR_UNSTABLE : WDLB_OK))
                          : -1;
    }
    return WDLB_OK;
}

wdlb_ctx *wdlb_batch_context(wdlb_batch *b, int32_t slot)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size()) return nullptr;
    return b->slots[slot].ctx;
}

int32_t wdlb_batch_active(const wdlb_batch *b)
{
    if (!b) return 0;
    int32_t n = 0;
    for (auto &s : b->slots) n += s.ctx != nullptr;
    return n;
}

uint64_t wdlb_batch_free_bytes(const wdlb_batch *b)
{
    if (!b) return 0;
    uint64_t f = 0;
    for (auto &fr : b->free_list) f += fr.second;
    return f;
}

int64_t wdlb_batch_launch_count(const wdlb_batch *b) { return b ? b->launches : 0; }

const char *wdlb_batch_last_error(const wdlb_batch *b) { return b ? b->err.c_str() : g_create_error.c_str(); }

void wdlb_batch_destroy(wdlb_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    for (auto &s : b->slots)
        if (s.ctx) wdlb_destroy(s.ctx);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_params) cudaFree(b->d_params);
    if (b->d_stat) cudaFree(b->d_stat);
    if (b->d_res) cudaFree(b->d_res);
    if (b->d_st) cudaFree(b->d_st);
    if (b->d_flow) cudaFree(b->d_flow);
    for (auto &p : b->d_bufs)
        if (p) cudaFree(p);
    if (b->owns_pool && b->pool) cudaFree(b->pool);
    for (int g = 0; g < kMaxBatchGroups; g++) {
        if (b->side[g]) cudaStreamDestroy(b->side[g]);
        if (b->fork[g]) cudaEventDestroy(b->fork[g]);
        if (b->join[g]) cudaEventDestroy(b->join[g]);
    }
    if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

// ===========================================================================
// Serving loop: requests arrive at any time (wdlb_server_submit, any thread);
// a worker thread admits them into a batch while its pool has room, steps all
// admitted pores together in blocks of check_every steps, tests every pore's
// FP64 steady-state residual after each block and retires the converged ones
// (continuous batching: admissions and retirements interleave with steps).
// ===========================================================================

#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

struct wdlb_server {
    wdlb_batch *batch = nullptr;
    int device = 0;
    int32_t check_every = 100;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    struct Pending {
        int64_t id;
        wdlb_request req;
        std::vector<double> n, u;
        double submit_s;
    };
    struct Active {
        int64_t id;
        wdlb_request req;
        double submit_s, start_s;
    };
    std::deque<Pending> queue;
    std::vector<Active> active;   // indexed by slot
    std::vector<wdlb_result> done;
    int64_t next_id = 1, submitted = 0, admitted = 0, completed = 0;
    int64_t node_steps = 0;       // lattice-node updates executed
    double gpu_step_s = 0.0;      // device time of the blocks of time steps
    // the batch's counters as the worker last saw them (read under mu by
    // wdlb_server_info, which must not touch the batch the worker mutates)
    int32_t snap_active = 0;
    uint64_t snap_free = 0;
    int64_t snap_launches = 0;
    std::chrono::steady_clock::time_point t0;
    std::string err;
};

namespace {

double server_now(const wdlb_server *s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Worker thread only: copy the batch's counters into the snapshot.
void server_publish(wdlb_server *s)
{
    const int32_t active = wdlb_batch_active(s->batch);
    const uint64_t free_bytes = wdlb_batch_free_bytes(s->batch);
    const int64_t launches = wdlb_batch_launch_count(s->batch);
    std::lock_guard<std::mutex> lock(s->mu);
    s->snap_active = active;
    s->snap_free = free_bytes;
    s->snap_launches = launches;
}

void server_finish(wdlb_server *s, int slot, int32_t status, double residual)
{
    wdlb_server::Active a = s->active[slot];
    wdlb_ctx *c = wdlb_batch_context(s->batch, slot);
    wdlb_result r;
    std::memset(&r, 0, sizeof(r));
    r.id = a.id;
    r.status = status;
    r.residual = residual;
    r.submit_s = a.submit_s;
    r.start_s = a.start_s;
    if (c) {
        r.steps = c->steps;
        if (wdlb_pore_average(c, &r.stats) != WDLB_OK && r.status == WDLB_OK) r.status = WDLB_ERR_UNSTABLE;
        r.stats.residual = residual;
        if (a.req.out_n || a.req.out_u) wdlb_moments(c, a.req.out_n, a.req.out_u);
    }
    wdlb_batch_remove(s->batch, slot);
    r.finish_s = server_now(s);
    s->active[slot].id = 0;
    std::lock_guard<std::mutex> lock(s->mu);
    s->done.push_back(r);
    s->completed++;
}

// Two CUDA events of the worker thread, bracketing a block of time steps.
struct StepTimer {
    cudaEvent_t ev[2] = {nullptr, nullptr};
    StepTimer()
    {
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
    }
    ~StepTimer()
    {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    bool ok() const { return ev[0] && ev[1]; }
};

void server_loop(wdlb_server *s)
{
    cudaSetDevice(s->device);
    StepTimer timer;
    std::vector<double> res(s->active.size()), tmp;
    std::vector<int32_t> st(s->active.size());
    for (;;) {
        // admit while there is room
        bool admitted_now = false;
        {
            TraceRange tr_admit("server_admit");
            for (;;) {
                wdlb_server::Pending p;
                {
                    std::unique_lock<std::mutex> lock(s->mu);
                    if (s->stop) return;
                    if (s->queue.empty()) {
                        if (wdlb_batch_active(s->batch) == 0) {
                            s->cv.wait_for(lock, std::chrono::milliseconds(2));
                            continue;
                        }
                        break;
                    }
                    uint64_t need = 0;
                    if (wdlb_batch_pore_bytes(s->batch, &s->queue.front().req.desc, &need) != WDLB_OK) need = 0;
                    if (need == 0 || need > wdlb_batch_free_bytes(s->batch)) {
                        if (wdlb_batch_active(s->batch) == 0 && need != 0) {
                            // larger than the whole pool: reject it
                            p = std::move(s->queue.front());
                            s->queue.pop_front();
                            lock.unlock();
                            wdlb_result r;
                            std::memset(&r, 0, sizeof(r));
                            r.id = p.id;
                            r.status = WDLB_ERR_OOM;
                            r.submit_s = r.start_s = p.submit_s;
                            r.finish_s = server_now(s);
                            std::lock_guard<std::mutex> l2(s->mu);
                            s->done.push_back(r);
                            s->completed++;
                            continue;
                        }
                        break;
                    }
                    p = std::move(s->queue.front());
                    s->queue.pop_front();
                }
                int32_t slot = -1;
                wdlb_status a = wdlb_batch_add(s->batch, &p.req.desc, p.n.data(),
                                               p.u.empty() ? nullptr : p.u.data(), &slot);
                if (a != WDLB_OK) {
                    std::lock_guard<std::mutex> lock(s->mu);
                    if (a == WDLB_ERR_OOM) {   // fragmentation or slots: retry later
                        s->queue.push_front(std::move(p));
                        break;
                    }
                    wdlb_result r;
                    std::memset(&r, 0, sizeof(r));
                    r.id = p.id;
                    r.status = a;
                    r.submit_s = r.start_s = p.submit_s;
                    r.finish_s = server_now(s);
                    s->done.push_back(r);
                    s->completed++;
                    continue;
                }
                s->active[slot] = wdlb_server::Active{p.id, p.req, p.submit_s, server_now(s)};
                s->active[slot].req.n = s->active[slot].req.u = nullptr;
                s->admitted++;
                admitted_now = true;
            }
        }
        // u_x snapshot of the new pores (the others' snapshots are re-taken at the same state)
        if (admitted_now) wdlb_batch_residuals(s->batch, s->check_every, res.data(), st.data());
        server_publish(s);
        if (wdlb_batch_active(s->batch) == 0) continue;
        int64_t block_nodes = 0;
        for (size_t k = 0; k < s->active.size(); k++)
            if (s->active[k].id) {
                wdlb_ctx *c = wdlb_batch_context(s->batch, (int)k);
                if (c) block_nodes += c->N;
            }
        // one block of steps for every admitted pore, then the residual test
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->node_steps += block_nodes * s->check_every;
        }
        // the tables and the graph first, so that the events bracket device work only
        bool timed = timer.ok();
        if (s->batch->dirty && batch_build(s->batch) != WDLB_OK) timed = false;
        if (timed && !s->batch->flow && batch_ensure_graph(s->batch) != WDLB_OK) timed = false;
        if (timed) timed = cudaEventRecord(timer.ev[0], s->batch->stream) == cudaSuccess;
        wdlb_status step_st = wdlb_batch_step(s->batch, s->check_every);
        if (timed) timed = cudaEventRecord(timer.ev[1], s->batch->stream) == cudaSuccess;
        if (step_st != WDLB_OK || wdlb_batch_residuals(s->batch, s->check_every, res.data(), st.data()) != WDLB_OK) {
            std::lock_guard<std::mutex> lock(s->mu);
            s->err = wdlb_batch_last_error(s->batch);
            for (size_t k = 0; k < s->active.size(); k++)
                if (s->active[k].id) st[k] = WDLB_ERR_CUDA;
        }
        float ms = 0.f;   // the residual test synchronised the stream
        if (timed && cudaEventElapsedTime(&ms, timer.ev[0], timer.ev[1]) == cudaSuccess) {
            std::lock_guard<std::mutex> lock(s->mu);
            s->gpu_step_s += 1e-3 * double(ms);
        }
        for (size_t k = 0; k < s->active.size(); k++) {
            if (!s->active[k].id) continue;
            wdlb_ctx *c = wdlb_batch_context(s->batch, (int)k);
            const wdlb_request &q = s->active[k].req;
            if (st[k] != WDLB_OK)
                server_finish(s, (int)k, st[k], res[k]);
            else if (res[k] < q.tol)
                server_finish(s, (int)k, WDLB_OK, res[k]);
            else if (c && c->steps >= q.max_steps)
                server_finish(s, (int)k, WDLB_ERR_TIMEOUT, res[k]);
        }
        server_publish(s);
    }
}

}  // namespace

extern "C" {

wdlb_status wdlb_server_create(const wdlb_options *opt, uint64_t hbm_budget, int32_t max_active, int32_t check_every,
                               wdlb_server **out)
{
    if (!out || check_every < 1) return WDLB_ERR_ARG;
    *out = nullptr;
    wdlb_server *s = new (std::nothrow) wdlb_server();
    if (!s) return WDLB_ERR_OOM;
    cudaGetDevice(&s->device);
    // no tile probes inside the worker thread: its pores take the autotuner's
    // table as it stands (built-in rule for keys not yet in it)
    wdlb_options o;
    if (opt)
        o = *opt;
    else
        wdlb_default_options(&o);
    o.autotune = 0;
    wdlb_status st = wdlb_batch_create(&o, hbm_budget, max_active, &s->batch);
    if (st != WDLB_OK) {
        delete s;
        return st;
    }
    s->check_every = check_every;
    s->active.resize(max_active);
    for (auto &a : s->active) a.id = 0;
    s->snap_free = wdlb_batch_free_bytes(s->batch);
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread(server_loop, s);
    *out = s;
    return WDLB_OK;
}

wdlb_status wdlb_server_submit(wdlb_server *s, const wdlb_request *r, int64_t *id)
{
    if (!s || !r || !r->n || !(r->tol > 0) || r->max_steps < 1) return WDLB_ERR_ARG;
    wdlb_lattice lat = r->desc.lat;
    if (lat.nx < 1 || lat.ny < 1 || lat.nz < 1) return WDLB_ERR_ARG;
    const size_t N = (size_t)lat.nx * lat.ny * lat.nz;
    wdlb_server::Pending p;
    p.req = *r;
    p.n.assign(r->n, r->n + N);
    if (r->u) p.u.assign(r->u, r->u + 3 * N);
    p.submit_s = server_now(s);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        p.id = s->next_id++;
        s->submitted++;
        if (id) *id = p.id;
        s->queue.push_back(std::move(p));
    }
    s->cv.notify_one();
    return WDLB_OK;
}

int32_t wdlb_server_poll(wdlb_server *s, wdlb_result *out, int32_t cap)
{
    if (!s || !out || cap < 1) return 0;
    std::lock_guard<std::mutex> lock(s->mu);
    int32_t n = (int32_t)std::min<size_t>(cap, s->done.size());
    for (int32_t k = 0; k < n; k++) out[k] = s->done[k];
    s->done.erase(s->done.begin(), s->done.begin() + n);
    return n;
}

wdlb_status wdlb_server_info(wdlb_server *s, wdlb_server_stats *info)
{
    if (!s || !info) return WDLB_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    info->submitted = s->submitted;
    info->admitted = s->admitted;
    info->completed = s->completed;
    info->queued = (int64_t)s->queue.size();
    info->active = s->snap_active;
    info->pool_free = s->snap_free;
    info->launches = s->snap_launches;
    info->clock_s = server_now(s);
    info->node_steps = s->node_steps;
    info->gpu_step_s = s->gpu_step_s;
    return WDLB_OK;
}

void wdlb_server_destroy(wdlb_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    wdlb_batch_destroy(s->batch);
    delete s;
}

}  // extern "C"
