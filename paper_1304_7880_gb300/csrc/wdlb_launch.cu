// Launchers for one population storage type, selected at compile time by
// WDLB_STORAGE (0: FP64, 1: FP32 deviation, 2: FP16 relative deviation).
#include "wdlb_kernels.cuh"
#include "wdlb_launch.h"
#include "wdlb_shell_tiled.cuh"
#include "wdlb_step_kernels.cuh"
#include "wdlb_tables.h"

#include <algorithm>
#include <cstring>

#ifndef WDLB_STORAGE
#error "compile with -DWDLB_STORAGE=0|1|2"
#endif

namespace wdlb {
namespace {

#if WDLB_STORAGE == 0
typedef double S;
#elif WDLB_STORAGE == 1
typedef float S;
#else
typedef __half S;
#endif
typedef Store<S>::T T;
// arithmetic of the collision: the storage's compute type, or (built with
// WDLB_DW_COLLISION, FP32 storage only) double-word pairs of floats
#if WDLB_DW_COLLISION
static_assert(WDLB_STORAGE == 1, "the double-word collision is built for FP32 storage");
typedef dwf A;
#else
typedef T A;
#endif
// the double-word collision is compiled for lattices with walls only (the
// library refuses it for periodic boxes, which FP32 already serves at 1e-5)
constexpr bool kPeriodic = !is_dw<A>::value;

constexpr int kThreads = 256;

inline int blocks_for(int n) { return (n + kThreads - 1) / kThreads; }

KBufs<S, T> typed(const DevBufs &d, int cur)
{
    KBufs<S, T> b;
    b.f_in = static_cast<const S *>(d.f[cur]);
    b.f_out = static_cast<S *>(d.f[cur ^ 1]);
    b.nu = static_cast<V4<T> *>(d.nu);
    b.hb = static_cast<T *>(d.hb);
    b.cprev = static_cast<T *>(d.cprev);
    b.tprev = static_cast<T *>(d.tprev);
    b.nscale = static_cast<T *>(d.nscale);
    b.shell_e = d.shell_e;
    b.shell_k = static_cast<const V4<T> *>(d.shell_k);
    b.ball = d.ball;
    b.status = d.status;
    b.out_nbar = b.out_C = b.out_A = b.out_u = nullptr;
    return b;
}

template <int CL, bool WALLS>
void launch_fields_shell(const KParams &p, const KBufs<S, T> &b, cudaStream_t st)
{
    if (p.shell_rule)
        k_shell_collide<S, CL, WALLS, true, true><<<blocks_for(p.N), kThreads, 0, st>>>(p, b);
    else
        k_shell_collide<S, CL, WALLS, true, false><<<blocks_for(p.N), kThreads, 0, st>>>(p, b);
}

#if WDLB_STORAGE != 0
// The tiled kernel is compiled for the Carnahan-Starling closure (the default),
// sigma in {3, 4, 6}, the three tile variants and both shell rules; other
// closures and sigmas use the generic kernel.
template <int S2, int V, bool WALLS, bool WT>
cudaError_t tiled_attr()
{
    return cudaFuncSetAttribute(k_step_shell_tiled<S, S2, V, WALLS, WT, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tiled::smem_bytes<S2, V, WT>());
}

template <int S2, int V, bool WT>
cudaError_t tiled_attr_w(bool walls)
{
    if constexpr (kPeriodic)
        return walls ? tiled_attr<S2, V, true, WT>() : tiled_attr<S2, V, false, WT>();
    else
        return walls ? tiled_attr<S2, V, true, WT>() : cudaErrorNotSupported;
}

template <int S2, bool WT>
cudaError_t tiled_attr_v(int v, bool walls)
{
    return v == 0 ? tiled_attr_w<S2, 0, WT>(walls)
                  : (v == 1 ? tiled_attr_w<S2, 1, WT>(walls) : tiled_attr_w<S2, 2, WT>(walls));
}

template <int S2>
cudaError_t tiled_attr_r(int v, bool walls, bool wt)
{
    return wt ? tiled_attr_v<S2, true>(v, walls) : tiled_attr_v<S2, false>(v, walls);
}

template <int S2, int V, bool WALLS, bool WT>
void launch_tiled_group(const BatchLaunch &L, const KBufs<S, float> *B, const BatchGroup &G, cudaStream_t st)
{
    k_step_shell_tiled<S, S2, V, WALLS, WT, A>
        <<<G.nitems, tiled::threads_of(V), tiled::smem_bytes<S2, V, WT>(), st>>>(L.params, B, G.items);
}

template <int S2, int V, bool WT>
void launch_tiled_r(const BatchLaunch &L, const KBufs<S, float> *B, const BatchGroup &G, cudaStream_t st)
{
    if (G.walls)
        launch_tiled_group<S2, V, true, WT>(L, B, G, st);
    else if constexpr (kPeriodic)
        launch_tiled_group<S2, V, false, WT>(L, B, G, st);
}

template <int S2, int V>
void launch_tiled_w(const BatchLaunch &L, const KBufs<S, float> *B, const BatchGroup &G, cudaStream_t st)
{
    if (G.rule)
        launch_tiled_r<S2, V, true>(L, B, G, st);
    else
        launch_tiled_r<S2, V, false>(L, B, G, st);
}

template <int S2>
void launch_tiled_v(const BatchLaunch &L, const KBufs<S, float> *B, const BatchGroup &G, cudaStream_t st)
{
    if (G.tile == 0)
        launch_tiled_w<S2, 0>(L, B, G, st);
    else if (G.tile == 1)
        launch_tiled_w<S2, 1>(L, B, G, st);
    else
        launch_tiled_w<S2, 2>(L, B, G, st);
}
#endif

#if WDLB_STORAGE != 0
// A compiled shell table (tiled::ct) is used only if it equals the library's
// table for this sigma and rule: the same vectors in the same order, and for
// the compact rule one weight per orbit.
template <int S2, bool WT>
bool compiled_table_matches()
{
    if constexpr (!tiled::ct::compiled<S2, WT>()) {
        return true;
    } else {
        const double sigma = 0.5 * S2;
        std::vector<int> e;
        std::vector<double> wts;
        double w = 0.0;
        if (WT) {
            if (!build_shell_compact(sigma, e, wts)) return false;
        } else {
            build_shell(sigma, e, &w);
        }
        constexpr tiled::ct::PairTable<S2, WT> T{};
        if ((int)e.size() != 6 * T.n) return false;
        for (int m = 0; m < T.n; m++) {
            if (e[6 * m] != T.ex[m] || e[6 * m + 1] != T.ey[m] || e[6 * m + 2] != T.ez[m]) return false;
            if (WT && wts[2 * m] != wts[2 * tiled::ct::first_pair_of_orbit<S2>(T.orb[m])]) return false;
        }
        return true;
    }
}

template <int S2>
bool table_ok(bool wt)
{
    static const bool full = compiled_table_matches<S2, false>(), compact = compiled_table_matches<S2, true>();
    return wt ? compact : full;
}
#endif

bool tiled_eligible(const KParams &p)
{
#if WDLB_STORAGE != 0
    return (p.s2 == 6 || p.s2 == 8 || p.s2 == 12) && p.closure == 0 && p.nx >= tiled::TX && p.ny >= tiled::TY;
#else
    (void)p;
    return false;
#endif
}

bool do_prepare(const KParams &p)
{
    if (!tiled_eligible(p) || p.tile < 0 || p.tile >= tiled::kVariants) return false;
#if WDLB_STORAGE != 0
    const bool walls = p.walls != 0, wt = p.shell_rule != 0;
    if (!(p.s2 == 6 ? table_ok<6>(wt) : (p.s2 == 8 ? table_ok<8>(wt) : table_ok<12>(wt)))) return false;
    cudaError_t e = p.s2 == 6 ? tiled_attr_r<6>(p.tile, walls, wt)
                              : (p.s2 == 8 ? tiled_attr_r<8>(p.tile, walls, wt) : tiled_attr_r<12>(p.tile, walls, wt));
    return e == cudaSuccess;
#else
    return false;
#endif
}

cudaError_t do_init(const KParams &p, const DevBufs &d, int cur, const double *d_n, const double *d_u,
                    cudaStream_t st, int64_t *launches)
{
    KBufs<S, T> b = typed(d, cur ^ 1);   // f_out = buffer `cur`
    k_init<S><<<blocks_for(p.N), kThreads, 0, st>>>(p, b, d_n, d_u);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t do_thermal(const KParams &p, const DevBufs &d, int cur, const double *T, double *Q, double *B,
                       double *FT, cudaStream_t st, int64_t *launches)
{
    k_thermal_fields<S><<<blocks_for(p.N), kThreads, 0, st>>>(p, typed(d, cur), T, Q, B, FT);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t do_fields(const KParams &p, const DevBufs &d, int cur, double *nbar, double *C, double *A, double *u,
                      cudaStream_t st, int64_t *launches)
{
    KBufs<S, T> b = typed(d, cur);
    b.out_nbar = nbar;
    b.out_C = C;
    b.out_A = A;
    b.out_u = u;
#define WDLB_CASE(CL, W)                                \
    if (p.closure == CL && (p.walls != 0) == W) {       \
        launch_fields_shell<CL, W>(p, b, st);           \
        *launches += 1;                                 \
        return cudaGetLastError();                      \
    }
    WDLB_CASE(0, true) WDLB_CASE(0, false) WDLB_CASE(1, true) WDLB_CASE(1, false) WDLB_CASE(2, true)
    WDLB_CASE(2, false)
#undef WDLB_CASE
    return cudaErrorInvalidValue;
}

cudaError_t do_moments(const KParams &p, const DevBufs &d, int cur, double *d_n, double *d_u, cudaStream_t st,
                       int64_t *launches)
{
    KBufs<S, T> b = typed(d, cur);
    k_moments<S, true><<<blocks_for(p.N), kThreads, 0, st>>>(p, b, d_n, d_u);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t do_population(const KParams &p, const DevBufs &d, int cur, int q, double *out, cudaStream_t st,
                          int64_t *launches)
{
    k_pop_to_f64<S><<<blocks_for(p.N), kThreads, 0, st>>>(p, static_cast<const S *>(d.f[cur]),
                                                          static_cast<const T *>(d.nscale), q, out);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t do_stats(const KParams &p, const DevBufs &d, int cur, int update_snap, cudaStream_t st,
                     int64_t *launches)
{
    KBufs<S, T> b = typed(d, cur);
    double *sn = d.stage, *su = d.stage + p.N;
    k_moments<S, true><<<blocks_for(p.N), kThreads, 0, st>>>(p, b, sn, su);
    k_stats<<<kStatBlocks, kThreads, 0, st>>>(p, sn, su, d.snap, update_snap, d.partial);
    k_stats_final<<<1, 32, 0, st>>>(d.partial, kStatBlocks, d.result);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t do_batch_stats(const BatchLaunch &L, int parity, const StatSlot *slots, int nslots, int update_snap,
                           double *res, int *st_out, cudaStream_t st, int64_t *launches)
{
    if (nslots < 1 || L.n_node_items < 1) return cudaSuccess;
    const KBufs<S, T> *B = static_cast<const KBufs<S, T> *>(L.bufs[parity & 1]);
    k_batch_stats_moments<S><<<L.n_node_items, kThreads, 0, st>>>(L.params, B, L.node_items, slots);
    k_batch_stats<<<nslots * kStatBlocks, kThreads, 0, st>>>(L.params, slots, update_snap);
    k_batch_stats_final<<<nslots, 32, 0, st>>>(slots, res, st_out);
    *launches += 3;
    return cudaGetLastError();
}

void kbufs_fill(const DevBufs &d, int cur, void *out)
{
    KBufs<S, T> b = typed(d, cur);
    std::memcpy(out, &b, sizeof(b));
}

cudaError_t do_batch_step(const BatchLaunch &L, int parity, int part, int group, cudaStream_t st,
                          int64_t *launches)
{
    const KBufs<S, T> *B = static_cast<const KBufs<S, T> *>(L.bufs[parity & 1]);
    if ((part < 0 || part == 0) && L.n_node_items > 0) {
        k_step_moments<S><<<L.n_node_items, kThreads, 0, st>>>(L.params, B, L.node_items);
        *launches += 1;
    }
    if (part < 0 || part == 1) {
        if (L.n_ball_items > 0) {
            k_step_ball_tiled<S><<<L.n_ball_items, kThreads, L.ball_smem, st>>>(L.params, B, L.ball_items);
            *launches += 1;
        }
        if (L.n_ball_node_items > 0) {
            k_step_ball<S><<<L.n_ball_node_items, kThreads, 0, st>>>(L.params, B, L.ball_node_items);
            *launches += 1;
        }
    }
    if (part >= 0 && part != 2) return cudaGetLastError();
    for (int g = 0; g < L.ngroups; g++) {
        const BatchGroup &G = L.groups[g];
        if (G.nitems == 0 || (group >= 0 && g != group)) continue;
#if WDLB_STORAGE != 0
        if (G.tiled) {
            if (G.s2 == 6)
                launch_tiled_v<6>(L, B, G, st);
            else if (G.s2 == 8)
                launch_tiled_v<8>(L, B, G, st);
            else
                launch_tiled_v<12>(L, B, G, st);
            *launches += 1;
            continue;
        }
#endif
#define WDLB_SB(CLV, WV)                                                                         \
    do {                                                                                         \
        if (G.rule)                                                                              \
            k_step_shell<S, CLV, WV, true, A><<<G.nitems, kThreads, 0, st>>>(L.params, B, G.items);  \
        else                                                                                     \
            k_step_shell<S, CLV, WV, false, A><<<G.nitems, kThreads, 0, st>>>(L.params, B, G.items); \
    } while (0)
        if (G.walls) {
            if (G.closure == 0) WDLB_SB(0, true);
            else if (G.closure == 1) WDLB_SB(1, true);
            else WDLB_SB(2, true);
        } else if constexpr (kPeriodic) {
            if (G.closure == 0) WDLB_SB(0, false);
            else if (G.closure == 1) WDLB_SB(1, false);
            else WDLB_SB(2, false);
        }
#undef WDLB_SB
        *launches += 1;
    }
    return cudaGetLastError();
}

bool do_flow_ok(const BatchLaunch &L)
{
#if WDLB_STORAGE != 0
    if (L.n_ball_node_items != 0 || L.ngroups != 1 || L.n_ball_items == 0) return false;
    const BatchGroup &G = L.groups[0];
    return G.tiled && G.s2 == 8 && G.tile == 2 && G.closure == 0 && G.nitems > 0;
#else
    (void)L;
    return false;
#endif
}

#if WDLB_STORAGE != 0
template <bool WALLS, bool WT>
cudaError_t launch_flow(const BatchLaunch &L, const FlowLaunch &F, cudaStream_t st)
{
    auto kern = k_step_flow<S, 8, 2, WALLS, WT, A>;
    const size_t smem = flow_smem_bytes<8, 2, WT>();
    static int grid = 0;   // one per template instance: resident blocks on the whole GPU
    if (grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0, sms = 0, per_sm = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
        if (e != cudaSuccess) return e;
        grid = std::max(1, sms * per_sm);
    }
    FlowArgs a;
    a.P = L.params;
    a.B[0] = L.bufs[0];
    a.B[1] = L.bufs[1];
    a.items = L.node_items;   // moments, smeared-density and shell items are contiguous in the table
    a.n0 = L.n_node_items;
    a.n1 = L.n_ball_items;
    a.n2 = L.groups[0].nitems;
    a.nsteps = F.nsteps;
    a.parity0 = F.parity0;
    a.nslots = F.nslots;
    a.count = F.count;
    a.done = F.done;
    a.next = F.next;
    a.abort_flag = F.abort_flag;
    a.wait_limit = F.wait_limit;
    kern<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}
#endif

cudaError_t do_flow_step(const BatchLaunch &L, const FlowLaunch &F, cudaStream_t st, int64_t *launches)
{
#if WDLB_STORAGE != 0
    if (!do_flow_ok(L)) return cudaErrorInvalidValue;
    const BatchGroup &G = L.groups[0];
    cudaError_t e = cudaErrorNotSupported;
    if (G.walls)
        e = G.rule ? launch_flow<true, true>(L, F, st) : launch_flow<true, false>(L, F, st);
    else if constexpr (kPeriodic)
        e = G.rule ? launch_flow<false, true>(L, F, st) : launch_flow<false, false>(L, F, st);
    *launches += 1;
    return e;
#else
    (void)L;
    (void)F;
    (void)st;
    (void)launches;
    return cudaErrorInvalidValue;
#endif
}

static_assert(sizeof(KBufs<S, T>) <= kKBufsMaxBytes, "KBufs larger than its table slot");
const Launchers kL = {do_prepare, sizeof(KBufs<S, T>), kbufs_fill, do_batch_step, do_init,      do_fields,
                      do_moments, do_population,       do_stats,   do_batch_stats, do_flow_ok, do_flow_step,
                      do_thermal};

}  // namespace

#if WDLB_STORAGE == 0
const Launchers &launchers_f64() { return kL; }

cudaError_t launch_sum_density(const KParams &p, const double *d_n, double *partial, double *result,
                               cudaStream_t st, int64_t *launches)
{
    k_sum_density<<<kStatBlocks, kThreads, 0, st>>>(p, d_n, partial);
    k_sum_final<<<1, 32, 0, st>>>(partial, kStatBlocks, result);
    *launches += 2;
    return cudaGetLastError();
}
#elif WDLB_STORAGE == 1 && WDLB_DW_COLLISION
const Launchers &launchers_f32dw() { return kL; }
#elif WDLB_STORAGE == 1
const Launchers &launchers_f32() { return kL; }
#else
const Launchers &launchers_f16() { return kL; }
#endif

}  // namespace wdlb
