// Launchers for one population storage type, selected at compile time by
// WDLB_STORAGE (0: FP64, 1: FP32 deviation, 2: FP16 relative deviation).
#include "wdlb_kernels.cuh"
#include "wdlb_launch.h"
#include "wdlb_shell_tiled.cuh"

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

constexpr int kThreads = 256;

inline int blocks_for(int n) { return (n + kThreads - 1) / kThreads; }

// ---- multi-lattice kernels: one launch for all slots, same kernel bodies ----
__global__ void __launch_bounds__(256) k_moments_batch(const KParams *P, const KBufs<S, T> *B, const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    moments_body<S, false>(P[w.slot], B[w.slot], w.bx, nullptr, nullptr);
}

__global__ void __launch_bounds__(256) k_ball_batch(const KParams *P, const KBufs<S, T> *B, const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    const KBufs<S, T> &b = B[w.slot];
    ball_body<T>(P[w.slot], b.nu, b.hb, b.ball, b.status, w.bx);
}

template <int CL, bool WALLS>
__global__ void __launch_bounds__(256) k_shell_batch(const KParams *P, const KBufs<S, T> *B, const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    shell_body<S, CL, WALLS, false>(P[w.slot], B[w.slot], w.bx);
}

#if WDLB_STORAGE != 0
template <int S2, bool WALLS>
__global__ void __launch_bounds__(tiled::THREADS, 2) k_tiled_batch(const KParams *P, const KBufs<S, float> *B,
                                                                  const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    tiled::tiled_body<S, S2, 0, WALLS, false>(P[w.slot], B[w.slot], w.bx, w.by, w.bz);
}
#endif

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

template <int CL, bool WALLS, bool FIELDS>
void launch_shell(const KParams &p, const KBufs<S, T> &b, cudaStream_t st)
{
    k_shell_collide<S, CL, WALLS, FIELDS><<<blocks_for(p.N), kThreads, 0, st>>>(p, b);
}

#if WDLB_STORAGE != 0
// The tiled kernel is compiled for the Carnahan-Starling closure (the default)
// and sigma in {3, 4, 6}; other closures and sigmas use k_shell_collide.
template <int S2, bool WALLS>
cudaError_t tiled_attr()
{
    cudaError_t e = cudaFuncSetAttribute(tiled::k_shell_tiled<S, S2, 0, WALLS, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiled::smem_bytes<S2>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tiled_batch<S2, WALLS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tiled::smem_bytes<S2>());
}

template <int S2, bool WALLS>
void launch_tiled(const KParams &p, const KBufs<S, T> &b, cudaStream_t st)
{
    dim3 grid((p.nx + tiled::TX - 1) / tiled::TX, (p.ny + tiled::TY - 1) / tiled::TY,
              (p.nz + tiled::TZ - 1) / tiled::TZ);
    tiled::k_shell_tiled<S, S2, 0, WALLS, false><<<grid, tiled::THREADS, tiled::smem_bytes<S2>(), st>>>(p, b);
}

template <int S2>
void tiled_s2(const KParams &p, const KBufs<S, T> *b, cudaStream_t st, cudaError_t *attr)
{
    if (p.walls) {
        if (attr) *attr = tiled_attr<S2, true>();
        else launch_tiled<S2, true>(p, *b, st);
    } else {
        if (attr) *attr = tiled_attr<S2, false>();
        else launch_tiled<S2, false>(p, *b, st);
    }
}

// attr != nullptr: set kernel attributes instead of launching
void dispatch_tiled(const KParams &p, const KBufs<S, T> *b, cudaStream_t st, cudaError_t *attr)
{
    switch (p.s2) {
    case 6: tiled_s2<6>(p, b, st, attr); break;
    case 8: tiled_s2<8>(p, b, st, attr); break;
    case 12: tiled_s2<12>(p, b, st, attr); break;
    default: break;
    }
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
    if (!tiled_eligible(p)) return false;
#if WDLB_STORAGE != 0
    cudaError_t e = cudaSuccess;
    dispatch_tiled(p, nullptr, nullptr, &e);
    return e == cudaSuccess;
#else
    return false;
#endif
}

template <bool FIELDS>
void dispatch_shell(const KParams &p, const KBufs<S, T> &b, cudaStream_t st)
{
#if WDLB_STORAGE != 0
    if (!FIELDS && p.tiled) {
        dispatch_tiled(p, &b, st, nullptr);
        return;
    }
#endif
#define WDLB_CASE(CL, W)                                \
    if (p.closure == CL && (p.walls != 0) == W) {       \
        launch_shell<CL, W, FIELDS>(p, b, st);          \
        return;                                         \
    }
    WDLB_CASE(0, true) WDLB_CASE(0, false) WDLB_CASE(1, true) WDLB_CASE(1, false) WDLB_CASE(2, true)
    WDLB_CASE(2, false)
#undef WDLB_CASE
}

void moments_ball(const KParams &p, const KBufs<S, T> &b, cudaStream_t st)
{
    k_moments<S, false><<<blocks_for(p.N), kThreads, 0, st>>>(p, b, nullptr, nullptr);
    k_ball<T><<<blocks_for(p.N), kThreads, 0, st>>>(p, b.nu, b.hb, b.ball, b.status);
}

cudaError_t do_init(const KParams &p, const DevBufs &d, int cur, const double *d_n, const double *d_u,
                    cudaStream_t st, int64_t *launches)
{
    KBufs<S, T> b = typed(d, cur ^ 1);   // f_out = buffer `cur`
    k_init<S><<<blocks_for(p.N), kThreads, 0, st>>>(p, b, d_n, d_u);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t do_step(const KParams &p, const DevBufs &d, int cur, cudaStream_t st, int64_t *launches)
{
    KBufs<S, T> b = typed(d, cur);
    moments_ball(p, b, st);
    dispatch_shell<false>(p, b, st);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t do_step_part(const KParams &p, const DevBufs &d, int cur, int part, cudaStream_t st, int64_t *launches)
{
    KBufs<S, T> b = typed(d, cur);
    if (part == 0)
        k_moments<S, false><<<blocks_for(p.N), kThreads, 0, st>>>(p, b, nullptr, nullptr);
    else if (part == 1)
        k_ball<T><<<blocks_for(p.N), kThreads, 0, st>>>(p, b.nu, b.hb, b.ball, b.status);
    else
        dispatch_shell<false>(p, b, st);
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
    moments_ball(p, b, st);
    dispatch_shell<true>(p, b, st);
    *launches += 3;
    return cudaGetLastError();
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

void kbufs_fill(const DevBufs &d, int cur, void *out)
{
    KBufs<S, T> b = typed(d, cur);
    std::memcpy(out, &b, sizeof(b));
}

cudaError_t do_batch_step(const BatchLaunch &L, int parity, cudaStream_t st, int64_t *launches)
{
    const KBufs<S, T> *B = static_cast<const KBufs<S, T> *>(L.bufs[parity & 1]);
    if (L.n_node_items > 0) {
        k_moments_batch<<<L.n_node_items, kThreads, 0, st>>>(L.params, B, L.node_items);
        k_ball_batch<<<L.n_node_items, kThreads, 0, st>>>(L.params, B, L.node_items);
        *launches += 2;
    }
    for (int g = 0; g < L.ngroups; g++) {
        const BatchGroup &G = L.groups[g];
        if (G.nitems == 0) continue;
#if WDLB_STORAGE != 0
        if (G.tiled) {
            const size_t sm = G.s2 == 6 ? tiled::smem_bytes<6>() : (G.s2 == 8 ? tiled::smem_bytes<8>()
                                                                               : tiled::smem_bytes<12>());
#define WDLB_TB(S2V, WV) k_tiled_batch<S2V, WV><<<G.nitems, tiled::THREADS, sm, st>>>(L.params, B, G.items)
            if (G.s2 == 6) { if (G.walls) WDLB_TB(6, true); else WDLB_TB(6, false); }
            else if (G.s2 == 8) { if (G.walls) WDLB_TB(8, true); else WDLB_TB(8, false); }
            else { if (G.walls) WDLB_TB(12, true); else WDLB_TB(12, false); }
#undef WDLB_TB
            *launches += 1;
            continue;
        }
#endif
#define WDLB_SB(CLV, WV) k_shell_batch<CLV, WV><<<G.nitems, kThreads, 0, st>>>(L.params, B, G.items)
        if (G.closure == 0) { if (G.walls) WDLB_SB(0, true); else WDLB_SB(0, false); }
        else if (G.closure == 1) { if (G.walls) WDLB_SB(1, true); else WDLB_SB(1, false); }
        else { if (G.walls) WDLB_SB(2, true); else WDLB_SB(2, false); }
#undef WDLB_SB
        *launches += 1;
    }
    return cudaGetLastError();
}

const Launchers kL = {do_prepare, sizeof(KBufs<S, T>), kbufs_fill, do_batch_step, do_init, do_step, do_step_part, do_fields, do_moments, do_population, do_stats};

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
#elif WDLB_STORAGE == 1
const Launchers &launchers_f32() { return kL; }
#else
const Launchers &launchers_f16() { return kL; }
#endif

}  // namespace wdlb
