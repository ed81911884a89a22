// Launchers for one population storage type, selected at compile time by
// WDLB_STORAGE (0: FP64, 1: FP32 deviation, 2: FP16 relative deviation).
#include "wdlb_kernels.cuh"
#include "wdlb_launch.h"
#include "wdlb_shell_tiled.cuh"

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
    return cudaFuncSetAttribute(tiled::k_shell_tiled<S, S2, 0, WALLS, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiled::smem_bytes<S2>());
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

const Launchers kL = {do_prepare, do_init, do_step, do_step_part, do_fields, do_moments, do_population, do_stats};

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
