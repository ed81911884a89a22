// Launchers for one population storage type, selected at compile time by
// WDLB_STORAGE (0: FP64, 1: FP32 deviation, 2: FP16 relative deviation).
#include "wdlb_kernels.cuh"
#include "wdlb_launch.h"

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
    b.shell_e = d.shell_e;
    b.shell_k = static_cast<const V4<T> *>(d.shell_k);
    b.ball = d.ball;
    b.status = d.status;
    b.out_nbar = b.out_C = b.out_A = b.out_u = nullptr;
    return b;
}

template <int CL, int OM, bool WALLS, bool FIELDS>
void launch_shell(const KParams &p, const KBufs<S, T> &b, cudaStream_t st)
{
    k_shell_collide<S, CL, OM, WALLS, FIELDS><<<blocks_for(p.N), kThreads, 0, st>>>(p, b);
}

template <bool FIELDS>
void dispatch_shell(const KParams &p, const KBufs<S, T> &b, cudaStream_t st)
{
#define WDLB_CASE(CL, OM, W)                                            \
    if (p.closure == CL && p.omega_mode == OM && (p.walls != 0) == W) { \
        launch_shell<CL, OM, W, FIELDS>(p, b, st);                      \
        return;                                                         \
    }
    WDLB_CASE(0, 0, true) WDLB_CASE(0, 0, false) WDLB_CASE(0, 1, true) WDLB_CASE(0, 1, false)
    WDLB_CASE(1, 0, true) WDLB_CASE(1, 0, false) WDLB_CASE(1, 1, true) WDLB_CASE(1, 1, false)
    WDLB_CASE(2, 0, true) WDLB_CASE(2, 0, false) WDLB_CASE(2, 1, true) WDLB_CASE(2, 1, false)
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
    k_pop_to_f64<S><<<blocks_for(p.N), kThreads, 0, st>>>(p, static_cast<const S *>(d.f[cur]), q, out);
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

const Launchers kL = {do_init, do_step, do_step_part, do_fields, do_moments, do_population, do_stats};

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
