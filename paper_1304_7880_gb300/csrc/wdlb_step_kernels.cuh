// Step kernels of the WDLB time step, one launch per phase for every
// lattice of a table of work items (BatchItem: slot and block coordinates).
// Every block copies its slot's parameters and buffer pointers into
// registers and runs the per-block body of wdlb_kernels.cuh or
// wdlb_shell_tiled.cuh.  A lattice stepped alone runs these same kernels
// through a one-slot table, so it steps bit-identically alone and in a batch.
#pragma once

#include "wdlb_kernels.cuh"
#include "wdlb_launch.h"
#include "wdlb_shell_tiled.cuh"

namespace wdlb {

template <class S>
__global__ void __launch_bounds__(256) k_step_moments(const KParams *P, const KBufs<S, typename Store<S>::T> *B,
                                                      const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    const KParams p = P[w.slot];
    const KBufs<S, typename Store<S>::T> b = B[w.slot];
    moments_body<S, false>(p, b, w.bx, nullptr, nullptr);
}

template <class S>
__global__ void __launch_bounds__(256) k_step_ball(const KParams *P, const KBufs<S, typename Store<S>::T> *B,
                                                   const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    const KParams p = P[w.slot];
    const KBufs<S, typename Store<S>::T> b = B[w.slot];
    ball_body<typename Store<S>::T>(p, b.nu, b.hb, b.ball, b.status, w.bx);
}

template <class S>
__global__ void __launch_bounds__(256) k_step_ball_tiled(const KParams *P, const KBufs<S, typename Store<S>::T> *B,
                                                         const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    const KParams p = P[w.slot];
    const KBufs<S, typename Store<S>::T> b = B[w.slot];
    typedef typename Store<S>::T T;
    switch (p.s2) {      // uniform over the block (one slot per block)
    case 6: ball_brick_ct<T, 6>(p, b.nu, b.hb, b.status, w.bx, w.by, w.bz); break;
    case 8: ball_brick_ct<T, 8>(p, b.nu, b.hb, b.status, w.bx, w.by, w.bz); break;
    case 12: ball_brick_ct<T, 12>(p, b.nu, b.hb, b.status, w.bx, w.by, w.bz); break;
    case 16: ball_brick_ct<T, 16>(p, b.nu, b.hb, b.status, w.bx, w.by, w.bz); break;
    default: ball_tiled_body<T>(p, b.nu, b.hb, b.ball, b.status, w.bx, w.by, w.bz); break;
    }
}

template <class S, int CL, bool WALLS, bool WT>
__global__ void __launch_bounds__(256) k_step_shell(const KParams *P, const KBufs<S, typename Store<S>::T> *B,
                                                    const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    const KParams p = P[w.slot];
    const KBufs<S, typename Store<S>::T> b = B[w.slot];
    shell_body<S, CL, WALLS, false, WT>(p, b, w.bx);
}

template <class S, int S2, int V, bool WALLS, bool WT>
__global__ void __launch_bounds__(tiled::threads_of(V), (tiled::blocks_per_sm<S2, V, WT>()))
    k_step_shell_tiled(const KParams *P, const KBufs<S, float> *B, const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    const KParams p = P[w.slot];
    const KBufs<S, float> b = B[w.slot];
    tiled::tiled_body<S, S2, V, 0, WALLS, false, WT>(p, b, w.bx, w.by, w.bz);
}

}  // namespace wdlb
