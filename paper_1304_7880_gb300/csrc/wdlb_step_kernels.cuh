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

template <class S, int CL, bool WALLS, bool WT, class A = typename Store<S>::T>
__global__ void __launch_bounds__(256) k_step_shell(const KParams *P, const KBufs<S, typename Store<S>::T> *B,
                                                    const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    const KParams p = P[w.slot];
    const KBufs<S, typename Store<S>::T> b = B[w.slot];
    shell_body<S, CL, WALLS, false, WT, A>(p, b, w.bx);
}

template <class S, int S2, int V, bool WALLS, bool WT, class A = float>
__global__ void __launch_bounds__(tiled::threads_of(V), (tiled::blocks_per_sm<S2, V, WT>()))
    k_step_shell_tiled(const KParams *P, const KBufs<S, float> *B, const BatchItem *it)
{
    const BatchItem w = it[blockIdx.x];
    const KParams p = P[w.slot];
    const KBufs<S, float> b = B[w.slot];
    tiled::tiled_body<S, S2, V, 0, WALLS, false, WT, A>(p, b, w.bx, w.by, w.bz);
}

}  // namespace wdlb

namespace wdlb {

// ---------------------------------------------------------------------------
// Persistent dataflow form of the batch step: one launch runs nsteps time
// steps of every pore.  The work items of one step are the batch's table in
// phase order (the moments blocks of every pore, then the smeared-density
// bricks, then the shell bricks, pore by pore within a phase); step t's items
// follow step t-1's.  A block takes the next item from an atomic counter and,
// before running it, waits until the same pore has completed every item of
// the phase it depends on:
//   smeared density (t) <- moments (t) <- shell sums + collision + push (t-1)
//   shell (t)           <- smeared density (t)
// (the earlier phases of the pore are implied).  Pores never wait for one
// another, so one pore's next phase starts while another pore's last blocks of
// the previous phase still run.  Items are handed out in dependency order, so
// a waiting block waits only on items held by running blocks: no deadlock,
// whatever the number of resident blocks.  Every wait is bounded
// (wait_limit tries); a wait that runs out sets the abort flag and the
// timeout bit of every slot, and all blocks return.
// ---------------------------------------------------------------------------
struct FlowArgs {
    const KParams *P;
    const void *B[2];           // KBufs tables of the two buffer parities
    const BatchItem *items;     // one step: moments items, then ball bricks, then shell bricks
    int n0, n1, n2;             // items per phase
    int nsteps, parity0;        // steps of this launch; buffer parity of its first step
    int nslots;
    const int *count;           // [slot * 3 + phase]: items of the slot in the phase
    int *done;                  // [slot * 3 + phase]: items completed in this launch (zeroed before)
    unsigned *next;             // the work counter (zeroed before)
    int *abort_flag;            // set when a wait gave up (zeroed before)
    int wait_limit;             // tries per wait; < 0 (tests only): a wait that is never met
};

// dynamic shared memory of the flow kernel: the shell tile (the largest of the
// three phases) and 16 bytes for the block's item and stop flag
template <int S2, int V, bool WT>
constexpr size_t flow_smem_bytes()
{
    return tiled::smem_bytes<S2, V, WT>() + 16;
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <class S, int S2, int V, bool WALLS, bool WT, class A = float>
__global__ void __launch_bounds__(tiled::threads_of(V), (tiled::blocks_per_sm<S2, V, WT>()))
    k_step_flow(FlowArgs a)
{
    typedef typename Store<S>::T T;
    static_assert(tiled::threads_of(V) == 256, "one block size for every phase");
    // the block's item and stop flag, past the shell tile in dynamic shared
    // memory (static shared memory would move the tile off its alignment)
    extern __shared__ __align__(128) unsigned char flow_smem[];
    int &s_item = reinterpret_cast<int *>(flow_smem + flow_smem_bytes<S2, V, WT>() - 16)[0];
    int &s_stop = reinterpret_cast<int *>(flow_smem + flow_smem_bytes<S2, V, WT>() - 16)[1];
    const long long per_step = (long long)a.n0 + a.n1 + a.n2;
    const long long total = per_step * a.nsteps;
    const bool probe = a.wait_limit < 0;
    const int limit = probe ? -a.wait_limit : a.wait_limit;
    for (;;) {
        if (threadIdx.x == 0) {
            long long k = (long long)atomicAdd(a.next, 1u);
            int stop = k >= total || ld_acquire_gpu(a.abort_flag) != 0;
            int item = -1;
            if (!stop) {
                const int t = (int)(k / per_step), r = (int)(k % per_step);
                const int phase = r < a.n0 ? 0 : (r < a.n0 + a.n1 ? 1 : 2);
                const int slot = a.items[r].slot;
                // the phase this one waits on, and how many of its items
                int dep = -1, target = 0;
                if (phase == 0 && t > 0) {
                    dep = 2;
                    target = t * a.count[slot * 3 + 2];
                } else if (phase > 0) {
                    dep = phase - 1;
                    target = (t + 1) * a.count[slot * 3 + dep];
                }
                if (dep >= 0 && probe) target += 1;      // tests: never met
                if (dep >= 0) {
                    int tries = 0;
                    while (ld_acquire_gpu(a.done + slot * 3 + dep) < target) {
                        if (ld_acquire_gpu(a.abort_flag) != 0 || ++tries > limit) {
                            // give up: stop every block and mark every slot
                            atomicExch(a.abort_flag, 1);
                            const KBufs<S, T> *B0 = static_cast<const KBufs<S, T> *>(a.B[0]);
                            for (int s = 0; s < a.nslots; s++)
                                if (B0[s].status) atomicOr(B0[s].status, kStatusTimeout);
                            stop = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                    // the data the producers wrote before their release are visible
                    // to this block's loads, the TMA's included
                    __threadfence();
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
                item = (int)k;
            }
            s_item = item;
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) return;
        const long long k = s_item;
        const int t = (int)(k / per_step), r = (int)(k % per_step);
        const int phase = r < a.n0 ? 0 : (r < a.n0 + a.n1 ? 1 : 2);
        const BatchItem w = a.items[r];
        const KParams p = a.P[w.slot];
        const KBufs<S, T> b = static_cast<const KBufs<S, T> *>(a.B[(a.parity0 + t) & 1])[w.slot];
        if (phase == 0)
            moments_body<S, false>(p, b, w.bx, nullptr, nullptr);
        else if (phase == 1)
            ball_brick_ct<T, S2>(p, b.nu, b.hb, b.status, w.bx, w.by, w.bz);
        else
            tiled::tiled_body<S, S2, V, 0, WALLS, false, WT, A>(p, b, w.bx, w.by, w.bz);
        __syncthreads();       // every thread's writes of this item are done
        if (threadIdx.x == 0) {
            __threadfence();   // release them before counting the item as done
            atomicAdd(a.done + w.slot * 3 + phase, 1);
        }
    }
}

// The residual test's statistics for every slot of a table, in three
// launches: FP64 moments over the slots' node blocks, then kStatBlocks blocks
// per slot with the partition of the per-lattice k_stats, then one warp per
// slot reducing its partial sums as k_stats_final does.
template <class S>
__global__ void __launch_bounds__(256) k_batch_stats_moments(const KParams *P, const KBufs<S, typename Store<S>::T> *B,
                                                             const BatchItem *it, const StatSlot *ss)
{
    const BatchItem w = it[blockIdx.x];
    const KParams p = P[w.slot];
    const KBufs<S, typename Store<S>::T> b = B[w.slot];
    double *stage = ss[w.slot].stage;
    moments_body<S, true>(p, b, w.bx, stage, stage + p.N);
}

static __global__ void __launch_bounds__(256) k_batch_stats(const KParams *P, const StatSlot *ss, int update_snap)
{
    const int slot = blockIdx.x / kStatBlocks, blk = blockIdx.x % kStatBlocks;
    const StatSlot t = ss[slot];
    if (!t.stage) return;
    const KParams p = P[slot];
    stats_body(p, t.stage, t.stage + p.N, t.snap, update_snap, t.partial, blk, kStatBlocks);
}

static __global__ void k_batch_stats_final(const StatSlot *ss, double *res, int *st)
{
    const StatSlot t = ss[blockIdx.x];
    if (!t.stage) return;
    stats_final_body(t.partial, kStatBlocks, res + 6 * blockIdx.x);
    if (threadIdx.x == 0) st[blockIdx.x] = *t.status;
}

}  // namespace wdlb
