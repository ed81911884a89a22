// Host-side launchers of the WDLB kernels, one set per population storage
// (compiled from wdlb_launch.cu once per storage type).  Every launcher
// enqueues on `st`, adds the number of kernels it launched to *launches and
// returns the first CUDA error.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wdlb_common.cuh"

namespace wdlb {

// Untyped device buffers of one lattice; the launcher casts them to its storage.
struct DevBufs {
    void *f[2];          // populations, double buffer
    void *nu;            // V4<T> per node
    void *hb;            // T per node
    void *cprev;         // 3 x Npad T
    void *tprev;         // Npad T
    void *nscale;        // Npad T
    const int4 *shell_e;
    const void *shell_k; // V4<T> per shell vector
    const int4 *ball;
    int *status;
    double *stage;       // >= 4 N doubles (FP64 staging of n and u)
    double *snap;        // N doubles (u_x snapshot)
    double *partial;     // >= kStatBlocks * 6 doubles
    double *result;      // >= 8 doubles
};

constexpr int kStatBlocks = 304;

// One block of work in a multi-lattice launch: lattice slot and block
// coordinates within it (bx: node block of 256 for the per-node kernels and
// the generic shell kernel; bx, by, bz: 8x8x8 tile for the tiled kernel).
struct BatchItem {
    int slot, bx, by, bz;
};

// Shell launch of one group of slots with the same kernel variant.
struct BatchGroup {
    int s2, walls, tiled, closure, tile, rule;   // rule: shell rule (0 full, 1 compact)
    const BatchItem *items;
    int nitems;
};

constexpr int kMaxBatchGroups = 16;

// Device tables of a multi-lattice step.  bufs[p]: one KBufs per slot (of the
// launcher's storage type), input buffer = the slot's buffer for parity p.
struct BatchLaunch {
    const KParams *params;
    const void *bufs[2];
    const BatchItem *node_items;      // blocks of 256 nodes of every slot (moments)
    int n_node_items;
    const BatchItem *ball_items;      // 8^3 bricks of the slots with a tiled ball sum
    int n_ball_items;
    size_t ball_smem;                 // largest tiled ball shared memory among them
    const BatchItem *ball_node_items; // blocks of 256 nodes of the other slots
    int n_ball_node_items;
    BatchGroup groups[kMaxBatchGroups];
    int ngroups;
};

constexpr size_t kKBufsMaxBytes = 256;   // room for one KBufs of any storage type in a table

// FP64 statistics of a batch's slots in one set of launches (the residual
// test): per slot its FP64 staging, u_x snapshot, partial sums and status
// word (stage == nullptr: empty slot).
struct StatSlot {
    double *stage, *snap, *partial;
    int *status;
};

// Persistent dataflow step of a batch (k_step_flow): per-slot item counts and
// completion counters, the work counter and the abort flag in device memory
// (done, next and abort_flag zeroed before each launch).
struct FlowLaunch {
    const int *count;    // [slot * 3 + phase]
    int *done;           // [slot * 3 + phase]
    unsigned *next;
    int *abort_flag;
    int nsteps, parity0, nslots, wait_limit;
};

struct Launchers {
    // per-context preparation outside any stream capture (kernel attributes);
    // returns whether the tiled shell kernel can serve these parameters
    bool (*prepare)(const KParams &);
    // step tables: size of one KBufs, writing it for input buffer `cur`
    size_t kbufs_bytes;
    void (*kbufs_fill)(const DevBufs &, int cur, void *out);
    // one time step of every slot in the tables (input buffers of parity p);
    // part -1: all three kernels, 0: moments, 1: smeared density, 2: shell
    // sums + collision + streaming (group -1: every shell group, else only
    // L.groups[group]).  A lattice stepped alone uses the same kernels
    // through a one-slot table, so it steps bit-identically alone and in a
    // batch.
    cudaError_t (*batch_step)(const BatchLaunch &, int parity, int part, int group, cudaStream_t,
                              int64_t *launches);
    cudaError_t (*init)(const KParams &, const DevBufs &, int cur, const double *d_n, const double *d_u,
                        cudaStream_t, int64_t *launches);
    // shell fields of the state in buffer `cur` after its moments and smeared
    // density were updated by batch_step parts 0 and 1 (no streaming)
    cudaError_t (*fields)(const KParams &, const DevBufs &, int cur, double *nbar, double *C, double *A,
                          double *u, cudaStream_t, int64_t *launches);
    // moments of the state in buffer `cur` into FP64 device arrays (either may be NULL)
    cudaError_t (*moments)(const KParams &, const DevBufs &, int cur, double *d_n, double *d_u, cudaStream_t,
                           int64_t *launches);
    // population q of buffer `cur` as FP64 into out (N doubles)
    cudaError_t (*population)(const KParams &, const DevBufs &, int cur, int q, double *out, cudaStream_t,
                              int64_t *launches);
    // moments of buffer `cur`, then FP64 statistics into result[0..5] (see k_stats)
    cudaError_t (*stats)(const KParams &, const DevBufs &, int cur, int update_snap, cudaStream_t,
                         int64_t *launches);
    // stats of every slot of the tables (input buffers of parity p) with the
    // same partition and reduction order as `stats` per slot: results into
    // res[6 slot ..], status words into st[slot]
    cudaError_t (*batch_stats)(const BatchLaunch &, int parity, const StatSlot *slots, int nslots, int update_snap,
                               double *res, int *st, cudaStream_t, int64_t *launches);
    // whether the persistent dataflow kernel serves these tables (one shell
    // group: tiled sigma 4, 8 x 8 x 4 bricks; tiled smeared density for all),
    // and its launch: F.nsteps time steps of every slot in one kernel
    bool (*flow_ok)(const BatchLaunch &);
    cudaError_t (*flow_step)(const BatchLaunch &, const FlowLaunch &F, cudaStream_t, int64_t *launches);
    // energy-equation fields Q, B, F^T (FP64 device arrays: N, 3N, 3N) on the
    // temperature T (N doubles) from the state in buffer `cur`, after its
    // moments and smeared density were updated by batch_step parts 0 and 1
    cudaError_t (*thermal)(const KParams &, const DevBufs &, int cur, const double *T, double *Q, double *B,
                           double *FT, cudaStream_t, int64_t *launches);
};

const Launchers &launchers_f64();
const Launchers &launchers_f32();
// FP32 storage with the collision in double-word arithmetic (WDLB_COLLISION_DW)
const Launchers &launchers_f32dw();
const Launchers &launchers_f16();

// FP64 sum of d_n over fluid nodes into *result (device), one launch pair.
cudaError_t launch_sum_density(const KParams &, const double *d_n, double *partial, double *result,
                               cudaStream_t, int64_t *launches);

}  // namespace wdlb
