// Shared definitions of the WDLB CUDA library (device and host side).
//
// Lattice: D3Q19 (Sec. 5, Numerical results), lattice units with k_B T = 1/3.
// This library's population order: rest; faces +x -x +y -y +z -z; edges
// (+x+y) (-x-y) (+x-y) (-x+y) (+x+z) (-x-z) (+x-z) (-x+z) (+y+z) (-y-z)
// (+y-z) (-y+z).  Opposite directions are adjacent (q, q^1 for q >= 1).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wdlb {

constexpr int NQ = 19;
constexpr double CS2 = 1.0 / 3.0;
constexpr double KAPPA = 2.0;   // implicit factor of the field-velocity predictor

__host__ __device__ constexpr int cx_of(int q)
{
    constexpr int t[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int cy_of(int q)
{
    constexpr int t[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[q];
}
__host__ __device__ constexpr int cz_of(int q)
{
    constexpr int t[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}
__host__ __device__ constexpr double w_of(int q)
{
    return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr int opp_of(int q) { return q == 0 ? 0 : (((q - 1) ^ 1) + 1); }

template <class T>
struct alignas(4 * sizeof(T)) V4 {
    T x, y, z, w;
};

// Scalar parameters of one lattice, passed by value to every kernel.
struct KParams {
    int nx, ny, nz, walls;   // walls: solid planes z = 0 and z = nz-1
    int N, Npad;             // node count, padded stride of per-node arrays
    int nshell, nball;
    int closure, omega_mode, interactions;
    int s2;                  // 2 sigma if it is an integer, else 0 (selects a compiled shell)
    int tiled;               // 1: use the shared-memory tiled shell kernel
    int tile;                // its shape (tile variant 0, 1, 2; see wdlb_shell_tiled.cuh)
    int ball_r;              // largest |component| of a ball vector (halo of the tiled ball sum)
    int ball_tiled;          // 1: use the shared-memory tiled ball sum
    int shell_rule;          // 0: full shell, uniform weight wshell; 1: compact shell,
                             // per-vector weights in shell_k[m].w (wshell = 1)
    int tma;                 // 1: the tiled shell kernel stages interior bricks' tiles by TMA
    int wait_limit;          // polls of an mbarrier wait before it gives up (status bit 4)
    const void *tmaps;       // device tensor maps of nu and hb for the TMA tile (64-byte aligned)
    double g[3];             // external acceleration
    double omega;            // 1/tau
    double tau;
    double k_cross;          // K of the A-term
    double n_off;            // storage offset density (0 for FP64)
    double sig2;             // sigma^2
    double beta;             // 2 sigma^2 sqrt(kT/pi)
    double wshell;           // uniform shell weight
    double chi_of_n;         // pi sigma^3 / 6
    double c_half;           // chi_of_n / (2 |ball|): half packing fraction per ball sum
    double h_off;            // half packing fraction of n_off: chi_of_n n_off / 2
    double ref_ng;           // n_ref g2(n_ref) (NBAR mode)
    double h_pred;           // kappa beta / 6: implicit factor of the field-velocity predictor per unit t
    // g, omega and K/(2 c_s^4) (0 without fields) split into pairs of floats
    // for the double-word collision (hi, lo)
    float g_dw[3][2];
    float omega_dw[2];
    float ka_dw[2];
    // the doubles above rounded to float once (set_float_params), for the
    // FP32 kernels: a per-thread conversion would run on the FP64 pipe
    float f_g[3], f_omega, f_tau, f_k_cross, f_n_off, f_sig2, f_beta, f_wshell, f_chi_of_n, f_c_half, f_h_off,
        f_ref_ng, f_h_pred;
};

// Fill the float copies of KParams' doubles (after any of them changes).
inline __host__ __device__ void set_float_params(KParams &p)
{
    for (int d = 0; d < 3; d++) p.f_g[d] = float(p.g[d]);
    p.f_omega = float(p.omega);
    p.f_tau = float(p.tau);
    p.f_k_cross = float(p.k_cross);
    p.f_n_off = float(p.n_off);
    p.f_sig2 = float(p.sig2);
    p.f_beta = float(p.beta);
    p.f_wshell = float(p.wshell);
    p.f_chi_of_n = float(p.chi_of_n);
    p.f_c_half = float(p.c_half);
    p.f_h_off = float(p.h_off);
    p.f_ref_ng = float(p.ref_ng);
    p.f_h_pred = float(p.h_pred);
}

// A parameter in the compute type T: the double itself, or its float copy
// (the same value a device conversion of the double gives).
template <class T>
__device__ __forceinline__ T prm(double d, float f);
template <>
__device__ __forceinline__ double prm<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float prm<float>(double, float f) { return f; }

// Tiled ball sum: an 8 x 8 x 8 brick of nodes per block with a halo of
// ball_r, the brick's n - n_off and the ball's offsets in shared memory.
constexpr int kBallTile = 8;

// Output brick depth of tile variant v of the tiled shell kernel.
inline __host__ __device__ int tile_depth(int v) { return v == 2 ? 4 : 8; }
constexpr size_t kBallTileMaxSmem = 48 * 1024;   // no opt-in attribute needed

inline __host__ __device__ size_t ball_tile_smem(int ball_r, int nball, size_t tsize)
{
    const size_t side = size_t(kBallTile + 2 * ball_r);
    return side * side * side * tsize + size_t(nball) * sizeof(int);
}

// Device buffers of one lattice.  S: storage type of populations; T: compute type.
template <class S, class T>
struct KBufs {
    const S *f_in;
    S *f_out;
    V4<T> *nu;           // (n - n_off, v_x, v_y, v_z) per node: density deviation and field velocity
    T *hb;               // half smeared packing fraction minus h_off, per node
    T *cprev;            // C of the previous step, 3 x Npad
    T *tprev;            // t = sum_e w g2 n(r+e) of the previous step
    T *nscale;           // storage scale of f_in minus n_off, per node
    const int4 *shell_e; // shell vectors
    const V4<T> *shell_k;// unit vectors e/|e| and, in w, the vector's weight (compact shell)
    const int4 *ball;    // ball vectors
    int *status;         // [0]: unstable flag
    double *out_nbar, *out_C, *out_A, *out_u;   // field outputs (fields kernel only)
};

// Checked build (compile with -DWDLB_CHECKED=1): every index the step
// kernels compute into a global or shared array is tested against the array's
// extent.  An index outside it sets bit 2 of the status word and the access is
// skipped, so a wrong index is reported instead of reading or writing another
// buffer.  In the normal build the test is the constant true.
#ifndef WDLB_CHECKED
#define WDLB_CHECKED 0
#endif
constexpr int kStatusUnstable = 1;   // status word bits
constexpr int kStatusBounds = 2;
constexpr int kStatusTimeout = 4;    // a bounded wait (TMA tile) gave up
constexpr int kDefaultWaitLimit = 1 << 20;   // mbarrier try_wait calls (each suspends briefly)

__device__ __forceinline__ bool in_bounds(long long i, long long n, int *status)
{
#if WDLB_CHECKED
    if (i >= 0 && i < n) return true;
    atomicOr(status, kStatusBounds);
    return false;
#else
    (void)i;
    (void)n;
    (void)status;
    return true;
#endif
}

// Asynchronous global -> shared copy of BYTES (4, 8 or 16) bytes, both
// addresses aligned to BYTES; cp_async_wait_all waits for all of the thread's
// copies (a __syncthreads must follow before other threads read them).
template <int BYTES>
__device__ __forceinline__ void cp_async_ca(void *smem, const void *gmem)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// TMA (cp.async.bulk.tensor) with an mbarrier in shared memory that counts
// the bytes the copies deliver.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One potentially blocking test of the barrier's phase: the hardware may
// suspend the thread until the phase completes or a short time limit passes.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Wait for the barrier's phase 0 with at most `limit` tries; true once it completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, int limit)
{
    for (int it = 0; it < limit; it++)
        if (mbar_try_wait(bar, 0)) return true;
    return false;
}
// Tiled loads of a 3-D / 4-D box of a tensor map into shared memory (the
// innermost coordinate first; coordinates outside the tensor read zero).
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const void *tmap, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Contact value of the homogeneous hard-sphere pair distribution at packing
// fraction chi (closure 0: Carnahan-Starling, 1: Percus-Yevick, 2: one).
template <int CL, class T>
__device__ __forceinline__ T contact_g(T chi)
{
    if (CL == 2) return T(1);
    T s = T(1) - chi;
    if (CL == 0) return (T(0.5) + T(0.5) * s) / (s * s * s);
    return (T(1.5) - T(0.5) * s) / (s * s);
}

inline double contact_g_host(int closure, double chi)
{
    if (closure == 2) return 1.0;
    double s = 1.0 - chi;
    if (closure == 0) return (0.5 + 0.5 * s) / (s * s * s);
    return (1.5 - 0.5 * s) / (s * s);
}

// Population storage relative to a rest state w_q s (s: a density per node).
// FP64 and FP32: f - w_q s.  FP16: (f - w_q s) / (w_q s).  load() takes the
// scale w_q s, put() its inverse.
template <class S>
struct Store;
template <>
struct Store<double> {
    typedef double T;
    __device__ __forceinline__ static double load(const double *p, double) { return *p; }
    __device__ __forceinline__ static void put(double *p, double v, double) { *p = v; }
};
template <>
struct Store<float> {
    typedef float T;
    __device__ __forceinline__ static float load(const float *p, float) { return *p; }
    __device__ __forceinline__ static void put(float *p, float v, float) { *p = v; }
};
template <>
struct Store<__half> {
    typedef float T;
    __device__ __forceinline__ static float load(const __half *p, float scale) { return __half2float(*p) * scale; }
    __device__ __forceinline__ static void put(__half *p, float v, float inv_scale) { *p = __float2half_rn(v * inv_scale); }
};

}  // namespace wdlb
