// wdlb_fields_static: the fields of a state (smeared density, C and A) for
// callers that cannot allocate device memory -- code running inside another
// framework's memory pool or a plugin host that forbids cudaMalloc, or that
// must not grow a process's device footprint after start-up.  It computes the
// same shell sums as the fields pass of the time step, from device arrays of
// n and u supplied by the caller, with its scratch (the FP32 field tile
// arrays, the stencil tables and a reduction slot) in one file-scope
// __device__ array of fixed size.  Every GPU that loads the library holds that
// array until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/wdlb.h"
#include "wdlb_kernels.cuh"
#include "wdlb_tables.h"

using namespace wdlb;

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kNuBytes = size_t(WDLB_STATIC_MAX_NODES) * sizeof(V4<float>);
constexpr size_t kHbBytes = size_t(WDLB_STATIC_MAX_NODES) * sizeof(float);
constexpr int kMaxShell = 1024, kMaxBall = 512;
constexpr size_t kOffHb = kNuBytes;
constexpr size_t kOffShellE = kOffHb + kHbBytes;
constexpr size_t kOffShellK = kOffShellE + kMaxShell * sizeof(int4);
constexpr size_t kOffBall = kOffShellK + kMaxShell * sizeof(V4<float>);
constexpr size_t kOffMisc = kOffBall + kMaxBall * sizeof(int4);   // [0] double reference density, [8] int status
constexpr size_t kScratchBytes = kOffMisc + 256;

// The scratch of every call on this device.  Host code must not take this
// name as a device address: the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

struct StaticBufs {
    V4<float> *nu;
    float *hb;
    const int4 *shell_e;
    const V4<float> *shell_k;
    const int4 *ball;
    double *ref;
    int *status;
};

StaticBufs carve(void *base)
{
    char *b = static_cast<char *>(base);
    StaticBufs s;
    s.nu = reinterpret_cast<V4<float> *>(b);
    s.hb = reinterpret_cast<float *>(b + kOffHb);
    s.shell_e = reinterpret_cast<const int4 *>(b + kOffShellE);
    s.shell_k = reinterpret_cast<const V4<float> *>(b + kOffShellK);
    s.ball = reinterpret_cast<const int4 *>(b + kOffBall);
    s.ref = reinterpret_cast<double *>(b + kOffMisc);
    s.status = reinterpret_cast<int *>(b + kOffMisc + 8);
    return s;
}

// p with the reference density computed on the device.
__device__ __forceinline__ KParams with_reference(KParams p, const double *ref)
{
    p.n_off = *ref;
    p.h_off = 0.5 * p.chi_of_n * p.n_off;
    set_float_params(p);
    return p;
}

// Mean density over fluid nodes (one block), the reference of the deviation form.
__global__ void __launch_bounds__(1024) k_static_reference(KParams p, const double *d_n, double *ref)
{
    __shared__ double sh[32];
    __shared__ double cnt[32];
    double a = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
        const int z = i / (p.nx * p.ny);
        if (p.walls && (z == 0 || z == p.nz - 1)) continue;
        a += d_n[i];
        c += 1.0;
    }
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        c += __shfl_down_sync(0xffffffffu, c, off);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5] = a;
        cnt[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, n = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            s += sh[w];
            n += cnt[w];
        }
        *ref = n > 0.0 ? s / n : 0.0;
    }
}

// Field arrays in deviation form from the caller's n and u (deviation formed in FP64).
__global__ void __launch_bounds__(256) k_static_prepare(KParams p0, StaticBufs s, const double *d_n,
                                                        const double *d_u)
{
    const KParams p = with_reference(p0, s.ref);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const int z = i / (p.nx * p.ny);
    if (p.walls && (z == 0 || z == p.nz - 1)) {
        s.nu[i] = V4<float>{-float(p.n_off), 0.f, 0.f, 0.f};
        return;
    }
    const double n = d_n[i], ux = d_u[i], uy = d_u[p.N + i], uz = d_u[2 * p.N + i];
    // a negative or non-finite density, or a non-finite velocity, is not a state
    if (!(n >= 0.0) || !isfinite(n) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz))
        atomicOr(s.status, kStatusUnstable);
    s.nu[i] = V4<float>{float(n - p.n_off), float(ux), float(uy), float(uz)};
}

__global__ void __launch_bounds__(256) k_static_ball(KParams p0, StaticBufs s)
{
    const KParams p = with_reference(p0, s.ref);
    ball_body<float>(p, s.nu, s.hb, s.ball, s.status, blockIdx.x);
}

template <int CL, bool WALLS>
__global__ void __launch_bounds__(256) k_static_fields(KParams p0, StaticBufs s, double *d_nbar, double *d_C,
                                                       double *d_A)
{
    const KParams p = with_reference(p0, s.ref);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const int N = p.N;
    const int x = i % p.nx, y = (i / p.nx) % p.ny, z = i / (p.nx * p.ny);
    if (WALLS && (z == 0 || z == p.nz - 1)) {
        if (d_nbar) d_nbar[i] = 0.0;
        for (int c = 0; c < 3; c++) d_C[c * N + i] = 0.0;
        for (int c = 0; c < 6; c++) d_A[c * N + i] = 0.0;
        return;
    }
    const float hr = float(p.h_off) + s.hb[i];
    const V4<float> me = s.nu[i];
    ShellAcc<float> a = {};
    shell_sums_generic<CL, WALLS, float>(p, s.nu, s.hb, s.shell_e, s.shell_k, x, y, z, hr, me.y, me.z, me.w, a,
                                         s.status);
    float C[3], A[6], t;
    shell_forces<float>(p, a, float(p.n_off) + me.x, me.y, me.z, me.w, C[0], C[1], C[2], A[0], A[1], A[2], A[3], A[4],
                        A[5], t);
    if (d_nbar) d_nbar[i] = double(hr) * 2.0 / p.chi_of_n;
    for (int c = 0; c < 3; c++) d_C[c * N + i] = C[c];
    for (int c = 0; c < 6; c++) d_A[c * N + i] = A[c];
}

template <int CL>
void launch_fields(bool walls, int blocks, cudaStream_t st, const KParams &p, const StaticBufs &s, double *nb,
                   double *C, double *A)
{
    if (walls)
        k_static_fields<CL, true><<<blocks, 256, 0, st>>>(p, s, nb, C, A);
    else
        k_static_fields<CL, false><<<blocks, 256, 0, st>>>(p, s, nb, C, A);
}

}  // namespace

extern "C" wdlb_status wdlb_fields_static(wdlb_lattice lat, double sigma, int32_t walls, int32_t closure,
                                          const double *d_n, const double *d_u, double *d_nbar, double *d_C,
                                          double *d_A, void *stream)
{
    if (!d_n || !d_u || !d_C || !d_A) return WDLB_ERR_ARG;
    if (lat.nx < 1 || lat.ny < 1 || lat.nz < 1) return WDLB_ERR_ARG;
    if (walls != WDLB_WALLS_NONE && walls != WDLB_WALLS_Z) return WDLB_ERR_ARG;
    if (walls == WDLB_WALLS_Z && lat.nz < 3) return WDLB_ERR_ARG;
    if (closure < 0 || closure > 2) return WDLB_ERR_ARG;
    if (!(sigma >= 1.0 && sigma <= 8.0)) return WDLB_ERR_ARG;
    const long long N = (long long)lat.nx * lat.ny * lat.nz;
    if (N > WDLB_STATIC_MAX_NODES) return WDLB_ERR_ARG;   // beyond the fixed scratch

    std::vector<int> ball, shell;
    double wshell = 0.0;
    build_ball(sigma, ball);
    build_shell(sigma, shell, &wshell);
    const int nball = (int)ball.size() / 3, nshell = (int)shell.size() / 3;
    if (nball > kMaxBall || nshell > kMaxShell) return WDLB_ERR_ARG;

    // device address of the static scratch, once per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return WDLB_ERR_CUDA;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return WDLB_ERR_CUDA;
            g_scratch_ptr[dev] = ptr;
        }
        base = g_scratch_ptr[dev];
    }
    const StaticBufs s = carve(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    std::vector<int4> se(nshell), be(nball);
    std::vector<V4<float>> sk(nshell);
    for (int m = 0; m < nshell; m++) {
        const int x = shell[3 * m], y = shell[3 * m + 1], z = shell[3 * m + 2];
        se[m] = make_int4(x, y, z, 0);
        const double len = std::sqrt(double(x * x + y * y + z * z));
        sk[m] = V4<float>{float(x / len), float(y / len), float(z / len), 0.f};
    }
    for (int m = 0; m < nball; m++) be[m] = make_int4(ball[3 * m], ball[3 * m + 1], ball[3 * m + 2], 0);
    char *b = static_cast<char *>(base);
    // pageable host sources: these copies have completed reading the vectors when they return
    if (cudaMemcpyAsync(b + kOffShellE, se.data(), nshell * sizeof(int4), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(b + kOffShellK, sk.data(), nshell * sizeof(V4<float>), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b + kOffBall, be.data(), nball * sizeof(int4), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(b + kOffMisc, 0, 256, st) != cudaSuccess)
        return WDLB_ERR_CUDA;

    KParams p;
    std::memset(&p, 0, sizeof(p));
    p.nx = lat.nx;
    p.ny = lat.ny;
    p.nz = lat.nz;
    p.walls = walls;
    p.N = (int)N;
    p.Npad = (int)N;
    p.nshell = nshell;
    p.nball = nball;
    p.closure = closure;
    p.interactions = 1;
    p.sig2 = sigma * sigma;
    p.beta = 2.0 * p.sig2 * std::sqrt(CS2 / M_PI);
    p.wshell = wshell;
    p.chi_of_n = M_PI * sigma * sigma * sigma / 6.0;
    p.c_half = p.chi_of_n / (2.0 * nball);
    set_float_params(p);

    const int blocks = (int)((N + 255) / 256);
    k_static_reference<<<1, 1024, 0, st>>>(p, d_n, s.ref);
    k_static_prepare<<<blocks, 256, 0, st>>>(p, s, d_n, d_u);
    k_static_ball<<<blocks, 256, 0, st>>>(p, s);
    if (closure == WDLB_CLOSURE_CS)
        launch_fields<0>(walls != 0, blocks, st, p, s, d_nbar, d_C, d_A);
    else if (closure == WDLB_CLOSURE_PY)
        launch_fields<1>(walls != 0, blocks, st, p, s, d_nbar, d_C, d_A);
    else
        launch_fields<2>(walls != 0, blocks, st, p, s, d_nbar, d_C, d_A);
    if (cudaGetLastError() != cudaSuccess) return WDLB_ERR_CUDA;
    // the status word the kernels set, read back after they finish: bit 1 a
    // non-physical state (smeared packing fraction >= 1, bad n or u), bit 2
    // (checked build only) an index outside its array, whose access was skipped
    int h = 0;
    if (cudaMemcpyAsync(&h, s.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return WDLB_ERR_CUDA;
    if (h & kStatusBounds) return WDLB_ERR_CUDA;
    if (h) return WDLB_ERR_UNSTABLE;
    return WDLB_OK;
}
