// Tiled shell kernel: the same step as k_shell_collide (steps 2 + 3 of
// Sec. 5), for FP32 arithmetic, with the field tile and its shell halo staged
// in shared memory and the contact shell unrolled at compile time.
//
// Block: 256 threads, an 8 x 8 x 8 brick of output nodes (two per thread, z
// and z + 4).  Shared memory holds (8 + 2R)^3 nodes of (n, v_x, v_y, v_z) and
// the half packing fraction hb, R = floor(sigma + 1/2), with periodic wrap in
// x, y (and z without walls) and n = 0 beyond the walls, so that the shell
// loop needs no bounds checks: a solid or missing neighbour has n = 0 and adds
// nothing.  Each shell vector is a compile-time constant, so the shared-memory
// offsets are immediates and khat enters as literal operands.  The shell is
// walked in (+e, -e) pairs (pair_weights, accumulate_pair): khat flips sign
// between the two, so the F^mf, F^viscous and A sums (Eq. campoc, Eq. campod)
// take the sum or the difference of the pair's terms, and the mean-field sum
// is formed from density deviations.
#pragma once

#include <utility>

#include "wdlb_kernels.cuh"

namespace wdlb {
namespace tiled {

constexpr int TX = 8, TY = 8, TZ = 8, THREADS = 256;

struct IV3 {
    int x, y, z;
};

// Shell of diameter sigma = S2 / 2: (S2 - 1)^2 < 4 |e|^2 <= (S2 + 1)^2, walked
// as (+e, -e) with +e lexicographically positive (x, then y, then z).
constexpr bool in_shell(int S2, int x, int y, int z)
{
    return (S2 - 1) * (S2 - 1) < 4 * (x * x + y * y + z * z) && 4 * (x * x + y * y + z * z) <= (S2 + 1) * (S2 + 1);
}

constexpr int shell_radius(int S2) { return (S2 + 1) / 2; }

constexpr int shell_count(int S2)
{
    int R = shell_radius(S2), m = 0;
    for (int x = -R; x <= R; x++)
        for (int y = -R; y <= R; y++)
            for (int z = -R; z <= R; z++)
                if (in_shell(S2, x, y, z)) m++;
    return m;
}

// M-th positive vector (+e of the M-th pair).
constexpr IV3 shell_pair(int S2, int M)
{
    int R = shell_radius(S2), m = 0;
    for (int x = 0; x <= R; x++)
        for (int y = -R; y <= R; y++)
            for (int z = -R; z <= R; z++) {
                bool positive = x > 0 || (x == 0 && (y > 0 || (y == 0 && z > 0)));
                if (positive && in_shell(S2, x, y, z)) {
                    if (m == M) return IV3{x, y, z};
                    m++;
                }
            }
    return IV3{0, 0, 0};
}

constexpr double csqrt(double v)
{
    double r = v > 1 ? v : 1.0;
    for (int k = 0; k < 60; k++) r = 0.5 * (r + v / r);
    return r;
}

template <int S2, int CL, int SX, int SY, int M>
__device__ __forceinline__ void pair_term(ShellAcc<float> &a, const float4 *__restrict__ sm4,
                                          const float *__restrict__ smh, int base, float s0, float noff, float vx,
                                          float vy, float vz)
{
    constexpr IV3 e = shell_pair(S2, M);
    constexpr int off = e.x + SX * (e.y + SY * e.z);
    constexpr double len = csqrt(double(e.x * e.x + e.y * e.y + e.z * e.z));
    constexpr float kx = float(e.x / len), ky = float(e.y / len), kz = float(e.z / len);

    const float4 np = sm4[base + off];
    const float hp = smh[base + off];
    const float4 nm = sm4[base - off];
    const float hm = smh[base - off];
    float qp, qm, qd;
    pair_weights<CL, float>(s0, noff, hp, np.x, hm, nm.x, qp, qm, qd);
    // q dv for both ends; khat(-e) = -khat(+e): W takes the sum, S the difference
    const float px = qp * (np.y - vx), py = qp * (np.z - vy), pz = qp * (np.w - vz);
    const float mx = qm * (nm.y - vx), my = qm * (nm.z - vy), mz = qm * (nm.w - vz);
    const float sx = px + mx, sy = py + my, sz = pz + mz;
    const float dx = px - mx, dy = py - my, dz = pz - mz;
    a.t += qp + qm;
    float ks = 0.f;
    if constexpr (e.x != 0) { a.Vx += kx * qd; ks += kx * sx; }
    if constexpr (e.y != 0) { a.Vy += ky * qd; ks += ky * sy; }
    if constexpr (e.z != 0) { a.Vz += kz * qd; ks += kz * sz; }
    if constexpr (e.x != 0) { a.Wx += kx * ks; a.Sxx += kx * dx; }
    if constexpr (e.y != 0) { a.Wy += ky * ks; a.Syy += ky * dy; }
    if constexpr (e.z != 0) { a.Wz += kz * ks; a.Szz += kz * dz; }
    if constexpr (e.y != 0) a.Sxy += ky * dx;
    if constexpr (e.x != 0) a.Sxy += kx * dy;
    if constexpr (e.z != 0) a.Sxz += kz * dx;
    if constexpr (e.x != 0) a.Sxz += kx * dz;
    if constexpr (e.z != 0) a.Syz += kz * dy;
    if constexpr (e.y != 0) a.Syz += ky * dz;
}

template <int S2, int CL, int SX, int SY, int... M>
__device__ __forceinline__ void shell_sum(ShellAcc<float> &a, const float4 *sm4, const float *smh, int base, float s0,
                                          float noff, float vx, float vy, float vz, std::integer_sequence<int, M...>)
{
    (pair_term<S2, CL, SX, SY, M>(a, sm4, smh, base, s0, noff, vx, vy, vz), ...);
}

template <int S2>
constexpr size_t smem_bytes()
{
    constexpr int R = shell_radius(S2);
    constexpr size_t n = size_t(TX + 2 * R) * (TY + 2 * R) * (TZ + 2 * R);
    return n * (sizeof(float4) + sizeof(float));
}

template <class S, int S2, int CL, bool WALLS, bool FIELDS>
__global__ void __launch_bounds__(THREADS) k_shell_tiled(KParams p, KBufs<S, float> b)
{
    constexpr int R = shell_radius(S2);
    constexpr int SX = TX + 2 * R, SY = TY + 2 * R, SZ = TZ + 2 * R;
    constexpr int NS = SX * SY * SZ;
    constexpr int NPAIR = shell_count(S2) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *sm4 = reinterpret_cast<float4 *>(smem_raw);
    float *smh = reinterpret_cast<float *>(smem_raw + sizeof(float4) * NS);

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;

    // stage the field tile with its halo
    for (int idx = threadIdx.x; idx < NS; idx += THREADS) {
        const int sx = idx % SX, sy = (idx / SX) % SY, sz = idx / (SX * SY);
        int gx = x0 - R + sx, gy = y0 - R + sy, gz = z0 - R + sz;
        gx = ((gx % nx) + nx) % nx;
        gy = ((gy % ny) + ny) % ny;
        bool inside = true;
        if (WALLS)
            inside = gz >= 0 && gz < nz;
        else
            gz = ((gz % nz) + nz) % nz;
        float4 v = make_float4(-float(p.n_off), 0.f, 0.f, 0.f);   // beyond a wall: n = 0
        float h = -float(p.h_off);
        if (inside) {
            const int g = gx + nx * (gy + ny * gz);
            const V4<float> t = b.nu[g];
            v = make_float4(t.x, t.y, t.z, t.w);
            h = b.hb[g];
        }
        sm4[idx] = v;
        smh[idx] = h;
    }
    __syncthreads();

    const int tx = threadIdx.x & 7, ty = (threadIdx.x >> 3) & 7, tzb = threadIdx.x >> 6;
#pragma unroll 1
    for (int half = 0; half < 2; half++) {
        const int tz = tzb + 4 * half;
        const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
        if (x >= nx || y >= ny || z >= nz) continue;
        if (WALLS && (z == 0 || z == nz - 1)) continue;
        const int i = x + nx * (y + ny * z);
        const int base = (tx + R) + SX * ((ty + R) + SY * (tz + R));
        const float4 me = sm4[base];
        const float noff = float(p.n_off);
        const float hr = float(p.h_off) + smh[base];

        float Cx = 0.f, Cy = 0.f, Cz = 0.f;
        float Axx = 0.f, Ayy = 0.f, Azz = 0.f, Axy = 0.f, Axz = 0.f, Ayz = 0.f, tsum = 0.f;
        if (p.interactions) {
            ShellAcc<float> a = {};
            shell_sum<S2, CL, SX, SY>(a, sm4, smh, base, 1.f - hr - float(p.h_off), noff, me.y, me.z, me.w,
                                      std::make_integer_sequence<int, NPAIR>{});
            const float w = float(p.wshell);
            const float n = noff + me.x;
            const float mf = -float(CS2) * float(p.sig2) * w * n;
            const float vi = float(p.beta) * w * n;
            Cx = mf * a.Vx + vi * a.Wx;
            Cy = mf * a.Vy + vi * a.Wy;
            Cz = mf * a.Vz + vi * a.Wz;
            const float pa = -(float(CS2) / 5.f) * float(p.sig2) * n * w;
            Axx = 2.f * pa * a.Sxx; Ayy = 2.f * pa * a.Syy; Azz = 2.f * pa * a.Szz;
            Axy = pa * a.Sxy; Axz = pa * a.Sxz; Ayz = pa * a.Syz;
            tsum = a.t * w;
        }
        collide_push<S, CL, WALLS, FIELDS>(
            p, b, i, x, y, z, hr, Cx, Cy, Cz, Axx, Ayy, Azz, Axy, Axz, Ayz, tsum, me.x,
            [&](int q, int) { return sm4[base + cx_of(q) + SX * (cy_of(q) + SY * cz_of(q))].x; });
    }
}

}  // namespace tiled
}  // namespace wdlb
