// Kernels of one WDLB time step (Sec. 5, Numerical results: the five-step
// algorithm), templated on population storage S, closure CL, relaxation mode
// OM and geometry (WALLS).  Compute type T = Store<S>::T.
//
//   k_moments        step 4 of Sec. 5 (Eq. colonna): n, j from f, and the
//                    field velocity v, a lagged linear-implicit predictor of
//                    the trapezoidal velocity u = j/n + g/2 + C/(2n):
//                      (1 + H) v = j/n + g/2 + C_prev/(2n) + H v_prev,
//                      H = kappa (beta/2) t_prev / 3,  t = sum_e w g2 n(r+e).
//   k_ball           smeared density of Sec. 3 over the lattice ball, stored
//                    as half packing fraction chi/2 per node.
//   k_shell_collide  steps 2 + 3 of Sec. 5: the shell sums of Eq. campoc
//                    (C = n (F^mf + F^viscous)) and Eq. campod (A) with
//                    du = v(r+e) - v(r), the collision of Eq. SMDB with the
//                    A-term of Eq. eq:dufty2 (second-order forcing), and push
//                    streaming with half-way bounce-back.
#pragma once

#include "wdlb_common.cuh"

namespace wdlb {

static __device__ __forceinline__ int wrap_coord(int v, int n)
{
    if (v >= 0 && v < n) return v;
    v %= n;
    return v < 0 ? v + n : v;
}

static __device__ __forceinline__ bool solid_plane(const KParams &p, int z)
{
    return p.walls && (z == 0 || z == p.nz - 1);
}

// ---------------------------------------------------------------------------
// Step 1 of Sec. 5: f = discrete local equilibrium of (n, u) from FP64
// staging; v_prev = u, C_prev = 0, t_prev = 0.
// ---------------------------------------------------------------------------
template <class S>
__global__ void __launch_bounds__(256) k_init(KParams p, KBufs<S, typename Store<S>::T> b, const double *st_n,
                                              const double *st_u)
{
    typedef typename Store<S>::T T;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int z = i / (p.nx * p.ny);
    bool solid = solid_plane(p, z);
    T n = solid ? T(0) : T(st_n[i]);
    T ux = solid || !st_u ? T(0) : T(st_u[i]);
    T uy = solid || !st_u ? T(0) : T(st_u[p.N + i]);
    T uz = solid || !st_u ? T(0) : T(st_u[2 * p.N + i]);
    T dn = n - T(p.n_off);
    T uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        T cu = T(cx_of(q)) * ux + T(cy_of(q)) * uy + T(cz_of(q)) * uz;
        T dev = T(w_of(q)) * (dn + n * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
        Store<S>::put(b.f_out + (size_t)q * p.Npad + i, dev, T(1.0 / w_of(q)) * T(p.inv_n_off));
    }
    b.nu[i] = V4<T>{n, ux, uy, uz};
    b.cprev[i] = T(0);
    b.cprev[p.Npad + i] = T(0);
    b.cprev[2 * p.Npad + i] = T(0);
    b.tprev[i] = T(0);
}

// ---------------------------------------------------------------------------
// Step 4 of Sec. 5 / Eq. colonna.  OUT = false: in-place update of nu (the
// time step); OUT = true: FP64 outputs only, state untouched.
// ---------------------------------------------------------------------------
template <class S, bool OUT>
__global__ void __launch_bounds__(256) k_moments(KParams p, KBufs<S, typename Store<S>::T> b, double *out_n,
                                                 double *out_u)
{
    typedef typename Store<S>::T T;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int z = i / (p.nx * p.ny);
    if (solid_plane(p, z)) {
        if (OUT) {
            if (out_n) out_n[i] = 0.0;
            if (out_u) out_u[i] = out_u[p.N + i] = out_u[2 * p.N + i] = 0.0;
        } else {
            b.nu[i] = V4<T>{T(0), T(0), T(0), T(0)};
        }
        return;
    }
    const T noff = T(p.n_off);
    T dn = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        T d = Store<S>::load(b.f_in + (size_t)q * p.Npad + i, T(w_of(q)) * noff);
        dn += d;
        if (cx_of(q)) jx += T(cx_of(q)) * d;
        if (cy_of(q)) jy += T(cy_of(q)) * d;
        if (cz_of(q)) jz += T(cz_of(q)) * d;
    }
    const T n = noff + dn;
    if (!(n > T(0)) || !isfinite(n)) atomicOr(b.status, 1);
    const T inv = T(1) / n;
    const V4<T> old = b.nu[i];
    const T H = T(p.h_pred) * b.tprev[i];
    const T den = T(1) / (T(1) + H);
    const T vx = ((jx + T(0.5) * (n * T(p.g[0]) + b.cprev[i])) * inv + H * old.y) * den;
    const T vy = ((jy + T(0.5) * (n * T(p.g[1]) + b.cprev[p.Npad + i])) * inv + H * old.z) * den;
    const T vz = ((jz + T(0.5) * (n * T(p.g[2]) + b.cprev[2 * p.Npad + i])) * inv + H * old.w) * den;
    if (OUT) {
        if (out_n) out_n[i] = double(n);
        if (out_u) {
            out_u[i] = double(vx);
            out_u[p.N + i] = double(vy);
            out_u[2 * p.N + i] = double(vz);
        }
    } else {
        b.nu[i] = V4<T>{n, vx, vy, vz};
    }
}

// ---------------------------------------------------------------------------
// Smeared density (Sec. 3) as half packing fraction: hb = (pi s^3/6) nbar / 2.
// Solid nodes get 0 (they carry n = 0 and never enter a pair with weight).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_ball(KParams p, const V4<T> *nu, T *hb, const int4 *ball, int *status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x = i % p.nx;
    int y = (i / p.nx) % p.ny;
    int z = i / (p.nx * p.ny);
    if (solid_plane(p, z)) {
        hb[i] = T(0);
        return;
    }
    T sum = T(0);
    for (int m = 0; m < p.nball; m++) {
        int4 e = ball[m];
        int zz = z + e.z;
        if (p.walls) {
            if (zz < 0 || zz >= p.nz) continue;
        } else {
            zz = wrap_coord(zz, p.nz);
        }
        int xx = wrap_coord(x + e.x, p.nx);
        int yy = wrap_coord(y + e.y, p.ny);
        sum += nu[xx + p.nx * (yy + p.ny * zz)].x;
    }
    T h = T(p.c_half) * sum;
    if (!(h < T(0.5))) atomicOr(status, 1);
    hb[i] = h;
}

// ---------------------------------------------------------------------------
// Fields + collision + streaming, one node per thread.
// ---------------------------------------------------------------------------
template <class S, int CL, int OM, bool WALLS, bool FIELDS>
__global__ void __launch_bounds__(256) k_shell_collide(KParams p, KBufs<S, typename Store<S>::T> b)
{
    typedef typename Store<S>::T T;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int x = i % nx;
    int y = (i / nx) % ny;
    int z = i / (nx * ny);
    if (WALLS && (z == 0 || z == nz - 1)) return;

    // own populations and moments
    const T noff = T(p.n_off), inoff = T(p.inv_n_off);
    T d[NQ];
    T dn = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        d[q] = Store<S>::load(b.f_in + (size_t)q * p.Npad + i, T(w_of(q)) * noff);
        dn += d[q];
        if (cx_of(q)) jx += T(cx_of(q)) * d[q];
        if (cy_of(q)) jy += T(cy_of(q)) * d[q];
        if (cz_of(q)) jz += T(cz_of(q)) * d[q];
    }
    const T n = noff + dn;
    const T inv_n = T(1) / n;
    const T gx = T(p.g[0]), gy = T(p.g[1]), gz = T(p.g[2]);
    const T hr = b.hb[i];
    const V4<T> me = b.nu[i];
    const T vx = me.y, vy = me.z, vz = me.w;

    T Cx = T(0), Cy = T(0), Cz = T(0);
    T Axx = T(0), Ayy = T(0), Azz = T(0), Axy = T(0), Axz = T(0), Ayz = T(0);
    T tsum = T(0);
    if (p.interactions) {
        T Vx = T(0), Vy = T(0), Vz = T(0);       // sum q khat           (F^mf)
        T Wx = T(0), Wy = T(0), Wz = T(0);       // sum q khat (khat.dv) (F^visc)
        T Sxx = T(0), Syy = T(0), Szz = T(0), Sxy = T(0), Sxz = T(0), Syz = T(0);
        for (int m = 0; m < p.nshell; m++) {
            const int4 e = b.shell_e[m];
            const V4<T> k = b.shell_k[m];
            int zz = z + e.z;
            if (WALLS) {
                if (zz <= 0 || zz >= nz - 1) continue;   // solid or beyond: n = 0
            } else {
                zz = wrap_coord(zz, nz);
            }
            const int xx = wrap_coord(x + e.x, nx);
            const int yy = wrap_coord(y + e.y, ny);
            const int j = xx + nx * (yy + ny * zz);
            const V4<T> ne = b.nu[j];
            const T q = contact_g<CL, T>(hr + b.hb[j]) * ne.x;
            const T dvx = ne.y - vx, dvy = ne.z - vy, dvz = ne.w - vz;
            const T qkd = q * (k.x * dvx + k.y * dvy + k.z * dvz);
            Vx += q * k.x; Vy += q * k.y; Vz += q * k.z;
            Wx += qkd * k.x; Wy += qkd * k.y; Wz += qkd * k.z;
            const T qx = q * dvx, qy = q * dvy, qz = q * dvz;
            Sxx += k.x * qx; Syy += k.y * qy; Szz += k.z * qz;
            Sxy += k.y * qx + k.x * qy;
            Sxz += k.z * qx + k.x * qz;
            Syz += k.z * qy + k.y * qz;
            tsum += q;
        }
        const T w = T(p.wshell);
        const T mf = -T(CS2) * T(p.sig2) * w * n;
        const T vi = T(p.beta) * w * n;
        Cx = mf * Vx + vi * Wx;
        Cy = mf * Vy + vi * Wy;
        Cz = mf * Vz + vi * Wz;
        const T pa = -(T(CS2) / T(5)) * T(p.sig2) * n * w;
        Axx = T(2) * pa * Sxx; Ayy = T(2) * pa * Syy; Azz = T(2) * pa * Szz;
        Axy = pa * Sxy; Axz = pa * Sxz; Ayz = pa * Syz;
        tsum *= w;
    }

    // collision velocity u = (j + F/2)/n with F = n g + C
    const T Fx = n * gx + Cx, Fy = n * gy + Cy, Fz = n * gz + Cz;
    const T ux = (jx + T(0.5) * Fx) * inv_n;
    const T uy = (jy + T(0.5) * Fy) * inv_n;
    const T uz = (jz + T(0.5) * Fz) * inv_n;

    if (FIELDS) {
        const int N = p.N;
        b.out_nbar[i] = double(hr) * 2.0 / p.chi_of_n;
        b.out_C[i] = Cx; b.out_C[N + i] = Cy; b.out_C[2 * N + i] = Cz;
        b.out_A[i] = Axx; b.out_A[N + i] = Ayy; b.out_A[2 * N + i] = Azz;
        b.out_A[3 * N + i] = Axy; b.out_A[4 * N + i] = Axz; b.out_A[5 * N + i] = Ayz;
        b.out_u[i] = ux; b.out_u[N + i] = uy; b.out_u[2 * N + i] = uz;
        return;
    }

    // relaxation frequency
    T omega = T(p.omega);
    if (OM == 1) {
        const T chib = T(2) * hr;
        const T loc = chib / T(p.chi_of_n) * contact_g<CL, T>(chib);
        T tau = loc > T(0) ? T(0.5) + (T(p.tau) - T(0.5)) * T(p.ref_ng) / loc : T(1e30);
        tau = tau < T(0.501) ? T(0.501) : tau;
        omega = T(1) / tau;
    }

    // collision (Eq. SMDB, second order): f* = f - omega (f - feq) + (1 - omega/2)(Phi + S^A)
    const T tr3 = (Axx + Ayy + Azz) * T(1.0 / 3.0);
    const T Bxx = Axx - tr3, Byy = Ayy - tr3, Bzz = Azz - tr3;   // traceless A
    const T kA = p.interactions ? T(p.k_cross) * T(4.5) : T(0);  // K / (2 c_s^4)
    const T uu = ux * ux + uy * uy + uz * uz;
    const T uF = ux * Fx + uy * Fy + uz * Fz;
    const T src_pref = T(1) - T(0.5) * omega;

#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const int cxq = cx_of(q), cyq = cy_of(q), czq = cz_of(q);
        const T wq = T(w_of(q));
        const T cu = T(cxq) * ux + T(cyq) * uy + T(czq) * uz;
        const T cF = T(cxq) * Fx + T(cyq) * Fy + T(czq) * Fz;
        const T feq_dev = wq * (dn + n * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
        const T phi = wq * (T(3) * (cF - uF) + T(9) * cu * cF);
        const T cAc = T(cxq * cxq) * Bxx + T(cyq * cyq) * Byy + T(czq * czq) * Bzz +
                      T(2 * cxq * cyq) * Axy + T(2 * cxq * czq) * Axz + T(2 * cyq * czq) * Ayz;
        const T sa = kA * wq * cAc;
        const T post = d[q] - omega * (d[q] - feq_dev) + src_pref * (phi + sa);
        // push streaming with half-way bounce-back
        int zt = z + czq;
        int dst;
        int qq = q;
        if (WALLS && (zt == 0 || zt == nz - 1)) {
            dst = i;
            qq = opp_of(q);
        } else {
            if (!WALLS) zt = wrap_coord(zt, nz);
            const int xt = wrap_coord(x + cxq, nx);
            const int yt = wrap_coord(y + cyq, ny);
            dst = xt + nx * (yt + ny * zt);
        }
        Store<S>::put(b.f_out + (size_t)qq * p.Npad + dst, post, T(1.0 / w_of(q)) * inoff);
    }
    b.cprev[i] = Cx;
    b.cprev[p.Npad + i] = Cy;
    b.cprev[2 * p.Npad + i] = Cz;
    b.tprev[i] = tsum;
}

// ---------------------------------------------------------------------------
// Outputs and FP64 reductions.
// ---------------------------------------------------------------------------
template <class S>
__global__ void __launch_bounds__(256) k_pop_to_f64(KParams p, const S *f, int q, double *out)
{
    typedef typename Store<S>::T T;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int z = i / (p.nx * p.ny);
    if (solid_plane(p, z)) {
        out[i] = 0.0;
        return;
    }
    T dv = Store<S>::load(f + (size_t)q * p.Npad + i, T(w_of(q)) * T(p.n_off));
    out[i] = double(dv) + w_of(q) * p.n_off;
}

// Per-block FP64 partial sums over fluid nodes of the FP64 moments n, u_x:
// [0] sum n, [1] sum u_x, [2] sum n u_x, [3] max |u_x - snap|, [4] max |u_x|, [5] count.
// If update_snap, the snapshot is overwritten with the current u_x.
static __global__ void __launch_bounds__(256) k_stats(KParams p, const double *n_, const double *ux_, double *snap,
                                                      int update_snap, double *partial)
{
    __shared__ double sh[6][8];
    double a0 = 0, a1 = 0, a2 = 0, m3 = 0, m4 = 0, c5 = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.N; i += gridDim.x * blockDim.x) {
        int z = i / (p.nx * p.ny);
        if (p.walls && (z == 0 || z == p.nz - 1)) continue;
        double n = n_[i], ux = ux_[i];
        a0 += n;
        a1 += ux;
        a2 += n * ux;
        double dd = fabs(ux - snap[i]);
        m3 = dd > m3 ? dd : m3;
        m4 = fabs(ux) > m4 ? fabs(ux) : m4;
        c5 += 1.0;
        if (update_snap) snap[i] = ux;
    }
    for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, off);
        a1 += __shfl_down_sync(0xffffffffu, a1, off);
        a2 += __shfl_down_sync(0xffffffffu, a2, off);
        m3 = fmax(m3, __shfl_down_sync(0xffffffffu, m3, off));
        m4 = fmax(m4, __shfl_down_sync(0xffffffffu, m4, off));
        c5 += __shfl_down_sync(0xffffffffu, c5, off);
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = a0; sh[1][wid] = a1; sh[2][wid] = a2;
        sh[3][wid] = m3; sh[4][wid] = m4; sh[5][wid] = c5;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[6] = {0, 0, 0, 0, 0, 0};
        int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; w++) {
            r[0] += sh[0][w]; r[1] += sh[1][w]; r[2] += sh[2][w];
            r[3] = fmax(r[3], sh[3][w]); r[4] = fmax(r[4], sh[4][w]); r[5] += sh[5][w];
        }
        for (int k = 0; k < 6; k++) partial[blockIdx.x * 6 + k] = r[k];
    }
}

static __global__ void k_stats_final(const double *partial, int nblocks, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double r[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; b++) {
        r[0] += partial[b * 6 + 0]; r[1] += partial[b * 6 + 1]; r[2] += partial[b * 6 + 2];
        r[3] = fmax(r[3], partial[b * 6 + 3]); r[4] = fmax(r[4], partial[b * 6 + 4]);
        r[5] += partial[b * 6 + 5];
    }
    for (int k = 0; k < 6; k++) out[k] = r[k];
}

// FP64 sum of the initial density over fluid nodes (for the default n_ref).
static __global__ void k_sum_density(KParams p, const double *st_n, double *partial)
{
    __shared__ double sh[8];
    double a = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.N; i += gridDim.x * blockDim.x) {
        int z = i / (p.nx * p.ny);
        if (p.walls && (z == 0 || z == p.nz - 1)) continue;
        a += st_n[i];
    }
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh[w];
        partial[blockIdx.x] = r;
    }
}

static __global__ void k_sum_final(const double *partial, int nblocks, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double r = 0;
    for (int b = 0; b < nblocks; b++) r += partial[b];
    out[0] = r;
}

}  // namespace wdlb
