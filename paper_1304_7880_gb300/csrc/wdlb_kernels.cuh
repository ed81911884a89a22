// Per-block bodies of one WDLB time step (Sec. 5, Numerical results: the
// five-step algorithm), templated on population storage S, closure CL and
// geometry (WALLS); the relaxation mode is a runtime branch.  Compute type
// T = Store<S>::T.  The step kernels that run them (one launch per phase for
// every lattice of a table) are in wdlb_launch.cu.
//
//   moments_body     step 4 of Sec. 5 (Eq. colonna): n, j from f, and the
//                    field velocity v, a lagged linear-implicit predictor of
//                    the trapezoidal velocity u = j/n + g/2 + C/(2n):
//                      (1 + H) v = j/n + g/2 + C_prev/(2n) + H v_prev,
//                      H = kappa (beta/2) t_prev / 3,  t = sum_e w g2 n(r+e).
//   ball_body,       smeared density of Sec. 3 over the lattice ball, stored
//   ball_tiled_body  as half packing fraction chi/2 per node (per node, or
//                    per 8^3 brick through shared memory; same sums).
//   shell_body       steps 2 + 3 of Sec. 5: the shell sums of Eq. campoc
//                    (C = n (F^mf + F^viscous)) and Eq. campod (A) with
//                    du = v(r+e) - v(r), the collision of Eq. SMDB with the
//                    A-term of Eq. eq:dufty2 (second-order forcing), and push
//                    streaming with half-way bounce-back (the tiled form for
//                    sigma 3, 4, 6 is in wdlb_shell_tiled.cuh).
//
// Deviation form: nu holds n - n_off and hb holds chi/2 - h_off (h_off the
// value of n_off), so that the mean-field sum, which cancels down to a
// density gradient, is formed from differences of deviations (see
// pair_weights) and keeps FP32 accuracy relative to the gradient itself.
//
// Population storage is relative to a local rest state: the value stored for
// f_q(r) is f_q - w_q s(r) (FP64, FP32) or (f_q - w_q s(r)) / (w_q s(r))
// (FP16), with s(r) = n_off + nscale[r] the density of node r one step
// earlier.  The pushes of a step encode with the target's current density,
// which becomes the target's scale for the next step; the stored values stay
// small near walls, where n departs far from n_off.
#pragma once

#include "wdlb_common.cuh"
#include "wdlb_dw.cuh"

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
    // deviations from n_off are formed in FP64 before rounding to T
    const T dnv = solid ? -prm<T>(p.n_off, p.f_n_off) : T(st_n[i] - p.n_off);
    T n = solid ? T(0) : prm<T>(p.n_off, p.f_n_off) + dnv;
    T ux = solid || !st_u ? T(0) : T(st_u[i]);
    T uy = solid || !st_u ? T(0) : T(st_u[p.N + i]);
    T uz = solid || !st_u ? T(0) : T(st_u[2 * p.N + i]);
    // local rest state s(r) = n (solid nodes: n_off, their slots are never read)
    const T dsc = solid ? T(0) : dnv;
    const T sc = prm<T>(p.n_off, p.f_n_off) + dsc;
    const T uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        T cu = T(cx_of(q)) * ux + T(cy_of(q)) * uy + T(cz_of(q)) * uz;
        T dev = solid ? T(0) : T(w_of(q)) * n * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
        Store<S>::put(b.f_out + (size_t)q * p.Npad + i, dev, T(1.0 / w_of(q)) / sc);
    }
    b.nu[i] = V4<T>{dnv, ux, uy, uz};
    b.nscale[i] = dsc;
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
__device__ __forceinline__ void moments_body(const KParams &p, const KBufs<S, typename Store<S>::T> &b, int blk,
                                             double *out_n, double *out_u)
{
    typedef typename Store<S>::T T;
    int i = blk * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int z = i / (p.nx * p.ny);
    if (solid_plane(p, z)) {
        if (OUT) {
            if (out_n) out_n[i] = 0.0;
            if (out_u) out_u[i] = out_u[p.N + i] = out_u[2 * p.N + i] = 0.0;
        } else {
            b.nu[i] = V4<T>{-prm<T>(p.n_off, p.f_n_off), T(0), T(0), T(0)};
        }
        return;
    }
    const T noff = prm<T>(p.n_off, p.f_n_off);
    const T dsc = b.nscale[i];
    const T sc = noff + dsc;
    T dl = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        T d = Store<S>::load(b.f_in + (size_t)q * p.Npad + i, T(w_of(q)) * sc);
        dl += d;
        if (cx_of(q)) jx += T(cx_of(q)) * d;
        if (cy_of(q)) jy += T(cy_of(q)) * d;
        if (cz_of(q)) jz += T(cz_of(q)) * d;
    }
    const T dn = dsc + dl;          // n - n_off
    const T n = noff + dn;
    if (!(n > T(0)) || !isfinite(n)) atomicOr(b.status, 1);
    const T inv = T(1) / n;
    const V4<T> old = b.nu[i];
    const T H = prm<T>(p.h_pred, p.f_h_pred) * b.tprev[i];
    const T den = T(1) / (T(1) + H);
    // every multiply-add written out, so each kernel that runs this body
    // (the per-phase step and the persistent one) computes the same bits
    const T vx = fma(H, old.y, fma(T(0.5), fma(n, prm<T>(p.g[0], p.f_g[0]), b.cprev[i]), jx) * inv) * den;
    const T vy = fma(H, old.z, fma(T(0.5), fma(n, prm<T>(p.g[1], p.f_g[1]), b.cprev[p.Npad + i]), jy) * inv) * den;
    const T vz = fma(H, old.w, fma(T(0.5), fma(n, prm<T>(p.g[2], p.f_g[2]), b.cprev[2 * p.Npad + i]), jz) * inv) * den;
    if (OUT) {
        if (out_n) out_n[i] = double(n);
        if (out_u) {
            out_u[i] = double(vx);
            out_u[p.N + i] = double(vy);
            out_u[2 * p.N + i] = double(vz);
        }
    } else {
        b.nu[i] = V4<T>{dn, vx, vy, vz};
    }
}

template <class S, bool OUT>
__global__ void __launch_bounds__(256) k_moments(KParams p, KBufs<S, typename Store<S>::T> b, double *out_n,
                                                 double *out_u)
{
    moments_body<S, OUT>(p, b, blockIdx.x, out_n, out_u);
}

// ---------------------------------------------------------------------------
// Smeared density (Sec. 3) as half packing fraction: hb = (pi s^3/6) nbar / 2.
// Solid nodes get 0 (they carry n = 0 and never enter a pair with weight).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void ball_body(const KParams &p, const V4<T> *nu, T *hb, const int4 *ball, int *status,
                                          int blk)
{
    int i = blk * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x = i % p.nx;
    int y = (i / p.nx) % p.ny;
    int z = i / (p.nx * p.ny);
    if (solid_plane(p, z)) {
        hb[i] = -prm<T>(p.h_off, p.f_h_off);    // n = 0: chi = 0
        return;
    }
    const T noff = prm<T>(p.n_off, p.f_n_off);
    T sum = T(0);               // sum over the ball of n - n_off
    for (int m = 0; m < p.nball; m++) {
        int4 e = ball[m];
        int zz = z + e.z;
        if (p.walls) {
            if (zz < 0 || zz >= p.nz) {
                sum -= noff;    // beyond a wall: n = 0
                continue;
            }
        } else {
            zz = wrap_coord(zz, p.nz);
        }
        int xx = wrap_coord(x + e.x, p.nx);
        int yy = wrap_coord(y + e.y, p.ny);
        const int j = xx + p.nx * (yy + p.ny * zz);
        if (in_bounds(j, p.N, status)) sum += nu[j].x;
    }
    T dh = prm<T>(p.c_half, p.f_c_half) * sum;
    if (!(prm<T>(p.h_off, p.f_h_off) + dh < T(0.5))) atomicOr(status, 1);
    hb[i] = dh;
}

// Tiled form of ball_body: one 8 x 8 x 8 brick of nodes per block of 256
// threads (two nodes per thread, z and z + 4), with n - n_off of the brick
// and its halo of ball_r, and the ball's offsets within it, in shared memory.
// Beyond a wall the staged value is -n_off (n = 0).  The brick arrives by
// cp.async (all of a thread's loads in flight at once).  The ball points are
// added in table order, so every sum is bitwise the one of ball_body.
template <class T>
__device__ __forceinline__ void ball_tiled_body(const KParams &p, const V4<T> *nu, T *hb, const int4 *ball,
                                                int *status, int bx, int by, int bz)
{
    extern __shared__ __align__(16) unsigned char ball_smem[];
    const int R = p.ball_r, SX = kBallTile + 2 * R, NS = SX * SX * SX;
    T *sn = reinterpret_cast<T *>(ball_smem);
    int *so = reinterpret_cast<int *>(ball_smem + size_t(NS) * sizeof(T));
    for (int m = threadIdx.x; m < p.nball; m += blockDim.x) {
        const int4 e = ball[m];
        so[m] = e.x + SX * (e.y + SX * e.z);
    }
    const T noff = prm<T>(p.n_off, p.f_n_off);
    const int x0 = bx * kBallTile, y0 = by * kBallTile, z0 = bz * kBallTile;
    for (int idx = threadIdx.x; idx < NS; idx += blockDim.x) {
        const int sx = idx % SX, sy = (idx / SX) % SX, sz = idx / (SX * SX);
        const int gx = wrap_coord(x0 - R + sx, p.nx), gy = wrap_coord(y0 - R + sy, p.ny);
        int gz = z0 - R + sz;
        bool inside = true;
        if (p.walls)
            inside = gz >= 0 && gz < p.nz;
        else
            gz = wrap_coord(gz, p.nz);
        const int g = gx + p.nx * (gy + p.ny * gz);
        if (inside && in_bounds(g, p.N, status))
            cp_async_ca<sizeof(T)>(sn + idx, &nu[g].x);
        else
            sn[idx] = -noff;
    }
    cp_async_wait_all();
    __syncthreads();
    const int tx = threadIdx.x & 7, ty = (threadIdx.x >> 3) & 7, tzb = threadIdx.x >> 6;
    for (int half = 0; half < 2; half++) {
        const int tz = tzb + 4 * half;
        const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
        if (x >= p.nx || y >= p.ny || z >= p.nz) continue;
        const int i = x + p.nx * (y + p.ny * z);
        if (solid_plane(p, z)) {
            hb[i] = -prm<T>(p.h_off, p.f_h_off);
            continue;
        }
        const int base = (tx + R) + SX * ((ty + R) + SX * (tz + R));
        T sum = T(0);
        for (int m = 0; m < p.nball; m++)
            if (in_bounds(base + so[m], NS, status)) sum += sn[base + so[m]];
        T dh = prm<T>(p.c_half, p.f_c_half) * sum;
        if (!(prm<T>(p.h_off, p.f_h_off) + dh < T(0.5))) atomicOr(status, 1);
        hb[i] = dh;
    }
}

// ball_tiled_body with 2 sigma = S2 known at compile time (sigma 3, 4, 6, 8): the
// brick side and the ball's offsets are constants, and the points are added
// in the order of the host's ball table (dx, then dy, then dz ascending), so
// the sums are bitwise those of ball_body and ball_tiled_body.
template <class T, int S2>
__device__ __forceinline__ void ball_brick_ct(const KParams &p, const V4<T> *nu, T *hb, int *status, int bx,
                                              int by, int bz)
{
    constexpr int R = S2 / 4;                       // floor(sigma / 2)
    constexpr int SX = kBallTile + 2 * R, NS = SX * SX * SX;
    extern __shared__ __align__(16) unsigned char ball_smem[];
    T *sn = reinterpret_cast<T *>(ball_smem);
    const T noff = prm<T>(p.n_off, p.f_n_off);
    const int x0 = bx * kBallTile, y0 = by * kBallTile, z0 = bz * kBallTile;
    for (int idx = threadIdx.x; idx < NS; idx += blockDim.x) {
        const int sx = idx % SX, sy = (idx / SX) % SX, sz = idx / (SX * SX);
        const int gx = wrap_coord(x0 - R + sx, p.nx), gy = wrap_coord(y0 - R + sy, p.ny);
        int gz = z0 - R + sz;
        bool inside = true;
        if (p.walls)
            inside = gz >= 0 && gz < p.nz;
        else
            gz = wrap_coord(gz, p.nz);
        const int g = gx + p.nx * (gy + p.ny * gz);
        if (inside && in_bounds(g, p.N, status))
            cp_async_ca<sizeof(T)>(sn + idx, &nu[g].x);
        else
            sn[idx] = -noff;
    }
    cp_async_wait_all();
    __syncthreads();
    const int tx = threadIdx.x & 7, ty = (threadIdx.x >> 3) & 7, tzb = threadIdx.x >> 6;
    for (int half = 0; half < 2; half++) {
        const int tz = tzb + 4 * half;
        const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
        if (x >= p.nx || y >= p.ny || z >= p.nz) continue;
        const int i = x + p.nx * (y + p.ny * z);
        if (solid_plane(p, z)) {
            hb[i] = -prm<T>(p.h_off, p.f_h_off);
            continue;
        }
        const T *c = sn + (tx + R) + SX * ((ty + R) + SX * (tz + R));
        T sum = T(0);
#pragma unroll
        for (int dx = -R; dx <= R; dx++)
#pragma unroll
            for (int dy = -R; dy <= R; dy++)
#pragma unroll
                for (int dz = -R; dz <= R; dz++)
                    if (16 * (dx * dx + dy * dy + dz * dz) <= S2 * S2 &&
                        in_bounds(c - sn + dx + SX * (dy + SX * dz), NS, status))
                        sum += c[dx + SX * (dy + SX * dz)];
        T dh = prm<T>(p.c_half, p.f_c_half) * sum;
        if (!(prm<T>(p.h_off, p.f_h_off) + dh < T(0.5))) atomicOr(status, 1);
        hb[i] = dh;
    }
}

// ---------------------------------------------------------------------------
// Pair weights of a (+e, -e) pair of the contact shell.  With
// q = g2(chi_mid) n(r+e) (without the quadrature weight), chi_mid/2 =
// hb(r) + hb(r+e), the weights are carried doubled, Q = 2q, which makes the
// Carnahan-Starling value one multiply-add: 2 g2 = (1 + s)/s^3 with
// s = 1 - chi_mid (Percus-Yevick: (3 - s)/s^2; closure one: 2).  s0 = 1 - h(r)
// - h_off; dh, dn: deviations of the two neighbours.  Besides Q+ and Q- it
// returns 2 (Q+ - Q-), formed from the deviations so that it is accurate
// relative to itself (it is what the mean-field sum accumulates):
//   2 (Q+ - Q-) = (G+ + G-)(dn+ - dn-) + (G+ - G-)(n+ + n-),   G = 2 g2,
//   CS:  G+ - G- = (dh+ - dh-) [s+^2 + s-^2 + s+ s- (1 + s+ + s-)] / (s+^3 s-^3)
//   PY:  G+ - G- = (dh+ - dh-) [3 (s+ + s-) - s+ s-] / (s+^2 s-^2)
// (exact divided differences of the closures; s- - s+ = dh+ - dh-).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T fast_rcp(T x);
template <>
__device__ __forceinline__ float fast_rcp<float>(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ double fast_rcp<double>(double x)
{
    return 1.0 / x;
}

// a + b rounded as a sum: never contracted with a product into a multiply-add,
// so the bits do not depend on how the surrounding code is compiled
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

template <int CL, class T>
__device__ __forceinline__ void pair_weights(T s0, T noff, T dhp, T dnp, T dhm, T dnm, T &qp, T &qm, T &qd)
{
    const T np = noff + dnp, nm = noff + dnm;
    if (CL == 2) {
        qp = T(2) * np;
        qm = T(2) * nm;
        qd = T(4) * (dnp - dnm);
        return;
    }
    const T sp = s0 - dhp, sm = s0 - dhm;
    const T spm = sp * sm;
    T gp, gm, gd;
    if (CL == 0) {
        const T sp2 = sp * sp, sm2 = sm * sm;
        const T rp = fast_rcp<T>(sp2 * sp), rm = fast_rcp<T>(sm2 * sm);
        gp = fma(sp, rp, rp);
        gm = fma(sm, rm, rm);
        gd = (dhp - dhm) * (add_rn(sp2, sm2) + fma(spm, sp + sm, spm)) * (rp * rm);
    } else {
        const T rp = fast_rcp<T>(sp * sp), rm = fast_rcp<T>(sm * sm);
        gp = fma(-sp, rp, T(3) * rp);
        gm = fma(-sm, rm, T(3) * rm);
        gd = (dhp - dhm) * fma(T(3), sp + sm, -spm) * (rp * rm);
    }
    qp = gp * np;
    qm = gm * nm;
    // Q+ - Q- in the form that is odd under swapping the two ends bit for bit:
    // (+e, -e) and its mirror image (-e, +e) swap the ends, so the mean-field sum
    // cancels between mirror pairs exactly where the state is mirror-symmetric.
    // (G+ (dn+ - dn-) + (G+ - G-) n- is the same number rounded differently at
    // each end; in a driven slit that left a net x-force of 0.3 % of the drive.)
    // Returned doubled, 2 (Q+ - Q-): the halving is one exact scaling of the
    // sum V in shell_forces instead of a product per pair.
    qd = fma(add_rn(gp, gm), dnp - dnm, gd * add_rn(np, nm));
}

// Shell-sum accumulators (doubled weights Q = 2q, no quadrature weight w).
// The velocity sums take the neighbours' velocities v' = v(r+e) directly; the
// node's own velocity v enters W per pair and S once, in shell_forces:
//   V    = 2 sum Q khat, doubled once more (halved in shell_forces)  (F^mf)
//   W    = sum Q khat (khat . (v' - v))                    (F^viscous)
//   S_ab = sum Q (khat_b v'_a + khat_a v'_b), diagonal once (A, before the
//          term - (V_a v_b + V_b v_a) that turns v' into v' - v)
//   t    = sum Q                                           (predictor)
template <class T>
struct ShellAcc {
    T Vx, Vy, Vz;
    T Wx, Wy, Wz;
    T Sxx, Syy, Szz, Sxy, Sxz, Syz;
    T t;
};

// Add the (+e, -e) pair with unit vector (kx, ky, kz) of +e.  khat(-e) = -khat(+e),
// so W takes the sum of the two ends' Q (v' - v) and S the difference of
// their Q v'.
template <class T>
__device__ __forceinline__ void accumulate_pair(ShellAcc<T> &a, T kx, T ky, T kz, T qp, T qm, T qd, T vpx, T vpy,
                                                T vpz, T vmx, T vmy, T vmz, T vx, T vy, T vz)
{
    const T px = qp * vpx, py = qp * vpy, pz = qp * vpz;
    const T dx = fma(-qm, vmx, px), dy = fma(-qm, vmy, py), dz = fma(-qm, vmz, pz);
    const T ex = fma(qm, vmx, px), ey = fma(qm, vmy, py), ez = fma(qm, vmz, pz);
    const T tq = add_rn(qp, qm);
    a.t += tq;
    const T sx = fma(-tq, vx, ex), sy = fma(-tq, vy, ey), sz = fma(-tq, vz, ez);
    a.Vx = fma(kx, qd, a.Vx); a.Vy = fma(ky, qd, a.Vy); a.Vz = fma(kz, qd, a.Vz);
    const T ks = fma(kx, sx, fma(ky, sy, kz * sz));
    a.Wx = fma(kx, ks, a.Wx); a.Wy = fma(ky, ks, a.Wy); a.Wz = fma(kz, ks, a.Wz);
    a.Sxx = fma(kx, dx, a.Sxx); a.Syy = fma(ky, dy, a.Syy); a.Szz = fma(kz, dz, a.Szz);
    a.Sxy = fma(ky, dx, fma(kx, dy, a.Sxy));
    a.Sxz = fma(kz, dx, fma(kx, dz, a.Sxz));
    a.Syz = fma(kz, dy, fma(ky, dz, a.Syz));
}

// Fields of one node from its shell sums: C = n (F^mf + F^viscous) with
// F^mf = -kT sigma^2 w V and F^viscous = beta w W (Eq. campoc),
// A = -(kT/5) n sigma^2 w S (Eq. campod, not yet traceless), and
// t = w sum q for the predictor.  w/2 undoes the doubled weights.
template <class T>
__device__ __forceinline__ void shell_forces(const KParams &p, const ShellAcc<T> &a, T n, T vx, T vy, T vz, T &Cx,
                                             T &Cy, T &Cz, T &Axx, T &Ayy, T &Azz, T &Axy, T &Axz, T &Ayz, T &tsum)
{
    const T wh = T(0.5) * prm<T>(p.wshell, p.f_wshell);
    // the mean-field sum, carried doubled (pair_weights): halving is exact
    const T Vx = T(0.5) * a.Vx, Vy = T(0.5) * a.Vy, Vz = T(0.5) * a.Vz;
    const T mf = -T(CS2) * prm<T>(p.sig2, p.f_sig2) * wh * n;
    const T vi = prm<T>(p.beta, p.f_beta) * wh * n;
    // multiply-adds written out (the same bits in every kernel); the product
    // with the mean-field sum V, the larger term next to a wall, enters exactly
    Cx = fma(mf, Vx, vi * a.Wx);
    Cy = fma(mf, Vy, vi * a.Wy);
    Cz = fma(mf, Vz, vi * a.Wz);
    const T pa = -(T(CS2) / T(5)) * prm<T>(p.sig2, p.f_sig2) * n * wh;
    Axx = T(2) * pa * fma(-Vx, vx, a.Sxx);
    Ayy = T(2) * pa * fma(-Vy, vy, a.Syy);
    Azz = T(2) * pa * fma(-Vz, vz, a.Szz);
    Axy = pa * (a.Sxy - fma(Vy, vx, Vx * vy));
    Axz = pa * (a.Sxz - fma(Vz, vx, Vx * vz));
    Ayz = pa * (a.Syz - fma(Vz, vy, Vy * vz));
    tsum = a.t * wh;
}

// ---------------------------------------------------------------------------
// Collision and push streaming of node i (step 3 of Sec. 5), given its fields.
// C = n (F^mf + F^viscous) (Eq. campoc); A (Eq. campod, not yet traceless);
// tsum = t of the field-velocity predictor for the next step.  FIELDS: write
// nbar, C, A and the collision velocity instead of advancing the state.
// ---------------------------------------------------------------------------
// Index offsets from node (x, y, z) to its neighbours one step down and up
// each axis, wrapped periodically in x and y (and z without walls; with walls,
// z +- 1 of a fluid node lies in the lattice).  Formed once per node, so that
// the push of every direction is the same branch-free sum of three offsets.
struct PushOffsets {
    int xm, xp, ym, yp, zm, zp;
};

template <bool WALLS>
__device__ __forceinline__ PushOffsets push_offsets(int x, int y, int z, int nx, int ny, int nz)
{
    const int nxy = nx * ny;
    PushOffsets o;
    o.xm = x > 0 ? -1 : nx - 1;
    o.xp = x < nx - 1 ? 1 : 1 - nx;
    o.ym = y > 0 ? -nx : (ny - 1) * nx;
    o.yp = y < ny - 1 ? nx : (1 - ny) * nx;
    o.zm = WALLS || z > 0 ? -nxy : (nz - 1) * nxy;
    o.zp = WALLS || z < nz - 1 ? nxy : (1 - nz) * nxy;
    return o;
}

// i + c for a lattice direction c with components in {-1, 0, 1}
__device__ __forceinline__ int push_target(const PushOffsets &o, int i, int cx, int cy, int cz)
{
    return i + (cx < 0 ? o.xm : cx > 0 ? o.xp : 0) + (cy < 0 ? o.ym : cy > 0 ? o.yp : 0) +
           (cz < 0 ? o.zm : cz > 0 ? o.zp : 0);
}

// target_dn(q, dst) returns n - n_off of the node a population is pushed to
// (this step's density there: its storage scale for the next step).
template <class S, int CL, bool WALLS, bool FIELDS, class T, class TargetDn>
__device__ __forceinline__ void collide_push(const KParams &p, const KBufs<S, T> &b, int i, int x, int y, int z,
                                             T hr, T Cx, T Cy, T Cz, T Axx, T Ayy, T Azz, T Axy, T Axz, T Ayz,
                                             T tsum, T dn_self, TargetDn target_dn)
{
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const T noff = prm<T>(p.n_off, p.f_n_off);
    const T dsc = b.nscale[i];           // this node's storage scale - n_off
    const T sc = noff + dsc;
    T d[NQ];
    T dn = T(0), jx = T(0), jy = T(0), jz = T(0);   // dn: n - s(r)
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        d[q] = Store<S>::load(b.f_in + (size_t)q * p.Npad + i, T(w_of(q)) * sc);
        dn += d[q];
        if (cx_of(q)) jx += T(cx_of(q)) * d[q];
        if (cy_of(q)) jy += T(cy_of(q)) * d[q];
        if (cz_of(q)) jz += T(cz_of(q)) * d[q];
    }
    const T n = sc + dn;
    const T inv_n = T(1) / n;

    // collision velocity u = (j + F/2)/n with F = n g + C
    const T Fx = n * prm<T>(p.g[0], p.f_g[0]) + Cx, Fy = n * prm<T>(p.g[1], p.f_g[1]) + Cy, Fz = n * prm<T>(p.g[2], p.f_g[2]) + Cz;
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
    T omega = prm<T>(p.omega, p.f_omega);
    if (p.omega_mode == 1) {
        const T chib = T(2) * hr;
        const T loc = chib / prm<T>(p.chi_of_n, p.f_chi_of_n) * contact_g<CL, T>(chib);
        T tau = loc > T(0) ? T(0.5) + (prm<T>(p.tau, p.f_tau) - T(0.5)) * prm<T>(p.ref_ng, p.f_ref_ng) / loc : T(1e30);
        tau = tau < T(0.501) ? T(0.501) : tau;
        omega = T(1) / tau;
    }

    // collision (Eq. SMDB, second order): f* = f - omega (f - feq) + (1 - omega/2)(Phi + S^A)
    const T tr3 = (Axx + Ayy + Azz) * T(1.0 / 3.0);
    const T Bxx = Axx - tr3, Byy = Ayy - tr3, Bzz = Azz - tr3;   // traceless A
    const T kA = p.interactions ? prm<T>(p.k_cross, p.f_k_cross) * T(4.5) : T(0);  // K / (2 c_s^4)
    const T uu = ux * ux + uy * uy + uz * uz;
    const T uF = ux * Fx + uy * Fy + uz * Fz;
    const T src_pref = T(1) - T(0.5) * omega;
    const PushOffsets po = push_offsets<WALLS>(x, y, z, nx, ny, nz);

    // push streaming with half-way bounce-back; re-encode relative to the
    // target's rest state w_q s(target), s(target) = its density now
    const auto push = [&](int q, T post) {
        const int cxq = cx_of(q), cyq = cy_of(q), czq = cz_of(q);
        const T wq = T(w_of(q));
        const int zt = z + czq;
        int dst;
        int qq = q;
        T dn_t;
        if (WALLS && (zt == 0 || zt == nz - 1)) {
            dst = i;
            qq = opp_of(q);
            dn_t = dn_self;
        } else {
            dst = push_target(po, i, cxq, cyq, czq);
            dn_t = q == 0 ? dn_self : target_dn(q, dst);
        }
        if (!in_bounds(dst, p.N, b.status)) return;
        const T stored = post + wq * (dsc - dn_t);
        Store<S>::put(b.f_out + (size_t)qq * p.Npad + dst, stored, T(1.0 / w_of(q)) * fast_rcp<T>(noff + dn_t));
    };
    // population q's equilibrium deviation and its forcing (Phi + S^A)
    const auto relax = [&](int q, T &feq_dev, T &forcing) {
        const int cxq = cx_of(q), cyq = cy_of(q), czq = cz_of(q);
        const T wq = T(w_of(q));
        const T cu = T(cxq) * ux + T(cyq) * uy + T(czq) * uz;
        const T cF = T(cxq) * Fx + T(cyq) * Fy + T(czq) * Fz;
        feq_dev = wq * (dn + n * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
        const T phi = wq * (T(3) * (cF - uF) + T(9) * cu * cF);
        const T cAc = T(cxq * cxq) * Bxx + T(cyq * cyq) * Byy + T(czq * czq) * Bzz +
                      T(2 * cxq * cyq) * Axy + T(2 * cxq * czq) * Axz + T(2 * cyq * czq) * Ayz;
        forcing = phi + kA * wq * cAc;
    };
    if constexpr (WALLS && sizeof(S) == sizeof(float) && sizeof(T) == sizeof(float)) {
        // FP32 storage in a slit: the momentum of the changes along the walls
        // (x, y), which is F exactly, is summed in double-word arithmetic and
        // 3 w_q c_q . (F - sum) is added back.  The roundings inside the changes
        // otherwise leave an x-momentum error that biases the steady flow of a
        // driven slit by up to 6e-5 of max|u_x|.  The correction carries no mass
        // (sum_q w_q c_q = 0).  The wall-normal component, which the walls take
        // up, is left as it is: correcting it too raised the density error of
        // the converged slit at n* 0.3 from 1.1e-7 to 8.3e-7.
        dwf Mx = dw_from(0.f), My = dw_from(0.f);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            T feq_dev, forcing;
            relax(q, feq_dev, forcing);
            const T dl = src_pref * forcing - omega * (d[q] - feq_dev);   // the change
            d[q] = d[q] + dl;
            if (cx_of(q)) Mx += cx_of(q) > 0 ? dl : -dl;
            if (cy_of(q)) My += cy_of(q) > 0 ? dl : -dl;
        }
        const T ex = T(3) * __fsub_rn(__fsub_rn(Fx, Mx.hi), Mx.lo);
        const T ey = T(3) * __fsub_rn(__fsub_rn(Fy, My.hi), My.lo);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const T cdel = T(cx_of(q)) * ex + T(cy_of(q)) * ey;
            push(q, cx_of(q) || cy_of(q) ? fma(T(w_of(q)), cdel, d[q]) : d[q]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            T feq_dev, forcing;
            relax(q, feq_dev, forcing);
            push(q, d[q] - omega * (d[q] - feq_dev) + src_pref * forcing);
        }
    }
    b.nscale[i] = dn_self;
    b.cprev[i] = Cx;
    b.cprev[p.Npad + i] = Cy;
    b.cprev[2 * p.Npad + i] = Cz;
    b.tprev[i] = tsum;
}

// ---------------------------------------------------------------------------
// Collision and push of node i as in collide_push, with the collision and the
// re-encoding for the target in double-word arithmetic (FP32 storage): the
// stored deviations, the fields and the results stay FP32.  In a driven slit
// each step changes the momentum by a fraction ~ nu/H^2 of itself (2e-4 at
// H = 159), so the ~6e-8 rounding of the FP32 collision is a few 1e-4 of the
// per-step drive, and part of it acts as a steady spurious force; here the
// collision's rounding sits ~2^-44 below its operands and the result is
// rounded once, at the store.  Velocity components that are zero for a
// lattice direction are skipped at compile time.
// ---------------------------------------------------------------------------
__device__ __forceinline__ dwf dw_signed(int c, dwf a) { return c > 0 ? a : -a; }

// c . (a, b, c3) for a lattice direction with components in {-1, 0, 1}
__device__ __forceinline__ dwf dw_cdot(int cx, int cy, int cz, dwf a, dwf b, dwf c)
{
    if (cx) {
        dwf r = dw_signed(cx, a);
        if (cy) r = r + dw_signed(cy, b);
        if (cz) r = r + dw_signed(cz, c);
        return r;
    }
    if (cy) {
        dwf r = dw_signed(cy, b);
        if (cz) r = r + dw_signed(cz, c);
        return r;
    }
    return cz ? dw_signed(cz, c) : dw_from(0.f);
}

template <class S, int CL, bool WALLS, class TargetDn>
__device__ __forceinline__ void collide_push_dw(const KParams &p, const KBufs<S, float> &b, int i, int x, int y,
                                                int z, float hr, float Cx, float Cy, float Cz, float Axx, float Ayy,
                                                float Azz, float Axy, float Axz, float Ayz, float tsum, float dn_self,
                                                TargetDn target_dn)
{
    static_assert(sizeof(S) == sizeof(float), "double-word collision: FP32 storage");
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const float noff = p.f_n_off;
    const float dsc = b.nscale[i];
    float d[NQ];
    dwf dn = dw_from(0.f), jx = dw_from(0.f), jy = dw_from(0.f), jz = dw_from(0.f);
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        d[q] = Store<S>::load(b.f_in + (size_t)q * p.Npad + i, 0.f);
        dn += d[q];
        if (cx_of(q)) jx += cx_of(q) > 0 ? d[q] : -d[q];
        if (cy_of(q)) jy += cy_of(q) > 0 ? d[q] : -d[q];
        if (cz_of(q)) jz += cz_of(q) > 0 ? d[q] : -d[q];
    }
    const dwf n = two_sum(noff, dsc) + dn;
    const dwf inv_n = dw_from(1.f) / n;

    // collision velocity u = (j + F/2)/n with F = n g + C
    const dwf Fx = n * dw_load(p.g_dw[0]) + Cx, Fy = n * dw_load(p.g_dw[1]) + Cy, Fz = n * dw_load(p.g_dw[2]) + Cz;
    const dwf ux = (jx + dw_scale2(Fx, 0.5f)) * inv_n;
    const dwf uy = (jy + dw_scale2(Fy, 0.5f)) * inv_n;
    const dwf uz = (jz + dw_scale2(Fz, 0.5f)) * inv_n;

    dwf omega = dw_load(p.omega_dw);
    if (p.omega_mode == 1) {
        const float chib = 2.f * hr;
        const float loc = chib / p.f_chi_of_n * contact_g<CL, float>(chib);
        float tau = loc > 0.f ? 0.5f + (p.f_tau - 0.5f) * p.f_ref_ng / loc : 1e30f;
        tau = tau < 0.501f ? 0.501f : tau;
        omega = dw_from(1.f) / dw_from(tau);
    }

    const dwf tr3 = (two_sum(Axx, Ayy) + Azz) * dw_const(1.0 / 3.0);
    const dwf Bxx = Axx - tr3, Byy = Ayy - tr3, Bzz = Azz - tr3;   // traceless A
    const dwf kA = dw_load(p.ka_dw);                               // K / (2 c_s^4), 0 without fields
    const dwf uu15 = (ux * ux + uy * uy + uz * uz) * 1.5f;
    const dwf uF = ux * Fx + uy * Fy + uz * Fz;
    const dwf src_pref = dw_from(1.f) - dw_scale2(omega, 0.5f);
    const PushOffsets po = push_offsets<WALLS>(x, y, z, nx, ny, nz);

#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const int cxq = cx_of(q), cyq = cy_of(q), czq = cz_of(q);
        const dwf wq = dw_const(w_of(q));
        const dwf cu = dw_cdot(cxq, cyq, czq, ux, uy, uz);
        const dwf cF = dw_cdot(cxq, cyq, czq, Fx, Fy, Fz);
        const dwf feq_dev = wq * (dn + n * (cu * 3.f + (cu * cu) * 4.5f - uu15));
        const dwf phi = wq * ((cF - uF) * 3.f + (cu * cF) * 9.f);
        // c_q^2-weighted diagonal of traceless A (the rest direction has none)
        dwf cAc = cxq ? Bxx : (cyq ? Byy : (czq ? Bzz : dw_from(0.f)));
        if (cxq && cyq) cAc = cAc + Byy;
        if ((cxq || cyq) && czq) cAc = cAc + Bzz;
        if (cxq && cyq) cAc = cAc + float(2 * cxq * cyq) * Axy;
        if (cxq && czq) cAc = cAc + float(2 * cxq * czq) * Axz;
        if (cyq && czq) cAc = cAc + float(2 * cyq * czq) * Ayz;
        const dwf sa = kA * wq * cAc;
        const dwf post = d[q] - omega * (d[q] - feq_dev) + src_pref * (phi + sa);
        const int zt = z + czq;
        int dst;
        int qq = q;
        float dn_t;
        if (WALLS && (zt == 0 || zt == nz - 1)) {
            dst = i;
            qq = opp_of(q);
            dn_t = dn_self;
        } else {
            dst = push_target(po, i, cxq, cyq, czq);
            dn_t = q == 0 ? dn_self : target_dn(q, dst);
        }
        if (!in_bounds(dst, p.N, b.status)) continue;
        const float stored = dw_round(post + wq * two_sum(dsc, -dn_t));
        Store<S>::put(b.f_out + (size_t)qq * p.Npad + dst, stored, 0.f);
    }
    b.nscale[i] = dn_self;
    b.cprev[i] = Cx;
    b.cprev[p.Npad + i] = Cy;
    b.cprev[2 * p.Npad + i] = Cz;
    b.tprev[i] = tsum;
}

// Shell sums of node (x, y, z) with the table in global memory (any sigma,
// any lattice shape): the (+e, -e) pairs of the library's table, neighbours
// wrapped periodically in x, y (and z without walls), n = 0 on and beyond the
// walls.  nu, hb in deviation form (see above).  WT: per-vector quadrature
// weights (the compact shell) in shell_k[m].w scale the pair's Q; without
// WT the uniform weight is applied once, in shell_forces.
template <int CL, bool WALLS, class T, bool WT = false>
__device__ __forceinline__ void shell_sums_generic(const KParams &p, const V4<T> *nu, const T *hb,
                                                   const int4 *shell_e, const V4<T> *shell_k, int x, int y, int z,
                                                   T hr, T vx, T vy, T vz, ShellAcc<T> &a, int *status)
{
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const T noff = prm<T>(p.n_off, p.f_n_off), hoff = prm<T>(p.h_off, p.f_h_off);
    const T s0 = T(1) - hr - hoff;
    auto fetch = [&](int ex, int ey, int ez, V4<T> &nb, T &hbv) {
        int zz = z + ez;
        bool solid = false;
        if (WALLS)
            solid = zz <= 0 || zz >= nz - 1;
        else
            zz = wrap_coord(zz, nz);
        const int j = solid ? 0 : wrap_coord(x + ex, nx) + nx * (wrap_coord(y + ey, ny) + ny * zz);
        if (solid || !in_bounds(j, p.N, status)) {
            nb = V4<T>{-noff, T(0), T(0), T(0)};
            hbv = -hoff;
        } else {
            nb = nu[j];
            hbv = hb[j];
        }
    };
    for (int m = 0; m + 1 < p.nshell; m += 2) {     // (+e, -e) pairs
        const int4 e = shell_e[m];
        const V4<T> k = shell_k[m];
        V4<T> nb[2];
        T hbv[2];
        fetch(e.x, e.y, e.z, nb[0], hbv[0]);
        fetch(-e.x, -e.y, -e.z, nb[1], hbv[1]);
        T qp, qm, qd;
        pair_weights<CL, T>(s0, noff, hbv[0], nb[0].x, hbv[1], nb[1].x, qp, qm, qd);
        if (WT) {
            qp *= k.w;
            qm *= k.w;
            qd *= k.w;
        }
        accumulate_pair<T>(a, k.x, k.y, k.z, qp, qm, qd, nb[0].y, nb[0].z, nb[0].w, nb[1].y, nb[1].z, nb[1].w, vx,
                           vy, vz);
    }
}

// ---------------------------------------------------------------------------
// Fields + collision + streaming, one node per thread, shell table from
// global memory (any sigma and lattice shape).
// ---------------------------------------------------------------------------
template <class S, int CL, bool WALLS, bool FIELDS, bool WT = false, class A = typename Store<S>::T>
__device__ __forceinline__ void shell_body(const KParams &p, const KBufs<S, typename Store<S>::T> &b, int blk)
{
    typedef typename Store<S>::T T;
    int i = blk * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int x = i % nx;
    int y = (i / nx) % ny;
    int z = i / (nx * ny);
    if (WALLS && (z == 0 || z == nz - 1)) return;

    const T noff = prm<T>(p.n_off, p.f_n_off), hoff = prm<T>(p.h_off, p.f_h_off);
    const T dhr = b.hb[i];
    const T hr = hoff + dhr;
    const V4<T> me = b.nu[i];
    const T n = noff + me.x;
    const T vx = me.y, vy = me.z, vz = me.w;

    T Cx = T(0), Cy = T(0), Cz = T(0);
    T Axx = T(0), Ayy = T(0), Azz = T(0), Axy = T(0), Axz = T(0), Ayz = T(0);
    T tsum = T(0);
    if (p.interactions) {
        ShellAcc<T> a = {};
        shell_sums_generic<CL, WALLS, T, WT>(p, b.nu, b.hb, b.shell_e, b.shell_k, x, y, z, hr, vx, vy, vz, a,
                                             b.status);
        shell_forces<T>(p, a, n, vx, vy, vz, Cx, Cy, Cz, Axx, Ayy, Azz, Axy, Axz, Ayz, tsum);
    }
    const auto target_dn = [&](int, int dst) { return in_bounds(dst, p.N, b.status) ? b.nu[dst].x : T(0); };
    if constexpr (is_dw<A>::value && !FIELDS)
        collide_push_dw<S, CL, WALLS>(p, b, i, x, y, z, hr, Cx, Cy, Cz, Axx, Ayy, Azz, Axy, Axz, Ayz, tsum, me.x,
                                      target_dn);
    else
        collide_push<S, CL, WALLS, FIELDS>(p, b, i, x, y, z, hr, Cx, Cy, Cz, Axx, Ayy, Azz, Axy, Axz, Ayz, tsum,
                                           me.x, target_dn);
}

template <class S, int CL, bool WALLS, bool FIELDS, bool WT>
__global__ void __launch_bounds__(256) k_shell_collide(KParams p, KBufs<S, typename Store<S>::T> b)
{
    shell_body<S, CL, WALLS, FIELDS, WT>(p, b, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Energy-equation fields of Sec. 3 on a prescribed temperature T (k_B T per
// node, lattice units, m = 1), in FP64 from the state's fields (n, the field
// velocity v, the smeared density) with the shell sum of C and A:
//   Q    = T n sigma^2 sum_e w g2 n(r+e) [-khat.(v(r+e) - v(r))/2
//                                         + sqrt(T/pi) (T(r+e) - T(r))/T]   (Eq. campob1)
//   B_i  = -2 T n sigma^2 sum_e w khat_i g2 n(r+e) (T(r+e) - T(r))           (Eq. campos)
//   F^T_i = -(sigma^2/2) sum_e w khat_i g2 n(r+e) (T(r+e) - T(r))            (Eq. thermalforce)
// g2 at the mean of the two ends' smeared densities; khat = e/|e| in FP64;
// w the uniform shell weight or, with the compact rule, the vector's own.
// Zero on solid nodes.  An inspection path: the time step is isothermal
// (Sec. 5) and never runs it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double g2_contact_f64(int closure, double chi)
{
    if (closure == 0) return (1.0 - 0.5 * chi) / ((1.0 - chi) * (1.0 - chi) * (1.0 - chi));
    if (closure == 1) return (1.0 + 0.5 * chi) / ((1.0 - chi) * (1.0 - chi));
    return 1.0;
}

template <class S>
__global__ void __launch_bounds__(256) k_thermal_fields(KParams p, KBufs<S, typename Store<S>::T> b, const double *T,
                                                        double *Qo, double *Bo, double *Fo)
{
    typedef typename Store<S>::T Tc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    const int nx = p.nx, ny = p.ny, nz = p.nz, N = p.N;
    const int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    double q = 0.0, bs[3] = {0.0, 0.0, 0.0};
    const bool solid = solid_plane(p, z);
    const V4<Tc> me = b.nu[i];
    const double ni = p.n_off + double(me.x), Ti = T[i];
    if (!solid && p.interactions) {
        const double hr = p.h_off + double(b.hb[i]);
        for (int m = 0; m < p.nshell; m++) {
            const int4 e = b.shell_e[m];
            int zz = z + e.z;
            if (p.walls) {
                if (zz <= 0 || zz >= nz - 1) continue;     // beyond or on a wall: n = 0
            } else {
                zz = wrap_coord(zz, nz);
            }
            const int j = wrap_coord(x + e.x, nx) + nx * (wrap_coord(y + e.y, ny) + ny * zz);
            if (!in_bounds(j, N, b.status)) continue;
            const V4<Tc> nb = b.nu[j];
            const double len = sqrt(double(e.x * e.x + e.y * e.y + e.z * e.z));
            const double kx = e.x / len, ky = e.y / len, kz = e.z / len;
            const double chi = hr + p.h_off + double(b.hb[j]);    // chi_mid = h(r) + h(r+e), h = chi/2
            const double w = p.shell_rule ? double(b.shell_k[m].w) : p.wshell;
            const double wgn = w * g2_contact_f64(p.closure, chi) * (p.n_off + double(nb.x));
            const double dT = T[j] - Ti;
            const double kdu = kx * (double(nb.y) - double(me.y)) + ky * (double(nb.z) - double(me.z)) +
                               kz * (double(nb.w) - double(me.w));
            q += wgn * (-0.5 * kdu + sqrt(Ti / M_PI) * dT / Ti);
            bs[0] += wgn * kx * dT;
            bs[1] += wgn * ky * dT;
            bs[2] += wgn * kz * dT;
        }
    }
    Qo[i] = solid ? 0.0 : Ti * ni * p.sig2 * q;
    for (int d = 0; d < 3; d++) {
        Bo[d * N + i] = solid ? 0.0 : -2.0 * Ti * ni * p.sig2 * bs[d];
        Fo[d * N + i] = solid ? 0.0 : -0.5 * p.sig2 * bs[d];
    }
}

// ---------------------------------------------------------------------------
// Outputs and FP64 reductions.
// ---------------------------------------------------------------------------
template <class S>
__global__ void __launch_bounds__(256) k_pop_to_f64(KParams p, const S *f, const typename Store<S>::T *nscale, int q,
                                                    double *out)
{
    typedef typename Store<S>::T T;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int z = i / (p.nx * p.ny);
    if (solid_plane(p, z)) {
        out[i] = 0.0;
        return;
    }
    const T sc = prm<T>(p.n_off, p.f_n_off) + nscale[i];
    T dv = Store<S>::load(f + (size_t)q * p.Npad + i, T(w_of(q)) * sc);
    out[i] = double(dv) + w_of(q) * double(sc);
}

// Per-block FP64 partial sums over fluid nodes of the FP64 moments n, u_x:
// [0] sum n, [1] sum u_x, [2] sum n u_x, [3] max |u_x - snap|, [4] max |u_x|, [5] count.
// If update_snap, the snapshot is overwritten with the current u_x.
__device__ __forceinline__ void stats_body(const KParams &p, const double *n_, const double *ux_, double *snap,
                                           int update_snap, double *partial, int blk, int nblk)
{
    __shared__ double sh[6][8];
    double a0 = 0, a1 = 0, a2 = 0, m3 = 0, m4 = 0, c5 = 0;
    for (int i = blk * blockDim.x + threadIdx.x; i < p.N; i += nblk * blockDim.x) {
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
        for (int k = 0; k < 6; k++) partial[blk * 6 + k] = r[k];
    }
}

static __global__ void __launch_bounds__(256) k_stats(KParams p, const double *n_, const double *ux_, double *snap,
                                                      int update_snap, double *partial)
{
    stats_body(p, n_, ux_, snap, update_snap, partial, blockIdx.x, gridDim.x);
}

// one warp: lane l takes blocks l, l + 32, ...; then a fixed shuffle tree
__device__ __forceinline__ void stats_final_body(const double *partial, int nblocks, double *out)
{
    if (threadIdx.x >= 32) return;
    double r[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        r[0] += partial[b * 6 + 0]; r[1] += partial[b * 6 + 1]; r[2] += partial[b * 6 + 2];
        r[3] = fmax(r[3], partial[b * 6 + 3]); r[4] = fmax(r[4], partial[b * 6 + 4]);
        r[5] += partial[b * 6 + 5];
    }
    for (int off = 16; off > 0; off >>= 1) {
        r[0] += __shfl_down_sync(0xffffffffu, r[0], off);
        r[1] += __shfl_down_sync(0xffffffffu, r[1], off);
        r[2] += __shfl_down_sync(0xffffffffu, r[2], off);
        r[3] = fmax(r[3], __shfl_down_sync(0xffffffffu, r[3], off));
        r[4] = fmax(r[4], __shfl_down_sync(0xffffffffu, r[4], off));
        r[5] += __shfl_down_sync(0xffffffffu, r[5], off);
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; k++) out[k] = r[k];
}

static __global__ void k_stats_final(const double *partial, int nblocks, double *out)
{
    if (blockIdx.x == 0) stats_final_body(partial, nblocks, out);
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
