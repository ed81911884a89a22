// Tiled shell kernel: the shell sums, collision and streaming of
// shell_body (steps 2 + 3 of Sec. 5), in FP32, with the field tile and its
// shell halo staged in shared memory.
//
// Block: a brick of 8 x 8 x TZ output nodes.  Three shapes (tile variants),
// chosen per (sigma, walls, nz) by the autotuner:
//   0: TZ = 8, 256 threads, two nodes each (z and z + 4);
//   1: TZ = 8, 512 threads, one node each (16 warps per SM when only one
//      block fits, as for sigma 6, whose tile takes 160 KB);
//   2: TZ = 4, 256 threads, one node each (less z padding in thin slits and
//      a smaller tile: three blocks per SM at sigma 4, more halo per node).
// Shared memory holds (8 + 2R)^2 (TZ + 2R) nodes of (n - n_off, v_x, v_y,
// v_z) and hb - h_off, R = floor(sigma + 1/2), with periodic wrap in x, y (and
// z without walls) and n = 0 beyond the walls, so the shell loop needs no
// bounds checks: a solid or missing neighbour has n = 0 and adds nothing.
// The tile arrives by cp.async (16 bytes of nu, 4 of hb per node), so all
// of a thread's halo loads are in flight together (measured 3 % faster for
// the full sigma-4 shell, 8 to 18 % for the compact shells).
// The (+e, -e) pairs of the contact shell are staged once per block as
// (khat_x, khat_y, khat_z, offset of +e in the tile); the loop over them is
// kept rolled (a few pairs per iteration) so the code stays in the
// instruction cache.  Each pair goes through pair_weights and accumulate_pair,
// the same arithmetic as shell_body.  WT (the compact shell): the pairs are
// the first nshell/2 of the table, staged with their weights, which scale
// each pair's Q as in shell_body.
#pragma once

#include <type_traits>

#include "wdlb_kernels.cuh"

namespace wdlb {
namespace tiled {


constexpr int TX = 8, TY = 8;
constexpr int kVariants = 3;

constexpr int tz_of(int V) { return V == 2 ? 4 : 8; }
constexpr int threads_of(int V) { return V == 1 ? 512 : 256; }

constexpr int shell_radius(int S2) { return (S2 + 1) / 2; }

constexpr int shell_count(int S2)
{
    int R = shell_radius(S2), m = 0;
    for (int x = -R; x <= R; x++)
        for (int y = -R; y <= R; y++)
            for (int z = -R; z <= R; z++) {
                int r4 = 4 * (x * x + y * y + z * z);
                if ((S2 - 1) * (S2 - 1) < r4 && r4 <= (S2 + 1) * (S2 + 1)) m++;
            }
    return m;
}

// ---------------------------------------------------------------------------
// Compile-time shell tables.  For the shells below, the (+e, -e) pairs are
// generated at compile time in the order of the library's table (dx from 0 to
// R, then dy and dz from -R to R, +e lexicographically positive), so the pair
// loop unrolls with constant unit vectors and constant tile offsets, and the
// products with a zero component of khat drop out.  The compact rule's orbits
// (sorted |components|) at sigma 3, 4 and 6 are the ones the library's rule
// selects; wdlb_launch.cu checks the library's table against these before it
// uses them.  The per-orbit weights stay runtime values.
// ---------------------------------------------------------------------------
namespace ct {

constexpr double sqrt_newton(double x)
{
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 64; i++) r = 0.5 * (r + x / r);
    return r;
}

constexpr int kMaxPairs = 128;

struct Orbits {
    int n;
    int key[3][3];
};

// the compact rule's orbits at 2 sigma = S2 (n = 0: no compiled table)
constexpr Orbits compact_orbits(int S2)
{
    return S2 == 6    ? Orbits{3, {{0, 0, 3}, {0, 2, 2}, {2, 2, 2}}}
           : S2 == 8  ? Orbits{3, {{0, 0, 4}, {0, 2, 3}, {0, 3, 3}}}
           : S2 == 12 ? Orbits{2, {{0, 0, 6}, {2, 4, 4}, {0, 0, 0}}}
                      : Orbits{0, {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}};
}

// orbit index of e under the compact rule, -1 if e is in none of its orbits
constexpr int orbit_of(int S2, int x, int y, int z)
{
    int v[3] = {x < 0 ? -x : x, y < 0 ? -y : y, z < 0 ? -z : z};
    for (int p = 0; p < 2; p++)
        for (int q = 0; q < 2 - p; q++)
            if (v[q] > v[q + 1]) {
                int t = v[q];
                v[q] = v[q + 1];
                v[q + 1] = t;
            }
    const Orbits o = compact_orbits(S2);
    for (int k = 0; k < o.n; k++)
        if (o.key[k][0] == v[0] && o.key[k][1] == v[1] && o.key[k][2] == v[2]) return k;
    return -1;
}

template <int S2, bool COMPACT>
struct PairTable {
    int n;
    int ex[kMaxPairs], ey[kMaxPairs], ez[kMaxPairs], orb[kMaxPairs];
    constexpr PairTable() : n(0), ex{}, ey{}, ez{}, orb{}
    {
        const int R = (S2 + 1) / 2;
        for (int dx = 0; dx <= R; dx++)
            for (int dy = -R; dy <= R; dy++)
                for (int dz = -R; dz <= R; dz++) {
                    const bool positive = dx > 0 || (dx == 0 && (dy > 0 || (dy == 0 && dz > 0)));
                    const int r4 = 4 * (dx * dx + dy * dy + dz * dz);
                    if (!positive || !((S2 - 1) * (S2 - 1) < r4 && r4 <= (S2 + 1) * (S2 + 1))) continue;
                    const int o = COMPACT ? orbit_of(S2, dx, dy, dz) : 0;
                    if (o < 0 || n >= kMaxPairs) continue;
                    ex[n] = dx;
                    ey[n] = dy;
                    ez[n] = dz;
                    orb[n] = o;
                    n++;
                }
    }
};

// largest |component| of the table's vectors
template <int S2, bool COMPACT>
constexpr int max_component()
{
    constexpr PairTable<S2, COMPACT> T{};
    int mx = 0;
    for (int m = 0; m < T.n; m++) {
        const int c[3] = {T.ex[m], T.ey[m], T.ez[m]};
        for (int d = 0; d < 3; d++) mx = (c[d] < 0 ? -c[d] : c[d]) > mx ? (c[d] < 0 ? -c[d] : c[d]) : mx;
    }
    return mx;
}

template <int S2>
constexpr int first_pair_of_orbit(int o)
{
    constexpr PairTable<S2, true> T{};
    for (int m = 0; m < T.n; m++)
        if (T.orb[m] == o) return m;
    return 0;
}

// Shells with a compiled table: the compact rule at sigma 3, 4 and 6 (13, 21
// and 15 pairs; 7-10 % faster than the runtime table on the 128^3 box).  The
// full shells keep the runtime loop: unrolled, their 49 to 225 pairs ran 4 %
// (sigma 3) and 21 % (sigma 4) slower, the code no longer fitting the
// instruction cache.
template <int S2, bool COMPACT>
constexpr bool compiled()
{
    return COMPACT && compact_orbits(S2).n > 0;
}

template <int B, int E, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// accumulate_pair with khat = e/|e| known at compile time: the products with
// a zero component are skipped (a multiply-add by zero is not folded away by
// the compiler, as it would change NaN and infinity propagation).
template <int EX, int EY, int EZ>
__device__ __forceinline__ void accumulate_pair_ct(ShellAcc<float> &a, float qp, float qm, float qd, float vpx,
                                                   float vpy, float vpz, float vmx, float vmy, float vmz, float vx,
                                                   float vy, float vz)
{
    constexpr double len = sqrt_newton(double(EX * EX + EY * EY + EZ * EZ));
    constexpr float kx = float(EX / len), ky = float(EY / len), kz = float(EZ / len);
    const float px = qp * vpx, py = qp * vpy, pz = qp * vpz;
    const float dx = fmaf(-qm, vmx, px), dy = fmaf(-qm, vmy, py), dz = fmaf(-qm, vmz, pz);
    const float ex = fmaf(qm, vmx, px), ey = fmaf(qm, vmy, py), ez = fmaf(qm, vmz, pz);
    const float tq = __fadd_rn(qp, qm);   // never contracted: the same bits in every build
    a.t += tq;
    float ks = 0.f;
    if constexpr (EZ != 0) ks = kz * fmaf(-tq, vz, ez);
    if constexpr (EY != 0) ks = fmaf(ky, fmaf(-tq, vy, ey), ks);
    if constexpr (EX != 0) ks = fmaf(kx, fmaf(-tq, vx, ex), ks);
    if constexpr (EX != 0) {
        a.Vx = fmaf(kx, qd, a.Vx);
        a.Wx = fmaf(kx, ks, a.Wx);
        a.Sxx = fmaf(kx, dx, a.Sxx);
    }
    if constexpr (EY != 0) {
        a.Vy = fmaf(ky, qd, a.Vy);
        a.Wy = fmaf(ky, ks, a.Wy);
        a.Syy = fmaf(ky, dy, a.Syy);
    }
    if constexpr (EZ != 0) {
        a.Vz = fmaf(kz, qd, a.Vz);
        a.Wz = fmaf(kz, ks, a.Wz);
        a.Szz = fmaf(kz, dz, a.Szz);
    }
    if constexpr (EX != 0) a.Sxy = fmaf(kx, dy, a.Sxy);
    if constexpr (EY != 0) a.Sxy = fmaf(ky, dx, a.Sxy);
    if constexpr (EX != 0) a.Sxz = fmaf(kx, dz, a.Sxz);
    if constexpr (EZ != 0) a.Sxz = fmaf(kz, dx, a.Sxz);
    if constexpr (EY != 0) a.Syz = fmaf(ky, dz, a.Syz);
    if constexpr (EZ != 0) a.Syz = fmaf(kz, dy, a.Syz);
}

}  // namespace ct

template <int S2, int V, bool WT = false>
constexpr size_t smem_bytes()
{
    constexpr int R = shell_radius(S2);
    constexpr size_t n = size_t(TX + 2 * R) * (TY + 2 * R) * (tz_of(V) + 2 * R);
    const size_t tables = size_t(shell_count(S2) / 2) * (sizeof(float4) + (WT ? sizeof(float) : 0));
    return n * (sizeof(float4) + sizeof(float)) + (tables + 7) / 8 * 8 + sizeof(uint64_t);   // + the mbarrier
}

// TMA staging of the tile: for a halo R that is a multiple of 4 (sigma 4),
// the tile's first x coordinate x0 - R is a multiple of 4 floats (16 bytes),
// so the nu tile is one box (4 floats x 16 x 16 x (TZ + 2R) nodes) of the 4-D
// tensor (component, x, y, z) and the hb tile one box of the 3-D tensor.
template <int S2>
constexpr bool tma_staging()
{
    return shell_radius(S2) % 4 == 0 && TX + 2 * shell_radius(S2) <= 256;
}

// Blocks per SM the launch bounds ask for: for 256 threads, three where three
// blocks' shared memory fits (227 KB per SM; the compiler then keeps to 85
// registers per thread), else two where two fit, else one; one for 512
// threads.  Three blocks measured 7-12 % faster than two for sigma 3 (8^3
// bricks) and sigma 4 (8 x 8 x 4 bricks), and 5 % faster for the double-word
// collision at sigma 4, whose 85 registers spill ~100 bytes.
template <int S2, int V, bool WT = false>
constexpr int blocks_per_sm()
{
    return threads_of(V) != 256                                ? 1
           : 3 * smem_bytes<S2, V, WT>() <= size_t(227) * 1024 ? 3
           : 2 * smem_bytes<S2, V, WT>() <= size_t(227) * 1024 ? 2
                                                                : 1;
}

template <class S, int S2, int V, int CL, bool WALLS, bool FIELDS, bool WT = false, class A = float>
__device__ __forceinline__ void tiled_body(const KParams &p, const KBufs<S, float> &b, int bx, int by, int bz)
{
    constexpr int R = shell_radius(S2);
    constexpr int TZ = tz_of(V);
    constexpr int SX = TX + 2 * R, SY = TY + 2 * R, SZ = TZ + 2 * R;
    constexpr int NS = SX * SY * SZ;
    constexpr int NPAIR = shell_count(S2) / 2;
    constexpr int NT = threads_of(V);
    constexpr int ZSTEP = NT / (TX * TY);     // z rows covered by one pass of the block
    // shared memory: nu tile (16 B per node), hb tile (4 B per node), pair
    // table, pair weights, mbarrier; the two tiles 128-byte aligned for TMA
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *sm4 = reinterpret_cast<float4 *>(smem_raw);
    float *smh = reinterpret_cast<float *>(smem_raw + sizeof(float4) * NS);
    float4 *smt = reinterpret_cast<float4 *>(smem_raw + (sizeof(float4) + sizeof(float)) * NS);
    float *smw = reinterpret_cast<float *>(smt + NPAIR);   // pair weights (WT)
    uint64_t *bar = reinterpret_cast<uint64_t *>(
        smem_raw + smem_bytes<S2, V, WT>() - sizeof(uint64_t));
    static_assert(((sizeof(float4) + sizeof(float)) * NS) % 16 == 0, "pair table alignment");
    const int npair = WT ? (p.nshell >> 1) : NPAIR;
    constexpr bool CT = ct::compiled<S2, WT>();

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;

    // shell pairs: +e is entry 2m of the library's table (-e is 2m + 1)
    if constexpr (!CT) {
        for (int m = threadIdx.x; m < npair; m += NT) {
            const int4 e = b.shell_e[2 * m];
            const V4<float> k = b.shell_k[2 * m];
            smt[m] = make_float4(k.x, k.y, k.z, __int_as_float(e.x + SX * (e.y + SY * e.z)));
            if (WT) smw[m] = k.w;
        }
    }
    // compiled table with the compact rule: the weight of each orbit, taken
    // from the first pair of the orbit in the library's table
    float wo[3] = {1.f, 1.f, 1.f};
    if constexpr (CT && WT) {
        ct::static_for<0, ct::compact_orbits(S2).n>([&](auto O) {
            constexpr int m = ct::first_pair_of_orbit<S2>(decltype(O)::value);
            wo[decltype(O)::value] = b.shell_k[2 * m].w;
        });
    }
    // the field tile with its halo: one TMA box per array where the tile needs
    // no periodic wrap in x and y (and z without walls), else per-node copies
    const float noff = p.f_n_off, hoff = p.f_h_off;
    bool use_tma = false;
    if constexpr (tma_staging<S2>()) {
        // (TMA writes shared memory at 128-byte aligned addresses only)
        use_tma = p.tma && (smem_u32(sm4) & 127u) == 0 && x0 - R >= 0 && x0 + TX + R <= nx && y0 - R >= 0 &&
                  y0 + TY + R <= ny && (WALLS || (z0 - R >= 0 && z0 + TZ + R <= nz));
    }
    if (use_tma) {
        // wait_limit < 0 (tests only): no copy is issued and the barrier is
        // never completed, so the wait runs out after -wait_limit polls
        const bool probe = p.wait_limit < 0;
        const int limit = probe ? -p.wait_limit : p.wait_limit;
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            if (!probe) {
                mbar_arrive_expect_tx(bar, (unsigned)(NS * (sizeof(float4) + sizeof(float))));
                const char *tm = static_cast<const char *>(p.tmaps);
                tma_load_4d(sm4, tm, 0, x0 - R, y0 - R, z0 - R, bar);
                tma_load_3d(smh, tm + 128, x0 - R, y0 - R, z0 - R, bar);
            }
        }
        __syncthreads();   // the barrier is initialised before anyone polls it
        const bool ok = mbar_wait_bounded(bar, limit);
        if (__syncthreads_or(!ok)) {
            // gave up: report it, then wait (bounded) for any copy in flight
            // before the block's shared memory is released
            if (threadIdx.x == 0) atomicOr(b.status, kStatusTimeout);
            if (!probe) mbar_wait_bounded(bar, kDefaultWaitLimit);
            return;
        }
        if (WALLS && (z0 - R < 0 || z0 + TZ + R > nz)) {
            // the box read zeros beyond the lattice; beyond a wall n = 0
            for (int idx = threadIdx.x; idx < NS; idx += NT) {
                const int gz = z0 - R + idx / (SX * SY);
                if (gz < 0 || gz >= nz) {
                    sm4[idx] = make_float4(-noff, 0.f, 0.f, 0.f);
                    smh[idx] = -hoff;
                }
            }
        }
    }
    for (int idx = threadIdx.x; idx < (use_tma ? 0 : NS); idx += NT) {
        const int sx = idx % SX, sy = (idx / SX) % SY, sz = idx / (SX * SY);
        int gx = x0 - R + sx, gy = y0 - R + sy, gz = z0 - R + sz;
        gx = wrap_coord(gx, nx);
        gy = wrap_coord(gy, ny);
        bool inside = true;
        if (WALLS)
            inside = gz >= 0 && gz < nz;
        else
            gz = wrap_coord(gz, nz);
        const int g = gx + nx * (gy + ny * gz);
        if (inside && in_bounds(g, p.N, b.status)) {   // asynchronous copies: all loads in flight at once
            cp_async_ca<16>(sm4 + idx, b.nu + g);
            cp_async_ca<4>(smh + idx, b.hb + g);
        } else {        // beyond a wall: n = 0
            sm4[idx] = make_float4(-noff, 0.f, 0.f, 0.f);
            smh[idx] = -hoff;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (use_tma && threadIdx.x == 0) mbar_inval(bar);

    const int tx = threadIdx.x & 7, ty = (threadIdx.x >> 3) & 7, tzb = threadIdx.x >> 6;
#pragma unroll 1
    for (int half = 0; half < TZ / ZSTEP; half++) {
        const int tz = tzb + ZSTEP * half;
        const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
        if (x >= nx || y >= ny || z >= nz) continue;
        if (WALLS && (z == 0 || z == nz - 1)) continue;
        const int i = x + nx * (y + ny * z);
        const int base = (tx + R) + SX * ((ty + R) + SY * (tz + R));
        const float4 me = sm4[base];
        const float hr = hoff + smh[base];

        float Cx = 0.f, Cy = 0.f, Cz = 0.f;
        float Axx = 0.f, Ayy = 0.f, Azz = 0.f, Axy = 0.f, Axz = 0.f, Ayz = 0.f, tsum = 0.f;
        if (p.interactions) {
            ShellAcc<float> a = {};
            const float s0 = 1.f - hr - hoff;
            if constexpr (CT) {
                constexpr ct::PairTable<S2, WT> T{};
                // The offsets are constants: every component of a table vector
                // is at most R, the tile's halo, so base +- off stays inside the
                // tile for every thread.  Proved here at compile time, which
                // keeps the pair loop the same code in the checked build.
                static_assert(ct::max_component<S2, WT>() <= R, "shell vector beyond the tile halo");
                ct::static_for<0, T.n>([&](auto M) {
                    constexpr int m = decltype(M)::value;
                    constexpr int EX = T.ex[m], EY = T.ey[m], EZ = T.ez[m];
                    constexpr int off = EX + SX * (EY + SY * EZ);
                    const float4 np = sm4[base + off];
                    const float hp = smh[base + off];
                    const float4 nm = sm4[base - off];
                    const float hm = smh[base - off];
                    float qp, qm, qd;
                    pair_weights<CL, float>(s0, noff, hp, np.x, hm, nm.x, qp, qm, qd);
                    if constexpr (WT) {
                        const float r = wo[T.orb[m]];
                        qp *= r;
                        qm *= r;
                        qd *= r;
                    }
                    ct::accumulate_pair_ct<EX, EY, EZ>(a, qp, qm, qd, np.y, np.z, np.w, nm.y, nm.z, nm.w, me.y,
                                                       me.z, me.w);
                });
            }
            // three pairs per iteration; kept rolled for sigma 6 (225 pairs), where
            // it measured 1.5 % faster
#pragma unroll(S2 >= 12 && !WT ? 1 : 3)
            for (int m = 0; m < (CT ? 0 : npair); m++) {
                const float4 t = smt[m];
                const int off = __float_as_int(t.w);
                if (!in_bounds(base + off, NS, b.status) || !in_bounds(base - off, NS, b.status)) continue;
                const float4 np = sm4[base + off];
                const float hp = smh[base + off];
                const float4 nm = sm4[base - off];
                const float hm = smh[base - off];
                float qp, qm, qd;
                pair_weights<CL, float>(s0, noff, hp, np.x, hm, nm.x, qp, qm, qd);
                if (WT) {
                    const float r = smw[m];
                    qp *= r;
                    qm *= r;
                    qd *= r;
                }
                accumulate_pair<float>(a, t.x, t.y, t.z, qp, qm, qd, np.y, np.z, np.w, nm.y, nm.z, nm.w, me.y,
                                       me.z, me.w);
            }
            shell_forces<float>(p, a, noff + me.x, me.y, me.z, me.w, Cx, Cy, Cz, Axx, Ayy, Azz, Axy, Axz, Ayz,
                                tsum);
        }
        const auto target_dn = [&](int q, int) {
            const int k = base + cx_of(q) + SX * (cy_of(q) + SY * cz_of(q));
            return in_bounds(k, NS, b.status) ? sm4[k].x : 0.f;
        };
        if constexpr (is_dw<A>::value && !FIELDS)
            collide_push_dw<S, CL, WALLS>(p, b, i, x, y, z, hr, Cx, Cy, Cz, Axx, Ayy, Azz, Axy, Axz, Ayz, tsum,
                                          me.x, target_dn);
        else
            collide_push<S, CL, WALLS, FIELDS>(p, b, i, x, y, z, hr, Cx, Cy, Cz, Axx, Ayy, Azz, Axy, Axz, Ayz,
                                               tsum, me.x, target_dn);
    }
}

}  // namespace tiled
}  // namespace wdlb
