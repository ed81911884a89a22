// Host-side stencil tables of the library (Sec. 3: the ball of the smeared
// density; Eq. campoc: the contact shell and its quadrature weight).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <utility>
#include <vector>

namespace wdlb {

// Ball of the smeared density: all b with |b|^2 <= (sigma/2)^2.
inline void build_ball(double sigma, std::vector<int> &out)
{
    out.clear();
    const double r2 = 0.25 * sigma * sigma;
    const int R = (int)std::floor(0.5 * sigma);
    for (int dx = -R; dx <= R; dx++)
        for (int dy = -R; dy <= R; dy++)
            for (int dz = -R; dz <= R; dz++)
                if (double(dx * dx + dy * dy + dz * dz) <= r2) {
                    out.push_back(dx);
                    out.push_back(dy);
                    out.push_back(dz);
                }
}

// Contact shell (sigma - 1/2)^2 < |e|^2 <= (sigma + 1/2)^2, ordered as (+e, -e)
// pairs with +e lexicographically positive; weight w such that
// sigma^2 * sum_e w e_z^2/|e| = 4 pi sigma^3 / 3.
inline void build_shell(double sigma, std::vector<int> &out, double *w)
{
    out.clear();
    const double lo = (sigma - 0.5) * (sigma - 0.5), hi = (sigma + 0.5) * (sigma + 0.5);
    const int R = (int)std::floor(sigma + 0.5);
    double second = 0.0;
    for (int dx = 0; dx <= R; dx++)
        for (int dy = -R; dy <= R; dy++)
            for (int dz = -R; dz <= R; dz++) {
                bool positive = dx > 0 || (dx == 0 && (dy > 0 || (dy == 0 && dz > 0)));
                if (!positive) continue;
                double r2 = double(dx * dx + dy * dy + dz * dz);
                if (!(r2 > lo && r2 <= hi)) continue;
                int v[2][3] = {{dx, dy, dz}, {-dx, -dy, -dz}};
                for (auto &e : v) {
                    out.push_back(e[0]);
                    out.push_back(e[1]);
                    out.push_back(e[2]);
                }
                second += 2.0 * double(dz * dz) / std::sqrt(r2);
            }
    *w = second > 0 ? (4.0 * M_PI / 3.0) * sigma / second : 0.0;
}

// Compact contact shell (shell rule 1; a quadrature of this library, the
// paper leaves the discrete integral over khat of Eq. campoc open): two or
// three orbits of the cubic group inside the full shell, one weight per orbit,
// fixed by
//   sigma^2 sum w khat_z e_z            = 4 pi sigma^3 / 3   (virial coefficient b)
//   sum w khat_x^2 e_z^2                = 4 pi sigma^2 / 15  (continuum value of the
//                                         collisional-viscosity moment)
//   sum w (khat_z^2 - 3 khat_x^2) e_z^2 = 0                  (isotropic fourth moment)
// with every weight above 1e-3 of the largest.  Of all such unions: the fewest
// vectors, then the smallest sum over its vectors of (|e|^2 - sigma^2)^2 (a
// later union must improve it by more than 1e-9 relative), then the first
// found with orbits ordered by |e|^2 and then by their sorted components, and
// unions of two orbits searched before unions of three.  Output as in
// build_shell ((+e, -e) pairs) with the weight of every vector in wts; false
// if no union qualifies.
inline bool build_shell_compact(double sigma, std::vector<int> &out, std::vector<double> &wts)
{
    out.clear();
    wts.clear();
    struct Orbit {
        int key[3];
        int r2, size;
        double col[3];
    };
    const double lo = (sigma - 0.5) * (sigma - 0.5), hi = (sigma + 0.5) * (sigma + 0.5);
    const int R = (int)std::floor(sigma + 0.5);
    auto sorted_abs = [](int x, int y, int z, int k[3]) {
        k[0] = std::abs(x);
        k[1] = std::abs(y);
        k[2] = std::abs(z);
        if (k[0] > k[1]) std::swap(k[0], k[1]);
        if (k[1] > k[2]) std::swap(k[1], k[2]);
        if (k[0] > k[1]) std::swap(k[0], k[1]);
    };
    // group the full shell by orbit, accumulating each orbit's three moments
    std::vector<Orbit> orb;
    for (int dx = -R; dx <= R; dx++)
        for (int dy = -R; dy <= R; dy++)
            for (int dz = -R; dz <= R; dz++) {
                const int r2 = dx * dx + dy * dy + dz * dz;
                if (!(double(r2) > lo && double(r2) <= hi)) continue;
                int k[3];
                sorted_abs(dx, dy, dz, k);
                size_t j = 0;
                while (j < orb.size() && !(orb[j].key[0] == k[0] && orb[j].key[1] == k[1] && orb[j].key[2] == k[2]))
                    j++;
                if (j == orb.size()) orb.push_back(Orbit{{k[0], k[1], k[2]}, r2, 0, {0.0, 0.0, 0.0}});
                const double x2 = double(dx) * dx, z2 = double(dz) * dz, len2 = double(r2);
                orb[j].size++;
                orb[j].col[0] += z2 / std::sqrt(len2);
                orb[j].col[1] += x2 * z2 / len2;
                orb[j].col[2] += (z2 * z2 - 3.0 * x2 * z2) / len2;
            }
    std::sort(orb.begin(), orb.end(), [](const Orbit &a, const Orbit &b) {
        if (a.r2 != b.r2) return a.r2 < b.r2;
        for (int d = 0; d < 3; d++)
            if (a.key[d] != b.key[d]) return a.key[d] < b.key[d];
        return false;
    });
    const double rhs[3] = {4.0 * M_PI * sigma / 3.0, 4.0 * M_PI * sigma * sigma / 15.0, 0.0};

    // least-squares weights of the orbits idx[0..k) by modified Gram-Schmidt;
    // true if the three conditions hold and every weight is positive
    auto solve = [&](const int *idx, int k, double *w) -> bool {
        double q[3][3], r[3][3] = {{0.0}};
        for (int j = 0; j < k; j++) {
            double v[3], norm0 = 0.0;
            for (int i = 0; i < 3; i++) {
                v[i] = orb[idx[j]].col[i];
                norm0 += v[i] * v[i];
            }
            for (int p = 0; p < j; p++) {
                r[p][j] = q[p][0] * v[0] + q[p][1] * v[1] + q[p][2] * v[2];
                for (int i = 0; i < 3; i++) v[i] -= r[p][j] * q[p][i];
            }
            r[j][j] = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (!(r[j][j] > 1e-12 * std::sqrt(norm0))) return false;
            for (int i = 0; i < 3; i++) q[j][i] = v[i] / r[j][j];
        }
        for (int j = k - 1; j >= 0; j--) {
            double y = q[j][0] * rhs[0] + q[j][1] * rhs[1] + q[j][2] * rhs[2];
            for (int p = j + 1; p < k; p++) y -= r[j][p] * w[p];
            w[j] = y / r[j][j];
        }
        double wmax = 0.0;
        for (int j = 0; j < k; j++) wmax = std::max(wmax, w[j]);
        for (int j = 0; j < k; j++)
            if (!(w[j] > 1e-3 * wmax)) return false;
        for (int i = 0; i < 3; i++) {
            double lhs = 0.0, mag = std::fabs(rhs[i]);
            for (int j = 0; j < k; j++) {
                lhs += orb[idx[j]].col[i] * w[j];
                mag += std::fabs(orb[idx[j]].col[i] * w[j]);
            }
            if (std::fabs(lhs - rhs[i]) > 1e-9 * mag) return false;
        }
        return true;
    };

    const int no = (int)orb.size();
    int best[3] = {-1, -1, -1}, bestk = 0, bestn = 0;
    double bestw[3] = {0.0, 0.0, 0.0}, bests = 0.0;
    auto consider = [&](const int *idx, int k) {
        double w[3];
        if (!solve(idx, k, w)) return;
        int n = 0;
        double spread = 0.0;
        for (int j = 0; j < k; j++) {
            const double d = double(orb[idx[j]].r2) - sigma * sigma;
            n += orb[idx[j]].size;
            spread += orb[idx[j]].size * d * d;
        }
        if (bestk == 0 || n < bestn || (n == bestn && spread < bests - 1e-9 * (1.0 + bests))) {
            bestk = k;
            bestn = n;
            bests = spread;
            for (int j = 0; j < k; j++) {
                best[j] = idx[j];
                bestw[j] = w[j];
            }
        }
    };
    for (int a = 0; a < no; a++)
        for (int b = a + 1; b < no; b++) {
            const int idx[2] = {a, b};
            consider(idx, 2);
        }
    for (int a = 0; a < no; a++)
        for (int b = a + 1; b < no; b++)
            for (int c = b + 1; c < no; c++) {
                const int idx[3] = {a, b, c};
                consider(idx, 3);
            }
    if (bestk == 0) return false;

    // the chosen orbits' vectors in build_shell's order, +e then -e
    for (int dx = 0; dx <= R; dx++)
        for (int dy = -R; dy <= R; dy++)
            for (int dz = -R; dz <= R; dz++) {
                const bool positive = dx > 0 || (dx == 0 && (dy > 0 || (dy == 0 && dz > 0)));
                if (!positive) continue;
                int k[3];
                sorted_abs(dx, dy, dz, k);
                for (int j = 0; j < bestk; j++) {
                    const Orbit &o = orb[best[j]];
                    if (o.key[0] != k[0] || o.key[1] != k[1] || o.key[2] != k[2]) continue;
                    const int v[2][3] = {{dx, dy, dz}, {-dx, -dy, -dz}};
                    for (auto &e : v) {
                        out.push_back(e[0]);
                        out.push_back(e[1]);
                        out.push_back(e[2]);
                        wts.push_back(bestw[j]);
                    }
                }
            }
    return true;
}

// Contact shell of either rule (0 full, 1 compact) with the weight of every
// vector; false if the rule has no shell at this sigma.
inline bool build_shell_rule(double sigma, int rule, std::vector<int> &out, std::vector<double> &wts)
{
    if (rule == 1) return build_shell_compact(sigma, out, wts);
    double w = 0.0;
    build_shell(sigma, out, &w);
    wts.assign(out.size() / 3, w);
    return rule == 0;
}

}  // namespace wdlb
