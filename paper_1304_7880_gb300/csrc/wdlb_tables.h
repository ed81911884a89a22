// Host-side stencil tables of the library (Sec. 3: the ball of the smeared
// density; Eq. campoc: the contact shell and its quadrature weight).
#pragma once

#include <cmath>
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

}  // namespace wdlb
