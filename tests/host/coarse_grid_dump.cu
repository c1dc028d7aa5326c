// Host-only dump of the coarse grids (d >= 5 path) that make_coarse_grid builds (no GPU
// needed) for seeded random extents and eps; tests/test_host_grid.py checks them.
//   coarse f32 eps mn_0 mx_0 mn_1 mx_1 mn_2 mx_2 | rc inv_side tau ncell_0 ncell_1 ncell_2
#include <math.h>
#include <stdio.h>

#include <random>

#include "hd_run.cuh"

int main() {
    std::mt19937_64 rng(1912 + 5);
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    for (int c = 0; c < 64; ++c) {
        const bool f32 = c % 2 == 0;
        const double eps = pow(10.0, -3.0 + 6.0 * u01(rng));
        double mn[3], mx[3];
        for (int i = 0; i < 3; ++i) {
            const double o = (u01(rng) - 0.5) * 2e4;
            mn[i] = o;
            mx[i] = o + eps * pow(10.0, -2.0 + 7.0 * u01(rng));
            if (f32) {
                mn[i] = (double)(float)mn[i];
                mx[i] = (double)(float)mx[i];
                if (mx[i] < mn[i]) mx[i] = mn[i];
            }
        }
        hca::GridParams g;
        double tau = 0.0;
        const int rc = hca::detail::make_coarse_grid(f32, eps, 5, 1000, mn, mx, 0, g, tau);
        printf("coarse %d %.17g", f32 ? 1 : 0, eps);
        for (int i = 0; i < 3; ++i) printf(" %.17g %.17g", mn[i], mx[i]);
        printf(" | %d %.17g %.17g %u %u %u\n", rc, g.inv_side, tau, g.ncell[0], g.ncell[1], g.ncell[2]);
    }
    return 0;
}
