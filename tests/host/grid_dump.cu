// Host-only dump of the hypercube grids that make_grid builds (no GPU needed) for seeded random
// extents, eps, d = 1..4 and float / double input; tests/test_host_grid.py checks them.
//   grid D f32 eps mn_0 mx_0 .. mn_{D-1} mx_{D-1} | rc bin_fp64 inv_side inv_side_f tau ncell_0 ..
//        key_bits lo32 hi32 box_ok tau_box box_full box_none
#include <math.h>
#include <stdio.h>

#include <random>

#include "lowd_run.cuh"

int main() {
    std::mt19937_64 rng(1912);
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    for (int c = 0; c < 96; ++c) {
        const int D = 1 + c % 4;
        const bool f32 = (c / 4) % 2 == 0;
        const double eps = pow(10.0, -3.0 + 6.0 * u01(rng));
        double mn[4], mx[4];
        for (int i = 0; i < D; ++i) {
            const double o = (u01(rng) - 0.5) * 2e4;
            const double ext = eps * pow(10.0, -2.0 + 7.0 * u01(rng));
            mn[i] = o;
            mx[i] = o + ext;
            if (f32) {  // float input: the extremes are float values
                mn[i] = (double)(float)mn[i];
                mx[i] = (double)(float)mx[i];
                if (mx[i] < mn[i]) mx[i] = mn[i];
            }
        }
        hca::GridParams g;
        double tau = 0.0;
        const int rc = hca::detail::make_grid(D, f32, eps, 5, 1000, mn, mx, 0, g, tau);
        printf("grid %d %d %.17g", D, f32 ? 1 : 0, eps);
        for (int i = 0; i < D; ++i) printf(" %.17g %.17g", mn[i], mx[i]);
        printf(" | %d %d %.17g %.9g %.17g", rc, g.bin_fp64, g.inv_side, (double)g.inv_side_f, tau);
        for (int i = 0; i < D; ++i) printf(" %u", g.ncell[i]);
        printf(" %d %.9g %.9g %d %.9g %.9g %.9g\n", g.key_bits, (double)g.lo32, (double)g.hi32, g.box_ok,
               (double)g.tau_box, (double)g.box_full, (double)g.box_none);
    }
    return 0;
}
