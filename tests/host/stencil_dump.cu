// Host-only dump of the neighbour stencil that the hypercube path builds (no GPU needed), for
// d = 1..4 and four binning error bounds tau; tests/test_host_stencil.py checks it.
//   case D tau side eps n_all n_half
//   pencil k off_0 .. off_{D-2} reach
//   near j k        (the j-th pencil of the counting order)
#include <math.h>
#include <stdio.h>

#include "lowd_run.cuh"

int main() {
    const double eps = 1.5;
    const double taus[] = {0.0, 1e-6, 0.01, 0.1};
    for (int D = 1; D <= 4; ++D) {
        for (double tau : taus) {
            const double side = eps / sqrt((double)D) * (1.0 - ldexp(1.0, -20)) / (1.0 + 2.0 * tau);
            hca::Stencil st;
            if (hca::detail::make_stencil(D, eps, side, tau, st) != HCA_OK) {
                printf("error %d %g\n", D, tau);
                return 1;
            }
            printf("case %d %.17g %.17g %.17g %d %d\n", D, tau, side, eps, st.n_all, st.n_half);
            for (int k = 0; k < st.n_all; ++k) {
                printf("pencil %d", k);
                for (int i = 0; i < D - 1; ++i) printf(" %d", (int)st.off[k][i]);
                printf(" %d\n", (int)st.reach[k]);
            }
            for (int j = 0; j < st.n_all; ++j) printf("near %d %d\n", j, (int)st.near[j]);
        }
    }
    return 0;
}
