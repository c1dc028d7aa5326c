// Instantiations of the hypercube-stencil path for double coordinates, d = 1..4.
#include "lowd_run.cuh"

namespace hca {
template int run_lowd<double, 1>(const RunArgs &);
template int run_lowd<double, 2>(const RunArgs &);
template int run_lowd<double, 3>(const RunArgs &);
template int run_lowd<double, 4>(const RunArgs &);
}  // namespace hca
