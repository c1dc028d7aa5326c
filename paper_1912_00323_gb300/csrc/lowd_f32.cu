// Instantiations of the hypercube-stencil path for float coordinates, d = 1..4.
#include "lowd_run.cuh"

namespace hca {
template int run_lowd<float, 1>(const RunArgs &);
template int run_lowd<float, 2>(const RunArgs &);
template int run_lowd<float, 3>(const RunArgs &);
template int run_lowd<float, 4>(const RunArgs &);
}  // namespace hca
