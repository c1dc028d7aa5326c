// Instantiations of the high-dimensional path for double coordinates (rows padded to 8..64).
#include "hd_run.cuh"

namespace hca {
template int run_hd<double, 8>(const RunArgs &);
template int run_hd<double, 16>(const RunArgs &);
template int run_hd<double, 32>(const RunArgs &);
template int run_hd<double, 64>(const RunArgs &);
}  // namespace hca
