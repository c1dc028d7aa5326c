// Instantiations of the high-dimensional path for float coordinates (rows padded to 8..64).
#include "hd_run.cuh"

namespace hca {
template int run_hd<float, 8>(const RunArgs &);
template int run_hd<float, 16>(const RunArgs &);
template int run_hd<float, 32>(const RunArgs &);
template int run_hd<float, 64>(const RunArgs &);
}  // namespace hca
