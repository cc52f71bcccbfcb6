// Kernel instantiations for one lattice and storage form (one unit each, so the build
// compiles them in parallel).
#include "dispatch.cuh"

namespace lbm {
Ops ops_d3q103_fp64() { return make_ops_st<LAT_D3Q103, ST_FP64>(); }
} // namespace lbm
