// Kernel instantiations for one lattice and storage form (one unit each, so the build
// compiles them in parallel).
#include "dispatch.cuh"

namespace lbm {
Ops ops_d2q77_fp16() { return make_ops_st<LAT_D2Q77, ST_FP16>(); }
} // namespace lbm
