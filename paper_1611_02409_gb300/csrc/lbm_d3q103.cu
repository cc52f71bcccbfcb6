// Kernel instantiations for the 3-D D3Q103 lattice.
#include "dispatch.cuh"

namespace lbm {
Ops ops_d3q103(int storage) { return make_ops<LAT_D3Q103>(storage); }
} // namespace lbm
