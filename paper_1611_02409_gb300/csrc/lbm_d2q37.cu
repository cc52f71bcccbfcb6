// Kernel instantiations for the D2Q37 lattice (Sec. VI A, Table D2Q37).
#include "dispatch.cuh"

namespace lbm {
Ops ops_d2q37(int storage) { return make_ops<LAT_D2Q37>(storage); }
} // namespace lbm
