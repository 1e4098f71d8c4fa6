// Compile-time instantiations: every shape, double elements, 32-byte vectors.
#include "inst.cuh"

namespace salt {
void register_f64_vb32(Registry& r) { register_width<double, 32>(r); }
}  // namespace salt
