// Compile-time instantiations: every shape, double elements, 16-byte vectors.
#include "inst.cuh"

namespace salt {
void register_f64_vb16(Registry& r) { register_width<double, 16>(r); }
}  // namespace salt
