// Compile-time instantiations: every shape, float elements, 32-byte vectors.
#include "inst.cuh"

namespace salt {
void register_f32_vb32(Registry& r) { register_width<float, 32>(r); }
}  // namespace salt
