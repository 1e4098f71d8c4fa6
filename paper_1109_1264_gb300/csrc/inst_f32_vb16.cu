// Compile-time instantiations: every shape, float elements, 16-byte vectors.
#include "inst.cuh"

namespace salt {
void register_f32_vb16(Registry& r) { register_width<float, 16>(r); }
}  // namespace salt
