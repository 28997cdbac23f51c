// Instantiation of the fused stream-and-collide kernels for f32 population storage.
#include "launchers.cuh"

namespace nomrt {
const Launchers &launchers_f32() {
    static const Launchers L = make_launchers<float>();
    return L;
}
}  // namespace nomrt
