// Instantiation of the fused stream-and-collide kernels for f16 population storage.
#include "launchers.cuh"

namespace nomrt {
const Launchers &launchers_f16() {
    static const Launchers L = make_launchers<__half>();
    return L;
}
}  // namespace nomrt
