// pattern_p64.cu -- pattern-kernel configurations for 64 x 64 detectors.
#include "pattern_kernels.cuh"

namespace pty {
extern const PatternImpl kImplP64[] = {make_impl<64, 64, 256>()};
extern const int kNumImplP64 = sizeof(kImplP64) / sizeof(kImplP64[0]);
}  // namespace pty
