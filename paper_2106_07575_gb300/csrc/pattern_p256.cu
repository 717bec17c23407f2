// pattern_p256.cu -- pattern-kernel configurations for 256 x 256 detectors: the 526 KB
// exit wave does not fit one SM, so a cluster of 8 (R = 32) or 4 (R = 64) CTAs shares it.
#include "pattern_kernels.cuh"

namespace pty {
extern const PatternImpl kImplP256[] = {make_impl<256, 32, 256>(), make_impl<256, 64, 512>()};
extern const int kNumImplP256 = sizeof(kImplP256) / sizeof(kImplP256[0]);
}  // namespace pty
