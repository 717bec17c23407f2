// pattern_p128.cu -- pattern-kernel configurations for 128 x 128 detectors: one CTA per
// pattern (R = 128, 512 or 1024 threads) or clusters of 2 or 4 CTAs (R = 64, 32).
#include "pattern_kernels.cuh"

namespace pty {
extern const PatternImpl kImplP128[] = {make_impl<128, 128, 512>(), make_impl<128, 64, 256>(),
                                        make_impl<128, 32, 256>(), make_impl<128, 128, 1024>()};
extern const int kNumImplP128 = sizeof(kImplP128) / sizeof(kImplP128[0]);
}  // namespace pty
