// pattern_misc.cu -- configuration lookup and the device self-test of the line-search
// logarithm.
#include "mathx.cuh"
#include "pattern_kernels.cuh"

namespace pty {

extern const PatternImpl kImplP64[];
extern const int kNumImplP64;
extern const PatternImpl kImplP128[];
extern const int kNumImplP128;
extern const PatternImpl kImplP256[];
extern const int kNumImplP256;

int pattern_impls(int P, const PatternImpl **out)
{
    switch (P) {
    case 64: *out = kImplP64; return kNumImplP64;
    case 128: *out = kImplP128; return kNumImplP128;
    case 256: *out = kImplP256; return kNumImplP256;
    default: *out = nullptr; return 0;
    }
}

bool pattern_supported(int P) { return P == 64 || P == 128 || P == 256; }
int ls_window_supported(int L) { return L == 4 || L == 8 || L == 16 || L == 32; }

__global__ void k_selftest_log1p(const float *__restrict__ t, float *__restrict__ out, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = log1p_fast(t[i]);
}

cudaError_t launch_selftest_log1p(const float *t, float *out, int n, cudaStream_t s)
{
    const int nb = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    k_selftest_log1p<<<nb, 256, 0, s>>>(t, out, n);
    return cudaGetLastError();
}

}  // namespace pty
