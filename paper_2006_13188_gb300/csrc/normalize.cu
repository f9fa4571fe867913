// Division of the extended-convolution numerators by the response to the
// constant signal (Sec. 8, Eq. normalization): out[c][p] /= D[p].
#include "internal.h"

namespace {

__global__ void k_divide_channels(float* __restrict__ out, const float* __restrict__ D, long long P, int channels) {
  const long long n = P * channels;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = out[i] / __ldg(D + i % P);
}

}  // namespace

void launch_divide_channels(float* out, const float* D, long long P, int channels, int sms, cudaStream_t st) {
  long long b = (P * channels + 255) / 256;
  if (b > (long long)sms * 16) b = (long long)sms * 16;
  if (b > 0) k_divide_channels<<<(unsigned)b, 256, 0, st>>>(out, D, P, channels);
}
