// Angular sweep with per-pixel max/argmax, plain FP32 on CUDA cores.
//
// For a grid of J rotations alpha_j = 2 pi j / J the extended correlation at
// p is (Sec. 4.1 "Linear Combination", evaluated at every alpha_j)
//   S(p, j) = G_0(p) + 2 sum_{k=1..K} Re(e^{i k alpha_j} G_k(p))
//           = G_0(p) + sum_c A(p, c) B[j][c],
// A(p, 2k-2) = Re G_k, A(p, 2k-1) = Im G_k; B from the FP64 table kernel.
// The maximum over j and the first j attaining it are written per pixel
// (Sec. 5: pattern detection keeps the largest response over rotations).
#include "internal.h"

#include <cfloat>

// Each thread handles two adjacent pixels so that every B value read from
// shared memory feeds two FMAs.  B rows are padded to CP floats (multiple of 4).
template <int K>
__global__ void __launch_bounds__(256) k_sweep_fp32(const float* __restrict__ G, long long P, int J,
                                                    const float* __restrict__ B, float* __restrict__ maxv,
                                                    int32_t* __restrict__ argmax) {
  constexpr int C2 = 2 * K;
  constexpr int CP = (C2 + 3) / 4 * 4;
  extern __shared__ float4 Bs4[];
  const float4* Bg = reinterpret_cast<const float4*>(B);
  for (int i = threadIdx.x; i < J * (CP / 4); i += blockDim.x) Bs4[i] = Bg[i];
  __syncthreads();
  const long long npairs = (P + 1) / 2;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npairs;
       q += (long long)gridDim.x * blockDim.x) {
    const long long p0 = 2 * q;
    const bool two = (p0 + 1) < P;
    float a0[CP], a1[CP];
    float g00, g01;
#pragma unroll
    for (int c = 0; c < CP; ++c) { a0[c] = 0.f; a1[c] = 0.f; }
    g00 = __ldg(G + p0);
    g01 = two ? __ldg(G + p0 + 1) : 0.f;
#pragma unroll
    for (int c = 0; c < C2; ++c) {
      const float* plane = G + (size_t)(c + 1) * P;
      a0[c] = __ldg(plane + p0);
      a1[c] = two ? __ldg(plane + p0 + 1) : 0.f;
    }
    float best0 = -FLT_MAX, best1 = -FLT_MAX;
    int bj0 = 0, bj1 = 0;
    bool first = true;
    for (int j = 0; j < J; ++j) {
      float s0 = g00, s1 = g01;
      const float4* row = Bs4 + j * (CP / 4);
#pragma unroll
      for (int c4 = 0; c4 < CP / 4; ++c4) {
        const float4 b = row[c4];
        s0 = fmaf(a0[4 * c4 + 0], b.x, s0); s1 = fmaf(a1[4 * c4 + 0], b.x, s1);
        s0 = fmaf(a0[4 * c4 + 1], b.y, s0); s1 = fmaf(a1[4 * c4 + 1], b.y, s1);
        s0 = fmaf(a0[4 * c4 + 2], b.z, s0); s1 = fmaf(a1[4 * c4 + 2], b.z, s1);
        s0 = fmaf(a0[4 * c4 + 3], b.w, s0); s1 = fmaf(a1[4 * c4 + 3], b.w, s1);
      }
      if (first || s0 > best0) { best0 = s0; bj0 = j; }
      if (first || s1 > best1) { best1 = s1; bj1 = j; }
      first = false;
    }
    maxv[p0] = best0;
    argmax[p0] = bj0;
    if (two) { maxv[p0 + 1] = best1; argmax[p0 + 1] = bj1; }
  }
}

template <int K>
static void launch_sweep_fp32(const float* G, long long P, int J, const float* B, float* maxv, int32_t* argmax,
                              cudaStream_t st) {
  constexpr int CP = (2 * K + 3) / 4 * 4;
  const int smem = J * CP * 4;
  static const bool once = (smem > 0 ? cudaFuncSetAttribute(k_sweep_fp32<K>,
                                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                            227 * 1024)
                                     : cudaSuccess,
                            true);
  (void)once;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long npairs = (P + 1) / 2;
  long long blocks = (npairs + 255) / 256;
  const long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_sweep_fp32<K><<<(unsigned)blocks, 256, smem, st>>>(G, P, J, B, maxv, argmax);
}

bool sweep_fp32(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv, int32_t* argmax,
                cudaStream_t st) {
  (void)cp;
  switch (K) {
#define EXT_SWEEP_CASE(KK) case KK: launch_sweep_fp32<KK>(G, P, J, B, maxv, argmax, st); return true;
    EXT_SWEEP_CASE(1) EXT_SWEEP_CASE(2) EXT_SWEEP_CASE(3) EXT_SWEEP_CASE(4)
    EXT_SWEEP_CASE(5) EXT_SWEEP_CASE(6) EXT_SWEEP_CASE(7) EXT_SWEEP_CASE(8)
    EXT_SWEEP_CASE(9) EXT_SWEEP_CASE(10) EXT_SWEEP_CASE(11) EXT_SWEEP_CASE(12)
    EXT_SWEEP_CASE(13) EXT_SWEEP_CASE(14) EXT_SWEEP_CASE(15) EXT_SWEEP_CASE(16)
#undef EXT_SWEEP_CASE
    default: return false;
  }
}
