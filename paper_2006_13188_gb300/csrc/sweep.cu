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
#include <mutex>
#include <string>

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

// Dynamic shared memory of the FP32 sweep: the J x CP steering table.
static int sweep_fp32_smem(int K, int J) { return J * ((2 * K + 3) / 4 * 4) * 4; }

bool sweep_fp32_fits(int K, int J) {
  int dev = 0, optin = 48 * 1024;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return sweep_fp32_smem(K, J) <= optin;
}

// The opt-in to more than 48 KB of dynamic shared memory is a per-device
// function attribute: set it once per (device, K).
static std::mutex g_attr_mutex;
static uint32_t g_attr_set[256] = {};   // bit K set: done on that device ordinal

template <int K>
static bool sweep_fp32_optin(int dev) {
  if (dev < 0 || dev >= 256) return false;
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  if (g_attr_set[dev] & (1u << K)) return true;
  int optin = 48 * 1024;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaFuncSetAttribute(k_sweep_fp32<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess)
    return false;
  g_attr_set[dev] |= 1u << K;
  return true;
}

template <int K>
static bool launch_sweep_fp32(const float* G, long long P, int J, const float* B, float* maxv, int32_t* argmax,
                              cudaStream_t st) {
  const int smem = sweep_fp32_smem(K, J);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  if (smem > 48 * 1024 && !sweep_fp32_optin<K>(dev)) return false;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long npairs = (P + 1) / 2;
  long long blocks = (npairs + 255) / 256;
  const long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_sweep_fp32<K><<<(unsigned)blocks, 256, smem, st>>>(G, P, J, B, maxv, argmax);
  return true;
}

bool sweep_fp32(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv, int32_t* argmax,
                cudaStream_t st) {
  (void)cp;
  switch (K) {
#define EXT_SWEEP_CASE(KK) case KK: return launch_sweep_fp32<KK>(G, P, J, B, maxv, argmax, st);
    EXT_SWEEP_CASE(1) EXT_SWEEP_CASE(2) EXT_SWEEP_CASE(3) EXT_SWEEP_CASE(4)
    EXT_SWEEP_CASE(5) EXT_SWEEP_CASE(6) EXT_SWEEP_CASE(7) EXT_SWEEP_CASE(8)
    EXT_SWEEP_CASE(9) EXT_SWEEP_CASE(10) EXT_SWEEP_CASE(11) EXT_SWEEP_CASE(12)
    EXT_SWEEP_CASE(13) EXT_SWEEP_CASE(14) EXT_SWEEP_CASE(15) EXT_SWEEP_CASE(16)
#undef EXT_SWEEP_CASE
    default: return false;
  }
}

// ------------------------------------------------- allocation-free variant ---
// Some callers cannot let a library allocate device memory: an application
// whose device memory is all handed out by its own allocator (a framework's
// caching pool sized to the whole budget), a latency-critical loop where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable,
// or a process running under a fixed device-memory reservation.  For them,
// ext_sweep_so2_noalloc keeps its only scratch -- the steering-weight table
// B[j][c] of the sweep -- in this file-scope device array.  Every GPU that
// loads the library holds these 16 KB until the process exits.
#define EXT_NOALLOC_MAX_ANGLES 128
#define EXT_NOALLOC_ROW 32   // 2K <= 32 channels per angle
static __device__ __align__(256) float g_noalloc_table[EXT_NOALLOC_MAX_ANGLES * EXT_NOALLOC_ROW];

namespace {
std::mutex g_noalloc_mutex;
float* g_noalloc_ptr[256] = {};   // device address of the table, per device ordinal

// The array's name is only a host-side stand-in in host code; its device
// address is looked up once per device, with that device current.
ext_status noalloc_table(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    ext_set_error("ext_sweep_so2_noalloc: no usable current device");
    return EXT_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_table);
    if (e != cudaSuccess || !p) {
      ext_set_error("ext_sweep_so2_noalloc: cudaGetSymbolAddress of the scratch table failed");
      return EXT_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return EXT_OK;
}

// Device memory of `dev` (the current device) or managed memory.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}
}  // namespace

extern "C" ext_status ext_sweep_so2_noalloc(const float* G, int64_t n_pix, int K, int n_angles, float* max_out,
                                            int32_t* argmax, void* stream) {
  if (n_pix < 0 || K < 1 || n_angles < 1) {
    ext_set_error("ext_sweep_so2_noalloc: need n_pix >= 0, K >= 1, n_angles >= 1");
    return EXT_ERR_INVALID_ARG;
  }
  if (K > EXT_NOALLOC_ROW / 2 || n_angles > EXT_NOALLOC_MAX_ANGLES) {
    ext_set_error("ext_sweep_so2_noalloc: K must be <= 16 and n_angles <= 128 (fixed scratch table)");
    return EXT_ERR_UNSUPPORTED;
  }
  if (n_pix == 0) return EXT_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    ext_set_error("ext_sweep_so2_noalloc: no usable current device");
    return EXT_ERR_CUDA;
  }
  if (!G || !max_out || !argmax || !on_device(G, dev) || !on_device(max_out, dev) || !on_device(argmax, dev)) {
    ext_set_error("ext_sweep_so2_noalloc: G, max_out and argmax must be device buffers of the current device");
    return EXT_ERR_INVALID_ARG;
  }
  // An error left by earlier, unrelated work on this thread would be read
  // below as this call's own: report it and leave it in place for its owner.
  cudaError_t prior = cudaPeekAtLastError();
  if (prior != cudaSuccess) {
    ext_set_error((std::string("ext_sweep_so2_noalloc: a CUDA error from earlier work is pending on this thread: ") +
                   cudaGetErrorString(prior)).c_str());
    return EXT_ERR_CUDA;
  }
  float* table = nullptr;
  ext_status s = noalloc_table(&table);
  if (s != EXT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int cp = (2 * K + 3) / 4 * 4;
  // the table is rewritten in full on every call (rows of cp floats, zero padded)
  launch_sweep_table(K, n_angles, cp, table, st);
  if (!sweep_fp32(G, n_pix, K, n_angles, table, cp, max_out, argmax, st)) {
    ext_set_error("ext_sweep_so2_noalloc: unsupported K");
    return EXT_ERR_UNSUPPORTED;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ext_set_error(cudaGetErrorString(e));
    return EXT_ERR_CUDA;
  }
  return EXT_OK;
}
