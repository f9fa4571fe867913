// Angular sweep on the 5th-generation tensor cores (tcgen05), split BF16.
//
// The sweep of Sec. 4.1's linear combination over J rotations is the dense
// contraction  S(p, j) = G_0(p) + sum_c A(p, c) B[j][c]  with A the 2K real
// component planes of each pixel and B the steering weights (2 cos, -2 sin).
// Each 128-pixel tile is one MMA of M = 128, N = J (padded to 16), and the
// FP32 operands are split into BF16 hi + lo parts,
//   A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi,
// by concatenating [A_hi | A_hi | A_lo] and [B_hi ; B_lo ; B_hi] along the
// contraction, with FP32 accumulation in tensor memory (TMEM).  The per-pixel
// max and first argmax over j are taken straight from TMEM.
//
// Shared-memory operands use the K-major layout without swizzle: 8 x 16-byte
// core matrices, adjacent along K at 128 B (LBO) and along M/N at
// KT/8 * 128 B (SBO).  One thread issues the MMAs; completion is signalled
// through an mbarrier; every wait is bounded in time and reports a timeout
// through the error word instead of hanging.
#include "internal.h"

#include <cuda_bf16.h>

namespace {

constexpr int TILE_M = 128;
constexpr int THREADS = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor cores
  return d;                 // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(addr), "r"(phase)
      : "memory");
  return done != 0;
}

// Waits for the mbarrier phase; gives up after `limit_ns` and reports it.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t phase, uint64_t limit_ns, int* err) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(addr, phase)) {
    if (global_ns() - t0 > limit_ns) {
      atomicExch(err, EXT_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

template <int NCOL>
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo_elem), b = __float2bfloat16_rn(hi_elem);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// KC: channels per split part (2K padded to 16); JP: angles padded to 16.
template <int KC, int JP>
__global__ void __launch_bounds__(THREADS, 4) k_sweep_tc(const float* __restrict__ G, long long P, int C2, int J,
                                                      const float* __restrict__ B, int cp, float* __restrict__ maxv,
                                                      int32_t* __restrict__ argmax, int* __restrict__ err,
                                                      unsigned long long limit_ns) {
  constexpr int KT = 3 * KC;            // concatenated contraction length
  constexpr int KB = KT / 8;            // core matrices along K
  constexpr int SBO = KB * 128;         // bytes between 8-row groups
  constexpr int A_BYTES = (TILE_M / 8) * SBO;
  constexpr int TCOLS = JP <= 32 ? 32 : (JP <= 64 ? 64 : (JP <= 128 ? 128 : 256));
  constexpr uint32_t IDESC = make_idesc(TILE_M, JP);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* As = smem;
  unsigned char* Bs = smem + A_BYTES;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  // B' = [B_hi ; B_lo ; B_hi] along the contraction, rows = angles j
  for (int q = tid; q < JP * KB; q += THREADS) {
    const int n = q / KB, kb = q % KB;
    const int part = (kb * 8) / KC;           // 0: hi, 1: lo, 2: hi
    const int c0 = kb * 8 - part * KC;
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float e[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = c0 + 2 * t + u;
        const float b = (n < J && c < C2) ? B[(size_t)n * cp + c] : 0.f;
        const float hi = __bfloat162float(__float2bfloat16_rn(b));
        e[u] = (part == 1) ? (b - hi) : hi;
      }
      w[t] = pack_bf16(e[0], e[1]);
    }
    *reinterpret_cast<uint4*>(Bs + (n / 8) * SBO + kb * 128 + (n % 8) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t mbar_addr = smem_u32(&mbar);
  const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
  uint32_t phase = 0;

  const long long ntiles = (P + TILE_M - 1) / TILE_M;
  // this thread's pixel row of the tile, prefetched one tile ahead
  float a[KC];
  float g0 = 0.f;
  auto load_tile = [&](long long t, float (&dst)[KC], float& g) {
    const long long p = t * TILE_M + tid;
    const bool live = t < ntiles && p < P;
#pragma unroll
    for (int c = 0; c < KC; ++c) dst[c] = (live && c < C2) ? __ldg(G + (size_t)(c + 1) * P + p) : 0.f;
    g = live ? __ldg(G + p) : 0.f;
  };
  load_tile(blockIdx.x, a, g0);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long p = tile * TILE_M + tid;
    const bool live = p < P;
    // A' row of this pixel: [A_hi | A_hi | A_lo]
    unsigned char* arow = As + (tid / 8) * SBO + (tid % 8) * 16;
#pragma unroll
    for (int kb = 0; kb < KC / 8; ++kb) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float x0 = a[kb * 8 + 2 * t], x1 = a[kb * 8 + 2 * t + 1];
        const float h0 = __bfloat162float(__float2bfloat16_rn(x0)), h1 = __bfloat162float(__float2bfloat16_rn(x1));
        hi[t] = pack_bf16(x0, x1);
        lo[t] = pack_bf16(x0 - h0, x1 - h1);
      }
      const uint4 vh = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(arow + kb * 128) = vh;
      *reinterpret_cast<uint4*>(arow + (kb + KC / 8) * 128) = vh;
      *reinterpret_cast<uint4*>(arow + (kb + 2 * KC / 8) * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    const float g0_cur = g0;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int s = 0; s < KT / 16; ++s) {
        const uint64_t ad = make_desc(a_base + s * 256, 128, SBO);
        const uint64_t bd = make_desc(b_base + s * 256, 128, SBO);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar_addr)
                   : "memory");
    }
    // the next tile's loads are in flight while the MMA and the epilogue run
    load_tile(tile + gridDim.x, a, g0);
    if (!mbar_wait_bounded(mbar_addr, phase, limit_ns, err)) abort_flag = 1;
    phase ^= 1u;
    __syncthreads();
    if (abort_flag) break;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // epilogue: this thread owns TMEM lane `tid` (warp w reads lanes 32w..32w+31)
    float best = -3.402823466e38f;
    int bj = 0;
#pragma unroll
    for (int c0 = 0; c0 < JP; c0 += 32) {
      float v[32];
      tmem_ld32<32>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int j = c0 + i;
        if (j < J && (j == 0 || v[i] > best)) {
          best = v[i];
          bj = j;
        }
      }
    }
    if (live) {
      maxv[p] = g0_cur + best;
      argmax[p] = bj;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
  }
}

template <int KC, int JP>
bool launch_tc(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv, int32_t* argmax,
               int* err, int sms, cudaStream_t st) {
  constexpr int KB = 3 * KC / 8;
  constexpr int SBO = KB * 128;
  constexpr int bytes = (TILE_M / 8) * SBO + (JP / 8) * SBO;
  // at most 512 / TCOLS blocks may share an SM's tensor memory (and at most 6):
  // request enough shared memory that no more fit
  constexpr int TCOLS = JP <= 32 ? 32 : (JP <= 64 ? 64 : (JP <= 128 ? 128 : 256));
  constexpr int per_sm = (512 / TCOLS) < 6 ? (512 / TCOLS) : 6;
  constexpr int floor_bytes = (220 * 1024) / per_sm;
  constexpr int request = bytes < floor_bytes ? floor_bytes : bytes;
  static const bool once =
      (cudaFuncSetAttribute(k_sweep_tc<KC, JP>, cudaFuncAttributeMaxDynamicSharedMemorySize, request), true);
  (void)once;
  const long long ntiles = (P + TILE_M - 1) / TILE_M;
  long long grid = (long long)sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  k_sweep_tc<KC, JP><<<(unsigned)grid, THREADS, request, st>>>(G, P, 2 * K, J, B, cp, maxv, argmax, err,
                                                              1000000000ull);
  return true;
}

template <int KC>
bool dispatch_j(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv, int32_t* argmax,
                int* err, int sms, cudaStream_t st) {
  const int jp = (J + 15) / 16 * 16;
  switch (jp) {
    case 16: return launch_tc<KC, 16>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
    case 32: return launch_tc<KC, 32>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
    case 48: return launch_tc<KC, 48>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
    case 64: return launch_tc<KC, 64>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
    case 80: return launch_tc<KC, 80>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
    case 96: return launch_tc<KC, 96>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
    case 112: return launch_tc<KC, 112>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
    case 128: return launch_tc<KC, 128>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
    default: return false;
  }
}

}  // namespace

bool sweep_bf16x3(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv, int32_t* argmax,
                  int* err, int sms, cudaStream_t st) {
  if (K < 1 || K > 16 || J < 1 || J > 128) return false;
  if (2 * K <= 16) return dispatch_j<16>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
  return dispatch_j<32>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
}
