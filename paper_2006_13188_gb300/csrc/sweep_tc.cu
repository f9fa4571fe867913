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
#include "tc_common.cuh"

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
// The budget comes from the plan's status block (byte 8) when it sets one.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t phase, uint64_t limit_ns, int* err) {
  if (mbar_try_wait(addr, phase)) return true;
  if (err) {
    const uint64_t b = *reinterpret_cast<const volatile unsigned long long*>(err + 2);
    if (b) limit_ns = b;
  }
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
  if (!ext_smem_optin((const void*)k_sweep_tc<KC, JP>, request)) return false;
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

// ---------------------------------------------------------------------------
// Pipelined variant.  The component planes of a 128-pixel tile (G_0 and the
// 2K channels: a [2K+1][128] FP32 box) arrive by one tensor copy into a ring
// of NST stages, issued NST tiles ahead; each thread splits its pixel's
// channels into BF16 hi / lo blocks; the three products A_hi B_hi, A_hi B_lo,
// A_lo B_hi accumulate into one of two TMEM accumulators, so the MMA of tile
// i runs while the max/argmax of tile i-1 is read from the other.  Waits are
// bounded; on expiry err = EXT_ERR_TIMEOUT and the block stops after its
// copies in flight have landed (bounded as well).
template <int KC, int JP, int NST>
struct Tc2Cfg {
  static constexpr int C1 = 2 * KC + 1;                 // box rows: G_0 + up to 2 KC channels (padded)
  static constexpr int STAGE_BYTES = 128 * 4 * 33;      // room for the largest box (K = 16: 33 rows)
  static constexpr int A_BYTES = TILE_M * KC * 2;       // one BF16 block of a tile
  static constexpr int B_BYTES = JP * KC * 2;
  static constexpr int SBO = (KC / 8) * 128;
  static constexpr int OFF_A = NST * STAGE_BYTES;       // A_hi[2], A_lo[2]
  static constexpr int OFF_B = OFF_A + 4 * A_BYTES;     // B_hi, B_lo
  static constexpr int SMEM = OFF_B + 2 * B_BYTES + 1024;
  static constexpr int TCOLS = 2 * JP <= 32 ? 32 : (2 * JP <= 64 ? 64 : (2 * JP <= 128 ? 128 : 256));
};

template <int KC, int JP, int NST>
__global__ void __launch_bounds__(THREADS, 1) k_sweep_tc2(const __grid_constant__ CUtensorMap tmG, long long P, int C2,
                                                         int J, const float* __restrict__ B, int cp,
                                                         float* __restrict__ maxv, int32_t* __restrict__ argmax,
                                                         int* __restrict__ err, unsigned long long limit_ns) {
  using CF = Tc2Cfg<KC, JP, NST>;
  constexpr uint32_t IDESC = make_idesc(TILE_M, JP);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t full[NST];
  __shared__ __align__(8) uint64_t mma_done[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* Bhi = smem + CF::OFF_B;
  unsigned char* Blo = Bhi + CF::B_BYTES;
  // B split into hi / lo blocks, rows = angles, K-major core matrices
  for (int q = tid; q < JP * (KC / 8); q += THREADS) {
    const int n = q / (KC / 8), kb = q % (KC / 8);
    uint32_t wh[4], wl[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float eh[2], el[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = kb * 8 + 2 * t + u;
        const float b = (n < J && c < C2) ? B[(size_t)n * cp + c] : 0.f;
        eh[u] = __bfloat162float(__float2bfloat16_rn(b));
        el[u] = b - eh[u];
      }
      wh[t] = pack_bf16(eh[0], eh[1]);
      wl[t] = pack_bf16(el[0], el[1]);
    }
    const int off = (n / 8) * CF::SBO + kb * 128 + (n % 8) * 16;
    *reinterpret_cast<uint4*>(Bhi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4*>(Blo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < NST; ++s) tc::mbar_init(tc::smem_u32(&full[s]), 1);
    tc::mbar_init(tc::smem_u32(&mma_done[0]), 1);
    tc::mbar_init(tc::smem_u32(&mma_done[1]), 1);
  }
  if (warp == 0) tc::tmem_alloc<CF::TCOLS>(tc::smem_u32(&tmem_slot));
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const long long ntiles = (P + TILE_M - 1) / TILE_M;
  const int rows = C2 + 1;
  const uint32_t stage_tx = (uint32_t)rows * TILE_M * 4u;
  auto tile_of = [&](long long li) { return (long long)blockIdx.x + li * gridDim.x; };
  auto issue = [&](long long li) {   // thread 0
    const int s = (int)(li % NST);
    tc::fence_proxy_async();
    tc::mbar_expect_tx(tc::smem_u32(&full[s]), stage_tx);
    tc::tma_load_2d(tc::smem_u32(smem + s * CF::STAGE_BYTES), &tmG, (int)(tile_of(li) * TILE_M), 0,
                    tc::smem_u32(&full[s]));
  };
  long long nloc = 0;   // tiles of this block
  if ((long long)blockIdx.x < ntiles) nloc = (ntiles - 1 - blockIdx.x) / gridDim.x + 1;
  if (tid == 0)
    for (long long li = 0; li < NST && li < nloc; ++li) issue(li);
  long long issued = nloc < NST ? nloc : NST;
  float g0_prev = 0.f;
  long long li = 0;
  // max/argmax of tile li_e (accumulator li_e & 1) to global memory
  auto epilogue = [&](long long li_e, float g0) {
    const int b = (int)(li_e & 1);
    if (!tc::mbar_wait_bounded(tc::smem_u32(&mma_done[b]), (uint32_t)((li_e >> 1) & 1), limit_ns, err,
                               EXT_ERR_TIMEOUT))
      abort_flag = 1;
    tc::fence_after();
    float best = 0.f;
    int bj = 0;
    const bool full = (J == JP);   // no padded angle columns to skip
#pragma unroll
    for (int c0 = 0; c0 < JP; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * JP + c0), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int j = c0 + i;
        if (j == 0) {
          best = v[i];
        } else if ((full || j < J) && v[i] > best) {
          best = v[i];
          bj = j;
        }
      }
    }
    const long long p = tile_of(li_e) * TILE_M + tid;
    if (p < P && !abort_flag) {
      maxv[p] = g0 + best;
      argmax[p] = bj;
    }
    tc::fence_before();
  };
  for (; li < nloc; ++li) {
    const int s = (int)(li % NST);
    const int b = (int)(li & 1);
    if (!tc::mbar_wait_bounded(tc::smem_u32(&full[s]), (uint32_t)((li / NST) & 1), limit_ns, err, EXT_ERR_TIMEOUT))
      abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    // this thread's pixel: channels from the stage, split into the A blocks of accumulator b
    const float* st = reinterpret_cast<const float*>(smem + s * CF::STAGE_BYTES);
    const float g0 = st[tid];
    unsigned char* Ahi = smem + CF::OFF_A + b * CF::A_BYTES;
    unsigned char* Alo = smem + CF::OFF_A + (2 + b) * CF::A_BYTES;
    const int rowoff = (tid / 8) * CF::SBO + (tid % 8) * 16;
#pragma unroll
    for (int kb = 0; kb < KC / 8; ++kb) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = kb * 8 + 2 * t;
        const float x0 = c < C2 ? st[(c + 1) * TILE_M + tid] : 0.f;
        const float x1 = c + 1 < C2 ? st[(c + 2) * TILE_M + tid] : 0.f;
        // packed conversions: one instruction rounds both values
        const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - __low2float(hb), x1 - __high2float(hb));
        hi[t] = *reinterpret_cast<const uint32_t*>(&hb);
        lo[t] = *reinterpret_cast<const uint32_t*>(&lb);
      }
      *reinterpret_cast<uint4*>(Ahi + rowoff + kb * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(Alo + rowoff + kb * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      if (issued < nloc) issue(issued);   // the stage just consumed takes tile `issued` (= li + NST)
      const uint32_t d = tmem + (uint32_t)(b * JP);
      const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll
      for (int k = 0; k < KC / 16; ++k) {
        tc::mma_bf16(d, tc::make_desc(ah + k * 256, 128, CF::SBO), tc::make_desc(bh + k * 256, 128, CF::SBO), IDESC,
                     k > 0 ? 1u : 0u);
        tc::mma_bf16(d, tc::make_desc(ah + k * 256, 128, CF::SBO), tc::make_desc(bl + k * 256, 128, CF::SBO), IDESC,
                     1u);
        tc::mma_bf16(d, tc::make_desc(al + k * 256, 128, CF::SBO), tc::make_desc(bh + k * 256, 128, CF::SBO), IDESC,
                     1u);
      }
      tc::mma_commit(tc::smem_u32(&mma_done[b]));
    }
    if (issued < nloc) ++issued;
    // the previous tile's max/argmax while this tile's MMAs run
    if (li > 0) epilogue(li - 1, g0_prev);
    g0_prev = g0;
  }
  if (!abort_flag && nloc > 0) epilogue(nloc - 1, g0_prev);
  // copies and MMAs still in flight after an abort: let them finish (bounded) before the block exits
  if (abort_flag && tid == 0) {
    for (long long q = li; q < issued; ++q)
      tc::mbar_wait_bounded(tc::smem_u32(&full[q % NST]), (uint32_t)((q / NST) & 1), limit_ns, err, EXT_ERR_TIMEOUT);
    if (li > 0)
      tc::mbar_wait_bounded(tc::smem_u32(&mma_done[(li - 1) & 1]), (uint32_t)(((li - 1) >> 1) & 1), limit_ns, err,
                            EXT_ERR_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc<CF::TCOLS>(tmem);
  }
}

template <int KC, int JP>
bool launch_tc2(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv, int32_t* argmax,
                int* err, int sms, cudaStream_t st) {
  constexpr int NST = 2;
  using CF = Tc2Cfg<KC, JP, NST>;
  CUtensorMap tm;
  // G as rows of P floats: plane 0 = G_0, planes 1..2K the channels; one box = 2K+1 planes x 128 pixels
  if (P % 4 != 0 || !make_tmap_2d_f32(G, (unsigned long long)P, (unsigned long long)(2 * K + 1),
                                      (unsigned long long)P * 4, TILE_M, (unsigned)(2 * K + 1), &tm))
    return false;
  if (!ext_smem_optin((const void*)k_sweep_tc2<KC, JP, NST>, CF::SMEM)) return false;
  const long long ntiles = (P + TILE_M - 1) / TILE_M;
  const int per_sm = (227 * 1024) / (CF::SMEM + 1024) < 1 ? 1 : (227 * 1024) / (CF::SMEM + 1024);
  long long grid = (long long)sms * (per_sm < 512 / CF::TCOLS ? per_sm : 512 / CF::TCOLS);
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  k_sweep_tc2<KC, JP, NST><<<(unsigned)grid, THREADS, CF::SMEM, st>>>(tm, P, 2 * K, J, B, cp, maxv, argmax, err,
                                                                      1000000000ull);
  return true;
}

}  // namespace

bool sweep_bf16x3(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv, int32_t* argmax,
                  int* err, int sms, cudaStream_t st) {
  if (K < 1 || K > 16 || J < 1 || J > 128) return false;
  // the pipelined tensor-copy variant for the common shapes; the register-prefetch one otherwise
  if (K > 8 && (J + 15) / 16 * 16 == 64 && launch_tc2<32, 64>(G, P, K, J, B, cp, maxv, argmax, err, sms, st))
    return true;
  if (2 * K <= 16) return dispatch_j<16>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
  return dispatch_j<32>(G, P, K, J, B, cp, maxv, argmax, err, sms, st);
}
