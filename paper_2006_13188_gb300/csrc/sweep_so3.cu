// Sweep over a grid of rotations for SO(3) (Sec. 9 "Linear Combination" at
// every grid rotation), with per-voxel max and first argmax:
//   S(p, j) = sum_c A(p, c) B[j][c],
// A = the real channels of the component correlations G_l^{ab} (planar, one
// plane per channel), B[j] = the steering row of rotation j (C^l_00 for a
// self channel, 2 Re C^l_ab and 2 Im C^l_ab for a pair of channels).
#include "internal.h"
#include "tc_common.cuh"

#include <cfloat>

// ------------------------------------------------------------ plain FP32 ---
// Block: 64 voxels x 64 rotations per tile, 256 threads with 4 x 4 outputs
// each, channels streamed through shared memory 32 at a time; the running
// per-voxel max over rotation tiles stays in shared memory.
namespace {
constexpr int FM = 64, FN = 64, FK = 32;
}

__global__ void __launch_bounds__(256) k_sweep_so3_fp32(const float* __restrict__ G, long long P, int C,
                                                        const float* __restrict__ B, int cpad, int J,
                                                        float* __restrict__ maxv, int32_t* __restrict__ argmax) {
  __shared__ float As[FK][FM];
  __shared__ float Bs[FK][FN + 1];
  __shared__ float best_v[FM][16];
  __shared__ int best_j[FM][16];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;   // tx: rotation group, ty: voxel group
  const long long p0 = (long long)blockIdx.x * FM;
  float vbest[4];
  int jbest[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) { vbest[i] = -FLT_MAX; jbest[i] = 0; }
  for (int n0 = 0; n0 < J; n0 += FN) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][k] = 0.f;
    for (int c0 = 0; c0 < C; c0 += FK) {
      for (int e = tid; e < FK * FM; e += 256) {
        const int c = e / FM, m = e % FM;
        const long long p = p0 + m;
        As[c][m] = (c0 + c < C && p < P) ? __ldg(G + (size_t)(c0 + c) * P + p) : 0.f;
      }
      for (int e = tid; e < FK * FN; e += 256) {
        const int n = e / FK, c = e % FK;
        Bs[c][n] = (n0 + n < J && c0 + c < cpad) ? __ldg(B + (size_t)(n0 + n) * cpad + c0 + c) : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int c = 0; c < FK; ++c) {
        float a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[c][ty * 4 + i];
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = Bs[c][tx * 4 + k];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[i][k] = fmaf(a[i], b[k], acc[i][k]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = n0 + tx * 4 + k;
        if (j < J && acc[i][k] > vbest[i]) { vbest[i] = acc[i][k]; jbest[i] = j; }
      }
  }
  // reduce over the 16 rotation groups; ties keep the smallest j
#pragma unroll
  for (int i = 0; i < 4; ++i) { best_v[ty * 4 + i][tx] = vbest[i]; best_j[ty * 4 + i][tx] = jbest[i]; }
  __syncthreads();
  if (tid < FM) {
    float v = -FLT_MAX;
    int jj = 0;
    bool first = true;
    for (int g = 0; g < 16; ++g) {
      const float x = best_v[tid][g];
      const int xj = best_j[tid][g];
      if (first || x > v || (x == v && xj < jj)) { v = x; jj = xj; first = false; }
    }
    const long long p = p0 + tid;
    if (p < P) { maxv[p] = v; argmax[p] = jj; }
  }
}

void sweep_so3_fp32(const float* G, long long P, int C, const float* B, int cpad, int J, float* maxv,
                    int32_t* argmax, cudaStream_t st) {
  const long long blocks = (P + FM - 1) / FM;
  k_sweep_so3_fp32<<<(unsigned)blocks, 256, 0, st>>>(G, P, C, B, cpad, J, maxv, argmax);
}

// ------------------------------------------------------------ tcgen05 -----
// M = 128 voxels per tile (one TMEM lane per voxel), N = 256 rotations per
// N tile (256 TMEM columns), K streamed in chunks of 32 channels; each chunk
// is split [A_hi | A_hi | A_lo] x [B_hi ; B_lo ; B_hi] (96 bf16) and issued as
// six K = 16 MMAs.  B' is prepared once per rotation set in the exact
// shared-memory image of each (N tile, K chunk) block.
namespace {
constexpr int TM = 128, TN = 256, TKC = 32, TKT = 3 * TKC, TKB = TKT / 8;
constexpr int T_SBO = TKB * 128;                   // 1536 B between 8-row groups
constexpr int TA_BYTES = (TM / 8) * T_SBO;          // 24 KB
constexpr int TB_BYTES = (TN / 8) * T_SBO;          // 48 KB
}

// B' blocks: [n_tile][k_chunk][TB_BYTES] in core-matrix order from B[j][cpad]
__global__ void k_so3_btc(const float* __restrict__ B, int cpad, int J, int ntn, int nkc, unsigned char* __restrict__ Bt) {
  const long long total = (long long)ntn * nkc * TN * TKB;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const int kb = (int)(q % TKB);
    const int n = (int)((q / TKB) % TN);
    const int kc = (int)((q / ((long long)TKB * TN)) % nkc);
    const int nt = (int)(q / ((long long)TKB * TN * nkc));
    const int part = kb / (TKC / 8);   // 0 hi, 1 lo, 2 hi
    const int c0 = kc * TKC + (kb % (TKC / 8)) * 8;
    const int j = nt * TN + n;
    uint32_t w[4];
    for (int t = 0; t < 4; ++t) {
      float e[2];
      for (int u = 0; u < 2; ++u) {
        const int c = c0 + 2 * t + u;
        const float b = (j < J && c < cpad) ? B[(size_t)j * cpad + c] : 0.f;
        const float hi = tc::bf16_round(b);
        e[u] = part == 1 ? b - hi : hi;
      }
      w[t] = tc::pack_bf16(e[0], e[1]);
    }
    unsigned char* blk = Bt + ((size_t)nt * nkc + kc) * TB_BYTES;
    *reinterpret_cast<uint4*>(blk + (n / 8) * T_SBO + kb * 128 + (n % 8) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// With gridDim.y > 1 the rotation tiles are split over blockIdx.y and every
// block folds its (max, first argmax) into keys[p] (ordered score bits above
// the complemented index: atomicMax keeps the larger score, then the smaller
// index); k_sweep_keys_finish decodes them.
__device__ __forceinline__ unsigned long long sweep_key(float v, int j) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return ((unsigned long long)o << 32) | (uint32_t)(0xFFFFFFFFu - (uint32_t)j);
}

__global__ void __launch_bounds__(128) k_sweep_so3_tc(const float* __restrict__ G, long long P, int C, int nkc,
                                                      const unsigned char* __restrict__ Bt, int ntn, int J,
                                                      float* __restrict__ maxv, int32_t* __restrict__ argmax,
                                                      unsigned long long* __restrict__ keys,
                                                      int* __restrict__ err, unsigned long long limit_ns) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* As = smem;
  unsigned char* Bs = smem + TA_BYTES;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    abort_flag = 0;
    tc::mbar_init(tc::smem_u32(&mbar), 1);
  }
  if (warp == 0) tc::tmem_alloc<TN>(tc::smem_u32(&tmem_slot));
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot, mbar_addr = tc::smem_u32(&mbar);
  const uint32_t a_base = tc::smem_u32(As), b_base = tc::smem_u32(Bs);
  constexpr uint32_t IDESC = tc::make_idesc(TM, TN);
  uint32_t phase = 0;
  const long long ntm = (P + TM - 1) / TM;
  const int nsplit = gridDim.y;
  const int nt0 = (int)((long long)ntn * blockIdx.y / nsplit), nt1 = (int)((long long)ntn * (blockIdx.y + 1) / nsplit);
  for (long long mt = blockIdx.x; mt < ntm && !abort_flag; mt += gridDim.x) {
    const long long p = mt * TM + tid;
    const bool live = p < P;
    float best = -FLT_MAX;
    int bj = nt0 * TN;
    for (int nt = nt0; nt < nt1 && !abort_flag; ++nt) {
      for (int kc = 0; kc < nkc; ++kc) {
        // B' block: straight copy of its shared-memory image
        const uint4* src = reinterpret_cast<const uint4*>(Bt + ((size_t)nt * nkc + kc) * TB_BYTES);
        uint4* dst = reinterpret_cast<uint4*>(Bs);
        for (int q = tid; q < TB_BYTES / 16; q += 128) dst[q] = __ldg(src + q);
        // A' row of this voxel for channels kc*32 .. kc*32+31
        float a[TKC];
#pragma unroll
        for (int c = 0; c < TKC; ++c) {
          const int ch = kc * TKC + c;
          a[c] = (live && ch < C) ? __ldg(G + (size_t)ch * P + p) : 0.f;
        }
        unsigned char* arow = As + (tid / 8) * T_SBO + (tid % 8) * 16;
#pragma unroll
        for (int kb = 0; kb < TKC / 8; ++kb) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float x0 = a[kb * 8 + 2 * t], x1 = a[kb * 8 + 2 * t + 1];
            hi[t] = tc::pack_bf16(x0, x1);
            lo[t] = tc::pack_bf16(x0 - tc::bf16_round(x0), x1 - tc::bf16_round(x1));
          }
          const uint4 vh = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(arow + kb * 128) = vh;
          *reinterpret_cast<uint4*>(arow + (kb + TKC / 8) * 128) = vh;
          *reinterpret_cast<uint4*>(arow + (kb + 2 * TKC / 8) * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after();
#pragma unroll
          for (int s = 0; s < TKT / 16; ++s)
            tc::mma_bf16(tmem, tc::make_desc(a_base + s * 256, 128, T_SBO), tc::make_desc(b_base + s * 256, 128, T_SBO),
                         IDESC, (kc > 0 || s > 0) ? 1u : 0u);
          tc::mma_commit(mbar_addr);
        }
        if (!tc::mbar_wait_bounded(mbar_addr, phase, limit_ns, err, EXT_ERR_TIMEOUT)) abort_flag = 1;
        phase ^= 1u;
        __syncthreads();
        if (abort_flag) break;
      }
      if (abort_flag) break;
      tc::fence_after();
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int j = nt * TN + c0 + i;
          if (j < J && (v[i] > best || (j == nt0 * TN))) { best = v[i]; bj = j; }
        }
      }
      tc::fence_before();
      __syncthreads();
    }
    if (live && !abort_flag) {
      if (nsplit == 1) {
        maxv[p] = best;
        argmax[p] = bj;
      } else {
        atomicMax(keys + p, sweep_key(best, bj));
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc<TN>(tmem);
  }
}

size_t so3_btc_bytes(int J, int cpad) {
  const int ntn = (J + TN - 1) / TN, nkc = (cpad + TKC - 1) / TKC;
  return (size_t)ntn * nkc * TB_BYTES;
}

void so3_build_btc(const float* B, int cpad, int J, unsigned char* Bt, cudaStream_t st) {
  const int ntn = (J + TN - 1) / TN, nkc = (cpad + TKC - 1) / TKC;
  k_so3_btc<<<1024, 256, 0, st>>>(B, cpad, J, ntn, nkc, Bt);
}

__global__ void k_sweep_keys_finish(const unsigned long long* __restrict__ keys, long long P, float* __restrict__ maxv,
                                    int32_t* __restrict__ argmax) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[p];
    const uint32_t o = (uint32_t)(k >> 32);
    const uint32_t b = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    maxv[p] = __uint_as_float(b);
    argmax[p] = (int32_t)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu));
  }
}

int sweep_so3_tc_split(long long P, int J, int sms) {
  const int ntn = (J + TN - 1) / TN;
  const long long ntm = (P + TM - 1) / TM;
  long long s = (2LL * sms) / (ntm > 0 ? ntm : 1);
  if (s < 1) s = 1;
  if (s > ntn) s = ntn;
  return (int)s;
}

void sweep_so3_tc(const float* G, long long P, int C, int cpad, const unsigned char* Bt, int J, float* maxv,
                  int32_t* argmax, unsigned long long* keys, int* err, int sms, cudaStream_t st) {
  const int ntn = (J + TN - 1) / TN, nkc = (cpad + TKC - 1) / TKC;
  // two blocks per SM share the 512 TMEM columns: request shared memory accordingly
  constexpr int request = 100 * 1024;
  ext_smem_optin((const void*)k_sweep_so3_tc, request);
  const long long ntm = (P + TM - 1) / TM;
  const int nsplit = keys ? sweep_so3_tc_split(P, J, sms) : 1;
  long long grid = ((long long)sms * 2 + nsplit - 1) / nsplit;
  if (grid > ntm) grid = ntm;
  if (nsplit > 1) cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * P, st);
  k_sweep_so3_tc<<<dim3((unsigned)grid, nsplit), 128, request, st>>>(G, P, C, nkc, Bt, ntn, J, maxv, argmax, keys,
                                                                     err, 2000000000ull);
  if (nsplit > 1) {
    long long b = (P + 255) / 256;
    if (b > 4096) b = 4096;
    k_sweep_keys_finish<<<(unsigned)b, 256, 0, st>>>(keys, P, maxv, argmax);
  }
}

// ------------------------------------------- warp-specialised tcgen05 sweep ---
// The split-BF16 GEMM S = A_hi B_hi + A_hi B_lo + A_lo B_hi over pre-split
// operands: A' (the voxel channels) and B' (the steering rows) are written
// once per call / rotation set in the exact shared-memory image of each
// (tile, 32-channel chunk) block, hi and lo halves only (the third product
// reuses A_hi and B_hi through the descriptors).  Per block (one per SM):
//   warp 0, one thread: bulk copies of the A' and B' blocks of each chunk into
//     a ring of NS stages (48 KB each), waiting for the stage to be free;
//   warp 1, one thread: six M128 N256 K16 MMAs per chunk into one of two TMEM
//     accumulators (512 columns), freeing the stage and, after the last chunk
//     of a tile, signalling the accumulator full;
//   warps 2-5: max / first argmax of each accumulator over its 256 rotations,
//     one voxel per thread (TMEM lane), while the MMAs fill the other one.
// Work: voxel tiles strided over the blocks, for each all rotation tiles of
// the block's rotation range (gridDim.y > 1 splits the rotation tiles and
// folds results through keys as k_sweep_so3_tc does).  Every wait is bounded;
// on expiry a role records EXT_ERR_TIMEOUT, stops, waits (bounded) for its own
// copies or MMAs in flight, and the block frees its tensor memory.
namespace ws {
constexpr int M = 128, N = 256, KC = 32;
constexpr int SBO = (KC / 8) * 128;         // 512 B between 8-row groups
constexpr int A_HALF = (M / 8) * SBO;       // 8 KB: A_hi or A_lo of one chunk
constexpr int B_HALF = (N / 8) * SBO;       // 16 KB: B_hi or B_lo of one chunk
constexpr int A_BYTES = 2 * A_HALF, B_BYTES = 2 * B_HALF;
constexpr int STAGE = A_BYTES + B_BYTES;    // 48 KB
constexpr int NS = 4;
constexpr int SMEM = NS * STAGE + 1024;     // + room to align the ring to 1 KB
constexpr int THREADS = 192;
constexpr int THREADS_GRID = 320;          // the grid variant: eight epilogue warps, two per lane quarter
}  // namespace ws

// A' [mt][kc]: hi block then lo block, 128 voxel rows x 32 channels each in
// core-matrix order; voxels beyond P and channels beyond C are zero.
__global__ void k_so3_a_split(const float* __restrict__ G, long long P, int C, int nkc, unsigned char* __restrict__ Ab) {
  using namespace ws;
  const long long rows = (P + M - 1) / M * M;
  const long long total = rows * nkc * (KC / 8);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const long long p = q % rows;           // voxel fastest: coalesced plane reads
    const int g = (int)(q / rows);          // 8-channel group
    const int kc = g / (KC / 8), kb = g % (KC / 8);
    const long long mt = p / M;
    const int r = (int)(p % M);
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float x[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int ch = g * 8 + 2 * t + u;
        x[u] = (p < P && ch < C) ? __ldg(G + (size_t)ch * P + p) : 0.f;
      }
      hi[t] = tc::pack_bf16(x[0], x[1]);
      lo[t] = tc::pack_bf16(x[0] - tc::bf16_round(x[0]), x[1] - tc::bf16_round(x[1]));
    }
    unsigned char* blk = Ab + ((size_t)mt * nkc + kc) * A_BYTES;
    const int off = (r / 8) * SBO + kb * 128 + (r % 8) * 16;
    *reinterpret_cast<uint4*>(blk + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(blk + A_HALF + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// B' [nt][kc]: hi block then lo block, 256 rotation rows x 32 channels each.
__global__ void k_so3_b_split(const float* __restrict__ B, int cpad, int J, int ntn, int nkc,
                              unsigned char* __restrict__ Bb) {
  using namespace ws;
  const long long total = (long long)ntn * nkc * N * (KC / 8);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const int kb = (int)(q % (KC / 8));
    const int n = (int)((q / (KC / 8)) % N);
    const int kc = (int)((q / ((long long)(KC / 8) * N)) % nkc);
    const int nt = (int)(q / ((long long)(KC / 8) * N * nkc));
    const int j = nt * N + n;
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float x[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = kc * KC + kb * 8 + 2 * t + u;
        x[u] = (j < J && c < cpad) ? B[(size_t)j * cpad + c] : 0.f;
      }
      hi[t] = tc::pack_bf16(x[0], x[1]);
      lo[t] = tc::pack_bf16(x[0] - tc::bf16_round(x[0]), x[1] - tc::bf16_round(x[1]));
    }
    unsigned char* blk = Bb + ((size_t)nt * nkc + kc) * B_BYTES;
    const int off = (n / 8) * SBO + kb * 128 + (n % 8) * 16;
    *reinterpret_cast<uint4*>(blk + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(blk + B_HALF + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// GRID: the B' rows are 16 per direction (in-plane harmonics H_0, Re/Im H_a of
// k_so3_grid_rows) and the epilogue forms S(psi_t) = H_0 + sum_a (2 cos(a psi_t)
// Re H_a - 2 sin(a psi_t) Im H_a) for t < n_psi, rotation index dir * n_psi + t;
// J is then the number of directions.
template <bool GRID>
__global__ void __launch_bounds__(GRID ? ws::THREADS_GRID : ws::THREADS, 1)
    k_sweep_so3_ws(const unsigned char* __restrict__ Ab, const unsigned char* __restrict__ Bb, long long P, int nkc,
                   int ntn, int J, int n_psi, float* __restrict__ maxv, int32_t* __restrict__ argmax,
                   unsigned long long* __restrict__ keys, int* __restrict__ err, unsigned long long limit_ns) {
  using namespace ws;
  extern __shared__ __align__(1024) unsigned char ws_smem[];
  __shared__ __align__(8) uint64_t full[NS], empty[NS], accf[2], acce[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ __align__(16) float psi_tab[GRID ? 64 * 12 : 4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = (tc::smem_u32(ws_smem) + 1023u) & ~1023u;
  if constexpr (GRID) {   // [q][t]: 2 cos(a psi_t) (q = 2a - 2), -2 sin(a psi_t) (q = 2a - 1), a = 1..6, t < n_psi
    for (int e = tid; e < 64 * 12; e += (GRID ? THREADS_GRID : THREADS)) {
      const int q = e / 64, t = e % 64, a = q / 2 + 1;
      double sv, cv;
      sincospi(2.0 * a * t / (double)(n_psi > 0 ? n_psi : 1), &sv, &cv);
      psi_tab[e] = t < n_psi ? (float)((q & 1) ? -2.0 * sv : 2.0 * cv) : 0.f;
    }
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(tc::smem_u32(&full[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(tc::smem_u32(&accf[b]), 1);
      tc::mbar_init(tc::smem_u32(&acce[b]), GRID ? 8 : 4);
    }
  }
  if (warp == 1) tc::tmem_alloc<512>(tc::smem_u32(&tmem_slot));
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const long long ntm = (P + M - 1) / M;
  const int nsplit = gridDim.y;
  const int nt0 = (int)((long long)ntn * blockIdx.y / nsplit), nt1 = (int)((long long)ntn * (blockIdx.y + 1) / nsplit);

  if (warp == 0) {
    if (lane == 0) {   // ---- producer: bulk copies into the ring
      long long it = 0;
      for (long long mt = blockIdx.x; mt < ntm && !abort_flag; mt += gridDim.x)
        for (int nt = nt0; nt < nt1 && !abort_flag; ++nt)
          for (int kc = 0; kc < nkc; ++kc) {
            const int s = (int)(it % NS);
            const uint32_t par = (uint32_t)(((it / NS) & 1) ^ 1);
            if (!tc::mbar_wait_bounded(tc::smem_u32(&empty[s]), par, limit_ns, err, EXT_ERR_TIMEOUT)) {
              abort_flag = 1;
              break;
            }
            const uint32_t fb = tc::smem_u32(&full[s]), dst = base + (uint32_t)s * STAGE;
            tc::mbar_expect_tx(fb, STAGE);
            tc::bulk_load(dst, Ab + ((size_t)mt * nkc + kc) * A_BYTES, A_BYTES, fb);
            tc::bulk_load(dst + A_BYTES, Bb + ((size_t)nt * nkc + kc) * B_BYTES, B_BYTES, fb);
            ++it;
          }
      // the copies of the last chunks issued must have landed before the block exits
      for (long long q = it > NS ? it - NS : 0; q < it; ++q)
        tc::mbar_wait_bounded(tc::smem_u32(&full[q % NS]), (uint32_t)((q / NS) & 1), limit_ns, err, EXT_ERR_TIMEOUT);
    }
  } else if (warp == 1) {
    if (lane == 0) {   // ---- MMA issue
      constexpr uint32_t IDESC = tc::make_idesc(M, N);
      long long it = 0;
      int t = 0;
      for (long long mt = blockIdx.x; mt < ntm && !abort_flag; mt += gridDim.x)
        for (int nt = nt0; nt < nt1 && !abort_flag; ++nt, ++t) {
          const int b = t & 1;
          if (!tc::mbar_wait_bounded(tc::smem_u32(&acce[b]), (uint32_t)(((t >> 1) & 1) ^ 1), limit_ns, err,
                                     EXT_ERR_TIMEOUT)) {
            abort_flag = 1;
            break;
          }
          tc::fence_after();
          const uint32_t d = tmem + (uint32_t)(b * N);
          for (int kc = 0; kc < nkc; ++kc) {
            const int s = (int)(it % NS);
            if (!tc::mbar_wait_bounded(tc::smem_u32(&full[s]), (uint32_t)((it / NS) & 1), limit_ns, err,
                                       EXT_ERR_TIMEOUT)) {
              abort_flag = 1;
              break;
            }
            tc::fence_after();
            const uint32_t a_hi = base + (uint32_t)s * STAGE, a_lo = a_hi + A_HALF;
            const uint32_t b_hi = a_hi + A_BYTES, b_lo = b_hi + B_HALF;
            // products in the order hi.hi, hi.lo, lo.hi, each over both K = 16 halves (the accumulation
            // order of k_sweep_so3_tc, so both kernels give identical sums)
            const uint32_t pa[3] = {a_hi, a_hi, a_lo}, pb[3] = {b_hi, b_lo, b_hi};
#pragma unroll
            for (int part = 0; part < 3; ++part)
#pragma unroll
              for (int k2 = 0; k2 < KC / 16; ++k2) {
                const uint32_t o = (uint32_t)k2 * 256;
                tc::mma_bf16(d, tc::make_desc(pa[part] + o, 128, SBO), tc::make_desc(pb[part] + o, 128, SBO), IDESC,
                             (kc > 0 || part > 0 || k2 > 0) ? 1u : 0u);
              }
            tc::mma_commit(tc::smem_u32(&empty[s]));
            ++it;
          }
          if (abort_flag) break;
          tc::mma_commit(tc::smem_u32(&accf[b]));
        }
      // every MMA issued must be complete before the tensor memory is freed
      if (it > 0)
        tc::mbar_wait_bounded(tc::smem_u32(&empty[(it - 1) % NS]), (uint32_t)(((it - 1) / NS) & 1), limit_ns, err,
                              EXT_ERR_TIMEOUT);
    }
  } else {   // ---- epilogue: warps 2..5 (grid variant: 2..9), one voxel row per thread
    const int q4 = warp & 3;                 // the TMEM lane quarter this warp may read
    const int row = q4 * 32 + lane;
    // grid variant: the two warps of a lane quarter take half of each tile's columns each and fold
    // their results through keys (the larger score, then the smaller index)
    const int part = GRID ? (warp - 2) / 4 : 0;
    constexpr int C_SPAN = GRID ? N / 2 : N;
    // every branch below is taken by the whole warp (the tensor-memory loads are warp-wide)
    int t = 0;
    for (long long mt = blockIdx.x; mt < ntm; mt += gridDim.x) {
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      float best = -FLT_MAX;
      int bj = nt0 * N;
      bool first = true, stop = false;
      for (int nt = nt0; nt < nt1; ++nt, ++t) {
        const int b = t & 1;
        int ok = 1;
        if (lane == 0)
          ok = tc::mbar_wait_bounded(tc::smem_u32(&accf[b]), (uint32_t)((t >> 1) & 1), limit_ns, err, EXT_ERR_TIMEOUT)
                   ? 1 : 0;
        if (__any_sync(0xffffffffu, ok == 0 || abort_flag != 0)) {
          abort_flag = 1;
          stop = true;
          break;
        }
        tc::fence_after();
#pragma unroll 1
        for (int c0 = part * C_SPAN; c0 < part * C_SPAN + C_SPAN; c0 += 32) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * N + c0), v);
          if constexpr (GRID) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              const int dir = nt * (N / 16) + c0 / 16 + half;   // the same for the whole warp
              if (dir >= J) continue;
              const float* hv = v + 16 * half;
              const float4* tab = reinterpret_cast<const float4*>(psi_tab);
              if (n_psi == 24) {
                // psi + pi flips the odd harmonics: S_t = E_t + O_t, S_{t+12} = E_t - O_t (t < 12), even-a
                // and odd-a partial sums E, O; then the 24 scores compared in index order
                float sc[24];
#pragma unroll
                for (int g = 0; g < 3; ++g) {
                  float e[4], o[4];
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    e[u] = hv[0];
                    o[u] = 0.f;
                  }
#pragma unroll
                  for (int q = 0; q < 12; ++q) {
                    const float4 c = tab[q * 16 + g];
                    const float hq = hv[q + 1];
                    if ((q / 2) % 2 == 1) {   // a = q / 2 + 1 even
                      e[0] = fmaf(c.x, hq, e[0]);
                      e[1] = fmaf(c.y, hq, e[1]);
                      e[2] = fmaf(c.z, hq, e[2]);
                      e[3] = fmaf(c.w, hq, e[3]);
                    } else {
                      o[0] = fmaf(c.x, hq, o[0]);
                      o[1] = fmaf(c.y, hq, o[1]);
                      o[2] = fmaf(c.z, hq, o[2]);
                      o[3] = fmaf(c.w, hq, o[3]);
                    }
                  }
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    sc[4 * g + u] = e[u] + o[u];
                    sc[12 + 4 * g + u] = e[u] - o[u];
                  }
                }
#pragma unroll
                for (int t = 0; t < 24; ++t) {
                  if (first || sc[t] > best) {
                    best = sc[t];
                    bj = dir * 24 + t;
                    first = false;
                  }
                }
                continue;
              }
              // eight angles at a time: independent accumulators, one coefficient row per harmonic term
#pragma unroll 1
              for (int t0 = 0; t0 < n_psi; t0 += 8) {
                float sc[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) sc[u] = hv[0];
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                  const float4 c0 = tab[q * 16 + t0 / 4], c1 = tab[q * 16 + t0 / 4 + 1];
                  const float hq = hv[q + 1];
                  sc[0] = fmaf(c0.x, hq, sc[0]);
                  sc[1] = fmaf(c0.y, hq, sc[1]);
                  sc[2] = fmaf(c0.z, hq, sc[2]);
                  sc[3] = fmaf(c0.w, hq, sc[3]);
                  sc[4] = fmaf(c1.x, hq, sc[4]);
                  sc[5] = fmaf(c1.y, hq, sc[5]);
                  sc[6] = fmaf(c1.z, hq, sc[6]);
                  sc[7] = fmaf(c1.w, hq, sc[7]);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  const int t = t0 + u;
                  if (t < n_psi && (first || sc[u] > best)) {
                    best = sc[u];
                    bj = dir * n_psi + t;
                    first = false;
                  }
                }
              }
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int j = nt * N + c0 + i;
              if (j < J && (first || v[i] > best)) {
                best = v[i];
                bj = j;
                first = false;
              }
            }
          }
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(tc::smem_u32(&acce[b]));
      }
      if (stop) break;
      const long long p = mt * M + row;
      if (p < P) {
        if (GRID) {
          if (!first) atomicMax(keys + p, sweep_key(best, bj));
        } else if (nsplit == 1) {
          maxv[p] = best;
          argmax[p] = bj;
        } else {
          atomicMax(keys + p, sweep_key(best, bj));
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc<512>(tmem);
  }
}

size_t so3_ws_a_bytes(long long P, int cpad) {
  return (size_t)((P + ws::M - 1) / ws::M) * (size_t)(cpad / ws::KC) * ws::A_BYTES;
}

size_t so3_ws_b_bytes(int J, int cpad) {
  return (size_t)((J + ws::N - 1) / ws::N) * (size_t)(cpad / ws::KC) * ws::B_BYTES;
}

void so3_ws_build_b(const float* B, int cpad, int J, unsigned char* Bb, cudaStream_t st) {
  const int ntn = (J + ws::N - 1) / ws::N, nkc = cpad / ws::KC;
  k_so3_b_split<<<1024, 256, 0, st>>>(B, cpad, J, ntn, nkc, Bb);
}

void so3_ws_split_a(const float* G, long long P, int C, int cpad, unsigned char* Ab, int sms, cudaStream_t st) {
  k_so3_a_split<<<sms * 8, 256, 0, st>>>(G, P, C, cpad / ws::KC, Ab);
}

bool sweep_so3_ws(long long P, int cpad, const unsigned char* Ab, const unsigned char* Bb, int J, float* maxv,
                  int32_t* argmax, int* err, int sms, cudaStream_t st) {
  if (cpad % ws::KC != 0 || P < 1) return false;
  if (!ext_smem_optin((const void*)k_sweep_so3_ws<false>, ws::SMEM)) return false;
  const int ntn = (J + ws::N - 1) / ws::N, nkc = cpad / ws::KC;
  const long long ntm = (P + ws::M - 1) / ws::M;
  long long grid = sms;
  if (grid > ntm) grid = ntm;
  k_sweep_so3_ws<false><<<dim3((unsigned)grid, 1), ws::THREADS, ws::SMEM, st>>>(Ab, Bb, P, nkc, ntn, J, 0, maxv,
                                                                               argmax, nullptr, err, 2000000000ull);
  return true;
}

bool sweep_so3_ws_grid(long long P, int cpad, const unsigned char* Ab, const unsigned char* Bb, int n_dirs,
                       int n_psi, float* maxv, int32_t* argmax, unsigned long long* keys, int* err, int sms,
                       cudaStream_t st) {
  if (cpad % ws::KC != 0 || P < 1 || n_psi < 1 || n_psi > 64 || !keys) return false;
  if (!ext_smem_optin((const void*)k_sweep_so3_ws<true>, ws::SMEM)) return false;
  const int ntn = (16 * n_dirs + ws::N - 1) / ws::N, nkc = cpad / ws::KC;
  const long long ntm = (P + ws::M - 1) / ws::M;
  long long grid = sms;
  if (grid > ntm) grid = ntm;
  cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * P, st);
  k_sweep_so3_ws<true><<<dim3((unsigned)grid, 1), ws::THREADS_GRID, ws::SMEM, st>>>(
      Ab, Bb, P, nkc, ntn, n_dirs, n_psi, maxv, argmax, keys, err, 2000000000ull);
  long long b = (P + 255) / 256;
  if (b > 4096) b = 4096;
  k_sweep_keys_finish<<<(unsigned)b, 256, 0, st>>>(keys, P, maxv, argmax);
  return true;
}
