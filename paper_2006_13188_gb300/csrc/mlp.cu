// The proposal network's arithmetic on the 5th-generation tensor cores: a
// BF16 GEMM C = A B^T (both operands K-major, FP32 accumulation in tensor
// memory) with a fused bias / ReLU / ReLU-mask epilogue, and the small
// kernels around it (input normalisation, quaternion loss and its gradient,
// bias gradients, transposes, Adam).
//
// Network: x = row / |row|, h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
// o = W3 h2 + b3 (4 outputs), q = o / |o|, loss mean(1 - <q, q*>^2).
#include "internal.h"
#include "tc_common.cuh"

#include <cfloat>

namespace {

constexpr int GBM = 128, GBK = 64;
constexpr int G_SBO = (GBK / 8) * 128;           // bytes between 8-row groups of a 64-wide K chunk
constexpr int GA_BYTES = (GBM / 8) * G_SBO;      // 16 KB
constexpr int G_SMEM_REQUEST = 100 * 1024;       // at most two blocks per SM (TMEM columns)
constexpr unsigned long long G_WAIT_NS = 1000000000ull;

}  // namespace

// One 128 x BN output tile per block; K in chunks of 64 staged by all 128
// threads (16-byte loads, zero beyond M, N, K), four K = 16 MMAs per chunk
// issued by one thread; thread t owns output row t (TMEM lane t).
template <int BN>
__global__ void __launch_bounds__(128) k_gemm_bf16(const __nv_bfloat16* __restrict__ A, int lda,
                                                   const __nv_bfloat16* __restrict__ B, int ldb, int M, int N, int K,
                                                   GemmEpilogue ep, int* __restrict__ err) {
  constexpr int TCOLS = BN < 32 ? 32 : BN;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* As = smem;
  unsigned char* Bs = smem + GA_BYTES;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * BN;
  if (tid == 0) {
    abort_flag = 0;
    tc::mbar_init(tc::smem_u32(&mbar), 1);
  }
  if (warp == 0) tc::tmem_alloc<TCOLS>(tc::smem_u32(&tmem_slot));
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot, mbar_addr = tc::smem_u32(&mbar);
  constexpr uint32_t IDESC = tc::make_idesc(GBM, BN);
  uint32_t phase = 0;
  const int nk = (K + GBK - 1) / GBK;
  // The K chunk's operand rows are loaded into registers all at once (every
  // thread's loads in flight together), and the next chunk's while the
  // tensor cores work on the current one.
  constexpr int NA = GBM * 8 / 128, NB = (BN * 8 + 127) / 128;
  uint4 va[NA], vb[NB];
  auto load_chunk = [&](int k0) {
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int q = tid + i * 128;
      const int m = q >> 3, k = k0 + (q & 7) * 8;
      va[i] = (m0 + m < M && k < K) ? __ldg(reinterpret_cast<const uint4*>(A + (size_t)(m0 + m) * lda + k))
                                    : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int q = tid + i * 128;
      const int n = q >> 3, k = k0 + (q & 7) * 8;
      vb[i] = (q < BN * 8 && n0 + n < N && k < K)
                  ? __ldg(reinterpret_cast<const uint4*>(B + (size_t)(n0 + n) * ldb + k))
                  : make_uint4(0, 0, 0, 0);
    }
  };
  if (nk > 0) load_chunk(0);
  for (int kc = 0; kc < nk; ++kc) {
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int q = tid + i * 128;
      const int m = q >> 3, kp = q & 7;
      *reinterpret_cast<uint4*>(As + (m >> 3) * G_SBO + kp * 128 + (m & 7) * 16) = va[i];
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int q = tid + i * 128;
      const int n = q >> 3, kp = q & 7;
      if (q < BN * 8) *reinterpret_cast<uint4*>(Bs + (n >> 3) * G_SBO + kp * 128 + (n & 7) * 16) = vb[i];
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int s = 0; s < GBK / 16; ++s)
        tc::mma_bf16(tmem, tc::make_desc(tc::smem_u32(As) + s * 256, 128, G_SBO),
                     tc::make_desc(tc::smem_u32(Bs) + s * 256, 128, G_SBO), IDESC, (kc > 0 || s > 0) ? 1u : 0u);
      tc::mma_commit(mbar_addr);
    }
    if (kc + 1 < nk) load_chunk((kc + 1) * GBK);
    if (!tc::mbar_wait_bounded(mbar_addr, phase, G_WAIT_NS, err, EXT_ERR_TIMEOUT)) abort_flag = 1;
    phase ^= 1u;
    __syncthreads();
    if (abort_flag) break;
  }
  if (!abort_flag) {
    tc::fence_after();
    const int lane = tid & 31;
    const int mw = m0 + warp * 32;   // first row of this warp's TMEM lanes
    // one output element: bias, ReLU, ReLU mask, FP32 and/or BF16 stores
    auto emit = [&](int m, int n, float x) {
      if (ep.bias) x += ep.bias[n];
      if (ep.relu) x = fmaxf(x, 0.f);
      if (ep.mask && !(__bfloat162float(ep.mask[(size_t)m * ep.ldm + n]) > 0.f)) x = 0.f;
      if (ep.out_f32) ep.out_f32[ep.trans ? (size_t)n * ep.ldo + m : (size_t)m * ep.ldo + n] = x;
      if (ep.out_bf16)
        ep.out_bf16[ep.trans ? (size_t)n * ep.ldo16 + m : (size_t)m * ep.ldo16 + n] = __float2bfloat16_rn(x);
    };
    // row-major outputs go through a per-warp 32 x 32 transpose in shared
    // memory, so that the lanes of a warp read the mask and store along a row
    // (coalesced); transposed outputs are already coalesced with one lane per row
    float* scratch = reinterpret_cast<float*>(Bs + BN * GBK * 2) + warp * 32 * 33;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (ep.trans) {
        const int m = mw + lane;
        if (m < M) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int n = n0 + c0 + i;
            if (c0 + i < BN && n < N) emit(m, n, v[i]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) scratch[lane * 33 + i] = v[i];
        __syncwarp();
        const int n = n0 + c0 + lane;
        const bool col_ok = c0 + lane < BN && n < N;
        // this lane's column of the warp's 32 rows: the bias once, the 32 mask
        // entries all in flight together, then the stores
        const float bn = (ep.bias && col_ok) ? ep.bias[n] : 0.f;
        float xs[32];
        __nv_bfloat16 mk[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          xs[r] = scratch[r * 33 + lane];
          mk[r] = (ep.mask && col_ok && mw + r < M) ? ep.mask[(size_t)(mw + r) * ep.ldm + n] : __float2bfloat16_rn(1.f);
        }
        __syncwarp();
        if (col_ok) {
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const int m = mw + r;
            if (m >= M) break;
            float x = ep.bias ? xs[r] + bn : xs[r];
            if (ep.relu) x = fmaxf(x, 0.f);
            if (ep.mask && !(__bfloat162float(mk[r]) > 0.f)) x = 0.f;
            if (ep.out_f32) ep.out_f32[(size_t)m * ep.ldo + n] = x;
            if (ep.out_bf16) ep.out_bf16[(size_t)m * ep.ldo16 + n] = __float2bfloat16_rn(x);
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc<TCOLS>(tmem);
  }
}

template <int BN>
static void launch_gemm_bn(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                           const GemmEpilogue& ep, int* err, cudaStream_t st) {
  ext_smem_optin((const void*)k_gemm_bf16<BN>, G_SMEM_REQUEST);
  dim3 grid((M + GBM - 1) / GBM, (N + BN - 1) / BN);
  k_gemm_bf16<BN><<<grid, 128, G_SMEM_REQUEST, st>>>(A, lda, B, ldb, M, N, K, ep, err);
}

void gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
               const GemmEpilogue& ep, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  if (N <= 16) launch_gemm_bn<16>(A, lda, B, ldb, M, N, K, ep, err, st);
  else if (N <= 64) launch_gemm_bn<64>(A, lda, B, ldb, M, N, K, ep, err, st);
  else launch_gemm_bn<256>(A, lda, B, ldb, M, N, K, ep, err, st);
}

// ------------------------------------------------------------ small pieces ---

// Y[i] = X[r] / |X[r]| (first C entries, r = idx ? idx[i] : i) as BF16, zero to pitch dp
__global__ void k_rows_normalize_bf16(const float* __restrict__ X, int ldx, const int32_t* __restrict__ idx, int n,
                                      int C, int dp, __nv_bfloat16* __restrict__ Y) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const float* row = X + (size_t)(idx ? idx[i] : i) * ldx;
  __shared__ float red[4];
  float s = 0.f;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const float v = row[c];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  const float tot = red[0] + red[1] + red[2] + red[3];
  const float inv = tot > 0.f ? rsqrtf(tot) : 0.f;
  for (int c = threadIdx.x; c < dp; c += blockDim.x)
    Y[(size_t)i * dp + c] = __float2bfloat16_rn(c < C ? row[c] * inv : 0.f);
}

void launch_rows_normalize_bf16(const float* X, int ldx, const int32_t* idx, int n, int C, int dp,
                                __nv_bfloat16* Y, cudaStream_t st) {
  if (n > 0) k_rows_normalize_bf16<<<n, 128, 0, st>>>(X, ldx, idx, n, C, dp, Y);
}

__global__ void k_gather_quats(const float* __restrict__ q, const int32_t* __restrict__ idx, int n,
                               float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 v = *reinterpret_cast<const float4*>(q + 4 * (size_t)idx[i]);
  *reinterpret_cast<float4*>(out + 4 * (size_t)i) = v;
}

void launch_gather_quats(const float* q, const int32_t* idx, int n, float* out, cudaStream_t st) {
  if (n > 0) k_gather_quats<<<(n + 127) / 128, 128, 0, st>>>(q, idx, n, out);
}

// loss += mean(1 - <q, q*>^2) with q = o / |o|; d loss / d o as rows of 16
// (entries 4..15 zero) in BF16 (dout) and FP32 (dout_f)
__global__ void k_quat_loss(const float* __restrict__ o, int ldo, const float* __restrict__ qt, int n,
                            float* __restrict__ loss, __nv_bfloat16* __restrict__ dout, float* __restrict__ dout_f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float li = 0.f;
  if (i < n) {
    float v[4], t[4], nn = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = o[(size_t)i * ldo + k];
      t[k] = qt[4 * (size_t)i + k];
      nn += v[k] * v[k];
    }
    const float norm = sqrtf(fmaxf(nn, 1e-30f));
    float q[4], d = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      q[k] = v[k] / norm;
      d += q[k] * t[k];
    }
    li = (1.f - d * d) / n;
    // d loss / d q = -2 d q* / n; through q = o / |o|: (dq - q <dq, q>) / |o|
    float dq[4], qdq = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      dq[k] = -2.f * d * t[k] / n;
      qdq += dq[k] * q[k];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float gk = k < 4 ? (dq[k] - q[k] * qdq) / norm : 0.f;
      if (dout) dout[(size_t)i * 16 + k] = __float2bfloat16_rn(gk);
      if (dout_f) dout_f[(size_t)i * 16 + k] = gk;
    }
  }
  for (int off = 16; off > 0; off >>= 1) li += __shfl_xor_sync(0xffffffffu, li, off);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, li);
}

void launch_quat_loss(const float* o, int ldo, const float* qt, int n, float* loss, __nv_bfloat16* dout,
                      float* dout_f, cudaStream_t st) {
  if (n > 0) k_quat_loss<<<(n + 127) / 128, 128, 0, st>>>(o, ldo, qt, n, loss, dout, dout_f);
}

// out[c] = sum_r X[r][c]
__global__ void k_colsum(const float* __restrict__ X, int rows, int cols, int ld, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += X[(size_t)r * ld + c];
  out[c] = s;
}

void launch_colsum(const float* X, int rows, int cols, int ld, float* out, cudaStream_t st) {
  k_colsum<<<(cols + 127) / 128, 128, 0, st>>>(X, rows, cols, ld, out);
}

// Y[c][r] = X[r][c] for r < rows, c < cols; zero elsewhere in Y's yrows x ycols
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ X, int rows, int cols, int ldx,
                                 __nv_bfloat16* __restrict__ Y, int yrows, int ycols, int ldy) {
  __shared__ __nv_bfloat16 t[32][34];
  const int yr0 = blockIdx.y * 32, yc0 = blockIdx.x * 32;   // Y tile origin: rows = source columns
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = yc0 + j, c = yr0 + threadIdx.x;            // source element (r, c)
    t[j][threadIdx.x] = (r < rows && c < cols) ? X[(size_t)r * ldx + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int yr = yr0 + j, yc = yc0 + threadIdx.x;
    if (yr < yrows && yc < ycols) Y[(size_t)yr * ldy + yc] = t[threadIdx.x][j];
  }
}

void launch_transpose_bf16(const __nv_bfloat16* X, int rows, int cols, int ldx, __nv_bfloat16* Y, int yrows,
                           int ycols, int ldy, cudaStream_t st) {
  dim3 grid((ycols + 31) / 32, (yrows + 31) / 32);
  k_transpose_bf16<<<grid, dim3(32, 8), 0, st>>>(X, rows, cols, ldx, Y, yrows, ycols, ldy);
}

// Adam (Kingma & Ba) on FP32 master weights; c1, c2 the bias corrections; refreshes the BF16 copy
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2, __nv_bfloat16* __restrict__ w16) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16_rn(wi);
  }
}

void launch_adam(float* w, float* m, float* v, const float* g, long long n, float lr, int step, __nv_bfloat16* w16,
                 cudaStream_t st) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - pow(b1, step)), c2 = (float)(1.0 - pow(b2, step));
  const long long blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  k_adam<<<(unsigned)blocks, 256, 0, st>>>(w, m, v, g, n, lr, (float)b1, (float)b2, 1e-8f, c1, c2, w16);
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

void launch_f32_to_bf16(const float* x, long long n, __nv_bfloat16* y, cudaStream_t st) {
  const long long blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  if (n > 0) k_f32_to_bf16<<<(unsigned)blocks, 256, 0, st>>>(x, n, y);
}

// q = o / |o| from the first 4 entries of each row (identity if o = 0)
__global__ void k_normalize_quat(const float* __restrict__ o, int ldo, int n, float* __restrict__ q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v[4], s = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = o[(size_t)i * ldo + k];
    s += v[k] * v[k];
  }
  const float inv = s > 0.f ? rsqrtf(s) : 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) q[4 * (size_t)i + k] = s > 0.f ? v[k] * inv : (k == 0 ? 1.f : 0.f);
}

void launch_normalize_quat(const float* o, int ldo, int n, float* q, cudaStream_t st) {
  if (n > 0) k_normalize_quat<<<(n + 127) / 128, 128, 0, st>>>(o, ldo, n, q);
}
