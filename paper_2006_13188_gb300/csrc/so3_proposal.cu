// SO(3) matching by proposal: the score bound that prunes voxels, ordered
// compaction of the survivors, gathering their component channels, the
// gradient-ascent refinement of a proposed rotation on the exact score,
// rotation augmentation of training rows, and the final merge.
//
// Score of one voxel for a rotation R (real filter and signal):
//   S(R) = sum over unique (l, a, b) of w * Re(conj(C^l_ab(R)) G_l^ab),
// w = 1 for the self entry (0, 0) and 2 for the others.  With
// R = R_z(alpha) R_y(beta) R_z(gamma) and the unit quaternion (w, x, y, z):
// cos(beta/2) = |(w, z)|, sin(beta/2) = |(x, y)|, e^{i sigma} = (w + i z) /
// cos(beta/2), e^{i delta} = (y - i x) / sin(beta/2) where sigma = (alpha +
// gamma)/2 and delta = (alpha - gamma)/2, so C^l_ab = d^l_ba(beta)
// e^{-i((a+b) sigma + (b-a) delta)} needs no trigonometric function.
#include "internal.h"

#include <cfloat>

namespace {

struct SteerTabs {
  float pw[26];     // cos(beta/2)^k (k = 0..12), then sin(beta/2)^k
  float2 es[13];    // e^{i k sigma}
  float2 ed[13];    // e^{i k delta}
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float4 quat_mul(float4 p, float4 q) {   // (w, x, y, z) in (x, y, z, w) slots
  return make_float4(p.x * q.x - p.y * q.y - p.z * q.z - p.w * q.w, p.x * q.y + p.y * q.x + p.z * q.w - p.w * q.z,
                     p.x * q.z - p.y * q.w + p.z * q.x + p.w * q.y, p.x * q.w + p.y * q.z - p.z * q.y + p.w * q.x);
}

__device__ __forceinline__ float4 quat_normalize(float4 q) {
  const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  return make_float4(q.x * inv, q.y * inv, q.z * inv, q.w * inv);
}

// unit quaternion of the rotation by angle t about the unit axis u
__device__ __forceinline__ float4 quat_exp(float t, float ux, float uy, float uz) {
  float s, c;
  sincosf(0.5f * t, &s, &c);
  return make_float4(c, s * ux, s * uy, s * uz);
}

// The warp's tables for rotation q (unit quaternion, (w, x, y, z) in (x, y, z, w)).
__device__ __forceinline__ void steer_tables(float4 q, SteerTabs* t, int lane) {
  const float cb = sqrtf(q.x * q.x + q.w * q.w), sb = sqrtf(q.y * q.y + q.z * q.z);
  const float2 es = cb > 1e-12f ? make_float2(q.x / cb, q.w / cb) : make_float2(1.f, 0.f);
  const float2 ed = sb > 1e-12f ? make_float2(q.z / sb, -q.y / sb) : make_float2(1.f, 0.f);
  __syncwarp();
  if (lane < 26) {
    const int k = lane < 13 ? lane : lane - 13;
    const float base = lane < 13 ? cb : sb;
    const float2 e = lane < 13 ? es : ed;
    float p = 1.f;
    float2 z = make_float2(1.f, 0.f);
    for (int j = 0; j < k; ++j) {
      p *= base;
      z = cmul(z, e);
    }
    t->pw[lane] = p;
    if (lane < 13) t->es[k] = z;
    else t->ed[k] = z;
  }
  __syncwarp();
}

// C^l_ab of one unique entry from the warp's tables
__device__ __forceinline__ float2 steer_entry(uint32_t meta, int e, const float (*coef)[256], const SteerTabs* t) {
  const int ks = (int)((meta >> 11) & 31u) - 12, kd = (int)((meta >> 16) & 31u) - 12;
  const int ns = (meta >> 21) & 7u, pc0 = (meta >> 24) & 15u, ps0 = meta >> 28;
  float d = 0.f;
  for (int j = 0; j < ns; ++j) d += coef[j][e] * t->pw[pc0 - 2 * j] * t->pw[13 + ps0 + 2 * j];
  const float2 A = ks >= 0 ? make_float2(t->es[ks].x, -t->es[ks].y) : t->es[-ks];
  const float2 B = kd >= 0 ? make_float2(t->ed[kd].x, -t->ed[kd].y) : t->ed[-kd];
  const float2 E = cmul(A, B);
  return make_float2(d * E.x, d * E.y);
}

constexpr int EPL = 8;   // unique entries per lane (8 x 32 >= 231)

struct LaneChannels {
  uint32_t meta[EPL];
  float g0[EPL], g1[EPL];
};

// S(q) for the warp's voxel; identical in every lane (lane 0's sum broadcast)
__device__ float eval_score(float4 q, const LaneChannels& lc, int nent, const float (*coef)[256], SteerTabs* t,
                            int lane) {
  steer_tables(quat_normalize(q), t, lane);
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int e = lane + 32 * k;
    if (e < nent) {
      const float2 C = steer_entry(lc.meta[k], e, coef, t);
      acc += (lc.meta[k] & (1u << 10)) ? C.x * lc.g0[k] : 2.f * (C.x * lc.g0[k] + C.y * lc.g1[k]);
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  return __shfl_sync(0xffffffffu, acc, 0);
}

__device__ void load_steer(const So3Steer* __restrict__ tab, float (*coef)[256], uint32_t* meta, int nent) {
  for (int i = threadIdx.x; i < 7 * 256; i += blockDim.x) coef[i / 256][i % 256] = tab->coef[i / 256][i % 256];
  if (meta)
    for (int i = threadIdx.x; i < nent; i += blockDim.x) meta[i] = tab->meta[i];
  __syncthreads();
}

}  // namespace

// ------------------------------------------------------------ upper bound ---
// UB(p) = sum_l sqrt(2l+1) |G_l(p)|_F.  In the channel layout degree l owns
// the (2l+1)^2 channels from l(2l-1)(2l+1)/3 on: first its self channel
// (weight 1 in |G_l|_F^2), then Re/Im pairs standing for two entries each
// (weight 2).  One voxel per thread; the channel loop is unrolled so that
// many independent loads are in flight.
template <int L>
__global__ void __launch_bounds__(256) k_so3_upper_bound(const float* __restrict__ G, long long P,
                                                         float* __restrict__ ub) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    float u = 0.f;
#pragma unroll
    for (int l = 0; l <= L; ++l) {
      const int c0 = l * (2 * l - 1) * (2 * l + 1) / 3, c1 = c0 + (2 * l + 1) * (2 * l + 1);
      const float g0 = __ldg(G + (size_t)c0 * P + p);
      float acc = g0 * g0, acc2 = 0.f;
      // loads in batches of 24, all in flight before their squares are summed
      for (int cb = c0 + 1; cb < c1; cb += 24) {
        float x[24];
#pragma unroll
        for (int t = 0; t < 24; ++t) x[t] = cb + t < c1 ? __ldg(G + (size_t)(cb + t) * P + p) : 0.f;
#pragma unroll
        for (int t = 0; t < 24; ++t) acc2 = fmaf(x[t], x[t], acc2);
      }
      u += sqrtf((2.f * l + 1.f) * (acc + 2.f * acc2));
    }
    ub[p] = u;
  }
}

void launch_so3_upper_bound(const float* G, long long P, const So3Steer* tab, float* ub, int L, int sms,
                            cudaStream_t st) {
  (void)tab;
  long long b = (P + 255) / 256;
  if (b > (long long)sms * 16) b = (long long)sms * 16;
  if (P <= 0) return;
  switch (L) {
    case 0: k_so3_upper_bound<0><<<(unsigned)b, 256, 0, st>>>(G, P, ub); break;
    case 1: k_so3_upper_bound<1><<<(unsigned)b, 256, 0, st>>>(G, P, ub); break;
    case 2: k_so3_upper_bound<2><<<(unsigned)b, 256, 0, st>>>(G, P, ub); break;
    case 3: k_so3_upper_bound<3><<<(unsigned)b, 256, 0, st>>>(G, P, ub); break;
    case 4: k_so3_upper_bound<4><<<(unsigned)b, 256, 0, st>>>(G, P, ub); break;
    case 5: k_so3_upper_bound<5><<<(unsigned)b, 256, 0, st>>>(G, P, ub); break;
    default: k_so3_upper_bound<6><<<(unsigned)b, 256, 0, st>>>(G, P, ub); break;
  }
}

// ------------------------------------------------------- ordered compaction ---
namespace {
constexpr int CP_THREADS = 256, CP_ITEMS = 16, CP_CHUNK = CP_THREADS * CP_ITEMS;

__device__ __forceinline__ bool cp_flag(const float* v, long long i, long long n, float thr, int below) {
  if (i >= n) return false;
  const float x = v[i];
  return below ? (x < thr) : (x >= thr);
}
}  // namespace

__global__ void k_compact_count(const float* __restrict__ v, long long n, float thr, int below, int* __restrict__ cnt) {
  const long long base = (long long)blockIdx.x * CP_CHUNK;
  int c = 0;
  for (int it = 0; it < CP_ITEMS; ++it) c += __syncthreads_count(cp_flag(v, base + it * CP_THREADS + threadIdx.x, n, thr, below));
  if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

// exclusive scan of nb block counts (one block), total into *count
__global__ void k_compact_scan(const int* __restrict__ cnt, int nb, int* __restrict__ off, int* __restrict__ count) {
  __shared__ int s[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    const int i = b0 + threadIdx.x;
    const int x = i < nb ? cnt[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
      const int y = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < nb) off[i] = carry + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = carry;
}

__global__ void k_compact_write(const float* __restrict__ v, long long n, float thr, int below,
                                const int* __restrict__ off, int32_t* __restrict__ idx) {
  __shared__ int wsum[CP_THREADS / 32];
  const long long base = (long long)blockIdx.x * CP_CHUNK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int run = off[blockIdx.x];
  for (int it = 0; it < CP_ITEMS; ++it) {
    const long long i = base + it * CP_THREADS + threadIdx.x;
    const bool f = cp_flag(v, i, n, thr, below);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < CP_THREADS / 32; ++w) {
      if (w < warp) before += wsum[w];
      total += wsum[w];
    }
    if (f) idx[run + before + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
    run += total;
    __syncthreads();
  }
}

size_t compact_scratch_bytes(long long n) {
  const long long nb = (n + CP_CHUNK - 1) / CP_CHUNK;
  return sizeof(int) * (size_t)(2 * nb + 1);
}

void compact(const float* v, long long n, float thr, int below, int32_t* idx, int* count, void* scratch,
             cudaStream_t st) {
  const long long nb = (n + CP_CHUNK - 1) / CP_CHUNK;
  int* cnt = static_cast<int*>(scratch);
  int* off = cnt + nb;
  if (nb == 0) {
    cudaMemsetAsync(count, 0, sizeof(int), st);
    return;
  }
  k_compact_count<<<(unsigned)nb, CP_THREADS, 0, st>>>(v, n, thr, below, cnt);
  k_compact_scan<<<1, 1024, 0, st>>>(cnt, (int)nb, off, count);
  k_compact_write<<<(unsigned)nb, CP_THREADS, 0, st>>>(v, n, thr, below, off, idx);
}

// ----------------------------------------------------------------- gathers ---
// X[i][c] = G[c][vox[i]] for c < C, zero for C <= c < ldx (32 x 32 tiles through shared memory)
__global__ void k_gather_rows(const float* __restrict__ G, long long P, int C, const int32_t* __restrict__ vox, int n,
                              float* __restrict__ X, int ldx) {
  __shared__ float t[32][33];
  const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int i = i0 + threadIdx.x;
  const long long p = i < n ? (long long)vox[i] : 0;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j;
    t[j][threadIdx.x] = (i < n && c < C) ? __ldg(G + (size_t)c * P + p) : 0.f;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = i0 + j, c = c0 + threadIdx.x;
    if (r < n && c < ldx) X[(size_t)r * ldx + c] = t[threadIdx.x][j];
  }
}

void launch_gather_rows(const float* G, long long P, int C, const int32_t* vox, int n, float* X, int ldx,
                        cudaStream_t st) {
  if (n <= 0) return;
  dim3 grid((n + 31) / 32, (ldx + 31) / 32);
  k_gather_rows<<<grid, dim3(32, 8), 0, st>>>(G, P, C, vox, n, X, ldx);
}

// out[c][i] = G[c][vox[sel ? sel[i] : i]]
__global__ void k_gather_channels(const float* __restrict__ G, long long P, int C, const int32_t* __restrict__ vox,
                                  const int32_t* __restrict__ sel, int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = vox[sel ? sel[i] : i];
  for (int c = blockIdx.y; c < C; c += gridDim.y) out[(size_t)c * n + i] = __ldg(G + (size_t)c * P + p);
}

void launch_gather_channels(const float* G, long long P, int C, const int32_t* vox, const int32_t* sel, int n,
                            float* out, cudaStream_t st) {
  if (n <= 0) return;
  dim3 grid((n + 127) / 128, C < 64 ? C : 64);
  k_gather_channels<<<grid, 128, 0, st>>>(G, P, C, vox, sel, n, out);
}

// -------------------------------------------------------------- refinement ---
// One warp per voxel: from q0, `steps` gradient-ascent steps on S in the body
// frame.  The gradient: d/dxi_i S(R exp(xi e_i)) = Re tr(C(R)^H A_i^H G) with
// A_i = d/dt C(exp(t e_i)) at 0 (the rotation generators: (A_i^H G)_ab =
// (i/2)(al_-(a) G_{a-1,b} + al_+(a) G_{a+1,b}) for x, (1/2)(al_+(a) G_{a+1,b} -
// al_-(a) G_{a-1,b}) for y, i a G_ab for z, al_+-(a) = sqrt(l(l+1) - a(a+-1))),
// so one evaluation of C(R) gives the score and the gradient.  A step moves
// q -> q exp(t g/|g|), t halved until S increases (at most `tries` times;
// none: stop); an accepted step keeps t for the next one.
namespace {

struct LaneGrad {
  float hx0[EPL], hx1[EPL], hy0[EPL], hy1[EPL], hz0[EPL], hz1[EPL];
};

// S and its body-frame gradient at q, identical in every lane
__device__ float4 eval_score_grad(float4 q, const LaneChannels& lc, const LaneGrad& lg, int nent,
                                  const float (*coef)[256], SteerTabs* t, int lane) {
  steer_tables(quat_normalize(q), t, lane);
  float a0 = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int e = lane + 32 * k;
    if (e < nent) {
      const float2 C = steer_entry(lc.meta[k], e, coef, t);
      const float w = (lc.meta[k] & (1u << 10)) ? 1.f : 2.f;
      a0 += w * (C.x * lc.g0[k] + C.y * lc.g1[k]);
      ax += w * (C.x * lg.hx0[k] + C.y * lg.hx1[k]);
      ay += w * (C.x * lg.hy0[k] + C.y * lg.hy1[k]);
      az += w * (C.x * lg.hz0[k] + C.y * lg.hz1[k]);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
    ax += __shfl_xor_sync(0xffffffffu, ax, off);
    ay += __shfl_xor_sync(0xffffffffu, ay, off);
    az += __shfl_xor_sync(0xffffffffu, az, off);
  }
  return make_float4(__shfl_sync(0xffffffffu, a0, 0), __shfl_sync(0xffffffffu, ax, 0),
                     __shfl_sync(0xffffffffu, ay, 0), __shfl_sync(0xffffffffu, az, 0));
}

}  // namespace

__global__ void __launch_bounds__(128) k_so3_refine(const float* __restrict__ X, int ldx, int n,
                                                    const float* __restrict__ q0, const So3Steer* __restrict__ tab,
                                                    int steps, float theta0, int tries,
                                                    float* __restrict__ q_out, float* __restrict__ s_out) {
  __shared__ float coef[7][256];
  __shared__ uint32_t meta_s[256];
  __shared__ unsigned char l_s[256];
  __shared__ SteerTabs tabs[4];
  __shared__ float2 Gm[4][455];
  const int nent = tab->n;
  for (int i = threadIdx.x; i < nent; i += blockDim.x) l_s[i] = tab->l[i];
  load_steer(tab, coef, meta_s, nent);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  SteerTabs* tw = &tabs[warp];
  float2* Gw = Gm[warp];
  LaneChannels lc;
  LaneGrad lg;
#pragma unroll
  for (int k = 0; k < EPL; ++k) lc.meta[k] = (lane + 32 * k) < nent ? meta_s[lane + 32 * k] : 0u;
  const int nw = gridDim.x * 4;
  for (int i = blockIdx.x * 4 + warp; i < n; i += nw) {
    const float* row = X + (size_t)i * ldx;
    __syncwarp();
    // the full matrices G_l of this voxel (unique entries and their partners)
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
      const int e = lane + 32 * k;
      const uint32_t m = lc.meta[k];
      const int ch = m & 1023u;
      lc.g0[k] = e < nent ? row[ch] : 0.f;
      lc.g1[k] = (e < nent && !(m & (1u << 10))) ? row[ch + 1] : 0.f;
      if (e < nent) {
        const int l = l_s[e], ks = (int)((m >> 11) & 31u) - 12, kd = (int)((m >> 16) & 31u) - 12;
        const int a = (ks - kd) / 2, b = (ks + kd) / 2, d = 2 * l + 1, base = l * (2 * l - 1) * (2 * l + 1) / 3;
        const float sg = ((a + b) & 1) ? -1.f : 1.f;
        Gw[base + (a + l) * d + (b + l)] = make_float2(lc.g0[k], lc.g1[k]);
        Gw[base + (-a + l) * d + (-b + l)] = make_float2(sg * lc.g0[k], -sg * lc.g1[k]);
      }
    }
    __syncwarp();
    // H_i = A_i^H G at this lane's entries
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
      const int e = lane + 32 * k;
      lg.hx0[k] = lg.hx1[k] = lg.hy0[k] = lg.hy1[k] = lg.hz0[k] = lg.hz1[k] = 0.f;
      if (e < nent) {
        const uint32_t m = lc.meta[k];
        const int l = l_s[e], ks = (int)((m >> 11) & 31u) - 12, kd = (int)((m >> 16) & 31u) - 12;
        const int a = (ks - kd) / 2, b = (ks + kd) / 2, d = 2 * l + 1, base = l * (2 * l - 1) * (2 * l + 1) / 3;
        const float ll = (float)(l * (l + 1));
        const float am = a > -l ? sqrtf(ll - (float)(a * (a - 1))) : 0.f;
        const float ap = a < l ? sqrtf(ll - (float)(a * (a + 1))) : 0.f;
        const float2 gm = a > -l ? Gw[base + (a - 1 + l) * d + (b + l)] : make_float2(0.f, 0.f);
        const float2 gp = a < l ? Gw[base + (a + 1 + l) * d + (b + l)] : make_float2(0.f, 0.f);
        const float2 g0 = make_float2(lc.g0[k], lc.g1[k]);
        // x: (i/2)(am gm + ap gp)
        const float sx = 0.5f * (am * gm.x + ap * gp.x), sy = 0.5f * (am * gm.y + ap * gp.y);
        lg.hx0[k] = -sy;
        lg.hx1[k] = sx;
        // y: (1/2)(ap gp - am gm)
        lg.hy0[k] = 0.5f * (ap * gp.x - am * gm.x);
        lg.hy1[k] = 0.5f * (ap * gp.y - am * gm.y);
        // z: i a G_ab
        lg.hz0[k] = -(float)a * g0.y;
        lg.hz1[k] = (float)a * g0.x;
      }
    }
    float4 q = quat_normalize(make_float4(q0[4 * (size_t)i], q0[4 * (size_t)i + 1], q0[4 * (size_t)i + 2],
                                          q0[4 * (size_t)i + 3]));
    float4 sg = eval_score_grad(q, lc, lg, nent, coef, tw, lane);
    float theta = theta0;
    for (int it = 0; it < steps; ++it) {
      const float gn = sqrtf(sg.y * sg.y + sg.z * sg.z + sg.w * sg.w);
      if (!(gn > 0.f)) break;
      const float ux = sg.y / gn, uy = sg.z / gn, uz = sg.w / gn;
      bool moved = false;
      float t = theta;
      for (int k = 0; k < tries; ++k) {
        const float4 qn = quat_mul(q, quat_exp(t, ux, uy, uz));
        const float4 sn = eval_score_grad(qn, lc, lg, nent, coef, tw, lane);
        if (sn.x > sg.x) {
          q = quat_normalize(qn);
          sg = sn;
          theta = t;
          moved = true;
          break;
        }
        t *= 0.5f;
      }
      if (!moved) break;
    }
    if (lane == 0) {
      *reinterpret_cast<float4*>(q_out + 4 * (size_t)i) = q;
      s_out[i] = sg.x;
    }
  }
}

void launch_so3_refine(const float* X, int ldx, int n, const float* q0, const So3Steer* tab, int steps, float theta0,
                       int tries, float* q_out, float* s_out, int sms, cudaStream_t st) {
  if (n <= 0) return;
  long long b = (n + 3) / 4;
  if (b > (long long)sms * 16) b = (long long)sms * 16;
  k_so3_refine<<<(unsigned)b, 128, 0, st>>>(X, ldx, n, q0, tab, steps, theta0, tries, q_out, s_out);
}

// ------------------------------------------------------------ augmentation ---
// Rotating the score function by Q: S'(R) = S(Q^-1 R) has components
// G'_l = G_l C^l(Q) (C(R1 R2) = C(R2) C(R1), C unitary), and its maximiser
// is Q R*, i.e. the label quaternion Q q*.  One warp per row.
__global__ void __launch_bounds__(128) k_so3_augment(const float* __restrict__ X, int ldx,
                                                     const int32_t* __restrict__ rows, int n,
                                                     const float* __restrict__ Q, const float* __restrict__ q_in,
                                                     const So3Steer* __restrict__ tab, int C,
                                                     float* __restrict__ X_out, int ldo, float* __restrict__ q_out) {
  __shared__ float coef[7][256];
  __shared__ uint32_t meta_s[256];
  __shared__ unsigned char l_s[256];
  __shared__ SteerTabs tabs[4];
  __shared__ float2 Cm[4][455], Gm[4][455];
  const int nent = tab->n;
  for (int i = threadIdx.x; i < nent; i += blockDim.x) l_s[i] = tab->l[i];
  load_steer(tab, coef, meta_s, nent);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = gridDim.x * 4;
  float2* Cw = Cm[warp];
  float2* Gw = Gm[warp];
  for (int i = blockIdx.x * 4 + warp; i < n; i += nw) {
    const float* row = X + (size_t)(rows ? rows[i] : i) * ldx;
    const float4 qq = quat_normalize(*reinterpret_cast<const float4*>(Q + 4 * (size_t)i));
    steer_tables(qq, &tabs[warp], lane);
    for (int e = lane; e < nent; e += 32) {
      const uint32_t m = meta_s[e];
      const int l = l_s[e], ch = m & 1023u;
      const int ks = (int)((m >> 11) & 31u) - 12, kd = (int)((m >> 16) & 31u) - 12;
      const int a = (ks - kd) / 2, b = (ks + kd) / 2, d = 2 * l + 1, base = l * (2 * l - 1) * (2 * l + 1) / 3;
      const float2 c = steer_entry(m, e, coef, &tabs[warp]);
      const float2 g = (m & (1u << 10)) ? make_float2(row[ch], 0.f) : make_float2(row[ch], row[ch + 1]);
      const float sg = ((a + b) & 1) ? -1.f : 1.f;
      Cw[base + (a + l) * d + (b + l)] = c;
      Gw[base + (a + l) * d + (b + l)] = g;
      Cw[base + (-a + l) * d + (-b + l)] = make_float2(sg * c.x, -sg * c.y);
      Gw[base + (-a + l) * d + (-b + l)] = make_float2(sg * g.x, -sg * g.y);
    }
    __syncwarp();
    float* orow = X_out + (size_t)i * ldo;
    for (int e = lane; e < nent; e += 32) {
      const uint32_t m = meta_s[e];
      const int l = l_s[e], ch = m & 1023u;
      const int ks = (int)((m >> 11) & 31u) - 12, kd = (int)((m >> 16) & 31u) - 12;
      const int a = (ks - kd) / 2, b = (ks + kd) / 2, d = 2 * l + 1, base = l * (2 * l - 1) * (2 * l + 1) / 3;
      float2 acc = make_float2(0.f, 0.f);
      for (int c = -l; c <= l; ++c) {
        const float2 g = Gw[base + (a + l) * d + (c + l)], r = Cw[base + (c + l) * d + (b + l)];
        acc.x += g.x * r.x - g.y * r.y;
        acc.y += g.x * r.y + g.y * r.x;
      }
      orow[ch] = acc.x;
      if (!(m & (1u << 10))) orow[ch + 1] = acc.y;
    }
    for (int c = C + lane; c < ldo; c += 32) orow[c] = 0.f;
    if (lane == 0) {
      const float4 qi = *reinterpret_cast<const float4*>(q_in + 4 * (size_t)(rows ? rows[i] : i));
      *reinterpret_cast<float4*>(q_out + 4 * (size_t)i) = quat_normalize(quat_mul(qq, qi));
    }
    __syncwarp();
  }
}

void launch_so3_augment(const float* X, int ldx, const int32_t* rows, int n, const float* Q, const float* q_in,
                        const So3Steer* tab, int C, float* X_out, int ldo, float* q_out, cudaStream_t st) {
  if (n <= 0) return;
  const int b = (n + 3) / 4 < 4096 ? (n + 3) / 4 : 4096;
  k_so3_augment<<<b, 128, 0, st>>>(X, ldx, rows, n, Q, q_in, tab, C, X_out, ldo, q_out);
}

// ------------------------------------------------------------------ merge ---
__global__ void k_so3_fill(long long P, float* __restrict__ score, float* __restrict__ quat,
                           int32_t* __restrict__ grid_idx) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    score[p] = -INFINITY;
    if (quat) *reinterpret_cast<float4*>(quat + 4 * p) = make_float4(1.f, 0.f, 0.f, 0.f);
    if (grid_idx) grid_idx[p] = -2;
  }
}

void launch_so3_fill(long long P, float* score, float* quat, int32_t* grid_idx, cudaStream_t st) {
  long long b = (P + 255) / 256;
  if (b > 4096) b = 4096;
  if (P > 0) k_so3_fill<<<(unsigned)b, 256, 0, st>>>(P, score, quat, grid_idx);
}

__global__ void k_so3_scatter(const int32_t* __restrict__ cand, int n, const float* __restrict__ s,
                              const float* __restrict__ q, float* __restrict__ score, float* __restrict__ quat,
                              int32_t* __restrict__ grid_idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = cand[i];
  score[p] = s[i];
  if (quat) *reinterpret_cast<float4*>(quat + 4 * p) = *reinterpret_cast<const float4*>(q + 4 * (size_t)i);
  if (grid_idx) grid_idx[p] = -1;
}

void launch_so3_scatter(const int32_t* cand, int n, const float* s, const float* q, float* score, float* quat,
                        int32_t* grid_idx, cudaStream_t st) {
  if (n > 0) k_so3_scatter<<<(n + 127) / 128, 128, 0, st>>>(cand, n, s, q, score, quat, grid_idx);
}

// fallback i: voxel cand[fb[i]] was swept (max m, argmax j); keep whichever of
// the refined and the grid rotation scores higher
__global__ void k_so3_merge(const int32_t* __restrict__ cand, const int32_t* __restrict__ fb, int n_fb,
                            const float* __restrict__ m, const int32_t* __restrict__ j, const double* __restrict__ grid,
                            float* __restrict__ score, float* __restrict__ quat, int32_t* __restrict__ grid_idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_fb) return;
  const long long p = cand[fb ? fb[i] : i];
  const int ji = j[i];
  if (grid_idx) grid_idx[p] = ji;
  if (m[i] >= score[p]) {
    score[p] = m[i];
    if (quat) {
      const double* g = grid + 4 * (size_t)ji;
      const double nrm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + g[3] * g[3]);
      *reinterpret_cast<float4*>(quat + 4 * p) =
          make_float4((float)(g[0] / nrm), (float)(g[1] / nrm), (float)(g[2] / nrm), (float)(g[3] / nrm));
    }
  }
}

void launch_so3_merge(const int32_t* cand, const int32_t* fb, int n_fb, const float* m, const int32_t* j,
                      const double* grid, float* score, float* quat, int32_t* grid_idx, cudaStream_t st) {
  if (n_fb > 0) k_so3_merge<<<(n_fb + 127) / 128, 128, 0, st>>>(cand, fb, n_fb, m, j, grid, score, quat, grid_idx);
}

// *bad = 1 if some idx[i] is outside [0, upper)
__global__ void k_check_index(const int32_t* __restrict__ idx, long long n, long long upper, int* __restrict__ bad) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (idx[i] < 0 || (long long)idx[i] >= upper) *bad = 1;
}

void launch_check_index(const int32_t* idx, long long n, long long upper, int* bad, cudaStream_t st) {
  long long b = (n + 255) / 256;
  if (b > 1024) b = 1024;
  if (n > 0) k_check_index<<<(unsigned)b, 256, 0, st>>>(idx, n, upper, bad);
}

// ---------------------------------------------------- refined score bound ---
// For every unitary U, Re tr(U^H G_l) <= |G_l|_* (nuclear norm), so
// sum_l |G_l|_* bounds |S(p, R)| as well, and is far tighter than the
// Frobenius form when G_l is close to low rank (as near a template).  It is
// bounded from above without an SVD: for orthonormal q1, q2 and P = [q1 q2]^H
// G_l, R = G_l - [q1 q2] P, |G_l|_* <= |P|_* + sqrt(m - 2) |R|_F (triangle
// inequality; rank R <= m - 2), with |P|_* = sqrt(|P|_F^2 + 2 sqrt(det P P^H))
// in closed form; q1, q2 from one block power step G G^H on the two columns of
// largest norm.  Per degree the smaller of this and sqrt(m) |G_l|_F is kept;
// small margins cover FP32 rounding.  One half-warp per row of X.
__global__ void __launch_bounds__(128) k_so3_refined_bound(const float* __restrict__ X, int ldx, int n,
                                                           const So3Steer* __restrict__ tab, int L,
                                                           float* __restrict__ out) {
  __shared__ uint32_t meta[256];
  __shared__ unsigned char lv[256];
  __shared__ float2 Gs[8][13][13];
  __shared__ float2 Vs[8][2][13];
  const int nent = tab->n;
  for (int i = threadIdx.x; i < nent; i += blockDim.x) {
    meta[i] = tab->meta[i];
    lv[i] = tab->l[i];
  }
  __syncthreads();
  // one voxel per half-warp (m = 2l+1 <= 13 <= 16 lanes)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane & 15, grp = lane >> 4;
  float2(*G)[13] = Gs[warp * 2 + grp];
  float2(*Vw)[13] = Vs[warp * 2 + grp];
  auto hsum = [](float v) {
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  for (int base = (blockIdx.x * 4 + warp) * 2; base < n; base += gridDim.x * 8) {
    const int i = base + grp;
    const bool valid = i < n;
    const float* row = X + (size_t)(valid ? i : base) * ldx;   // the spare half of a warp repeats a real row
    float total = 0.f;
    int e0 = 0;
    for (int l = 0; l <= L; ++l) {
      const int m = 2 * l + 1;
      int e1 = e0;
      while (e1 < nent && lv[e1] == l) ++e1;
      __syncwarp();
      for (int e = e0 + sub; e < e1; e += 16) {
        const uint32_t mt = meta[e];
        const int ks = (int)((mt >> 11) & 31u) - 12, kd = (int)((mt >> 16) & 31u) - 12;
        const int a = (ks - kd) / 2, b = (ks + kd) / 2, ch = mt & 1023u;
        const float2 g = (mt & (1u << 10)) ? make_float2(row[ch], 0.f) : make_float2(row[ch], row[ch + 1]);
        const float sg = ((a + b) & 1) ? -1.f : 1.f;
        G[a + l][b + l] = g;
        G[-a + l][-b + l] = make_float2(sg * g.x, -sg * g.y);
      }
      __syncwarp();
      e0 = e1;
      float cn = -1.f;
      if (sub < m) {
        cn = 0.f;
        for (int r = 0; r < m; ++r) cn += G[r][sub].x * G[r][sub].x + G[r][sub].y * G[r][sub].y;
      }
      const float fro2 = hsum(sub < m ? cn : 0.f);
      const float fro_bound = sqrtf((float)m * fro2);
      if (m == 1) {
        total += sqrtf(fro2);
        continue;
      }
      // the two columns of largest norm
      float best = cn;
      int j1 = sub;
      for (int o = 8; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
        if (ob > best || (ob == best && oj < j1)) { best = ob; j1 = oj; }
      }
      best = (sub == j1) ? -1.f : cn;
      int j2 = sub;
      for (int o = 8; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j2, o);
        if (ob > best || (ob == best && oj < j2)) { best = ob; j2 = oj; }
      }
      // w_t = G^H g_{j_t} (sub = column), v_t = G w_t (sub = row)
      float2 w1 = make_float2(0.f, 0.f), w2 = make_float2(0.f, 0.f);
      if (sub < m) {
        for (int r = 0; r < m; ++r) {
          const float2 gr = G[r][sub], a1 = G[r][j1], a2 = G[r][j2];
          w1.x += gr.x * a1.x + gr.y * a1.y;
          w1.y += gr.x * a1.y - gr.y * a1.x;
          w2.x += gr.x * a2.x + gr.y * a2.y;
          w2.y += gr.x * a2.y - gr.y * a2.x;
        }
        Vw[0][sub] = w1;
        Vw[1][sub] = w2;
      }
      __syncwarp();
      float2 v1 = make_float2(0.f, 0.f), v2 = make_float2(0.f, 0.f);
      if (sub < m) {
        for (int j = 0; j < m; ++j) {
          const float2 g = G[sub][j], a1 = Vw[0][j], a2 = Vw[1][j];
          v1.x += g.x * a1.x - g.y * a1.y;
          v1.y += g.x * a1.y + g.y * a1.x;
          v2.x += g.x * a2.x - g.y * a2.y;
          v2.y += g.x * a2.y + g.y * a2.x;
        }
      }
      // Gram-Schmidt, the second vector orthogonalised twice
      const float n1 = sqrtf(hsum(v1.x * v1.x + v1.y * v1.y));
      const float inv1 = n1 > 0.f ? 1.f / n1 : 0.f;
      const float2 q1 = make_float2(v1.x * inv1, v1.y * inv1);
      const float n2raw = sqrtf(hsum(v2.x * v2.x + v2.y * v2.y));
      for (int pass = 0; pass < 2; ++pass) {
        const float dre = hsum(q1.x * v2.x + q1.y * v2.y), dim = hsum(q1.x * v2.y - q1.y * v2.x);
        v2.x -= q1.x * dre - q1.y * dim;
        v2.y -= q1.x * dim + q1.y * dre;
      }
      const float n2 = sqrtf(hsum(v2.x * v2.x + v2.y * v2.y));
      const int k = (n2 > 1e-6f * n2raw && n2 > 0.f) ? 2 : 1;
      const float inv2 = k == 2 ? 1.f / n2 : 0.f;
      const float2 q2 = make_float2(v2.x * inv2, v2.y * inv2);
      __syncwarp();
      if (sub < m) {
        Vw[0][sub] = q1;
        Vw[1][sub] = q2;
      }
      __syncwarp();
      // P = [q1 q2]^H G (sub = column), R = G - [q1 q2] P (sub = row)
      float2 p1 = make_float2(0.f, 0.f), p2 = make_float2(0.f, 0.f);
      if (sub < m) {
        for (int r = 0; r < m; ++r) {
          const float2 g = G[r][sub], a1 = Vw[0][r], a2 = Vw[1][r];
          p1.x += a1.x * g.x + a1.y * g.y;
          p1.y += a1.x * g.y - a1.y * g.x;
          p2.x += a2.x * g.x + a2.y * g.y;
          p2.y += a2.x * g.y - a2.y * g.x;
        }
      }
      const float a11 = hsum(p1.x * p1.x + p1.y * p1.y), a22 = hsum(p2.x * p2.x + p2.y * p2.y);
      const float c_re = hsum(p1.x * p2.x + p1.y * p2.y), c_im = hsum(p1.x * p2.y - p1.y * p2.x);
      float rr = 0.f;
      for (int j = 0; j < m; ++j) {
        const float p1x = __shfl_sync(0xffffffffu, p1.x, j, 16), p1y = __shfl_sync(0xffffffffu, p1.y, j, 16);
        const float p2x = __shfl_sync(0xffffffffu, p2.x, j, 16), p2y = __shfl_sync(0xffffffffu, p2.y, j, 16);
        if (sub < m) {
          const float2 g = G[sub][j];
          const float rx = g.x - (q1.x * p1x - q1.y * p1y) - (q2.x * p2x - q2.y * p2y);
          const float ry = g.y - (q1.x * p1y + q1.y * p1x) - (q2.x * p2y + q2.y * p2x);
          rr += rx * rx + ry * ry;
        }
      }
      rr = hsum(rr);
      const float det = fmaxf(a11 * a22 - (c_re * c_re + c_im * c_im), 0.f) + 4.8e-7f * a11 * a22;
      const float nucP = sqrtf(a11 + a22 + 2.f * sqrtf(det));
      const float defl = nucP * (1.f + 1e-5f) + sqrtf((float)(m - k)) * sqrtf(rr) + 1e-5f * fro_bound;
      total += n1 > 0.f ? fminf(fro_bound, defl) : fro_bound;
    }
    if (sub == 0 && valid) out[i] = total;
  }
}

void launch_so3_refined_bound(const float* X, int ldx, int n, const So3Steer* tab, int L, float* out, int sms,
                              cudaStream_t st) {
  if (n <= 0) return;
  long long b = (n + 7) / 8;
  if (b > (long long)sms * 16) b = (long long)sms * 16;
  k_so3_refined_bound<<<(unsigned)b, 128, 0, st>>>(X, ldx, n, tab, L, out);
}

// Y[i] = X[sel[i]] (rows of ld floats), i < n
__global__ void k_gather_row_copies(const float* __restrict__ X, int ld, const int32_t* __restrict__ sel, int n,
                                    float* __restrict__ Y) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const float* src = X + (size_t)sel[i] * ld;
  for (int c = threadIdx.x; c < ld; c += blockDim.x) Y[(size_t)i * ld + c] = src[c];
}

// y[i] = x[sel[i]]
__global__ void k_gather_int(const int32_t* __restrict__ x, const int32_t* __restrict__ sel, int n,
                             int32_t* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[sel[i]];
}

void launch_gather_row_copies(const float* X, int ld, const int32_t* sel, int n, float* Y, cudaStream_t st) {
  if (n > 0) k_gather_row_copies<<<n, 128, 0, st>>>(X, ld, sel, n, Y);
}

void launch_gather_int(const int32_t* x, const int32_t* sel, int n, int32_t* y, cudaStream_t st) {
  if (n > 0) k_gather_int<<<(n + 255) / 256, 256, 0, st>>>(x, sel, n, y);
}
