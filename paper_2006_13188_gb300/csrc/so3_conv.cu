// SO(3) extended convolution (Eq. Def-EConv with a rotation at every input
// voxel; component form of Sec. 9):
//   O = Re sum over unique (l, a, b) of w (V C^l_ab(R(.))) (*) (f_l^a Y_l^b),
// w = 1 for the self entry (0, 0) and 2 for the others (the (-a, -b) partner
// is the complex conjugate for a real filter).  This file holds the
// modulation of the volume by its own rotation's matrix entries and the
// accumulation of chunked partial results; the transforms are the shared
// FFT passes.
//
// Matrix entries from the unit quaternion (w, x, y, z) of R = R_z(alpha)
// R_y(beta) R_z(gamma) without trigonometric functions: cos(beta/2) =
// |(w, z)|, sin(beta/2) = |(x, y)|, e^{i sigma} = (w + i z) / cos(beta/2),
// e^{i delta} = (y - i x) / sin(beta/2) with sigma = (alpha + gamma)/2 and
// delta = (alpha - gamma)/2; C^l_ab = d^l_ba(beta) e^{-i((a+b) sigma + (b-a)
// delta)}, d^l_ba from Wigner's sum formula (coefficients fixed at compile
// time per entry, so that every table index is a constant and the tables
// live in registers).
#include "internal.h"

#include <algorithm>
#include <utility>

namespace {

constexpr int MOD_THREADS = 128;

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ----- compile-time steering entries (same order as the channel layout:
// for each l the self entry (0, 0), then (0, b > 0), then (a > 0, b = -l..l))
__host__ __device__ constexpr double cfact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// square root by Newton's iteration (x > 0), for constant expressions
__host__ __device__ constexpr double csqrt(double x) {
  if (!(x > 0.0)) return 0.0;
  double r = x > 1.0 ? x : 1.0;
  for (int i = 0; i < 400; ++i) {
    const double n = 0.5 * (r + x / r);
    if (n >= r) break;
    r = n;
  }
  return r;
}

struct WEntry {
  int ns = 0, pc0 = 0, ps0 = 0, ks = 0, kd = 0;
  bool self = false;
  float coef[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
};

// Entry e of degree <= L: C^l_ab = d^l_ba(beta) e^{-i(ks sigma + kd delta)}
// with ks = a + b, kd = b - a, and Wigner's sum formula
//   d^l_ba = sum_s c_s cos(beta/2)^{pc0 - 2j} sin(beta/2)^{ps0 + 2j},  s = smin + j.
__host__ __device__ constexpr WEntry went(int e) {
  int idx = 0;
  for (int l = 0; l <= 6; ++l)
    for (int a = 0; a <= l; ++a)
      for (int b = -l; b <= l; ++b) {
        if (a == 0 && b < 0) continue;
        if (idx++ != e) continue;
        WEntry w;
        const int m = a, mp = b;
        const int smin = m - mp > 0 ? m - mp : 0;
        const int smax = (l + m < l - mp) ? l + m : l - mp;
        w.ns = smax - smin + 1;
        const double pre = csqrt(cfact(l + mp) * cfact(l - mp) * cfact(l + m) * cfact(l - m));
        for (int j = 0; j < w.ns; ++j) {
          const int s = smin + j;
          const double sg = ((mp - m + s) % 2 != 0) ? -1.0 : 1.0;
          w.coef[j] = (float)(sg * pre / (cfact(l + m - s) * cfact(s) * cfact(mp - m + s) * cfact(l - mp - s)));
        }
        w.pc0 = 2 * l + m - mp - 2 * smin;
        w.ps0 = mp - m + 2 * smin;
        w.ks = m + mp;
        w.kd = mp - m;
        w.self = (m == 0 && mp == 0);
        return w;
      }
  return WEntry{};
}

__host__ __device__ constexpr int n_entries(int L) { return (L + 1) * (2 * L * L + 4 * L + 3) / 3; }   // sum_l (2 l (l + 1) + 1)

// Per-voxel powers: pw[k] = cos(beta/2)^k, pw[13 + k] = sin(beta/2)^k,
// es[k] = e^{ik sigma}, ed[k] = e^{ik delta} (k <= 2L), all in registers.
template <int L>
struct VoxelTabs {
  float pw[26];
  float2 es[2 * L + 1], ed[2 * L + 1];
};

template <int L, int E>
__device__ __forceinline__ void mod_entry(const VoxelTabs<L>& t, float val, int e0, int ne, float2* dst, size_t P) {
  if (E < e0 || E >= e0 + ne) return;
  constexpr WEntry w = went(E);
  float d = 0.f;
#pragma unroll
  for (int j = 0; j < w.ns; ++j) d = fmaf(w.coef[j], t.pw[w.pc0 - 2 * j] * t.pw[13 + w.ps0 + 2 * j], d);
  // conj(e^{i ks sigma}) conj(e^{i kd delta})
  const float2 A = w.ks >= 0 ? make_float2(t.es[w.ks].x, -t.es[w.ks].y) : t.es[-w.ks];
  const float2 B = w.kd >= 0 ? make_float2(t.ed[w.kd].x, -t.ed[w.kd].y) : t.ed[-w.kd];
  const float2 E2 = cmul2(A, B);
  const float wv = (w.self ? 1.f : 2.f) * val * d;
  dst[(size_t)(E - e0) * P] = make_float2(wv * E2.x, wv * E2.y);
}

template <int L, int... E>
__device__ __forceinline__ void mod_all(std::integer_sequence<int, E...>, const VoxelTabs<L>& t, float val, int e0,
                                        int ne, float2* dst, size_t P) {
  (mod_entry<L, E>(t, val, e0, ne, dst, P), ...);
}

// One thread per voxel (no grid-stride loop: the per-entry plane offsets
// would be hoisted out of it and exhaust the registers): the voxel's tables
// in registers, then every entry e0 .. e0 + ne - 1, each store of a warp
// covering 32 consecutive voxels of one plane.
template <int L>
__global__ void __launch_bounds__(MOD_THREADS) k_so3_modulate(const float* __restrict__ V,
                                                             const float4* __restrict__ Q, long long P, int e0,
                                                             int ne, float2* __restrict__ U) {
  const long long v = (long long)blockIdx.x * MOD_THREADS + threadIdx.x;
  if (v < P) {
    float4 q = __ldg(Q + v);
    float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    if (!(n2 > 1e-30f)) {   // a zero quaternion acts as the identity
      q = make_float4(1.f, 0.f, 0.f, 0.f);
      n2 = 1.f;
    }
    const float inv = rsqrtf(n2);
    q = make_float4(q.x * inv, q.y * inv, q.z * inv, q.w * inv);   // (w, x, y, z) in (x, y, z, w)
    const float cb = sqrtf(q.x * q.x + q.w * q.w), sb = sqrtf(q.y * q.y + q.z * q.z);
    const float2 s1 = cb > 1e-12f ? make_float2(q.x / cb, q.w / cb) : make_float2(1.f, 0.f);
    const float2 d1 = sb > 1e-12f ? make_float2(q.z / sb, -q.y / sb) : make_float2(1.f, 0.f);
    VoxelTabs<L> t;
    float pc = 1.f, ps = 1.f;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
      t.pw[k] = pc;
      t.pw[13 + k] = ps;
      pc *= cb;
      ps *= sb;
    }
    float2 zs = make_float2(1.f, 0.f), zd = make_float2(1.f, 0.f);
#pragma unroll
    for (int k = 0; k <= 2 * L; ++k) {
      t.es[k] = zs;
      t.ed[k] = zd;
      zs = cmul2(zs, s1);
      zd = cmul2(zd, d1);
    }
    mod_all<L>(std::make_integer_sequence<int, n_entries(L)>{}, t, __ldg(V + v), e0, ne, U + v, (size_t)P);
  }
}

__global__ void k_add_complex(float2* __restrict__ acc, const float2* __restrict__ y, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float2 a = acc[i], b = __ldg(y + i);
    acc[i] = make_float2(a.x + b.x, a.y + b.y);
  }
}

}  // namespace

void launch_so3_modulate(const float* V, const float* Q, long long P, int L, int e0, int ne, float2* U,
                         cudaStream_t st) {
  if (P <= 0 || ne <= 0) return;
  const long long blocks = (P + MOD_THREADS - 1) / MOD_THREADS;
  const float4* q = reinterpret_cast<const float4*>(Q);
  switch (L) {
#define EXT_MOD(LL) \
  case LL: k_so3_modulate<LL><<<(unsigned)blocks, MOD_THREADS, 0, st>>>(V, q, P, e0, ne, U); break;
    EXT_MOD(0) EXT_MOD(1) EXT_MOD(2) EXT_MOD(3) EXT_MOD(4) EXT_MOD(5) EXT_MOD(6)
#undef EXT_MOD
    default: break;
  }
}

void launch_add_complex(float2* acc, const float2* y, long long n, int sms, cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)sms * 8);
  k_add_complex<<<blocks, 256, 0, st>>>(acc, y, n);
}
