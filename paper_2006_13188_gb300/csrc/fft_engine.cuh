// Shared-memory FP32 FFT engine (device side).
//
// The paper computes every standard correlation/convolution of Sec. 4.1
// ("Standard Correlation") with the 2D FFT.  This engine performs the 1D
// transforms those 2D FFTs are made of, for many lines at once, inside one
// thread block:
//
//   * Stockham autosort formulation, mixed radix.  A length n = R_0 R_1 ...
//     is processed in stages; stage s with radix R and span Ns = R_0..R_{s-1}
//     reads R values j + r n/R, multiplies value r by W_{Ns R}^{r (j mod Ns)},
//     takes a length-R DFT, and writes the results to
//     (j / Ns) Ns R + (j mod Ns) + r Ns.  No bit reversal is needed.
//   * Radices 16, 8, 4, 2 (hand-written butterflies) and 3, 5, 7, 11, 13
//     (direct DFTs with symmetric pairing), so every image side of the form
//     2^a 3^b 5^c 7^d 11^e 13^f is supported.
//   * Twiddles come from a per-length table W_n^m = exp(-2 pi i m / n),
//     m in [0, n), computed in FP64 and rounded once to FP32.
//   * In place: every thread loads all of its butterfly inputs for a stage
//     into registers, the block synchronises, and the outputs are written
//     back.  A thread holds at most ceil(FFT_MAXE / R) butterflies, so the
//     block must have at least nlines * n / FFT_MAXE threads.
//   * Element i of line l lives at buf[l * ls + sidx(i) * es]; sidx inserts
//     one padding slot every 16 elements to spread the strided Stockham
//     accesses over the shared-memory banks.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#define FFT_MAXE 16
#define FFT_MAX_STAGES 12

struct FftLine {
  int n;                        // line length
  int nst;                      // number of stages
  int radix[FFT_MAX_STAGES];    // radices in application order
  const float2* tw;             // W_n^m, m in [0, n)
};

__device__ __forceinline__ int sidx(int i) { return i + (i >> 4); }
__host__ __device__ inline int sidx_len(int n) { return n + ((n - 1) >> 4) + 1; }

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 c_rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------------ small DFTs ---
template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 s02 = c_add(x0, x2), d02 = c_sub(x0, x2);
  float2 s13 = c_add(x1, x3), d13 = c_rot<INV>(c_sub(x1, x3));
  x0 = c_add(s02, s13);
  x2 = c_sub(s02, s13);
  x1 = c_add(d02, d13);
  x3 = c_sub(d02, d13);
}

// exp(-2 pi i m / 16): cosine and sine parts (constant-folded after unrolling)
__host__ __device__ constexpr float w16c(int m) {
  constexpr float c[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                           0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                           -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                           0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
  return c[m & 15];
}
__host__ __device__ constexpr float w16s(int m) {
  constexpr float s[16] = {0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                           -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                           0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                           1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};
  return s[m & 15];
}

template <bool INV>
__device__ __forceinline__ float2 tw16(float2 a, int m) {
  // a * W16^m (forward) or a * conj(W16^m) (inverse); m is a compile-time constant after unrolling
  const float c = w16c(m);
  const float s = INV ? -w16s(m) : w16s(m);
  return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* v) {
  float2 t = v[0];
  v[0] = c_add(t, v[1]);
  v[1] = c_sub(t, v[1]);
}

template <bool INV>
__device__ __forceinline__ void dft4v(float2* v) { dft4<INV>(v[0], v[1], v[2], v[3]); }

// n = 2 n1 + n2 : inner DFT-4 over n1, twiddle W8^{n2 k1}, outer DFT-2 over n2.
template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  float2 a0 = v[0], a1 = v[2], a2 = v[4], a3 = v[6];
  float2 b0 = v[1], b1 = v[3], b2 = v[5], b3 = v[7];
  dft4<INV>(a0, a1, a2, a3);
  dft4<INV>(b0, b1, b2, b3);
  b1 = tw16<INV>(b1, 2);
  b2 = tw16<INV>(b2, 4);
  b3 = tw16<INV>(b3, 6);
  v[0] = c_add(a0, b0); v[4] = c_sub(a0, b0);
  v[1] = c_add(a1, b1); v[5] = c_sub(a1, b1);
  v[2] = c_add(a2, b2); v[6] = c_sub(a2, b2);
  v[3] = c_add(a3, b3); v[7] = c_sub(a3, b3);
}

// n = 4 n1 + n2 : DFT-4 over n1, twiddle W16^{n2 k1}, DFT-4 over n2.
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  float2 a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    a[n2][0] = v[n2]; a[n2][1] = v[4 + n2]; a[n2][2] = v[8 + n2]; a[n2][3] = v[12 + n2];
    dft4<INV>(a[n2][0], a[n2][1], a[n2][2], a[n2][3]);
  }
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) a[n2][k1] = tw16<INV>(a[n2][k1], n2 * k1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 x0 = a[0][k1], x1 = a[1][k1], x2 = a[2][k1], x3 = a[3][k1];
    dft4<INV>(x0, x1, x2, x3);
    v[k1] = x0; v[k1 + 4] = x1; v[k1 + 8] = x2; v[k1 + 12] = x3;
  }
}

// cos / sin of 2 pi m / R for the odd radices (constant-folded after unrolling)
template <int R> __host__ __device__ constexpr float odd_c(int m);
template <int R> __host__ __device__ constexpr float odd_s(int m);
template <> __host__ __device__ constexpr float odd_c<3>(int m) {
  constexpr float t[3] = {1.0f, -0.5f, -0.5f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_s<3>(int m) {
  constexpr float t[3] = {0.0f, 8.660254038e-01f, -8.660254038e-01f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_c<5>(int m) {
  constexpr float t[5] = {1.0f, 3.090169944e-01f, -8.090169944e-01f, -8.090169944e-01f, 3.090169944e-01f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_s<5>(int m) {
  constexpr float t[5] = {0.0f, 9.510565163e-01f, 5.877852523e-01f, -5.877852523e-01f, -9.510565163e-01f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_c<7>(int m) {
  constexpr float t[7] = {1.0f, 6.234898019e-01f, -2.225209340e-01f, -9.009688679e-01f,
                                 -9.009688679e-01f, -2.225209340e-01f, 6.234898019e-01f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_s<7>(int m) {
  constexpr float t[7] = {0.0f, 7.818314825e-01f, 9.749279122e-01f, 4.338837391e-01f,
                                 -4.338837391e-01f, -9.749279122e-01f, -7.818314825e-01f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_c<11>(int m) {
  constexpr float t[11] = {1.0f, 8.412535328e-01f, 4.154150130e-01f, -1.423148383e-01f,
                                  -6.548607339e-01f, -9.594929736e-01f, -9.594929736e-01f, -6.548607339e-01f,
                                  -1.423148383e-01f, 4.154150130e-01f, 8.412535328e-01f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_s<11>(int m) {
  constexpr float t[11] = {0.0f, 5.406408175e-01f, 9.096319954e-01f, 9.898214419e-01f,
                                  7.557495744e-01f, 2.817325568e-01f, -2.817325568e-01f, -7.557495744e-01f,
                                  -9.898214419e-01f, -9.096319954e-01f, -5.406408175e-01f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_c<13>(int m) {
  constexpr float t[13] = {1.0f, 8.854560257e-01f, 5.680647467e-01f, 1.205366803e-01f,
                                  -3.546048870e-01f, -7.485107482e-01f, -9.709418174e-01f, -9.709418174e-01f,
                                  -7.485107482e-01f, -3.546048870e-01f, 1.205366803e-01f, 5.680647467e-01f,
                                  8.854560257e-01f};
  return t[m];
}
template <> __host__ __device__ constexpr float odd_s<13>(int m) {
  constexpr float t[13] = {0.0f, 4.647231720e-01f, 8.229838659e-01f, 9.927088741e-01f,
                                  9.350162427e-01f, 6.631226582e-01f, 2.393156643e-01f, -2.393156643e-01f,
                                  -6.631226582e-01f, -9.350162427e-01f, -9.927088741e-01f, -8.229838659e-01f,
                                  -4.647231720e-01f};
  return t[m];
}

// y_m = sum_r v_r exp(-/+ 2 pi i r m / R), pairing r and R - r:
// v_r e^{-i t} + v_{R-r} e^{i t} = (v_r + v_{R-r}) cos t - i (v_r - v_{R-r}) sin t.
template <int R, bool INV>
__device__ __forceinline__ void dft_odd(float2* v) {
  constexpr int H = (R - 1) / 2;
  float2 sum[H + 1], dif[H + 1];
  float2 y0 = v[0];
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    sum[r] = c_add(v[r], v[R - r]);
    dif[r] = c_sub(v[r], v[R - r]);
    y0 = c_add(y0, sum[r]);
  }
  float2 out[R];
  out[0] = y0;
#pragma unroll
  for (int m = 1; m < R; ++m) {
    float2 acc = v[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const float c = odd_c<R>((r * m) % R);
      const float s = odd_s<R>((r * m) % R);
      acc.x = fmaf(sum[r].x, c, acc.x);
      acc.y = fmaf(sum[r].y, c, acc.y);
      if (INV) {
        acc.x = fmaf(-dif[r].y, s, acc.x);
        acc.y = fmaf(dif[r].x, s, acc.y);
      } else {
        acc.x = fmaf(dif[r].y, s, acc.x);
        acc.y = fmaf(-dif[r].x, s, acc.y);
      }
    }
    out[m] = acc;
  }
#pragma unroll
  for (int m = 0; m < R; ++m) v[m] = out[m];
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) dft2<INV>(v);
  else if constexpr (R == 4) dft4v<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
  else dft_odd<R, INV>(v);
}

// ------------------------------------------------------------- one stage ---
// LINE_FAST: consecutive threads take consecutive lines (column tiles, where
// lines are adjacent in memory); otherwise consecutive butterflies of a line.
template <int R, bool INV, bool LINE_FAST>
__device__ __noinline__ void fft_stage(float2* buf, int n, int nlines, int ls, int es, int Ns,
                                          const float2* __restrict__ tw) {
  constexpr int S = (FFT_MAXE + R - 1) / R;
  const int nb = n / R;
  const int total = nb * nlines;
  const int tstep = n / (Ns * R);
  float2 v[S][R];
  int base_s[S], dst_s[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int it = threadIdx.x + s * blockDim.x;
    base_s[s] = -1;
    if (it < total) {
      int line, j;
      if (LINE_FAST) { line = it % nlines; j = it / nlines; }
      else { j = it % nb; line = it / nb; }
      const int k = j % Ns;
      float2* base = buf + line * ls;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 a = base[sidx(j + r * nb) * es];
        if (r > 0 && k > 0) {
          float2 w = __ldg(tw + r * k * tstep);
          if (INV) w.y = -w.y;
          a = c_mul(a, w);
        }
        v[s][r] = a;
      }
      base_s[s] = line * ls;
      dst_s[s] = (j / Ns) * Ns * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if (base_s[s] >= 0) {
      dft<R, INV>(v[s]);
      float2* base = buf + base_s[s];
#pragma unroll
      for (int r = 0; r < R; ++r) base[sidx(dst_s[s] + r * Ns) * es] = v[s][r];
    }
  }
  __syncthreads();
}

// Whole transform of `nlines` lines.  Caller must __syncthreads() after
// filling `buf`; on return the result is in `buf` and visible to all threads.
template <bool INV, bool LINE_FAST>
__device__ void fft_lines(float2* buf, const FftLine& L, int nlines, int ls, int es) {
  int Ns = 1;
  for (int st = 0; st < L.nst; ++st) {
    const int R = L.radix[st];
    switch (R) {
      case 16: fft_stage<16, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      case 8: fft_stage<8, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      case 4: fft_stage<4, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      case 2: fft_stage<2, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      case 3: fft_stage<3, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      case 5: fft_stage<5, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      case 7: fft_stage<7, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      case 11: fft_stage<11, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      case 13: fft_stage<13, INV, LINE_FAST>(buf, L.n, nlines, ls, es, Ns, L.tw); break;
      default: break;
    }
    Ns *= R;
  }
}
