// 2D FFT passes with the extended-convolution/correlation work fused into
// their loads and stores (Sec. 4.1).  Every kernel is a template on the 1D
// length N it transforms, so that the Stockham stages unroll completely.
//
// Layouts (all row-major, x = column index fastest):
//   H      real signal, h x w floats
//   Hh     half spectrum of H after the row and column passes,
//          h x (w/2 + 1) complex  (Hermitian: H^(-u,-v) = conj(H^(u,v)))
//   S_k    filter-component spectra in column tiles of width CW(h):
//          S[k][tile][v][c] = (scaled, possibly conjugated) F^_k(tile*CW + c, v)
//   Z      k-chunk of partially inverted products, nk x h x w complex
//   G      component correlations, (2K+1) planes of P = h*w floats:
//          plane 0 = G_0, plane 2k-1 = Re G_k, plane 2k = Im G_k (k >= 1)
#pragma once
#include "fft_engine.cuh"
#include "tc_common.cuh"
#include "../../include/extconv.h"

#include <cuda.h>

// ---------------------------------------------------------- compile time ---
struct RadixList {
  int cnt;
  int r[FFT_MAX_STAGES];
};

__host__ __device__ constexpr RadixList factor_radices(int n) {
  RadixList L{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
  int m = n;
  const int odd[5] = {13, 11, 7, 5, 3};
  for (int i = 0; i < 5; ++i)
    while (m % odd[i] == 0 && L.cnt < FFT_MAX_STAGES) { L.r[L.cnt++] = odd[i]; m /= odd[i]; }
  while (m % 16 == 0 && L.cnt < FFT_MAX_STAGES) { L.r[L.cnt++] = 16; m /= 16; }
  if (m % 8 == 0) { L.r[L.cnt++] = 8; m /= 8; }
  if (m % 4 == 0) { L.r[L.cnt++] = 4; m /= 4; }
  if (m % 2 == 0) { L.r[L.cnt++] = 2; m /= 2; }
  return L;
}

__host__ __device__ constexpr int ct_sidx_len(int n) { return n + ((n - 1) >> 4) + 1; }

template <int N>
struct LineCfg {
  static constexpr int TPL = (N + FFT_MAXE - 1) / FFT_MAXE;   // threads per line
  static constexpr int LS = ct_sidx_len(N);                   // padded line length
  // row passes: RL lines per block; column passes: CW adjacent columns per block
  static constexpr int RL = (8192 / N) < 1 ? 1 : ((8192 / N) > 16 ? 16 : (8192 / N));
  static constexpr int CW = RL;
  static constexpr int ROW_THREADS = ((RL * TPL + 31) / 32) * 32;
  static constexpr int TW_BYTES = N * 8;   // twiddle table copy in shared memory
  static constexpr int ROW_SMEM = RL * LS * 8 + TW_BYTES;
  static constexpr int ROW_EPT = (RL * N + ROW_THREADS - 1) / ROW_THREADS;
  static constexpr int COL_THREADS = ((CW * TPL + 31) / 32) * 32;
  static constexpr int COL_SMEM = CW * LS * 8 + TW_BYTES;
  static constexpr int COL_EPT = (CW * N + COL_THREADS - 1) / COL_THREADS;
  // blocks per SM the register budget is sized for
  static constexpr int ROW_MINB = ROW_THREADS >= 512 ? 2 : 1;
  static constexpr int COL_MINB = COL_THREADS >= 512 ? 2 : 1;
};

// Visit the elements of a block's lines: element e = threadIdx.x + i * THREADS,
// i < EPT, all indices compile-time except threadIdx.x.  fn(i, e).
template <int TOTAL, int THREADS, class Fn>
__device__ __forceinline__ void for_elems(Fn&& fn) {
  constexpr int EPT = (TOTAL + THREADS - 1) / THREADS;
#pragma unroll
  for (int i = 0; i < EPT; ++i) {
    const int e = threadIdx.x + i * THREADS;
    if (TOTAL % THREADS == 0 || e < TOTAL) fn(i, e);
  }
}

// Same visit in chunks of G elements per thread: load(i, e) for the whole
// chunk first (so G loads are in flight together), then store(i, e).
template <int TOTAL, int THREADS, int G, class Load, class Store>
__device__ __forceinline__ void for_elems_staged(Load&& load, Store&& store) {
  constexpr int EPT = (TOTAL + THREADS - 1) / THREADS;
#pragma unroll
  for (int i0 = 0; i0 < EPT; i0 += G) {
#pragma unroll
    for (int i = i0; i < i0 + G && i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      if (TOTAL % THREADS == 0 || e < TOTAL) load(i - i0, e);
    }
#pragma unroll
    for (int i = i0; i < i0 + G && i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      if (TOTAL % THREADS == 0 || e < TOTAL) store(i - i0, e);
    }
  }
}

constexpr int STAGE_G = 8;

// Twiddle sources of the stages: the stage table (see stage_twiddles), or a
// split table W_N^m = lo[m mod 64] hi[m / 64] (64 + N / 64 entries, one
// extra complex product per twiddle) for passes whose shared memory has no
// room for the N - 1 entries of the stage table.
struct SplitTw {
  const float2* lo;
  const float2* hi;
};
template <int NS, int STEP>
__device__ __forceinline__ float2 tw_get(const float2* __restrict__ t, int r, int k) {
  return t[r * NS - 1 + k];
}
template <int NS, int STEP>
__device__ __forceinline__ float2 tw_get(const SplitTw& t, int r, int k) {
  const int m = r * k * STEP;
  return c_mul(t.lo[m & 63], t.hi[m >> 6]);
}

template <int N, int R, int NS, bool INV, bool LINE_FAST, int NLINES, int THREADS, class TWT>
__device__ __forceinline__ void ct_stage(float2* buf, int ls, int es, TWT tw) {
  constexpr int NB = N / R;
  constexpr int TSTEP = N / (NS * R);
  constexpr int total = NB * NLINES;
  constexpr int S = (total + THREADS - 1) / THREADS;
  static_assert(S * R <= FFT_MAXE + R, "too many butterflies per thread");
  constexpr int nlines = NLINES;
  float2 v[S][R];
  int base_s[S], dst_s[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int it = threadIdx.x + s * THREADS;
    base_s[s] = -1;
    dst_s[s] = 0;
    if (it < total) {
      int line, j;
      if (LINE_FAST) { line = it % nlines; j = it / nlines; }
      else { j = it % NB; line = it / NB; }
      const int k = j % NS;
      const float2* base = buf + line * ls;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 a = base[sidx(j + r * NB) * es];
        if (NS > 1 && r > 0) {
          float2 w = tw_get<NS, TSTEP>(tw, r, k);
          if (INV) w.y = -w.y;
          a = c_mul(a, w);
        }
        v[s][r] = a;
      }
      base_s[s] = line * ls;
      dst_s[s] = (j / NS) * NS * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if (base_s[s] >= 0) {
      dft<R, INV>(v[s]);
      float2* base = buf + base_s[s];
#pragma unroll
      for (int r = 0; r < R; ++r) base[sidx(dst_s[s] + r * NS) * es] = v[s][r];
    }
  }
  __syncthreads();
}

template <int N, bool INV, bool LINE_FAST, int NLINES, int THREADS, int ST = 0, int NS = 1, class TWT>
__device__ __forceinline__ void ct_fft(float2* buf, int ls, int es, TWT tw) {
  constexpr RadixList L = factor_radices(N);
  if constexpr (ST < L.cnt) {
    constexpr int R = L.r[ST];
    ct_stage<N, R, NS, INV, LINE_FAST, NLINES, THREADS>(buf, ls, es, tw);
    ct_fft<N, INV, LINE_FAST, NLINES, THREADS, ST + 1, NS * R>(buf, ls, es, tw);
  }
}

// Stages ST .. END-1 of the transform (in place, as ct_fft).
template <int N, bool INV, bool LINE_FAST, int NLINES, int THREADS, int ST, int END, int NS, class TWT>
__device__ __forceinline__ void ct_fft_range(float2* buf, int ls, int es, TWT tw) {
  constexpr RadixList L = factor_radices(N);
  if constexpr (ST < END) {
    constexpr int R = L.r[ST];
    ct_stage<N, R, NS, INV, LINE_FAST, NLINES, THREADS>(buf, ls, es, tw);
    ct_fft_range<N, INV, LINE_FAST, NLINES, THREADS, ST + 1, END, NS * R>(buf, ls, es, tw);
  }
}

// Output (line, x) of butterfly s, value r of the last forward stage of a
// column transform (LINE_FAST: line = it mod NLINES); valid() is false for
// butterflies past the end.
template <int N, int NLINES, int THREADS>
struct LastColStage {
  static constexpr RadixList L = factor_radices(N);
  static constexpr int R = L.r[L.cnt - 1];
  static constexpr int NS = N / R;
  static constexpr int NB = N / R;
  static constexpr int TOTAL = NB * NLINES;
  static constexpr int S = (TOTAL + THREADS - 1) / THREADS;
  __device__ static __forceinline__ bool valid(int s) {
    return TOTAL % THREADS == 0 || (int)threadIdx.x + s * THREADS < TOTAL;
  }
  __device__ static __forceinline__ int line(int s) { return ((int)threadIdx.x + s * THREADS) % NLINES; }
  // NS R = N, so the butterfly's first output is j itself
  __device__ static __forceinline__ int x(int s, int r) { return ((int)threadIdx.x + s * THREADS) / NLINES + r * NS; }
};

// The last forward stage of a column transform (buf in the column layout,
// line stride 1, element stride es), its outputs handed to fn(s, r, value)
// instead of being stored; s and r are compile-time after unrolling.
template <int N, int NLINES, int THREADS, class TWT, class Fn>
__device__ __forceinline__ void ct_last_stage_cols(const float2* buf, int es, TWT tw, Fn&& fn) {
  using LS_ = LastColStage<N, NLINES, THREADS>;
  constexpr int R = LS_::R, NS = LS_::NS, NB = LS_::NB;
#pragma unroll
  for (int s = 0; s < LS_::S; ++s) {
    if (LS_::valid(s)) {
      const int it = threadIdx.x + s * THREADS;
      const int line = it % NLINES, j = it / NLINES;
      const int k = j % NS;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 a = buf[line + sidx(j + r * NB) * es];
        if (NS > 1 && r > 0) a = c_mul(a, tw_get<NS, 1>(tw, r, k));
        v[r] = a;
      }
      dft<R, false>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) fn(s, r, v[r]);
    }
  }
}

// Stage with functor I/O: load(line, idx) supplies the inputs (FIRST: from
// anywhere, e.g. a staging buffer with a product fused in; INPLACE_FIRST: the
// first stage's loads read buf itself, so all reads finish before any write)
// and store(line, idx, value) consumes the outputs (LAST: e.g. straight to
// global memory); otherwise both use the padded shared-memory layout of buf.
template <int N, int R, int NS, bool INV, bool LINE_FAST, int NLINES, int THREADS, bool FIRST, bool LAST,
          bool INPLACE_FIRST = false, class TWT, class Load, class Store>
__device__ __forceinline__ void ct_stage_io(float2* buf, int ls, int es, TWT tw, Load&& load,
                                            Store&& store) {
  constexpr int NB = N / R;
  constexpr int TSTEP = N / (NS * R);
  constexpr int total = NB * NLINES;
  constexpr int S = (total + THREADS - 1) / THREADS;
  static_assert(S * R <= FFT_MAXE + R, "too many butterflies per thread");
  float2 v[S][R];
  int line_s[S], dst_s[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int it = threadIdx.x + s * THREADS;
    line_s[s] = -1;
    dst_s[s] = 0;
    if (total % THREADS == 0 || it < total) {
      int line, j;
      if (LINE_FAST) { line = it % NLINES; j = it / NLINES; }
      else { j = it % NB; line = it / NB; }
      const int k = j % NS;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 a = FIRST ? load(line, j + r * NB) : buf[line * ls + sidx(j + r * NB) * es];
        if (NS > 1 && r > 0) {
          float2 w = tw_get<NS, TSTEP>(tw, r, k);
          if (INV) w.y = -w.y;
          a = c_mul(a, w);
        }
        v[s][r] = a;
      }
      line_s[s] = line;
      dst_s[s] = (j / NS) * NS * R + k;
    }
  }
  if ((!FIRST || INPLACE_FIRST) && !LAST) __syncthreads();   // in place: all reads before any write
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if (line_s[s] >= 0) {
      dft<R, INV>(v[s]);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (LAST) store(line_s[s], dst_s[s] + r * NS, v[s][r]);
        else buf[line_s[s] * ls + sidx(dst_s[s] + r * NS) * es] = v[s][r];
      }
    }
  }
  if (!LAST) __syncthreads();
}

// Whole transform with functor input (first stage) and output (last stage).
// The caller must __syncthreads() before re-using buf or the load source.
template <int N, bool INV, bool LINE_FAST, int NLINES, int THREADS, int ST = 0, int NS = 1, class TWT, class Load,
          class Store>
__device__ __forceinline__ void ct_fft_io(float2* buf, int ls, int es, TWT tw, Load&& load, Store&& store) {
  constexpr RadixList L = factor_radices(N);
  if constexpr (ST < L.cnt) {
    constexpr int R = L.r[ST];
    ct_stage_io<N, R, NS, INV, LINE_FAST, NLINES, THREADS, ST == 0, ST == L.cnt - 1>(buf, ls, es, tw, load, store);
    ct_fft_io<N, INV, LINE_FAST, NLINES, THREADS, ST + 1, NS * R>(buf, ls, es, tw, load, store);
  }
}

// ------------------------------------------------------------- cp.async ---
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;   // 0 source bytes: the 16 destination bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Builds the per-stage twiddle tables in shared memory right after the
// block's data region and returns them (the caller's next __syncthreads makes
// them visible).  The stage with span NS and radix R needs
// W_N^(r k N / (NS R)) for r = 1..R-1, k = 0..NS-1; it is stored at
// r * NS - 1 + k, contiguous in k so that adjacent butterflies read adjacent
// words.  The stage blocks telescope to N - 1 entries in total.  Values are
// copied from the FP64-derived table W_N^m = exp(-2 pi i m / N).
// Product of the radices before stage S.
__host__ __device__ constexpr int radix_prefix(int n, int S) {
  int p = 1;
  const RadixList L = factor_radices(n);
  for (int i = 0; i < S; ++i) p *= L.r[i];
  return p;
}

// Stage table of the Stockham passes: for stage s (NS = product of the
// earlier radices, radix R), entry NS - 1 + (r - 1) NS + k = w^(r k N / (NS R)),
// 1 <= r < R, 0 <= k < NS; N - 1 entries.  Filled stage by stage so every
// division is by a compile-time constant.
template <int N, int S>
__device__ __forceinline__ void stage_twiddles_fill(float2* t, const float2* __restrict__ tw, int threads) {
  constexpr RadixList L = factor_radices(N);
  if constexpr (S < L.cnt) {
    constexpr int NS = radix_prefix(N, S);
    constexpr int R = L.r[S];
    constexpr int STEP = N / (NS * R);
    for (int e = threadIdx.x; e < (R - 1) * NS; e += threads) {
      const int r = e / NS + 1, k = e % NS;
      t[NS - 1 + e] = __ldg(tw + r * k * STEP);
    }
    stage_twiddles_fill<N, S + 1>(t, tw, threads);
  }
}

template <int N, int DATA_ELEMS>
__device__ __forceinline__ const float2* stage_twiddles(float2* sm, const float2* __restrict__ tw, int threads) {
  float2* t = sm + DATA_ELEMS;
  stage_twiddles_fill<N, 0>(t, tw, threads);
  return t;
}

// Row layout: line l, element x at sm[l * LS + sidx(x)].
template <int N, bool INV>
__device__ __forceinline__ void row_fft(float2* sm, const float2* tw) {
  using C = LineCfg<N>;
  ct_fft<N, INV, false, C::RL, C::ROW_THREADS>(sm, C::LS, 1, tw);
}
// Column layout: column c, element v at sm[c + sidx(v) * CW].
template <int N, bool INV, class TWT>
__device__ __forceinline__ void col_fft(float2* sm, TWT tw) {
  using C = LineCfg<N>;
  ct_fft<N, INV, true, C::CW, C::COL_THREADS>(sm, 1, C::CW, tw);
}

// exp(i k alpha) for an FP32 angle: k*alpha is formed exactly as p + e
// (two-product with an FMA), reduced by an additive three-part split of 2 pi
// (Cody & Waite's argument reduction), and only then passed to sincosf.
__device__ __forceinline__ void sincos_kalpha(int k, float alpha, float* s, float* c) {
  const float kf = (float)k;
  const float p = kf * alpha;
  const float e = fmaf(kf, alpha, -p);
  const float n = rintf(p * 0.15915494309189535f);
  float r = fmaf(-n, 6.28125f, p);
  r = fmaf(-n, 0.0019353071693331003f, r);
  r = fmaf(-n, 1.0253131677018246e-11f, r);
  r += e;
  sincosf(r, s, c);
}

// The same reduction with the remainder (|r| <= pi + |e|) passed to
// sincospif as r / pi: branch-free, so loads ahead of it can be hoisted; the
// extra rounding of r / pi adds at most about 3e-7 rad.
__device__ __forceinline__ void sincos_kalpha_pi(int k, float alpha, float* s, float* c) {
  const float kf = (float)k;
  const float p = kf * alpha;
  const float e = fmaf(kf, alpha, -p);
  const float n = rintf(p * 0.15915494309189535f);
  float r = fmaf(-n, 6.28125f, p);
  r = fmaf(-n, 0.0019353071693331003f, r);
  r = fmaf(-n, 1.0253131677018246e-11f, r);
  r += e;
  sincospif(r * 0.31830988618379067f, s, c);
}

// The same reduction with the remainder (|r| <= pi + |e|) passed to the
// hardware sine and cosine (__sincosf): absolute error about 4e-7.
__device__ __forceinline__ void sincos_kalpha_fast(int k, float alpha, float* s, float* c) {
  const float kf = (float)k;
  const float p = kf * alpha;
  const float e = fmaf(kf, alpha, -p);
  const float n = rintf(p * 0.15915494309189535f);
  float r = fmaf(-n, 6.28125f, p);
  r = fmaf(-n, 0.0019353071693331003f, r);
  r = fmaf(-n, 1.0253131677018246e-11f, r);
  r += e;
  __sincosf(r, s, c);
}

// exp(i w x) for FP32 w, x: the product is formed exactly as p + e and
// reduced like sincos_kalpha.
__device__ __forceinline__ void sincos_wx(float wk, float x, float* s, float* c) {
  const float p = wk * x;
  const float e = fmaf(wk, x, -p);
  const float n = rintf(p * 0.15915494309189535f);
  float r = fmaf(-n, 6.28125f, p);
  r = fmaf(-n, 0.0019353071693331003f, r);
  r = fmaf(-n, 1.0253131677018246e-11f, r);
  r += e;
  sincosf(r, s, c);
}

// ------------------------------------------------------------ row passes ---
// All global loads of a block are first gathered into registers (every
// thread has its EPT loads in flight at once), then written to shared memory.

// Forward real-to-complex transform of the rows of H, two rows per complex
// line: z = H[2p] + i H[2p+1], Z = FFT(z), then
//   X_even[u] = (Z[u] + conj Z[-u]) / 2,  X_odd[u] = -i (Z[u] - conj Z[-u]) / 2.
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_r2c(const float* __restrict__ H, int h, float2* __restrict__ Hh, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::ROW_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  const int pair0 = blockIdx.x * C::RL;
  float2 v[STAGE_G];
  for_elems_staged<C::RL * N, T, STAGE_G>(
      [&](int i, int e) {
        const int l = e / N, x = e % N;
        const int y0 = 2 * (pair0 + l);
        v[i].x = (y0 < h) ? __ldg(H + (size_t)y0 * N + x) : 0.f;
        v[i].y = (y0 + 1 < h) ? __ldg(H + (size_t)(y0 + 1) * N + x) : 0.f;
      },
      [&](int i, int e) { sm[(e / N) * C::LS + sidx(e % N)] = v[i]; });
  __syncthreads();
  row_fft<N, false>(sm, twl);
  constexpr int WH = N / 2 + 1;
  for_elems<C::RL * WH, T>([&](int i, int e) {
    const int l = e / WH, u = e % WH;
    const int y0 = 2 * (pair0 + l);
    if (y0 >= h) return;
    const float2 z = sm[l * C::LS + sidx(u)];
    const float2 zm = c_conj(sm[l * C::LS + sidx((N - u) % N)]);
    const float2 x0 = c_scale(c_add(z, zm), 0.5f);
    const float2 d = c_scale(c_sub(z, zm), 0.5f);
    Hh[(size_t)y0 * WH + u] = x0;
    if (y0 + 1 < h) Hh[(size_t)(y0 + 1) * WH + u] = make_float2(d.y, -d.x);
  });
}

// Forward transform of the steered signals A_k = H exp(-i k alpha) (Sec. 4.1,
// extended convolution: the signal is pre-multiplied before convolving with
// F_k).  blockIdx.x selects k = k0 + blockIdx.x, blockIdx.y the row block.
// H == nullptr stands for the constant signal 1 (the denominator of Eq.
// normalization).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_fwd_phase(const float* __restrict__ H, const float* __restrict__ alpha, int h, int k0,
                 float2* __restrict__ A, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::ROW_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  // blockIdx.x = component (fastest): the blocks of all components of one row
  // block run together, so H and alpha are read from HBM once and then from L2
  const int y0 = blockIdx.y * C::RL;
  const int k = k0 + blockIdx.x;
  float hv[STAGE_G], av[STAGE_G];
  for_elems_staged<C::RL * N, T, STAGE_G>(
      [&](int i, int e) {
        const int y = y0 + e / N;
        const size_t idx = (size_t)y * N + e % N;
        hv[i] = (y < h) ? (H ? __ldg(H + idx) : 1.0f) : 0.f;
        av[i] = (y < h) ? __ldg(alpha + idx) : 0.f;
      },
      [&](int i, int e) {
        float s, c;
        sincos_kalpha(k, av[i], &s, &c);
        sm[(e / N) * C::LS + sidx(e % N)] = make_float2(hv[i] * c, -hv[i] * s);
      });
  __syncthreads();
  row_fft<N, false>(sm, twl);
  float2* out = A + (size_t)blockIdx.x * h * N;
  for_elems<C::RL * N, T>([&](int i, int e) {
    const int y = y0 + e / N;
    if (y < h) out[(size_t)y * N + e % N] = sm[(e / N) * C::LS + sidx(e % N)];
  });
}

// Forward transform of the scale-steered signals of Sec. 8:
//   A_k = H wgt exp(-i w_k ln s),  w_k = omega_step * (k0 + blockIdx.y),
// wgt = 1/s^2 when unit_integral (the normalised signal H~ = H/|T|^2), else 1;
// H == nullptr stands for the constant signal 1 (the denominator of
// Eq. normalization).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_fwd_scale(const float* __restrict__ H, const float* __restrict__ sfield, int h, int k0, float omega_step,
                 int unit_integral, float2* __restrict__ A, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::ROW_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::RL * C::LS>(sm, tw, C::ROW_THREADS);
  const int y0 = blockIdx.x * C::RL;
  const float wk = omega_step * (float)(k0 + (int)blockIdx.y);
  float hv[STAGE_G], sv[STAGE_G];
  for_elems_staged<C::RL * N, T, STAGE_G>(
      [&](int i, int e) {
        const int y = y0 + e / N;
        const size_t idx = (size_t)y * N + e % N;
        hv[i] = (y < h) ? (H ? __ldg(H + idx) : 1.0f) : 0.f;
        sv[i] = (y < h) ? __ldg(sfield + idx) : 1.0f;
      },
      [&](int i, int e) {
        float sn, cs;
        sincos_wx(wk, logf(sv[i]), &sn, &cs);
        const float a = unit_integral ? hv[i] / (sv[i] * sv[i]) : hv[i];
        sm[(e / N) * C::LS + sidx(e % N)] = make_float2(a * cs, -a * sn);
      });
  __syncthreads();
  row_fft<N, false>(sm, twl);
  float2* out = A + (size_t)blockIdx.y * h * N;
  for_elems<C::RL * N, T>([&](int i, int e) {
    const int y = y0 + e / N;
    if (y < h) out[(size_t)y * N + e % N] = sm[(e / N) * C::LS + sidx(e % N)];
  });
}

// Forward transform of the similarity-steered signals (rotation and scale
// fields together, in log-polar harmonics):
//   A_c = H wgt exp(-i (k alpha + w_j ln s)) = H wgt u^k v^j,  (k, j) = kj[blockIdx.x],
// with the per-pixel phasors uv = (u, v) = (e^{-i alpha}, e^{-i w_1 ln s})
// formed once per call (k_simil_phasors) and raised to the harmonic's powers
// by repeated squaring (|k|, |j| <= 64: at most 7 squarings each);
// wgt = 1/s^2 when unit_integral, else 1; H == nullptr stands for the constant
// signal 1.  blockIdx.x = component (fastest), so the row block's inputs come
// from L2 for all harmonics.  (A variant that carried each element's value
// from one harmonic to the next ran 1.8x slower at 2048 points: the carried
// state spilled and its long blocks lost occupancy.)
__device__ __forceinline__ float2 c_pow(float2 b, int e) {
  float2 r = make_float2(1.f, 0.f);
  if (e < 0) {
    b.y = -b.y;
    e = -e;
  }
  while (e) {
    if (e & 1) r = c_mul(r, b);
    b = c_mul(b, b);
    e >>= 1;
  }
  return r;
}

template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_fwd_simil(const float* __restrict__ H, const float4* __restrict__ uv, const float* __restrict__ sfield,
                 int h, const int2* __restrict__ kj, int unit_integral, float2* __restrict__ A,
                 const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::ROW_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::RL * C::LS>(sm, tw, C::ROW_THREADS);
  const int y0 = blockIdx.y * C::RL;
  const int2 c = kj[blockIdx.x];
  float hv[STAGE_G], sv[STAGE_G];
  float4 pv[STAGE_G];
  for_elems_staged<C::RL * N, T, STAGE_G>(
      [&](int i, int e) {
        const int y = y0 + e / N;
        const size_t idx = (size_t)y * N + e % N;
        hv[i] = (y < h) ? (H ? __ldg(H + idx) : 1.0f) : 0.f;
        sv[i] = (y < h && unit_integral) ? __ldg(sfield + idx) : 1.0f;
        pv[i] = (y < h) ? __ldg(uv + idx) : make_float4(1.f, 0.f, 1.f, 0.f);
      },
      [&](int i, int e) {
        const float a = unit_integral ? hv[i] / (sv[i] * sv[i]) : hv[i];
        const float2 z = c_mul(c_pow(make_float2(pv[i].x, pv[i].y), c.x), c_pow(make_float2(pv[i].z, pv[i].w), c.y));
        sm[(e / N) * C::LS + sidx(e % N)] = make_float2(a * z.x, a * z.y);
      });
  __syncthreads();
  row_fft<N, false>(sm, twl);
  float2* out = A + (size_t)blockIdx.x * h * N;
  for_elems<C::RL * N, T>([&](int i, int e) {
    const int y = y0 + e / N;
    if (y < h) out[(size_t)y * N + e % N] = sm[(e / N) * C::LS + sidx(e % N)];
  });
}

// ------------------------------------------ steered forward row passes ---
// e^{-2 pi i q} for q = m t (t a fraction of a turn, m an integer held in a
// float): the product is formed exactly as p + e (two-product with an FMA),
// its integer part is dropped (p - rint(p) is exact), and the remainder,
// |r| <= 1/2 + |e|, goes to sincospif.  No range reduction by 2 pi is needed.
__device__ __forceinline__ float2 turn_phasor(float m, float t) {
  const float p = m * t;
  const float e = fmaf(m, t, -p);
  const float r = (p - rintf(p)) + e;
  float sn, cs;
  sincospif(2.f * r, &sn, &cs);
  return make_float2(cs, -sn);
}

// The same phasor with the remainder passed to the hardware sine and cosine
// (__sincosf on 2 pi r, |2 pi r| <= pi): absolute error about 4e-7, against
// about 1e-7 for sincospif, for a fifth of the instructions of the
// component-loop row pass.
__device__ __forceinline__ float2 turn_phasor_fast(float m, float t) {
  const float p = m * t;
  const float e = fmaf(m, t, -p);
  const float r = (p - rintf(p)) + e;
  float sn, cs;
  __sincosf(6.283185307179586f * r, &sn, &cs);
  return make_float2(cs, -sn);
}

// Steering policies of k_rows_fwd_steered: comp(c) gives the constants of
// component c, at(cc, p) the steered signal of that component at pixel p.
// H == nullptr stands for the constant signal 1 (the denominator of Eq.
// normalization).
struct SteerPhase {   // A_k = H e^{-i k alpha} (Sec. 4.1, extended convolution)
  const float* H;
  const float* alpha;
  int k0;
  __device__ __forceinline__ int comp(int c) const { return k0 + c; }
  __device__ __forceinline__ float2 at(int k, size_t p) const {
    const float hv = H ? __ldg(H + p) : 1.0f;
    float sn, cs;
    sincos_kalpha_pi(k, __ldg(alpha + p), &sn, &cs);
    return make_float2(hv * cs, -hv * sn);
  }
};

struct SteerScale {   // A_k = H wgt e^{-i w_k ln s} = H wgt e^{-2 pi i k t}, (t, wgt) = T[p] (Sec. 8)
  const float* H;
  const float2* T;
  int k0;
  __device__ __forceinline__ float comp(int c) const { return (float)(k0 + c); }
  __device__ __forceinline__ float2 at(float k, size_t p) const {
    const float2 tv = __ldg(T + p);
    const float a = (H ? __ldg(H + p) : 1.0f) * tv.y;
    const float2 z = turn_phasor(k, tv.x);
    return make_float2(a * z.x, a * z.y);
  }
};

struct SteerSimil {   // A_(k,j) = H wgt e^{-i (k alpha + w_j ln s)}, (a, b, wgt) = T[p], turns a = alpha / 2 pi, b = ln s / log_period
  const float* H;
  const float4* T;
  const int2* kj;
  __device__ __forceinline__ float2 comp(int c) const {
    const int2 v = kj[c];
    return make_float2((float)v.x, (float)v.y);
  }
  __device__ __forceinline__ float2 at(float2 c, size_t p) const {
    const float4 tv = __ldg(T + p);
    const float a = (H ? __ldg(H + p) : 1.0f) * tv.z;
    const float p1 = c.x * tv.x, e1 = fmaf(c.x, tv.x, -p1);
    const float p2 = c.y * tv.y, e2 = fmaf(c.y, tv.y, -p2);
    const float r = ((p1 - rintf(p1)) + (p2 - rintf(p2))) + (e1 + e2);
    float sn, cs;
    sincospif(2.f * r, &sn, &cs);
    return make_float2(a * cs, -a * sn);
  }
};

// Forward row transform of steered signals: the steering is evaluated in the
// first butterfly stage's loads (straight from global memory, coalesced) and
// the last stage writes its outputs straight to global memory, so each
// element passes through shared memory twice fewer than when the lines are
// staged first.  blockIdx.x = component (fastest: the blocks of all
// components of a row block run together and read its inputs from L2),
// blockIdx.y = row block; component c's plane is A + c h N.
template <int N, class Steer>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_fwd_steered(const Steer sp, int h, float2* __restrict__ A, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::ROW_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::RL * C::LS>(sm, tw, T);
  const int y0 = blockIdx.y * C::RL;
  const auto cc = sp.comp((int)blockIdx.x);
  float2* out = A + (size_t)blockIdx.x * h * N;
  auto load = [&](int l, int x) -> float2 {
    const int y = y0 + l;
    return y < h ? sp.at(cc, (size_t)y * N + x) : make_float2(0.f, 0.f);
  };
  auto store = [&](int l, int x, float2 v) {
    const int y = y0 + l;
    if (y < h) out[(size_t)y * N + x] = v;
  };
  ct_fft_io<N, false, false, C::RL, T>(sm, C::LS, 1, twl, load, store);
}

// --------------------------- steered forward row passes, component loop ---
// RB rows per block (one for 1024 points and more, enough to make 128
// threads for shorter rows), N / 16 threads per row, 16 elements per thread:
// the per-pixel inputs of the rows are read once into registers and every
// component of the block's group is then steered from them and transformed
// (first radix-16 stage in registers, the other stages between two
// shared-memory row buffers, the last one writing straight to global
// memory), so the loads and the stage-twiddle staging are paid once per row
// block instead of once per row block and component.  Three-stage lengths
// take two barriers per component, two-stage lengths one (the two buffers
// alternate between components).
template <int N>
struct HloopCfg {
  static constexpr RadixList L = factor_radices(N);
  static constexpr int TPL = N / 16;                                     // threads per row
  static constexpr int RB = TPL >= 64 ? 1 : (TPL > 0 ? 128 / TPL : 1);   // rows per block
  static constexpr int THREADS = RB * TPL;
  static constexpr int LS = ct_sidx_len(N);
  static constexpr int SMEM = 2 * RB * LS * 8 + N * 8;   // two buffers of RB padded rows + the stage twiddles
  static constexpr int MINB = THREADS > 0 && 512 / THREADS > 0 ? 512 / THREADS : 1;
  static constexpr bool OK = (L.cnt == 3 || L.cnt == 2) && L.r[0] == 16 && N % 16 == 0 && THREADS >= 64 &&
                             THREADS % 32 == 0 && SMEM * MINB <= 220 * 1024;
};

// Ping-pong Stockham stage over NL lines of pitch ls: reads `in`, writes
// `out` (or, LAST, hands each output to store(line, x, value)); no barrier
// inside.
template <int N, int R, int NS, int NL, int THREADS, bool LAST, class Store>
__device__ __forceinline__ void pp_stage(const float2* in, float2* out, int ls, const float2* __restrict__ tw,
                                         Store&& store) {
  constexpr int NB = N / R;
  constexpr int TOTAL = NB * NL;
  constexpr int S = (TOTAL + THREADS - 1) / THREADS;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int it = threadIdx.x + s * THREADS;
    if (TOTAL % THREADS == 0 || it < TOTAL) {
      const int line = it / NB, j = it % NB;
      const int k = j % NS;
      const float2* src = in + line * ls;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 a = src[sidx(j + r * NB)];
        if (r > 0) a = c_mul(a, tw[r * NS - 1 + k]);
        v[r] = a;
      }
      dft<R, false>(v);
      const int dst = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (LAST) store(line, dst + r * NS, v[r]);
        else out[line * ls + sidx(dst + r * NS)] = v[r];
      }
    }
  }
}

// Steering policies of k_rows_fwd_hloop: load(p) gives the per-pixel state q
// held across components, comp(c) the constants of component c, at(cc, q)
// the steered signal.  H == nullptr stands for the constant signal 1.  FAST:
// the phasor from the hardware sine and cosine after the exact reduction
// (absolute error about 4e-7), else from sincospif (about 1e-7).
template <bool FAST>
struct HloopScale {   // A_k = H wgt e^{-2 pi i k t}; q = (H wgt, t)
  const float* H;
  const float2* T;
  int k0;
  using Q = float2;
  __device__ __forceinline__ Q load(size_t p) const {
    const float2 tv = __ldg(T + p);
    return make_float2((H ? __ldg(H + p) : 1.0f) * tv.y, tv.x);
  }
  __device__ __forceinline__ float comp(int c) const { return (float)(k0 + c); }
  __device__ __forceinline__ float2 at(float k, const Q& q) const {
    const float2 z = FAST ? turn_phasor_fast(k, q.y) : turn_phasor(k, q.y);
    return make_float2(q.x * z.x, q.x * z.y);
  }
};

template <bool FAST>
struct HloopSimil {   // A_(k,j) = H wgt e^{-2 pi i (k a + j b)}; q = (H wgt, a, b)
  const float* H;
  const float4* T;
  const int2* kj;
  using Q = float3;
  __device__ __forceinline__ Q load(size_t p) const {
    const float4 tv = __ldg(T + p);
    return make_float3((H ? __ldg(H + p) : 1.0f) * tv.z, tv.x, tv.y);
  }
  __device__ __forceinline__ float2 comp(int c) const {
    const int2 v = kj[c];
    return make_float2((float)v.x, (float)v.y);
  }
  __device__ __forceinline__ float2 at(float2 c, const Q& q) const {
    const float p1 = c.x * q.y, e1 = fmaf(c.x, q.y, -p1);
    const float p2 = c.y * q.z, e2 = fmaf(c.y, q.z, -p2);
    float r = ((p1 - rintf(p1)) + (p2 - rintf(p2))) + (e1 + e2);
    r -= rintf(r);   // exact: |r| <= 1/2
    float sn, cs;
    if (FAST) __sincosf(6.283185307179586f * r, &sn, &cs);
    else sincospif(2.f * r, &sn, &cs);
    return make_float2(q.x * cs, -q.x * sn);
  }
};

template <bool FAST>
struct HloopPhase {   // A_k = H e^{-i k alpha}; q = (H, alpha)
  const float* H;
  const float* alpha;
  int k0;
  using Q = float2;
  __device__ __forceinline__ Q load(size_t p) const {
    return make_float2(H ? __ldg(H + p) : 1.0f, __ldg(alpha + p));
  }
  __device__ __forceinline__ int comp(int c) const { return k0 + c; }
  __device__ __forceinline__ float2 at(int k, const Q& q) const {
    float sn, cs;
    if (FAST) sincos_kalpha_fast(k, q.y, &sn, &cs);
    else sincos_kalpha_pi(k, q.y, &sn, &cs);
    return make_float2(q.x * cs, -q.x * sn);
  }
};

// blockIdx.x = row block (rows blockIdx.x RB ..), blockIdx.y = component
// group [c0, c1), c0 = blockIdx.y * cpb; component c's plane is A + c h N.
template <int N, class Steer>
__global__ void __launch_bounds__(HloopCfg<N>::THREADS, HloopCfg<N>::MINB)
k_rows_fwd_hloop(const Steer sp, int h, int ncomp, int cpb, float2* __restrict__ A, const float2* __restrict__ tw) {
  using HC = HloopCfg<N>;
  constexpr int T = HC::THREADS;
  constexpr int LS = HC::LS;
  constexpr int RB = HC::RB;
  constexpr int TPL = HC::TPL;
  constexpr int NST = HC::L.cnt;
  constexpr int R1 = HC::L.r[1];
  extern __shared__ float2 sm[];
  float2* X = sm;
  float2* Y = sm + RB * LS;
  const float2* twl = stage_twiddles<N, 2 * RB * LS>(sm, tw, T);
  const int l = threadIdx.x / TPL, j = threadIdx.x % TPL;
  const int yb = blockIdx.x * RB;
  const int c0 = blockIdx.y * cpb;
  const int c1 = min(ncomp, c0 + cpb);
  typename Steer::Q q[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) q[r] = yb + l < h ? sp.load((size_t)(yb + l) * N + j + r * TPL) : typename Steer::Q{};
  auto nostore = [](int, int, float2) {};
  for (int c = c0; c < c1; ++c) {
    const auto cc = sp.comp(c);
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = sp.at(cc, q[r]);
    dft<16, false>(v);
    // two-stage lengths alternate the buffers between components
    float2* B0 = (NST == 2 && ((c - c0) & 1)) ? Y : X;
#pragma unroll
    for (int r = 0; r < 16; ++r) B0[l * LS + sidx(j * 16 + r)] = v[r];
    __syncthreads();   // B0 complete (and, on the first pass, the stage twiddles)
    float2* out = A + (size_t)c * h * N;
    auto store = [&](int line, int x, float2 v2) {
      if (yb + line < h) out[(size_t)(yb + line) * N + x] = v2;
    };
    if constexpr (NST == 3) {
      constexpr int R2 = HC::L.r[2];
      pp_stage<N, R1, 16, RB, T, false>(X, Y, LS, twl, nostore);
      __syncthreads();   // Y complete; X free for the next component
      pp_stage<N, R2, 16 * R1, RB, T, true>(Y, nullptr, LS, twl, store);
      // the next component writes X (read before the barrier above) and then Y
      // (after its own first barrier, when every thread has finished this read)
    } else {
      pp_stage<N, R1, 16, RB, T, true>(B0, nullptr, LS, twl, store);
      // the next component writes the other buffer; this one is rewritten two
      // components on, after a barrier that follows this read
    }
  }
}

template <int N>
__device__ __forceinline__ void rows_load_complex(float2* sm, const float2* src, int y0, int h) {
  using C = LineCfg<N>;
  constexpr int T = C::ROW_THREADS;
  float2 v[STAGE_G];
  for_elems_staged<C::RL * N, T, STAGE_G>(
      [&](int i, int e) {
        const int y = y0 + e / N;
        v[i] = (y < h) ? src[(size_t)y * N + e % N] : make_float2(0.f, 0.f);
      },
      [&](int i, int e) { sm[(e / N) * C::LS + sidx(e % N)] = v[i]; });
}

// Complex rows, forward or inverse, X -> Y (may alias); blockIdx.y = plane.
template <int N, bool INV>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_c2c(const float2* X, int h, float2* Y, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  const int y0 = blockIdx.x * C::RL;
  const size_t plane = (size_t)blockIdx.y * h * N;
  rows_load_complex<N>(sm, X + plane, y0, h);
  __syncthreads();
  row_fft<N, INV>(sm, twl);
  for_elems<C::RL * N, C::ROW_THREADS>([&](int i, int e) {
    const int y = y0 + e / N;
    if (y < h) Y[plane + (size_t)y * N + e % N] = sm[(e / N) * C::LS + sidx(e % N)];
  });
}

// Inverse row pass writing the component correlations G_k (k = k0 + blockIdx.y)
// into their planes.
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_inv_components(const float2* __restrict__ Z, int h, int k0, float* __restrict__ G,
                      const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  const int y0 = blockIdx.x * C::RL;
  const int k = k0 + blockIdx.y;
  const size_t P = (size_t)h * N;
  rows_load_complex<N>(sm, Z + (size_t)blockIdx.y * P, y0, h);
  __syncthreads();
  row_fft<N, true>(sm, twl);
  float* re = G + (k == 0 ? 0 : (size_t)(2 * k - 1) * P);
  float* im = G + (size_t)(2 * k) * P;
  for_elems<C::RL * N, C::ROW_THREADS>([&](int i, int e) {
    const int y = y0 + e / N;
    if (y >= h) return;
    const float2 v = sm[(e / N) * C::LS + sidx(e % N)];
    const size_t idx = (size_t)y * N + e % N;
    re[idx] = v.x;
    if (k != 0) im[idx] = v.y;
  });
}

// Inverse row pass with the steering sum of Sec. 4.1 ("Linear Combination")
// fused in: out(p) = G_0(p) + 2 sum_{k=1..K} Re(exp(i k alpha(p)) G_k(p)),
// looping over all K+1 components inside the block (real filter and signal).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, 1)
k_rows_inv_field(const float2* __restrict__ Z, int h, int K, const float* __restrict__ alpha,
                 float* __restrict__ out, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::ROW_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  float* acc = reinterpret_cast<float*>(sm + C::RL * C::LS + N);
  const int y0 = blockIdx.x * C::RL;
  const size_t P = (size_t)h * N;
  for_elems<C::RL * N, T>([&](int i, int e) { acc[e] = 0.f; });
  for (int k = 0; k <= K; ++k) {
    rows_load_complex<N>(sm, Z + (size_t)k * P, y0, h);
    __syncthreads();
    row_fft<N, true>(sm, twl);
    for_elems<C::RL * N, T>([&](int i, int e) {
      const int y = y0 + e / N;
      if (y >= h) return;
      const float2 g = sm[(e / N) * C::LS + sidx(e % N)];
      if (k == 0) {
        acc[e] += g.x;
      } else {
        float s, c;
        sincos_kalpha(k, __ldg(alpha + (size_t)y * N + e % N), &s, &c);
        acc[e] += 2.f * (c * g.x - s * g.y);
      }
    });
    __syncthreads();
  }
  for_elems<C::RL * N, T>([&](int i, int e) {
    const int y = y0 + e / N;
    if (y < h) out[(size_t)y * N + e % N] = acc[e];
  });
}

// Inverse row pass keeping the real part (extended convolution output).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_inv_real(const float2* __restrict__ Y, int h, float* __restrict__ out, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  const int y0 = blockIdx.x * C::RL;
  // the first butterfly stage reads the rows straight from global memory and
  // the last one writes the real parts straight back
  auto load = [&](int l, int x) -> float2 {
    return y0 + l < h ? Y[(size_t)(y0 + l) * N + x] : make_float2(0.f, 0.f);
  };
  auto store = [&](int l, int x, float2 v) {
    if (y0 + l < h) out[(size_t)(y0 + l) * N + x] = v.x;
  };
  ct_fft_io<N, true, false, C::RL, C::ROW_THREADS>(sm, C::LS, 1, twl, load, store);
}

// --------------------------------------------------------- column passes ---
// Element (v, c) of a tile of CW adjacent columns sits at sm[c + sidx(v) * CW];
// element e of a block maps to v = e / CW, c = e % CW (adjacent threads read
// adjacent columns of one row).

template <int N>
__device__ __forceinline__ void cols_store_sm(float2* sm, const float2* v) {
  using C = LineCfg<N>;
  for_elems<C::CW * N, C::COL_THREADS>([&](int i, int e) { sm[e % C::CW + sidx(e / C::CW) * C::CW] = v[i]; });
}

// Forward column pass of the half spectrum, in place (pitch ncols).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, LineCfg<N>::COL_MINB)
k_cols_fwd_half(float2* Hh, int ncols, const float2* __restrict__ tw, float2* __restrict__ Hf, int w) {
  using C = LineCfg<N>;
  constexpr int T = C::COL_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  const int u0 = blockIdx.x * C::CW;
  float2 v[STAGE_G];
  for_elems_staged<C::CW * N, T, STAGE_G>(
      [&](int i, int e) {
        const int u = u0 + e % C::CW;
        v[i] = (u < ncols) ? Hh[(size_t)(e / C::CW) * ncols + u] : make_float2(0.f, 0.f);
      },
      [&](int i, int e) { sm[e % C::CW + sidx(e / C::CW) * C::CW] = v[i]; });
  __syncthreads();
  col_fft<N, false>(sm, twl);
  for_elems<C::CW * N, T>([&](int i, int e) {
    const int u = u0 + e % C::CW, v = e / C::CW;
    if (u < ncols) {
      const float2 x = sm[e % C::CW + sidx(v) * C::CW];
      Hh[(size_t)v * ncols + u] = x;
      if (Hf) {   // the full spectrum too: Hf(v, u) = x and, by Hermitian symmetry, Hf(-v, w - u) = conj x
        Hf[(size_t)v * w + u] = x;
        if (u > 0 && 2 * u < w) Hf[(size_t)((N - v) % N) * w + (w - u)] = c_conj(x);
      }
    }
  });
}

// Forward column pass of a component grid (already row-transformed, pitch w),
// stored as a tiled spectrum: conj(X) * scale (correlation) or X * scale
// (convolution).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, LineCfg<N>::COL_MINB)
k_cols_fwd_spectrum(const float2* __restrict__ X, int w, int conj_out, float scale, float scale_rest,
                    float2* __restrict__ S, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::COL_THREADS;
  extern __shared__ float2 sm[];
  // blockIdx.y = plane: plane 0 is scaled by `scale`, the others by `scale_rest`
  X += (size_t)blockIdx.y * N * w;
  S += (size_t)blockIdx.y * ((w + C::CW - 1) / C::CW) * N * C::CW;
  if (blockIdx.y > 0) scale = scale_rest;
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  const int tile = blockIdx.x;
  const int u0 = tile * C::CW;
  float2 v[STAGE_G];
  for_elems_staged<C::CW * N, T, STAGE_G>(
      [&](int i, int e) {
        const int u = u0 + e % C::CW;
        v[i] = (u < w) ? X[(size_t)(e / C::CW) * w + u] : make_float2(0.f, 0.f);
      },
      [&](int i, int e) { sm[e % C::CW + sidx(e / C::CW) * C::CW] = v[i]; });
  __syncthreads();
  col_fft<N, false>(sm, twl);
  float2* dst = S + (size_t)tile * N * C::CW;
  for_elems<C::CW * N, T>([&](int i, int e) {
    float2 val = c_scale(sm[e % C::CW + sidx(e / C::CW) * C::CW], scale);
    if (conj_out) val.y = -val.y;
    dst[e] = val;   // e = v * CW + c
  });
}

// Inverse column pass of the correlation products H^(u,v) conj(F^_k(u,v))
// (Sec. 4.1 "Standard Correlation"), with H^ rebuilt from its half by
// Hermitian symmetry; k = k0 + blockIdx.y, output Z[blockIdx.y] (pitch w).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, LineCfg<N>::COL_MINB)
k_cols_inv_corr(const float2* __restrict__ Hh, int w, const float2* __restrict__ S, int k0,
                float2* __restrict__ Z, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::COL_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  const int tile = blockIdx.x;
  const int u0 = tile * C::CW;
  const int wh = w / 2 + 1;
  const int ntiles = (w + C::CW - 1) / C::CW;
  const float2* spec = S + ((size_t)(k0 + blockIdx.y) * ntiles + tile) * N * C::CW;
  float2 hv[STAGE_G], sv[STAGE_G];
  for_elems_staged<C::CW * N, T, STAGE_G>(
      [&](int i, int e) {
        const int v = e / C::CW, u = u0 + e % C::CW;
        sv[i] = __ldg(spec + e);
        if (u < wh) hv[i] = __ldg(Hh + (size_t)v * wh + u);
        else if (u < w) hv[i] = c_conj(__ldg(Hh + (size_t)((N - v) % N) * wh + (w - u)));
        else hv[i] = make_float2(0.f, 0.f);
      },
      [&](int i, int e) { sm[e % C::CW + sidx(e / C::CW) * C::CW] = c_mul(hv[i], sv[i]); });
  __syncthreads();
  col_fft<N, true>(sm, twl);
  float2* dst = Z + (size_t)blockIdx.y * N * w;
  for_elems<C::CW * N, T>([&](int i, int e) {
    const int u = u0 + e % C::CW;
    if (u < w) dst[(size_t)(e / C::CW) * w + u] = sm[e % C::CW + sidx(e / C::CW) * C::CW];
  });
}

// Extended convolution, column stage: forward column FFT of every steered
// signal A_k, product with its (weighted) spectrum, sum over k in registers,
// and the inverse column FFT of the sum (Sec. 4.1, last paragraph).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, 1)
k_cols_conv(const float2* __restrict__ A, int w, int K, const float2* __restrict__ S,
            float2* __restrict__ Y, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::COL_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, C::COL_THREADS);
  const int tile = blockIdx.x;
  const int u0 = tile * C::CW;
  const int ntiles = (w + C::CW - 1) / C::CW;
  float2 acc[C::COL_EPT];
  for_elems<C::CW * N, T>([&](int i, int e) { acc[i] = make_float2(0.f, 0.f); });
  for (int k = 0; k <= K; ++k) {
    const float2* src = A + (size_t)k * N * w;
    {
      float2 v[STAGE_G];
      for_elems_staged<C::CW * N, T, STAGE_G>(
          [&](int i, int e) {
            const int u = u0 + e % C::CW;
            v[i] = (u < w) ? __ldg(src + (size_t)(e / C::CW) * w + u) : make_float2(0.f, 0.f);
          },
          [&](int i, int e) { sm[e % C::CW + sidx(e / C::CW) * C::CW] = v[i]; });
    }
    __syncthreads();
    col_fft<N, false>(sm, twl);
    const float2* spec = S + ((size_t)k * ntiles + tile) * N * C::CW;
    for_elems<C::CW * N, T>([&](int i, int e) {
      const float2 sp = __ldg(spec + e);
      const float2 x = sm[e % C::CW + sidx(e / C::CW) * C::CW];
      acc[i].x = fmaf(x.x, sp.x, fmaf(-x.y, sp.y, acc[i].x));
      acc[i].y = fmaf(x.x, sp.y, fmaf(x.y, sp.x, acc[i].y));
    });
    __syncthreads();
  }
  cols_store_sm<N>(sm, acc);
  __syncthreads();
  col_fft<N, true>(sm, twl);
  for_elems<C::CW * N, T>([&](int i, int e) {
    const int u = u0 + e % C::CW;
    if (u < w) Y[(size_t)(e / C::CW) * w + u] = sm[e % C::CW + sidx(e / C::CW) * C::CW];
  });
}

// In-place complex column pass over `planes` planes of N x w (plane stride N w):
// the y-pass of a 3D transform (planes = z slices) or the z-pass (planes = 1,
// w = ny * nx).
template <int N, bool INV>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, LineCfg<N>::COL_MINB)
k_cols_c2c(float2* X, int w, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::COL_THREADS;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::CW * C::LS>(sm, tw, T);
  float2* P = X + (size_t)blockIdx.y * N * w;
  const int u0 = blockIdx.x * C::CW;
  float2 v[STAGE_G];
  for_elems_staged<C::CW * N, T, STAGE_G>(
      [&](int i, int e) {
        const int u = u0 + e % C::CW;
        v[i] = (u < w) ? P[(size_t)(e / C::CW) * w + u] : make_float2(0.f, 0.f);
      },
      [&](int i, int e) { sm[e % C::CW + sidx(e / C::CW) * C::CW] = v[i]; });
  __syncthreads();
  col_fft<N, INV>(sm, twl);
  for_elems<C::CW * N, T>([&](int i, int e) {
    const int u = u0 + e % C::CW;
    if (u < w) P[(size_t)(e / C::CW) * w + u] = sm[e % C::CW + sidx(e / C::CW) * C::CW];
  });
}

// Inverse row pass of component planes (each `rows` rows of N) writing the
// real and imaginary parts of component k0 + blockIdx.y into the channel
// planes chan[k].x and chan[k].y of G (chan[k].y < 0: imaginary part dropped).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, LineCfg<N>::ROW_MINB)
k_rows_inv_channels(const float2* __restrict__ Z, int rows, int k0, const int2* __restrict__ chan,
                    float* __restrict__ G, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  extern __shared__ float2 sm[];
  const float2* twl = stage_twiddles<N, C::RL * C::LS>(sm, tw, C::ROW_THREADS);
  const int y0 = blockIdx.x * C::RL;
  const size_t P = (size_t)rows * N;
  rows_load_complex<N>(sm, Z + (size_t)blockIdx.y * P, y0, rows);
  __syncthreads();
  row_fft<N, true>(sm, twl);
  const int2 ch = chan[k0 + blockIdx.y];
  float* re = G + (size_t)ch.x * P;
  float* im = G + (size_t)(ch.y < 0 ? 0 : ch.y) * P;
  for_elems<C::RL * N, C::ROW_THREADS>([&](int i, int e) {
    const int y = y0 + e / N;
    if (y >= rows) return;
    const float2 v = sm[(e / N) * C::LS + sidx(e % N)];
    const size_t idx = (size_t)y * N + e % N;
    re[idx] = v.x;
    if (ch.y >= 0) im[idx] = v.y;
  });
}

// Fused inverse y and x passes of the SO(3) components: one block per
// (component, z) plane of N x N complex values (after the z pass), with the
// whole plane resident in shared memory (rows of pitch LS).  The plane comes
// in by N bulk copies (one per row) on an mbarrier; column FFTs run in
// groups of 32 columns in place, then row FFTs in groups of 32 rows write the
// real channel planes of G.  As soon as a row group has been read, its rows
// of the block's next plane are requested, so the next plane streams in
// while this one finishes.  Waits are bounded (err = EXT_ERR_TIMEOUT).
template <int N>
struct PlaneCfg {
  using C = LineCfg<N>;
  // lines per group: as many as the shared memory left by the plane allows (up to N)
  static constexpr int PB = N * C::LS;               // plane, rows of pitch LS
  static constexpr int LINES_FIT = (227 * 1024 / 8 - PB - N) / C::LS;
  static constexpr int LINES = LINES_FIT >= 64 && N % 64 == 0 ? 64 : (LINES_FIT >= 32 && N % 32 == 0 ? 32 : 16);
  static constexpr int THREADS = ((LINES * C::TPL + 31) / 32) * 32 > 1024 ? 1024 : ((LINES * C::TPL + 31) / 32) * 32;
  static constexpr int WB = LINES * C::LS;           // work buffer of one group of lines
  static constexpr int SMEM = (PB + WB + N) * 8;
  static constexpr bool OK = (N % LINES == 0) && SMEM <= 227 * 1024 && (C::LS * 8) % 16 == 0 &&
                             THREADS >= LINES * N / FFT_MAXE;
};

template <int N>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS, 1)
k_planes_inv_channels(const float2* __restrict__ Z, int nz, int k0, int nk, const int2* __restrict__ chan,
                      float* __restrict__ G, const float2* __restrict__ tw, int* __restrict__ err) {
  using C = LineCfg<N>;
  using PC = PlaneCfg<N>;
  constexpr int T = PC::THREADS;
  constexpr int LINES = PC::LINES;
  constexpr int LS = C::LS;
  extern __shared__ float2 sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int abort_flag;
  float2* PBuf = sm;
  float2* W = sm + PC::PB;
  const float2* TWs = stage_twiddles<N, PC::PB + PC::WB>(sm, tw, T);
  const size_t plane = (size_t)N * N;
  const size_t P = plane * nz;
  const int nplanes = nk * nz;
  const uint32_t mb = tc::smem_u32(&mbar);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    tc::mbar_init(mb, 1);
  }
  __syncthreads();
  // thread 0: rows [r0, r1) of plane pz into the plane buffer (first call of a plane sets the byte count)
  auto fetch_rows = [&](int pz, int r0, int r1) {
    const float2* src = Z + (size_t)pz * plane;
    if (r0 == 0) {
      tc::fence_proxy_async();
      tc::mbar_expect_tx(mb, (uint32_t)(plane * 8));
    }
    for (int y = r0; y < r1; ++y) tc::bulk_load(tc::smem_u32(PBuf + y * LS), src + (size_t)y * N, N * 8u, mb);
  };
  int pz = blockIdx.x;
  uint32_t phase = 0;
  bool pending = pz < nplanes;
  if (pending && threadIdx.x == 0) fetch_rows(pz, 0, N);
  constexpr RadixList L = factor_radices(N);
  constexpr int R0 = L.r[0];
  for (; pz < nplanes; pz += gridDim.x) {
    if (!tc::mbar_wait_bounded(mb, phase, 1000000000ull, err, EXT_ERR_TIMEOUT)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    phase ^= 1u;
    pending = false;
    // y pass: groups of LINES columns, in place
    for (int g = 0; g < N / LINES; ++g) {
      const int x0 = g * LINES;
      auto load = [&](int c, int v) -> float2 { return PBuf[v * LS + x0 + c]; };
      auto store = [&](int c, int v, float2 val) { PBuf[v * LS + x0 + c] = val; };
      ct_stage_io<N, R0, 1, true, true, LINES, T, true, L.cnt == 1>(W, 1, LINES, TWs, load, store);
      if constexpr (L.cnt > 1) ct_fft_io<N, true, true, LINES, T, 1, R0>(W, 1, LINES, TWs, load, store);
      __syncthreads();
    }
    // x pass: groups of LINES rows, written to the channel planes
    const int kk = pz / nz, z = pz % nz;
    const int2 ch = chan[k0 + kk];
    float* re = G + (size_t)ch.x * P + (size_t)z * plane;
    float* im = G + (size_t)(ch.y < 0 ? ch.x : ch.y) * P + (size_t)z * plane;
    const int next = pz + gridDim.x;
    for (int g = 0; g < N / LINES; ++g) {
      const int y0 = g * LINES;
      auto load = [&](int l, int x) -> float2 { return PBuf[(y0 + l) * LS + x]; };
      auto store = [&](int l, int x, float2 val) {
        const size_t idx = (size_t)(y0 + l) * N + x;
        re[idx] = val.x;
        if (ch.y >= 0) im[idx] = val.y;
      };
      ct_stage_io<N, R0, 1, true, false, LINES, T, true, L.cnt == 1>(W, LS, 1, TWs, load, store);
      // the first stage has read these rows: the next plane may fill them
      if (next < nplanes) {
        if (threadIdx.x == 0) tc::fence_proxy_async();
        if (threadIdx.x == 0) fetch_rows(next, y0, y0 + LINES);
        pending = true;
      }
      if constexpr (L.cnt > 1) ct_fft_io<N, true, false, LINES, T, 1, R0>(W, LS, 1, TWs, load, store);
      __syncthreads();
    }
  }
  if (pending) tc::mbar_wait_bounded(mb, phase, 1000000000ull, err, EXT_ERR_TIMEOUT);
}

// Fused forward x and y passes of the SO(3) convolution's modulated planes,
// in place: one block per (entry, z) plane of N x N complex values at a time
// (persistent over planes), the same structure as k_planes_inv_channels.
// The plane comes in by N bulk copies on an mbarrier; the column (y) FFTs run
// in groups of LINES columns in shared memory, then the row (x) FFTs store
// their last stage straight back to the plane in global memory.  The 2D DFT
// is separable, so transforming y before x gives the same spectrum.  Rows of
// the block's next plane are requested as soon as a row group has been read.
// Waits are bounded (err = EXT_ERR_TIMEOUT).
template <int N>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS, 1)
k_planes_fwd_c2c(float2* __restrict__ U, int nplanes, const float2* __restrict__ tw, int* __restrict__ err) {
  using C = LineCfg<N>;
  using PC = PlaneCfg<N>;
  constexpr int T = PC::THREADS;
  constexpr int LINES = PC::LINES;
  constexpr int LS = C::LS;
  extern __shared__ float2 sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int abort_flag;
  float2* PBuf = sm;
  float2* W = sm + PC::PB;
  const float2* TWs = stage_twiddles<N, PC::PB + PC::WB>(sm, tw, T);
  const size_t plane = (size_t)N * N;
  const uint32_t mb = tc::smem_u32(&mbar);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    tc::mbar_init(mb, 1);
  }
  __syncthreads();
  auto fetch_rows = [&](int pz, int r0, int r1) {
    const float2* src = U + (size_t)pz * plane;
    if (r0 == 0) {
      tc::fence_proxy_async();
      tc::mbar_expect_tx(mb, (uint32_t)(plane * 8));
    }
    for (int y = r0; y < r1; ++y) tc::bulk_load(tc::smem_u32(PBuf + y * LS), src + (size_t)y * N, N * 8u, mb);
  };
  int pz = blockIdx.x;
  uint32_t phase = 0;
  bool pending = pz < nplanes;
  if (pending && threadIdx.x == 0) fetch_rows(pz, 0, N);
  constexpr RadixList L = factor_radices(N);
  constexpr int R0 = L.r[0];
  for (; pz < nplanes; pz += gridDim.x) {
    if (!tc::mbar_wait_bounded(mb, phase, 1000000000ull, err, EXT_ERR_TIMEOUT)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    phase ^= 1u;
    pending = false;
    // y pass: groups of LINES columns, in place in shared memory
    for (int g = 0; g < N / LINES; ++g) {
      const int x0 = g * LINES;
      auto load = [&](int c, int v) -> float2 { return PBuf[v * LS + x0 + c]; };
      auto store = [&](int c, int v, float2 val) { PBuf[v * LS + x0 + c] = val; };
      ct_stage_io<N, R0, 1, false, true, LINES, T, true, L.cnt == 1>(W, 1, LINES, TWs, load, store);
      if constexpr (L.cnt > 1) ct_fft_io<N, false, true, LINES, T, 1, R0>(W, 1, LINES, TWs, load, store);
      __syncthreads();
    }
    // x pass: groups of LINES rows, stored back to the plane
    float2* dst = U + (size_t)pz * plane;
    const int next = pz + gridDim.x;
    for (int g = 0; g < N / LINES; ++g) {
      const int y0 = g * LINES;
      auto load = [&](int l, int x) -> float2 { return PBuf[(y0 + l) * LS + x]; };
      auto store = [&](int l, int x, float2 val) { dst[(size_t)(y0 + l) * N + x] = val; };
      ct_stage_io<N, R0, 1, false, false, LINES, T, true, L.cnt == 1>(W, LS, 1, TWs, load, store);
      if constexpr (L.cnt == 1) __syncthreads();   // a single-stage transform has no barrier after its reads
      // the first stage has read these rows: the next plane may fill them
      if (next < nplanes) {
        if (threadIdx.x == 0) tc::fence_proxy_async();
        if (threadIdx.x == 0) fetch_rows(next, y0, y0 + LINES);
        pending = true;
      }
      if constexpr (L.cnt > 1) ct_fft_io<N, false, false, LINES, T, 1, R0>(W, LS, 1, TWs, load, store);
      __syncthreads();
    }
  }
  if (pending) tc::mbar_wait_bounded(mb, phase, 1000000000ull, err, EXT_ERR_TIMEOUT);
}

// ------------------------------------------------- pipelined hot passes ---
// Persistent versions of the two passes that run once per filter component
// in the correlation path.  Each block owns one SM (grid = min(items, SMs))
// and walks its tiles; the global data of the next tile is prefetched into
// shared memory with cp.async while the current tile is transformed.

template <int N>
struct PipeCfg {
  using C = LineCfg<N>;
  // columns: work buffer, spectrum and half-spectrum staging, twiddles
  static constexpr int COL_SMEM = C::CW * C::LS * 8 + 2 * C::CW * N * 8 + N * 8;
  // rows: work buffer, staging of the next rows, twiddles
  static constexpr int ROW_SMEM = C::RL * C::LS * 8 + C::RL * N * 8 + N * 8;
  static constexpr bool COL_OK = COL_SMEM <= 227 * 1024;
  static constexpr bool ROW_OK = ROW_SMEM <= 227 * 1024;
};

// Inverse column pass of H^ conj(F^_k) for k = k0 + (item / ntiles); output
// Z[item / ntiles] (pitch w).  Half spectrum pitch wh = w/2 + 1.
// HERM: Hh is the half spectrum (pitch w/2+1) of a real signal and the other
// half is rebuilt by Hermitian symmetry; otherwise Hh is the full spectrum
// (pitch w).
template <int N, bool HERM>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, 1)
k_cols_inv_corr_pipe(const float2* __restrict__ Hh, int w, const float2* __restrict__ S, int k0, int nk,
                     float2* __restrict__ Z, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::COL_THREADS;
  constexpr int CW = C::CW;
  constexpr int TILE = CW * N;
  extern __shared__ float2 sm[];
  float2* W = sm;                          // CW * LS
  float2* SS = sm + CW * C::LS;            // TILE, linear e = v * CW + c
  float2* HS = SS + TILE;                  // TILE
  const float2* TWs = stage_twiddles<N, CW * C::LS + 2 * TILE>(sm, tw, T);   // N - 1 entries
  const int wh = w / 2 + 1;
  const int ntiles = (w + CW - 1) / CW;
  const int nitems = ntiles * nk;

  auto prefetch = [&](int item) {
    const int kk = item / ntiles, tile = item % ntiles;
    const float2* spec = S + ((size_t)(k0 + kk) * ntiles + tile) * TILE;
    for (int q = threadIdx.x; q < TILE / 2; q += T) cp_async16(SS + 2 * q, spec + 2 * q, true);
    const int u0 = tile * CW;
    for (int e = threadIdx.x; e < TILE; e += T) {
      const int v = e / CW, u = u0 + e % CW;
      const float2* src = Hh;
      bool valid = u < w;
      if (!HERM) src = valid ? Hh + (size_t)v * w + u : Hh;
      else if (u < wh) src = Hh + (size_t)v * wh + u;
      else if (valid) src = Hh + (size_t)((N - v) % N) * wh + (w - u);
      cp_async8(HS + e, src, valid);
    }
    cp_async_commit();
  };

  int item = blockIdx.x;
  if (item < nitems) prefetch(item);
  for (; item < nitems; item += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    const int kk = item / ntiles, tile = item % ntiles;
    const int u0 = tile * CW;
    float2* dst = Z + (size_t)kk * N * w;
    const int next = item + gridDim.x;
    auto load = [&](int c, int v) -> float2 {
      const int e = v * CW + c;
      float2 hv = HS[e];
      if (HERM && u0 + c >= wh) hv.y = -hv.y;
      return c_mul(hv, SS[e]);
    };
    auto store = [&](int c, int v, float2 val) {
      if (u0 + c < w) dst[(size_t)v * w + u0 + c] = val;
    };
    // first stage consumes the staging buffers, then the next tile is prefetched
    constexpr RadixList L = factor_radices(N);
    constexpr int R0 = L.r[0];
    ct_stage_io<N, R0, 1, true, true, CW, T, true, L.cnt == 1>(W, 1, CW, TWs, load, store);
    if (next < nitems) prefetch(next);
    if constexpr (L.cnt > 1) ct_fft_io<N, true, true, CW, T, 1, R0>(W, 1, CW, TWs, load, store);
  }
  cp_async_wait_all();
}

__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Shared memory of k_cols_inv_corr_pipe2: two work buffers in the padded
// column layout, the resident H tile (linear), the twiddles.
template <int N>
struct Pipe2Cfg {
  using C = LineCfg<N>;
  static constexpr int SMEM = 2 * C::CW * C::LS * 8 + C::CW * N * 8 + N * 8;
  static constexpr bool OK = SMEM <= 227 * 1024;
};

// Inverse column pass of H^ conj(F^_k) (Sec. 4.1 "Standard Correlation"),
// double-buffered: the spectrum tile of the next item streams into the other
// work buffer while this one is transformed in place.  Item order:
//   REUSE: items (tile, component), component fastest, split into contiguous
//          ranges, one per block; the H tile is loaded once per tile and
//          reused by all its components (wide tiles: long contiguous writes);
//   otherwise: component-major items, block-strided, so blocks running at
//          the same time write adjacent tiles of one component plane (narrow
//          tiles: their short row segments merge in L2); H is loaded per item.
// Output Z[kk] row-major (pitch w).  HERM as in k_cols_inv_corr_pipe.
template <int N, bool HERM, bool REUSE>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, 1)
k_cols_inv_corr_pipe2(const float2* __restrict__ Hh, int w, const float2* __restrict__ S, int k0, int nk,
                      float2* __restrict__ Z, const float2* __restrict__ tw) {
  using C = LineCfg<N>;
  constexpr int T = C::COL_THREADS;
  constexpr int CW = C::CW;
  constexpr int TILE = CW * N;
  constexpr int LS = C::LS;
  extern __shared__ float2 sm[];
  float2* B0 = sm;                       // CW * LS, element (v, c) at c + sidx(v) * CW
  float2* B1 = sm + CW * LS;
  float2* HT = sm + 2 * CW * LS;         // TILE, linear e = v * CW + c
  const float2* TWs = stage_twiddles<N, 2 * CW * LS + TILE>(sm, tw, T);
  const int wh = w / 2 + 1;
  const int ntiles = (w + CW - 1) / CW;
  const long long nitems = (long long)ntiles * nk;
  // this block's items: i = first, first + step, ... < last
  const int first = REUSE ? (int)(nitems * blockIdx.x / gridDim.x) : (int)blockIdx.x;
  const int last = REUSE ? (int)(nitems * (blockIdx.x + 1) / gridDim.x) : (int)nitems;
  const int step = REUSE ? 1 : (int)gridDim.x;
  auto tile_of = [&](int item) { return REUSE ? item / nk : item % ntiles; };
  auto comp_of = [&](int item) { return REUSE ? item % nk : item / ntiles; };

  auto prefetch_spec = [&](int item, float2* buf) {
    const float2* spec = S + ((size_t)(k0 + comp_of(item)) * ntiles + tile_of(item)) * TILE;
    if (CW % 2 == 0) {
      for (int q = threadIdx.x; q < TILE / 2; q += T) {
        const int e = 2 * q, v = e / CW, c = e % CW;
        cp_async16(buf + c + sidx(v) * CW, spec + e, true);
      }
    } else {
      for (int e = threadIdx.x; e < TILE; e += T) cp_async8(buf + e % CW + sidx(e / CW) * CW, spec + e, true);
    }
    cp_async_commit();
  };
  auto load_h = [&](int tile) {
    const int u0 = tile * CW;
    for (int e = threadIdx.x; e < TILE; e += T) {
      const int v = e / CW, u = u0 + e % CW;
      const float2* src = Hh;
      bool valid = u < w;
      if (!HERM) src = valid ? Hh + (size_t)v * w + u : Hh;
      else if (u < wh) src = Hh + (size_t)v * wh + u;
      else if (valid) src = Hh + (size_t)((N - v) % N) * wh + (w - u);
      cp_async8(HT + e, src, valid);
    }
    cp_async_commit();
  };

  if (first < last) prefetch_spec(first, B0);
  int htile = -1, parity = 0;
  for (int item = first; item < last; item += step, parity ^= 1) {
    __syncthreads();                       // the previous item is done with both buffers and HT
    float2* Bc = parity ? B1 : B0;
    float2* Bn = parity ? B0 : B1;
    const int tile = tile_of(item), kk = comp_of(item);
    if (!REUSE || tile != htile) {
      load_h(tile);
      htile = tile;
    }
    if (item + step < last) {
      prefetch_spec(item + step, Bn);
      cp_async_wait_one();                 // this item's spectrum and H tile have landed
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const int u0 = tile * CW;
    float2* dst = Z + (size_t)kk * N * w;
    auto load = [&](int c, int v) -> float2 {
      float2 hv = HT[v * CW + c];
      if (HERM && u0 + c >= wh) hv.y = -hv.y;
      return c_mul(hv, Bc[c + sidx(v) * CW]);
    };
    auto store = [&](int c, int v, float2 val) {
      if (u0 + c < w) dst[(size_t)v * w + u0 + c] = val;
    };
    constexpr RadixList L = factor_radices(N);
    constexpr int R0 = L.r[0];
    ct_stage_io<N, R0, 1, true, true, CW, T, true, L.cnt == 1, true>(Bc, 1, CW, TWs, load, store);
    if constexpr (L.cnt > 1) ct_fft_io<N, true, true, CW, T, 1, R0>(Bc, 1, CW, TWs, load, store);
  }
  cp_async_wait_all();
}

// Inverse column pass of H^ conj(F^_k) staged by the tensor memory
// accelerator: per item one 1D bulk copy brings the spectrum tile (TILE
// contiguous elements) and N / br 2D tensor copies bring the H tile (CW
// columns of the FULL spectrum, rows y .. y+br-1 each) into shared memory,
// both completing on one mbarrier; thread 0 issues them, so the other
// threads spend no instructions on loading.  Items are component-major and
// block-strided (blocks running together write adjacent tiles of one
// component plane).  The next item's copies are issued as soon as the first
// butterfly stage has consumed the staging buffers.  Every wait is bounded:
// on expiry err = EXT_ERR_TIMEOUT and the block stops.  Output Z[kk]
// row-major (pitch w).
template <int N>
struct TmaColCfg {
  using C = LineCfg<N>;
  static constexpr int TILE = C::CW * N;
  // work buffer, then the two staging tiles at 128-byte aligned offsets, then twiddles
  static constexpr int OFF_S = ((C::CW * C::LS + 15) / 16) * 16;
  static constexpr int OFF_H = OFF_S + ((TILE + 15) / 16) * 16;
  static constexpr int OFF_TW = OFF_H + ((TILE + 15) / 16) * 16;
  static constexpr int SMEM = (OFF_TW + N) * 8 + 128;   // + slack to align the base to 128 bytes
  static constexpr bool OK = SMEM <= 227 * 1024 && C::CW % 2 == 0;
  // without the twiddle copy (the stage table read from global memory through L1)
  static constexpr int SMEM_GTW = OFF_TW * 8 + 128;
  static constexpr bool OK_GTW = !OK && SMEM_GTW <= 227 * 1024 && C::CW % 2 == 0;
  // with the split twiddle table (64 + N / 64 entries) instead of the stage table
  static constexpr int SMEM_SPLIT = (OFF_TW + 64 + N / 64) * 8 + 128;
  static constexpr bool OK_SPLIT = !OK && N % 64 == 0 && SMEM_SPLIT <= 227 * 1024 && C::CW % 2 == 0;
};

// Builds the split twiddle table (lo[b] = W_N^b, b < 64; hi[a] = W_N^{64 a},
// a < N / 64, copied from the FP64-derived table W_N^m) in shared memory at
// float2 offset OFF; visible after the caller's next barrier.
template <int N, int OFF>
__device__ __forceinline__ SplitTw split_twiddles(float2* sm, const float2* __restrict__ tw, int threads) {
  float2* lo = sm + OFF;
  float2* hi = lo + 64;
  for (int e = threadIdx.x; e < 64 + N / 64; e += threads) {
    if (e < 64) lo[e] = __ldg(tw + e);
    else hi[e - 64] = __ldg(tw + (size_t)(e - 64) * 64);
  }
  return SplitTw{lo, hi};
}

template <int N>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, 1)
k_cols_inv_corr_tma(const __grid_constant__ CUtensorMap tmH, int w, int br, const float2* __restrict__ S, int k0,
                    int nk, float2* __restrict__ Z, const float2* __restrict__ tw, int* __restrict__ err) {
  using C = LineCfg<N>;
  using TC = TmaColCfg<N>;
  constexpr int T = C::COL_THREADS;
  constexpr int CW = C::CW;
  constexpr int TILE = TC::TILE;
  extern __shared__ float2 sm_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int abort_flag;
  // 128-byte aligned base for the tensor copies
  float2* sm = reinterpret_cast<float2*>(sm_raw) + ((128 - (tc::smem_u32(sm_raw) & 127)) & 127) / 8;
  float2* W = sm;
  float2* SS = sm + TC::OFF_S;
  float2* HS = sm + TC::OFF_H;
  const float2* TWs = stage_twiddles<N, TC::OFF_TW>(sm, tw, T);
  const int ntiles = (w + CW - 1) / CW;
  const int nitems = ntiles * nk;
  const uint32_t mb = tc::smem_u32(&mbar);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    tc::mbar_init(mb, 1);
  }
  __syncthreads();
  // The image spectrum is read once per component: keep it in L2 (evict_last)
  // while the component spectra, read once, stream through (evict_first).
  const uint64_t keep = tc::policy_evict_last(), once = tc::policy_evict_first();
  auto issue = [&](int item) {   // thread 0
    const int kk = item / ntiles, tile = item % ntiles;
    tc::fence_proxy_async();      // earlier generic-proxy reads of the staging tiles come first
    tc::mbar_expect_tx(mb, 2u * TILE * 8u);
    tc::bulk_load_hint(tc::smem_u32(SS), S + ((size_t)(k0 + kk) * ntiles + tile) * TILE, TILE * 8u, mb, once);
    for (int y = 0; y < N; y += br)
      tc::tma_load_2d_hint(tc::smem_u32(HS + y * CW), &tmH, 2 * tile * CW, y, mb, keep);
  };
  uint32_t phase = 0;
  int item = blockIdx.x;
  bool pending = false;
  if (item < nitems && threadIdx.x == 0) issue(item);
  pending = item < nitems;
  for (; item < nitems; item += gridDim.x) {
    if (!tc::mbar_wait_bounded(mb, phase, 1000000000ull, err, EXT_ERR_TIMEOUT)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    phase ^= 1u;
    pending = false;
    const int kk = item / ntiles, tile = item % ntiles;
    const int u0 = tile * CW;
    float2* dst = Z + (size_t)kk * N * w;
    const int next = item + gridDim.x;
    auto load = [&](int c, int v) -> float2 {
      const int e = v * CW + c;
      return c_mul(HS[e], SS[e]);
    };
    auto store = [&](int c, int v, float2 val) {
      // plain stores: the last components written are still in L2 when the
      // inverse row pass, which takes the components in reverse, starts
      if (u0 + c < w) dst[(size_t)v * w + u0 + c] = val;
    };
    constexpr RadixList L = factor_radices(N);
    constexpr int R0 = L.r[0];
    ct_stage_io<N, R0, 1, true, true, CW, T, true, L.cnt == 1>(W, 1, CW, TWs, load, store);
    if (next < nitems) {
      if (threadIdx.x == 0) issue(next);
      pending = true;
    }
    if constexpr (L.cnt > 1) ct_fft_io<N, true, true, CW, T, 1, R0>(W, 1, CW, TWs, load, store);
  }
  // a copy still in flight (timeout path): wait for it, bounded, before the block exits
  if (pending) tc::mbar_wait_bounded(mb, phase, 1000000000ull, err, EXT_ERR_TIMEOUT);
}

// Convolution column pass (extended convolution, Sec. 4.1 last paragraph:
// Y = sum_k FFT(A_k) F^_k, then the inverse column transform) with the
// steered signals and the spectra staged by the tensor memory accelerator:
// per (column tile, k) one set of 2D tensor copies of the A_k tile (A seen as
// (K+1) h rows of 2w floats) and one bulk copy of the spectrum tile, each on
// its own mbarrier.  The next A tile is requested as soon as the first
// butterfly stage has read the current one, the next spectrum tile as soon as
// the products have been accumulated (in registers).  Column tiles are
// strided over the blocks; waits are bounded (err = EXT_ERR_TIMEOUT, the
// block stops).
template <int N, bool FUSED>
__global__ void __launch_bounds__(LineCfg<N>::COL_THREADS, 1)
k_cols_conv_tma(const __grid_constant__ CUtensorMap tmA, int w, int br, int K, int nsig, const float2* __restrict__ S,
                float2* __restrict__ Y, const float2* __restrict__ tw, const float2* __restrict__ stw_g,
                int* __restrict__ err) {
  using C = LineCfg<N>;
  using TC = TmaColCfg<N>;
  using LC = LastColStage<N, C::CW, C::COL_THREADS>;
  constexpr int T = C::COL_THREADS;
  constexpr int CW = C::CW;
  constexpr int TILE = TC::TILE;
  constexpr int NACC = FUSED ? LC::S * LC::R : C::COL_EPT;
  extern __shared__ float2 sm_raw[];
  __shared__ __align__(8) uint64_t bar_a, bar_s;
  __shared__ int abort_a, abort_s;   // separate flags: each is read only after a barrier that follows its writes
  float2* sm = reinterpret_cast<float2*>(sm_raw) + ((128 - (tc::smem_u32(sm_raw) & 127)) & 127) / 8;
  float2* W = sm;
  float2* SS = sm + TC::OFF_S;
  float2* AS = sm + TC::OFF_H;
  // stage twiddles: copied into shared memory where they fit, else the split
  // table in shared memory, else the global stage table (stw_g)
  const auto TWs = [&]() {
    if constexpr (TC::OK) return stage_twiddles<N, TC::OFF_TW>(sm, tw, T);
    else if constexpr (TC::OK_SPLIT) return split_twiddles<N, TC::OFF_TW>(sm, tw, T);
    else return stw_g;
  }();
  const int ntiles = (w + CW - 1) / CW;
  const uint32_t ma = tc::smem_u32(&bar_a), ms = tc::smem_u32(&bar_s);
  if (threadIdx.x == 0) {
    abort_a = 0;
    abort_s = 0;
    tc::mbar_init(ma, 1);
    tc::mbar_init(ms, 1);
  }
  __syncthreads();
  // items: (column tile, signal), signal fastest, so the blocks of all signals of a tile run
  // together and read each spectrum tile from HBM once and from L2 for the other signals
  const int nitems = ntiles * nsig;
  auto issue_a = [&](int item, int k) {   // thread 0; signal sig's component k is A row block sig (K+1) + k
    const int tile = item / nsig, sig = item % nsig;
    tc::fence_proxy_async();
    tc::mbar_expect_tx(ma, TILE * 8u);
    for (int y = 0; y < N; y += br)
      tc::tma_load_2d(tc::smem_u32(AS + y * CW), &tmA, 2 * tile * CW, (sig * (K + 1) + k) * N + y, ma);
  };
  auto issue_s = [&](int item, int k) {   // thread 0
    const int tile = item / nsig;
    tc::fence_proxy_async();
    tc::mbar_expect_tx(ms, TILE * 8u);
    tc::bulk_load(tc::smem_u32(SS), S + ((size_t)k * ntiles + tile) * TILE, TILE * 8u, ms);
  };
  constexpr RadixList L = factor_radices(N);
  constexpr int R0 = L.r[0];
  static_assert(L.cnt > 1, "at least two radix stages");
  uint32_t pa = 0, ps = 0;
  bool pend_a = false, pend_s = false;
  if ((int)blockIdx.x < nitems) {
    if (threadIdx.x == 0) {
      issue_a(blockIdx.x, 0);
      issue_s(blockIdx.x, 0);
    }
    pend_a = pend_s = true;
  }
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item / nsig;
    const int u0 = tile * CW;
    float2* const Ysig = Y + (size_t)(item % nsig) * N * w;
    const int next_item = item + gridDim.x;
    float2 acc[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int k = 0; k <= K; ++k) {
      const bool more = k < K || next_item < nitems;
      const int nt = k < K ? item : next_item, nk = k < K ? k + 1 : 0;
      if (!tc::mbar_wait_bounded(ma, pa, 1000000000ull, err, EXT_ERR_TIMEOUT)) abort_a = 1;
      if constexpr (!FUSED) {
        __syncthreads();
        if (abort_a) break;
      }
      pa ^= 1u;
      pend_a = false;
      auto load = [&](int c, int v) -> float2 { return AS[v * CW + c]; };
      auto nostore = [](int, int, float2) {};
      ct_stage_io<N, R0, 1, false, true, CW, T, true, false>(W, 1, CW, TWs, load, nostore);   // ends with a barrier
      if constexpr (FUSED) {
        if (abort_a) break;
      }
      if (more) {   // the first stage has read the A tile
        if (threadIdx.x == 0) issue_a(nt, nk);
        pend_a = true;
      }
      if constexpr (FUSED) {
        // middle stages in place, then the last stage multiplies its outputs
        // with the staged spectrum tile (laid out in the order of the
        // outputs) and accumulates them in registers
        ct_fft_range<N, false, true, CW, T, 1, L.cnt - 1, R0>(W, 1, CW, TWs);
        if (!tc::mbar_wait_bounded(ms, ps, 1000000000ull, err, EXT_ERR_TIMEOUT)) abort_s = 1;
        ps ^= 1u;
        pend_s = false;
        ct_last_stage_cols<N, CW, T>(W, CW, TWs, [&](int s2, int r, float2 v) {
          const float2 sp = SS[LC::x(s2, r) * CW + LC::line(s2)];
          float2& a = acc[s2 * LC::R + r];
          a.x = fmaf(v.x, sp.x, fmaf(-v.y, sp.y, a.x));
          a.y = fmaf(v.x, sp.y, fmaf(v.y, sp.x, a.y));
        });
        __syncthreads();   // W and the spectrum tile read
        if (abort_s) break;
      } else {
        ct_fft<N, false, true, CW, T, 1, R0>(W, 1, CW, TWs);
        if (!tc::mbar_wait_bounded(ms, ps, 1000000000ull, err, EXT_ERR_TIMEOUT)) abort_s = 1;
        __syncthreads();
        if (abort_s) break;
        ps ^= 1u;
        pend_s = false;
        for_elems<C::CW * N, T>([&](int i, int e) {
          const float2 sp = SS[e];
          const float2 x = W[e % CW + sidx(e / CW) * CW];
          acc[i].x = fmaf(x.x, sp.x, fmaf(-x.y, sp.y, acc[i].x));
          acc[i].y = fmaf(x.x, sp.y, fmaf(x.y, sp.x, acc[i].y));
        });
        __syncthreads();   // products read W and the spectrum tile
      }
      if (more) {
        if (threadIdx.x == 0) issue_s(nt, nk);
        pend_s = true;
      }
    }
    if (abort_a || abort_s) break;
    if constexpr (FUSED) {
#pragma unroll
      for (int s2 = 0; s2 < LC::S; ++s2)
#pragma unroll
        for (int r = 0; r < LC::R; ++r)
          if (LC::valid(s2)) W[LC::line(s2) + sidx(LC::x(s2, r)) * CW] = acc[s2 * LC::R + r];
    } else {
      cols_store_sm<N>(W, acc);
    }
    __syncthreads();
    col_fft<N, true>(W, TWs);
    for_elems<C::CW * N, T>([&](int i, int e) {
      const int u = u0 + e % CW;
      if (u < w) Ysig[(size_t)(e / CW) * w + u] = W[e % CW + sidx(e / CW) * CW];
    });
    __syncthreads();
  }
  // copies still in flight (timeout path): wait for them, bounded, before the block exits
  if (threadIdx.x == 0) {
    if (pend_a) tc::mbar_wait_bounded(ma, pa, 1000000000ull, err, EXT_ERR_TIMEOUT);
    if (pend_s) tc::mbar_wait_bounded(ms, ps, 1000000000ull, err, EXT_ERR_TIMEOUT);
  }
}

// Inverse row pass of Z writing the component planes of G (k = k0 + item / nblk).
// The RL rows of the next item (contiguous in Z) arrive by one bulk copy
// completing on an mbarrier, issued by thread 0 as soon as the first
// butterfly stage has consumed the staging buffer; waits are bounded (err =
// EXT_ERR_TIMEOUT, the block stops).
template <int N>
__global__ void __launch_bounds__(LineCfg<N>::ROW_THREADS, 1)
k_rows_inv_components_pipe(const float2* __restrict__ Z, int h, int k0, int nk, float* __restrict__ G,
                           const float2* __restrict__ tw, int* __restrict__ err) {
  using C = LineCfg<N>;
  constexpr int T = C::ROW_THREADS;
  constexpr int RL = C::RL;
  static_assert((RL * C::LS) % 2 == 0, "staging buffer must be 16-byte aligned");
  extern __shared__ float2 sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int abort_flag;
  float2* W = sm;
  float2* ZS = sm + RL * C::LS;   // RL * N linear
  const float2* TWs = stage_twiddles<N, RL * C::LS + RL * N>(sm, tw, T);
  const size_t P = (size_t)h * N;
  const int nblk = (h + RL - 1) / RL;
  const int nitems = nblk * nk;
  const uint32_t mb = tc::smem_u32(&mbar);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    tc::mbar_init(mb, 1);
  }
  __syncthreads();
  auto prefetch = [&](int item) {   // thread 0
    const int kk = nk - 1 - item / nblk, y0 = (item % nblk) * RL;   // last-written components first
    const int rows = (h - y0) < RL ? (h - y0) : RL;
    const uint32_t bytes = (uint32_t)rows * N * 8u;
    tc::fence_proxy_async();
    tc::mbar_expect_tx(mb, bytes);
    tc::bulk_load(tc::smem_u32(ZS), Z + (size_t)kk * P + (size_t)y0 * N, bytes, mb);
  };

  uint32_t phase = 0;
  int item = blockIdx.x;
  bool pending = item < nitems;
  if (pending && threadIdx.x == 0) prefetch(item);
  for (; item < nitems; item += gridDim.x) {
    if (!tc::mbar_wait_bounded(mb, phase, 1000000000ull, err, EXT_ERR_TIMEOUT)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    phase ^= 1u;
    pending = false;
    const int kk = nk - 1 - item / nblk, y0 = (item % nblk) * RL;   // last-written components first
    const int k = k0 + kk;
    float* re = G + (k == 0 ? 0 : (size_t)(2 * k - 1) * P);
    float* im = G + (size_t)(2 * k) * P;
    const int next = item + gridDim.x;
    auto load = [&](int l, int x) -> float2 { return ZS[l * N + x]; };
    auto store = [&](int l, int x, float2 val) {
      const int y = y0 + l;
      if (y < h) {
        const size_t idx = (size_t)y * N + x;
        re[idx] = val.x;
        if (k != 0) im[idx] = val.y;
      }
    };
    constexpr RadixList L = factor_radices(N);
    constexpr int R0 = L.r[0];
    ct_stage_io<N, R0, 1, true, false, RL, T, true, L.cnt == 1>(W, C::LS, 1, TWs, load, store);
    if (next < nitems) {
      if (threadIdx.x == 0) prefetch(next);
      pending = true;
    }
    if constexpr (L.cnt > 1) ct_fft_io<N, true, false, RL, T, 1, R0>(W, C::LS, 1, TWs, load, store);
  }
  if (pending) tc::mbar_wait_bounded(mb, phase, 1000000000ull, err, EXT_ERR_TIMEOUT);
}

// ------------------------------------------------------------- launchers ---
template <int N>
struct FftOps {
  using C = LineCfg<N>;
  static bool cols_inv_corr_tma(const CUtensorMap& tmH, int w, int br, const float2* S, int k0, int nk, float2* Z,
                                const float2* tw, int* err, int sms, cudaStream_t st);
  static bool planes_fwd_c2c(float2* U, int nplanes, const float2* tw, int* err, int sms, cudaStream_t st);
  static bool planes_inv_channels(const float2* Z, int nz, int k0, int nk, const int2* chan, float* G,
                                  const float2* tw, int* err, int sms, cudaStream_t st);
  static void rows_r2c(const float* H, int h, float2* Hh, const float2* tw, cudaStream_t st);
  static void rows_fwd_phase(const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                             const float2* tw, cudaStream_t st);
  static void rows_c2c(const float2* X, int h, int nplanes, float2* Y, bool inv, const float2* tw,
                       cudaStream_t st);
  static void rows_fwd_simil(const float* H, const float4* uv, const float* s, int h, const int2* kj, int ncomp,
                             int unit_integral, float2* A, const float2* tw, cudaStream_t st);
  static void rows_fwd_scale_turns(const float* H, const float2* T, int h, int k0, int nk, float2* A,
                                   const float2* tw, cudaStream_t st);
  static void rows_fwd_simil_turns(const float* H, const float4* T, int h, const int2* kj, int ncomp, float2* A,
                                   const float2* tw, cudaStream_t st);
  static void rows_fwd_phase_io(const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                                const float2* tw, cudaStream_t st);
  // component-loop variants (false where the line length has no 16 x R1 x R2 plan)
  static bool rows_fwd_hloop_scale(const float* H, const float2* T, int h, int k0, int nk, float2* A,
                                   const float2* tw, int sms, bool fast, cudaStream_t st);
  static bool rows_fwd_hloop_simil(const float* H, const float4* T, int h, const int2* kj, int ncomp, float2* A,
                                   const float2* tw, int sms, bool fast, cudaStream_t st);
  static bool rows_fwd_hloop_phase(const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                                   const float2* tw, int sms, bool fast, cudaStream_t st);
  static void rows_fwd_scale(const float* H, const float* s, int h, int k0, int nk, float omega_step,
                             int unit_integral, float2* A, const float2* tw, cudaStream_t st);
  static void rows_inv_components(const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                                  cudaStream_t st);
  static void rows_inv_field(const float2* Z, int h, int K, const float* alpha, float* out,
                             const float2* tw, cudaStream_t st);
  static void rows_inv_real(const float2* Y, int h, float* out, const float2* tw, cudaStream_t st);
  static void cols_fwd_half(float2* Hh, int ncols, const float2* tw, cudaStream_t st, float2* Hf, int w);
  static void cols_fwd_spectrum(const float2* X, int w, int conj_out, float scale, float2* S,
                                const float2* tw, cudaStream_t st, int nplanes, float scale_rest);
  static void cols_inv_corr(const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                            const float2* tw, cudaStream_t st);
  static void cols_conv(const float2* A, int w, int K, const float2* S, float2* Y, const float2* tw,
                        cudaStream_t st);
  static bool cols_conv_tma(const CUtensorMap& tmA, int w, int br, int K, int nsig, const float2* S, float2* Y,
                            const float2* tw, const float2* stw_g, int* err, int sms, bool fused, cudaStream_t st);
  static void cols_c2c(float2* X, int w, int planes, bool inv, const float2* tw, cudaStream_t st);
  static void rows_inv_channels(const float2* Z, int rows, int k0, int nk, const int2* chan, float* G,
                                const float2* tw, cudaStream_t st);
  static bool cols_inv_full_pipe(const float2* H, int w, const float2* S, int k0, int nk, float2* Z,
                                 const float2* tw, int sms, cudaStream_t st);
  // pipelined persistent variants (false if the shared-memory plan does not fit)
  static bool cols_inv_corr_pipe(const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                                 const float2* tw, int sms, cudaStream_t st);
  static bool rows_inv_components_pipe(const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                                       int* err, int sms, cudaStream_t st);
};

bool ext_smem_optin(const void* func, int bytes);   // api.cu

// The dynamic shared-memory opt-in is a per-device function attribute: it is
// requested on every launch path and set once per (device, kernel, size).
template <typename KernelT>
static inline bool ext_set_smem(KernelT kernel, int bytes) {
  return ext_smem_optin((const void*)kernel, bytes);
}

template <int N>
void FftOps<N>::rows_r2c(const float* H, int h, float2* Hh, const float2* tw, cudaStream_t st) {
  const bool once = (ext_set_smem(k_rows_r2c<N>, C::ROW_SMEM), true);
  (void)once;
  const int pairs = (h + 1) / 2;
  dim3 grid((pairs + C::RL - 1) / C::RL);
  k_rows_r2c<N><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(H, h, Hh, tw);
}

template <int N>
void FftOps<N>::rows_fwd_phase(const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                               const float2* tw, cudaStream_t st) {
  const bool once = (ext_set_smem(k_rows_fwd_phase<N>, C::ROW_SMEM), true);
  (void)once;
  dim3 grid(nk, (h + C::RL - 1) / C::RL);
  k_rows_fwd_phase<N><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(H, alpha, h, k0, A, tw);
}

template <int N>
void FftOps<N>::rows_c2c(const float2* X, int h, int nplanes, float2* Y, bool inv, const float2* tw,
                         cudaStream_t st) {
  const bool once = (ext_set_smem(k_rows_c2c<N, false>, C::ROW_SMEM),
                            ext_set_smem(k_rows_c2c<N, true>, C::ROW_SMEM), true);
  (void)once;
  dim3 grid((h + C::RL - 1) / C::RL, nplanes);
  if (inv) k_rows_c2c<N, true><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(X, h, Y, tw);
  else k_rows_c2c<N, false><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(X, h, Y, tw);
}

template <int N>
void FftOps<N>::rows_inv_components(const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                                    cudaStream_t st) {
  const bool once = (ext_set_smem(k_rows_inv_components<N>, C::ROW_SMEM), true);
  (void)once;
  dim3 grid((h + C::RL - 1) / C::RL, nk);
  k_rows_inv_components<N><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(Z, h, k0, G, tw);
}

template <int N>
void FftOps<N>::rows_inv_field(const float2* Z, int h, int K, const float* alpha, float* out,
                               const float2* tw, cudaStream_t st) {
  constexpr int smem = C::ROW_SMEM + C::RL * N * 4;
  const bool once = (ext_set_smem(k_rows_inv_field<N>, smem), true);
  (void)once;
  dim3 grid((h + C::RL - 1) / C::RL);
  k_rows_inv_field<N><<<grid, C::ROW_THREADS, smem, st>>>(Z, h, K, alpha, out, tw);
}

template <int N>
void FftOps<N>::rows_inv_real(const float2* Y, int h, float* out, const float2* tw, cudaStream_t st) {
  const bool once = (ext_set_smem(k_rows_inv_real<N>, C::ROW_SMEM), true);
  (void)once;
  dim3 grid((h + C::RL - 1) / C::RL);
  k_rows_inv_real<N><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(Y, h, out, tw);
}

template <int N>
void FftOps<N>::cols_fwd_half(float2* Hh, int ncols, const float2* tw, cudaStream_t st, float2* Hf, int w) {
  const bool once = (ext_set_smem(k_cols_fwd_half<N>, C::COL_SMEM), true);
  (void)once;
  dim3 grid((ncols + C::CW - 1) / C::CW);
  k_cols_fwd_half<N><<<grid, C::COL_THREADS, C::COL_SMEM, st>>>(Hh, ncols, tw, Hf, w);
}

template <int N>
void FftOps<N>::cols_fwd_spectrum(const float2* X, int w, int conj_out, float scale, float2* S,
                                  const float2* tw, cudaStream_t st, int nplanes, float scale_rest) {
  const bool once = (ext_set_smem(k_cols_fwd_spectrum<N>, C::COL_SMEM), true);
  (void)once;
  dim3 grid((w + C::CW - 1) / C::CW, nplanes);
  k_cols_fwd_spectrum<N><<<grid, C::COL_THREADS, C::COL_SMEM, st>>>(X, w, conj_out, scale, scale_rest, S, tw);
}

template <int N>
void FftOps<N>::cols_inv_corr(const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                              const float2* tw, cudaStream_t st) {
  const bool once = (ext_set_smem(k_cols_inv_corr<N>, C::COL_SMEM), true);
  (void)once;
  dim3 grid((w + C::CW - 1) / C::CW, nk);
  k_cols_inv_corr<N><<<grid, C::COL_THREADS, C::COL_SMEM, st>>>(Hh, w, S, k0, Z, tw);
}

template <int N>
void FftOps<N>::cols_conv(const float2* A, int w, int K, const float2* S, float2* Y, const float2* tw,
                          cudaStream_t st) {
  const bool once = (ext_set_smem(k_cols_conv<N>, C::COL_SMEM), true);
  (void)once;
  dim3 grid((w + C::CW - 1) / C::CW);
  k_cols_conv<N><<<grid, C::COL_THREADS, C::COL_SMEM, st>>>(A, w, K, S, Y, tw);
}

template <int N>
static inline int pipe_grid(int items, int sms, int smem, int threads) {
  int bps = (227 * 1024) / (smem + 1024);
  const int by_threads = 2048 / threads;
  if (bps > by_threads) bps = by_threads;
  if (bps > 16) bps = 16;
  if (bps < 1) bps = 1;
  const long long cap = (long long)sms * bps;
  return items < cap ? items : (int)cap;
}

template <int N>
bool FftOps<N>::cols_inv_corr_pipe(const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                                   const float2* tw, int sms, cudaStream_t st) {
  if constexpr (!PipeCfg<N>::COL_OK) {
    return false;
  } else {
    const int items = ((w + C::CW - 1) / C::CW) * nk;
    // the double-buffered pass wins for wide tiles (measured: 128-point columns
    // 1.94 -> 1.33 ms over 231 components of 128^3); for 2048-point columns
    // (4-column tiles) the single-buffered pass is faster (0.45 vs 0.50 ms)
    if constexpr (Pipe2Cfg<N>::OK && C::CW >= 16) {
      constexpr bool REUSE = true;
      const bool once2 = (ext_set_smem(k_cols_inv_corr_pipe2<N, true, REUSE>, Pipe2Cfg<N>::SMEM), true);
      (void)once2;
      const int grid = pipe_grid<N>(items, sms, Pipe2Cfg<N>::SMEM, C::COL_THREADS);
      k_cols_inv_corr_pipe2<N, true, REUSE><<<grid, C::COL_THREADS, Pipe2Cfg<N>::SMEM, st>>>(Hh, w, S, k0, nk, Z, tw);
      return true;
    }
    const bool once = (ext_set_smem(k_cols_inv_corr_pipe<N, true>, PipeCfg<N>::COL_SMEM), true);
    (void)once;
    const int grid = pipe_grid<N>(items, sms, PipeCfg<N>::COL_SMEM, C::COL_THREADS);
    k_cols_inv_corr_pipe<N, true><<<grid, C::COL_THREADS, PipeCfg<N>::COL_SMEM, st>>>(Hh, w, S, k0, nk, Z, tw);
    return true;
  }
}

template <int N>
bool FftOps<N>::cols_inv_corr_tma(const CUtensorMap& tmH, int w, int br, const float2* S, int k0, int nk, float2* Z,
                                  const float2* tw, int* err, int sms, cudaStream_t st) {
  if constexpr (!TmaColCfg<N>::OK) {
    return false;
  } else {
    const bool once = (ext_set_smem(k_cols_inv_corr_tma<N>, TmaColCfg<N>::SMEM), true);
    (void)once;
    const int items = ((w + C::CW - 1) / C::CW) * nk;
    const int grid = pipe_grid<N>(items, sms, TmaColCfg<N>::SMEM, C::COL_THREADS);
    k_cols_inv_corr_tma<N><<<grid, C::COL_THREADS, TmaColCfg<N>::SMEM, st>>>(tmH, w, br, S, k0, nk, Z, tw, err);
    return true;
  }
}

template <int N>
bool FftOps<N>::cols_conv_tma(const CUtensorMap& tmA, int w, int br, int K, int nsig, const float2* S, float2* Y,
                              const float2* tw, const float2* stw_g, int* err, int sms, bool fused,
                              cudaStream_t st) {
  using TC = TmaColCfg<N>;
  if constexpr (!(TC::OK || TC::OK_GTW) || factor_radices(N).cnt < 2) {
    return false;
  } else {
    if (!TC::OK && !TC::OK_SPLIT && !stw_g) return false;
    constexpr int smem = TC::OK ? TC::SMEM : (TC::OK_SPLIT ? TC::SMEM_SPLIT : TC::SMEM_GTW);
    const int items = (w + C::CW - 1) / C::CW * nsig;
    const int grid = pipe_grid<N>(items, sms, smem, C::COL_THREADS);
    if (fused) {
      if (!ext_set_smem(k_cols_conv_tma<N, true>, smem)) return false;
      k_cols_conv_tma<N, true><<<grid, C::COL_THREADS, smem, st>>>(tmA, w, br, K, nsig, S, Y, tw, stw_g, err);
    } else {
      if (!ext_set_smem(k_cols_conv_tma<N, false>, smem)) return false;
      k_cols_conv_tma<N, false><<<grid, C::COL_THREADS, smem, st>>>(tmA, w, br, K, nsig, S, Y, tw, stw_g, err);
    }
    return true;
  }
}

// Stage twiddle table of length n (the layout stage_twiddles builds) in global memory.
template <int N>
__global__ void k_stage_table(const float2* __restrict__ tw, float2* __restrict__ out) {
  stage_twiddles<N, 0>(out, tw, blockDim.x);
}

template <int N>
bool FftOps<N>::planes_fwd_c2c(float2* U, int nplanes, const float2* tw, int* err, int sms, cudaStream_t st) {
  if constexpr (!PlaneCfg<N>::OK) {
    return false;
  } else {
    const bool once = (ext_set_smem(k_planes_fwd_c2c<N>, PlaneCfg<N>::SMEM), true);
    (void)once;
    int per_sm = (227 * 1024) / (PlaneCfg<N>::SMEM + 1024);
    const int by_threads = 2048 / PlaneCfg<N>::THREADS;
    if (per_sm > by_threads) per_sm = by_threads;
    if (per_sm < 1) per_sm = 1;
    const int grid = nplanes < sms * per_sm ? nplanes : sms * per_sm;
    k_planes_fwd_c2c<N><<<grid, PlaneCfg<N>::THREADS, PlaneCfg<N>::SMEM, st>>>(U, nplanes, tw, err);
    return true;
  }
}

template <int N>
bool FftOps<N>::planes_inv_channels(const float2* Z, int nz, int k0, int nk, const int2* chan, float* G,
                                    const float2* tw, int* err, int sms, cudaStream_t st) {
  if constexpr (!PlaneCfg<N>::OK) {
    return false;
  } else {
    const bool once = (ext_set_smem(k_planes_inv_channels<N>, PlaneCfg<N>::SMEM), true);
    (void)once;
    const int planes = nk * nz;
    int per_sm = (227 * 1024) / (PlaneCfg<N>::SMEM + 1024);
    const int by_threads = 2048 / PlaneCfg<N>::THREADS;
    if (per_sm > by_threads) per_sm = by_threads;
    if (per_sm < 1) per_sm = 1;
    const int grid = planes < sms * per_sm ? planes : sms * per_sm;
    k_planes_inv_channels<N><<<grid, PlaneCfg<N>::THREADS, PlaneCfg<N>::SMEM, st>>>(Z, nz, k0, nk, chan, G, tw, err);
    return true;
  }
}

template <int N>
bool FftOps<N>::cols_inv_full_pipe(const float2* H, int w, const float2* S, int k0, int nk, float2* Z,
                                   const float2* tw, int sms, cudaStream_t st) {
  if constexpr (!PipeCfg<N>::COL_OK) {
    return false;
  } else {
    const int items = ((w + C::CW - 1) / C::CW) * nk;
    if constexpr (Pipe2Cfg<N>::OK && C::CW >= 16) {
      constexpr bool REUSE = true;
      const bool once2 = (ext_set_smem(k_cols_inv_corr_pipe2<N, false, REUSE>, Pipe2Cfg<N>::SMEM), true);
      (void)once2;
      const int grid = pipe_grid<N>(items, sms, Pipe2Cfg<N>::SMEM, C::COL_THREADS);
      k_cols_inv_corr_pipe2<N, false, REUSE><<<grid, C::COL_THREADS, Pipe2Cfg<N>::SMEM, st>>>(H, w, S, k0, nk, Z, tw);
      return true;
    }
    const bool once = (ext_set_smem(k_cols_inv_corr_pipe<N, false>, PipeCfg<N>::COL_SMEM), true);
    (void)once;
    const int grid = pipe_grid<N>(items, sms, PipeCfg<N>::COL_SMEM, C::COL_THREADS);
    k_cols_inv_corr_pipe<N, false><<<grid, C::COL_THREADS, PipeCfg<N>::COL_SMEM, st>>>(H, w, S, k0, nk, Z, tw);
    return true;
  }
}

template <int N>
void FftOps<N>::cols_c2c(float2* X, int w, int planes, bool inv, const float2* tw, cudaStream_t st) {
  const bool once = (ext_set_smem(k_cols_c2c<N, false>, C::COL_SMEM),
                            ext_set_smem(k_cols_c2c<N, true>, C::COL_SMEM), true);
  (void)once;
  dim3 grid((w + C::CW - 1) / C::CW, planes);
  if (inv) k_cols_c2c<N, true><<<grid, C::COL_THREADS, C::COL_SMEM, st>>>(X, w, tw);
  else k_cols_c2c<N, false><<<grid, C::COL_THREADS, C::COL_SMEM, st>>>(X, w, tw);
}

template <int N>
void FftOps<N>::rows_inv_channels(const float2* Z, int rows, int k0, int nk, const int2* chan, float* G,
                                  const float2* tw, cudaStream_t st) {
  const bool once = (ext_set_smem(k_rows_inv_channels<N>, C::ROW_SMEM), true);
  (void)once;
  dim3 grid((rows + C::RL - 1) / C::RL, nk);
  k_rows_inv_channels<N><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(Z, rows, k0, chan, G, tw);
}

template <int N>
bool FftOps<N>::rows_inv_components_pipe(const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                                         int* err, int sms, cudaStream_t st) {
  if constexpr (!PipeCfg<N>::ROW_OK) {
    return false;
  } else {
    const bool once = (ext_set_smem(k_rows_inv_components_pipe<N>, PipeCfg<N>::ROW_SMEM), true);
    (void)once;
    const int items = ((h + C::RL - 1) / C::RL) * nk;
    const int grid = pipe_grid<N>(items, sms, PipeCfg<N>::ROW_SMEM, C::ROW_THREADS);
    k_rows_inv_components_pipe<N><<<grid, C::ROW_THREADS, PipeCfg<N>::ROW_SMEM, st>>>(Z, h, k0, nk, G, tw, err);
    return true;
  }
}

template <int N>
void FftOps<N>::rows_fwd_simil(const float* H, const float4* uv, const float* s, int h, const int2* kj, int ncomp,
                               int unit_integral, float2* A, const float2* tw, cudaStream_t st) {
  const bool once = (ext_set_smem(k_rows_fwd_simil<N>, C::ROW_SMEM), true);
  (void)once;
  dim3 grid(ncomp, (h + C::RL - 1) / C::RL);
  k_rows_fwd_simil<N><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(H, uv, s, h, kj, unit_integral, A, tw);
}

template <int N, class Steer>
static void launch_rows_fwd_steered(const Steer& sp, int h, int ncomp, float2* A, const float2* tw, cudaStream_t st) {
  using C = LineCfg<N>;
  const bool once = (ext_set_smem(k_rows_fwd_steered<N, Steer>, C::ROW_SMEM), true);
  (void)once;
  dim3 grid(ncomp, (h + C::RL - 1) / C::RL);
  k_rows_fwd_steered<N, Steer><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(sp, h, A, tw);
}

// Component groups of the component-loop pass: the group count G minimises
// waves(h G blocks) x (ceil(ncomp / G) + 1), a block taking about one
// component's time for its loads and twiddle staging plus one per component.
inline int hloop_groups(int nrb, int ncomp, int slots) {
  long long best = -1;
  int bg = 1;
  for (int g = 1; g <= ncomp; ++g) {
    const int cpb = (ncomp + g - 1) / g;
    if (g > 1 && (ncomp + cpb - 1) / cpb < g) continue;   // same split as a smaller g
    const long long waves = ((long long)nrb * g + slots - 1) / slots;
    const long long cost = waves * (cpb + 1);
    if (best < 0 || cost < best) {
      best = cost;
      bg = g;
    }
  }
  return bg;
}

template <int N, class Steer>
static bool launch_rows_fwd_hloop(const Steer& sp, int h, int ncomp, float2* A, const float2* tw, int sms,
                                  cudaStream_t st) {
  using HC = HloopCfg<N>;
  if constexpr (!HC::OK) {
    return false;
  } else {
    if (!ext_set_smem(k_rows_fwd_hloop<N, Steer>, HC::SMEM)) return false;
    const int nrb = (h + HC::RB - 1) / HC::RB;
    const int g = hloop_groups(nrb, ncomp, sms * HC::MINB);
    const int cpb = (ncomp + g - 1) / g;
    dim3 grid(nrb, (ncomp + cpb - 1) / cpb);
    k_rows_fwd_hloop<N, Steer><<<grid, HC::THREADS, HC::SMEM, st>>>(sp, h, ncomp, cpb, A, tw);
    return true;
  }
}

template <int N>
bool FftOps<N>::rows_fwd_hloop_scale(const float* H, const float2* T, int h, int k0, int nk, float2* A,
                                     const float2* tw, int sms, bool fast, cudaStream_t st) {
  if (fast) return launch_rows_fwd_hloop<N>(HloopScale<true>{H, T, k0}, h, nk, A, tw, sms, st);
  return launch_rows_fwd_hloop<N>(HloopScale<false>{H, T, k0}, h, nk, A, tw, sms, st);
}

template <int N>
bool FftOps<N>::rows_fwd_hloop_simil(const float* H, const float4* T, int h, const int2* kj, int ncomp, float2* A,
                                     const float2* tw, int sms, bool fast, cudaStream_t st) {
  if (fast) return launch_rows_fwd_hloop<N>(HloopSimil<true>{H, T, kj}, h, ncomp, A, tw, sms, st);
  return launch_rows_fwd_hloop<N>(HloopSimil<false>{H, T, kj}, h, ncomp, A, tw, sms, st);
}

template <int N>
bool FftOps<N>::rows_fwd_hloop_phase(const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                                     const float2* tw, int sms, bool fast, cudaStream_t st) {
  if (fast) return launch_rows_fwd_hloop<N>(HloopPhase<true>{H, alpha, k0}, h, nk, A, tw, sms, st);
  return launch_rows_fwd_hloop<N>(HloopPhase<false>{H, alpha, k0}, h, nk, A, tw, sms, st);
}

template <int N>
void FftOps<N>::rows_fwd_scale_turns(const float* H, const float2* T, int h, int k0, int nk, float2* A,
                                     const float2* tw, cudaStream_t st) {
  launch_rows_fwd_steered<N>(SteerScale{H, T, k0}, h, nk, A, tw, st);
}

template <int N>
void FftOps<N>::rows_fwd_simil_turns(const float* H, const float4* T, int h, const int2* kj, int ncomp, float2* A,
                                     const float2* tw, cudaStream_t st) {
  launch_rows_fwd_steered<N>(SteerSimil{H, T, kj}, h, ncomp, A, tw, st);
}

template <int N>
void FftOps<N>::rows_fwd_phase_io(const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                                  const float2* tw, cudaStream_t st) {
  launch_rows_fwd_steered<N>(SteerPhase{H, alpha, k0}, h, nk, A, tw, st);
}

template <int N>
void FftOps<N>::rows_fwd_scale(const float* H, const float* s, int h, int k0, int nk, float omega_step,
                               int unit_integral, float2* A, const float2* tw, cudaStream_t st) {
  const bool once = (ext_set_smem(k_rows_fwd_scale<N>, C::ROW_SMEM), true);
  (void)once;
  dim3 grid((h + C::RL - 1) / C::RL, nk);
  k_rows_fwd_scale<N><<<grid, C::ROW_THREADS, C::ROW_SMEM, st>>>(H, s, h, k0, omega_step, unit_integral, A, tw);
}
