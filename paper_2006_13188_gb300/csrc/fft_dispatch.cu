// Runtime dispatch of the 2D FFT passes onto the compile-time line lengths.
#include "fft2d.cuh"
#include "internal.h"

#include <algorithm>

#define EXT_EXTERN(N) extern template struct FftOps<N>;
EXT_FFT_SIZES(EXT_EXTERN)
#undef EXT_EXTERN

bool fft_size_supported(int n) {
  switch (n) {
#define EXT_CASE(N) case N: return true;
    EXT_FFT_SIZES(EXT_CASE)
#undef EXT_CASE
    default: return false;
  }
}

int fft_col_tile(int n) {
  switch (n) {
#define EXT_CASE(N) case N: return LineCfg<N>::CW;
    EXT_FFT_SIZES(EXT_CASE)
#undef EXT_CASE
    default: return 0;
  }
}

#define EXT_C1(N) case N: FftOps<N>::rows_r2c(H, h, Hh, tw, st); return;
void fft_rows_r2c(int w, const float* H, int h, float2* Hh, const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_fwd_phase(H, alpha, h, k0, nk, A, tw, st); return;
void fft_rows_fwd_phase(int w, const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                        const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_c2c(X, h, nplanes, Y, inv, tw, st); return;
void fft_rows_c2c(int w, const float2* X, int h, int nplanes, float2* Y, bool inv, const float2* tw,
                  cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_inv_components(Z, h, k0, nk, G, tw, st); return;
void fft_rows_inv_components(int w, const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                             cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_inv_field(Z, h, K, alpha, out, tw, st); return;
void fft_rows_inv_field(int w, const float2* Z, int h, int K, const float* alpha, float* out,
                        const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_inv_real(Y, h, out, tw, st); return;
void fft_rows_inv_real(int w, const float2* Y, int h, float* out, const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::cols_fwd_half(Hh, ncols, tw, st, Hf, w); return;
void fft_cols_fwd_half(int h, float2* Hh, int ncols, const float2* tw, cudaStream_t st, float2* Hf, int w) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::cols_fwd_spectrum(X, w, conj_out, scale, S, tw, st, nplanes, scale_rest); return;
void fft_cols_fwd_spectrum(int h, const float2* X, int w, int conj_out, float scale, float2* S,
                           const float2* tw, cudaStream_t st, int nplanes, float scale_rest) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::cols_inv_corr(Hh, w, S, k0, nk, Z, tw, st); return;
void fft_cols_inv_corr(int h, const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                       const float2* tw, cudaStream_t st) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::cols_conv(A, w, K, S, Y, tw, st); return;
void fft_cols_conv(int h, const float2* A, int w, int K, const float2* S, float2* Y, const float2* tw,
                   cudaStream_t st) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: return FftOps<N>::cols_inv_corr_pipe(Hh, w, S, k0, nk, Z, tw, sms, st);
bool fft_cols_inv_corr_pipe(int h, const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                            const float2* tw, int sms, cudaStream_t st) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

#define EXT_C1(N) case N: return FftOps<N>::rows_inv_components_pipe(Z, h, k0, nk, G, tw, err, sms, st);
bool fft_rows_inv_components_pipe(int w, const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                                  int* err, int sms, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_fwd_simil(H, uv, s, h, kj, ncomp, unit_integral, A, tw, st); return;
void fft_rows_fwd_simil(int w, const float* H, const float4* uv, const float* s, int h, const int2* kj, int ncomp,
                        int unit_integral, float2* A, const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

// Per-pixel phasors of the similarity field: (e^{-i alpha}, e^{-i w_1 ln s}),
// phases by the two-product range reduction of sincos_kalpha / sincos_wx.
__global__ void k_simil_phasors(const float* __restrict__ alpha, const float* __restrict__ sfield, long long P,
                                float omega_step, float4* __restrict__ uv) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    float s1, c1, s2, c2;
    sincos_kalpha(1, __ldg(alpha + p), &s1, &c1);
    sincos_wx(omega_step, logf(__ldg(sfield + p)), &s2, &c2);
    uv[p] = make_float4(c1, -s1, c2, -s2);
  }
}

void launch_simil_phasors(const float* alpha, const float* s, long long P, float omega_step, float4* uv, int sms,
                          cudaStream_t st) {
  if (P <= 0) return;
  const int blocks = (int)std::min<long long>((P + 255) / 256, (long long)sms * 8);
  k_simil_phasors<<<blocks, 256, 0, st>>>(alpha, s, P, omega_step, uv);
}

#define EXT_C1(N) case N: FftOps<N>::rows_fwd_scale_turns(H, T, h, k0, nk, A, tw, st); return;
void fft_rows_fwd_scale_turns(int w, const float* H, const float2* T, int h, int k0, int nk, float2* A,
                              const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_fwd_simil_turns(H, T, h, kj, ncomp, A, tw, st); return;
void fft_rows_fwd_simil_turns(int w, const float* H, const float4* T, int h, const int2* kj, int ncomp, float2* A,
                              const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_fwd_phase_io(H, alpha, h, k0, nk, A, tw, st); return;
void fft_rows_fwd_phase_io(int w, const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                           const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: return FftOps<N>::rows_fwd_hloop_scale(H, T, h, k0, nk, A, tw, sms, fast, st);
bool fft_rows_fwd_hloop_scale(int w, const float* H, const float2* T, int h, int k0, int nk, float2* A,
                              const float2* tw, int sms, cudaStream_t st, bool fast) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

#define EXT_C1(N) case N: return FftOps<N>::rows_fwd_hloop_simil(H, T, h, kj, ncomp, A, tw, sms, fast, st);
bool fft_rows_fwd_hloop_simil(int w, const float* H, const float4* T, int h, const int2* kj, int ncomp, float2* A,
                              const float2* tw, int sms, cudaStream_t st, bool fast) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

#define EXT_C1(N) case N: return FftOps<N>::rows_fwd_hloop_phase(H, alpha, h, k0, nk, A, tw, sms, fast, st);
bool fft_rows_fwd_hloop_phase(int w, const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                              const float2* tw, int sms, cudaStream_t st, bool fast) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

// Per-pixel turns of the scale steering: t = ln s / log_period reduced to
// [-1/2, 1/2] (the phase of harmonic k is 2 pi k t, since w_k = 2 pi k /
// log_period) and the weight 1/s^2 (unit_integral) or 1.
__global__ void k_scale_turns(const float* __restrict__ sfield, long long P, float inv_log_period, int unit_integral,
                              float2* __restrict__ T) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    const float sv = __ldg(sfield + p);
    const float t = logf(sv) * inv_log_period;
    T[p] = make_float2(t - rintf(t), unit_integral ? 1.0f / (sv * sv) : 1.0f);
  }
}

void launch_scale_turns(const float* s, long long P, float inv_log_period, int unit_integral, float2* T, int sms,
                        cudaStream_t st) {
  if (P <= 0) return;
  const int blocks = (int)std::min<long long>((P + 255) / 256, (long long)sms * 8);
  k_scale_turns<<<blocks, 256, 0, st>>>(s, P, inv_log_period, unit_integral, T);
}

// Per-pixel turns of the similarity steering: (alpha / 2 pi, ln s / log_period),
// each reduced to [-1/2, 1/2], and the weight 1/s^2 (unit_integral) or 1.
__global__ void k_simil_turns(const float* __restrict__ alpha, const float* __restrict__ sfield, long long P,
                              float inv_log_period, int unit_integral, float4* __restrict__ T) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    const float sv = __ldg(sfield + p);
    const float a = __ldg(alpha + p) * 0.15915494309189535f;
    const float b = logf(sv) * inv_log_period;
    T[p] = make_float4(a - rintf(a), b - rintf(b), unit_integral ? 1.0f / (sv * sv) : 1.0f, 0.f);
  }
}

void launch_simil_turns(const float* alpha, const float* s, long long P, float inv_log_period, int unit_integral,
                        float4* T, int sms, cudaStream_t st) {
  if (P <= 0) return;
  const int blocks = (int)std::min<long long>((P + 255) / 256, (long long)sms * 8);
  k_simil_turns<<<blocks, 256, 0, st>>>(alpha, s, P, inv_log_period, unit_integral, T);
}

#define EXT_C1(N) case N: FftOps<N>::rows_fwd_scale(H, s, h, k0, nk, omega_step, unit_integral, A, tw, st); return;
void fft_rows_fwd_scale(int w, const float* H, const float* s, int h, int k0, int nk, float omega_step,
                        int unit_integral, float2* A, const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::cols_c2c(X, w, planes, inv, tw, st); return;
void fft_cols_c2c(int h, float2* X, int w, int planes, bool inv, const float2* tw, cudaStream_t st) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: FftOps<N>::rows_inv_channels(Z, rows, k0, nk, chan, G, tw, st); return;
void fft_rows_inv_channels(int w, const float2* Z, int rows, int k0, int nk, const int2* chan, float* G,
                           const float2* tw, cudaStream_t st) {
  switch (w) { EXT_FFT_SIZES(EXT_C1) default: return; }
}
#undef EXT_C1

#define EXT_C1(N) case N: return FftOps<N>::cols_inv_full_pipe(H, w, S, k0, nk, Z, tw, sms, st);
bool fft_cols_inv_full_pipe(int h, const float2* H, int w, const float2* S, int k0, int nk, float2* Z,
                            const float2* tw, int sms, cudaStream_t st) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

#define EXT_C1(N) case N: return FftOps<N>::cols_conv_tma(tmA, w, br, K, nsig, S, Y, tw, stw_g, err, sms, fused, st);
bool fft_cols_conv_tma(int h, const CUtensorMap& tmA, int w, int br, int K, const float2* S, float2* Y,
                       const float2* tw, const float2* stw_g, int* err, int sms, cudaStream_t st, bool fused,
                       int nsig) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

bool fft_cols_conv_tma_ok(int h, bool* needs_stage_table) {
  switch (h) {
#define EXT_CASE(N)                                         \
  case N:                                                   \
    *needs_stage_table = !TmaColCfg<N>::OK && !TmaColCfg<N>::OK_SPLIT; \
    return TmaColCfg<N>::OK || TmaColCfg<N>::OK_GTW;
    EXT_FFT_SIZES(EXT_CASE)
#undef EXT_CASE
    default: return false;
  }
}

void fft_build_stage_table(int n, const float2* tw, float2* out, cudaStream_t st) {
  switch (n) {
#define EXT_CASE(N) case N: k_stage_table<N><<<1, 256, 0, st>>>(tw, out); return;
    EXT_FFT_SIZES(EXT_CASE)
#undef EXT_CASE
    default: return;
  }
}

#define EXT_C1(N) case N: return FftOps<N>::cols_inv_corr_tma(tmH, w, br, S, k0, nk, Z, tw, err, sms, st);
bool fft_cols_inv_corr_tma(int h, const CUtensorMap& tmH, int w, int br, const float2* S, int k0, int nk, float2* Z,
                           const float2* tw, int* err, int sms, cudaStream_t st) {
  switch (h) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

bool fft_cols_tma_ok(int h) {
  switch (h) {
#define EXT_CASE(N) case N: return TmaColCfg<N>::OK;
    EXT_FFT_SIZES(EXT_CASE)
#undef EXT_CASE
    default: return false;
  }
}

// fused y and x inverse passes of square N x N planes (N = ny = nx)
#define EXT_C1(N) case N: return FftOps<N>::planes_fwd_c2c(U, nplanes, tw, err, sms, st);
bool fft_planes_fwd_c2c(int n, float2* U, int nplanes, const float2* tw, int* err, int sms, cudaStream_t st) {
  switch (n) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1

#define EXT_C1(N) case N: return FftOps<N>::planes_inv_channels(Z, nz, k0, nk, chan, G, tw, err, sms, st);
bool fft_planes_inv_channels(int n, const float2* Z, int nz, int k0, int nk, const int2* chan, float* G,
                             const float2* tw, int* err, int sms, cudaStream_t st) {
  switch (n) { EXT_FFT_SIZES(EXT_C1) default: return false; }
}
#undef EXT_C1
