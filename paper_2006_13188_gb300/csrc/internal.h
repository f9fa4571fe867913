// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/extconv.h"

// FFT sizes compiled into the library, split into groups that are
// instantiated in separate translation units (compiled in parallel).
#define EXT_FFT_SIZES_A(X) X(32) X(48) X(64) X(96) X(128) X(160)
#define EXT_FFT_SIZES_B(X) X(192) X(256) X(320) X(384)
#define EXT_FFT_SIZES_C(X) X(448) X(512) X(576) X(640)
#define EXT_FFT_SIZES_D(X) X(704) X(768) X(832) X(896)
#define EXT_FFT_SIZES_E(X) X(960) X(1024) X(1536)
#define EXT_FFT_SIZES_F(X) X(2048) X(3072) X(4096)
#define EXT_FFT_SIZES(X) \
  EXT_FFT_SIZES_A(X) EXT_FFT_SIZES_B(X) EXT_FFT_SIZES_C(X) EXT_FFT_SIZES_D(X) EXT_FFT_SIZES_E(X) EXT_FFT_SIZES_F(X)

// Sets the thread-local message returned by ext_last_error (api.cu).
void ext_set_error(const char* msg);

// ----- 2D FFT passes, dispatched on the runtime line length n (fft_dispatch.cu)
bool fft_size_supported(int n);
int fft_col_tile(int n);   // columns per block of the length-n column passes
void fft_rows_r2c(int w, const float* H, int h, float2* Hh, const float2* tw, cudaStream_t st);
void fft_rows_fwd_phase(int w, const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                        const float2* tw, cudaStream_t st);
void fft_rows_fwd_scale(int w, const float* H, const float* s, int h, int k0, int nk, float omega_step,
                        int unit_integral, float2* A, const float2* tw, cudaStream_t st);
void fft_rows_c2c(int w, const float2* X, int h, int nplanes, float2* Y, bool inv, const float2* tw,
                  cudaStream_t st);
void fft_rows_inv_components(int w, const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                             cudaStream_t st);
void fft_rows_inv_field(int w, const float2* Z, int h, int K, const float* alpha, float* out,
                        const float2* tw, cudaStream_t st);
void fft_rows_inv_real(int w, const float2* Y, int h, float* out, const float2* tw, cudaStream_t st);
void fft_cols_fwd_half(int h, float2* Hh, int ncols, const float2* tw, cudaStream_t st);
void fft_cols_fwd_spectrum(int h, const float2* X, int w, int conj_out, float scale, float2* S,
                           const float2* tw, cudaStream_t st, int nplanes = 1, float scale_rest = 0.f);
void fft_cols_inv_corr(int h, const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                       const float2* tw, cudaStream_t st);
bool fft_cols_inv_corr_pipe(int h, const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                            const float2* tw, int sms, cudaStream_t st);
bool fft_rows_inv_components_pipe(int w, const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                                  int sms, cudaStream_t st);
// 3D building blocks: in-place complex column pass over planes; inverse row
// pass into real channel planes; full-spectrum product column pass.
void fft_cols_c2c(int h, float2* X, int w, int planes, bool inv, const float2* tw, cudaStream_t st);
void fft_rows_inv_channels(int w, const float2* Z, int rows, int k0, int nk, const int2* chan, float* G,
                           const float2* tw, cudaStream_t st);
bool fft_cols_inv_full_pipe(int h, const float2* H, int w, const float2* S, int k0, int nk, float2* Z,
                            const float2* tw, int sms, cudaStream_t st);
void fft_cols_conv(int h, const float2* A, int w, int K, const float2* S, float2* Y, const float2* tw,
                   cudaStream_t st);

// ----- filter side, FP64 (filter.cu)
void launch_twiddle(float2* tw, int n, cudaStream_t st);
void launch_decompose_sampled(const double* img, int side, double dr, int n_r, int n_theta, int K,
                              double* P, double2* fk, cudaStream_t st);
// ncomp consecutive components k .. k+ncomp-1 into consecutive h x w planes of grid
void launch_component_grid(int kind, int K, int k, const double2* coef, int n_r, double dr, double sigma,
                           int R, int h, int w, float2* grid, cudaStream_t st, int ncomp = 1);
void launch_sweep_table(int K, int J, int cp, float* B, cudaStream_t st);
void launch_component_grid_mellin(double2 ck, double omega, double r_min, double r_max, int R, int h, int w,
                                  float2* grid, cudaStream_t st);
void launch_scale_finalize(const float* H, const float* s, const float* N, const float* D, int channels, long long P,
                           int mode, float cd, float* out, int sms, cudaStream_t st);

// ----- sweep (sweep.cu)
// B: J rows of cp floats (cp = 2K rounded up to a multiple of 4).
bool sweep_fp32(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv,
                int32_t* argmax, cudaStream_t st);
// tcgen05 split-BF16 sweep (sweep_tc.cu); err receives EXT_ERR_TIMEOUT if a bounded wait expires.
bool sweep_bf16x3(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv, int32_t* argmax,
                  int* err, int sms, cudaStream_t st);

// ----- SO(3) (so3.cu, sweep_so3.cu)
void launch_so3_component_grid(const int4* comp, int k0, int nk, const double2* tables, int n_r, double dr, int L,
                               int R, int nz, int ny, int nx, float2* grid, cudaStream_t st);
void launch_so3_wigner(const double* quats, int n, int L, double2* C, const int4* chans, int nchan, int cpad,
                       float* Brow, cudaStream_t st);
void launch_real_to_complex(const float* V, long long n, float2* X, int sms, cudaStream_t st);
void sweep_so3_fp32(const float* G, long long P, int C, const float* B, int cpad, int J, float* maxv,
                    int32_t* argmax, cudaStream_t st);
size_t so3_btc_bytes(int J, int cpad);
void so3_build_btc(const float* B, int cpad, int J, unsigned char* Bt, cudaStream_t st);
void sweep_so3_tc(const float* G, long long P, int C, int cpad, const unsigned char* Bt, int J, float* maxv,
                  int32_t* argmax, int* err, int sms, cudaStream_t st);
