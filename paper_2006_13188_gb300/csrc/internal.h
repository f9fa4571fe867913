// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
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
// similarity-steered signals: component c < ncomp has (k, j) = kj[c]; uv the
// per-pixel phasors (e^{-i alpha}, e^{-i w_1 ln s}) of launch_simil_phasors
void fft_rows_fwd_simil(int w, const float* H, const float4* uv, const float* s, int h, const int2* kj, int ncomp,
                        int unit_integral, float2* A, const float2* tw, cudaStream_t st);
void fft_rows_fwd_scale_turns(int w, const float* H, const float2* T, int h, int k0, int nk, float2* A,
                              const float2* tw, cudaStream_t st);
void fft_rows_fwd_simil_turns(int w, const float* H, const float4* T, int h, const int2* kj, int ncomp, float2* A,
                              const float2* tw, cudaStream_t st);
void fft_rows_fwd_phase_io(int w, const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                           const float2* tw, cudaStream_t st);
// component-loop steered row passes (false: no plan for this line length; use the others);
// fast: phasors from the hardware sine and cosine after the exact reduction
bool fft_rows_fwd_hloop_scale(int w, const float* H, const float2* T, int h, int k0, int nk, float2* A,
                              const float2* tw, int sms, cudaStream_t st, bool fast);
bool fft_rows_fwd_hloop_simil(int w, const float* H, const float4* T, int h, const int2* kj, int ncomp, float2* A,
                              const float2* tw, int sms, cudaStream_t st, bool fast);
bool fft_rows_fwd_hloop_phase(int w, const float* H, const float* alpha, int h, int k0, int nk, float2* A,
                              const float2* tw, int sms, cudaStream_t st, bool fast);
// per-pixel turns (t, wgt) / (alpha / 2 pi, ln s / log_period, wgt) of the steered row passes
void launch_scale_turns(const float* s, long long P, float inv_log_period, int unit_integral, float2* T, int sms,
                        cudaStream_t st);
void launch_simil_turns(const float* alpha, const float* s, long long P, float inv_log_period, int unit_integral,
                        float4* T, int sms, cudaStream_t st);
void launch_simil_phasors(const float* alpha, const float* s, long long P, float omega_step, float4* uv, int sms,
                          cudaStream_t st);
void fft_rows_fwd_scale(int w, const float* H, const float* s, int h, int k0, int nk, float omega_step,
                        int unit_integral, float2* A, const float2* tw, cudaStream_t st);
void fft_rows_c2c(int w, const float2* X, int h, int nplanes, float2* Y, bool inv, const float2* tw,
                  cudaStream_t st);
void fft_rows_inv_components(int w, const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                             cudaStream_t st);
void fft_rows_inv_field(int w, const float2* Z, int h, int K, const float* alpha, float* out,
                        const float2* tw, cudaStream_t st);
void fft_rows_inv_real(int w, const float2* Y, int h, float* out, const float2* tw, cudaStream_t st);
// Hf (optional): the full h x w spectrum written as well (Hermitian mirror of the half spectrum)
void fft_cols_fwd_half(int h, float2* Hh, int ncols, const float2* tw, cudaStream_t st, float2* Hf = nullptr,
                       int w = 0);
void fft_cols_fwd_spectrum(int h, const float2* X, int w, int conj_out, float scale, float2* S,
                           const float2* tw, cudaStream_t st, int nplanes = 1, float scale_rest = 0.f);
void fft_cols_inv_corr(int h, const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                       const float2* tw, cudaStream_t st);
bool fft_cols_inv_corr_pipe(int h, const float2* Hh, int w, const float2* S, int k0, int nk, float2* Z,
                            const float2* tw, int sms, cudaStream_t st);
bool fft_rows_inv_components_pipe(int w, const float2* Z, int h, int k0, int nk, float* G, const float2* tw,
                                  int* err, int sms, cudaStream_t st);
// 2D FP32 tensor map (dim0 fastest, row pitch stride1_bytes, box box0 x box1);
// false if the driver entry point is missing or alignment rules are not met.
bool make_tmap_2d_f32(const void* base, unsigned long long dim0, unsigned long long dim1,
                      unsigned long long stride1_bytes, unsigned box0, unsigned box1, CUtensorMap* out);
// Inverse column pass staged by the tensor memory accelerator: tmH maps the
// FULL spectrum (h rows of 2w floats, boxes of 2 * col_tile floats x br rows);
// false if this length has no such variant.
bool fft_cols_tma_ok(int h);
bool fft_cols_inv_corr_tma(int h, const CUtensorMap& tmH, int w, int br, const float2* S, int k0, int nk, float2* Z,
                           const float2* tw, int* err, int sms, cudaStream_t st);
// 3D building blocks: in-place complex column pass over planes; inverse row
// pass into real channel planes; full-spectrum product column pass.
void fft_cols_c2c(int h, float2* X, int w, int planes, bool inv, const float2* tw, cudaStream_t st);
void fft_rows_inv_channels(int w, const float2* Z, int rows, int k0, int nk, const int2* chan, float* G,
                           const float2* tw, cudaStream_t st);
// fused forward y and x passes, in place, over nplanes planes of n x n complex
// values (false: not available for n)
bool fft_planes_fwd_c2c(int n, float2* U, int nplanes, const float2* tw, int* err, int sms, cudaStream_t st);
// fused inverse y and x passes over nk * nz planes of n x n (false: not available for n)
bool fft_planes_inv_channels(int n, const float2* Z, int nz, int k0, int nk, const int2* chan, float* G,
                             const float2* tw, int* err, int sms, cudaStream_t st);
bool fft_cols_inv_full_pipe(int h, const float2* H, int w, const float2* S, int k0, int nk, float2* Z,
                            const float2* tw, int sms, cudaStream_t st);
void fft_cols_conv(int h, const float2* A, int w, int K, const float2* S, float2* Y, const float2* tw,
                   cudaStream_t st);
// The same pass with the A_k and spectrum tiles staged by the tensor memory
// accelerator: tmA maps A as (K+1) h rows of 2w floats, boxes of 2 * col_tile
// floats x br rows; false if this length has no such variant.  fused: the
// last butterfly stage multiplies and accumulates its outputs in registers
// (no shared-memory pass of the products).  nsig > 1: nsig signals in one
// launch, signal s's components at A rows (s (K+1) + k) h, its sum at
// Y + s h w; they share each spectrum tile.
bool fft_cols_conv_tma(int h, const CUtensorMap& tmA, int w, int br, int K, const float2* S, float2* Y,
                       const float2* tw, const float2* stw_g, int* err, int sms, cudaStream_t st,
                       bool fused = true, int nsig = 1);
// whether the staged convolution pass exists for column length h, and whether it
// reads its stage twiddles from a global table (fft_build_stage_table) instead of
// a shared-memory copy
bool fft_cols_conv_tma_ok(int h, bool* needs_stage_table);
void fft_build_stage_table(int n, const float2* tw, float2* out, cudaStream_t st);

// ----- filter side, FP64 (filter.cu)
void launch_twiddle(float2* tw, int n, cudaStream_t st);
void launch_decompose_sampled(const double* img, int side, double dr, int n_r, int n_theta, int K,
                              double* P, double2* fk, cudaStream_t st);
// ncomp consecutive components k .. k+ncomp-1 into consecutive h x w planes of grid
void launch_component_grid(int kind, int K, int k, const double2* coef, int n_r, double dr, double sigma,
                           int R, int h, int w, float2* grid, cudaStream_t st, int ncomp = 1);
void launch_sweep_table(int K, int J, int cp, float* B, cudaStream_t st);
// the same for a component list (ks[0] = 0, ks[1..K] the steered components, device)
void launch_sweep_table_list(const int* ks, int K, int J, int cp, float* B, cudaStream_t st);
// E_k = sum over the box [-R, R]^2 of |F_k(d)|^2, k = 0..K, accumulated into E (zeroed by the caller)
void launch_component_energy(int kind, int K, const double2* coef, int n_r, double dr, double sigma, int R,
                             double* E, cudaStream_t st);
void launch_component_grid_mellin(double2 ck, double omega, double r_min, double r_max, int R, int h, int w,
                                  float2* grid, cudaStream_t st);
// log-polar harmonic grids coef[c] e^{i (k theta + w_j ln r)}, (k, j) = kj[c],
// w_j = omega_step j, for c = k0 .. k0 + nk - 1 (one h x w plane each)
void launch_component_grid_simil(const double2* coef, const int2* kj, int k0, int nk, double omega_step, double r_min,
                                 double r_max, int R, int h, int w, float2* grid, cudaStream_t st);
void launch_scale_finalize(const float* H, const float* s, const float* N, const float* D, int channels, long long P,
                           int mode, float cd, float* out, int sms, cudaStream_t st);

// ----- pattern detection front end (ght.cu): H = |grad I|, theta = atan2(dI/dy, dI/dx)
void launch_gradient_field(const float* I, int h, int w, float* H, float* theta, int sms, cudaStream_t st);

// out[c][p] /= D[p] for c < channels (normalize.cu)
void launch_divide_channels(float* out, const float* D, long long P, int channels, int sms, cudaStream_t st);

// ----- failure-path self-test (status.cu): one wait that nothing completes, bounded by the status block's budget
void launch_selftest_timeout(int* err, cudaStream_t st);
// Opt-in to `bytes` of dynamic shared memory for `func` on the current device
// (a per-device function attribute; set once per (device, function, size)).
bool ext_smem_optin(const void* func, int bytes);

// ----- sweep (sweep.cu)
// B: J rows of cp floats (cp = 2K rounded up to a multiple of 4).
bool sweep_fp32(const float* G, long long P, int K, int J, const float* B, int cp, float* maxv,
                int32_t* argmax, cudaStream_t st);
// whether the J x 2K steering table of the FP32 sweep fits the current device's shared memory
bool sweep_fp32_fits(int K, int J);
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
// warp-specialised split-BF16 sweep over pre-split operands: B' blocks built once per rotation set
// (so3_ws_build_b), A' blocks of the voxels written into Ab (so3_ws_a_bytes) by the call itself
size_t so3_ws_a_bytes(long long P, int cpad);
size_t so3_ws_b_bytes(int J, int cpad);
void so3_ws_build_b(const float* B, int cpad, int J, unsigned char* Bb, cudaStream_t st);
void so3_ws_split_a(const float* G, long long P, int C, int cpad, unsigned char* Ab, int sms, cudaStream_t st);
bool sweep_so3_ws(long long P, int cpad, const unsigned char* Ab, const unsigned char* Bb, int J, float* maxv,
                  int32_t* argmax, int* err, int sms, cudaStream_t st);
// the grid sweep over R_d R_z(2 pi t / n_psi): B' = 16 in-plane-harmonic rows per direction (launch_so3_grid_rows),
// hi/lo split as so3_ws_build_b with J = 16 n_dirs rows; index dir * n_psi + t
bool sweep_so3_ws_grid(long long P, int cpad, const unsigned char* Ab, const unsigned char* Bb, int n_dirs,
                       int n_psi, float* maxv, int32_t* argmax, unsigned long long* keys, int* err, int sms,
                       cudaStream_t st);
void launch_so3_grid_rows(const double2* C, int n_dirs, int L, const int4* comps, int ncomp, int cpad, float* Brow,
                          cudaStream_t st);
size_t so3_btc_bytes(int J, int cpad);
void so3_build_btc(const float* B, int cpad, int J, unsigned char* Bt, cudaStream_t st);
// keys (P entries of scratch, or NULL): lets small voxel counts split the
// rotation tiles over more blocks (sweep_so3_tc_split(P, J, sms) > 1)
int sweep_so3_tc_split(long long P, int J, int sms);
void sweep_so3_tc(const float* G, long long P, int C, int cpad, const unsigned char* Bt, int J, float* maxv,
                  int32_t* argmax, unsigned long long* keys, int* err, int sms, cudaStream_t st);

// ----- learned SO(3) proposal: tensor-core GEMM and network kernels (mlp.cu)
// Epilogue of C = A B^T: optional bias[n], ReLU, zeroing where mask[m][n] <= 0,
// FP32 and/or BF16 stores, row-major or transposed (out[n][m]).
struct GemmEpilogue {
  const float* bias = nullptr;
  int relu = 0;
  const __nv_bfloat16* mask = nullptr;
  int ldm = 0;
  float* out_f32 = nullptr;
  int ldo = 0;
  __nv_bfloat16* out_bf16 = nullptr;
  int ldo16 = 0;
  int trans = 0;
};
// A [M][lda], B [N][ldb], BF16, K-major; K, lda, ldb multiples of 8; 16-byte aligned rows.
void gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
               const GemmEpilogue& ep, int* err, cudaStream_t st);
// rows (optionally selected by idx) of X [.][ldx] (first C entries) -> unit-norm BF16 rows of pitch dp
void launch_rows_normalize_bf16(const float* X, int ldx, const int32_t* idx, int n, int C, int dp,
                                __nv_bfloat16* Y, cudaStream_t st);
void launch_gather_quats(const float* q, const int32_t* idx, int n, float* out, cudaStream_t st);
void launch_quat_loss(const float* o, int ldo, const float* qt, int n, float* loss, __nv_bfloat16* dout,
                      float* dout_f, cudaStream_t st);
void launch_colsum(const float* X, int rows, int cols, int ld, float* out, cudaStream_t st);
void launch_transpose_bf16(const __nv_bfloat16* X, int rows, int cols, int ldx, __nv_bfloat16* Y, int yrows,
                           int ycols, int ldy, cudaStream_t st);
void launch_adam(float* w, float* m, float* v, const float* g, long long n, float lr, int step, __nv_bfloat16* w16,
                 cudaStream_t st);
void launch_normalize_quat(const float* o, int ldo, int n, float* q, cudaStream_t st);
void launch_f32_to_bf16(const float* x, long long n, __nv_bfloat16* y, cudaStream_t st);

// ----- SO(3) proposal support (so3_proposal.cu)
// Unique entries (l, a, b) of the rotation matrices, C^l_ab(R) = d^l_ba(beta) e^{-i((a+b) sigma + (b-a) delta)}
// with sigma = (alpha + gamma) / 2, delta = (alpha - gamma) / 2 (zyz Euler angles); d from Wigner's sum
// formula as sum_j coef[j] cos(beta/2)^(pc0 - 2j) sin(beta/2)^(ps0 + 2j).
struct So3Steer {
  int n;                 // entries (231 for L = 6)
  uint32_t meta[256];    // ch | self << 10 | (ks + 12) << 11 | (kd + 12) << 16 | ns << 21 | pc0 << 24 | ps0 << 28
  unsigned char l[256];  // degree of each entry (entries are ordered by degree)
  float coef[7][256];
};
// SO(3) extended convolution: U[i] = w V C^l_ab(R(q)) for the steering
// entries e0 + i (i < ne) of degree <= L, Q the per-voxel quaternions
// (w, x, y, z), U planes of P complex values; acc += y over n complex values.
void launch_so3_modulate(const float* V, const float* Q, long long P, int L, int e0, int ne, float2* U,
                         cudaStream_t st);
void launch_add_complex(float2* acc, const float2* y, long long n, int sms, cudaStream_t st);
void launch_so3_upper_bound(const float* G, long long P, const So3Steer* tab, float* ub, int L, int sms,
                            cudaStream_t st);
// ordered compaction: idx[k] = the k-th i with (below ? v[i] < thr : v[i] >= thr); *count = their number
size_t compact_scratch_bytes(long long n);
void compact(const float* v, long long n, float thr, int below, int32_t* idx, int* count, void* scratch,
             cudaStream_t st);
void launch_gather_rows(const float* G, long long P, int C, const int32_t* vox, int n, float* X, int ldx,
                        cudaStream_t st);
void launch_gather_channels(const float* G, long long P, int C, const int32_t* vox, const int32_t* sel, int n,
                            float* out, cudaStream_t st);
void launch_so3_refine(const float* X, int ldx, int n, const float* q0, const So3Steer* tab, int steps, float theta0,
                       int tries, float* q_out, float* s_out, int sms, cudaStream_t st);
void launch_so3_augment(const float* X, int ldx, const int32_t* rows, int n, const float* Q, const float* q_in,
                        const So3Steer* tab, int C, float* X_out, int ldo, float* q_out, cudaStream_t st);
void launch_so3_fill(long long P, float* score, float* quat, int32_t* grid_idx, cudaStream_t st);
void launch_so3_scatter(const int32_t* cand, int n, const float* s, const float* q, float* score, float* quat,
                        int32_t* grid_idx, cudaStream_t st);
void launch_so3_merge(const int32_t* cand, const int32_t* fb, int n_fb, const float* m, const int32_t* j,
                      const double* grid, float* score, float* quat, int32_t* grid_idx, cudaStream_t st);
void launch_check_index(const int32_t* idx, long long n, long long upper, int* bad, cudaStream_t st);
// per row of X (channel layout of degree L): sum_l min(sqrt(2l+1) |G_l|_F, deflated bound of |G_l|_*)
void launch_so3_refined_bound(const float* X, int ldx, int n, const So3Steer* tab, int L, float* out, int sms,
                              cudaStream_t st);
void launch_gather_row_copies(const float* X, int ld, const int32_t* sel, int n, float* Y, cudaStream_t st);
void launch_gather_int(const int32_t* x, const int32_t* sel, int n, int32_t* y, cudaStream_t st);
