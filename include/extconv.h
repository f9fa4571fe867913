/*
 * extconv -- extended convolution and correlation on GB300 (sm_103a).
 *
 * C ABI of libextconv.so.  It computes the spatially adaptive filtering
 * operators of Mitchel et al., "Efficient Spatially Adaptive Convolution and
 * Correlation" (arXiv 2006.13188):
 *
 *   extended correlation  {H,T} * F (p) = sum_q H(q) conj((T(p)F)(q - p))   (Sec. 2.1, Eq. Def-ECorr)
 *   extended convolution  {H,T} * F (p) = sum_q H(q) (T(q)F)(p - q)         (Sec. 2.2, Eq. Def-EConv)
 *
 * on the integer lattice with periodic boundaries (indices mod (h, w)), for
 * rotation fields (SO(2), Sec. 4.1).  The filter is split into angular
 * harmonics F_k(r, theta) = f_k(r) e^{i k theta}, |k| <= K (Sec. 4.1
 * "Filter Decomposition"); every component is correlated/convolved with the
 * signal by FFT ("Standard Correlation"); the result is steered per pixel
 * ("Linear Combination"), or swept over J uniformly spaced angles with a
 * per-pixel max/argmax (the rotation search of Sec. 5, "Band-Limiting
 * Revisited").
 *
 * Conventions shared by every entry point:
 *   - Images are row-major, x = column index, y = row index, no padding
 *     (leading dimension = w).  Angles are radians; rotating a filter by
 *     alpha means (T_alpha F)(d) = F(R(-alpha) d), R(a) = [[cos a, -sin a],
 *     [sin a, cos a]], which multiplies harmonic k by e^{-i k alpha}.
 *   - Image/field/output pointers may be DEVICE or HOST memory; the library
 *     tells them apart with cudaPointerGetAttributes.  Host buffers are
 *     staged through plan-owned device memory and the call then returns only
 *     after its results are back in host memory.  With device buffers the
 *     call is asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *     stream).  The caller owns every buffer it passes; the library never
 *     frees them.
 *   - Filter descriptions (ext_filter_so2 and the arrays it points to) are
 *     HOST memory, read during the call only.
 *   - Supported image sides: 32, 48, 96, 160, every multiple of 64 up to
 *     1024, 1536, 2048, 3072 and 4096 (all of the form 2^a 3^b 5^c 7^d 11^e 13^f);
 *     w must be even.  Other sizes return EXT_ERR_UNSUPPORTED before any
 *     launch.  h == 0 or w == 0 is a no-op returning EXT_OK.
 *   - Errors: argument errors return before any launch; CUDA errors return
 *     EXT_ERR_CUDA.  ext_last_error() gives a thread-local message.  No C++
 *     exception crosses this interface.  There is no CPU fallback.
 */
#ifndef EXTCONV_H
#define EXTCONV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ext_status;
#define EXT_OK 0
#define EXT_ERR_INVALID_ARG 1
#define EXT_ERR_UNSUPPORTED 2
#define EXT_ERR_CUDA 3
#define EXT_ERR_OOM 4
#define EXT_ERR_TIMEOUT 5
#define EXT_ERR_CHECKPOINT 6   /* a checkpoint file is missing, truncated, corrupt or of other shapes */

/* Filter kinds (ext_filter_so2.kind). */
#define EXT_FILTER_ANALYTIC_GAUSSPOW 0 /* f_k(r) = a_k r^|k| exp(-r^2 / (2 sigma^2))                */
#define EXT_FILTER_TABLE 1             /* f_k(i dr) given; cubic Hermite in r (see below)            */
#define EXT_FILTER_SAMPLED 2           /* (2R+1)^2 image, decomposed by the library (Sec. 4.1)      */

/* Sweep precision (ext_corr_so2 / ext_sweep_so2). */
#define EXT_PREC_FP32 0   /* plain FP32 on CUDA cores                                              */
#define EXT_PREC_BF16X3 1 /* split BF16 hi+lo operands on tcgen05 tensor cores, FP32 accumulation */
#define EXT_PREC_DEFAULT (-1) /* the plan's default precision (ext_options.precision)                */

/*
 * SO(2) filter with angular bandwidth K (|k| <= K) on the box [-R, R]^2:
 *   F(d) = sum_{|k|<=K} f_k(|d|) e^{i k theta(d)},  theta(d) = atan2(d_y, d_x),
 *   F(0) = f_0(0)  (the k != 0 terms vanish at the origin).
 * ANALYTIC_GAUSSPOW: a = 2(2K+1) doubles, interleaved (re, im) of a_k for
 *   k = -K..K; sigma > 0.
 * TABLE: fk = 2(2K+1)n_r doubles, row k+K holds (re, im) of f_k(i dr),
 *   i = 0..n_r-1.  Between samples f_k is the cubic Hermite spline with
 *   tangents (v_{i+1} - v_{i-1}) / 2, v_{-1} = (-1)^k v_1, v_{n_r} = 0, and
 *   f_k(r) = 0 for r / dr > (n_r - 1) + 1e-9 (closed support).
 * SAMPLED: img = (2R+1)^2 doubles, row-major, centre pixel (R, R).  The
 *   library resamples it at radii i dr <= R and n_theta angles with the Keys
 *   cubic kernel (a = -1/2, zero outside), takes the DFT along each circle
 *   (Sec. 4.1 "Filter Decomposition"), and uses the resulting TABLE.
 * The operators below require a real filter (f_{-k} = conj f_k); this holds
 *   for SAMPLED and is the caller's promise for the other kinds.
 */
typedef struct {
  int K;
  int R;
  int kind;
  const double* a;
  double sigma;
  const double* fk;
  int n_r;
  double dr;
  const double* img;
  int n_theta;
} ext_filter_so2;

typedef struct ext_plan_s* ext_plan;

const char* ext_status_string(ext_status s);
/* Thread-local message describing the last error returned on this thread. */
const char* ext_last_error(void);

/*
 * Plan options (no counterpart in the paper: run-time policy of the library).
 *   device          CUDA device ordinal the plan works on.
 *   precision       EXT_PREC_FP32 or EXT_PREC_BF16X3: the sweep precision used
 *                   wherever a call passes EXT_PREC_DEFAULT.
 *   wait_budget_ns  limit of every bounded device-side wait (a kernel waiting
 *                   for its own bulk copies or tensor-core work); on expiry the
 *                   kernel records EXT_ERR_TIMEOUT in the plan's status word,
 *                   waits (bounded) for its own work in flight, frees its
 *                   tensor memory and returns.  0 = 1 second.
 *   autotune        EXT_TUNE_ON: the first ext_corr_so2 / ext_batch_corr_so2
 *                   call of a shape class times the pass variants the library
 *                   has for it (tensor-copy staged or not, persistent
 *                   prefetching or not, components per inverse launch) and keeps
 *                   the fastest; EXT_TUNE_OFF (default): the built-in choice.
 *   tune_cache      path of the autotuner's cache (text, one line per shape
 *                   class, keyed by GPU name and driver version), read at plan
 *                   creation and rewritten when a new class is tuned; NULL:
 *                   in memory only.  The string is copied.
 *   fault_inject    EXT_FAULT_ALLOC: after `fault_after` successful device
 *                   allocations of the plan, the next one fails as if the
 *                   device were out of memory (EXT_ERR_OOM; once).  For tests
 *                   of the error paths; EXT_FAULT_NONE (default) in use.
 * ext_options_init fills the defaults (device 0).  ext_plan_create with
 * options == NULL uses them.
 */
#define EXT_TUNE_OFF 0
#define EXT_TUNE_ON 1
#define EXT_FAULT_NONE 0
#define EXT_FAULT_ALLOC 1
typedef struct {
  int device;
  int precision;
  uint64_t wait_budget_ns;
  int autotune;
  const char* tune_cache;
  int fault_inject;
  int fault_after;
} ext_options;
void ext_options_init(ext_options* options);

/* Plan: caches twiddle tables, filter spectra (per filter, size and mode),
 * sweep tables and workspace on options->device.  Not thread-safe: one plan
 * per host thread.  ext_plan_destroy frees everything the plan allocated. */
ext_status ext_plan_create(ext_plan* plan, const ext_options* options);
ext_status ext_plan_destroy(ext_plan plan);
/* Frees cached filter spectra and workspace (kept otherwise for reuse). */
ext_status ext_plan_trim(ext_plan plan);

/* Waits for `stream` and reports device-side failures of earlier calls on
 * this plan: EXT_ERR_TIMEOUT if a bounded wait inside a kernel expired (the
 * kernel then abandoned its work, freed its tensor memory and returned; the
 * affected outputs are invalid).  Calls with host buffers do this check
 * themselves before returning. */
ext_status ext_plan_sync(ext_plan plan, void* stream);

/*
 * Self-test of the failure path above (no counterpart in the paper).  Launches
 * on `stream` one kernel that waits on a shared-memory mbarrier which nothing
 * will ever complete (no copy, no tensor-core work and no other thread is in
 * flight), bounded by the plan's wait budget; when the budget runs out the
 * kernel records EXT_ERR_TIMEOUT and returns, so the next ext_plan_sync
 * returns EXT_ERR_TIMEOUT (and clears it) and the plan stays usable.
 */
ext_status ext_plan_selftest_timeout(ext_plan plan, void* stream);

/* Per-kernel accounting for benchmarks and tracing (no counterpart in the
 * paper).  Every kernel launch of the plan is counted per kernel name; with
 * profiling enabled each launch is also bracketed by CUDA events recorded on
 * the launch's stream.  ext_plan_profile_read waits for those events, writes
 * up to n_max entries (names: n_max * 64 chars, NUL-terminated; total_ms:
 * summed event time; launches: count), sets *n_out, and clears the
 * accumulators.  Any output array may be NULL. */
ext_status ext_plan_profile(ext_plan plan, int enable);
ext_status ext_plan_profile_read(ext_plan plan, int n_max, char* names, double* total_ms, int64_t* launches,
                                 int* n_out);

/*
 * Filter decomposition (Sec. 4.1 "Filter Decomposition"), FP64 on the
 * device.  Writes the radial table f_k(i dr), k = -K..K, as 2(2K+1)n_r
 * interleaved doubles to HOST memory fk_out (capacity fk_cap doubles) and
 * n_r to *n_r_out.  SAMPLED filters are decomposed; TABLE filters are
 * returned as given; ANALYTIC filters return EXT_ERR_UNSUPPORTED.
 */
ext_status ext_filter_so2_decompose(ext_plan plan, const ext_filter_so2* F, double* fk_out,
                                    int64_t fk_cap, int* n_r_out);

/*
 * Extended convolution with a rotation field (Sec. 2.2 Eq. Def-EConv; the
 * algorithm of Sec. 4.1, last paragraph): out = Re sum_k (H e^{-ik alpha}) * F_k.
 * H, alpha (radians), out: h x w float32.
 */
ext_status ext_conv_so2(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F,
                        const float* alpha, float* out, void* stream);

/*
 * Normalised extended convolution with a rotation field (Sec. 8, Eq.
 * normalization; the Line Integral Convolution application): for every
 * channel c,
 *   out_c = ({H_c, alpha} * F) / ({1, alpha} * F),
 * each extended convolution as in ext_conv_so2, so that every output is the
 * weighted average of the values scattered onto it (for rotations no
 * division of the signal by |T|^2 is needed).  H, out: channels x h x w
 * float32 (channel-major); alpha: h x w float32 radians.  The denominator is
 * not guarded: a filter whose band-limited response to 1 changes sign gives
 * unbounded outputs there.  EXT_ERR_INVALID_ARG for channels outside [1, 64].
 */
ext_status ext_conv_so2_normalized(ext_plan plan, const float* H, int channels, int h, int w,
                                   const ext_filter_so2* F, const float* alpha, float* out, void* stream);

/*
 * Extended correlation with a rotation field (Sec. 2.1 Eq. Def-ECorr; Sec. 4.1
 * "Linear Combination"):
 *   field mode (alpha != NULL): out(p) = sum_k e^{ik alpha(p)} G_k(p),
 *                               G_k = H (*) F_k  (standard correlation);
 *   sweep mode (alpha == NULL): S(p, j) = sum_k e^{ik alpha_j} G_k(p) with
 *     alpha_j = 2 pi j / n_angles; out_or_max(p) = max_j S(p, j) and
 *     argmax(p) = the smallest j attaining it.
 * H, alpha, out_or_max: h x w float32; argmax: h x w int32 (sweep mode only,
 * NULL in field mode).  precision: EXT_PREC_FP32 or EXT_PREC_BF16X3 (sweep
 * mode; ignored in field mode).
 */
ext_status ext_corr_so2(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F,
                        const float* alpha, int n_angles, float* out_or_max, int32_t* argmax,
                        int precision, void* stream);

/*
 * Fixed-budget component selection (Sec. 5 "Band-Limiting Revisited": with a
 * budget of standard convolutions the least-squares best choice, averaged
 * over rotations, is the components with the largest coefficients).
 * ext_filter_so2_energy writes the lattice energies
 *   E_k = sum_{d in [-R, R]^2} |F_k(d)|^2,  k = 0..K,
 * (F_k(0) = 0 for k != 0; FP64) to HOST memory energy_out (K+1 doubles): the
 * rotation-averaged squared error of steering with a subset is the energy of
 * the components left out (each k >= 1 counts twice, with -k).
 * ext_corr_so2_subset is ext_corr_so2 in sweep mode restricted to the listed
 * components: ks[0] = 0 (G_0, the angle-independent mean, always kept), then
 * nks - 1 <= 16 ascending components 1 <= ks[i] <= K;
 *   S(p, j) = G_0(p) + 2 sum_{i >= 1} Re(e^{i 2 pi ks[i] j / J} G_{ks[i]}(p)),
 * max_out(p) = max_j S(p, j), argmax(p) = the smallest maximising j.  Its
 * cost is that of ext_corr_so2 with K = nks - 1.
 */
ext_status ext_filter_so2_energy(ext_plan plan, const ext_filter_so2* F, double* energy_out);
/* The selection rule (host only, no device work): from the energies E_k,
 * k = 0..K (energy, HOST, K+1 doubles) and a budget of standard correlations,
 * writes ks_out[0] = 0 (G_0 always kept), then the budget - 1 components
 * k >= 1 of largest energy (ties to the smaller k) in ascending order, and
 * their count min(budget, K + 1) to *n_out.  ks_out must hold K + 1 ints.
 * EXT_ERR_INVALID_ARG for K < 0, budget < 1 or a NaN energy. */
ext_status ext_select_components(const double* energy, int K, int budget, int* ks_out, int* n_out);
ext_status ext_corr_so2_subset(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F, const int* ks,
                               int nks, int n_angles, float* max_out, int32_t* argmax, int precision, void* stream);

/*
 * The component correlations G_k = H (*) F_k, k = 0..K (Sec. 4.1 "Standard
 * Correlation"), as 2K+1 planes of h*w float32: plane 0 = G_0 (real for a
 * real filter), plane 2k-1 = Re G_k, plane 2k = Im G_k.
 */
ext_status ext_corr_so2_components(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F,
                                   float* G, void* stream);

/*
 * The angular sweep over precomputed components (Sec. 5 "Band-Limiting
 * Revisited": max over rotations), G laid out as ext_corr_so2_components
 * writes it for n_pix pixels:
 *   S(p, j) = G_0(p) + 2 sum_{k=1..K} Re(e^{i 2 pi k j / J} G_k(p)),
 *   max_out(p) = max_j S(p, j), argmax(p) = smallest maximising j.
 */
ext_status ext_sweep_so2(ext_plan plan, const float* G, int64_t n_pix, int K, int n_angles, float* max_out,
                         int32_t* argmax, int precision, void* stream);

/*
 * Batched correlation sweep over many images of uneven sizes, bandwidths and
 * angle counts (each image as ext_corr_so2 in sweep mode with its own
 * filter).  All image and output buffers must be DEVICE memory; filter
 * descriptions are HOST memory read during the call.  The batch is recorded
 * as two CUDA graphs: a setup graph (per-image filter decomposition and the
 * component spectra of every template, kept in plan workspace: the sum over
 * the images of (K_i + 1) h_i w_i complex values, plus tile padding) replayed
 * when the descriptor list or a filter changes, and a step graph (forward
 * FFT, inverse correlation passes and sweep of every image) replayed on every
 * call -- a fixed template library matched against new image data in the
 * same buffers.  The call is asynchronous on `stream` (a changed batch first
 * waits for its filter data to be copied).
 */
typedef struct {
  const float* H;          /* h x w image, device */
  int h, w;
  const ext_filter_so2* F; /* its filter, host */
  int n_angles;            /* sweep angles J */
  float* max_out;          /* h x w, device */
  int32_t* argmax;         /* h x w, device */
} ext_image_desc;
ext_status ext_batch_corr_so2(ext_plan plan, const ext_image_desc* imgs, int n, int precision, void* stream);

/*
 * Scale-adaptive extended convolution and smoothing (Sec. 8).  The filter is
 * a radially symmetric function written in log-radial (Mellin) harmonics,
 *   F(d) = P(ln|d|) for r_min <= |d| <= r_max,  F(0) = centre_tap, else 0,
 *   P(u) = sum_{k=-(n_h-1)}^{n_h-1} c_k e^{i w_k u},  w_k = 2 pi k / log_period,
 *   c_{-k} = conj(c_k)  (mellin_c: n_h complex c_0..c_{n_h-1}, interleaved
 *   doubles, HOST memory).
 * Scaling the filter by s(q) multiplies harmonic k by e^{-i w_k ln s(q)} on the
 * same support (the centre tap is scale invariant).  With A * B denoting the
 * extended convolution of Eq. Def-EConv under this scale field,
 *   mode 0: out_c = {H_c, s} * F
 *   mode 1: out_c = {H_c, s} * F / {1, s} * F                 (Eq. normalization)
 *   mode 2: out_c = {H_c / s^2, s} * F / {1 / s^2, s} * F     (unit-integral signal)
 * H, out: channels planes of h x w float32; s: h x w float32 scale field, > 0.
 * Accuracy: FP32 transforms; each harmonic's phasor e^{-i w_k ln s} comes from
 * an exact reduction of k ln s / log_period and the hardware sine and cosine
 * (absolute error about 4e-7; the environment variable EXT_STEER_MODE=3 at
 * plan creation selects sincospif, about 1e-7).  Against the FP64 definition
 * the results stay within 1e-5 of the output scale (rel-L2 about 4e-6 on the
 * 4096 x 4096 x 3, 24-harmonic workload).  The same holds for ext_conv_so2,
 * ext_conv_so2_normalized and ext_conv_similarity.
 */
ext_status ext_conv_scale(ext_plan plan, const float* H, int channels, int h, int w, const double* mellin_c, int n_h,
                          double log_period, double r_min, double r_max, double centre_tap, const float* s, int mode,
                          float* out, void* stream);

/*
 * Extended convolution with a joint rotation x scale field (transformation
 * fields of rotations and isotropic scales; Eq. Def-EConv with the angular
 * harmonics of Sec. 4.1 and the log-radial harmonics of Sec. 8).  Filter in
 * log-polar harmonics,
 *   F(d) = sum_{|k|<=K} sum_{|j|<n_h} c_{k,j} e^{i k theta(d)} e^{i w_j ln|d|}
 *          for r_min <= |d| <= r_max,  F(0) = centre_tap,  else 0,
 *   w_j = 2 pi j / log_period,  c_{-k,-j} = conj(c_{k,j})  (F real);
 * coef (HOST): c_{k,j} for k = 0..K, j = -(n_h-1)..n_h-1 as interleaved
 * complex doubles, row k, column j + n_h - 1 (row k = 0 is read for j >= 0
 * only).  The similarity g(q) = (alpha(q), s(q)) multiplies harmonic (k, j)
 * by e^{-i k alpha} e^{-i w_j ln s} on the same support (the centre tap is
 * invariant), i.e. (T_g F)(d) is F's log-polar expansion at (theta(d) -
 * alpha, ln|d| - ln s).  Modes as for ext_conv_scale:
 *   mode 0: out_c = {H_c, g} * F
 *   mode 1: out_c = {H_c, g} * F / {1, g} * F
 *   mode 2: out_c = {H_c / s^2, g} * F / {1 / s^2, g} * F
 * H, out: channels planes of h x w float32; alpha (radians), s (> 0): h x w
 * float32.  Cost: one steered transform per unique harmonic, n_h + K (2 n_h
 * - 1) of them, per signal (channels, plus the denominator in modes 1, 2);
 * EXT_ERR_UNSUPPORTED when their spectra would exceed 8 GiB.
 */
ext_status ext_conv_similarity(ext_plan plan, const float* H, int channels, int h, int w, const double* coef, int K,
                               int n_h, double log_period, double r_min, double r_max, double centre_tap,
                               const float* alpha, const float* s, int mode, float* out, void* stream);

/*
 * SO(3) extended correlation (Sec. 9).  Volume V: nz x ny x nx float32
 * (z slowest; x = column, y = row, z = slice), periodic.  Filter
 *   F(x) = sum_{l<=L} sum_{|a|<=l} f_l^a(|x|) Y_l^a(x^)
 * with orthonormal Condon-Shortley spherical harmonics (theta from +z,
 * phi = atan2(y, x)); `tables` (HOST) holds f_l^a(i dr), i < n_r, as complex
 * doubles, row l^2 + l + a; cubic Hermite in r with parity (-1)^l and closed
 * support as for ext_filter_so2 tables; at x = 0 only l = 0 contributes; the
 * box is [-R, R]^3.  A real filter (f_l^{-a} = (-1)^a conj f_l^a) is assumed.
 * Rotations act as (T_R F)(x) = F(R^-1 x); C^l_ab(R) is the coefficient of
 * Y_l^b in T_R Y_l^a; the score of rotation R at voxel p is
 *   S(p, R) = sum_d V(p+d) conj((T_R F)(d)) = sum_{l,a,b} conj(C^l_ab(R)) G_l^{ab}(p),
 * G_l^{ab} = V (*) (f_l^a Y_l^b).  Rotations are unit quaternions (w, x, y, z),
 * HOST memory.  L <= 6.
 *
 * Real channel layout of G (ext_so3_channels(L) channels, one plane each):
 * for l = 0..L: the self pair (a, b) = (0, 0) (one channel, Re G), then the
 * pairs (0, b > 0) and (a > 0, any b) in order of a then b (two channels,
 * Re G and Im G); (-a, -b) is implied by G_l^{-a,-b} = (-1)^{a+b} conj G_l^{ab}.
 */
int ext_so3_channels(int L);
/* C^l(R) for every rotation, l = 0..L, row-major (2l+1)^2 blocks per l, as
 * complex doubles into HOST out (n_rot * sum_l (2l+1)^2 complex values). */
ext_status ext_so3_wigner(ext_plan plan, const double* quats, int n_rot, int L, double* out);
/* The component correlations in the real channel layout (Sec. 9 "Standard
 * Correlation"): G = ext_so3_channels(L) planes of nz*ny*nx floats. */
ext_status ext_corr_so3_components(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L,
                                   int n_r, double dr, int R, float* G, void* stream);
/* Sweep over n_rot rotations (Sec. 9 "Linear Combination" at every rotation):
 * per voxel max_R S and the first maximising rotation index. */
ext_status ext_sweep_so3(ext_plan plan, const float* G, int64_t n_vox, int L, const double* quats, int n_rot,
                         float* max_out, int32_t* argmax, int precision, void* stream);
/*
 * SO(3) extended convolution (Eq. Def-EConv, scatter form, with a rotation at
 * every INPUT voxel; component form of Sec. 9):
 *   out(p) = sum_q V(q) (T_{R(q)} F)(p - q)
 *          = sum_{l,a,b} ((V C^l_ab(R(.))) (*) (f_l^a Y_l^b))(p),
 * periodic, with the volume, filter tables, box and C^l_ab conventions of
 * ext_corr_so3 above (a real filter, so out is real).  quats: nz*ny*nx unit
 * quaternions (w, x, y, z) as float32 [n_vox][4], HOST or device (a device
 * pointer 16-byte aligned, else EXT_ERR_INVALID_ARG); they are
 * normalised on use and a zero quaternion acts as the identity.  V, out:
 * nz*ny*nx float32.  Cost: one complex 3D transform per unique (l, a, b)
 * (231 for L = 6) and one inverse; the component spectra are cached per
 * filter and volume shape.  Workspace: up to 4 GiB of modulated planes.
 */
ext_status ext_conv_so3(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L, int n_r,
                        double dr, int R, const float* quats, float* out, void* stream);
/* Components then sweep. */
ext_status ext_corr_so3(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L, int n_r,
                        double dr, int R, const double* quats, int n_rot, float* max_out, int32_t* argmax,
                        int precision, void* stream);
/*
 * The sweep over a product grid of rotations R_{d,t} = R_d R_z(2 pi t / n_psi)
 * (n_dirs direction rotations R_d, HOST quaternions [n_dirs][4], each followed
 * on the right by n_psi uniformly spaced rotations about z; rotation index
 * d * n_psi + t), e.g. a Hopf-fibration grid.  Sec. 9's score factors over
 * the in-plane angle: C(R_d R_z(psi)) = C(R_z(psi)) C(R_d) with
 * C^l_ab(R_z(psi)) = delta_ab e^{-i a psi}, so
 *   S(p, R_{d,t}) = H_0 + 2 sum_{a=1..L} Re(e^{i a psi_t} H_a),
 *   H_a(p, d) = sum_{l >= a, b} conj(C^l_ab(R_d)) G_l^{ab}(p)
 * (H_{-a} = conj(H_a) for a real score).  With EXT_PREC_BF16X3 the 2L+1 real
 * H values of every direction come from a split-BF16 tensor-core GEMM and the
 * n_psi angles are steered in its epilogue; EXT_PREC_FP32 sweeps the
 * expanded rotation list as ext_sweep_so3.  Outputs as ext_sweep_so3 (max and
 * the first maximising index).  n_psi <= 64; L <= 6.
 */
ext_status ext_sweep_so3_grid(ext_plan plan, const float* G, int64_t n_vox, int L, const double* dir_quats,
                              int n_dirs, int n_psi, float* max_out, int32_t* argmax, int precision, void* stream);
/* Components then the product-grid sweep. */
ext_status ext_corr_so3_grid(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L,
                             int n_r, double dr, int R, const double* dir_quats, int n_dirs, int n_psi,
                             float* max_out, int32_t* argmax, int precision, void* stream);

/*
 * Learned SO(3) proposal (Sec. 9 matching, with a network proposing the
 * rotation instead of sweeping a grid everywhere).
 *
 * Score bounds.  For every rotation R, |S(p, R)| <= UB(p) = sum_l sqrt(2l+1)
 * |G_l(p)|_F (Cauchy-Schwarz; C^l(R) is unitary with |C^l|_F^2 = 2l+1), and
 * also <= sum_l |G_l(p)|_* (nuclear norm: Re tr(U^H G) <= |G|_* for every
 * unitary U).  The proposal evaluates UB at every voxel; where UB >= B it
 * bounds the nuclear norms from above without an SVD (two orthonormal
 * directions from one block power step, the rest by sqrt(rank) times the
 * Frobenius norm) and keeps the smaller bound per degree.  Voxels whose bound
 * is below the detection threshold B cannot reach it and are not evaluated
 * further.
 *
 * Proposal.  For the other voxels (the candidates) the network maps the
 * unit-normalised channel vector x = G(p)/|G(p)| to a unit quaternion, which
 * `refine` improves by gradient ascent on the exact score S(p, R) (5 steps;
 * the gradient in the body frame, d/dxi_i S(R exp(xi e_i)), exactly from the
 * rotation generators acting on C^l(R); a step moves by an angle t along it,
 * t = 0.25 at first, halved up to 6 times until S increases, none: stop; an
 * accepted step keeps t).  The refinement runs in FP32.
 *
 * Fallback.  Every candidate whose refined score is below B is swept over the
 * rotation grid as in ext_sweep_so3; the higher of the two results is kept.
 * So every voxel with max_R S(p, R) >= B on the grid ends with a score >= B.
 *
 * Quaternions are (w, x, y, z) with the rotation matrix of a unit quaternion;
 * q and -q are the same rotation.
 */
typedef struct ext_mlp_s* ext_mlp;

/* A network n_in -> hidden -> hidden -> 4 with ReLU; x = row / |row| on input,
 * output o normalised to q = o / |o|; loss mean_i (1 - <q_i, q*_i>^2).  BF16
 * weights and activations on the tensor cores, FP32 accumulation, FP32 master
 * weights for Adam (Kingma & Ba: beta1 0.9, beta2 0.999, eps 1e-8).  hidden a
 * multiple of 16 in [16, 1024]; 1 <= n_in <= 4096.  Weights start at zero:
 * set them with ext_mlp_set_params.  The network runs on its plan's device
 * and workspace: every call but ext_mlp_destroy needs the plan alive. */
ext_status ext_mlp_create(ext_plan plan, int n_in, int hidden, ext_mlp* out);
ext_status ext_mlp_destroy(ext_mlp net);
/* Row-major FP32 W1 [hidden][n_in], b1 [hidden], W2 [hidden][hidden], b2
 * [hidden], W3 [4][hidden], b3 [4]; host or device pointers.  Resets Adam. */
ext_status ext_mlp_set_params(ext_mlp net, const float* W1, const float* b1, const float* W2, const float* b2,
                              const float* W3, const float* b3);
ext_status ext_mlp_get_params(ext_mlp net, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3);
/*
 * Checkpoint of the network's whole training state, so that training resumes
 * where it stopped: FP32 master weights, both Adam moments and the step count.
 * File layout (little endian):
 *   bytes 0..7    magic "EXTMLP01"
 *   8..11         uint32 version (1)
 *   12..15        uint32 n_in;   16..19 uint32 hidden;   20..23 uint32 zero
 *   24..31        uint64 Adam steps taken
 *   32..39        uint64 n = hidden (n_in + hidden + 6) + 4, floats per block
 *   40..          float32 weights [n], first moments [n], second moments [n],
 *                 each block W1, b1, W2, b2, W3, b3 in the shapes of
 *                 ext_mlp_set_params
 *   last 4 bytes  uint32 CRC-32 (IEEE 802.3: reflected polynomial 0xEDB88320,
 *                 initial value and final xor 0xFFFFFFFF) of all bytes before it
 * ext_mlp_save writes it (after waiting for the device); ext_mlp_load checks
 * magic, version, length, CRC and that n_in and hidden equal the network's,
 * and only then replaces the state: EXT_ERR_CHECKPOINT (state unchanged) on
 * any mismatch or unreadable file.  ext_mlp_checkpoint_info checks a file the
 * same way on the host alone (no device work) and returns its shapes and step.
 */
ext_status ext_mlp_save(ext_mlp net, const char* path);
ext_status ext_mlp_load(ext_mlp net, const char* path);
ext_status ext_mlp_checkpoint_info(const char* path, int* n_in, int* hidden, int64_t* step);
/* q [n][4] = the network's unit quaternion of each row of X [n][n_in]. */
ext_status ext_mlp_forward(ext_mlp net, const float* X, int n, float* q, void* stream);
/* Mean loss of rows X [n][n_in] against targets qt [n][4] into *loss (host or
 * device float) and its gradients, concatenated in the parameter order and
 * shapes of ext_mlp_set_params, into grads (host or device; NULL: none). */
ext_status ext_mlp_grads(ext_mlp net, const float* X, const float* qt, int n, float* loss, float* grads,
                         void* stream);
/* `steps` Adam steps of learning rate lr on batches of `batch` rows of the
 * training set X [n_train][n_in], targets qt [n_train][4]: step s uses rows
 * rows[s*batch .. s*batch+batch-1] (int32, in [0, n_train)).  If Q (float
 * [steps*batch][4] unit quaternions) is given, row i of step s is first
 * rotated by Q[s*batch+i] as in ext_so3_augment (then n_in must equal
 * ext_so3_channels(L)).  losses [steps] (host or device, or NULL) receives
 * each step's mean loss.  All arrays host or device. */
ext_status ext_mlp_train(ext_mlp net, const float* X, const float* qt, int n_train, int L, const int32_t* rows,
                         const float* Q, int steps, int batch, float lr, float* losses, void* stream);

/* UB(p) for every voxel of G (channel layout of ext_corr_so3_components). */
ext_status ext_so3_upper_bound(ext_plan plan, const float* G, int64_t n_vox, int L, float* ub, void* stream);
/* The refined bound of each row of X [n][ext_so3_channels(L)] (channel
 * vectors): sum_l min(sqrt(2l+1) |G_l|_F, an upper bound of |G_l|_*) into
 * out [n]; it is >= sum_l |G_l|_* >= max_R |S(R)|. */
ext_status ext_so3_refined_bound(ext_plan plan, const float* X, int n, int L, float* out, void* stream);
/* X [n][ext_so3_channels(L)] = the channel vectors G(:, vox[i]) (raw, not
 * normalised); vox int32 in [0, n_vox). */
ext_status ext_so3_gather(ext_plan plan, const float* G, int64_t n_vox, int L, const int32_t* vox, int n, float* X,
                          void* stream);
/* Rotation augmentation: the score function S'(R) = S(Q^-1 R) of row X[i]
 * has the channels X_out[i] (G'_l = G_l C^l(Q)), and its maximiser is Q R*:
 * q_out[i] = Q[i] q_in[i] (float quaternions [n][4]). */
ext_status ext_so3_augment(ext_plan plan, const float* X, int n, int L, const float* Q, const float* q_in,
                           float* X_out, float* q_out, void* stream);
/* The refinement alone: from q0 [n][4] on the channel rows X [n][C], C =
 * ext_so3_channels(L): refined unit quaternions q_out [n][4] and scores
 * s_out [n]. */
ext_status ext_so3_refine(ext_plan plan, const float* X, int n, int L, const float* q0, float* q_out, float* s_out,
                          void* stream);
/* The whole proposal on component channels G (n_vox voxels).  net may be NULL:
 * then every candidate goes to the grid sweep.  Outputs per voxel: score
 * (-infinity where UB < B), quat [n_vox][4] (the rotation found; identity
 * where UB < B; may be NULL) and grid_idx (-2: not a candidate, -1: refined
 * rotation kept, j >= 0: swept, j the grid argmax; may be NULL).  counts
 * (host int64[3], may be NULL): voxels with UB >= B, candidates (refined
 * bound >= B), swept candidates.  The call synchronises `stream` up to three
 * times to size its launches. */
ext_status ext_so3_propose(ext_plan plan, const float* G, int64_t n_vox, int L, ext_mlp net, const double* quats,
                           int n_rot, float bound, float* score, float* quat, int32_t* grid_idx, int precision,
                           int64_t* counts, void* stream);
/* Components (ext_corr_so3_components) then ext_so3_propose. */
ext_status ext_corr_so3_propose(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L,
                                int n_r, double dr, int R, ext_mlp net, const double* quats, int n_rot, float bound,
                                float* score, float* quat, int32_t* grid_idx, int precision, int64_t* counts,
                                void* stream);

/*
 * Pattern detection front end (Sec. 5 "Defining the Filter and Transformation
 * Field").  Signal and field of an image I (Eq. signal, Eq. theta):
 *   H_out = |grad I|,  theta_out = atan2(dI/dy, dI/dx)  (radians),
 * with central differences and periodic indices,
 *   dI/dx(y, x) = (I(y, x+1) - I(y, x-1)) / 2,  x = column, y = row.
 * I, H_out, theta_out: h x w float32, row-major (host or device).  H_out and
 * theta_out feed ext_conv_so2 as the signal and the rotation field.
 */
ext_status ext_gradient_field(ext_plan plan, const float* I, int h, int w, float* H_out, float* theta_out,
                              void* stream);

/*
 * Consensus filter (Sec. 5, Eq. opt_filt; the appendix derives it as the
 * filter maximising the extended-convolution response at the centre): every
 * pixel q of the pattern P with |q - c| <= eps votes with weight |grad P(q)|
 * (gradient as in ext_gradient_field, periodic within P, FP64) into the bin
 *   d = R(-theta_P(q)) (c - q),  R(a) = [[cos a, -sin a], [sin a, cos a]],
 * the unit impulse being a bilinear splat onto integer offsets.  P: hp x wp
 * float64 row-major; c = (cy, cx) a pixel of P; F_out: (2R+1) x (2R+1)
 * float64 with R = ext_consensus_radius(eps) = ceil(eps) + 1, offset (dx, dy)
 * at F_out[(dy + R)(2R + 1) + dx + R].  Use it as a SAMPLED ext_filter_so2
 * (img = F_out, R) for ext_conv_so2.  EXT_ERR_INVALID_ARG for an empty
 * pattern, a centre outside it or eps outside [0, 4096].
 */
int ext_consensus_radius(double eps);
ext_status ext_consensus_filter(ext_plan plan, const double* P, int hp, int wp, int cy, int cx, double eps,
                                double* F_out, void* stream);

/*
 * Pattern detection (Sec. 5): the response {H, theta} * F of Eq. Def-EConv
 * with the signal H = |grad I| and field theta of ext_gradient_field, F
 * typically the consensus filter of ext_consensus_filter (as a SAMPLED
 * filter).  I, out: h x w float32 (host or device); the gradient and the
 * steered transforms stay in plan workspace.
 */
ext_status ext_ght_detect(ext_plan plan, const float* I, int h, int w, const ext_filter_so2* F, float* out,
                          void* stream);

/*
 * Allocation-free variant of the FP32 angular sweep (the paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * allocate device memory -- an application whose device memory is all owned
 * by its own allocator, a latency-critical loop that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree imply, or a process under a
 * fixed device-memory reservation).  Same arithmetic and outputs as
 * ext_sweep_so2 with EXT_PREC_FP32, but no plan and no allocation of any
 * kind: its only scratch, the steering-weight table, lives in a fixed 16 KB
 * device array inside the library (every GPU that loads the library keeps it
 * until the process exits).  Limits: 1 <= K <= 16, 1 <= n_angles <= 128;
 * larger sizes return EXT_ERR_UNSUPPORTED.  G, max_out and argmax must be
 * DEVICE buffers of the current device (EXT_ERR_INVALID_ARG otherwise).  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; make that first call before any stream capture.  A reset of
 * the device's primary context (cudaDeviceReset) while the library is loaded
 * is not supported by this entry point.  If a CUDA error from earlier work is
 * already pending on the calling thread, the call launches nothing, returns
 * EXT_ERR_CUDA and leaves that error in place.  All calls share the one table
 * and each call rewrites it in full on `stream`: calls that overlap on the GPU
 * (different streams, or different threads) race on it.
 */
ext_status ext_sweep_so2_noalloc(const float* G, int64_t n_pix, int K, int n_angles, float* max_out,
                                 int32_t* argmax, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* EXTCONV_H */
