// FP64 filter-side kernels: the filter decomposition of Sec. 4.1 ("Filter
// Decomposition"), the sampling of every component F_k = f_k(r) e^{ik theta}
// on the FFT grid, and the tables (twiddles, sweep steering weights).  These
// run once per filter/size and are cached by the plan; they are the only
// FP64 arithmetic on the device.
#include "internal.h"

#include <cmath>

// ------------------------------------------------------------- twiddles ---
__global__ void k_twiddle(float2* tw, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)n, &s, &c);
  tw[m] = make_float2((float)c, (float)(-s));   // exp(-2 pi i m / n)
}

void launch_twiddle(float2* tw, int n, cudaStream_t st) {
  k_twiddle<<<(n + 255) / 256, 256, 0, st>>>(tw, n);
}

// ------------------------------------------------ polar decomposition ---
// Keys cubic convolution kernel, a = -1/2.
__device__ __forceinline__ double keys_w(double x) {
  const double a = -0.5;
  x = fabs(x);
  if (x <= 1.0) return ((a + 2.0) * x - (a + 3.0)) * x * x + 1.0;
  if (x < 2.0) return ((a * x - 5.0 * a) * x + 8.0 * a) * x - 4.0 * a;
  return 0.0;
}

// P[i][t] = image sampled (Keys bicubic, zero outside) at radius i*dr and
// angle 2 pi t / n_theta around the centre pixel (R, R); x = column, y = row.
__global__ void k_polar_sample(const double* __restrict__ img, int side, double dr, int n_r, int n_theta,
                               double* __restrict__ P) {
  const int i = blockIdx.x;
  const int R = (side - 1) / 2;
  for (int t = threadIdx.x; t < n_theta; t += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)t / (double)n_theta, &s, &c);
    const double r = i * dr;
    const double cx = R + r * c, cy = R + r * s;
    const double fx = floor(cx), fy = floor(cy);
    const int x0 = (int)fx, y0 = (int)fy;
    const double tx = cx - fx, ty = cy - fy;
    double acc = 0.0;
    for (int jy = -1; jy <= 2; ++jy) {
      const int yy = y0 + jy;
      if (yy < 0 || yy >= side) continue;
      const double wy = keys_w(ty - jy);
      for (int jx = -1; jx <= 2; ++jx) {
        const int xx = x0 + jx;
        if (xx < 0 || xx >= side) continue;
        acc += wy * keys_w(tx - jx) * img[(size_t)yy * side + xx];
      }
    }
    P[(size_t)i * n_theta + t] = acc;
  }
}

// f_k(r_i) = (1/n_theta) sum_t P[i][t] e^{-i k theta_t}, k = -K..K at row k+K.
// At r = 0 only k = 0 is kept (the angle is undefined there).
__global__ void k_angular_dft(const double* __restrict__ P, int n_r, int n_theta, int K,
                              double2* __restrict__ fk) {
  const int kk = blockIdx.y;            // 0..2K
  const int k = kk - K;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_r) return;
  double re = 0.0, im = 0.0;
  for (int t = 0; t < n_theta; ++t) {
    int m = (int)(((long long)k * t) % n_theta);
    if (m < 0) m += n_theta;
    double s, c;
    sincospi(2.0 * (double)m / (double)n_theta, &s, &c);
    const double p = P[(size_t)i * n_theta + t];
    re += p * c;
    im -= p * s;
  }
  re /= n_theta;
  im /= n_theta;
  if (i == 0) {
    if (k != 0) { re = 0.0; im = 0.0; }
    else { re = P[0]; im = 0.0; }
  }
  fk[(size_t)kk * n_r + i] = make_double2(re, im);
}

void launch_decompose_sampled(const double* img, int side, double dr, int n_r, int n_theta, int K,
                              double* P, double2* fk, cudaStream_t st) {
  k_polar_sample<<<n_r, 128, 0, st>>>(img, side, dr, n_r, n_theta, P);
  dim3 grid((n_r + 127) / 128, 2 * K + 1);
  k_angular_dft<<<grid, 128, 0, st>>>(P, n_r, n_theta, K, fk);
}

// ----------------------------------------------------- component sampling ---
// Cubic Hermite interpolation of a radial table v_i = f_k(i dr):
// tangents m_i = (v_{i+1} - v_{i-1}) / 2, v_{-1} = (-1)^k v_1, v_n = 0,
// f = 0 for r / dr > (n-1) + 1e-9 (closed support; boundary points inside).
__device__ double2 radial_table(const double2* __restrict__ v, int n, double dr, int k, double r) {
  const double u = r / dr;
  if (u > (double)(n - 1) + 1e-9 || n < 2) return make_double2(0.0, 0.0);
  int i = (int)floor(u);
  if (i > n - 1) i = n - 1;
  const double t = u - i;
  auto at = [&](int j) -> double2 {
    if (j < 0) {
      const double2 a = v[1];
      return (k & 1) ? make_double2(-a.x, -a.y) : a;
    }
    if (j >= n) return make_double2(0.0, 0.0);
    return v[j];
  };
  const double2 vm = at(i - 1), v0 = at(i), v1 = at(i + 1), v2 = at(i + 2);
  const double t2 = t * t, t3 = t2 * t;
  const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
  const double m0x = 0.5 * (v1.x - vm.x), m0y = 0.5 * (v1.y - vm.y);
  const double m1x = 0.5 * (v2.x - v0.x), m1y = 0.5 * (v2.y - v0.y);
  return make_double2(h00 * v0.x + h10 * m0x + h01 * v1.x + h11 * m1x,
                      h00 * v0.y + h10 * m0y + h01 * v1.y + h11 * m1y);
}

// F_k(d) for every offset d in the box [-R, R]^2, placed at (d mod (h, w)).
// kind: EXT_FILTER_ANALYTIC_GAUSSPOW uses a[k+K] r^|k| exp(-r^2 / 2 sigma^2);
// tables use radial_table.  With wrap != 0 several offsets share a cell and
// are accumulated atomically.
__global__ void k_component_grid(int kind, int K, int k, const double2* __restrict__ coef, int n_r,
                                 double dr, double sigma, int R, int h, int w, int wrap,
                                 float2* __restrict__ grid) {
  // blockIdx.y selects component k + blockIdx.y, written to plane blockIdx.y
  k += blockIdx.y;
  grid += (size_t)blockIdx.y * h * w;
  const int side = 2 * R + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)side * side) return;
  const int dy = (int)(idx / side) - R, dx = (int)(idx % side) - R;
  const double r = hypot((double)dx, (double)dy);
  double2 f;
  if (kind == EXT_FILTER_ANALYTIC_GAUSSPOW) {
    const double2 a = coef[k + K];
    const double mag = pow(r, (double)abs(k)) * exp(-r * r / (2.0 * sigma * sigma));
    f = make_double2(a.x * mag, a.y * mag);
  } else {
    f = radial_table(coef + (size_t)(k + K) * n_r, n_r, dr, k, r);
  }
  double2 val;
  if (r == 0.0) {
    val = (k == 0) ? f : make_double2(0.0, 0.0);
  } else {
    double s, c;
    sincos((double)k * atan2((double)dy, (double)dx), &s, &c);
    val = make_double2(f.x * c - f.y * s, f.x * s + f.y * c);
  }
  const int gy = ((dy % h) + h) % h, gx = ((dx % w) + w) % w;
  float2* cell = grid + (size_t)gy * w + gx;
  if (wrap) {
    atomicAdd(&cell->x, (float)val.x);
    atomicAdd(&cell->y, (float)val.y);
  } else {
    *cell = make_float2((float)val.x, (float)val.y);
  }
}

void launch_component_grid(int kind, int K, int k, const double2* coef, int n_r, double dr, double sigma,
                           int R, int h, int w, float2* grid, cudaStream_t st, int ncomp) {
  const int side = 2 * R + 1;
  const long long n = (long long)side * side;
  const int wrap = (side > h || side > w) ? 1 : 0;
  dim3 grid_dim((unsigned)((n + 255) / 256), ncomp);
  k_component_grid<<<grid_dim, 256, 0, st>>>(kind, K, k, coef, n_r, dr, sigma, R, h, w, wrap, grid);
}

// -------------------------------------------------------- sweep weights ---
// B[j][c], row padded to `cp` floats: c = 2(k-1) -> 2 cos(2 pi k j / J),
// c = 2(k-1)+1 -> -2 sin(2 pi k j / J), so that
// S(p, j) = G_0 + sum_c A(p, c) B[j][c] = G_0 + 2 sum_k Re(e^{i k alpha_j} G_k).
__global__ void k_sweep_table(int K, int J, int cp, float* __restrict__ B) {
  const int j = blockIdx.x;
  for (int c = threadIdx.x; c < cp; c += blockDim.x) {
    float val = 0.f;
    if (c < 2 * K) {
      const int k = c / 2 + 1;
      const int m = (int)(((long long)k * j) % J);
      double s, co;
      sincospi(2.0 * (double)m / (double)J, &s, &co);
      val = (c & 1) ? (float)(-2.0 * s) : (float)(2.0 * co);
    }
    B[(size_t)j * cp + c] = val;
  }
}

void launch_sweep_table(int K, int J, int cp, float* B, cudaStream_t st) {
  k_sweep_table<<<J, 64, 0, st>>>(K, J, cp, B);
}

// Steering weights of a component list: as k_sweep_table with k = ks[c / 2 + 1].
__global__ void k_sweep_table_list(const int* __restrict__ ks, int K, int J, int cp, float* __restrict__ B) {
  const int j = blockIdx.x;
  for (int c = threadIdx.x; c < cp; c += blockDim.x) {
    float val = 0.f;
    if (c < 2 * K) {
      const int k = ks[c / 2 + 1];
      const int m = (int)(((long long)k * j) % J);
      double s, co;
      sincospi(2.0 * (double)m / (double)J, &s, &co);
      val = (c & 1) ? (float)(-2.0 * s) : (float)(2.0 * co);
    }
    B[(size_t)j * cp + c] = val;
  }
}

void launch_sweep_table_list(const int* ks, int K, int J, int cp, float* B, cudaStream_t st) {
  k_sweep_table_list<<<J, 64, 0, st>>>(ks, K, J, cp, B);
}

// Lattice energy of every component, E_k = sum_{d in [-R, R]^2} |F_k(d)|^2
// (F_k(0) = 0 for k != 0), FP64, one thread per (offset, k = blockIdx.y).
__global__ void k_component_energy(int kind, int K, const double2* __restrict__ coef, int n_r, double dr,
                                   double sigma, int R, double* __restrict__ E) {
  const int k = blockIdx.y;
  const int side = 2 * R + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (idx < (long long)side * side) {
    const int dy = (int)(idx / side) - R, dx = (int)(idx % side) - R;
    const double r = hypot((double)dx, (double)dy);
    double2 f;
    if (kind == EXT_FILTER_ANALYTIC_GAUSSPOW) {
      const double2 a = coef[k + K];
      const double mag = pow(r, (double)k) * exp(-r * r / (2.0 * sigma * sigma));
      f = make_double2(a.x * mag, a.y * mag);
    } else {
      f = radial_table(coef + (size_t)(k + K) * n_r, n_r, dr, k, r);
    }
    if (r > 0.0 || k == 0) e = f.x * f.x + f.y * f.y;   // |e^{ik theta}| = 1
  }
  for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(E + k, e);
}

void launch_component_energy(int kind, int K, const double2* coef, int n_r, double dr, double sigma, int R,
                             double* E, cudaStream_t st) {
  const long long n = (long long)(2 * R + 1) * (2 * R + 1);
  dim3 grid((unsigned)((n + 255) / 256), K + 1);
  k_component_energy<<<grid, 256, 0, st>>>(kind, K, coef, n_r, dr, sigma, R, E);
}

// ------------------------------------------------------ Mellin components ---
// Scale harmonics of Sec. 8, F_k(r) = e^{i w_k ln r} (times the constant f_k of
// a radially symmetric filter): M_k(d) = c_k exp(i w_k ln|d|) on the annulus
// r_min <= |d| <= r_max, w_k = 2 pi k / L.  The centre tap is applied by the
// normalisation epilogue, not here.
__global__ void k_component_grid_mellin(double2 ck, double omega, double r_min, double r_max, int R, int h, int w,
                                        int wrap, float2* __restrict__ grid) {
  const int side = 2 * R + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)side * side) return;
  const int dy = (int)(idx / side) - R, dx = (int)(idx % side) - R;
  const double r = hypot((double)dx, (double)dy);
  if (r < r_min || r > r_max || r == 0.0) return;
  double s, c;
  sincos(omega * log(r), &s, &c);
  const double2 val = make_double2(ck.x * c - ck.y * s, ck.x * s + ck.y * c);
  const int gy = ((dy % h) + h) % h, gx = ((dx % w) + w) % w;
  float2* cell = grid + (size_t)gy * w + gx;
  if (wrap) {
    atomicAdd(&cell->x, (float)val.x);
    atomicAdd(&cell->y, (float)val.y);
  } else {
    *cell = make_float2((float)val.x, (float)val.y);
  }
}

void launch_component_grid_mellin(double2 ck, double omega, double r_min, double r_max, int R, int h, int w,
                                  float2* grid, cudaStream_t st) {
  const int side = 2 * R + 1;
  const long long n = (long long)side * side;
  const int wrap = (side > h || side > w) ? 1 : 0;
  k_component_grid_mellin<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ck, omega, r_min, r_max, R, h, w, wrap, grid);
}

// Log-polar harmonic (k, j) of a similarity filter on its support window,
// coef e^{i (k theta + w_j ln r)}, one plane per blockIdx.y (FP64, plan time).
__global__ void k_component_grid_simil(const double2* __restrict__ coef, const int2* __restrict__ kj, int k0,
                                       double omega_step, double r_min, double r_max, int R, int h, int w, int wrap,
                                       float2* __restrict__ grid) {
  const int side = 2 * R + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)side * side) return;
  const int dy = (int)(idx / side) - R, dx = (int)(idx % side) - R;
  const double r = hypot((double)dx, (double)dy);
  if (r < r_min || r > r_max || r == 0.0) return;
  const int c = k0 + (int)blockIdx.y;
  const double2 ck = coef[c];
  double s, co;
  sincos((double)kj[c].x * atan2((double)dy, (double)dx) + omega_step * kj[c].y * log(r), &s, &co);
  const double2 val = make_double2(ck.x * co - ck.y * s, ck.x * s + ck.y * co);
  const int gy = ((dy % h) + h) % h, gx = ((dx % w) + w) % w;
  float2* cell = grid + (size_t)blockIdx.y * h * w + (size_t)gy * w + gx;
  if (wrap) {
    atomicAdd(&cell->x, (float)val.x);
    atomicAdd(&cell->y, (float)val.y);
  } else {
    *cell = make_float2((float)val.x, (float)val.y);
  }
}

void launch_component_grid_simil(const double2* coef, const int2* kj, int k0, int nk, double omega_step, double r_min,
                                 double r_max, int R, int h, int w, float2* grid, cudaStream_t st) {
  const int side = 2 * R + 1;
  const long long n = (long long)side * side;
  const int wrap = (side > h || side > w) ? 1 : 0;
  dim3 g((unsigned)((n + 255) / 256), (unsigned)nk);
  k_component_grid_simil<<<g, 256, 0, st>>>(coef, kj, k0, omega_step, r_min, r_max, R, h, w, wrap, grid);
}

// ------------------------------------------------ smoothing epilogue ---
// Adds the centre tap c_delta A(p) to every accumulated convolution and, for
// modes 1 and 2, divides each channel by the denominator (Eq. normalization):
//   mode 0: out_c = N_c + c_delta H_c
//   mode 1: out_c = (N_c + c_delta H_c) / (D + c_delta)
//   mode 2: out_c = (N_c + c_delta H_c / s^2) / (D + c_delta / s^2)
__global__ void k_scale_finalize(const float* __restrict__ H, const float* __restrict__ s, const float* __restrict__ N,
                                 const float* __restrict__ D, int channels, long long P, int mode, float cd,
                                 float* __restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    const float sv = __ldg(s + p);
    const float wgt = mode == 2 ? 1.0f / (sv * sv) : 1.0f;
    const float den = mode == 0 ? 1.0f : (__ldg(D + p) + cd * wgt);
    for (int c = 0; c < channels; ++c) {
      const size_t i = (size_t)c * P + p;
      const float num = __ldg(N + i) + cd * wgt * __ldg(H + i);
      out[i] = mode == 0 ? num : num / den;
    }
  }
}

void launch_scale_finalize(const float* H, const float* s, const float* N, const float* D, int channels, long long P,
                           int mode, float cd, float* out, int sms, cudaStream_t st) {
  long long blocks = (P + 255) / 256;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  if (blocks < 1) blocks = 1;
  k_scale_finalize<<<(unsigned)blocks, 256, 0, st>>>(H, s, N, D, channels, P, mode, cd, out);
}
