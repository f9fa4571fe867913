// SO(3) filter side (Sec. 9), FP64 on the device: spherical harmonics, the
// components f_l^a(r) Y_l^b sampled on the voxel grid, the rotation matrices
// C^l(R) of every rotation of a sweep, and the steering table in the real
// channel layout used by the sweep.
//
// Conventions: orthonormal Y_l^m with the Condon-Shortley phase, theta from
// +z, phi = atan2(y, x); (T_R F)(x) = F(R^-1 x); C^l_ab(R) is the coefficient
// of Y_l^b in T_R Y_l^a.  With R = R_z(alpha) R_y(beta) R_z(gamma) this is
// C^l_ab = e^{-i b alpha} d^l_ba(beta) e^{-i a gamma}, d from Wigner's sum
// formula.
#include "internal.h"

#include <cmath>

namespace {

__device__ double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Y_l^m(theta, phi) for all l <= L (L <= 8) at one direction given by
// cos(theta), sin(theta) and phi; Y[l*l + l + m].
__device__ void sh_all(int L, double ct, double stheta, double phi, double2* Y) {
  const double inv4pi = 0.079577471545947667884;   // 1 / (4 pi)
  double pmm = sqrt(inv4pi);                          // normalised P_0^0
  for (int m = 0; m <= L; ++m) {
    if (m > 0) pmm = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * stheta * pmm;   // Condon-Shortley sign
    double pl2 = 0.0, pl1 = pmm;
    for (int l = m; l <= L; ++l) {
      double p;
      if (l == m) {
        p = pmm;
      } else if (l == m + 1) {
        p = sqrt(2.0 * m + 3.0) * ct * pmm;
      } else {
        const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        const double b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
        p = a * (ct * pl1 - b * pl2);
      }
      if (l > m) {
        pl2 = pl1;
        pl1 = p;
      }
      double s, c;
      sincos(m * phi, &s, &c);
      Y[l * l + l + m] = make_double2(p * c, p * s);
      if (m > 0) {
        const double sg = (m & 1) ? -1.0 : 1.0;     // Y_l^{-m} = (-1)^m conj(Y_l^m)
        Y[l * l + l - m] = make_double2(sg * p * c, -sg * p * s);
      }
    }
  }
}

// cubic Hermite radial interpolant (parity (-1)^l), closed support
__device__ double2 radial_hermite(const double2* __restrict__ v, int n, double dr, int parity, double r) {
  const double u = r / dr;
  if (u > (double)(n - 1) + 1e-9 || n < 2) return make_double2(0.0, 0.0);
  int i = (int)floor(u);
  if (i > n - 1) i = n - 1;
  const double t = u - i;
  auto at = [&](int j) -> double2 {
    if (j < 0) {
      const double2 a = v[1];
      return (parity & 1) ? make_double2(-a.x, -a.y) : a;
    }
    if (j >= n) return make_double2(0.0, 0.0);
    return v[j];
  };
  const double2 vm = at(i - 1), v0 = at(i), v1 = at(i + 1), v2 = at(i + 2);
  const double t2 = t * t, t3 = t2 * t;
  const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
  return make_double2(h00 * v0.x + h10 * 0.5 * (v1.x - vm.x) + h01 * v1.x + h11 * 0.5 * (v2.x - v0.x),
                      h00 * v0.y + h10 * 0.5 * (v1.y - vm.y) + h01 * v1.y + h11 * 0.5 * (v2.y - v0.y));
}

}  // namespace

// Components (l, a, b) = comp[k0 + blockIdx.y]: Phi(d) = f_l^a(|d|) Y_l^b(d^)
// on the box [-R, R]^3, wrapped onto the nz x ny x nx grid (plane blockIdx.y).
__global__ void k_so3_component_grid(const int4* __restrict__ comp, int k0, const double2* __restrict__ tables, int n_r,
                                     double dr, int L, int R, int nz, int ny, int nx, int wrap,
                                     float2* __restrict__ grid) {
  const int side = 2 * R + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)side * side * side) return;
  const int4 c = comp[k0 + blockIdx.y];
  const int l = c.x, a = c.y, b = c.z;
  float2* g = grid + (size_t)blockIdx.y * nz * ny * nx;
  const int dz = (int)(idx / (side * side)) - R;
  const int dy = (int)((idx / side) % side) - R;
  const int dx = (int)(idx % side) - R;
  const double r = sqrt((double)dx * dx + (double)dy * dy + (double)dz * dz);
  double2 val;
  if (r == 0.0) {
    if (l != 0) return;
    const double2 f = radial_hermite(tables, n_r, dr, 0, 0.0);
    const double y00 = 0.28209479177387814347;   // Y_0^0
    val = make_double2(f.x * y00, f.y * y00);
  } else {
    const double2 f = radial_hermite(tables + (size_t)(l * l + a + l) * n_r, n_r, dr, l, r);
    if (f.x == 0.0 && f.y == 0.0) return;
    double2 Y[81];
    const double ct = dz / r;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    sh_all(l, ct, st, atan2((double)dy, (double)dx), Y);
    const double2 y = Y[l * l + l + b];
    val = make_double2(f.x * y.x - f.y * y.y, f.x * y.y + f.y * y.x);
  }
  const int gz = ((dz % nz) + nz) % nz, gy = ((dy % ny) + ny) % ny, gx = ((dx % nx) + nx) % nx;
  float2* cell = g + ((size_t)gz * ny + gy) * nx + gx;
  if (wrap) {
    atomicAdd(&cell->x, (float)val.x);
    atomicAdd(&cell->y, (float)val.y);
  } else {
    *cell = make_float2((float)val.x, (float)val.y);
  }
}

void launch_so3_component_grid(const int4* comp, int k0, int nk, const double2* tables, int n_r, double dr, int L,
                               int R, int nz, int ny, int nx, float2* grid, cudaStream_t st) {
  const int side = 2 * R + 1;
  const long long n = (long long)side * side * side;
  const int wrap = (side > nz || side > ny || side > nx) ? 1 : 0;
  dim3 g((unsigned)((n + 127) / 128), nk);
  k_so3_component_grid<<<g, 128, 0, st>>>(comp, k0, tables, n_r, dr, L, R, nz, ny, nx, wrap, grid);
}

// Rotation matrices C^l(R_j), l <= L, for every quaternion (w, x, y, z):
// C[j][l^2 ... ] row-major (2l+1)^2 blocks (offset sum_{l'<l} (2l'+1)^2).
// Optionally the steering row of the sweep for every channel:
//   self channel (l, 0, 0): C^l_00;  pair (l, a, b): 2 Re C^l_ab, 2 Im C^l_ab.
__global__ void k_so3_wigner(const double* __restrict__ quats, int n, int L, double2* __restrict__ Cout,
                             const int4* __restrict__ chans, int nchan, int cpad, float* __restrict__ Brow) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double w = quats[4 * j], x = quats[4 * j + 1], y = quats[4 * j + 2], z = quats[4 * j + 3];
  const double nrm = sqrt(w * w + x * x + y * y + z * z);
  w /= nrm; x /= nrm; y /= nrm; z /= nrm;
  const double R00 = 1 - 2 * (y * y + z * z), R01 = 2 * (x * y - w * z), R02 = 2 * (x * z + w * y);
  const double R10 = 2 * (x * y + w * z), R11 = 1 - 2 * (x * x + z * z), R12 = 2 * (y * z - w * x);
  const double R20 = 2 * (x * z - w * y), R21 = 2 * (y * z + w * x), R22 = 1 - 2 * (x * x + y * y);
  (void)R01; (void)R11;
  // zyz Euler angles: R = R_z(alpha) R_y(beta) R_z(gamma)
  const double beta = acos(fmin(1.0, fmax(-1.0, R22)));
  double alpha, gamma;
  if (sin(beta) > 1e-12) {
    alpha = atan2(R12, R02);
    gamma = atan2(R21, -R20);
  } else if (R22 > 0) {
    alpha = atan2(R10, R00);
    gamma = 0.0;
  } else {
    alpha = atan2(-R10, -R00);
    gamma = 0.0;
  }
  const double cb = cos(0.5 * beta), sb = sin(0.5 * beta);
  size_t off = 0;
  double2* C = Cout ? Cout + (size_t)j * ((L + 1) * (2 * L + 1) * (2 * L + 3) / 3) : nullptr;
  // also keep the blocks locally for the steering row (L <= 6: 455 entries)
  double2 loc[455];
  for (int l = 0; l <= L; ++l) {
    const int d = 2 * l + 1;
    for (int a = -l; a <= l; ++a) {
      for (int b = -l; b <= l; ++b) {
        // d^l_{m' m}(beta) with m' = b, m = a
        const int mp = b, m = a;
        double sum = 0.0;
        const int smin = (m - mp) > 0 ? (m - mp) : 0;
        const int smax = (l + m) < (l - mp) ? (l + m) : (l - mp);
        for (int s = smin; s <= smax; ++s) {
          const double num = ((mp - m + s) & 1) ? -1.0 : 1.0;
          const double den = fact(l + m - s) * fact(s) * fact(mp - m + s) * fact(l - mp - s);
          sum += num / den * pow(cb, 2 * l + m - mp - 2 * s) * pow(sb, mp - m + 2 * s);
        }
        const double dval = sqrt(fact(l + mp) * fact(l - mp) * fact(l + m) * fact(l - m)) * sum;
        double s1, c1;
        sincos(-(b * alpha + a * gamma), &s1, &c1);
        const double2 cab = make_double2(dval * c1, dval * s1);
        const size_t e = off + (size_t)(a + l) * d + (b + l);
        if (C) C[e] = cab;
        if (e < 455) loc[e] = cab;
      }
    }
    off += (size_t)d * d;
  }
  if (Brow && L <= 6) {
    float* row = Brow + (size_t)j * cpad;
    for (int c = 0; c < cpad; ++c) row[c] = 0.f;
    for (int q = 0; q < nchan; ++q) {
      const int4 ch = chans[q];   // (l, a, b, first channel); a = b = 0 is the self channel
      const int l = ch.x;
      const size_t base = (size_t)l * (2 * l - 1) * (2 * l + 1) / 3;   // sum_{l'<l} (2l'+1)^2
      const double2 cab = loc[base + (size_t)(ch.y + l) * (2 * l + 1) + (ch.z + l)];
      if (ch.y == 0 && ch.z == 0) {
        row[ch.w] = (float)cab.x;
      } else {
        row[ch.w] = (float)(2.0 * cab.x);
        row[ch.w + 1] = (float)(2.0 * cab.y);
      }
    }
  }
}

void launch_so3_wigner(const double* quats, int n, int L, double2* C, const int4* chans, int nchan, int cpad,
                       float* Brow, cudaStream_t st) {
  k_so3_wigner<<<(n + 63) / 64, 64, 0, st>>>(quats, n, L, C, chans, nchan, cpad, Brow);
}

__global__ void k_real_to_complex(const float* __restrict__ V, long long n, float2* __restrict__ X) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    X[i] = make_float2(__ldg(V + i), 0.f);
}

void launch_real_to_complex(const float* V, long long n, float2* X, int sms, cudaStream_t st) {
  long long b = (n + 255) / 256;
  if (b > (long long)sms * 8) b = (long long)sms * 8;
  k_real_to_complex<<<(unsigned)b, 256, 0, st>>>(V, n, X);
}

// Steering rows of a direction set for the grid sweep over R = R_d R_z(psi)
// (rotation about z applied first).  C(R_d R_z(psi)) = C(R_z(psi)) C(R_d) and
// C(R_z(psi)) = diag(e^{-i a psi}), so
//   S(p, R) = sum_{l,a,b} conj(C^l_ab(R)) G_l^{ab}(p) = sum_a e^{i a psi} H_a(p),
//   H_a = sum_{l >= |a|, b} conj(C^l_ab(R_d)) G_l^{ab},
// and since S is real, H_{-a} = conj(H_a): S = H_0 + 2 sum_{a >= 1} Re(e^{i a psi} H_a).
// Per direction 16 rows over the real channels: row 0 = H_0 (real), rows 2a-1
// and 2a = Re H_a and Im H_a (a = 1..L), the rest zero.  C: the Wigner blocks of
// every direction as k_so3_wigner writes them; comps: (l, a, b, first channel)
// of the stored components (G^{-a,-b} = (-1)^{a+b} conj G^{ab}).
__global__ void k_so3_grid_rows(const double2* __restrict__ C, int n_dirs, int L, const int4* __restrict__ comps,
                                int ncomp, int cpad, float* __restrict__ Brow) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dirs) return;
  const size_t per = (size_t)(L + 1) * (2 * L + 1) * (2 * L + 3) / 3;
  const double2* Cd = C + (size_t)d * per;
  float* rows = Brow + (size_t)d * 16 * cpad;
  for (int i = 0; i < 16 * cpad; ++i) rows[i] = 0.f;
  for (int q = 0; q < ncomp; ++q) {
    const int4 cp = comps[q];
    const int l = cp.x, a = cp.y, b = cp.z, ch = cp.w;
    const size_t off = (size_t)l * (2 * l - 1) * (2 * l + 1) / 3;
    const double2 c = Cd[off + (size_t)(a + l) * (2 * l + 1) + (b + l)];
    if (a == 0 && b == 0) {
      rows[ch] += (float)c.x;                                    // H_0 += Re C_00 G (G real)
    } else if (a == 0) {                                         // (0, b) and its partner (0, -b)
      const double2 cm = Cd[off + (size_t)l * (2 * l + 1) + (-b + l)];
      const double sg = (b & 1) ? -1.0 : 1.0;
      rows[ch] += (float)(c.x + sg * cm.x);
      rows[ch + 1] += (float)(c.y - sg * cm.y);
    } else {                                                     // a > 0: H_a += conj(C_ab) G^{ab}
      float* re = rows + (size_t)(2 * a - 1) * cpad;
      float* im = rows + (size_t)(2 * a) * cpad;
      re[ch] += (float)c.x;
      re[ch + 1] += (float)c.y;
      im[ch] += (float)(-c.y);
      im[ch + 1] += (float)c.x;
    }
  }
}

void launch_so3_grid_rows(const double2* C, int n_dirs, int L, const int4* comps, int ncomp, int cpad, float* Brow,
                          cudaStream_t st) {
  k_so3_grid_rows<<<(n_dirs + 63) / 64, 64, 0, st>>>(C, n_dirs, L, comps, ncomp, cpad, Brow);
}
