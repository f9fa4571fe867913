// Pattern-detection front end of Sec. 5: the signal H = |grad I| and the
// rotation field theta = atan2(dI/dy, dI/dx) of an image (Eq. signal, Eq.
// theta), and the consensus filter of Eq. opt_filt built by voting.
//
// Derivatives are central differences with periodic indices,
// dI/dx(y, x) = (I(y, x+1) - I(y, x-1)) / 2 (x = column, y = row).  A
// pattern pixel q with |q - c| <= eps votes with weight |grad P(q)| into the
// bin d = R(-theta_P(q)) (c - q) of the filter box [-R, R]^2, R = ceil(eps) + 1,
// the unit impulse discretised as a bilinear splat (FP64 atomics).
#include <cmath>

#include "plan.h"

namespace {

// H and theta of a float image, one thread per pixel (grid-stride)
__global__ void k_gradient_field(const float* __restrict__ I, int h, int w, float* __restrict__ H,
                                 float* __restrict__ theta) {
  const long long n = (long long)h * w;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / w), x = (int)(i % w);
    const int xp = x + 1 == w ? 0 : x + 1, xm = x == 0 ? w - 1 : x - 1;
    const int yp = y + 1 == h ? 0 : y + 1, ym = y == 0 ? h - 1 : y - 1;
    const float gx = 0.5f * (__ldg(I + (size_t)y * w + xp) - __ldg(I + (size_t)y * w + xm));
    const float gy = 0.5f * (__ldg(I + (size_t)yp * w + x) - __ldg(I + (size_t)ym * w + x));
    H[i] = hypotf(gx, gy);
    theta[i] = atan2f(gy, gx);
  }
}

// votes of the pattern pixels inside the support disk, FP64
__global__ void k_consensus_vote(const double* __restrict__ P, int hp, int wp, int cy, int cx, double eps, int R,
                                 double* __restrict__ F) {
  const long long n = (long long)hp * wp;
  const int side = 2 * R + 1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int qy = (int)(i / wp), qx = (int)(i % wp);
    const double ox = (double)(cx - qx), oy = (double)(cy - qy);   // c - q
    if (ox * ox + oy * oy > eps * eps) continue;
    const int xp = qx + 1 == wp ? 0 : qx + 1, xm = qx == 0 ? wp - 1 : qx - 1;
    const int yp = qy + 1 == hp ? 0 : qy + 1, ym = qy == 0 ? hp - 1 : qy - 1;
    const double gx = 0.5 * (P[(size_t)qy * wp + xp] - P[(size_t)qy * wp + xm]);
    const double gy = 0.5 * (P[(size_t)yp * wp + qx] - P[(size_t)ym * wp + qx]);
    const double mag = hypot(gx, gy);
    if (mag == 0.0) continue;
    const double th = atan2(gy, gx);
    double s, c;
    sincos(th, &s, &c);
    const double dx = c * ox + s * oy, dy = -s * ox + c * oy;   // R(-theta) (c - q)
    const double x0 = floor(dx), y0 = floor(dy);
    const double fx = dx - x0, fy = dy - y0;
    const int ix = (int)x0 + R, iy = (int)y0 + R;
    // |d| <= eps < R - 1, so all four cells are inside the box; checked anyway
    if (ix < 0 || iy < 0 || ix + 1 >= side || iy + 1 >= side) continue;
    atomicAdd(F + (size_t)iy * side + ix, mag * (1.0 - fx) * (1.0 - fy));
    atomicAdd(F + (size_t)iy * side + ix + 1, mag * fx * (1.0 - fy));
    atomicAdd(F + (size_t)(iy + 1) * side + ix, mag * (1.0 - fx) * fy);
    atomicAdd(F + (size_t)(iy + 1) * side + ix + 1, mag * fx * fy);
  }
}

}  // namespace

void launch_gradient_field(const float* I, int h, int w, float* H, float* theta, int sms, cudaStream_t st) {
  long long b = ((long long)h * w + 255) / 256;
  if (b > (long long)sms * 16) b = (long long)sms * 16;
  if (b > 0) k_gradient_field<<<(unsigned)b, 256, 0, st>>>(I, h, w, H, theta);
}

extern "C" {

ext_status ext_gradient_field(ext_plan plan, const float* I, int h, int w, float* H_out, float* theta_out,
                              void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  if (h < 0 || w < 0) return fail(EXT_ERR_INVALID_ARG, "negative image size");
  if (h == 0 || w == 0) return EXT_OK;
  if (!I || !H_out || !theta_out) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)h * w;
  Staged sI, sH, sT;
  EXT_TRY(stage_in(plan, "in_I", I, sizeof(float) * P, st, &sI));
  EXT_TRY(stage_out_alloc(plan, "out_0", H_out, sizeof(float) * P, &sH));
  EXT_TRY(stage_out_alloc(plan, "out_1", theta_out, sizeof(float) * P, &sT));
  launch(plan, "gradient_field", st, [&] {
    launch_gradient_field((const float*)sI.dev, h, w, (float*)sH.dev, (float*)sT.dev, plan->sms, st);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sH, st));
  EXT_TRY(stage_out_finish(sT, st));
  return finish_host(plan, sI.host || sH.host || sT.host, st);
}

int ext_consensus_radius(double eps) { return eps >= 0 ? (int)std::ceil(eps) + 1 : -1; }

ext_status ext_consensus_filter(ext_plan plan, const double* P, int hp, int wp, int cy, int cx, double eps,
                                double* F_out, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  if (hp < 1 || wp < 1) return fail(EXT_ERR_INVALID_ARG, "empty pattern");
  if (!P || !F_out) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  if (!(eps >= 0) || eps > 4096) return fail(EXT_ERR_INVALID_ARG, "eps must be in [0, 4096]");
  if (cy < 0 || cy >= hp || cx < 0 || cx >= wp) return fail(EXT_ERR_INVALID_ARG, "centre outside the pattern");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int R = ext_consensus_radius(eps);
  const size_t side = 2 * (size_t)R + 1;
  Staged sP, sF;
  EXT_TRY(stage_in(plan, "in_P", P, sizeof(double) * (size_t)hp * wp, st, &sP));
  EXT_TRY(stage_out_alloc(plan, "out_F", F_out, sizeof(double) * side * side, &sF));
  EXT_CUDA(cudaMemsetAsync(sF.dev, 0, sizeof(double) * side * side, st));
  long long b = ((long long)hp * wp + 255) / 256;
  if (b > (long long)plan->sms * 16) b = (long long)plan->sms * 16;
  launch(plan, "consensus_vote", st, [&] {
    k_consensus_vote<<<(unsigned)b, 256, 0, st>>>((const double*)sP.dev, hp, wp, cy, cx, eps, R, (double*)sF.dev);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sF, st));
  return finish_host(plan, sP.host || sF.host, st);
}

}  // extern "C"
