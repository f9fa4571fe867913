// C ABI of libextconv.so, SO(3) operators: components, sweeps and the
// learned proposal.
#include "plan.h"

#include <cmath>

// ------------------------------------------------------------------ SO(3) ---
namespace {

struct So3Layout {
  std::vector<int4> comp;    // unique components (l, a, b, first channel)
  std::vector<int2> chan;    // per component: (real channel, imaginary channel or -1)
  int nchan = 0;
};

// Unique (l, a, b) up to the pairing (a, b) <-> (-a, -b) of a real filter and
// signal: for each l the self pair (0, 0) (one real channel), then (0, b > 0)
// and (a > 0, any b) (two channels: real and imaginary part).
So3Layout so3_layout(int L) {
  So3Layout o;
  for (int l = 0; l <= L; ++l) {
    o.comp.push_back(make_int4(l, 0, 0, o.nchan));
    o.chan.push_back(make_int2(o.nchan, -1));
    o.nchan += 1;
    for (int a = 0; a <= l; ++a)
      for (int b = -l; b <= l; ++b) {
        if (a == 0 && b <= 0) continue;
        o.comp.push_back(make_int4(l, a, b, o.nchan));
        o.chan.push_back(make_int2(o.nchan, o.nchan + 1));
        o.nchan += 2;
      }
  }
  return o;
}

ext_status check_so3_args(int nz, int ny, int nx, int L, int n_r, double dr, int R) {
  if (nz <= 0 || ny <= 0 || nx <= 0) return fail(EXT_ERR_INVALID_ARG, "empty volume");
  if (!fft_size_supported(nz) || !fft_size_supported(ny) || !fft_size_supported(nx))
    return fail(EXT_ERR_UNSUPPORTED, "volume side is not a supported FFT length");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "SO(3) path supports degrees L <= 6");
  if (n_r < 2 || !(dr > 0) || R < 0 || R > 64) return fail(EXT_ERR_INVALID_ARG, "bad radial table or box");
  return EXT_OK;
}

// Component spectra FFT(f_l^a Y_l^b) / P of every unique (l, a, b) in the
// column-tiled layout of the z pass (conj_out: their conjugates, as the
// correlation uses them), cached per filter, volume shape and kind.  dcomp,
// dtab: device copies of the layout and of the host `tables`.
ext_status so3_spectra(ext_plan plan, int ncomp, const int4* dcomp, const double* tables, const double2* dtab, int L,
                       int n_r, double dr, int R, int nz, int ny, int nx, int conj_out, cudaStream_t st,
                       const float2** out) {
  const size_t P = (size_t)nz * ny * nx;
  const int w2 = ny * nx;   // z-pass: a 2D array of nz rows and ny*nx columns
  const size_t tab_bytes = sizeof(double2) * (size_t)(L + 1) * (L + 1) * n_r;
  const float2 *tw_x, *tw_y, *tw_z;
  EXT_TRY(twiddle(plan, nx, st, &tw_x));
  EXT_TRY(twiddle(plan, ny, st, &tw_y));
  EXT_TRY(twiddle(plan, nz, st, &tw_z));
  uint64_t key = conj_out ? 0x503503503ull : 0x503c0503c0ull;
  key = fnv1a(key, tables, tab_bytes);
  int meta[5] = {L, n_r, R, nz, ny};
  key = fnv1a(key, meta, sizeof(meta));
  key = fnv1a(key, &dr, sizeof(dr));
  key = fnv1a(key, &nx, sizeof(nx));
  const int cw = fft_col_tile(nz);
  const size_t per_k = (size_t)((w2 + cw - 1) / cw) * nz * cw;
  const float scale = 1.0f / (float)P;
  auto build = [&](float2* Sdst) -> ext_status {
    int chunk = (int)((1024ull << 20) / (sizeof(float2) * P));
    chunk = std::max(1, std::min(chunk, ncomp));
    void* grid;
    EXT_TRY(ensure(plan, "grid", sizeof(float2) * P * chunk, &grid));
    for (int k0 = 0; k0 < ncomp; k0 += chunk) {
      const int nk = std::min(chunk, ncomp - k0);
      EXT_CUDA(cudaMemsetAsync(grid, 0, sizeof(float2) * P * nk, st));
      launch_so3_component_grid(dcomp, k0, nk, dtab, n_r, dr, L, R, nz, ny, nx, (float2*)grid, st);
      fft_rows_c2c(nx, (const float2*)grid, nz * ny, nk, (float2*)grid, false, tw_x, st);
      fft_cols_c2c(ny, (float2*)grid, nx, nz * nk, false, tw_y, st);
      fft_cols_fwd_spectrum(nz, (const float2*)grid, w2, conj_out, scale, Sdst + per_k * k0, tw_z, st, nk, scale);
    }
    EXT_CUDA(cudaGetLastError());
    return EXT_OK;
  };
  for (auto& e : plan->specs)
    if (e.key == key) {
      e.stamp = ++plan->clock;
      *out = e.S;
      return EXT_OK;
    }
  if (plan->specs.size() >= plan->max_specs) {
    size_t oldest = 0;
    for (size_t i = 1; i < plan->specs.size(); ++i)
      if (plan->specs[i].stamp < plan->specs[oldest].stamp) oldest = i;
    EXT_CUDA(cudaStreamSynchronize(st));
    EXT_CUDA(cudaFree(plan->specs[oldest].S));
    plan->specs.erase(plan->specs.begin() + oldest);
  }
  SpecEntry e;
  e.key = key;
  e.bytes = sizeof(float2) * per_k * ncomp;
  EXT_TRY(plan_malloc(plan, (void**)&e.S, e.bytes));
  ext_status bs = build(e.S);
  if (bs != EXT_OK) {
    cudaFree(e.S);
    return bs;
  }
  e.stamp = ++plan->clock;
  plan->specs.push_back(e);
  *out = e.S;
  return EXT_OK;
}

// Device copies of the layout (components, channels) and of the radial tables.
ext_status so3_upload(ext_plan plan, const So3Layout& lay, const double* tables, int L, int n_r, cudaStream_t st,
                      const int4** dcomp, const int2** dchan, const double2** dtab) {
  const int ncomp = (int)lay.comp.size();
  void *c, *h, *t;
  EXT_TRY(ensure(plan, "so3_comp", sizeof(int4) * ncomp, &c));
  EXT_TRY(ensure(plan, "so3_chan", sizeof(int2) * ncomp, &h));
  const size_t tab_bytes = sizeof(double2) * (size_t)(L + 1) * (L + 1) * n_r;
  EXT_TRY(ensure(plan, "so3_tab", tab_bytes, &t));
  EXT_CUDA(cudaMemcpyAsync(c, lay.comp.data(), sizeof(int4) * ncomp, cudaMemcpyHostToDevice, st));
  EXT_CUDA(cudaMemcpyAsync(h, lay.chan.data(), sizeof(int2) * ncomp, cudaMemcpyHostToDevice, st));
  EXT_CUDA(cudaMemcpyAsync(t, tables, tab_bytes, cudaMemcpyHostToDevice, st));
  *dcomp = (const int4*)c;
  *dchan = (const int2*)h;
  *dtab = (const double2*)t;
  return EXT_OK;
}

// G (nchan planes of nz*ny*nx floats) for volume V (device).
ext_status so3_components(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L, int n_r,
                          double dr, int R, float* G, cudaStream_t st) {
  const So3Layout lay = so3_layout(L);
  const int ncomp = (int)lay.comp.size();
  const size_t P = (size_t)nz * ny * nx;
  const int w2 = ny * nx;
  const int4* dcomp;
  const int2* dchan;
  const double2* dtab;
  EXT_TRY(so3_upload(plan, lay, tables, L, n_r, st, &dcomp, &dchan, &dtab));
  const float2 *tw_x, *tw_y, *tw_z;
  EXT_TRY(twiddle(plan, nx, st, &tw_x));
  EXT_TRY(twiddle(plan, ny, st, &tw_y));
  EXT_TRY(twiddle(plan, nz, st, &tw_z));
  const float2* S = nullptr;
  EXT_TRY(so3_spectra(plan, ncomp, dcomp, tables, dtab, L, n_r, dr, R, nz, ny, nx, 1, st, &S));
  // forward transform of the volume (full complex spectrum)
  void* Hf;
  EXT_TRY(ensure(plan, "so3_H", sizeof(float2) * P, &Hf));
  launch(plan, "so3_forward", st, [&] {
    launch_real_to_complex(V, (long long)P, (float2*)Hf, plan->sms, st);
    fft_rows_c2c(nx, (const float2*)Hf, nz * ny, 1, (float2*)Hf, false, tw_x, st);
    fft_cols_c2c(ny, (float2*)Hf, nx, nz, false, tw_y, st);
    fft_cols_c2c(nz, (float2*)Hf, w2, 1, false, tw_z, st);
  });
  // inverse passes, components in chunks
  int chunk = (int)((2048ull << 20) / (sizeof(float2) * P));
  chunk = std::max(1, std::min(chunk, ncomp));
  void* Z;
  EXT_TRY(ensure(plan, "Z", sizeof(float2) * P * chunk, &Z));
  for (int k0 = 0; k0 < ncomp; k0 += chunk) {
    const int nk = std::min(chunk, ncomp - k0);
    bool ok = false;
    launch(plan, "so3_cols_z_prod", st, [&] {
      ok = fft_cols_inv_full_pipe(nz, (const float2*)Hf, w2, S, k0, nk, (float2*)Z, tw_z, plan->sms, st);
    });
    if (!ok) return fail(EXT_ERR_UNSUPPORTED, "no pipelined z pass for this volume depth");
    bool fused = false;
    if (ny == nx && plan->pipelined)
      launch(plan, "so3_planes_yx", st, [&] {
        fused = fft_planes_inv_channels(nx, (const float2*)Z, nz, k0, nk, (const int2*)dchan, G, tw_x, plan->dev_err,
                                        plan->sms, st);
      });
    if (!fused) {
      launch(plan, "so3_cols_y", st, [&] { fft_cols_c2c(ny, (float2*)Z, nx, nz * nk, true, tw_y, st); });
      launch(plan, "so3_rows_x", st, [&] {
        fft_rows_inv_channels(nx, (const float2*)Z, nz * ny, k0, nk, (const int2*)dchan, G, tw_x, st);
      });
    }
  }
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

// Steering table B[j][c] (FP32, rows padded to cpad) of a rotation set, and
// for the tensor-core sweep its split-BF16 blocks; cached for the last set.
ext_status so3_tables(ext_plan plan, const double* quats, int n_rot, int L, cudaStream_t st, const float** B,
                      const unsigned char** Bt, int* cpad_out, int* nchan_out, const unsigned char** Bws = nullptr) {
  const So3Layout lay = so3_layout(L);
  const int nchan = lay.nchan;
  const int cpad = (nchan + 31) / 32 * 32;
  uint64_t key = fnv1a(0x7ab1e5ull, quats, sizeof(double) * 4 * n_rot);
  key = fnv1a(key, &L, sizeof(int));
  void *dq, *dB, *dBt, *dch;
  EXT_TRY(ensure(plan, "so3_quats", sizeof(double) * 4 * n_rot, &dq));
  EXT_TRY(ensure(plan, "so3_B", sizeof(float) * (size_t)n_rot * cpad, &dB));
  EXT_TRY(ensure(plan, "so3_Bt", so3_btc_bytes(n_rot, cpad), &dBt));
  EXT_TRY(ensure(plan, "so3_chans", sizeof(int4) * lay.comp.size(), &dch));
  void* dBw = nullptr;
  EXT_TRY(ensure(plan, "so3_Bws", so3_ws_b_bytes(n_rot, cpad), &dBw));
  for (void* q : {dq, dB, dBt, dBw}) key = fnv1a(key, &q, sizeof(q));
  if (plan->so3_rot_key != key) {
    EXT_CUDA(cudaMemcpyAsync(dq, quats, sizeof(double) * 4 * n_rot, cudaMemcpyHostToDevice, st));
    EXT_CUDA(cudaMemcpyAsync(dch, lay.comp.data(), sizeof(int4) * lay.comp.size(), cudaMemcpyHostToDevice, st));
    launch_so3_wigner((const double*)dq, n_rot, L, nullptr, (const int4*)dch, (int)lay.comp.size(), cpad, (float*)dB, st);
    so3_build_btc((const float*)dB, cpad, n_rot, (unsigned char*)dBt, st);
    so3_ws_build_b((const float*)dB, cpad, n_rot, (unsigned char*)dBw, st);
    EXT_CUDA(cudaGetLastError());
    EXT_CUDA(cudaStreamSynchronize(st));   // the host quaternions may change after return
    plan->so3_rot_key = key;
  }
  *B = (const float*)dB;
  *Bt = (const unsigned char*)dBt;
  if (Bws) *Bws = (const unsigned char*)dBw;
  *cpad_out = cpad;
  *nchan_out = nchan;
  return EXT_OK;
}

ext_status so3_sweep(ext_plan plan, const float* G, long long P, int L, const double* quats, int n_rot, float* maxv,
                     int32_t* argmax, int precision, cudaStream_t st) {
  const float* B;
  const unsigned char *Bt, *Bws;
  int cpad, nchan;
  EXT_TRY(so3_tables(plan, quats, n_rot, L, st, &B, &Bt, &cpad, &nchan, &Bws));
  // many voxel tiles: the warp-specialised sweep over pre-split operands, one block per SM
  if (precision == EXT_PREC_BF16X3 && plan->so3_ws && P >= 128LL * plan->sms) {
    void* Ab = nullptr;
    EXT_TRY(ensure(plan, "so3_Aws", so3_ws_a_bytes(P, cpad), &Ab));
    bool ok = false;
    launch(plan, "so3_split_a", st,
           [&] { so3_ws_split_a(G, P, nchan, cpad, (unsigned char*)Ab, plan->sms, st); });
    launch(plan, "so3_sweep_ws", st, [&] {
      ok = sweep_so3_ws(P, cpad, (const unsigned char*)Ab, Bws, n_rot, maxv, argmax, plan->dev_err, plan->sms, st);
    });
    if (ok) {
      EXT_CUDA(cudaGetLastError());
      return EXT_OK;
    }
  }
  if (precision == EXT_PREC_BF16X3) {
    void* keys = nullptr;
    if (sweep_so3_tc_split(P, n_rot, plan->sms) > 1)
      EXT_TRY(ensure(plan, "so3_keys", sizeof(unsigned long long) * P, &keys));
    launch(plan, "so3_sweep_bf16x3", st, [&] {
      sweep_so3_tc(G, P, nchan, cpad, Bt, n_rot, maxv, argmax, (unsigned long long*)keys, plan->dev_err, plan->sms,
                   st);
    });
  }
  else
    launch(plan, "so3_sweep_fp32", st, [&] { sweep_so3_fp32(G, P, nchan, B, cpad, n_rot, maxv, argmax, st); });
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

// The grid R_d R_z(2 pi t / n_psi): full quaternion list (for the FP32 sweep)
// q_d q_z(psi_t), and the split B' blocks of the 16 in-plane-harmonic rows of
// every direction (cached for the last direction set).
void grid_quats(const double* dirs, int n_dirs, int n_psi, std::vector<double>* out) {
  out->resize((size_t)4 * n_dirs * n_psi);
  for (int d = 0; d < n_dirs; ++d)
    for (int t = 0; t < n_psi; ++t) {
      const double h = 3.141592653589793238462643383279502884 * t / n_psi;   // half angle
      const double w1 = dirs[4 * d], x1 = dirs[4 * d + 1], y1 = dirs[4 * d + 2], z1 = dirs[4 * d + 3];
      const double w2 = std::cos(h), z2 = std::sin(h);
      double* q = out->data() + (size_t)4 * (d * n_psi + t);
      q[0] = w1 * w2 - z1 * z2;
      q[1] = x1 * w2 + y1 * z2;
      q[2] = y1 * w2 - x1 * z2;
      q[3] = w1 * z2 + z1 * w2;
    }
}

ext_status so3_grid_tables(ext_plan plan, const double* dirs, int n_dirs, int L, cudaStream_t st,
                           const unsigned char** Bb, int* cpad_out) {
  const So3Layout lay = so3_layout(L);
  const int cpad = (lay.nchan + 31) / 32 * 32;
  const size_t per = (size_t)(L + 1) * (2 * L + 1) * (2 * L + 3) / 3;
  uint64_t key = fnv1a(0x9a1d5ull, dirs, sizeof(double) * 4 * n_dirs);
  key = fnv1a(key, &L, sizeof(int));
  void *dq, *dC, *dB, *dBb, *dch;
  EXT_TRY(ensure(plan, "grid_quats", sizeof(double) * 4 * n_dirs, &dq));
  EXT_TRY(ensure(plan, "grid_C", sizeof(double2) * per * n_dirs, &dC));
  EXT_TRY(ensure(plan, "grid_rows", sizeof(float) * (size_t)16 * n_dirs * cpad, &dB));
  EXT_TRY(ensure(plan, "grid_Bws", so3_ws_b_bytes(16 * n_dirs, cpad), &dBb));
  EXT_TRY(ensure(plan, "grid_chans", sizeof(int4) * lay.comp.size(), &dch));
  for (void* q : {dq, dC, dB, dBb, dch}) key = fnv1a(key, &q, sizeof(q));
  if (plan->so3_grid_key != key) {
    EXT_CUDA(cudaMemcpyAsync(dq, dirs, sizeof(double) * 4 * n_dirs, cudaMemcpyHostToDevice, st));
    EXT_CUDA(cudaMemcpyAsync(dch, lay.comp.data(), sizeof(int4) * lay.comp.size(), cudaMemcpyHostToDevice, st));
    launch_so3_wigner((const double*)dq, n_dirs, L, (double2*)dC, nullptr, 0, 0, nullptr, st);
    launch_so3_grid_rows((const double2*)dC, n_dirs, L, (const int4*)dch, (int)lay.comp.size(), cpad, (float*)dB, st);
    so3_ws_build_b((const float*)dB, cpad, 16 * n_dirs, (unsigned char*)dBb, st);
    EXT_CUDA(cudaGetLastError());
    EXT_CUDA(cudaStreamSynchronize(st));   // the host directions may change after return
    plan->so3_grid_key = key;
  }
  *Bb = (const unsigned char*)dBb;
  *cpad_out = cpad;
  return EXT_OK;
}

ext_status so3_sweep_grid(ext_plan plan, const float* G, long long P, int L, const double* dirs, int n_dirs, int n_psi,
                          float* maxv, int32_t* argmax, int precision, cudaStream_t st) {
  if (precision == EXT_PREC_BF16X3) {
    const unsigned char* Bb;
    int cpad;
    EXT_TRY(so3_grid_tables(plan, dirs, n_dirs, L, st, &Bb, &cpad));
    void* Ab = nullptr;
    EXT_TRY(ensure(plan, "so3_Aws", so3_ws_a_bytes(P, cpad), &Ab));
    void* keys = nullptr;
    EXT_TRY(ensure(plan, "so3_keys", sizeof(unsigned long long) * P, &keys));
    const int nchan = so3_layout(L).nchan;
    bool ok = false;
    launch(plan, "so3_split_a", st, [&] { so3_ws_split_a(G, P, nchan, cpad, (unsigned char*)Ab, plan->sms, st); });
    launch(plan, "so3_sweep_grid", st, [&] {
      ok = sweep_so3_ws_grid(P, cpad, (const unsigned char*)Ab, Bb, n_dirs, n_psi, maxv, argmax,
                             (unsigned long long*)keys, plan->dev_err, plan->sms, st);
    });
    if (!ok) return fail(EXT_ERR_UNSUPPORTED, "grid sweep: unsupported shape");
    EXT_CUDA(cudaGetLastError());
    return EXT_OK;
  }
  std::vector<double> q;
  grid_quats(dirs, n_dirs, n_psi, &q);
  return so3_sweep(plan, G, P, L, q.data(), n_dirs * n_psi, maxv, argmax, precision, st);
}

ext_status check_grid_args(const double* dirs, int n_dirs, int n_psi) {
  if (!dirs || n_dirs < 1 || n_psi < 1) return fail(EXT_ERR_INVALID_ARG, "need directions and n_psi >= 1");
  if (n_psi > 64) return fail(EXT_ERR_UNSUPPORTED, "n_psi must be <= 64");
  if ((long long)n_dirs * n_psi > (1LL << 30)) return fail(EXT_ERR_UNSUPPORTED, "too many grid rotations");
  return EXT_OK;
}

}  // namespace

extern "C" {

ext_status ext_sweep_so3_grid(ext_plan plan, const float* G, int64_t n_vox, int L, const double* dir_quats,
                              int n_dirs, int n_psi, float* max_out, int32_t* argmax, int precision, void* stream) {
  if (!plan || !G || !max_out || !argmax || n_vox < 0) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  EXT_TRY(check_grid_args(dir_quats, n_dirs, n_psi));
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3) return fail(EXT_ERR_INVALID_ARG, "precision");
  if (n_vox == 0) return EXT_OK;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  Staged sG, sM, sA;
  EXT_TRY(stage_in(plan, "in_G", G, sizeof(float) * n_vox * so3_layout(L).nchan, st, &sG));
  EXT_TRY(stage_out_alloc(plan, "out_max", max_out, sizeof(float) * n_vox, &sM));
  EXT_TRY(stage_out_alloc(plan, "out_arg", argmax, sizeof(int32_t) * n_vox, &sA));
  EXT_TRY(so3_sweep_grid(plan, (const float*)sG.dev, n_vox, L, dir_quats, n_dirs, n_psi, (float*)sM.dev,
                         (int32_t*)sA.dev, precision, st));
  EXT_TRY(stage_out_finish(sM, st));
  EXT_TRY(stage_out_finish(sA, st));
  return finish_host(plan, sG.host || sM.host || sA.host, st);
}

ext_status ext_corr_so3_grid(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L,
                             int n_r, double dr, int R, const double* dir_quats, int n_dirs, int n_psi,
                             float* max_out, int32_t* argmax, int precision, void* stream) {
  if (!plan || !V || !tables || !max_out || !argmax) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_TRY(check_so3_args(nz, ny, nx, L, n_r, dr, R));
  EXT_TRY(check_grid_args(dir_quats, n_dirs, n_psi));
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3) return fail(EXT_ERR_INVALID_ARG, "precision");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)nz * ny * nx;
  Staged sV, sM, sA;
  EXT_TRY(stage_in(plan, "in_V", V, sizeof(float) * P, st, &sV));
  EXT_TRY(stage_out_alloc(plan, "out_max", max_out, sizeof(float) * P, &sM));
  EXT_TRY(stage_out_alloc(plan, "out_arg", argmax, sizeof(int32_t) * P, &sA));
  void* G;
  EXT_TRY(ensure(plan, "so3_G", sizeof(float) * P * so3_layout(L).nchan, &G));
  EXT_TRY(so3_components(plan, (const float*)sV.dev, nz, ny, nx, tables, L, n_r, dr, R, (float*)G, st));
  EXT_TRY(so3_sweep_grid(plan, (const float*)G, (long long)P, L, dir_quats, n_dirs, n_psi, (float*)sM.dev,
                         (int32_t*)sA.dev, precision, st));
  EXT_TRY(stage_out_finish(sM, st));
  EXT_TRY(stage_out_finish(sA, st));
  return finish_host(plan, sV.host || sM.host || sA.host, st);
}

int ext_so3_channels(int L) { return (L < 0 || L > 6) ? -1 : so3_layout(L).nchan; }

ext_status ext_so3_wigner(ext_plan plan, const double* quats, int n_rot, int L, double* out) {
  if (!plan || !quats || !out || n_rot < 1) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  EXT_CUDA(cudaSetDevice(plan->device));
  const size_t per = (size_t)(L + 1) * (2 * L + 1) * (2 * L + 3) / 3;
  void *dq, *dC;
  EXT_TRY(ensure(plan, "wig_q", sizeof(double) * 4 * n_rot, &dq));
  EXT_TRY(ensure(plan, "wig_C", sizeof(double2) * per * n_rot, &dC));
  EXT_CUDA(cudaMemcpy(dq, quats, sizeof(double) * 4 * n_rot, cudaMemcpyHostToDevice));
  launch_so3_wigner((const double*)dq, n_rot, L, (double2*)dC, nullptr, 0, 0, nullptr, 0);
  EXT_CUDA(cudaGetLastError());
  EXT_CUDA(cudaMemcpy(out, dC, sizeof(double2) * per * n_rot, cudaMemcpyDeviceToHost));
  return EXT_OK;
}

ext_status ext_corr_so3_components(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L,
                                   int n_r, double dr, int R, float* G, void* stream) {
  if (!plan || !V || !tables || !G) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_TRY(check_so3_args(nz, ny, nx, L, n_r, dr, R));
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)nz * ny * nx;
  Staged sV, sG;
  EXT_TRY(stage_in(plan, "in_V", V, sizeof(float) * P, st, &sV));
  EXT_TRY(stage_out_alloc(plan, "out_G", G, sizeof(float) * P * so3_layout(L).nchan, &sG));
  EXT_TRY(so3_components(plan, (const float*)sV.dev, nz, ny, nx, tables, L, n_r, dr, R, (float*)sG.dev, st));
  EXT_TRY(stage_out_finish(sG, st));
  return finish_host(plan, sV.host || sG.host, st);
}

ext_status ext_sweep_so3(ext_plan plan, const float* G, int64_t n_vox, int L, const double* quats, int n_rot,
                         float* max_out, int32_t* argmax, int precision, void* stream) {
  if (!plan || !G || !quats || !max_out || !argmax || n_vox < 0 || n_rot < 1)
    return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3) return fail(EXT_ERR_INVALID_ARG, "precision");
  if (n_vox == 0) return EXT_OK;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  Staged sG, sM, sA;
  EXT_TRY(stage_in(plan, "in_G", G, sizeof(float) * n_vox * so3_layout(L).nchan, st, &sG));
  EXT_TRY(stage_out_alloc(plan, "out_max", max_out, sizeof(float) * n_vox, &sM));
  EXT_TRY(stage_out_alloc(plan, "out_arg", argmax, sizeof(int32_t) * n_vox, &sA));
  EXT_TRY(so3_sweep(plan, (const float*)sG.dev, n_vox, L, quats, n_rot, (float*)sM.dev, (int32_t*)sA.dev, precision,
                    st));
  EXT_TRY(stage_out_finish(sM, st));
  EXT_TRY(stage_out_finish(sA, st));
  return finish_host(plan, sG.host || sM.host || sA.host, st);
}

ext_status ext_corr_so3(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L, int n_r,
                        double dr, int R, const double* quats, int n_rot, float* max_out, int32_t* argmax,
                        int precision, void* stream) {
  if (!plan || !V || !tables || !quats || !max_out || !argmax || n_rot < 1)
    return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_TRY(check_so3_args(nz, ny, nx, L, n_r, dr, R));
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3) return fail(EXT_ERR_INVALID_ARG, "precision");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)nz * ny * nx;
  Staged sV, sM, sA;
  EXT_TRY(stage_in(plan, "in_V", V, sizeof(float) * P, st, &sV));
  EXT_TRY(stage_out_alloc(plan, "out_max", max_out, sizeof(float) * P, &sM));
  EXT_TRY(stage_out_alloc(plan, "out_arg", argmax, sizeof(int32_t) * P, &sA));
  void* G;
  EXT_TRY(ensure(plan, "so3_G", sizeof(float) * P * so3_layout(L).nchan, &G));
  EXT_TRY(so3_components(plan, (const float*)sV.dev, nz, ny, nx, tables, L, n_r, dr, R, (float*)G, st));
  EXT_TRY(so3_sweep(plan, (const float*)G, (long long)P, L, quats, n_rot, (float*)sM.dev, (int32_t*)sA.dev, precision,
                    st));
  EXT_TRY(stage_out_finish(sM, st));
  EXT_TRY(stage_out_finish(sA, st));
  return finish_host(plan, sV.host || sM.host || sA.host, st);
}

}  // extern "C"

// ---------------------------------------------------------- learned proposal ---
struct ext_mlp_s {
  ext_plan plan = nullptr;
  int device = 0;
  int n_in = 0, dp = 0, H = 0;
  size_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, n_par = 0;
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // FP32 master, Adam moments, gradients
  __nv_bfloat16* w16 = nullptr;                                    // BF16 copy used by the GEMMs
  int step = 0;
  std::map<std::string, DevBuf> ws;
};

namespace {

double factd(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Unique entries of the rotation matrices in the channel layout, with the
// coefficients of Wigner's sum formula for d^l_ba (FP64, stored as FP32).
void build_steer(int L, So3Steer* t) {
  std::memset(t, 0, sizeof(So3Steer));
  const So3Layout lay = so3_layout(L);
  t->n = (int)lay.comp.size();
  for (int e = 0; e < t->n; ++e) {
    const int4 c = lay.comp[e];
    const int l = c.x, m = c.y, mp = c.z;   // C^l_ab uses d^l_{m' m} with m' = b, m = a
    const int smin = std::max(0, m - mp), smax = std::min(l + m, l - mp), ns = smax - smin + 1;
    const double pre = std::sqrt(factd(l + mp) * factd(l - mp) * factd(l + m) * factd(l - m));
    for (int j = 0; j < ns; ++j) {
      const int s = smin + j;
      const double sg = ((mp - m + s) % 2) ? -1.0 : 1.0;
      t->coef[j][e] = (float)(sg * pre / (factd(l + m - s) * factd(s) * factd(mp - m + s) * factd(l - mp - s)));
    }
    const uint32_t self = (m == 0 && mp == 0) ? 1u : 0u;
    const uint32_t pc0 = (uint32_t)(2 * l + m - mp - 2 * smin), ps0 = (uint32_t)(mp - m + 2 * smin);
    t->meta[e] = (uint32_t)c.w | self << 10 | (uint32_t)(m + mp + 12) << 11 | (uint32_t)(mp - m + 12) << 16 |
                 (uint32_t)ns << 21 | pc0 << 24 | ps0 << 28;
    t->l[e] = (unsigned char)l;
  }
}

ext_status steer_table(ext_plan plan, int L, cudaStream_t st, const So3Steer** out) {
  void* d = nullptr;
  EXT_TRY(ensure(plan, "so3_steer", sizeof(So3Steer), &d));
  if (plan->so3_steer_L != L) {
    So3Steer h;
    build_steer(L, &h);
    EXT_CUDA(cudaMemcpyAsync(d, &h, sizeof(So3Steer), cudaMemcpyHostToDevice, st));
    EXT_CUDA(cudaStreamSynchronize(st));
    plan->so3_steer_L = L;
  }
  *out = (const So3Steer*)d;
  return EXT_OK;
}

ext_status pinned_counts(ext_plan plan, int** out) {
  if (!plan->pinned) EXT_CUDA(cudaMallocHost(&plan->pinned, 64));
  *out = plan->pinned;
  return EXT_OK;
}

// device int -> host, synchronising the stream
ext_status read_count(ext_plan plan, const int* dcount, cudaStream_t st, int* out) {
  int* h = nullptr;
  EXT_TRY(pinned_counts(plan, &h));
  EXT_CUDA(cudaMemcpyAsync(h, dcount, sizeof(int), cudaMemcpyDeviceToHost, st));
  EXT_CUDA(cudaStreamSynchronize(st));
  EXT_TRY(device_status(plan));
  *out = *h;
  return EXT_OK;
}

// fails with EXT_ERR_INVALID_ARG if some idx is outside [0, upper)
ext_status check_indices(ext_plan plan, const int32_t* idx, long long n, long long upper, cudaStream_t st) {
  void* bad = nullptr;
  EXT_TRY(ensure(plan, "idx_bad", sizeof(int), &bad));
  EXT_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  launch(plan, "check_index", st, [&] { launch_check_index(idx, n, upper, (int*)bad, st); });
  int b = 0;
  EXT_TRY(read_count(plan, (const int*)bad, st, &b));
  if (b) return fail(EXT_ERR_INVALID_ARG, "an index is out of range");
  return EXT_OK;
}

ext_status mlp_buf(ext_mlp net, const char* name, size_t bytes, void** out) {
  DevBuf& b = net->ws[name];
  if (b.bytes < bytes) {
    if (b.p) EXT_CUDA(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
    EXT_CUDA(cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
  }
  *out = b.p;
  return EXT_OK;
}

template <class T>
ext_status mlp_get(ext_mlp net, const char* name, size_t count, T** out) {
  void* p = nullptr;
  EXT_TRY(mlp_buf(net, name, sizeof(T) * (count ? count : 1), &p));
  *out = (T*)p;
  return EXT_OK;
}

// Forward pass of n rows already in "x16" [n][dp]; logits o [n][16] in "o".
ext_status mlp_forward_x16(ext_mlp net, int n, cudaStream_t st, float** o_out) {
  ext_plan plan = net->plan;
  const int H = net->H, dp = net->dp;
  __nv_bfloat16 *x16, *h1, *h2;
  float* o;
  EXT_TRY(mlp_get(net, "x16", (size_t)n * dp, &x16));
  EXT_TRY(mlp_get(net, "h1", (size_t)n * H, &h1));
  EXT_TRY(mlp_get(net, "h2", (size_t)n * H, &h2));
  EXT_TRY(mlp_get(net, "o", (size_t)n * 16, &o));
  GemmEpilogue e1;
  e1.bias = net->w + net->ob1;
  e1.relu = 1;
  e1.out_bf16 = h1;
  e1.ldo16 = H;
  launch(plan, "mlp_gemm", st, [&] { gemm_bf16(x16, dp, net->w16 + net->oW1, dp, n, H, dp, e1, plan->dev_err, st); });
  GemmEpilogue e2 = e1;
  e2.bias = net->w + net->ob2;
  e2.out_bf16 = h2;
  launch(plan, "mlp_gemm", st, [&] { gemm_bf16(h1, H, net->w16 + net->oW2, H, n, H, H, e2, plan->dev_err, st); });
  GemmEpilogue e3;
  e3.bias = net->w + net->ob3;
  e3.out_f32 = o;
  e3.ldo = 16;
  launch(plan, "mlp_gemm", st, [&] { gemm_bf16(h2, H, net->w16 + net->oW3, H, n, 16, H, e3, plan->dev_err, st); });
  EXT_CUDA(cudaGetLastError());
  *o_out = o;
  return EXT_OK;
}

// Backward pass after mlp_forward_x16 on the same n rows: gradients of the
// mean loss against targets qt [n][4] into net->g, loss added to *loss_dev.
ext_status mlp_backward(ext_mlp net, int n, const float* qt, float* loss_dev, cudaStream_t st) {
  ext_plan plan = net->plan;
  const int H = net->H, dp = net->dp, npad = (n + 63) / 64 * 64;
  __nv_bfloat16 *x16, *h1, *h2, *do16, *doT, *h2T, *W3T, *dz2, *dz2T, *h1T, *W2T, *dz1, *dz1T, *xT;
  float *o, *dof, *dz2f, *dz1f;
  EXT_TRY(mlp_get(net, "x16", (size_t)n * dp, &x16));
  EXT_TRY(mlp_get(net, "h1", (size_t)n * H, &h1));
  EXT_TRY(mlp_get(net, "h2", (size_t)n * H, &h2));
  EXT_TRY(mlp_get(net, "o", (size_t)n * 16, &o));
  EXT_TRY(mlp_get(net, "do16", (size_t)n * 16, &do16));
  EXT_TRY(mlp_get(net, "dof", (size_t)n * 16, &dof));
  EXT_TRY(mlp_get(net, "doT", (size_t)16 * npad, &doT));
  EXT_TRY(mlp_get(net, "h2T", (size_t)H * npad, &h2T));
  EXT_TRY(mlp_get(net, "W3T", (size_t)H * 16, &W3T));
  EXT_TRY(mlp_get(net, "dz2", (size_t)n * H, &dz2));
  EXT_TRY(mlp_get(net, "dz2f", (size_t)n * H, &dz2f));
  EXT_TRY(mlp_get(net, "dz2T", (size_t)H * npad, &dz2T));
  EXT_TRY(mlp_get(net, "h1T", (size_t)H * npad, &h1T));
  EXT_TRY(mlp_get(net, "W2T", (size_t)H * H, &W2T));
  EXT_TRY(mlp_get(net, "dz1", (size_t)n * H, &dz1));
  EXT_TRY(mlp_get(net, "dz1f", (size_t)n * H, &dz1f));
  EXT_TRY(mlp_get(net, "dz1T", (size_t)H * npad, &dz1T));
  EXT_TRY(mlp_get(net, "xT", (size_t)dp * npad, &xT));
  float* g = net->g;
  int* err = plan->dev_err;
  launch(plan, "mlp_loss", st, [&] { launch_quat_loss(o, 16, qt, n, loss_dev, do16, dof, st); });
  // dW3^T = h2^T do (stored transposed), db3 = column sums of do
  launch(plan, "mlp_transpose", st, [&] {
    launch_transpose_bf16(do16, n, 16, 16, doT, 16, npad, npad, st);
    launch_transpose_bf16(h2, n, H, H, h2T, H, npad, npad, st);
    launch_transpose_bf16(net->w16 + net->oW3, 16, H, H, W3T, H, 16, 16, st);
  });
  GemmEpilogue eW3;
  eW3.out_f32 = g + net->oW3;
  eW3.ldo = H;
  eW3.trans = 1;
  launch(plan, "mlp_gemm", st, [&] { gemm_bf16(h2T, npad, doT, npad, H, 16, npad, eW3, err, st); });
  // dz2 = (do W3) * [h2 > 0]
  GemmEpilogue ez2;
  ez2.mask = h2;
  ez2.ldm = H;
  ez2.out_f32 = dz2f;
  ez2.ldo = H;
  ez2.out_bf16 = dz2;
  ez2.ldo16 = H;
  launch(plan, "mlp_gemm", st, [&] { gemm_bf16(do16, 16, W3T, 16, n, H, 16, ez2, err, st); });
  launch(plan, "mlp_transpose", st, [&] {
    launch_transpose_bf16(dz2, n, H, H, dz2T, H, npad, npad, st);
    launch_transpose_bf16(h1, n, H, H, h1T, H, npad, npad, st);
    launch_transpose_bf16(net->w16 + net->oW2, H, H, H, W2T, H, H, H, st);
  });
  GemmEpilogue eW2;
  eW2.out_f32 = g + net->oW2;
  eW2.ldo = H;
  launch(plan, "mlp_gemm", st, [&] { gemm_bf16(dz2T, npad, h1T, npad, H, H, npad, eW2, err, st); });
  // dz1 = (dz2 W2) * [h1 > 0]
  GemmEpilogue ez1 = ez2;
  ez1.mask = h1;
  ez1.out_f32 = dz1f;
  ez1.out_bf16 = dz1;
  launch(plan, "mlp_gemm", st, [&] { gemm_bf16(dz2, H, W2T, H, n, H, H, ez1, err, st); });
  launch(plan, "mlp_transpose", st, [&] {
    launch_transpose_bf16(dz1, n, H, H, dz1T, H, npad, npad, st);
    launch_transpose_bf16(x16, n, dp, dp, xT, dp, npad, npad, st);
  });
  GemmEpilogue eW1;
  eW1.out_f32 = g + net->oW1;
  eW1.ldo = dp;
  launch(plan, "mlp_gemm", st, [&] { gemm_bf16(dz1T, npad, xT, npad, H, dp, npad, eW1, err, st); });
  launch(plan, "mlp_colsum", st, [&] {
    launch_colsum(dof, n, 16, 16, g + net->ob3, st);
    launch_colsum(dz2f, n, H, H, g + net->ob2, st);
    launch_colsum(dz1f, n, H, H, g + net->ob1, st);
  });
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

// SO(3) extended convolution (scatter) of volume V (device) with the rotation
// field Q (device, P quaternions) into out (device):
//   U_e = w_e V C_e(R(.))               (k_so3_modulate, every unique entry e)
//   U^_e over x and y                   (in place: one fused plane pass for square
//                                        slices, else a row and a column pass)
//   Y = IFFT_z sum_e FFT_z(U^_e) S_e    (column pass accumulating the products)
//   out = Re IFFT_yx Y                  (S_e carries the 1 / P of the inverse)
// The entries go in chunks when all of them do not fit the workspace budget,
// their partial Y summed.
ext_status so3_conv(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L, int n_r,
                    double dr, int R, const float* Q, float* out, cudaStream_t st) {
  const So3Layout lay = so3_layout(L);
  const int ncomp = (int)lay.comp.size();
  const long long P = (long long)nz * ny * nx;
  const int w2 = ny * nx;
  const int4* dcomp;
  const int2* dchan;
  const double2* dtab;
  EXT_TRY(so3_upload(plan, lay, tables, L, n_r, st, &dcomp, &dchan, &dtab));
  const float2 *tw_x, *tw_y, *tw_z;
  EXT_TRY(twiddle(plan, nx, st, &tw_x));
  EXT_TRY(twiddle(plan, ny, st, &tw_y));
  EXT_TRY(twiddle(plan, nz, st, &tw_z));
  const float2* S = nullptr;
  EXT_TRY(so3_spectra(plan, ncomp, dcomp, tables, dtab, L, n_r, dr, R, nz, ny, nx, 0, st, &S));
  const int cw = fft_col_tile(nz);
  const size_t per_k = (size_t)((w2 + cw - 1) / cw) * nz * cw;
  int chunk = (int)((4096ull << 20) / (sizeof(float2) * (size_t)P));
  chunk = std::max(1, std::min(chunk, ncomp));
  void *U, *Y, *Yk = nullptr, *dch;
  EXT_TRY(ensure(plan, "so3c_U", sizeof(float2) * P * chunk, &U));
  EXT_TRY(ensure(plan, "so3c_Y", sizeof(float2) * P, &Y));
  if (chunk < ncomp) EXT_TRY(ensure(plan, "so3c_Yk", sizeof(float2) * P, &Yk));
  EXT_TRY(ensure(plan, "so3c_chan", sizeof(int2), &dch));
  const int2 real_only = make_int2(0, -1);
  EXT_CUDA(cudaMemcpyAsync(dch, &real_only, sizeof(int2), cudaMemcpyHostToDevice, st));
  bool gtw = false;
  const int br = plan->tma && fft_cols_conv_tma_ok(nz, &gtw) ? tma_rows(nz, cw) : 0;
  const float2* stw = nullptr;
  if (br > 0 && gtw) EXT_TRY(stage_table(plan, nz, st, &stw));
  for (int e0 = 0; e0 < ncomp; e0 += chunk) {
    const int ne = std::min(chunk, ncomp - e0);
    float2* Ydst = (float2*)(e0 == 0 ? Y : Yk);
    launch(plan, "so3c_modulate", st,
           [&] { launch_so3_modulate(V, Q, P, L, e0, ne, (float2*)U, st); });
    bool planes = false;
    if (ny == nx && plan->pipelined)
      launch(plan, "so3c_planes_yx_fwd", st, [&] {
        planes = fft_planes_fwd_c2c(nx, (float2*)U, ne * nz, tw_x, plan->dev_err, plan->sms, st);
      });
    if (!planes) {
      launch(plan, "so3c_rows_x", st,
             [&] { fft_rows_c2c(nx, (const float2*)U, nz * ny, ne, (float2*)U, false, tw_x, st); });
      launch(plan, "so3c_cols_y", st, [&] { fft_cols_c2c(ny, (float2*)U, nx, nz * ne, false, tw_y, st); });
    }
    CUtensorMap tmU;
    bool done = false;
    if (br > 0 && make_tmap_2d_f32(U, (unsigned long long)2 * w2, (unsigned long long)ne * nz,
                                   (unsigned long long)2 * w2 * sizeof(float), (unsigned)(2 * cw), (unsigned)br, &tmU))
      launch(plan, "so3c_cols_z_conv_tma", st, [&] {
        done = fft_cols_conv_tma(nz, tmU, w2, br, ne - 1, S + per_k * e0, Ydst, tw_z, stw, plan->dev_err, plan->sms,
                                 st);
      });
    if (!done)
      launch(plan, "so3c_cols_z_conv", st,
             [&] { fft_cols_conv(nz, (const float2*)U, w2, ne - 1, S + per_k * e0, Ydst, tw_z, st); });
    if (e0 > 0) launch(plan, "so3c_add", st, [&] { launch_add_complex((float2*)Y, (const float2*)Yk, P, plan->sms, st); });
  }
  bool fused = false;
  if (ny == nx && plan->pipelined)
    launch(plan, "so3c_planes_yx", st, [&] {
      fused = fft_planes_inv_channels(nx, (const float2*)Y, nz, 0, 1, (const int2*)dch, out, tw_x, plan->dev_err,
                                      plan->sms, st);
    });
  if (!fused) {
    launch(plan, "so3c_cols_y_inv", st, [&] { fft_cols_c2c(ny, (float2*)Y, nx, nz, true, tw_y, st); });
    launch(plan, "so3c_rows_x_inv", st, [&] {
      fft_rows_inv_channels(nx, (const float2*)Y, nz * ny, 0, 1, (const int2*)dch, out, tw_x, st);
    });
  }
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

}  // namespace

extern "C" {

ext_status ext_conv_so3(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L, int n_r,
                        double dr, int R, const float* quats, float* out, void* stream) {
  if (!plan || !V || !tables || !quats || !out) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_TRY(check_so3_args(nz, ny, nx, L, n_r, dr, R));
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)nz * ny * nx;
  Staged sV, sQ, sO;
  EXT_TRY(stage_in(plan, "in_V", V, sizeof(float) * P, st, &sV));
  EXT_TRY(stage_in(plan, "in_Q", quats, sizeof(float) * 4 * P, st, &sQ));
  if (reinterpret_cast<uintptr_t>(sQ.dev) % 16 != 0)
    return fail(EXT_ERR_INVALID_ARG, "device quaternion field must be 16-byte aligned");
  EXT_TRY(stage_out_direct(plan, "out_O", out, sizeof(float) * P, &sO));
  EXT_TRY(so3_conv(plan, (const float*)sV.dev, nz, ny, nx, tables, L, n_r, dr, R, (const float*)sQ.dev,
                   (float*)sO.dev, st));
  EXT_TRY(stage_out_finish(sO, st));
  return finish_host(plan, sV.host || sQ.host || sO.host || sO.mapped, st);
}

ext_status ext_mlp_create(ext_plan plan, int n_in, int hidden, ext_mlp* out) {
  if (!plan || !out) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (n_in < 1 || n_in > 4096) return fail(EXT_ERR_INVALID_ARG, "n_in must be in [1, 4096]");
  if (hidden < 16 || hidden > 1024 || hidden % 16) return fail(EXT_ERR_INVALID_ARG, "hidden: multiple of 16 in [16, 1024]");
  EXT_CUDA(cudaSetDevice(plan->device));
  ext_mlp net = new ext_mlp_s();
  net->plan = plan;
  net->device = plan->device;
  net->n_in = n_in;
  net->dp = (n_in + 15) / 16 * 16;
  net->H = hidden;
  const size_t H = hidden, dp = net->dp;
  net->oW1 = 0;
  net->ob1 = net->oW1 + H * dp;
  net->oW2 = net->ob1 + H;
  net->ob2 = net->oW2 + H * H;
  net->oW3 = net->ob2 + H;
  net->ob3 = net->oW3 + 16 * H;
  net->n_par = net->ob3 + 16;
  const size_t bytes = sizeof(float) * net->n_par;
  bool ok = cudaMalloc(&net->w, bytes) == cudaSuccess && cudaMalloc(&net->m, bytes) == cudaSuccess &&
            cudaMalloc(&net->v, bytes) == cudaSuccess && cudaMalloc(&net->g, bytes) == cudaSuccess &&
            cudaMalloc(&net->w16, sizeof(__nv_bfloat16) * net->n_par) == cudaSuccess;
  ok = ok && cudaMemset(net->w, 0, bytes) == cudaSuccess && cudaMemset(net->m, 0, bytes) == cudaSuccess &&
       cudaMemset(net->v, 0, bytes) == cudaSuccess && cudaMemset(net->g, 0, bytes) == cudaSuccess &&
       cudaMemset(net->w16, 0, sizeof(__nv_bfloat16) * net->n_par) == cudaSuccess;
  if (!ok) {
    ext_mlp_destroy(net);
    return fail(EXT_ERR_OOM, "cannot allocate the network");
  }
  *out = net;
  return EXT_OK;
}

ext_status ext_mlp_destroy(ext_mlp net) {
  if (!net) return EXT_OK;
  // uses only the network's own device: its plan may already be gone
  cudaSetDevice(net->device);
  cudaDeviceSynchronize();
  for (void* p : {(void*)net->w, (void*)net->m, (void*)net->v, (void*)net->g, (void*)net->w16})
    if (p) cudaFree(p);
  for (auto& kv : net->ws) cudaFree(kv.second.p);
  delete net;
  cudaGetLastError();   // leave no error of this teardown to a later call
  return EXT_OK;
}

ext_status ext_mlp_set_params(ext_mlp net, const float* W1, const float* b1, const float* W2, const float* b2,
                              const float* W3, const float* b3) {
  if (!net || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_CUDA(cudaSetDevice(net->plan->device));
  const size_t H = net->H, f = sizeof(float), bytes = f * net->n_par;
  EXT_CUDA(cudaDeviceSynchronize());
  EXT_CUDA(cudaMemset(net->w, 0, bytes));
  EXT_CUDA(cudaMemcpy2D(net->w + net->oW1, f * net->dp, W1, f * net->n_in, f * net->n_in, H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(net->w + net->ob1, b1, f * H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(net->w + net->oW2, W2, f * H * H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(net->w + net->ob2, b2, f * H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(net->w + net->oW3, W3, f * 4 * H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(net->w + net->ob3, b3, f * 4, cudaMemcpyDefault));
  EXT_CUDA(cudaMemset(net->m, 0, bytes));
  EXT_CUDA(cudaMemset(net->v, 0, bytes));
  net->step = 0;
  launch(net->plan, "mlp_to_bf16", 0, [&] { launch_f32_to_bf16(net->w, (long long)net->n_par, net->w16, 0); });
  EXT_CUDA(cudaGetLastError());
  EXT_CUDA(cudaDeviceSynchronize());
  return EXT_OK;
}

ext_status ext_mlp_get_params(ext_mlp net, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3) {
  if (!net || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_CUDA(cudaSetDevice(net->plan->device));
  const size_t H = net->H, f = sizeof(float);
  EXT_CUDA(cudaDeviceSynchronize());
  EXT_CUDA(cudaMemcpy2D(W1, f * net->n_in, net->w + net->oW1, f * net->dp, f * net->n_in, H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(b1, net->w + net->ob1, f * H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(W2, net->w + net->oW2, f * H * H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(b2, net->w + net->ob2, f * H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(W3, net->w + net->oW3, f * 4 * H, cudaMemcpyDefault));
  EXT_CUDA(cudaMemcpy(b3, net->w + net->ob3, f * 4, cudaMemcpyDefault));
  return EXT_OK;
}

ext_status ext_mlp_forward(ext_mlp net, const float* X, int n, float* q, void* stream) {
  if (!net || !X || !q || n < 0) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return EXT_OK;
  ext_plan plan = net->plan;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  Staged sX, sQ;
  EXT_TRY(stage_in(plan, "mlp_X", X, sizeof(float) * (size_t)n * net->n_in, st, &sX));
  EXT_TRY(stage_out_alloc(plan, "mlp_q", q, sizeof(float) * 4 * (size_t)n, &sQ));
  __nv_bfloat16* x16;
  EXT_TRY(mlp_get(net, "x16", (size_t)n * net->dp, &x16));
  launch(plan, "mlp_normalize", st,
         [&] { launch_rows_normalize_bf16((const float*)sX.dev, net->n_in, nullptr, n, net->n_in, net->dp, x16, st); });
  float* o = nullptr;
  EXT_TRY(mlp_forward_x16(net, n, st, &o));
  launch(plan, "mlp_quat", st, [&] { launch_normalize_quat(o, 16, n, (float*)sQ.dev, st); });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sQ, st));
  return finish_host(plan, sX.host || sQ.host, st);
}

ext_status ext_mlp_grads(ext_mlp net, const float* X, const float* qt, int n, float* loss, float* grads,
                         void* stream) {
  if (!net || !X || !qt || n < 1) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  ext_plan plan = net->plan;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  Staged sX, sT, sL;
  EXT_TRY(stage_in(plan, "mlp_X", X, sizeof(float) * (size_t)n * net->n_in, st, &sX));
  EXT_TRY(stage_in(plan, "mlp_qt", qt, sizeof(float) * 4 * (size_t)n, st, &sT));
  float* dloss = nullptr;
  EXT_TRY(mlp_get(net, "loss", 1, &dloss));
  EXT_CUDA(cudaMemsetAsync(dloss, 0, sizeof(float), st));
  __nv_bfloat16* x16;
  EXT_TRY(mlp_get(net, "x16", (size_t)n * net->dp, &x16));
  launch(plan, "mlp_normalize", st,
         [&] { launch_rows_normalize_bf16((const float*)sX.dev, net->n_in, nullptr, n, net->n_in, net->dp, x16, st); });
  float* o = nullptr;
  EXT_TRY(mlp_forward_x16(net, n, st, &o));
  EXT_TRY(mlp_backward(net, n, (const float*)sT.dev, dloss, st));
  if (loss) EXT_CUDA(cudaMemcpyAsync(loss, dloss, sizeof(float), cudaMemcpyDefault, st));
  if (grads) {
    const size_t H = net->H, f = sizeof(float), ni = net->n_in;
    float* d = grads;
    EXT_CUDA(cudaMemcpy2DAsync(d, f * ni, net->g + net->oW1, f * net->dp, f * ni, H, cudaMemcpyDefault, st));
    d += H * ni;
    EXT_CUDA(cudaMemcpyAsync(d, net->g + net->ob1, f * H, cudaMemcpyDefault, st));
    d += H;
    EXT_CUDA(cudaMemcpyAsync(d, net->g + net->oW2, f * H * H, cudaMemcpyDefault, st));
    d += H * H;
    EXT_CUDA(cudaMemcpyAsync(d, net->g + net->ob2, f * H, cudaMemcpyDefault, st));
    d += H;
    EXT_CUDA(cudaMemcpyAsync(d, net->g + net->oW3, f * 4 * H, cudaMemcpyDefault, st));
    d += 4 * H;
    EXT_CUDA(cudaMemcpyAsync(d, net->g + net->ob3, f * 4, cudaMemcpyDefault, st));
  }
  (void)sL;
  EXT_CUDA(cudaStreamSynchronize(st));
  return device_status(plan);
}

ext_status ext_mlp_train(ext_mlp net, const float* X, const float* qt, int n_train, int L, const int32_t* rows,
                         const float* Q, int steps, int batch, float lr, float* losses, void* stream) {
  if (!net || !X || !qt || !rows || n_train < 1 || steps < 0 || batch < 1)
    return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (Q && (L < 0 || L > 6 || so3_layout(L).nchan != net->n_in))
    return fail(EXT_ERR_INVALID_ARG, "augmentation needs n_in == ext_so3_channels(L)");
  if (steps == 0) return EXT_OK;
  ext_plan plan = net->plan;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nrows = (size_t)steps * batch;
  Staged sX, sT, sR, sQ, sL;
  EXT_TRY(stage_in(plan, "mlp_X", X, sizeof(float) * (size_t)n_train * net->n_in, st, &sX));
  EXT_TRY(stage_in(plan, "mlp_qt", qt, sizeof(float) * 4 * (size_t)n_train, st, &sT));
  EXT_TRY(stage_in(plan, "mlp_rows", rows, sizeof(int32_t) * nrows, st, &sR));
  if (Q) EXT_TRY(stage_in(plan, "mlp_Q", Q, sizeof(float) * 4 * nrows, st, &sQ));
  EXT_TRY(check_indices(plan, (const int32_t*)sR.dev, (long long)nrows, n_train, st));
  float* dl = nullptr;
  EXT_TRY(mlp_get(net, "losses", (size_t)steps, &dl));
  EXT_CUDA(cudaMemsetAsync(dl, 0, sizeof(float) * steps, st));
  const So3Steer* tab = nullptr;
  if (Q) EXT_TRY(steer_table(plan, L, st, &tab));
  float *xa = nullptr, *qa = nullptr;
  __nv_bfloat16* x16 = nullptr;
  EXT_TRY(mlp_get(net, "train_xa", (size_t)batch * net->n_in, &xa));
  EXT_TRY(mlp_get(net, "train_qa", (size_t)batch * 4, &qa));
  EXT_TRY(mlp_get(net, "x16", (size_t)batch * net->dp, &x16));
  const int32_t* R = (const int32_t*)sR.dev;
  for (int s = 0; s < steps; ++s) {
    const int32_t* r = R + (size_t)s * batch;
    if (Q) {
      const float* Qs = (const float*)sQ.dev + (size_t)s * batch * 4;
      launch(plan, "so3_augment", st, [&] {
        launch_so3_augment((const float*)sX.dev, net->n_in, r, batch, Qs, (const float*)sT.dev, tab, net->n_in, xa,
                           net->n_in, qa, st);
      });
      launch(plan, "mlp_normalize", st,
             [&] { launch_rows_normalize_bf16(xa, net->n_in, nullptr, batch, net->n_in, net->dp, x16, st); });
    } else {
      launch(plan, "mlp_normalize", st, [&] {
        launch_rows_normalize_bf16((const float*)sX.dev, net->n_in, r, batch, net->n_in, net->dp, x16, st);
        launch_gather_quats((const float*)sT.dev, r, batch, qa, st);
      });
    }
    float* o = nullptr;
    EXT_TRY(mlp_forward_x16(net, batch, st, &o));
    EXT_TRY(mlp_backward(net, batch, qa, dl + s, st));
    net->step += 1;
    launch(plan, "mlp_adam", st,
           [&] { launch_adam(net->w, net->m, net->v, net->g, (long long)net->n_par, lr, net->step, net->w16, st); });
  }
  EXT_CUDA(cudaGetLastError());
  if (losses) EXT_CUDA(cudaMemcpyAsync(losses, dl, sizeof(float) * steps, cudaMemcpyDefault, st));
  (void)sL;
  EXT_CUDA(cudaStreamSynchronize(st));
  return device_status(plan);
}

ext_status ext_so3_upper_bound(ext_plan plan, const float* G, int64_t n_vox, int L, float* ub, void* stream) {
  if (!plan || !G || !ub || n_vox < 0) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  if (n_vox == 0) return EXT_OK;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  Staged sG, sU;
  EXT_TRY(stage_in(plan, "in_G", G, sizeof(float) * n_vox * so3_layout(L).nchan, st, &sG));
  EXT_TRY(stage_out_alloc(plan, "out_ub", ub, sizeof(float) * n_vox, &sU));
  const So3Steer* tab = nullptr;
  EXT_TRY(steer_table(plan, L, st, &tab));
  launch(plan, "so3_upper_bound", st,
         [&] { launch_so3_upper_bound((const float*)sG.dev, n_vox, tab, (float*)sU.dev, L, plan->sms, st); });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sU, st));
  return finish_host(plan, sG.host || sU.host, st);
}

ext_status ext_so3_refined_bound(ext_plan plan, const float* X, int n, int L, float* out, void* stream) {
  if (!plan || !X || !out || n < 0) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  if (n == 0) return EXT_OK;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int C = so3_layout(L).nchan;
  Staged sX, sO;
  EXT_TRY(stage_in(plan, "in_X", X, sizeof(float) * (size_t)n * C, st, &sX));
  EXT_TRY(stage_out_alloc(plan, "out_ub", out, sizeof(float) * n, &sO));
  const So3Steer* tab = nullptr;
  EXT_TRY(steer_table(plan, L, st, &tab));
  launch(plan, "so3_refined_bound", st,
         [&] { launch_so3_refined_bound((const float*)sX.dev, C, n, tab, L, (float*)sO.dev, plan->sms, st); });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sO, st));
  return finish_host(plan, sX.host || sO.host, st);
}

ext_status ext_so3_gather(ext_plan plan, const float* G, int64_t n_vox, int L, const int32_t* vox, int n, float* X,
                          void* stream) {
  if (!plan || !G || !vox || !X || n_vox < 1 || n < 0) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  if (n == 0) return EXT_OK;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int C = so3_layout(L).nchan;
  Staged sG, sV, sX;
  EXT_TRY(stage_in(plan, "in_G", G, sizeof(float) * n_vox * C, st, &sG));
  EXT_TRY(stage_in(plan, "in_vox", vox, sizeof(int32_t) * n, st, &sV));
  EXT_TRY(stage_out_alloc(plan, "out_X", X, sizeof(float) * (size_t)n * C, &sX));
  EXT_TRY(check_indices(plan, (const int32_t*)sV.dev, n, n_vox, st));
  launch(plan, "so3_gather_rows", st, [&] {
    launch_gather_rows((const float*)sG.dev, n_vox, C, (const int32_t*)sV.dev, n, (float*)sX.dev, C, st);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sX, st));
  return finish_host(plan, sG.host || sV.host || sX.host, st);
}

ext_status ext_so3_augment(ext_plan plan, const float* X, int n, int L, const float* Q, const float* q_in,
                           float* X_out, float* q_out, void* stream) {
  if (!plan || !X || !Q || !q_in || !X_out || !q_out || n < 0) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  if (n == 0) return EXT_OK;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int C = so3_layout(L).nchan;
  Staged sX, sQ, sq, sXo, sqo;
  EXT_TRY(stage_in(plan, "in_X", X, sizeof(float) * (size_t)n * C, st, &sX));
  EXT_TRY(stage_in(plan, "in_Q", Q, sizeof(float) * 4 * (size_t)n, st, &sQ));
  EXT_TRY(stage_in(plan, "in_q", q_in, sizeof(float) * 4 * (size_t)n, st, &sq));
  EXT_TRY(stage_out_alloc(plan, "out_X", X_out, sizeof(float) * (size_t)n * C, &sXo));
  EXT_TRY(stage_out_alloc(plan, "out_q", q_out, sizeof(float) * 4 * (size_t)n, &sqo));
  const So3Steer* tab = nullptr;
  EXT_TRY(steer_table(plan, L, st, &tab));
  launch(plan, "so3_augment", st, [&] {
    launch_so3_augment((const float*)sX.dev, C, nullptr, n, (const float*)sQ.dev, (const float*)sq.dev, tab, C,
                       (float*)sXo.dev, C, (float*)sqo.dev, st);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sXo, st));
  EXT_TRY(stage_out_finish(sqo, st));
  return finish_host(plan, sX.host || sQ.host || sq.host || sXo.host || sqo.host, st);
}

ext_status ext_so3_refine(ext_plan plan, const float* X, int n, int L, const float* q0, float* q_out, float* s_out,
                          void* stream) {
  if (!plan || !X || !q0 || !q_out || !s_out || n < 0) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  if (n == 0) return EXT_OK;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int C = so3_layout(L).nchan;
  Staged sX, sq, sqo, sso;
  EXT_TRY(stage_in(plan, "in_X", X, sizeof(float) * (size_t)n * C, st, &sX));
  EXT_TRY(stage_in(plan, "in_q", q0, sizeof(float) * 4 * (size_t)n, st, &sq));
  EXT_TRY(stage_out_alloc(plan, "out_q", q_out, sizeof(float) * 4 * (size_t)n, &sqo));
  EXT_TRY(stage_out_alloc(plan, "out_s", s_out, sizeof(float) * (size_t)n, &sso));
  const So3Steer* tab = nullptr;
  EXT_TRY(steer_table(plan, L, st, &tab));
  launch(plan, "so3_refine", st, [&] {
    launch_so3_refine((const float*)sX.dev, C, n, (const float*)sq.dev, tab, 5, 0.25f, 6, (float*)sqo.dev,
                      (float*)sso.dev, plan->sms, st);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sqo, st));
  EXT_TRY(stage_out_finish(sso, st));
  return finish_host(plan, sX.host || sq.host || sqo.host || sso.host, st);
}

}  // extern "C"

namespace {

// Proposal on device channels G (P voxels) into device outputs.
ext_status so3_propose(ext_plan plan, const float* G, long long P, int L, ext_mlp net, const double* quats, int n_rot,
                       float bound, float* score, float* quat, int32_t* grid_idx, int precision, int64_t* counts,
                       cudaStream_t st) {
  const int C = so3_layout(L).nchan;
  const So3Steer* tab = nullptr;
  EXT_TRY(steer_table(plan, L, st, &tab));
  void *ub, *cand1, *cnt, *scratch;
  EXT_TRY(ensure(plan, "prop_ub", sizeof(float) * P, &ub));
  EXT_TRY(ensure(plan, "prop_cand1", sizeof(int32_t) * P, &cand1));
  EXT_TRY(ensure(plan, "prop_cnt", sizeof(int) * 4, &cnt));
  EXT_TRY(ensure(plan, "prop_scratch", compact_scratch_bytes(P), &scratch));
  int* dcnt = (int*)cnt;
  // stage 1: the Frobenius bound over every voxel
  launch(plan, "so3_upper_bound", st, [&] { launch_so3_upper_bound(G, P, tab, (float*)ub, L, plan->sms, st); });
  launch(plan, "compact", st, [&] { compact((const float*)ub, P, bound, 0, (int32_t*)cand1, dcnt, scratch, st); });
  launch(plan, "so3_fill", st, [&] { launch_so3_fill(P, score, quat, grid_idx, st); });
  EXT_CUDA(cudaGetLastError());
  int nc1 = 0, nc = 0, nf = 0;
  EXT_TRY(read_count(plan, dcnt, st, &nc1));
  // stage 2: the refined bound on the survivors
  void *X1 = nullptr, *ub2 = nullptr, *sel = nullptr, *cand = nullptr, *X = nullptr;
  if (nc1 > 0) {
    EXT_TRY(ensure(plan, "prop_X1", sizeof(float) * (size_t)nc1 * C, &X1));
    EXT_TRY(ensure(plan, "prop_ub2", sizeof(float) * nc1, &ub2));
    EXT_TRY(ensure(plan, "prop_sel", sizeof(int32_t) * nc1, &sel));
    EXT_TRY(ensure(plan, "prop_cand", sizeof(int32_t) * nc1, &cand));
    EXT_TRY(ensure(plan, "prop_X", sizeof(float) * (size_t)nc1 * C, &X));
    void* scr = nullptr;
    EXT_TRY(ensure(plan, "prop_scratch2", compact_scratch_bytes(nc1), &scr));
    launch(plan, "so3_gather_rows", st, [&] { launch_gather_rows(G, P, C, (const int32_t*)cand1, nc1, (float*)X1, C, st); });
    launch(plan, "so3_refined_bound", st,
           [&] { launch_so3_refined_bound((const float*)X1, C, nc1, tab, L, (float*)ub2, plan->sms, st); });
    launch(plan, "compact", st, [&] { compact((const float*)ub2, nc1, bound, 0, (int32_t*)sel, dcnt + 1, scr, st); });
    EXT_CUDA(cudaGetLastError());
    EXT_TRY(read_count(plan, dcnt + 1, st, &nc));
    launch(plan, "so3_select", st, [&] {
      launch_gather_int((const int32_t*)cand1, (const int32_t*)sel, nc, (int32_t*)cand, st);
      launch_gather_row_copies((const float*)X1, C, (const int32_t*)sel, nc, (float*)X, st);
    });
  }
  const int32_t* fb = nullptr;
  if (nc > 0 && net) {
    float *q0, *qr, *sr;
    int32_t* fbi;
    EXT_TRY(mlp_get(net, "prop_q0", (size_t)nc * 4, &q0));
    EXT_TRY(mlp_get(net, "prop_qr", (size_t)nc * 4, &qr));
    EXT_TRY(mlp_get(net, "prop_sr", (size_t)nc, &sr));
    EXT_TRY(mlp_get(net, "prop_fb", (size_t)nc, &fbi));
    __nv_bfloat16* x16;
    EXT_TRY(mlp_get(net, "x16", (size_t)nc * net->dp, &x16));
    launch(plan, "mlp_normalize", st,
           [&] { launch_rows_normalize_bf16((const float*)X, C, nullptr, nc, C, net->dp, x16, st); });
    float* o = nullptr;
    EXT_TRY(mlp_forward_x16(net, nc, st, &o));
    launch(plan, "mlp_quat", st, [&] { launch_normalize_quat(o, 16, nc, q0, st); });
    launch(plan, "so3_refine", st, [&] {
      launch_so3_refine((const float*)X, C, nc, q0, tab, 5, 0.25f, 6, qr, sr, plan->sms, st);
    });
    launch(plan, "so3_scatter", st,
           [&] { launch_so3_scatter((const int32_t*)cand, nc, sr, qr, score, quat, grid_idx, st); });
    void* scr3 = nullptr;
    EXT_TRY(ensure(plan, "prop_scratch3", compact_scratch_bytes(nc), &scr3));
    launch(plan, "compact", st, [&] { compact(sr, nc, bound, 1, fbi, dcnt + 2, scr3, st); });
    EXT_CUDA(cudaGetLastError());
    EXT_TRY(read_count(plan, dcnt + 2, st, &nf));
    fb = fbi;
  } else {
    nf = nc;
  }
  if (nf > 0) {
    void *Gf, *mf, *jf;
    EXT_TRY(ensure(plan, "prop_Gf", sizeof(float) * (size_t)nf * C, &Gf));
    EXT_TRY(ensure(plan, "prop_mf", sizeof(float) * nf, &mf));
    EXT_TRY(ensure(plan, "prop_jf", sizeof(int32_t) * nf, &jf));
    launch(plan, "so3_gather_channels", st,
           [&] { launch_gather_channels(G, P, C, (const int32_t*)cand, fb, nf, (float*)Gf, st); });
    EXT_TRY(so3_sweep(plan, (const float*)Gf, nf, L, quats, n_rot, (float*)mf, (int32_t*)jf, precision, st));
    void* dq = nullptr;
    EXT_TRY(ensure(plan, "so3_quats", sizeof(double) * 4 * n_rot, &dq));
    launch(plan, "so3_merge", st, [&] {
      launch_so3_merge((const int32_t*)cand, fb, nf, (const float*)mf, (const int32_t*)jf, (const double*)dq, score,
                       quat, grid_idx, st);
    });
    EXT_CUDA(cudaGetLastError());
  }
  if (counts) {
    counts[0] = nc1;
    counts[1] = nc;
    counts[2] = nf;
  }
  return EXT_OK;
}

}  // namespace

extern "C" {

ext_status ext_so3_propose(ext_plan plan, const float* G, int64_t n_vox, int L, ext_mlp net, const double* quats,
                           int n_rot, float bound, float* score, float* quat, int32_t* grid_idx, int precision,
                           int64_t* counts, void* stream) {
  if (!plan || !G || !quats || !score || n_vox < 0 || n_rot < 1) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  if (L < 0 || L > 6) return fail(EXT_ERR_UNSUPPORTED, "L <= 6");
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3) return fail(EXT_ERR_INVALID_ARG, "precision");
  if (n_vox > INT32_MAX) return fail(EXT_ERR_UNSUPPORTED, "at most 2^31 - 1 voxels");
  if (net && net->n_in != so3_layout(L).nchan) return fail(EXT_ERR_INVALID_ARG, "network n_in != channels of L");
  if (net && net->plan != plan) return fail(EXT_ERR_INVALID_ARG, "network belongs to another plan");
  if (counts) counts[0] = counts[1] = counts[2] = 0;
  if (n_vox == 0) return EXT_OK;
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int C = so3_layout(L).nchan;
  Staged sG, sS, sQ, sI;
  EXT_TRY(stage_in(plan, "in_G", G, sizeof(float) * n_vox * C, st, &sG));
  EXT_TRY(stage_out_alloc(plan, "out_score", score, sizeof(float) * n_vox, &sS));
  EXT_TRY(stage_out_alloc(plan, "out_quat", quat, sizeof(float) * 4 * n_vox, &sQ));
  EXT_TRY(stage_out_alloc(plan, "out_idx", grid_idx, sizeof(int32_t) * n_vox, &sI));
  EXT_TRY(so3_propose(plan, (const float*)sG.dev, n_vox, L, net, quats, n_rot, bound, (float*)sS.dev,
                      (float*)sQ.dev, (int32_t*)sI.dev, precision, counts, st));
  EXT_TRY(stage_out_finish(sS, st));
  if (quat) EXT_TRY(stage_out_finish(sQ, st));
  if (grid_idx) EXT_TRY(stage_out_finish(sI, st));
  return finish_host(plan, sG.host || sS.host || sQ.host || sI.host, st);
}

ext_status ext_corr_so3_propose(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L,
                                int n_r, double dr, int R, ext_mlp net, const double* quats, int n_rot, float bound,
                                float* score, float* quat, int32_t* grid_idx, int precision, int64_t* counts,
                                void* stream) {
  if (!plan || !V || !tables || !quats || !score || n_rot < 1) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_TRY(check_so3_args(nz, ny, nx, L, n_r, dr, R));
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3) return fail(EXT_ERR_INVALID_ARG, "precision");
  if (net && net->n_in != so3_layout(L).nchan) return fail(EXT_ERR_INVALID_ARG, "network n_in != channels of L");
  if (net && net->plan != plan) return fail(EXT_ERR_INVALID_ARG, "network belongs to another plan");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)nz * ny * nx;
  Staged sV, sS, sQ, sI;
  EXT_TRY(stage_in(plan, "in_V", V, sizeof(float) * P, st, &sV));
  EXT_TRY(stage_out_alloc(plan, "out_score", score, sizeof(float) * P, &sS));
  EXT_TRY(stage_out_alloc(plan, "out_quat", quat, sizeof(float) * 4 * P, &sQ));
  EXT_TRY(stage_out_alloc(plan, "out_idx", grid_idx, sizeof(int32_t) * P, &sI));
  void* G;
  EXT_TRY(ensure(plan, "so3_G", sizeof(float) * P * so3_layout(L).nchan, &G));
  EXT_TRY(so3_components(plan, (const float*)sV.dev, nz, ny, nx, tables, L, n_r, dr, R, (float*)G, st));
  EXT_TRY(so3_propose(plan, (const float*)G, (long long)P, L, net, quats, n_rot, bound, (float*)sS.dev,
                      (float*)sQ.dev, (int32_t*)sI.dev, precision, counts, st));
  EXT_TRY(stage_out_finish(sS, st));
  if (quat) EXT_TRY(stage_out_finish(sQ, st));
  if (grid_idx) EXT_TRY(stage_out_finish(sI, st));
  return finish_host(plan, sV.host || sS.host || sQ.host || sI.host, st);
}

}  // extern "C"

// ----------------------------------------------------------- checkpoints ---
// The network's whole training state in one file (layout in extconv.h):
// resuming from it continues Adam exactly where it stopped.
namespace {

// CRC-32 of IEEE 802.3 (reflected polynomial 0xEDB88320, register preset to
// all ones, result complemented), one bit at a time from its definition.
uint32_t crc32_ieee(const unsigned char* p, size_t n) {
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) {
    c ^= p[i];
    for (int b = 0; b < 8; ++b) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
  }
  return ~c;
}

constexpr char CKPT_MAGIC[9] = "EXTMLP01";
constexpr uint32_t CKPT_VERSION = 1;
constexpr size_t CKPT_HEADER = 40;

void put_u32(unsigned char* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
void put_u64(unsigned char* p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
uint32_t get_u32(const unsigned char* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
uint64_t get_u64(const unsigned char* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

uint64_t ckpt_floats(uint64_t n_in, uint64_t hidden) { return hidden * (n_in + hidden + 6) + 4; }

struct CkptInfo {
  int n_in = 0, hidden = 0;
  uint64_t step = 0, n = 0;
};

// Reads and checks a checkpoint file; on success the whole file is in `bytes`.
ext_status ckpt_read(const char* path, std::vector<unsigned char>* bytes, CkptInfo* info) {
  if (!path) return fail(EXT_ERR_INVALID_ARG, "checkpoint path is NULL");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(EXT_ERR_CHECKPOINT, std::string("cannot open checkpoint ") + path);
  std::vector<unsigned char>& b = *bytes;
  b.clear();
  unsigned char buf[1 << 16];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) b.insert(b.end(), buf, buf + got);
  const bool bad = std::ferror(f) != 0;
  std::fclose(f);
  if (bad) return fail(EXT_ERR_CHECKPOINT, "error reading the checkpoint");
  if (b.size() < CKPT_HEADER + 4) return fail(EXT_ERR_CHECKPOINT, "checkpoint truncated (shorter than its header)");
  if (std::memcmp(b.data(), CKPT_MAGIC, 8) != 0) return fail(EXT_ERR_CHECKPOINT, "not a network checkpoint (magic)");
  if (get_u32(b.data() + 8) != CKPT_VERSION) return fail(EXT_ERR_CHECKPOINT, "unknown checkpoint version");
  const uint32_t n_in = get_u32(b.data() + 12), hidden = get_u32(b.data() + 16);
  const uint64_t n = get_u64(b.data() + 32);
  if (n_in < 1 || n_in > 4096 || hidden < 16 || hidden > 1024 || hidden % 16 || n != ckpt_floats(n_in, hidden))
    return fail(EXT_ERR_CHECKPOINT, "checkpoint header has impossible shapes");
  if (b.size() != CKPT_HEADER + 3 * 4 * n + 4) return fail(EXT_ERR_CHECKPOINT, "checkpoint length does not match its header");
  if (crc32_ieee(b.data(), b.size() - 4) != get_u32(b.data() + b.size() - 4))
    return fail(EXT_ERR_CHECKPOINT, "checkpoint CRC-32 mismatch (corrupt file)");
  info->n_in = (int)n_in;
  info->hidden = (int)hidden;
  info->step = get_u64(b.data() + 24);
  info->n = n;
  return EXT_OK;
}

// One parameter-sized device buffer (padded layout of the network) <-> the
// packed layout of ext_mlp_set_params: W1, b1, W2, b2, W3, b3.
ext_status ckpt_pack(ext_mlp net, const float* base, float* out) {
  const size_t H = net->H, f = sizeof(float), ni = net->n_in;
  float* o = out;
  EXT_CUDA(cudaMemcpy2D(o, f * ni, base + net->oW1, f * net->dp, f * ni, H, cudaMemcpyDeviceToHost));
  o += H * ni;
  EXT_CUDA(cudaMemcpy(o, base + net->ob1, f * H, cudaMemcpyDeviceToHost));
  o += H;
  EXT_CUDA(cudaMemcpy(o, base + net->oW2, f * H * H, cudaMemcpyDeviceToHost));
  o += H * H;
  EXT_CUDA(cudaMemcpy(o, base + net->ob2, f * H, cudaMemcpyDeviceToHost));
  o += H;
  EXT_CUDA(cudaMemcpy(o, base + net->oW3, f * 4 * H, cudaMemcpyDeviceToHost));
  o += 4 * H;
  EXT_CUDA(cudaMemcpy(o, base + net->ob3, f * 4, cudaMemcpyDeviceToHost));
  return EXT_OK;
}

ext_status ckpt_unpack(ext_mlp net, const float* in, float* base) {
  const size_t H = net->H, f = sizeof(float), ni = net->n_in;
  EXT_CUDA(cudaMemset(base, 0, f * net->n_par));
  const float* s = in;
  EXT_CUDA(cudaMemcpy2D(base + net->oW1, f * net->dp, s, f * ni, f * ni, H, cudaMemcpyHostToDevice));
  s += H * ni;
  EXT_CUDA(cudaMemcpy(base + net->ob1, s, f * H, cudaMemcpyHostToDevice));
  s += H;
  EXT_CUDA(cudaMemcpy(base + net->oW2, s, f * H * H, cudaMemcpyHostToDevice));
  s += H * H;
  EXT_CUDA(cudaMemcpy(base + net->ob2, s, f * H, cudaMemcpyHostToDevice));
  s += H;
  EXT_CUDA(cudaMemcpy(base + net->oW3, s, f * 4 * H, cudaMemcpyHostToDevice));
  s += 4 * H;
  EXT_CUDA(cudaMemcpy(base + net->ob3, s, f * 4, cudaMemcpyHostToDevice));
  return EXT_OK;
}

}  // namespace

extern "C" {

ext_status ext_mlp_save(ext_mlp net, const char* path) {
  if (!net || !path) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_CUDA(cudaSetDevice(net->device));
  EXT_CUDA(cudaDeviceSynchronize());
  const uint64_t n = ckpt_floats(net->n_in, net->H);
  std::vector<unsigned char> b(CKPT_HEADER + 3 * 4 * n + 4, 0);
  std::memcpy(b.data(), CKPT_MAGIC, 8);
  put_u32(b.data() + 8, CKPT_VERSION);
  put_u32(b.data() + 12, (uint32_t)net->n_in);
  put_u32(b.data() + 16, (uint32_t)net->H);
  put_u64(b.data() + 24, (uint64_t)net->step);
  put_u64(b.data() + 32, n);
  std::vector<float> blk(n);
  const float* bases[3] = {net->w, net->m, net->v};
  for (int i = 0; i < 3; ++i) {
    EXT_TRY(ckpt_pack(net, bases[i], blk.data()));
    unsigned char* dst = b.data() + CKPT_HEADER + (size_t)i * 4 * n;
    for (uint64_t j = 0; j < n; ++j) {
      uint32_t u;
      std::memcpy(&u, &blk[j], 4);
      put_u32(dst + 4 * j, u);
    }
  }
  put_u32(b.data() + b.size() - 4, crc32_ieee(b.data(), b.size() - 4));
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(EXT_ERR_CHECKPOINT, std::string("cannot create ") + tmp);
  const bool ok = std::fwrite(b.data(), 1, b.size(), f) == b.size();
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(EXT_ERR_CHECKPOINT, std::string("cannot write checkpoint ") + path);
  }
  return EXT_OK;
}

ext_status ext_mlp_load(ext_mlp net, const char* path) {
  if (!net || !path) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  std::vector<unsigned char> b;
  CkptInfo info;
  EXT_TRY(ckpt_read(path, &b, &info));
  if (info.n_in != net->n_in || info.hidden != net->H)
    return fail(EXT_ERR_CHECKPOINT, "checkpoint shapes differ from the network's");
  EXT_CUDA(cudaSetDevice(net->device));
  EXT_CUDA(cudaDeviceSynchronize());
  std::vector<float> blk(info.n);
  float* bases[3] = {net->w, net->m, net->v};
  for (int i = 0; i < 3; ++i) {
    const unsigned char* src = b.data() + CKPT_HEADER + (size_t)i * 4 * info.n;
    for (uint64_t j = 0; j < info.n; ++j) {
      const uint32_t u = get_u32(src + 4 * j);
      std::memcpy(&blk[j], &u, 4);
    }
    EXT_TRY(ckpt_unpack(net, blk.data(), bases[i]));
  }
  net->step = (int)info.step;
  launch(net->plan, "mlp_to_bf16", 0, [&] { launch_f32_to_bf16(net->w, (long long)net->n_par, net->w16, 0); });
  EXT_CUDA(cudaGetLastError());
  EXT_CUDA(cudaDeviceSynchronize());
  return EXT_OK;
}

ext_status ext_mlp_checkpoint_info(const char* path, int* n_in, int* hidden, int64_t* step) {
  std::vector<unsigned char> b;
  CkptInfo info;
  EXT_TRY(ckpt_read(path, &b, &info));
  if (n_in) *n_in = info.n_in;
  if (hidden) *hidden = info.hidden;
  if (step) *step = (int64_t)info.step;
  return EXT_OK;
}

}  // extern "C"
