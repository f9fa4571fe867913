// C ABI of libextconv.so, SO(3) operators: components, sweeps and the
// learned proposal.
#include "plan.h"

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

// G (nchan planes of nz*ny*nx floats) for volume V (device).
ext_status so3_components(ext_plan plan, const float* V, int nz, int ny, int nx, const double* tables, int L, int n_r,
                          double dr, int R, float* G, cudaStream_t st) {
  const So3Layout lay = so3_layout(L);
  const int ncomp = (int)lay.comp.size();
  const size_t P = (size_t)nz * ny * nx;
  const int w2 = ny * nx;   // z-pass: a 2D array of nz rows and ny*nx columns
  // device copies of the layout and the tables
  void *dcomp, *dchan, *dtab;
  EXT_TRY(ensure(plan, "so3_comp", sizeof(int4) * ncomp, &dcomp));
  EXT_TRY(ensure(plan, "so3_chan", sizeof(int2) * ncomp, &dchan));
  const size_t tab_bytes = sizeof(double2) * (size_t)(L + 1) * (L + 1) * n_r;
  EXT_TRY(ensure(plan, "so3_tab", tab_bytes, &dtab));
  EXT_CUDA(cudaMemcpyAsync(dcomp, lay.comp.data(), sizeof(int4) * ncomp, cudaMemcpyHostToDevice, st));
  EXT_CUDA(cudaMemcpyAsync(dchan, lay.chan.data(), sizeof(int2) * ncomp, cudaMemcpyHostToDevice, st));
  EXT_CUDA(cudaMemcpyAsync(dtab, tables, tab_bytes, cudaMemcpyHostToDevice, st));
  const float2 *tw_x, *tw_y, *tw_z;
  EXT_TRY(twiddle(plan, nx, st, &tw_x));
  EXT_TRY(twiddle(plan, ny, st, &tw_y));
  EXT_TRY(twiddle(plan, nz, st, &tw_z));
  // component spectra, cached per filter and volume shape
  uint64_t key = 0x503503503ull;
  key = fnv1a(key, tables, tab_bytes);
  int meta[5] = {L, n_r, R, nz, ny};
  key = fnv1a(key, meta, sizeof(meta));
  key = fnv1a(key, &dr, sizeof(dr));
  key = fnv1a(key, &nx, sizeof(nx));
  const float2* S = nullptr;
  {
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
        launch_so3_component_grid((const int4*)dcomp, k0, nk, (const double2*)dtab, n_r, dr, L, R, nz, ny, nx,
                                  (float2*)grid, st);
        fft_rows_c2c(nx, (const float2*)grid, nz * ny, nk, (float2*)grid, false, tw_x, st);
        fft_cols_c2c(ny, (float2*)grid, nx, nz * nk, false, tw_y, st);
        fft_cols_fwd_spectrum(nz, (const float2*)grid, w2, 1, scale, Sdst + per_k * k0, tw_z, st, nk, scale);
      }
      EXT_CUDA(cudaGetLastError());
      return EXT_OK;
    };
    bool hit = false;
    for (auto& e : plan->specs)
      if (e.key == key) { e.stamp = ++plan->clock; S = e.S; hit = true; }
    if (!hit) {
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
      EXT_CUDA(cudaMalloc(&e.S, e.bytes));
      ext_status bs = build(e.S);
      if (bs != EXT_OK) { cudaFree(e.S); return bs; }
      e.stamp = ++plan->clock;
      plan->specs.push_back(e);
      S = e.S;
    }
  }
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
    launch(plan, "so3_cols_y", st, [&] { fft_cols_c2c(ny, (float2*)Z, nx, nz * nk, true, tw_y, st); });
    launch(plan, "so3_rows_x", st, [&] {
      fft_rows_inv_channels(nx, (const float2*)Z, nz * ny, k0, nk, (const int2*)dchan, G, tw_x, st);
    });
  }
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

// Steering table B[j][c] (FP32, rows padded to cpad) of a rotation set, and
// for the tensor-core sweep its split-BF16 blocks; cached for the last set.
ext_status so3_tables(ext_plan plan, const double* quats, int n_rot, int L, cudaStream_t st, const float** B,
                      const unsigned char** Bt, int* cpad_out, int* nchan_out) {
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
  for (void* q : {dq, dB, dBt}) key = fnv1a(key, &q, sizeof(q));
  if (plan->so3_rot_key != key) {
    EXT_CUDA(cudaMemcpyAsync(dq, quats, sizeof(double) * 4 * n_rot, cudaMemcpyHostToDevice, st));
    EXT_CUDA(cudaMemcpyAsync(dch, lay.comp.data(), sizeof(int4) * lay.comp.size(), cudaMemcpyHostToDevice, st));
    launch_so3_wigner((const double*)dq, n_rot, L, nullptr, (const int4*)dch, (int)lay.comp.size(), cpad, (float*)dB, st);
    so3_build_btc((const float*)dB, cpad, n_rot, (unsigned char*)dBt, st);
    EXT_CUDA(cudaGetLastError());
    EXT_CUDA(cudaStreamSynchronize(st));   // the host quaternions may change after return
    plan->so3_rot_key = key;
  }
  *B = (const float*)dB;
  *Bt = (const unsigned char*)dBt;
  *cpad_out = cpad;
  *nchan_out = nchan;
  return EXT_OK;
}

ext_status so3_sweep(ext_plan plan, const float* G, long long P, int L, const double* quats, int n_rot, float* maxv,
                     int32_t* argmax, int precision, cudaStream_t st) {
  const float* B;
  const unsigned char* Bt;
  int cpad, nchan;
  EXT_TRY(so3_tables(plan, quats, n_rot, L, st, &B, &Bt, &cpad, &nchan));
  if (precision == EXT_PREC_BF16X3)
    launch(plan, "so3_sweep_bf16x3", st,
           [&] { sweep_so3_tc(G, P, nchan, cpad, Bt, n_rot, maxv, argmax, plan->dev_err, plan->sms, st); });
  else
    launch(plan, "so3_sweep_fp32", st, [&] { sweep_so3_fp32(G, P, nchan, B, cpad, n_rot, maxv, argmax, st); });
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

}  // namespace

extern "C" {

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
