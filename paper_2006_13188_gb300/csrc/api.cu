// C ABI of libextconv.so, SO(2) and scale operators: argument checking, the
// filter caches, and the launch sequences of each operator.
#include "plan.h"

#include <fstream>
#include <mutex>
#include <set>
#include <sstream>
#include <tuple>

namespace {
thread_local std::string g_last_error;
}  // namespace

void ext_set_error(const char* msg) { g_last_error = msg; }

namespace {
std::mutex g_optin_mutex;
std::set<std::tuple<int, const void*, int>> g_optin_done;
}  // namespace

bool ext_smem_optin(const void* func, int bytes) {
  if (bytes <= 48 * 1024) return true;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  // launch paths ask on every launch: answer repeats from a per-thread list without the lock
  thread_local std::vector<std::tuple<int, const void*, int>> seen;
  const auto key0 = std::make_tuple(dev, func, bytes);
  for (const auto& e : seen)
    if (e == key0) return true;
  std::lock_guard<std::mutex> lock(g_optin_mutex);
  auto key = std::make_tuple(dev, func, bytes);
  if (g_optin_done.count(key)) {
    seen.push_back(key);
    return true;
  }
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  g_optin_done.insert(key);
  seen.push_back(key);
  return true;
}

namespace {

ext_status check_filter(const ext_filter_so2* F) {
  if (!F) return fail(EXT_ERR_INVALID_ARG, "filter is NULL");
  if (F->K < 0 || F->K > 64) return fail(EXT_ERR_INVALID_ARG, "filter K must be in [0, 64]");
  if (F->R < 0 || F->R > 1024) return fail(EXT_ERR_INVALID_ARG, "filter R must be in [0, 1024]");
  switch (F->kind) {
    case EXT_FILTER_ANALYTIC_GAUSSPOW:
      if (!F->a) return fail(EXT_ERR_INVALID_ARG, "analytic filter needs a");
      if (!(F->sigma > 0)) return fail(EXT_ERR_INVALID_ARG, "analytic filter needs sigma > 0");
      break;
    case EXT_FILTER_TABLE:
      if (!F->fk || F->n_r < 2 || !(F->dr > 0))
        return fail(EXT_ERR_INVALID_ARG, "table filter needs fk, n_r >= 2, dr > 0");
      break;
    case EXT_FILTER_SAMPLED:
      if (!F->img || !(F->dr > 0) || F->n_theta < 1)
        return fail(EXT_ERR_INVALID_ARG, "sampled filter needs img, dr > 0, n_theta >= 1");
      break;
    default:
      return fail(EXT_ERR_INVALID_ARG, "unknown filter kind");
  }
  return EXT_OK;
}

// Content hash of a filter's arrays, read as 64-bit words in four independent
// multiply-xor lanes (a batch hashes every template on every call, so the
// byte-serial FNV of the other keys would cost milliseconds there).
uint64_t hash_words(uint64_t h, const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t lane[4] = {h ^ 0x9E3779B97F4A7C15ull, h + 0xC2B2AE3D27D4EB4Full, h ^ 0x165667B19E3779F9ull,
                      h + 0x27D4EB2F165667C5ull};
  size_t i = 0;
  for (; i + 32 <= n; i += 32) {
    uint64_t w[4];
    std::memcpy(w, p + i, 32);
    for (int q = 0; q < 4; ++q) lane[q] = (lane[q] ^ w[q]) * 0x100000001B3ull;
  }
  uint64_t out = fnv1a(h, p + i, n - i);
  for (int q = 0; q < 4; ++q) {
    out ^= lane[q] + 0x9E3779B97F4A7C15ull + (out << 6) + (out >> 2);
    out *= 0xff51afd7ed558ccdull;
  }
  return out ^ (out >> 33);
}

uint64_t filter_key(const ext_filter_so2* F) {
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, &F->kind, sizeof(int));
  h = fnv1a(h, &F->K, sizeof(int));
  h = fnv1a(h, &F->R, sizeof(int));
  const size_t nk = (size_t)(2 * F->K + 1);
  if (F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW) {
    h = fnv1a(h, F->a, sizeof(double) * 2 * nk);
    h = fnv1a(h, &F->sigma, sizeof(double));
  } else if (F->kind == EXT_FILTER_TABLE) {
    h = fnv1a(h, &F->n_r, sizeof(int));
    h = fnv1a(h, &F->dr, sizeof(double));
    h = hash_words(h, F->fk, sizeof(double) * 2 * nk * F->n_r);
  } else {
    const size_t side = (size_t)(2 * F->R + 1);
    h = fnv1a(h, &F->dr, sizeof(double));
    h = fnv1a(h, &F->n_theta, sizeof(int));
    h = hash_words(h, F->img, sizeof(double) * side * side);
  }
  return h;
}

int sampled_nr(const ext_filter_so2* F) {
  // radii i * dr <= R
  return (int)((double)F->R / F->dr + 1e-9) + 1;
}

// Radial coefficients on the device: analytic a_k, or the f_k table (given or
// decomposed from a sampled image).  Returns pointer into workspace "coef".
ext_status filter_coefficients(ext_plan plan, const ext_filter_so2* F, cudaStream_t st, const double2** coef,
                               int* n_r, double* dr) {
  const int nk = 2 * F->K + 1;
  void* p = nullptr;
  if (F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW) {
    EXT_TRY(ensure(plan, "coef", sizeof(double2) * nk, &p));
    EXT_CUDA(cudaMemcpyAsync(p, F->a, sizeof(double2) * nk, cudaMemcpyHostToDevice, st));
    *n_r = 0;
    *dr = 0.0;
  } else if (F->kind == EXT_FILTER_TABLE) {
    EXT_TRY(ensure(plan, "coef", sizeof(double2) * nk * F->n_r, &p));
    EXT_CUDA(cudaMemcpyAsync(p, F->fk, sizeof(double2) * nk * F->n_r, cudaMemcpyHostToDevice, st));
    *n_r = F->n_r;
    *dr = F->dr;
  } else {
    const int side = 2 * F->R + 1;
    const int nr = sampled_nr(F);
    void *img = nullptr, *P = nullptr;
    EXT_TRY(ensure(plan, "fimg", sizeof(double) * side * side, &img));
    EXT_TRY(ensure(plan, "fpolar", sizeof(double) * nr * F->n_theta, &P));
    EXT_TRY(ensure(plan, "coef", sizeof(double2) * nk * nr, &p));
    EXT_CUDA(cudaMemcpyAsync(img, F->img, sizeof(double) * side * side, cudaMemcpyHostToDevice, st));
    launch_decompose_sampled((const double*)img, side, F->dr, nr, F->n_theta, F->K, (double*)P, (double2*)p, st);
    EXT_CUDA(cudaGetLastError());
    *n_r = nr;
    *dr = F->dr;
  }
  *coef = (const double2*)p;
  return EXT_OK;
}

enum SpecMode { SPEC_CORR = 0, SPEC_CONV = 1 };

// Spectra of `ncomp` filter components on an h x w grid, tiled for the column
// passes; sample(k, grid) writes component k into a zeroed h x w grid.
//   SPEC_CORR: S_k = conj(F^_k) / (h w)
//   SPEC_CONV: S_k = w_k F^_k / (h w), w_0 = 1, w_k = 2 (k >= 1; the -k terms
//              of a real filter give the complex conjugate contribution)
// Writes the spectra of `ncomp` components into S (tiled layout, see below).
// sample(k0, nk, grid) writes components k0..k0+nk-1 into consecutive zeroed
// h x w planes of grid; components are processed in chunks bounded by memory.
template <class Sampler>
ext_status build_spectra(ext_plan plan, int h, int w, int ncomp, int mode, cudaStream_t st, Sampler&& sample,
                         float2* S, const char* grid_name = "grid") {
  const int cw = fft_col_tile(h);
  const size_t per_k = (size_t)((w + cw - 1) / cw) * h * cw;
  const size_t plane = sizeof(float2) * (size_t)h * w;
  int chunk = (int)((512ull << 20) / plane);
  if (chunk < 1) chunk = 1;
  if (chunk > ncomp) chunk = ncomp;
  const float2 *tw_w = nullptr, *tw_h = nullptr;
  EXT_TRY(twiddle(plan, w, st, &tw_w));
  EXT_TRY(twiddle(plan, h, st, &tw_h));
  void* grid = nullptr;
  EXT_TRY(ensure(plan, grid_name, plane * chunk, &grid));
  const float inv_hw = 1.0f / ((float)h * (float)w);
  for (int k0 = 0; k0 < ncomp; k0 += chunk) {
    const int nk = k0 + chunk <= ncomp ? chunk : ncomp - k0;
    EXT_CUDA(cudaMemsetAsync(grid, 0, plane * nk, st));
    sample(k0, nk, (float2*)grid);
    fft_rows_c2c(w, (const float2*)grid, h, nk, (float2*)grid, false, tw_w, st);
    const float s_rest = mode == 1 ? 2.0f * inv_hw : inv_hw;   // SPEC_CONV weights k >= 1 by 2
    const float s0 = k0 == 0 ? inv_hw : s_rest;
    fft_cols_fwd_spectrum(h, (const float2*)grid, w, mode == 0 ? 1 : 0, s0, S + per_k * k0, tw_h, st, nk, s_rest);
  }
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

template <class Sampler>
ext_status spectra_generic(ext_plan plan, uint64_t key, int h, int w, int ncomp, SpecMode mode, cudaStream_t st,
                           Sampler&& sample, const float2** out) {
  key = fnv1a(key, &h, sizeof(int));
  key = fnv1a(key, &w, sizeof(int));
  int m = (int)mode;
  key = fnv1a(key, &m, sizeof(int));
  for (auto& e : plan->specs) {
    if (e.key == key) {
      e.stamp = ++plan->clock;
      *out = e.S;
      return EXT_OK;
    }
  }
  const int cw = fft_col_tile(h);
  const int ntiles = (w + cw - 1) / cw;
  const size_t per_k = (size_t)ntiles * h * cw;
  const size_t bytes = sizeof(float2) * per_k * ncomp;
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
  e.bytes = bytes;
  EXT_TRY(plan_malloc(plan, (void**)&e.S, bytes));
  const float2 *tw_w = nullptr, *tw_h = nullptr;
  EXT_TRY(twiddle(plan, w, st, &tw_w));
  EXT_TRY(twiddle(plan, h, st, &tw_h));
  EXT_TRY(build_spectra(plan, h, w, ncomp, mode, st, sample, e.S));
  e.stamp = ++plan->clock;
  plan->specs.push_back(e);
  *out = e.S;
  return EXT_OK;
}

// Component spectra of an SO(2) filter F_k = f_k(r) e^{ik theta}, k = 0..K.
ext_status spectra(ext_plan plan, const ext_filter_so2* F, int h, int w, SpecMode mode, cudaStream_t st,
                   const float2** out) {
  const uint64_t key = filter_key(F);
  // the radial coefficients are only needed on a cache miss; compute them lazily
  const double2* coef = nullptr;
  int n_r = 0;
  double dr = 0;
  ext_status cs = EXT_OK;
  bool have = false;
  const int kind = F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW ? EXT_FILTER_ANALYTIC_GAUSSPOW : EXT_FILTER_TABLE;
  auto sample = [&](int k0, int nk, float2* grid) {
    if (!have) {
      cs = filter_coefficients(plan, F, st, &coef, &n_r, &dr);
      have = true;
    }
    if (cs == EXT_OK) launch_component_grid(kind, F->K, k0, coef, n_r, dr, F->sigma, F->R, h, w, grid, st, nk);
  };
  EXT_TRY(spectra_generic(plan, key, h, w, F->K + 1, mode, st, sample, out));
  return cs;
}

// Spectra of the listed components ks[0..nks) (ks[0] = 0), in list order.
ext_status spectra_list(ext_plan plan, const ext_filter_so2* F, const int* ks, int nks, int h, int w, SpecMode mode,
                        cudaStream_t st, const float2** out) {
  uint64_t key = fnv1a(filter_key(F), &nks, sizeof(int));
  key = fnv1a(key, ks, sizeof(int) * nks);
  const double2* coef = nullptr;
  int n_r = 0;
  double dr = 0;
  ext_status cs = EXT_OK;
  bool have = false;
  const int kind = F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW ? EXT_FILTER_ANALYTIC_GAUSSPOW : EXT_FILTER_TABLE;
  const size_t plane = (size_t)h * w;
  auto sample = [&](int p0, int np, float2* grid) {
    if (!have) {
      cs = filter_coefficients(plan, F, st, &coef, &n_r, &dr);
      have = true;
    }
    if (cs == EXT_OK)
      for (int i = 0; i < np; ++i)
        launch_component_grid(kind, F->K, ks[p0 + i], coef, n_r, dr, F->sigma, F->R, h, w, grid + plane * i, st, 1);
  };
  EXT_TRY(spectra_generic(plan, key, h, w, nks, mode, st, sample, out));
  return cs;
}

// Steering weights of a component list (ks[0] = 0): B[j][2(i-1)] = 2 cos(2 pi ks[i] j / J),
// B[j][2(i-1)+1] = -2 sin(2 pi ks[i] j / J), i = 1..nks-1; rows padded to cp floats.
ext_status sweep_table_list(ext_plan plan, const int* ks, int nks, int J, cudaStream_t st, const float** out,
                            int* cp_out) {
  const int K = nks - 1;
  const int cp = (2 * K + 3) / 4 * 4;
  uint64_t key = fnv1a(0x5eedull, &J, sizeof(int));
  key = fnv1a(key, ks, sizeof(int) * nks) | 1ull;   // odd: apart from the (K << 32 | J) keys
  auto it = plan->sweep_tables.find(key);
  if (it == plan->sweep_tables.end()) {
    float* B = nullptr;
    EXT_TRY(plan_malloc(plan, (void**)&B, sizeof(float) * (size_t)J * (cp > 0 ? cp : 4)));
    if (cp > 0) {
      void* dks = nullptr;
      EXT_TRY(ensure(plan, "sweep_ks", sizeof(int) * nks, &dks));
      EXT_CUDA(cudaMemcpyAsync(dks, ks, sizeof(int) * nks, cudaMemcpyHostToDevice, st));
      launch_sweep_table_list((const int*)dks, K, J, cp, B, st);
      EXT_CUDA(cudaStreamSynchronize(st));   // the host list may go out of scope
    }
    EXT_CUDA(cudaGetLastError());
    it = plan->sweep_tables.emplace(key, B).first;
  }
  *out = it->second;
  *cp_out = cp;
  return EXT_OK;
}

ext_status sweep_table(ext_plan plan, int K, int J, cudaStream_t st, const float** out, int* cp_out) {
  const int cp = (2 * K + 3) / 4 * 4;
  const uint64_t key = ((uint64_t)K << 32) | (uint32_t)J;
  auto it = plan->sweep_tables.find(key);
  if (it == plan->sweep_tables.end()) {
    float* B = nullptr;
    EXT_TRY(plan_malloc(plan, (void**)&B, sizeof(float) * (size_t)J * (cp > 0 ? cp : 4)));
    if (cp > 0) launch_sweep_table(K, J, cp, B, st);
    EXT_CUDA(cudaGetLastError());
    it = plan->sweep_tables.emplace(key, B).first;
  }
  *out = it->second;
  *cp_out = cp;
  return EXT_OK;
}

ext_status check_size(int h, int w) {
  if (h < 0 || w < 0) return fail(EXT_ERR_INVALID_ARG, "negative image size");
  if (h == 0 || w == 0) return EXT_OK;
  if (!fft_size_supported(h) || !fft_size_supported(w))
    return fail(EXT_ERR_UNSUPPORTED, "image side " + std::to_string(!fft_size_supported(h) ? h : w) +
                                         " is not a supported FFT length");
  if (w % 2) return fail(EXT_ERR_UNSUPPORTED, "image width must be even");
  return EXT_OK;
}

// Tensor map of the full h x w complex spectrum as h rows of 2w floats, box
// 2 cw floats x br rows.
bool spectrum_tmap(const float2* Hf, int h, int w, int cw, int br, CUtensorMap* out) {
  return make_tmap_2d_f32(Hf, (unsigned long long)2 * w, (unsigned long long)h, (unsigned long long)2 * w * sizeof(float),
                          (unsigned)(2 * cw), (unsigned)br, out);
}

// G_k = H (*) F_k for k = 0..K into G (device, planes G_0, Re G_1, Im G_1, ...);
// with a component list ks (ks[0] = 0), for the listed components in list order.
ext_status run_components(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F, float* G,
                          cudaStream_t st, const int* ks = nullptr, int nks = 0) {
  const int K = ks ? nks - 1 : F->K;
  const float2* S = nullptr;
  if (ks)
    EXT_TRY(spectra_list(plan, F, ks, nks, h, w, SPEC_CORR, st, &S));
  else
    EXT_TRY(spectra(plan, F, h, w, SPEC_CORR, st, &S));
  const float2 *tw_w = nullptr, *tw_h = nullptr;
  EXT_TRY(twiddle(plan, w, st, &tw_w));
  EXT_TRY(twiddle(plan, h, st, &tw_h));
  const int wh = w / 2 + 1;
  void* Hh = nullptr;
  EXT_TRY(ensure(plan, "Hh", sizeof(float2) * (size_t)h * wh, &Hh));
  // TMA-staged column pass on the full spectrum where the tile shape allows it;
  // the forward column pass then writes the full spectrum as well
  CUtensorMap tmH;
  const int cw = fft_col_tile(h);
  const int br = plan->tma && fft_cols_tma_ok(h) ? tma_rows(h, cw) : 0;
  bool use_tma = false;
  void* Hf = nullptr;
  if (br > 0) {
    EXT_TRY(ensure(plan, "Hf", sizeof(float2) * (size_t)h * w, &Hf));
    use_tma = spectrum_tmap((const float2*)Hf, h, w, cw, br, &tmH);
  }
  launch(plan, "rows_r2c", st, [&] { fft_rows_r2c(w, H, h, (float2*)Hh, tw_w, st); });
  launch(plan, "cols_fwd_half", st,
         [&] { fft_cols_fwd_half(h, (float2*)Hh, wh, tw_h, st, use_tma ? (float2*)Hf : nullptr, w); });
  // All components go through each inverse pass in one launch: measured on
  // 2048^2 x 17 components, one launch beats per-component launches that keep
  // the partial products L2-resident (tail imbalance dominates), at the cost
  // of a (K+1)-plane intermediate.
  const size_t plane = sizeof(float2) * (size_t)h * w;
  int kc = K + 1;
  if (plan->kchunk > 0) kc = plan->kchunk < K + 1 ? plan->kchunk : K + 1;
  void* Z = nullptr;
  EXT_TRY(ensure(plan, "Z", plane * kc, &Z));
  for (int k0 = 0; k0 <= K; k0 += kc) {
    const int nk = (k0 + kc <= K + 1) ? kc : (K + 1 - k0);
    bool piped = false;
    if (use_tma)
      launch(plan, "cols_inv_corr_tma", st, [&] {
        piped = fft_cols_inv_corr_tma(h, tmH, w, br, S, k0, nk, (float2*)Z, tw_h, plan->dev_err, plan->sms, st);
      });
    if (!piped && plan->pipelined)
      launch(plan, "cols_inv_corr_pipe", st, [&] {
        piped = fft_cols_inv_corr_pipe(h, (const float2*)Hh, w, S, k0, nk, (float2*)Z, tw_h, plan->sms, st);
      });
    if (!piped)
      launch(plan, "cols_inv_corr", st,
             [&] { fft_cols_inv_corr(h, (const float2*)Hh, w, S, k0, nk, (float2*)Z, tw_h, st); });
    piped = false;
    if (plan->pipelined)
      launch(plan, "rows_inv_components_pipe", st, [&] {
        piped = fft_rows_inv_components_pipe(w, (const float2*)Z, h, k0, nk, G, tw_w, plan->dev_err, plan->sms, st);
      });
    if (!piped)
      launch(plan, "rows_inv_components", st,
             [&] { fft_rows_inv_components(w, (const float2*)Z, h, k0, nk, G, tw_w, st); });
  }
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

// ----- autotuner of the component passes (ext_options.autotune)
// A shape class (h, w, K) has several pass variants that compute the same
// components: the inverse column pass staged by tensor copies or not, the
// persistent prefetching passes or the plain ones, and all components per
// inverse launch or two chunks.  The first call of a class with autotuning on
// times every variant on the call's own data (one warm-up run, then three
// timed runs each, CUDA events on the call's stream) and keeps the fastest;
// the choice is cached per plan and, with a cache file, across processes.
struct PassVariant {
  bool tma = true, pipelined = true;
  int kchunk = 0;
};

std::string gpu_tag(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  int drv = 0;
  cudaDriverGetVersion(&drv);
  std::string name = prop.name;
  for (char& c : name)
    if (c == '\t' || c == '\n') c = ' ';
  return name + " driver " + std::to_string(drv);
}

void tune_cache_read(ext_plan plan) {
  if (plan->tune_cache.empty()) return;
  std::ifstream f(plan->tune_cache);
  const std::string tag = gpu_tag(plan->device);
  std::string line;
  while (std::getline(f, line)) {
    const size_t a = line.find('\t'), b = line.find('\t', a == std::string::npos ? a : a + 1);
    if (a == std::string::npos || b == std::string::npos) continue;
    if (line.compare(0, a, tag) == 0 && a == tag.size()) plan->tuned[line.substr(a + 1, b - a - 1)] = line.substr(b + 1);
  }
}

void tune_cache_write(ext_plan plan) {
  if (plan->tune_cache.empty()) return;
  const std::string tag = gpu_tag(plan->device);
  std::vector<std::string> keep;
  {
    std::ifstream f(plan->tune_cache);
    std::string line;
    while (std::getline(f, line))
      if (!(line.size() > tag.size() && line.compare(0, tag.size(), tag) == 0 && line[tag.size()] == '\t'))
        keep.push_back(line);
  }
  const std::string tmp = plan->tune_cache + ".tmp";
  {
    std::ofstream f(tmp, std::ios::trunc);
    for (const auto& l : keep) f << l << "\n";
    for (const auto& kv : plan->tuned) f << tag << "\t" << kv.first << "\t" << kv.second << "\n";
  }
  std::rename(tmp.c_str(), plan->tune_cache.c_str());
}

PassVariant parse_variant(const std::string& v) {
  PassVariant p;
  int t = 1, q = 1, k = 0;
  std::istringstream in(v);
  in >> t >> q >> k;
  p.tma = t != 0;
  p.pipelined = q != 0;
  p.kchunk = k;
  return p;
}

struct VariantScope {   // applies a variant to the plan for one call
  ext_plan plan;
  bool tma, pipelined;
  int kchunk;
  VariantScope(ext_plan p, const PassVariant& v) : plan(p), tma(p->tma), pipelined(p->pipelined), kchunk(p->kchunk) {
    p->tma = v.tma;
    p->pipelined = v.pipelined;
    p->kchunk = v.kchunk;
  }
  ~VariantScope() {
    plan->tma = tma;
    plan->pipelined = pipelined;
    plan->kchunk = kchunk;
  }
};

std::string class_key(int h, int w, int K) {
  return "components " + std::to_string(h) + "x" + std::to_string(w) + " K=" + std::to_string(K);
}

ext_status tune_components(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F, float* G,
                           cudaStream_t st, PassVariant* best) {
  const int K = F->K;
  std::vector<PassVariant> cands;
  for (int t = 1; t >= 0; --t)
    for (int q = 1; q >= 0; --q)
      for (int k : {0, (K + 2) / 2}) {
        if (k != 0 && k >= K + 1) continue;
        PassVariant v;
        v.tma = t != 0;
        v.pipelined = q != 0;
        v.kchunk = k;
        cands.push_back(v);
      }
  cudaEvent_t a = take_event(plan), b = take_event(plan);
  const bool profiling = plan->profiling;
  plan->profiling = false;
  float best_ms = -1.f;
  for (const PassVariant& v : cands) {
    VariantScope scope(plan, v);
    ext_status s = run_components(plan, H, h, w, F, G, st);
    if (s == EXT_OK) {
      cudaEventRecord(a, st);
      for (int r = 0; r < 3 && s == EXT_OK; ++r) s = run_components(plan, H, h, w, F, G, st);
      cudaEventRecord(b, st);
    }
    if (s == EXT_OK && cudaEventSynchronize(b) == cudaSuccess && device_status(plan) == EXT_OK) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (best_ms < 0.f || ms < best_ms) {
        best_ms = ms;
        *best = v;
      }
    }
    cudaGetLastError();
  }
  plan->profiling = profiling;
  plan->event_pool.push_back(a);
  plan->event_pool.push_back(b);
  if (best_ms < 0.f) return fail(EXT_ERR_CUDA, "autotuning: no pass variant ran");
  char buf[96];
  std::snprintf(buf, sizeof(buf), "%d %d %d %.4f", best->tma ? 1 : 0, best->pipelined ? 1 : 0, best->kchunk,
                best_ms / 3.f);
  plan->tuned[class_key(h, w, K)] = buf;
  tune_cache_write(plan);
  return EXT_OK;
}

// run_components with the tuned variant of its shape class (tuned now if
// autotuning is on, the class is new and the stream is not being captured).
ext_status run_components_tuned(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F, float* G,
                                cudaStream_t st) {
  if (!plan->autotune) return run_components(plan, H, h, w, F, G, st);
  PassVariant v;
  auto it = plan->tuned.find(class_key(h, w, F->K));
  if (it != plan->tuned.end()) {
    v = parse_variant(it->second);
  } else {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    EXT_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return run_components(plan, H, h, w, F, G, st);
    EXT_TRY(tune_components(plan, H, h, w, F, G, st, &v));
  }
  VariantScope scope(plan, v);
  return run_components(plan, H, h, w, F, G, st);
}

// Extended convolution of nsig signals by the steered-spectrum route of
// Sec. 4.1 / Sec. 8: for each signal, rows(sig, A) writes the row transforms
// of its ncomp steered copies into A; the column pass (tensor-copy staged
// where the tile shape allows) sums their products with the cached spectra S
// and inverts the columns; the inverse row pass writes the real result to
// dst(sig).  Workspaces "Aall" and "Y".
template <class Rows, class Dst>
ext_status conv_signals(ext_plan plan, int h, int w, int ncomp, int nsig, const float2* S, cudaStream_t st,
                        const char* row_name, Rows&& rows, Dst&& dst) {
  const size_t P = (size_t)h * w;
  const float2 *tw_w = nullptr, *tw_h = nullptr;
  EXT_TRY(twiddle(plan, w, st, &tw_w));
  EXT_TRY(twiddle(plan, h, st, &tw_h));
  const int cw = fft_col_tile(h);
  bool gtw = false;
  const int br = plan->tma && fft_cols_conv_tma_ok(h, &gtw) ? tma_rows(h, cw) : 0;
  const float2* stw = nullptr;
  if (br > 0 && gtw) EXT_TRY(stage_table(plan, h, st, &stw));
  // All signals through one column-pass launch where their steered row
  // transforms fit the workspace budget: the launch interleaves the signals
  // tile by tile, so each spectrum tile comes from HBM once instead of once
  // per signal.
  const size_t all_bytes = sizeof(float2) * P * ncomp * (size_t)nsig;
  const bool together = br > 0 && nsig > 1 && plan->colconv_form == 2 && plan->conv_together &&
                        all_bytes <= ((size_t)16 << 30) && (size_t)ncomp * nsig * h < (1ull << 31);
  void *A = nullptr, *Y = nullptr;
  EXT_TRY(ensure(plan, "Aall", together ? all_bytes : sizeof(float2) * P * ncomp, &A));
  EXT_TRY(ensure(plan, "Y", sizeof(float2) * P * (together ? nsig : 1), &Y));
  CUtensorMap tmA;
  const bool tma_A = br > 0 && make_tmap_2d_f32(A, (unsigned long long)2 * w,
                                                (unsigned long long)ncomp * h * (together ? nsig : 1),
                                                (unsigned long long)2 * w * sizeof(float), (unsigned)(2 * cw),
                                                (unsigned)br, &tmA);
  if (together && tma_A) {
    for (int sig = 0; sig < nsig; ++sig)
      launch(plan, row_name, st, [&] { rows(sig, (float2*)A + P * ncomp * sig, tw_w); });
    bool done = false;
    launch(plan, "cols_conv_tma", st, [&] {
      done = fft_cols_conv_tma(h, tmA, w, br, ncomp - 1, S, (float2*)Y, tw_h, stw, plan->dev_err, plan->sms, st,
                               true, nsig);
    });
    if (!done) return fail(EXT_ERR_CUDA, "the multi-signal convolution column pass could not be launched");
    for (int sig = 0; sig < nsig; ++sig)
      launch(plan, "rows_inv_real", st,
             [&] { fft_rows_inv_real(w, (const float2*)Y + P * sig, h, dst(sig), tw_w, st); });
    EXT_CUDA(cudaGetLastError());
    return EXT_OK;
  }
  for (int sig = 0; sig < nsig; ++sig) {
    launch(plan, row_name, st, [&] { rows(sig, (float2*)A, tw_w); });
    bool done = false;
    if (tma_A)
      launch(plan, "cols_conv_tma", st, [&] {
        done = fft_cols_conv_tma(h, tmA, w, br, ncomp - 1, S, (float2*)Y, tw_h, stw, plan->dev_err, plan->sms, st,
                                 plan->colconv_form == 2);
      });
    if (!done)
      launch(plan, "cols_conv", st,
             [&] { fft_cols_conv(h, (const float2*)A, w, ncomp - 1, S, (float2*)Y, tw_h, st); });
    launch(plan, "rows_inv_real", st, [&] { fft_rows_inv_real(w, (const float2*)Y, h, dst(sig), tw_w, st); });
  }
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

// Extended convolution of device buffers (Sec. 2.2 Eq. Def-EConv, the algorithm
// of Sec. 4.1): out = Re sum_k (H e^{-ik alpha}) * F_k.
// Several signals with one angle field: Hs[i] (nullptr: the constant signal 1) -> outs[i].
ext_status run_conv_so2_signals(ext_plan plan, const float* const* Hs, float* const* outs, int nsig, const float* alpha,
                                int h, int w, const ext_filter_so2* F, cudaStream_t st) {
  const int K = F->K;
  const float2* S = nullptr;
  EXT_TRY(spectra(plan, F, h, w, SPEC_CONV, st, &S));
  return conv_signals(
      plan, h, w, K + 1, nsig, S, st, "rows_fwd_phase",
      [&](int sig, float2* A, const float2* tw_w) {
        const float* H = Hs[sig];
        if (plan->steer_mode >= 2 &&
            fft_rows_fwd_hloop_phase(w, H, alpha, h, 0, K + 1, A, tw_w, plan->sms, st, plan->steer_mode == 2))
          return;
        if (plan->steer_mode == 1) fft_rows_fwd_phase_io(w, H, alpha, h, 0, K + 1, A, tw_w, st);
        else fft_rows_fwd_phase(w, H, alpha, h, 0, K + 1, A, tw_w, st);
      },
      [&](int sig) { return outs[sig]; });
}

ext_status run_conv_so2(ext_plan plan, const float* H, const float* alpha, int h, int w, const ext_filter_so2* F,
                        float* out, cudaStream_t st) {
  return run_conv_so2_signals(plan, &H, &out, 1, alpha, h, w, F, st);
}

ext_status run_sweep(ext_plan plan, const float* G, long long P, int K, int J, float* maxv, int32_t* argmax,
                     int precision, cudaStream_t st) {
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3)
    return fail(EXT_ERR_INVALID_ARG, "unknown precision");
  if (K == 0) {
    EXT_CUDA(cudaMemcpyAsync(maxv, G, sizeof(float) * P, cudaMemcpyDeviceToDevice, st));
    EXT_CUDA(cudaMemsetAsync(argmax, 0, sizeof(int32_t) * P, st));
    return EXT_OK;
  }
  if (K > 16) return fail(EXT_ERR_UNSUPPORTED, "sweep supports K <= 16");
  const float* B = nullptr;
  int cp = 0;
  EXT_TRY(sweep_table(plan, K, J, st, &B, &cp));
  bool ok = true;
  if (precision == EXT_PREC_BF16X3) {
    if (J > 128) return fail(EXT_ERR_UNSUPPORTED, "BF16x3 sweep supports at most 128 angles");
    launch(plan, "sweep_bf16x3", st,
           [&] { ok = sweep_bf16x3(G, P, K, J, B, cp, maxv, argmax, plan->dev_err, plan->sms, st); });
  } else {
    if (!sweep_fp32_fits(K, J))
      return fail(EXT_ERR_UNSUPPORTED, "FP32 sweep: the steering table of this many angles exceeds shared memory");
    launch(plan, "sweep_fp32", st, [&] { ok = sweep_fp32(G, P, K, J, B, cp, maxv, argmax, st); });
  }
  if (!ok) return fail(EXT_ERR_UNSUPPORTED, "sweep K");
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI ---
extern "C" {

const char* ext_status_string(ext_status s) {
  switch (s) {
    case EXT_OK: return "EXT_OK";
    case EXT_ERR_INVALID_ARG: return "EXT_ERR_INVALID_ARG";
    case EXT_ERR_UNSUPPORTED: return "EXT_ERR_UNSUPPORTED";
    case EXT_ERR_CUDA: return "EXT_ERR_CUDA";
    case EXT_ERR_OOM: return "EXT_ERR_OOM";
    case EXT_ERR_TIMEOUT: return "EXT_ERR_TIMEOUT";
    case EXT_ERR_CHECKPOINT: return "EXT_ERR_CHECKPOINT";
    default: return "EXT_ERR_UNKNOWN";
  }
}

const char* ext_last_error(void) { return g_last_error.c_str(); }

void ext_options_init(ext_options* o) {
  if (!o) return;
  o->device = 0;
  o->precision = EXT_PREC_FP32;
  o->wait_budget_ns = 0;
  o->autotune = EXT_TUNE_OFF;
  o->tune_cache = nullptr;
  o->fault_inject = EXT_FAULT_NONE;
  o->fault_after = 0;
}

ext_status ext_plan_create(ext_plan* plan, const ext_options* options) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  ext_options o;
  ext_options_init(&o);
  if (options) o = *options;
  if (o.precision != EXT_PREC_FP32 && o.precision != EXT_PREC_BF16X3)
    return fail(EXT_ERR_INVALID_ARG, "options.precision must be EXT_PREC_FP32 or EXT_PREC_BF16X3");
  if (o.autotune != EXT_TUNE_OFF && o.autotune != EXT_TUNE_ON) return fail(EXT_ERR_INVALID_ARG, "options.autotune");
  if (o.fault_inject != EXT_FAULT_NONE && o.fault_inject != EXT_FAULT_ALLOC)
    return fail(EXT_ERR_INVALID_ARG, "options.fault_inject");
  if (o.fault_after < 0) return fail(EXT_ERR_INVALID_ARG, "options.fault_after must be >= 0");
  int n = 0;
  EXT_CUDA(cudaGetDeviceCount(&n));
  if (o.device < 0 || o.device >= n) return fail(EXT_ERR_INVALID_ARG, "no such device");
  EXT_CUDA(cudaSetDevice(o.device));
  ext_plan p = new ext_plan_s();
  p->device = o.device;
  p->precision = o.precision;
  p->wait_budget_ns = o.wait_budget_ns ? o.wait_budget_ns : 1000000000ull;
  p->fault_inject = o.fault_inject;
  p->fault_countdown = o.fault_inject == EXT_FAULT_ALLOC ? o.fault_after : -1;
  p->autotune = o.autotune == EXT_TUNE_ON;
  if (o.tune_cache) p->tune_cache = o.tune_cache;
  cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, o.device);
  // status block: the status word at byte 0, the wait budget at byte 8
  unsigned long long block[2] = {0ull, p->wait_budget_ns};
  if (cudaMalloc(&p->dev_err, sizeof(block)) != cudaSuccess ||
      cudaMemcpy(p->dev_err, block, sizeof(block), cudaMemcpyHostToDevice) != cudaSuccess) {
    if (p->dev_err) cudaFree(p->dev_err);
    delete p;
    return fail(EXT_ERR_CUDA, "cannot allocate the plan status block");
  }
  if (const char* e = getenv("EXT_KCHUNK")) p->kchunk = atoi(e);
  if (const char* e = getenv("EXT_PIPELINED")) p->pipelined = atoi(e) != 0;
  if (const char* e = getenv("EXT_TMA")) p->tma = atoi(e) != 0;
  if (const char* e = getenv("EXT_SO3_WS")) p->so3_ws = atoi(e) != 0;
  if (const char* e = getenv("EXT_STEER_MODE")) p->steer_mode = atoi(e);
  if (const char* e = getenv("EXT_COLCONV")) p->colconv_form = atoi(e);
  if (const char* e = getenv("EXT_CONV_TOGETHER")) p->conv_together = atoi(e) != 0;
  if (const char* e = getenv("EXT_BATCH_BRANCHES")) p->batch_branches = atoi(e);
  if (p->autotune) tune_cache_read(p);
  *plan = p;
  return EXT_OK;
}

ext_status ext_plan_selftest_timeout(ext_plan plan, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  launch(plan, "selftest_timeout", st, [&] { launch_selftest_timeout(plan->dev_err, st); });
  EXT_CUDA(cudaGetLastError());
  return EXT_OK;
}

ext_status ext_select_components(const double* energy, int K, int budget, int* ks_out, int* n_out) {
  if (!energy || !ks_out || K < 0 || budget < 1) return fail(EXT_ERR_INVALID_ARG, "bad arguments");
  for (int k = 0; k <= K; ++k)
    if (energy[k] != energy[k]) return fail(EXT_ERR_INVALID_ARG, "NaN energy");
  std::vector<int> order;
  for (int k = 1; k <= K; ++k) order.push_back(k);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return energy[a] > energy[b]; });
  const int m = std::min(budget, K + 1) - 1;
  std::vector<int> chosen(order.begin(), order.begin() + m);
  std::sort(chosen.begin(), chosen.end());
  ks_out[0] = 0;
  for (int i = 0; i < m; ++i) ks_out[1 + i] = chosen[i];
  if (n_out) *n_out = m + 1;
  return EXT_OK;
}

ext_status ext_plan_trim(ext_plan plan) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_CUDA(cudaSetDevice(plan->device));
  EXT_CUDA(cudaDeviceSynchronize());
  for (auto& e : plan->specs) cudaFree(e.S);
  plan->specs.clear();
  for (auto& kv : plan->ws) cudaFree(kv.second.p);
  plan->ws.clear();
  // everything cached in the workspace is gone: the captured batch graph and
  // the SO(3) tables point into it
  if (plan->batch_exec) cudaGraphExecDestroy(plan->batch_exec);
  if (plan->batch_setup_exec) cudaGraphExecDestroy(plan->batch_setup_exec);
  plan->batch_exec = nullptr;
  plan->batch_setup_exec = nullptr;
  plan->batch_key = 0;
  plan->so3_rot_key = 0;
  plan->so3_grid_key = 0;
  plan->so3_steer_L = -1;
  return EXT_OK;
}

ext_status ext_plan_destroy(ext_plan plan) {
  if (!plan) return EXT_OK;
  cudaSetDevice(plan->device);
  cudaDeviceSynchronize();
  for (auto& e : plan->specs) cudaFree(e.S);
  for (auto& kv : plan->ws) cudaFree(kv.second.p);
  for (auto& kv : plan->twiddles) cudaFree(kv.second);
  for (auto& kv : plan->sweep_tables) cudaFree(kv.second);
  for (auto& p : plan->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : plan->event_pool) cudaEventDestroy(e);
  if (plan->batch_exec) cudaGraphExecDestroy(plan->batch_exec);
  if (plan->batch_setup_exec) cudaGraphExecDestroy(plan->batch_setup_exec);
  if (plan->pinned) cudaFreeHost(plan->pinned);
  cudaFree(plan->dev_err);
  delete plan;
  return EXT_OK;
}

ext_status ext_plan_sync(ext_plan plan, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_CUDA(cudaSetDevice(plan->device));
  EXT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return device_status(plan);
}

ext_status ext_plan_profile(ext_plan plan, int enable) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  plan->profiling = enable != 0;
  return EXT_OK;
}

ext_status ext_plan_profile_read(ext_plan plan, int n_max, char* names, double* total_ms, int64_t* launches,
                                 int* n_out) {
  if (!plan || !n_out) return fail(EXT_ERR_INVALID_ARG, "NULL argument");
  EXT_CUDA(cudaSetDevice(plan->device));
  for (auto& p : plan->pending) {
    EXT_CUDA(cudaEventSynchronize(p.b));
    float ms = 0.f;
    EXT_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
    ProfStat& stt = plan->prof[p.name];
    stt.ms += ms;
    stt.launches += 1;
    plan->event_pool.push_back(p.a);
    plan->event_pool.push_back(p.b);
  }
  plan->pending.clear();
  int n = 0;
  for (auto& kv : plan->prof) {
    if (n < n_max) {
      if (names) {
        std::strncpy(names + 64 * n, kv.first.c_str(), 63);
        names[64 * n + 63] = 0;
      }
      if (total_ms) total_ms[n] = kv.second.ms;
      if (launches) launches[n] = kv.second.launches;
    }
    ++n;
  }
  *n_out = n < n_max ? n : n_max;
  plan->prof.clear();
  return EXT_OK;
}

ext_status ext_filter_so2_decompose(ext_plan plan, const ext_filter_so2* F, double* fk_out, int64_t fk_cap,
                                    int* n_r_out) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_filter(F));
  if (!fk_out || !n_r_out) return fail(EXT_ERR_INVALID_ARG, "output is NULL");
  if (F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW)
    return fail(EXT_ERR_UNSUPPORTED, "analytic filters have no radial table");
  EXT_CUDA(cudaSetDevice(plan->device));
  const int nr = F->kind == EXT_FILTER_TABLE ? F->n_r : sampled_nr(F);
  const int64_t need = (int64_t)2 * (2 * F->K + 1) * nr;
  if (fk_cap < need) return fail(EXT_ERR_INVALID_ARG, "fk_out too small");
  cudaStream_t st = 0;
  const double2* coef = nullptr;
  int n_r = 0;
  double dr = 0;
  EXT_TRY(filter_coefficients(plan, F, st, &coef, &n_r, &dr));
  EXT_CUDA(cudaMemcpyAsync(fk_out, coef, sizeof(double) * need, cudaMemcpyDeviceToHost, st));
  EXT_CUDA(cudaStreamSynchronize(st));
  *n_r_out = n_r;
  return EXT_OK;
}

ext_status ext_corr_so2_components(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F,
                                   float* G, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_filter(F));
  EXT_TRY(check_size(h, w));
  if (h == 0 || w == 0) return EXT_OK;
  if (!H || !G) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)h * w;
  Staged sH, sG;
  EXT_TRY(stage_in(plan, "in_H", H, sizeof(float) * P, st, &sH));
  EXT_TRY(stage_out_alloc(plan, "out_G", G, sizeof(float) * P * (2 * F->K + 1), &sG));
  EXT_TRY(run_components_tuned(plan, (const float*)sH.dev, h, w, F, (float*)sG.dev, st));
  EXT_TRY(stage_out_finish(sG, st));
  return finish_host(plan, sH.host || sG.host, st);
}

ext_status ext_sweep_so2(ext_plan plan, const float* G, int64_t n_pix, int K, int n_angles, float* max_out,
                         int32_t* argmax, int precision, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  if (n_pix < 0 || K < 0 || n_angles < 1) return fail(EXT_ERR_INVALID_ARG, "bad sweep sizes");
  if (n_pix == 0) return EXT_OK;
  if (!G || !max_out || !argmax) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  Staged sG, sM, sA;
  EXT_TRY(stage_in(plan, "in_G", G, sizeof(float) * n_pix * (2 * K + 1), st, &sG));
  EXT_TRY(stage_out_alloc(plan, "out_max", max_out, sizeof(float) * n_pix, &sM));
  EXT_TRY(stage_out_alloc(plan, "out_arg", argmax, sizeof(int32_t) * n_pix, &sA));
  EXT_TRY(run_sweep(plan, (const float*)sG.dev, n_pix, K, n_angles, (float*)sM.dev, (int32_t*)sA.dev,
                    precision, st));
  EXT_TRY(stage_out_finish(sM, st));
  EXT_TRY(stage_out_finish(sA, st));
  return finish_host(plan, sG.host || sM.host || sA.host, st);
}

ext_status ext_corr_so2(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F, const float* alpha,
                        int n_angles, float* out_or_max, int32_t* argmax, int precision, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_filter(F));
  EXT_TRY(check_size(h, w));
  if (h == 0 || w == 0) return EXT_OK;
  if (!H || !out_or_max) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  if (!alpha) {
    if (n_angles < 1) return fail(EXT_ERR_INVALID_ARG, "sweep mode needs n_angles >= 1");
    if (!argmax) return fail(EXT_ERR_INVALID_ARG, "sweep mode needs argmax");
    precision = resolve_precision(plan, precision);
    if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3)
      return fail(EXT_ERR_INVALID_ARG, "unknown precision");
    if (F->K > 16) return fail(EXT_ERR_UNSUPPORTED, "sweep supports K <= 16");
  }
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)h * w;
  const int K = F->K;
  Staged sH, sAl, sO, sA;
  if (alpha) {
    EXT_TRY(stage_in(plan, "in_H", H, sizeof(float) * P, st, &sH));
    EXT_TRY(stage_out_alloc(plan, "out_0", out_or_max, sizeof(float) * P, &sO));
    EXT_TRY(stage_in(plan, "in_alpha", alpha, sizeof(float) * P, st, &sAl));
    const float2* S = nullptr;
    EXT_TRY(spectra(plan, F, h, w, SPEC_CORR, st, &S));
    const float2 *tw_w = nullptr, *tw_h = nullptr;
    EXT_TRY(twiddle(plan, w, st, &tw_w));
    EXT_TRY(twiddle(plan, h, st, &tw_h));
    const int wh = w / 2 + 1;
    void *Hh = nullptr, *Z = nullptr;
    EXT_TRY(ensure(plan, "Hh", sizeof(float2) * P / w * wh, &Hh));
    EXT_TRY(ensure(plan, "Zall", sizeof(float2) * P * (K + 1), &Z));
    launch(plan, "rows_r2c", st, [&] { fft_rows_r2c(w, (const float*)sH.dev, h, (float2*)Hh, tw_w, st); });
    launch(plan, "cols_fwd_half", st, [&] { fft_cols_fwd_half(h, (float2*)Hh, wh, tw_h, st); });
    launch(plan, "cols_inv_corr", st,
           [&] { fft_cols_inv_corr(h, (const float2*)Hh, w, S, 0, K + 1, (float2*)Z, tw_h, st); });
    launch(plan, "rows_inv_field", st,
           [&] { fft_rows_inv_field(w, (const float2*)Z, h, K, (const float*)sAl.dev, (float*)sO.dev, tw_w, st); });
    EXT_CUDA(cudaGetLastError());
    EXT_TRY(stage_out_finish(sO, st));
    return finish_host(plan, sH.host || sAl.host || sO.host, st);
  }
  // max and argmax are written once, by the sweep: page-locked host outputs are
  // written in place (K >= 1).  (Reading a page-locked H in place in the first row
  // pass measured no faster than the staged copy.)
  EXT_TRY(stage_in(plan, "in_H", H, sizeof(float) * P, st, &sH));
  Staged sM;
  if (K >= 1) {
    EXT_TRY(stage_out_direct(plan, "out_0", out_or_max, sizeof(float) * P, &sM));
    EXT_TRY(stage_out_direct(plan, "out_1", argmax, sizeof(int32_t) * P, &sA));
  } else {
    EXT_TRY(stage_out_alloc(plan, "out_0", out_or_max, sizeof(float) * P, &sM));
    EXT_TRY(stage_out_alloc(plan, "out_1", argmax, sizeof(int32_t) * P, &sA));
  }
  void* G = nullptr;
  EXT_TRY(ensure(plan, "G", sizeof(float) * P * (2 * K + 1), &G));
  EXT_TRY(run_components_tuned(plan, (const float*)sH.dev, h, w, F, (float*)G, st));
  EXT_TRY(run_sweep(plan, (const float*)G, (long long)P, K, n_angles, (float*)sM.dev, (int32_t*)sA.dev, precision,
                    st));
  EXT_TRY(stage_out_finish(sM, st));
  EXT_TRY(stage_out_finish(sA, st));
  return finish_host(plan, sH.host || sM.host || sA.host || sM.mapped || sA.mapped, st);
}

ext_status ext_corr_so2_subset(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F, const int* ks,
                               int nks, int n_angles, float* max_out, int32_t* argmax, int precision, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_filter(F));
  EXT_TRY(check_size(h, w));
  if (!ks || nks < 1 || nks > 17) return fail(EXT_ERR_INVALID_ARG, "component list must hold 1..17 entries");
  if (ks[0] != 0) return fail(EXT_ERR_INVALID_ARG, "the component list must start with 0");
  for (int i = 1; i < nks; ++i)
    if (ks[i] <= ks[i - 1] || ks[i] > F->K)
      return fail(EXT_ERR_INVALID_ARG, "components must ascend and lie in 1..K");
  if (n_angles < 1) return fail(EXT_ERR_INVALID_ARG, "n_angles must be >= 1");
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3)
    return fail(EXT_ERR_INVALID_ARG, "unknown precision");
  if (precision == EXT_PREC_BF16X3 && n_angles > 128)
    return fail(EXT_ERR_UNSUPPORTED, "BF16x3 sweep supports at most 128 angles");
  if (h == 0 || w == 0) return EXT_OK;
  if (!H || !max_out || !argmax) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)h * w;
  const int Ks = nks - 1;
  Staged sH, sM, sA;
  EXT_TRY(stage_in(plan, "in_H", H, sizeof(float) * P, st, &sH));
  if (Ks >= 1) {
    EXT_TRY(stage_out_direct(plan, "out_0", max_out, sizeof(float) * P, &sM));
    EXT_TRY(stage_out_direct(plan, "out_1", argmax, sizeof(int32_t) * P, &sA));
  } else {
    EXT_TRY(stage_out_alloc(plan, "out_0", max_out, sizeof(float) * P, &sM));
    EXT_TRY(stage_out_alloc(plan, "out_1", argmax, sizeof(int32_t) * P, &sA));
  }
  void* G = nullptr;
  EXT_TRY(ensure(plan, "G", sizeof(float) * P * (2 * Ks + 1), &G));
  EXT_TRY(run_components(plan, (const float*)sH.dev, h, w, F, (float*)G, st, ks, nks));
  if (Ks == 0) {   // only G_0: the same score at every angle, the first angle
    EXT_CUDA(cudaMemcpyAsync(sM.dev, G, sizeof(float) * P, cudaMemcpyDeviceToDevice, st));
    EXT_CUDA(cudaMemsetAsync(sA.dev, 0, sizeof(int32_t) * P, st));
  } else {
    const float* B = nullptr;
    int cp = 0;
    EXT_TRY(sweep_table_list(plan, ks, nks, n_angles, st, &B, &cp));
    bool ok = true;
    if (precision == EXT_PREC_BF16X3)
      launch(plan, "sweep_bf16x3", st, [&] {
        ok = sweep_bf16x3((const float*)G, (long long)P, Ks, n_angles, B, cp, (float*)sM.dev, (int32_t*)sA.dev,
                          plan->dev_err, plan->sms, st);
      });
    else if (!sweep_fp32_fits(Ks, n_angles))
      return fail(EXT_ERR_UNSUPPORTED, "FP32 sweep: the steering table of this many angles exceeds shared memory");
    else
      launch(plan, "sweep_fp32", st, [&] {
        ok = sweep_fp32((const float*)G, (long long)P, Ks, n_angles, B, cp, (float*)sM.dev, (int32_t*)sA.dev, st);
      });
    if (!ok) return fail(EXT_ERR_UNSUPPORTED, "sweep shape");
  }
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sM, st));
  EXT_TRY(stage_out_finish(sA, st));
  return finish_host(plan, sH.host || sM.host || sA.host || sM.mapped || sA.mapped, st);
}

ext_status ext_filter_so2_energy(ext_plan plan, const ext_filter_so2* F, double* energy_out) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_filter(F));
  if (!energy_out) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = 0;
  const double2* coef = nullptr;
  int n_r = 0;
  double dr = 0;
  EXT_TRY(filter_coefficients(plan, F, st, &coef, &n_r, &dr));
  const int kind = F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW ? EXT_FILTER_ANALYTIC_GAUSSPOW : EXT_FILTER_TABLE;
  void* E = nullptr;
  EXT_TRY(ensure(plan, "energy", sizeof(double) * (F->K + 1), &E));
  EXT_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * (F->K + 1), st));
  launch(plan, "component_energy", st, [&] {
    launch_component_energy(kind, F->K, coef, n_r, dr, F->sigma, F->R, (double*)E, st);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_CUDA(cudaMemcpyAsync(energy_out, E, sizeof(double) * (F->K + 1), cudaMemcpyDeviceToHost, st));
  EXT_CUDA(cudaStreamSynchronize(st));
  return EXT_OK;
}

ext_status ext_conv_so2(ext_plan plan, const float* H, int h, int w, const ext_filter_so2* F, const float* alpha,
                        float* out, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_filter(F));
  EXT_TRY(check_size(h, w));
  if (h == 0 || w == 0) return EXT_OK;
  if (!H || !alpha || !out) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)h * w;
  Staged sH, sAl, sO;
  EXT_TRY(stage_in(plan, "in_H", H, sizeof(float) * P, st, &sH));
  EXT_TRY(stage_in(plan, "in_alpha", alpha, sizeof(float) * P, st, &sAl));
  EXT_TRY(stage_out_alloc(plan, "out_0", out, sizeof(float) * P, &sO));
  EXT_TRY(run_conv_so2(plan, (const float*)sH.dev, (const float*)sAl.dev, h, w, F, (float*)sO.dev, st));
  EXT_TRY(stage_out_finish(sO, st));
  return finish_host(plan, sH.host || sAl.host || sO.host, st);
}

ext_status ext_conv_so2_normalized(ext_plan plan, const float* H, int channels, int h, int w, const ext_filter_so2* F,
                                   const float* alpha, float* out, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_filter(F));
  EXT_TRY(check_size(h, w));
  if (channels < 1 || channels > 64) return fail(EXT_ERR_INVALID_ARG, "channels must be in [1, 64]");
  if (h == 0 || w == 0) return EXT_OK;
  if (!H || !alpha || !out) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)h * w;
  Staged sH, sAl, sO;
  EXT_TRY(stage_in(plan, "in_H", H, sizeof(float) * P * channels, st, &sH));
  EXT_TRY(stage_in(plan, "in_alpha", alpha, sizeof(float) * P, st, &sAl));
  EXT_TRY(stage_out_alloc(plan, "out_0", out, sizeof(float) * P * channels, &sO));
  void* D = nullptr;
  EXT_TRY(ensure(plan, "norm_D", sizeof(float) * P, &D));
  // the channels and the denominator (the response to the constant signal 1,
  // the phase row pass's H = NULL) in one call, sharing the column pass
  std::vector<const float*> srcs;
  std::vector<float*> dsts;
  for (int c = 0; c < channels; ++c) {
    srcs.push_back((const float*)sH.dev + P * c);
    dsts.push_back((float*)sO.dev + P * c);
  }
  srcs.push_back(nullptr);
  dsts.push_back((float*)D);
  EXT_TRY(run_conv_so2_signals(plan, srcs.data(), dsts.data(), channels + 1, (const float*)sAl.dev, h, w, F, st));
  launch(plan, "divide_channels", st, [&] {
    launch_divide_channels((float*)sO.dev, (const float*)D, (long long)P, channels, plan->sms, st);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sO, st));
  return finish_host(plan, sH.host || sAl.host || sO.host, st);
}

ext_status ext_ght_detect(ext_plan plan, const float* I, int h, int w, const ext_filter_so2* F, float* out,
                          void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_filter(F));
  EXT_TRY(check_size(h, w));
  if (h == 0 || w == 0) return EXT_OK;
  if (!I || !out) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)h * w;
  Staged sI, sO;
  EXT_TRY(stage_in(plan, "in_I", I, sizeof(float) * P, st, &sI));
  // the response is written once, by the last row pass: page-locked host output in place
  EXT_TRY(stage_out_direct(plan, "out_0", out, sizeof(float) * P, &sO));
  void *Hs = nullptr, *Ts = nullptr;
  EXT_TRY(ensure(plan, "ght_H", sizeof(float) * P, &Hs));
  EXT_TRY(ensure(plan, "ght_theta", sizeof(float) * P, &Ts));
  launch(plan, "gradient_field", st,
         [&] { launch_gradient_field((const float*)sI.dev, h, w, (float*)Hs, (float*)Ts, plan->sms, st); });
  EXT_TRY(run_conv_so2(plan, (const float*)Hs, (const float*)Ts, h, w, F, (float*)sO.dev, st));
  EXT_TRY(stage_out_finish(sO, st));
  return finish_host(plan, sI.host || sO.host || sO.mapped, st);
}

ext_status ext_conv_scale(ext_plan plan, const float* H, int channels, int h, int w, const double* mellin_c, int n_h,
                          double log_period, double r_min, double r_max, double centre_tap, const float* s, int mode,
                          float* out, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_size(h, w));
  if (h == 0 || w == 0) return EXT_OK;
  if (!H || !s || !out || !mellin_c) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  if (channels < 1 || channels > 64) return fail(EXT_ERR_INVALID_ARG, "channels must be in [1, 64]");
  if (n_h < 1 || n_h > 256) return fail(EXT_ERR_INVALID_ARG, "n_h must be in [1, 256]");
  if (!(log_period > 0)) return fail(EXT_ERR_INVALID_ARG, "log_period must be > 0");
  if (!(r_min > 0) || !(r_max >= r_min) || r_max > 1024) return fail(EXT_ERR_INVALID_ARG, "need 0 < r_min <= r_max <= 1024");
  if (mode < 0 || mode > 2) return fail(EXT_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)h * w;
  Staged sH, sS, sO;
  EXT_TRY(stage_in(plan, "in_H", H, sizeof(float) * P * channels, st, &sH));
  EXT_TRY(stage_in(plan, "in_s", s, sizeof(float) * P, st, &sS));
  EXT_TRY(stage_out_alloc(plan, "out_0", out, sizeof(float) * P * channels, &sO));
  // spectra of the Mellin components (Sec. 8), cached per filter and size
  uint64_t key = 0x5ca1e5ca1e5ca1eull;
  key = fnv1a(key, mellin_c, sizeof(double) * 2 * n_h);
  key = fnv1a(key, &n_h, sizeof(int));
  key = fnv1a(key, &log_period, sizeof(double));
  key = fnv1a(key, &r_min, sizeof(double));
  key = fnv1a(key, &r_max, sizeof(double));
  const int R = (int)r_max;
  const double two_pi = 6.283185307179586476925286766559;
  auto sample = [&](int k0, int nk, float2* grid) {
    for (int k = k0; k < k0 + nk; ++k)
      launch_component_grid_mellin(make_double2(mellin_c[2 * k], mellin_c[2 * k + 1]), two_pi * k / log_period,
                                   r_min, r_max, R, h, w, grid + (size_t)(k - k0) * h * w, st);
  };
  const float2* S = nullptr;
  EXT_TRY(spectra_generic(plan, key, h, w, n_h, SPEC_CONV, st, sample, &S));
  void *Nb = nullptr, *Db = nullptr;
  EXT_TRY(ensure(plan, "Nscale", sizeof(float) * P * channels, &Nb));
  EXT_TRY(ensure(plan, "Dscale", sizeof(float) * P, &Db));
  const float omega_step = (float)(two_pi / log_period);
  const int unit = mode == 2 ? 1 : 0;
  void* Tt = nullptr;
  if (plan->steer_mode >= 1) {
    EXT_TRY(ensure(plan, "scale_turns", sizeof(float2) * P, &Tt));
    launch(plan, "scale_turns", st, [&] {
      launch_scale_turns((const float*)sS.dev, (long long)P, (float)(1.0 / log_period), unit, (float2*)Tt,
                         plan->sms, st);
    });
  }
  EXT_TRY(conv_signals(
      plan, h, w, n_h, channels + (mode == 0 ? 0 : 1), S, st, "rows_fwd_scale",
      [&](int sig, float2* A, const float2* tw_w) {
        const float* src = sig < channels ? (const float*)sH.dev + P * sig : nullptr;   // nullptr: the signal 1
        if (Tt && plan->steer_mode >= 2 &&
            fft_rows_fwd_hloop_scale(w, src, (const float2*)Tt, h, 0, n_h, A, tw_w, plan->sms, st,
                                     plan->steer_mode == 2))
          return;
        if (Tt)
          fft_rows_fwd_scale_turns(w, src, (const float2*)Tt, h, 0, n_h, A, tw_w, st);
        else
          fft_rows_fwd_scale(w, src, (const float*)sS.dev, h, 0, n_h, omega_step, unit, A, tw_w, st);
      },
      [&](int sig) { return sig < channels ? (float*)Nb + P * sig : (float*)Db; }));
  launch(plan, "scale_finalize", st, [&] {
    launch_scale_finalize((const float*)sH.dev, (const float*)sS.dev, (const float*)Nb, (const float*)Db, channels,
                          (long long)P, mode, (float)centre_tap, (float*)sO.dev, plan->sms, st);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sO, st));
  return finish_host(plan, sH.host || sS.host || sO.host, st);
}

ext_status ext_conv_similarity(ext_plan plan, const float* H, int channels, int h, int w, const double* coef, int K,
                               int n_h, double log_period, double r_min, double r_max, double centre_tap,
                               const float* alpha, const float* s, int mode, float* out, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  EXT_TRY(check_size(h, w));
  if (h == 0 || w == 0) return EXT_OK;
  if (!H || !alpha || !s || !out || !coef) return fail(EXT_ERR_INVALID_ARG, "NULL buffer");
  if (channels < 1 || channels > 64) return fail(EXT_ERR_INVALID_ARG, "channels must be in [1, 64]");
  if (K < 0 || K > 64) return fail(EXT_ERR_INVALID_ARG, "K must be in [0, 64]");
  if (n_h < 1 || n_h > 64) return fail(EXT_ERR_INVALID_ARG, "n_h must be in [1, 64]");
  if (!(log_period > 0)) return fail(EXT_ERR_INVALID_ARG, "log_period must be > 0");
  if (!(r_min > 0) || !(r_max >= r_min) || r_max > 1024) return fail(EXT_ERR_INVALID_ARG, "need 0 < r_min <= r_max <= 1024");
  if (mode < 0 || mode > 2) return fail(EXT_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
  const size_t P = (size_t)h * w;
  // unique harmonics up to the pairing (k, j) <-> (-k, -j): (0, 0), (0, j > 0), (k > 0, any j)
  const int nj = 2 * n_h - 1;
  std::vector<int2> kj;
  std::vector<double2> ck;
  for (int k = 0; k <= K; ++k)
    for (int j = (k == 0 ? 0 : -(n_h - 1)); j < n_h; ++j) {
      kj.push_back(make_int2(k, j));
      const size_t at = 2 * ((size_t)k * nj + (size_t)(j + n_h - 1));
      ck.push_back(make_double2(coef[at], coef[at + 1]));
    }
  const int ncomp = (int)kj.size();
  if (sizeof(float2) * P * ncomp > (8ull << 30))
    return fail(EXT_ERR_UNSUPPORTED, "steered spectra of all harmonics exceed 8 GiB");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  Staged sH, sA, sS, sO;
  EXT_TRY(stage_in(plan, "in_H", H, sizeof(float) * P * channels, st, &sH));
  EXT_TRY(stage_in(plan, "in_alpha", alpha, sizeof(float) * P, st, &sA));
  EXT_TRY(stage_in(plan, "in_s", s, sizeof(float) * P, st, &sS));
  EXT_TRY(stage_out_alloc(plan, "out_0", out, sizeof(float) * P * channels, &sO));
  void *dkj = nullptr, *dck = nullptr;
  EXT_TRY(ensure(plan, "simil_kj", sizeof(int2) * ncomp, &dkj));
  EXT_TRY(ensure(plan, "simil_coef", sizeof(double2) * ncomp, &dck));
  EXT_CUDA(cudaMemcpyAsync(dkj, kj.data(), sizeof(int2) * ncomp, cudaMemcpyHostToDevice, st));
  EXT_CUDA(cudaMemcpyAsync(dck, ck.data(), sizeof(double2) * ncomp, cudaMemcpyHostToDevice, st));
  // spectra of the harmonics, cached per filter and size
  uint64_t key = 0x5e5e5e1a1a1a1ull;
  key = fnv1a(key, ck.data(), sizeof(double2) * ncomp);
  key = fnv1a(key, &K, sizeof(int));
  key = fnv1a(key, &n_h, sizeof(int));
  key = fnv1a(key, &log_period, sizeof(double));
  key = fnv1a(key, &r_min, sizeof(double));
  key = fnv1a(key, &r_max, sizeof(double));
  const int R = (int)r_max;
  const double two_pi = 6.283185307179586476925286766559;
  auto sample = [&](int k0, int nk, float2* grid) {
    launch_component_grid_simil((const double2*)dck, (const int2*)dkj, k0, nk, two_pi / log_period, r_min, r_max, R,
                                h, w, grid, st);
  };
  const float2* S = nullptr;
  EXT_TRY(spectra_generic(plan, key, h, w, ncomp, SPEC_CONV, st, sample, &S));
  void *Nb = nullptr, *Db = nullptr, *UV = nullptr;
  EXT_TRY(ensure(plan, "Nscale", sizeof(float) * P * channels, &Nb));
  EXT_TRY(ensure(plan, "Dscale", sizeof(float) * P, &Db));
  EXT_TRY(ensure(plan, "simil_uv", sizeof(float4) * P, &UV));
  const float omega_step = (float)(two_pi / log_period);
  const int unit = mode == 2 ? 1 : 0;
  if (plan->steer_mode >= 1)
    launch(plan, "simil_turns", st, [&] {
      launch_simil_turns((const float*)sA.dev, (const float*)sS.dev, (long long)P, (float)(1.0 / log_period), unit,
                         (float4*)UV, plan->sms, st);
    });
  else
    launch(plan, "simil_phasors", st, [&] {
      launch_simil_phasors((const float*)sA.dev, (const float*)sS.dev, (long long)P, omega_step, (float4*)UV,
                           plan->sms, st);
    });
  EXT_TRY(conv_signals(
      plan, h, w, ncomp, channels + (mode == 0 ? 0 : 1), S, st, "rows_fwd_simil",
      [&](int sig, float2* A, const float2* tw_w) {
        const float* src = sig < channels ? (const float*)sH.dev + P * sig : nullptr;   // nullptr: the signal 1
        if (plan->steer_mode >= 2 &&
            fft_rows_fwd_hloop_simil(w, src, (const float4*)UV, h, (const int2*)dkj, ncomp, A, tw_w, plan->sms, st,
                                     plan->steer_mode == 2))
          return;
        if (plan->steer_mode >= 1)
          fft_rows_fwd_simil_turns(w, src, (const float4*)UV, h, (const int2*)dkj, ncomp, A, tw_w, st);
        else
          fft_rows_fwd_simil(w, src, (const float4*)UV, (const float*)sS.dev, h, (const int2*)dkj, ncomp, unit, A,
                             tw_w, st);
      },
      [&](int sig) { return sig < channels ? (float*)Nb + P * sig : (float*)Db; }));
  launch(plan, "scale_finalize", st, [&] {
    launch_scale_finalize((const float*)sH.dev, (const float*)sS.dev, (const float*)Nb, (const float*)Db, channels,
                          (long long)P, mode, (float)centre_tap, (float*)sO.dev, plan->sms, st);
  });
  EXT_CUDA(cudaGetLastError());
  EXT_TRY(stage_out_finish(sO, st));
  return finish_host(plan, sH.host || sA.host || sS.host || sO.host, st);
}

ext_status ext_batch_corr_so2(ext_plan plan, const ext_image_desc* imgs, int n, int precision, void* stream) {
  if (!plan) return fail(EXT_ERR_INVALID_ARG, "plan is NULL");
  if (n < 0 || (n > 0 && !imgs)) return fail(EXT_ERR_INVALID_ARG, "bad image list");
  if (n == 0) return EXT_OK;
  precision = resolve_precision(plan, precision);
  if (precision != EXT_PREC_FP32 && precision != EXT_PREC_BF16X3) return fail(EXT_ERR_INVALID_ARG, "unknown precision");
  EXT_CUDA(cudaSetDevice(plan->device));
  cudaStream_t st = (cudaStream_t)stream;
  // ---- validate, size the workspaces, pack the filter data
  size_t max_S = 0, max_grid = 0, max_Hh = 0, max_Hf = 0, max_Z = 0, max_G = 0, max_polar = 0;
  std::vector<size_t> off_in(n), off_coef(n);
  std::vector<int> nr(n);
  size_t host_bytes = 0, coef_bytes = 0;
  uint64_t key = 0xba7c4ba7c4ull;
  for (int i = 0; i < n; ++i) {
    const ext_image_desc& d = imgs[i];
    EXT_TRY(check_filter(d.F));
    EXT_TRY(check_size(d.h, d.w));
    if (d.h == 0 || d.w == 0) return fail(EXT_ERR_INVALID_ARG, "empty image in a batch");
    if (!d.H || !d.max_out || !d.argmax) return fail(EXT_ERR_INVALID_ARG, "NULL buffer in a batch");
    if (!is_device_ptr(d.H, plan->device) || !is_device_ptr(d.max_out, plan->device) ||
        !is_device_ptr(d.argmax, plan->device))
      return fail(EXT_ERR_INVALID_ARG, "batched images and outputs must be device buffers");
    const int K = d.F->K;
    if (d.n_angles < 1 || K > 16 || (precision == EXT_PREC_BF16X3 && d.n_angles > 128))
      return fail(EXT_ERR_UNSUPPORTED, "batched sweep supports K <= 16 and 1..128 angles (BF16x3)");
    const size_t P = (size_t)d.h * d.w;
    const int cw = fft_col_tile(d.h);
    max_S = std::max(max_S, sizeof(float2) * (size_t)(K + 1) * ((d.w + cw - 1) / cw) * d.h * cw);
    max_grid = std::max(max_grid, sizeof(float2) * P * std::min<size_t>(K + 1, std::max<size_t>(1, (512ull << 20) / (8 * P))));
    max_Hh = std::max(max_Hh, sizeof(float2) * (size_t)d.h * (d.w / 2 + 1));
    max_Hf = std::max(max_Hf, sizeof(float2) * P);
    max_Z = std::max(max_Z, sizeof(float2) * P * (K + 1));
    max_G = std::max(max_G, sizeof(float) * P * (2 * K + 1));
    const size_t nk = (size_t)(2 * K + 1);
    size_t in_bytes = 0;
    if (d.F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW) { in_bytes = sizeof(double2) * nk; nr[i] = 0; }
    else if (d.F->kind == EXT_FILTER_TABLE) { in_bytes = sizeof(double2) * nk * d.F->n_r; nr[i] = d.F->n_r; }
    else {
      const size_t side = 2 * d.F->R + 1;
      in_bytes = sizeof(double) * side * side;
      nr[i] = sampled_nr(d.F);
      max_polar = std::max(max_polar, sizeof(double) * nr[i] * d.F->n_theta);
    }
    off_in[i] = host_bytes;
    host_bytes += (in_bytes + 255) / 256 * 256;
    off_coef[i] = coef_bytes;
    coef_bytes += (sizeof(double2) * nk * std::max(nr[i], 1) + 255) / 256 * 256;
    const uint64_t fk = filter_key(d.F);
    key = fnv1a(key, &fk, sizeof(fk));
    key = fnv1a(key, &d, sizeof(d));
  }
  key = fnv1a(key, &precision, sizeof(int));
  // the template spectra of every image, kept in plan workspace while the batch stays the same
  std::vector<size_t> off_S(n);
  size_t spec_bytes = 0;
  for (int i = 0; i < n; ++i) {
    const ext_image_desc& d = imgs[i];
    const int cw = fft_col_tile(d.h);
    off_S[i] = spec_bytes;
    spec_bytes += (sizeof(float2) * (size_t)(d.F->K + 1) * ((d.w + cw - 1) / cw) * d.h * cw + 255) / 256 * 256;
  }
  (void)max_S;
  // independent images run on NB parallel branches of the graphs, each with its own workspace set
  constexpr int NBMAX = 32;
  const int nbr = std::max(1, std::min(NBMAX, plan->batch_branches));
  const int NB = n < nbr ? n : nbr;
  key = fnv1a(key, &NB, sizeof(int));
  std::string kGrid[NBMAX], kHh[NBMAX], kHf[NBMAX], kZ[NBMAX], kG[NBMAX], kP[NBMAX];
  void *dgrid[NBMAX], *dHh[NBMAX], *dHf[NBMAX], *dZ[NBMAX], *dG[NBMAX], *dpolar[NBMAX], *din, *dcoef, *dspec;
  for (int b = 0; b < NB; ++b) {
    const std::string t = std::to_string(b);
    kGrid[b] = "grid" + t;
    kHh[b] = "Hh" + t;
    kHf[b] = "Hf" + t;
    kZ[b] = "Z" + t;
    kG[b] = "G" + t;
    kP[b] = "fpolar" + t;
    EXT_TRY(ensure(plan, kGrid[b].c_str(), max_grid, &dgrid[b]));
    EXT_TRY(ensure(plan, kHh[b].c_str(), max_Hh, &dHh[b]));
    EXT_TRY(ensure(plan, kHf[b].c_str(), plan->tma || plan->autotune ? max_Hf : 16, &dHf[b]));
    EXT_TRY(ensure(plan, kZ[b].c_str(), max_Z, &dZ[b]));
    EXT_TRY(ensure(plan, kG[b].c_str(), max_G, &dG[b]));
    EXT_TRY(ensure(plan, kP[b].c_str(), std::max<size_t>(max_polar, 8), &dpolar[b]));
    for (void* q : {dgrid[b], dHh[b], dHf[b], dZ[b], dG[b], dpolar[b]}) key = fnv1a(key, &q, sizeof(q));
  }
  EXT_TRY(ensure(plan, "batch_in", host_bytes, &din));
  EXT_TRY(ensure(plan, "batch_coef", coef_bytes, &dcoef));
  EXT_TRY(ensure(plan, "batch_spectra", std::max<size_t>(spec_bytes, 256), &dspec));
  for (void* q : {din, dcoef, dspec}) key = fnv1a(key, &q, sizeof(q));
  // tables used inside the graphs are created beforehand
  for (int i = 0; i < n; ++i) {
    const float2* t;
    EXT_TRY(twiddle(plan, imgs[i].w, st, &t));
    EXT_TRY(twiddle(plan, imgs[i].h, st, &t));
    if (imgs[i].F->K > 0) {
      const float* B;
      int cp;
      EXT_TRY(sweep_table(plan, imgs[i].F->K, imgs[i].n_angles, st, &B, &cp));
    }
  }
  const bool fresh = plan->batch_exec == nullptr || plan->batch_setup_exec == nullptr || plan->batch_key != key;
  if (fresh) {
    // ---- upload the filter data (the setup graph reads it from batch_in)
    plan->batch_host.resize(std::max<size_t>(host_bytes, 1));
    for (int i = 0; i < n; ++i) {
      const ext_filter_so2* F = imgs[i].F;
      const size_t nk = (size_t)(2 * F->K + 1);
      unsigned char* dst = plan->batch_host.data() + off_in[i];
      if (F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW) std::memcpy(dst, F->a, sizeof(double2) * nk);
      else if (F->kind == EXT_FILTER_TABLE) std::memcpy(dst, F->fk, sizeof(double2) * nk * F->n_r);
      else std::memcpy(dst, F->img, sizeof(double) * (2 * F->R + 1) * (2 * F->R + 1));
    }
    EXT_CUDA(cudaMemcpyAsync(din, plan->batch_host.data(), host_bytes, cudaMemcpyHostToDevice, st));
    EXT_CUDA(cudaStreamSynchronize(st));   // the host staging buffer is reused by the next call
  }
  // ---- autotuning: every new shape class is tuned on its first image
  if (plan->autotune) {
    for (int i = 0; i < n; ++i) {
      const ext_image_desc& d = imgs[i];
      if (plan->tuned.count(class_key(d.h, d.w, d.F->K))) continue;
      PassVariant v;
      EXT_TRY(tune_components(plan, d.H, d.h, d.w, d.F, (float*)dG[0], st, &v));
    }
  }
  // ---- capture the per-image launch sequences once (setup: filter decomposition and template
  // spectra; step: forward transform, inverse correlation passes, sweep), then replay
  // branch of each image: largest images first, each to the least-loaded branch (work ~ (K+1) h w)
  std::vector<int> branch(n, 0);
  {
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto cost = [&](int i) { return (double)(imgs[i].F->K + 1) * imgs[i].h * imgs[i].w; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<double> load(NB, 0.0);
    for (int i : order) {
      const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      branch[i] = b;
      load[b] += cost(i);
    }
  }
  auto capture = [&](bool setup, cudaGraphExec_t* out) -> ext_status {
    const bool profiling = plan->profiling;
    plan->profiling = false;   // no event records inside the graph
    cudaStream_t cs = nullptr, br[NBMAX] = {};
    cudaEvent_t fork = nullptr, join[NBMAX] = {};
    EXT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    for (int b = 0; b < NB; ++b) {
      EXT_CUDA(cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking));
      EXT_CUDA(cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming));
    }
    EXT_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    EXT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    EXT_CUDA(cudaEventRecord(fork, cs));
    for (int b = 0; b < NB; ++b) EXT_CUDA(cudaStreamWaitEvent(br[b], fork, 0));
    ext_status ss = EXT_OK;
    for (int i = 0; i < n && ss == EXT_OK; ++i) {
      const int b = branch[i];
      cudaStream_t bs = br[b];
      const ext_image_desc& d = imgs[i];
      const ext_filter_so2* F = d.F;
      const int K = F->K, h = d.h, w = d.w;
      const size_t P = (size_t)h * w;
      float2* Si = (float2*)((unsigned char*)dspec + off_S[i]);
      if (setup) {
        const double2* coef = (const double2*)((unsigned char*)din + off_in[i]);
        if (F->kind == EXT_FILTER_SAMPLED) {
          double2* table = (double2*)((unsigned char*)dcoef + off_coef[i]);
          launch_decompose_sampled((const double*)coef, 2 * F->R + 1, F->dr, nr[i], F->n_theta, K, (double*)dpolar[b],
                                   table, bs);
          coef = table;
        }
        const int kind = F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW ? EXT_FILTER_ANALYTIC_GAUSSPOW : EXT_FILTER_TABLE;
        const double dr = F->kind == EXT_FILTER_ANALYTIC_GAUSSPOW ? 0.0 : F->dr;
        auto sample = [&](int k0, int nk, float2* grid) {
          launch_component_grid(kind, K, k0, coef, nr[i], dr, F->sigma, F->R, h, w, grid, bs, nk);
        };
        ss = build_spectra(plan, h, w, K + 1, SPEC_CORR, bs, sample, Si, kGrid[b].c_str());
        continue;
      }
      PassVariant v;
      v.tma = plan->tma;
      v.pipelined = plan->pipelined;
      v.kchunk = plan->kchunk;
      if (plan->autotune) {
        auto it = plan->tuned.find(class_key(h, w, K));
        if (it != plan->tuned.end()) v = parse_variant(it->second);
      }
      VariantScope scope(plan, v);
      const float2 *tw_w = nullptr, *tw_h = nullptr;
      twiddle(plan, w, bs, &tw_w);
      twiddle(plan, h, bs, &tw_h);
      const int wh = w / 2 + 1;
      bool done = false;
      const int cw = fft_col_tile(h);
      const int brows = plan->tma && fft_cols_tma_ok(h) ? tma_rows(h, cw) : 0;
      CUtensorMap tmH;
      const bool tma_ok = brows > 0 && spectrum_tmap((const float2*)dHf[b], h, w, cw, brows, &tmH);
      fft_rows_r2c(w, d.H, h, (float2*)dHh[b], tw_w, bs);
      fft_cols_fwd_half(h, (float2*)dHh[b], wh, tw_h, bs, tma_ok ? (float2*)dHf[b] : nullptr, w);
      if (tma_ok)
        done = fft_cols_inv_corr_tma(h, tmH, w, brows, Si, 0, K + 1, (float2*)dZ[b], tw_h, plan->dev_err, plan->sms, bs);
      if (!done && (!plan->pipelined ||
                    !fft_cols_inv_corr_pipe(h, (const float2*)dHh[b], w, Si, 0, K + 1, (float2*)dZ[b], tw_h, plan->sms,
                                            bs)))
        fft_cols_inv_corr(h, (const float2*)dHh[b], w, Si, 0, K + 1, (float2*)dZ[b], tw_h, bs);
      if (!plan->pipelined || !fft_rows_inv_components_pipe(w, (const float2*)dZ[b], h, 0, K + 1, (float*)dG[b], tw_w,
                                                            plan->dev_err, plan->sms, bs))
        fft_rows_inv_components(w, (const float2*)dZ[b], h, 0, K + 1, (float*)dG[b], tw_w, bs);
      ss = run_sweep(plan, (const float*)dG[b], (long long)P, K, d.n_angles, d.max_out, d.argmax, precision, bs);
    }
    for (int b = 0; b < NB; ++b) {
      cudaEventRecord(join[b], br[b]);
      cudaStreamWaitEvent(cs, join[b], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    plan->profiling = profiling;
    cudaStreamDestroy(cs);
    for (int b = 0; b < NB; ++b) {
      cudaStreamDestroy(br[b]);
      cudaEventDestroy(join[b]);
    }
    cudaEventDestroy(fork);
    if (ss != EXT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return ss;
    }
    if (ce != cudaSuccess) return fail(EXT_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(EXT_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(ce));
    return EXT_OK;
  };
  if (fresh) {
    for (cudaGraphExec_t* g : {&plan->batch_exec, &plan->batch_setup_exec})
      if (*g) {
        EXT_CUDA(cudaGraphExecDestroy(*g));
        *g = nullptr;
      }
    plan->batch_key = 0;
    EXT_TRY(capture(true, &plan->batch_setup_exec));
    EXT_TRY(capture(false, &plan->batch_exec));
    plan->prof["batch_setup_graph"].launches += 1;
    EXT_CUDA(cudaGraphLaunch(plan->batch_setup_exec, st));
    plan->batch_key = key;
  }
  plan->prof["batch_graph"].launches += 1;
  EXT_CUDA(cudaGraphLaunch(plan->batch_exec, st));
  return EXT_OK;
}

}  // extern "C"
