// The plan object behind the C ABI and the helpers every operator uses:
// workspace, per-kernel launch accounting, host/device staging of arguments
// and the device status word.
#pragma once
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>   // header-only NVTX v3: ranges cost nothing unless a profiler is attached

#include "internal.h"

namespace {

inline ext_status fail(ext_status s, const std::string& msg) {
  ext_set_error(msg.c_str());
  return s;
}

#define EXT_CUDA(call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? EXT_ERR_OOM : EXT_ERR_CUDA,                    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                              \
    }                                                                                               \
  } while (0)

#define EXT_TRY(expr)                  \
  do {                                 \
    ext_status s_ = (expr);            \
    if (s_ != EXT_OK) return s_;       \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct SpecEntry {
  uint64_t key = 0;
  float2* S = nullptr;
  size_t bytes = 0;
  uint64_t stamp = 0;
};

uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace
struct ProfStat {
  double ms = 0.0;
  int64_t launches = 0;
};

struct ProfPending {
  std::string name;
  cudaEvent_t a, b;
};

struct ext_plan_s {
  int device = 0;
  bool profiling = false;
  std::map<std::string, ProfStat> prof;
  std::vector<ProfPending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::map<int, float2*> twiddles;
  std::map<std::string, DevBuf> ws;
  std::vector<SpecEntry> specs;
  std::map<uint64_t, float*> sweep_tables;
  uint64_t clock = 0;
  size_t max_specs = 4;
  int sms = 0;           // multiprocessors of the device
  int kchunk = 0;        // components per inverse launch (0 = by L2 budget)
  bool pipelined = true; // persistent prefetching passes where they fit
  bool tma = true;       // tensor-memory-accelerator staged column pass where it fits
  bool so3_ws = true;    // warp-specialised SO(3) sweep for many voxels
  bool conv_together = true; // all signals of a convolution through one column-pass launch (workspace permitting)
  int colconv_form = 2;    // convolution column pass: 1 products through shared memory, 2 fused into the last stage
  int steer_mode = 2;      // steered row passes: 0 staged lines, 1 steering in the first stage's loads,
                           // 2 component loop (hardware sine/cosine), 3 component loop (sincospif)
  int batch_branches = 4; // parallel graph branches of the batched correlation (4: measured best of 1-16)
  int* dev_err = nullptr; // device-side status block: int status word, then (byte 8) the wait budget in ns
  int precision = EXT_PREC_FP32;        // used where a call passes EXT_PREC_DEFAULT
  unsigned long long wait_budget_ns = 1000000000ull;
  int fault_inject = EXT_FAULT_NONE;    // host-side fault injection (tests of the error paths)
  long long fault_countdown = -1;       // allocations left before the injected failure (-1: none)
  // autotuner: chosen pass variant per shape class, and where the cache lives
  bool autotune = false;
  std::string tune_cache;
  std::map<std::string, std::string> tuned;   // shape-class key -> "tma pipelined kchunk ms"
  // batched correlation: captured CUDA graph of the last batch and its key
  cudaGraphExec_t batch_exec = nullptr;         // per step: forward transforms, correlations, sweeps
  cudaGraphExec_t batch_setup_exec = nullptr;   // once per batch: filter decomposition, template spectra
  uint64_t batch_key = 0;
  std::vector<unsigned char> batch_host;   // packed filter data (host staging)
  // SO(3): steering tables of the last rotation set
  uint64_t so3_rot_key = 0;
  uint64_t so3_grid_key = 0;       // direction set of the grid sweep's cached rows
  int so3_rot_n = 0, so3_rot_L = -1;
  int so3_steer_L = -1;            // degree of the steering-entry table in workspace "so3_steer"
  int* pinned = nullptr;           // small pinned host buffer for counts read back mid-call
};

namespace {

cudaEvent_t take_event(ext_plan plan) {
  if (!plan->event_pool.empty()) {
    cudaEvent_t e = plan->event_pool.back();
    plan->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Every kernel launch of the operators goes through here: it is counted per
// kernel name and, when profiling is on, bracketed by events on its stream.
template <typename F>
void launch(ext_plan plan, const char* name, cudaStream_t st, F&& f) {
  struct Range {   // an NVTX range named after the kernel around its launch (tracing tools)
    explicit Range(const char* n) { nvtxRangePushA(n); }
    ~Range() { nvtxRangePop(); }
  } range(name);
  if (!plan->profiling) {
    plan->prof[name].launches += 1;
    f();
    return;
  }
  ProfPending p;
  p.name = name;
  p.a = take_event(plan);
  p.b = take_event(plan);
  cudaEventRecord(p.a, st);
  f();
  cudaEventRecord(p.b, st);
  plan->pending.push_back(p);
}

// Every device allocation of a plan goes through here, so that an injected
// allocation failure (ext_options.fault_inject) takes the same error path as
// a real one.
ext_status plan_malloc(ext_plan plan, void** p, size_t bytes) {
  if (plan->fault_inject == EXT_FAULT_ALLOC && plan->fault_countdown >= 0) {
    if (plan->fault_countdown == 0) {
      plan->fault_countdown = -1;
      *p = nullptr;
      return fail(EXT_ERR_OOM, "device allocation failed (injected by ext_options.fault_inject)");
    }
    --plan->fault_countdown;
  }
  EXT_CUDA(cudaMalloc(p, bytes));
  return EXT_OK;
}

int resolve_precision(ext_plan plan, int precision) {
  return precision == EXT_PREC_DEFAULT ? plan->precision : precision;
}

ext_status ensure(ext_plan plan, const char* name, size_t bytes, void** out) {
  DevBuf& b = plan->ws[name];
  if (b.bytes < bytes) {
    if (b.p) EXT_CUDA(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
    EXT_TRY(plan_malloc(plan, &b.p, bytes));
    b.bytes = bytes;
  }
  *out = b.p;
  return EXT_OK;
}

ext_status twiddle(ext_plan plan, int n, cudaStream_t st, const float2** out) {
  auto it = plan->twiddles.find(n);
  if (it == plan->twiddles.end()) {
    float2* tw = nullptr;
    EXT_TRY(plan_malloc(plan, (void**)&tw, sizeof(float2) * n));
    launch_twiddle(tw, n, st);
    EXT_CUDA(cudaGetLastError());
    it = plan->twiddles.emplace(n, tw).first;
  }
  *out = it->second;
  return EXT_OK;
}

// Rows per tensor copy of the H tile: a divisor of h, at most 256, whose box
// (br rows x cw complex) is a multiple of 128 bytes; 0 if none.
int tma_rows(int h, int cw) {
  for (int br = 256; br >= 1; --br)
    if (h % br == 0 && (br * cw * 8) % 128 == 0) return br;
  return 0;
}

// Stage twiddle table of length n in device memory (cached in the twiddle map
// under the key -n), for passes whose shared memory has no room for a copy.
ext_status stage_table(ext_plan plan, int n, cudaStream_t st, const float2** out) {
  auto it = plan->twiddles.find(-n);
  if (it == plan->twiddles.end()) {
    const float2* tw = nullptr;
    EXT_TRY(twiddle(plan, n, st, &tw));
    float2* t = nullptr;
    EXT_TRY(plan_malloc(plan, (void**)&t, sizeof(float2) * n));
    fft_build_stage_table(n, tw, t, st);
    EXT_CUDA(cudaGetLastError());
    it = plan->twiddles.emplace(-n, t).first;
  }
  *out = it->second;
  return EXT_OK;
}

// 1: device (or managed) memory the kernels of `device` can use; 0: host
// memory (pageable or page-locked); -1: device memory of another GPU.
int pointer_kind(const void* p, int device) {
  if (!p) return 0;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type == cudaMemoryTypeManaged) return 1;
  if (at.type == cudaMemoryTypeDevice) return at.device == device ? 1 : -1;
  return 0;
}

bool is_device_ptr(const void* p, int device) { return pointer_kind(p, device) == 1; }

ext_status foreign_device(const char* name) {
  return fail(EXT_ERR_INVALID_ARG, std::string(name) + ": device buffer on another GPU than the plan's");
}

// Host/device staging of one argument.
struct Staged {
  const void* user = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
  bool host = false;     // staged through a device buffer and copied
  bool mapped = false;   // page-locked host memory written in place through its device mapping
};

ext_status stage_in(ext_plan plan, const char* name, const void* user, size_t bytes, cudaStream_t st,
                    Staged* s) {
  s->user = user;
  s->bytes = bytes;
  const int kind = pointer_kind(user, plan->device);
  if (kind < 0) return foreign_device(name);
  s->host = user && kind == 0;
  if (!s->host) {
    s->dev = const_cast<void*>(user);
    return EXT_OK;
  }
  EXT_TRY(ensure(plan, name, bytes, &s->dev));
  EXT_CUDA(cudaMemcpyAsync(s->dev, user, bytes, cudaMemcpyHostToDevice, st));
  return EXT_OK;
}

ext_status stage_out_alloc(ext_plan plan, const char* name, void* user, size_t bytes, Staged* s) {
  s->user = user;
  s->bytes = bytes;
  const int kind = pointer_kind(user, plan->device);
  if (kind < 0) return foreign_device(name);
  s->host = user && kind == 0;
  if (!s->host) {
    s->dev = user;
    return EXT_OK;
  }
  return ensure(plan, name, bytes, &s->dev);
}

// An output written exactly once, by plain stores of the call's last kernel:
// page-locked host memory with a device mapping is written in place, so the
// transfer to the host overlaps that kernel instead of following it as a
// copy; other host memory is staged as usual.
ext_status stage_out_direct(ext_plan plan, const char* name, void* user, size_t bytes, Staged* s) {
  if (user && !is_device_ptr(user, plan->device)) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, user) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
      s->user = user;
      s->bytes = bytes;
      s->dev = at.devicePointer;
      s->host = false;
      s->mapped = true;
      return EXT_OK;
    }
    cudaGetLastError();
  }
  return stage_out_alloc(plan, name, user, bytes, s);
}

ext_status stage_out_finish(const Staged& s, cudaStream_t st) {
  if (!s.host) return EXT_OK;
  EXT_CUDA(cudaMemcpyAsync(const_cast<void*>(s.user), s.dev, s.bytes, cudaMemcpyDeviceToHost, st));
  return EXT_OK;
}

// G_k = H (*) F_k for k = 0..K into G (device, (2K+1) planes).
ext_status device_status(ext_plan plan) {
  int e = 0;
  EXT_CUDA(cudaMemcpy(&e, plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    EXT_CUDA(cudaMemset(plan->dev_err, 0, sizeof(int)));
    return fail(e, "a device-side wait timed out; results of the affected call are invalid");
  }
  return EXT_OK;
}

ext_status finish_host(ext_plan plan, bool any_host, cudaStream_t st) {
  if (any_host) {
    // the status word rides on the stream with the outputs: one synchronisation
    if (!plan->pinned) EXT_CUDA(cudaMallocHost(&plan->pinned, 64));
    int* word = plan->pinned + 15;
    EXT_CUDA(cudaMemcpyAsync(word, plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    EXT_CUDA(cudaStreamSynchronize(st));
    if (*word != 0) {
      const int e = *word;
      EXT_CUDA(cudaMemset(plan->dev_err, 0, sizeof(int)));
      return fail((ext_status)e, "a device-side wait timed out; results of the affected call are invalid");
    }
  }
  return EXT_OK;
}

}  // namespace
