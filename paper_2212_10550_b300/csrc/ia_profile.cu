// Launch tracing for measurement: per-kernel device times from CUDA events.
#include <cstring>
#include <string>
#include <vector>

#include "ia.h"
#include "ia_measure.h"
#include "ia_profile.h"

namespace ia {
namespace {

struct Record {
  const char* name;
  cudaEvent_t start, stop;
};

struct Profile {
  bool open = false;
  std::vector<Record> recs;
  std::vector<cudaEvent_t> pool;  // events of closed profiles, reused
  cudaError_t err = cudaSuccess;  // first failure while recording

  cudaEvent_t event() {
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess && err == cudaSuccess) err = r;
    return r == cudaSuccess ? e : nullptr;
  }
};

thread_local Profile g_profile;

}  // namespace

KernelSpan::KernelSpan(const char* name, cudaStream_t s) : s_(s), rec_(-1) {
  Profile& p = g_profile;
  if (!p.open) return;
  Record r{name, p.event(), p.event()};
  if (!r.start || !r.stop) return;
  cudaError_t e = cudaEventRecord(r.start, s);
  if (e != cudaSuccess) {
    if (p.err == cudaSuccess) p.err = e;
    return;
  }
  rec_ = (int)p.recs.size();
  p.recs.push_back(r);
}

KernelSpan::~KernelSpan() {
  if (rec_ < 0) return;
  Profile& p = g_profile;
  cudaError_t e = cudaEventRecord(p.recs[rec_].stop, s_);
  if (e != cudaSuccess && p.err == cudaSuccess) p.err = e;
}

}  // namespace ia

namespace {
thread_local std::string g_profile_err;
}

extern "C" {

const char* ia_profile_error(void) { return g_profile_err.c_str(); }

ia_status ia_profile_begin(void) {
  ia::Profile& p = ia::g_profile;
  if (p.open) {
    g_profile_err = "a profile is already open on this thread";
    return IA_ERR_STATE;
  }
  p.open = true;
  p.err = cudaSuccess;
  p.recs.clear();
  return IA_OK;
}

ia_status ia_profile_end(ia_kernel_time* out, int max_out, int* n_out) {
  ia::Profile& p = ia::g_profile;
  if (!p.open) {
    g_profile_err = "no profile is open on this thread";
    return IA_ERR_STATE;
  }
  if (max_out < 0 || (max_out > 0 && !out) || !n_out) {
    g_profile_err = "bad output arguments";
    return IA_ERR_ARG;
  }
  p.open = false;
  ia_status st = IA_OK;
  std::vector<ia_kernel_time> acc;
  for (const ia::Record& r : p.recs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.stop);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
    if (e != cudaSuccess) {
      g_profile_err = std::string("event timing failed: ") + cudaGetErrorString(e);
      st = IA_ERR_CUDA;
      break;
    }
    ia_kernel_time* k = nullptr;
    for (auto& a : acc)
      if (std::strncmp(a.name, r.name, sizeof(a.name)) == 0) k = &a;
    if (!k) {
      acc.push_back(ia_kernel_time{});
      k = &acc.back();
      std::strncpy(k->name, r.name, sizeof(k->name) - 1);
    }
    k->launches += 1;
    k->total_ms += ms;
    if (ms > k->max_ms) k->max_ms = ms;
  }
  for (const ia::Record& r : p.recs) {
    p.pool.push_back(r.start);
    p.pool.push_back(r.stop);
  }
  p.recs.clear();
  if (st == IA_OK && p.err != cudaSuccess) {
    g_profile_err = std::string("event recording failed: ") + cudaGetErrorString(p.err);
    st = IA_ERR_CUDA;
  }
  *n_out = (int)acc.size();
  for (int i = 0; i < (int)acc.size() && i < max_out; ++i) out[i] = acc[i];
  return st;
}

}  // extern "C"
