// Launch tracing for measurement (ia_profile_begin / ia_profile_end in
// include/ia_measure.h).  While a profile is open on the calling host thread,
// every launch site wrapped in a KernelSpan records one CUDA event before and
// one after its launch, on the launch's own stream; ia_profile_end turns the
// pairs into per-kernel launch counts and device times.  With no profile open
// a KernelSpan costs one thread-local load.
#pragma once

#include <cuda_runtime.h>

namespace ia {

class KernelSpan {
 public:
  KernelSpan(const char* name, cudaStream_t s);  // name: a string literal
  ~KernelSpan();
  KernelSpan(const KernelSpan&) = delete;
  KernelSpan& operator=(const KernelSpan&) = delete;

 private:
  cudaStream_t s_;
  int rec_;  // index of this launch's record, -1 when not profiling
};

}  // namespace ia
