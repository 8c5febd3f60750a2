// Internal profiling hooks (see dpp_profile.cu).
#pragma once

#include <cuda_runtime.h>

namespace dpp {

enum ProfCat {
  kProfPanel = 0,
  kProfUpdateFp64 = 1,
  kProfUpdateF32 = 2,
  kProfUpdateTc = 3,
  kProfConvert = 4,
  kProfRecompute = 5,
  kProfOther = 6,
  kProfBatched = 7,
  kProfAdjoint = 8,
  kProfLEnsemble = 9,
  kProfBelow = 10,
  kProfElementary = 11,
  kProfCategories = 12
};

// Counts one launch; while profiling is on, records an event pair around the
// scope on stream `s` with the launch's algorithmic flops and bytes.
class ProfScope {
 public:
  ProfScope(int cat, cudaStream_t s, double flops = 0.0, double bytes = 0.0);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int idx_;
  cudaStream_t s_;
};

void count_launch(unsigned n);

}  // namespace dpp
