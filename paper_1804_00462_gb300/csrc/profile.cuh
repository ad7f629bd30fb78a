// Launch accounting hooks (profile.cu).
#pragma once
#include <cuda_runtime.h>

namespace sorsvd {

// kernel classes reported by sorsvd_profile_end (same numbering as the header)
enum KClass { K_GAUSSIAN = 0, K_PASS = 1, K_CORE = 2, K_SMALL_GEMM = 3, K_REDUCE = 4, K_CHOL = 5,
              K_JACOBI = 6, K_MISC = 7, K_PASS_SPLIT = 8, K_RPCA = 9, K_NCLASS = 10 };

void count_launches(int n);
int prof_start(int cls, cudaStream_t st);   // -1 when profiling is off
void prof_stop(int slot, cudaStream_t st);

// RAII scope: counts `n` launches and brackets them with an event pair.
struct ProfScope {
  int slot;
  cudaStream_t st;
  ProfScope(int cls, cudaStream_t s, int n = 1) : slot(prof_start(cls, s)), st(s) { count_launches(n); }
  ~ProfScope() { prof_stop(slot, st); }
};

}  // namespace sorsvd
