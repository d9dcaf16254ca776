// Per-kernel launch accounting: a launch counter and optional CUDA-event
// timing around every kernel launch, with the algorithmic bytes and flops
// each launch is charged (used for roofline reporting).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ssa {

enum KClass {
  K_SPECTRUM = 0,
  K_MATVEC_SMALL,
  K_MATVEC_COLFWD,
  K_MATVEC_ROW,
  K_MATVEC_COLINV,
  K_PROJ,
  K_UPDATE,
  K_UPDATE_PROJ,
  K_NORMALIZE,
  K_SMALL_SVD,
  K_SVD_PRE,
  K_RITZ,
  K_HANKEL_SMALL,
  K_HANKEL_FS,
  K_MISC,
  K_SKIPPED,  // launches of passes that the device decided to skip (no bytes)
  K_BATCH,
  K_NCLASS
};

void prof_begin(cudaStream_t s);
void prof_end(cudaStream_t s, int cls, double bytes, double flops, int launches = 1);
void prof_flush();
bool prof_enabled();
// launches counted on the calling thread (for the launch count of a captured CUDA graph), and
// launches replayed from such a graph
uint64_t prof_thread_launches();
void prof_add_launches(uint64_t n);
void prof_sub_launches(uint64_t n);
// while on (this thread), launches are counted but not timed (no host allocation)
void prof_suppress(bool on);
void host_set_error(const char* msg);

}  // namespace ssa
