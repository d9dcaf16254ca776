// Device-memory estimates used for admission by the request server: the
// bytes one decomposition holds on the device while it runs.
#pragma once
#include <cstdint>
#include <vector>

namespace ssa {

// ssa_embed_plan + ssa_decompose of one series (default Krylov dimension)
int64_t plan_path_bytes(int64_t N, int64_t L, int k, int precision);

// one ssa_decompose_batch call over the given series (N, L, k each)
struct BatchItem {
  int64_t N, L;
  int k;
};
int64_t batch_path_bytes(const std::vector<BatchItem>& items, int refine);
// a series can run in the batched engine
bool batch_eligible(int64_t N, int64_t L, int k, int precision);

// raise (never lower) the freed device memory that the library's own stream-ordered pool keeps
// for reuse on the current device (default 4 GiB); the request server keeps its whole budget
void lib_pool_keep(uint64_t bytes);

}  // namespace ssa

// device array of all left vectors of a batch (series after series, each
// L x k column-major in submission order); valid until ssa_batch_destroy
typedef struct ssa_batch_s* ssa_batch_t;
namespace ssa {
const double* batch_device_U(ssa_batch_t b);

}  // namespace ssa
