// bf16 tensor-core (tcgen05) distance GEMM with fused top-K: not built yet.
#include "common.cuh"
#include "knn.cuh"

namespace ssg {

bool knn_tc_available() { return false; }

void knn_exact_tc(const float*, int64_t, int, const float*, const float*, int64_t, int,
                  const float*, int, int, int, int32_t*, float*, cudaStream_t, StageTimer*) {
  set_error("bf16 tensor-core kNN is not available");
  throw Fail{SSG_EINTERNAL};
}

}  // namespace ssg
