// Tensor-core (tcgen05) pair engine for sm_103a.
#include "ftk_internal.h"
#include "tc_engine.h"

namespace ftk {

bool tc_supported(const ftk_plan_s*) { return false; }
size_t tc_pair_bytes(const ftk_plan_s*) { return 0; }
int tc_template_quantum(const ftk_plan_s*) { return 1; }
cudaError_t tc_build_tables(ftk_plan_s*, const std::vector<float2>&) { return cudaSuccess; }
void tc_free_tables(ftk_plan_s*) {}
ftk_status tc_run_chunk(ftk_plan_s*, int, const float2*, int, const float2*, int, int, int, int, float2*, char*,
                        float*, unsigned long long*, cudaStream_t) {
  return FTK_ERR_UNSUPPORTED;
}

}  // namespace ftk
