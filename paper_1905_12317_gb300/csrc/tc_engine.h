// Tensor-core (tcgen05) pair engine: interface used by the C-ABI layer.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "ftk_internal.h"

namespace ftk {

// Whether the plan's sizes fit the tcgen05 kernels.
bool tc_supported(const ftk_plan_s* p);
// Extra per-pair scratch (bytes) of the tensor path, on top of the fp32 Zhat buffer.
size_t tc_pair_bytes(const ftk_plan_s* p);
// Per-chunk fixed scratch (bytes) of the tensor path (tail tile, alignment).
size_t tc_fixed_bytes(const ftk_plan_s* p);
// Template-block granularity of a chunk.
int tc_template_quantum(const ftk_plan_s* p);
// Builds/frees the split-precision shift-factor tables.
cudaError_t tc_build_tables(ftk_plan_s* p, const std::vector<float2>& Y);
void tc_free_tables(ftk_plan_s* p);
// One chunk of ni images x nj templates.
ftk_status tc_run_chunk(ftk_plan_s* p, int precision, const float2* a, int ni, const float2* b, int nj, int i0,
                        int j0, int NT, float2* zbuf, char* tcbuf, float* d_scores, unsigned long long* d_keys,
                        cudaStream_t s);

}  // namespace ftk
