// ftk_align_best_static: the best-pose search with its scratch in a static
// device array instead of a caller workspace, for callers that cannot allocate
// device memory when they call the library (see include/ftk.h).
#include <cuda_runtime.h>

#include <mutex>

#include "ftk_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = FTK_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch itself. In host code this name is only a handle for the CUDA
// runtime; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device, looked up once
// per device (with that device current).
ftk_status static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FTK_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return FTK_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return FTK_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FTK_OK;
}

}  // namespace

extern "C" ftk_status ftk_align_best_static(ftk_plan_t plan, int precision, const float* d_img_coeffs, int NI,
                                            const float* d_tpl_coeffs, int NT, int* d_tpl, int* d_rot, int* d_shift,
                                            float* d_score, void* stream) {
  if (!plan || NI < 0 || NT < 0) return FTK_ERR_ARG;
  // the scratch is looked up on the current device, which must hold the plan's tables
  if (!ftk::on_plan_device(plan)) return FTK_ERR_ARG;
  size_t min_bytes = 0;
  ftk_status st = ftk_workspace_size(plan, precision, NI, NT, &min_bytes, nullptr);
  if (st != FTK_OK) return st;
  if (min_bytes > kStaticScratchBytes) return FTK_ERR_SCRATCH_LIMIT;
  if (NI == 0) return FTK_OK;
  void* scratch = nullptr;
  st = static_scratch(&scratch);
  if (st != FTK_OK) return st;
  // ftk_align_best initializes the per-image maxima it keeps in the scratch
  // before use; everything else in it is written before it is read.
  return ftk_align_best(plan, precision, d_img_coeffs, NI, d_tpl_coeffs, NT, d_tpl, d_rot, d_shift, d_score, scratch,
                        kStaticScratchBytes, stream);
}
