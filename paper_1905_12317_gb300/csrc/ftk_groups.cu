// Grouped best-pose search: ftk_align_best for several (plan, images, templates)
// groups in one call, each group on a stream of the library's own pool, forked from
// and joined to the caller's stream with events (legal under stream capture, so the
// call can be recorded into one CUDA graph).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ftk_internal.h"

namespace {

constexpr size_t kGroupAlign = 256;
constexpr int kPoolStreams = 8;
constexpr int kMaxDevices = 64;

size_t galign(size_t x) { return (x + kGroupAlign - 1) / kGroupAlign * kGroupAlign; }

std::mutex g_pool_mu;
cudaStream_t g_pool[kMaxDevices][kPoolStreams] = {};

// The pool of the current device, created on first use.
cudaError_t pool_streams(cudaStream_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  for (int k = 0; k < kPoolStreams; ++k) {
    if (!g_pool[dev][k]) {
      e = cudaStreamCreateWithFlags(&g_pool[dev][k], cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        g_pool[dev][k] = nullptr;
        return e;
      }
    }
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

ftk_status group_sizes(const ftk_group* groups, int n_groups, int precision, std::vector<size_t>* mn,
                       std::vector<size_t>* gd) {
  if (!groups || n_groups < 1 || n_groups > FTK_MAX_GROUPS) return FTK_ERR_ARG;
  mn->assign(n_groups, 0);
  gd->assign(n_groups, 0);
  for (int g = 0; g < n_groups; ++g) {
    const ftk_group& G = groups[g];
    if (!G.plan || G.NI < 0 || G.NT < 0) return FTK_ERR_ARG;
    if (G.NI == 0) continue;
    size_t a = 0, b = 0;
    const ftk_status st = ftk_workspace_size(G.plan, precision, G.NI, G.NT, &a, &b);
    if (st != FTK_OK) return st;
    (*mn)[g] = galign(a);
    (*gd)[g] = galign(std::max(a, b));
  }
  return FTK_OK;
}

ftk_status align_best_groups(const ftk_group* groups, int n_groups, int precision, void* d_work, size_t work_bytes,
                             void* stream);

}  // namespace

extern "C" {

ftk_status ftk_groups_workspace_size(const ftk_group* groups, int n_groups, int precision, size_t* min_bytes,
                                     size_t* good_bytes) {
  std::vector<size_t> mn, gd;
  const ftk_status st = group_sizes(groups, n_groups, precision, &mn, &gd);
  if (st != FTK_OK) return st;
  size_t smin = 0, sgood = 0;
  for (int g = 0; g < n_groups; ++g) {
    smin += mn[g];
    sgood += gd[g];
  }
  if (min_bytes) *min_bytes = smin;
  if (good_bytes) *good_bytes = sgood;
  return FTK_OK;
}

ftk_status ftk_align_best_groups(const ftk_group* groups, int n_groups, int precision, void* d_work,
                                 size_t work_bytes, void* stream) {
  nvtxRangePushA("ftk_align_best_groups");
  const ftk_status st = align_best_groups(groups, n_groups, precision, d_work, work_bytes, stream);
  nvtxRangePop();
  return st;
}

}  // extern "C"

namespace {
ftk_status align_best_groups(const ftk_group* groups, int n_groups, int precision, void* d_work, size_t work_bytes,
                             void* stream) {
  std::vector<size_t> mn, gd;
  ftk_status st = group_sizes(groups, n_groups, precision, &mn, &gd);
  if (st != FTK_OK) return st;
  if (!d_work || reinterpret_cast<uintptr_t>(d_work) % kGroupAlign) return FTK_ERR_ARG;
  size_t smin = 0, sgood = 0;
  for (int g = 0; g < n_groups; ++g) {
    smin += mn[g];
    sgood += gd[g];
  }
  if (work_bytes < smin) return FTK_ERR_NOMEM;
  // slices: good sizes if they fit, else min + a share of the rest in proportion to (good - min)
  std::vector<size_t> size(n_groups);
  const size_t extra = work_bytes - smin, want = sgood - smin;
  for (int g = 0; g < n_groups; ++g) {
    if (work_bytes >= sgood || want == 0) {
      size[g] = gd[g];
    } else {
      const double share = static_cast<double>(gd[g] - mn[g]) / static_cast<double>(want);
      const size_t add = static_cast<size_t>(share * static_cast<double>(extra)) / kGroupAlign * kGroupAlign;
      size[g] = mn[g] + std::min(add, gd[g] - mn[g]);  // the slices sum to at most work_bytes
    }
  }
  cudaStream_t* pool = nullptr;
  if (pool_streams(&pool) != cudaSuccess) return FTK_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t fork;
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return FTK_ERR_CUDA;
  if (cudaEventRecord(fork, s) != cudaSuccess) {
    cudaEventDestroy(fork);
    return FTK_ERR_CUDA;
  }
  ftk_status first = FTK_OK;
  bool used[kPoolStreams] = {};
  char* w = static_cast<char*>(d_work);
  for (int g = 0; g < n_groups; ++g) {
    const ftk_group& G = groups[g];
    if (G.NI == 0) continue;
    const int k = g % kPoolStreams;
    if (!used[k]) {
      if (cudaStreamWaitEvent(pool[k], fork, 0) != cudaSuccess) {
        first = FTK_ERR_CUDA;
        break;
      }
      used[k] = true;
    }
    st = ftk_align_best(G.plan, precision, G.d_img_coeffs, G.NI, G.d_tpl_coeffs, G.NT, G.d_tpl, G.d_rot, G.d_shift,
                        G.d_score, w, size[g], pool[k]);
    w += size[g];
    if (st != FTK_OK) {
      first = st;
      break;
    }
  }
  // join every stream that was forked, also after a failure
  for (int k = 0; k < kPoolStreams; ++k) {
    if (!used[k]) continue;
    cudaEvent_t join = nullptr;
    if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
      if (first == FTK_OK) first = FTK_ERR_CUDA;
      continue;
    }
    if (cudaEventRecord(join, pool[k]) != cudaSuccess || cudaStreamWaitEvent(s, join, 0) != cudaSuccess) {
      if (first == FTK_OK) first = FTK_ERR_CUDA;
    }
    cudaEventDestroy(join);
  }
  cudaEventDestroy(fork);
  return first;
}

}  // namespace
