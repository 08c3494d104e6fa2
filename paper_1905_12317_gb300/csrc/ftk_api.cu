// C ABI of libftk: planning, transform, pair-engine orchestration.
//
// Planning (Section 4.5) runs on the host in FP64 and uploads small tables. The
// pair engine walks the (image, template) pair space in chunks that fit the
// caller's workspace; per chunk it runs Step 1 -> Step 2 -> Step 3 of eq. (fbk3)
// and either writes every score or folds them into a per-image running maximum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ftk_internal.h"
#include "plan_math.h"
#include "tc_engine.h"

using ftk::FftSchedule;

namespace {

// NVTX range over one C-ABI call (host timeline; free when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool valid_two_Q(int L) {
  if (L < 8 || L > 768 || (L & 3)) return false;
  FftSchedule s = ftk::make_fft_schedule(L);
  return s.n > 0;
}

// the spectral weight exp(-decay (k/K)^2) of the modal SVDs: 0 (plain weights) .. 256
bool valid_decay(double decay) { return std::isfinite(decay) && decay >= 0.0 && decay <= 256.0; }

// Gauss--Jacobi nodes of the modal SVDs: enough for J_l(x y) on [0, 2 pi W] x [0, 1], the
// CTF's oscillation (|tau| half turns) and the weight's Gaussian sqrt(rho) = exp(-decay y^2 / 2)
int modal_nodes(double W, double tmax, double decay) {
  return static_cast<int>(std::ceil(2.0 * M_PI * W)) + 48 + static_cast<int>(std::ceil(2.0 * tmax)) +
         static_cast<int>(std::ceil(2.0 * std::sqrt(decay)));
}

template <typename T>
cudaError_t upload(T** dptr, const std::vector<T>& h) {
  *dptr = nullptr;
  if (h.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dptr), h.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_tables(ftk_plan_s* p) {
  cudaFree(p->d_G);
  cudaFree(p->d_l);
  cudaFree(p->d_Y);
  cudaFree(p->d_shifts);
  p->d_shifts = nullptr;
  cudaFree(p->d_Ex);
  cudaFree(p->d_Ey);
  cudaFree(p->d_tw);
  cudaFree(p->d_tw_rot);
  cudaFree(p->d_err);
  ftk::xform_free_tables(p);
  ftk::tc_free_tables(p);
  p->d_G = nullptr;
  p->d_l = nullptr;
  p->d_Y = nullptr;
  p->d_Ex = p->d_Ey = p->d_tw = p->d_tw_rot = nullptr;
  p->d_err = nullptr;
}

#define FTK_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return FTK_ERR_CUDA;          \
  } while (0)

// Per-pair scratch of the FP32 pair engine (bytes): Zhat / Z in FP32.
size_t pair_bytes(const ftk_plan_s* p) { return static_cast<size_t>(p->Hh) * p->two_Q * sizeof(float2); }

size_t keys_bytes(int NI) { return align_up(static_cast<size_t>(NI) * sizeof(unsigned long long)); }

struct Chunking {
  int ib = 0, tb = 0;
};

Chunking choose_chunks(const ftk_plan_s* p, int NI, int NT, size_t avail) {
  Chunking c;
  const size_t pb = pair_bytes(p);
  const size_t fixed = 2 * kAlign;
  if (avail <= fixed) return c;
  size_t maxpairs = (avail - fixed) / pb;
  if (maxpairs < 1) return c;
  if (maxpairs > (1u << 20)) maxpairs = 1u << 20;
  int tb = static_cast<int>(std::min<size_t>(NT, maxpairs));
  if (tb <= 0) return c;
  int ib = static_cast<int>(std::min<size_t>(NI, maxpairs / tb));
  ib = std::min(ib, 65535);
  c.ib = std::max(ib, 1);
  c.tb = tb;
  return c;
}

ftk_status check_common(const ftk_plan_s* p, int precision, const void* a, int NI, const void* b, int NT) {
  if (!p) return FTK_ERR_ARG;
  if (!ftk::on_plan_device(p)) return FTK_ERR_ARG;
  if (precision != FTK_FP32 && precision != FTK_BF16X3 && precision != FTK_BF16 &&
      precision != FTK_FP16) return FTK_ERR_ARG;
  if (NI < 0 || NT < 0) return FTK_ERR_ARG;
  if ((NI > 0 && !a) || (NT > 0 && !b)) return FTK_ERR_ARG;
  if (precision != FTK_FP32 && !ftk::tc_supported(p)) return FTK_ERR_UNSUPPORTED;
  if (precision == FTK_FP32 && p->n_rot != p->two_Q) return FTK_ERR_UNSUPPORTED;  // finer grids: tensor path
  return FTK_OK;
}

// Best-pose bookkeeping: with pose indices below 2^32 one 64-bit key per image (score
// bits | complemented pose index) decides the maximum and k_best_finalize decodes it;
// past 2^32 (the template part needs more bits) each chunk's keys count templates from
// the chunk's first template, or by shortlist position, and are merged after the chunk
// into per-image records kept in the outputs.
ftk::BestRecords records_for(const ftk_plan_s* p, long long n_tpl_index, int* tpl, int* rot, int* shift,
                             float* score) {
  ftk::BestRecords r;
  r.wide = ftk::pose_index_wide(n_tpl_index, p->n_rot, p->N);
  if (r.wide) {
    r.tpl = tpl;
    r.rot = rot;
    r.shift = shift;
    r.score = score;
  }
  return r;
}

ftk_status finish_best(ftk_plan_s* p, const unsigned long long* keys, int NI, const ftk::BestRecords& rec, int* tpl,
                       int* rot, int* shift, float* score, cudaStream_t s) {
  if (rec.wide)  // every chunk is merged already: this pass latches images left without a pose
    FTK_LAUNCH(p, ftk::kKBestMerge, s,
               ftk::launch_best_merge(p, const_cast<unsigned long long*>(keys), 0, NI, 0, nullptr, 0, rec, true, s));
  else
    FTK_LAUNCH(p, ftk::kKBestFinalize, s, ftk::launch_best_finalize(p, keys, NI, tpl, rot, shift, score, s));
  return FTK_OK;
}

// Runs Steps 1-3 over all pairs, chunk by chunk. With rec.wide (best pose, NT * R * N >=
// 2^32) each chunk's keys count templates from its first template and are merged into the
// records after it; chunks then cover fewer than 2^32 / (R N) templates.
ftk_status run_engine(ftk_plan_s* p, int precision, const float2* a, int NI, const float2* b, int NT,
                      float* d_scores, unsigned long long* d_keys, const ftk::BestRecords& rec, char* work,
                      size_t work_bytes, cudaStream_t s) {
  if (precision != FTK_FP32)
    return ftk::tc_run_all(p, precision, a, NI, b, NT, d_scores, d_keys, rec, work, work_bytes, s);
  Chunking ch = choose_chunks(p, NI, NT, work_bytes);
  if (ch.ib <= 0 || ch.tb <= 0) return FTK_ERR_NOMEM;
  while (rec.wide && ch.tb > 1 && ftk::pose_index_wide(ch.tb, p->n_rot, p->N)) ch.tb /= 2;
  const size_t MQ2 = static_cast<size_t>(p->M) * p->two_Q;
  float2* zbuf = reinterpret_cast<float2*>(work);
  for (int i0 = 0; i0 < NI; i0 += ch.ib) {
    const int ni = std::min(ch.ib, NI - i0);
    for (int j0 = 0; j0 < NT; j0 += ch.tb) {
      const int nj = std::min(ch.tb, NT - j0);
      FTK_LAUNCH(p, ftk::kKStep1Simt, s, ftk::launch_step1_simt(p, a + i0 * MQ2, ni, b + j0 * MQ2, nj, zbuf, s));
      FTK_LAUNCH(p, ftk::kKFftRows, s, ftk::launch_fft_rows(p, zbuf, static_cast<long long>(ni) * nj * p->Hh, 1.0f, s));
      FTK_LAUNCH(p, ftk::kKStep3Simt, s,
                 ftk::launch_step3_simt(p, zbuf, ni, nj, i0, j0, NT, d_scores, d_keys, s, nullptr, nullptr, 0.f,
                                        rec.wide ? j0 : 0, 0));
      if (rec.wide && d_keys)
        FTK_LAUNCH(p, ftk::kKBestMerge, s, ftk::launch_best_merge(p, d_keys, i0, ni, j0, nullptr, 0, rec, false, s));
    }
  }
  return FTK_OK;
}

}  // namespace

namespace ftk {

bool on_plan_device(const ftk_plan_s* p) {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev == p->device;
}

static_assert(FTK_NUM_KERNELS == kKNumKernels, "FTK_NUM_KERNELS must count the profiled kernels");

const char* kernel_name(int id) {
  static const char* names[kKNumKernels] = {"polar_transform", "fft_rows",     "step1_simt",
                                            "step3_simt",      "best_init",    "best_finalize",
                                            "step1_tc",        "fft_pack",     "step3_tc",
                                            "pack_templates",  "polar_tc",     "pack_pixels",
                                            "step23_tc",       "best_merge",   "step23c_tc"};
  return (id >= 0 && id < kKNumKernels) ? names[id] : "?";
}

void prof_start(ftk_plan_s* p, int id, cudaStream_t s) {
  if (!p->prof.on) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, s);
  p->prof.pending_start[id].push_back(e);
}

void prof_stop(ftk_plan_s* p, int id, cudaStream_t s) {
  if (!p->prof.on) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, s);
  p->prof.pending_stop[id].push_back(e);
}

}  // namespace ftk

extern "C" {

ftk_status ftk_profile_begin(ftk_plan_t p) {
  if (!p) return FTK_ERR_ARG;
  for (int k = 0; k < ftk::kKNumKernels; ++k) {
    p->prof.total_ms[k] = 0;
    p->prof.count[k] = 0;
  }
  p->prof.on = true;
  return FTK_OK;
}

ftk_status ftk_profile_end(ftk_plan_t p, void* stream) {
  if (!p) return FTK_ERR_ARG;
  p->prof.on = false;
  ftk_status st = FTK_OK;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) st = FTK_ERR_CUDA;
  for (int k = 0; k < ftk::kKNumKernels; ++k) {
    auto& a = p->prof.pending_start[k];
    auto& b = p->prof.pending_stop[k];
    for (size_t i = 0; i < a.size() && i < b.size(); ++i) {
      float ms = 0.f;
      if (cudaEventSynchronize(b[i]) == cudaSuccess && cudaEventElapsedTime(&ms, a[i], b[i]) == cudaSuccess) {
        p->prof.total_ms[k] += ms;
        p->prof.count[k] += 1;
      }
    }
    for (cudaEvent_t e : a) cudaEventDestroy(e);
    for (cudaEvent_t e : b) cudaEventDestroy(e);
    a.clear();
    b.clear();
  }
  return st;
}

ftk_status ftk_profile_kernel(ftk_plan_t p, int id, const char** name, double* total_ms, long long* launches) {
  if (!p || id < 0 || id >= ftk::kKNumKernels) return FTK_ERR_ARG;
  if (name) *name = ftk::kernel_name(id);
  if (total_ms) *total_ms = p->prof.total_ms[id];
  if (launches) *launches = p->prof.count[id];
  return FTK_OK;
}

const char* ftk_status_string(ftk_status st) {
  switch (st) {
    case FTK_OK: return "ok";
    case FTK_ERR_ARG: return "invalid argument";
    case FTK_ERR_SHIFT_RANGE: return "shift outside the disk of radius 2W pixels";
    case FTK_ERR_NOMEM: return "out of memory or workspace too small";
    case FTK_ERR_CUDA: return "CUDA error";
    case FTK_ERR_TIMEOUT: return "device-side wait timed out";
    case FTK_ERR_PLAN_MISMATCH: return "buffer does not match the plan";
    case FTK_ERR_UNSUPPORTED: return "configuration not supported by this kernel";
    case FTK_ERR_SCRATCH_LIMIT: return "problem needs more scratch than the library's fixed static buffer";
  }
  return "unknown status";
}

ftk_status ftk_rank_profile(double W, double eps, int max_l, int* H_l, double* sigma, int n_sigma,
                            int* H_total) {
  return ftk_rank_profile_weighted(W, eps, 0.0, max_l, H_l, sigma, n_sigma, H_total);
}

ftk_status ftk_rank_profile_weighted(double W, double eps, double decay, int max_l, int* H_l, double* sigma,
                                     int n_sigma, int* H_total) {
  if (!(W > 0) || !(eps > 0) || eps >= 1 || max_l < 0 || max_l > 4096 || n_sigma < 0) return FTK_ERR_ARG;
  if (!valid_decay(decay)) return FTK_ERR_ARG;
  const int nq = modal_nodes(W, 0.0, decay);
  int total = 0, zero_run = 0;
  for (int l = 0; l <= 4096; ++l) {
    const bool report = l <= max_l;
    if (!report && zero_run >= 4) break;
    ftk::ModalSVD ms = ftk::modal_svd(l, W, nq, {}, 0.0, decay);
    int h = 0;
    while (h < static_cast<int>(ms.sigma.size()) && ms.sigma[h] > eps) ++h;
    total += (l == 0 ? 1 : 2) * h;
    zero_run = h == 0 ? zero_run + 1 : 0;
    if (report) {
      if (H_l) H_l[l] = h;
      if (sigma)
        for (int e = 0; e < n_sigma; ++e)
          sigma[static_cast<size_t>(l) * n_sigma + e] = e < static_cast<int>(ms.sigma.size()) ? ms.sigma[e] : 0.0;
    }
  }
  if (H_total) *H_total = total;
  return FTK_OK;
}

}  // extern "C"

namespace {

// plan files (ftk_plan_save / ftk_plan_load)
constexpr char kPlanMagic[8] = {'F', 'T', 'K', 'P', 'L', 'A', 'N', '1'};
constexpr int32_t kPlanVersion = 2;  // 2 adds the spectral decay; 1 is still read

template <typename T>
bool put(std::FILE* f, const T* v, size_t n) { return n == 0 || std::fwrite(v, sizeof(T), n, f) == n; }
template <typename T>
bool get(std::FILE* f, T* v, size_t n) { return n == 0 || std::fread(v, sizeof(T), n, f) == n; }

// Device tables of a plan whose host fields (rule, terms, h_G, h_Y, shifts) are set:
// transform tables, factors, shifts, error word, tensor-core tables. Deletes the plan
// on failure.
ftk_status plan_upload(ftk_plan_s* p, const std::vector<int>& lz) {
  const int n = p->n, M = p->M, two_Q = p->two_Q, N = p->N_shift;
  // ---- transform tables (eq. Ahattrap), half plane p < Q ----
  const int MQ = M * p->Q;
  std::vector<float2> Ex(static_cast<size_t>(n) * MQ), Ey(static_cast<size_t>(n) * MQ);
  std::vector<double> ey_re(static_cast<size_t>(n) * MQ), ey_im(static_cast<size_t>(n) * MQ);
  for (int m = 0; m < M; ++m) {
    for (int pp = 0; pp < p->Q; ++pp) {
      const double psi = M_PI * pp / p->Q;
      const double kx = p->h_k[m] * std::cos(psi), ky = p->h_k[m] * std::sin(psi);
      for (int i = 0; i < n; ++i) {
        const double x = i * p->dx - 1.0;
        const size_t at = static_cast<size_t>(i) * MQ + m * p->Q + pp;
        Ex[at] = make_float2(static_cast<float>(std::cos(kx * x)), static_cast<float>(-std::sin(kx * x)));
        ey_re[at] = std::cos(ky * x);
        ey_im[at] = -std::sin(ky * x);
        Ey[at] = make_float2(static_cast<float>(ey_re[at]), static_cast<float>(ey_im[at]));
      }
    }
  }
  std::vector<float2> tw(two_Q);
  for (int t = 0; t < two_Q; ++t) {
    const double a = -2.0 * M_PI * t / two_Q;
    tw[t] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
  }

  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(&p->d_G, p->h_G);
  if (e == cudaSuccess) e = upload(&p->d_l, lz);
  if (e == cudaSuccess) e = upload(&p->d_Y, p->h_Y);
  if (e == cudaSuccess) {  // the shift of every row (repeated per defocus value)
    std::vector<float2> sh(p->N);
    for (int r = 0; r < p->N; ++r) {
      const int s = r % N;
      sh[r] = make_float2(static_cast<float>(p->h_shifts[2 * s]), static_cast<float>(p->h_shifts[2 * s + 1]));
    }
    e = upload(&p->d_shifts, sh);
  }
  if (e == cudaSuccess) e = upload(&p->d_Ex, Ex);
  if (e == cudaSuccess) e = upload(&p->d_Ey, Ey);
  if (e == cudaSuccess) e = upload(&p->d_tw, tw);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->d_err), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = ftk::tc_build_tables(p, p->h_Y);
  if (e == cudaSuccess && ftk::xform_tc_supported(p)) {
    e = ftk::xform_build_tables(p, ey_re, ey_im);
    if (e == cudaSuccess) e = ftk::xform_alloc_scratch(p);
  }
  if (e != cudaSuccess) {
    free_tables(p);
    delete p;
    return e == cudaErrorMemoryAllocation ? FTK_ERR_NOMEM : FTK_ERR_CUDA;
  }
  return FTK_OK;
}

ftk_status plan_create(int n, double K, double W, double eps, int M, int two_Q, const double* shifts_px, int N,
                       const std::vector<double>& taus, double phase, double decay, ftk_plan_t* out) {
  if (!out) return FTK_ERR_ARG;
  *out = nullptr;
  if (!valid_decay(decay)) return FTK_ERR_ARG;
  for (double t : taus)
    if (!std::isfinite(t) || std::fabs(t) > 64.0) return FTK_ERR_ARG;
  if (!std::isfinite(phase)) return FTK_ERR_ARG;
  const int nt = taus.empty() ? 1 : static_cast<int>(taus.size());
  if (static_cast<long long>(N) * nt > (1 << 24)) return FTK_ERR_ARG;
  if (n < 8 || n > 256 || (n & 1)) return FTK_ERR_ARG;
  if (!(W > 0) || !(eps > 0) || eps >= 1 || M < 1 || M > 256 || !valid_two_Q(two_Q)) return FTK_ERR_ARG;
  if (N < 1 || !shifts_px) return FTK_ERR_ARG;
  for (int s = 0; s < 2 * N; ++s)
    if (!std::isfinite(shifts_px[s])) return FTK_ERR_ARG;
  for (int s = 0; s < N; ++s) {
    const double r = std::hypot(shifts_px[2 * s], shifts_px[2 * s + 1]);
    if (r > 2.0 * W * (1.0 + 1e-12) + 1e-12) return FTK_ERR_SHIFT_RANGE;
  }
  ftk_plan_s* p = new (std::nothrow) ftk_plan_s();
  if (!p) return FTK_ERR_NOMEM;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return FTK_ERR_CUDA;
  }
  p->n = n;
  p->M = M;
  p->two_Q = two_Q;
  p->n_rot = two_Q;
  p->Q = two_Q / 2;
  p->N_shift = N;
  p->n_tau = nt;
  p->N = N * nt;
  p->K = K > 0 ? K : 0.5 * M_PI * n;
  p->W = W;
  p->eps = eps;
  p->dx = 2.0 / n;
  p->fft = ftk::make_fft_schedule(two_Q);

  // ---- radial rule, Section 3.1: Gauss--Jacobi(0,1) mapped to [0, K] ----
  {
    std::vector<double> t, v;
    ftk::gauss_jacobi(M, 0.0, 1.0, t, v);
    p->h_k.resize(M);
    p->h_w.resize(M);
    for (int m = 0; m < M; ++m) {
      p->h_k[m] = 0.5 * p->K * (1.0 + t[m]);
      p->h_w[m] = 0.25 * p->K * p->K * v[m];
    }
  }

  // ---- per-order operator SVD, Section 4.5; keep Sigma > eps, orders l >= 0 ----
  double tmax = 0.0;
  for (double t : taus) tmax = std::max(tmax, std::fabs(t));
  const int nq = modal_nodes(W, tmax, decay);
  std::vector<ftk::ModalSVD> modes;
  std::vector<int> Hl;
  int zero_run = 0;
  for (int l = 0; l <= 4096; ++l) {
    ftk::ModalSVD ms = ftk::modal_svd(l, W, nq, taus, phase, decay);
    int h = 0;
    while (h < static_cast<int>(ms.sigma.size()) && ms.sigma[h] > eps) ++h;
    if (h == 0) {
      if (++zero_run >= 4) break;
      continue;
    }
    zero_run = 0;
    while (static_cast<int>(Hl.size()) < l) Hl.push_back(0);
    Hl.push_back(h);
    modes.push_back(std::move(ms));
  }
  std::vector<float> G;
  std::vector<int> lz;
  std::vector<std::vector<double>> Urows;  // per term: U at each shift
  {
    int H = 0, Hh = 0;
    for (const auto& ms : modes) {
      int h = 0;
      while (h < static_cast<int>(ms.sigma.size()) && ms.sigma[h] > eps) ++h;
      H += (ms.l == 0 ? 1 : 2) * h;
      Hh += h;
      p->L = std::max(p->L, ms.l);
    }
    p->H = H;
    p->Hh = Hh;
  }
  if (p->L >= two_Q) {  // Step 1 reads a(k; q - l) with q - l taken modulo 2Q once
    delete p;
    return FTK_ERR_UNSUPPORTED;
  }
  G.resize(static_cast<size_t>(p->Hh) * M);
  lz.resize(p->Hh);
  std::vector<float2> Y(static_cast<size_t>(p->N) * p->Hh);  // row b N + s: defocus b, shift s
  {
    int z = 0;
    for (const auto& ms : modes) {
      int h = 0;
      while (h < static_cast<int>(ms.sigma.size()) && ms.sigma[h] > eps) ++h;
      for (int eta = 0; eta < h; ++eta, ++z) {
        lz[z] = ms.l;
        p->h_l.push_back(ms.l);
        p->h_sigma.push_back(ms.sigma[eta]);
        for (int m = 0; m < M; ++m)
          G[static_cast<size_t>(z) * M + m] =
              static_cast<float>(2.0 * M_PI * p->h_w[m] * ms.G(eta, p->h_k[m] / p->K));
        const double c = ms.l == 0 ? 1.0 : 2.0;
        for (int b = 0; b < nt; ++b)
          for (int s = 0; s < N; ++s) {
            const double dxs = shifts_px[2 * s] * p->dx, dys = shifts_px[2 * s + 1] * p->dx;
            const double d = std::hypot(dxs, dys);
            const double om = std::atan2(dys, dxs);
            const double u = ms.U(eta, p->K * d, b);
            const double ph = -ms.l * (om + 0.5 * M_PI);
            Y[(static_cast<size_t>(b) * N + s) * p->Hh + z] =
                make_float2(static_cast<float>(c * u * std::cos(ph)), static_cast<float>(c * u * std::sin(ph)));
          }
      }
    }
  }

  p->h_Y = std::move(Y);
  p->h_G = std::move(G);
  p->h_shifts.assign(shifts_px, shifts_px + 2 * N);
  p->h_taus = taus;
  p->phase = phase;
  p->decay = decay;
  const ftk_status st = plan_upload(p, lz);
  if (st != FTK_OK) return st;
  *out = p;
  return FTK_OK;
}

}  // namespace

extern "C" {

ftk_status ftk_plan_create(int n, double K, double W, double eps, int M, int two_Q, const double* shifts_px,
                           int N, ftk_plan_t* out) {
  NvtxRange nvtx_("ftk_plan_create");
  return plan_create(n, K, W, eps, M, two_Q, shifts_px, N, {}, 0.0, 0.0, out);
}

ftk_status ftk_plan_create_weighted(int n, double K, double W, double eps, int M, int two_Q, const double* shifts_px,
                                    int N, double decay, ftk_plan_t* out) {
  NvtxRange nvtx_("ftk_plan_create_weighted");
  return plan_create(n, K, W, eps, M, two_Q, shifts_px, N, {}, 0.0, decay, out);
}

double ftk_plan_spectral_decay(ftk_plan_t p) { return p ? p->decay : -1.0; }

ftk_status ftk_plan_create_ctf(int n, double K, double W, double eps, int M, int two_Q, const double* shifts_px,
                               int N, const double* defocus, int n_defocus, double phase, ftk_plan_t* out) {
  NvtxRange nvtx_("ftk_plan_create_ctf");
  if (n_defocus < 1 || n_defocus > 256 || !defocus) {
    if (out) *out = nullptr;
    return FTK_ERR_ARG;
  }
  return plan_create(n, K, W, eps, M, two_Q, shifts_px, N, std::vector<double>(defocus, defocus + n_defocus), phase,
                     0.0, out);
}

int ftk_plan_defocus_count(ftk_plan_t p) { return p ? p->n_tau : 0; }

// ---- plan files: everything the host computed (rule, terms, factors, shifts, tuning) ----
ftk_status ftk_plan_save(ftk_plan_t p, const char* path) {
  if (!p || !path) return FTK_ERR_ARG;
  std::FILE* f = std::fopen(path, "wb");
  if (!f) return FTK_ERR_ARG;
  const int32_t hdr[18] = {kPlanVersion, p->n, p->M, p->two_Q, p->N_shift, p->n_tau, p->H, p->Hh, p->L, p->n_rot,
                           p->tune.step3_group_max, p->tune.step3_a_stages, p->tune.step1_stages,
                           p->tune.step1_ctas_per_sm, p->tune.fft_lanes, p->xf.use_simt ? 1 : 0,
                           static_cast<int32_t>(p->h_taus.size()), p->tune.step23};
  const double dv[5] = {p->K, p->W, p->eps, p->phase, p->decay};
  bool ok = put(f, kPlanMagic, 8) && put(f, hdr, 18) && put(f, dv, 5) && put(f, p->h_taus.data(), p->h_taus.size()) &&
            put(f, p->h_shifts.data(), p->h_shifts.size()) && put(f, p->h_k.data(), p->h_k.size()) &&
            put(f, p->h_w.data(), p->h_w.size()) && put(f, p->h_l.data(), p->h_l.size()) &&
            put(f, p->h_sigma.data(), p->h_sigma.size()) && put(f, p->h_G.data(), p->h_G.size()) &&
            put(f, reinterpret_cast<const float*>(p->h_Y.data()), 2 * p->h_Y.size());
  ok = (std::fclose(f) == 0) && ok;
  return ok ? FTK_OK : FTK_ERR_ARG;
}

ftk_status ftk_plan_load(const char* path, ftk_plan_t* out) {
  NvtxRange nvtx_("ftk_plan_load");
  if (!out) return FTK_ERR_ARG;
  *out = nullptr;
  if (!path) return FTK_ERR_ARG;
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return FTK_ERR_ARG;
  char magic[8];
  int32_t h[18];
  double dv[5] = {0, 0, 0, 0, 0};
  bool ok = get(f, magic, 8) && std::memcmp(magic, kPlanMagic, 8) == 0 && get(f, h, 18) && (h[0] == 1 || h[0] == 2) &&
            get(f, dv, h[0] == 2 ? 5 : 4);
  ok = ok && h[1] >= 8 && h[1] <= 256 && h[2] >= 1 && h[2] <= 256 && valid_two_Q(h[3]) &&
       h[4] >= 1 && h[5] >= 1 && h[5] <= 256 && static_cast<long long>(h[4]) * h[5] <= (1 << 24) && h[7] >= 1 &&
       h[7] <= 8192 && h[6] >= h[7] && h[8] >= 0 && h[8] < h[3] && h[9] >= h[3] && h[9] % h[3] == 0 && h[16] >= 0 &&
       h[16] <= 256 && (h[16] == 0 ? h[5] == 1 : h[16] == h[5]);
  // tuning knobs, in the ranges ftk_plan_tune accepts
  ok = ok && (h[10] == 0 || (h[10] >= 16 && h[10] <= 256 && h[10] % 16 == 0)) && h[11] >= 0 && h[11] <= 12 &&
       h[12] >= 0 && h[12] <= 8 && h[13] >= 0 && h[13] <= 8 &&
       (h[14] == 0 || h[14] == 8 || h[14] == 16 || h[14] == 32) && (h[15] == 0 || h[15] == 1) &&
       (h[17] == 0 || h[17] == 1);
  ok = ok && std::isfinite(dv[0]) && dv[0] > 0 && std::isfinite(dv[1]) && dv[1] > 0 && dv[2] > 0 && dv[2] < 1 &&
       std::isfinite(dv[3]) && valid_decay(dv[4]);
  ftk_plan_s* p = ok ? new (std::nothrow) ftk_plan_s() : nullptr;
  if (!p) {
    std::fclose(f);
    return ok ? FTK_ERR_NOMEM : FTK_ERR_ARG;
  }
  p->n = h[1];
  p->M = h[2];
  p->two_Q = h[3];
  p->Q = h[3] / 2;
  p->n_rot = h[3];
  p->N_shift = h[4];
  p->n_tau = h[5];
  p->N = h[4] * h[5];
  p->H = h[6];
  p->Hh = h[7];
  p->L = h[8];
  p->tune.step3_group_max = h[10];
  p->tune.step3_a_stages = h[11];
  p->tune.step1_stages = h[12];
  p->tune.step1_ctas_per_sm = h[13];
  p->tune.fft_lanes = h[14];
  p->xf.use_simt = h[15] != 0;
  p->tune.step23 = h[17];
  p->K = dv[0];
  p->W = dv[1];
  p->eps = dv[2];
  p->phase = dv[3];
  p->decay = dv[4];
  p->dx = 2.0 / p->n;
  p->fft = ftk::make_fft_schedule(p->two_Q);
  p->h_taus.resize(h[16]);
  p->h_shifts.resize(2 * static_cast<size_t>(p->N_shift));
  p->h_k.resize(p->M);
  p->h_w.resize(p->M);
  p->h_l.resize(p->Hh);
  p->h_sigma.resize(p->Hh);
  p->h_G.resize(static_cast<size_t>(p->Hh) * p->M);
  p->h_Y.resize(static_cast<size_t>(p->N) * p->Hh);
  ok = get(f, p->h_taus.data(), p->h_taus.size()) && get(f, p->h_shifts.data(), p->h_shifts.size()) &&
       get(f, p->h_k.data(), p->h_k.size()) && get(f, p->h_w.data(), p->h_w.size()) &&
       get(f, p->h_l.data(), p->h_l.size()) && get(f, p->h_sigma.data(), p->h_sigma.size()) &&
       get(f, p->h_G.data(), p->h_G.size()) &&
       get(f, reinterpret_cast<float*>(p->h_Y.data()), 2 * p->h_Y.size());
  char extra;
  ok = ok && std::fread(&extra, 1, 1, f) == 0;  // nothing after the tables
  std::fclose(f);
  for (int z = 0; ok && z < p->Hh; ++z) ok = p->h_l[z] >= 0 && p->h_l[z] <= p->L;
  if (!ok || cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return ok ? FTK_ERR_CUDA : FTK_ERR_ARG;
  }
  const std::vector<int> lz(p->h_l.begin(), p->h_l.end());
  const ftk_status st = plan_upload(p, lz);  // deletes p on failure
  if (st != FTK_OK) return st;
  if (h[9] != p->two_Q) {
    const ftk_status sr = ftk_plan_set_rotations(p, h[9]);
    if (sr != FTK_OK) {
      ftk_plan_destroy(p);
      return sr;
    }
  }
  *out = p;
  return FTK_OK;
}

ftk_status ftk_plan_tune(ftk_plan_t p, const char* knob, int value) {
  if (!p || !knob || value < 0) return FTK_ERR_ARG;
  const std::string k(knob);
  if (k == "step3_group_max") {
    if (value != 0 && (value < 16 || value > 256 || value % 16)) return FTK_ERR_ARG;
    p->tune.step3_group_max = value;
  } else if (k == "step3_a_stages") {
    if (value > 12) return FTK_ERR_ARG;
    p->tune.step3_a_stages = value;
  } else if (k == "step1_stages") {
    if (value > 8) return FTK_ERR_ARG;
    p->tune.step1_stages = value;
  } else if (k == "step1_ctas_per_sm") {
    if (value > 8) return FTK_ERR_ARG;
    p->tune.step1_ctas_per_sm = value;
    return FTK_OK;
  } else if (k == "fft_lanes") {
    if (value != 0 && value != 8 && value != 16 && value != 32) return FTK_ERR_ARG;
    p->tune.fft_lanes = value;
    return FTK_OK;
  } else if (k == "checks") {
    if (value > 1) return FTK_ERR_ARG;
    p->tune.checks = value;
    return FTK_OK;
  } else if (k == "step23") {
    if (value > 1) return FTK_ERR_ARG;
    p->tune.step23 = value;
    return FTK_OK;
  } else if (k == "cluster23") {
    if (value > 1) return FTK_ERR_ARG;
    p->tune.cluster23 = value;
    return FTK_OK;
  } else if (k == "transform") {
    if (value > 1) return FTK_ERR_ARG;
    p->xf.use_simt = value == 1;
    return FTK_OK;
  } else {
    return FTK_ERR_ARG;
  }
  if (k == "step1_stages") return FTK_OK;
  // the Step-3 grouping changes the layout of the split shift-factor tables
  if (cudaDeviceSynchronize() != cudaSuccess) return FTK_ERR_CUDA;
  ftk::tc_free_tables(p);
  const cudaError_t e = ftk::tc_build_tables(p, p->h_Y);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FTK_ERR_NOMEM : FTK_ERR_CUDA;
  return FTK_OK;
}

ftk_status ftk_plan_tuning(ftk_plan_t p, int* step3_group, int* step3_groups, int* step3_a_stages) {
  if (!p) return FTK_ERR_ARG;
  if (step3_group) *step3_group = p->tc.G;
  if (step3_groups) *step3_groups = p->tc.n_groups;
  if (step3_a_stages) *step3_a_stages = p->tc.nsa;
  return FTK_OK;
}

void ftk_plan_destroy(ftk_plan_t p) {
  if (!p) return;
  free_tables(p);
  delete p;
}

ftk_status ftk_plan_info(ftk_plan_t p, int* H, int* H_half, int* L, int* M, int* two_Q, int* N, int* n) {
  if (!p) return FTK_ERR_ARG;
  if (H) *H = p->H;
  if (H_half) *H_half = p->Hh;
  if (L) *L = p->L;
  if (M) *M = p->M;
  if (two_Q) *two_Q = p->two_Q;
  if (N) *N = p->N;
  if (n) *n = p->n;
  return FTK_OK;
}

ftk_status ftk_plan_set_rotations(ftk_plan_t p, int n_rot) {
  if (!p || n_rot < p->two_Q || n_rot % p->two_Q) return FTK_ERR_ARG;
  if (n_rot == p->two_Q) {
    cudaFree(p->d_tw_rot);
    p->d_tw_rot = nullptr;
    p->n_rot = n_rot;
    return FTK_OK;
  }
  // the zero-padded transform runs in the warp-register FFT: L = 32 c with a supported c
  if (n_rot != 96 && n_rot != 192 && n_rot != 288 && n_rot != 384 && n_rot != 576 && n_rot != 768)
    return FTK_ERR_UNSUPPORTED;
  if (!ftk::tc_supported(p)) return FTK_ERR_UNSUPPORTED;
  std::vector<float2> tw(n_rot);
  for (int t = 0; t < n_rot; ++t) {
    const double a = -2.0 * M_PI * t / n_rot;
    tw[t] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return FTK_ERR_CUDA;
  cudaFree(p->d_tw_rot);
  p->d_tw_rot = nullptr;
  const cudaError_t e = upload(&p->d_tw_rot, tw);
  if (e != cudaSuccess) {
    p->d_tw_rot = nullptr;
    p->n_rot = p->two_Q;
    return e == cudaErrorMemoryAllocation ? FTK_ERR_NOMEM : FTK_ERR_CUDA;
  }
  p->n_rot = n_rot;
  return FTK_OK;
}

int ftk_plan_rotations(ftk_plan_t p) { return p ? p->n_rot : 0; }

ftk_status ftk_plan_terms(ftk_plan_t p, int* l, double* sigma) {
  if (!p) return FTK_ERR_ARG;
  for (int z = 0; z < p->Hh; ++z) {
    if (l) l[z] = p->h_l[z];
    if (sigma) sigma[z] = p->h_sigma[z];
  }
  return FTK_OK;
}

ftk_status ftk_plan_radial_rule(ftk_plan_t p, double* k, double* w) {
  if (!p) return FTK_ERR_ARG;
  for (int m = 0; m < p->M; ++m) {
    if (k) k[m] = p->h_k[m];
    if (w) w[m] = p->h_w[m];
  }
  return FTK_OK;
}

long long ftk_plan_launch_count(ftk_plan_t p) { return p ? p->launches : -1; }

ftk_status ftk_transform(ftk_plan_t p, const float* d_images, int B, float* d_coeffs, void* stream) {
  NvtxRange nvtx_("ftk_transform");
  if (!p || B < 0) return FTK_ERR_ARG;
  if (!ftk::on_plan_device(p)) return FTK_ERR_ARG;
  if (B == 0) return FTK_OK;
  if (!d_images || !d_coeffs) return FTK_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float2* out = reinterpret_cast<float2*>(d_coeffs);
  if (p->xf.d_ehi && !p->xf.use_simt) {
    const ftk_status st = ftk::xform_run(p, d_images, B, out, s);
    if (st != FTK_OK) return st;
  } else {
    FTK_LAUNCH(p, ftk::kKPolar, s, ftk::launch_polar_transform(p, d_images, B, out, s));
  }
  FTK_LAUNCH(p, ftk::kKFftRows, s, ftk::launch_fft_rows(p, out, static_cast<long long>(B) * p->M, 1.0f / p->two_Q, s));
  return FTK_OK;
}

ftk_status ftk_workspace_size(ftk_plan_t p, int precision, int NI, int NT, size_t* min_bytes,
                              size_t* good_bytes) {
  if (!p || NI < 0 || NT < 0) return FTK_ERR_ARG;
  if (precision != FTK_FP32 && precision != FTK_BF16X3 && precision != FTK_BF16 &&
      precision != FTK_FP16) return FTK_ERR_ARG;
  const size_t base = keys_bytes(NI) + 2 * kAlign;
  if (precision != FTK_FP32) {
    if (!ftk::tc_supported(p)) return FTK_ERR_UNSUPPORTED;
    size_t mn = 0, gd = 0;
    ftk::tc_workspace(p, NI, NT, &mn, &gd);
    if (min_bytes) *min_bytes = base + mn;
    if (good_bytes) *good_bytes = base + gd;
    return FTK_OK;
  }
  const size_t pb = pair_bytes(p);
  if (min_bytes) *min_bytes = base + pb;
  if (good_bytes) {
    size_t pairs = static_cast<size_t>(std::max(NI, 1)) * std::max(NT, 1);
    const size_t cap = std::max<size_t>(1, (size_t(1) << 30) / pb);
    pairs = std::min(pairs, cap);
    *good_bytes = base + pb * std::max<size_t>(pairs, 1);
  }
  return FTK_OK;
}

ftk_status ftk_align_scores(ftk_plan_t p, int precision, const float* d_img, int NI, const float* d_tpl, int NT,
                            float* d_scores, void* d_work, size_t work_bytes, void* stream) {
  NvtxRange nvtx_("ftk_align_scores");
  ftk_status st = check_common(p, precision, d_img, NI, d_tpl, NT);
  if (st != FTK_OK) return st;
  if (NI == 0 || NT == 0) return FTK_OK;
  if (!d_scores || !d_work) return FTK_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return FTK_ERR_ARG;
  return run_engine(p, precision, reinterpret_cast<const float2*>(d_img), NI, reinterpret_cast<const float2*>(d_tpl),
                    NT, d_scores, nullptr, ftk::BestRecords(), static_cast<char*>(d_work), work_bytes,
                    static_cast<cudaStream_t>(stream));
}

ftk_status ftk_align_best(ftk_plan_t p, int precision, const float* d_img, int NI, const float* d_tpl, int NT,
                          int* d_tplo, int* d_rot, int* d_shift, float* d_score, void* d_work, size_t work_bytes,
                          void* stream) {
  NvtxRange nvtx_("ftk_align_best");
  ftk_status st = check_common(p, precision, d_img, NI, d_tpl, NT);
  if (st != FTK_OK) return st;
  if (NI == 0) return FTK_OK;
  if (NT == 0) return FTK_ERR_ARG;
  if (!d_tplo || !d_rot || !d_shift || !d_score || !d_work) return FTK_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return FTK_ERR_ARG;
  if (ftk::pose_index_wide(1, p->n_rot, p->N)) return FTK_ERR_UNSUPPORTED;
  const size_t kb = keys_bytes(NI);
  if (work_bytes < kb) return FTK_ERR_NOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* keys = static_cast<unsigned long long*>(d_work);
  const ftk::BestRecords rec = records_for(p, NT, d_tplo, d_rot, d_shift, d_score);
  if (rec.wide)
    FTK_LAUNCH(p, ftk::kKBestInit, s, ftk::launch_best_init_records(keys, NI, d_tplo, d_rot, d_shift, d_score, s));
  else
    FTK_LAUNCH(p, ftk::kKBestInit, s, ftk::launch_best_init(keys, NI, s));
  st = run_engine(p, precision, reinterpret_cast<const float2*>(d_img), NI, reinterpret_cast<const float2*>(d_tpl),
                  NT, nullptr, keys, rec, static_cast<char*>(d_work) + kb, work_bytes - kb, s);
  if (st != FTK_OK) return st;
  return finish_best(p, keys, NI, rec, d_tplo, d_rot, d_shift, d_score, s);
}

ftk_status ftk_shortlist_workspace_size(ftk_plan_t p, int precision, int NI, int NT, int K, size_t* min_bytes,
                                        size_t* good_bytes) {
  if (!p || NI < 0 || K < 1 || NT < K) return FTK_ERR_ARG;
  if (precision != FTK_FP32 && precision != FTK_BF16X3 && precision != FTK_BF16 &&
      precision != FTK_FP16) return FTK_ERR_ARG;
  if (precision != FTK_FP32 && !ftk::tc_supported(p)) return FTK_ERR_UNSUPPORTED;
  const size_t base = keys_bytes(NI) + align_up(static_cast<size_t>(NI) * K * sizeof(int)) + 2 * kAlign;
  auto chunk = [&](int ni) {
    return precision == FTK_FP32 ? pair_bytes(p) * K * ni : ftk::tc_shortlist_bytes(p, ni, K, NT);
  };
  if (min_bytes) *min_bytes = base + chunk(1);
  if (good_bytes) {  // up to 512 images per launch, within 16 GiB
    int ni = std::max(1, std::min(NI, 512));
    while (ni > 1 && chunk(ni) > (size_t(1) << 34)) ni = (ni + 1) / 2;
    *good_bytes = base + chunk(ni);
  }
  return FTK_OK;
}

ftk_status ftk_align_best_shortlist(ftk_plan_t p, int precision, const float* d_img, int NI, const float* d_tpl,
                                    int NT, const int* d_shortlist, int K, const float* d_center_px, float window_px,
                                    int* d_tplo, int* d_rot, int* d_shift, float* d_score, void* d_work,
                                    size_t work_bytes, void* stream) {
  NvtxRange nvtx_("ftk_align_best_shortlist");
  ftk_status st = check_common(p, precision, d_img, NI, d_tpl, NT);
  if (st != FTK_OK) return st;
  if (NT < 1 || K < 1 || K > NT || (NI > 0 && !d_shortlist)) return FTK_ERR_ARG;
  if (d_center_px && !(window_px >= 0.f)) return FTK_ERR_ARG;
  if (NI == 0) return FTK_OK;
  if (!d_tplo || !d_rot || !d_shift || !d_score || !d_work) return FTK_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return FTK_ERR_ARG;
  // past 2^32 pose indices the keys count list positions (K R N must stay below 2^32)
  if (ftk::pose_index_wide(K, p->n_rot, p->N)) return FTK_ERR_UNSUPPORTED;
  const size_t kb = keys_bytes(NI);
  const size_t lb = align_up(static_cast<size_t>(NI) * K * sizeof(int));
  if (work_bytes < kb + lb + 2 * kAlign) return FTK_ERR_NOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* keys = static_cast<unsigned long long*>(d_work);
  int* list = reinterpret_cast<int*>(static_cast<char*>(d_work) + kb);
  char* rest = static_cast<char*>(d_work) + kb + lb;
  const size_t avail = work_bytes - kb - lb - 2 * kAlign;
  const float2* a = reinterpret_cast<const float2*>(d_img);
  const float2* b = reinterpret_cast<const float2*>(d_tpl);
  const float2* center = reinterpret_cast<const float2*>(d_center_px);
  const ftk::BestRecords rec = records_for(p, NT, d_tplo, d_rot, d_shift, d_score);
  auto init = [&]() -> ftk_status {
    if (rec.wide)
      FTK_LAUNCH(p, ftk::kKBestInit, s, ftk::launch_best_init_records(keys, NI, d_tplo, d_rot, d_shift, d_score, s));
    else
      FTK_LAUNCH(p, ftk::kKBestInit, s, ftk::launch_best_init(keys, NI, s));
    return FTK_OK;
  };
  if (precision != FTK_FP32) {
    if (ftk::tc_shortlist_bytes(p, 1, K, NT) > avail) return FTK_ERR_NOMEM;
    FTK_CUDA(ftk::launch_sanitize_list(p, d_shortlist, static_cast<long long>(NI) * K, NT, list, s));
    if ((st = init()) != FTK_OK) return st;
    st = ftk::tc_run_shortlist(p, precision, a, NI, b, NT, list, K, center, window_px, keys, rec, rest, avail, s);
    if (st != FTK_OK) return st;
    return finish_best(p, keys, NI, rec, d_tplo, d_rot, d_shift, d_score, s);
  }
  float2* zbuf = reinterpret_cast<float2*>(rest);
  const size_t per_image = pair_bytes(p) * K;
  if (avail < per_image) return FTK_ERR_NOMEM;
  const int ib = static_cast<int>(std::min<size_t>({static_cast<size_t>(NI), avail / per_image, 65535}));
  const size_t MQ2 = static_cast<size_t>(p->M) * p->two_Q;
  FTK_CUDA(ftk::launch_sanitize_list(p, d_shortlist, static_cast<long long>(NI) * K, NT, list, s));
  if ((st = init()) != FTK_OK) return st;
  for (int i0 = 0; i0 < NI; i0 += ib) {
    const int ni = std::min(ib, NI - i0);
    FTK_LAUNCH(p, ftk::kKStep1Simt, s,
               ftk::launch_step1_simt(p, a + i0 * MQ2, ni, b, K, zbuf, s, list + static_cast<size_t>(i0) * K));
    FTK_LAUNCH(p, ftk::kKFftRows, s, ftk::launch_fft_rows(p, zbuf, static_cast<long long>(ni) * K * p->Hh, 1.0f, s));
    FTK_LAUNCH(p, ftk::kKStep3Simt, s,
               ftk::launch_step3_simt(p, zbuf, ni, K, i0, 0, NT, nullptr, keys, s, list, center, window_px, 0,
                                      rec.wide ? 1 : 0));
    if (rec.wide)
      FTK_LAUNCH(p, ftk::kKBestMerge, s, ftk::launch_best_merge(p, keys, i0, ni, 0, list, K, rec, false, s));
  }
  return finish_best(p, keys, NI, rec, d_tplo, d_rot, d_shift, d_score, s);
}

ftk_status ftk_search_workspace_size(ftk_plan_t p, int precision, int NI, int NT, size_t* min_bytes,
                                     size_t* good_bytes) {
  if (!p || NI < 0 || NT < 0) return FTK_ERR_ARG;
  size_t mn = 0, gd = 0;
  ftk_status st = ftk_workspace_size(p, precision, NI, NT, &mn, &gd);
  if (st != FTK_OK) return st;
  const size_t px = align_up(static_cast<size_t>(NI + NT) * p->n * p->n * sizeof(float));
  const size_t cf = align_up(static_cast<size_t>(NI + NT) * p->M * p->two_Q * sizeof(float2));
  const size_t outb = 4 * align_up(static_cast<size_t>(NI) * sizeof(int));
  if (min_bytes) *min_bytes = px + cf + outb + mn;
  if (good_bytes) *good_bytes = px + cf + outb + gd;
  return FTK_OK;
}

ftk_status ftk_search_host(ftk_plan_t p, int precision, const float* h_images, int NI, const float* h_templates,
                           int NT, int* h_tpl, int* h_rot, int* h_shift, float* h_score, void* d_work,
                           size_t work_bytes, void* stream) {
  NvtxRange nvtx_("ftk_search_host");
  if (!p || NI < 0 || NT <= 0 || !h_templates || (NI > 0 && (!h_images || !h_tpl || !h_rot || !h_shift || !h_score)))
    return FTK_ERR_ARG;
  if (!d_work || reinterpret_cast<uintptr_t>(d_work) % kAlign) return FTK_ERR_ARG;
  if (NI == 0) return FTK_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(d_work);
  const size_t npx = static_cast<size_t>(p->n) * p->n;
  const size_t px = align_up(static_cast<size_t>(NI + NT) * npx * sizeof(float));
  const size_t cf = align_up(static_cast<size_t>(NI + NT) * p->M * p->two_Q * sizeof(float2));
  const size_t outb = 4 * align_up(static_cast<size_t>(NI) * sizeof(int));
  if (work_bytes < px + cf + outb) return FTK_ERR_NOMEM;
  float* d_px = reinterpret_cast<float*>(w);
  float* d_cf = reinterpret_cast<float*>(w + px);
  int* d_out = reinterpret_cast<int*>(w + px + cf);
  const size_t ob = align_up(static_cast<size_t>(NI) * sizeof(int));
  int* d_tpl = d_out;
  int* d_rot = reinterpret_cast<int*>(reinterpret_cast<char*>(d_out) + ob);
  int* d_shift = reinterpret_cast<int*>(reinterpret_cast<char*>(d_out) + 2 * ob);
  float* d_score = reinterpret_cast<float*>(reinterpret_cast<char*>(d_out) + 3 * ob);
  FTK_CUDA(cudaMemcpyAsync(d_px, h_images, static_cast<size_t>(NI) * npx * sizeof(float), cudaMemcpyHostToDevice, s));
  FTK_CUDA(cudaMemcpyAsync(d_px + static_cast<size_t>(NI) * npx, h_templates,
                           static_cast<size_t>(NT) * npx * sizeof(float), cudaMemcpyHostToDevice, s));
  ftk_status st = ftk_transform(p, d_px, NI + NT, d_cf, stream);
  if (st != FTK_OK) return st;
  const float* d_a = d_cf;
  const float* d_b = d_cf + static_cast<size_t>(NI) * p->M * p->two_Q * 2;
  st = ftk_align_best(p, precision, d_a, NI, d_b, NT, d_tpl, d_rot, d_shift, d_score, w + px + cf + outb,
                      work_bytes - (px + cf + outb), stream);
  if (st != FTK_OK) return st;
  FTK_CUDA(cudaMemcpyAsync(h_tpl, d_tpl, NI * sizeof(int), cudaMemcpyDeviceToHost, s));
  FTK_CUDA(cudaMemcpyAsync(h_rot, d_rot, NI * sizeof(int), cudaMemcpyDeviceToHost, s));
  FTK_CUDA(cudaMemcpyAsync(h_shift, d_shift, NI * sizeof(int), cudaMemcpyDeviceToHost, s));
  FTK_CUDA(cudaMemcpyAsync(h_score, d_score, NI * sizeof(float), cudaMemcpyDeviceToHost, s));
  FTK_CUDA(cudaStreamSynchronize(s));
  return ftk_stream_check(p, stream);
}

ftk_status ftk_stream_check(ftk_plan_t p, void* stream) {
  if (!p) return FTK_ERR_ARG;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return FTK_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return FTK_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FTK_ERR_CUDA;
  if (err) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return (err & ftk::kErrTimeout) ? FTK_ERR_TIMEOUT : FTK_ERR_ARG;
  }
  return FTK_OK;
}

}  // extern "C"
